"""Dense matrices of the discrete Helmholtz operators for tiny grids (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Independent of the FFT
code in ``helmholtz``: the 2D DFT is the Kronecker product of 1D DFT matrices
F[j, k] = exp(-2 pi i j k / N) written from the definition, acting on
row-major flattened fields.  Used to pin the FFT-based oracle to exact linear
algebra: Prop. 3.1 (I - G V = G A, the disk and condition-number bounds),
dense direct solves, the CBS iteration matrix, and M = (I - G V)^{-1}.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(N: int) -> np.ndarray:
    j = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(j, j) / N)


def signed_modes(N: int) -> np.ndarray:
    """Integer mode of DFT index k taken in -N/2 .. N/2 - 1 (App. Pseudospectral)."""
    k = np.arange(N)
    return ((k + N // 2) % N) - N // 2


def dft2(ny: int, nx: int) -> np.ndarray:
    return np.kron(dft_matrix(ny), dft_matrix(nx))


def neg_laplacian(ny: int, nx: int, h: float = 1.0) -> np.ndarray:
    """F^{-1} diag(|xi|^2) F with xi = 2 pi n / (N h)."""
    F = dft2(ny, nx)
    Finv = F.conj().T / (ny * nx)
    ky = 2 * np.pi * signed_modes(ny) / (ny * h)
    kx = 2 * np.pi * signed_modes(nx) / (nx * h)
    xi2 = (ky[:, None] ** 2 + kx[None, :] ** 2).reshape(-1)
    return Finv @ np.diag(xi2) @ F


def operators(k2: np.ndarray, h: float, k0sq: float, eps: float) -> dict:
    """Dense A, L_eta, G_eta = L_eta^{-1}, V, gamma, B = I - G V and the CBS
    iteration matrix I - gamma B (= gamma G V - gamma + 1)."""
    ny, nx = k2.shape
    n = ny * nx
    Lap = neg_laplacian(ny, nx, h)
    K2 = np.diag(k2.reshape(-1))
    A = Lap - K2
    L = Lap - (k0sq + 1j * eps) * np.eye(n)
    G = np.linalg.inv(L)
    Vd = k2.reshape(-1) - (k0sq + 1j * eps)
    V = np.diag(Vd)
    gam = np.diag(1j * Vd / eps)
    B = np.eye(n) - G @ V
    Mcbs = np.eye(n) - gam @ B
    return dict(A=A, L=L, G=G, V=V, gamma=gam, B=B, Mcbs=Mcbs, Lap=Lap)
