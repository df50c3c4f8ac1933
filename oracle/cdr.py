"""Convection-diffusion-reaction operators and the Born / NPBS iteration for
them (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  complex128 / float64 on
the CPU with plain PyTorch ops (``torch.fft`` as the FFT step).

The paper's CDR extension (App. Full Derivations, Convection-Diffusion-Reaction;
Eqs. cdr_pde, cdr_L0, cdr_V, cdr_integral, cdr_identity, cdr_bs_loss,
cdr_G_symbol):

    A u  = -div(kappa grad u) + v . grad u + sigma u            (Eq. cdr_pde)
    L0 u = -kappa0 Lap u + v0 . grad u + sigma0 u               (Eq. cdr_L0)
    V    = L0 - A = div(dkappa grad u) - dv . grad u - dsigma u  (Eq. cdr_V)
    G    = L0^{-1}, symbol 1 / (kappa0 |xi|^2 + i v0 . xi + sigma0)  (Eq. cdr_G_symbol)
    (I - G V) u = G f,   I - G V = G A                           (Eqs. cdr_integral, cdr_identity)

and the same NPBS template as for Helmholtz: u <- u + M(G(V u + f) - u).

Readings where the paper is silent: the periodic grid of the Helmholtz
problem (x_j = j h, the same mode set, first derivatives with symbol i xi on
every mode); the background constants are kappa0 = the midpoint of the range
of kappa, sigma0 = the midpoint of the range of sigma and v0 = the grid mean
of v (the choice that makes the diffusion and reaction parts of G V contract,
|kappa - kappa0| / kappa0 < 1 and |sigma - sigma0| / sigma0 < 1, as the
midpoint k0^2 and eps = max |k^2 - k0^2| do for Helmholtz; for a velocity from
a periodic stream function the mean is zero, so L0 is the symmetric
-kappa0 Lap + sigma0 and all of the convection sits in V); fields are complex
(real data stay real up to rounding).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np
import torch

from . import helmholtz as H

C128 = torch.complex128
F64 = torch.float64


@dataclasses.dataclass
class CdrProblem:
    kappa: torch.Tensor   # [ny, nx] float64 diffusion
    vx: torch.Tensor      # [ny, nx] float64 velocity, x component (along the last axis)
    vy: torch.Tensor      # [ny, nx] float64 velocity, y component
    sigma: torch.Tensor   # [ny, nx] float64 reaction
    f: torch.Tensor       # [ny, nx] complex128 source
    h: float
    kappa0: float
    v0x: float
    v0y: float
    sigma0: float
    kx: torch.Tensor      # [1, nx] float64 xi_x
    ky: torch.Tensor      # [ny, 1] float64 xi_y
    lam: torch.Tensor     # [ny, nx] complex128 symbol of L0


def wavenumbers(ny: int, nx: int, h: float):
    """xi_y [ny, 1], xi_x [1, nx] with xi = 2 pi n / (N h) on the Helmholtz mode set."""
    ky = 2.0 * math.pi * H.mode_index(ny) / (ny * h)
    kx = 2.0 * math.pi * H.mode_index(nx) / (nx * h)
    return ky[:, None], kx[None, :]


def make_problem(kappa, vx, vy, sigma, f, h: float, consts=None) -> CdrProblem:
    """consts = (kappa0, v0x, v0y, sigma0), by default the midpoints of the
    ranges of kappa and sigma and the grid means of v."""
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=F64)
    kappa, vx, vy, sigma = t(kappa), t(vx), t(vy), t(sigma)
    f = H.as_c128(f)
    if consts is None:
        consts = (0.5 * (float(kappa.min()) + float(kappa.max())), float(vx.mean()), float(vy.mean()),
                  0.5 * (float(sigma.min()) + float(sigma.max())))
    k0, v0x, v0y, s0 = (float(c) for c in consts)
    ky, kx = wavenumbers(*kappa.shape, h)
    lam = (k0 * (kx ** 2 + ky ** 2)).to(C128) + 1j * (v0x * kx + v0y * ky) + s0
    return CdrProblem(kappa, vx, vy, sigma, f, float(h), k0, v0x, v0y, s0, kx, ky, lam)


def ddx(p: CdrProblem, u: torch.Tensor) -> torch.Tensor:
    return torch.fft.ifft2(1j * p.kx * torch.fft.fft2(u))


def ddy(p: CdrProblem, u: torch.Tensor) -> torch.Tensor:
    return torch.fft.ifft2(1j * p.ky * torch.fft.fft2(u))


def apply_A(p: CdrProblem, u: torch.Tensor) -> torch.Tensor:
    """A u = -div(kappa grad u) + v . grad u + sigma u (Eq. cdr_pde)."""
    ux, uy = ddx(p, u), ddy(p, u)
    return -(ddx(p, p.kappa * ux) + ddy(p, p.kappa * uy)) + p.vx * ux + p.vy * uy + p.sigma * u


def apply_L0(p: CdrProblem, u: torch.Tensor) -> torch.Tensor:
    """L0 u = -kappa0 Lap u + v0 . grad u + sigma0 u (Eq. cdr_L0), by its symbol."""
    return torch.fft.ifft2(p.lam * torch.fft.fft2(u))


def apply_V(p: CdrProblem, u: torch.Tensor) -> torch.Tensor:
    """V u = div(dkappa grad u) - dv . grad u - dsigma u (Eq. cdr_V)."""
    ux, uy = ddx(p, u), ddy(p, u)
    dk = p.kappa - p.kappa0
    return (ddx(p, dk * ux) + ddy(p, dk * uy)) - (p.vx - p.v0x) * ux - (p.vy - p.v0y) * uy - (p.sigma - p.sigma0) * u


def green(p: CdrProblem, q: torch.Tensor) -> torch.Tensor:
    """G q = F^{-1}(F q / symbol(L0)) (Eq. cdr_G_symbol)."""
    return torch.fft.ifft2(torch.fft.fft2(q) / p.lam)


def born_residual(p: CdrProblem, u: torch.Tensor) -> torch.Tensor:
    """G(V u + f) - u (the integral form, Eq. cdr_integral)."""
    return green(p, apply_V(p, u) + p.f) - u


def op_B(p: CdrProblem, x: torch.Tensor) -> torch.Tensor:
    """(I - G V) x."""
    return x - green(p, apply_V(p, x))


def green_adjoint(p: CdrProblem, q: torch.Tensor) -> torch.Tensor:
    """G^* q = F^{-1}(F q / conj(symbol(L0)))."""
    return torch.fft.ifft2(torch.fft.fft2(q) / p.lam.conj())


def apply_A_adjoint(p: CdrProblem, g: torch.Tensor) -> torch.Tensor:
    """A^* g = -div(kappa grad g) - div(v g) + sigma g (the real coefficients
    make the diffusion and reaction parts self-adjoint; the adjoint of v . grad
    is -div(v .))."""
    gx, gy = ddx(p, g), ddy(p, g)
    return -(ddx(p, p.kappa * gx + p.vx * g) + ddy(p, p.kappa * gy + p.vy * g)) + p.sigma * g


def op_BH(p: CdrProblem, y: torch.Tensor) -> torch.Tensor:
    """(I - G V)^* y = (G A)^* y = A^* G^* y (Eq. cdr_identity)."""
    return apply_A_adjoint(p, green_adjoint(p, y))


def rtol(p: CdrProblem, u: torch.Tensor) -> float:
    """||f - A u|| / ||f|| (the stopping rule of Sec. 5)."""
    return float(torch.linalg.norm(p.f - apply_A(p, u)) / torch.linalg.norm(p.f))


@dataclasses.dataclass
class SolveResult:
    u: torch.Tensor
    iters: int
    history: list


def npbs_solve(p: CdrProblem, M: Callable[[torch.Tensor], torch.Tensor], tol: float = 1e-6, max_iter: int = 2500,
               u0=None) -> SolveResult:
    """u <- u + M(G(V u + f) - u) until rTol <= tol (M = identity: the Born series)."""
    u = torch.zeros_like(p.f) if u0 is None else H.as_c128(u0).clone()
    hist = [rtol(p, u)]
    it = 0
    while hist[-1] > tol and it < max_iter:
        u = u + M(born_residual(p, u))
        it += 1
        hist.append(rtol(p, u))
    return SolveResult(u, it, hist)
