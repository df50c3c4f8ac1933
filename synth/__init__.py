"""Seeded synthetic Helmholtz workloads (media, absorbing layers, sources).

This module is the one piece shared by the CPU oracle (``oracle/``), the CUDA
library's tests and ``bench.py``.  It holds only the *problem statement* of the
Helmholtz equation (Sec. 3.1, Eq. (helm): coefficient k(x)^2 = omega^2 n(x)^2,
an absorbing layer folded into the operator) and the random recipes that stand
in for the paper's OpenFWI media (App. Dataset Illustration: 256^2 interior plus
an absorbing layer, 1500-4500 m/s, at least 12 points per wavelength).  It holds
none of the method's arithmetic: no reference wavenumber k0, no damping eps, no
potential V, no preconditioner gamma, no Green symbol.  Those are computed
independently by each side.

Readings of the paper that this recipe fixes (the paper gives only "sponge or
PML" and OpenFWI media):

* absorbing layer: k^2 = omega^2 n^2 + i*sigma with sigma = 0.5*omega^2*rho^2,
  rho = depth/W inside a W-cell layer on every side (depth 1..W, outermost cell
  = W), rho = max(rho_x, rho_y) in the corners;
* grid spacing h = 1 cell, periodic full grid including the layer;
* "wavelengths across the domain" are counted across the interior width;
* Gaussian sources have peak 1 and width 1.5 cells; point sources are 1 at one
  cell.

Every instance draws from ``numpy.random.default_rng(1000 * cfg + index)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

__all__ = [
    "Instance", "grf", "layer_rho", "make_instance", "workload_96",
    "workload_mixed", "workload_contrast", "workload_layered", "small_instance",
]


@dataclasses.dataclass
class Instance:
    """One Helmholtz problem on a periodic ``ny x nx`` grid (layer included)."""
    ny: int
    nx: int
    h: float
    omega: float
    layer: int
    n: np.ndarray        # refractive index, float64 [ny, nx]
    k2: np.ndarray       # complex128 [ny, nx]: omega^2 n^2 + i*sigma
    f: np.ndarray        # complex128 [ny, nx]: source
    seed: int
    source_kind: str


def grf(rng: np.random.Generator, ny: int, nx: int, ell: float) -> np.ndarray:
    """Periodic Gaussian random field with covariance ~exp(-r^2 / (2 ell^2)).

    Unit-variance white noise filtered by exp(-|xi|^2 ell^2 / 4) (xi in rad per
    cell), then re-normalised to zero mean and unit standard deviation.
    """
    w = rng.standard_normal((ny, nx))
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    kx = 2.0 * np.pi * np.fft.fftfreq(nx)
    filt = np.exp(-(ky[:, None] ** 2 + kx[None, :] ** 2) * ell * ell / 4.0)
    g = np.fft.ifft2(np.fft.fft2(w) * filt).real
    g -= g.mean()
    s = g.std()
    return g / s if s > 0 else g


def _depth_1d(n: int, w: int) -> np.ndarray:
    """Depth (in cells, 1..w) into a w-cell layer at both ends; 0 inside."""
    d = np.zeros(n)
    if w <= 0:
        return d
    j = np.arange(n)
    d = np.where(j < w, w - j, d)
    d = np.where(j >= n - w, j - (n - w) + 1, d)
    return d.astype(np.float64)


def layer_rho(ny: int, nx: int, w: int) -> np.ndarray:
    """Normalised layer depth rho in [0, 1]: max of the x and y depths over w."""
    if w <= 0:
        return np.zeros((ny, nx))
    ry = _depth_1d(ny, w) / w
    rx = _depth_1d(nx, w) / w
    return np.maximum(ry[:, None], rx[None, :])


def _gaussian_source(ny: int, nx: int, cy: float, cx: float, width: float = 1.5) -> np.ndarray:
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    r2 = (y - cy) ** 2 + (x - cx) ** 2
    return np.exp(-r2 / (2.0 * width * width)).astype(np.complex128)


def _point_source(ny: int, nx: int, cy: int, cx: int) -> np.ndarray:
    f = np.zeros((ny, nx), np.complex128)
    f[cy, cx] = 1.0
    return f


def make_instance(n: np.ndarray, omega: float, layer: int, f: np.ndarray, *,
                  seed: int = -1, source_kind: str = "gaussian",
                  abs_amp_over_omega2: float = 0.5) -> Instance:
    """Assemble k^2 = omega^2 n^2 + i*A*rho^2 with A = abs_amp_over_omega2*omega^2."""
    ny, nx = n.shape
    sigma = abs_amp_over_omega2 * omega * omega * layer_rho(ny, nx, layer) ** 2
    k2 = (omega * omega) * n.astype(np.float64) ** 2 + 1j * sigma
    return Instance(ny=ny, nx=nx, h=1.0, omega=float(omega), layer=int(layer),
                    n=n.astype(np.float64), k2=k2.astype(np.complex128),
                    f=f.astype(np.complex128), seed=seed, source_kind=source_kind)


def small_instance(ny: int, nx: int | None = None, *, seed: int = 0, layer: int | None = None,
                   ell: float = 8.0, contrast: float = 0.3, ppw: float = 10.0,
                   source: str = "gaussian") -> Instance:
    """The 96^2 medium law at any grid size (tests): n = 1 + c*tanh(GRF)."""
    nx = ny if nx is None else nx
    rng = np.random.default_rng(seed)
    if layer is None:
        layer = max(1, min(ny, nx) // 6)
    g = grf(rng, ny, nx, ell)
    n = 1.0 + contrast * np.tanh(g)
    omega = 2.0 * math.pi / ppw
    if source == "gaussian":
        f = _gaussian_source(ny, nx, ny // 2, nx // 2)
    elif source == "point":
        f = _point_source(ny, nx, ny // 2, nx // 2)
    elif source == "random":
        f = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex128)
    else:
        raise ValueError(source)
    return make_instance(n, omega, layer, f, seed=seed, source_kind=source)


def workload_96() -> List[Instance]:
    """One 96^2 instance: 64^2 interior + 16-cell layer, n = 1 + 0.3 tanh(g),
    correlation length 8, omega = 2*pi/10 (10 points per wavelength at n = 1),
    Gaussian source at the centre."""
    rng = np.random.default_rng(0)
    g = grf(rng, 96, 96, 8.0)
    n = 1.0 + 0.3 * np.tanh(g)
    f = _gaussian_source(96, 96, 48, 48)
    return [make_instance(n, 2.0 * math.pi / 10.0, 16, f, seed=0, source_kind="gaussian")]


def _interior_source(rng: np.random.Generator, N: int, W: int, kind: str) -> np.ndarray:
    cy = int(rng.integers(W, N - W))
    cx = int(rng.integers(W, N - W))
    if kind == "point":
        return _point_source(N, N, cy, cx)
    return _gaussian_source(N, N, cy, cx)


def _mixed_one(seed: int, N: int) -> Instance:
    rng = np.random.default_rng(seed)
    W = N // 16
    n = 1.0 + 0.3 * np.tanh(grf(rng, N, N, 8.0))
    waves = rng.uniform(10.0, 40.0)
    omega = 2.0 * math.pi * waves / (N - 2 * W)
    kind = "point" if rng.uniform() < 0.5 else "gaussian"
    f = _interior_source(rng, N, W, kind)
    return make_instance(n, omega, W, f, seed=seed, source_kind=kind)


def workload_mixed(n256: int = 256, n_other: int = 64, sizes=(128, 192, 384, 512)) -> List[Instance]:
    """Uneven batch: n256 instances at 256^2 plus n_other at sizes drawn
    uniformly from ``sizes``; the 96^2 medium law, 10-40 wavelengths across the
    interior, point or Gaussian sources at random interior positions."""
    out = [_mixed_one(1000 + i, 256) for i in range(n256)]
    pick = np.random.default_rng(1999)
    for j in range(n_other):
        N = int(sizes[int(pick.integers(0, len(sizes)))])
        out.append(_mixed_one(1000 + n256 + j, N))
    return out


def _contrast_one(seed: int, N: int) -> Instance:
    rng = np.random.default_rng(seed)
    W = N // 16
    g = grf(rng, N, N, 16.0)
    na, nb = rng.uniform(0.7, 1.6, size=2)
    n = na + (nb - na) * 0.5 * (1.0 + np.tanh(g / 0.25))
    waves = rng.uniform(20.0, 40.0)
    omega = 2.0 * math.pi * waves / (N - 2 * W)
    f = _interior_source(rng, N, W, "gaussian")
    return make_instance(n, omega, W, f, seed=seed, source_kind="gaussian")


def workload_contrast(count: int = 64, N: int = 256, cfg: int = 2) -> List[Instance]:
    """Thresholded-GRF media with smoothed edges (n in [0.7, 1.6]), 20-40
    wavelengths across the interior, Gaussian sources at random interior
    positions.  ``cfg`` only selects the seed block (2: inference, 3: training)."""
    return [_contrast_one(1000 * cfg + i, N) for i in range(count)]


def _layered_one(seed: int, N: int, waves: float) -> Instance:
    rng = np.random.default_rng(seed)
    W = N // 16
    min_th = N / 24.0
    while True:
        cuts = np.sort(rng.uniform(0.0, 1.0, size=5)) * N
        edges = np.concatenate([[0.0], cuts, [float(N)]])
        if np.all(np.diff(edges) >= min_th):
            break
    vals = rng.uniform(1.0, 2.0, size=6)
    y = np.arange(N) + 0.5
    layer_id = np.searchsorted(cuts, y)
    n = vals[layer_id][:, None] * np.ones((1, N)) + 0.1 * grf(rng, N, N, 16.0)
    omega = 2.0 * math.pi * waves / (N - 2 * W)
    f = _interior_source(rng, N, W, "gaussian")
    return make_instance(n, omega, W, f, seed=seed, source_kind="gaussian")


def workload_layered(count: int = 8, N: int = 1024, waves: float = 100.0) -> List[Instance]:
    """Six horizontal layers (n ~ U[1, 2], minimum thickness N/24) plus a
    0.1-amplitude GRF (correlation length 16), ``waves`` wavelengths across the
    interior, Gaussian source at a random interior position."""
    return [_layered_one(4000 + i, N, waves) for i in range(count)]


def random_weights(shapes, seed: int = 0, out_scale: float = 0.1) -> np.ndarray:
    """Seeded He-normal weights in a flat float32 array, one block per shape.

    1-D shapes are biases (N(0, 0.01^2)); other shapes are weights with fan-in
    prod(shape[1:]).  The last block is scaled by ``out_scale`` so that an
    untrained network makes small corrections.  Used as test/bench input only.
    """
    rng = np.random.default_rng(seed)
    parts = []
    shapes = list(shapes)
    for i, shape in enumerate(shapes):
        shape = tuple(int(s) for s in shape)
        if len(shape) == 1:
            parts.append(0.01 * rng.standard_normal(shape[0]))
        else:
            fan_in = int(np.prod(shape[1:]))
            std = math.sqrt(2.0 / fan_in) * (out_scale if i == len(shapes) - 1 else 1.0)
            parts.append(std * rng.standard_normal(int(np.prod(shape))))
    return np.concatenate(parts).astype(np.float32)


@dataclasses.dataclass
class CdrInstance:
    """One periodic convection-diffusion-reaction problem on the unit square."""
    n: int
    h: float
    kappa: np.ndarray    # float64 [n, n] diffusion (> 0)
    vx: np.ndarray       # float64 [n, n] velocity along the last axis
    vy: np.ndarray       # float64 [n, n] velocity along the first axis
    sigma: np.ndarray    # float64 [n, n] reaction (> 0)
    f: np.ndarray        # complex128 [n, n] source (real Gaussian bump)
    seed: int


def cdr_instance(n: int = 128, seed: int = 0, kappa_mean: float = 0.01, speed: float = 1.0,
                 kappa_contrast: float = 0.5) -> CdrInstance:
    """The CDR benchmark's recipe on a periodic n x n grid of [0, 1)^2 (h = 1/n):
    kappa from a GRF (log-normal around kappa_mean, log-amplitude kappa_contrast), an incompressible velocity
    v = (d psi / dy, -d psi / dx) from a GRF stream function psi (spectral
    derivatives; scaled to a maximum speed `speed`), sigma = 1 + 0.5 tanh(GRF),
    and a Gaussian bump source of random centre and width (periodic distance)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    kappa = kappa_mean * np.exp(kappa_contrast * grf(rng, n, n, n / 16.0))
    psi = grf(rng, n, n, n / 8.0)
    k = 2.0 * math.pi * np.fft.fftfreq(n, d=h)
    P = np.fft.fft2(psi)
    vx = np.fft.ifft2(1j * k[:, None] * P).real       # d psi / dy (first axis)
    vy = -np.fft.ifft2(1j * k[None, :] * P).real      # -d psi / dx (last axis)
    vmax = max(float(np.max(np.hypot(vx, vy))), 1e-30)
    vx, vy = vx * (speed / vmax), vy * (speed / vmax)
    sigma = 1.0 + 0.5 * np.tanh(grf(rng, n, n, n / 16.0))
    cy, cx = rng.uniform(0.0, 1.0, size=2)
    width = rng.uniform(0.03, 0.08)
    y = np.arange(n)[:, None] * h
    x = np.arange(n)[None, :] * h
    dy = np.minimum(np.abs(y - cy), 1.0 - np.abs(y - cy))
    dx = np.minimum(np.abs(x - cx), 1.0 - np.abs(x - cx))
    f = np.exp(-(dy ** 2 + dx ** 2) / (2.0 * width * width)).astype(np.complex128)
    return CdrInstance(n=n, h=h, kappa=kappa, vx=vx, vy=vy, sigma=sigma, f=f, seed=seed)


@dataclasses.dataclass
class NewtonInstance:
    """The nonlinear Dirichlet problem -Lap u - u^2 = f on [0, 1]^2 with N x N
    interior unknowns (h = 1/(N + 1)) and an initial guess."""
    n: int
    h: float
    f: np.ndarray        # float64 [n, n] source -s sin(pi x) sin(pi y)
    u0: np.ndarray       # float64 [n, n] initial guess
    seed: int


def newton_instance(n: int = 64, seed: int = 0, amplitude: float = 1600.0, base: float = -20.0,
                    alpha: float = 4.0) -> NewtonInstance:
    """The Newton benchmark's recipe (N = 64, h = 1/65, s = 1600): f = -s
    sin(pi x) sin(pi y) on the interior nodes x_j = j h, and an initial guess
    base sin(pi x) sin(pi y) + alpha sum_{i,j=1..4} c_ij sin(i pi x) sin(j pi y)
    with c_ij ~ N(0, 0.1^2) (the paper perturbs a reference solution; here the
    perturbation rides on a fixed smooth guess, and Newton finds the branch)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n + 1)
    t = np.arange(1, n + 1) * h
    y, x = t[:, None], t[None, :]
    f = -amplitude * np.sin(math.pi * x) * np.sin(math.pi * y)
    c = rng.normal(0.0, 0.1, size=(4, 4))
    u0 = base * np.sin(math.pi * x) * np.sin(math.pi * y)
    for i in range(4):
        for j in range(4):
            u0 = u0 + alpha * c[i, j] * np.sin((i + 1) * math.pi * x) * np.sin((j + 1) * math.pi * y)
    return NewtonInstance(n=n, h=h, f=f, u0=u0, seed=seed)
