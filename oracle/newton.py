"""Newton-Born linearisation of a nonlinear PDE with a DST-I Green operator
(CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  float64 torch tensors
[N, N] of interior unknowns on Omega = [0, 1]^2 with homogeneous Dirichlet
boundaries, h = 1/(N + 1), x_j = j h (j = 1..N).

The paper's nonlinear example (App. Full Derivations, Nonlinear PDE via
Newton-Born Linearization; Sec. 5.2, Eq. newton; App. Verification, Newton
linear systems):

    F(u)  = -Lap u - u^2 - f                                   (Eq. nonlinear_residual)
    J_m   = -Lap - 2 u_m,   r_m = -F(u_m),  u_{m+1} = u_m + delta_m   (Eq. newton_linear_system)
    discretely L_D = the five-point negative Laplacian / h^2, J = L_D - 2 diag(u_m)
    J0_m  = L_D + (alpha_m - 2 mean(u_m)) I                    (Eq. newton_ref)
    V_m   = J0_m - J_m = 2 (u_m - mean(u_m)) + alpha_m        (Eq. newton_vm)
    G_m   = J0_m^{-1} = S^{-1} diag(1 / lambda) S, S the 2D DST-I,
            lambda_pq = (4/h^2)(sin^2(p pi h/2) + sin^2(q pi h/2)) + alpha_m - 2 mean(u_m)
    (I - G_m V_m) delta = G_m r  <=>  I - G_m V_m = G_m J_m    (Eq. newton_born_identity)
    inner iteration delta <- delta + M(G_m (r - J_m delta))    (Eq. newton_inner_iter)

Readings where the paper is silent: the shift keeps the mean-reaction term
(-2 mean(u_m), the paper's "spatial average" choice) with alpha_m = 0 unless a
caller gives another; the inner stopping rule is ||r - J delta|| / ||r|| <=
rTol (rTol = 1e-4 in the paper); the outer loop stops when ||F(u)|| / ||f|| <=
tol or after a given number of Newton steps.  Fields may be complex (the
library carries complex64 fields; real data stay real).

The DST-I is written as products with the sine matrix (S^2 = (N + 1)/2 I
per axis, so S^{-1} = (2 / (N + 1)) S); the pins check it against scipy's
DST-I.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import torch

F64 = torch.float64


def spacing(N: int) -> float:
    return 1.0 / (N + 1)


def grid(N: int):
    """Interior coordinates (y [N, 1], x [1, N]) with x_j = j h, j = 1..N."""
    h = spacing(N)
    t = torch.arange(1, N + 1, dtype=F64) * h
    return t[:, None], t[None, :]


def lap_D(u: torch.Tensor, h: float) -> torch.Tensor:
    """The five-point negative Laplacian on interior unknowns with zero
    Dirichlet values outside: (4 u_ij - u_i+1,j - u_i-1,j - u_i,j+1 - u_i,j-1) / h^2."""
    p = torch.nn.functional.pad(u[None, None] if not u.is_complex() else u.real[None, None], (1, 1, 1, 1))[0, 0]
    if u.is_complex():
        q = torch.nn.functional.pad(u.imag[None, None], (1, 1, 1, 1))[0, 0]
        return torch.complex(_stencil(p, h), _stencil(q, h))
    return _stencil(p, h)


def _stencil(p: torch.Tensor, h: float) -> torch.Tensor:
    c = p[1:-1, 1:-1]
    return (4.0 * c - p[2:, 1:-1] - p[:-2, 1:-1] - p[1:-1, 2:] - p[1:-1, :-2]) / (h * h)


def nonlinear_residual(u: torch.Tensor, f: torch.Tensor, h: float) -> torch.Tensor:
    """F(u) = L_D u - u^2 - f (Eq. nonlinear_residual, discretely)."""
    return lap_D(u, h) - u * u - f


def jacobian(u: torch.Tensor, x: torch.Tensor, h: float) -> torch.Tensor:
    """J x = L_D x - 2 u x."""
    return lap_D(x, h) - 2.0 * u * x


def sine_matrix(N: int) -> torch.Tensor:
    """S_jk = sin(pi j k / (N + 1)), j, k = 1..N (symmetric)."""
    j = torch.arange(1, N + 1, dtype=F64)
    return torch.sin(math.pi * torch.outer(j, j) / (N + 1))


def dst2(q: torch.Tensor) -> torch.Tensor:
    """The 2D DST-I: S q S along both axes (a plain matrix product, so that
    autograd passes through the Green operator)."""
    S = sine_matrix(q.shape[0]).to(q.dtype)
    return S @ q @ S


def laplacian_eigenvalues(N: int) -> torch.Tensor:
    """lambda_pq of L_D: (4/h^2)(sin^2(p pi h / 2) + sin^2(q pi h / 2)), p, q = 1..N."""
    h = spacing(N)
    s = torch.sin(torch.arange(1, N + 1, dtype=F64) * math.pi * h / 2.0) ** 2
    return 4.0 / (h * h) * (s[:, None] + s[None, :])


@dataclasses.dataclass
class NewtonState:
    """One linearisation: the iterate u_m, its shift c = alpha - 2 mean(u_m),
    the symbol lambda of J0 and the right-hand side r = -F(u_m)."""
    u: torch.Tensor
    f: torch.Tensor
    h: float
    alpha: float
    shift: float
    lam: torch.Tensor
    r: torch.Tensor


def linearise(u: torch.Tensor, f: torch.Tensor, alpha: float = 0.0) -> NewtonState:
    N = u.shape[0]
    h = spacing(N)
    shift = alpha - 2.0 * float(u.real.mean())
    lam = laplacian_eigenvalues(N) + shift
    return NewtonState(u, f, h, float(alpha), shift, lam, -nonlinear_residual(u, f, h))


def green(s: NewtonState, q: torch.Tensor) -> torch.Tensor:
    """G q = S^{-1}(S q / lambda), S^{-1} = (2/(N+1))^2 S in 2D."""
    N = q.shape[0]
    return dst2(dst2(q) / s.lam) * (2.0 / (N + 1)) ** 2


def apply_J0(s: NewtonState, x: torch.Tensor) -> torch.Tensor:
    """J0 x = L_D x + shift x."""
    return lap_D(x, s.h) + s.shift * x


def apply_V(s: NewtonState, x: torch.Tensor) -> torch.Tensor:
    """V x = (J0 - J) x = (shift + 2 u) x."""
    return (s.shift + 2.0 * s.u) * x


def born_residual(s: NewtonState, d: torch.Tensor, r: Optional[torch.Tensor] = None) -> torch.Tensor:
    """G(r - J d) (the network input of Eq. newton_inner_iter)."""
    r = s.r if r is None else r
    return green(s, r - jacobian(s.u, d, s.h))


def op_B(s: NewtonState, x: torch.Tensor) -> torch.Tensor:
    """(I - G V) x."""
    return x - green(s, apply_V(s, x))


def op_BH(s: NewtonState, y: torch.Tensor) -> torch.Tensor:
    """(I - G V)^* y = y - V G y (G, V real symmetric: conj(V) = V, G^* = G on real data
    and G^* y = conj(G conj y) in general)."""
    return y - apply_V(s, green(s, y))


def inner_rtol(s: NewtonState, d: torch.Tensor) -> float:
    return float(torch.linalg.norm(s.r - jacobian(s.u, d, s.h)) / torch.linalg.norm(s.r))


@dataclasses.dataclass
class InnerResult:
    delta: torch.Tensor
    iters: int
    history: List[float]


def inner_solve(s: NewtonState, M: Callable[[torch.Tensor], torch.Tensor], tol: float = 1e-4,
                max_iter: int = 1000) -> InnerResult:
    """delta <- delta + M(G(r - J delta)) from delta = 0 until ||r - J delta|| / ||r|| <= tol
    (M = identity: the Born series)."""
    d = torch.zeros_like(s.r)
    hist = [inner_rtol(s, d)]
    it = 0
    while hist[-1] > tol and it < max_iter:
        d = d + M(born_residual(s, d))
        it += 1
        hist.append(inner_rtol(s, d))
    return InnerResult(d, it, hist)


@dataclasses.dataclass
class NewtonResult:
    u: torch.Tensor
    steps: int
    inner_iters: List[int]
    history: List[float]


def newton(u0: torch.Tensor, f: torch.Tensor, M: Callable[[NewtonState, torch.Tensor], torch.Tensor],
           alpha: float = 0.0, tol: float = 1e-8, max_steps: int = 20, inner_tol: float = 1e-4,
           inner_max: int = 1000) -> NewtonResult:
    """Newton on F(u) = 0 with inner Born / NPBS solves of each Jacobian system;
    M(state, r) is the correction of one inner iteration.  Stops when
    ||F(u)|| / ||f|| <= tol."""
    u = u0.clone()
    h = spacing(u.shape[0])
    fn = float(torch.linalg.norm(f))
    hist = [float(torch.linalg.norm(nonlinear_residual(u, f, h))) / fn]
    inner = []
    m = 0
    while hist[-1] > tol and m < max_steps:
        s = linearise(u, f, alpha)
        res = inner_solve(s, lambda q: M(s, q), inner_tol, inner_max)
        u = u + res.delta
        inner.append(res.iters)
        m += 1
        hist.append(float(torch.linalg.norm(nonlinear_residual(u, f, h))) / fn)
    return NewtonResult(u, m, inner, hist)


def source(N: int, amplitude: float = 1600.0) -> torch.Tensor:
    """f = -s sin(pi x) sin(pi y) (Sec. 5.2, the nonlinear example)."""
    y, x = grid(N)
    return -amplitude * torch.sin(math.pi * x) * torch.sin(math.pi * y)
