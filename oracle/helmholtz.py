"""Helmholtz operators, CBS and NPBS iterations in complex128 (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Fields are complex128
torch tensors of shape [ny, nx] on a periodic grid with spacing h.

Discretisation (App. Fourier Pseudospectral Discretization): grid x_j = j h,
multi-index n_a in {-N/2, ..., N/2 - 1} (so the Nyquist mode carries -N/2),
xi = 2 pi n / (N h), forward DFT unnormalised and inverse scaled by 1/N.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import torch

C128 = torch.complex128
F64 = torch.float64


def as_c128(a) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(C128)
    return torch.from_numpy(np.asarray(a, dtype=np.complex128))


def mode_index(N: int) -> torch.Tensor:
    """n in FFT order: 0, 1, ..., N/2 - 1, -N/2, ..., -1 (App. Pseudospectral:
    n_a ranges over -N/2 .. N/2 - 1)."""
    n = torch.arange(N, dtype=F64)
    return torch.where(n < N // 2, n, n - N) if N % 2 == 0 else torch.where(n <= N // 2, n, n - N)


def xi_squared(ny: int, nx: int, h: float = 1.0) -> torch.Tensor:
    """|xi_n|^2 with xi = 2 pi n / (N h) (App. Pseudospectral, physical wavenumbers)."""
    ky = 2.0 * math.pi * mode_index(ny) / (ny * h)
    kx = 2.0 * math.pi * mode_index(nx) / (nx * h)
    return ky[:, None] ** 2 + kx[None, :] ** 2


def reference_constants(k2: torch.Tensor) -> tuple[float, float]:
    """k0^2 = midpoint of the range of Re k^2, eps = max |k^2 - k0^2|.

    The paper leaves k0 as the background wavenumber (Sec. 3.1) and eta to a
    validation sweep (App. Role of eta); these are the readings used here, which
    make |1 - gamma| <= 1 pointwise for gamma = i V / eps (CBS convergence).
    """
    re = k2.real
    k0sq = 0.5 * (float(re.min()) + float(re.max()))
    eps = float((k2 - k0sq).abs().max())
    return k0sq, eps


def absorbing_medium(n, omega: float, layer_cells: int, ramp_amp_over_omega2: float = 0.5) -> torch.Tensor:
    """k^2(x) = omega^2 n(x)^2 + i a omega^2 rho(x)^2 on the padded grid.

    Sec. 3.1 truncates the domain with an absorbing layer folded into the
    operator; the paper names only "sponge or PML".  The reading used here: a
    W-cell layer (W = layer_cells) along every side whose imaginary part rises
    quadratically with the depth, a = ramp_amp_over_omega2.  Per cell, the depth
    into the layer along one axis counts 1 at the innermost layer cell up to W
    at the outermost one (0 in the interior); rho is the larger of the two axis
    depths divided by W.  Written cell by cell.
    """
    n = np.asarray(n, dtype=np.float64)
    ny, nx = n.shape
    W = int(layer_cells)
    k2 = np.zeros((ny, nx), dtype=np.complex128)
    for y in range(ny):
        for x in range(nx):
            depths = []
            for j, N in ((y, ny), (x, nx)):
                d = 0
                if j < W:
                    d = W - j
                if j >= N - W:
                    d = j - (N - W) + 1
                depths.append(d)
            rho = max(depths) / W if W > 0 else 0.0
            k2[y, x] = complex((omega * omega) * (n[y, x] * n[y, x]),
                               ramp_amp_over_omega2 * omega * omega * (rho * rho))
    return torch.from_numpy(k2)


def symbol(ny: int, nx: int, h: float, k0sq: float, eps: float) -> torch.Tensor:
    """lambda_n = |xi_n|^2 - (k0^2 + i eta): symbol of L_eta (App. Pseudospectral)."""
    return xi_squared(ny, nx, h).to(C128) - complex(k0sq, eps)


def potential(k2: torch.Tensor, k0sq: float, eps: float) -> torch.Tensor:
    """V_eta = k^2 - k0^2 - i eta (coefficient-only split, Sec. 3.1 and App. Pseudospectral)."""
    return k2 - complex(k0sq, eps)


def gamma_of(V: torch.Tensor, eps: float) -> torch.Tensor:
    """Diagonal CBS preconditioner gamma = i V / eta.  Eq. (CBS) only says gamma is
    'derived from V'; this is the convergent-Born-series choice of the cited CBS
    paper (Osnabrugge et al. 2016)."""
    return 1j * V / eps


def green(q: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
    """G_eta q = F^{-1}(F q / lambda): the three-step FFT recipe (App. Pseudospectral)."""
    return torch.fft.ifft2(torch.fft.fft2(q) / lam)


def green_adjoint(q: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
    """G_eta^* q = F^{-1}(F q / conj(lambda)) (G = F^{-1} diag(1/lambda) F, App.
    Transform-diagonalizable, and F^{-1} = F^* / N for the unnormalised DFT)."""
    return torch.fft.ifft2(torch.fft.fft2(q) / lam.conj())


def laplacian_neg(u: torch.Tensor, h: float = 1.0) -> torch.Tensor:
    """-Delta u = F^{-1}(|xi|^2 F u) (App. Pseudospectral, relation to A)."""
    ny, nx = u.shape
    return torch.fft.ifft2(xi_squared(ny, nx, h).to(C128) * torch.fft.fft2(u))


def apply_A(u: torch.Tensor, k2: torch.Tensor, h: float = 1.0) -> torch.Tensor:
    """A u = -Delta u - k^2 u with the layer folded into Im k^2 (Eq. helm, App. Pseudospectral)."""
    return laplacian_neg(u, h) - k2 * u


@dataclasses.dataclass
class Problem:
    """A discretised Helmholtz instance with the method's derived quantities."""
    k2: torch.Tensor
    f: torch.Tensor
    h: float
    k0sq: float
    eps: float
    V: torch.Tensor
    lam: torch.Tensor
    gamma: torch.Tensor
    n: Optional[torch.Tensor] = None

    @property
    def shape(self):
        return tuple(self.k2.shape)


def make_problem(k2, f, h: float = 1.0, k0sq: float | None = None, eps: float | None = None,
                 n=None) -> Problem:
    k2 = as_c128(k2)
    f = as_c128(f)
    a, b = reference_constants(k2)
    k0sq = a if k0sq is None else float(k0sq)
    eps = b if eps is None else float(eps)
    ny, nx = k2.shape
    V = potential(k2, k0sq, eps)
    lam = symbol(ny, nx, h, k0sq, eps)
    nt = None if n is None else torch.as_tensor(np.asarray(n), dtype=F64)
    return Problem(k2=k2, f=f, h=float(h), k0sq=k0sq, eps=eps, V=V, lam=lam,
                   gamma=gamma_of(V, eps), n=nt)


def problem_from_instance(inst) -> Problem:
    return make_problem(inst.k2, inst.f, inst.h, n=inst.n)


# ---------------------------------------------------------------- apply modes

def born_residual(p: Problem, u: torch.Tensor) -> torch.Tensor:
    """Preconditioned residual in integral form, r = G(V u + f) - u (Eq. npbs_integral)."""
    return green(p.V * u + p.f, p.lam) - u


def born_residual_left(p: Problem, u: torch.Tensor) -> torch.Tensor:
    """The same residual in left-preconditioned form, G(f - A u) (Eq. npbs_iter)."""
    return green(p.f - apply_A(u, p.k2, p.h), p.lam)


def cbs_step(p: Problem, u: torch.Tensor) -> torch.Tensor:
    """u + gamma (G(V u + f) - u) (Eq. CBS)."""
    return u + p.gamma * born_residual(p, u)


def op_B(p: Problem, x: torch.Tensor) -> torch.Tensor:
    """B x = (I - G V) x, the Lippmann-Schwinger operator (Eq. LS_discrete)."""
    return x - green(p.V * x, p.lam)


def op_BH(p: Problem, y: torch.Tensor) -> torch.Tensor:
    """B^* y = y - conj(V) (G^* y)."""
    return y - p.V.conj() * green_adjoint(y, p.lam)


def true_residual(p: Problem, u: torch.Tensor) -> torch.Tensor:
    """f - A u over the full padded grid (Sec. 5, unified stopping rule)."""
    return p.f - apply_A(u, p.k2, p.h)


def rtol(p: Problem, u: torch.Tensor) -> float:
    """rTol = ||f - A u||_2 / ||f||_2 (Sec. 5)."""
    return float(torch.linalg.vector_norm(true_residual(p, u)) / torch.linalg.vector_norm(p.f))


def prec_cbs_sweep(p: Problem, z: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """One Richardson sweep with the CBS diagonal for B z = v: z + gamma (v - B z).
    With v = G f this is exactly Eq. (CBS)."""
    return z + p.gamma * (v - op_B(p, z))


# ---------------------------------------------------------------- iterations

@dataclasses.dataclass
class SolveResult:
    u: torch.Tensor
    iters: int
    rtol: float
    history: List[float]
    converged: bool


def cbs_solve(p: Problem, tol: float = 1e-6, max_iter: int = 2500, u0=None,
              check_every: int = 1) -> SolveResult:
    """Stationary CBS (Eq. CBS) from u^0 = 0, stopped by rTol (Sec. 5).

    The count is the number of updates applied before the first passing check.
    """
    u = torch.zeros_like(p.f) if u0 is None else as_c128(u0).clone()
    hist = []
    it = 0
    r = rtol(p, u)
    hist.append(r)
    while r > tol and it < max_iter:
        u = cbs_step(p, u)
        it += 1
        if it % check_every == 0 or it == max_iter:
            r = rtol(p, u)
            hist.append(r)
    return SolveResult(u=u, iters=it, rtol=r, history=hist, converged=r <= tol)


def npbs_solve(p: Problem, M: Callable[[torch.Tensor], torch.Tensor], tol: float = 1e-6,
               max_iter: int = 2500, u0=None, check_every: int = 1) -> SolveResult:
    """NPBS in integral form, u <- u + M(G(V u + f) - u) (Eq. npbs_integral)."""
    u = torch.zeros_like(p.f) if u0 is None else as_c128(u0).clone()
    hist = []
    it = 0
    r = rtol(p, u)
    hist.append(r)
    while r > tol and it < max_iter:
        u = u + M(born_residual(p, u))
        it += 1
        if it % check_every == 0 or it == max_iter:
            r = rtol(p, u)
            hist.append(r)
    return SolveResult(u=u, iters=it, rtol=r, history=hist, converged=r <= tol)


def direct_solve(p: Problem, M: Callable[[torch.Tensor], torch.Tensor], tol: float = 1e-6,
                 max_iter: int = 2500, u0=None, check_every: int = 1) -> SolveResult:
    """Learned iteration in unpreconditioned residual coordinates,
    u <- u + M(f - A u) (Eq. direct_iter), the baseline format of Sec. 4."""
    u = torch.zeros_like(p.f) if u0 is None else as_c128(u0).clone()
    hist = []
    it = 0
    r = rtol(p, u)
    hist.append(r)
    while r > tol and it < max_iter:
        u = u + M(true_residual(p, u))
        it += 1
        if it % check_every == 0 or it == max_iter:
            r = rtol(p, u)
            hist.append(r)
    return SolveResult(u=u, iters=it, rtol=r, history=hist, converged=r <= tol)
