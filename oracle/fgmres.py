"""Restarted flexible GMRES on the Lippmann-Schwinger system (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Solves B u = G f with B = I - G V (Eq. LS_discrete), with a right
preconditioner that may change from step to step (flexible GMRES, the FGMRES
comparison of Sec. 5.1.3 after Saad 1993): z_j = P(v_j), w = B z_j,
modified Gram-Schmidt against v_1..v_j, Givens rotations on the Hessenberg
column, and at the end of a cycle u += Z y.  The inner estimate is
||G f - B u||_2; the cycle ends early when that estimate reaches the current
inner target, and the stopping test is the true rTol of Sec. 5 checked at the
end of every cycle.  Iteration counts are the number of preconditioned
Arnoldi steps (each one application of B).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import torch

from . import helmholtz as H


@dataclasses.dataclass
class FgmresResult:
    u: torch.Tensor
    iters: int
    rtol: float
    history: List[float]
    converged: bool


def _dot(a: torch.Tensor, b: torch.Tensor) -> complex:
    """<a, b> = sum conj(a) b."""
    return complex(torch.vdot(a.reshape(-1), b.reshape(-1)))


def _norm(a: torch.Tensor) -> float:
    return float(torch.linalg.vector_norm(a))


def fgmres_solve(p: H.Problem, precond: Optional[Callable[[torch.Tensor], torch.Tensor]] = None,
                 restart: int = 20, tol: float = 1e-5, max_iter: int = 2500,
                 u0: Optional[torch.Tensor] = None) -> FgmresResult:
    P = precond if precond is not None else (lambda v: v)
    u = torch.zeros_like(p.f) if u0 is None else H.as_c128(u0).clone()
    b = H.green(p.f, p.lam)
    bnorm = _norm(b)
    total = 0
    r_true = H.rtol(p, u)
    hist = [r_true]
    inner_target = tol * bnorm
    while r_true > tol and total < max_iter:
        r0 = b - H.op_B(p, u)
        beta = _norm(r0)
        if beta == 0.0:
            break
        Vb = [r0 / beta]
        Z = []
        Hm = torch.zeros((restart + 1, restart), dtype=torch.complex128)
        cs = torch.zeros(restart, dtype=torch.complex128)
        sn = torch.zeros(restart, dtype=torch.complex128)
        g = torch.zeros(restart + 1, dtype=torch.complex128)
        g[0] = beta
        j_used = 0
        for j in range(restart):
            z = P(Vb[j])
            Z.append(z)
            w = H.op_B(p, z)
            for i in range(j + 1):
                hij = _dot(Vb[i], w)
                Hm[i, j] = hij
                w = w - hij * Vb[i]
            hn = _norm(w)
            Hm[j + 1, j] = hn
            Vb.append(w / hn if hn > 0 else w)
            # apply the previous rotations to the new column
            for i in range(j):
                a, c = complex(Hm[i, j]), complex(Hm[i + 1, j])
                Hm[i, j] = cs[i].conj() * a + sn[i].conj() * c
                Hm[i + 1, j] = -sn[i] * a + cs[i] * c
            a, c = complex(Hm[j, j]), complex(Hm[j + 1, j])
            den = (abs(a) ** 2 + abs(c) ** 2) ** 0.5
            cs[j] = a / den if den > 0 else 1.0
            sn[j] = c / den if den > 0 else 0.0
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            gj = complex(g[j])
            g[j + 1] = -sn[j] * gj
            g[j] = cs[j].conj() * gj
            total += 1
            j_used = j + 1
            if abs(complex(g[j + 1])) <= inner_target or total >= max_iter or hn == 0.0:
                break
        R = Hm[:j_used, :j_used]
        y = torch.linalg.solve_triangular(R, g[:j_used].reshape(-1, 1), upper=True).reshape(-1)
        for i in range(j_used):
            u = u + y[i] * Z[i]
        r_true = H.rtol(p, u)
        hist.append(r_true)
        if r_true > tol:
            est = abs(complex(g[j_used])) / bnorm
            if est <= tol:
                # the estimate passed but the true residual did not: tighten the
                # inner target in proportion to the observed gap
                inner_target = inner_target * max(0.05, 0.5 * tol / r_true)
    return FgmresResult(u=u, iters=total, rtol=r_true, history=hist, converged=r_true <= tol)
