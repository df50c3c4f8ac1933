"""Pins of the oracle's CDR operators (App. Full Derivations, CDR; Eqs. cdr_pde,
cdr_L0, cdr_V, cdr_integral, cdr_identity, cdr_G_symbol): V written out
against L0 - A, the key identity, closed forms for constant coefficients,
dense direct solves built from the DFT definition, the NPBS special cases, and
the input recipe's incompressible velocity."""
import numpy as np
import pytest
import torch

import synth
from oracle import cdr as CD
from oracle import dense as D


def _random_problem(n=12, seed=0, consts=None, strength=1.0):
    rng = np.random.default_rng(seed)
    kappa = 0.05 * np.exp(0.3 * strength * rng.standard_normal((n, n)))
    vx = 0.5 * strength * rng.standard_normal((n, n))
    vy = 0.5 * strength * rng.standard_normal((n, n))
    sigma = 1.0 + 0.3 * strength * rng.standard_normal((n, n))
    f = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return CD.make_problem(kappa, vx, vy, sigma, f, 1.0 / n, consts)


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))


def test_V_written_out_equals_L0_minus_A():
    p = _random_problem(consts=(0.04, 0.2, -0.1, 0.9))
    u = _rand(12, 1)
    lhs = CD.apply_V(p, u)
    rhs = CD.apply_L0(p, u) - CD.apply_A(p, u)
    assert torch.allclose(lhs, rhs, rtol=0, atol=1e-12 * float(rhs.abs().max()))


def test_key_identity_I_minus_GV_equals_GA():
    p = _random_problem(seed=2)
    x = _rand(12, 3)
    assert torch.allclose(CD.op_B(p, x), CD.green(p, CD.apply_A(p, x)), atol=1e-12)


def test_constant_coefficients_plane_wave():
    """kappa, v, sigma constant: V = 0 and A on exp(i xi . x) is the symbol
    kappa0 |xi|^2 + i v0 . xi + sigma0 times it (Eq. cdr_G_symbol)."""
    n, h = 8, 1.0 / 8
    k0, vx0, vy0, s0 = 0.07, 0.4, -0.3, 1.3
    c = np.ones((n, n))
    p = CD.make_problem(k0 * c, vx0 * c, vy0 * c, s0 * c, np.ones((n, n)), h)
    assert (p.kappa0, p.v0x, p.v0y, p.sigma0) == pytest.approx((k0, vx0, vy0, s0))
    y = np.arange(n)[:, None] * h
    x = np.arange(n)[None, :] * h
    for my, mx in [(1, 2), (-3, 1), (0, -2)]:
        xi_y, xi_x = 2 * np.pi * my, 2 * np.pi * mx
        e = torch.from_numpy(np.exp(1j * (xi_y * y + xi_x * x)))
        sym = k0 * (xi_x ** 2 + xi_y ** 2) + 1j * (vx0 * xi_x + vy0 * xi_y) + s0
        assert torch.allclose(CD.apply_A(p, e), sym * e, atol=1e-11)
        assert torch.allclose(CD.apply_V(p, e), torch.zeros_like(e), atol=1e-11)


def _dense_A(p, n):
    """A = -Dx K Dx - Dy K Dy + diag(vx) Dx + diag(vy) Dy + diag(sigma) from DFT matrices."""
    F = D.dft2(n, n)
    Fi = F.conj().T / (n * n)
    k = 2 * np.pi * D.signed_modes(n) / (n * p.h)
    Dx = Fi @ np.diag(np.tile(1j * k, n)) @ F
    Dy = Fi @ np.diag(np.repeat(1j * k, n)) @ F
    diag = lambda a: np.diag(a.numpy().reshape(-1))
    K = diag(p.kappa)
    return -(Dx @ K @ Dx + Dy @ K @ Dy) + diag(p.vx) @ Dx + diag(p.vy) @ Dy + diag(p.sigma)


def test_dense_operator_and_direct_solve():
    n = 8
    p = _random_problem(n=n, seed=4)
    A = _dense_A(p, n)
    u = _rand(n, 5)
    assert np.allclose((A @ u.numpy().reshape(-1)).reshape(n, n), CD.apply_A(p, u).numpy(), atol=1e-10)
    ustar = np.linalg.solve(A, p.f.numpy().reshape(-1)).reshape(n, n)
    assert CD.rtol(p, torch.from_numpy(ustar)) < 1e-12
    # NPBS with M = (I - G V)^{-1} reaches it in one step from u = 0 (Eq. cdr_integral)
    B = np.stack([CD.op_B(p, torch.from_numpy(e.reshape(n, n))).numpy().reshape(-1) for e in np.eye(n * n)], axis=1)
    Binv = np.linalg.inv(B)
    M = lambda r: torch.from_numpy((Binv @ r.numpy().reshape(-1)).reshape(n, n))
    res = CD.npbs_solve(p, M, tol=1e-12, max_iter=3)
    assert res.iters == 1 and np.allclose(res.u.numpy(), ustar, atol=1e-10)


def test_born_series_converges_for_a_weak_perturbation():
    """M = identity (the Born series u <- G(V u + f)) contracts when ||G V|| < 1."""
    p = _random_problem(n=12, seed=6, strength=0.1)
    res = CD.npbs_solve(p, lambda r: r, tol=1e-10, max_iter=500)
    assert res.history[-1] <= 1e-10 and res.iters < 500
    assert all(b <= a * 1.0000001 for a, b in zip(res.history[1:], res.history[2:]))


def test_recipe_velocity_is_incompressible():
    inst = synth.cdr_instance(64, seed=3)
    p = CD.make_problem(inst.kappa, inst.vx, inst.vy, inst.sigma, inst.f, inst.h)
    div = CD.ddx(p, torch.from_numpy(inst.vx).to(torch.complex128)) + CD.ddy(p, torch.from_numpy(inst.vy).to(torch.complex128))
    assert float(div.abs().max()) < 1e-10 * float(np.abs(inst.vx).max() / inst.h)
    assert abs(p.v0x) < 1e-12 and abs(p.v0y) < 1e-12 and inst.kappa.min() > 0 and inst.sigma.min() > 0


def test_adjoint_dot_product_and_dense_transpose():
    """<B x, y> = <x, B^* y> with B = I - G V; and B^* equals the conjugate
    transpose of B's dense matrix."""
    n = 8
    p = _random_problem(n=n, seed=7)
    x, y = _rand(n, 8), _rand(n, 9)
    lhs = torch.vdot(y.reshape(-1), CD.op_B(p, x).reshape(-1))
    rhs = torch.vdot(CD.op_BH(p, y).reshape(-1), x.reshape(-1))
    assert abs(complex(lhs - rhs)) <= 1e-12 * abs(complex(lhs))
    B = np.stack([CD.op_B(p, torch.from_numpy(e.reshape(n, n))).numpy().reshape(-1) for e in np.eye(n * n)], axis=1)
    BH = np.stack([CD.op_BH(p, torch.from_numpy(e.reshape(n, n))).numpy().reshape(-1) for e in np.eye(n * n)], axis=1)
    assert np.allclose(BH, B.conj().T, atol=1e-10)
