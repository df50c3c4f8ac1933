"""Pins of the Newton-Born oracle (App. Full Derivations, Nonlinear PDE via
Newton-Born Linearization; App. Verification, Newton linear systems): the
five-point Laplacian against the dense Kronecker matrix, the DST-I against
scipy's DST-I, the closed-form eigenpairs of L_D,
the Born identity I - G V = G J, the adjoint, and Newton against a
manufactured exact solution."""
import math

import numpy as np
import pytest
import torch

from oracle import newton as NW


def _dense_lap(N):
    """(T (x) I + I (x) T) / h^2 with T = tridiag(-1, 2, -1): row-major [y][x] unknowns."""
    h = NW.spacing(N)
    T = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    return (np.kron(T, np.eye(N)) + np.kron(np.eye(N), T)) / (h * h)


def _dense_sine(N):
    j = np.arange(1, N + 1)
    return np.sin(math.pi * np.outer(j, j) / (N + 1))


@pytest.mark.parametrize("N", [5, 8])
def test_lap_D_is_the_kronecker_five_point_matrix(N):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((N, N))
    got = NW.lap_D(torch.from_numpy(x), NW.spacing(N)).numpy().ravel()
    assert np.allclose(got, _dense_lap(N) @ x.ravel(), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("N", [4, 7])
def test_dst2_is_scipys_dst_one_on_both_axes(N):
    """Against a library routine: scipy's DST-I is 2 sum_n x_n sin(pi (k+1)(n+1)/(N+1)),
    so S q S = dst(dst(q, axis 0), axis 1) / 4; and S^2 = (N + 1)/2 I per axis."""
    import scipy.fft as sfft
    rng = np.random.default_rng(2)
    q = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    ref = sfft.dst(sfft.dst(q, type=1, axis=0), type=1, axis=1) / 4.0
    got = NW.dst2(torch.from_numpy(q)).numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    S = _dense_sine(N)
    assert np.allclose(S @ S, (N + 1) / 2 * np.eye(N), atol=1e-12)


def test_sine_modes_are_eigenfunctions_of_L_D():
    """L_D sin(p pi x) sin(q pi y) = lambda_pq sin(p pi x) sin(q pi y) on the
    grid, lambda_pq = (4/h^2)(sin^2(p pi h/2) + sin^2(q pi h/2))."""
    N = 9
    h = NW.spacing(N)
    y, x = NW.grid(N)
    lam = NW.laplacian_eigenvalues(N)
    for p, q in [(1, 1), (2, 5), (9, 3)]:
        phi = torch.sin(q * math.pi * x) * torch.sin(p * math.pi * y)
        assert torch.allclose(NW.lap_D(phi, h), lam[p - 1, q - 1] * phi, rtol=1e-10, atol=1e-8)
    assert float(lam[0, 0]) == pytest.approx(8.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2, rel=1e-14)


def _state(N, seed, alpha=0.0):
    rng = np.random.default_rng(seed)
    u = torch.from_numpy(-10.0 + 5.0 * rng.standard_normal((N, N)))
    f = NW.source(N)
    return NW.linearise(u, f, alpha)


def test_green_inverts_the_reference_jacobian():
    s = _state(8, 3, alpha=1.5)
    rng = np.random.default_rng(4)
    q = torch.from_numpy(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    assert torch.allclose(NW.apply_J0(s, NW.green(s, q)), q, rtol=1e-10, atol=1e-10)
    J0 = _dense_lap(8) + s.shift * np.eye(64)
    assert np.allclose(NW.green(s, q).numpy().ravel(), np.linalg.solve(J0, q.numpy().ravel()), rtol=1e-10)
    # the shift keeps the mean reaction: alpha - 2 mean(u)
    assert s.shift == pytest.approx(1.5 - 2.0 * float(s.u.mean()), rel=1e-14)


def test_born_identity_and_adjoint():
    """I - G V = G J (Eq. newton_born_identity) on random fields, and
    <B x, y> = <x, B^* y>; V = J0 - J is the pointwise 2 (u - mean u) + alpha."""
    s = _state(8, 5, alpha=0.7)
    rng = np.random.default_rng(6)
    x = torch.from_numpy(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    y = torch.from_numpy(rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    assert torch.allclose(NW.op_B(s, x), NW.green(s, NW.jacobian(s.u, x, s.h)), rtol=1e-10, atol=1e-10)
    Jd = _dense_lap(8) - 2.0 * np.diag(s.u.numpy().ravel())
    J0d = _dense_lap(8) + s.shift * np.eye(64)
    assert np.allclose(np.diag(J0d - Jd), (2.0 * (s.u - s.u.mean()) + 0.7).numpy().ravel())
    lhs = complex((NW.op_B(s, x) * y.conj()).sum())
    rhs = complex((x * NW.op_BH(s, y).conj()).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_inner_solve_with_the_exact_inverse_takes_one_step_and_born_matches_dense():
    s = _state(8, 7)
    Jd = _dense_lap(8) - 2.0 * np.diag(s.u.numpy().ravel())
    B = np.linalg.solve(_dense_lap(8) + s.shift * np.eye(64), Jd)  # G J
    Minv = lambda q: torch.from_numpy(np.linalg.solve(B, q.numpy().ravel()).reshape(8, 8))
    res = NW.inner_solve(s, Minv, tol=1e-10)
    assert res.iters == 1
    born = NW.inner_solve(s, lambda q: q, tol=1e-11, max_iter=5000)
    exact = np.linalg.solve(Jd, s.r.numpy().ravel())
    assert np.allclose(born.delta.numpy().ravel(), exact, rtol=1e-8, atol=1e-8 * np.abs(exact).max())


def test_newton_recovers_a_manufactured_solution():
    """f := L_D u* - u*^2 for a chosen u* (so F(u*) = 0 exactly); Newton with
    Born inner solves from a perturbed start returns u*, and the last steps
    converge quadratically."""
    N = 16
    h = NW.spacing(N)
    y, x = NW.grid(N)
    ustar = -20.0 * torch.sin(math.pi * x) * torch.sin(math.pi * y) + 3.0 * torch.sin(2 * math.pi * x) * torch.sin(
        3 * math.pi * y)
    f = NW.lap_D(ustar, h) - ustar * ustar
    assert float(torch.linalg.norm(NW.nonlinear_residual(ustar, f, h))) < 1e-9
    u0 = ustar + 2.0 * torch.sin(math.pi * x) * torch.sin(2 * math.pi * y)
    res = NW.newton(u0, f, lambda s, q: q, tol=1e-12, max_steps=20, inner_tol=1e-12, inner_max=5000)
    assert torch.allclose(res.u, ustar, rtol=1e-9, atol=1e-9)
    e = res.history
    k = next(i for i in range(len(e)) if e[i] < 1e-3)
    assert e[k + 1] <= 10.0 * e[k] ** 2 + 1e-13


def test_paper_source_and_grid():
    N = 64
    assert NW.spacing(N) == pytest.approx(1.0 / 65.0)
    f = NW.source(N)
    y, x = NW.grid(N)
    assert float(x[0, 0]) == pytest.approx(1.0 / 65.0) and float(x[0, -1]) == pytest.approx(64.0 / 65.0)
    assert float(f.min()) == pytest.approx(-1600.0 * math.sin(32 * math.pi / 65) ** 2, rel=1e-12)
