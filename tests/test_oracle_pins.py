"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test compares the FFT-based oracle with something that is not itself:
dense matrices written from the DFT definition, closed forms, or algebraic
identities of Prop. 3.1 / Prop. 3.2, so that a dropped term, a wrong sign, a
transposed operand or a wrong mode ordering fails at least one of them.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import dense as D
from oracle import fgmres as FG
from oracle import helmholtz as H


def _vec(t):
    return t.numpy().reshape(-1)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tiny():
    # non-square grid so that an x/y transposition cannot pass
    inst = synth.small_instance(8, 12, seed=3, layer=2, ppw=5.0)
    p = H.problem_from_instance(inst)
    ops = D.operators(inst.k2, 1.0, p.k0sq, p.eps)
    return inst, p, ops


def _modes(N):
    """-N/2 .. N/2 - 1 for even N (App. Pseudospectral); for odd N (sides 3^b)
    the symmetric -(N-1)/2 .. (N-1)/2, the one band-limited choice."""
    return range(-N // 2, N // 2) if N % 2 == 0 else range(-(N - 1) // 2, (N + 1) // 2)


@pytest.mark.parametrize("ny,nx,h", [(6, 10, 0.7), (9, 6, 1.3)])
def test_plane_wave_symbols(ny, nx, h):
    """G and A act on e^{i xi.x} as 1/lambda and |xi|^2 - k^2 (App. Transform-
    diagonalizable, Helmholtz case), with xi = 2 pi n/(N h) and n taken in
    -N/2..N/2-1, for every mode including the Nyquist ones; h != 1 and
    nx != ny exercise the scaling and orientation, an odd side (9) the
    symmetric mode range of odd lengths."""
    k0sq, eps, k2c = 1.3, 0.45, 1.1 + 0.2j
    lam = H.symbol(ny, nx, h, k0sq, eps)
    y = torch.arange(ny, dtype=torch.float64)[:, None] * h
    x = torch.arange(nx, dtype=torch.float64)[None, :] * h
    for my in _modes(ny):
        for mx in _modes(nx):
            xy = 2 * math.pi * my / (ny * h)
            xx = 2 * math.pi * mx / (nx * h)
            u = torch.exp(1j * (xy * y + xx * x))
            lam_exact = xy * xy + xx * xx - k0sq - 1j * eps
            g = H.green(u, lam)
            assert torch.allclose(g, u / lam_exact, atol=1e-12, rtol=0)
            Au = H.apply_A(u, torch.full((ny, nx), k2c, dtype=torch.complex128), h)
            assert torch.allclose(Au, (xy * xy + xx * xx - k2c) * u, atol=1e-11, rtol=0)


def test_reference_constants_closed_form():
    k2 = torch.tensor([[1.0 + 0.0j, 3.0 + 0.5j], [2.0 + 0.0j, 1.5 + 0.0j]], dtype=torch.complex128)
    k0sq, eps = H.reference_constants(k2)
    assert k0sq == pytest.approx(2.0)
    # |k^2 - 2|: 1, |1 + 0.5i| = 1.118, 0, 0.5
    assert eps == pytest.approx(math.sqrt(1.25))
    V = H.potential(k2, k0sq, eps)
    g = H.gamma_of(V, eps)
    # |1 - gamma| <= 1 pointwise (the CBS convergence condition)
    assert float((1 - g).abs().max()) <= 1 + 1e-15


def test_green_and_A_match_dense(tiny):
    inst, p, ops = tiny
    rng = np.random.default_rng(0)
    q = rng.standard_normal((8, 12)) + 1j * rng.standard_normal((8, 12))
    qt = torch.from_numpy(q)
    assert _rel(_vec(H.green(qt, p.lam)), ops["G"] @ q.reshape(-1)) < 1e-12
    assert _rel(_vec(H.apply_A(qt, p.k2)), ops["A"] @ q.reshape(-1)) < 1e-12
    assert _rel(_vec(H.green_adjoint(qt, p.lam)), ops["G"].conj().T @ q.reshape(-1)) < 1e-12
    assert _rel(_vec(H.op_B(p, qt)), ops["B"] @ q.reshape(-1)) < 1e-12
    assert _rel(_vec(H.op_BH(p, qt)), ops["B"].conj().T @ q.reshape(-1)) < 1e-12


def test_key_identity_prop31(tiny):
    """I - G V = G A (Eq. key_identity), densely and through the FFT oracle."""
    inst, p, ops = tiny
    lhs = np.eye(96) - ops["G"] @ ops["V"]
    rhs = ops["G"] @ ops["A"]
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-12
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((8, 12)) + 0j)
    a = H.op_B(p, x)
    b = H.green(H.apply_A(x, p.k2), p.lam)
    assert float((a - b).norm() / b.norm()) < 1e-13


def test_left_and_integral_forms_agree(tiny):
    """G(V u + f) - u == G(f - A u) (Eq. npbs_integral vs Eq. npbs_iter)."""
    inst, p, ops = tiny
    u = torch.from_numpy(np.random.default_rng(2).standard_normal((8, 12)) * (1 + 1j))
    a = H.born_residual(p, u)
    b = H.born_residual_left(p, u)
    assert float((a - b).norm() / b.norm()) < 1e-13


def test_disk_and_condition_bounds():
    """Low contrast so that q = ||G V||_2 < 1: spectrum of I - G V inside
    |z - 1| <= q and kappa_2 <= (1 + q)/(1 - q) (Eqs. disk_bound, kappa_bound)."""
    inst = synth.small_instance(16, 16, seed=5, layer=3, contrast=0.05, ppw=8.0)
    p = H.problem_from_instance(inst)
    # a larger damping than the default makes ||G V|| < 1
    ops = D.operators(inst.k2, 1.0, p.k0sq, 4.0 * p.eps)
    GV = ops["G"] @ ops["V"]
    q = np.linalg.norm(GV, 2)
    assert q < 1
    B = np.eye(GV.shape[0]) - GV
    ev = np.linalg.eigvals(B)
    assert np.all(np.abs(ev - 1) <= q + 1e-12)
    assert np.linalg.cond(B) <= (1 + q) / (1 - q) + 1e-9


def test_cbs_contraction_spectral_radius():
    """With eps = max|k^2 - k0^2|, the CBS iteration matrix
    M = gamma G V - gamma + 1 has spectral radius below 1."""
    for seed, (ny, nx) in [(7, (16, 16)), (8, (12, 16))]:
        inst = synth.small_instance(ny, nx, seed=seed, layer=3, contrast=0.3, ppw=6.0)
        p = H.problem_from_instance(inst)
        ops = D.operators(inst.k2, 1.0, p.k0sq, p.eps)
        Mdense = ops["gamma"] @ ops["G"] @ ops["V"] - ops["gamma"] + np.eye(ny * nx)
        assert np.allclose(Mdense, ops["Mcbs"])
        rho = max(abs(np.linalg.eigvals(Mdense)))
        assert rho < 1.0


@pytest.mark.parametrize("shape", [(16, 16), (32, 32)])
def test_cbs_converges_to_dense_direct_solve(shape):
    ny, nx = shape
    inst = synth.small_instance(ny, nx, seed=11, layer=ny // 4, ppw=8.0)
    p = H.problem_from_instance(inst)
    A = D.neg_laplacian(ny, nx) - np.diag(inst.k2.reshape(-1))
    ustar = np.linalg.solve(A, inst.f.reshape(-1))
    res = H.cbs_solve(p, tol=1e-12, max_iter=20000)
    assert res.converged
    assert _rel(_vec(res.u), ustar) < 1e-10
    # fixed-point invariants: A u* = f and the Born residual vanishes
    us = torch.from_numpy(ustar.reshape(ny, nx))
    assert H.rtol(p, us) < 1e-12
    assert float(H.born_residual(p, us).norm() / us.norm()) < 1e-12


def test_homogeneous_closed_form():
    """Constant k^2 = kr^2 + i kappa, k0^2 = kr^2, eps = 2 kappa (so V = -i kappa,
    gamma = 1/2): the exact solution is F^{-1}(F f / (|xi|^2 - k^2)), written here
    with the dense DFT; CBS reaches it."""
    ny = nx = 16
    kr2, kappa = 0.8, 0.3
    k2 = np.full((ny, nx), kr2 + 1j * kappa)
    f = synth.small_instance(ny, nx, seed=1, source="random").f
    p = H.make_problem(k2, f, 1.0, k0sq=kr2, eps=2 * kappa)
    assert torch.allclose(p.gamma, torch.full_like(p.gamma, 0.5))
    F = D.dft2(ny, nx)
    ky = 2 * np.pi * D.signed_modes(ny) / ny
    kx = 2 * np.pi * D.signed_modes(nx) / nx
    xi2 = (ky[:, None] ** 2 + kx[None, :] ** 2).reshape(-1)
    uex = (F.conj().T / (ny * nx)) @ ((F @ f.reshape(-1)) / (xi2 - (kr2 + 1j * kappa)))
    res = H.cbs_solve(p, tol=1e-13, max_iter=5000)
    assert _rel(_vec(res.u), uex) < 1e-12


def test_npbs_with_gamma_is_cbs(tiny):
    """M = gamma reduces Eq. npbs_integral to Eq. CBS: identical iterates."""
    inst, p, ops = tiny
    a = H.cbs_solve(p, tol=0, max_iter=25)
    b = H.npbs_solve(p, lambda r: p.gamma * r, tol=0, max_iter=25)
    assert torch.equal(a.u, b.u)


def test_npbs_with_exact_inverse_one_step(tiny):
    """M = (I - G V)^{-1} gives the exact solution after one step from u = 0."""
    inst, p, ops = tiny
    Binv = np.linalg.inv(ops["B"])
    M = lambda r: torch.from_numpy((Binv @ _vec(r)).reshape(8, 12))
    res = H.npbs_solve(p, M, tol=1e-12, max_iter=1)
    ustar = np.linalg.solve(ops["A"], inst.f.reshape(-1))
    assert res.iters == 1
    assert _rel(_vec(res.u), ustar) < 1e-11


def test_direct_solve_with_exact_inverse_one_step(tiny):
    """Eq. direct_iter with M = A^{-1}: the exact solution after one step."""
    inst, p, ops = tiny
    Ainv = np.linalg.inv(ops["A"])
    M = lambda r: torch.from_numpy((Ainv @ _vec(r)).reshape(8, 12))
    res = H.direct_solve(p, M, tol=1e-12, max_iter=1)
    ustar = np.linalg.solve(ops["A"], inst.f.reshape(-1))
    assert res.iters == 1 and _rel(_vec(res.u), ustar) < 1e-11


def test_direct_solve_with_scaled_identity_is_richardson(tiny):
    """Eq. direct_iter with M = alpha I is Richardson's iteration on A u = f:
    five steps against the same recurrence on the dense matrix."""
    inst, p, ops = tiny
    alpha = 0.01 + 0.002j
    res = H.direct_solve(p, lambda r: alpha * r, tol=0, max_iter=5)
    u = np.zeros(96, dtype=np.complex128)
    f = inst.f.reshape(-1)
    for _ in range(5):
        u = u + alpha * (f - ops["A"] @ u)
    assert _rel(_vec(res.u), u) < 1e-12


def test_riesz_equivalence(tiny):
    """Prop. 3.2: ||(I - G V) c - G r|| / ||G r|| = ||A c - r||_R / ||r||_R with
    ||x||_R = ||G x||_2, for arbitrary c and r."""
    inst, p, ops = tiny
    rng = np.random.default_rng(4)
    r = torch.from_numpy(rng.standard_normal((8, 12)) + 1j * rng.standard_normal((8, 12)))
    c = torch.from_numpy(rng.standard_normal((8, 12)) + 1j * rng.standard_normal((8, 12)))
    Gr = H.green(r, p.lam)
    lhs = (H.op_B(p, c) - Gr).norm() / Gr.norm()
    Rn = lambda x: H.green(x, p.lam).norm()
    rhs = Rn(H.apply_A(c, p.k2) - r) / Rn(r)
    assert float(abs(lhs - rhs) / rhs) < 1e-13


def test_adjoint_dot_product(tiny):
    inst, p, ops = tiny
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal((8, 12)) + 1j * rng.standard_normal((8, 12)))
    y = torch.from_numpy(rng.standard_normal((8, 12)) + 1j * rng.standard_normal((8, 12)))
    lhs = torch.vdot(H.op_B(p, x).reshape(-1), y.reshape(-1))
    rhs = torch.vdot(x.reshape(-1), H.op_BH(p, y).reshape(-1))
    assert abs(complex(lhs - rhs)) / abs(complex(lhs)) < 1e-13


@pytest.mark.parametrize("which", ["none", "cbs", "exact"])
def test_fgmres_converges_to_direct(which):
    inst = synth.small_instance(16, 16, seed=21, layer=4, ppw=7.0)
    p = H.problem_from_instance(inst)
    ops = D.operators(inst.k2, 1.0, p.k0sq, p.eps)
    ustar = np.linalg.solve(ops["A"], inst.f.reshape(-1))
    if which == "none":
        P = None
    elif which == "cbs":
        def P(v):
            z = torch.zeros_like(v)
            for _ in range(16):
                z = H.prec_cbs_sweep(p, z, v)
            return z
    else:
        Binv = np.linalg.inv(ops["B"])
        P = lambda v: torch.from_numpy((Binv @ _vec(v)).reshape(16, 16))
    res = FG.fgmres_solve(p, P, restart=20, tol=1e-11, max_iter=3000)
    assert res.converged
    assert _rel(_vec(res.u), ustar) < 1e-9
    if which == "exact":
        assert res.iters == 1


def test_fgmres_full_restart_is_exact_in_n_steps():
    """Unpreconditioned GMRES without restart terminates in at most n steps."""
    inst = synth.small_instance(4, 6, seed=2, layer=1, ppw=4.0, source="random")
    p = H.problem_from_instance(inst)
    res = FG.fgmres_solve(p, None, restart=24, tol=1e-12, max_iter=24)
    A = D.neg_laplacian(4, 6) - np.diag(inst.k2.reshape(-1))
    ustar = np.linalg.solve(A, inst.f.reshape(-1))
    assert _rel(_vec(res.u), ustar) < 1e-9


def test_prec_sweep_is_richardson_on_B_and_the_cbs_step_for_v_equal_G_f(tiny):
    """The FGMRES CBS preconditioner sweep z + gamma (v - B z) against the dense
    B and gamma, and for v = G f it is Eq. (CBS) itself (G(V z + f) - z =
    G f - B z), through a different code path (the Born residual)."""
    inst, p, ops = tiny
    rng = np.random.default_rng(11)
    shape = inst.k2.shape
    z = torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    v = torch.from_numpy(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    ref = _vec(z) + ops["gamma"] @ (_vec(v) - ops["B"] @ _vec(z))
    assert _rel(_vec(H.prec_cbs_sweep(p, z, v)), ref) < 1e-12
    Gf = H.green(p.f, p.lam)
    assert _rel(_vec(H.prec_cbs_sweep(p, z, Gf)), _vec(H.cbs_step(p, z))) < 1e-12


@pytest.mark.parametrize("k", [1, 3, 6])
def test_fgmres_iterate_minimises_the_residual_over_the_krylov_space(tiny, k):
    """k unpreconditioned FGMRES steps from u = 0 inside one cycle give the
    element of K_k(B, b) = span{b, B b, ..., B^(k-1) b}, b = G f, with the least
    ||b - B u||_2 (the defining property of GMRES, Saad 1993), found here by
    least squares with the dense B: a dropped Givens term, a wrong conjugate or
    a misplaced Hessenberg entry moves the iterate off the minimiser."""
    inst, p, ops = tiny
    B = ops["B"]
    b = ops["G"] @ inst.f.reshape(-1)
    cols = [b]
    for _ in range(k - 1):
        cols.append(B @ cols[-1])
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))  # orthonormal basis of the same space
    c, *_ = np.linalg.lstsq(B @ Q, b, rcond=None)
    u_ls = Q @ c
    res = FG.fgmres_solve(p, None, restart=20, tol=1e-14, max_iter=k)
    assert res.iters == k
    assert _rel(_vec(res.u), u_ls) < 1e-8
    # and the residual can only fall from one k to the next
    assert np.linalg.norm(b - B @ _vec(res.u)) <= np.linalg.norm(b) * (1 + 1e-12)


def test_free_space_green_function_trend():
    """Physics sanity, not parity: with an absorbing layer the field of a point
    source in a homogeneous medium approaches (i/4) H0^(1)(k r) in an annulus,
    and the mismatch falls as the layer widens."""
    scipy_special = pytest.importorskip("scipy.special")
    errs = []
    for N, W in [(128, 16), (192, 48)]:
        omega = 2 * math.pi / 12
        n = np.ones((N, N))
        f = np.zeros((N, N), np.complex128)
        c = N // 2
        f[c, c] = 1.0
        inst = synth.make_instance(n, omega, W, f, abs_amp_over_omega2=0.5)
        # a homogeneous medium: the layer sets eps; damping far from the source is small
        p = H.problem_from_instance(inst)
        res = H.cbs_solve(p, tol=1e-7, max_iter=20000, check_every=50)
        yy, xx = np.mgrid[0:N, 0:N]
        r = np.hypot(yy - c, xx - c)
        ring = (r > 6) & (r < 20)
        ex = 0.25j * scipy_special.hankel1(0, omega * r[ring])
        num = res.u.numpy()[ring]
        errs.append(np.linalg.norm(num - ex) / np.linalg.norm(ex))
    assert errs[1] < errs[0]
    assert errs[1] < 0.15


def test_absorbing_medium_special_cells():
    """The layer reading of Sec. 3.1 on a 7 x 9 grid with a 2-cell layer:
    interior cells carry no absorption, the outermost ring the full a omega^2,
    one cell in a quarter of it (rho = 1/2, quadratic ramp), corners take the
    larger depth, and the real part is omega^2 n^2."""
    rng = np.random.default_rng(5)
    n = 1.0 + 0.3 * rng.standard_normal((7, 9))
    om, a, W = 0.7, 0.5, 2
    k2 = H.absorbing_medium(n, om, W, a).numpy()
    full = a * om * om
    assert np.array_equal(k2.real, (om * om) * (n * n))
    assert k2[3, 4].imag == 0.0 and k2[2, 2].imag == 0.0 and k2[4, 6].imag == 0.0
    for y, x in [(0, 4), (6, 4), (3, 0), (3, 8), (0, 0), (6, 8)]:
        assert k2[y, x].imag == pytest.approx(full, rel=1e-15)
    for y, x in [(1, 4), (5, 4), (3, 1), (3, 7), (1, 1), (5, 7)]:
        assert k2[y, x].imag == pytest.approx(full / 4, rel=1e-15)
    assert k2[1, 0].imag == pytest.approx(full, rel=1e-15)  # corner: the deeper axis wins
    assert np.allclose(k2.imag, k2.imag[::-1, ::-1], rtol=0, atol=0)
    assert not np.any(H.absorbing_medium(n, om, 0, a).numpy().imag)


def test_absorbing_medium_is_the_workload_recipe():
    """The synthetic workloads assemble k^2 with the same layer (96^2 law)."""
    inst = synth.workload_96()[0]
    k2 = H.absorbing_medium(inst.n, inst.omega, inst.layer, 0.5).numpy()
    assert np.allclose(k2, inst.k2, rtol=1e-15, atol=0)
