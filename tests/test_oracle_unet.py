"""Pins of the oracle's network, unrolled loss and optimiser.

conv2d is a library step; these tests pin how the oracle uses it (kernel
orientation, padding, channel order) to brute force, the scale wrapper to
positive homogeneity, the reference gradient to central finite differences
(h = 1e-3, float64, 8 instances at 32x32) and AdamW to its closed form.
"""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import synth
from oracle import helmholtz as H
from oracle import unet as U


def _params(seed=0):
    flat = torch.from_numpy(synth.random_weights([s for _, s in U.PARAM_SPEC], seed=seed)).double()
    return flat, U.unflatten(flat)


def test_param_count():
    # 9 * sum(Cin*Cout) over the 17 3x3 convs + biases + the 32->2 head
    assert U.n_params() == 9 * 237664 + sum(c for _, _, c in U.CONVS) + 64


def test_conv_orientation_brute_force():
    """Cross-correlation with zero padding 1 and OIHW weights, by loops."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 4, 5))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    ref = np.zeros((1, 3, 4, 5))
    for co in range(3):
        for y in range(4):
            for xx in range(5):
                acc = b[co]
                for ci in range(2):
                    for dy in range(3):
                        for dx in range(3):
                            yy, xs = y + dy - 1, xx + dx - 1
                            if 0 <= yy < 4 and 0 <= xs < 5:
                                acc += w[co, ci, dy, dx] * x[0, ci, yy, xs]
                ref[0, co, y, xx] = acc
    got = Fnn.conv2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), padding=1)
    assert np.allclose(got.numpy(), ref, atol=1e-12)


def test_pool_up_and_gelu_definitions():
    x = torch.arange(16, dtype=torch.float64).reshape(1, 1, 4, 4)
    p = U._pool(x)
    assert p[0, 0, 0, 0] == (0 + 1 + 4 + 5) / 4
    u = U._up(p)
    assert u.shape == x.shape and u[0, 0, 1, 1] == p[0, 0, 0, 0] and u[0, 0, 2, 3] == p[0, 0, 1, 1]
    t = torch.tensor([-1.5, 0.0, 0.7], dtype=torch.float64)
    ref = torch.tensor([v * 0.5 * (1 + math.erf(v / math.sqrt(2))) for v in t.tolist()], dtype=torch.float64)
    assert torch.allclose(Fnn.gelu(t), ref, atol=1e-15)


def test_each_convolution_runs_at_its_level_resolution(monkeypatch):
    """U-Net layout (pool, then the level's two convolutions; upsample, then
    the up convolution): every convolution named for level l sees an input of
    (H / 2^l) x (W / 2^l), recorded at the library conv2d call itself."""
    _, P = _params(9)
    seen = {}
    conv = U.Fnn.conv2d

    def spy(x, w, *a, **k):
        seen[id(w)] = tuple(x.shape[-2:])
        return conv(x, w, *a, **k)

    monkeypatch.setattr(U.Fnn, "conv2d", spy)
    H_, W_ = 32, 48
    U.network(torch.zeros(1, 3, H_, W_, dtype=torch.float64), P)
    for name, _, _ in U.CONVS:
        lvl = int(name[-2] if name[-1] in "ab" else name[-1])
        assert seen[id(P[name + ".w"])] == (H_ >> lvl, W_ >> lvl), name
    assert seen[id(P["out.w"])] == (H_, W_)


def test_oracle_conv_applies_the_erf_gelu():
    """The oracle's conv + activation with a centre-tap identity kernel is the
    erf-form GELU x Phi(x) (the tanh approximation differs by up to ~1e-3)."""
    t = torch.linspace(-3.0, 3.0, 25, dtype=torch.float64).reshape(1, 1, 5, 5)
    w = torch.zeros(1, 1, 3, 3, dtype=torch.float64)
    w[0, 0, 1, 1] = 1.0
    got = U._conv_gelu(t, {"c.w": w, "c.b": torch.zeros(1, dtype=torch.float64)}, "c")
    ref = torch.tensor([v * 0.5 * (1 + math.erf(v / math.sqrt(2))) for v in t.reshape(-1).tolist()],
                       dtype=torch.float64).reshape(t.shape)
    assert torch.allclose(got, ref, atol=1e-15, rtol=0)


def test_decoder_concatenates_skip_then_up():
    """Channel order of the decoder input (the reading: [skip, up]): with the
    up-branch convolution zeroed its GELU output is exactly 0, so the weights
    that dec<l>a applies to channels [C, 2C) cannot change the output, while
    those on [0, C) (the skip) do."""
    _, P = _params(7)
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.standard_normal((1, 3, 16, 16)))
    for lvl, C in [(2, 128), (0, 32)]:
        Q = {k: v.clone() for k, v in P.items()}
        Q[f"up{lvl}.w"].zero_()
        Q[f"up{lvl}.b"].zero_()
        y0 = U.network(x, Q)
        Q1 = {k: v.clone() for k, v in Q.items()}
        Q1[f"dec{lvl}a.w"][:, C:] += 0.5
        assert torch.equal(U.network(x, Q1), y0), lvl
        Q2 = {k: v.clone() for k, v in Q.items()}
        Q2[f"dec{lvl}a.w"][:, :C] += 0.5
        assert not torch.allclose(U.network(x, Q2), y0), lvl


def test_output_channels_are_real_then_imaginary():
    """Head channel 0 is Re c and channel 1 is Im c: zeroing one head row
    makes the correction purely imaginary or purely real."""
    _, P = _params(8)
    rng = np.random.default_rng(6)
    r = torch.from_numpy(rng.standard_normal((1, 16, 16)) + 1j * rng.standard_normal((1, 16, 16)))
    n = torch.from_numpy(1 + 0.1 * rng.standard_normal((1, 16, 16)))
    for row, part in [(1, "imag"), (0, "real")]:
        Q = {k: v.clone() for k, v in P.items()}
        Q["out.w"][row].zero_()
        c = U.correction(r, n, Q)
        assert float(getattr(c, part).abs().max()) == 0.0
        other = "real" if part == "imag" else "imag"
        assert float(getattr(c, other).abs().max()) > 0.0


def test_scale_wrapper_positive_homogeneity():
    _, P = _params(1)
    rng = np.random.default_rng(3)
    r = torch.from_numpy(rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16)))
    n = torch.from_numpy(1 + 0.2 * rng.standard_normal((2, 16, 16)))
    a = U.correction(3.7 * r, n, P)
    b = 3.7 * U.correction(r, n, P)
    assert float((a - b).abs().max() / b.abs().max()) < 1e-12


def _batch(count=8, N=32):
    insts = [synth.small_instance(N, N, seed=100 + i, layer=4, ppw=8.0) for i in range(count)]
    probs = [H.problem_from_instance(i) for i in insts]
    V, lam, f, n = U.problems_to_batch(probs)
    # residual snapshots from short CBS runs of different lengths
    u0 = torch.stack([H.cbs_solve(p, tol=0, max_iter=3 * i).u for i, p in enumerate(probs)])
    return V, lam, f, n, u0


def test_loss_is_one_when_network_is_zero():
    flat, _ = _params(2)
    P = U.unflatten(torch.zeros_like(flat))
    V, lam, f, n, u0 = _batch(2, 16)
    assert float(U.unrolled_loss(P, V, lam, f, n, u0)) == pytest.approx(1.0, abs=1e-14)


def test_loss_gradient_matches_central_fd():
    """Autograd of the float64 oracle loss vs central finite differences,
    h = 1e-3, on 8 instances at 32x32."""
    flat, _ = _params(4)
    V, lam, f, n, u0 = _batch(8, 32)
    th = flat.clone().requires_grad_(True)
    L = U.unrolled_loss(U.unflatten(th), V, lam, f, n, u0)
    (g,) = torch.autograd.grad(L, th)
    rng = np.random.default_rng(7)
    # a few coordinates in each of: first conv, bottleneck, decoder, head
    names = [nm for nm, _ in U.PARAM_SPEC]
    offs = np.cumsum([0] + [math.prod(s) for _, s in U.PARAM_SPEC])
    picks = []
    for nm in ["enc0a.w", "enc0a.b", "enc3b.w", "dec0b.w", "out.w"]:
        k = names.index(nm)
        picks += list(rng.integers(offs[k], offs[k + 1], size=2))
    h = 1e-3
    for idx in picks:
        e = torch.zeros_like(flat)
        e[idx] = h
        lp = float(U.unrolled_loss(U.unflatten(flat + e), V, lam, f, n, u0))
        lm = float(U.unrolled_loss(U.unflatten(flat - e), V, lam, f, n, u0))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(g[idx])) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (idx, fd, float(g[idx]))


def _batch_kinds(count=2, N=16):
    insts = [synth.small_instance(N, N, seed=200 + i, layer=3, ppw=6.0) for i in range(count)]
    probs = [H.problem_from_instance(i) for i in insts]
    V, lam, f, n = U.problems_to_batch(probs)
    k2 = torch.stack([p.k2 for p in probs])
    xi2 = H.xi_squared(N, N, 1.0).to(torch.complex128)
    u0 = torch.stack([H.cbs_solve(p, tol=0, max_iter=2 + 3 * i).u for i, p in enumerate(probs)])
    return insts, probs, V, lam, k2, xi2, f, n, u0


@pytest.mark.parametrize("kind", U.LOSS_KINDS)
def test_loss_kinds_are_one_for_a_zero_network(kind):
    insts, probs, V, lam, k2, xi2, f, n, u0 = _batch_kinds()
    L = U.unrolled_loss_kind(lambda x: torch.zeros_like(x), kind, V, lam, k2, xi2, f, u0)
    assert float(L) == pytest.approx(1.0, abs=1e-14)


def test_loss_kinds_vanish_for_the_exact_inverse_of_their_format():
    """Each objective is zero for the operator its format asks the network to
    learn (Sec. 4): A^{-1} for Eq. L_dir (input: the plain residual), (G A)^{-1}
    for Eq. L_bs_l2 and (I - G V)^{-1} for Eq. L_bs_Reta_integral (input: the
    Born residual).  Dense inverses from the DFT definition, 8 x 12 grid."""
    from oracle import dense as D
    inst = synth.small_instance(8, 12, seed=3, layer=2, ppw=5.0)
    p = H.problem_from_instance(inst)
    ops = D.operators(inst.k2, 1.0, p.k0sq, p.eps)
    V, lam, f, n = U.problems_to_batch([p])
    k2 = p.k2[None]
    xi2 = H.xi_squared(8, 12, 1.0).to(torch.complex128)
    u0 = H.cbs_solve(p, tol=0, max_iter=3).u[None]
    inv = {"dir": np.linalg.inv(ops["A"]), "bs_l2": np.linalg.inv(ops["G"] @ ops["A"]),
           "bs_reta": np.linalg.inv(ops["B"])}
    for kind in U.LOSS_KINDS:
        Mi = inv[kind]
        M = lambda x, Mi=Mi: torch.from_numpy((Mi @ x[0].numpy().reshape(-1)).reshape(1, 8, 12))
        L = float(U.unrolled_loss_kind(M, kind, V, lam, k2, xi2, f, u0, unroll=2))
        assert L < 1e-20, (kind, L)
        # and the other formats' inverses do not zero it
        for other in U.LOSS_KINDS:
            if other != kind and not (kind != "dir" and other != "dir"):
                Mo = inv[other]
                Mx = lambda x, Mo=Mo: torch.from_numpy((Mo @ x[0].numpy().reshape(-1)).reshape(1, 8, 12))
                assert float(U.unrolled_loss_kind(Mx, kind, V, lam, k2, xi2, f, u0, unroll=2)) > 1e-6


@pytest.mark.parametrize("kind", U.LOSS_KINDS)
def test_loss_kinds_match_dense_one_and_two_step_formulas(kind):
    """Each objective of Sec. 4 for the network M = alpha I, from dense A and G
    (DFT definition): t_{k+1} = t_k - A alpha P_in t_k, loss = mean over k of
    ||P_out t_{k+1}||^2 / ||P_out t_0||^2 with (P_in, P_out) = (I, I) for
    Eq. L_dir, (G, I) for Eq. L_bs_l2 and (G, G) for Eq. L_bs_Reta_integral;
    a swapped projection fails it."""
    from oracle import dense as D
    inst = synth.small_instance(8, 12, seed=3, layer=2, ppw=5.0)
    p = H.problem_from_instance(inst)
    ops = D.operators(inst.k2, 1.0, p.k0sq, p.eps)
    V, lam, f, n = U.problems_to_batch([p])
    k2 = p.k2[None]
    xi2 = H.xi_squared(8, 12, 1.0).to(torch.complex128)
    u0 = H.cbs_solve(p, tol=0, max_iter=3).u[None]
    A, G = ops["A"], ops["G"]
    I = np.eye(A.shape[0])
    Pin = I if kind == "dir" else G
    Pout = G if kind == "bs_reta" else I
    alpha = 0.37 - 0.21j
    t = inst.f.reshape(-1) - A @ u0[0].numpy().reshape(-1)
    t0n = np.linalg.norm(Pout @ t) ** 2
    for unroll in (1, 2):
        tk, acc = t.copy(), 0.0
        for _ in range(unroll):
            tk = tk - A @ (alpha * (Pin @ tk))
            acc += np.linalg.norm(Pout @ tk) ** 2 / t0n
        L = float(U.unrolled_loss_kind(lambda x: alpha * x, kind, V, lam, k2, xi2, f, u0, unroll=unroll))
        assert L == pytest.approx(acc / unroll, rel=1e-10), (kind, unroll)


def test_reta_kind_in_true_residual_coordinates_equals_born_state_loss():
    """Eq. L_bs_Reta_integral through the true residual t (x = G t, metric
    ||G t||) equals the Born-state form r_{k+1} = r_k - (I - G V) c_k used for
    training: the key identity G A = I - G V (Eq. key_identity) inside the loss."""
    flat, P = _params(5)
    insts, probs, V, lam, k2, xi2, f, n, u0 = _batch_kinds(3, 16)
    a = U.unrolled_loss_kind(lambda x: U.correction(x, n, P), "bs_reta", V, lam, k2, xi2, f, u0)
    b = U.unrolled_loss(P, V, lam, f, n, u0)
    assert float(abs(a - b) / b) < 1e-12


@pytest.mark.parametrize("kind", ["dir", "bs_l2"])
def test_loss_kind_gradient_matches_central_fd(kind):
    """Autograd of the float64 oracle objective vs central differences, h = 1e-3."""
    flat, _ = _params(6)
    insts, probs, V, lam, k2, xi2, f, n, u0 = _batch_kinds(2, 16)
    th = flat.clone().requires_grad_(True)
    loss = lambda t: U.unrolled_loss_kind(lambda x: U.correction(x, n, U.unflatten(t)), kind, V, lam, k2, xi2, f,
                                          u0, unroll=2)
    (g,) = torch.autograd.grad(loss(th), th)
    names = [nm for nm, _ in U.PARAM_SPEC]
    offs = np.cumsum([0] + [math.prod(s) for _, s in U.PARAM_SPEC])
    rng = np.random.default_rng(9)
    picks = [int(rng.integers(offs[names.index(nm)], offs[names.index(nm) + 1])) for nm in
             ["enc0a.w", "enc2b.w", "dec1a.b", "out.w"]]
    h = 1e-3
    with torch.no_grad():
        for idx in picks:
            e = torch.zeros_like(flat)
            e[idx] = h
            fd = (float(loss(flat + e)) - float(loss(flat - e))) / (2 * h)
            assert abs(fd - float(g[idx])) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (kind, idx, fd, float(g[idx]))


def test_adamw_first_step_closed_form():
    """At step 1, mhat = g and vhat = g^2, so the update is
    -lr * g / (|g| + eps) after decay by (1 - lr wd)."""
    # the last gradient is tiny against sqrt(eps): eps added outside the root
    # (Adam's form) and inside it differ by a factor of ~10 there
    th = torch.tensor([1.0, -2.0, 0.5, 0.25], dtype=torch.float64)
    g = torch.tensor([0.3, -0.01, 0.0, 1e-6], dtype=torch.float64)
    lr, wd, eps = 1e-3, 1e-2, 1e-8
    z = torch.zeros(4, dtype=torch.float64)
    new, m, v = U.adamw_step(th, g, z, z.clone(), 1, lr=lr, weight_decay=wd, eps=eps)
    expect = th * (1 - lr * wd) - lr * g / (g.abs() + eps)
    assert torch.allclose(new, expect, atol=1e-15, rtol=0)
    assert torch.allclose(m, 0.1 * g) and torch.allclose(v, 0.001 * g * g)
