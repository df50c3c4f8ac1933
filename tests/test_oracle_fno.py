"""Pins of the oracle's FNO map (App. Architectural Instantiations, Eqs.
fno_impl / lfl / nlfl): the spectral block against DFT sums written out
cell by cell, its special cases, the linearity of M in r that the paper
designs for, and the adjoint / weight-gradient formulas the library's
backward kernels implement (against central differences)."""
import math

import numpy as np
import pytest
import torch

from oracle import fno as FN


def _brute_spectral(x, W, m):
    """irfft2(W * R(rfft2(x))) written as explicit DFT sums: the forward
    half-plane DFT, the channel mixing on the retained modes, then the inverse
    over the Hermitian extension (Y[ky, kx] for kx <= N/2, conj(Y[-ky, N - kx])
    beyond) and the real part."""
    B, Ci, N, _ = x.shape
    Co = W.shape[1]
    rows, cols = FN.retained_rows(N, m), FN.retained_cols(N, m)
    xs = x.numpy()
    Wn = W.numpy()
    y = np.zeros((B, Co, N, N))
    for b in range(B):
        Y = np.zeros((Co, N, N // 2 + 1), dtype=np.complex128)
        for a, ky in enumerate(rows):
            for c, kx in enumerate(cols):
                X = np.zeros(Ci, dtype=np.complex128)
                for i in range(Ci):
                    s = 0j
                    for p in range(N):
                        for q in range(N):
                            s += xs[b, i, p, q] * np.exp(-2j * math.pi * (ky * p + kx * q) / N)
                    X[i] = s
                for o in range(Co):
                    Y[o, ky, kx] = sum(Wn[i, o, a, c] * X[i] for i in range(Ci))
        for o in range(Co):
            for p in range(N):
                for q in range(N):
                    s = 0j
                    for ky in range(N):
                        for kx in range(N):
                            v = Y[o, ky, kx] if kx <= N // 2 else np.conj(Y[o, (-ky) % N, N - kx])
                            s += v * np.exp(2j * math.pi * (ky * p + kx * q) / N)
                    y[b, o, p, q] = (s / (N * N)).real
    return torch.from_numpy(y)


def _rand_w(rng, ci, co, n, m):
    ky, kx = len(FN.retained_rows(n, m)), len(FN.retained_cols(n, m))
    return torch.from_numpy(rng.standard_normal((ci, co, ky, kx)) + 1j * rng.standard_normal((ci, co, ky, kx)))


@pytest.mark.parametrize("m", [2, 4])
def test_spectral_block_matches_dft_sums(m):
    rng = np.random.default_rng(1)
    N = 6
    x = torch.from_numpy(rng.standard_normal((1, 2, N, N)))
    W = _rand_w(rng, 2, 3, N, m)
    assert torch.allclose(FN.spectral(x, W, m), _brute_spectral(x, W, m), rtol=0, atol=1e-12)


def test_retained_mode_sets():
    assert FN.retained_rows(8, 2) == [0, 1, 7]
    assert FN.retained_cols(8, 2) == [0, 1]
    assert FN.retained_rows(8, 5) == list(range(8)) and FN.retained_cols(8, 5) == list(range(5))
    cfg = FN.FnoConfig(n=256)
    assert FN.spectral_shape(cfg, cfg.modes) == (89, 45)
    assert FN.spectral_shape(cfg, cfg.full) == (256, 129)


def test_identity_weights_on_every_mode_give_the_identity():
    rng = np.random.default_rng(2)
    N, C = 8, 3
    x = torch.from_numpy(rng.standard_normal((2, C, N, N)))
    ky, kx = len(FN.retained_rows(N, N // 2 + 1)), len(FN.retained_cols(N, N // 2 + 1))
    W = torch.zeros(C, C, ky, kx, dtype=torch.complex128)
    for i in range(C):
        W[i, i] = 1.0
    assert torch.allclose(FN.spectral(x, W, N // 2 + 1), x, atol=1e-13)


def test_correction_is_real_linear_in_the_residual():
    cfg = FN.FnoConfig(n=16, width=4, modes=3, layers=2)
    P = FN.unflatten(cfg, FN.init_params(cfg, 3) + 0.05)  # nonzero biases on the coefficient branch
    rng = np.random.default_rng(4)
    a = torch.from_numpy(1.0 + 0.3 * rng.standard_normal((2, 16, 16)))
    r1 = torch.from_numpy(rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16)))
    r2 = torch.from_numpy(rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16)))
    lhs = FN.correction(1.7 * r1 - 0.4 * r2, a, P, cfg)
    rhs = 1.7 * FN.correction(r1, a, P, cfg) - 0.4 * FN.correction(r2, a, P, cfg)
    assert torch.allclose(lhs, rhs, atol=1e-12)
    assert FN.correction(torch.zeros_like(r1), a, P, cfg).abs().max() == 0.0


def test_layer_norm_moments():
    rng = np.random.default_rng(5)
    a = torch.from_numpy(3.0 + 2.0 * rng.standard_normal((3, 16, 16)))
    z = FN.layer_norm(a)
    assert torch.allclose(z.mean(dim=(-2, -1)), torch.zeros(3, dtype=torch.float64), atol=1e-13)
    assert torch.allclose((z ** 2).mean(dim=(-2, -1)), torch.ones(3, dtype=torch.float64), atol=1e-5)


@pytest.mark.parametrize("m", [2, 5])
def test_spectral_adjoint_is_the_conjugate_transposed_block(m):
    """<spectral(x; W), g> = <x, spectral(g; conj(W) with channels swapped)>."""
    rng = np.random.default_rng(6)
    N = 8
    x = torch.from_numpy(rng.standard_normal((2, 3, N, N)))
    g = torch.from_numpy(rng.standard_normal((2, 4, N, N)))
    W = _rand_w(rng, 3, 4, N, m)
    lhs = (FN.spectral(x, W, m) * g).sum()
    rhs = (x * FN.spectral(g, W.conj().transpose(0, 1), m)).sum()
    assert float(lhs) == pytest.approx(float(rhs), rel=1e-12)


@pytest.mark.parametrize("m", [2, 5])
def test_spectral_weight_gradient_formula(m):
    """d<spectral(x; W), g>/dW (re + i im) = c_kx / N^2 sum_b G_o conj(X_i), with
    X = rfft2(x), G = rfft2(g) on the retained modes and c = 2 except on the
    self-mirrored columns kx = 0 and kx = N/2 (c = 1): against central
    differences of the real and imaginary parts."""
    rng = np.random.default_rng(7)
    N, Ci, Co = 8, 2, 3
    x = torch.from_numpy(rng.standard_normal((2, Ci, N, N)))
    g = torch.from_numpy(rng.standard_normal((2, Co, N, N)))
    W = _rand_w(rng, Ci, Co, N, m)
    rows = torch.tensor(FN.retained_rows(N, m))
    cols = torch.tensor(FN.retained_cols(N, m))
    X = torch.fft.rfft2(x)[:, :, rows][:, :, :, cols]
    G = torch.fft.rfft2(g)[:, :, rows][:, :, :, cols]
    c = torch.where((cols == 0) | (cols == N // 2), 1.0, 2.0).to(torch.float64)
    grad = torch.einsum("bokl,bikl->iokl", G, X.conj()) * c / (N * N)
    h = 1e-6
    L = lambda Wt: float((FN.spectral(x, Wt, m) * g).sum())
    for (i, o, a, b) in [(0, 0, 0, 0), (1, 2, 1, 1), (0, 1, len(rows) - 1, len(cols) - 1), (1, 0, 2, 0)]:
        E = torch.zeros_like(W)
        E[i, o, a, b] = 1.0
        dre = (L(W + h * E) - L(W - h * E)) / (2 * h)
        dim = (L(W + 1j * h * E) - L(W - 1j * h * E)) / (2 * h)
        assert complex(grad[i, o, a, b]) == pytest.approx(complex(dre, dim), rel=1e-6, abs=1e-9)


def test_param_count_of_the_paper_configuration():
    cfg = FN.FnoConfig(n=256)
    C = 25
    spec = lambda ky, kx: C * C * ky * kx * 2
    expect = (C + C) + 3 * (spec(89, 45) + C * C + C) + 2 * C + spec(256, 129) + C * C + spec(89, 45) + C * C + 2 * C
    assert FN.n_params(cfg) == expect


def test_layer_norm_normalises_each_coefficient_channel_separately():
    """Several coefficient channels (the CDR input kappa, v, sigma): each
    channel of each instance gets zero mean and unit variance on its own."""
    rng = np.random.default_rng(8)
    scale = np.array([1.0, 30.0, 0.01])[None, :, None, None]
    a = torch.from_numpy(5.0 + scale * rng.standard_normal((2, 3, 16, 16)))
    z = FN.layer_norm(a)
    assert torch.allclose(z.mean(dim=(-2, -1)), torch.zeros(2, 3, dtype=torch.float64), atol=1e-12)
    # unit variance up to the eps in the denominator (var / (var + 1e-5))
    v = a.var(dim=(-2, -1), unbiased=False)
    assert torch.allclose((z ** 2).mean(dim=(-2, -1)), v / (v + 1e-5), rtol=1e-12)


def test_several_coefficient_channels_reduce_to_one_and_permute():
    """With lift_a.w nonzero in column 0 only, a coef = 3 network equals the
    coef = 1 network fed channel 0; permuting the channels of a together
    with the columns of lift_a.w leaves M unchanged."""
    rng = np.random.default_rng(9)
    c1 = FN.FnoConfig(n=16, width=4, modes=3, layers=2)
    c3 = FN.FnoConfig(n=16, width=4, modes=3, layers=2, coef=3)
    flat1 = FN.init_params(c1, 3) + 0.05
    P1 = FN.unflatten(c1, flat1)
    P3 = dict(P1)
    w3 = torch.zeros(4, 3, dtype=torch.float64)
    w3[:, 0] = P1["lift_a.w"][:, 0]
    P3["lift_a.w"] = w3
    a = torch.from_numpy(rng.standard_normal((2, 3, 16, 16)) * np.array([1.0, 4.0, 0.1])[None, :, None, None])
    r = torch.from_numpy(rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16)))
    y1 = FN.correction(r, a[:, 0], P1, c1)
    y3 = FN.correction(r, a, P3, c3)
    assert torch.allclose(y1, y3, rtol=1e-12, atol=1e-12)
    P3["lift_a.w"] = torch.from_numpy(rng.standard_normal((4, 3)))
    perm = [2, 0, 1]
    Pp = dict(P3)
    Pp["lift_a.w"] = P3["lift_a.w"][:, perm]
    assert torch.allclose(FN.correction(r, a, P3, c3), FN.correction(r, a[:, perm], Pp, c3), rtol=1e-12, atol=1e-12)
    assert FN.n_params(c3) == FN.n_params(c1) + 2 * 4


def test_residual_branch_reads_re_then_im_and_projects_to_re_then_im():
    """With the lifting's Im column zero, M sees only Re r: M(i s) = 0 for a
    real field s while M(s) != 0; with proj's second row zero the output is
    real.  Pins the (Re, Im) order of Psi's input and of P's output."""
    rng = np.random.default_rng(10)
    cfg = FN.FnoConfig(n=16, width=4, modes=3, layers=1)
    P = FN.unflatten(cfg, FN.init_params(cfg, 4) + 0.05)
    P["lift_r.w"] = P["lift_r.w"].clone()
    P["lift_r.w"][:, 1] = 0.0
    a = torch.from_numpy(rng.standard_normal((1, 16, 16)))
    s = torch.from_numpy(rng.standard_normal((1, 16, 16))).to(torch.complex128)
    assert FN.correction(1j * s, a, P, cfg).abs().max() == 0.0
    assert FN.correction(s, a, P, cfg).abs().max() > 1e-6
    P["proj.w"] = P["proj.w"].clone()
    P["proj.w"][1] = 0.0
    y = FN.correction(s, a, P, cfg)
    assert y.imag.abs().max() == 0.0 and y.real.abs().max() > 1e-6


def test_identity_skip_adds_the_input_and_starts_as_the_born_series():
    """With cfg.skip, M(r) = r + N(r): the difference to the same parameters
    without the skip is r itself, M stays real-linear in r, and the initial
    parameters (zero projection) give M = I exactly."""
    rng = np.random.default_rng(11)
    c0 = FN.FnoConfig(n=16, width=4, modes=3, layers=1)
    c1 = FN.FnoConfig(n=16, width=4, modes=3, layers=1, skip=True)
    P = FN.unflatten(c0, FN.init_params(c0, 5) + 0.05)
    a = torch.from_numpy(rng.standard_normal((2, 16, 16)))
    r1 = torch.from_numpy(rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16)))
    r2 = torch.from_numpy(rng.standard_normal((2, 16, 16)) + 1j * rng.standard_normal((2, 16, 16)))
    assert torch.allclose(FN.correction(r1, a, P, c1) - FN.correction(r1, a, P, c0), r1, atol=1e-12)
    lhs = FN.correction(2.0 * r1 - 3.0 * r2, a, P, c1)
    rhs = 2.0 * FN.correction(r1, a, P, c1) - 3.0 * FN.correction(r2, a, P, c1)
    assert torch.allclose(lhs, rhs, atol=1e-10)
    P0 = FN.unflatten(c1, FN.init_params(c1, 6))
    assert float(P0["proj.w"].abs().max()) == 0.0
    assert torch.allclose(FN.correction(r1, a, P0, c1), r1, atol=0)
