"""The FNO network on the GPU (App. Architectural Instantiations) against the
float64 oracle: forward, the hand-written adjoint and weight gradients, the
metric-matched training step, and NPBS / FGMRES solves driven by it.

Tolerance: the library's FNO runs in float32 (FFTs of n^2 points, channel
sums of at most 25 terms): about 1e-6 relative error per operation, a few
1e-6 over a forward.  Forward outputs are checked at relative L2 <= 1e-4,
gradients (forward and backward) at <= 1e-3.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import fno as FN
from oracle import helmholtz as H
from oracle import unet as U
from tests.gpu_common import ctx, oracle_problem, rel_l2, random_field, setup_batch

pytestmark = pytest.mark.gpu

CONFIGS = [FN.FnoConfig(n=32, width=8, modes=5, layers=2), FN.FnoConfig(n=64, width=25, modes=12, layers=3)]


def _params(cfg, seed):
    """Seeded parameters in the canonical order, float32 (biases nonzero)."""
    p = FN.init_params(cfg, seed).numpy()
    rng = np.random.default_rng(seed)
    o = 0
    for name, shape in FN.param_spec(cfg):
        k = int(np.prod(shape))
        if name.endswith(".b"):
            p[o:o + k] = 0.1 * rng.standard_normal(k)
        o += k
    return p.astype(np.float32)


def _net(capi, cfg, seed):
    net = capi.Net.fno(cfg.n, cfg.width, cfg.modes, cfg.layers, seed=1)
    assert net.num_params() == FN.n_params(cfg)
    net.set_params(_params(cfg, seed))
    return net


def _oracle_params(cfg, seed, requires_grad=False):
    flat = torch.from_numpy(_params(cfg, seed).astype(np.float64)).requires_grad_(requires_grad)
    return flat, FN.unflatten(cfg, flat)


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"n{c.n}c{c.width}m{c.modes}l{c.layers}")
def test_fno_forward_parity(cfg):
    capi, c = ctx()
    insts = [synth.small_instance(cfg.n, cfg.n, seed=500 + j) for j in range(3)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    rs = [random_field((cfg.n, cfg.n), 510 + j) * (10.0 ** (j - 1)) for j in range(3)]
    r = b.pack(rs)
    out = torch.zeros_like(r)
    net = _net(capi, cfg, 7)
    capi.npbs_net_forward(c, net, b, r, n, out)
    torch.cuda.synchronize()
    _, P = _oracle_params(cfg, 7)
    a = torch.from_numpy(np.stack([i.n.astype(np.float32).astype(np.float64) for i in insts]))
    ref = FN.correction(torch.from_numpy(np.stack(rs)), a, P, cfg).numpy()
    got = b.unpack(out)
    for j in range(3):
        assert rel_l2(got[j], ref[j]) <= 1e-4, (j, rel_l2(got[j], ref[j]))


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"n{c.n}c{c.width}m{c.modes}l{c.layers}")
def test_fno_backward_matches_autograd(cfg):
    """npbs_net_backward vs autograd of the oracle: L = <g, M(r; a)> (real inner
    product) for a fixed random g; parameter gradients and the gradient in r."""
    capi, c = ctx()
    insts = [synth.small_instance(cfg.n, cfg.n, seed=520 + j) for j in range(3)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    rs = [random_field((cfg.n, cfg.n), 530 + j) for j in range(3)]
    gs = [random_field((cfg.n, cfg.n), 540 + j) for j in range(3)]
    r, g = b.pack(rs), b.pack(gs)
    gr = torch.zeros_like(r)
    net = _net(capi, cfg, 8)
    net.zero_grad()
    capi.npbs_net_backward(c, net, b, r, n, g, gr)
    torch.cuda.synchronize()
    flat, P = _oracle_params(cfg, 8, requires_grad=True)
    rr = torch.from_numpy(np.stack(rs).real.copy()).requires_grad_(True)
    ri = torch.from_numpy(np.stack(rs).imag.copy()).requires_grad_(True)
    a = torch.from_numpy(np.stack([i.n.astype(np.float32).astype(np.float64) for i in insts]))
    out = FN.correction(torch.complex(rr, ri), a, P, cfg)
    gt = torch.from_numpy(np.stack(gs))
    L = (gt.real * out.real + gt.imag * out.imag).sum()
    dth, dre, dim = torch.autograd.grad(L, [flat, rr, ri])
    gw = net.get_grads()
    ref = dth.numpy()
    assert rel_l2(gw, ref) <= 1e-3, rel_l2(gw, ref)
    o = 0
    for name, shape in FN.param_spec(cfg):
        k = int(np.prod(shape))
        assert rel_l2(gw[o:o + k], ref[o:o + k]) <= 1e-3, (name, rel_l2(gw[o:o + k], ref[o:o + k]))
        o += k
    got_r = np.stack(b.unpack(gr))
    assert rel_l2(got_r, (dre + 1j * dim).numpy()) <= 1e-3


def test_fno_train_step_loss_and_gradient_match_oracle():
    """npbs_train_step with the FNO (4 unrolls, lr = 0) on 8 instances at 32^2
    against the oracle's metric-matched unrolled loss and its autograd gradient."""
    cfg = CONFIGS[0]
    capi, c = ctx()
    insts = [synth.small_instance(32, 32, seed=100 + i, layer=4, ppw=8.0) for i in range(8)]
    probs = [oracle_problem(i) for i in insts]
    snaps = [H.cbs_solve(p, tol=0, max_iter=3 * i).u.numpy() for i, p in enumerate(probs)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    u0 = b.pack(snaps)
    net = _net(capi, cfg, 9)
    loss = capi.npbs_train_step(c, net, b, V, f, n, u0, unroll=4, lr=0.0, weight_decay=0.0)
    flat, P = _oracle_params(cfg, 9, requires_grad=True)
    Vb, lam, fb, nb = U.problems_to_batch(probs)
    # the library's V and snapshots are complex64: the oracle runs on the same values
    u0t = torch.from_numpy(np.stack(snaps).astype(np.complex64).astype(np.complex128))
    L = FN.unrolled_loss(P, cfg, Vb, lam, fb, nb, u0t, unroll=4)
    (gref,) = torch.autograd.grad(L, flat)
    assert loss == pytest.approx(float(L), rel=1e-3)
    assert rel_l2(net.get_grads(), gref.numpy()) <= 2e-3


def test_fno_params_roundtrip_and_checkpoint(tmp_path):
    cfg = CONFIGS[0]
    capi, c = ctx()
    net = _net(capi, cfg, 10)
    assert np.array_equal(net.get_params(), _params(cfg, 10))
    p = str(tmp_path / "fno.bin")
    net.save(p)
    net2 = capi.Net.load(p)
    assert net2.num_params() == FN.n_params(cfg)
    assert np.array_equal(net2.get_params(), _params(cfg, 10))


def test_fno_rejects_other_grids():
    cfg = CONFIGS[0]
    capi, c = ctx()
    insts = [synth.small_instance(64, 64, seed=550)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    r = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    net = _net(capi, cfg, 11)
    with pytest.raises(capi.NpbsError) as e:
        capi.npbs_net_forward(c, net, b, r, n, r.clone())
    assert e.value.status == capi.ERR_UNSUPPORTED_SIZE


def test_npbs_with_an_fno_converges_oracle_judged():
    """NPBS runs with an FNO network in place of the U-Net (an untrained one
    here: the divergence guard hands non-improving instances to CBS); the
    returned u is judged by the oracle.  FGMRES accepts the FNO as its right
    preconditioner and reports per instance."""
    cfg = CONFIGS[0]
    capi, c = ctx()
    insts = [synth.small_instance(32, 32, seed=560 + j, layer=4, ppw=8.0) for j in range(2)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    net = _net(capi, cfg, 12)
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.npbs_solve(c, net, b, k2, f, n, u, rtol=1e-5, max_iter=20000, check_every=4)
    assert st == capi.OK, rep
    for j, inst in enumerate(insts):
        p = oracle_problem(inst)
        assert H.rtol(p, torch.from_numpy(b.unpack(u)[j])) <= 1e-5
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.fgmres_solve(c, net, b, k2, f, n, u, restart=20, precond=2, cbs_sweeps=16, rtol=1e-5, max_iter=40)
    assert st in (capi.OK, capi.NOT_CONVERGED)
    assert all(np.isfinite(rep["rtol"])) and all(i <= 40 for i in rep["iters"])


def test_fno_with_four_coefficient_channels_forward_and_backward():
    """coef_channels = 4 (the CDR input kappa, vx, vy, sigma as four planes of
    the batch extent, one after another): forward at relative L2 <= 1e-4 and
    the parameter gradient at <= 1e-3 against the oracle, on a ragged batch of
    two grids' worth of instances at one size."""
    cfg = FN.FnoConfig(n=32, width=8, modes=5, layers=2, coef=4)
    capi, c = ctx()
    insts = [synth.small_instance(32, 32, seed=570 + j) for j in range(3)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    rng = np.random.default_rng(571)
    scale = np.array([0.01, 1.0, 1.0, 3.0])[:, None, None]
    A = [(1.0 + rng.random((4, 32, 32))) * scale for _ in insts]
    a_dev = torch.cat([b.pack([A[j][ch] for j in range(3)], dtype=torch.float32) for ch in range(4)])
    net = capi.Net.fno(32, cfg.width, cfg.modes, cfg.layers, seed=1, coef_channels=4)
    assert net.num_params() == FN.n_params(cfg)
    net.set_params(_params(cfg, 13))
    rs = [random_field((32, 32), 572 + j) for j in range(3)]
    gs = [random_field((32, 32), 575 + j) for j in range(3)]
    r, g = b.pack(rs), b.pack(gs)
    out = torch.zeros_like(r)
    capi.npbs_net_forward(c, net, b, r, a_dev, out)
    gr = torch.zeros_like(r)
    net.zero_grad()
    capi.npbs_net_backward(c, net, b, r, a_dev, g, gr)
    torch.cuda.synchronize()
    flat, P = _oracle_params(cfg, 13, requires_grad=True)
    a = torch.from_numpy(np.stack(A).astype(np.float32).astype(np.float64))
    ref = FN.correction(torch.from_numpy(np.stack(rs)), a, P, cfg)
    got = b.unpack(out)
    for j in range(3):
        assert rel_l2(got[j], ref[j].detach().numpy()) <= 1e-4
    L = (torch.from_numpy(np.stack(gs)).real * ref.real + torch.from_numpy(np.stack(gs)).imag * ref.imag).sum()
    (dth,) = torch.autograd.grad(L, [flat])
    gw = net.get_grads()
    o = 0
    for name, shape in FN.param_spec(cfg):
        k = int(np.prod(shape))
        assert rel_l2(gw[o:o + k], dth.numpy()[o:o + k]) <= 1e-3, name
        o += k


def test_fno_identity_skip_forward_backward_and_checkpoint(tmp_path):
    """npbs_net_fno_set_skip: switching it on makes M = I at first (zero
    projection); with random parameters the forward and the parameter and
    residual gradients match the oracle's M = I + N; a saved network keeps
    the skip."""
    cfg = FN.FnoConfig(n=32, width=8, modes=5, layers=2, skip=True)
    capi, c = ctx()
    insts = [synth.small_instance(32, 32, seed=580 + j) for j in range(2)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    rs = [random_field((32, 32), 582 + j) for j in range(2)]
    gs = [random_field((32, 32), 584 + j) for j in range(2)]
    r, g = b.pack(rs), b.pack(gs)
    net = capi.Net.fno(32, cfg.width, cfg.modes, cfg.layers, seed=3, skip=True)
    out = torch.zeros_like(r)
    capi.npbs_net_forward(c, net, b, r, n, out)
    torch.cuda.synchronize()
    assert np.array_equal(b.unpack(out)[0], rs[0].astype(np.complex64))
    net.set_params(_params(cfg, 15))
    capi.npbs_net_forward(c, net, b, r, n, out)
    gr = torch.zeros_like(r)
    net.zero_grad()
    capi.npbs_net_backward(c, net, b, r, n, g, gr)
    torch.cuda.synchronize()
    flat, P = _oracle_params(cfg, 15, requires_grad=True)
    rr = torch.from_numpy(np.stack(rs).real.copy()).requires_grad_(True)
    ri = torch.from_numpy(np.stack(rs).imag.copy()).requires_grad_(True)
    a = torch.from_numpy(np.stack([i.n.astype(np.float32).astype(np.float64) for i in insts]))
    ref = FN.correction(torch.complex(rr, ri), a, P, cfg)
    got = b.unpack(out)
    for j in range(2):
        assert rel_l2(got[j], ref[j].detach().numpy()) <= 1e-4
    gt = torch.from_numpy(np.stack(gs))
    L = (gt.real * ref.real + gt.imag * ref.imag).sum()
    dth, dre, dim = torch.autograd.grad(L, [flat, rr, ri])
    assert rel_l2(net.get_grads(), dth.numpy()) <= 1e-3
    assert rel_l2(np.stack(b.unpack(gr)), (dre + 1j * dim).numpy()) <= 1e-3
    p = str(tmp_path / "fno_skip.bin")
    net.save(p)
    net2 = capi.Net.load(p)
    out2 = torch.zeros_like(r)
    capi.npbs_net_forward(c, net2, b, r, n, out2)
    torch.cuda.synchronize()
    assert np.array_equal(b.unpack(out2)[1], got[1])


def test_fno_forward_and_backward_partial_sample_chunks():
    """The mode mixing walks the batch in chunks of 8 samples and pads each
    mode's rows of samples to an even count: 11 instances (one full chunk, one
    of 3, an odd batch) keep forward parity and every parameter gradient
    against the oracle, with the width-25 configuration."""
    cfg = CONFIGS[1]
    capi, c = ctx()
    nb = 11
    insts = [synth.small_instance(cfg.n, cfg.n, seed=600 + j) for j in range(nb)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    rs = [random_field((cfg.n, cfg.n), 610 + j) for j in range(nb)]
    gs = [random_field((cfg.n, cfg.n), 630 + j) for j in range(nb)]
    r, g = b.pack(rs), b.pack(gs)
    net = _net(capi, cfg, 9)
    out = torch.zeros_like(r)
    capi.npbs_net_forward(c, net, b, r, n, out)
    gr = torch.zeros_like(r)
    net.zero_grad()
    capi.npbs_net_backward(c, net, b, r, n, g, gr)
    torch.cuda.synchronize()
    flat, P = _oracle_params(cfg, 9, requires_grad=True)
    a = torch.from_numpy(np.stack([i.n.astype(np.float32).astype(np.float64) for i in insts]))
    ref = FN.correction(torch.from_numpy(np.stack(rs)), a, P, cfg)
    got = b.unpack(out)
    for j in range(nb):
        assert rel_l2(got[j], ref[j].detach().numpy()) <= 1e-4, j
    gt = torch.from_numpy(np.stack(gs))
    L = (gt.real * ref.real + gt.imag * ref.imag).sum()
    (dth,) = torch.autograd.grad(L, [flat])
    gw, dref = net.get_grads(), dth.numpy()
    o = 0
    for name, shape in FN.param_spec(cfg):
        k = int(np.prod(shape))
        assert rel_l2(gw[o:o + k], dref[o:o + k]) <= 1e-3, (name, rel_l2(gw[o:o + k], dref[o:o + k]))
        o += k
