"""The CDR operators on the GPU (App. Full Derivations, CDR) against the
float64 oracle: background constants, every apply mode, the adjoint, and the
Born-series solve judged by the oracle's rTol.

Tolerance: float32 FFTs of n^2 points and pointwise products; the operator
scales modes by up to kappa |xi|^2 ~ 10^3 at 128^2, so a random (rough) input
loses about three digits more than a smooth one: applies are checked at
relative L2 <= 1e-4 on random complex inputs.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import cdr as CD
from tests.gpu_common import ctx, rel_l2, random_field

pytestmark = pytest.mark.gpu


def _setup(capi, insts):
    b = capi.Batch([(i.n, i.n) for i in insts], h=[i.h for i in insts])
    fields = capi.CdrFields(b, [i.kappa for i in insts], [i.vx for i in insts], [i.vy for i in insts],
                            [i.sigma for i in insts])
    f = b.pack([i.f for i in insts])
    return b, fields, f


def _oracle(inst, consts):
    r32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return CD.make_problem(r32(inst.kappa), r32(inst.vx), r32(inst.vy), r32(inst.sigma),
                           inst.f.astype(np.complex64).astype(np.complex128), inst.h, consts)


# grid sides 64, 128 and 256 run the compile-time fused kernels, 96 the run-time ones
INSTS = [(64, 11, 1.0), (128, 12, 1.0), (64, 13, 0.1), (96, 14, 0.5), (256, 15, 1.0)]


def test_cdr_background_constants():
    capi, c = ctx()
    insts = [synth.cdr_instance(n, seed=s, speed=v) for n, s, v in INSTS]
    b, fields, f = _setup(capi, insts)
    got = capi.npbs_cdr_background(c, b, fields)
    for j, inst in enumerate(insts):
        p = _oracle(inst, None)
        assert got[j] == pytest.approx((p.kappa0, p.v0x, p.v0y, p.sigma0), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("mode", ["RESIDUAL", "OP_B", "TRUE_RESIDUAL", "ADJ_B"])
def test_cdr_apply_parity(mode):
    capi, c = ctx()
    insts = [synth.cdr_instance(n, seed=s, speed=v) for n, s, v in INSTS]
    b, fields, f = _setup(capi, insts)
    consts = capi.npbs_cdr_background(c, b, fields)
    xs = [random_field((i.n, i.n), 700 + j) for j, i in enumerate(insts)]
    x = b.pack(xs)
    out = torch.zeros_like(x)
    n2 = torch.zeros(b.count, dtype=torch.float64, device="cuda")
    capi.cdr_apply(c, b, consts, fields, f, x, out, getattr(capi, mode), n2)
    torch.cuda.synchronize()
    got = b.unpack(out)
    for j, inst in enumerate(insts):
        p = _oracle(inst, consts[j])
        xt = torch.from_numpy(xs[j].astype(np.complex64).astype(np.complex128))
        ref = {"RESIDUAL": lambda: CD.born_residual(p, xt), "OP_B": lambda: CD.op_B(p, xt),
               "TRUE_RESIDUAL": lambda: p.f - CD.apply_A(p, xt), "ADJ_B": lambda: CD.op_BH(p, xt)}[mode]().numpy()
        assert rel_l2(got[j], ref) <= 1e-4, (mode, j, rel_l2(got[j], ref))
        assert float(n2[j]) == pytest.approx(float(np.sum(np.abs(ref) ** 2)), rel=2e-4)


def test_cdr_adjoint_dot_product_on_the_gpu():
    capi, c = ctx()
    insts = [synth.cdr_instance(64, seed=14, speed=1.0)]
    b, fields, f = _setup(capi, insts)
    consts = capi.npbs_cdr_background(c, b, fields)
    x, y = b.pack([random_field((64, 64), 720)]), b.pack([random_field((64, 64), 721)])
    bx, bhy = torch.zeros_like(x), torch.zeros_like(y)
    capi.cdr_apply(c, b, consts, fields, None, x, bx, capi.OP_B)
    capi.cdr_apply(c, b, consts, fields, None, y, bhy, capi.ADJ_B)
    lhs = complex(torch.vdot(y.to(torch.complex128), bx.to(torch.complex128)))
    rhs = complex(torch.vdot(bhy.to(torch.complex128), x.to(torch.complex128)))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_cdr_born_series_solve_is_oracle_judged():
    """Weak convection (the Born series contracts): cdr_solve without a network
    reaches rTol 1e-7, below the float32 floor, through its float64 refresh of
    the iterate; the oracle judges the returned u, the reported rTol is the
    float64 one, and the count is the oracle's Born-series count (checked
    every iteration there, every 4 here: rounded up to a multiple of 4, one
    check of slack for the float32 inner iteration)."""
    capi, c = ctx()
    insts = [synth.cdr_instance(64, seed=15, speed=0.05), synth.cdr_instance(128, seed=16, speed=0.05)]
    b, fields, f = _setup(capi, insts)
    consts = capi.npbs_cdr_background(c, b, fields)
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    tol = 1e-7
    st, rep = capi.cdr_solve(c, None, b, consts, fields, f, None, u, rtol=tol, max_iter=600, check_every=4)
    assert st == capi.OK, rep
    U = b.unpack(u)
    for j, inst in enumerate(insts):
        p = _oracle(inst, consts[j])
        r = CD.rtol(p, torch.from_numpy(U[j]))
        assert r <= tol * (1 + 1e-3), (j, r, rep)
        assert rep["rtol"][j] == pytest.approx(r, rel=1e-3)
        ref = CD.npbs_solve(p, lambda q: q, tol=tol, max_iter=600).iters
        up4 = -(-ref // 4) * 4
        assert up4 - 4 <= rep["iters"][j] <= up4 + 4, (j, ref, rep["iters"][j])


def _fno_case(capi, c, seed, cfg=None):
    """A four-channel FNO with seeded parameters and four 32^2 CDR instances at
    full convection speed; the oracle's parameters and problems beside them."""
    from oracle import fno as FN
    from tests.test_gpu_fno import _oracle_params, _params
    cfg = cfg or FN.FnoConfig(n=32, width=8, modes=5, layers=2, coef=4)
    insts = [synth.cdr_instance(32, seed=seed + j, speed=1.0) for j in range(4)]
    b, fields, f = _setup(capi, insts)
    consts = capi.npbs_cdr_background(c, b, fields)
    net = capi.Net.fno(32, cfg.width, cfg.modes, cfg.layers, seed=1, coef_channels=4)
    net.set_params(_params(cfg, seed))
    flat, P = _oracle_params(cfg, seed, requires_grad=True)
    probs = [_oracle(i, consts[j]) for j, i in enumerate(insts)]
    A = torch.stack([torch.stack([p.kappa, p.vx, p.vy, p.sigma]) for p in probs])
    return cfg, b, fields, f, consts, net, flat, P, probs, A


@pytest.mark.parametrize("loss", ["bs_reta", "bs_l2", "dir"])
def test_cdr_train_step_matches_the_oracle_loss_and_gradient(loss):
    """cdr_train_step (an FNO with the four coefficient channels kappa, vx,
    vy, sigma; 3 unrolls; lr = 0) against the unrolled losses composed from
    the oracle's CDR operators, and their autograd gradients:
    bs_reta: r_0 = G(V u + f) - u, r_{k+1} = r_k - (I - G V) M(r_k), weights 1/||r_0||^2;
    bs_l2 / dir: t_0 = f - A u, t_{k+1} = t_k - A M(G t_k) / A M(t_k), weights 1/||t_0||^2;
    loss = mean_j (1/U) sum_k ||state_k||^2 * weight.  Autograd through the
    oracle's A and G pins the library's explicit adjoints A^* and G^* (convection
    makes A not complex symmetric)."""
    from oracle import fno as FN
    capi, c = ctx()
    cfg, b, fields, f, consts, net, flat, P, probs, A = _fno_case(capi, c, 800)
    snaps = [np.zeros((32, 32), np.complex64)] + [(0.1 * random_field((32, 32), 810 + j)).astype(np.complex64)
                                                 for j in range(3)]
    u0 = b.pack(snaps)
    got = capi.cdr_train_step(c, net, b, consts, fields, f, fields.a, u0, unroll=3, lr=0.0, weight_decay=0.0,
                              loss=loss)
    feats = FN.coefficient_features(A, P, cfg)
    us = [torch.from_numpy(s.astype(np.complex128)) for s in snaps]
    if loss == "bs_reta":
        x = torch.stack([CD.born_residual(p, u) for p, u in zip(probs, us)])
        step = lambda j, cj: CD.op_B(probs[j], cj)
    else:
        x = torch.stack([p.f - CD.apply_A(p, u) for p, u in zip(probs, us)])
        step = lambda j, cj: CD.apply_A(probs[j], cj)
    inp = (lambda t: torch.stack([CD.green(p, t[j]) for j, p in enumerate(probs)])) if loss == "bs_l2" else \
        (lambda t: t)
    n0 = (x.real ** 2 + x.imag ** 2).sum(dim=(-2, -1))
    acc = torch.zeros_like(n0)
    for _ in range(3):
        corr = FN.correction_from_features(inp(x), feats, P, cfg)
        x = x - torch.stack([step(j, corr[j]) for j in range(len(probs))])
        acc = acc + (x.real ** 2 + x.imag ** 2).sum(dim=(-2, -1)) / n0
    L = (acc / 3).mean()
    (gref,) = torch.autograd.grad(L, flat)
    assert got == pytest.approx(float(L.detach()), rel=1e-3)
    assert rel_l2(net.get_grads(), gref.numpy()) <= 2e-3


@pytest.mark.parametrize("direct", [False, True])
def test_cdr_solve_with_a_network_follows_the_oracle_iteration(direct):
    """Three iterations of NPBS (u <- u + M(G(f - A u))) or of the Direct
    format (u <- u + M(f - A u)) with an FNO from u = 0, against the same
    iteration written with the oracle's operators and network; the reported
    rTol is the oracle's rTol of the returned u."""
    from oracle import fno as FN
    capi, c = ctx()
    cfg, b, fields, f, consts, net, flat, P, probs, A = _fno_case(capi, c, 820)
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.cdr_solve(c, net, b, consts, fields, f, fields.a, u, rtol=0.0, max_iter=3, check_every=3,
                             direct=direct)
    assert st == capi.NOT_CONVERGED
    got = b.unpack(u)
    with torch.no_grad():
        feats = FN.coefficient_features(A, P, cfg)
        U = torch.zeros(len(probs), 32, 32, dtype=torch.complex128)
        for _ in range(3):
            t = torch.stack([p.f - CD.apply_A(p, U[j]) for j, p in enumerate(probs)])
            x = t if direct else torch.stack([CD.green(p, t[j]) for j, p in enumerate(probs)])
            U = U + FN.correction_from_features(x, feats, P, cfg)
    for j, p in enumerate(probs):
        assert rel_l2(got[j], U[j].numpy()) <= 1e-3, j
        assert rep["rtol"][j] == pytest.approx(CD.rtol(p, torch.from_numpy(got[j])), rel=1e-6)
