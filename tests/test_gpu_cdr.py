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


INSTS = [(64, 11, 1.0), (128, 12, 1.0), (64, 13, 0.1)]


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
    reaches the float32 floor of the iterate; the oracle judges the returned u."""
    capi, c = ctx()
    insts = [synth.cdr_instance(64, seed=15, speed=0.05), synth.cdr_instance(128, seed=16, speed=0.05)]
    b, fields, f = _setup(capi, insts)
    consts = capi.npbs_cdr_background(c, b, fields)
    u = torch.zeros_like(f)
    st, rep = capi.cdr_solve(c, None, b, consts, fields, f, None, u, rtol=1e-4, max_iter=600, check_every=4)
    assert st == capi.OK, rep
    U = b.unpack(u)
    for j, inst in enumerate(insts):
        p = _oracle(inst, consts[j])
        r = CD.rtol(p, torch.from_numpy(U[j].astype(np.complex128)))
        assert r <= 1e-4, (j, r, rep)
        # the reported rtol is ||f - A u|| / ||f|| evaluated in float32 (seven
        # FFTs and the flux products): near 1e-4 its rounding error is a few
        # 1e-5 of ||f|| (eps32 times ||kappa grad u|| |xi|_max / ||f||)
        assert abs(r - rep["rtol"][j]) <= 0.05 * r + 3e-5
