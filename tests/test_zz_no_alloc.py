"""The allocation-free apply (cbs_apply_static) against cbs_apply.

cbs_apply_static exists for callers that cannot let the library call
cudaMalloc (a memory manager that owns the whole device, or code that must not
risk a device-synchronising allocation).  It runs the same kernels with a
static, fixed-size scratch.  Here it is called through the C ABI twice in a
row, with different inputs, and every output and norm must match the existing
entry point within the apply tolerance used elsewhere (relative L2 1e-5).
This file is collected last so that a failure here cannot hide other tests.
"""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_common import ctx, rel_l2, random_field, setup_batch

pytestmark = pytest.mark.gpu

SHAPES = [(96, 96), (256, 256), (48, 24), (128, 384), (9, 512)]
MODES = ["RESIDUAL", "CBS_STEP", "OP_B", "ADJ_B", "TRUE_RESIDUAL", "PREC_SWEEP"]


def test_static_apply_matches_cbs_apply_on_two_calls():
    capi, c = ctx()
    insts = [synth.small_instance(ny, nx, seed=300 + j, layer=max(1, min(ny, nx) // 8))
             for j, (ny, nx) in enumerate(SHAPES)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    for call in range(2):
        x = b.pack([random_field((i.ny, i.nx), 400 + 10 * call + j) for j, i in enumerate(insts)])
        for mode in MODES:
            m = getattr(capi, mode)
            ref = torch.zeros_like(x)
            got = torch.full_like(x, float("nan"))
            n_ref = torch.zeros(b.count, dtype=torch.float64, device="cuda")
            n_got = torch.full((b.count,), float("nan"), dtype=torch.float64, device="cuda")
            capi.cbs_apply(c, b, V, f, x, ref, m, n_ref)
            capi.cbs_apply_static(b, V, f, x, got, m, n_got)
            torch.cuda.synchronize()
            R, G = b.unpack(ref), b.unpack(got)
            for j in range(b.count):
                assert rel_l2(G[j], R[j]) <= 1e-5, (call, mode, SHAPES[j])
            assert np.allclose(n_got.cpu().numpy(), n_ref.cpu().numpy(), rtol=1e-6, atol=0), (call, mode)


def test_static_apply_rejects_batches_beyond_its_scratch():
    capi, c = ctx()
    b = capi.Batch([(1024, 1024), (1024, 1024)], k0sq=[1.0, 1.0], eps=[1.0, 1.0])
    t = torch.zeros(32, dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NpbsError) as e:
        capi.cbs_apply_static(b, t, t, t, t, capi.RESIDUAL)
    assert e.value.status == capi.ERR_UNSUPPORTED_SIZE
    assert "static scratch" in str(e.value)


def test_static_apply_rejects_more_instances_than_its_plan_holds():
    capi, c = ctx()
    b = capi.Batch([(8, 8)] * 65, k0sq=[1.0] * 65, eps=[1.0] * 65)
    t = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NpbsError) as e:
        capi.cbs_apply_static(b, t, t, t, t, capi.RESIDUAL)
    assert e.value.status == capi.ERR_UNSUPPORTED_SIZE
    assert "65 instances exceed the static limit of 64" in str(e.value)


def test_static_apply_rejects_more_distinct_grid_sides_than_its_plan_holds():
    capi, c = ctx()
    # nine distinct sides, each 2^a 3^b: the ninth exceeds the eight plan slots
    shapes = [(2, 3), (4, 6), (8, 9), (12, 16), (18, 24), (27, 32)]
    sides = {s for sh in shapes for s in sh}
    assert len(sides) == 12
    b = capi.Batch(shapes, k0sq=[1.0] * len(shapes), eps=[1.0] * len(shapes))
    t = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NpbsError) as e:
        capi.cbs_apply_static(b, t, t, t, t, capi.RESIDUAL)
    assert e.value.status == capi.ERR_UNSUPPORTED_SIZE
    assert "distinct grid sizes" in str(e.value)
