"""The library's medium and potential builder (npbs_build_potential) against
the oracle: k^2 with its absorbing layer (Sec. 3.1), the reference constants,
and a CBS solve from the library-built k^2 judged by the oracle's rTol."""
import numpy as np
import pytest
import torch

import synth
from oracle import helmholtz as H
from tests.gpu_common import ctx, oracle_problem

pytestmark = pytest.mark.gpu


def _batch(capi, insts):
    b = capi.Batch([(i.ny, i.nx) for i in insts], h=[i.h for i in insts])
    n32 = [i.n.astype(np.float32) for i in insts]
    return b, n32, b.pack(n32, dtype=torch.float32)


@pytest.mark.parametrize("layer", [16, 5, 0])
def test_build_potential_matches_the_oracle_medium(layer):
    capi, c = ctx()
    insts = [synth.small_instance(96, 96, seed=31, layer=16), synth.small_instance(64, 128, seed=32, layer=16),
             synth.small_instance(48, 32, seed=33, layer=8)]
    b, n32, n = _batch(capi, insts)
    k2 = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    V = torch.zeros_like(k2)
    k0, ep = capi.npbs_build_potential(c, b, n, [i.omega for i in insts], layer, 0.5, k2, V)
    got_k2, got_V = b.unpack(k2), b.unpack(V)
    for j, i in enumerate(insts):
        ref = H.absorbing_medium(n32[j].astype(np.float64), i.omega, layer, 0.5).numpy()
        # the same float64 arithmetic rounded to complex64 on both sides
        assert np.array_equal(got_k2[j], ref.astype(np.complex64)), j
        k0_ref, ep_ref = H.reference_constants(torch.from_numpy(ref.astype(np.complex64).astype(np.complex128)))
        assert k0[j] == pytest.approx(k0_ref, rel=1e-12, abs=1e-12)
        assert ep[j] == pytest.approx(ep_ref, rel=1e-12)
        V_ref = H.potential(torch.from_numpy(ref.astype(np.complex64).astype(np.complex128)), k0_ref, ep_ref).numpy()
        assert np.max(np.abs(got_V[j] - V_ref)) <= 2e-7 * np.max(np.abs(V_ref))


def test_build_potential_without_k2_output_and_bad_arguments():
    capi, c = ctx()
    insts = [synth.small_instance(64, 64, seed=34, layer=8)]
    b, n32, n = _batch(capi, insts)
    V = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    k0, ep = capi.npbs_build_potential(c, b, n, [insts[0].omega], 8, 0.5, None, V)
    ref = H.absorbing_medium(n32[0].astype(np.float64), insts[0].omega, 8, 0.5).numpy().astype(np.complex64)
    k0_ref, ep_ref = H.reference_constants(torch.from_numpy(ref.astype(np.complex128)))
    assert k0[0] == pytest.approx(k0_ref, rel=1e-12) and ep[0] == pytest.approx(ep_ref, rel=1e-12)
    for bad in [dict(omega=[0.0]), dict(layer=-1), dict(ramp=float("nan"))]:
        with pytest.raises(capi.NpbsError) as e:
            capi.npbs_build_potential(c, b, n, bad.get("omega", [insts[0].omega]), bad.get("layer", 8),
                                      bad.get("ramp", 0.5), None, V)
        assert e.value.status == capi.ERR_INVALID_ARG


def test_cbs_solve_from_the_library_built_medium_is_oracle_judged():
    capi, c = ctx()
    inst = synth.workload_96()[0]
    b, n32, n = _batch(capi, [inst])
    k2 = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    capi.npbs_build_potential(c, b, n, [inst.omega], inst.layer, 0.5, k2, None)
    f = b.pack([inst.f])
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.cbs_solve(c, b, k2, f, u, rtol=1e-5, max_iter=5000, check_every=16)
    assert st == capi.OK
    k2_h = b.unpack(k2)[0]
    p = H.make_problem(k2_h.astype(np.complex128), inst.f.astype(np.complex64).astype(np.complex128), inst.h)
    assert H.rtol(p, torch.from_numpy(b.unpack(u)[0])) <= 1e-5
