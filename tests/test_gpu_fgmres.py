"""GPU FGMRES (restart 20) with no / CBS / network preconditioning, judged by
the complex128 oracle's rTol on the returned solution."""
import numpy as np
import pytest
import torch

import synth
from oracle import fgmres as FG
from oracle import helmholtz as H
from tests.gpu_common import ctx, setup_batch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_fgmres_reaches_tolerance(precond):
    capi, c = ctx()
    insts = [synth.small_instance(64, 64, seed=120 + j, layer=8, ppw=8.0) for j in range(2)] + \
            [synth.small_instance(96, 48, seed=130, layer=8, ppw=8.0)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    net = capi.Net(0, seed=2) if precond == 2 else None
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.fgmres_solve(c, net, b, V, f, n, u, restart=20, precond=precond, cbs_sweeps=16, rtol=1e-5,
                                max_iter=3000)
    assert st == capi.OK, rep
    got = b.unpack(u)
    for j, inst in enumerate(insts):
        p = H.problem_from_instance(inst)
        r = H.rtol(p, torch.from_numpy(got[j]))
        assert r <= 1e-5, (j, r, rep)
        assert rep["rtol"][j] == pytest.approx(r, rel=1e-3, abs=1e-10)
    if precond == 0:
        # same Krylov method as the oracle: iteration counts agree to a restart cycle
        for j, inst in enumerate(insts):
            ref = FG.fgmres_solve(H.problem_from_instance(inst), None, restart=20, tol=1e-5, max_iter=3000)
            assert abs(ref.iters - rep["iters"][j]) <= 20 + 0.1 * ref.iters, (ref.iters, rep["iters"][j])
