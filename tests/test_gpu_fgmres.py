"""GPU FGMRES (restart 20) with no / CBS / network preconditioning, judged by
the complex128 oracle's rTol on the returned solution."""
import numpy as np
import pytest
import torch

import synth
from oracle import fgmres as FG
from oracle import helmholtz as H
from tests.gpu_common import oracle_problem, ctx, setup_batch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", [0, 1])
def test_fgmres_reaches_tolerance(precond):
    capi, c = ctx()
    insts = [synth.small_instance(64, 64, seed=120 + j, layer=8, ppw=8.0) for j in range(2)] + \
            [synth.small_instance(96, 48, seed=130, layer=8, ppw=8.0)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    net = capi.Net(0, seed=2) if precond == 2 else None
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.fgmres_solve(c, net, b, k2, f, n, u, restart=20, precond=precond, cbs_sweeps=16, rtol=1e-5,
                                max_iter=3000)
    assert st == capi.OK, rep
    got = b.unpack(u)
    for j, inst in enumerate(insts):
        p = oracle_problem(inst)
        r = H.rtol(p, torch.from_numpy(got[j]))
        assert r <= 1e-5, (j, r, rep)
        assert rep["rtol"][j] == pytest.approx(r, rel=1e-3, abs=1e-10)
    if precond == 0:
        # same Krylov method as the oracle: iteration counts agree to a restart cycle
        for j, inst in enumerate(insts):
            ref = FG.fgmres_solve(oracle_problem(inst), None, restart=20, tol=1e-5, max_iter=3000)
            assert abs(ref.iters - rep["iters"][j]) <= 20 + 0.1 * ref.iters, (ref.iters, rep["iters"][j])


def test_fgmres_network_preconditioner_is_flexible_minimal_residual():
    """With an (untrained) network as right preconditioner, one FGMRES cycle
    minimises ||G rho - B delta|| over span(Z): the Born residual G(f - A u)
    of the returned u cannot grow with more Arnoldi steps of the same cycle,
    and the float64 rTol the solver reports is the oracle's."""
    capi, c = ctx()
    insts = [synth.small_instance(64, 64, seed=120, layer=8, ppw=8.0)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    p = oracle_problem(insts[0])
    net = capi.Net(0, seed=2)
    born = []
    for steps in [1, 3, 6, 12]:
        u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
        st, rep = capi.fgmres_solve(c, net, b, k2, f, n, u, restart=20, precond=2, rtol=1e-5, max_iter=steps)
        ug = torch.from_numpy(b.unpack(u)[0])
        assert rep["rtol"][0] == pytest.approx(H.rtol(p, ug), rel=1e-6)
        born.append(float(H.born_residual_left(p, ug).norm()))
    # float32 Arnoldi: allow rounding-level increases
    assert all(born[i + 1] <= born[i] * (1 + 1e-4) for i in range(len(born) - 1)), born
    assert born[-1] < born[0]


@pytest.mark.parametrize("precond", [0, 1])
def test_fgmres_short_trajectory_matches_oracle(precond):
    """Six FGMRES steps inside one restart cycle (Arnoldi, Givens, least
    squares) with no preconditioner or 16 CBS sweeps: the GPU iterate is the
    oracle's minimal-residual iterate over the same Krylov space (float32 basis
    against float64: agreement to ~1e-5)."""
    capi, c = ctx()
    insts = [synth.small_instance(64, 64, seed=140 + j, layer=8, ppw=8.0) for j in range(2)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.fgmres_solve(c, None, b, k2, f, n, u, restart=20, precond=precond, cbs_sweeps=16, rtol=1e-12,
                                max_iter=6)
    assert rep["iters"] == [6, 6], rep
    got = b.unpack(u)
    for j, inst in enumerate(insts):
        p = oracle_problem(inst)

        def cbs16(v, p=p):
            z = torch.zeros_like(v)
            for _ in range(16):
                z = H.prec_cbs_sweep(p, z, v)
            return z

        ref = FG.fgmres_solve(p, cbs16 if precond == 1 else None, restart=20, tol=1e-12, max_iter=6)
        err = float(np.linalg.norm(got[j] - ref.u.numpy()) / np.linalg.norm(ref.u.numpy()))
        assert err <= 1e-4, (precond, j, err)
