"""Parity at the benchmark's full sizes and launch configuration.

The mixed-size batch of the bench (256 x 256^2 + 64 instances of 128/192/384/
512) is applied and solved exactly as bench.py does (autotuned cluster-kernel
variants, CUDA-graph chunks); sampled instances are checked one by one against
the complex128 oracle.  The 1024^2 layered FGMRES and the 256^2 NPBS solve with
the shipped network are judged by the oracle's rTol.
"""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import helmholtz as H
from tests.gpu_common import ctx, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mixed():
    capi, c = ctx()
    insts = synth.workload_mixed(256, 64)
    b = capi.Batch([(i.ny, i.nx) for i in insts], h=[i.h for i in insts])
    k2 = b.pack([i.k2 for i in insts])
    f = b.pack([i.f for i in insts])
    V = torch.zeros_like(k2)
    capi.npbs_potential_from_k2(c, b, k2, V)
    x = torch.zeros_like(k2)
    capi.npbs_autotune_apply(c, b, V, f, x, reps=2)
    return capi, c, insts, b, k2, f, V


def _samples(insts):
    pick = [0, 100, 255]
    for n in (128, 192, 384, 512):
        js = [j for j, i in enumerate(insts) if i.nx == n]
        if js:
            pick.append(js[0])
    return pick


def test_full_batch_apply_sampled_parity(mixed):
    capi, c, insts, b, k2, f, V = mixed
    rng = np.random.default_rng(5)
    xs = b.pack([(rng.standard_normal((i.ny, i.nx)) + 1j * rng.standard_normal((i.ny, i.nx))) * 1e-2
                 for i in insts])
    out = torch.zeros_like(xs)
    capi.cbs_apply(c, b, V, f, xs, out, capi.CBS_STEP)
    torch.cuda.synchronize()
    for j in _samples(insts):
        x0 = b.view(xs, j).cpu().numpy().astype(np.complex128)
        ref = H.cbs_step(oracle_problem(insts[j]), torch.from_numpy(x0)).numpy()
        assert rel_l2(b.view(out, j).cpu().numpy(), ref) <= 1e-5, (j, insts[j].nx)


def test_full_batch_solve_sampled_rtol(mixed):
    capi, c, insts, b, k2, f, V = mixed
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.cbs_solve(c, b, k2, f, u, rtol=1e-5, max_iter=20000, check_every=16)
    assert st == capi.OK and all(s == capi.OK for s in rep["status"])
    for j in _samples(insts):
        r = H.rtol(oracle_problem(insts[j]), torch.from_numpy(b.view(u, j).cpu().numpy()))
        assert r <= 1e-5, (j, r)
        assert rep["rtol"][j] == pytest.approx(r, rel=1e-6)


def test_layered_1024_fgmres_cbs_preconditioned():
    capi, c = ctx()
    insts = synth.workload_layered(2, 1024)
    b = capi.Batch([(i.ny, i.nx) for i in insts], h=[i.h for i in insts])
    k2, f = b.pack([i.k2 for i in insts]), b.pack([i.f for i in insts])
    n = b.pack([i.n for i in insts], dtype=torch.float32)
    V = torch.zeros_like(k2)
    capi.npbs_potential_from_k2(c, b, k2, V)
    u = torch.zeros(b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.fgmres_solve(c, None, b, k2, f, n, u, restart=20, precond=1, cbs_sweeps=16, rtol=1e-5,
                                max_iter=1000)
    assert st == capi.OK, rep
    for j, inst in enumerate(insts):
        assert H.rtol(oracle_problem(inst), torch.from_numpy(b.view(u, j).cpu().numpy())) <= 1e-5


def test_npbs_solve_with_shipped_network_256():
    capi, c = ctx()
    from paper_2603_18527_gb300 import train_unet as T
    w = np.load(os.path.join(ROOT, "paper_2603_18527_gb300", "weights", "unet_contrast256.npz"))["params"]
    net = capi.Net(0, seed=0)
    net.set_params(w.astype(np.float32))
    insts = T.media(256, 4, 30000)  # seeds outside every training pool
    pool = T.Pool(c, insts)
    u = torch.zeros(pool.b.extent, dtype=torch.complex128, device="cuda")
    st, rep = capi.npbs_solve(c, net, pool.b, pool.k2, pool.f, pool.n, u, rtol=1e-5, max_iter=20000, check_every=4)
    # Every instance reports the oracle's rTol of the iterate it returns; those
    # reported converged are; the guard hands non-contracting ones to CBS.
    ok = 0
    for j, inst in enumerate(insts):
        r = H.rtol(oracle_problem(inst), torch.from_numpy(pool.b.view(u, j).cpu().numpy()))
        assert rep["rtol"][j] == pytest.approx(r, rel=1e-6), (j, rep)
        if rep["status"][j] == capi.OK:
            assert r <= 1e-5, (j, r)
            ok += 1
        else:
            assert rep["fallback"][j] == 1 and rep["iters"][j] == 20000, (j, rep)
    assert ok >= 2, rep
