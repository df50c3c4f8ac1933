"""What the trained network gains over the method without it.

The U-Net is trained on the GPU by the library's own forward/backward
kernels (metric-matched loss over CBS snapshots, AdamW), then NPBS with it is
compared with plain CBS on held-out media of the same law.  Every returned u
is judged by the float64 oracle's rTol.
"""
import numpy as np
import pytest
import torch

from oracle import helmholtz as H
from tests.gpu_common import ctx

pytestmark = pytest.mark.gpu


def test_trained_network_cuts_iterations_against_cbs():
    capi, c = ctx()
    from paper_2603_18527_gb300 import train_unet as T
    net = capi.Net(0, seed=0)
    hist = T.train(c, net, grid=64, steps=300, batch=32, pool_size=128, log=None)
    # the metric-matched loss falls well below its untrained value (about 1)
    assert np.mean(hist[-50:]) < 0.5 * np.mean(hist[:5])
    insts = T.media(64, 8, 9000)
    pool = T.Pool(c, insts)
    res = {}
    us = {}
    for name in ["cbs", "npbs"]:
        u = torch.zeros(pool.b.extent, dtype=torch.complex128, device="cuda")
        if name == "cbs":
            st, rep = capi.cbs_solve(c, pool.b, pool.k2, pool.f, u, rtol=1e-5, max_iter=20000, check_every=16)
        else:
            st, rep = capi.npbs_solve(c, net, pool.b, pool.k2, pool.f, pool.n, u, rtol=1e-5, max_iter=20000,
                                      check_every=4)
        res[name] = rep
        us[name] = pool.b.unpack(u)
    # NPBS reaches the tolerance everywhere, judged by the oracle
    for j, inst in enumerate(insts):
        k2 = inst.k2.astype(np.complex64).astype(np.complex128)
        f = inst.f.astype(np.complex64).astype(np.complex128)
        p = H.make_problem(k2, f, inst.h)
        assert res["npbs"]["status"][j] == capi.OK
        assert H.rtol(p, torch.from_numpy(us["npbs"][j])) <= 1e-5
    # and needs far fewer iterations than CBS (counting CBS's cap as its count)
    med_cbs = float(np.median(res["cbs"]["iters"]))
    med_npbs = float(np.median(res["npbs"]["iters"]))
    assert med_npbs * 4 < med_cbs, (res["cbs"]["iters"], res["npbs"]["iters"])
