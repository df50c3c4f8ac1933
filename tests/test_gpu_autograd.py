"""The torch.autograd front-end over the library's adjoints: the Born operator's
backward is its adjoint (oracle, float64), the network Function's backward is
the library's network backward, and the metric-matched loss written with the
two Functions gives the loss and parameter gradients of the library's
checkpointed training step."""
import numpy as np
import pytest
import torch

import synth
from oracle import helmholtz as H
from oracle import unet as U
from tests.gpu_common import ctx, oracle_problem, random_field, rel_l2, setup_batch

pytestmark = pytest.mark.gpu


def _weights(seed):
    return synth.random_weights([s for _, s in U.PARAM_SPEC], seed=seed, out_scale=1.0)


def test_born_operator_forward_and_backward_match_oracle():
    capi, c = ctx()
    from paper_2603_18527_gb300 import autograd as AG
    insts = [synth.small_instance(128, 128, seed=300, layer=8), synth.small_instance(96, 48, seed=301, layer=6)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    xs = [random_field((i.ny, i.nx), 310 + j) for j, i in enumerate(insts)]
    gs = [random_field((i.ny, i.nx), 320 + j) for j, i in enumerate(insts)]
    x = b.pack(xs).requires_grad_(True)
    g = b.pack(gs)
    w = AG.BornOperator.apply(c, b, V, x)
    L = torch.real(torch.vdot(g, w))  # Re <g, B x>: dL/dw = g, so x.grad = B^* g
    L.backward()
    for j, inst in enumerate(insts):
        p = oracle_problem(inst)
        wref = H.op_B(p, torch.from_numpy(xs[j].astype(np.complex128))).numpy()
        gref = H.op_BH(p, torch.from_numpy(gs[j].astype(np.complex128))).numpy()
        assert rel_l2(b.view(w.detach(), j).cpu().numpy(), wref) <= 1e-5
        assert rel_l2(b.view(x.grad, j).cpu().numpy(), gref) <= 1e-5


def test_net_correction_backward_is_the_library_backward():
    capi, c = ctx()
    from paper_2603_18527_gb300 import autograd as AG
    insts = [synth.small_instance(64, 64, seed=330 + j) for j in range(3)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    r = b.pack([random_field((64, 64), 340 + j) for j in range(3)])
    g = b.pack([random_field((64, 64), 350 + j) for j in range(3)])
    net = capi.Net(0, seed=1)
    net.set_params(_weights(12))
    rr = r.clone().requires_grad_(True)
    net.zero_grad()
    out = AG.NetCorrection.apply(c, net, b, n, rr)
    torch.real(torch.vdot(g, out)).backward()
    gw_auto = net.get_grads().copy()
    net.zero_grad()
    gr = torch.zeros_like(r)
    capi.npbs_net_backward(c, net, b, r, n, g, gr)
    torch.cuda.synchronize()
    gw_lib = net.get_grads()
    assert torch.equal(rr.grad, gr)
    assert rel_l2(gw_auto, gw_lib) <= 1e-5  # float32 atomics in another order


def test_unrolled_metric_loss_matches_the_library_train_step():
    """Eq. L_bs_Reta_integral over 4 unrolled NPBS steps: autograd through the
    two Functions vs npbs_train_step (lr = 0), same network and snapshots."""
    capi, c = ctx()
    from paper_2603_18527_gb300 import autograd as AG
    insts = [synth.small_instance(32, 32, seed=100 + i, layer=4, ppw=8.0) for i in range(8)]
    probs = [H.problem_from_instance(i) for i in insts]
    snaps = [H.cbs_solve(p, tol=0, max_iter=3 * i).u.numpy() for i, p in enumerate(probs)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    u0 = b.pack(snaps)
    net = capi.Net(0, seed=1)
    net.set_params(_weights(4))
    net.zero_grad()
    L = AG.unrolled_metric_loss(c, net, b, V, f, n, u0, unroll=4)
    L.backward()
    g_auto = net.get_grads().copy()
    loss_lib = capi.npbs_train_step(c, net, b, V, f, n, u0, unroll=4, lr=0.0, weight_decay=0.0)
    g_lib = net.get_grads()
    assert float(L) == pytest.approx(loss_lib, rel=1e-4)
    assert rel_l2(g_auto, g_lib) <= 1e-4, rel_l2(g_auto, g_lib)
