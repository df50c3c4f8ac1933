"""torch.autograd front-end over the library's hand-written adjoints.

Every forward and backward below is one call into libnpbs (the CUDA kernels);
this module only wires them into PyTorch's autograd so that the method's
operators compose with ordinary torch code:

* ``BornOperator``: w = B x = (I - G V) x (Eq. LS_discrete), backward B^* g
  (the ADJ_B apply: g - conj(V) G^* g).
* ``NetCorrection``: c = M(r; n), the residual-to-correction network with its
  scale wrapper (Eq. npbs_integral), backward J_M(r)^* g by the library's
  network backward, which also accumulates the parameter gradients in the
  library-side network (read them with ``Net.get_grads()``, step with
  ``npbs_net_adamw``).
* ``born_residual``: G(V u + f) - u (the RESIDUAL apply), no gradient.
* ``unrolled_metric_loss``: the metric-matched objective (Eq.
  L_bs_Reta_integral) over unrolled NPBS steps written with the two
  Functions; ``npbs_train_step`` computes the same loss and gradients with
  activation checkpointing inside the library.

PyTorch's complex convention applies: for a real loss L of complex z the
gradient is dL/dRe z + i dL/dIm z, and the vector-Jacobian product of a
complex-linear map is its adjoint; the library's adjoints use the same
convention.
"""
from __future__ import annotations

import torch

from . import capi


class BornOperator(torch.autograd.Function):
    """w = (I - G V) x for every instance of the batch; complex64, packed layout."""

    @staticmethod
    def forward(ctx, lib_ctx, batch, V, x):
        x = x.contiguous()
        w = torch.empty_like(x)
        capi.cbs_apply(lib_ctx, batch, V, None, x, w, capi.OP_B)
        ctx.lib = (lib_ctx, batch, V)
        return w

    @staticmethod
    def backward(ctx, g):
        lib_ctx, batch, V = ctx.lib
        gx = torch.empty_like(g)
        capi.cbs_apply(lib_ctx, batch, V, None, g.contiguous(), gx, capi.ADJ_B)
        return None, None, None, gx


def param_token(net) -> torch.Tensor:
    """A zero-size tensor that stands for the library-side weights of `net` in
    the autograd graph (it requires grad, so outputs of the network do even
    when their input does not); its gradient is always empty, the weight
    gradients accumulate in the library."""
    tok = getattr(net, "_autograd_token", None)
    if tok is None:
        tok = torch.zeros(0, requires_grad=True)
        net._autograd_token = tok
    return tok


class _NetCorrection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lib_ctx, net, batch, n, token, r):
        r = r.contiguous()
        c = torch.empty_like(r)
        capi.npbs_net_forward(lib_ctx, net, batch, r, n, c)
        ctx.lib = (lib_ctx, net, batch, n)
        ctx.save_for_backward(r)
        return c

    @staticmethod
    def backward(ctx, g):
        lib_ctx, net, batch, n = ctx.lib
        (r,) = ctx.saved_tensors
        gr = torch.empty_like(g)
        capi.npbs_net_backward(lib_ctx, net, batch, r, n, g.contiguous(), gr)
        return None, None, None, None, None, gr


class NetCorrection:
    """c = M(r; n) with the library network; parameter gradients accumulate in `net`."""

    @staticmethod
    def apply(lib_ctx, net, batch, n, r):
        return _NetCorrection.apply(lib_ctx, net, batch, n, param_token(net), r)


def born_residual(lib_ctx, batch, V, f, u) -> torch.Tensor:
    """G(V u + f) - u (Eq. npbs_integral), complex64; not differentiated."""
    r = torch.empty_like(u)
    capi.cbs_apply(lib_ctx, batch, V, f, u.contiguous(), r, capi.RESIDUAL)
    return r


def instance_sq_norms(batch, x: torch.Tensor) -> torch.Tensor:
    """||x_j||^2 per instance of the packed layout (differentiable torch ops)."""
    return torch.stack([(batch.view(x, j).abs() ** 2).sum() for j in range(batch.count)])


def unrolled_metric_loss(lib_ctx, net, batch, V, f, n, u_snap, unroll: int = 4) -> torch.Tensor:
    """Mean over instances of (1/unroll) sum_k ||r_k||^2 / ||r_0||^2 with
    r_0 = G(V u + f) - u, c_k = M(r_k), r_{k+1} = r_k - (I - G V) c_k."""
    r = born_residual(lib_ctx, batch, V, f, u_snap)
    r0 = instance_sq_norms(batch, r).detach()
    acc = torch.zeros_like(r0)
    for _ in range(unroll):
        c = NetCorrection.apply(lib_ctx, net, batch, n, r)
        r = r - BornOperator.apply(lib_ctx, batch, V, c)
        acc = acc + instance_sq_norms(batch, r) / r0
    return (acc / unroll).mean()
