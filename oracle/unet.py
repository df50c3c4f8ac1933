"""Residual-to-correction U-Net and the metric-matched unrolled loss (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  float64 on the CPU with
plain PyTorch ops (``conv2d`` as the convolution step, autograd only where a
test asks for a reference gradient).

Network (App. Experimental Setup, U-Net backbone: 4 levels, 32 channels,
skip connections).  Readings where the paper is silent:

* per level two 3x3 convolutions, each followed by GELU (erf form), zero
  padding 1, with bias;
* down: 2x2 average pooling; up: nearest-neighbour x2, a 3x3 convolution
  followed by GELU, then channel concatenation [skip, up];
* channels 32, 64, 128, 256 (base 32 doubling per level);
* input channels [Re r / s, Im r / s, n]; output a 1x1 convolution 32 -> 2
  without bias giving (Re, Im) of the correction;
* scale wrapper M(r) = s * N(r / s, n) with s = ||r||_2 / sqrt(#points), so that
  M is positively homogeneous in r (the paper asks the residual path to be
  linear; GELU alone would not be).

Parameter order and shapes (the canonical exchange format with the CUDA
library): ``PARAM_SPEC`` lists (name, shape) with torch's OIHW weight layout,
each 3x3 conv contributing a weight then a bias, and the final 1x1 conv a
weight only.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Sequence, Tuple

import torch
import torch.nn.functional as Fnn

from . import helmholtz as H

BASE = 32
LEVELS = 4


def _conv_list() -> List[Tuple[str, int, int]]:
    ch = [BASE * (2 ** i) for i in range(LEVELS)]  # 32 64 128 256
    convs = []
    cin = 3
    for lvl in range(LEVELS):
        convs.append((f"enc{lvl}a", cin, ch[lvl]))
        convs.append((f"enc{lvl}b", ch[lvl], ch[lvl]))
        cin = ch[lvl]
    for lvl in range(LEVELS - 2, -1, -1):
        convs.append((f"up{lvl}", ch[lvl + 1], ch[lvl]))
        convs.append((f"dec{lvl}a", 2 * ch[lvl], ch[lvl]))
        convs.append((f"dec{lvl}b", ch[lvl], ch[lvl]))
    return convs


CONVS = _conv_list()


def param_spec() -> List[Tuple[str, Tuple[int, ...]]]:
    spec = []
    for name, cin, cout in CONVS:
        spec.append((name + ".w", (cout, cin, 3, 3)))
        spec.append((name + ".b", (cout,)))
    spec.append(("out.w", (2, BASE, 1, 1)))
    return spec


PARAM_SPEC = param_spec()


def n_params() -> int:
    return sum(math.prod(s) for _, s in PARAM_SPEC)


def unflatten(flat: torch.Tensor) -> Dict[str, torch.Tensor]:
    out, o = {}, 0
    for name, shape in PARAM_SPEC:
        k = math.prod(shape)
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    return out


def _conv_gelu(x, P, name):
    return Fnn.gelu(Fnn.conv2d(x, P[name + ".w"], P[name + ".b"], padding=1))


def _pool(x):
    return Fnn.avg_pool2d(x, 2)


def _up(x):
    return x.repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)


def network(x: torch.Tensor, P: Dict[str, torch.Tensor]) -> torch.Tensor:
    """N(x) for x of shape [B, 3, H, W] (H, W divisible by 8) -> [B, 2, H, W]."""
    skips = []
    h = x
    for lvl in range(LEVELS):
        if lvl > 0:
            h = _pool(h)
        h = _conv_gelu(h, P, f"enc{lvl}a")
        h = _conv_gelu(h, P, f"enc{lvl}b")
        skips.append(h)
    for lvl in range(LEVELS - 2, -1, -1):
        u = _conv_gelu(_up(h), P, f"up{lvl}")
        h = torch.cat([skips[lvl], u], dim=1)
        h = _conv_gelu(h, P, f"dec{lvl}a")
        h = _conv_gelu(h, P, f"dec{lvl}b")
    return Fnn.conv2d(h, P["out.w"])


def rms(r: torch.Tensor) -> torch.Tensor:
    """s = ||r||_2 / sqrt(#points) per instance; r: [B, H, W] complex."""
    return torch.sqrt((r.real ** 2 + r.imag ** 2).mean(dim=(-2, -1)))


def correction(r: torch.Tensor, n: torch.Tensor, P: Dict[str, torch.Tensor]) -> torch.Tensor:
    """M(r; n) = s * N([Re r/s, Im r/s, n]) with s = rms(r) (scale wrapper);
    r: [B, H, W] complex128, n: [B, H, W] float64 -> [B, H, W] complex128."""
    s = rms(r)
    sc = s[:, None, None]
    x = torch.stack([r.real / sc, r.imag / sc, n], dim=1)
    y = network(x, P)
    return sc * torch.complex(y[:, 0], y[:, 1])


# ------------------------------------------------------------- unrolled loss

def batched_op_B(V: torch.Tensor, lam: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """(I - G V) x for a batch: V, x [B, H, W]; lam [B, H, W]."""
    return x - torch.fft.ifft2(torch.fft.fft2(V * x) / lam)


def batched_born_residual(V, lam, f, u):
    """G(V u + f) - u (Eq. npbs_integral) for a batch."""
    return torch.fft.ifft2(torch.fft.fft2(V * u + f) / lam) - u


def unrolled_loss(P: Dict[str, torch.Tensor], V, lam, f, n, u0, unroll: int = 4) -> torch.Tensor:
    """Metric-matched loss (Eq. L_bs_Reta_integral) over ``unroll`` NPBS steps.

    Per instance r_0 = G(V u_0 + f) - u_0; for k = 0..unroll-1,
    c_k = M(r_k) and r_{k+1} = r_k - (I - G V) c_k, which is the Born residual
    after u_{k+1} = u_k + c_k.  Loss = mean over the batch of
    (1/unroll) sum_k ||r_{k+1}||^2 / ||r_0||^2.  The k = 0 term is the squared
    form of the paper's one-step metric-matched ratio with G r = r_0.
    """
    r = batched_born_residual(V, lam, f, u0)
    r0n = (r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1))
    acc = torch.zeros_like(r0n)
    for _ in range(unroll):
        c = correction(r, n, P)
        r = r - batched_op_B(V, lam, c)
        acc = acc + (r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1)) / r0n
    return (acc / unroll).mean()


def problems_to_batch(problems: Sequence[H.Problem]):
    V = torch.stack([p.V for p in problems])
    lam = torch.stack([p.lam for p in problems])
    f = torch.stack([p.f for p in problems])
    n = torch.stack([p.n for p in problems])
    return V, lam, f, n


def batched_apply_A(k2: torch.Tensor, xi2: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """A x = -Delta x - k^2 x (Eq. helm) for a batch: k2, x [B, H, W]; xi2 [H, W] = |xi|^2."""
    return torch.fft.ifft2(xi2 * torch.fft.fft2(x)) - k2 * x


def batched_green(lam: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """G x = F^{-1}(F x / lambda) for a batch."""
    return torch.fft.ifft2(torch.fft.fft2(x) / lam)


LOSS_KINDS = ("bs_reta", "bs_l2", "dir")


def unrolled_loss_kind(M: Callable[[torch.Tensor], torch.Tensor], kind: str, V, lam, k2, xi2, f, u0,
                       unroll: int = 4) -> torch.Tensor:
    """The three training objectives of Sec. 4 in the unrolled squared form.

    With the true residual t = f - A u as the state, one unrolled step is
    x_k = P_in t_k, c_k = M(x_k), t_{k+1} = t_k - A c_k (u_{k+1} = u_k + c_k),
    and the loss is the batch mean of (1/unroll) sum_k ||P_out t_{k+1}||^2 /
    ||P_out t_0||^2, where
      dir      (Eq. L_dir):            P_in = I, P_out = I (the Direct format, Eq. direct_iter);
      bs_l2    (Eq. L_bs_l2):          P_in = G, P_out = I;
      bs_reta  (Eq. L_bs_Reta_integral): P_in = G, P_out = G (the metric-matched objective).
    For bs_reta, G t is the Born residual and G A = I - G V (Eq. key_identity), so
    this equals ``unrolled_loss`` written in Born-residual coordinates.
    """
    if kind not in LOSS_KINDS:
        raise ValueError(kind)
    t = f - batched_apply_A(k2, xi2, u0)
    proj_in = (lambda v: v) if kind == "dir" else (lambda v: batched_green(lam, v))
    proj_out = (lambda v: batched_green(lam, v)) if kind == "bs_reta" else (lambda v: v)

    def sq(v):
        return (v.real ** 2 + v.imag ** 2).sum(dim=(-2, -1))

    t0n = sq(proj_out(t))
    acc = torch.zeros_like(t0n)
    for _ in range(unroll):
        c = M(proj_in(t))
        t = t - batched_apply_A(k2, xi2, c)
        acc = acc + sq(proj_out(t)) / t0n
    return (acc / unroll).mean()


def adamw_step(theta: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
               step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
               eps: float = 1e-8, weight_decay: float = 1e-6):
    """One AdamW update (decoupled weight decay, Loshchilov and Hutter 2019):
    theta <- theta (1 - lr wd); m, v moment updates; theta -= lr mhat / (sqrt(vhat) + eps),
    with bias corrections 1 - beta^step (step counted from 1).  Returns new (theta, m, v)."""
    theta = theta * (1.0 - lr * weight_decay)
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = theta - lr * mhat / (torch.sqrt(vhat) + eps)
    return theta, m, v
