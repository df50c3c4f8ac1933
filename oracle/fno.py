"""FNO residual-to-correction map (CPU oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  float64 on the CPU with
plain PyTorch ops (``torch.fft.rfft2`` / ``irfft2`` as the FFT steps).

The paper's primary learned map (App. Architectural Instantiations, Eqs.
fno_impl, fno_lift, fno_proj, lfl, nlfl):

    M(r; a) = P( LFL_f[ NLFL_L(...NLFL_1(Phi(a))) * LFL_r(Psi(r)) ] )

with Phi(a) = W_a LayerNorm(a) + b_a (lifting of the coefficient field),
Psi(r) = W_r [Re r, Im r] (lifting of the residual, no bias), P(z) = W_p z
(projection to (Re, Im) of the correction, no bias), and the Fourier blocks

    LFL(x)  = F^{-1}(W^F * F(x)) + W^loc x (+ b on the coefficient branch)
    NLFL(x) = GELU(LFL(x)).

Hyper-parameters (App. Experimental Setup, FNO backbone): three NLFL layers,
25 hidden channels, 45 retained Fourier modes per layer; the residual LFL keeps
the full bandwidth (N/2 + 1).  Readings where the paper is silent:

* F is the real 2D DFT of each channel (half plane kx = 0 .. N/2, the rfft2 /
  irfft2 pair); a layer with "m retained modes" keeps the rows with
  min(ky, N - ky) < m (both signs, symmetric) and the columns kx < m, the
  full-bandwidth layer every row and kx = 0 .. N/2;
* W^F is a complex weight per retained mode and channel pair,
  out[o, k] = sum_i W^F[i, o, k] X[i, k]; other modes are zero;
* the lifting / projection and W^loc are 1x1 convolutions; only the
  coefficient branch (lift and NLFL layers) carries biases, so that M is
  linear in r (the paper's design principle) and no scale wrapper is needed;
* LayerNorm normalises each coefficient channel over the grid of each
  instance (zero mean, unit variance, eps 1e-5, no affine: the lifting
  supplies it); pad / unpad are the identity, since the periodic grid already
  carries the absorbing layer; the CDR problems feed several coefficient
  channels (kappa, v, sigma), Helmholtz one;
* the coefficient channel a is the one the U-Net reads (the local wavenumber
  omega n(x)); GELU is the erf form;
* optionally (cfg.skip) M = I + N with N the network above and its
  projection initialised to zero, so that M starts as the Born series: the
  metric-matched loss weights a residual mode by 1/|lambda|^2 of the Green
  symbol, so the high modes of N receive almost no gradient, and without the
  identity their untrained response can make the iteration diverge there.

The canonical flat parameter order (the exchange format with the CUDA
library) is ``param_spec(cfg)``: real arrays, complex spectral weights stored
as trailing (re, im) pairs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Tuple

import torch
import torch.nn.functional as Fnn


@dataclasses.dataclass(frozen=True)
class FnoConfig:
    n: int            # grid side N (square grids)
    width: int = 25   # hidden channels
    modes: int = 45   # retained modes of the NLFL and fusion layers
    layers: int = 3   # NLFL layers on the coefficient branch
    coef: int = 1     # coefficient channels of a
    skip: bool = False  # M = I + N: the network's output plus its input (Born series at N = 0)

    @property
    def full(self) -> int:
        """Modes of the full-bandwidth residual layer: N/2 + 1."""
        return self.n // 2 + 1


def retained_rows(n: int, m: int) -> List[int]:
    """Rows ky (FFT order) with min(ky, n - ky) < m."""
    return [k for k in range(n) if min(k, n - k) < m]


def retained_cols(n: int, m: int) -> List[int]:
    """Columns kx = 0 .. m - 1 of the half plane (m <= n/2 + 1)."""
    return list(range(min(m, n // 2 + 1)))


def spectral_shape(cfg: FnoConfig, m: int) -> Tuple[int, int]:
    return len(retained_rows(cfg.n, m)), len(retained_cols(cfg.n, m))


def param_spec(cfg: FnoConfig) -> List[Tuple[str, Tuple[int, ...]]]:
    C = cfg.width
    ky, kx = spectral_shape(cfg, cfg.modes)
    fy, fx = spectral_shape(cfg, cfg.full)
    spec = [("lift_a.w", (C, cfg.coef)), ("lift_a.b", (C,))]
    for l in range(cfg.layers):
        spec += [(f"spec{l}.w", (C, C, ky, kx, 2)), (f"loc{l}.w", (C, C)), (f"loc{l}.b", (C,))]
    spec += [("lift_r.w", (C, 2)), ("spec_r.w", (C, C, fy, fx, 2)), ("loc_r.w", (C, C)),
             ("spec_f.w", (C, C, ky, kx, 2)), ("loc_f.w", (C, C)), ("proj.w", (2, C))]
    return spec


def n_params(cfg: FnoConfig) -> int:
    return sum(math.prod(s) for _, s in param_spec(cfg))


def unflatten(cfg: FnoConfig, flat: torch.Tensor) -> Dict[str, torch.Tensor]:
    """Dict of named tensors (float64); spectral weights become complex [Ci, Co, Ky, Kx]."""
    out, o = {}, 0
    for name, shape in param_spec(cfg):
        k = math.prod(shape)
        t = flat[o:o + k].reshape(shape).to(torch.float64)
        if name.startswith("spec"):
            t = torch.complex(t[..., 0], t[..., 1])
        out[name] = t
        o += k
    return out


def spectral(x: torch.Tensor, W: torch.Tensor, m: int) -> torch.Tensor:
    """irfft2( W * R(rfft2(x)) ): x [B, Ci, N, N] real, W [Ci, Co, Ky, Kx] complex
    over the retained modes of ``m`` -> [B, Co, N, N] real."""
    N = x.shape[-1]
    rows = torch.tensor(retained_rows(N, m))
    cols = torch.tensor(retained_cols(N, m))
    X = torch.fft.rfft2(x)                                   # [B, Ci, N, N/2+1]
    Xr = X[:, :, rows][:, :, :, cols]                        # [B, Ci, Ky, Kx]
    Yr = torch.einsum("bikl,iokl->bokl", Xr, W)
    Y = torch.zeros(x.shape[0], W.shape[1], N, N // 2 + 1, dtype=X.dtype)
    Y[:, :, rows[:, None], cols[None, :]] = Yr
    return torch.fft.irfft2(Y, s=(N, N))


def conv1x1(x: torch.Tensor, w: torch.Tensor, b: torch.Tensor | None = None) -> torch.Tensor:
    """Pointwise channel mixing out[o] = sum_i w[o, i] x[i] (+ b[o])."""
    y = torch.einsum("oi,bihw->bohw", w, x)
    return y if b is None else y + b[None, :, None, None]


def layer_norm(a: torch.Tensor, eps: float = 1e-5) -> torch.Tensor:
    """Normalise each instance's field (each channel) over its grid: a [..., N, N]."""
    mu = a.mean(dim=(-2, -1), keepdim=True)
    var = ((a - mu) ** 2).mean(dim=(-2, -1), keepdim=True)
    return (a - mu) / torch.sqrt(var + eps)


def coefficient_features(a: torch.Tensor, P: Dict[str, torch.Tensor], cfg: FnoConfig) -> torch.Tensor:
    """NLFL_L(...NLFL_1(Phi(a))): a [B, N, N] (one channel) or [B, coef, N, N]
    real -> [B, C, N, N]."""
    if a.dim() == 3:
        a = a[:, None]
    c = conv1x1(layer_norm(a), P["lift_a.w"], P["lift_a.b"])
    for l in range(cfg.layers):
        c = Fnn.gelu(spectral(c, P[f"spec{l}.w"], cfg.modes) + conv1x1(c, P[f"loc{l}.w"], P[f"loc{l}.b"]))
    return c


def correction_from_features(r: torch.Tensor, c: torch.Tensor, P: Dict[str, torch.Tensor],
                             cfg: FnoConfig) -> torch.Tensor:
    """P(LFL_f[c * LFL_r(Psi(r))]) (plus r with cfg.skip): r [B, N, N] complex,
    c [B, C, N, N] -> [B, N, N] complex."""
    x = conv1x1(torch.stack([r.real, r.imag], dim=1), P["lift_r.w"])
    x = spectral(x, P["spec_r.w"], cfg.full) + conv1x1(x, P["loc_r.w"])
    z = c * x
    z = spectral(z, P["spec_f.w"], cfg.modes) + conv1x1(z, P["loc_f.w"])
    y = conv1x1(z, P["proj.w"])
    out = torch.complex(y[:, 0], y[:, 1])
    return out + r if cfg.skip else out


def correction(r: torch.Tensor, a: torch.Tensor, P: Dict[str, torch.Tensor], cfg: FnoConfig) -> torch.Tensor:
    """M(r; a) of Eq. fno_impl for a batch."""
    return correction_from_features(r, coefficient_features(a, P, cfg), P, cfg)


def unrolled_loss(P: Dict[str, torch.Tensor], cfg: FnoConfig, V, lam, f, a, u0, unroll: int = 4) -> torch.Tensor:
    """The metric-matched unrolled loss (Eq. L_bs_Reta_integral, squared form)
    with this network as M: r_0 = G(V u_0 + f) - u_0, r_{k+1} = r_k - (I - G V) M(r_k),
    loss = batch mean of (1/unroll) sum_k ||r_{k+1}||^2 / ||r_0||^2."""
    r = torch.fft.ifft2(torch.fft.fft2(V * u0 + f) / lam) - u0
    r0n = (r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1))
    c = coefficient_features(a, P, cfg)
    acc = torch.zeros_like(r0n)
    for _ in range(unroll):
        corr = correction_from_features(r, c, P, cfg)
        r = r - (corr - torch.fft.ifft2(torch.fft.fft2(V * corr) / lam))
        acc = acc + (r.real ** 2 + r.imag ** 2).sum(dim=(-2, -1)) / r0n
    return (acc / unroll).mean()


def init_params(cfg: FnoConfig, seed: int) -> torch.Tensor:
    """Seeded initial parameters in the canonical order (float64): 1x1 weights
    uniform in +-1/sqrt(fan_in), spectral weights uniform in [0, 1/(C*C)) for
    both parts, biases zero; with cfg.skip the projection starts at zero, so
    the initial M is the identity (the Born series)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for name, shape in param_spec(cfg):
        if name.endswith(".b") or (cfg.skip and name == "proj.w"):
            parts.append(torch.zeros(math.prod(shape), dtype=torch.float64))
        elif name.startswith("spec"):
            parts.append(torch.rand(math.prod(shape), generator=g, dtype=torch.float64) / (cfg.width ** 2))
        else:
            bound = 1.0 / math.sqrt(shape[1])
            parts.append((2 * torch.rand(math.prod(shape), generator=g, dtype=torch.float64) - 1) * bound)
    return torch.cat(parts)

