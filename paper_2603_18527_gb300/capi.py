"""Thin ctypes binding of ``libnpbs.so`` (argument marshalling only).

Function names follow the C ABI in ``include/npbs.h``.  Field arguments are
torch CUDA tensors (complex64 / complex128 / float32, contiguous, covering
the whole packed batch); nothing here computes any part of the method.  If
the shared library is missing or was not built for this machine, loading
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnpbs.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED_SIZE, ERR_NONFINITE, NOT_CONVERGED, ERR_DEVICE_TIMEOUT, ERR_CUDA, ERR_OOM = range(8)
STATUS_NAMES = ["OK", "ERR_INVALID_ARG", "ERR_UNSUPPORTED_SIZE", "ERR_NONFINITE", "NOT_CONVERGED",
                "ERR_DEVICE_TIMEOUT", "ERR_CUDA", "ERR_OOM"]
RESIDUAL, CBS_STEP, OP_B, ADJ_B, TRUE_RESIDUAL, PREC_SWEEP = range(6)
ALIGN = 32  # offsets are multiples of 32 elements (256 bytes of complex64)


class npbs_instance(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("h", C.c_double), ("k0sq", C.c_double),
                ("eps", C.c_double), ("offset", C.c_int64)]


class npbs_batch(C.Structure):
    _fields_ = [("count", C.c_int32), ("inst", C.POINTER(npbs_instance))]


class npbs_solve_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("check_every", C.c_int32),
                ("use_graph", C.c_int32)]


class npbs_report(C.Structure):
    _fields_ = [("iters", C.POINTER(C.c_int32)), ("rtol", C.POINTER(C.c_double)),
                ("status", C.POINTER(C.c_int32)), ("flags", C.POINTER(C.c_int32))]


class npbs_cdr_consts(C.Structure):
    _fields_ = [("kappa0", C.c_double), ("v0x", C.c_double), ("v0y", C.c_double), ("sigma0", C.c_double)]


class npbs_newton_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_steps", C.c_int32), ("inner_rtol", C.c_double),
                ("inner_max_iter", C.c_int32), ("check_every", C.c_int32), ("direct_format", C.c_int32)]


class npbs_newton_report(C.Structure):
    _fields_ = [("steps", C.POINTER(C.c_int32)), ("inner_iters", C.POINTER(C.c_int32)),
                ("residual", C.POINTER(C.c_double)), ("status", C.POINTER(C.c_int32))]


class NpbsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_LIB = None

_SIGS = {
    "npbs_version": (C.c_char_p, []),
    "npbs_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "npbs_destroy": (C.c_int, [C.c_void_p]),
    "npbs_last_error": (C.c_char_p, [C.c_void_p]),
    "npbs_launch_count": (C.c_int64, [C.c_void_p]),
    "npbs_conv_stats": (None, [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "npbs_potential_from_k2": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "npbs_build_potential": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.POINTER(C.c_double),
                                       C.c_int32, C.c_double, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "cbs_apply": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "npbs_device_status": (C.c_int, [C.c_void_p]),
    "npbs_test_device_timeout": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "cbs_steps": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_int, C.c_int32, C.c_void_p, C.c_void_p]),
    "cbs_solve": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(npbs_solve_opts), C.POINTER(npbs_report), C.c_void_p]),
    "npbs_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.POINTER(npbs_solve_opts), C.POINTER(npbs_report),
                             C.c_void_p]),
    "npbs_solve_direct": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.POINTER(npbs_solve_opts), C.POINTER(npbs_report),
                                    C.c_void_p]),
    "fgmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                               C.POINTER(npbs_solve_opts), C.POINTER(npbs_report), C.c_void_p]),
    "npbs_autotune_apply": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int32, C.c_void_p, C.c_void_p]),
    "cbs_apply_static": (C.c_int, [C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_void_p, C.c_void_p, C.c_char_p, C.c_int32]),
    "npbs_cdr_background": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.POINTER(npbs_cdr_consts), C.c_void_p]),
    "cdr_apply": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.POINTER(npbs_cdr_consts), C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                            C.c_void_p]),
    "cdr_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.POINTER(npbs_cdr_consts), C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(npbs_solve_opts), C.POINTER(npbs_report), C.c_void_p]),
    "cdr_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.POINTER(npbs_cdr_consts),
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int32, C.c_float, C.c_float, C.POINTER(C.c_float), C.c_void_p]),
    "cdr_solve_direct": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.POINTER(npbs_cdr_consts),
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.POINTER(npbs_solve_opts), C.POINTER(npbs_report), C.c_void_p]),
    "cdr_train_step_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.POINTER(npbs_cdr_consts),
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int32, C.c_int, C.c_float, C.c_float, C.POINTER(C.c_float),
                                      C.c_void_p]),
    "newton_apply": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.POINTER(C.c_double), C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "newton_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_double,
                               C.POINTER(npbs_newton_opts), C.POINTER(npbs_newton_report), C.c_void_p]),
    "newton_linearise": (C.c_int, [C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p, C.c_double,
                                   C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_void_p]),
    "newton_train_step_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.POINTER(C.c_double),
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int, C.c_float,
                                         C.c_float, C.POINTER(C.c_float), C.c_void_p]),
    "npbs_net_fno_set_skip": (C.c_int, [C.c_void_p, C.c_int32]),
    "npbs_net_num_params": (C.c_int64, []),
    "npbs_net_param_count": (C.c_int64, [C.c_void_p]),
    "npbs_net_create_fno": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_int, C.c_uint64]),
    "npbs_net_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_uint64]),
    "npbs_net_destroy": (C.c_int, [C.c_void_p]),
    "npbs_net_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "npbs_net_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "npbs_net_get_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "npbs_net_zero_grad": (C.c_int, [C.c_void_p, C.c_void_p]),
    "npbs_net_adamw": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float, C.c_float, C.c_void_p]),
    "npbs_net_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "npbs_net_load": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_char_p]),
    "npbs_net_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    "npbs_net_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "npbs_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_float,
                                  C.POINTER(C.c_float), C.c_void_p]),
    "npbs_train_step_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(npbs_batch), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_int32, C.c_int, C.c_float, C.c_float,
                                       C.POINTER(C.c_float), C.c_void_p]),
}


def exported_symbols() -> List[str]:
    return list(_SIGS)


def lib():
    """Load libnpbs.so (raises if it is absent: build it with ``build.build()``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2603_18527_gb300.build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """An npbs_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        st = lib().npbs_create(C.byref(self._h), int(device))
        if st != OK:
            raise NpbsError(st, "npbs_create failed")
        self.device = device

    @property
    def handle(self):
        return self._h

    def last_error(self) -> str:
        return lib().npbs_last_error(self._h).decode()

    def check(self, st: int):
        if st != OK:
            raise NpbsError(st, self.last_error())
        return st

    def close(self):
        if self._h:
            lib().npbs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Packed batch layout: per-instance (nx, ny, h, k0sq, eps, offset)."""

    def __init__(self, shapes: Sequence[tuple], h: Sequence[float] | None = None,
                 k0sq: Sequence[float] | None = None, eps: Sequence[float] | None = None):
        self.shapes = [(int(ny), int(nx)) for ny, nx in shapes]
        n = len(self.shapes)
        self.h = list(h) if h is not None else [1.0] * n
        self.k0sq = list(k0sq) if k0sq is not None else [0.0] * n
        self.eps = list(eps) if eps is not None else [1.0] * n
        self.offsets = []
        o = 0
        for ny, nx in self.shapes:
            self.offsets.append(o)
            o += (ny * nx + ALIGN - 1) // ALIGN * ALIGN
        self.extent = o
        # E = max_j (offset_j + nx_j ny_j): the stride of the planes of a
        # several-channel network input
        self.plane_stride = max((o + ny * nx for o, (ny, nx) in zip(self.offsets, self.shapes)), default=0)
        self._c = None

    @property
    def count(self):
        return len(self.shapes)

    def points(self) -> int:
        return sum(ny * nx for ny, nx in self.shapes)

    def c_batch(self):
        """The C description; rebuilt only when h, k0sq or eps changed since the last call."""
        key = (tuple(self.h), tuple(self.k0sq), tuple(self.eps))
        if self._c is not None and self._c[2] == key:
            return self._c[1]
        arr = (npbs_instance * max(1, self.count))()
        for j, (ny, nx) in enumerate(self.shapes):
            arr[j] = npbs_instance(nx, ny, float(self.h[j]), float(self.k0sq[j]), float(self.eps[j]),
                                   int(self.offsets[j]))
        self._c = (arr, npbs_batch(self.count, arr), key)
        return self._c[1]

    def pack(self, fields: Sequence[np.ndarray], dtype=torch.complex64, device="cuda") -> torch.Tensor:
        """Copy per-instance arrays into one packed device tensor."""
        out = torch.zeros(self.extent, dtype=dtype)
        for j, a in enumerate(fields):
            ny, nx = self.shapes[j]
            a = np.asarray(a).reshape(ny * nx)
            out[self.offsets[j]:self.offsets[j] + ny * nx] = torch.from_numpy(a).to(dtype)
        return out.to(device)

    def unpack(self, t: torch.Tensor) -> List[np.ndarray]:
        h = t.detach().cpu()
        return [h[o:o + ny * nx].reshape(ny, nx).numpy() for o, (ny, nx) in zip(self.offsets, self.shapes)]

    def view(self, t: torch.Tensor, j: int) -> torch.Tensor:
        ny, nx = self.shapes[j]
        return t[self.offsets[j]:self.offsets[j] + ny * nx].view(ny, nx)


def npbs_version() -> str:
    return lib().npbs_version().decode()


def npbs_conv_stats() -> dict:
    tc, mma = C.c_int64(0), C.c_int64(0)
    lib().npbs_conv_stats(C.byref(tc), C.byref(mma))
    return {"tensor_core": int(tc.value), "warp_mma": int(mma.value)}


def launch_count(ctx: Context) -> int:
    return int(lib().npbs_launch_count(ctx.handle))


def npbs_potential_from_k2(ctx: Context, batch: Batch, k2: torch.Tensor, V_out: Optional[torch.Tensor],
                           stream=None):
    """Fill V_out from k^2 and return (k0sq, eps) lists; also stores them in ``batch``."""
    n = batch.count
    k0 = (C.c_double * max(1, n))()
    ep = (C.c_double * max(1, n))()
    ctx.check(lib().npbs_potential_from_k2(ctx.handle, C.byref(batch.c_batch()), _ptr(k2), _ptr(V_out), k0, ep,
                                           _stream(stream)))
    batch.k0sq = [k0[j] for j in range(n)]
    batch.eps = [ep[j] for j in range(n)]
    return batch.k0sq, batch.eps


def npbs_build_potential(ctx: Context, batch: Batch, n: torch.Tensor, omega: Sequence[float], layer_cells: int,
                         ramp_amp_over_omega2: float, k2_out: Optional[torch.Tensor], V_out: Optional[torch.Tensor],
                         stream=None):
    """Build k^2 (absorbing layer included) and V from n and omega on the GPU;
    return (k0sq, eps) lists and store them in ``batch``."""
    if n.dtype != torch.float32:
        raise ValueError("n must be float32")
    cnt = batch.count
    om = (C.c_double * max(1, cnt))(*[float(w) for w in omega])
    k0 = (C.c_double * max(1, cnt))()
    ep = (C.c_double * max(1, cnt))()
    ctx.check(lib().npbs_build_potential(ctx.handle, C.byref(batch.c_batch()), _ptr(n), om, int(layer_cells),
                                         float(ramp_amp_over_omega2), _ptr(k2_out), _ptr(V_out), k0, ep,
                                         _stream(stream)))
    batch.k0sq = [k0[j] for j in range(cnt)]
    batch.eps = [ep[j] for j in range(cnt)]
    return batch.k0sq, batch.eps


def cbs_apply(ctx: Context, batch: Batch, V, f, x, out, mode: int, norm2: Optional[torch.Tensor] = None,
              stream=None):
    if norm2 is not None and norm2.dtype != torch.float64:
        raise ValueError("norm2 must be float64")
    ctx.check(lib().cbs_apply(ctx.handle, C.byref(batch.c_batch()), _ptr(V), _ptr(f), _ptr(x), _ptr(out),
                              int(mode), _ptr(norm2), _stream(stream)))


def npbs_device_status(ctx: Context) -> int:
    """Synchronise; ERR_DEVICE_TIMEOUT (once) if a bounded device wait gave up, else OK."""
    return int(lib().npbs_device_status(ctx.handle))


def npbs_test_device_timeout(ctx: Context, seconds: float = 0.05, stream=None):
    """Make one bounded device wait give up after `seconds` (tests the error path)."""
    ctx.check(lib().npbs_test_device_timeout(ctx.handle, float(seconds), _stream(stream)))


def cbs_steps(ctx: Context, batch: Batch, V, f, x, out, mode: int, steps: int,
              norm2: Optional[torch.Tensor] = None, stream=None):
    """`steps` consecutive in-place CBS_STEP / PREC_SWEEP applies in one launch per grid side."""
    if norm2 is not None and norm2.dtype != torch.float64:
        raise ValueError("norm2 must be float64")
    ctx.check(lib().cbs_steps(ctx.handle, C.byref(batch.c_batch()), _ptr(V), _ptr(f), _ptr(x), _ptr(out),
                              int(mode), int(steps), _ptr(norm2), _stream(stream)))


def npbs_autotune_apply(ctx: Context, batch: Batch, V, f, x, reps=5, stream=None) -> dict:
    """Pick the fastest cluster-kernel variant per grid side; returns {side: variant}."""
    out = (C.c_int32 * 8)()
    ctx.check(lib().npbs_autotune_apply(ctx.handle, C.byref(batch.c_batch()), _ptr(V), _ptr(f), _ptr(x), int(reps),
                                        out, _stream(stream)))
    return {int(v) // 16: int(v) % 16 for v in out if v > 0}


def cbs_apply_static(batch: Batch, V, f, x, out, mode: int, norm2: Optional[torch.Tensor] = None, stream=None):
    """cbs_apply without a context and without device allocation (static scratch)."""
    if norm2 is not None and norm2.dtype != torch.float64:
        raise ValueError("norm2 must be float64")
    buf = C.create_string_buffer(256)
    st = lib().cbs_apply_static(C.byref(batch.c_batch()), _ptr(V), _ptr(f), _ptr(x), _ptr(out), int(mode),
                                _ptr(norm2), _stream(stream), buf, 256)
    if st != OK:
        raise NpbsError(st, buf.value.decode())


class Report:
    def __init__(self, n: int):
        self.iters = (C.c_int32 * max(1, n))()
        self.rtol = (C.c_double * max(1, n))()
        self.status = (C.c_int32 * max(1, n))()
        self.flags = (C.c_int32 * max(1, n))()
        self.n = n
        self.c = npbs_report(self.iters, self.rtol, self.status, self.flags)

    def as_dict(self):
        return {"iters": [self.iters[i] for i in range(self.n)],
                "rtol": [self.rtol[i] for i in range(self.n)],
                "status": [self.status[i] for i in range(self.n)],
                "fallback": [self.flags[i] for i in range(self.n)]}


def _opts(rtol, max_iter, check_every, use_graph):
    return npbs_solve_opts(float(rtol), int(max_iter), int(check_every), int(use_graph))


def cbs_solve(ctx: Context, batch: Batch, k2, f, u, rtol=1e-5, max_iter=2500, check_every=16, use_graph=1,
              stream=None):
    """Returns (status, report dict); u (complex128) is updated in place.  OK,
    NOT_CONVERGED and ERR_NONFINITE come with the per-instance report; other
    statuses raise NpbsError."""
    rep = Report(batch.count)
    o = _opts(rtol, max_iter, check_every, use_graph)
    st = lib().cbs_solve(ctx.handle, C.byref(batch.c_batch()), _ptr(k2), _ptr(f), _ptr(u), C.byref(o),
                         C.byref(rep.c), _stream(stream))
    if st not in (OK, NOT_CONVERGED, ERR_NONFINITE):  # these fill the per-instance report
        ctx.check(st)
    return st, rep.as_dict()


def npbs_solve(ctx: Context, net: "Net", batch: Batch, k2, f, n, u, rtol=1e-5, max_iter=2500, check_every=4,
               use_graph=1, stream=None):
    rep = Report(batch.count)
    o = _opts(rtol, max_iter, check_every, use_graph)
    st = lib().npbs_solve(ctx.handle, net.handle, C.byref(batch.c_batch()), _ptr(k2), _ptr(f), _ptr(n), _ptr(u),
                          C.byref(o), C.byref(rep.c), _stream(stream))
    if st not in (OK, NOT_CONVERGED, ERR_NONFINITE):  # these fill the per-instance report
        ctx.check(st)
    return st, rep.as_dict()


def npbs_solve_direct(ctx: Context, net: "Net", batch: Batch, k2, f, n, u, rtol=1e-5, max_iter=2500,
                      check_every=4, use_graph=1, stream=None):
    """The Direct format u <- u + M(f - A u) (no CBS guard); as npbs_solve otherwise."""
    rep = Report(batch.count)
    o = _opts(rtol, max_iter, check_every, use_graph)
    st = lib().npbs_solve_direct(ctx.handle, net.handle, C.byref(batch.c_batch()), _ptr(k2), _ptr(f), _ptr(n),
                                 _ptr(u), C.byref(o), C.byref(rep.c), _stream(stream))
    if st not in (OK, NOT_CONVERGED, ERR_NONFINITE):
        ctx.check(st)
    return st, rep.as_dict()


PRECOND_NONE, PRECOND_CBS, PRECOND_NPBS = 0, 1, 2
LOSS_BS_RETA, LOSS_BS_L2, LOSS_DIR = 0, 1, 2
LOSS_KINDS = {"bs_reta": LOSS_BS_RETA, "bs_l2": LOSS_BS_L2, "dir": LOSS_DIR}


def fgmres_solve(ctx: Context, net, batch: Batch, k2, f, n, u, restart=20, precond=PRECOND_NONE, cbs_sweeps=16,
                 rtol=1e-5, max_iter=2500, stream=None):
    rep = Report(batch.count)
    o = _opts(rtol, max_iter, 1, 0)
    st = lib().fgmres_solve(ctx.handle, net.handle if net is not None else None, C.byref(batch.c_batch()), _ptr(k2),
                            _ptr(f), _ptr(n), _ptr(u), int(restart), int(precond), int(cbs_sweeps), C.byref(o),
                            C.byref(rep.c), _stream(stream))
    if st not in (OK, NOT_CONVERGED, ERR_NONFINITE):  # these fill the per-instance report
        ctx.check(st)
    return st, rep.as_dict()


def npbs_net_num_params() -> int:
    return int(lib().npbs_net_num_params())


class Net:
    """An npbs_net (U-Net or FNO weights, gradients, AdamW moments) on one device."""

    def __init__(self, device: int = 0, seed: int = 0, handle=None):
        if handle is not None:
            self._h = handle
        else:
            self._h = C.c_void_p()
            st = lib().npbs_net_create(C.byref(self._h), int(device), C.c_uint64(seed))
            if st != OK:
                raise NpbsError(st, "npbs_net_create failed")
        self.device = device

    @property
    def handle(self):
        return self._h

    @classmethod
    def fno(cls, n: int, width: int = 25, modes: int = 45, layers: int = 3, device: int = 0,
            seed: int = 0, coef_channels: int = 1, skip: bool = False) -> "Net":
        """An FNO network (App. Architectural Instantiations) for n x n grids;
        skip=True makes M = I + N (a zero projection: the Born series at start)."""
        h = C.c_void_p()
        st = lib().npbs_net_create_fno(C.byref(h), int(device), int(n), int(width), int(modes), int(layers),
                                       int(coef_channels), C.c_uint64(seed))
        if st != OK:
            raise NpbsError(st, "npbs_net_create_fno failed")
        net = cls(device, handle=h)
        if skip:
            st = lib().npbs_net_fno_set_skip(h, 1)
            if st != OK:
                raise NpbsError(st, "npbs_net_fno_set_skip failed")
        return net

    def num_params(self) -> int:
        return int(lib().npbs_net_param_count(self._h))

    @classmethod
    def load(cls, path: str, device: int = 0) -> "Net":
        h = C.c_void_p()
        st = lib().npbs_net_load(C.byref(h), int(device), path.encode())
        if st != OK:
            raise NpbsError(st, f"npbs_net_load({path}) failed")
        return cls(device, handle=h)

    def save(self, path: str):
        st = lib().npbs_net_save(self._h, path.encode())
        if st != OK:
            raise NpbsError(st, f"npbs_net_save({path}) failed")

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        st = lib().npbs_net_set_params(self._h, a.ctypes.data_as(C.c_void_p), a.size)
        if st != OK:
            raise NpbsError(st, "npbs_net_set_params failed")

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.num_params(), np.float32)
        st = lib().npbs_net_get_params(self._h, a.ctypes.data_as(C.c_void_p), a.size)
        if st != OK:
            raise NpbsError(st, "npbs_net_get_params failed")
        return a

    def get_grads(self) -> np.ndarray:
        a = np.zeros(self.num_params(), np.float32)
        st = lib().npbs_net_get_grads(self._h, a.ctypes.data_as(C.c_void_p), a.size)
        if st != OK:
            raise NpbsError(st, "npbs_net_get_grads failed")
        return a

    def zero_grad(self, stream=None):
        st = lib().npbs_net_zero_grad(self._h, _stream(stream))
        if st != OK:
            raise NpbsError(st, "npbs_net_zero_grad failed")

    def close(self):
        if self._h:
            lib().npbs_net_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def npbs_net_forward(ctx: Context, net: Net, batch: Batch, r, n, c_out, stream=None):
    ctx.check(lib().npbs_net_forward(ctx.handle, net.handle, C.byref(batch.c_batch()), _ptr(r), _ptr(n), _ptr(c_out),
                                     _stream(stream)))


def npbs_net_backward(ctx: Context, net: Net, batch: Batch, r, n, grad_c, grad_r, stream=None):
    ctx.check(lib().npbs_net_backward(ctx.handle, net.handle, C.byref(batch.c_batch()), _ptr(r), _ptr(n),
                                      _ptr(grad_c), _ptr(grad_r), _stream(stream)))


def npbs_net_adamw(ctx: Context, net: Net, lr: float, weight_decay: float, stream=None):
    ctx.check(lib().npbs_net_adamw(ctx.handle, net.handle, float(lr), float(weight_decay), _stream(stream)))


def npbs_train_step(ctx: Context, net: Net, batch: Batch, V, f, n, u_snap, unroll=4, lr=1e-3, weight_decay=1e-6,
                    stream=None, loss: str = "bs_reta") -> float:
    """One training step; loss "bs_reta" (metric-matched), "bs_l2" or "dir"."""
    out = C.c_float(0.0)
    if loss == "bs_reta":
        ctx.check(lib().npbs_train_step(ctx.handle, net.handle, C.byref(batch.c_batch()), _ptr(V), _ptr(f), _ptr(n),
                                        _ptr(u_snap), int(unroll), float(lr), float(weight_decay), C.byref(out),
                                        _stream(stream)))
    else:
        ctx.check(lib().npbs_train_step_loss(ctx.handle, net.handle, C.byref(batch.c_batch()), _ptr(V), _ptr(f),
                                             _ptr(n), _ptr(u_snap), int(unroll), LOSS_KINDS[loss], float(lr),
                                             float(weight_decay), C.byref(out), _stream(stream)))
    return float(out.value)


# ---- convection-diffusion-reaction ------------------------------------------

class CdrFields:
    """Packed DEVICE float32 coefficient fields (kappa, vx, vy, sigma) of a CDR batch."""

    def __init__(self, batch: "Batch", kappa, vx, vy, sigma):
        self.kappa = batch.pack(kappa, dtype=torch.float32)
        self.vx = batch.pack(vx, dtype=torch.float32)
        self.vy = batch.pack(vy, dtype=torch.float32)
        self.sigma = batch.pack(sigma, dtype=torch.float32)
        # the four-plane network input (kappa, vx, vy, sigma), planes batch.plane_stride apart
        E = batch.plane_stride
        self.a = torch.cat([t[:E] for t in (self.kappa, self.vx, self.vy, self.sigma)]).contiguous()

    def ptrs(self):
        return _ptr(self.kappa), _ptr(self.vx), _ptr(self.vy), _ptr(self.sigma)


def cdr_consts_array(consts):
    """The per-instance constants as the C array the entries take; pass the
    result instead of a list to skip the conversion on repeated calls."""
    if isinstance(consts, C.Array):
        return consts
    arr = (npbs_cdr_consts * max(1, len(consts)))()
    for j, c in enumerate(consts):
        arr[j] = npbs_cdr_consts(*[float(v) for v in c])
    return arr


_consts = cdr_consts_array


def npbs_cdr_background(ctx: Context, batch: "Batch", fields: CdrFields, stream=None):
    """Background constants (kappa0, v0x, v0y, sigma0) per instance: range midpoints of kappa and sigma, means of v."""
    out = (npbs_cdr_consts * max(1, batch.count))()
    ctx.check(lib().npbs_cdr_background(ctx.handle, C.byref(batch.c_batch()), *fields.ptrs(), out, _stream(stream)))
    return [(out[j].kappa0, out[j].v0x, out[j].v0y, out[j].sigma0) for j in range(batch.count)]


def cdr_apply(ctx: Context, batch: "Batch", consts, fields: CdrFields, f, x, out, mode: int,
              norm2: Optional[torch.Tensor] = None, stream=None):
    ctx.check(lib().cdr_apply(ctx.handle, C.byref(batch.c_batch()), _consts(consts), *fields.ptrs(), _ptr(f), _ptr(x),
                              _ptr(out), int(mode), _ptr(norm2), _stream(stream)))


def cdr_solve(ctx: Context, net, batch: "Batch", consts, fields: CdrFields, f, a, u, rtol=1e-6, max_iter=2500,
              check_every=4, stream=None, direct: bool = False):
    """NPBS (net) or the Born series (net None) for CDR, or with direct=True
    the Direct format u <- u + M(f - A u); u (complex128) is updated in place.
    Returns (status, report dict)."""
    if u.dtype != torch.complex128:
        raise TypeError("cdr_solve: u must be complex128")
    rep = Report(batch.count)
    o = _opts(rtol, max_iter, check_every, 0)
    fn = lib().cdr_solve_direct if direct else lib().cdr_solve
    st = fn(ctx.handle, net.handle if net is not None else None, C.byref(batch.c_batch()), _consts(consts),
            *fields.ptrs(), _ptr(f), _ptr(a), _ptr(u), C.byref(o), C.byref(rep.c), _stream(stream))
    if st not in (OK, NOT_CONVERGED, ERR_NONFINITE):
        ctx.check(st)
    return st, rep.as_dict()


def cdr_train_step(ctx: Context, net, batch: "Batch", consts, fields: CdrFields, f, a, u_snap, unroll=4, lr=1e-3,
                   weight_decay=1e-6, stream=None, loss: str = "bs_reta") -> float:
    """One training step with the CDR operators; loss "bs_reta"
    (metric-matched), "bs_l2" or "dir".  Returns the loss before the update."""
    out = C.c_float(0.0)
    ctx.check(lib().cdr_train_step_loss(ctx.handle, net.handle, C.byref(batch.c_batch()), _consts(consts),
                                        *fields.ptrs(), _ptr(f), _ptr(a), _ptr(u_snap), int(unroll),
                                        LOSS_KINDS[loss], float(lr), float(weight_decay), C.byref(out),
                                        _stream(stream)))
    return float(out.value)


# ---- Newton-Born linearisation (Dirichlet, DST-I Green operator) --------------

def newton_shifts_array(shift):
    """The per-instance shifts as the C array the entries take; pass the
    result instead of a list to skip the conversion on repeated calls."""
    if isinstance(shift, C.Array):
        return shift
    arr = (C.c_double * max(1, len(shift)))()
    for j, c in enumerate(shift):
        arr[j] = float(c)
    return arr


_shifts = newton_shifts_array


def newton_apply(ctx: Context, batch: "Batch", shift, u, r, x, out, mode, norm2=None, stream=None):
    """One Newton-Born apply at linearisation points u (float32) with host shifts c."""
    if u.dtype != torch.float32:
        raise TypeError("newton_apply: u must be float32")
    ctx.check(lib().newton_apply(ctx.handle, C.byref(batch.c_batch()), _shifts(shift), _ptr(u), _ptr(r), _ptr(x),
                                 _ptr(out), int(mode), _ptr(norm2), _stream(stream)))


def newton_linearise(ctx: Context, batch: "Batch", u, f, alpha=0.0, stream=None):
    """The Newton state at u (float64): (shifts list, u32 float32, r complex64)."""
    if f.dtype != torch.float64 or u.dtype != torch.float64:
        raise TypeError("newton_linearise: f and u must be float64")
    n = batch.count
    sh = (C.c_double * max(1, n))()
    u32 = torch.zeros(batch.extent, dtype=torch.float32, device=u.device)
    r = torch.zeros(batch.extent, dtype=torch.complex64, device=u.device)
    ctx.check(lib().newton_linearise(ctx.handle, C.byref(batch.c_batch()), _ptr(u), _ptr(f), float(alpha), sh,
                                     _ptr(u32), _ptr(r), _stream(stream)))
    return [sh[i] for i in range(n)], u32, r


def newton_solve(ctx: Context, net, batch: "Batch", f, u, alpha=0.0, tol=1e-8, max_steps=20, inner_rtol=1e-4,
                 inner_max_iter=1000, check_every=2, direct=False, stream=None):
    """Newton with inner Born (net None) or NPBS solves (or the Direct format,
    direct=True); f, u float64 (u in place).  Returns (status, report dict)."""
    if f.dtype != torch.float64 or u.dtype != torch.float64:
        raise TypeError("newton_solve: f and u must be float64")
    n = batch.count
    steps, inner = (C.c_int32 * max(1, n))(), (C.c_int32 * max(1, n))()
    res, stat = (C.c_double * max(1, n))(), (C.c_int32 * max(1, n))()
    rep = npbs_newton_report(steps, inner, res, stat)
    o = npbs_newton_opts(float(tol), int(max_steps), float(inner_rtol), int(inner_max_iter), int(check_every),
                         1 if direct else 0)
    st = lib().newton_solve(ctx.handle, net.handle if net is not None else None, C.byref(batch.c_batch()), _ptr(f),
                            _ptr(u), float(alpha), C.byref(o), C.byref(rep), _stream(stream))
    if st not in (OK, NOT_CONVERGED, ERR_NONFINITE):
        ctx.check(st)
    return st, {"steps": [steps[i] for i in range(n)], "inner_iters": [inner[i] for i in range(n)],
                "residual": [res[i] for i in range(n)], "status": [stat[i] for i in range(n)]}


def newton_train_step(ctx: Context, net, batch: "Batch", shift, u, r, d_snap, unroll=4, lr=1e-3,
                      weight_decay=1e-6, loss: str = "bs_reta", stream=None) -> float:
    """One training step on Newton inner systems; returns the loss before the update."""
    out = C.c_float(0.0)
    ctx.check(lib().newton_train_step_loss(ctx.handle, net.handle, C.byref(batch.c_batch()), _shifts(shift), _ptr(u),
                                           _ptr(r), _ptr(d_snap), int(unroll), LOSS_KINDS[loss], float(lr),
                                           float(weight_decay), C.byref(out), _stream(stream)))
    return float(out.value)
