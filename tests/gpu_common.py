"""Helpers for the GPU parity tests: pack seeded instances, run the oracle."""
from __future__ import annotations

import numpy as np
import torch

import synth
from oracle import helmholtz as H


def ctx():
    from paper_2603_18527_gb300 import build, capi
    build.build()
    return capi, capi.Context(0)


def setup_batch(capi, c, insts):
    """Pack k^2, f, n of the instances; the library builds V and k0^2, eps."""
    b = capi.Batch([(i.ny, i.nx) for i in insts], h=[i.h for i in insts])
    k2 = b.pack([i.k2 for i in insts])
    f = b.pack([i.f for i in insts])
    n = b.pack([i.n for i in insts], dtype=torch.float32)
    V = torch.zeros_like(k2)
    capi.npbs_potential_from_k2(c, b, k2, V)
    return b, k2, f, n, V


def oracle_problem(inst):
    """The oracle's problem on exactly the data handed to the GPU (k^2, f and n
    rounded to the complex64 / float32 inputs of the library)."""
    k2 = inst.k2.astype(np.complex64).astype(np.complex128)
    f = inst.f.astype(np.complex64).astype(np.complex128)
    n = inst.n.astype(np.float32).astype(np.float64)
    return H.make_problem(k2, f, inst.h, n=n)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def random_field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
