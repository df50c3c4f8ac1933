"""Host-side logic on the CPU: the packed batch layout the C ABI expects, and
the bench's workload selection (no GPU, no kernel launches)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _capi():
    from paper_2603_18527_gb300 import capi
    return capi


SHAPES = [(96, 96), (3, 6), (1024, 64), (9, 512), (2, 2), (256, 256)]


def test_batch_offsets_are_aligned_disjoint_and_cover_the_extent():
    capi = _capi()
    b = capi.Batch(SHAPES)
    assert b.count == len(SHAPES) and b.points() == sum(ny * nx for ny, nx in SHAPES)
    ends = []
    for o, (ny, nx) in zip(b.offsets, SHAPES):
        assert o % 32 == 0  # the C ABI rejects other offsets
        ends.append(o + ny * nx)
    spans = sorted(zip(b.offsets, ends))
    assert all(e0 <= s1 for (_, e0), (s1, _) in zip(spans, spans[1:]))
    assert b.extent >= max(ends) and b.extent % 32 == 0


def test_c_batch_carries_nx_ny_h_and_offsets_in_abi_order():
    capi = _capi()
    b = capi.Batch(SHAPES, h=[0.5 + j for j in range(len(SHAPES))], k0sq=[2.0] * len(SHAPES),
                   eps=[3.0] * len(SHAPES))
    cb = b.c_batch()
    assert cb.count == len(SHAPES)
    for j, (ny, nx) in enumerate(SHAPES):
        s = cb.inst[j]
        assert (s.nx, s.ny) == (nx, ny)
        assert (s.h, s.k0sq, s.eps, s.offset) == (0.5 + j, 2.0, 3.0, b.offsets[j])


def test_pack_unpack_and_view_round_trip_on_cpu():
    capi = _capi()
    b = capi.Batch(SHAPES)
    rng = np.random.default_rng(5)
    fields = [(rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex64)
              for ny, nx in SHAPES]
    t = b.pack(fields, device="cpu")
    assert t.dtype == torch.complex64 and t.numel() == b.extent
    for j, (got, ref) in enumerate(zip(b.unpack(t), fields)):
        assert np.array_equal(got, ref)
        assert np.array_equal(b.view(t, j).numpy(), ref)
    # the gaps between instances stay zero
    mask = torch.ones(b.extent, dtype=torch.bool)
    for o, (ny, nx) in zip(b.offsets, SHAPES):
        mask[o:o + ny * nx] = False
    assert bool((t[mask] == 0).all())


def test_bench_layered_workload_is_1024_grids():
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    insts, name = bench.make_workload(argparse.Namespace(workload="layered1024", fgmres_count=2))
    assert name == "layered_2x1024^2"
    assert [(i.ny, i.nx) for i in insts] == [(1024, 1024)] * 2
    for i in insts:
        assert np.isfinite(i.k2).all() and np.isfinite(i.f).all()
        assert 0.5 < float(i.n.min()) and float(i.n.max()) < 2.5  # layers in [1, 2] plus a 0.1-amplitude field


def test_bench_rejects_the_layered_workload_outside_apply_only():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "layered1024"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 2 and "apply-only" in r.stderr


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the CPU oracle on a bounded sample of
    the bench workload and prints one JSON line with the contract's keys."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
