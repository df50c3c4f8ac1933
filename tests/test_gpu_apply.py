"""GPU parity of the fused Born apply (every mode) against the complex128 oracle.

Tolerance: relative L2 error <= 1e-5 per instance and apply (float32 FFT
round-off is ~1e-7 * log2 N; the bound leaves two orders of margin).
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import helmholtz as H
from tests.gpu_common import ctx, oracle_problem, rel_l2, random_field, setup_batch

pytestmark = pytest.mark.gpu

TOL = 1e-5

# sizes spanning several row/column tiles, ragged tails, radix 3, non-square grids
SHAPES = [(16, 16), (96, 96), (24, 48), (48, 24), (2, 2), (3, 6), (288, 288), (256, 256), (1024, 64),
          (64, 1024), (384, 128), (9, 512), (128, 128), (192, 192), (384, 384), (512, 512), (256, 256),
          (1024, 1024)]


@pytest.fixture(scope="module")
def env():
    capi, c = ctx()
    insts = [synth.small_instance(ny, nx, seed=10 + j, layer=max(1, min(ny, nx) // 8), ppw=6.0)
             for j, (ny, nx) in enumerate(SHAPES)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    probs = [H.problem_from_instance(i) for i in insts]
    xs = [random_field((i.ny, i.nx), 100 + j) for j, i in enumerate(insts)]
    x = b.pack(xs)
    return capi, c, insts, probs, b, k2, f, V, xs, x


def test_reference_constants_match_oracle(env):
    capi, c, insts, probs, b, *_ = env
    for j, p in enumerate(probs):
        assert b.k0sq[j] == pytest.approx(p.k0sq, rel=1e-6, abs=1e-7)
        assert b.eps[j] == pytest.approx(p.eps, rel=1e-6)


def _oracle(mode, p, x):
    x = torch.from_numpy(x)
    if mode == "RESIDUAL":
        return H.born_residual(p, x), None
    if mode == "CBS_STEP":
        return H.cbs_step(p, x), H.born_residual(p, x)
    if mode == "OP_B":
        return H.op_B(p, x), None
    if mode == "ADJ_B":
        return H.op_BH(p, x), None
    if mode == "TRUE_RESIDUAL":
        return H.true_residual(p, x), None
    if mode == "PREC_SWEEP":
        # f plays the role of the preconditioned-coordinate right-hand side v
        return H.prec_cbs_sweep(p, x, p.f), p.f - H.op_B(p, x)
    raise ValueError(mode)


@pytest.mark.parametrize("mode", ["RESIDUAL", "CBS_STEP", "OP_B", "ADJ_B", "TRUE_RESIDUAL", "PREC_SWEEP"])
def test_apply_mode_parity(env, mode):
    capi, c, insts, probs, b, k2, f, V, xs, x = env
    out = torch.zeros_like(x)
    norm2 = torch.zeros(b.count, dtype=torch.float64, device="cuda")
    capi.cbs_apply(c, b, V, f, x, out, getattr(capi, mode), norm2)
    torch.cuda.synchronize()
    got = b.unpack(out)
    n2 = norm2.cpu().numpy()
    for j, p in enumerate(probs):
        ref, normed = _oracle(mode, p, xs[j])
        err = rel_l2(got[j], ref.numpy())
        assert err <= TOL, (mode, insts[j].ny, insts[j].nx, err)
        q = ref if normed is None else normed
        refn = float((q.abs() ** 2).sum())
        assert n2[j] == pytest.approx(refn, rel=1e-4), (mode, j)


def test_cbs_step_in_place(env):
    capi, c, insts, probs, b, k2, f, V, xs, x = env
    u = x.clone()
    capi.cbs_apply(c, b, V, f, u, u, capi.CBS_STEP)
    torch.cuda.synchronize()
    got = b.unpack(u)
    for j, p in enumerate(probs):
        assert rel_l2(got[j], H.cbs_step(p, torch.from_numpy(xs[j])).numpy()) <= TOL


def test_adjoint_dot_product_gpu(env):
    """<B x, y> = <x, B^* y> with both sides on the GPU (float32)."""
    capi, c, insts, probs, b, k2, f, V, xs, x = env
    y = b.pack([random_field((i.ny, i.nx), 500 + j) for j, i in enumerate(insts)])
    Bx = torch.zeros_like(x)
    BHy = torch.zeros_like(x)
    capi.cbs_apply(c, b, V, None, x, Bx, capi.OP_B)
    capi.cbs_apply(c, b, V, None, y, BHy, capi.ADJ_B)
    torch.cuda.synchronize()
    for j in range(b.count):
        yv = b.view(y, j)
        lhs = torch.vdot(b.view(Bx, j).reshape(-1).to(torch.complex128), yv.reshape(-1).to(torch.complex128))
        rhs = torch.vdot(b.view(x, j).reshape(-1).to(torch.complex128), b.view(BHy, j).reshape(-1).to(torch.complex128))
        assert abs(complex(lhs - rhs)) <= 1e-5 * abs(complex(lhs)) + 1e-6


def test_empty_batch_is_a_noop():
    capi, c = ctx()
    b = capi.Batch([])
    t = torch.zeros(32, dtype=torch.complex64, device="cuda")
    capi.cbs_apply(c, b, t, t, t, t, capi.RESIDUAL)


@pytest.mark.parametrize("shape", [(97, 96), (96, 2048), (1, 8), (96, 7)])
def test_unsupported_sizes_are_rejected(shape):
    capi, c = ctx()
    b = capi.Batch([shape], k0sq=[1.0], eps=[1.0])
    t = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NpbsError) as e:
        capi.cbs_apply(c, b, t, t, t, t, capi.RESIDUAL)
    assert e.value.status == capi.ERR_UNSUPPORTED_SIZE


def test_invalid_arguments_are_rejected():
    capi, c = ctx()
    b = capi.Batch([(16, 16)], k0sq=[1.0], eps=[0.0])
    t = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.NpbsError) as e:
        capi.cbs_apply(c, b, t, t, t, t, capi.RESIDUAL)
    assert e.value.status == capi.ERR_INVALID_ARG
    b = capi.Batch([(16, 16)], k0sq=[1.0], eps=[1.0])
    b.offsets = [8]
    with pytest.raises(capi.NpbsError) as e:
        capi.cbs_apply(c, b, t, t, t, t, capi.RESIDUAL)
    assert e.value.status == capi.ERR_INVALID_ARG
    b = capi.Batch([(16, 16)], k0sq=[1.0], eps=[1.0])
    with pytest.raises(capi.NpbsError):
        capi.cbs_apply(c, b, t, None, t, t, capi.RESIDUAL)


def test_cluster_path_matches_three_pass_path(env, monkeypatch):
    """Square 128..512 grids run on the single-launch cluster kernel and 1024
    on the band kernels; a context created with NPBS_APPLY_PATH=three_pass runs
    the generic three-launch kernels.  Both must agree to float32 round-off for
    every mode."""
    capi, c, insts, probs, b, k2, f, V, xs, x = env
    monkeypatch.setenv("NPBS_APPLY_PATH", "three_pass")
    c3 = capi.Context(0)
    for mode in ["RESIDUAL", "CBS_STEP", "OP_B", "ADJ_B", "TRUE_RESIDUAL", "PREC_SWEEP"]:
        o1, o2 = torch.zeros_like(x), torch.zeros_like(x)
        n1 = torch.zeros(b.count, dtype=torch.float64, device="cuda")
        n2 = torch.zeros(b.count, dtype=torch.float64, device="cuda")
        capi.cbs_apply(c, b, V, f, x, o1, getattr(capi, mode), n1)
        capi.cbs_apply(c3, b, V, f, x, o2, getattr(capi, mode), n2)
        torch.cuda.synchronize()
        A, B = b.unpack(o1), b.unpack(o2)
        for j in range(b.count):
            assert rel_l2(A[j], B[j]) <= 2e-6, (mode, SHAPES[j])
        assert np.allclose(n1.cpu().numpy(), n2.cpu().numpy(), rtol=1e-5)


# compiled (N1, N2, cluster, threads, min CTAs, exchange path) configurations per side; each
# also exists with the L2 prefetch of the next instance (variant + count)
KERNEL_VARIANTS = {128: 5, 192: 4, 256: 6, 384: 6, 512: 3}
# compiled band configurations (rows / columns per block) of the 1024 kernels
BAND_VARIANTS = {1024: 2}


def selectable_variants(side):
    """Variants NPBS_FAST_VARIANT may pin for a square side (0: none)."""
    if side in KERNEL_VARIANTS:
        return 2 * KERNEL_VARIANTS[side]
    return BAND_VARIANTS.get(side, 0)


@pytest.mark.parametrize("side,variants", [(s, 2 * v) for s, v in KERNEL_VARIANTS.items()])
def test_every_cluster_variant_matches_three_pass(side, variants, monkeypatch):
    """Each compiled (factorisation, cluster size, threads) variant that the
    autotuner may pick, with and without the L2 prefetch, gives the
    three-launch result for every mode."""
    capi, c0 = ctx()
    insts = [synth.small_instance(side, side, seed=200 + j, layer=side // 16) for j in range(2)]
    b, k2, f, n, V = setup_batch(capi, c0, insts)
    x = b.pack([random_field((side, side), 210 + j) for j in range(2)])
    monkeypatch.setenv("NPBS_APPLY_PATH", "three_pass")
    c3 = capi.Context(0)
    monkeypatch.delenv("NPBS_APPLY_PATH")
    for v in range(variants):
        monkeypatch.setenv("NPBS_FAST_VARIANT", f"{side}:{v}")
        cv = capi.Context(0)
        for mode in ["RESIDUAL", "CBS_STEP", "OP_B", "ADJ_B", "TRUE_RESIDUAL", "PREC_SWEEP"]:
            o1, o2 = torch.zeros_like(x), torch.zeros_like(x)
            capi.cbs_apply(cv, b, V, f, x, o1, getattr(capi, mode))
            capi.cbs_apply(c3, b, V, f, x, o2, getattr(capi, mode))
            torch.cuda.synchronize()
            A, B = b.unpack(o1), b.unpack(o2)
            for j in range(2):
                assert rel_l2(A[j], B[j]) <= 2e-6, (side, v, mode)


@pytest.mark.parametrize("side,variants", list(BAND_VARIANTS.items()))
def test_every_band_variant_matches_three_pass(side, variants, monkeypatch):
    """The 1024 band kernels (rows forward, columns with the symbol, rows
    inverse with the epilogue; spectrum kept in digit order) give the generic
    three-launch result for every mode and every compiled band shape, norms
    included."""
    capi, c0 = ctx()
    insts = [synth.small_instance(side, side, seed=250 + j, layer=side // 16) for j in range(2)]
    b, k2, f, n, V = setup_batch(capi, c0, insts)
    x = b.pack([random_field((side, side), 260 + j) for j in range(2)])
    monkeypatch.setenv("NPBS_APPLY_PATH", "three_pass")
    c3 = capi.Context(0)
    monkeypatch.delenv("NPBS_APPLY_PATH")
    for v in range(variants):
        monkeypatch.setenv("NPBS_FAST_VARIANT", f"{side}:{v}")
        cv = capi.Context(0)
        for mode in ["RESIDUAL", "CBS_STEP", "OP_B", "ADJ_B", "TRUE_RESIDUAL", "PREC_SWEEP"]:
            o1, o2 = torch.zeros_like(x), torch.zeros_like(x)
            n1 = torch.zeros(b.count, dtype=torch.float64, device="cuda")
            n2 = torch.zeros(b.count, dtype=torch.float64, device="cuda")
            capi.cbs_apply(cv, b, V, f, x, o1, getattr(capi, mode), n1)
            capi.cbs_apply(c3, b, V, f, x, o2, getattr(capi, mode), n2)
            torch.cuda.synchronize()
            A, B = b.unpack(o1), b.unpack(o2)
            for j in range(2):
                assert rel_l2(A[j], B[j]) <= 2e-6, (side, v, mode)
            assert np.allclose(n1.cpu().numpy(), n2.cpu().numpy(), rtol=1e-5), (side, v, mode)


def test_autotuner_picks_a_valid_band_variant():
    capi, c = ctx()
    insts = [synth.small_instance(1024, 1024, seed=270 + j, layer=64) for j in range(2)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    x = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    tuned = capi.npbs_autotune_apply(c, b, V, f, x, reps=2)
    assert set(tuned) == {1024} and 0 <= tuned[1024] < BAND_VARIANTS[1024]


def test_autotuner_picks_a_valid_variant():
    capi, c = ctx()
    insts = [synth.small_instance(256, 256, seed=230 + j, layer=16) for j in range(4)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    x = torch.zeros(b.extent, dtype=torch.complex64, device="cuda")
    tuned = capi.npbs_autotune_apply(c, b, V, f, x, reps=2)
    assert set(tuned) == {256} and 0 <= tuned[256] < 2 * KERNEL_VARIANTS[256]


@pytest.mark.parametrize("side", [128, 256])
def test_prefetch_variants_identical_on_batches_beyond_residency(side, monkeypatch):
    """With more instances than clusters resident at once, every cluster slot
    prefetches the instance it runs next; a prefetch is only a cache hint, so
    every mode's output is bit-identical to the same kernel without it (the
    per-instance norms are summed by float64 atomics in any order)."""
    capi, c0 = ctx()
    count = 200 if side == 128 else 96
    insts = [synth.small_instance(side, side, seed=400 + j, layer=side // 16) for j in range(count)]
    b, k2, f, n, V = setup_batch(capi, c0, insts)
    x = b.pack([random_field((side, side), 500 + j) for j in range(count)])
    nv = KERNEL_VARIANTS[side]
    for v in range(nv):
        outs = []
        for vv in (v, v + nv):
            monkeypatch.setenv("NPBS_FAST_VARIANT", f"{side}:{vv}")
            cv = capi.Context(0)
            res = []
            for mode in ["CBS_STEP", "ADJ_B", "TRUE_RESIDUAL"]:
                o = torch.zeros_like(x)
                nrm = torch.zeros(b.count, dtype=torch.float64, device="cuda")
                capi.cbs_apply(cv, b, V, f, x, o, getattr(capi, mode), nrm)
                res.append((o, nrm))
            torch.cuda.synchronize()
            outs.append(res)
        for (o1, n1), (o2, n2) in zip(*outs):
            assert torch.equal(o1, o2), (side, v)
            assert torch.allclose(n1, n2, rtol=1e-12, atol=0), (side, v)


@pytest.mark.parametrize("side,count", [(96, 3), (128, 3), (128, 10), (192, 3), (256, 3), (384, 3), (512, 3),
                                        (1024, 2)])
def test_fused_steps_bit_identical_to_repeated_applies(side, count, monkeypatch):
    """cbs_steps(K) is K in-place CBS_STEP (or PREC_SWEEP) applies, fused into
    one launch per grid side for small groups (3 instances) and one launch per
    step for groups above the fused count (10 > 8): every compiled variant
    gives exactly the output of K separate cbs_apply calls (96^2 takes the
    generic three-launch path, 1024^2 the band kernels, three launches a step)."""
    capi, c0 = ctx()
    insts = [synth.small_instance(side, side, seed=600 + j, layer=side // 16) for j in range(count)]
    b, k2, f, n, V = setup_batch(capi, c0, insts)
    x0 = b.pack([random_field((side, side), 610 + j) for j in range(count)])
    K = 5
    for v in range(selectable_variants(side) or 1):
        if selectable_variants(side):
            monkeypatch.setenv("NPBS_FAST_VARIANT", f"{side}:{v}")
        cv = capi.Context(0)
        for mode in ("CBS_STEP", "PREC_SWEEP"):
            m = getattr(capi, mode)
            ref = x0.clone()
            n_ref = torch.zeros(b.count, dtype=torch.float64, device="cuda")
            for k in range(K):
                capi.cbs_apply(cv, b, V, f, ref, ref, m, n_ref if k == K - 1 else None)
            got = torch.zeros_like(x0)
            n_got = torch.zeros(b.count, dtype=torch.float64, device="cuda")
            capi.cbs_steps(cv, b, V, f, x0, got, m, K, n_got)  # out of place: step 0 reads x0
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (side, v, mode)
            assert torch.allclose(n_got, n_ref, rtol=1e-12, atol=0), (side, v, mode)


def test_zero_fused_steps_is_a_noop(env):
    capi, c, insts, probs, b, k2, f, V, xs, x = env
    out = torch.full_like(x, 7.0)
    capi.cbs_steps(c, b, V, f, x, out, capi.CBS_STEP, 0)
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    with pytest.raises(capi.NpbsError):
        capi.cbs_steps(c, b, V, f, x, out, capi.OP_B, 3)


@pytest.mark.parametrize("mode", ["RESIDUAL", "CBS_STEP", "ADJ_B", "TRUE_RESIDUAL"])
def test_apply_parity_with_grid_spacing(mode):
    """h != 1 (xi = 2 pi n / (N h), App. Pseudospectral): every instance of a
    batch carries its own h, on cluster (128^2, 192^2), band (1024^2) and
    three-launch (96 x 48) grids; a dropped or misplaced 1/h fails this."""
    import dataclasses
    capi, c = ctx()
    base = [synth.small_instance(128, 128, seed=60, layer=8), synth.small_instance(192, 192, seed=61, layer=12),
            synth.small_instance(96, 48, seed=62, layer=6), synth.small_instance(128, 128, seed=63, layer=8),
            synth.small_instance(1024, 1024, seed=64, layer=64)]
    hs = [0.5, 2.5, 0.5, 1.7, 0.8]
    insts = [dataclasses.replace(i, h=h) for i, h in zip(base, hs)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    xs = [random_field((i.ny, i.nx), 70 + j) for j, i in enumerate(insts)]
    x = b.pack(xs)
    out = torch.zeros_like(x)
    capi.cbs_apply(c, b, V, f, x, out, getattr(capi, mode))
    torch.cuda.synchronize()
    got = b.unpack(out)
    for j, inst in enumerate(insts):
        p = oracle_problem(inst)
        ref, _ = _oracle(mode, p, xs[j].astype(np.complex128))
        assert rel_l2(got[j], ref.numpy()) <= TOL, (mode, j, inst.h, rel_l2(got[j], ref.numpy()))


def test_custom_offsets_with_gaps_leave_gaps_untouched():
    """The batch layout is the caller's (offsets multiples of 32, any order,
    holes allowed): reversed instances with holes give bit-identical results
    to the packed layout, and nothing is written into the holes (applies,
    fused steps, a CBS solve)."""
    capi, c = ctx()
    insts = [synth.small_instance(128, 128, seed=80, layer=8), synth.small_instance(96, 48, seed=81, layer=6),
             synth.small_instance(128, 128, seed=82, layer=8)]
    b0, k2_0, f_0, n_0, V_0 = setup_batch(capi, c, insts)
    x0 = b0.pack([random_field((i.ny, i.nx), 90 + j) for j, i in enumerate(insts)])
    # the same instances, reversed, with 64- and 96-element holes
    bg = capi.Batch([(i.ny, i.nx) for i in insts], h=[i.h for i in insts])
    sizes = [i.ny * i.nx for i in insts]
    bg.offsets = [64 + sizes[2] + 96 + sizes[1] + 64, 64 + sizes[2] + 96, 64]
    bg.extent = bg.offsets[0] + sizes[0] + 32
    hole = torch.ones(bg.extent, dtype=torch.bool)
    for o, sz in zip(bg.offsets, sizes):
        hole[o:o + sz] = False
    hole = hole.cuda()

    def regap(t, fill):
        out = torch.full((bg.extent,), fill, dtype=t.dtype, device="cuda")
        for j in range(len(insts)):
            bg.view(out, j).copy_(b0.view(t, j))
        return out

    SENT = complex(7.0, -3.0)
    k2_g, f_g, x_g = regap(k2_0, SENT), regap(f_0, SENT), regap(x0, SENT)
    V_g = torch.full_like(k2_g, SENT)
    capi.npbs_potential_from_k2(c, bg, k2_g, V_g)
    assert bool((V_g[hole] == SENT).all())
    for mode in ["RESIDUAL", "CBS_STEP", "OP_B", "ADJ_B", "TRUE_RESIDUAL", "PREC_SWEEP"]:
        o0 = torch.zeros_like(x0)
        capi.cbs_apply(c, b0, V_0, f_0, x0, o0, getattr(capi, mode))
        og = torch.full_like(x_g, SENT)
        capi.cbs_apply(c, bg, V_g, f_g, x_g, og, getattr(capi, mode))
        torch.cuda.synchronize()
        assert bool((og[hole] == SENT).all()), mode
        for j in range(len(insts)):
            assert torch.equal(bg.view(og, j), b0.view(o0, j)), (mode, j)
    s0, sg = x0.clone(), x_g.clone()
    capi.cbs_steps(c, b0, V_0, f_0, s0, s0, capi.CBS_STEP, 7)
    capi.cbs_steps(c, bg, V_g, f_g, sg, sg, capi.CBS_STEP, 7)
    torch.cuda.synchronize()
    assert bool((sg[hole] == SENT).all())
    for j in range(len(insts)):
        assert torch.equal(bg.view(sg, j), b0.view(s0, j)), j
    u0 = torch.zeros(b0.extent, dtype=torch.complex128, device="cuda")
    ug = torch.full((bg.extent,), SENT, dtype=torch.complex128, device="cuda")
    for j in range(len(insts)):
        bg.view(ug, j).zero_()
    st0, r0 = capi.cbs_solve(c, b0, k2_0, f_0, u0, rtol=1e-5, max_iter=5000, check_every=16)
    stg, rg = capi.cbs_solve(c, bg, k2_g, f_g, ug, rtol=1e-5, max_iter=5000, check_every=16)
    assert st0 == stg == capi.OK and r0["iters"] == rg["iters"]
    assert bool((ug[hole] == SENT).all())
    for j in range(len(insts)):
        assert torch.equal(bg.view(ug, j), b0.view(u0, j)), j


def test_apply_and_fused_steps_capture_into_a_cuda_graph():
    """After a first call with the batch (which builds its plan and workspace),
    cbs_apply and cbs_steps issue only stream work, so a caller can capture
    them into a CUDA graph (here torch's) and replay it: identical results,
    grid sides on the forked side streams included."""
    capi, c = ctx()
    insts = [synth.small_instance(128, 128, seed=50, layer=8), synth.small_instance(256, 256, seed=51, layer=16),
             synth.small_instance(96, 48, seed=52, layer=6)]
    b, k2, f, n, V = setup_batch(capi, c, insts)
    x0 = b.pack([random_field((i.ny, i.nx), 53 + j) for j, i in enumerate(insts)])
    ref = x0.clone()
    nref = torch.zeros(b.count, dtype=torch.float64, device="cuda")
    capi.cbs_apply(c, b, V, f, ref, ref, capi.CBS_STEP, nref)
    capi.cbs_steps(c, b, V, f, ref, ref, capi.CBS_STEP, 4, nref)
    torch.cuda.synchronize()
    x = x0.clone()
    nrm = torch.zeros(b.count, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside capture on the capture stream
        capi.cbs_apply(c, b, V, f, x, x, capi.CBS_STEP, nrm)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        capi.cbs_apply(c, b, V, f, x, x, capi.CBS_STEP, nrm)
        capi.cbs_steps(c, b, V, f, x, x, capi.CBS_STEP, 4, nrm)
    x.copy_(x0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, ref)
    assert torch.allclose(nrm, nref, rtol=1e-12, atol=0)


def test_bounded_device_wait_reports_timeout_and_context_stays_usable(env):
    """Failure detection without a fault: a kernel thread waits 50 ms on a
    barrier that nothing completes, gives up and sets the device flag; the
    host reads NPBS_ERR_DEVICE_TIMEOUT once, and the context and device keep
    working (the next apply matches the oracle)."""
    capi, c, insts, probs, b, k2, f, V, xs, x = env
    assert capi.npbs_device_status(c) == capi.OK
    capi.npbs_test_device_timeout(c, 0.05)
    assert capi.npbs_device_status(c) == capi.ERR_DEVICE_TIMEOUT
    assert "bounded device wait" in c.last_error()
    assert capi.npbs_device_status(c) == capi.OK
    out = torch.zeros_like(x)
    capi.cbs_apply(c, b, V, f, x, out, capi.CBS_STEP)
    torch.cuda.synchronize()
    got = b.unpack(out)
    for j in (0, 7):
        ref, _ = _oracle("CBS_STEP", probs[j], xs[j])
        assert rel_l2(got[j], ref.numpy()) <= TOL
    with pytest.raises(capi.NpbsError):
        capi.npbs_test_device_timeout(c, 5.0)
