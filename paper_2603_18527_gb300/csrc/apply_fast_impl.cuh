// Single-launch Born apply for square N x N instances, one thread-block
// cluster per instance (the hot path of every CBS / NPBS / FGMRES step).
//
// CTA `rank` of a cluster of CS CTAs owns rows [rank*ROWS, (rank+1)*ROWS) of
// the instance in shared memory (ROWS = N / CS).  Each 1D transform of length
// N = N1 * N2 is a four-step FFT done in registers (n = N2 n1 + n2,
// k = k1 + N1 k2):
//   pass 1: N2 DFTs of length N1 over stride-N2 elements, twiddle W_N^{n2 k1};
//   pass 2: N1 DFTs of length N2 over contiguous blocks,
// which leaves the spectrum in "digit order" (position N2 k1 + k2 holds
// frequency k1 + N1 k2).  The Green symbol is applied in that order (App.
// Pseudospectral: lambda = |xi|^2 - k0^2 - i eps, step 2), and the inverse
// transform consumes digit order and returns natural order, so no reordering
// pass exists.  The row -> column and column -> row transposes go through
// distributed shared memory: each thread stores its register results directly
// into the owning CTA's slab between two cluster barriers.
//
// The row -> column exchange has a second form (template parameter XP = 1):
// each thread writes its row-pass results straight to the instance's region
// of the spectrum scratch in column-major order (coalesced 256-byte stores),
// one cluster barrier, and the column pass loads its columns from L2; the
// CTA then discards its columns' lines from L2 (discard.global.L2) so that
// the dirty scratch is never written back to DRAM.  On GB300 the L2 route
// moves the exchange faster than distributed shared memory (measured
// GPU-wide: about 3.8 TB/s through L2 against 2.5 TB/s through DSMEM); the
// autotuner chooses per grid side.
//
// DRAM traffic is the algorithmic minimum: the prologue reads x, V, f once
// (Eq. CBS: q = V x + f), the epilogue re-reads x and V (they are still in L2)
// and writes out once.  Phases per apply:
//   P1 row pass 1 (from global, prologue)   P2 row pass 2 -> DSMEM transpose
//   P3 column pass 1                         P4 column pass 2, symbol, inverse pass A
//   P5 column inverse pass B -> DSMEM        P6 row inverse pass A
//   P7 row inverse pass B, epilogue (to global), per-instance norm
#include <cooperative_groups.h>
#include <algorithm>
#include <cstdlib>

#pragma once
#include "apply.cuh"
#include "apply_fast.cuh"
#include "dftreg.cuh"

namespace cg = cooperative_groups;

// Optional per-phase instrumentation hook (expands to nothing in the library).
#ifndef NPBS_PHASE_MARK
#define NPBS_PHASE_MARK(i)
#endif

namespace npbs {

namespace fastimpl {

template <int N2> __device__ __forceinline__ int pad(int p) { return p + p / N2; }
// Twiddle table W_N^{n2 k1} stored as [k1][n2] with row stride N2 + 1: the
// first passes read it with n2 varying across a warp (consecutive words), the
// second passes with k1 varying (stride N2 + 1, odd for every factorisation
// here), so neither pattern has shared-memory bank conflicts.
template <int N2> __device__ __forceinline__ int twi(int k1, int n2) { return k1 * (N2 + 1) + n2; }

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Hint the L2 to fetch this CTA's rows of instance `next` (the operands the
// apply of MODE reads: x and V always, f where the mode uses it) while the
// current instance is transformed on chip; one bulk prefetch per chunk of
// about 16 KB, issued by one thread each.  Skipped unless 16-byte aligned.
template <int N, int ROWS, int MODE>
__device__ __forceinline__ void prefetch_rows(const int next, const int rank, const BatchDev& bd, const ApplyArgs& a) {
    constexpr int BYTES = ROWS * N * 8;
    constexpr int CH = BYTES >= 32768 ? BYTES / 16384 : 1;
    constexpr int CB = BYTES / CH;
    static_assert(BYTES % (16 * CH) == 0, "prefetch chunks must be multiples of 16 bytes");
    constexpr bool USE_F = MODE == NPBS_RESIDUAL || MODE == NPBS_CBS_STEP || MODE == NPBS_TRUE_RESIDUAL ||
                           MODE == NPBS_PREC_SWEEP;
    const int t = threadIdx.x;
    if (t >= (USE_F ? 3 : 2) * CH) return;
    const int arr = t / CH, ch = t - arr * CH;
    const float2* base = arr == 0 ? a.x : (arr == 1 ? a.V : a.f);
    const char* p = reinterpret_cast<const char*>(base + bd.inst[next].offset + (long long)rank * ROWS * N) +
                    (long long)ch * CB;
    if ((reinterpret_cast<unsigned long long>(p) & 15ull) != 0) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(CB)
                 : "memory");
}

// One apply (phases P1..P7) of instance `in` by this CTA; returns this
// thread's share of the squared residual norm when `last`.  CBS_STEP and
// PREC_SWEEP may run several steps in place: a step with !first reads x from
// out (each thread reads back exactly the points it wrote in the previous
// step, so the thread's own program order suffices; coherent loads, never the
// read-only path, since out changes during the kernel).
template <int N1, int N2, int CS, int T, int MODE, bool first, bool last, int XP>
__device__ __forceinline__ double cluster_step(const InstDev& in, const BatchDev& bd, const ApplyArgs& a, float2* S,
                                               const float2* tw, const int rank, const int tid, const int next) {
    constexpr int N = N1 * N2;
    constexpr int ROWS = N / CS;
    constexpr int LD = N + N1 + 1;
    constexpr int J1 = (ROWS * N2 + T - 1) / T;  // jobs per thread, passes over N1 (P1, P3, P5, P7)
    constexpr int J2 = (ROWS * N1 + T - 1) / T;  // jobs per thread, passes over N2 (P2, P4, P6)
    cg::cluster_group cluster = cg::this_cluster();
    const long long base = in.offset;

    NPBS_PHASE_MARK(0);
    // ---------------- P1: row pass 1 from global with the prologue
#pragma unroll
    for (int s = 0; s < J1; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N2) {
            const int n2 = j % N2, r = j / N2;
            const long long g0 = base + (long long)(rank * ROWS + r) * N + n2;
            float2 v[N1];
            {
                float2 Vs[N1], fs[N1];
#pragma unroll
                for (int m = 0; m < N1; ++m) {
                    const long long g = g0 + N2 * m;
                    v[m] = first ? __ldg(a.x + g) : __ldcg(a.out + g);
                    if constexpr (MODE != NPBS_ADJ_B && MODE != NPBS_TRUE_RESIDUAL) Vs[m] = __ldg(a.V + g);
                    if constexpr (MODE == NPBS_RESIDUAL || MODE == NPBS_CBS_STEP) fs[m] = __ldg(a.f + g);
                }
#pragma unroll
                for (int m = 0; m < N1; ++m) {
                    const float2 x = v[m];
                    if constexpr (MODE == NPBS_RESIDUAL || MODE == NPBS_CBS_STEP) {
                        v[m] = make_float2(Vs[m].x * x.x - Vs[m].y * x.y + fs[m].x, Vs[m].x * x.y + Vs[m].y * x.x + fs[m].y);
                    } else if constexpr (MODE == NPBS_OP_B || MODE == NPBS_PREC_SWEEP) {
                        v[m] = make_float2(Vs[m].x * x.x - Vs[m].y * x.y, Vs[m].x * x.y + Vs[m].y * x.x);
                    }
                }
            }
            DftR<N1, -1>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                const float2 w = tw[twi<N2>(k1, n2)];
                const float2 t = v[k1];
                S[r * LD + pad<N2>(N2 * k1 + n2)] = make_float2(t.x * w.x - t.y * w.y, t.x * w.y + t.y * w.x);
            }
        }
    }
    __syncthreads();
    if (next >= 0) prefetch_rows<N, ROWS, MODE>(next, rank, bd, a);

    NPBS_PHASE_MARK(1);
    // ---------------- P2: row pass 2, results held for the transpose
    float2 h2[J2][N2];
#pragma unroll
    for (int s = 0; s < J2; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N1) {
            const int r = j % ROWS, k1 = j / ROWS;
#pragma unroll
            for (int i = 0; i < N2; ++i) h2[s][i] = S[r * LD + pad<N2>(N2 * k1 + i)];
            DftR<N2, -1>::run(h2[s]);
        }
    }
    if constexpr (XP == 1) {
        // exchange through L2: column-major [position][row] in the scratch
        float2* regA = static_cast<float2*>(a.scratch) + base;
#pragma unroll
        for (int s = 0; s < J2; ++s) {
            const int j = tid + s * T;
            if (j < ROWS * N1) {
                const int r = j % ROWS, k1 = j / ROWS;
                const int R = rank * ROWS + r;
#pragma unroll
                for (int i = 0; i < N2; ++i) __stcg(regA + (long long)(N2 * k1 + i) * N + R, h2[s][i]);
            }
        }
        cluster.sync();
    } else {
        cluster.sync();
#pragma unroll
        for (int s = 0; s < J2; ++s) {
            const int j = tid + s * T;
            if (j < ROWS * N1) {
                const int r = j % ROWS, k1 = j / ROWS;
                const int p0 = N2 * k1;
                const int d = p0 / ROWS, pl = p0 - d * ROWS;
                float2* dst = cluster.map_shared_rank(S, d);
                const int R = rank * ROWS + r;
#pragma unroll
                for (int i = 0; i < N2; ++i) dst[(pl + i) * LD + pad<N2>(R)] = h2[s][i];
            }
        }
        cluster.sync();
    }

    NPBS_PHASE_MARK(2);
    // ---------------- P3: column pass 1 (slab now [ROWS columns][N rows])
#pragma unroll
    for (int s = 0; s < J1; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N2) {
            const int n2 = j % N2, c = j / N2;
            float2 v[N1];
            if constexpr (XP == 1) {
                const float2* col = static_cast<const float2*>(a.scratch) + base + (long long)(rank * ROWS + c) * N;
#pragma unroll
                for (int m = 0; m < N1; ++m) v[m] = __ldcg(col + n2 + N2 * m);
            } else {
#pragma unroll
                for (int m = 0; m < N1; ++m) v[m] = S[c * LD + pad<N2>(n2 + N2 * m)];
            }
            DftR<N1, -1>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
                const float2 w = tw[twi<N2>(k1, n2)];
                const float2 t = v[k1];
                S[c * LD + pad<N2>(N2 * k1 + n2)] = make_float2(t.x * w.x - t.y * w.y, t.x * w.y + t.y * w.x);
            }
        }
    }
    __syncthreads();
    if constexpr (XP == 1) {
        // this CTA's columns of the scratch are consumed: drop them from L2
        // without a write-back (their contents become undefined)
        const char* col0 = reinterpret_cast<const char*>(static_cast<const float2*>(a.scratch) + base +
                                                         (long long)rank * ROWS * N);
        for (int l = tid; l < ROWS * N * 8 / 128; l += T)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(__cvta_generic_to_global(col0 + 128 * l)) : "memory");
    }

    NPBS_PHASE_MARK(3);
    // ---------------- P4: column pass 2, Green symbol, inverse pass A
    {
        const float cxi = (float)(6.283185307179586476925 / ((double)N * in.h));
        const float k0sq = (float)in.k0sq, eps = (float)in.eps;
#pragma unroll
        for (int s = 0; s < J2; ++s) {
            const int j = tid + s * T;
            if (j < ROWS * N1) {
                const int k1 = j % N1, c = j / N1;
                float2 v[N2];
#pragma unroll
                for (int i = 0; i < N2; ++i) v[i] = S[c * LD + pad<N2>(N2 * k1 + i)];
                DftR<N2, -1>::run(v);
                const int px = rank * ROWS + c;
                const int kx = signed_mode(px / N2 + N1 * (px % N2), N);
                const float xx = cxi * (float)kx;
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) {
                    const int ky = signed_mode(k1 + N1 * k2, N);
                    const float xy = cxi * (float)ky;
                    const float xi2 = xx * xx + xy * xy;
                    const float2 t = v[k2];
                    if constexpr (MODE == NPBS_TRUE_RESIDUAL) {
                        v[k2] = make_float2(t.x * xi2, t.y * xi2);
                    } else {
                        const float lr = xi2 - k0sq;
                        const float li = (MODE == NPBS_ADJ_B) ? eps : -eps;
                        // hardware reciprocal (rcp.approx, ~1 ulp): the symbol
                        // needs far less than float32 round-to-nearest division
                        float inv;
                        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(fmaf(lr, lr, li * li)));
                        v[k2] = make_float2((t.x * lr + t.y * li) * inv, (t.y * lr - t.x * li) * inv);
                    }
                }
                DftR<N2, +1>::run(v);
#pragma unroll
                for (int n2 = 0; n2 < N2; ++n2) {
                    const float2 w = tw[twi<N2>(k1, n2)];  // conjugate twiddle for the inverse
                    const float2 t = v[n2];
                    S[c * LD + pad<N2>(N2 * k1 + n2)] = make_float2(t.x * w.x + t.y * w.y, t.y * w.x - t.x * w.y);
                }
            }
        }
    }
    __syncthreads();

    NPBS_PHASE_MARK(4);
    // ---------------- P5: column inverse pass B, results held for the transpose back
    float2 h5[J1][N1];
#pragma unroll
    for (int s = 0; s < J1; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N2) {
            const int c = j % ROWS, n2 = j / ROWS;
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) h5[s][k1] = S[c * LD + pad<N2>(N2 * k1 + n2)];
            DftR<N1, +1>::run(h5[s]);
        }
    }
    cluster.sync();
#pragma unroll
    for (int s = 0; s < J1; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N2) {
            const int c = j % ROWS, n2 = j / ROWS;
            const int px = rank * ROWS + c;
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int Ry = N2 * n1 + n2;
                const int d = Ry / ROWS, rl = Ry - d * ROWS;
                float2* dst = cluster.map_shared_rank(S, d);
                dst[rl * LD + pad<N2>(px)] = h5[s][n1];
            }
        }
    }
    cluster.sync();

    NPBS_PHASE_MARK(5);
    // ---------------- P6: row inverse pass A
#pragma unroll
    for (int s = 0; s < J2; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N1) {
            const int k1 = j % N1, r = j / N1;
            float2 v[N2];
#pragma unroll
            for (int i = 0; i < N2; ++i) v[i] = S[r * LD + pad<N2>(N2 * k1 + i)];
            DftR<N2, +1>::run(v);
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) {
                const float2 w = tw[twi<N2>(k1, n2)];
                const float2 t = v[n2];
                S[r * LD + pad<N2>(N2 * k1 + n2)] = make_float2(t.x * w.x + t.y * w.y, t.y * w.x - t.x * w.y);
            }
        }
    }
    __syncthreads();

    NPBS_PHASE_MARK(6);
    // ---------------- P7: row inverse pass B and the epilogue
    const float scale = 1.f / ((float)N * (float)N);
    const float ie = (float)(1.0 / in.eps);
    // this thread's share of the norm in float32 (a few dozen points); the
    // block and instance sums are float64 (per-point float64 work would load
    // the FP64 pipe, a small fraction of the FP32 rate on GB300)
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < J1; ++s) {
        const int j = tid + s * T;
        if (j < ROWS * N2) {
            const int n2 = j % N2, r = j / N2;
            float2 v[N1];
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) v[k1] = S[r * LD + pad<N2>(N2 * k1 + n2)];
            DftR<N1, +1>::run(v);
            const long long g0 = base + (long long)(rank * ROWS + r) * N + n2;
            // every point of this job is read and written by this thread only:
            // load all operands first so the loads overlap (out may alias x)
            float2 xs[N1], Vs[N1], fs[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const long long g = g0 + N2 * n1;
                xs[n1] = first ? a.x[g] : a.out[g];
                if constexpr (MODE != NPBS_RESIDUAL && MODE != NPBS_OP_B) Vs[n1] = __ldg(a.V + g);
                if constexpr (MODE == NPBS_TRUE_RESIDUAL || MODE == NPBS_PREC_SWEEP) fs[n1] = __ldg(a.f + g);
            }
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const long long g = g0 + N2 * n1;
                const float zr = v[n1].x * scale, zi = v[n1].y * scale;
                const float2 x = xs[n1];
                float rr, ri;
                float2 o;
                if constexpr (MODE == NPBS_RESIDUAL) {
                    rr = zr - x.x;
                    ri = zi - x.y;
                    o = make_float2(rr, ri);
                } else if constexpr (MODE == NPBS_CBS_STEP) {
                    rr = zr - x.x;
                    ri = zi - x.y;
                    const float2 V = Vs[n1];
                    const float gr = -V.y * ie, gi = V.x * ie;
                    o = make_float2(x.x + gr * rr - gi * ri, x.y + gr * ri + gi * rr);
                } else if constexpr (MODE == NPBS_OP_B) {
                    rr = x.x - zr;
                    ri = x.y - zi;
                    o = make_float2(rr, ri);
                } else if constexpr (MODE == NPBS_ADJ_B) {
                    const float2 V = Vs[n1];
                    rr = x.x - (V.x * zr + V.y * zi);
                    ri = x.y - (V.x * zi - V.y * zr);
                    o = make_float2(rr, ri);
                } else if constexpr (MODE == NPBS_TRUE_RESIDUAL) {
                    const float2 V = Vs[n1], f = fs[n1];
                    const float kr = V.x + (float)in.k0sq, ki = V.y + (float)in.eps;
                    rr = f.x + kr * x.x - ki * x.y - zr;
                    ri = f.y + kr * x.y + ki * x.x - zi;
                    o = make_float2(rr, ri);
                } else {  // PREC_SWEEP
                    const float2 V = Vs[n1], f = fs[n1];
                    rr = f.x - x.x + zr;
                    ri = f.y - x.y + zi;
                    const float gr = -V.y * ie, gi = V.x * ie;
                    o = make_float2(x.x + gr * rr - gi * ri, x.y + gr * ri + gi * rr);
                }
                a.out[g] = o;
                if (last) acc = fmaf(rr, rr, fmaf(ri, ri, acc));
            }
        }
    }
    NPBS_PHASE_MARK(7);
    return (double)acc;
}

// The same step compiled as a separate function: the fused multi-step loop
// calls it, so nothing loop-invariant (addresses, the symbol 1/lambda,
// twiddles) is hoisted out of the loop and kept live across the phases.
template <int N1, int N2, int CS, int T, int MODE, bool first, bool last, int XP>
__device__ __noinline__ double cluster_step_call(const InstDev& in, const BatchDev& bd, const ApplyArgs& a, float2* S,
                                                 const float2* tw, const int rank, const int tid) {
    return cluster_step<N1, N2, CS, T, MODE, first, last, XP>(in, bd, a, S, tw, rank, tid, -1);
}

template <int N1, int N2, int CS, int T, int MODE, int XP>
__device__ __forceinline__ void cluster_apply_one(const int instx, const BatchDev& bd, const ApplyArgs& a,
                                                  float2* smem, double* red, const int next = -1) {
    constexpr int N = N1 * N2;
    constexpr int ROWS = N / CS;
    constexpr int LD = N + N1 + 1;
    static_assert(N % CS == 0 && ROWS % N2 == 0, "slab must hold whole N2 blocks");
    float2* S = smem;               // [ROWS][LD]: row slab, then column slab
    float2* tw = smem + ROWS * LD;  // [N1][N2 + 1]: W_N^{n2 k1}, W_N^j = exp(-2 pi i j / N)
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const InstDev in = bd.inst[instx];
    const int tid = threadIdx.x;
    for (int e = tid; e < N; e += T) {
        const int k1 = e / N2, n2 = e - k1 * N2;
        tw[twi<N2>(k1, n2)] = bd.tw32[in.tw_x + n2 * k1];
    }
    __syncthreads();
    double acc;
    constexpr bool ITER = MODE == NPBS_CBS_STEP || MODE == NPBS_PREC_SWEEP;
    if (!ITER || a.steps <= 1) {
        acc = cluster_step<N1, N2, CS, T, MODE, true, true, XP>(in, bd, a, S, tw, rank, tid, next);
    } else if constexpr (ITER) {
        // fused steps: after the first, u, V and f of the instance come from L2
        cluster_step_call<N1, N2, CS, T, MODE, true, false, XP>(in, bd, a, S, tw, rank, tid);
        __syncthreads();  // the next step rewrites the slab
        for (int it = 1; it < a.steps - 1; ++it) {
            cluster_step_call<N1, N2, CS, T, MODE, false, false, XP>(in, bd, a, S, tw, rank, tid);
            __syncthreads();
        }
        acc = cluster_step_call<N1, N2, CS, T, MODE, false, true, XP>(in, bd, a, S, tw, rank, tid);
    }
    if (a.norm2) {
        acc = warp_sum_d(acc);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < T / 32; ++w) t += red[w];
            atomicAdd(a.norm2 + instx, t);
        }
    }
    __syncthreads();  // smem (slab, twiddles, red) is reused by the next instance
}

// One cluster per instance.
template <int N1, int N2, int CS, int T, int MODE, int MINB = 1, int XP = 0>
__global__ void __launch_bounds__(T, MINB) k_apply_cluster(FastDev fd, BatchDev bd, ApplyArgs a) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ double red[T / 32];
    const int cl = blockIdx.x / CS;
    const int instx = fd.list[cl];
    if (bd.active && !bd.active[instx]) return;  // uniform over the cluster
    int next = -1;
    if (fd.ahead > 0 && cl + fd.ahead < fd.count) {
        next = fd.list[cl + fd.ahead];
        if (bd.active && !bd.active[next]) next = -1;
    }
    cluster_apply_one<N1, N2, CS, T, MODE, XP>(instx, bd, a, smem, red, next);
}

// Prefetch distance in clusters: a third of the resident count (measured on
// 256 x 256^2, 57 resident clusters: 282.8 us without prefetch, 271.8 / 295.3 /
// 300.5 us at distance 19 / 38 / 57; a whole wave ahead the prefetched operands
// do not survive in L2 next to the current wave's), or NPBS_FAST_AHEAD.
inline int prefetch_ahead(int resident) {
    static const int forced = [] {
        const char* e = getenv("NPBS_FAST_AHEAD");
        return e ? atoi(e) : -1;
    }();
    return forced >= 0 ? forced : std::max(1, resident / 3);
}

// Clusters of one variant resident on the device at once (set when the
// attributes are; 0 when unknown, which disables the prefetch).
template <int N1, int N2, int CS, int T, int MODE, int MINB, int XP>
int& resident_clusters() {
    static int v = 0;
    return v;
}

template <int N1, int N2, int CS, int T> constexpr size_t fast_smem() {
    return sizeof(float2) * ((size_t)(N1 * N2 / CS) * (N1 * N2 + N1 + 1) + (size_t)N1 * (N2 + 1));
}

template <int N1, int N2, int CS, int T, int MODE, int MINB = 1, int XP = 0>
cudaError_t set_attr_one() {
    auto k = k_apply_cluster<N1, N2, CS, T, MODE, MINB, XP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast_smem<N1, N2, CS, T>());
    if (e == cudaSuccess && CS > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CS, 1, 1);
        cfg.blockDim = dim3(T, 1, 1);
        cfg.dynamicSmemBytes = fast_smem<N1, N2, CS, T>();
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess) resident_clusters<N1, N2, CS, T, MODE, MINB, XP>() = n;
        else (void)cudaGetLastError();
    }
    return e;
}

template <int N1, int N2, int CS, int T, int MINB, int XP = 0>
cudaError_t set_attr_size() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_one<N1, N2, CS, T, NPBS_RESIDUAL, MINB, XP>();
    if (e == cudaSuccess) e = set_attr_one<N1, N2, CS, T, NPBS_CBS_STEP, MINB, XP>();
    if (e == cudaSuccess) e = set_attr_one<N1, N2, CS, T, NPBS_OP_B, MINB, XP>();
    if (e == cudaSuccess) e = set_attr_one<N1, N2, CS, T, NPBS_ADJ_B, MINB, XP>();
    if (e == cudaSuccess) e = set_attr_one<N1, N2, CS, T, NPBS_TRUE_RESIDUAL, MINB, XP>();
    if (e == cudaSuccess) e = set_attr_one<N1, N2, CS, T, NPBS_PREC_SWEEP, MINB, XP>();
    return e;
}

template <int N1, int N2, int CS, int T, int MODE, int MINB = 1, int XP = 0>
cudaError_t launch_one(const FastDev& fd, const BatchDev& bd, const ApplyArgs& a, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(fd.count * CS), 1, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cfg.dynamicSmemBytes = fast_smem<N1, N2, CS, T>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FastDev f2 = fd;
    f2.ahead = fd.ahead > 0 ? prefetch_ahead(resident_clusters<N1, N2, CS, T, MODE, MINB, XP>()) : 0;
    return cudaLaunchKernelEx(&cfg, k_apply_cluster<N1, N2, CS, T, MODE, MINB, XP>, f2, bd, a);
}

template <int N1, int N2, int CS, int T, int MINB, int XP = 0>
cudaError_t launch_size(int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a, cudaStream_t st) {
    switch (mode) {
        case NPBS_RESIDUAL: return launch_one<N1, N2, CS, T, NPBS_RESIDUAL, MINB, XP>(fd, bd, a, st);
        case NPBS_CBS_STEP: return launch_one<N1, N2, CS, T, NPBS_CBS_STEP, MINB, XP>(fd, bd, a, st);
        case NPBS_OP_B: return launch_one<N1, N2, CS, T, NPBS_OP_B, MINB, XP>(fd, bd, a, st);
        case NPBS_ADJ_B: return launch_one<N1, N2, CS, T, NPBS_ADJ_B, MINB, XP>(fd, bd, a, st);
        case NPBS_TRUE_RESIDUAL: return launch_one<N1, N2, CS, T, NPBS_TRUE_RESIDUAL, MINB, XP>(fd, bd, a, st);
        case NPBS_PREC_SWEEP: return launch_one<N1, N2, CS, T, NPBS_PREC_SWEEP, MINB, XP>(fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fastimpl
}  // namespace npbs
