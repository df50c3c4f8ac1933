// Born apply for square grids too large for one cluster's shared memory
// (N x N with N = N1 * N2 = 1024): three launches over bands of whole rows or
// whole columns, each 1D transform a four-step FFT in registers (the same
// factorisation as the cluster kernel, n = N2 n1 + n2, k = k1 + N1 k2):
//
//   rows forward   q = prologue(x, V, f) (Eq. CBS / npbs_integral); per row
//                  N2 DFTs of length N1 (stride N2), twiddle W_N^{n2 k1}, N1
//                  DFTs of length N2; the row spectrum goes to the scratch in
//                  digit order (position N2 k1 + k2 holds frequency k1 + N1 k2)
//   columns        per column the forward four-step FFT, the Green symbol
//                  1/lambda (App. Pseudospectral, step 2) applied in digit
//                  order, the inverse four-step FFT back to natural row order
//   rows inverse   the inverse row FFT consumes digit order and returns
//                  natural order; epilogue (e.g. x + gamma (z - x), Eq. CBS)
//                  and the per-instance squared norm
//
// so no pass reorders data.  A CTA holds its band in a padded shared-memory
// slab (pad(p) = p + p / N2; row stride LD = 2 mod 16 float2, so both the
// 8-column x 2-row accesses of the column kernel and the contiguous accesses
// of the row kernels are free of bank conflicts).  HBM traffic: the row
// kernels read x, V, f and write the spectrum (32 B/point), the column kernel
// reads and writes it (16 B), the inverse row kernel reads it, x and V and
// writes the result (32 B).
#include <algorithm>

#include "apply.cuh"
#include "apply_fast.cuh"
#include "dftreg.cuh"

namespace npbs {
namespace bandimpl {

template <int N2> __device__ __forceinline__ int pad(int p) { return p + p / N2; }
// W_N^{n2 k1} stored as [k1][N2 + 1]
template <int N2> __device__ __forceinline__ int twi(int k1, int n2) { return k1 * (N2 + 1) + n2; }

template <int N1, int N2> constexpr int slab_ld() { return ((N1 * N2 + N1 + 13) / 16) * 16 + 2; }

// slab of W rows (or columns) plus the twiddle table
template <int N1, int N2, int W> constexpr size_t band_smem() {
    return sizeof(float2) * ((size_t)W * slab_ld<N1, N2>() + (size_t)N1 * (N2 + 1));
}

__device__ __forceinline__ float2 cmul_w(float2 t, float2 w) {
    return make_float2(t.x * w.x - t.y * w.y, t.x * w.y + t.y * w.x);
}
// t * conj(w)
__device__ __forceinline__ float2 cmul_wc(float2 t, float2 w) {
    return make_float2(t.x * w.x + t.y * w.y, t.y * w.x - t.x * w.y);
}

template <int N1, int N2, int T> __device__ __forceinline__ void load_twiddles(float2* tw, const float2* src) {
    for (int e = threadIdx.x; e < N1 * N2; e += T) {
        const int k1 = e / N2, n2 = e - k1 * N2;
        tw[twi<N2>(k1, n2)] = src[n2 * k1];
    }
}

// ---------------------------------------------------------------- rows forward
template <int N1, int N2, int RB, int T, int MODE, int MINB>
__global__ void __launch_bounds__(T, MINB) k_band_rows_fwd(FastDev fd, BatchDev bd, ApplyArgs a) {
    constexpr int N = N1 * N2, LD = slab_ld<N1, N2>(), NB = N / RB;
    static_assert(N % RB == 0 && (RB * N) % T == 0, "bands of whole rows, copied in whole strides");
    extern __shared__ __align__(16) float2 smem[];
    float2* S = smem;            // [RB][LD]
    float2* tw = smem + RB * LD;  // [N1][N2 + 1]
    const int li = blockIdx.x / NB, band = blockIdx.x - li * NB;
    const int instx = fd.list[li];
    if (bd.active && !bd.active[instx]) return;  // uniform over the block
    const InstDev in = bd.inst[instx];
    const int tid = threadIdx.x;
    load_twiddles<N1, N2, T>(tw, bd.tw32 + in.tw_x);
    __syncthreads();
    const long long row0 = in.offset + (long long)band * RB * N;
    // pass 1: length-N1 DFTs over stride-N2 points of q, twiddled
    for (int j = tid; j < RB * N2; j += T) {
        const int n2 = j % N2, r = j / N2;
        const long long g0 = row0 + (long long)r * N + n2;
        float2 v[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) {
            const long long g = g0 + N2 * m;
            const float2 x = __ldg(a.x + g);
            if constexpr (MODE == NPBS_RESIDUAL || MODE == NPBS_CBS_STEP) {
                const float2 V = __ldg(a.V + g), f = __ldg(a.f + g);
                v[m] = make_float2(V.x * x.x - V.y * x.y + f.x, V.x * x.y + V.y * x.x + f.y);
            } else if constexpr (MODE == NPBS_OP_B || MODE == NPBS_PREC_SWEEP) {
                const float2 V = __ldg(a.V + g);
                v[m] = make_float2(V.x * x.x - V.y * x.y, V.x * x.y + V.y * x.x);
            } else {  // ADJ_B, TRUE_RESIDUAL transform x itself
                v[m] = x;
            }
        }
        DftR<N1, -1>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) S[r * LD + pad<N2>(N2 * k1 + n2)] = cmul_w(v[k1], tw[twi<N2>(k1, n2)]);
    }
    __syncthreads();
    // pass 2: length-N2 DFTs over contiguous blocks, in place (digit order)
    for (int j = tid; j < RB * N1; j += T) {
        const int k1 = j % N1, r = j / N1;
        float2* p = S + r * LD;
        float2 v[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = p[pad<N2>(N2 * k1 + i)];
        DftR<N2, -1>::run(v);
#pragma unroll
        for (int i = 0; i < N2; ++i) p[pad<N2>(N2 * k1 + i)] = v[i];
    }
    __syncthreads();
    // coalesced copy of the band to the scratch (row-major, x in digit order)
    float2* Tr = reinterpret_cast<float2*>(a.scratch) + row0;
#pragma unroll
    for (int s = 0; s < RB * N / T; ++s) {
        const int e = tid + s * T, r = e / N, p = e - r * N;
        __stcg(Tr + e, S[r * LD + pad<N2>(p)]);
    }
}

// ---------------------------------------------------------------- columns
template <int N1, int N2, int CB, int T, int MODE, int MINB>
__global__ void __launch_bounds__(T, MINB) k_band_cols(FastDev fd, BatchDev bd, ApplyArgs a) {
    constexpr int N = N1 * N2, LD = slab_ld<N1, N2>(), NB = N / CB;
    static_assert(N % CB == 0, "bands of whole columns");
    extern __shared__ __align__(16) float2 smem[];
    float2* S = smem;             // [CB][LD]: column c of the band, padded row position
    float2* tw = smem + CB * LD;  // [N1][N2 + 1]
    const int li = blockIdx.x / NB, band = blockIdx.x - li * NB;
    const int instx = fd.list[li];
    if (bd.active && !bd.active[instx]) return;
    const InstDev in = bd.inst[instx];
    const int tid = threadIdx.x;
    load_twiddles<N1, N2, T>(tw, bd.tw32 + in.tw_x);
    __syncthreads();
    const int p0 = band * CB;
    float2* Tg = reinterpret_cast<float2*>(a.scratch) + in.offset + p0;  // element (y, c) at Tg[y N + c]
    // pass 1: length-N1 DFTs over rows n2 + N2 m, twiddled
    for (int j = tid; j < CB * N2; j += T) {
        const int c = j % CB, n2 = j / CB;
        float2 v[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = __ldcg(Tg + (long long)(n2 + N2 * m) * N + c);
        DftR<N1, -1>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) S[c * LD + pad<N2>(N2 * k1 + n2)] = cmul_w(v[k1], tw[twi<N2>(k1, n2)]);
    }
    __syncthreads();
    // pass 2: length-N2 DFTs, the symbol at (xi_y, xi_x) in digit order,
    // inverse length-N2 DFTs, conjugate twiddle
    {
        const float cxi = (float)(6.283185307179586476925 / ((double)N * in.h));
        const float k0sq = (float)in.k0sq, eps = (float)in.eps;
        for (int j = tid; j < CB * N1; j += T) {
            const int k1 = j % N1, c = j / N1;
            float2* p = S + c * LD;
            float2 v[N2];
#pragma unroll
            for (int i = 0; i < N2; ++i) v[i] = p[pad<N2>(N2 * k1 + i)];
            DftR<N2, -1>::run(v);
            const int px = p0 + c;  // digit-order x position: frequency px / N2 + N1 (px % N2)
            const float xx = cxi * (float)signed_mode(px / N2 + N1 * (px % N2), N);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const float xy = cxi * (float)signed_mode(k1 + N1 * k2, N);
                const float xi2 = xx * xx + xy * xy;
                const float2 t = v[k2];
                if constexpr (MODE == NPBS_TRUE_RESIDUAL) {
                    v[k2] = make_float2(t.x * xi2, t.y * xi2);
                } else {
                    // lambda = xi2 - k0^2 - i eps; 1/lambda = conj(lambda) / |lambda|^2
                    const float lr = xi2 - k0sq;
                    const float lim = (MODE == NPBS_ADJ_B) ? eps : -eps;  // conj for the adjoint
                    float inv;  // hardware reciprocal (rcp.approx, ~1 ulp)
                    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(fmaf(lr, lr, lim * lim)));
                    v[k2] = make_float2((t.x * lr + t.y * lim) * inv, (t.y * lr - t.x * lim) * inv);
                }
            }
            DftR<N2, +1>::run(v);
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) p[pad<N2>(N2 * k1 + n2)] = cmul_wc(v[n2], tw[twi<N2>(k1, n2)]);
        }
    }
    __syncthreads();
    // pass 3: inverse length-N1 DFTs -> natural row y = N2 n1 + n2
    for (int j = tid; j < CB * N2; j += T) {
        const int c = j % CB, n2 = j / CB;
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = S[c * LD + pad<N2>(N2 * k1 + n2)];
        DftR<N1, +1>::run(v);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) __stcg(Tg + (long long)(N2 * n1 + n2) * N + c, v[n1]);
    }
}

// ---------------------------------------------------------------- rows inverse
template <int N1, int N2, int RB, int T, int MODE, int MINB>
__global__ void __launch_bounds__(T, MINB) k_band_rows_inv(FastDev fd, BatchDev bd, ApplyArgs a) {
    constexpr int N = N1 * N2, LD = slab_ld<N1, N2>(), NB = N / RB;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ double red[T / 32];
    float2* S = smem;
    float2* tw = smem + RB * LD;
    const int li = blockIdx.x / NB, band = blockIdx.x - li * NB;
    const int instx = fd.list[li];
    if (bd.active && !bd.active[instx]) return;
    const InstDev in = bd.inst[instx];
    const int tid = threadIdx.x;
    load_twiddles<N1, N2, T>(tw, bd.tw32 + in.tw_x);
    const long long row0 = in.offset + (long long)band * RB * N;
    const float2* Tr = reinterpret_cast<const float2*>(a.scratch) + row0;
    {
        float2 u[RB * N / T];  // every load of the band in flight before the first shared store
#pragma unroll
        for (int s = 0; s < RB * N / T; ++s) u[s] = __ldcg(Tr + tid + s * T);
#pragma unroll
        for (int s = 0; s < RB * N / T; ++s) {
            const int e = tid + s * T, r = e / N, p = e - r * N;
            S[r * LD + pad<N2>(p)] = u[s];
        }
    }
    __syncthreads();
    // pass A: inverse length-N2 DFTs on digit order, conjugate twiddle
    for (int j = tid; j < RB * N1; j += T) {
        const int k1 = j % N1, r = j / N1;
        float2* p = S + r * LD;
        float2 v[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = p[pad<N2>(N2 * k1 + i)];
        DftR<N2, +1>::run(v);
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) p[pad<N2>(N2 * k1 + n2)] = cmul_wc(v[n2], tw[twi<N2>(k1, n2)]);
    }
    __syncthreads();
    // pass B: inverse length-N1 DFTs -> natural x = N2 n1 + n2, then the epilogue
    constexpr bool USE_V = MODE != NPBS_RESIDUAL && MODE != NPBS_OP_B;
    constexpr bool USE_F = MODE == NPBS_TRUE_RESIDUAL || MODE == NPBS_PREC_SWEEP;
    // out may alias x, so no load can move past an earlier store: the operands
    // of EC points are loaded together, then those points are written
    constexpr int EC = 8;
    static_assert(N1 % EC == 0, "whole chunks");
    const float scale = 1.f / ((float)N * (float)N);
    const float ie = (float)(1.0 / in.eps);
    float acc = 0.f;  // this thread's share of the norm (float64 across threads)
    for (int j = tid; j < RB * N2; j += T) {
        const int n2 = j % N2, r = j / N2;
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = S[r * LD + pad<N2>(N2 * k1 + n2)];
        DftR<N1, +1>::run(v);
        const long long g0 = row0 + (long long)r * N + n2;
#pragma unroll
        for (int c0 = 0; c0 < N1; c0 += EC) {
            float2 xs[EC], Vs[EC], fs[EC];
#pragma unroll
            for (int i = 0; i < EC; ++i) {
                const long long g = g0 + N2 * (c0 + i);
                xs[i] = a.x[g];  // plain load: out may alias x (each point is read, then written, by one thread)
                if constexpr (USE_V) Vs[i] = __ldg(a.V + g);
                if constexpr (USE_F) fs[i] = __ldg(a.f + g);
            }
#pragma unroll
            for (int i = 0; i < EC; ++i) {
                const int n1 = c0 + i;
                const long long g = g0 + N2 * n1;
                const float zr = v[n1].x * scale, zi = v[n1].y * scale;
                const float2 x = xs[i];
                float rr, ri;  // the quantity whose squared norm is reported
                float2 o;
                if constexpr (MODE == NPBS_RESIDUAL) {
                    rr = zr - x.x;
                    ri = zi - x.y;
                    o = make_float2(rr, ri);
                } else if constexpr (MODE == NPBS_CBS_STEP) {
                    rr = zr - x.x;
                    ri = zi - x.y;
                    const float2 V = Vs[i];
                    const float gr = -V.y * ie, gi = V.x * ie;  // gamma = i V / eps
                    o = make_float2(x.x + gr * rr - gi * ri, x.y + gr * ri + gi * rr);
                } else if constexpr (MODE == NPBS_OP_B) {
                    rr = x.x - zr;
                    ri = x.y - zi;
                    o = make_float2(rr, ri);
                } else if constexpr (MODE == NPBS_ADJ_B) {
                    const float2 V = Vs[i];  // x - conj(V) z
                    rr = x.x - (V.x * zr + V.y * zi);
                    ri = x.y - (V.x * zi - V.y * zr);
                    o = make_float2(rr, ri);
                } else if constexpr (MODE == NPBS_TRUE_RESIDUAL) {
                    const float2 V = Vs[i], f = fs[i];
                    const float kr = V.x + (float)in.k0sq, ki = V.y + (float)in.eps;
                    rr = f.x + kr * x.x - ki * x.y - zr;
                    ri = f.y + kr * x.y + ki * x.x - zi;
                    o = make_float2(rr, ri);
                } else {  // PREC_SWEEP: r = f - B x = f - x + z, out = x + gamma r
                    const float2 V = Vs[i], f = fs[i];
                    rr = f.x - x.x + zr;
                    ri = f.y - x.y + zi;
                    const float gr = -V.y * ie, gi = V.x * ie;
                    o = make_float2(x.x + gr * rr - gi * ri, x.y + gr * ri + gi * rr);
                }
                a.out[g] = o;
                acc = fmaf(rr, rr, fmaf(ri, ri, acc));
            }
        }
    }
    if (a.norm2) {
        double accd = acc;
        for (int o = 16; o > 0; o >>= 1) accd += __shfl_xor_sync(0xffffffffu, accd, o);
        if ((tid & 31) == 0) red[tid >> 5] = accd;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < T / 32; ++w) t += red[w];
            atomicAdd(a.norm2 + instx, t);
        }
    }
}

// ---------------------------------------------------------------- launch
// A variant: (N1, N2), rows per row-kernel block RB with TR threads and MR
// blocks per SM, columns per column-kernel block CB with TC threads and MC.
template <int N1, int N2, int RB, int TR, int MR, int CB, int TC, int MC> struct Variant {
    static_assert(RB * N2 == TR && RB * N1 == TR, "one row job per thread in every row pass");
    static_assert(CB * N2 == TC && CB * N1 == TC, "one column job per thread in every column pass");

    template <int MODE> static cudaError_t set_attrs() {
        cudaError_t e = cudaFuncSetAttribute(k_band_rows_fwd<N1, N2, RB, TR, MODE, MR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem<N1, N2, RB>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_band_cols<N1, N2, CB, TC, MODE, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)band_smem<N1, N2, CB>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_band_rows_inv<N1, N2, RB, TR, MODE, MR>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_smem<N1, N2, RB>());
        return e;
    }

    static cudaError_t prepare() {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = set_attrs<NPBS_RESIDUAL>();
        if (e == cudaSuccess) e = set_attrs<NPBS_CBS_STEP>();
        if (e == cudaSuccess) e = set_attrs<NPBS_OP_B>();
        if (e == cudaSuccess) e = set_attrs<NPBS_ADJ_B>();
        if (e == cudaSuccess) e = set_attrs<NPBS_TRUE_RESIDUAL>();
        if (e == cudaSuccess) e = set_attrs<NPBS_PREC_SWEEP>();
        return e;
    }

    template <int MODE>
    static cudaError_t launch_mode(const FastDev& fd, const BatchDev& bd, const ApplyArgs& a, cudaStream_t st) {
        constexpr int N = N1 * N2;
        constexpr bool ITER = MODE == NPBS_CBS_STEP || MODE == NPBS_PREC_SWEEP;
        const int steps = ITER ? std::max(1, a.steps) : 1;
        const unsigned gr = (unsigned)(fd.count * (N / RB)), gc = (unsigned)(fd.count * (N / CB));
        for (int k = 0; k < steps; ++k) {
            ApplyArgs ak = a;
            if (k > 0) ak.x = a.out;
            if (k < steps - 1) ak.norm2 = nullptr;
            k_band_rows_fwd<N1, N2, RB, TR, MODE, MR><<<gr, TR, band_smem<N1, N2, RB>(), st>>>(fd, bd, ak);
            k_band_cols<N1, N2, CB, TC, MODE, MC><<<gc, TC, band_smem<N1, N2, CB>(), st>>>(fd, bd, ak);
            k_band_rows_inv<N1, N2, RB, TR, MODE, MR><<<gr, TR, band_smem<N1, N2, RB>(), st>>>(fd, bd, ak);
        }
        return cudaGetLastError();
    }

    static cudaError_t launch(int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a, cudaStream_t st) {
        switch (mode) {
            case NPBS_RESIDUAL: return launch_mode<NPBS_RESIDUAL>(fd, bd, a, st);
            case NPBS_CBS_STEP: return launch_mode<NPBS_CBS_STEP>(fd, bd, a, st);
            case NPBS_OP_B: return launch_mode<NPBS_OP_B>(fd, bd, a, st);
            case NPBS_ADJ_B: return launch_mode<NPBS_ADJ_B>(fd, bd, a, st);
            case NPBS_TRUE_RESIDUAL: return launch_mode<NPBS_TRUE_RESIDUAL>(fd, bd, a, st);
            case NPBS_PREC_SWEEP: return launch_mode<NPBS_PREC_SWEEP>(fd, bd, a, st);
            default: return cudaErrorInvalidValue;
        }
    }
};

// 1024 = 32 x 32: 8 rows per 256-thread block (2 per SM) or 4 rows per
// 128-thread block (4 per SM); 8 columns per 256-thread block
using V0 = Variant<32, 32, 8, 256, 2, 8, 256, 2>;
using V1 = Variant<32, 32, 4, 128, 4, 8, 256, 2>;

}  // namespace bandimpl

int band_variants_1024() { return 2; }

cudaError_t prepare_band_1024() {
    cudaError_t e = bandimpl::V0::prepare();
    if (e == cudaSuccess) e = bandimpl::V1::prepare();
    return e;
}

cudaError_t launch_band_1024(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                             cudaStream_t st) {
    switch (variant) {
        case 0: return bandimpl::V0::launch(mode, fd, bd, a, st);
        case 1: return bandimpl::V1::launch(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
