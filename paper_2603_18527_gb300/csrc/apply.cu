// The fused Born apply: pointwise prologue + row FFTs, column FFT -> symbol ->
// column inverse FFT, row inverse FFTs + pointwise epilogue.
//
//   q   = prologue(x, V, f)            e.g. V x + f            (Eq. CBS / npbs_integral)
//   q^  = F q                          rows then columns       (App. Pseudospectral, step 1)
//   z^  = symbol(xi) q^                1/lambda, 1/conj(lambda) or |xi|^2 (step 2)
//   z   = F^{-1} z^                    columns then rows       (step 3)
//   out = epilogue(z, x, V, f)         e.g. x + gamma (z - x)  (Eq. CBS)
//
// Three launches per apply over the whole batch (every instance of every
// size in the same launch, one work item per band of rows or columns).  The
// intermediate spectrum lives in a context-owned scratch buffer.  The float64
// refresh (kTrueRes64) instantiates the same kernels with the double-single
// real type of dsfloat.cuh.
#include "apply.cuh"
#include "dsfloat.cuh"
#include "fft.cuh"

namespace npbs {

template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    }
    return s;  // valid in thread 0
}

template <typename R> __device__ __forceinline__ const cpx<R>* twiddles(const BatchDev& bd, int off);
template <> __device__ __forceinline__ const float2* twiddles<float>(const BatchDev& bd, int off) { return bd.tw32 + off; }
template <> __device__ __forceinline__ const dscpx* twiddles<dsf>(const BatchDev& bd, int off) {
    return reinterpret_cast<const dscpx*>(bd.twds + off);
}

// ---------------------------------------------------------------- kernel 1
template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) k_rows_forward(BatchDev bd, ApplyArgs a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RowItem it = bd.rows[blockIdx.x];
    if (bd.active && !bd.active[it.inst]) return;
    const InstDev in = bd.inst[it.inst];
    __shared__ RadixPlan plan;
    if (threadIdx.x == 0) plan = bd.plans[in.plan_x];
    const int nx = in.nx;
    const int n = it.nrows * nx;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + kTileElems<R>();
    const long long base = in.offset + (long long)it.row0 * nx;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const long long g = base + e;
        C q;
        if constexpr (MODE == kTrueRes64) {
            // fold the float32 correction into the float64 solution, then transform u
            double2 u = a.uhi[g];
            if (a.delta) {
                const float2 d = ld(a.delta + g);
                u.x += (double)d.x;
                u.y += (double)d.y;
                a.uhi[g] = u;
            }
            q = from_double2<C>(u);
        } else {
            const float2 x = ld(a.x + g);
            if constexpr (MODE == NPBS_RESIDUAL || MODE == NPBS_CBS_STEP) {
                const float2 v = ld(a.V + g), f = ld(a.f + g);
                q = mk<C>(v.x * x.x - v.y * x.y + f.x, v.x * x.y + v.y * x.x + f.y);
            } else if constexpr (MODE == NPBS_OP_B || MODE == NPBS_PREC_SWEEP) {
                const float2 v = ld(a.V + g);
                q = mk<C>(v.x * x.x - v.y * x.y, v.x * x.y + v.y * x.x);
            } else {  // ADJ_B, TRUE_RESIDUAL
                q = mk<C>(x.x, x.y);
            }
        }
        buf0[e] = q;
    }
    __syncthreads();
    C* res = fft_tile<C, -1, false>(buf0, buf1, plan, it.nrows, 1, nx, twiddles<R>(bd, in.tw_x), threadIdx.x,
                                    blockDim.x);
    C* T = reinterpret_cast<C*>(a.scratch);
    for (int e = threadIdx.x; e < n; e += blockDim.x) T[base + e] = res[e];
}

// ---------------------------------------------------------------- kernel 2
template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) k_cols(BatchDev bd, ApplyArgs a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ColItem it = bd.cols[blockIdx.x];
    if (bd.active && !bd.active[it.inst]) return;
    const InstDev in = bd.inst[it.inst];
    __shared__ RadixPlan plan;
    if (threadIdx.x == 0) plan = bd.plans[in.plan_y];
    const int nx = in.nx, ny = in.ny, nc = it.ncols;
    const int n = ny * nc;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + kTileElems<R>();
    C* T = reinterpret_cast<C*>(a.scratch);
    const long long base = in.offset + it.col0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / nc, c = e - i * nc;
        buf0[e] = T[base + (long long)i * nx + c];
    }
    __syncthreads();
    const C* tw = twiddles<R>(bd, in.tw_y);
    C* s = fft_tile<C, -1, true>(buf0, buf1, plan, nc, nc, 1, tw, threadIdx.x, blockDim.x);
    // symbol of the reference operator at (xi_y, xi_x)
    const R cy = R(6.283185307179586476925 / (in.ny * in.h));
    const R cx = R(6.283185307179586476925 / (in.nx * in.h));
    const R k0sq = R(in.k0sq), eps = R(in.eps);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / nc, c = e - i * nc;
        const R xy = cy * R(signed_mode(i, ny));
        const R xx = cx * R(signed_mode(it.col0 + c, nx));
        const R xi2 = xy * xy + xx * xx;
        C v = s[e];
        if constexpr (MODE == NPBS_TRUE_RESIDUAL || MODE == kTrueRes64) {
            v = mk<C>(v.x * xi2, v.y * xi2);
        } else {
            // lambda = xi2 - k0^2 - i eps; 1/lambda = conj(lambda)/|lambda|^2
            const R lr = xi2 - k0sq;
            const R li = (MODE == NPBS_ADJ_B) ? eps : -eps;  // conj for the adjoint
            const R inv = R(1) / (lr * lr + li * li);
            v = mk<C>((v.x * lr + v.y * li) * inv, (v.y * lr - v.x * li) * inv);
        }
        s[e] = v;
    }
    __syncthreads();
    C* o = (s == buf0) ? buf1 : buf0;
    C* r = fft_tile<C, +1, true>(s, o, plan, nc, nc, 1, tw, threadIdx.x, blockDim.x);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / nc, c = e - i * nc;
        T[base + (long long)i * nx + c] = r[e];
    }
}

// ---------------------------------------------------------------- kernel 3
template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) k_rows_inverse(BatchDev bd, ApplyArgs a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kThreads / 32];
    __shared__ double red2[kThreads / 32];
    const RowItem it = bd.rows[blockIdx.x];
    if (bd.active && !bd.active[it.inst]) return;
    const InstDev in = bd.inst[it.inst];
    __shared__ RadixPlan plan;
    if (threadIdx.x == 0) plan = bd.plans[in.plan_x];
    const int nx = in.nx;
    const int n = it.nrows * nx;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + kTileElems<R>();
    const long long base = in.offset + (long long)it.row0 * nx;
    const C* T = reinterpret_cast<const C*>(a.scratch);
    for (int e = threadIdx.x; e < n; e += blockDim.x) buf0[e] = T[base + e];
    __syncthreads();
    C* z = fft_tile<C, +1, false>(buf0, buf1, plan, it.nrows, 1, nx, twiddles<R>(bd, in.tw_x), threadIdx.x,
                                  blockDim.x);
    const R scale = R(1) / (R(in.nx) * R(in.ny));
    const R ie = R(1) / R(in.eps);
    double acc = 0.0, acc2 = 0.0;
    float accf = 0.f;  // float32 modes: this thread's share in float32, float64 across threads
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const long long g = base + e;
        const C zz = z[e];
        const R zr = zz.x * scale, zi = zz.y * scale;
        if constexpr (MODE == kTrueRes64) {
            // rho = f + k^2 u - z with k^2 = V + k0^2 + i eps
            const double2 u = a.uhi[g];
            const float2 f = ld(a.f + g);
            double kr, ki;
            if (a.k2) {
                const float2 k = ld(a.k2 + g);
                kr = (double)k.x;
                ki = (double)k.y;
            } else {
                const float2 v = ld(a.V + g);
                kr = (double)v.x + in.k0sq;
                ki = (double)v.y + in.eps;
            }
            const double rr = (double)f.x + kr * u.x - ki * u.y - to_double(zr);
            const double ri = (double)f.y + kr * u.y + ki * u.x - to_double(zi);
            if (a.out) a.out[g] = make_float2((float)rr, (float)ri);
            acc += rr * rr + ri * ri;
            acc2 += (double)f.x * f.x + (double)f.y * f.y;
        } else {
            const float2 x = a.x[g];  // plain load: out may alias x
            float2 o;
            float rr, ri;  // the quantity whose squared norm is reported
            if constexpr (MODE == NPBS_RESIDUAL) {
                rr = zr - x.x;
                ri = zi - x.y;
                o = make_float2(rr, ri);
            } else if constexpr (MODE == NPBS_CBS_STEP) {
                rr = zr - x.x;
                ri = zi - x.y;
                const float2 v = ld(a.V + g);
                // gamma = i V / eps
                const float gr = -v.y * ie, gi = v.x * ie;
                o = make_float2(x.x + gr * rr - gi * ri, x.y + gr * ri + gi * rr);
            } else if constexpr (MODE == NPBS_OP_B) {
                rr = x.x - zr;
                ri = x.y - zi;
                o = make_float2(rr, ri);
            } else if constexpr (MODE == NPBS_ADJ_B) {
                const float2 v = ld(a.V + g);
                // x - conj(V) z
                rr = x.x - (v.x * zr + v.y * zi);
                ri = x.y - (v.x * zi - v.y * zr);
                o = make_float2(rr, ri);
            } else if constexpr (MODE == NPBS_TRUE_RESIDUAL) {
                const float2 v = ld(a.V + g), f = ld(a.f + g);
                const float kr = v.x + (float)in.k0sq, ki = v.y + (float)in.eps;
                rr = f.x + kr * x.x - ki * x.y - zr;
                ri = f.y + kr * x.y + ki * x.x - zi;
                o = make_float2(rr, ri);
            } else {  // PREC_SWEEP: r = f - B x = f - x + z, out = x + gamma r
                const float2 v = ld(a.V + g), f = ld(a.f + g);
                rr = f.x - x.x + zr;
                ri = f.y - x.y + zi;
                const float gr = -v.y * ie, gi = v.x * ie;
                o = make_float2(x.x + gr * rr - gi * ri, x.y + gr * ri + gi * rr);
            }
            a.out[g] = o;
            accf = fmaf(rr, rr, fmaf(ri, ri, accf));
        }
    }
    acc += (double)accf;
    if (a.norm2 || a.norm2b) {
        const double s = block_sum(acc, red);
        double s2 = 0.0;
        if constexpr (MODE == kTrueRes64) s2 = block_sum(acc2, red2);
        if (threadIdx.x == 0) {
            if (a.norm2) atomicAdd(a.norm2 + it.inst, s);
            if (a.norm2b) atomicAdd(a.norm2b + it.inst, s2);
        }
    }
}

// ---------------------------------------------------------------- launch
template <typename R, int MODE>
static cudaError_t set_attrs() {
    const int smem = (int)(2 * kTileElems<R>() * sizeof(cpx<R>));
    cudaError_t e = cudaFuncSetAttribute(k_rows_forward<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rows_inverse<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t prepare_apply() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attrs<float, NPBS_RESIDUAL>();
    if (e == cudaSuccess) e = set_attrs<float, NPBS_CBS_STEP>();
    if (e == cudaSuccess) e = set_attrs<float, NPBS_OP_B>();
    if (e == cudaSuccess) e = set_attrs<float, NPBS_ADJ_B>();
    if (e == cudaSuccess) e = set_attrs<float, NPBS_TRUE_RESIDUAL>();
    if (e == cudaSuccess) e = set_attrs<float, NPBS_PREC_SWEEP>();
    if (e == cudaSuccess) e = set_attrs<dsf, kTrueRes64>();
    return e;
}

template <typename R, int MODE>
static cudaError_t launch3(const BatchDev& bd, int nrow_items, int ncol_items, const ApplyArgs& a, cudaStream_t st) {
    const size_t smem = 2 * kTileElems<R>() * sizeof(cpx<R>);
    if (nrow_items == 0) return cudaSuccess;
    k_rows_forward<R, MODE><<<nrow_items, kThreads, smem, st>>>(bd, a);
    k_cols<R, MODE><<<ncol_items, kThreads, smem, st>>>(bd, a);
    k_rows_inverse<R, MODE><<<nrow_items, kThreads, smem, st>>>(bd, a);
    return cudaGetLastError();
}

cudaError_t launch_apply(int mode, const BatchDev& bd, int nrow_items, int ncol_items, const ApplyArgs& a,
                         cudaStream_t st) {
    switch (mode) {
        case NPBS_RESIDUAL: return launch3<float, NPBS_RESIDUAL>(bd, nrow_items, ncol_items, a, st);
        case NPBS_CBS_STEP: return launch3<float, NPBS_CBS_STEP>(bd, nrow_items, ncol_items, a, st);
        case NPBS_OP_B: return launch3<float, NPBS_OP_B>(bd, nrow_items, ncol_items, a, st);
        case NPBS_ADJ_B: return launch3<float, NPBS_ADJ_B>(bd, nrow_items, ncol_items, a, st);
        case NPBS_TRUE_RESIDUAL: return launch3<float, NPBS_TRUE_RESIDUAL>(bd, nrow_items, ncol_items, a, st);
        case NPBS_PREC_SWEEP: return launch3<float, NPBS_PREC_SWEEP>(bd, nrow_items, ncol_items, a, st);
        case kTrueRes64: return launch3<dsf, kTrueRes64>(bd, nrow_items, ncol_items, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
