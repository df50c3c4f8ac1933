// Newton-Born linearisation with a DST-I Green operator (App. Full
// Derivations, Nonlinear PDE via Newton-Born Linearization; Eqs.
// nonlinear_residual, newton_linear_system, newton_ref, newton_vm,
// newton_born_identity, newton_inner_iter; App. Verification, Newton linear
// systems):
//
//   F(u) = L_D u - u^2 - f on N x N interior unknowns, homogeneous Dirichlet,
//          L_D the five-point negative Laplacian / h^2, h = 1/(N + 1)
//   J    = L_D - 2 diag(u_m),  J0 = L_D + c I,  c = alpha - 2 mean(u_m)
//   V    = J0 - J = c + 2 u_m,  G = J0^{-1} = S^{-1} diag(1/lambda) S
//   lambda_pq = (4/h^2)(sin^2(p pi h/2) + sin^2(q pi h/2)) + c
//   S the 2D DST-I, S_jk = sin(pi j k / (N + 1)), S^{-1} = (2/(N+1))^2 S.
//
// The transform is a dense contraction with the sine matrix in shared memory:
// the paper's grid (N = 64) has N + 1 = 65, which no 2^a 3^b FFT of length
// 2(N + 1) covers, and at N <= 96 the two N^3 products per transform are a
// few microseconds per instance.  One CTA holds one instance: the stencil,
// both transforms, the symbol and the epilogue never leave shared memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "ctx.cuh"
#include "net.cuh"
#include "umma.cuh"

namespace npbs {
namespace {

constexpr int kNtMaxN = 96;

struct NtInst {
    int n;
    long long off;
};

// mode values of the fused apply beside the public ones
constexpr int kNtGreen = 100;  // out = G x

// sine-matrix products on an n x n tile (n a multiple of 4), 4 x 4 outputs per
// thread: LEFT out = S Q, else out = Q S (S real symmetric, Q complex)
template <bool LEFT>
__device__ __forceinline__ void sine_mul(const float* __restrict__ S, const float2* __restrict__ Q,
                                         float2* __restrict__ out, int n) {
    const int nb = n >> 2;
    for (int blk = threadIdx.x; blk < nb * nb; blk += blockDim.x) {
        const int i0 = (blk / nb) * 4, j0 = (blk % nb) * 4;
        float2 acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
        for (int k = 0; k < n; ++k) {
            if (LEFT) {
                // out[i][j] += S[i][k] Q[k][j], S[i][k] = S[k][i]
                const float4 s = *reinterpret_cast<const float4*>(S + k * n + i0);
                const float a[4] = {s.x, s.y, s.z, s.w};
                const float4 q01 = *reinterpret_cast<const float4*>(Q + k * n + j0);
                const float4 q23 = *reinterpret_cast<const float4*>(Q + k * n + j0 + 2);
                const float2 b[4] = {make_float2(q01.x, q01.y), make_float2(q01.z, q01.w),
                                     make_float2(q23.x, q23.y), make_float2(q23.z, q23.w)};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[r][c].x = fmaf(a[r], b[c].x, acc[r][c].x);
                        acc[r][c].y = fmaf(a[r], b[c].y, acc[r][c].y);
                    }
            } else {
                // out[i][j] += Q[i][k] S[k][j]
                const float4 s = *reinterpret_cast<const float4*>(S + k * n + j0);
                const float b[4] = {s.x, s.y, s.z, s.w};
                float2 a[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = Q[(i0 + r) * n + k];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[r][c].x = fmaf(a[r].x, b[c], acc[r][c].x);
                        acc[r][c].y = fmaf(a[r].y, b[c], acc[r][c].y);
                    }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) out[(i0 + r) * n + j0 + c] = acc[r][c];
    }
}

// A <- G A in place (B scratch): S A S, divided by lambda / (2/(n+1))^2, S . S
__device__ __forceinline__ void green_tile(const float* S, const float* eig, float2* A, float2* B, int n,
                                           float shift) {
    sine_mul<true>(S, A, B, n);
    __syncthreads();
    sine_mul<false>(S, B, A, n);
    __syncthreads();
    const float sc = 4.f / ((float)(n + 1) * (float)(n + 1));
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        const float l = eig[i] + eig[j] + shift;
        const float w = sc / l;
        A[e] = make_float2(A[e].x * w, A[e].y * w);
    }
    __syncthreads();
    sine_mul<true>(S, A, B, n);
    __syncthreads();
    sine_mul<false>(S, B, A, n);
    __syncthreads();
}

// (J x)(e) from a tile X: L_D x - 2 u x with zero values outside the grid
__device__ __forceinline__ float2 jac_point(const float2* X, int n, int i, int j, float inv_h2, float uv) {
    const float2 c = X[i * n + j];
    float2 s = make_float2(4.f * c.x, 4.f * c.y);
    if (i > 0) { s.x -= X[(i - 1) * n + j].x; s.y -= X[(i - 1) * n + j].y; }
    if (i < n - 1) { s.x -= X[(i + 1) * n + j].x; s.y -= X[(i + 1) * n + j].y; }
    if (j > 0) { s.x -= X[i * n + j - 1].x; s.y -= X[i * n + j - 1].y; }
    if (j < n - 1) { s.x -= X[i * n + j + 1].x; s.y -= X[i * n + j + 1].y; }
    return make_float2(s.x * inv_h2 - 2.f * uv * c.x, s.y * inv_h2 - 2.f * uv * c.y);
}

// One fused float32 apply per CTA (instance blockIdx.x of the group):
//   RESIDUAL      out = G(r - J x)      OP_B  out = G J x
//   TRUE_RESIDUAL out = r - J x (r nullable: -J x)
//   ADJ_B         out = (G J)^* x = J G x (J and G real symmetric)
//   kNtGreen      out = G x
// tab: the group's sine matrix [n][n] then the 1D eigenvalues (4/h^2) sin^2(p pi h/2) [n].
__global__ void __launch_bounds__(256) k_nt_apply(const NtInst* ins, const int* ids, const float* tab,
                                                  const double* shift, const float* u, const float2* r,
                                                  const float2* x, float2* out, double* norm2, int mode) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const NtInst in = ins[blockIdx.x];
    const int n = in.n, np = n * n;
    float* S = reinterpret_cast<float*>(smraw);
    float* eig = S + np;
    float2* A = reinterpret_cast<float2*>(eig + ((n + 3) & ~3));
    float2* B = A + np;
    __shared__ double red[8];
    const int j = ids[blockIdx.x];
    const float c = (float)shift[j];
    const float inv_h2 = (float)(n + 1) * (float)(n + 1);
    for (int e = threadIdx.x; e < np + n; e += blockDim.x) S[e] = tab[e];
    for (int e = threadIdx.x; e < np; e += blockDim.x) A[e] = x[in.off + e];
    __syncthreads();
    const float2* res = A;
    if (mode == NPBS_ADJ_B || mode == kNtGreen) {
        green_tile(S, eig, A, B, n, c);
        if (mode == NPBS_ADJ_B) {
            for (int e = threadIdx.x; e < np; e += blockDim.x) {
                const int i = e / n, jj = e - i * n;
                B[e] = jac_point(A, n, i, jj, inv_h2, u[in.off + e]);
            }
            __syncthreads();
            res = B;
        }
    } else {
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            const int i = e / n, jj = e - i * n;
            float2 q = jac_point(A, n, i, jj, inv_h2, u[in.off + e]);
            if (mode != NPBS_OP_B) {
                const float2 rv = r ? r[in.off + e] : make_float2(0.f, 0.f);
                q = make_float2(rv.x - q.x, rv.y - q.y);
            }
            B[e] = q;
        }
        __syncthreads();
        if (mode != NPBS_TRUE_RESIDUAL) green_tile(S, eig, B, A, n, c);
        res = B;
    }
    double acc = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const float2 v = res[e];
        out[in.off + e] = v;
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    if (norm2) {
        for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            atomicAdd(norm2 + j, t);
        }
    }
}

// block sum of a double (blockDim.x <= 256); every thread gets the total
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int w = 16; w > 0; w >>= 1) v += __shfl_xor_sync(0xffffffffu, v, w);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// five-point L_D x at (i, j) in float64 from global memory
__device__ __forceinline__ double lap64(const double* X, int n, int i, int j) {
    const double c = X[i * n + j];
    double s = 4.0 * c;
    if (i > 0) s -= X[(i - 1) * n + j];
    if (i < n - 1) s -= X[(i + 1) * n + j];
    if (j > 0) s -= X[i * n + j - 1];
    if (j < n - 1) s -= X[i * n + j + 1];
    return s * (double)(n + 1) * (double)(n + 1);
}

// Newton linearisation per instance (one CTA): r = -F(u) = f - L_D u + u^2,
// shift = alpha - 2 mean(u), u32 = (float)u, and the squared norms of r and f
// (out4[4 j ..]: ||r||^2, ||f||^2).  Frozen instances are skipped.
__global__ void k_nt_linearise(const NtInst* ins, const int* ids, const int* frozen, const double* u,
                               const double* f, double alpha, double* r, float* u32, double* shift, double* out4) {
    __shared__ double red[8];
    const NtInst in = ins[blockIdx.x];
    const int j = ids[blockIdx.x];
    if (frozen && frozen[j]) return;
    const int n = in.n, np = n * n;
    const double* U = u + in.off;
    double su = 0.0, sr = 0.0, sf = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int i = e / n, jj = e - i * n;
        const double uv = U[e], fv = f[in.off + e];
        const double rv = fv - lap64(U, n, i, jj) + uv * uv;
        r[in.off + e] = rv;
        u32[in.off + e] = (float)uv;
        su += uv;
        sr += rv * rv;
        sf += fv * fv;
    }
    su = block_sum(su, red);
    sr = block_sum(sr, red);
    sf = block_sum(sf, red);
    if (threadIdx.x == 0) {
        shift[j] = alpha - 2.0 * su / (double)np;
        out4[4 * j] = sr;
        out4[4 * j + 1] = sf;
    }
}

// The inner solve's float64 check per instance (one CTA): delta += eps
// (complex), eps = 0, rho = r - J delta in float64 (rounded to complex64 into
// rho32) and out4[4 j + 2] = ||rho||^2.  Instances with frozen set are skipped.
// its_out non-null: the check also freezes the instance on the device when
// it passes (||rho||^2 <= rtol2 ||r||^2, ||r||^2 from out4[4 j]), is not
// finite, or it >= max_it, recording it in its_out[j].
__global__ void k_nt_check(const NtInst* ins, const int* ids, int* frozen, const double* u, const double* r,
                           float2* eps, double2* delta, float2* rho32, double* out4, int* its_out, double rtol2,
                           int it, int max_it) {
    __shared__ double red[8];
    const NtInst in = ins[blockIdx.x];
    const int j = ids[blockIdx.x];
    if (frozen[j]) return;
    const int n = in.n, np = n * n;
    double2* D = delta + in.off;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const float2 d = eps[in.off + e];
        D[e] = make_double2(D[e].x + (double)d.x, D[e].y + (double)d.y);
        eps[in.off + e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const double inv_h2 = (double)(n + 1) * (double)(n + 1);
    double s2 = 0.0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int i = e / n, jj = e - i * n;
        double lx = 4.0 * D[e].x, ly = 4.0 * D[e].y;
        if (i > 0) { lx -= D[e - n].x; ly -= D[e - n].y; }
        if (i < n - 1) { lx -= D[e + n].x; ly -= D[e + n].y; }
        if (jj > 0) { lx -= D[e - 1].x; ly -= D[e - 1].y; }
        if (jj < n - 1) { lx -= D[e + 1].x; ly -= D[e + 1].y; }
        const double uv = u[in.off + e];
        const double jx = lx * inv_h2 - 2.0 * uv * D[e].x, jy = ly * inv_h2 - 2.0 * uv * D[e].y;
        const double px = r[in.off + e] - jx, py = -jy;
        rho32[in.off + e] = make_float2((float)px, (float)py);
        s2 += px * px + py * py;
    }
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
        out4[4 * j + 2] = s2;
        if (its_out) {
            const double q = s2 / fmax(out4[4 * j], 1e-300);
            if (!isfinite(q) || q <= rtol2 || it >= max_it) {
                frozen[j] = 1;
                its_out[j] = it;
            }
        }
    }
}

// u += Re delta, delta = 0 (instances with active set)
__global__ void k_nt_update(const NtInst* ins, const int* ids, const int* active, double* u, double2* delta) {
    const NtInst in = ins[blockIdx.x];
    if (!active[ids[blockIdx.x]]) return;
    const int np = in.n * in.n;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        u[in.off + e] += delta[in.off + e].x;
        delta[in.off + e] = make_double2(0.0, 0.0);
    }
}

// out = (complex64) r for one instance per CTA
__global__ void k_nt_to_c64(const NtInst* ins, const double* r, float2* out) {
    const NtInst in = ins[blockIdx.x];
    const int np = in.n * in.n;
    for (int e = threadIdx.x; e < np; e += blockDim.x) out[in.off + e] = make_float2((float)r[in.off + e], 0.f);
}

// eps += rr on the instances not frozen (the Born step, M = identity)
__global__ void k_nt_axpy(const NtInst* ins, const int* ids, const int* frozen, const float2* rr, float2* eps) {
    const NtInst in = ins[blockIdx.x];
    if (frozen[ids[blockIdx.x]]) return;
    const int np = in.n * in.n;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const float2 a = rr[in.off + e];
        float2 b = eps[in.off + e];
        eps[in.off + e] = make_float2(b.x + a.x, b.y + a.y);
    }
}

// ---------------------------------------------------------------- tensor cores

// The same apply on the 5th-generation tensor cores for side 64 (modes
// RESIDUAL, OP_B, ADJ_B and kNtGreen).  G = S diag(w) (S q S) S is four real
// 64 x 64 sine-matrix products of a complex tile, each one MMA of M = 128
// (rows: real parts of 64 rows, then imaginary parts), N = 64, K = 64 against
// S in TF32 with a three-term split (hi hi + hi lo + lo hi, hi = tf32(v), lo =
// tf32(v - hi)), which keeps float32 accuracy.  The accumulator sits in TMEM,
// lane = operand row; between products every thread moves its lane into the
// next operand transposed (lane (p, a) holding columns b becomes column a of
// rows (p, b)), which is a conflict-free row write of the swizzled tile, so
// S q S, the symbol and S Z S chain without a separate transpose:
//   A0 = q        -> D0[(p,i)][j] = (q S)[i][j]
//   A1 = D0^T     -> D1[(p,j)][i] = (S q S)[i][j]   (scaled by w[i][j] on the way out)
//   A2 = D1^T     -> D2[(p,i)][j] = (Z S)[i][j]
//   A3 = D2^T     -> D3[(p,j)][i] = (S Z S)[i][j] = (G q)[i][j]
// One CTA (eight warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns
// 32 (w / 4) .. + 31) walks instances blockIdx.x, blockIdx.x + gridDim.x, ...;
// thread 0 issues the MMAs and waits (bounded) on their commit; a wait that
// gives up sets g_nt_tc_timeout and the CTA stops.
constexpr int kNtTcN = 64;
constexpr int kNtTcBytes = 98304 + 1024 + 512;  // A hi/lo, S hi/lo, alignment slack, eig / flags
__device__ int g_nt_tc_timeout = 0;

// v = hi + lo as two TF32 values, each rounded to nearest (ties away from
// zero) by adding half a unit of the 10-bit mantissa to the magnitude bits and
// clearing the 13 bits below it; v - hi is exact in float32
__device__ __forceinline__ uint32_t tf32_round(uint32_t b) { return (b + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
    const uint32_t h = tf32_round(__float_as_uint(v));
    const uint32_t l = tf32_round(__float_as_uint(v - __uint_as_float(h)));
    *reinterpret_cast<uint32_t*>(hi + off) = h;
    *reinterpret_cast<uint32_t*>(lo + off) = l;
}

constexpr int kNtTcThreads = 256;
__global__ void __launch_bounds__(kNtTcThreads, 2) k_nt_apply_tc(const NtInst* ins, const int* ids, int cnt, const float* tab,
                                                     const double* shift, const float* u, const float2* r,
                                                     const float2* x, float2* out, double* norm2, int mode,
                                                     long long wait_limit) {
    using namespace umma;
    extern __shared__ unsigned char smraw_tc[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw_tc + 1023) & ~(uintptr_t)1023);
    unsigned char* Ah = base;           // operand A: 128 rows x 64, tf32 high parts (2 x 16 KB)
    unsigned char* Al = base + 32768;   // low parts
    unsigned char* Sh = base + 65536;   // the sine matrix as operand B: 64 rows x 64 (2 x 8 KB)
    unsigned char* Sl = base + 81920;
    float* eig = reinterpret_cast<float*>(base + 98304);
    double* red = reinterpret_cast<double*>(eig + kNtTcN);
    uint64_t* bar = reinterpret_cast<uint64_t*>(red + kNtTcThreads / 32);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    int* okflag = reinterpret_cast<int*>(tslot + 1);
    float2* O = reinterpret_cast<float2*>(base);  // result staging over A once the last product is done
    constexpr int n = kNtTcN, np = kNtTcN * kNtTcN;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    if (t == 0) {
        mbar_init(su32(bar), 1);
        *okflag = 1;
    }
    if (w == 0) tmem_alloc(tslot, 64);
    {
        // the table as float4 (4 per thread, all loads in flight before the stores)
        float4 tv[np / 4 / kNtTcThreads];
#pragma unroll
        for (int m = 0; m < np / 4 / kNtTcThreads; ++m) tv[m] = reinterpret_cast<const float4*>(tab)[t + kNtTcThreads * m];
#pragma unroll
        for (int m = 0; m < np / 4 / kNtTcThreads; ++m) {
            const int e = 4 * (t + kNtTcThreads * m), row = e >> 6, k = e & 63;
            put_split(Sh, Sl, sw128_off(row, k, n), tv[m].x);
            put_split(Sh, Sl, sw128_off(row, k + 1, n), tv[m].y);
            put_split(Sh, Sl, sw128_off(row, k + 2, n), tv[m].z);
            put_split(Sh, Sl, sw128_off(row, k + 3, n), tv[m].w);
        }
    }
    if (t < n) eig[t] = tab[np + t];
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_tf32(128, n);
    // operand descriptors at the tile bases (shared addresses < 256 KB: the 14-bit
    // start field never carries when a K sub-step is added)
    const uint64_t dAh = desc_sw128(su32(Ah)), dAl = desc_sw128(su32(Al));
    const uint64_t dSh = desc_sw128(su32(Sh)), dSl = desc_sw128(su32(Sl));
    const float inv_h2 = (float)(n + 1) * (float)(n + 1);
    const float sc = 4.f / inv_h2;
    const int lrow = 32 * (w & 3) + lane;  // this thread's TMEM lane = operand row (part p, index a)
    const int p = lrow >> 6, a = lrow & 63;
    const int col0 = 32 * (w >> 2);          // and its half of the accumulator columns
    uint32_t phase = 0;
    bool ok = true;
    for (int q = blockIdx.x; q < cnt && ok; q += gridDim.x) {
        const NtInst in = ins[q];
        const int j = ids[q];
        const float c = (float)shift[j];
        // the first operand in natural order: rows (part, i), column k.  Warp w
        // takes the band of rows 8 w .. 8 w + 7, lanes = columns k and k + 32;
        // the band's rows (with a halo row on each side), u and r are loaded
        // before any is used, and the left / right neighbours come from the
        // adjacent lanes.
        const bool stencil = mode == NPBS_RESIDUAL || mode == NPBS_OP_B;
        const bool with_r = mode == NPBS_RESIDUAL && r != nullptr;
        {
            const int i0 = 8 * w;
            float2 X[10][2];
            float U[8][2];
            float2 R[8][2];
#pragma unroll
            for (int rr = 0; rr < 10; ++rr) {
                const int i = i0 - 1 + rr;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    X[rr][h] = (i >= 0 && i < n && (stencil || (rr >= 1 && rr <= 8)))
                                   ? x[in.off + (long long)i * n + lane + 32 * h]
                                   : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int rr = 0; rr < 8; ++rr)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const long long e = in.off + (long long)(i0 + rr) * n + lane + 32 * h;
                    U[rr][h] = stencil ? u[e] : 0.f;
                    R[rr][h] = with_r ? r[e] : make_float2(0.f, 0.f);
                }
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                const int i = i0 + rr;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;
                    const float2 cc = X[rr + 1][h];
                    float2 v = cc;
                    if (stencil) {
                        // neighbours in the row: lanes +-1, across the two column halves at lanes 0 / 31
                        const float2 o0 = X[rr + 1][0], o1 = X[rr + 1][1];
                        float2 lf, rt;
                        const float2 up0 = make_float2(__shfl_up_sync(0xffffffffu, o0.x, 1), __shfl_up_sync(0xffffffffu, o0.y, 1));
                        const float2 up1 = make_float2(__shfl_up_sync(0xffffffffu, o1.x, 1), __shfl_up_sync(0xffffffffu, o1.y, 1));
                        const float2 dn0 = make_float2(__shfl_down_sync(0xffffffffu, o0.x, 1), __shfl_down_sync(0xffffffffu, o0.y, 1));
                        const float2 dn1 = make_float2(__shfl_down_sync(0xffffffffu, o1.x, 1), __shfl_down_sync(0xffffffffu, o1.y, 1));
                        const float2 l31 = make_float2(__shfl_sync(0xffffffffu, o0.x, 31), __shfl_sync(0xffffffffu, o0.y, 31));
                        const float2 r0 = make_float2(__shfl_sync(0xffffffffu, o1.x, 0), __shfl_sync(0xffffffffu, o1.y, 0));
                        if (h == 0) {
                            lf = lane == 0 ? make_float2(0.f, 0.f) : up0;
                            rt = lane == 31 ? r0 : dn0;
                        } else {
                            lf = lane == 0 ? l31 : up1;
                            rt = lane == 31 ? make_float2(0.f, 0.f) : dn1;
                        }
                        const float2 a1 = X[rr][h], a2 = X[rr + 2][h];
                        const float sx = 4.f * cc.x - a1.x - a2.x - lf.x - rt.x;
                        const float sy = 4.f * cc.y - a1.y - a2.y - lf.y - rt.y;
                        const float uv = U[rr][h];
                        v = make_float2(sx * inv_h2 - 2.f * uv * cc.x, sy * inv_h2 - 2.f * uv * cc.y);
                        if (mode == NPBS_RESIDUAL) v = make_float2(R[rr][h].x - v.x, R[rr][h].y - v.y);
                    }
                    put_split(Ah, Al, sw128_off(i, k, 128), v.x);
                    put_split(Ah, Al, sw128_off(n + i, k, 128), v.y);
                }
            }
        }
        for (int st = 0; st < 4; ++st) {
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            if (t == 0) {
                fence_after_sync();
                // a K sub-step moves the start address field (bytes / 16) of the base descriptors
#pragma unroll
                for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ao = (uint64_t)((kb * 16384 + kk * 32) >> 4);
                        const uint64_t bo = (uint64_t)((kb * 8192 + kk * 32) >> 4);
                        mma_tf32(tmem, dAl + ao, dSh + bo, idesc, (kb | kk) ? 1u : 0u);
                        mma_tf32(tmem, dAh + ao, dSl + bo, idesc, 1u);
                        mma_tf32(tmem, dAh + ao, dSh + bo, idesc, 1u);
                    }
                commit(su32(bar));
                if (!mbar_wait(su32(bar), phase, wait_limit)) {
                    atomicExch(&g_nt_tc_timeout, 1);
                    *okflag = 0;
                }
            }
            phase ^= 1;
            __syncthreads();
            if (!*okflag) {
                ok = false;
                break;
            }
            fence_after_sync();
            // this lane's 32 accumulator columns, 16 at a time
            const float ea = eig[a] + c;
#pragma unroll
            for (int cq = 0; cq < 2; ++cq) {
                const int cb = (col0 >> 4) + cq;
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(cb * 16), v);
                if (st == 1) {
                    // lane (p, j = a) holds (S q S)[i][a] over i: the Green symbol
#pragma unroll
                    for (int q2 = 0; q2 < 16; ++q2) v[q2] *= sc / (eig[cb * 16 + q2] + ea);
                }
                if (st < 3) {
#pragma unroll
                    for (int q2 = 0; q2 < 16; ++q2) put_split(Ah, Al, sw128_off(p * n + cb * 16 + q2, a, 128), v[q2]);
                } else {
                    // lane (p, j = a) holds (G q)[i][a] over i: stage it in natural order
                    float* Of = reinterpret_cast<float*>(O);
#pragma unroll
                    for (int q2 = 0; q2 < 16; ++q2) Of[2 * ((cb * 16 + q2) * n + a) + p] = v[q2];
                }
            }
        }
        if (!ok) break;
        fence_before_sync();
        __syncthreads();
        double acc = 0.0;
#pragma unroll 8
        for (int e = t; e < np; e += blockDim.x) {
            float2 vv = O[e];
            if (mode == NPBS_ADJ_B) {
                // J (G x): the stencil on the staged tile
                const int i = e >> 6, k = e & 63;
                float2 s = make_float2(4.f * vv.x, 4.f * vv.y);
                if (i > 0) { const float2 y = O[e - n]; s.x -= y.x; s.y -= y.y; }
                if (i < n - 1) { const float2 y = O[e + n]; s.x -= y.x; s.y -= y.y; }
                if (k > 0) { const float2 y = O[e - 1]; s.x -= y.x; s.y -= y.y; }
                if (k < n - 1) { const float2 y = O[e + 1]; s.x -= y.x; s.y -= y.y; }
                const float uv = u[in.off + e];
                vv = make_float2(s.x * inv_h2 - 2.f * uv * vv.x, s.y * inv_h2 - 2.f * uv * vv.y);
            }
            out[in.off + e] = vv;
            acc += (double)vv.x * vv.x + (double)vv.y * vv.y;
        }
        if (norm2) {
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) red[w] = acc;
            __syncthreads();
            if (t == 0) {
                double tot = 0.0;
                for (int q2 = 0; q2 < kNtTcThreads / 32; ++q2) tot += red[q2];
                atomicAdd(norm2 + j, tot);
            }
        }
        __syncthreads();  // the staging tile is the next instance's operand
    }
    if (!ok && t == 0) {
        // a wait gave up: give the MMAs in flight one more bounded wait before TMEM is released
        (void)mbar_wait(su32(bar), phase ^ 1, wait_limit);
    }
    fence_before_sync();
    __syncthreads();
    if (w == 0) tmem_dealloc(tmem, 64);
}

}  // namespace
}  // namespace npbs

namespace npbs {
namespace {

struct NtGroup {
    int n = 0, cnt = 0;
    const NtInst* ins = nullptr;  // device [cnt]
    const int* ids = nullptr;     // device [cnt]: batch index of each
    const float* tab = nullptr;   // device: sine matrix [n][n], 1D eigenvalues [n]
};

struct NtPrep {
    std::vector<NtGroup> groups;
    long long extent = 0;
    int tc_ctas = 0;             // CTAs of the tensor-core apply (two per SM)
    long long wait_limit = 0;    // its bounded waits, in clock cycles (about two seconds)
};

// The tensor-core apply serves side-64 groups unless NPBS_NEWTON_TC=0 (read
// at each apply, so that the two kernels can be compared in one process).
bool nt_tc_enabled() {
    const char* e = getenv("NPBS_NEWTON_TC");
    return !(e && e[0] == '0');
}

size_t nt_smem(int n) { return sizeof(float) * ((size_t)n * n + ((n + 3) & ~3)) + 2 * sizeof(float2) * (size_t)n * n; }

// The last prepared batch: its exact description and the prepared plan, whose
// device tables stay in work[18].
struct NtCached {
    std::vector<char> desc;
    NtPrep P;
};

npbs_status nt_prepare(npbs_ctx* ctx, const npbs_batch* batch, NtPrep* P, cudaStream_t st) {
    if (!batch || batch->count < 0 || (batch->count > 0 && !batch->inst))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton: NULL batch");
    // a batch identical to the last one prepared reuses its tables: no upload, no synchronisation
    std::vector<char> desc(sizeof(int) + (size_t)batch->count * sizeof(npbs_instance));
    memcpy(desc.data(), &batch->count, sizeof(int));
    if (batch->count > 0) memcpy(desc.data() + sizeof(int), batch->inst, sizeof(npbs_instance) * batch->count);
    if (ctx->nt_prep) {
        const NtCached* c = static_cast<const NtCached*>(ctx->nt_prep.get());
        if (c->desc == desc) {
            *P = c->P;
            return NPBS_OK;
        }
    }
    std::map<int, std::vector<int>> by;
    long long ext = 0;
    for (int j = 0; j < batch->count; ++j) {
        const npbs_instance& s = batch->inst[j];
        if (s.nx != s.ny || s.nx % 4 != 0 || s.nx < 8 || s.nx > kNtMaxN) {
            char buf[160];
            snprintf(buf, sizeof buf, "newton: instance %d is %d x %d; need square grids, side a multiple of 4 in 8..%d",
                     j, s.ny, s.nx, kNtMaxN);
            return set_err(ctx, NPBS_ERR_UNSUPPORTED_SIZE, buf);
        }
        if (s.offset < 0 || s.offset % 32 != 0)
            return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton: need offsets >= 0, multiples of 32");
        by[s.nx].push_back(j);
        ext = std::max<long long>(ext, s.offset + (long long)s.nx * s.ny);
    }
    P->extent = ext;
    P->groups.clear();
    std::vector<char> host;
    auto put = [&](const void* src, size_t bytes) {
        const size_t o = (host.size() + 255) & ~size_t(255);
        host.resize(o + bytes);
        memcpy(host.data() + o, src, bytes);
        return o;
    };
    struct Offs { size_t ins, ids, tab; };
    std::vector<Offs> offs;
    for (auto& kv : by) {
        const int n = kv.first;
        NtGroup g;
        g.n = n;
        g.cnt = (int)kv.second.size();
        std::vector<float> tab((size_t)n * n + n);
        const double h = 1.0 / (n + 1);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                // sin(pi (a+1)(b+1)/(n+1)) with the integer argument reduced mod 2(n+1)
                const long long m = ((long long)(a + 1) * (b + 1)) % (2LL * (n + 1));
                tab[(size_t)a * n + b] = (float)std::sin(M_PI * (double)m / (double)(n + 1));
            }
        for (int p = 0; p < n; ++p) {
            const double sp = std::sin(0.5 * M_PI * (double)(p + 1) * h);
            tab[(size_t)n * n + p] = (float)(4.0 / (h * h) * sp * sp);
        }
        std::vector<NtInst> ins;
        for (int j : kv.second) ins.push_back(NtInst{n, batch->inst[j].offset});
        Offs o;
        o.ins = put(ins.data(), sizeof(NtInst) * ins.size());
        o.ids = put(kv.second.data(), sizeof(int) * kv.second.size());
        o.tab = put(tab.data(), sizeof(float) * tab.size());
        offs.push_back(o);
        P->groups.push_back(g);
    }
    NPBS_CK(ctx, ctx->work[18].ensure(std::max<size_t>(host.size(), 256)));
    char* d = static_cast<char*>(ctx->work[18].p);
    NPBS_CK(ctx, cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    NPBS_CK(ctx, cudaStreamSynchronize(st));  // the staging vector goes out of scope
    for (size_t i = 0; i < P->groups.size(); ++i) {
        P->groups[i].ins = reinterpret_cast<const NtInst*>(d + offs[i].ins);
        P->groups[i].ids = reinterpret_cast<const int*>(d + offs[i].ids);
        P->groups[i].tab = reinterpret_cast<const float*>(d + offs[i].tab);
    }
    NPBS_CK(ctx, cudaFuncSetAttribute(k_nt_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)nt_smem(kNtMaxN)));
    NPBS_CK(ctx, cudaFuncSetAttribute(k_nt_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kNtTcBytes));
    {
        int dev = 0, sms = 0, khz = 0;
        NPBS_CK(ctx, cudaGetDevice(&dev));
        NPBS_CK(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NPBS_CK(ctx, cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
        P->tc_ctas = 2 * std::max(1, sms);
        P->wait_limit = 2LL * std::max(1, khz) * 1000;
    }
    auto cached = std::make_shared<NtCached>();
    cached->desc = std::move(desc);
    cached->P = *P;
    ctx->nt_prep = cached;
    return NPBS_OK;
}

// one fused float32 apply over the prepared batch (shift: DEVICE double [count])
npbs_status nt_run(npbs_ctx* ctx, const NtPrep& P, int mode, const double* shift, const float* u, const float2* r,
                   const float2* x, float2* out, double* norm2, int count, cudaStream_t st) {
    if (norm2) NPBS_CK(ctx, cudaMemsetAsync(norm2, 0, sizeof(double) * count, st));
    const bool tc = mode != NPBS_TRUE_RESIDUAL && nt_tc_enabled();
    for (const NtGroup& g : P.groups) {
        if (tc && g.n == kNtTcN)
            k_nt_apply_tc<<<std::min(g.cnt, P.tc_ctas), kNtTcThreads, kNtTcBytes, st>>>(g.ins, g.ids, g.cnt, g.tab, shift, u,
                                                                             r, x, out, norm2, mode, P.wait_limit);
        else
            k_nt_apply<<<g.cnt, 256, nt_smem(g.n), st>>>(g.ins, g.ids, g.tab, shift, u, r, x, out, norm2, mode);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(st, 1);
    }
    return NPBS_OK;
}

// a context plan over the batch for the network (its k0sq / eps are placeholders)
const Plan* nt_net_plan(npbs_ctx* ctx, const npbs_batch* batch, npbs_status* st) {
    std::vector<npbs_instance> tmp(batch->inst, batch->inst + batch->count);
    for (auto& t : tmp) {
        t.k0sq = 0.0;
        t.eps = 1.0;
        if (!(t.h > 0.0)) t.h = 1.0 / (t.nx + 1);
    }
    npbs_batch b2{batch->count, tmp.data()};
    return get_plan(ctx, &b2, st);
}

}  // namespace
}  // namespace npbs

namespace npbs {

// 1 once a bounded wait of the tensor-core apply gave up (synchronous read), and its reset
int newton_tc_timeout_flag() {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_nt_tc_timeout, sizeof(int));
    return v;
}
void newton_tc_clear_timeout() {
    const int z = 0;
    cudaMemcpyToSymbol(g_nt_tc_timeout, &z, sizeof(int));
}

}  // namespace npbs

using namespace npbs;

extern "C" {

npbs_status newton_apply(npbs_ctx* ctx, const npbs_batch* batch, const double* shift, const float* u, const void* r,
                         const void* x, void* out, npbs_mode mode, double* norm2, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (mode != NPBS_RESIDUAL && mode != NPBS_OP_B && mode != NPBS_TRUE_RESIDUAL && mode != NPBS_ADJ_B)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_apply: mode must be RESIDUAL, OP_B, TRUE_RESIDUAL or ADJ_B");
    if (!batch || batch->count == 0) return batch ? NPBS_OK : NPBS_ERR_INVALID_ARG;
    if (!shift || !u || !x || !out || (mode == NPBS_RESIDUAL && !r))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_apply: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NtPrep P;
    npbs_status st = nt_prepare(ctx, batch, &P, s);
    if (st != NPBS_OK) return st;
    NPBS_CK(ctx, ctx->work[20].ensure(sizeof(double) * batch->count));
    double* dsh = static_cast<double*>(ctx->work[20].p);
    NPBS_CK(ctx, cudaMemcpyAsync(dsh, shift, sizeof(double) * batch->count, cudaMemcpyHostToDevice, s));
    return nt_run(ctx, P, (int)mode, dsh, u, static_cast<const float2*>(r), static_cast<const float2*>(x),
                  static_cast<float2*>(out), norm2, batch->count, s);
}

npbs_status newton_linearise(npbs_ctx* ctx, const npbs_batch* batch, const double* u, const double* f, double alpha,
                             double* shift_out, float* u32_out, void* r_out, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!batch || batch->count < 0) return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_linearise: NULL batch");
    const int cnt = batch->count;
    if (cnt == 0) return NPBS_OK;
    if (!u || !f || !shift_out || !u32_out || !r_out || !std::isfinite(alpha))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_linearise: NULL argument or non-finite alpha");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NtPrep P;
    npbs_status st = nt_prepare(ctx, batch, &P, s);
    if (st != NPBS_OK) return st;
    const size_t ext = (size_t)std::max<long long>(P.extent, 1);
    NPBS_CK(ctx, ctx->work[20].ensure(sizeof(double) * (ext + 5 * (size_t)cnt)));
    double* r64 = static_cast<double*>(ctx->work[20].p);
    double* dsh = r64 + ext;
    double* out4 = dsh + cnt;
    for (const NtGroup& g : P.groups) {
        k_nt_linearise<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, nullptr, u, f, alpha, r64, u32_out, dsh, out4);
        k_nt_to_c64<<<g.cnt, 256, 0, s>>>(g.ins, r64, static_cast<float2*>(r_out));
    }
    NPBS_CK(ctx, cudaGetLastError());
    ctx->count(s, 2LL * (long long)P.groups.size());
    NPBS_CK(ctx, cudaMemcpyAsync(shift_out, dsh, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaStreamSynchronize(s));
    return NPBS_OK;
}

npbs_status newton_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const double* f, double* u,
                         double alpha, const npbs_newton_opts* opts, npbs_newton_report* report,
                         npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!batch || batch->count < 0) return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_solve: NULL batch");
    const int cnt = batch->count;
    if (cnt == 0) return NPBS_OK;
    if (!f || !u || !opts) return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_solve: NULL argument");
    if (opts->direct_format && !net)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_solve: the Direct format needs a network");
    if (!(opts->tol >= 0.0) || opts->max_steps < 0 || !(opts->inner_rtol >= 0.0) || opts->inner_max_iter < 0 ||
        opts->check_every < 1 || !std::isfinite(alpha))
        return set_err(ctx, NPBS_ERR_INVALID_ARG,
                       "newton_solve: need tol, inner_rtol >= 0, max_steps, inner_max_iter >= 0, check_every >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NtPrep P;
    npbs_status st = nt_prepare(ctx, batch, &P, s);
    if (st != NPBS_OK) return st;
    const size_t ext = (size_t)std::max<long long>(P.extent, 1);
    // delta (double2), r (double), eps, rho32, rr (float2), u32 (float), shift, out4 (double), flags (int)
    const size_t bytes = ext * (16 + 8 + 3 * 8) + ((ext * 4 + 255) & ~size_t(255)) + sizeof(double) * 5 * cnt +
                         sizeof(int) * 4 * cnt + 1024;
    NPBS_CK(ctx, ctx->work[19].ensure(bytes));
    char* w = static_cast<char*>(ctx->work[19].p);
    double2* delta = reinterpret_cast<double2*>(w);
    double* r64 = reinterpret_cast<double*>(delta + ext);
    float2* eps = reinterpret_cast<float2*>(r64 + ext);
    float2* rho32 = eps + ext;
    float2* rr = rho32 + ext;
    float* u32 = reinterpret_cast<float*>(rr + ext);
    double* shift = reinterpret_cast<double*>(reinterpret_cast<char*>(u32) + ((ext * 4 + 255) & ~size_t(255)));
    double* out4 = shift + cnt;
    int* nfrozen = reinterpret_cast<int*>(out4 + 4 * cnt);
    int* ifrozen = nfrozen + cnt;
    int* active = ifrozen + cnt;
    int* itsd = active + cnt;
    NPBS_CK(ctx, cudaMemsetAsync(delta, 0, sizeof(double2) * ext, s));
    NPBS_CK(ctx, cudaMemsetAsync(out4, 0, sizeof(double) * 4 * cnt, s));
    const Net* N = reinterpret_cast<const Net*>(net);
    const Plan* pl = nullptr;
    std::vector<int> all(cnt);
    for (int j = 0; j < cnt; ++j) all[j] = j;
    if (N) {
        pl = nt_net_plan(ctx, batch, &st);
        if (!pl) return st;
    }
    std::vector<int> steps(cnt, 0), inner(cnt, 0), hn(cnt, 0), hi(cnt, 0), hact(cnt, 0), its(cnt, 0);
    std::vector<double> res(cnt, 1.0), h4(4 * (size_t)cnt);
    std::vector<npbs_status> stat(cnt, NPBS_NOT_CONVERGED);
    auto upload = [&](int* dst, const std::vector<int>& v) -> npbs_status {
        NPBS_CK(ctx, cudaMemcpyAsync(dst, v.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        return NPBS_OK;
    };
    auto read4 = [&]() -> npbs_status {
        NPBS_CK(ctx, cudaMemcpyAsync(h4.data(), out4, sizeof(double) * 4 * cnt, cudaMemcpyDeviceToHost, s));
        NPBS_CK(ctx, cudaStreamSynchronize(s));
        return NPBS_OK;
    };
    for (int m = 0;; ++m) {
        if ((st = upload(nfrozen, hn)) != NPBS_OK) return st;
        for (const NtGroup& g : P.groups)
            k_nt_linearise<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, nfrozen, u, f, alpha, r64, u32, shift, out4);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(s, (long long)P.groups.size());
        if ((st = read4()) != NPBS_OK) return st;
        bool any = false;
        for (int j = 0; j < cnt; ++j) {
            if (hn[j]) continue;
            res[j] = std::sqrt(h4[4 * j] / std::max(h4[4 * j + 1], 1e-300));
            steps[j] = m;
            if (!std::isfinite(res[j])) stat[j] = NPBS_ERR_NONFINITE;
            else if (res[j] <= opts->tol) stat[j] = NPBS_OK;
            else if (m >= opts->max_steps) stat[j] = NPBS_NOT_CONVERGED;
            else {
                any = true;
                continue;
            }
            hn[j] = 1;
        }
        if (!any) break;
        NetRun run;
        if (N) {
            // the coefficient channel is this step's linearisation point
            st = net_prepare(ctx, *N, *pl, all, false, &run, s, u32);
            if (st != NPBS_OK) return st;
        }
        // the inner solve of J delta = r on the instances still iterating
        NPBS_CK(ctx, cudaMemsetAsync(eps, 0, sizeof(float2) * ext, s));
        hi = hn;
        for (int j = 0; j < cnt; ++j) its[j] = 0;
        int it = 0;
        auto check = [&]() -> npbs_status {
            npbs_status s2 = upload(ifrozen, hi);
            if (s2 != NPBS_OK) return s2;
            for (const NtGroup& g : P.groups)
                k_nt_check<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, ifrozen, u, r64, eps, delta, rho32, out4, nullptr,
                                                 0.0, 0, 0);
            NPBS_CK(ctx, cudaGetLastError());
            ctx->count(s, (long long)P.groups.size());
            if ((s2 = read4()) != NPBS_OK) return s2;
            for (int j = 0; j < cnt; ++j) {
                if (hi[j]) continue;
                const double irt = std::sqrt(h4[4 * j + 2] / std::max(h4[4 * j], 1e-300));
                its[j] = it;
                if (!std::isfinite(irt) || irt <= opts->inner_rtol || it >= opts->inner_max_iter) hi[j] = 1;
            }
            return upload(ifrozen, hi);
        };
        if (!N) {
            // Born inner solves: the check freezes each instance on the device at
            // its first passing check, so the host reads the flags only every
            // kNtSyncChecks checks (iterations on frozen instances after that are
            // never folded in, and the update skips them)
            constexpr int kNtSyncChecks = 4;
            const double rtol2 = opts->inner_rtol * opts->inner_rtol;
            if ((st = upload(ifrozen, hi)) != NPBS_OK) return st;
            auto check_dev = [&]() -> npbs_status {
                for (const NtGroup& g : P.groups)
                    k_nt_check<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, ifrozen, u, r64, eps, delta, rho32, out4, itsd,
                                                     rtol2, it, opts->inner_max_iter);
                NPBS_CK(ctx, cudaGetLastError());
                ctx->count(s, (long long)P.groups.size());
                return NPBS_OK;
            };
            if ((st = check_dev()) != NPBS_OK) return st;
            for (;;) {
                NPBS_CK(ctx, cudaMemcpyAsync(hi.data(), ifrozen, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
                NPBS_CK(ctx, cudaStreamSynchronize(s));
                bool busy = false;
                for (int j = 0; j < cnt; ++j) busy |= !hi[j];
                if (!busy) break;
                for (int sc = 0; sc < kNtSyncChecks; ++sc) {
                    for (int k = 0; k < opts->check_every && it < opts->inner_max_iter; ++k, ++it) {
                        st = nt_run(ctx, P, NPBS_RESIDUAL, shift, u32, rho32, eps, rr, nullptr, cnt, s);
                        if (st != NPBS_OK) return st;
                        for (const NtGroup& g : P.groups)
                            k_nt_axpy<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, ifrozen, rr, eps);
                        NPBS_CK(ctx, cudaGetLastError());
                        ctx->count(s, (long long)P.groups.size());
                    }
                    if ((st = check_dev()) != NPBS_OK) return st;
                }
            }
            std::vector<int> hits(cnt);
            NPBS_CK(ctx, cudaMemcpyAsync(hits.data(), itsd, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
            NPBS_CK(ctx, cudaStreamSynchronize(s));
            for (int j = 0; j < cnt; ++j)
                if (!hn[j]) its[j] = hits[j];
        }
        if (N && (st = check()) != NPBS_OK) return st;
        for (; N;) {
            bool busy = false;
            for (int j = 0; j < cnt; ++j) busy |= !hi[j];
            if (!busy) break;
            for (int k = 0; k < opts->check_every && it < opts->inner_max_iter; ++k, ++it) {
                // the network input: G(rho - J eps), or rho - J eps in the Direct format
                st = nt_run(ctx, P, opts->direct_format ? NPBS_TRUE_RESIDUAL : NPBS_RESIDUAL, shift, u32, rho32, eps,
                            rr, nullptr, cnt, s);
                if (st != NPBS_OK) return st;
                if (N) {
                    st = net_run_forward(ctx, *N, run, rr, u32, eps, 1, s);
                    if (st != NPBS_OK) return st;
                } else {
                    for (const NtGroup& g : P.groups) k_nt_axpy<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, ifrozen, rr, eps);
                    NPBS_CK(ctx, cudaGetLastError());
                    ctx->count(s, (long long)P.groups.size());
                }
            }
            if ((st = check()) != NPBS_OK) return st;
        }
        for (int j = 0; j < cnt; ++j) {
            hact[j] = !hn[j];
            if (hact[j]) inner[j] += its[j];
        }
        if ((st = upload(active, hact)) != NPBS_OK) return st;
        for (const NtGroup& g : P.groups) k_nt_update<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, active, u, delta);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(s, (long long)P.groups.size());
    }
    npbs_status ret = NPBS_OK;
    for (int j = 0; j < cnt; ++j) {
        if (report) {
            if (report->steps) report->steps[j] = steps[j];
            if (report->inner_iters) report->inner_iters[j] = inner[j];
            if (report->residual) report->residual[j] = res[j];
            if (report->status) report->status[j] = stat[j];
        }
        if (stat[j] == NPBS_ERR_NONFINITE) ret = NPBS_ERR_NONFINITE;
        else if (stat[j] != NPBS_OK && ret == NPBS_OK) ret = NPBS_NOT_CONVERGED;
    }
    return ret;
}

npbs_status newton_train_step_loss(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const double* shift,
                                   const float* u, const void* r, const void* d_snap, int32_t unroll,
                                   npbs_loss kind, float lr, float weight_decay, float* loss_host,
                                   npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!net || !batch || !shift || !u || !r || !d_snap || !loss_host)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_train_step: NULL argument");
    if (kind != NPBS_LOSS_BS_RETA && kind != NPBS_LOSS_BS_L2 && kind != NPBS_LOSS_DIR)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_train_step: unknown loss");
    if (unroll < 1 || unroll > 16 || !(lr >= 0.f) || !(weight_decay >= 0.f))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "newton_train_step: need 1 <= unroll <= 16, lr >= 0, weight_decay >= 0");
    *loss_host = 0.f;
    const int cnt = batch->count;
    if (cnt <= 0) return cnt == 0 ? NPBS_OK : NPBS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NtPrep P;
    npbs_status st = nt_prepare(ctx, batch, &P, s);
    if (st != NPBS_OK) return st;
    NPBS_CK(ctx, ctx->work[20].ensure(sizeof(double) * cnt));
    double* dsh = static_cast<double*>(ctx->work[20].p);
    NPBS_CK(ctx, cudaMemcpyAsync(dsh, shift, sizeof(double) * cnt, cudaMemcpyHostToDevice, s));
    const Plan* pl = nt_net_plan(ctx, batch, &st);
    if (!pl) return st;
    const float2* R = static_cast<const float2*>(r);
    const float2* D = static_cast<const float2*>(d_snap);
    Net& Nn = *reinterpret_cast<Net*>(net);
    if (kind != NPBS_LOSS_BS_RETA) {
        // J and G are real symmetric: J^* = J, G^* = G
        EuclidOps op;
        op.minus_a = [&](const float2* x, const float2* f_in, float2* out, double* norm2) -> npbs_status {
            return nt_run(ctx, P, NPBS_TRUE_RESIDUAL, dsh, u, f_in, x, out, norm2, cnt, s);
        };
        op.minus_a_adj = [&](const float2* y, float2* out) -> npbs_status {
            return nt_run(ctx, P, NPBS_TRUE_RESIDUAL, dsh, u, nullptr, y, out, nullptr, cnt, s);
        };
        op.green = [&](const float2* x, float2* out) -> npbs_status {
            return nt_run(ctx, P, kNtGreen, dsh, u, nullptr, x, out, nullptr, cnt, s);
        };
        op.green_adj = op.green;
        return train_step_euclid(ctx, Nn, pl, u, R, D, unroll, kind == NPBS_LOSS_BS_L2, lr, weight_decay, loss_host,
                                 s, op);
    }
    BornOp op = [&](int mode, const float2* x, float2* out, double* norm2) -> npbs_status {
        return nt_run(ctx, P, mode, dsh, u, R, mode == NPBS_RESIDUAL ? D : x, out, norm2, cnt, s);
    };
    return train_step_reta(ctx, Nn, pl, u, unroll, lr, weight_decay, loss_host, s, op);
}

}  // extern "C"
