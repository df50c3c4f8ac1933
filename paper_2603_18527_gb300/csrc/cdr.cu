// Convection-diffusion-reaction operators (App. Full Derivations, CDR; Eqs.
// cdr_pde, cdr_L0, cdr_V, cdr_integral, cdr_identity, cdr_G_symbol) and their
// Born / NPBS iteration on the GPU:
//
//   A u  = -div(kappa grad u) + v . grad u + sigma u
//   L0   = -kappa0 Lap + v0 . grad + sigma0,  G = L0^{-1} (symbol 1 / lambda0,
//          lambda0 = kappa0 |xi|^2 + i v0 . xi + sigma0)
//   V    = L0 - A,  I - G V = G A  (so G(V x + f) - x = G(f - A x))
//
// On the same periodic pseudospectral grid as the Helmholtz operators (first
// derivatives by i xi on the mode set n in -N/2..N/2-1).  One apply:
//   b0 = F x;  b1, b2 = F^{-1}(i xi_x b0), F^{-1}(i xi_y b0)        (grad x)
//   b3, b4 = F(kappa grad x),  b5 = F(v . grad x + sigma x [- f])
//   W = -i xi_x b3 - i xi_y b4 + b5 = F(A x [- f])
//   RESIDUAL: F^{-1}(-W / lambda0) = G(f - A x);  OP_B: F^{-1}(W / lambda0) = G A x;
//   TRUE_RESIDUAL: F^{-1}(-W) = f - A x
// and the adjoint ADJ_B: (G A)^* y = A^* G^* y with G^* of symbol 1/conj(lambda0)
// and A^* g = -div(kappa grad g + v g) + sigma g.  Seven (eight) batched 2D
// FFTs of the instances' square grids (fft2d.cuh) and four pointwise kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "ctx.cuh"
#include "dftreg.cuh"
#include "fft2d.cuh"
#include "net.cuh"

namespace npbs {
namespace {

struct CdrInst {
    int n;
    double h;
    long long off;
    double k0, v0x, v0y, s0;
};

template <typename R> __device__ __forceinline__ R xi_of(int i, int n, double h) {
    return (R)(6.283185307179586476925 * (double)signed_mode(i, n) / ((double)n * h));
}

__device__ __forceinline__ void field_point(const CdrInst* ins, long long np, long long g, int* j, long long* p) {
    *j = (int)(g / np);
    *p = g - (long long)(*j) * np;
}

// The kernels below run in float32 (R = float: the complex64 iteration) or in
// float64 (R = double: the stopping residual f - A u of a complex128 iterate).
// Coefficient fields are float32 and the source complex64 in both.

// b0 = x (then transformed in place)
template <typename R>
__global__ void k_cdr_copy(const CdrInst* ins, int cnt, long long np, const cpx<R>* x, cpx<R>* b0) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        const long long o = ins[j].off + p;
        b0[o] = x[o];
    }
}

// spectral gradients b1 = i xi_x b0, b2 = i xi_y b0 (adj == 1: b0 /= conj(lambda0) first, G^*)
template <typename R>
__global__ void k_cdr_grad(const CdrInst* ins, int cnt, long long np, cpx<R>* b0, cpx<R>* b1, cpx<R>* b2, int adj) {
    using C = cpx<R>;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        const CdrInst in = ins[j];
        const int y = (int)(p / in.n), x = (int)(p % in.n);
        const R kx = xi_of<R>(x, in.n, in.h), ky = xi_of<R>(y, in.n, in.h);
        const long long o = in.off + p;
        C u = b0[o];
        if (adj == 1) {
            // G^*: divide by conj(lambda0) = kappa0 |xi|^2 + sigma0 - i v0 . xi
            const R lr = (R)in.k0 * (kx * kx + ky * ky) + (R)in.s0;
            const R li = -((R)in.v0x * kx + (R)in.v0y * ky);
            const R d = (R)1 / (lr * lr + li * li);
            u = mk<C>((u.x * lr + u.y * li) * d, (u.y * lr - u.x * li) * d);
            b0[o] = u;
        }
        b1[o] = mk<C>(-kx * u.y, kx * u.x);
        b2[o] = mk<C>(-ky * u.y, ky * u.x);
    }
}

// pointwise products in physical space (s = 1/n^2 undoes the unnormalised transforms)
//   forward:  b3 = kappa ux, b4 = kappa uy, b5 = vx ux + vy uy + sigma x - f
//   adjoint:  g = b0 s: b3 = kappa gx + vx g, b4 = kappa gy + vy g, b5 = sigma g
template <typename R>
__global__ void k_cdr_flux(const CdrInst* ins, int cnt, long long np, const float* kappa, const float* vx,
                           const float* vy, const float* sigma, const cpx<R>* x, const float2* f, const cpx<R>* b0,
                           const cpx<R>* b1, const cpx<R>* b2, cpx<R>* b3, cpx<R>* b4, cpx<R>* b5, int adj) {
    using C = cpx<R>;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        const CdrInst in = ins[j];
        const long long o = in.off + p;
        const R s = (R)1 / ((R)in.n * (R)in.n);
        const R k = kappa[o], ax = vx[o], ay = vy[o], sg = sigma[o];
        const C ux = mk<C>(b1[o].x * s, b1[o].y * s), uy = mk<C>(b2[o].x * s, b2[o].y * s);
        if (!adj) {
            const C xv = x[o];
            C r = mk<C>(ax * ux.x + ay * uy.x + sg * xv.x, ax * ux.y + ay * uy.y + sg * xv.y);
            if (f) r = mk<C>(r.x - (R)f[o].x, r.y - (R)f[o].y);
            b3[o] = mk<C>(k * ux.x, k * ux.y);
            b4[o] = mk<C>(k * uy.x, k * uy.y);
            b5[o] = r;
        } else {
            const C gv = mk<C>(b0[o].x * s, b0[o].y * s);
            b3[o] = mk<C>(k * ux.x + ax * gv.x, k * ux.y + ax * gv.y);
            b4[o] = mk<C>(k * uy.x + ay * gv.x, k * uy.y + ay * gv.y);
            b5[o] = mk<C>(sg * gv.x, sg * gv.y);
        }
    }
}

// W = -i xi_x b3 - i xi_y b4 + b5; b0 = mode-dependent multiple of W
//   kind 0 (RESIDUAL): -W / lambda0, 1 (OP_B): W / lambda0, 2 (TRUE_RESIDUAL): -W, 3 (ADJ_B): W
template <typename R>
__global__ void k_cdr_assemble(const CdrInst* ins, int cnt, long long np, const cpx<R>* b3, const cpx<R>* b4,
                               const cpx<R>* b5, cpx<R>* b0, int kind) {
    using C = cpx<R>;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        const CdrInst in = ins[j];
        const int y = (int)(p / in.n), x = (int)(p % in.n);
        const R kx = xi_of<R>(x, in.n, in.h), ky = xi_of<R>(y, in.n, in.h);
        const long long o = in.off + p;
        const C a = b3[o], b = b4[o], c = b5[o];
        // -i xi (a) = (xi a.y, -xi a.x)
        C w = mk<C>(kx * a.y + ky * b.y + c.x, -kx * a.x - ky * b.x + c.y);
        if (kind == 0 || kind == 2) w = mk<C>(-w.x, -w.y);
        if (kind == 0 || kind == 1) {
            const R lr = (R)in.k0 * (kx * kx + ky * ky) + (R)in.s0;
            const R li = (R)in.v0x * kx + (R)in.v0y * ky;
            const R d = (R)1 / (lr * lr + li * li);
            w = mk<C>((w.x * lr + w.y * li) * d, (w.y * lr - w.x * li) * d);
        }
        b0[o] = w;
    }
}

// b0 /= lambda0 (G) or conj(lambda0) (G^*)
template <typename R>
__global__ void k_cdr_green(const CdrInst* ins, int cnt, long long np, cpx<R>* b0, int adj) {
    using C = cpx<R>;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        const CdrInst in = ins[j];
        const int y = (int)(p / in.n), x = (int)(p % in.n);
        const R kx = xi_of<R>(x, in.n, in.h), ky = xi_of<R>(y, in.n, in.h);
        const long long o = in.off + p;
        const R lr = (R)in.k0 * (kx * kx + ky * ky) + (R)in.s0;
        const R li = (adj ? (R)-1 : (R)1) * ((R)in.v0x * kx + (R)in.v0y * ky);
        const R d = (R)1 / (lr * lr + li * li);
        const C w = b0[o];
        b0[o] = mk<C>((w.x * lr + w.y * li) * d, (w.y * lr - w.x * li) * d);
    }
}

// out = b0 / n^2 (rounded to complex64), norm2[j] += ||b0 / n^2||^2 (R per
// thread, float64 across threads)
template <typename R>
__global__ void k_cdr_out(const CdrInst* ins, int cnt, long long np, const cpx<R>* b0, float2* out, const int* ids,
                          double* norm2) {
    __shared__ double red[8];
    const long long tot = cnt * np;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < tot; base += (long long)gridDim.x * blockDim.x) {
        const long long g = base + threadIdx.x;
        R acc = 0;
        int j = (int)(base / np);
        if (g < tot) {
            long long p;
            field_point(ins, np, g, &j, &p);
            const CdrInst in = ins[j];
            const R s = (R)1 / ((R)in.n * (R)in.n);
            const long long o = in.off + p;
            const R vr = b0[o].x * s, vi = b0[o].y * s;
            out[o] = make_float2((float)vr, (float)vi);
            acc = vr * vr + vi * vi;
        }
        if (norm2) {
            // a block of 256 points never straddles two instances (np is a multiple of 256)
            double a = acc;
            for (int w = 16; w > 0; w >>= 1) a += __shfl_xor_sync(0xffffffffu, a, w);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
            __syncthreads();
            if (threadIdx.x == 0 && base < tot) {
                double t = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
                atomicAdd(norm2 + ids[j], t);
            }
            __syncthreads();
        }
    }
}

// norm2[j] += ||f_j||^2 (float64)
__global__ void k_cdr_norm2(const CdrInst* ins, int cnt, long long np, const float2* f, const int* ids,
                            double* norm2) {
    __shared__ double red[8];
    const long long tot = cnt * np;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < tot; base += (long long)gridDim.x * blockDim.x) {
        const long long g = base + threadIdx.x;
        double acc = 0;
        int j = (int)(base / np);
        if (g < tot) {
            long long p;
            field_point(ins, np, g, &j, &p);
            const float2 v = f[ins[j].off + p];
            acc = (double)v.x * v.x + (double)v.y * v.y;
        }
        for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0 && base < tot) {
            double t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            atomicAdd(norm2 + ids[j], t);
        }
        __syncthreads();
    }
}

// u += delta, delta = 0 (the float32 correction folded into the complex128
// iterate) on the instances not yet frozen (frozen: by batch index)
__global__ void k_cdr_fold(const CdrInst* ins, const int* ids, const int* frozen, int cnt, long long np, float2* delta,
                           double2* u) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        if (frozen[ids[j]]) continue;
        const long long o = ins[j].off + p;
        const float2 d = delta[o];
        u[o] = make_double2(u[o].x + (double)d.x, u[o].y + (double)d.y);
        delta[o] = make_float2(0.f, 0.f);
    }
}

// ---- the fused float32 apply: five launches per grid side -----------------
// K1 rows:  x -> F_x x                                        (b0)
// K2 cols:  F_y -> X; [adjoint: X /= conj(lambda0)]; i xi_x X, i xi_y X [, X]
//           -> F_y^{-1}                                       (b1, b2 [, b0])
// K3 rows:  F_x^{-1} of those fields; the flux of k_cdr_flux; F_x of the
//           three flux fields                                 (b3, b4, b5)
// K4 cols:  F_y of the three; W = -i xi_x b3 - i xi_y b4 + b5, the mode's
//           multiple of W; F_y^{-1}                           (b0)
// K5 rows:  F_x^{-1}, out = b0 / n^2 and ||out||^2
// The same arithmetic as the unfused kernels, with the pointwise steps done
// inside the transform kernels (about 160 B/point moved instead of 380).
// complex elements per tile buffer (24 KB); two per block, so four blocks of
// 256 threads fit an SM (latency of the shared-memory passes needs the warps)
constexpr int kFTile = 3072;

__device__ __forceinline__ float2 cdr_lambda(const CdrInst& in, float kx, float ky, bool conj) {
    return make_float2((float)in.k0 * (kx * kx + ky * ky) + (float)in.s0,
                       (conj ? -1.f : 1.f) * ((float)in.v0x * kx + (float)in.v0y * ky));
}
__device__ __forceinline__ float2 cdiv(float2 w, float2 l) {
    const float d = 1.f / (l.x * l.x + l.y * l.y);
    return make_float2((w.x * l.x + w.y * l.y) * d, (w.y * l.x - w.x * l.y) * d);
}

// A tile transform: compile-time geometry when N > 0, else the run-time plan.
template <int N, int NB, int SI, int SB, int DIR, bool COLS>
__device__ __forceinline__ float2* tile_fft(float2* a, float2* b, const RadixPlan& plan, int nb, int si, int sb,
                                            const float2* tw) {
    if constexpr (N > 0) return fft_tile_ct<float2, DIR, COLS, N, NB, SI, SB>(a, b, tw, threadIdx.x, blockDim.x);
    else return fft_tile<float2, DIR, COLS>(a, b, plan, nb, si, sb, tw, threadIdx.x, blockDim.x);
}

// The kernels take the grid side N, rows per row block RB, columns per column
// block CB and the number F of gradient fields as template constants (N = 0:
// run-time n, rb, cb; F is always a template constant).

// K1: rb rows of one instance per block: b0 rows = F_x(x rows)
template <int N, int RB>
__global__ void __launch_bounds__(256) k_cdrf_rows_fwd(const CdrInst* ins, int n_, int rb_, RadixPlan plan,
                                                       const float2* tw, const float2* x, float2* b0) {
    extern __shared__ __align__(16) float2 sm[];
    const int n = N ? N : n_, rb = N ? RB : rb_;
    const int nbk = n / rb;
    const CdrInst in = ins[blockIdx.x / nbk];
    const long long base = in.off + (long long)(blockIdx.x % nbk) * rb * n;
    const int cnt = rb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) sm[e] = x[base + e];
    __syncthreads();
    float2* res = tile_fft<N, RB, 1, N, -1, false>(sm, sm + kFTile, plan, rb, 1, n, tw);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) b0[base + e] = res[e];
}

// K2: cb columns of one instance per block.  F fields out: forward 2 (gx, gy),
// adjoint 3 (gx, gy, g), adj == 1 dividing by conj(lambda0) first (G^*).
// Tile layout [row i][field f * cb + column b].
template <int N, int CB, int F>
__global__ void __launch_bounds__(256) k_cdrf_cols_grad(const CdrInst* ins, int n_, int cb_, RadixPlan plan,
                                                        const float2* tw, float2* b0, float2* b1, float2* b2,
                                                        int adj) {
    extern __shared__ __align__(16) float2 sm[];
    const int n = N ? N : n_, cb = N ? CB : cb_;
    const int nbk = n / cb;
    const CdrInst in = ins[blockIdx.x / nbk];
    const int c0 = (blockIdx.x % nbk) * cb;
    const long long base = in.off + c0;
    const int cnt = cb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        sm[e] = b0[base + (long long)i * n + b];
    }
    __syncthreads();
    float2* X = tile_fft<N, CB, CB, 1, -1, true>(sm, sm + kFTile, plan, cb, cb, 1, tw);
    // spread into F fields in the other buffer (X is in sm or sm + kFTile)
    float2* T = X == sm ? sm + kFTile : sm;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        const float kx = xi_of<float>(c0 + b, n, in.h), ky = xi_of<float>(i, n, in.h);
        float2 u = X[e];
        if (adj == 1) u = cdiv(u, cdr_lambda(in, kx, ky, true));
        float2* row = T + (long long)i * F * cb;
        row[b] = make_float2(-kx * u.y, kx * u.x);
        row[cb + b] = make_float2(-ky * u.y, ky * u.x);
        if (F == 3) row[2 * cb + b] = u;
    }
    __syncthreads();
    // the buffer X occupied is the scratch of the inverse
    float2* res = tile_fft<N, F * CB, F * CB, 1, 1, true>(T, X, plan, F * cb, F * cb, 1, tw);
    for (int e = threadIdx.x; e < F * cnt; e += blockDim.x) {
        const int i = e / (F * cb), r = e - i * (F * cb), f = r / cb, b = r - f * cb;
        float2* o = f == 0 ? b1 : f == 1 ? b2 : b0;
        o[base + (long long)i * n + b] = res[e];
    }
}

// K3: rb rows per block: F_x^{-1} of the F gradient fields, the flux, F_x of
// the three flux fields.  Tile layout [field][row][n].
template <int N, int RB, int F>
__global__ void __launch_bounds__(256) k_cdrf_rows_flux(const CdrInst* ins, int n_, int rb_, RadixPlan plan,
                                                        const float2* tw, const float* kappa, const float* vx,
                                                        const float* vy, const float* sigma, const float2* x,
                                                        const float2* f, float2* b0, float2* b1, float2* b2,
                                                        float2* b3, float2* b4, float2* b5) {
    extern __shared__ __align__(16) float2 sm[];
    const int n = N ? N : n_, rb = N ? RB : rb_;
    const int nbk = n / rb;
    const CdrInst in = ins[blockIdx.x / nbk];
    const long long base = in.off + (long long)(blockIdx.x % nbk) * rb * n;
    const int cnt = rb * n;
    for (int e = threadIdx.x; e < F * cnt; e += blockDim.x) {
        const int fld = e / cnt, p = e - fld * cnt;
        const float2* src = fld == 0 ? b1 : fld == 1 ? b2 : b0;
        sm[e] = src[base + p];
    }
    __syncthreads();
    float2* G = tile_fft<N, F * RB, 1, N, 1, false>(sm, sm + kFTile, plan, F * rb, 1, n, tw);
    float2* T = G == sm ? sm + kFTile : sm;
    const float s = 1.f / ((float)n * (float)n);
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        const long long o = base + p;
        const float k = kappa[o], ax = vx[o], ay = vy[o], sg = sigma[o];
        const float2 ux = make_float2(G[p].x * s, G[p].y * s), uy = make_float2(G[cnt + p].x * s, G[cnt + p].y * s);
        if (F == 2) {
            const float2 xv = x[o];
            float2 r = make_float2(ax * ux.x + ay * uy.x + sg * xv.x, ax * ux.y + ay * uy.y + sg * xv.y);
            if (f) r = make_float2(r.x - f[o].x, r.y - f[o].y);
            T[p] = make_float2(k * ux.x, k * ux.y);
            T[cnt + p] = make_float2(k * uy.x, k * uy.y);
            T[2 * cnt + p] = r;
        } else {
            const float2 gv = make_float2(G[2 * cnt + p].x * s, G[2 * cnt + p].y * s);
            T[p] = make_float2(k * ux.x + ax * gv.x, k * ux.y + ax * gv.y);
            T[cnt + p] = make_float2(k * uy.x + ay * gv.x, k * uy.y + ay * gv.y);
            T[2 * cnt + p] = make_float2(sg * gv.x, sg * gv.y);
        }
    }
    __syncthreads();
    float2* res = tile_fft<N, 3 * RB, 1, N, -1, false>(T, G, plan, 3 * rb, 1, n, tw);
    for (int e = threadIdx.x; e < 3 * cnt; e += blockDim.x) {
        const int fld = e / cnt, p = e - fld * cnt;
        float2* o = fld == 0 ? b3 : fld == 1 ? b4 : b5;
        o[base + p] = res[e];
    }
}

// K4: cb columns per block: F_y of b3, b4, b5, the assembly (kinds of
// k_cdr_assemble), F_y^{-1} of the result into b0.  Tile [row][field * cb + b].
template <int N, int CB>
__global__ void __launch_bounds__(256) k_cdrf_cols_asm(const CdrInst* ins, int n_, int cb_, RadixPlan plan,
                                                       const float2* tw, const float2* b3, const float2* b4,
                                                       const float2* b5, float2* b0, int kind) {
    extern __shared__ __align__(16) float2 sm[];
    const int n = N ? N : n_, cb = N ? CB : cb_;
    const int nbk = n / cb;
    const CdrInst in = ins[blockIdx.x / nbk];
    const int c0 = (blockIdx.x % nbk) * cb;
    const long long base = in.off + c0;
    const int cnt = cb * n;
    for (int e = threadIdx.x; e < 3 * cnt; e += blockDim.x) {
        const int i = e / (3 * cb), r = e - i * (3 * cb), fld = r / cb, b = r - fld * cb;
        const float2* src = fld == 0 ? b3 : fld == 1 ? b4 : b5;
        sm[e] = src[base + (long long)i * n + b];
    }
    __syncthreads();
    float2* S = tile_fft<N, 3 * CB, 3 * CB, 1, -1, true>(sm, sm + kFTile, plan, 3 * cb, 3 * cb, 1, tw);
    float2* T = S == sm ? sm + kFTile : sm;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        const float kx = xi_of<float>(c0 + b, n, in.h), ky = xi_of<float>(i, n, in.h);
        const float2* row = S + (long long)i * 3 * cb;
        const float2 a = row[b], bb = row[cb + b], c = row[2 * cb + b];
        float2 w = make_float2(kx * a.y + ky * bb.y + c.x, -kx * a.x - ky * bb.x + c.y);
        if (kind == 0 || kind == 2) w = make_float2(-w.x, -w.y);
        if (kind == 0 || kind == 1) w = cdiv(w, cdr_lambda(in, kx, ky, false));
        T[e] = w;
    }
    __syncthreads();
    float2* res = tile_fft<N, CB, CB, 1, 1, true>(T, S, plan, cb, cb, 1, tw);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        b0[base + (long long)i * n + b] = res[e];
    }
}

// K5: rb rows per block: F_x^{-1}, out = b0 / n^2, norm2[ids[j]] += ||out||^2
template <int N, int RB>
__global__ void __launch_bounds__(256) k_cdrf_rows_out(const CdrInst* ins, const int* ids, int n_, int rb_,
                                                       RadixPlan plan, const float2* tw, const float2* b0,
                                                       float2* out, double* norm2) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[8];
    const int n = N ? N : n_, rb = N ? RB : rb_;
    const int nbk = n / rb;
    const int j = blockIdx.x / nbk;
    const CdrInst in = ins[j];
    const long long base = in.off + (long long)(blockIdx.x % nbk) * rb * n;
    const int cnt = rb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) sm[e] = b0[base + e];
    __syncthreads();
    float2* res = tile_fft<N, RB, 1, N, 1, false>(sm, sm + kFTile, plan, rb, 1, n, tw);
    const float s = 1.f / ((float)n * (float)n);
    double acc = 0.0;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const float2 v = make_float2(res[e].x * s, res[e].y * s);
        out[base + e] = v;
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    if (norm2) {
        for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            atomicAdd(norm2 + ids[j], t);
        }
    }
}

// ---- register four-step column kernels (compile-time sides) --------------
// The column transforms of K2 and K4 as four-step FFTs in registers (N = N1 N2,
// n = N2 n1 + n2, k = k1 + N1 k2): pass 1 reads each column's N1 points n2 +
// N2 m from global, transforms them and writes the twiddled results to a
// padded shared slab; pass 2 transforms along n2, so that a thread holds the
// spectrum X[k1 + N1 k2] of one column for all k2 in registers, where the
// spectral step runs before the inverse length-N2 transform; pass 3 finishes
// the inverse and writes natural rows.  Two shared round trips per transform
// pair, against two per Stockham pass.
template <int N2> __device__ __forceinline__ int rpad(int p) { return p + p / N2; }
template <int N1, int N2> constexpr int rld() { return ((N1 * N2 + N1 + 13) / 16) * 16 + 2; }
template <int N1, int N2, int CB, int NF> constexpr size_t reg_smem() {
    return sizeof(float2) * ((size_t)NF * CB * rld<N1, N2>() + (size_t)N1 * (N2 + 1));
}
__device__ __forceinline__ float2 rmul(float2 t, float2 w) {
    return make_float2(t.x * w.x - t.y * w.y, t.x * w.y + t.y * w.x);
}
__device__ __forceinline__ float2 rmulc(float2 t, float2 w) {  // t * conj(w)
    return make_float2(t.x * w.x + t.y * w.y, t.y * w.x - t.x * w.y);
}
// twiddles W_N^{n2 k1} stored [k1][N2 + 1] from the length-N table
template <int N1, int N2> __device__ __forceinline__ void reg_twiddles(float2* tw, const float2* src) {
    for (int e = threadIdx.x; e < N1 * N2; e += blockDim.x) {
        const int k1 = e / N2, n2 = e - k1 * N2;
        tw[k1 * (N2 + 1) + n2] = src[n2 * k1];
    }
}
// pass 1 on field f of the slab: length-N1 DFTs over rows n2 + N2 m of cb columns
template <int N1, int N2, int CB>
__device__ __forceinline__ void reg_pass1(const float2* src, long long base, float2* S, const float2* tw) {
    constexpr int N = N1 * N2, LD = rld<N1, N2>();
    for (int j = threadIdx.x; j < CB * N2; j += blockDim.x) {
        const int c = j % CB, n2 = j / CB;
        float2 v[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = src[base + (long long)(n2 + N2 * m) * N + c];
        DftR<N1, -1>::run(v);
        float2* col = S + c * LD;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) col[rpad<N2>(N2 * k1 + n2)] = rmul(v[k1], tw[k1 * (N2 + 1) + n2]);
    }
}

// K2 (register form): b0 columns -> X; [adjoint: / conj(lambda0)]; i xi_x X,
// i xi_y X [, X] -> inverse; F output fields (b1, b2 [, b0]).
template <int N1, int N2, int CB, int F>
__global__ void __launch_bounds__(256) k_cdrr_cols_grad(const CdrInst* ins, const float2* twg, float2* b0,
                                                        float2* b1, float2* b2, int adj) {
    constexpr int N = N1 * N2, LD = rld<N1, N2>(), NBK = N / CB;
    extern __shared__ __align__(16) float2 smem[];
    float2* S = smem;                  // [F][CB][LD]
    float2* tw = smem + F * CB * LD;   // [N1][N2 + 1]
    const CdrInst in = ins[blockIdx.x / NBK];
    const int c0 = (blockIdx.x % NBK) * CB;
    const long long base = in.off + c0;
    reg_twiddles<N1, N2>(tw, twg);
    __syncthreads();
    reg_pass1<N1, N2, CB>(b0, base, S, tw);
    __syncthreads();
    // pass 2: forward along n2, the spectral step, inverse along k2 per output field
    for (int j = threadIdx.x; j < CB * N1; j += blockDim.x) {
        const int k1 = j % N1, c = j / N1;
        float2 v[N2];
        const float2* col = S + c * LD;
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = col[rpad<N2>(N2 * k1 + i)];
        DftR<N2, -1>::run(v);
        const float kx = xi_of<float>(c0 + c, N, in.h);
        if (adj == 1) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const float ky = xi_of<float>(k1 + N1 * k2, N, in.h);
                v[k2] = cdiv(v[k2], cdr_lambda(in, kx, ky, true));
            }
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float2 w[N2];
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const float u = f == 0 ? kx : xi_of<float>(k1 + N1 * k2, N, in.h);
                w[k2] = f < 2 ? make_float2(-u * v[k2].y, u * v[k2].x) : v[k2];
            }
            DftR<N2, +1>::run(w);
            float2* out = S + (f * CB + c) * LD;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) out[rpad<N2>(N2 * k1 + n2)] = rmulc(w[n2], tw[k1 * (N2 + 1) + n2]);
        }
    }
    __syncthreads();
    // pass 3: inverse along k1 -> natural rows N2 n1 + n2
    for (int j = threadIdx.x; j < F * CB * N2; j += blockDim.x) {
        const int f = j / (CB * N2), rem = j - f * (CB * N2);
        const int c = rem % CB, n2 = rem / CB;
        const float2* col = S + (f * CB + c) * LD;
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = col[rpad<N2>(N2 * k1 + n2)];
        DftR<N1, +1>::run(v);
        float2* o = f == 0 ? b1 : f == 1 ? b2 : b0;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) o[base + (long long)(N2 * n1 + n2) * N + c] = v[n1];
    }
}

// K4 (register form): b3, b4, b5 columns -> spectra; W = -i xi_x F1 - i xi_y F2
// + F3 with the mode's multiple (kinds of k_cdr_assemble); inverse into b0.
template <int N1, int N2, int CB>
__global__ void __launch_bounds__(256) k_cdrr_cols_asm(const CdrInst* ins, const float2* twg, const float2* b3,
                                                       const float2* b4, const float2* b5, float2* b0, int kind) {
    constexpr int N = N1 * N2, LD = rld<N1, N2>(), NBK = N / CB;
    extern __shared__ __align__(16) float2 smem[];
    float2* S = smem;                  // [3][CB][LD]
    float2* tw = smem + 3 * CB * LD;   // [N1][N2 + 1]
    const CdrInst in = ins[blockIdx.x / NBK];
    const int c0 = (blockIdx.x % NBK) * CB;
    const long long base = in.off + c0;
    reg_twiddles<N1, N2>(tw, twg);
    __syncthreads();
    reg_pass1<N1, N2, CB>(b3, base, S, tw);
    reg_pass1<N1, N2, CB>(b4, base, S + CB * LD, tw);
    reg_pass1<N1, N2, CB>(b5, base, S + 2 * CB * LD, tw);
    __syncthreads();
    // pass 2a: forward along n2 for each field, spectra back in place (slot N2 k1 + k2 holds k1 + N1 k2)
    for (int j = threadIdx.x; j < 3 * CB * N1; j += blockDim.x) {
        const int fc = j / N1, k1 = j - fc * N1;
        float2* col = S + fc * LD;
        float2 v[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = col[rpad<N2>(N2 * k1 + i)];
        DftR<N2, -1>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) col[rpad<N2>(N2 * k1 + k2)] = v[k2];
    }
    __syncthreads();
    // pass 2b: the assembly, the inverse along k2 into field 0
    for (int j = threadIdx.x; j < CB * N1; j += blockDim.x) {
        const int k1 = j % N1, c = j / N1;
        const float kx = xi_of<float>(c0 + c, N, in.h);
        const float2* c3 = S + c * LD;
        const float2* c4 = S + (CB + c) * LD;
        const float2* c5 = S + (2 * CB + c) * LD;
        float2 w[N2];
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int p = rpad<N2>(N2 * k1 + k2);
            const float ky = xi_of<float>(k1 + N1 * k2, N, in.h);
            const float2 a = c3[p], bb = c4[p], cc = c5[p];
            float2 x = make_float2(kx * a.y + ky * bb.y + cc.x, -kx * a.x - ky * bb.x + cc.y);
            if (kind == 0 || kind == 2) x = make_float2(-x.x, -x.y);
            if (kind == 0 || kind == 1) x = cdiv(x, cdr_lambda(in, kx, ky, false));
            w[k2] = x;
        }
        DftR<N2, +1>::run(w);
        // field 0's slots of this (c, k1) were read above by this thread only
        float2* out = S + c * LD;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) out[rpad<N2>(N2 * k1 + n2)] = rmulc(w[n2], tw[k1 * (N2 + 1) + n2]);
    }
    __syncthreads();
    // pass 3: inverse along k1 -> natural rows
    for (int j = threadIdx.x; j < CB * N2; j += blockDim.x) {
        const int c = j % CB, n2 = j / CB;
        const float2* col = S + c * LD;
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = col[rpad<N2>(N2 * k1 + n2)];
        DftR<N1, +1>::run(v);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) b0[base + (long long)(N2 * n1 + n2) * N + c] = v[n1];
    }
}

// the register column configuration of a compile-time side
template <int N> struct RegCols;
template <> struct RegCols<64> { static constexpr int N1 = 8, N2 = 8, CB = 16; };
template <> struct RegCols<128> { static constexpr int N1 = 8, N2 = 16, CB = 16; };
template <> struct RegCols<256> { static constexpr int N1 = 16, N2 = 16, CB = 8; };

}  // namespace
}  // namespace npbs

namespace npbs {
namespace {

bool cdr_radix_plan(int n, RadixPlan* p) {
    if (n < 2 || n > kMaxN) return false;
    p->n = n;
    p->npass = 0;
    int m = n;
    while (m % 8 == 0) { p->radix[p->npass++] = 8; m /= 8; }
    while (m % 4 == 0) { p->radix[p->npass++] = 4; m /= 4; }
    while (m % 2 == 0) { p->radix[p->npass++] = 2; m /= 2; }
    while (m % 3 == 0) { p->radix[p->npass++] = 3; m /= 3; }
    return m == 1 && p->npass <= kMaxPass;
}

// One grid size of a CDR batch, prepared on the device.
struct CdrGroup {
    int n = 0, cnt = 0;
    RadixPlan plan{};
    const float2* tw = nullptr;
    const double2* tw64 = nullptr;
    const CdrInst* ins = nullptr;   // device [cnt]
    const int* ids = nullptr;       // device [cnt]: batch index of each
    const long long* off = nullptr; // device [6 cnt]: field offsets of buffer k (k * extent + offset)
};

struct CdrPrep {
    std::vector<CdrGroup> groups;
    long long extent = 0;
    float2* buf = nullptr;     // 6 complex64 fields of the batch extent
    double2* buf64 = nullptr;  // 6 complex128 fields (cdr_prepare64 only)
    template <typename R> cpx<R>* fields() const;
    template <typename R> const cpx<R>* twiddles(const CdrGroup& g) const;
};
template <> float2* CdrPrep::fields<float>() const { return buf; }
template <> double2* CdrPrep::fields<double>() const { return buf64; }
template <> const float2* CdrPrep::twiddles<float>(const CdrGroup& g) const { return g.tw; }
template <> const double2* CdrPrep::twiddles<double>(const CdrGroup& g) const { return g.tw64; }

npbs_status cdr_fused_attrs(npbs_ctx* ctx);

// The last prepared batch: its exact description (instances and constants)
// and the prepared plan, whose device tables stay in work[12].
struct CdrCached {
    std::vector<char> desc;
    CdrPrep P;
};

npbs_status cdr_prepare(npbs_ctx* ctx, const npbs_batch* batch, const npbs_cdr_consts* consts, CdrPrep* P,
                        cudaStream_t st) {
    if (!batch || batch->count < 0 || (batch->count > 0 && (!batch->inst || !consts)))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr: NULL batch or constants");
    // a batch identical to the last one prepared reuses its tables: no upload, no synchronisation
    std::vector<char> desc(sizeof(int) + (size_t)batch->count * (sizeof(npbs_instance) + sizeof(npbs_cdr_consts)));
    memcpy(desc.data(), &batch->count, sizeof(int));
    if (batch->count > 0) {
        memcpy(desc.data() + sizeof(int), batch->inst, sizeof(npbs_instance) * batch->count);
        memcpy(desc.data() + sizeof(int) + sizeof(npbs_instance) * batch->count, consts,
               sizeof(npbs_cdr_consts) * batch->count);
    }
    if (ctx->cdr_prep) {
        const CdrCached* c = static_cast<const CdrCached*>(ctx->cdr_prep.get());
        if (c->desc == desc) {
            *P = c->P;
            return NPBS_OK;
        }
    }
    std::map<int, std::vector<int>> by;
    long long ext = 0;
    for (int j = 0; j < batch->count; ++j) {
        const npbs_instance& s = batch->inst[j];
        RadixPlan rp;
        if (s.nx != s.ny || s.nx % 16 != 0 || !cdr_radix_plan(s.nx, &rp)) {
            char buf[160];
            snprintf(buf, sizeof buf, "cdr: instance %d is %d x %d; need square grids, side a multiple of 16, 2^a 3^b <= %d",
                     j, s.ny, s.nx, kMaxN);
            return set_err(ctx, NPBS_ERR_UNSUPPORTED_SIZE, buf);
        }
        if (!(s.h > 0.0) || !std::isfinite(s.h) || s.offset < 0 || s.offset % 32 != 0)
            return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr: need h > 0 and offsets >= 0, multiples of 32");
        const npbs_cdr_consts& c = consts[j];
        if (!(c.kappa0 > 0.0) || !std::isfinite(c.v0x) || !std::isfinite(c.v0y) || !std::isfinite(c.sigma0) ||
            !std::isfinite(c.kappa0))
            return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr: need kappa0 > 0 and finite background constants");
        by[s.nx].push_back(j);
        ext = std::max<long long>(ext, s.offset + (long long)s.nx * s.ny);
    }
    P->extent = ext;
    P->groups.clear();
    // host staging of every group's tables, then one upload
    std::vector<char> host;
    auto put = [&](const void* src, size_t bytes) {
        const size_t o = (host.size() + 255) & ~size_t(255);
        host.resize(o + bytes);
        memcpy(host.data() + o, src, bytes);
        return o;
    };
    struct Offs { size_t tw, tw64, ins, ids, off; };
    std::vector<Offs> offs;
    for (auto& kv : by) {
        const int n = kv.first;
        CdrGroup g;
        g.n = n;
        g.cnt = (int)kv.second.size();
        cdr_radix_plan(n, &g.plan);
        std::vector<float2> tw(n);
        std::vector<double2> tw64(n);
        for (int k = 0; k < n; ++k) {
            const double a = -2.0 * M_PI * (double)k / (double)n;
            tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
            tw64[k] = make_double2(std::cos(a), std::sin(a));
        }
        std::vector<CdrInst> ins;
        std::vector<long long> off;
        for (int j : kv.second) {
            const npbs_instance& s = batch->inst[j];
            const npbs_cdr_consts& c = consts[j];
            ins.push_back(CdrInst{s.nx, s.h, s.offset, c.kappa0, c.v0x, c.v0y, c.sigma0});
        }
        for (int k = 0; k < 6; ++k)
            for (int j : kv.second) off.push_back((long long)k * ext + batch->inst[j].offset);
        Offs o;
        o.tw = put(tw.data(), sizeof(float2) * tw.size());
        o.tw64 = put(tw64.data(), sizeof(double2) * tw64.size());
        o.ins = put(ins.data(), sizeof(CdrInst) * ins.size());
        o.ids = put(kv.second.data(), sizeof(int) * kv.second.size());
        o.off = put(off.data(), sizeof(long long) * off.size());
        offs.push_back(o);
        P->groups.push_back(g);
    }
    NPBS_CK(ctx, ctx->work[12].ensure(std::max<size_t>(host.size(), 256)));
    NPBS_CK(ctx, ctx->work[13].ensure(sizeof(float2) * 6 * (size_t)std::max<long long>(ext, 1)));
    char* d = static_cast<char*>(ctx->work[12].p);
    NPBS_CK(ctx, cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    NPBS_CK(ctx, cudaStreamSynchronize(st));  // the staging vector goes out of scope
    for (size_t i = 0; i < P->groups.size(); ++i) {
        P->groups[i].tw = reinterpret_cast<const float2*>(d + offs[i].tw);
        P->groups[i].tw64 = reinterpret_cast<const double2*>(d + offs[i].tw64);
        P->groups[i].ins = reinterpret_cast<const CdrInst*>(d + offs[i].ins);
        P->groups[i].ids = reinterpret_cast<const int*>(d + offs[i].ids);
        P->groups[i].off = reinterpret_cast<const long long*>(d + offs[i].off);
    }
    P->buf = static_cast<float2*>(ctx->work[13].p);
    NPBS_CK(ctx, fft2d::set_attrs());
    npbs_status fs = cdr_fused_attrs(ctx);
    if (fs != NPBS_OK) return fs;
    auto cached = std::make_shared<CdrCached>();
    cached->desc = std::move(desc);
    cached->P = *P;
    cached->P.buf64 = nullptr;  // cdr_prepare64 sets it per call
    ctx->cdr_prep = cached;
    return NPBS_OK;
}

// the complex128 field buffers of the float64 residual (after cdr_prepare)
npbs_status cdr_prepare64(npbs_ctx* ctx, CdrPrep* P) {
    NPBS_CK(ctx, ctx->work[16].ensure(sizeof(double2) * 6 * (size_t)std::max<long long>(P->extent, 1)));
    P->buf64 = static_cast<double2*>(ctx->work[16].p);
    NPBS_CK(ctx, fft2d::set_attrs_of<double2>());
    return NPBS_OK;
}

int cdr_grid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

// internal apply modes beside the public ones: out = -A^* y, and the Green
// operators alone
constexpr int kCdrMinusAdjA = 100;
constexpr int kCdrGreen = 101;
constexpr int kCdrGreenAdj = 102;

inline int divisor_at_most(int n, int lim) {
    for (int d = std::min(n, lim); d >= 1; --d)
        if (n % d == 0) return d;
    return 1;
}

template <int N, int RB, int CB> cudaError_t fused_attrs_of() {
    const int sm = (int)(2 * kFTile * sizeof(float2));
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    if constexpr (N > 0) {
        using RC = RegCols<N>;
        const int rs = (int)reg_smem<RC::N1, RC::N2, RC::CB, 3>();
        e = cudaFuncSetAttribute(k_cdrr_cols_grad<RC::N1, RC::N2, RC::CB, 2>, at, rs);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrr_cols_grad<RC::N1, RC::N2, RC::CB, 3>, at, rs);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrr_cols_asm<RC::N1, RC::N2, RC::CB>, at, rs);
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_rows_fwd<N, RB>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_cols_grad<N, CB, 2>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_cols_grad<N, CB, 3>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_rows_flux<N, RB, 2>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_rows_flux<N, RB, 3>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_cols_asm<N, CB>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdrf_rows_out<N, RB>, at, sm);
    return e;
}

npbs_status cdr_fused_attrs(npbs_ctx* ctx) {
    NPBS_CK(ctx, (fused_attrs_of<0, 0, 0>()));
    NPBS_CK(ctx, (fused_attrs_of<64, 8, 8>()));
    NPBS_CK(ctx, (fused_attrs_of<128, 8, 8>()));
    NPBS_CK(ctx, (fused_attrs_of<256, 4, 4>()));
    return NPBS_OK;
}

// The five launches of one grid side (N > 0: compile-time geometry RB, CB).
template <int N, int RB, int CB>
void fused_launch(const CdrGroup& g, int rb, int cb, int mode, const float* kappa, const float* vx, const float* vy,
                  const float* sigma, const float2* f, const float2* x, float2* const* b, float2* out, double* norm2,
                  cudaStream_t st) {
    const int n = g.n;
    const size_t sm = 2 * kFTile * sizeof(float2);
    const bool adj = mode == NPBS_ADJ_B || mode == kCdrMinusAdjA;
    const int kind = mode == NPBS_RESIDUAL ? 0 : mode == NPBS_OP_B ? 1
                   : (mode == NPBS_TRUE_RESIDUAL || mode == kCdrMinusAdjA) ? 2 : 3;
    const unsigned gr = (unsigned)(g.cnt * (n / rb)), gc = (unsigned)(g.cnt * (n / cb));
    const float2* fs = (mode == NPBS_OP_B || adj) ? nullptr : f;
    k_cdrf_rows_fwd<N, RB><<<gr, 256, sm, st>>>(g.ins, n, rb, g.plan, g.tw, x, b[0]);
    // column kernels: register four-step transforms for the compile-time sides
    auto cols_grad = [&](auto fct) {
        constexpr int F = decltype(fct)::value;
        if constexpr (N > 0) {
            using RC = RegCols<N>;
            const unsigned gcr = (unsigned)(g.cnt * (N / RC::CB));
            k_cdrr_cols_grad<RC::N1, RC::N2, RC::CB, F><<<gcr, 256, reg_smem<RC::N1, RC::N2, RC::CB, 3>(), st>>>(
                g.ins, g.tw, b[0], b[1], b[2], mode == NPBS_ADJ_B ? 1 : 0);
        } else {
            k_cdrf_cols_grad<N, CB, F><<<gc, 256, sm, st>>>(g.ins, n, cb, g.plan, g.tw, b[0], b[1], b[2],
                                                            mode == NPBS_ADJ_B ? 1 : 0);
        }
    };
    if (adj) {
        cols_grad(std::integral_constant<int, 3>{});
        k_cdrf_rows_flux<N, RB, 3><<<gr, 256, sm, st>>>(g.ins, n, rb, g.plan, g.tw, kappa, vx, vy, sigma, x, fs, b[0],
                                                        b[1], b[2], b[3], b[4], b[5]);
    } else {
        cols_grad(std::integral_constant<int, 2>{});
        k_cdrf_rows_flux<N, RB, 2><<<gr, 256, sm, st>>>(g.ins, n, rb, g.plan, g.tw, kappa, vx, vy, sigma, x, fs, b[0],
                                                        b[1], b[2], b[3], b[4], b[5]);
    }
    if constexpr (N > 0) {
        using RC = RegCols<N>;
        const unsigned gcr = (unsigned)(g.cnt * (N / RC::CB));
        k_cdrr_cols_asm<RC::N1, RC::N2, RC::CB><<<gcr, 256, reg_smem<RC::N1, RC::N2, RC::CB, 3>(), st>>>(
            g.ins, g.tw, b[3], b[4], b[5], b[0], kind);
    } else {
        k_cdrf_cols_asm<N, CB><<<gc, 256, sm, st>>>(g.ins, n, cb, g.plan, g.tw, b[3], b[4], b[5], b[0], kind);
    }
    k_cdrf_rows_out<N, RB><<<gr, 256, sm, st>>>(g.ins, g.ids, n, rb, g.plan, g.tw, b[0], out, norm2);
}

// The fused float32 apply (RESIDUAL, OP_B, TRUE_RESIDUAL, ADJ_B, -A^*): grid
// sides 64, 128 and 256 with compile-time geometry, the others at run time.
npbs_status cdr_run_fused(npbs_ctx* ctx, const CdrPrep& P, int mode, const float* kappa, const float* vx,
                          const float* vy, const float* sigma, const float2* f, const float2* x, float2* out,
                          double* norm2, int count, cudaStream_t st) {
    const long long E = P.extent;
    float2* b[6];
    for (int k = 0; k < 6; ++k) b[k] = P.buf + k * E;
    if (norm2) NPBS_CK(ctx, cudaMemsetAsync(norm2, 0, sizeof(double) * count, st));
    for (const CdrGroup& g : P.groups) {
        const int n = g.n;
        // three fields of rb rows (cb columns) fit one tile buffer
        const int rb = divisor_at_most(n, std::min(8, kFTile / (3 * n)));
        const int cb = divisor_at_most(n, std::min(8, kFTile / (3 * n)));
        if (n == 64 && rb == 8 && cb == 8)
            fused_launch<64, 8, 8>(g, rb, cb, mode, kappa, vx, vy, sigma, f, x, b, out, norm2, st);
        else if (n == 128 && rb == 8 && cb == 8)
            fused_launch<128, 8, 8>(g, rb, cb, mode, kappa, vx, vy, sigma, f, x, b, out, norm2, st);
        else if (n == 256 && rb == 4 && cb == 4)
            fused_launch<256, 4, 4>(g, rb, cb, mode, kappa, vx, vy, sigma, f, x, b, out, norm2, st);
        else
            fused_launch<0, 0, 0>(g, rb, cb, mode, kappa, vx, vy, sigma, f, x, b, out, norm2, st);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(st, 5);
    }
    return NPBS_OK;
}

// One CDR apply over a prepared batch (mode: RESIDUAL, OP_B, TRUE_RESIDUAL,
// ADJ_B or an internal one) in precision R; out is complex64 in both.  The
// float32 operator modes run fused (cdr_run_fused); the float64 residual and
// the Green operators run the step-by-step kernels.
template <typename R>
npbs_status cdr_run(npbs_ctx* ctx, const CdrPrep& P, int mode, const float* kappa, const float* vx, const float* vy,
                    const float* sigma, const float2* f, const cpx<R>* x, float2* out, double* norm2, int count,
                    cudaStream_t st) {
    using C = cpx<R>;
    if constexpr (std::is_same<R, float>::value) {
        if (mode != kCdrGreen && mode != kCdrGreenAdj)
            return cdr_run_fused(ctx, P, mode, kappa, vx, vy, sigma, f, x, out, norm2, count, st);
    }
    const long long E = P.extent;
    C* const buf = P.fields<R>();
    if (!buf) return set_err(ctx, NPBS_ERR_CUDA, "cdr: float64 buffers not prepared");
    C* b[6];
    for (int k = 0; k < 6; ++k) b[k] = buf + k * E;
    if (norm2) NPBS_CK(ctx, cudaMemsetAsync(norm2, 0, sizeof(double) * count, st));
    if (mode == kCdrGreen || mode == kCdrGreenAdj) {
        for (const CdrGroup& g : P.groups) {
            const long long np = (long long)g.n * g.n, tot = (long long)g.cnt * np;
            const int grid = cdr_grid(tot);
            const C* tw = P.twiddles<R>(g);
            k_cdr_copy<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, x, b[0]);
            NPBS_CK(ctx, fft2d::run<C>(buf, g.off, g.cnt, g.n, -1, g.plan, tw, st));
            k_cdr_green<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, b[0], mode == kCdrGreenAdj ? 1 : 0);
            NPBS_CK(ctx, fft2d::run<C>(buf, g.off, g.cnt, g.n, 1, g.plan, tw, st));
            k_cdr_out<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, b[0], out, g.ids, norm2);
            NPBS_CK(ctx, cudaGetLastError());
            ctx->count(st, 3 + 2 * 2);
        }
        return NPBS_OK;
    }
    const bool adj = mode == NPBS_ADJ_B || mode == kCdrMinusAdjA;
    const int kind = mode == NPBS_RESIDUAL ? 0 : mode == NPBS_OP_B ? 1
                   : (mode == NPBS_TRUE_RESIDUAL || mode == kCdrMinusAdjA) ? 2 : 3;
    for (const CdrGroup& g : P.groups) {
        const long long np = (long long)g.n * g.n, tot = (long long)g.cnt * np;
        const int grid = cdr_grid(tot);
        const C* tw = P.twiddles<R>(g);
        k_cdr_copy<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, x, b[0]);
        NPBS_CK(ctx, fft2d::run<C>(buf, g.off, g.cnt, g.n, -1, g.plan, tw, st));
        k_cdr_grad<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, b[0], b[1], b[2],
                                            mode == NPBS_ADJ_B ? 1 : adj ? 2 : 0);
        // b1, b2 (and for the adjoint b0 = G^* x) back to physical space
        NPBS_CK(ctx, fft2d::run<C>(buf, g.off + g.cnt, 2LL * g.cnt, g.n, 1, g.plan, tw, st));
        if (adj) NPBS_CK(ctx, fft2d::run<C>(buf, g.off, g.cnt, g.n, 1, g.plan, tw, st));
        k_cdr_flux<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, kappa, vx, vy, sigma, x,
                                            (mode == NPBS_OP_B || adj) ? nullptr : f, b[0], b[1], b[2], b[3], b[4],
                                            b[5], adj ? 1 : 0);
        NPBS_CK(ctx, fft2d::run<C>(buf, g.off + 3 * g.cnt, 3LL * g.cnt, g.n, -1, g.plan, tw, st));
        k_cdr_assemble<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, b[3], b[4], b[5], b[0], kind);
        NPBS_CK(ctx, fft2d::run<C>(buf, g.off, g.cnt, g.n, 1, g.plan, tw, st));
        k_cdr_out<R><<<grid, 256, 0, st>>>(g.ins, g.cnt, np, b[0], out, g.ids, norm2);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(st, 5 + 2 * (adj ? 5 : 4));
    }
    return NPBS_OK;
}

// background constants per instance: the midpoints of the ranges of kappa and
// sigma, the grid means of vx and vy
__global__ void k_cdr_background(const CdrInst* ins, const int* ids, const float* kappa, const float* vx,
                                 const float* vy, const float* sigma, double* out) {
    const CdrInst in = ins[blockIdx.x];
    const long long np = (long long)in.n * in.n;
    double mx = 0, my = 0;
    float kmin = 3.0e38f, kmax = -3.0e38f, smin = 3.0e38f, smax = -3.0e38f;
    for (long long p = threadIdx.x; p < np; p += blockDim.x) {
        const long long o = in.off + p;
        kmin = fminf(kmin, kappa[o]);
        kmax = fmaxf(kmax, kappa[o]);
        smin = fminf(smin, sigma[o]);
        smax = fmaxf(smax, sigma[o]);
        mx += vx[o];
        my += vy[o];
    }
    for (int w = 16; w > 0; w >>= 1) {
        mx += __shfl_xor_sync(0xffffffffu, mx, w);
        my += __shfl_xor_sync(0xffffffffu, my, w);
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, w));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, w));
        smin = fminf(smin, __shfl_xor_sync(0xffffffffu, smin, w));
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, w));
    }
    __shared__ double rd[2][8];
    __shared__ float rf[4][8];
    const int wp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        rd[0][wp] = mx;
        rd[1][wp] = my;
        rf[0][wp] = kmin;
        rf[1][wp] = kmax;
        rf[2][wp] = smin;
        rf[3][wp] = smax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (int)(blockDim.x >> 5);
        double a = 0, b = 0;
        float k0 = rf[0][0], k1 = rf[1][0], s0 = rf[2][0], s1 = rf[3][0];
        for (int w = 0; w < nw; ++w) {
            a += rd[0][w];
            b += rd[1][w];
            k0 = fminf(k0, rf[0][w]);
            k1 = fmaxf(k1, rf[1][w]);
            s0 = fminf(s0, rf[2][w]);
            s1 = fmaxf(s1, rf[3][w]);
        }
        double* o = out + 4 * ids[blockIdx.x];
        o[0] = 0.5 * ((double)k0 + (double)k1);
        o[1] = a / (double)np;
        o[2] = b / (double)np;
        o[3] = 0.5 * ((double)s0 + (double)s1);
    }
}

// u += r (the Born series step, M = identity)
__global__ void k_cdr_axpy(const CdrInst* ins, int cnt, long long np, const float2* r, float2* u) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt * np; g += (long long)gridDim.x * blockDim.x) {
        int j; long long p;
        field_point(ins, np, g, &j, &p);
        const long long o = ins[j].off + p;
        u[o] = make_float2(u[o].x + r[o].x, u[o].y + r[o].y);
    }
}

}  // namespace
}  // namespace npbs

using namespace npbs;

extern "C" {

npbs_status npbs_cdr_background(npbs_ctx* ctx, const npbs_batch* batch, const float* kappa, const float* vx,
                                const float* vy, const float* sigma, npbs_cdr_consts* out, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!batch || batch->count < 0 || (batch->count > 0 && (!kappa || !vx || !vy || !sigma || !out)))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_cdr_background: NULL argument");
    if (batch->count == 0) return NPBS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<npbs_cdr_consts> dummy(batch->count, npbs_cdr_consts{1.0, 0.0, 0.0, 0.0});
    CdrPrep P;
    npbs_status st = cdr_prepare(ctx, batch, dummy.data(), &P, s);
    if (st != NPBS_OK) return st;
    NPBS_CK(ctx, ctx->work[14].ensure(sizeof(double) * 4 * batch->count));
    double* dm = static_cast<double*>(ctx->work[14].p);
    for (const CdrGroup& g : P.groups) k_cdr_background<<<g.cnt, 256, 0, s>>>(g.ins, g.ids, kappa, vx, vy, sigma, dm);
    NPBS_CK(ctx, cudaGetLastError());
    ctx->count(s, (long long)P.groups.size());
    std::vector<double> h(4 * batch->count);
    NPBS_CK(ctx, cudaMemcpyAsync(h.data(), dm, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaStreamSynchronize(s));
    for (int j = 0; j < batch->count; ++j) out[j] = npbs_cdr_consts{h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]};
    return NPBS_OK;
}

npbs_status cdr_apply(npbs_ctx* ctx, const npbs_batch* batch, const npbs_cdr_consts* consts, const float* kappa,
                      const float* vx, const float* vy, const float* sigma, const void* f, const void* x, void* out,
                      npbs_mode mode, double* norm2, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (mode != NPBS_RESIDUAL && mode != NPBS_OP_B && mode != NPBS_TRUE_RESIDUAL && mode != NPBS_ADJ_B)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_apply: mode must be RESIDUAL, OP_B, TRUE_RESIDUAL or ADJ_B");
    if (!batch || batch->count == 0) return batch ? NPBS_OK : NPBS_ERR_INVALID_ARG;
    const bool need_f = mode == NPBS_RESIDUAL || mode == NPBS_TRUE_RESIDUAL;
    if (!kappa || !vx || !vy || !sigma || !x || !out || (need_f && !f))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_apply: NULL field pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CdrPrep P;
    npbs_status st = cdr_prepare(ctx, batch, consts, &P, s);
    if (st != NPBS_OK) return st;
    return cdr_run<float>(ctx, P, (int)mode, kappa, vx, vy, sigma, static_cast<const float2*>(f),
                   static_cast<const float2*>(x), static_cast<float2*>(out), norm2, batch->count, s);
}

}  // extern "C"

// NPBS (direct = false: u <- u + M(G(f - A u))) or the Direct format
// (direct = true: u <- u + M(f - A u)) with the CDR operators
static npbs_status cdr_solve_impl(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch,
                                  const npbs_cdr_consts* consts, const float* kappa, const float* vx, const float* vy,
                                  const float* sigma, const void* f, const float* a, void* u,
                                  const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream, bool direct) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (direct && !net) return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_solve_direct: need a network");
    if (!batch || batch->count < 0) return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_solve: NULL batch");
    const int cnt = batch->count;
    if (cnt == 0) return NPBS_OK;
    if (!opts || !(opts->rtol >= 0.0) || opts->max_iter < 0 || opts->check_every < 1)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_solve: need rtol >= 0, max_iter >= 0, check_every >= 1");
    if (!kappa || !vx || !vy || !sigma || !f || !u || (net && !a))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_solve: NULL field pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CdrPrep P;
    npbs_status st = cdr_prepare(ctx, batch, consts, &P, s);
    if (st != NPBS_OK) return st;
    st = cdr_prepare64(ctx, &P);
    if (st != NPBS_OK) return st;
    const long long E = P.extent;
    const size_t ext = (size_t)std::max<long long>(E, 1);
    // r: the Born residual of the correction equation; rho = f - A u (complex64
    // copy of the float64 residual); delta: the correction since the last fold
    NPBS_CK(ctx, ctx->work[15].ensure(sizeof(double) * 2 * cnt + sizeof(int) * cnt));
    NPBS_CK(ctx, ctx->work[17].ensure(sizeof(float2) * 3 * ext));
    double* n2 = static_cast<double*>(ctx->work[15].p);
    double* f2 = n2 + cnt;
    int* frozen = reinterpret_cast<int*>(f2 + cnt);
    float2* r = static_cast<float2*>(ctx->work[17].p);
    float2* rho = r + ext;
    float2* delta = rho + ext;
    double2* U = static_cast<double2*>(u);
    const float2* F = static_cast<const float2*>(f);
    NPBS_CK(ctx, cudaMemsetAsync(delta, 0, sizeof(float2) * ext, s));
    NPBS_CK(ctx, cudaMemsetAsync(f2, 0, sizeof(double) * cnt, s));
    NPBS_CK(ctx, cudaMemsetAsync(frozen, 0, sizeof(int) * cnt, s));
    for (const CdrGroup& g : P.groups) {
        const long long np = (long long)g.n * g.n;
        k_cdr_norm2<<<cdr_grid(g.cnt * np), 256, 0, s>>>(g.ins, g.cnt, np, F, g.ids, f2);
    }
    NPBS_CK(ctx, cudaGetLastError());
    ctx->count(s, (long long)P.groups.size());
    std::vector<double> hf(cnt), hr(cnt);
    NPBS_CK(ctx, cudaMemcpyAsync(hf.data(), f2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    NetRun run;
    std::vector<int> all(cnt);
    for (int j = 0; j < cnt; ++j) all[j] = j;
    const Net* N = reinterpret_cast<const Net*>(net);
    if (N) {
        npbs_status s2;
        // the network groups instances through a context plan (constants there are placeholders)
        std::vector<npbs_instance> tmp(batch->inst, batch->inst + cnt);
        for (auto& t : tmp) { t.k0sq = 0.0; t.eps = 1.0; }
        npbs_batch b2{cnt, tmp.data()};
        const Plan* pl = get_plan(ctx, &b2, &s2);
        if (!pl) return s2;
        s2 = net_prepare(ctx, *N, *pl, all, false, &run, s, a);
        if (s2 != NPBS_OK) return s2;
    }
    std::vector<int> iters(cnt, 0);
    std::vector<double> rt(cnt, 1.0);
    std::vector<npbs_status> stat(cnt, NPBS_NOT_CONVERGED);
    int it = 0;
    // every check folds delta into u and recomputes rho = f - A u in float64:
    // the inner complex64 iteration then solves A delta = rho from delta = 0,
    // whose Born residuals G(rho - A delta) are those of the uninterrupted
    // iteration (M is linear in r), so the count is the method's while the
    // stopping test carries no float32 floor.  An instance that passed is
    // frozen: its u stays the iterate of its first passing check.
    std::vector<int> hfrozen(cnt, 0);
    auto check = [&]() -> npbs_status {
        for (const CdrGroup& g : P.groups) {
            const long long np = (long long)g.n * g.n;
            k_cdr_fold<<<cdr_grid(g.cnt * np), 256, 0, s>>>(g.ins, g.ids, frozen, g.cnt, np, delta, U);
        }
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(s, (long long)P.groups.size());
        npbs_status s2 = cdr_run<double>(ctx, P, NPBS_TRUE_RESIDUAL, kappa, vx, vy, sigma, F, U, rho, n2, cnt, s);
        if (s2 != NPBS_OK) return s2;
        NPBS_CK(ctx, cudaMemcpyAsync(hr.data(), n2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        NPBS_CK(ctx, cudaStreamSynchronize(s));
        for (int j = 0; j < cnt; ++j) {
            if (stat[j] != NPBS_NOT_CONVERGED) continue;
            rt[j] = std::sqrt(hr[j] / std::max(hf[j], 1e-300));
            iters[j] = it;
            if (!std::isfinite(rt[j])) stat[j] = NPBS_ERR_NONFINITE;
            else if (rt[j] <= opts->rtol) stat[j] = NPBS_OK;
            hfrozen[j] = stat[j] != NPBS_NOT_CONVERGED;
        }
        NPBS_CK(ctx, cudaMemcpyAsync(frozen, hfrozen.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        return NPBS_OK;
    };
    st = check();
    if (st != NPBS_OK) return st;
    while (it < opts->max_iter) {
        bool any = false;
        for (int j = 0; j < cnt; ++j) any |= stat[j] == NPBS_NOT_CONVERGED;
        if (!any) break;
        // every instance iterates; frozen ones are no longer folded into u
        for (int k = 0; k < opts->check_every && it < opts->max_iter; ++k, ++it) {
            // the network input of the correction equation: G(rho - A delta), or rho - A delta
            st = cdr_run<float>(ctx, P, direct ? NPBS_TRUE_RESIDUAL : NPBS_RESIDUAL, kappa, vx, vy, sigma, rho, delta,
                                r, nullptr, cnt, s);
            if (st != NPBS_OK) return st;
            if (N) {
                st = net_run_forward(ctx, *N, run, r, a, delta, 1, s);
                if (st != NPBS_OK) return st;
            } else {
                for (const CdrGroup& g : P.groups) {
                    const long long np = (long long)g.n * g.n;
                    k_cdr_axpy<<<cdr_grid(g.cnt * np), 256, 0, s>>>(g.ins, g.cnt, np, r, delta);
                }
                NPBS_CK(ctx, cudaGetLastError());
                ctx->count(s, (long long)P.groups.size());
            }
        }
        st = check();
        if (st != NPBS_OK) return st;
    }
    npbs_status ret = NPBS_OK;
    for (int j = 0; j < cnt; ++j) {
        if (stat[j] == NPBS_NOT_CONVERGED) iters[j] = it;
        if (report) {
            if (report->iters) report->iters[j] = iters[j];
            if (report->rtol) report->rtol[j] = rt[j];
            if (report->status) report->status[j] = stat[j];
            if (report->flags) report->flags[j] = 0;
        }
        if (stat[j] == NPBS_ERR_NONFINITE) ret = NPBS_ERR_NONFINITE;
        else if (stat[j] != NPBS_OK && ret == NPBS_OK) ret = NPBS_NOT_CONVERGED;
    }
    return ret;
}

extern "C" {

npbs_status cdr_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const npbs_cdr_consts* consts,
                      const float* kappa, const float* vx, const float* vy, const float* sigma, const void* f,
                      const float* a, void* u, const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream) {
    return cdr_solve_impl(ctx, net, batch, consts, kappa, vx, vy, sigma, f, a, u, opts, report, stream, false);
}

npbs_status cdr_solve_direct(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch,
                             const npbs_cdr_consts* consts, const float* kappa, const float* vx, const float* vy,
                             const float* sigma, const void* f, const float* a, void* u, const npbs_solve_opts* opts,
                             npbs_report* report, npbs_stream stream) {
    return cdr_solve_impl(ctx, net, batch, consts, kappa, vx, vy, sigma, f, a, u, opts, report, stream, true);
}

npbs_status cdr_train_step_loss(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch,
                                const npbs_cdr_consts* consts, const float* kappa, const float* vx, const float* vy,
                                const float* sigma, const void* f, const float* a, const void* u_snap,
                                int32_t unroll, npbs_loss kind, float lr, float weight_decay, float* loss_host,
                                npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (kind != NPBS_LOSS_BS_RETA && kind != NPBS_LOSS_BS_L2 && kind != NPBS_LOSS_DIR)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_train_step: unknown loss");
    if (!net || !batch || !kappa || !vx || !vy || !sigma || !f || !a || !u_snap || !loss_host)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_train_step: NULL argument");
    if (unroll < 1 || unroll > 16 || !(lr >= 0.f) || !(weight_decay >= 0.f))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cdr_train_step: need 1 <= unroll <= 16, lr >= 0, weight_decay >= 0");
    *loss_host = 0.f;
    const int cnt = batch->count;
    if (cnt <= 0) return cnt == 0 ? NPBS_OK : NPBS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CdrPrep P;
    npbs_status st = cdr_prepare(ctx, batch, consts, &P, s);
    if (st != NPBS_OK) return st;
    // the network and the step's vector kernels walk the instances through a
    // context plan (its k0sq / eps are placeholders, unused here)
    std::vector<npbs_instance> tmp(batch->inst, batch->inst + cnt);
    for (auto& t : tmp) { t.k0sq = 0.0; t.eps = 1.0; }
    npbs_batch b2{cnt, tmp.data()};
    const Plan* pl = get_plan(ctx, &b2, &st);
    if (!pl) return st;
    const float2* F = static_cast<const float2*>(f);
    const float2* usnap = static_cast<const float2*>(u_snap);
    Net& N = *reinterpret_cast<Net*>(net);
    if (kind != NPBS_LOSS_BS_RETA) {
        // explicit adjoints: the convection term makes A not complex symmetric
        EuclidOps op;
        op.minus_a = [&](const float2* x, const float2* f_in, float2* out, double* norm2) -> npbs_status {
            return cdr_run<float>(ctx, P, NPBS_TRUE_RESIDUAL, kappa, vx, vy, sigma, f_in, x, out, norm2, cnt, s);
        };
        op.minus_a_adj = [&](const float2* y, float2* out) -> npbs_status {
            return cdr_run<float>(ctx, P, kCdrMinusAdjA, kappa, vx, vy, sigma, nullptr, y, out, nullptr, cnt, s);
        };
        op.green = [&](const float2* x, float2* out) -> npbs_status {
            return cdr_run<float>(ctx, P, kCdrGreen, kappa, vx, vy, sigma, nullptr, x, out, nullptr, cnt, s);
        };
        op.green_adj = [&](const float2* y, float2* out) -> npbs_status {
            return cdr_run<float>(ctx, P, kCdrGreenAdj, kappa, vx, vy, sigma, nullptr, y, out, nullptr, cnt, s);
        };
        return train_step_euclid(ctx, N, pl, a, F, usnap, unroll, kind == NPBS_LOSS_BS_L2, lr, weight_decay,
                                 loss_host, s, op);
    }
    BornOp op = [&](int mode, const float2* x, float2* out, double* norm2) -> npbs_status {
        return cdr_run<float>(ctx, P, mode, kappa, vx, vy, sigma, F, mode == NPBS_RESIDUAL ? usnap : x, out, norm2,
                              cnt, s);
    };
    return train_step_reta(ctx, N, pl, a, unroll, lr, weight_decay, loss_host, s, op);
}

npbs_status cdr_train_step(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const npbs_cdr_consts* consts,
                           const float* kappa, const float* vx, const float* vy, const float* sigma, const void* f,
                           const float* a, const void* u_snap, int32_t unroll, float lr, float weight_decay,
                           float* loss_host, npbs_stream stream) {
    return cdr_train_step_loss(ctx, net, batch, consts, kappa, vx, vy, sigma, f, a, u_snap, unroll,
                               NPBS_LOSS_BS_RETA, lr, weight_decay, loss_host, stream);
}

}  // extern "C"
