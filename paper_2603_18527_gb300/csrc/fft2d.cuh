// Batched 2D complex FFTs of square n x n fields for the parts of the library
// that run plain transforms (the FNO's Fourier layers, the CDR operators):
// a row kernel and a column kernel of radix-2/3/4/8 Stockham passes in shared
// memory (fft.cuh), forward unnormalised, inverse without the 1/n^2 factor.
// Field i of a call starts at data + off[i] (or at data + i n^2 when off is
// null).  C is float2 or double2 (the twiddle table has the same type).  Two
// tile buffers of kTile complex elements per block (64 KB of dynamic shared
// memory in float32, 128 KB in float64: set_attrs() opts the kernels in).
#pragma once

#include <algorithm>
#include <type_traits>

#include "fft.cuh"

namespace npbs {
namespace fft2d {
namespace {

constexpr int kTile = 4096;

// A tile transform: compile-time geometry when N > 0, else the run-time plan.
template <typename C, int N, int NB, int SI, int SB, int DIR, bool COLS>
__device__ __forceinline__ C* tile(C* a, C* b, const RadixPlan& plan, int nb, int si, int sb, const C* tw) {
    if constexpr (N > 0) return fft_tile_ct<C, DIR, COLS, N, NB, SI, SB>(a, b, tw, threadIdx.x, blockDim.x);
    else return fft_tile<C, DIR, COLS>(a, b, plan, nb, si, sb, tw, threadIdx.x, blockDim.x);
}

// Real channel planes feeding a forward transform: field f = b * P + j of
// the transform is (channel 2 j) + i (channel 2 j + 1) of sample b of planes
// x [nb][ci][n n] (P = ceil(ci / 2); a missing odd channel is zero).
struct RealPairs {
    const float* x = nullptr;
    int ci = 0;
};

// rb rows of one field per block, the transform along each row (N > 0: the
// side and RB = rb are compile-time constants); src.x non-null: the rows are
// loaded from real channel pairs instead of the field
template <typename C, int DIR, int N = 0, int RB = 0>
__global__ void __launch_bounds__(256) k_rows(C* data, const long long* off, int n_, int rb_, RadixPlan plan,
                                              const C* tw, RealPairs src) {
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = N ? N : n_, rb = N ? RB : rb_;
    const int nb = n / rb;
    const long long field = blockIdx.x / nb;
    const long long r0 = (long long)(blockIdx.x % nb) * rb * n;
    C* p = data + (off ? off[field] : field * n * n) + r0;
    const int cnt = rb * n;
    if (src.x) {
        const int P = (src.ci + 1) / 2;
        const long long b = field / P, j = field - b * P, np = (long long)n * n;
        const float* re = src.x + (b * src.ci + 2 * j) * np + r0;
        const bool has_im = 2 * j + 1 < src.ci;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            C v;
            v.x = re[e];
            v.y = has_im ? re[np + e] : 0.f;
            sm[e] = v;
        }
    } else {
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) sm[e] = p[e];
    }
    __syncthreads();
    C* res = tile<C, N, RB, 1, N, DIR, false>(sm, sm + kTile, plan, rb, 1, n, tw);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) p[e] = res[e];
}

// cb columns of one field per block, the transform along each column; only
// the first nlo and the last nhi column blocks of every field (all of them
// when nlo + nhi covers the field)
template <typename C, int DIR, int N = 0, int CB = 0>
__global__ void __launch_bounds__(256) k_cols(C* data, const long long* off, int n_, int cb_, RadixPlan plan,
                                              const C* tw, int nlo, int nhi) {
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = N ? N : n_, cb = N ? CB : cb_;
    const int nb = n / cb, nsel = nlo + nhi;
    const long long field = blockIdx.x / nsel;
    const int bi = (int)(blockIdx.x % nsel);
    const int blk = bi < nlo ? bi : nb - nhi + (bi - nlo);
    C* p = data + (off ? off[field] : field * n * n) + (long long)blk * cb;
    const int cnt = cb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        sm[e] = p[(long long)i * n + b];
    }
    __syncthreads();
    C* res = tile<C, N, CB, CB, 1, DIR, true>(sm, sm + kTile, plan, cb, cb, 1, tw);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        p[(long long)i * n + b] = res[e];
    }
}

inline int largest_divisor_at_most(int n, int lim) {
    for (int d = std::min(n, lim); d >= 1; --d)
        if (n % d == 0) return d;
    return 1;
}

template <typename C, int N, int RB, int CB> inline cudaError_t set_attrs_one() {
    const int sm = (int)(2 * kTile * sizeof(C));
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_rows<C, -1, N, RB>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows<C, 1, N, RB>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<C, -1, N, CB>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<C, 1, N, CB>, at, sm);
    return e;
}

// compile-time sides (float32 only): 64, 128 and 256 with rb = min(n, kTile / n), cb = 16
template <typename C> inline cudaError_t set_attrs_of() {
    cudaError_t e = set_attrs_one<C, 0, 0, 0>();
    if constexpr (std::is_same<C, float2>::value) {
        if (e == cudaSuccess) e = set_attrs_one<C, 64, 64, 16>();
        if (e == cudaSuccess) e = set_attrs_one<C, 128, 32, 16>();
        if (e == cudaSuccess) e = set_attrs_one<C, 256, 16, 16>();
    }
    return e;
}

inline cudaError_t set_attrs() { return set_attrs_of<float2>(); }

// Forward: rows, then the selected column blocks.  Inverse: the selected
// column blocks first (the others must hold zeros), then rows.  The two
// orders give the same 2D transform where every column is transformed.
template <typename C, int N, int RB, int CB>
inline void launch(C* data, const long long* off, long long fields, int n, int rb, int cb, int dir, int nlo,
                   int nhi, const RadixPlan& plan, const C* tw, cudaStream_t st, RealPairs src) {
    const size_t sm = 2 * kTile * sizeof(C);
    const unsigned gr = (unsigned)(fields * (n / rb)), gc = (unsigned)(fields * (nlo + nhi));
    if (dir < 0) {
        k_rows<C, -1, N, RB><<<gr, 256, sm, st>>>(data, off, n, rb, plan, tw, src);
        k_cols<C, -1, N, CB><<<gc, 256, sm, st>>>(data, off, n, cb, plan, tw, nlo, nhi);
    } else {
        k_cols<C, 1, N, CB><<<gc, 256, sm, st>>>(data, off, n, cb, plan, tw, nlo, nhi);
        k_rows<C, 1, N, RB><<<gr, 256, sm, st>>>(data, off, n, rb, plan, tw, RealPairs{});
    }
}

// 2D transform of `fields` fields in place (dir < 0 forward, > 0 inverse).
// kx > 0: only columns 0 .. kx - 1 and n - kx + 1 .. n - 1 matter (the
// retained modes of a real field's half-plane spectrum and their mirrors):
// a forward transform computes those columns only (the others hold row
// spectra), an inverse one requires the others to be zero.  src (forward,
// float2 fields without offsets only): read the input from real channel pairs.
template <typename C>
inline cudaError_t run(C* data, const long long* off, long long fields, int n, int dir, const RadixPlan& plan,
                       const C* tw, cudaStream_t st, int kx = 0, RealPairs src = RealPairs{}) {
    const int rb = largest_divisor_at_most(n, kTile / n), cb = largest_divisor_at_most(n, std::min(16, kTile / n));
    const int nb = n / cb;
    int nlo = nb, nhi = 0;
    if (kx > 0) {
        const int lo = (kx + cb - 1) / cb, hi = (kx - 1 + cb - 1) / cb;
        if (lo + hi < nb) {
            nlo = lo;
            nhi = hi;
        }
    }
    if constexpr (std::is_same<C, float2>::value) {
        if (n == 64 && rb == 64 && cb == 16) launch<C, 64, 64, 16>(data, off, fields, n, rb, cb, dir, nlo, nhi, plan, tw, st, src);
        else if (n == 128 && rb == 32 && cb == 16) launch<C, 128, 32, 16>(data, off, fields, n, rb, cb, dir, nlo, nhi, plan, tw, st, src);
        else if (n == 256 && rb == 16 && cb == 16) launch<C, 256, 16, 16>(data, off, fields, n, rb, cb, dir, nlo, nhi, plan, tw, st, src);
        else launch<C, 0, 0, 0>(data, off, fields, n, rb, cb, dir, nlo, nhi, plan, tw, st, src);
    } else {
        launch<C, 0, 0, 0>(data, off, fields, n, rb, cb, dir, nlo, nhi, plan, tw, st, RealPairs{});
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace fft2d
}  // namespace npbs
