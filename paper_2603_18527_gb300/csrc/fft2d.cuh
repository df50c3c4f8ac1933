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

#include "fft.cuh"

namespace npbs {
namespace fft2d {
namespace {

constexpr int kTile = 4096;

// rb rows of one field per block, the transform along each row
template <typename C, int DIR>
__global__ void __launch_bounds__(256) k_rows(C* data, const long long* off, int n, int rb, RadixPlan plan,
                                              const C* tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int nb = n / rb;
    const long long field = blockIdx.x / nb;
    C* p = data + (off ? off[field] : field * n * n) + (long long)(blockIdx.x % nb) * rb * n;
    const int cnt = rb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) sm[e] = p[e];
    __syncthreads();
    C* res = fft_tile<C, DIR, false>(sm, sm + kTile, plan, rb, 1, n, tw, threadIdx.x, blockDim.x);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) p[e] = res[e];
}

// cb columns of one field per block, the transform along each column
template <typename C, int DIR>
__global__ void __launch_bounds__(256) k_cols(C* data, const long long* off, int n, int cb, RadixPlan plan,
                                              const C* tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int nb = n / cb;
    const long long field = blockIdx.x / nb;
    C* p = data + (off ? off[field] : field * n * n) + (long long)(blockIdx.x % nb) * cb;
    const int cnt = cb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        sm[e] = p[(long long)i * n + b];
    }
    __syncthreads();
    C* res = fft_tile<C, DIR, true>(sm, sm + kTile, plan, cb, cb, 1, tw, threadIdx.x, blockDim.x);
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

template <typename C> inline cudaError_t set_attrs_of() {
    const int sm = (int)(2 * kTile * sizeof(C));
    cudaError_t e = cudaFuncSetAttribute(k_rows<C, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<C, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

inline cudaError_t set_attrs() { return set_attrs_of<float2>(); }

// 2D transform of `fields` fields in place (dir < 0 forward, > 0 inverse)
template <typename C>
inline cudaError_t run(C* data, const long long* off, long long fields, int n, int dir, const RadixPlan& plan,
                       const C* tw, cudaStream_t st) {
    const int rb = largest_divisor_at_most(n, kTile / n), cb = largest_divisor_at_most(n, std::min(16, kTile / n));
    const size_t sm = 2 * kTile * sizeof(C);
    if (dir < 0) {
        k_rows<C, -1><<<(unsigned)(fields * (n / rb)), 256, sm, st>>>(data, off, n, rb, plan, tw);
        k_cols<C, -1><<<(unsigned)(fields * (n / cb)), 256, sm, st>>>(data, off, n, cb, plan, tw);
    } else {
        k_rows<C, 1><<<(unsigned)(fields * (n / rb)), 256, sm, st>>>(data, off, n, rb, plan, tw);
        k_cols<C, 1><<<(unsigned)(fields * (n / cb)), 256, sm, st>>>(data, off, n, cb, plan, tw);
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace fft2d
}  // namespace npbs
