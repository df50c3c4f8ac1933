// Batched 2D complex FFTs of square n x n fields for the parts of the library
// that run plain transforms (the FNO's Fourier layers, the CDR operators):
// a row kernel and a column kernel of radix-2/3/4/8 Stockham passes in shared
// memory (fft.cuh), forward unnormalised, inverse without the 1/n^2 factor.
// Field i of a call starts at data + off[i] (or at data + i n^2 when off is
// null).  Two tile buffers of kTile complex elements per block (64 KB of
// dynamic shared memory: set_attrs() opts the kernels in).
#pragma once

#include <algorithm>

#include "fft.cuh"

namespace npbs {
namespace fft2d {
namespace {

constexpr int kTile = 4096;

// rb rows of one field per block, the transform along each row
template <int DIR>
__global__ void __launch_bounds__(256) k_rows(float2* data, const long long* off, int n, int rb, RadixPlan plan,
                                              const float2* tw) {
    extern __shared__ __align__(16) float2 sm[];
    const int nb = n / rb;
    const long long field = blockIdx.x / nb;
    float2* p = data + (off ? off[field] : field * n * n) + (long long)(blockIdx.x % nb) * rb * n;
    const int cnt = rb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) sm[e] = p[e];
    __syncthreads();
    float2* res = fft_tile<float2, DIR, false>(sm, sm + kTile, plan, rb, 1, n, tw, threadIdx.x, blockDim.x);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) p[e] = res[e];
}

// cb columns of one field per block, the transform along each column
template <int DIR>
__global__ void __launch_bounds__(256) k_cols(float2* data, const long long* off, int n, int cb, RadixPlan plan,
                                              const float2* tw) {
    extern __shared__ __align__(16) float2 sm[];
    const int nb = n / cb;
    const long long field = blockIdx.x / nb;
    float2* p = data + (off ? off[field] : field * n * n) + (long long)(blockIdx.x % nb) * cb;
    const int cnt = cb * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / cb, b = e - i * cb;
        sm[e] = p[(long long)i * n + b];
    }
    __syncthreads();
    float2* res = fft_tile<float2, DIR, true>(sm, sm + kTile, plan, cb, cb, 1, tw, threadIdx.x, blockDim.x);
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

inline cudaError_t set_attrs() {
    const int sm = (int)(2 * kTile * sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(k_rows<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cols<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

// 2D transform of `fields` fields in place (dir < 0 forward, > 0 inverse)
inline cudaError_t run(float2* data, const long long* off, long long fields, int n, int dir, const RadixPlan& plan,
                       const float2* tw, cudaStream_t st) {
    const int rb = largest_divisor_at_most(n, kTile / n), cb = largest_divisor_at_most(n, std::min(16, kTile / n));
    const size_t sm = 2 * kTile * sizeof(float2);
    if (dir < 0) {
        k_rows<-1><<<(unsigned)(fields * (n / rb)), 256, sm, st>>>(data, off, n, rb, plan, tw);
        k_cols<-1><<<(unsigned)(fields * (n / cb)), 256, sm, st>>>(data, off, n, cb, plan, tw);
    } else {
        k_rows<1><<<(unsigned)(fields * (n / rb)), 256, sm, st>>>(data, off, n, rb, plan, tw);
        k_cols<1><<<(unsigned)(fields * (n / cb)), 256, sm, st>>>(data, off, n, cb, plan, tw);
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace fft2d
}  // namespace npbs
