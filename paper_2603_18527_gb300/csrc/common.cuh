// Shared definitions of the CUDA library: complex helpers, device-side batch
// descriptors, status plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/npbs.h"

namespace npbs {

template <typename R> struct cpx_t;
template <> struct cpx_t<float> { using type = float2; };
template <> struct cpx_t<double> { using type = double2; };
template <typename R> using cpx = typename cpx_t<R>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
    C c; c.x = a; c.y = b; return c;
}
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cmul_conj_b(C a, C b) {  // a * conj(b)
    return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
template <typename C> __device__ __forceinline__ decltype(C::x) cabs2(C a) { return a.x * a.x + a.y * a.y; }

// Largest supported transform length and the maximum number of radix passes.
constexpr int kMaxN = 1024;
constexpr int kMaxPass = 12;

// Radix schedule of one transform length: passes applied in order (Stockham,
// stride of already-combined sub-transforms Ns = product of earlier radices).
struct RadixPlan {
    int n;
    int npass;
    int radix[kMaxPass];
};

// Device-side description of one instance of a batch.
struct InstDev {
    int nx, ny;
    int plan_x, plan_y;     // index into the plan table
    int tw_x, tw_y;         // element offset of the twiddle table for nx / ny
    double h, k0sq, eps;
    long long offset;       // first element in every field buffer
};

// Work items: a band of rows or a band of columns of one instance.
struct RowItem { int inst, row0, nrows, pad; };
struct ColItem { int inst, col0, ncols, pad; };
// A contiguous chunk of one instance for pointwise / reduction kernels.
struct VecItem { int inst, start, len, pad; };
constexpr int kVecChunk = 8192;

// Everything a launch needs to know about a batch (all device pointers).
struct BatchDev {
    const InstDev* inst;
    const RadixPlan* plans;
    const float2* tw32;      // W_N^k = exp(-2 pi i k / N), per distinct N
    const float4* twds;      // the same in double-single (re hi, re lo, im hi, im lo): float64 refresh
    const RowItem* rows;
    const ColItem* cols;
    const int* active;       // nullable: per-instance mask (0 = skip)
    int count;
};

}  // namespace npbs
