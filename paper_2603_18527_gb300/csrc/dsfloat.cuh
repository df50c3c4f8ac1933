// Double-single ("float-float") arithmetic: a real number held as the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significant bits, computed on the FP32 pipes.  The operations are the
// error-free transformations of Knuth (two-sum: the exact rounding error of
// a + b from six additions) and of the fused multiply-add (two-product: the
// exact error of a * b is fma(a, b, -p)), followed by renormalisation, as in
// Dekker's 1971 double-length arithmetic.  The float64 refresh of the solvers
// (f - A u, the arbiter of rTol) runs its FFTs in this type: on GB300 the FP64
// rate is a small fraction of the FP32 rate, and 48 bits keep the residual of
// a solution converged to 1e-5 accurate to better than 1e-7 of itself.
#pragma once

#include "common.cuh"

namespace npbs {

struct dsf {
    float hi, lo;
    __host__ __device__ dsf() : hi(0.f), lo(0.f) {}
    __host__ __device__ dsf(float h, float l) : hi(h), lo(l) {}
    // nearest double-single to a double (exact for |x| in the float range)
    __host__ __device__ dsf(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ dsf(int x) : dsf((double)x) {}
};

__device__ __forceinline__ double to_double(dsf a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ dsf two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dsf(s, e);
}
// s + e = a + b exactly, given |a| >= |b|
__device__ __forceinline__ dsf quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dsf(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
    // both parts summed error-free, then renormalised twice (accurate under cancellation)
    dsf s = two_sum(a.hi, b.hi);
    const dsf t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }
__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ dsf operator/(dsf a, dsf b) {
    // q1 = a / b to float accuracy, then one correction from the remainder a - q1 b
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dsf r = a - b * dsf(q1, 0.f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return quick_two_sum(q1, q2);
}

struct dscpx {
    dsf x, y;
};
template <> struct cpx_t<dsf> { using type = dscpx; };
__device__ __forceinline__ dscpx operator+(dscpx a, dscpx b) { return dscpx{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dscpx operator-(dscpx a, dscpx b) { return dscpx{a.x - b.x, a.y - b.y}; }

// conversions at the edges of a transform
template <typename C> __device__ __forceinline__ C from_double2(double2 v);
template <> __device__ __forceinline__ double2 from_double2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ dscpx from_double2<dscpx>(double2 v) { return dscpx{dsf(v.x), dsf(v.y)}; }
__device__ __forceinline__ double to_double(double a) { return a; }

}  // namespace npbs
