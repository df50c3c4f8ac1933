// Register-resident DFTs of small composite lengths (6, 8, 9, 12, 16, 18, 24,
// 32, ...) with compile-time roots of unity.
//
// DftR<R, DIR>::run(v) replaces v[0..R) by X[k] = sum_n v[n] exp(DIR 2 pi i n k / R)
// in natural order.  Composite R = A * B is split Cooley-Tukey style
// (n = B n1 + n2, k = k1 + A k2): B DFTs of length A over stride-B elements,
// twiddles W_R^{n2 k1}, then A DFTs of length B.  Every index is a compile-time
// constant, so the arrays live in registers and the twiddles are immediates.
#pragma once

#include <type_traits>
#include <utility>

#include "fft.cuh"

namespace npbs {

namespace cx {
constexpr double kPi = 3.14159265358979323846264338327950288;
// Taylor series after reduction to [-pi, pi]; exact to double rounding there.
constexpr double sin_t(double x) {
    double t = x, s = x;
    for (int n = 1; n < 32; ++n) {
        t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        s += t;
    }
    return s;
}
constexpr double cos_t(double x) {
    double t = 1.0, s = 1.0;
    for (int n = 1; n < 32; ++n) {
        t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        s += t;
    }
    return s;
}
}  // namespace cx

// exp(2 pi i K / R) split into cos and sin (float)
template <int R, int K> struct Root {
    static constexpr int k = ((K % R) + R) % R;
    static constexpr double ang0 = 2.0 * cx::kPi * (double)k / (double)R;
    static constexpr double ang = ang0 > cx::kPi ? ang0 - 2.0 * cx::kPi : ang0;
    static constexpr float c = (float)cx::cos_t(ang);
    static constexpr float s = (float)cx::sin_t(ang);
};

template <typename F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F> __host__ __device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// x * exp(DIR 2 pi i K / R)
template <int R, int K, int DIR> __host__ __device__ __forceinline__ float2 twid(float2 x) {
    if constexpr (((K % R) + R) % R == 0) {
        return x;
    } else {
        constexpr float c = Root<R, K>::c;
        constexpr float s = DIR * Root<R, K>::s;
        return make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
    }
}

template <int R> struct Factor {
    static constexpr int A = (R % 8 == 0 && R > 8) ? 8 : (R % 4 == 0 && R > 4) ? 4 : (R % 3 == 0 && R > 3) ? 3 : 2;
    static constexpr int B = R / A;
};

template <int R, int DIR> struct DftR {
    static __host__ __device__ __forceinline__ void run(float2* v) {
        if constexpr (R == 1) {
        } else if constexpr (R == 2 || R == 3 || R == 4 || R == 8) {
            Dft<R, DIR, float2>::run(v);
        } else {
            constexpr int A = Factor<R>::A, B = Factor<R>::B;
            float2 y[R];
            static_for<B>([&](auto n2c) {
                constexpr int n2 = decltype(n2c)::value;
                float2 t[A];
                static_for<A>([&](auto n1c) {
                    constexpr int n1 = decltype(n1c)::value;
                    t[n1] = v[B * n1 + n2];
                });
                DftR<A, DIR>::run(t);
                static_for<A>([&](auto k1c) {
                    constexpr int k1 = decltype(k1c)::value;
                    y[k1 * B + n2] = twid<R, n2 * k1, DIR>(t[k1]);
                });
            });
            static_for<A>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                float2 t[B];
                static_for<B>([&](auto n2c) {
                    constexpr int n2 = decltype(n2c)::value;
                    t[n2] = y[k1 * B + n2];
                });
                DftR<B, DIR>::run(t);
                static_for<B>([&](auto k2c) {
                    constexpr int k2 = decltype(k2c)::value;
                    v[k1 + A * k2] = t[k2];
                });
            });
        }
    }
};

}  // namespace npbs
