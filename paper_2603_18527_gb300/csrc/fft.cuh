// Mixed-radix (2, 3, 4, 8) Stockham FFT passes on shared-memory tiles.
//
// A tile holds `nbatch` independent transforms of length N; element i of
// transform b sits at tile[i * si + b * sb].  Row tiles (transforms along a
// contiguous grid row) use si = 1; column tiles use sb = 1 so that adjacent
// threads touch adjacent columns.  Each pass reads R values at stride N/R,
// multiplies by the twiddles W_{Ns R}^{r k}, does a length-R DFT in registers
// and writes the autosorted result at stride Ns into the other buffer, so the
// output of the last pass is in natural order (Stockham autosort).  Forward
// transforms use W = exp(-2 pi i / N) (DIR = -1), inverse ones its conjugate
// (DIR = +1) without the 1/N factor.  Twiddles come from tables computed on the
// host in double precision.
#pragma once

#include "common.cuh"

namespace npbs {

// x * (DIR * i): multiply by +i (DIR = +1) or -i (DIR = -1).
template <int DIR, typename C> __host__ __device__ __forceinline__ C mul_i(C a) {
    return DIR > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

template <int R, int DIR, typename C> struct Dft;

template <int DIR, typename C> struct Dft<2, DIR, C> {
    static __host__ __device__ __forceinline__ void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
};

template <int DIR, typename C> struct Dft<4, DIR, C> {
    static __host__ __device__ __forceinline__ void run(C* v) {
        C t0 = v[0] + v[2], t1 = v[0] - v[2];
        C t2 = v[1] + v[3], t3 = mul_i<DIR>(v[1] - v[3]);
        v[0] = t0 + t2;
        v[2] = t0 - t2;
        v[1] = t1 + t3;
        v[3] = t1 - t3;
    }
};

template <int DIR, typename C> struct Dft<8, DIR, C> {
    static __host__ __device__ __forceinline__ void run(C* v) {
        using S = decltype(C::x);
        const S h = S(0.70710678118654752440);  // sqrt(2)/2
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, DIR, C>::run(e);
        Dft<4, DIR, C>::run(o);
        // w8^q o_q with w8 = exp(DIR 2 pi i / 8)
        C o1 = mk<C>(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
        C o2 = mul_i<DIR>(o[2]);
        C o3 = mk<C>(h * (-o[3].x - DIR * o[3].y), h * (-o[3].y + DIR * o[3].x));
        v[0] = e[0] + o[0];
        v[4] = e[0] - o[0];
        v[1] = e[1] + o1;
        v[5] = e[1] - o1;
        v[2] = e[2] + o2;
        v[6] = e[2] - o2;
        v[3] = e[3] + o3;
        v[7] = e[3] - o3;
    }
};

template <int DIR, typename C> struct Dft<3, DIR, C> {
    static __host__ __device__ __forceinline__ void run(C* v) {
        using S = decltype(C::x);
        const S s3 = S(0.86602540378443864676);  // sqrt(3)/2
        C t = v[1] + v[2];
        C d = v[1] - v[2];
        C m = mk<C>(v[0].x - S(0.5) * t.x, v[0].y - S(0.5) * t.y);
        C j = mul_i<DIR>(mk<C>(s3 * d.x, s3 * d.y));
        v[0] = v[0] + t;
        v[1] = m + j;
        v[2] = m - j;
    }
};

// One Stockham pass of radix RAD over every transform of the tile.
template <typename C, int RAD, int DIR, bool COLS>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ in, C* __restrict__ out, int N, int Ns,
                                              int nbatch, int si, int sb, const C* __restrict__ tw,
                                              int tid, int nth) {
    const int nb = N / RAD;
    const int total = nb * nbatch;
    const int twstep = N / (Ns * RAD);
    for (int w = tid; w < total; w += nth) {
        int b, j;
        if (COLS) {
            b = w % nbatch;
            j = w / nbatch;
        } else {
            j = w % nb;
            b = w / nb;
        }
        const int k = j % Ns;
        C v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[r] = in[(j + r * nb) * si + b * sb];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                C t = tw[r * k * twstep];
                if (DIR > 0) t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        Dft<RAD, DIR, C>::run(v);
        const int d = (j / Ns) * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) out[(d + r * Ns) * si + b * sb] = v[r];
    }
}

// Full transform of a tile; returns the buffer holding the result (a or b).
// Ends with a __syncthreads(), so the result is visible to the whole block.
template <typename C, int DIR, bool COLS>
__device__ C* fft_tile(C* a, C* b, const RadixPlan& p, int nbatch, int si, int sb, const C* __restrict__ tw,
                       int tid, int nth) {
    int Ns = 1;
    const int N = p.n;
    for (int s = 0; s < p.npass; ++s) {
        const int R = p.radix[s];
        switch (R) {
            case 8: stockham_pass<C, 8, DIR, COLS>(a, b, N, Ns, nbatch, si, sb, tw, tid, nth); break;
            case 4: stockham_pass<C, 4, DIR, COLS>(a, b, N, Ns, nbatch, si, sb, tw, tid, nth); break;
            case 3: stockham_pass<C, 3, DIR, COLS>(a, b, N, Ns, nbatch, si, sb, tw, tid, nth); break;
            default: stockham_pass<C, 2, DIR, COLS>(a, b, N, Ns, nbatch, si, sb, tw, tid, nth); break;
        }
        __syncthreads();
        C* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Compile-time variants: the length, the pass stride and the tile geometry are
// template constants, so the index arithmetic of every pass compiles to
// shifts and multiplies.  Same radix order as the run-time plans (8s, then
// 4, 2, 3) and the same length-N twiddle table.
template <typename C, int RAD, int DIR, bool COLS, int N, int NS, int NB, int SI, int SB>
__device__ __forceinline__ void stockham_pass_ct(const C* __restrict__ in, C* __restrict__ out,
                                                 const C* __restrict__ tw, int tid, int nth) {
    constexpr int nb = N / RAD;
    constexpr int total = nb * NB;
    constexpr int twstep = N / (NS * RAD);
    for (int w = tid; w < total; w += nth) {
        int b, j;
        if (COLS) {
            b = w % NB;
            j = w / NB;
        } else {
            j = w % nb;
            b = w / nb;
        }
        const int k = j % NS;
        C v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[r] = in[(j + r * nb) * SI + b * SB];
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                C t = tw[r * k * twstep];
                if (DIR > 0) t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        Dft<RAD, DIR, C>::run(v);
        const int d = (j / NS) * NS * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) out[(d + r * NS) * SI + b * SB] = v[r];
    }
}

template <int M> struct NextRadix {
    static constexpr int value = M % 8 == 0 ? 8 : M % 4 == 0 ? 4 : M % 2 == 0 ? 2 : 3;
};

// The transform of a tile with compile-time geometry (NB transforms of length
// N, element i of transform b at tile[i * SI + b * SB]); returns the buffer
// holding the result and ends with a __syncthreads().
template <typename C, int DIR, bool COLS, int N, int NB, int SI, int SB, int NS = 1>
__device__ __forceinline__ C* fft_tile_ct(C* a, C* b, const C* __restrict__ tw, int tid, int nth) {
    if constexpr (NS >= N) {
        return a;
    } else {
        constexpr int R = NextRadix<N / NS>::value;
        stockham_pass_ct<C, R, DIR, COLS, N, NS, NB, SI, SB>(a, b, tw, tid, nth);
        __syncthreads();
        return fft_tile_ct<C, DIR, COLS, N, NB, SI, SB, NS * R>(b, a, tw, tid, nth);
    }
}

// Signed mode of DFT index i for length N: 0..ceil(N/2)-1, then negative
// (the Nyquist index of an even N maps to -N/2).
__device__ __forceinline__ int signed_mode(int i, int N) { return i < (N + 1) / 2 ? i : i - N; }

}  // namespace npbs
