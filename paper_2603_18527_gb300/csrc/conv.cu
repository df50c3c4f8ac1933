// BF16 implicit-GEMM 3x3 convolutions (forward / data gradient via the forward
// kernel with transformed weights / weight gradient) on the warp-level tensor
// core MMA (m16n8k16, float32 accumulate), cp.async double buffering and
// ldmatrix fragment loads.
#include <atomic>
#include <cstdlib>
#include <cstring>

#include "conv.cuh"

namespace npbs {

namespace {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm4(uint32_t a, uint32_t* r) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t a, uint32_t* r) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// Source element offset of input pixel (b, iy, ix) of an output-resolution
// tap, or -1 outside the zero-padded image.
__device__ __forceinline__ long long gather_off(int b, int iy, int ix, int H, int W, int ups, int xs) {
    if (iy < 0 || iy >= H || ix < 0 || ix >= W) return -1;
    if (ups) {
        const int Hi = H >> 1, Wi = W >> 1;
        return (((long long)b * Hi + (iy >> 1)) * Wi + (ix >> 1)) * xs;
    }
    return (((long long)b * H + iy) * W + ix) * xs;
}

constexpr int kBM = 128;
constexpr int kConvThreads = 256;

template <int BN, int BK>
__global__ void __launch_bounds__(kConvThreads) k_conv_fwd(ConvFwd a) {
    constexpr int LDA = BK + 8, LDB = BK + 8;
    constexpr int CPP = BK / 8;                 // 16-byte chunks per pixel row
    constexpr int APT = kBM * CPP / kConvThreads;  // A chunks per thread (1 or 2)
    constexpr int WN = BN / 2, NI = WN / 8;
    __shared__ __align__(128) bf16 As[2][kBM * LDA];
    __shared__ __align__(128) bf16 Bs[2][BN * LDB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm0 = (warp & 3) * 32, wn0 = (warp >> 2) * WN;
    const long long M = (long long)a.B * a.H * a.W;
    const long long m0 = (long long)blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const int nck = a.Cin / BK;
    const int KT = 9 * nck;

    int pb[APT], py[APT], px[APT], ppart[APT], prow[APT];
    bool pv[APT];
#pragma unroll
    for (int i = 0; i < APT; ++i) {
        const int id = tid + i * kConvThreads;
        prow[i] = id / CPP;
        ppart[i] = id % CPP;
        const long long p = m0 + prow[i];
        pv[i] = p < M;
        const long long pp = pv[i] ? p : 0;
        px[i] = (int)(pp % a.W);
        const long long t = pp / a.W;
        py[i] = (int)(t % a.H);
        pb[i] = (int)(t / a.H);
    }

    auto load = [&](int stage, int kt) {
        const int tap = kt / nck, c0 = (kt % nck) * BK;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int i = 0; i < APT; ++i) {
            long long off = pv[i] ? gather_off(pb[i], py[i] + dy, px[i] + dx, a.H, a.W, a.ups, a.xs) : -1;
            const bf16* src = off >= 0 ? a.x + off + a.xo + c0 + ppart[i] * 8 : a.x;
            cp16(su32(&As[stage][prow[i] * LDA + ppart[i] * 8]), src, off >= 0 ? 16 : 0);
        }
        for (int id = tid; id < BN * CPP; id += kConvThreads) {
            const int row = id / CPP, part = id % CPP;
            const int n = n0 + row;
            const bool ok = n < a.Cout;
            const bf16* src = ok ? a.w + ((long long)n * 9 + tap) * a.Cin + c0 + part * 8 : a.w;
            cp16(su32(&Bs[stage][row * LDB + part * 8]), src, ok ? 16 : 0);
        }
    };

    float acc[2][NI][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    load(0, 0);
    cp_commit();
    for (int kt = 0; kt < KT; ++kt) {
        if (kt + 1 < KT) load((kt + 1) & 1, kt + 1);
        cp_commit();
        cp_wait1();
        __syncthreads();
        const bf16* as = As[kt & 1];
        const bf16* bs = Bs[kt & 1];
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
            uint32_t af[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int row = wm0 + mi * 16 + (lane & 15);
                const int col = kk * 16 + (lane >> 4) * 8;
                ldsm4(su32(&as[row * LDA + col]), af[mi]);
            }
#pragma unroll
            for (int nj = 0; nj < NI / 2; ++nj) {
                uint32_t bf[4];
                const int row = wn0 + nj * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int col = kk * 16 + ((lane >> 3) & 1) * 8;
                ldsm4(su32(&bs[row * LDB + col]), bf);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    mma(acc[mi][2 * nj], af[mi], bf[0], bf[1]);
                    mma(acc[mi][2 * nj + 1], af[mi], bf[2], bf[3]);
                }
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long p = m0 + wm0 + mi * 16 + (lane >> 2) + h * 8;
                const int n = n0 + wn0 + ni * 8 + (lane & 3) * 2;
                if (p >= M || n >= a.Cout) continue;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (a.bias) {
                    v0 += a.bias[n];
                    v1 += a.bias[n + 1];
                }
                const long long o = p * a.ys + a.yo + n;
                if (a.yf) {
                    *reinterpret_cast<float2*>(a.yf + o) = make_float2(v0, v1);
                    continue;
                }
                if (a.z) *reinterpret_cast<__nv_bfloat162*>(a.z + o) = __floats2bfloat162_rn(v0, v1);
                if (a.act) {
                    v0 = gelu(v0);
                    v1 = gelu(v1);
                }
                *reinterpret_cast<__nv_bfloat162*>(a.y + o) = __floats2bfloat162_rn(v0, v1);
            }
}

template <int BM>
__global__ void __launch_bounds__(kConvThreads) k_conv_wgrad(ConvWgrad a) {
    constexpr int BN = 64, BK = 32;
    constexpr int LDA = BM + 8, LDB = BN + 8;
    constexpr int MI = BM / 32;  // m16 tiles per warp (2 warps along M)
    __shared__ __align__(128) bf16 As[2][BK * LDA];
    __shared__ __align__(128) bf16 Bs[2][BK * LDB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm0 = (warp & 1) * (BM / 2), wn0 = (warp >> 1) * 16;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const long long P = (long long)a.B * a.H * a.W;
    const long long pbeg = (long long)blockIdx.z * a.pix_per_cta;
    const long long pend = min(P, pbeg + a.pix_per_cta);
    const int NT = 9 * a.Cin;
    if (pbeg >= pend) return;
    const int KT = (int)((pend - pbeg + BK - 1) / BK);

    auto load = [&](int stage, int kt) {
        const long long p0 = pbeg + (long long)kt * BK;
        for (int id = tid; id < BK * (BM / 8); id += kConvThreads) {
            const int pix = id / (BM / 8), part = id % (BM / 8);
            const long long p = p0 + pix;
            const int m = m0 + part * 8;
            const bool ok = p < pend && m < a.Cout;
            const bf16* src = ok ? a.dz + p * a.Cout + m : a.dz;
            cp16(su32(&As[stage][pix * LDA + part * 8]), src, ok ? 16 : 0);
        }
        {
            const int id = tid;  // BK * BN / 8 == 256 chunks
            const int pix = id / (BN / 8), part = id % (BN / 8);
            const long long p = p0 + pix;
            const int n = n0 + part * 8;
            long long off = -1;
            if (p < pend && n < NT) {
                const int tap = n / a.Cin, ci = n % a.Cin;
                const int xx = (int)(p % a.W);
                const long long t = p / a.W;
                const int yy = (int)(t % a.H), bb = (int)(t / a.H);
                off = gather_off(bb, yy + tap / 3 - 1, xx + tap % 3 - 1, a.H, a.W, a.ups, a.xs);
                if (off >= 0) off += a.xo + ci;
            }
            cp16(su32(&Bs[stage][pix * LDB + part * 8]), off >= 0 ? a.x + off : a.x, off >= 0 ? 16 : 0);
        }
    };

    float acc[MI][2][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    load(0, 0);
    cp_commit();
    for (int kt = 0; kt < KT; ++kt) {
        if (kt + 1 < KT) load((kt + 1) & 1, kt + 1);
        cp_commit();
        cp_wait1();
        __syncthreads();
        const bf16* as = As[kt & 1];
        const bf16* bs = Bs[kt & 1];
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
            uint32_t af[MI][4];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                const int k = kk * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int m = wm0 + mi * 16 + ((lane >> 3) & 1) * 8;
                ldsm4t(su32(&as[k * LDA + m]), af[mi]);
            }
            uint32_t bf[4];
            {
                const int k = kk * 16 + (lane & 7) + (((lane >> 3) & 1) << 3);
                const int n = wn0 + (lane >> 4) * 8;
                ldsm4t(su32(&bs[k * LDB + n]), bf);
            }
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                mma(acc[mi][0], af[mi], bf[0], bf[1]);
                mma(acc[mi][1], af[mi], bf[2], bf[3]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm0 + mi * 16 + (lane >> 2) + h * 8;
                const int n = n0 + wn0 + ni * 8 + (lane & 3) * 2;
                if (m >= a.Cout || n >= NT) continue;
                atomicAdd(a.dw + (long long)m * NT + n, acc[mi][ni][2 * h]);
                atomicAdd(a.dw + (long long)m * NT + n + 1, acc[mi][ni][2 * h + 1]);
            }
}

}  // namespace

std::atomic<long long> g_conv_tc_launches{0}, g_conv_mma_launches{0};

cudaError_t conv_fwd(const ConvFwd& a, cudaStream_t st) {
    const long long M = (long long)a.B * a.H * a.W;
    if (M == 0) return cudaSuccess;
    const char* force = getenv("NPBS_CONV");
    if (!(force && strcmp(force, "mma") == 0) && conv_tc_supported(a)) {
        g_conv_tc_launches++;
        return conv_fwd_tc(a, st);
    }
    g_conv_mma_launches++;
    if (a.Cin % 16 || a.Cout % 8 || a.xs % 8 || a.xo % 8 || a.ys % 2 || a.yo % 2) return cudaErrorInvalidValue;
    const unsigned gm = (unsigned)((M + kBM - 1) / kBM);
    const bool bk32 = a.Cin % 32 == 0;
    if (a.Cout > 32) {
        dim3 g(gm, (a.Cout + 63) / 64);
        if (bk32) k_conv_fwd<64, 32><<<g, kConvThreads, 0, st>>>(a);
        else k_conv_fwd<64, 16><<<g, kConvThreads, 0, st>>>(a);
    } else {
        dim3 g(gm, 1);
        if (bk32) k_conv_fwd<32, 32><<<g, kConvThreads, 0, st>>>(a);
        else k_conv_fwd<32, 16><<<g, kConvThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t conv_wgrad(const ConvWgrad& a, cudaStream_t st) {
    const long long P = (long long)a.B * a.H * a.W;
    if (P == 0) return cudaSuccess;
    const char* force = getenv("NPBS_WGRAD");
    if (!(force && strcmp(force, "mma") == 0) && conv_wgrad_tc_supported(a)) {
        g_conv_tc_launches++;
        return conv_wgrad_tc(a, st);
    }
    g_conv_mma_launches++;
    if (a.Cin % 8 || a.Cout % 8 || a.xs % 8 || a.xo % 8 || a.pix_per_cta <= 0) return cudaErrorInvalidValue;
    const unsigned gz = (unsigned)((P + a.pix_per_cta - 1) / a.pix_per_cta);
    const int NT = 9 * a.Cin;
    if (a.Cout > 32) {
        dim3 g((NT + 63) / 64, (a.Cout + 63) / 64, gz);
        k_conv_wgrad<64><<<g, kConvThreads, 0, st>>>(a);
    } else {
        dim3 g((NT + 63) / 64, (a.Cout + 31) / 32, gz);
        k_conv_wgrad<32><<<g, kConvThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace npbs

extern "C" void npbs_conv_stats(int64_t* tensor_core_launches, int64_t* warp_mma_launches) {
    if (tensor_core_launches) *tensor_core_launches = npbs::g_conv_tc_launches.load();
    if (warp_mma_launches) *warp_mma_launches = npbs::g_conv_mma_launches.load();
}
