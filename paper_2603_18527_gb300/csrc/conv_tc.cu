// 3x3 convolution (implicit GEMM) on the 5th-generation tensor cores:
// TMA loads of the shifted input tile and of the weights into swizzled shared
// memory, tcgen05.mma (BF16 x BF16 -> FP32) accumulating in tensor memory,
// tcgen05.ld for the bias / GELU / BF16 epilogue.
//
// One CTA computes a 128-pixel x Cout tile (Cout <= 256, all output channels,
// so each input tile is read once).  K = 9 taps x Cin in chunks of BK channels
// (BK = 64 with the 128-byte swizzle, or 32 / 16 for narrow inputs).  The
// 128 output pixels are a run of one image row (W >= 128) or whole rows
// (W < 128): for tap (dy, dx) the input tile is the same run shifted by
// (dy, dx), which a 4D TMA box [1][rows][cols][BK] at (c0, x0 + dx, y0 + dy, b)
// fetches with hardware zero fill outside the image (the convolution's zero
// padding).  Pipeline: 4 stages, thread 0 issues TMA, thread 32 issues MMAs
// and commits stage releases; all 128 threads (one warpgroup, TMEM lanes
// 0..127 = tile rows) run the epilogue.  Every mbarrier wait is bounded; a
// timeout sets g_conv_tc_timeout and the CTA cleans up and returns.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "conv.cuh"

namespace npbs {

__device__ int g_conv_tc_timeout = 0;

namespace {

constexpr int kStages = 4;
constexpr int kTM = 128;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and the global flag set) after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicExch(&g_conv_tc_timeout, 1);
            return false;
        }
    }
    return true;
}

// Exercises the bounded-wait path: thread 0 waits on an mbarrier that nothing
// arrives at, gives up after `limit` cycles and sets the timeout flag; the
// kernel then returns normally.
__global__ void k_wait_selftest(long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(su32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        (void)mbar_wait(su32(&bar), 0, limit);
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// K-major shared-memory matrix descriptor with swizzle (rows of `row_bytes`,
// 8-row atoms `8 * row_bytes` apart).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int row_bytes) {
    const uint64_t layout = row_bytes == 128 ? 2ull : row_bytes == 64 ? 4ull : 6ull;  // SW128 / SW64 / SW32
    const uint64_t sbo = (uint64_t)(8 * row_bytes) >> 4;
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;  // leading byte offset (unused for swizzled K-major)
    d |= (sbo & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    d |= layout << 61;
    return d;
}

// Instruction descriptor: BF16 x BF16 -> F32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(int n) {
    uint32_t d = 0;
    d |= 1u << 4;                      // D format F32
    d |= 1u << 7;                      // A format BF16
    d |= 1u << 10;                     // B format BF16
    d |= (uint32_t)(n >> 3) << 17;     // N / 8
    d |= (uint32_t)(kTM >> 4) << 24;   // M / 16
    return d;
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

struct TcArgs {
    int B, H, W, Cin, Cout, BK;   // H, W: the grid the 128-pixel tiles walk (half resolution for sub-pixel)
    int ntaps;                    // 9 (3x3) or 4 (2x2 sub-pixel convolution)
    int tdy[9], tdx[9];           // input offsets of each tap
    int sub, py, px, Ho, Wo;      // sub-pixel output: pixel (Y, X) of the tile grid -> (2Y + py, 2X + px) of Ho x Wo
    int rows_per_tile;      // output rows per 128-pixel tile (W < 128), else 1
    int tiles_per_row;      // W / 128 when W >= 128, else 1
    const float* bias;
    int act;
    bf16* y;
    bf16* z;
    float* yf;
    int ys, yo;
    int xo;                 // channel offset of the input slice
    int bn;                 // N of the MMA (Cout rounded up to 16)
    int tmem_cols;
    int halo;               // 1: halo rows (one per dy, shared by the three dx taps), see k_conv_tc_persist
};

// Halo mode: one TMA box of kHaloRows pixels (x0 - 4 .. x0 + 131) x 8 channels
// per dy row and 8-channel slice of a K chunk, unswizzled, so that the A
// operand of tap dx starts at pixel row 4 + dx of the box (16-byte steps).
constexpr int kHaloRows = 136;

// K-major shared-memory descriptor without swizzle: 8-row x 16-byte core
// matrices, `lbo` bytes apart along K, `sbo` bytes apart along M / N.
__device__ __forceinline__ uint64_t smem_desc_nosw(uint32_t addr, int lbo, int sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(((uint32_t)lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(((uint32_t)sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; layout type 0 = no swizzle
    return d;
}

__global__ void __launch_bounds__(128, 1) k_conv_tc(const __grid_constant__ CUtensorMap mapx,
                                                    const __grid_constant__ CUtensorMap mapw, TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage buffers (swizzle atoms), then barriers
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int a_bytes = kTM * a.BK * 2;
    const int b_bytes = a.bn * a.BK * 2;
    const int stage_bytes = a_bytes + b_bytes;
    unsigned char* stage0 = base;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kStages * stage_bytes);  // full[4], empty[4], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);

    const int tid = threadIdx.x, warp = tid >> 5;
    const long long m0 = (long long)blockIdx.x * kTM;
    // tile origin
    const long long HW = (long long)a.H * a.W;
    const int b = (int)(m0 / HW);
    const long long rem = m0 - (long long)b * HW;
    const int y0 = (int)(rem / a.W);
    const int x0 = (int)(rem % a.W);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(su32(&bars[s]), 1);
            mbar_init(su32(&bars[kStages + s]), 1);
        }
        mbar_init(su32(&bars[2 * kStages]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int nck = a.Cin / a.BK;
    const int KT = a.ntaps * nck;
    bool ok = true;
    if (tid == 0) {
        // TMA producer
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % kStages;
            if (kt >= kStages) ok = mbar_wait(su32(&bars[kStages + s]), ((kt / kStages) - 1) & 1);
            if (!ok) break;
            const int tap = kt / nck, c0 = (kt % nck) * a.BK;
            const int dy = a.tdy[tap], dx = a.tdx[tap];
            const uint32_t full = su32(&bars[s]);
            mbar_expect_tx(full, (uint32_t)stage_bytes);
            unsigned char* st = stage0 + s * stage_bytes;
            tma_load_4d(su32(st), &mapx, full, a.xo + c0, x0 + dx, y0 + dy, b);
            tma_load_2d(su32(st + a_bytes), &mapw, full, tap * a.Cin + c0, 0);
        }
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = instr_desc(a.bn);
        const int row_bytes = a.BK * 2;
        for (int kt = 0; kt < KT && ok; ++kt) {
            const int s = kt % kStages;
            ok = mbar_wait(su32(&bars[s]), (kt / kStages) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* st = stage0 + s * stage_bytes;
            const uint32_t abase = su32(st), bbase = su32(st + a_bytes);
            for (int kk = 0; kk < a.BK / 16; ++kk) {
                const uint64_t ad = smem_desc(abase + kk * 32, row_bytes);
                const uint64_t bd = smem_desc(bbase + kk * 32, row_bytes);
                umma(tmem, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(su32(&bars[kStages + s]));  // stage s free once these MMAs complete
        }
        umma_commit(su32(&bars[2 * kStages]));  // accumulator complete
    }
    __syncwarp();
    // epilogue: every thread owns one tile row (TMEM lane = tid)
    const bool done = mbar_wait(su32(&bars[2 * kStages]), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const long long q = m0 + tid;
    const long long P = (long long)a.B * HW;
    long long p = q;
    if (a.sub) {
        const int qb = (int)(q / HW);
        const long long qr = q - (long long)qb * HW;
        p = ((long long)qb * a.Ho + 2 * (qr / a.W) + a.py) * a.Wo + 2 * (qr % a.W) + a.px;
    }
    if (done) {
        for (int c = 0; c < a.bn; c += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (q >= P) continue;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                v[j] = __uint_as_float(r[j]);
                if (a.bias && c + j < a.Cout) v[j] += a.bias[c + j];
            }
            const long long o = p * a.ys + a.yo + c;
            if (a.yf) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    if (c + j < a.Cout) *reinterpret_cast<float4*>(a.yf + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                continue;
            }
            __align__(16) bf16 zb[16], yb[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                zb[j] = __float2bfloat16_rn(v[j]);
                yb[j] = __float2bfloat16_rn(a.act ? gelu(v[j]) : v[j]);
            }
            if (c + 16 <= a.Cout) {
                uint4* yd = reinterpret_cast<uint4*>(a.y + o);
                yd[0] = reinterpret_cast<uint4*>(yb)[0];
                yd[1] = reinterpret_cast<uint4*>(yb)[1];
                if (a.z) {
                    uint4* zd = reinterpret_cast<uint4*>(a.z + o);
                    zd[0] = reinterpret_cast<uint4*>(zb)[0];
                    zd[1] = reinterpret_cast<uint4*>(zb)[1];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}


// Persistent, warp-specialised variant: warps 0-3 drain TMEM (epilogue),
// warp 4 issues TMA, warp 5 issues MMAs.  Each CTA walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; the smem pipeline runs across tile
// boundaries and two TMEM accumulators let the epilogue of one tile overlap
// the MMAs of the next.
__global__ void __launch_bounds__(192, 1) k_conv_tc_persist(const __grid_constant__ CUtensorMap mapx,
                                                            const __grid_constant__ CUtensorMap mapw, TcArgs a,
                                                            int ntiles) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // halo mode: A = BK/8 boxes of 8 channels x kHaloRows pixels, B = the three
    // dx taps' weights for BK channels; K step = (dy, BK-channel chunk)
    const int a_bytes = a.halo ? (a.BK / 8) * kHaloRows * 16 : kTM * a.BK * 2;
    const int b_bytes = a.halo ? 3 * a.bn * a.BK * 2 : a.bn * a.BK * 2;
    const int stage_bytes = a_bytes + b_bytes;
    unsigned char* stage0 = base;
    // full[S], empty[S], tfull[2], tempty[2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + kStages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* tfull = bars + 2 * kStages;
    uint64_t* tempty = bars + 2 * kStages + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long HW = (long long)a.H * a.W;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(su32(&full[s]), 1);
            mbar_init(su32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(su32(&tfull[b]), 1);
            mbar_init(su32(&tempty[b]), 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int nck = a.Cin / a.BK;
    const int KT = a.halo ? 3 * nck : a.ntaps * nck;
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 4) {
        if (lane == 0) {
            bool ok = true;
            long long g = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const long long m0 = (long long)(blockIdx.x + (long long)i * gridDim.x) * kTM;
                const int b = (int)(m0 / HW);
                const long long rem = m0 - (long long)b * HW;
                const int y0 = (int)(rem / a.W), x0 = (int)(rem % a.W);
                for (int kt = 0; kt < KT && ok; ++kt, ++g) {
                    const int s = (int)(g % kStages);
                    if (g >= kStages) ok = mbar_wait(su32(&empty[s]), (uint32_t)(((g / kStages) - 1) & 1));
                    if (!ok) break;
                    mbar_expect_tx(su32(&full[s]), (uint32_t)stage_bytes);
                    unsigned char* st = stage0 + s * stage_bytes;
                    if (a.halo) {
                        const int dyi = kt / nck, c0 = (kt % nck) * a.BK;
                        for (int hh = 0; hh < a.BK / 8; ++hh)
                            tma_load_4d(su32(st + hh * kHaloRows * 16), &mapx, su32(&full[s]), a.xo + c0 + 8 * hh,
                                        x0 - 4, y0 + dyi - 1, b);
                        for (int dxi = 0; dxi < 3; ++dxi)
                            tma_load_2d(su32(st + a_bytes + dxi * a.bn * a.BK * 2), &mapw, su32(&full[s]),
                                        (3 * dyi + dxi) * a.Cin + c0, 0);
                    } else {
                        const int tap = kt / nck, c0 = (kt % nck) * a.BK;
                        tma_load_4d(su32(st), &mapx, su32(&full[s]), a.xo + c0, x0 + a.tdx[tap], y0 + a.tdy[tap], b);
                        tma_load_2d(su32(st + a_bytes), &mapw, su32(&full[s]), tap * a.Cin + c0, 0);
                    }
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(a.bn);
            const int row_bytes = a.BK * 2;
            bool ok = true;
            long long g = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int buf = i & 1;
                if (i >= 2) ok = mbar_wait(su32(&tempty[buf]), (uint32_t)(((i >> 1) - 1) & 1));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc_addr = tmem + (uint32_t)(buf * a.bn);
                for (int kt = 0; kt < KT && ok; ++kt, ++g) {
                    const int s = (int)(g % kStages);
                    ok = mbar_wait(su32(&full[s]), (uint32_t)((g / kStages) & 1));
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char* st = stage0 + s * stage_bytes;
                    const uint32_t abase = su32(st), bbase = su32(st + a_bytes);
                    if (a.halo) {
                        // tap dx = dxi - 1 reads pixel rows 3 + dxi .. 130 + dxi of the halo
                        // boxes; K sub-step kk takes boxes 2 kk and 2 kk + 1 (16 channels)
                        for (int dxi = 0; dxi < 3; ++dxi)
                            for (int kk = 0; kk < a.BK / 16; ++kk)
                                umma(acc_addr,
                                     smem_desc_nosw(abase + kk * 2 * kHaloRows * 16 + (3 + dxi) * 16, kHaloRows * 16, 128),
                                     smem_desc(bbase + dxi * a.bn * a.BK * 2 + kk * 32, row_bytes), idesc,
                                     (kt > 0 || dxi > 0 || kk > 0) ? 1u : 0u);
                    } else {
                        for (int kk = 0; kk < a.BK / 16; ++kk)
                            umma(acc_addr, smem_desc(abase + kk * 32, row_bytes), smem_desc(bbase + kk * 32, row_bytes),
                                 idesc, (kt > 0 || kk > 0) ? 1u : 0u);
                    }
                    umma_commit(su32(&empty[s]));
                }
                umma_commit(su32(&tfull[buf]));
            }
        }
    } else {
        // epilogue warps 0..3: TMEM lanes 32 * warp .. 32 * warp + 31
        const long long P = (long long)a.B * HW;
        for (int i = 0; i < my_tiles; ++i) {
            const int buf = i & 1;
            if (!mbar_wait(su32(&tfull[buf]), (uint32_t)((i >> 1) & 1))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long long q = (long long)(blockIdx.x + (long long)i * gridDim.x) * kTM + tid;
            long long p = q;
            if (a.sub) {
                const int qb = (int)(q / HW);
                const long long qr = q - (long long)qb * HW;
                p = ((long long)qb * a.Ho + 2 * (qr / a.W) + a.py) * a.Wo + 2 * (qr % a.W) + a.px;
            }
            for (int c = 0; c < a.bn; c += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * a.bn + c);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (q >= P) continue;
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]);
                    if (a.bias && c + j < a.Cout) v[j] += a.bias[c + j];
                }
                const long long o = p * a.ys + a.yo + c;
                if (a.yf) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        if (c + j < a.Cout)
                            *reinterpret_cast<float4*>(a.yf + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    continue;
                }
                __align__(16) bf16 zb[16], yb[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    zb[j] = __float2bfloat16_rn(v[j]);
                    yb[j] = __float2bfloat16_rn(a.act ? gelu(v[j]) : v[j]);
                }
                if (c + 16 <= a.Cout) {
                    uint4* yd = reinterpret_cast<uint4*>(a.y + o);
                    yd[0] = reinterpret_cast<uint4*>(yb)[0];
                    yd[1] = reinterpret_cast<uint4*>(yb)[1];
                    if (a.z) {
                        uint4* zd = reinterpret_cast<uint4*>(a.z + o);
                        zd[0] = reinterpret_cast<uint4*>(zb)[0];
                        zd[1] = reinterpret_cast<uint4*>(zb)[1];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tempty[buf])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------- weight gradient
//
// dW[n][tap][c] = sum_p x[nbr(p, tap)][c] * dz[p][n] as one GEMM per tap with
// K = pixels: D[m][n] = sum_k A[m][k] B[k][n], A = the tap-shifted input (m =
// input channel), B = dz (n = output channel).  Both operands sit in memory
// channel-contiguous per pixel, i.e. MN-major: a TMA box of 64 pixels x BC
// channels lands as 64 rows of 2*BC bytes, the canonical MN-major swizzled
// layout (8-row atoms SBO apart along K, BC-element blocks LBO apart along
// M/N), so no transpose is needed.  The 128 rows of one M-tile are 128/BC
// (tap, channel block) pairs: narrow inputs pack several taps into one MMA.
// A CTA owns MT M-tiles (accumulators side by side in TMEM, sharing each dz
// tile; the host uses MT = 1 so that two short pipelines share an SM) over a
// range of 64-pixel K-tiles; ranges are combined with float32 atomics
// (coalesced along the input channel).  Warp 4 issues TMA,
// warp 5 the MMAs, warps 0-3 drain TMEM; every wait is bounded.

constexpr int kWKP = 64;  // pixels per K-tile

// MN-major swizzled descriptor: rows of `row_bytes` along K (8-row atoms
// 8 * row_bytes apart = SBO), MN blocks of row_bytes / 2 elements `lbo` apart.
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr, int row_bytes, int lbo) {
    const uint64_t layout = row_bytes == 128 ? 2ull : row_bytes == 64 ? 4ull : 6ull;
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(((uint32_t)lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(((uint32_t)(8 * row_bytes) >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

// BF16 x BF16 -> F32, A and B MN-major, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc_mn(int n) {
    return instr_desc(n) | (1u << 15) | (1u << 16);
}

struct WgArgs {
    int H, W;            // grid of the convolution (input = output resolution)
    int Cin, Cout, xo;   // Cin channels read at channel offset xo; dW is [Cout][9][Cin]
    int BC, cpb;         // channels per x box (16 / 32 / 64), boxes per tap (Cin / BC)
    int pairs;           // 9 * cpb (tap, channel block) pairs
    int per_tile;        // 128 / BC pairs per M-tile
    int nm, MT;          // M-tiles in total, per CTA
    int bnw, nbox_b;     // dz box width (channels) and boxes per K-tile
    int KT, ktp;         // K-tiles in total, per CTA (blockIdx.y)
    int stages, stage_bytes, a_bytes;
    int tmem_cols;
    float* dw;
};

__global__ void __launch_bounds__(192, 2) k_wgrad_tc(const __grid_constant__ CUtensorMap mapx,
                                                     const __grid_constant__ CUtensorMap mapd, WgArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + S * a.stage_bytes);
    uint64_t* empty = full + S;
    uint64_t* done = full + 2 * S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 2 * S + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt0 = blockIdx.x * a.MT;
    const int mtn = min(a.MT, a.nm - mt0);
    const int kb = blockIdx.y * a.ktp, ke = min(a.KT, kb + a.ktp);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(su32(&full[s]), 1);
            mbar_init(su32(&empty[s]), 1);
        }
        mbar_init(su32(done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const long long HW = (long long)a.H * a.W;
    const int xbox = a.BC * kWKP * 2, dbox = a.bnw * kWKP * 2;

    if (warp == 4) {
        if (lane == 0) {
            int nx = 0;  // x boxes per K-tile
            for (int t = 0; t < mtn; ++t) nx += min(a.per_tile, a.pairs - (mt0 + t) * a.per_tile);
            const uint32_t bytes = (uint32_t)(a.nbox_b * dbox + nx * xbox);
            bool ok = true;
            for (int kt = kb; kt < ke && ok; ++kt) {
                const int i = kt - kb, s = i % S;
                if (i >= S) ok = mbar_wait(su32(&empty[s]), (uint32_t)(((i / S) - 1) & 1));
                if (!ok) break;
                const long long p0 = (long long)kt * kWKP;
                const int b = (int)(p0 / HW);
                const long long rem = p0 - (long long)b * HW;
                const int y0 = (int)(rem / a.W), x0 = (int)(rem % a.W);
                unsigned char* st = base + s * a.stage_bytes;
                mbar_expect_tx(su32(&full[s]), bytes);
                for (int k = 0; k < a.nbox_b; ++k)
                    tma_load_2d(su32(st + a.a_bytes + k * dbox), &mapd, su32(&full[s]), k * a.bnw, (int)p0);
                for (int t = 0; t < mtn; ++t)
                    for (int j = 0; j < a.per_tile; ++j) {
                        const int q = (mt0 + t) * a.per_tile + j;
                        if (q >= a.pairs) break;
                        const int tap = q / a.cpb, cb = q - tap * a.cpb;
                        tma_load_4d(su32(st + t * (kTM * kWKP * 2) + j * xbox), &mapx, su32(&full[s]),
                                    a.xo + cb * a.BC, x0 + tap % 3 - 1, y0 + tap / 3 - 1, b);
                    }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc_mn(a.Cout);
            const int ra = 2 * a.BC, rb = 2 * a.bnw;
            bool ok = true;
            for (int kt = kb; kt < ke && ok; ++kt) {
                const int i = kt - kb, s = i % S;
                ok = mbar_wait(su32(&full[s]), (uint32_t)((i / S) & 1));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* st = base + s * a.stage_bytes;
                const uint32_t abase = su32(st), bbase = su32(st + a.a_bytes);
                for (int t = 0; t < mtn; ++t)
                    for (int kk = 0; kk < kWKP / 16; ++kk)
                        umma(tmem + (uint32_t)(t * a.Cout),
                             smem_desc_mn(abase + t * (kTM * kWKP * 2) + kk * 16 * ra, ra, kWKP * ra),
                             smem_desc_mn(bbase + kk * 16 * rb, rb, kWKP * rb), idesc, (i > 0 || kk > 0) ? 1u : 0u);
                umma_commit(su32(&empty[s]));
            }
            if (ok) umma_commit(su32(done));
        }
    } else {
        // epilogue warps 0..3: TMEM lane m = tid is row m of each M-tile
        const bool okd = ke > kb && mbar_wait(su32(done), 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (okd) {
            const int j = tid / a.BC, c = tid - j * a.BC;
            for (int t = 0; t < mtn; ++t) {
                const int q = (mt0 + t) * a.per_tile + j;
                const bool valid = q < a.pairs;
                const int tap = valid ? q / a.cpb : 0;
                const int ci = valid ? (q - tap * a.cpb) * a.BC + c : 0;
                for (int n0 = 0; n0 < a.Cout; n0 += 16) {
                    uint32_t r[16];
                    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * a.Cout + n0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(taddr)
                        : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (!valid) continue;
                    float* d = a.dw + ((long long)n0 * 9 + tap) * a.Cin + ci;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) atomicAdd(d + (long long)jj * 9 * a.Cin, __uint_as_float(r[jj]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

size_t tc_smem(int bn, int bk) { return (size_t)kStages * (kTM + bn) * bk * 2 + 1024 + 256; }

bool g_tc_persistent = true;
bool g_tc_halo = true;  // NPBS_CONV_HALO=0 disables the halo mode
// CTAs of the persistent convolution per SM: two by default (measured: the
// network forward of 16 x 256^2 takes 1.66 / 1.25 / 1.30 / 1.32 ms with 1 / 2 /
// 3 / 4), fewer where registers or shared memory do not fit them.
int g_tc_blocks_per_sm_cap = 2;
bool g_tc_blocks_forced = false;  // NPBS_CONV_CTAS_PER_SM given: size the grid by it alone

// CTAs of the persistent convolution that fit on one SM with `smem` bytes of
// dynamic shared memory, from the kernel's registers and the SM's register
// file, shared memory and thread limits.  (The occupancy query reports one CTA
// for this kernel whatever the launch's shared memory, which left SMs idle.)
int conv_tc_blocks_per_sm(size_t smem) {
    cudaFuncAttributes fa{};
    int dev = 0, regs_sm = 65536, smem_sm = 228 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (cudaFuncGetAttributes(&fa, k_conv_tc_persist) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    const int by_regs = regs_sm / std::max(1, fa.numRegs * 192);
    const int by_smem = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
    return std::max(1, std::min(std::min(by_regs, by_smem), 2048 / 192));
}

}  // namespace

// Whether the tensor-core path takes this convolution (else the caller uses
// the warp-level MMA kernel).
static bool tc_grid_ok(int H, int W) {
    const long long HW = (long long)H * W;
    if (W >= kTM) return W % kTM == 0;
    return kTM % W == 0 && HW % kTM == 0;
}

bool conv_tc_supported(const ConvFwd& a) {
    if (!encoder()) return false;
    if (a.ups) {
        if (!a.w_sub || (a.H & 1) || (a.W & 1) || !tc_grid_ok(a.H / 2, a.W / 2)) return false;
    } else if (!tc_grid_ok(a.H, a.W)) {
        return false;
    }
    if (!(a.Cin == 16 || a.Cin == 32 || a.Cin % 64 == 0)) return false;
    if (a.Cout % 16 || a.Cout > 256 || a.Cout < 16) return false;
    if (a.xs % 8 || a.xo % 8 || (reinterpret_cast<uintptr_t>(a.x) & 15)) return false;
    if (a.ys % 8 || a.yo % 8) return false;
    return true;
}

static cudaError_t conv_fwd_tc_one(const ConvFwd& a, cudaStream_t st, int sub, int py, int px);

cudaError_t conv_fwd_tc(const ConvFwd& a, cudaStream_t st) {
    if (!a.ups) return conv_fwd_tc_one(a, st, 0, 0, 0);
    // nearest x2 upsampling + 3x3 conv == four 2x2 convolutions of the half-res
    // input (one per output parity) with pre-summed weights
    for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px) {
            cudaError_t e = conv_fwd_tc_one(a, st, 1, py, px);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

static cudaError_t conv_fwd_tc_one(const ConvFwd& a0, cudaStream_t st, int sub, int py, int px) {
    ConvFwd a = a0;
    const int ntaps = sub ? 4 : 9;
    if (sub) {
        a.H = a0.H / 2;
        a.W = a0.W / 2;
        a.w = a0.w_sub + (size_t)(py * 2 + px) * a0.Cout * 4 * a0.Cin;
    }
    // halo rows for 3x3 convolutions over whole 128-pixel row runs with narrow
    // inputs (the level-0/1 convolutions, bound by the tap tiles' L2 stream)
    const bool halo = g_tc_persistent && g_tc_halo && !sub && a.W % kTM == 0 && a.Cin % 16 == 0 && a.Cin <= 32;
    const int bk = a.Cin >= 64 ? 64 : a.Cin;
    const int bn = a.Cout;
    int tcols = 32;
    while (tcols < bn) tcols <<= 1;
    CUtensorMapSwizzle sw = bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                                : CU_TENSOR_MAP_SWIZZLE_32B;
    // input: dims (C, W, H, B), box (bk, cols, rows, 1); halo: (8, kHaloRows, 1, 1) unswizzled
    const int cols = a.W >= kTM ? kTM : a.W;
    const int rows = a.W >= kTM ? 1 : kTM / a.W;
    CUtensorMap mx, mw;
    {
        cuuint64_t dims[4] = {(cuuint64_t)a.xs, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
        cuuint64_t strides[3] = {(cuuint64_t)a.xs * 2, (cuuint64_t)a.xs * 2 * a.W, (cuuint64_t)a.xs * 2 * a.W * a.H};
        cuuint32_t box[4] = {(cuuint32_t)bk, (cuuint32_t)cols, (cuuint32_t)rows, 1};
        if (halo) {
            box[0] = 8;
            box[1] = kHaloRows;
        }
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (encoder()(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.x), dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, halo ? CU_TENSOR_MAP_SWIZZLE_NONE : sw,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)ntaps * a.Cin, (cuuint64_t)a.Cout};
        cuuint64_t strides[1] = {(cuuint64_t)ntaps * a.Cin * 2};
        cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)bn};
        cuuint32_t es[2] = {1, 1};
        if (encoder()(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(a.w), dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    TcArgs t{};
    t.B = a.B;
    t.H = a.H;
    t.W = a.W;
    t.Cin = a.Cin;
    t.Cout = a.Cout;
    t.BK = bk;
    t.ntaps = ntaps;
    for (int k = 0; k < ntaps; ++k) {
        if (sub) {
            // offsets {p - 1, p} at half resolution for output parity p
            t.tdy[k] = (k >> 1) + py - 1;
            t.tdx[k] = (k & 1) + px - 1;
        } else {
            t.tdy[k] = k / 3 - 1;
            t.tdx[k] = k % 3 - 1;
        }
    }
    t.sub = sub;
    t.py = py;
    t.px = px;
    t.Ho = a0.H;
    t.Wo = a0.W;
    t.rows_per_tile = rows;
    t.tiles_per_row = a.W >= kTM ? a.W / kTM : 1;
    t.bias = a.bias;
    t.act = a.act;
    t.y = a.y;
    t.z = a.z;
    t.yf = a.yf;
    t.ys = a.ys;
    t.yo = a.yo;
    t.xo = a.xo;
    t.bn = bn;
    t.tmem_cols = tcols;
    t.halo = halo ? 1 : 0;
    const size_t smem = halo ? (size_t)kStages * ((bk / 8) * kHaloRows * 16 + 3 * bn * bk * 2) + 1024 + 256
                             : tc_smem(bn, bk);
    const long long M = (long long)a.B * a.H * a.W;
    const int ntiles = (int)((M + kTM - 1) / kTM);
    if (g_tc_persistent) {
        int tc2 = 32;
        while (tc2 < 2 * bn) tc2 <<= 1;
        t.tmem_cols = tc2;
        const int per_sm = std::max(1, std::min(512 / tc2, g_tc_blocks_per_sm_cap));
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        occ = g_tc_blocks_forced ? g_tc_blocks_per_sm_cap : conv_tc_blocks_per_sm(smem);
        const int grid = std::max(1, std::min(ntiles, nsm * std::max(1, std::min(occ, per_sm))));
        k_conv_tc_persist<<<grid, 192, smem, st>>>(mx, mw, t, ntiles);
        return cudaGetLastError();
    }
    k_conv_tc<<<(unsigned)ntiles, 128, smem, st>>>(mx, mw, t);
    return cudaGetLastError();
}

// 64-pixel K-tiles: a run of one row (W a multiple of 64) or whole rows.
static bool wg_grid_ok(int H, int W) {
    if (W % kWKP == 0) return true;
    return kWKP % W == 0 && H % (kWKP / W) == 0;
}

bool conv_wgrad_tc_supported(const ConvWgrad& a) {
    if (!encoder() || a.ups) return false;
    if (!wg_grid_ok(a.H, a.W)) return false;
    if (!(a.Cin == 16 || a.Cin == 32 || a.Cin % 64 == 0)) return false;
    if (!(a.Cout == 32 || a.Cout % 64 == 0) || a.Cout > 256) return false;
    if (a.xs % 8 || a.xo % 8 || (reinterpret_cast<uintptr_t>(a.x) & 15) || (reinterpret_cast<uintptr_t>(a.dz) & 15))
        return false;
    return true;
}

static constexpr size_t kWgSmemMax = 200 * 1024 + 2048;

cudaError_t conv_wgrad_tc(const ConvWgrad& a, cudaStream_t st) {
    const long long P = (long long)a.B * a.H * a.W;
    WgArgs t{};
    t.H = a.H;
    t.W = a.W;
    t.Cin = a.Cin;
    t.Cout = a.Cout;
    t.xo = a.xo;
    t.BC = a.Cin >= 64 ? 64 : a.Cin;
    t.cpb = a.Cin / t.BC;
    t.pairs = 9 * t.cpb;
    t.per_tile = kTM / t.BC;
    t.nm = (t.pairs + t.per_tile - 1) / t.per_tile;
    // one M-tile per CTA and a pipeline sized so that two CTAs share an SM:
    // the kernel is bound by TMA round trips, not by the tensor pipe, so
    // more independent pipelines beat sharing each dz tile across M-tiles
    t.MT = 1;
    t.bnw = a.Cout >= 64 ? 64 : a.Cout;
    t.nbox_b = a.Cout / t.bnw;
    t.a_bytes = t.MT * kTM * kWKP * 2;
    t.stage_bytes = t.a_bytes + a.Cout * kWKP * 2;
    t.stages = (int)std::max<size_t>(2, std::min<size_t>(6, (100 * 1024) / (size_t)t.stage_bytes));
    int cols = 32;
    while (cols < t.MT * a.Cout) cols <<= 1;
    t.tmem_cols = cols;
    t.dw = a.dw;
    t.KT = (int)(P / kWKP);
    const int G = (t.nm + t.MT - 1) / t.MT;
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int want = std::max(1, (4 * std::max(nsm, 1) + G - 1) / G);
    int S = std::max(1, std::min(t.KT / 8, want));
    t.ktp = (t.KT + S - 1) / S;
    S = (t.KT + t.ktp - 1) / t.ktp;
    const size_t smem = (size_t)t.stages * t.stage_bytes + 1024 + 256;
    if (smem > kWgSmemMax) return cudaErrorInvalidValue;
    CUtensorMap mx, md;
    const CUtensorMapSwizzle swx = t.BC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : t.BC == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                : CU_TENSOR_MAP_SWIZZLE_32B;
    {
        const int cols_ = a.W >= kWKP ? kWKP : a.W;
        const int rows_ = a.W >= kWKP ? 1 : kWKP / a.W;
        cuuint64_t dims[4] = {(cuuint64_t)a.xs, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
        cuuint64_t strides[3] = {(cuuint64_t)a.xs * 2, (cuuint64_t)a.xs * 2 * a.W, (cuuint64_t)a.xs * 2 * a.W * a.H};
        cuuint32_t box[4] = {(cuuint32_t)t.BC, (cuuint32_t)cols_, (cuuint32_t)rows_, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (encoder()(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.x), dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swx, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)a.Cout, (cuuint64_t)P};
        cuuint64_t strides[1] = {(cuuint64_t)a.Cout * 2};
        cuuint32_t box[2] = {(cuuint32_t)t.bnw, (cuuint32_t)kWKP};
        cuuint32_t es[2] = {1, 1};
        const CUtensorMapSwizzle swd = t.bnw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
        if (encoder()(&md, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(a.dz), dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swd, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    k_wgrad_tc<<<dim3((unsigned)G, (unsigned)S), 192, smem, st>>>(mx, md, t);
    return cudaGetLastError();
}

cudaError_t prepare_conv_tc() {
    encoder();
    if (const char* e = getenv("NPBS_CONV_TC")) g_tc_persistent = strcmp(e, "tile") != 0;
    if (const char* e = getenv("NPBS_CONV_HALO")) g_tc_halo = strcmp(e, "0") != 0;
    // NPBS_CONV_CTAS_PER_SM=k launches k CTAs of the persistent convolution per SM (default: 2 where they fit)
    if (const char* e = getenv("NPBS_CONV_CTAS_PER_SM")) {
        g_tc_blocks_per_sm_cap = std::max(1, atoi(e));
        g_tc_blocks_forced = true;
    }
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(256, 64));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_tc_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(256, 64));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmemMax);
    return e;
}

int conv_tc_timeout_flag() {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_conv_tc_timeout, sizeof(int));
    return v;
}

void conv_tc_clear_timeout() {
    const int z = 0;
    cudaMemcpyToSymbol(g_conv_tc_timeout, &z, sizeof(int));
}

cudaError_t wait_selftest(double seconds, cudaStream_t st) {
    int dev = 0, khz = 2000000;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const long long limit = (long long)(seconds * (double)khz * 1e3);
    k_wait_selftest<<<1, 32, 0, st>>>(limit > 0 ? limit : 1);
    return cudaGetLastError();
}

}  // namespace npbs
