// The residual-to-correction network M(r; n) = s N([Re r/s, Im r/s, n]),
// s = ||r||_2 / sqrt(#points): a 4-level U-Net (32, 64, 128, 256 channels, two
// 3x3 conv + GELU per level, 2x2 average pooling, nearest x2 upsampling + 3x3
// conv + GELU, concatenated skips, a bias-free 1x1 head to (Re, Im)).  This is
// the U-Net backbone of App. Experimental Setup with the readings listed in the
// design notes; parameters follow the canonical order (per conv: weight
// [Cout][Cin][3][3], bias [Cout]; then the head [2][32]).
//
// Forward, backward (data and weight gradients), AdamW and the parameter I/O
// of the C ABI live here.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "conv.cuh"
#include "krylov.cuh"
#include "net.cuh"

namespace npbs {

const std::vector<LayerDef>& layer_defs() {
    static std::vector<LayerDef> defs = [] {
        std::vector<LayerDef> d;
        const int ch[4] = {32, 64, 128, 256};
        int cin = 3;
        for (int l = 0; l < 4; ++l) {
            d.push_back({"enc_a", l, cin, ch[l], 0});
            d.push_back({"enc_b", l, ch[l], ch[l], 0});
            cin = ch[l];
        }
        for (int l = 2; l >= 0; --l) {
            d.push_back({"up", l, ch[l + 1], ch[l], 1});
            d.push_back({"dec_a", l, 2 * ch[l], ch[l], 0});
            d.push_back({"dec_b", l, ch[l], ch[l], 0});
        }
        long long off = 0, coff = 0;
        for (auto& L : d) {
            L.cin_pad = L.cin < 16 ? 16 : L.cin;
            L.w_off = off;
            off += (long long)L.cout * 9 * L.cin_pad;
            L.b_off = off;
            off += L.cout;
            L.cw_off = coff;
            coff += (long long)L.cout * L.cin * 9;
            L.cb_off = coff;
            coff += L.cout;
        }
        return d;
    }();
    return defs;
}

long long dev_param_count() {
    const auto& d = layer_defs();
    return d.back().b_off + d.back().cout + 2 * 32;
}
long long canon_param_count() {
    const auto& d = layer_defs();
    return d.back().cb_off + d.back().cout + 2 * 32;
}
long long head_dev_off() { return dev_param_count() - 64; }
long long head_canon_off() { return canon_param_count() - 64; }

// ------------------------------------------------------------- small kernels

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// acc[slot] += sum |r|^2 over a chunk of the slot's instance (grid: chunks x slots)
__global__ void k_slot_sumsq(const SlotDev sd, const float2* r, double* acc2) {
    const int slot = blockIdx.y;
    const long long base = sd.off[slot];
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < sd.np; e += (long long)gridDim.x * blockDim.x) {
        const float2 v = r[base + e];
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(acc2 + slot, t);
    }
}

// s[slot] = sqrt(mean |r|^2)
__global__ void k_slot_rms_finish(int nb, long long np, const double* acc2, float* s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb) s[i] = (float)sqrt(acc2[i] / (double)np);
}

static cudaError_t slot_rms(const SlotDev& sd, const float2* r, double* acc2, float* s, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc2, 0, sizeof(double) * sd.nb, st);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)std::max<long long>(1, std::min<long long>(64, (sd.np + 255) / 256)), sd.nb);
    k_slot_sumsq<<<g, 256, 0, st>>>(sd, r, acc2);
    k_slot_rms_finish<<<(sd.nb + 127) / 128, 128, 0, st>>>(sd.nb, sd.np, acc2, s);
    return cudaGetLastError();
}

// net input [slot][H][W][16]: Re r / s, Im r / s, n, zeros
__global__ void k_pack_input(const SlotDev sd, const float2* r, const float* n, const float* s, bf16* out) {
    const long long P = (long long)sd.nb * sd.np;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(p / sd.np);
        const long long e = p - (long long)slot * sd.np;
        const long long g = sd.off[slot] + e;
        const float sc = s[slot];
        const float is = sc > 0.f ? 1.f / sc : 0.f;
        const float2 v = r[g];
        __align__(16) bf16 c[16];
        c[0] = __float2bfloat16_rn(v.x * is);
        c[1] = __float2bfloat16_rn(v.y * is);
        c[2] = __float2bfloat16_rn(n[g]);
#pragma unroll
        for (int k = 3; k < 16; ++k) c[k] = __float2bfloat16_rn(0.f);
        uint4* dst = reinterpret_cast<uint4*>(out + p * 16);
        dst[0] = reinterpret_cast<uint4*>(c)[0];
        dst[1] = reinterpret_cast<uint4*>(c)[1];
    }
}

// 2x2 average pooling of channels [0, C) of src [B][R][Rw][S] -> dst [B][R/2][Rw/2][C]
__global__ void k_pool(int nb, int R, int Rw, int C, int S, const bf16* src, bf16* dst) {
    const int Ro = R / 2, Rwo = Rw / 2;
    const int cc = C / 8;
    const long long total = (long long)nb * Ro * Rwo * cc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(i % cc);
        const long long q = i / cc;
        const int x = (int)(q % Rwo);
        const long long t = q / Rwo;
        const int y = (int)(t % Ro), b = (int)(t / Ro);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long sp = ((long long)b * R + 2 * y + dy) * Rw + 2 * x + dx;
                const uint4 v = *reinterpret_cast<const uint4*>(src + sp * S + c8 * 8);
                const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] += __bfloat162float(e[k]);
            }
        __align__(16) bf16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16_rn(0.25f * acc[k]);
        *reinterpret_cast<uint4*>(dst + q * C + c8 * 8) = *reinterpret_cast<uint4*>(o);
    }
}

// head: y = Wh e (2 x 32), c = s (y0 + i y1); mode 0: out = c, 1: out += c
__global__ void k_head(const SlotDev sd, const bf16* e, const float* wh, const float* s, float2* out, int add) {
    __shared__ float w[64];
    if (threadIdx.x < 64) w[threadIdx.x] = wh[threadIdx.x];
    __syncthreads();
    const long long P = (long long)sd.nb * sd.np;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(p / sd.np);
        const long long g = sd.off[slot] + (p - (long long)slot * sd.np);
        const uint4* src = reinterpret_cast<const uint4*>(e + p * 32);
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = src[q];
            const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float x = __bfloat162float(h[k]);
                y0 += w[q * 8 + k] * x;
                y1 += w[32 + q * 8 + k] * x;
            }
        }
        const float sc = s[slot];
        float2 c = make_float2(sc * y0, sc * y1);
        if (add) {
            const float2 o = out[g];
            c.x += o.x;
            c.y += o.y;
        }
        out[g] = c;
    }
}

// head backward: gy = s (Re gc, Im gc); dZ_e = (Wh^T gy) * gelu'(z_e) (bf16);
// dWh += sum gy e^T; S1[slot] += sum (Re gc y0 + Im gc y1)
__global__ void k_head_bwd(const SlotDev sd, const bf16* e, const bf16* ze, const float* wh, const float* s,
                           const float2* gc, bf16* dz, float* dwh, double* S1) {
    __shared__ float w[64];
    __shared__ float dws[64];
    __shared__ double s1s;
    if (threadIdx.x < 64) { w[threadIdx.x] = wh[threadIdx.x]; dws[threadIdx.x] = 0.f; }
    if (threadIdx.x == 0) s1s = 0.0;
    __syncthreads();
    const long long P = (long long)sd.nb * sd.np;
    float dwl[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) dwl[k] = 0.f;
    // one slot per block range: blocks are assigned to whole slots below
    const int slot = blockIdx.y;
    double s1 = 0.0;
    for (long long e2 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e2 < sd.np; e2 += (long long)gridDim.x * blockDim.x) {
        const long long p = (long long)slot * sd.np + e2;
        const long long g = sd.off[slot] + e2;
        const float2 gg = gc[g];
        const float sc = s[slot];
        const float g0 = sc * gg.x, g1 = sc * gg.y;
        float hx[32];
        const uint4* src = reinterpret_cast<const uint4*>(e + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = src[q];
            const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) hx[q * 8 + k] = __bfloat162float(h[k]);
        }
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            y0 += w[k] * hx[k];
            y1 += w[32 + k] * hx[k];
            dwl[k] += g0 * hx[k];
            dwl[32 + k] += g1 * hx[k];
        }
        s1 += (double)gg.x * y0 + (double)gg.y * y1;
        const uint4* zsrc = reinterpret_cast<const uint4*>(ze + p * 32);
        __align__(16) bf16 o[32];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = zsrc[q];
            const bf16* zz = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = q * 8 + k;
                const float d = (w[c] * g0 + w[32 + c] * g1) * gelu_grad(__bfloat162float(zz[k]));
                o[c] = __float2bfloat16_rn(d);
            }
        }
        uint4* dst = reinterpret_cast<uint4*>(dz + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<uint4*>(o)[q];
    }
    (void)P;
#pragma unroll
    for (int k = 0; k < 64; ++k) {
        float v = dwl[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&dws[k], v);
    }
    for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s1s, s1);
    __syncthreads();
    if (threadIdx.x < 64) atomicAdd(dwh + threadIdx.x, dws[threadIdx.x]);
    if (threadIdx.x == 0) atomicAdd(S1 + slot, s1s);
}

// dZ = dY * gelu'(Z): dY float32 (pixel stride ds, offset do), Z bf16 (stride zs,
// offset zo) -> dZ bf16 [P][C]; with db, also db[c] += sum_p dZ[p][c] (the bias
// gradient of the convolution that produced Z, from the bf16 dZ it consumes).
// Launched with 256 threads and C / 8 dividing 256, so every thread keeps one
// group of 8 channels across the grid-stride loop.
__global__ void k_gelu_bwd(long long P, int C, const float* dy, int ds, int dof, const bf16* z, int zs, int zo, bf16* dz,
                           float* db) {
    __shared__ float red[256 * 8];
    const int cc = C / 8;
    const long long total = P * cc;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / cc;
        const int c8 = (int)(i % cc);
        const float4 a = *reinterpret_cast<const float4*>(dy + p * ds + dof + c8 * 8);
        const float4 b = *reinterpret_cast<const float4*>(dy + p * ds + dof + c8 * 8 + 4);
        const uint4 zv = *reinterpret_cast<const uint4*>(z + p * zs + zo + c8 * 8);
        const bf16* zz = reinterpret_cast<const bf16*>(&zv);
        const float d[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        __align__(16) bf16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            o[k] = __float2bfloat16_rn(d[k] * gelu_grad(__bfloat162float(zz[k])));
            acc[k] += __bfloat162float(o[k]);
        }
        *reinterpret_cast<uint4*>(dz + p * C + c8 * 8) = *reinterpret_cast<uint4*>(o);
    }
    if (!db) return;  // uniform over the launch
    const int g = threadIdx.x % cc, l = threadIdx.x / cc;
#pragma unroll
    for (int k = 0; k < 8; ++k) red[l * C + g * 8 + k] = acc[k];
    __syncthreads();
    const int lanes = blockDim.x / cc;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float t = 0.f;
        for (int j = 0; j < lanes; ++j) t += red[j * C + c];
        atomicAdd(db + c, t);
    }
}

// adjoint of 2x2 average pooling, accumulated: dst[b][2y+dy][2x+dx][c] (stride S)
// += 0.25 * src[b][y][x][c]   (src [B][R][Rw][C], R x Rw the coarse size)
__global__ void k_pool_adj_add(int nb, int R, int Rw, int C, const float* src, float* dst, int S) {
    const long long total = (long long)nb * R * Rw * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long q = i / C;
        const int x = (int)(q % Rw);
        const long long t = q / Rw;
        const int y = (int)(t % R), b = (int)(t / R);
        const float v = 0.25f * src[i];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long dp = ((long long)b * 2 * R + 2 * y + dy) * 2 * Rw + 2 * x + dx;
                dst[dp * S + c] += v;
            }
    }
}

// adjoint of nearest x2 upsampling: dst[b][y][x][c] = sum of the 2x2 block of src
// (src [B][2R][2Rw][C], dst [B][R][Rw][C])
__global__ void k_sumpool(int nb, int R, int Rw, int C, const float* src, float* dst) {
    const long long total = (long long)nb * R * Rw * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long q = i / C;
        const int x = (int)(q % Rw);
        const long long t = q / Rw;
        const int y = (int)(t % R), b = (int)(t / R);
        float acc = 0.f;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const long long sp = ((long long)b * 2 * R + 2 * y + dy) * 2 * Rw + 2 * x + dx;
                acc += src[sp * C + c];
            }
        dst[i] = acc;
    }
}

// db[c] += sum_p dz[p][c]
// db[c] += sum_p dz[p, c]: each thread sums 8 channels (one 16-byte load) of
// a strided set of pixels, the block reduces its pixel lanes in shared memory
// and adds one partial per channel.  C is a multiple of 8, at most 8 * 256.
__global__ void k_bias_grad(long long P, int C, const bf16* dz, float* db) {
    __shared__ float red[256 * 8];
    const int cg = C / 8;
    const int lanes = blockDim.x / cg;
    const int g = threadIdx.x % cg, l = threadIdx.x / cg;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (l < lanes) {
        for (long long p = (long long)blockIdx.x * lanes + l; p < P; p += (long long)gridDim.x * lanes) {
            const uint4 v = *reinterpret_cast<const uint4*>(dz + p * C + g * 8);
            const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += __bfloat162float(e[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) red[l * C + g * 8 + k] = acc[k];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float t = 0.f;
        for (int j = 0; j < lanes; ++j) t += red[j * C + c];
        atomicAdd(db + c, t);
    }
}

// dst[b][y][x][0..C) = src[b][y/2][x/2][0..C): the nearest x2 upsampling the
// up convolutions fold into their gather, written out (R x Rw the fine size)
__global__ void k_upsample2(int nb, int R, int Rw, int C, const bf16* src, bf16* dst) {
    const int c8n = C / 8;
    const long long total = (long long)nb * R * Rw * c8n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / c8n;
        const int c8 = (int)(i - p * c8n);
        const int x = (int)(p % Rw);
        const long long t = p / Rw;
        const int y = (int)(t % R), b = (int)(t / R);
        const long long q = ((long long)b * (R / 2) + y / 2) * (Rw / 2) + x / 2;
        *reinterpret_cast<uint4*>(dst + p * C + c8 * 8) = *reinterpret_cast<const uint4*>(src + q * C + c8 * 8);
    }
}

// S2[slot] += sum (dx0 Re r + dx1 Im r) / s^2 over the slot
__global__ void k_input_grad_reduce(const SlotDev sd, const float* dx, const float2* r, const float* s, double* S2) {
    const int slot = blockIdx.y;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < sd.np; e += (long long)gridDim.x * blockDim.x) {
        const long long p = (long long)slot * sd.np + e;
        const float2 v = r[sd.off[slot] + e];
        acc += (double)dx[p * 16] * v.x + (double)dx[p * 16 + 1] * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double sc = s[slot];
        atomicAdd(S2 + slot, sc > 0 ? t / (sc * sc) : 0.0);
    }
}

// g_r = (dx0 + i dx1) / s + (S1 - S2) r / (N s)   (scale-wrapper chain rule)
__global__ void k_input_grad(const SlotDev sd, const float* dx, const float2* r, const float* s, const double* S1,
                             const double* S2, float2* gr, int add) {
    const long long P = (long long)sd.nb * sd.np;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(p / sd.np);
        const long long g = sd.off[slot] + (p - (long long)slot * sd.np);
        const float sc = s[slot];
        const float is = sc > 0.f ? 1.f / sc : 0.f;
        const float k = (float)((S1[slot] - S2[slot]) / (double)sd.np) * is;
        const float2 v = r[g];
        float2 o = make_float2(dx[p * 16] * is + k * v.x, dx[p * 16 + 1] * is + k * v.y);
        if (add) {
            const float2 q = gr[g];
            o.x += q.x;
            o.y += q.y;
        }
        gr[g] = o;
    }
}

// master fp32 [Cout][9][Cinp] -> bf16 copy and the flipped transpose used by
// the data gradient: wt[ci][8 - tap][co] = w[co][tap][ci]
__global__ void k_weights_bf16(const float* w, int cout, int cinp, bf16* wb, bf16* wt) {
    const long long total = (long long)cout * 9 * cinp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cinp);
        const long long q = i / cinp;
        const int tap = (int)(q % 9), co = (int)(q / 9);
        const bf16 v = __float2bfloat16_rn(w[i]);
        wb[i] = v;
        wt[((long long)ci * 9 + (8 - tap)) * cout + co] = v;
    }
}

// 2x2 sub-pixel weights of an upsampling conv: for output parity (py, px) and
// tap (a, b) at half-resolution offsets (a + py - 1, b + px - 1), the sum of the
// 3x3 weights whose input falls on that half-resolution pixel.
__device__ __forceinline__ void dy_range(int p, int a, int* lo, int* hi) {
    // p = 0: a = 0 <- {-1}, a = 1 <- {0, 1};  p = 1: a = 0 <- {-1, 0}, a = 1 <- {1}
    if (p == 0) { *lo = a == 0 ? -1 : 0; *hi = a == 0 ? -1 : 1; }
    else { *lo = a == 0 ? -1 : 1; *hi = a == 0 ? 0 : 1; }
}
__global__ void k_weights_subpixel(const float* w, int cout, int cinp, bf16* ws) {
    const long long total = 4LL * cout * 4 * cinp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cinp);
        long long q = i / cinp;
        const int k = (int)(q % 4);
        q /= 4;
        const int co = (int)(q % cout);
        const int par = (int)(q / cout);
        const int py = par >> 1, px = par & 1, a = k >> 1, b = k & 1;
        int y0, y1, x0, x1;
        dy_range(py, a, &y0, &y1);
        dy_range(px, b, &x0, &x1);
        float acc = 0.f;
        for (int dy = y0; dy <= y1; ++dy)
            for (int dx = x0; dx <= x1; ++dx) acc += w[((long long)co * 9 + (dy + 1) * 3 + (dx + 1)) * cinp + ci];
        ws[i] = __float2bfloat16_rn(acc);
    }
}

__global__ void k_adamw(long long n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        float x = p[i] * (1.f - lr * wd);
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        x -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = x;
    }
}

static unsigned grid_for(long long n, int threads = 256, int cap = 152 * 16) {
    long long g = (n + threads - 1) / threads;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, cap));
}

// ------------------------------------------------------------- net object

npbs_status Net::alloc(int dev) {
    device = dev;
    const long long P = dev_param_count();
    const auto& d = layer_defs();
    long long nbf = 0;
    for (auto& L : d) nbf += (long long)L.cout * 9 * L.cin_pad;
    if (cudaMalloc(&params, sizeof(float) * P) != cudaSuccess) return NPBS_ERR_OOM;
    if (cudaMalloc(&grads, sizeof(float) * P) != cudaSuccess) return NPBS_ERR_OOM;
    if (cudaMalloc(&m1, sizeof(float) * P) != cudaSuccess) return NPBS_ERR_OOM;
    if (cudaMalloc(&m2, sizeof(float) * P) != cudaSuccess) return NPBS_ERR_OOM;
    if (cudaMalloc(&wb, sizeof(bf16) * nbf) != cudaSuccess) return NPBS_ERR_OOM;
    if (cudaMalloc(&wt, sizeof(bf16) * nbf) != cudaSuccess) return NPBS_ERR_OOM;
    long long nsub = 0;
    for (auto& L : d) {
        wsub_off.push_back(L.ups ? nsub : -1);
        if (L.ups) nsub += 4LL * L.cout * 4 * L.cin_pad;
    }
    if (nsub && cudaMalloc(&wsub, sizeof(bf16) * nsub) != cudaSuccess) return NPBS_ERR_OOM;
    cudaMemset(params, 0, sizeof(float) * P);
    cudaMemset(grads, 0, sizeof(float) * P);
    cudaMemset(m1, 0, sizeof(float) * P);
    cudaMemset(m2, 0, sizeof(float) * P);
    long long o = 0;
    for (auto& L : d) {
        wb_off.push_back(o);
        o += (long long)L.cout * 9 * L.cin_pad;
    }
    return NPBS_OK;
}

Net::~Net() {
    cudaFree(params);
    cudaFree(grads);
    cudaFree(m1);
    cudaFree(m2);
    cudaFree(wb);
    cudaFree(wt);
    cudaFree(wsub);
    if (fno) {
        cudaFree(fno->tw);
        cudaFree(fno->cache);
        cudaFree(fno->wt);
        delete fno;
    }
}

cudaError_t Net::refresh_bf16(cudaStream_t st) const {
    const auto& d = layer_defs();
    for (size_t i = 0; i < d.size(); ++i) {
        const auto& L = d[i];
        const long long n = (long long)L.cout * 9 * L.cin_pad;
        k_weights_bf16<<<grid_for(n), 256, 0, st>>>(params + L.w_off, L.cout, L.cin_pad, wb + wb_off[i], wt + wb_off[i]);
        if (L.ups)
            k_weights_subpixel<<<grid_for(16LL * L.cout * L.cin_pad), 256, 0, st>>>(params + L.w_off, L.cout, L.cin_pad,
                                                                                    wsub + wsub_off[i]);
    }
    return cudaGetLastError();
}

// canonical (OIHW) <-> device ([Cout][9][Cinp]) parameter layouts on the host
void canon_to_dev(const float* c, std::vector<float>& dv) {
    const auto& d = layer_defs();
    dv.assign(dev_param_count(), 0.f);
    for (auto& L : d) {
        for (int co = 0; co < L.cout; ++co)
            for (int ci = 0; ci < L.cin; ++ci)
                for (int t = 0; t < 9; ++t)
                    dv[L.w_off + ((long long)co * 9 + t) * L.cin_pad + ci] = c[L.cw_off + ((long long)co * L.cin + ci) * 9 + t];
        for (int co = 0; co < L.cout; ++co) dv[L.b_off + co] = c[L.cb_off + co];
    }
    for (int k = 0; k < 64; ++k) dv[head_dev_off() + k] = c[head_canon_off() + k];
}

void dev_to_canon(const std::vector<float>& dv, float* c) {
    const auto& d = layer_defs();
    for (auto& L : d) {
        for (int co = 0; co < L.cout; ++co)
            for (int ci = 0; ci < L.cin; ++ci)
                for (int t = 0; t < 9; ++t)
                    c[L.cw_off + ((long long)co * L.cin + ci) * 9 + t] = dv[L.w_off + ((long long)co * 9 + t) * L.cin_pad + ci];
        for (int co = 0; co < L.cout; ++co) c[L.cb_off + co] = dv[L.b_off + co];
    }
    for (int k = 0; k < 64; ++k) c[head_canon_off() + k] = dv[head_dev_off() + k];
}

// ------------------------------------------------------------- workspace

// Activation layout of one forward (and backward) over nb slots of H x W.
struct Acts {
    int nb, H, W;
    bf16* netin;
    bf16 *in[4], *a[4], *za[4], *cat[4], *zcat[4], *d[3], *zd[3], *e[3], *ze[3];
    // gradients (float32 except dz scratch)
    float *dnetin, *din[4], *da[4], *dcat[4], *dd[3], *de[3], *tmp;
    bf16* dz;
    float* s;
    double *S1, *S2;
    int* slot_dev;
    long long* off_dev;
};

static size_t acts_bytes(int nb, int H, int W, bool train, Acts* A, char* base) {
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + o : nullptr;
        o += (bytes + 255) / 256 * 256;
        return p;
    };
    const int ch[4] = {32, 64, 128, 256};
    const long long P0 = (long long)nb * H * W;
    auto px = [&](int l) { return P0 >> (2 * l); };
    Acts a{};
    a.nb = nb;
    a.H = H;
    a.W = W;
    a.netin = (bf16*)take(sizeof(bf16) * P0 * 16);
    for (int l = 0; l < 4; ++l) {
        const int C = ch[l];
        const int CC = l < 3 ? 2 * C : C;
        a.in[l] = l ? (bf16*)take(sizeof(bf16) * px(l) * ch[l - 1]) : nullptr;
        a.a[l] = (bf16*)take(sizeof(bf16) * px(l) * C);
        a.cat[l] = (bf16*)take(sizeof(bf16) * px(l) * CC);
        a.za[l] = train ? (bf16*)take(sizeof(bf16) * px(l) * C) : nullptr;
        a.zcat[l] = train ? (bf16*)take(sizeof(bf16) * px(l) * CC) : nullptr;
        if (l < 3) {
            a.d[l] = (bf16*)take(sizeof(bf16) * px(l) * C);
            a.e[l] = (bf16*)take(sizeof(bf16) * px(l) * C);
            a.zd[l] = train ? (bf16*)take(sizeof(bf16) * px(l) * C) : nullptr;
            a.ze[l] = train ? (bf16*)take(sizeof(bf16) * px(l) * C) : nullptr;
        }
    }
    if (train) {
        a.dnetin = (float*)take(sizeof(float) * P0 * 16);
        for (int l = 0; l < 4; ++l) {
            const int C = ch[l];
            const int CC = l < 3 ? 2 * C : C;
            a.din[l] = l ? (float*)take(sizeof(float) * px(l) * ch[l - 1]) : nullptr;
            a.da[l] = (float*)take(sizeof(float) * px(l) * C);
            a.dcat[l] = (float*)take(sizeof(float) * px(l) * CC);
            if (l < 3) {
                a.dd[l] = (float*)take(sizeof(float) * px(l) * C);
                a.de[l] = (float*)take(sizeof(float) * px(l) * C);
            }
        }
        a.tmp = (float*)take(sizeof(float) * P0 * 64);     // full-res dgrad of an up conv
        a.dz = (bf16*)take(sizeof(bf16) * P0 * 64);        // largest P x C product is P0 x 64
    }
    a.s = (float*)take(sizeof(float) * nb);
    a.S1 = (double*)take(sizeof(double) * nb);
    a.S2 = (double*)take(sizeof(double) * nb);
    a.slot_dev = (int*)take(sizeof(int) * nb);
    a.off_dev = (long long*)take(sizeof(long long) * nb);
    if (A) *A = a;
    return o;
}

// ------------------------------------------------------------- forward

static cudaError_t conv(const Net& net, int li, const bf16* x, int xs, int xo, int nb, int H, int W, bf16* y, int ys,
                        int yo, bf16* z, cudaStream_t st) {
    const LayerDef& L = layer_defs()[li];
    ConvFwd a{};
    a.x = x;
    a.xs = xs;
    a.xo = xo;
    a.B = nb;
    a.H = H;
    a.W = W;
    a.ups = L.ups;
    a.Cin = L.cin_pad;
    a.Cout = L.cout;
    a.w = net.wb + net.wb_off[li];
    a.w_sub = L.ups ? net.wsub + net.wsub_off[li] : nullptr;
    a.bias = net.params + L.b_off;
    a.act = 1;
    a.y = y;
    a.ys = ys;
    a.yo = yo;
    a.z = z;
    return conv_fwd(a, st);
}

// Layer indices in layer_defs(): enc l a = 2l, enc l b = 2l + 1; decoder level l
// (2, 1, 0): up = 8 + 3 (2 - l), dec_a = +1, dec_b = +2.
static int enc_a(int l) { return 2 * l; }
static int enc_b(int l) { return 2 * l + 1; }
static int up_i(int l) { return 8 + 3 * (2 - l); }

static cudaError_t forward_body(const Net& net, const Acts& A, cudaStream_t st, long long* kernels) {
    const int ch[4] = {32, 64, 128, 256};
    const int nb = A.nb;
    cudaError_t e = cudaSuccess;
    long long k = 0;
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        const int R = A.H >> l, Rw = A.W >> l;
        const int C = ch[l], CC = l < 3 ? 2 * C : C;
        const bf16* xin;
        int xs;
        if (l == 0) {
            xin = A.netin;
            xs = 16;
        } else {
            const int Cp = ch[l - 1];
            k_pool<<<grid_for((long long)nb * R * Rw * Cp / 8), 256, 0, st>>>(nb, 2 * R, 2 * Rw, Cp, 2 * Cp, A.cat[l - 1], A.in[l]);
            ++k;
            xin = A.in[l];
            xs = Cp;
        }
        e = conv(net, enc_a(l), xin, xs, 0, nb, R, Rw, A.a[l], C, 0, A.za[l], st);
        if (e == cudaSuccess) e = conv(net, enc_b(l), A.a[l], C, 0, nb, R, Rw, A.cat[l], CC, 0, A.zcat[l], st);
        k += 2;
    }
    for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
        const int R = A.H >> l, Rw = A.W >> l;
        const int C = ch[l];
        const bf16* src = l == 2 ? A.cat[3] : A.e[l + 1];
        const int ss = l == 2 ? ch[3] : ch[l + 1];
        e = conv(net, up_i(l), src, ss, 0, nb, R, Rw, A.cat[l], 2 * C, C, A.zcat[l], st);
        if (e == cudaSuccess) e = conv(net, up_i(l) + 1, A.cat[l], 2 * C, 0, nb, R, Rw, A.d[l], C, 0, A.zd[l], st);
        if (e == cudaSuccess) e = conv(net, up_i(l) + 2, A.d[l], C, 0, nb, R, Rw, A.e[l], C, 0, A.ze[l], st);
        k += 3;
    }
    if (kernels) *kernels += k;
    return e;
}

// Group instances by grid size.
static std::map<std::pair<int, int>, std::vector<int>> group(const Plan& pl, const std::vector<int>& which) {
    std::map<std::pair<int, int>, std::vector<int>> g;
    for (int j : which) g[{pl.inst_h[j].ny, pl.inst_h[j].nx}].push_back(j);
    return g;
}

npbs_status net_prepare(npbs_ctx* ctx, const Net& net, const Plan& pl, const std::vector<int>& which, bool train,
                        NetRun* run, cudaStream_t st, const float* a) {
    if (net.fno) return fno_prepare(ctx, net, pl, which, train, run, st, a);
    run->groups.clear();
    run->train = train;
    auto gr = group(pl, which);
    size_t ws = 0;
    std::vector<long long> off;
    for (auto& kv : gr) {
        const int H = kv.first.first, W = kv.first.second;
        if (H % 8 || W % 8 || H < 8 || W < 8)
            return set_err(ctx, NPBS_ERR_UNSUPPORTED_SIZE, "network: grid sides must be multiples of 8 (>= 8)");
        ws = std::max(ws, acts_bytes((int)kv.second.size(), H, W, train, nullptr, nullptr));
        for (int j : kv.second) off.push_back(pl.inst_h[j].offset);
    }
    NPBS_CK(ctx, ctx->net_ws.ensure(std::max<size_t>(ws, 256)));
    NPBS_CK(ctx, ctx->work[5].ensure(sizeof(long long) * std::max<size_t>(off.size(), 1)));
    long long* doff = static_cast<long long*>(ctx->work[5].p);
    NPBS_CK(ctx, cudaMemcpyAsync(doff, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
    NPBS_CK(ctx, cudaStreamSynchronize(st));
    size_t o = 0;
    for (auto& kv : gr) {
        NetGroup g;
        g.H = kv.first.first;
        g.W = kv.first.second;
        g.sd.nb = (int)kv.second.size();
        g.sd.np = (long long)g.H * g.W;
        g.sd.off = doff + o;
        o += kv.second.size();
        run->groups.push_back(g);
    }
    return NPBS_OK;
}

static Acts acts_of(npbs_ctx* ctx, const NetGroup& g, bool train) {
    Acts A;
    acts_bytes(g.sd.nb, g.H, g.W, train, &A, static_cast<char*>(ctx->net_ws.p));
    return A;
}

npbs_status net_run_forward(npbs_ctx* ctx, const Net& net, const NetRun& run, const float2* r, const float* n,
                            float2* out, int add, cudaStream_t st) {
    if (net.fno) return fno_run_forward(ctx, net, run, r, n, out, add, st);
    for (const NetGroup& g : run.groups) {
        Acts A = acts_of(ctx, g, false);
        const SlotDev sd = g.sd;
        NPBS_CK(ctx, slot_rms(sd, r, A.S2, A.s, st));
        k_pack_input<<<grid_for((long long)sd.nb * sd.np), 256, 0, st>>>(sd, r, n, A.s, A.netin);
        long long k = 2;
        NPBS_CK(ctx, forward_body(net, A, st, &k));
        k_head<<<grid_for((long long)sd.nb * sd.np), 256, 0, st>>>(sd, A.e[0], net.params + head_dev_off(), A.s, out, add);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(st, k + 1);
    }
    return NPBS_OK;
}

// Backward of out = M(r): accumulates the weight gradients into net.grads and
// writes (or adds) g_r.  Recomputes the forward (activation checkpointing).
npbs_status net_run_backward(npbs_ctx* ctx, Net& net, const NetRun& run, const float2* r, const float* n,
                             const float2* gc, float2* gr, int add, cudaStream_t st) {
    if (!run.train) return set_err(ctx, NPBS_ERR_INVALID_ARG, "network backward needs a training preparation");
    if (net.fno) return fno_run_backward(ctx, net, run, r, n, gc, gr, add, st);
    const int ch[4] = {32, 64, 128, 256};
    const auto& defs = layer_defs();
    for (const NetGroup& grp : run.groups) {
        const int H = grp.H, W = grp.W;
        Acts A = acts_of(ctx, grp, true);
        const SlotDev sd = grp.sd;
        const int nb = sd.nb;
        long long k = 0;
        NPBS_CK(ctx, slot_rms(sd, r, A.S2, A.s, st));
        k_pack_input<<<grid_for((long long)nb * sd.np), 256, 0, st>>>(sd, r, n, A.s, A.netin);
        k += 2;
        NPBS_CK(ctx, forward_body(net, A, st, &k));
        NPBS_CK(ctx, cudaMemsetAsync(A.S1, 0, sizeof(double) * nb, st));
        NPBS_CK(ctx, cudaMemsetAsync(A.S2, 0, sizeof(double) * nb, st));
        // head
        {
            dim3 g(std::max(1u, std::min(64u, (unsigned)((sd.np + 255) / 256))), nb);
            k_head_bwd<<<g, 256, 0, st>>>(sd, A.e[0], A.ze[0], net.params + head_dev_off(), A.s, gc, A.dz,
                                         net.grads + head_dev_off(), A.S1);
            ++k;
        }
        // helpers for one conv's backward given dZ (bf16, contiguous [P][Cout]) in A.dz
        auto wgrad = [&](int li, const bf16* x, int xs, int xo, int R, int Rw, bool bias_in_gelu = true) -> cudaError_t {
            const LayerDef& L = defs[li];
            ConvWgrad w{};
            w.x = x;
            w.xs = xs;
            w.xo = xo;
            w.B = nb;
            w.H = R;
            w.W = Rw;
            w.ups = L.ups;
            w.Cin = L.cin_pad;
            w.Cout = L.cout;
            w.dz = A.dz;
            w.dw = net.grads + L.w_off;
            const long long P = (long long)nb * R * Rw;
            if (L.ups) {
                // the tensor-core kernel reads TMA boxes of the input: write the
                // upsampled input out first (into the up conv's dgrad scratch,
                // which is free until the dgrad that follows)
                ConvWgrad w2 = w;
                w2.ups = 0;
                w2.x = reinterpret_cast<const bf16*>(A.tmp);
                w2.xs = L.cin_pad;
                w2.xo = 0;
                const char* force = getenv("NPBS_WGRAD");
                if (!(force && strcmp(force, "mma") == 0) && xs == L.cin_pad && xo == 0 && conv_wgrad_tc_supported(w2)) {
                    k_upsample2<<<grid_for(P * L.cin_pad / 8), 256, 0, st>>>(nb, R, Rw, L.cin_pad, x,
                                                                            reinterpret_cast<bf16*>(A.tmp));
                    ++k;
                    w = w2;
                }
            }
            const long long tiles = (long long)((9 * L.cin_pad + 63) / 64) * ((L.cout + 63) / 64);
            long long ppc = std::max<long long>(256, (P * tiles + 1215) / 1216);  // ~8 CTAs per SM
            ppc = (ppc + 31) / 32 * 32;
            w.pix_per_cta = (int)std::min<long long>(ppc, 1 << 20);
            cudaError_t e = conv_wgrad(w, st);
            if (e != cudaSuccess) return e;
            ++k;
            if (!bias_in_gelu) {
                const int lanes = 256 / (L.cout / 8);
                const long long nblk = std::min<long long>((P + lanes - 1) / lanes, 152LL * 8);
                k_bias_grad<<<(unsigned)nblk, 256, 0, st>>>(P, L.cout, A.dz, net.grads + L.b_off);
                ++k;
            }
            return cudaGetLastError();
        };
        auto dgrad = [&](int li, int R, int Rw, float* dst, int ds, int dof) -> cudaError_t {
            // dX = conv(dZ, flipped transposed W) at output resolution
            const LayerDef& L = defs[li];
            ConvFwd a{};
            a.x = A.dz;
            a.xs = L.cout;
            a.xo = 0;
            a.B = nb;
            a.H = R;
            a.W = Rw;
            a.ups = 0;
            a.Cin = L.cout;
            a.Cout = L.cin_pad;
            a.w = net.wt + net.wb_off[li];
            a.yf = dst;
            a.ys = ds;
            a.yo = dof;
            ++k;
            return conv_fwd(a, st);
        };
        // dZ of layer li's output; accumulates that layer's bias gradient too
        auto gelu_b = [&](int li, long long P, int C, const float* dy, int ds, int dof, const bf16* z, int zs, int zo) {
            k_gelu_bwd<<<grid_for(P * C / 8), 256, 0, st>>>(P, C, dy, ds, dof, z, zs, zo, A.dz,
                                                             net.grads + defs[li].b_off);
            ++k;
        };
        cudaError_t e = cudaSuccess;
        // decoder levels 0, 1, 2 (reverse of the forward order)
        for (int l = 0; l <= 2 && e == cudaSuccess; ++l) {
            const int R = H >> l, Rw = W >> l, C = ch[l];
            const long long P = (long long)nb * R * Rw;
            const int ib = up_i(l) + 2, ia = up_i(l) + 1, iu = up_i(l);
            if (l > 0) gelu_b(ib, P, C, A.de[l], C, 0, A.ze[l], C, 0);  // level 0: dz of dec_b from the head
            e = wgrad(ib, A.d[l], C, 0, R, Rw, l > 0);
            if (e == cudaSuccess) e = dgrad(ib, R, Rw, A.dd[l], C, 0);
            if (e != cudaSuccess) break;
            gelu_b(ia, P, C, A.dd[l], C, 0, A.zd[l], C, 0);
            e = wgrad(ia, A.cat[l], 2 * C, 0, R, Rw);
            if (e == cudaSuccess) e = dgrad(ia, R, Rw, A.dcat[l], 2 * C, 0);
            if (e != cudaSuccess) break;
            // up conv: output channels [C, 2C) of cat
            gelu_b(iu, P, C, A.dcat[l], 2 * C, C, A.zcat[l], 2 * C, C);
            const bf16* usrc = l == 2 ? A.cat[3] : A.e[l + 1];
            const int uss = l == 2 ? ch[3] : ch[l + 1];
            e = wgrad(iu, usrc, uss, 0, R, Rw);
            if (e == cudaSuccess) e = dgrad(iu, R, Rw, A.tmp, uss, 0);
            if (e != cudaSuccess) break;
            float* dsrc = l == 2 ? A.dcat[3] : A.de[l + 1];
            k_sumpool<<<grid_for((long long)nb * (R / 2) * (Rw / 2) * uss), 256, 0, st>>>(nb, R / 2, Rw / 2, uss, A.tmp, dsrc);
            ++k;
        }
        // encoder levels 3 .. 0
        for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
            const int R = H >> l, Rw = W >> l, C = ch[l];
            const int CC = l < 3 ? 2 * C : C;
            const long long P = (long long)nb * R * Rw;
            // enc b: output = cat channels [0, C); dY in dcat (already has the pool adjoint for l < 3)
            gelu_b(enc_b(l), P, C, A.dcat[l], CC, 0, A.zcat[l], CC, 0);
            e = wgrad(enc_b(l), A.a[l], C, 0, R, Rw);
            if (e == cudaSuccess) e = dgrad(enc_b(l), R, Rw, A.da[l], C, 0);
            if (e != cudaSuccess) break;
            gelu_b(enc_a(l), P, C, A.da[l], C, 0, A.za[l], C, 0);
            const bf16* x = l == 0 ? A.netin : A.in[l];
            const int xs = l == 0 ? 16 : ch[l - 1];
            e = wgrad(enc_a(l), x, xs, 0, R, Rw);
            if (e != cudaSuccess) break;
            if (l == 0) {
                e = dgrad(enc_a(0), R, Rw, A.dnetin, 16, 0);
            } else {
                e = dgrad(enc_a(l), R, Rw, A.din[l], ch[l - 1], 0);
                if (e == cudaSuccess) {
                    k_pool_adj_add<<<grid_for((long long)nb * R * Rw * ch[l - 1]), 256, 0, st>>>(
                        nb, R, Rw, ch[l - 1], A.din[l], A.dcat[l - 1], 2 * ch[l - 1]);
                    ++k;
                }
            }
        }
        NPBS_CK(ctx, e);
        {
            dim3 g(std::max(1u, std::min(64u, (unsigned)((sd.np + 255) / 256))), nb);
            k_input_grad_reduce<<<g, 256, 0, st>>>(sd, A.dnetin, r, A.s, A.S2);
            k_input_grad<<<grid_for((long long)nb * sd.np), 256, 0, st>>>(sd, A.dnetin, r, A.s, A.S1, A.S2, gr, add);
            k += 2;
        }
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(st, k);
    }
    return NPBS_OK;
}

npbs_status net_adamw(npbs_ctx* ctx, Net& net, float lr, float wd, cudaStream_t st) {
    net.step += 1;
    net.version += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float bc1 = 1.f - std::pow(b1, (float)net.step), bc2 = 1.f - std::pow(b2, (float)net.step);
    const long long P = net.count();
    k_adamw<<<grid_for(P), 256, 0, st>>>(P, net.params, net.grads, net.m1, net.m2, lr, b1, b2, eps, wd, bc1, bc2);
    NPBS_CK(ctx, cudaGetLastError());
    if (net.fno) {
        ctx->count(st, 1);
        return NPBS_OK;
    }
    NPBS_CK(ctx, net.refresh_bf16(st));
    ctx->count(st, 1 + (long long)layer_defs().size());
    return NPBS_OK;
}

}  // namespace npbs

using namespace npbs;

// ------------------------------------------------------------- C ABI

static uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" {

int64_t npbs_net_num_params(void) { return (int64_t)canon_param_count(); }

npbs_status npbs_net_create(npbs_net** out, int device, uint64_t seed) {
    if (!out) return NPBS_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return NPBS_ERR_INVALID_ARG;
    Net* n = new (std::nothrow) Net();
    if (!n) return NPBS_ERR_OOM;
    npbs_status st = n->alloc(device);
    if (st != NPBS_OK) {
        delete n;
        return st;
    }
    // He-normal weights, N(0, 0.01^2) biases, head scaled by 0.1 (Box-Muller on splitmix64)
    const long long C = canon_param_count();
    std::vector<float> c(C);
    uint64_t s = seed * 0x2545F4914F6CDD1Dull + 1;
    auto normal = [&]() {
        const double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    };
    for (auto& L : layer_defs()) {
        const double sd = std::sqrt(2.0 / (L.cin * 9.0));
        for (long long i = 0; i < (long long)L.cout * L.cin * 9; ++i) c[L.cw_off + i] = (float)(sd * normal());
        for (int i = 0; i < L.cout; ++i) c[L.cb_off + i] = (float)(0.01 * normal());
    }
    for (int k = 0; k < 64; ++k) c[head_canon_off() + k] = (float)(0.1 * std::sqrt(2.0 / 32.0) * normal());
    std::vector<float> dv;
    canon_to_dev(c.data(), dv);
    cudaMemcpy(n->params, dv.data(), sizeof(float) * dv.size(), cudaMemcpyHostToDevice);
    n->refresh_bf16(nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete n;
        return NPBS_ERR_CUDA;
    }
    *out = reinterpret_cast<npbs_net*>(n);
    return NPBS_OK;
}

npbs_status npbs_net_destroy(npbs_net* net) {
    if (!net) return NPBS_ERR_INVALID_ARG;
    delete reinterpret_cast<Net*>(net);
    return NPBS_OK;
}

static npbs_status copy_out(const Net& N, const float* dev, float* host, int64_t n) {
    if (N.fno) {
        if (!dev || !host || n != (int64_t)N.fno->count) return NPBS_ERR_INVALID_ARG;
        return cudaMemcpy(host, dev, sizeof(float) * n, cudaMemcpyDeviceToHost) == cudaSuccess ? NPBS_OK
                                                                                               : NPBS_ERR_CUDA;
    }
    if (!dev || !host || n != (int64_t)canon_param_count()) return NPBS_ERR_INVALID_ARG;
    std::vector<float> dv(dev_param_count());
    if (cudaMemcpy(dv.data(), dev, sizeof(float) * dv.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return NPBS_ERR_CUDA;
    dev_to_canon(dv, host);
    return NPBS_OK;
}

npbs_status npbs_net_set_params(npbs_net* net, const float* host, int64_t n) {
    if (!net || !host) return NPBS_ERR_INVALID_ARG;
    Net* N = reinterpret_cast<Net*>(net);
    cudaSetDevice(N->device);
    N->version += 1;
    if (N->fno) {
        if (n != (int64_t)N->fno->count) return NPBS_ERR_INVALID_ARG;
        return cudaMemcpy(N->params, host, sizeof(float) * n, cudaMemcpyHostToDevice) == cudaSuccess ? NPBS_OK
                                                                                                      : NPBS_ERR_CUDA;
    }
    if (n != (int64_t)canon_param_count()) return NPBS_ERR_INVALID_ARG;
    std::vector<float> dv;
    canon_to_dev(host, dv);
    if (cudaMemcpy(N->params, dv.data(), sizeof(float) * dv.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return NPBS_ERR_CUDA;
    if (N->refresh_bf16(nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return NPBS_ERR_CUDA;
    return NPBS_OK;
}

npbs_status npbs_net_get_params(const npbs_net* net, float* host, int64_t n) {
    if (!net) return NPBS_ERR_INVALID_ARG;
    const Net* N = reinterpret_cast<const Net*>(net);
    cudaSetDevice(N->device);
    return copy_out(*N, N->params, host, n);
}

npbs_status npbs_net_get_grads(const npbs_net* net, float* host, int64_t n) {
    if (!net) return NPBS_ERR_INVALID_ARG;
    const Net* N = reinterpret_cast<const Net*>(net);
    cudaSetDevice(N->device);
    return copy_out(*N, N->grads, host, n);
}

npbs_status npbs_net_zero_grad(npbs_net* net, npbs_stream stream) {
    if (!net) return NPBS_ERR_INVALID_ARG;
    Net* N = reinterpret_cast<Net*>(net);
    if (cudaMemsetAsync(N->grads, 0, sizeof(float) * N->count(), reinterpret_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return NPBS_ERR_CUDA;
    return NPBS_OK;
}

npbs_status npbs_net_adamw(npbs_ctx* ctx, npbs_net* net, float lr, float weight_decay, npbs_stream stream) {
    if (!ctx || !net || !(lr >= 0.f) || !(weight_decay >= 0.f)) return NPBS_ERR_INVALID_ARG;
    return net_adamw(ctx, *reinterpret_cast<Net*>(net), lr, weight_decay, reinterpret_cast<cudaStream_t>(stream));
}

// file: magic, version, step, count, params, m1, m2 (device layout, float32)
npbs_status npbs_net_save(const npbs_net* net, const char* path) {
    if (!net || !path) return NPBS_ERR_INVALID_ARG;
    const Net* N = reinterpret_cast<const Net*>(net);
    cudaSetDevice(N->device);
    const long long P = N->count();
    std::vector<float> buf(3 * P);
    if (cudaMemcpy(buf.data(), N->params, sizeof(float) * P, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + P, N->m1, sizeof(float) * P, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + 2 * P, N->m2, sizeof(float) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
        return NPBS_ERR_CUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return NPBS_ERR_INVALID_ARG;
    // an FNO file carries its shape (n, width, modes, layers, coefficient channels, identity skip)
    // after the magic
    const char magic[8] = {'N', 'P', 'B', 'S', N->fno ? 'F' : 'N', N->fno ? 'N' : 'E', N->fno ? 'O' : 'T',
                           N->fno ? '2' : '1'};
    const long long hdr[2] = {N->step, P};
    const int shape[6] = {N->fno ? N->fno->n : 0, N->fno ? N->fno->C : 0, N->fno ? N->fno->m : 0,
                          N->fno ? N->fno->L : 0, N->fno ? N->fno->ca : 0, N->fno ? N->fno->skip : 0};
    bool ok = fwrite(magic, 1, 8, f) == 8 && (!N->fno || fwrite(shape, sizeof(int), 6, f) == 6) &&
              fwrite(hdr, sizeof(long long), 2, f) == 2 &&
              fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? NPBS_OK : NPBS_ERR_INVALID_ARG;
}

npbs_status npbs_net_load(npbs_net** out, int device, const char* path) {
    if (!out || !path) return NPBS_ERR_INVALID_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return NPBS_ERR_INVALID_ARG;
    char magic[8];
    long long hdr[2];
    int shape[6] = {0, 0, 0, 0, 0, 0};
    bool ok = fread(magic, 1, 8, f) == 8;
    // FNO files: version 1 without the skip flag, version 2 with it
    const bool fno1 = ok && memcmp(magic, "NPBSFNO1", 8) == 0, fno2 = ok && memcmp(magic, "NPBSFNO2", 8) == 0;
    const bool is_fno = fno1 || fno2;
    ok = ok && (is_fno || memcmp(magic, "NPBSNET1", 8) == 0);
    if (ok && is_fno) {
        const size_t ns = fno2 ? 6 : 5;
        ok = fread(shape, sizeof(int), ns, f) == ns && shape[0] > 0 && shape[0] <= kMaxN;
    }
    long long P = 0;
    if (ok) P = is_fno ? fno_def(shape[0], shape[1], shape[2], shape[3], shape[4]).count : dev_param_count();
    ok = ok && P > 0 && fread(hdr, sizeof(long long), 2, f) == 2 && hdr[1] == P;
    std::vector<float> buf(ok ? 3 * P : 0);
    ok = ok && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return NPBS_ERR_INVALID_ARG;
    npbs_net* h = nullptr;
    npbs_status st = is_fno ? npbs_net_create_fno(&h, device, shape[0], shape[1], shape[2], shape[3], shape[4], 0)
                            : npbs_net_create(&h, device, 0);
    if (st != NPBS_OK) return st;
    Net* N = reinterpret_cast<Net*>(h);
    N->step = hdr[0];
    N->version += 1;
    if (N->fno) N->fno->skip = shape[5] ? 1 : 0;
    if (cudaMemcpy(N->params, buf.data(), sizeof(float) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(N->m1, buf.data() + P, sizeof(float) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(N->m2, buf.data() + 2 * P, sizeof(float) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        (!N->fno && N->refresh_bf16(nullptr) != cudaSuccess) || cudaDeviceSynchronize() != cudaSuccess) {
        npbs_net_destroy(h);
        return NPBS_ERR_CUDA;
    }
    *out = h;
    return NPBS_OK;
}

static npbs_status net_args(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const Plan** pl,
                            std::vector<int>* which) {
    if (!ctx || !net) return NPBS_ERR_INVALID_ARG;
    npbs_status st;
    *pl = get_plan(ctx, batch, &st);
    if (!*pl) return st;
    which->clear();
    for (int j = 0; j < (*pl)->count; ++j) which->push_back(j);
    return NPBS_OK;
}

npbs_status npbs_net_forward(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const void* r,
                             const float* n, void* c_out, npbs_stream stream) {
    const Plan* pl;
    std::vector<int> which;
    npbs_status st = net_args(ctx, net, batch, &pl, &which);
    if (st != NPBS_OK) return st;
    if (which.empty()) return NPBS_OK;
    if (!r || !n || !c_out) return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_net_forward: NULL field pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NetRun run;
    st = net_prepare(ctx, *reinterpret_cast<const Net*>(net), *pl, which, false, &run, s, n);
    if (st != NPBS_OK) return st;
    return net_run_forward(ctx, *reinterpret_cast<const Net*>(net), run, static_cast<const float2*>(r), n,
                           static_cast<float2*>(c_out), 0, s);
}

npbs_status npbs_net_backward(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* r, const float* n,
                              const void* grad_c, void* grad_r, npbs_stream stream) {
    const Plan* pl;
    std::vector<int> which;
    npbs_status st = net_args(ctx, net, batch, &pl, &which);
    if (st != NPBS_OK) return st;
    if (which.empty()) return NPBS_OK;
    if (!r || !n || !grad_c || !grad_r)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_net_backward: NULL field pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NetRun run;
    st = net_prepare(ctx, *reinterpret_cast<const Net*>(net), *pl, which, true, &run, s);
    if (st != NPBS_OK) return st;
    return net_run_backward(ctx, *reinterpret_cast<Net*>(net), run, static_cast<const float2*>(r), n,
                            static_cast<const float2*>(grad_c), static_cast<float2*>(grad_r), 0, s);
}

}  // extern "C"
