// The FNO residual-to-correction map (App. Architectural Instantiations, Eqs.
// fno_impl, fno_lift, fno_proj, lfl, nlfl) on the GPU: forward, hand-written
// adjoint and weight gradients, as a second kind of npbs_net.
//
//   M(r; a) = P( LFL_f[ NLFL_L(...NLFL_1(Phi(a))) * LFL_r(Psi(r)) ] )
//   Phi(a) = W_a LayerNorm(a) + b_a,  Psi(r) = W_r [Re r, Im r],  P(z) = W_p z
//   LFL(x) = irfft2(W^F * R(rfft2(x))) + W^loc x (+ b),  NLFL = GELU(LFL)
//
// Hyper-parameters of the paper's backbone: 25 channels, three NLFL layers,
// 45 retained modes (rows with min(ky, N - ky) < 45, columns kx < 45 of the
// half plane), the residual layer at full bandwidth (every row, kx = 0..N/2).
//
// Layout, per group of nb instances of one N x N grid: channel planes
// [nb][C][N*N] float32; spectra of channel pairs [nb][P][N*N] complex64
// (channel 2j in the real part and 2j + 1 in the imaginary part, so that one
// complex FFT transforms two real channels); retained modes compact
// [nb][C][Ky*Kx] complex64 (rows in FFT order, then columns).
//
// A spectral block y = irfft2(W * R(rfft2(x))) runs as: pack channel pairs,
// 2D FFT (row and column kernels of radix-2/3/4/8 Stockham passes in shared
// memory), extract the retained modes of each real channel
// (X_a = (Z_k + conj Z_-k) / 2, X_b = (Z_k - conj Z_-k) / 2i), mix channels
// per mode, complete the half plane to a Hermitian spectrum (on the kx = 0 and
// N/2 columns the Hermitian part, which is all the real part of irfft2 keeps)
// packed two channels per complex field, inverse 2D FFT, and an epilogue
// (1/N^2, the 1x1 convolution, bias, GELU).  Its adjoint is the same pipeline
// with the conjugate channel-transposed weights; the spectral weight gradient
// is c_kx / N^2 sum_b G_o conj(X_i), c = 2 except on the kx = 0 and N/2
// columns (c = 1).  The coefficient branch depends on a only; every call
// recomputes it (activation checkpointing in the backward).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fft2d.cuh"
#include "net.cuh"

namespace npbs {

namespace {

constexpr int kMaxC = 32;     // channel bound of the register-blocked kernels
constexpr int kModesPerBlock = 8;

int grid_of(long long n, int per = 256) { return (int)std::min<long long>((n + per - 1) / per, 152LL * 64); }

// rows of the compact mode list for m retained modes: min(ky, n - ky) < m
__host__ __device__ inline int rows_kept(int n, int m) {
    int c = 0;
    for (int k = 0; k < n; ++k) c += (k < n - k ? k : n - k) < m;
    return c;
}
// compact row index of ky (-1 if not retained)
__device__ __forceinline__ int row_index(int ky, int n, int m) {
    if (2 * m - 1 >= n) return ky;
    if (ky < m) return ky;
    if (ky >= n - m + 1) return ky - (n - 2 * m + 1);
    return -1;
}
// FFT-order row of compact row index ri
__device__ __forceinline__ int row_of(int ri, int n, int m) {
    if (2 * m - 1 >= n) return ri;
    return ri < m ? ri : ri + (n - 2 * m + 1);
}

// Mode-major layouts (complex elements), padded so that every mode's block
// and every channel row starts 16-byte aligned: weights
// Wt[k * wstride(C) + i * C + o]; spectra X[k * xstride(nb, C) + c * nbp(nb) + b]
// (per mode, one row of samples per channel).
__host__ __device__ inline long long wstride(int C) { return ((long long)C * C + 1) & ~1LL; }
__host__ __device__ inline int nbp(int nb) { return (nb + 1) & ~1; }
__host__ __device__ inline long long xstride(int nb, int C) { return (long long)C * nbp(nb); }

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

}  // namespace

namespace {

// ------------------------------------------------------------- pointwise kernels

// LayerNorm statistics of each instance's coefficient channels: mean and
// 1/sqrt(var + 1e-5); block b * ca + c reads channel c (ca channels, astride
// elements apart) of instance b
__global__ void k_ln_stats(SlotDev sd, const float* a, int ca, long long astride, float* stats) {
    __shared__ double s1[32], s2[32];
    const int b = blockIdx.x / ca, ch = blockIdx.x - (blockIdx.x / ca) * ca;
    const float* p = a + (long long)ch * astride + sd.off[b];
    double m = 0.0, q = 0.0;
    for (long long e = threadIdx.x; e < sd.np; e += blockDim.x) {
        const double v = p[e];
        m += v;
        q += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s1[w] = m; s2[w] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a1 += s1[i]; a2 += s2[i]; }
        const double mu = a1 / (double)sd.np;
        const double var = fmax(a2 / (double)sd.np - mu * mu, 0.0);
        stats[2 * blockIdx.x] = (float)mu;
        stats[2 * blockIdx.x + 1] = (float)(1.0 / sqrt(var + 1e-5));
    }
}

// z = LayerNorm(a) as channel planes [nb][ca][np]
__global__ void k_ln_plane(SlotDev sd, const float* a, int ca, long long astride, const float* stats, float* z) {
    const long long tot = (long long)sd.nb * ca * sd.np;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot; g += (long long)gridDim.x * blockDim.x) {
        const long long bc = g / sd.np;
        const long long p = g - bc * sd.np;
        const int b = (int)(bc / ca), ch = (int)(bc - (long long)b * ca);
        z[g] = (a[(long long)ch * astride + sd.off[b] + p] - stats[2 * bc]) * stats[2 * bc + 1];
    }
}

// [Re r, Im r] (or [Re, Im] of any complex field at the batch offsets) as a two-channel plane
__global__ void k_complex_planes(SlotDev sd, const float2* r, float* z) {
    const long long tot = (long long)sd.nb * sd.np;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot; g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / sd.np);
        const long long p = g - (long long)b * sd.np;
        const float2 v = r[sd.off[b] + p];
        z[((long long)b * 2) * sd.np + p] = v.x;
        z[((long long)b * 2 + 1) * sd.np + p] = v.y;
    }
}

// out[b][o][p] = sum_i M(o, i) x[b][i][p] + bias[o] (+ part of a spectral
// result Z / N^2), pre-activation optionally kept, GELU optionally applied,
// then optionally multiplied by mul[b][o][p] and added to the old out.
// M(o, i) = w[o * so + i * si] (si = 1, so = Ci for the forward 1x1; swapped
// strides give the transpose).  Z (nullable): channel o is the real (o even)
// or imaginary (o odd) part of field o / 2 of [nb][ceil(Co/2)][np].
__global__ void __launch_bounds__(256) k_mix_points(int nb, long long np, const float* x, int Ci, const float* w,
                                                    int so, int si, const float* bias, const float2* Z, float zscale,
                                                    int Co, int act, float* pre, const float* mul, float* out,
                                                    int add) {
    // the matrix (rows padded to an even length) and the bias in shared
    // memory; each thread takes two adjacent points (np is even: n is), so one
    // shared load of two weights feeds four FMAs, and the plane accesses are
    // float2 (every plane starts 256-byte aligned and np is a multiple of 4)
    __shared__ __align__(16) float Ms[kMaxC * (kMaxC + 1)];
    __shared__ float Bs[kMaxC];
    const int Ci2 = (Ci + 1) & ~1;
    for (int e = threadIdx.x; e < Co * Ci2; e += blockDim.x) {
        const int o = e / Ci2, i = e - o * Ci2;
        Ms[e] = i < Ci ? w[o * so + i * si] : 0.f;
    }
    for (int o = threadIdx.x; o < Co; o += blockDim.x) Bs[o] = bias ? bias[o] : 0.f;
    __syncthreads();
    const int Q = (Co + 1) / 2;
    const long long pairs = (long long)nb * np / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < pairs; q += (long long)gridDim.x * blockDim.x) {
        const long long g = 2 * q;
        const int b = (int)(g / np);
        const long long p = g - (long long)b * np;
        float2 xv[kMaxC];
#pragma unroll
        for (int i = 0; i < kMaxC; ++i)
            if (i < Ci2)
                xv[i] = i < Ci ? *reinterpret_cast<const float2*>(x + ((long long)b * Ci + i) * np + p)
                               : make_float2(0.f, 0.f);
        // output channels in pairs (one complex field of Z each); the next
        // pair's Z values and old outputs are loaded before this pair's
        // stores, so their latency overlaps the arithmetic
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        auto ldz = [&](int o) -> float4 {
            return Z ? *reinterpret_cast<const float4*>(Z + ((long long)b * Q + o / 2) * np + p) : zero4;
        };
        // two adjacent points of planes o and o + 1 of a [nb][Co][np] array
        auto ld2 = [&](const float* a, int o) -> float4 {
            const float2 u = *reinterpret_cast<const float2*>(a + ((long long)b * Co + o) * np + p);
            const float2 v = o + 1 < Co ? *reinterpret_cast<const float2*>(a + ((long long)b * Co + o + 1) * np + p)
                                        : make_float2(0.f, 0.f);
            return make_float4(u.x, u.y, v.x, v.y);
        };
        auto ldo = [&](int o) -> float4 { return add ? ld2(out, o) : zero4; };
        auto ldm = [&](int o) -> float4 { return mul ? ld2(mul, o) : make_float4(1.f, 1.f, 1.f, 1.f); };
        float4 zn = ldz(0), on = ldo(0), mn = ldm(0);
        for (int o = 0; o < Co; o += 2) {
            const float4 z = zn, old = on, mv = mn;
            if (o + 2 < Co) {
                zn = ldz(o + 2);
                on = ldo(o + 2);
                mn = ldm(o + 2);
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int oo = o + t;
                if (oo >= Co) break;
                float s0 = Bs[oo], s1 = Bs[oo];
                const float* mo = Ms + oo * Ci2;
#pragma unroll
                for (int i = 0; i < kMaxC; i += 2) {
                    if (i < Ci2) {
                        const float2 m = *reinterpret_cast<const float2*>(mo + i);
                        s0 = fmaf(m.x, xv[i].x, s0);
                        s1 = fmaf(m.x, xv[i].y, s1);
                        s0 = fmaf(m.y, xv[i + 1].x, s0);
                        s1 = fmaf(m.y, xv[i + 1].y, s1);
                    }
                }
                s0 = fmaf(t ? z.y : z.x, zscale, s0);
                s1 = fmaf(t ? z.w : z.z, zscale, s1);
                const long long oi = ((long long)b * Co + oo) * np + p;
                if (pre) *reinterpret_cast<float2*>(pre + oi) = make_float2(s0, s1);
                float v0 = act ? gelu_f(s0) : s0, v1 = act ? gelu_f(s1) : s1;
                v0 = fmaf(v0, t ? mv.z : mv.x, t ? old.z : old.x);
                v1 = fmaf(v1, t ? mv.w : mv.y, t ? old.w : old.y);
                *reinterpret_cast<float2*>(out + oi) = make_float2(v0, v1);
            }
        }
    }
}

// Retained half-plane modes of each real channel from the pair spectra, in
// the mode-major layout X[k * xstride(nb, Ci) + i * nbp(nb) + b] (row
// f = i * nb + b).  A block takes 32 modes x 32 rows through a shared tile:
// the spectra are read along the modes (consecutive k are consecutive kx of a
// row) and X is written along the rows.
__global__ void k_extract(int nb, int n, int m, int Kx, int K, const float2* __restrict__ Z, int Ci,
                          float2* __restrict__ X) {
    __shared__ float2 t[32][33];  // [channel row][mode]
    const int P = (Ci + 1) / 2, F = nb * Ci;
    const long long np = (long long)n * n;
    const int k0 = blockIdx.x * 32, f0 = blockIdx.y * 32;
    const int k = k0 + threadIdx.x;
    if (k < K) {
        const int ky = row_of(k / Kx, n, m), kx = k % Kx;
        const int my = ky == 0 ? 0 : n - ky, mx = kx == 0 ? 0 : n - kx;
        const long long ik = (long long)ky * n + kx, im = (long long)my * n + mx;
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int f = f0 + r;
            if (f >= F) break;
            const int i = f / nb, b = f - i * nb;
            const float2* z = Z + ((long long)b * P + i / 2) * np;
            const float2 zk = z[ik], zm = z[im];
            t[r][threadIdx.x] = (i & 1) ? make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x))
                                        : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        }
    }
    __syncthreads();
    const int f = f0 + threadIdx.x;
    if (f >= F) return;
    const int i = f / nb, b = f - i * nb;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int kk = k0 + r;
        if (kk >= K) break;
        X[(long long)kk * xstride(nb, Ci) + (long long)i * nbp(nb) + b] = t[threadIdx.x][r];
    }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Channel mixing on the retained modes, mode-major: Y[k][b][o] = sum_i
// X[k][i][b] Wt[k][i][o] (adj: Y[k][b][i] = sum_o conj(Wt[k][i][o]) X[k][o][b]),
// Wt the mode-major copy of the [Ci][Co][K] weight block, X in the padded
// layout above, Y unpadded [K][nb][O].  Work items are (mode, chunk of kMixNB
// samples), mode-major, so the items of one mode are neighbours and share its
// weights in L2.  Every warp runs its own kMixStages-deep cp.async ring: the
// weight matrix and the X chunk ([channel][kMixNB], zero past the batch) of
// the items ahead stream into the warp's shared stages while it mixes the
// current item.  Lane q = output channel; per summed channel one weight load
// and kMixNB / 2 broadcast 16-byte X loads feed 4 kMixNB FMAs.
constexpr int kMixNB = 8;
constexpr int kMixStages = 3;
constexpr int kMixWarps = 4;
__host__ __device__ inline int mix_stage(int C) {  // complex elements per stage
    return (int)(wstride(C) + kMixNB * C);
}
__global__ void __launch_bounds__(32 * kMixWarps) k_mix_modes(int nb, int K, const float2* __restrict__ X,
                                                              const float2* __restrict__ Wt, int C, int adj,
                                                              float2* __restrict__ Y) {
    extern __shared__ __align__(16) float2 ring_all[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int SZ = mix_stage(C);
    float2* ring = ring_all + (long long)wib * kMixStages * SZ;
    const long long WS = wstride(C), XS = xstride(nb, C);
    const int nch = (nb + kMixNB - 1) / kMixNB;
    const long long items = (long long)K * nch;
    const long long nw = (long long)gridDim.x * kMixWarps;
    const long long w0 = (long long)blockIdx.x * kMixWarps + wib;
    // stage item `it` into ring slot `slot` (16-byte pieces; the tail of the
    // last sample chunk is zero-filled, nothing past it is read)
    auto issue = [&](long long it, int slot) {
        const long long k = it / nch;
        const int c = (int)(it - k * nch);
        float2* sw = ring + (long long)slot * SZ;
        float2* sx = sw + WS;
        const char* gw = reinterpret_cast<const char*>(Wt + k * WS);
        const int wb = (int)(WS * 8);
        for (int o = lane * 16; o < wb; o += 32 * 16) cp_async16(reinterpret_cast<char*>(sw) + o, gw + o, 16);
        // channel p's kMixNB samples: kMixNB / 2 pieces of 16 bytes, zero-filled past nb
        const int xb = min(kMixNB, nb - c * kMixNB) * 8;
        const char* gx = reinterpret_cast<const char*>(X + k * XS + (long long)c * kMixNB);
        for (int q = lane; q < (kMixNB / 2) * C; q += 32) {
            const int p = q / (kMixNB / 2), h = q % (kMixNB / 2);
            const int bytes = max(0, min(16, xb - 16 * h));
            const char* src = gx + (long long)p * nbp(nb) * 8 + (bytes > 0 ? 16 * h : 0);
            cp_async16(reinterpret_cast<char*>(sx + p * kMixNB) + 16 * h, src, bytes);
        }
    };
#pragma unroll
    for (int s = 0; s < kMixStages - 1; ++s) {
        const long long it = w0 + s * nw;
        if (it < items) issue(it, s);
        cp_async_commit();
    }
    const bool on = lane < C;
    for (long long i = 0;; ++i) {
        const long long it = w0 + i * nw;
        if (it >= items) break;
        const long long ahead = it + (kMixStages - 1) * nw;
        if (ahead < items) issue(ahead, (int)((i + kMixStages - 1) % kMixStages));
        cp_async_commit();
        cp_async_wait<kMixStages - 1>();
        __syncwarp();
        const float2* sw = ring + (long long)(i % kMixStages) * SZ;
        const float2* sx = sw + WS;
        const long long k = it / nch;
        const int c = (int)(it - k * nch);
        const int b0 = c * kMixNB, nbc = min(kMixNB, nb - b0);
        float2 acc[kMixNB];
#pragma unroll
        for (int j = 0; j < kMixNB; ++j) acc[j] = make_float2(0.f, 0.f);
        // lane q's weight for summed channel p: Wt[k][p][q], or conj(Wt[k][q][p])
        const float2* wq = sw + (adj ? lane * C : lane);
        const int ws = adj ? 1 : C;
#pragma unroll 2
        for (int p = 0; p < C; ++p) {
            float2 w = on ? wq[p * ws] : make_float2(0.f, 0.f);
            if (adj) w.y = -w.y;
            const float4* xp = reinterpret_cast<const float4*>(sx + p * kMixNB);
#pragma unroll
            for (int h = 0; h < kMixNB / 2; ++h) {
                const float4 x2 = xp[h];
                acc[2 * h].x = fmaf(w.x, x2.x, fmaf(-w.y, x2.y, acc[2 * h].x));
                acc[2 * h].y = fmaf(w.x, x2.y, fmaf(w.y, x2.x, acc[2 * h].y));
                acc[2 * h + 1].x = fmaf(w.x, x2.z, fmaf(-w.y, x2.w, acc[2 * h + 1].x));
                acc[2 * h + 1].y = fmaf(w.x, x2.w, fmaf(w.y, x2.z, acc[2 * h + 1].y));
            }
        }
        if (on) {
            float2* yk = Y + (k * nb + b0) * C + lane;
#pragma unroll
            for (int j = 0; j < kMixNB; ++j)
                if (j < nbc) yk[(long long)j * C] = acc[j];
        }
        __syncwarp();  // this slot is refilled by the next iteration's issue
    }
    cp_async_wait<0>();
}

size_t mix_smem(int C) { return sizeof(float2) * (size_t)kMixWarps * kMixStages * mix_stage(C); }

// Y = mix(X) on K modes (see k_mix_modes); square C x C blocks
cudaError_t mix_modes(int nb, int K, const float2* X, const float2* Wt, int C, int adj, float2* Y,
                      cudaStream_t st) {
    const size_t sm = mix_smem(C);  // within the limit set_fft_attrs() raised for C <= kMaxC
    const long long items = (long long)K * ((nb + kMixNB - 1) / kMixNB);
    const int blocks = (int)std::min<long long>((items + kMixWarps - 1) / kMixWarps, 152LL * 4);
    k_mix_modes<<<blocks, 32 * kMixWarps, sm, st>>>(nb, K, X, Wt, C, adj, Y);
    return cudaGetLastError();
}

// Wt[k * WS + io] = W[io][k] for one spectral block (io = i * Co + o, W as
// float pairs at a possibly odd offset), through a 32 x 32 shared tile.
__global__ void k_wt_transpose(const float* __restrict__ W, int K, int IO, long long WS, float2* __restrict__ Wt) {
    __shared__ float2 t[32][33];
    const int k0 = blockIdx.x * 32, io0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int io = io0 + r, k = k0 + threadIdx.x;
        if (io < IO && k < K) {
            const long long e = 2 * ((long long)io * K + k);
            t[r][threadIdx.x] = make_float2(W[e], W[e + 1]);
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, io = io0 + threadIdx.x;
        if (io < IO && k < K) Wt[(long long)k * WS + io] = t[threadIdx.x][r];
    }
}

// Hermitian completion of the retained half-plane spectra, two channels per
// complex field: Z[b][q] = H(Y[.][b][2q]) + i H(Y[.][b][2q + 1]), Y mode-major
// [K][nb][Co].  Grid: points x chunks of kHermF fields (f = b * Q + q); where
// a point takes its value from (one or two) retained modes is decided once per
// thread, its fields' two channel values are read straight from the
// (L2-resident) spectra, and Z is written along the points, without shared
// memory or barriers.
constexpr int kHermF = 8;
__global__ void __launch_bounds__(256) k_hermite(int nb, int n, int m, int Kx, int K, const float2* __restrict__ Y,
                                                 int Co, float2* __restrict__ Z) {
    const int Q = (Co + 1) / 2;
    const int np = n * n;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    // value = the mode itself (form 1, kx < n/2), the conjugate of the
    // mirrored mode (form 2, kx > n/2), or half the sum of the mode and the
    // conjugate of its mirror (form 0, kx = 0 or n/2)
    const int ky = p / n, kx = p - ky * n;
    const int mky = ky == 0 ? 0 : n - ky;
    auto idx = [&](int yy, int xx) -> int {
        const int ri = row_index(yy, n, m);
        return (ri < 0 || xx >= Kx) ? -1 : ri * Kx + xx;
    };
    int i1, i2 = -1, form = 1;
    if (kx == 0 || 2 * kx == n) {
        form = 0;
        i1 = idx(ky, kx);
        i2 = idx(mky, kx);
    } else if (2 * kx < n) {
        i1 = idx(ky, kx);
    } else {
        form = 2;
        i1 = idx(mky, n - kx);
    }
    const long long rowY = (long long)nb * Co;  // entries per mode
    const float2* y1 = Y + (long long)(i1 < 0 ? 0 : i1) * rowY;
    const float2* y2 = Y + (long long)(i2 < 0 ? 0 : i2) * rowY;
    const float2 zero = make_float2(0.f, 0.f);
    const int f0 = blockIdx.y * kHermF, f1 = min(nb * Q, f0 + kHermF);
#pragma unroll 4
    for (int f = f0; f < f1; ++f) {
        const int b = f / Q, q = f - b * Q;
        const int c0 = 2 * q, c1 = 2 * q + 1;
        const long long e0 = (long long)b * Co + c0;
        const bool has1 = c1 < Co;
        float2 u0 = i1 >= 0 ? y1[e0] : zero;
        float2 u1 = (i1 >= 0 && has1) ? y1[e0 + 1] : zero;
        if (form == 0) {
            const float2 v0 = i2 >= 0 ? y2[e0] : zero;
            const float2 v1 = (i2 >= 0 && has1) ? y2[e0 + 1] : zero;
            u0 = make_float2(0.5f * (u0.x + v0.x), 0.5f * (u0.y - v0.y));
            u1 = make_float2(0.5f * (u1.x + v1.x), 0.5f * (u1.y - v1.y));
        } else if (form == 2) {
            u0.y = -u0.y;
            u1.y = -u1.y;
        }
        Z[(long long)f * np + p] = make_float2(u0.x - u1.y, u0.y + u1.x);
    }
}

// ------------------------------------------------------------- gradients

// dW[i][o][k] += c_kx / n^2 sum_b G[k][b][o] conj(X[k][b][i]) (mode-major
// spectra) for kModesPerBlock modes per block, one thread per channel pair.
__global__ void k_wgrad_modes(int nb, int n, int Kx, int K, const float2* G, const float2* X, int Ci, int Co,
                              float* dW) {
    // rows padded by one element: a warp reads gs[o][q] for up to kMaxC channels o at one q
    __shared__ float2 xs[kMaxC][kModesPerBlock + 1], gs[kMaxC][kModesPerBlock + 1];
    const int k0 = blockIdx.x * kModesPerBlock;
    const int t = threadIdx.x;
    const int i = t / Co, o = t - (t / Co) * Co;
    const bool mine = t < Ci * Co;
    float2 acc[kModesPerBlock];
#pragma unroll
    for (int q = 0; q < kModesPerBlock; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int b = 0; b < nb; ++b) {
        for (int e = t; e < (Ci + Co) * kModesPerBlock; e += blockDim.x) {
            // consecutive threads take consecutive channels of one mode
            const int q = e / (Ci + Co), c = e - q * (Ci + Co);
            const int k = k0 + q;
            if (c < Ci) xs[c][q] = k < K ? X[(long long)k * xstride(nb, Ci) + (long long)c * nbp(nb) + b]
                                         : make_float2(0.f, 0.f);
            else gs[c - Ci][q] = k < K ? G[(long long)k * xstride(nb, Co) + (long long)(c - Ci) * nbp(nb) + b]
                                       : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (mine) {
#pragma unroll
            for (int q = 0; q < kModesPerBlock; ++q) {
                const float2 g = gs[o][q], x = xs[i][q];
                acc[q].x = fmaf(g.x, x.x, fmaf(g.y, x.y, acc[q].x));
                acc[q].y = fmaf(g.y, x.x, fmaf(-g.x, x.y, acc[q].y));
            }
        }
        __syncthreads();
    }
    if (!mine) return;
    const float inv = 1.f / ((float)n * (float)n);
#pragma unroll
    for (int q = 0; q < kModesPerBlock; ++q) {
        const int k = k0 + q;
        if (k >= K) break;
        const int kx = k % Kx;
        const float c = (kx == 0 || 2 * kx == n) ? inv : 2.f * inv;
        float* w = dW + 2 * (((long long)i * Co + o) * K + k);  // (re, im) pairs, possibly odd offset
        w[0] += c * acc[q].x;
        w[1] += c * acc[q].y;
    }
}

// 1x1 weight (and bias) gradients: dW[o][i] += sum_{b,p} G[b][o][p] X[b][i][p],
// db[o] += sum G[b][o][p]; 32-pixel chunks staged in shared memory.
constexpr int kPairsPerThread = 5;
__global__ void __launch_bounds__(256) k_wgrad_points(int nb, long long np, const float* G, int Co, const float* X,
                                                      int Ci, float* dW, float* db) {
    // rows padded to 33 floats: the pair (o, i) loop reads xs[i][j] for up to
    // kMaxC channels i at one j within a warp, which a 32-float stride would
    // put in one bank
    __shared__ float gs[kMaxC][33], xs[kMaxC][33];
    const int npair = Co * Ci + (db ? Co : 0);
    float acc[kPairsPerThread];
#pragma unroll
    for (int q = 0; q < kPairsPerThread; ++q) acc[q] = 0.f;
    const long long chunks = (long long)nb * np / 32;
    for (long long ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const long long g0 = ch * 32;
        const int b = (int)(g0 / np);
        const long long p0 = g0 - (long long)b * np;
        for (int e = threadIdx.x; e < (Co + Ci) * 32; e += blockDim.x) {
            const int c = e >> 5, j = e & 31;
            if (c < Co) gs[c][j] = G[((long long)b * Co + c) * np + p0 + j];
            else xs[c - Co][j] = X ? X[((long long)b * Ci + (c - Co)) * np + p0 + j] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPairsPerThread; ++q) {
            const int t = threadIdx.x + q * blockDim.x;
            if (t < npair) {
                float s = 0.f;
                if (t < Co * Ci) {
                    const int o = t / Ci, i = t - (t / Ci) * Ci;
#pragma unroll 8
                    for (int j = 0; j < 32; ++j) s = fmaf(gs[o][j], xs[i][j], s);
                } else {
                    const int o = t - Co * Ci;
#pragma unroll 8
                    for (int j = 0; j < 32; ++j) s += gs[o][j];
                }
                acc[q] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kPairsPerThread; ++q) {
        const int t = threadIdx.x + q * blockDim.x;
        if (t < npair) {
            if (t < Co * Ci) atomicAdd(dW + t, acc[q]);
            else atomicAdd(db + (t - Co * Ci), acc[q]);
        }
    }
}

__global__ void k_gelu_back(long long cnt, const float* dy, const float* pre, float* dx) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt; g += (long long)gridDim.x * blockDim.x)
        dx[g] = dy[g] * gelu_grad(pre[g]);
}

__global__ void k_mul(long long cnt, const float* a, const float* b, float* out) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt; g += (long long)gridDim.x * blockDim.x)
        out[g] = a[g] * b[g];
}

// z = c * x: dx = c * dz, dc = x * dz
__global__ void k_mul_back(long long cnt, const float* dz, const float* c, const float* x, float* dx, float* dc) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < cnt; g += (long long)gridDim.x * blockDim.x) {
        const float d = dz[g];
        dx[g] = c[g] * d;
        dc[g] = x[g] * d;
    }
}

// out (complex, batch offsets) (+)= (sum_c w[0][c] z[c], sum_c w[1][c] z[c])
// out (+)= P z (+ r when r is non-null: the identity skip)
__global__ void k_proj(SlotDev sd, const float* z, int C, const float* w, float2* out, int add, const float2* r) {
    const long long tot = (long long)sd.nb * sd.np;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot; g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / sd.np);
        const long long p = g - (long long)b * sd.np;
        float re = 0.f, im = 0.f;
        for (int c = 0; c < C; ++c) {
            const float v = z[((long long)b * C + c) * sd.np + p];
            re = fmaf(__ldg(w + c), v, re);
            im = fmaf(__ldg(w + C + c), v, im);
        }
        if (r) {
            const float2 rv = r[sd.off[b] + p];
            re += rv.x;
            im += rv.y;
        }
        float2* o = out + sd.off[b] + p;
        *o = add ? make_float2(o->x + re, o->y + im) : make_float2(re, im);
    }
}

// dz[b][c][p] = w[0][c] Re g + w[1][c] Im g
__global__ void k_proj_back(SlotDev sd, const float2* gc, int C, const float* w, float* dz) {
    const long long tot = (long long)sd.nb * sd.np;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot; g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / sd.np);
        const long long p = g - (long long)b * sd.np;
        const float2 v = gc[sd.off[b] + p];
        for (int c = 0; c < C; ++c) dz[((long long)b * C + c) * sd.np + p] = fmaf(__ldg(w + c), v.x, __ldg(w + C + c) * v.y);
    }
}

// gr (complex, batch offsets) (+)= (sum_c w[c][0] dx[c], sum_c w[c][1] dx[c])
// gr (+)= Psi^T dx (+ gc when gc is non-null: the identity skip's gradient)
__global__ void k_lift_r_back(SlotDev sd, const float* dx, int C, const float* w, float2* gr, int add,
                              const float2* gc) {
    const long long tot = (long long)sd.nb * sd.np;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot; g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / sd.np);
        const long long p = g - (long long)b * sd.np;
        float re = 0.f, im = 0.f;
        for (int c = 0; c < C; ++c) {
            const float v = dx[((long long)b * C + c) * sd.np + p];
            re = fmaf(__ldg(w + 2 * c), v, re);
            im = fmaf(__ldg(w + 2 * c + 1), v, im);
        }
        if (gc) {
            const float2 gv = gc[sd.off[b] + p];
            re += gv.x;
            im += gv.y;
        }
        float2* o = gr + sd.off[b] + p;
        *o = add ? make_float2(o->x + re, o->y + im) : make_float2(re, im);
    }
}

}  // namespace

// ------------------------------------------------------------- host side

static bool fno_radix_plan(int n, RadixPlan* p) {
    if (n < 2 || n > kMaxN) return false;
    p->n = n;
    p->npass = 0;
    int m = n;
    while (m % 8 == 0) { p->radix[p->npass++] = 8; m /= 8; }
    while (m % 4 == 0) { p->radix[p->npass++] = 4; m /= 4; }
    while (m % 2 == 0) { p->radix[p->npass++] = 2; m /= 2; }
    while (m % 3 == 0) { p->radix[p->npass++] = 3; m /= 3; }
    return m == 1 && p->npass <= kMaxPass;
}

FnoDef fno_def(int n, int C, int m, int L, int ca) {
    FnoDef d;
    d.n = n;
    d.C = C;
    d.m = m;
    d.L = L;
    d.ca = ca;
    if (n < 2 || C < 1 || m < 1 || L < 0 || L > 8 || ca < 1 || ca > kMaxC) return d;  // count stays 0: invalid
    d.ky = rows_kept(n, m);
    d.kx = std::min(m, n / 2 + 1);
    d.fy = n;
    d.fx = n / 2 + 1;
    const long long spec = 2LL * C * C * d.ky * d.kx, full = 2LL * C * C * d.fy * d.fx;
    long long o = 0;
    d.lift_a_w = o; o += (long long)C * ca;
    d.lift_a_b = o; o += C;
    for (int l = 0; l < L; ++l) {
        d.spec[l] = o; o += spec;
        d.loc_w[l] = o; o += (long long)C * C;
        d.loc_b[l] = o; o += C;
    }
    d.lift_r = o; o += 2LL * C;
    d.spec_r = o; o += full;
    d.loc_r = o; o += (long long)C * C;
    d.spec_f = o; o += spec;
    d.loc_f = o; o += (long long)C * C;
    d.proj = o; o += 2LL * C;
    d.count = o;
    return d;
}

namespace {

// Workspace of one instance group (nb instances of the FNO's grid).
struct FnoWS {
    float* stats = nullptr;
    float *lnp = nullptr, *rp = nullptr, *gp = nullptr;
    float* c[9] = {};
    float* pre[8] = {};
    float *x0 = nullptr, *x1 = nullptr, *z = nullptr, *z1 = nullptr;
    float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *dc = nullptr;
    float2 *Zp = nullptr, *Xc = nullptr, *Yc = nullptr, *Gc = nullptr;
};

size_t ws_layout(const FnoDef& d, int nb, bool train, FnoWS* w, char* base) {
    const long long np = (long long)d.n * d.n;
    const long long plane = (long long)nb * np;            // floats per channel-plane set
    const long long K = std::max((long long)d.ky * d.kx, (long long)d.fy * d.fx);
    const long long P = (d.C + 1) / 2;
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + o : nullptr;
        o += (bytes + 255) & ~size_t(255);
        return p;
    };
    auto f = [&](long long n) { return reinterpret_cast<float*>(take(sizeof(float) * n)); };
    auto c2 = [&](long long n) { return reinterpret_cast<float2*>(take(sizeof(float2) * n)); };
    FnoWS t;
    t.stats = f(2LL * nb * d.ca);
    t.lnp = f(d.ca * plane);
    t.rp = f(2 * plane);
    const int ncoef = train ? d.L + 1 : 2;
    for (int l = 0; l < ncoef; ++l) t.c[l] = f(d.C * plane);
    t.x0 = f(d.C * plane);
    t.x1 = f(d.C * plane);
    t.z = f(d.C * plane);
    t.z1 = f(d.C * plane);
    t.Zp = c2((long long)nb * P * np);
    t.Xc = c2(xstride(nb, d.C) * K);
    t.Yc = c2((long long)nb * d.C * K);
    if (train) {
        t.gp = f(2 * plane);
        for (int l = 0; l < d.L; ++l) t.pre[l] = f(d.C * plane);
        t.g1 = f(d.C * plane);
        t.g2 = f(d.C * plane);
        t.g3 = f(d.C * plane);
        t.dc = f(d.C * plane);
        t.Gc = c2(xstride(nb, d.C) * K);
    }
    if (w) *w = t;
    return o;
}

// the coefficient activation after layer l (inference keeps two buffers)
float* coef(const FnoWS& w, const FnoDef& d, int l, bool train) { return train ? w.c[l] : w.c[l & 1]; }

// 2D transforms of Z; kx: the retained columns (and their mirrors) of the
// layer, so that a layer with few modes transforms only those columns
cudaError_t fft2(const FnoDef& d, float2* Z, long long fields, int dir, cudaStream_t st, int kx,
                 fft2d::RealPairs src = fft2d::RealPairs{}) {
    return fft2d::run(Z, nullptr, fields, d.n, dir, d.plan, d.tw, st, kx, src);
}

// Spectral layer j's block of the mode-major weight copy: j < L the NLFL
// layers, j = L the residual layer, j = L + 1 the fusion layer.
long long wt_modes(const FnoDef& d, int j) {
    return j == d.L ? (long long)d.fy * d.fx : (long long)d.ky * d.kx;
}
long long wt_canon(const FnoDef& d, int j) { return j < d.L ? d.spec[j] : j == d.L ? d.spec_r : d.spec_f; }
const float2* wt_of(const FnoDef& d, int j) {
    long long o = 0;
    for (int q = 0; q < j; ++q) o += wt_modes(d, q) * wstride(d.C);
    return d.wt + o;
}

// Refresh the mode-major weight copy from the parameters when they changed
// (allocated on first use; never called inside a graph capture with stale
// weights: every run is prepared first, and preparing refreshes it).
cudaError_t ensure_wt(const FnoDef& d, const float* P, long long version, cudaStream_t st) {
    if (d.wt && d.wt_version == version) return cudaSuccess;
    const int IO = d.C * d.C;
    if (!d.wt) {
        long long tot = 0;
        for (int j = 0; j < d.L + 2; ++j) tot += wt_modes(d, j) * wstride(d.C);
        cudaError_t e = cudaMalloc(&d.wt, sizeof(float2) * tot);
        if (e != cudaSuccess) {
            d.wt = nullptr;
            return e;
        }
    }
    for (int j = 0; j < d.L + 2; ++j) {
        const long long K = wt_modes(d, j);
        k_wt_transpose<<<dim3((unsigned)((K + 31) / 32), (unsigned)((IO + 31) / 32)), dim3(32, 8), 0, st>>>(
            P + wt_canon(d, j), (int)K, IO, wstride(d.C), const_cast<float2*>(wt_of(d, j)));
    }
    d.wt_version = version;
    return cudaGetLastError();
}

// Retained-mode spectra of the real channel planes x [nb][Ci][np] into the
// mode-major X [K][xstride(nb, Ci)] (row b * Ci + i of mode k).
cudaError_t spectra(const FnoDef& d, const FnoWS& w, int nb, const float* x, int Ci, int m, float2* X,
                    cudaStream_t st, long long* kc) {
    const int P = (Ci + 1) / 2;
    const int Kx = std::min(m, d.n / 2 + 1), K = rows_kept(d.n, m) * Kx;
    // the row transforms read the channel pairs of x directly (no packed copy)
    cudaError_t e = fft2(d, w.Zp, (long long)nb * P, -1, st, Kx, fft2d::RealPairs{x, Ci});
    if (e != cudaSuccess) return e;
    k_extract<<<dim3((unsigned)((K + 31) / 32), (unsigned)((nb * Ci + 31) / 32)), dim3(32, 8), 0, st>>>(
        nb, d.n, m, Kx, K, w.Zp, Ci, X);
    *kc += 3;
    return cudaGetLastError();
}

// out = act(irfft2(mix(Y)) / ... + M x + bias): Y [K][nb][Co] already mixed;
// the local matrix M(o, i) = wl[o * so + i * si] acts on x [nb][Ci][np].
cudaError_t synthesize(const FnoDef& d, const FnoWS& w, int nb, const float2* Y, int Co, int m, const float* x,
                       int Ci, const float* wl, int so, int si, const float* bias, int act, float* pre, float* out,
                       int add, cudaStream_t st, long long* kc, const float* mul = nullptr) {
    const long long np = (long long)d.n * d.n;
    const int Q = (Co + 1) / 2;
    const int Kx = std::min(m, d.n / 2 + 1), K = rows_kept(d.n, m) * Kx;
    k_hermite<<<dim3((unsigned)((np + 255) / 256), (unsigned)((nb * Q + kHermF - 1) / kHermF)), 256, 0, st>>>(
        nb, d.n, m, Kx, K, Y, Co, w.Zp);
    cudaError_t e = fft2(d, w.Zp, (long long)nb * Q, 1, st, Kx);
    if (e != cudaSuccess) return e;
    k_mix_points<<<grid_of((long long)nb * np / 2), 256, 0, st>>>(nb, np, x, Ci, wl, so, si, bias, w.Zp,
                                                              1.f / (float)np, Co, act, pre, mul, out, add);
    *kc += 4;
    return cudaGetLastError();
}

// One Fourier layer: out = act(irfft2(W * R(rfft2(x))) + W^loc x + b), times mul (nullable)
cudaError_t layer_fwd(const FnoDef& d, const FnoWS& w, int nb, const float* x, const float2* Wt, int m,
                      const float* wl, const float* bias, int act, float* pre, float* out, cudaStream_t st,
                      long long* kc, const float* mul = nullptr) {
    const int C = d.C;
    const int K = rows_kept(d.n, m) * std::min(m, d.n / 2 + 1);
    cudaError_t e = spectra(d, w, nb, x, C, m, w.Xc, st, kc);
    if (e != cudaSuccess) return e;
    e = mix_modes(nb, K, w.Xc, Wt, C, 0, w.Yc, st);
    *kc += 1;
    if (e != cudaSuccess) return e;
    return synthesize(d, w, nb, w.Yc, C, m, x, C, wl, C, 1, bias, act, pre, out, 0, st, kc, mul);
}

// Backward of one Fourier layer from G = dL/d(pre-activation): accumulates the
// spectral, local and bias gradients; dx = adjoint(G) (nullable).
cudaError_t layer_bwd(const FnoDef& d, const FnoWS& w, int nb, const float* x, const float2* Wt, float* dWsp, int m,
                      const float* wl, float* dwl, float* dbias, const float* G, float* dx, cudaStream_t st,
                      long long* kc) {
    const int C = d.C;
    const long long np = (long long)d.n * d.n;
    const int Kx = std::min(m, d.n / 2 + 1), K = rows_kept(d.n, m) * Kx;
    cudaError_t e = spectra(d, w, nb, x, C, m, w.Xc, st, kc);
    if (e == cudaSuccess) e = spectra(d, w, nb, G, C, m, w.Gc, st, kc);
    if (e != cudaSuccess) return e;
    const int thr = std::max(32, ((C * C + 31) / 32) * 32);
    k_wgrad_modes<<<(K + kModesPerBlock - 1) / kModesPerBlock, thr, 0, st>>>(nb, d.n, Kx, K, w.Gc, w.Xc, C, C,
                                                                             dWsp);
    k_wgrad_points<<<304, 256, 0, st>>>(nb, np, G, C, x, C, dwl, dbias);
    *kc += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!dx) return cudaSuccess;
    e = mix_modes(nb, K, w.Gc, Wt, C, 1, w.Yc, st);
    *kc += 1;
    if (e != cudaSuccess) return e;
    return synthesize(d, w, nb, w.Yc, C, m, G, C, wl, 1, C, nullptr, 0, nullptr, dx, 0, st, kc);
}

// NLFL_L(...NLFL_1(Phi(a))) of one group into coef(w, d, L), keeping every
// activation when `train`.
cudaError_t coefficient_branch(const FnoDef& d, const float* P, const FnoWS& w, const SlotDev& sd, const float* a,
                               long long astride, bool train, cudaStream_t st, long long* kc) {
    const int C = d.C, nb = sd.nb;
    const long long np = sd.np;
    k_ln_stats<<<nb * d.ca, 256, 0, st>>>(sd, a, d.ca, astride, w.stats);
    k_ln_plane<<<grid_of((long long)nb * d.ca * np), 256, 0, st>>>(sd, a, d.ca, astride, w.stats, w.lnp);
    k_mix_points<<<grid_of((long long)nb * np / 2), 256, 0, st>>>(nb, np, w.lnp, d.ca, P + d.lift_a_w, d.ca, 1,
                                                              P + d.lift_a_b, nullptr, 0.f, C, 0, nullptr,
                                                              nullptr, coef(w, d, 0, train), 0);
    *kc += 3;
    cudaError_t e = cudaGetLastError();
    for (int l = 0; l < d.L && e == cudaSuccess; ++l)
        e = layer_fwd(d, w, nb, coef(w, d, l, train), wt_of(d, l), d.m, P + d.loc_w[l], P + d.loc_b[l], 1,
                      train ? w.pre[l] : nullptr, coef(w, d, l + 1, train), st, kc);
    return e;
}

// The forward of one group, keeping every activation when `train`; cf (nullable)
// holds the coefficient branch's output already (the inference cache).
cudaError_t forward_group(const FnoDef& d, const float* P, const FnoWS& w, const NetGroup& grp, const float2* r,
                          const float* a, float2* out, int add, bool train, cudaStream_t st, long long* kc,
                          const float* cf = nullptr) {
    const SlotDev& sd = grp.sd;
    const int C = d.C, nb = sd.nb;
    const long long np = sd.np;
    cudaError_t e = cudaSuccess;
    if (!cf) {
        e = coefficient_branch(d, P, w, sd, a, grp.astride, train, st, kc);
        if (e != cudaSuccess) return e;
        cf = coef(w, d, d.L, train);
    }
    k_complex_planes<<<grid_of((long long)nb * np), 256, 0, st>>>(sd, r, w.rp);
    k_mix_points<<<grid_of((long long)nb * np / 2), 256, 0, st>>>(nb, np, w.rp, 2, P + d.lift_r, 2, 1, nullptr, nullptr,
                                                              0.f, C, 0, nullptr, nullptr, w.x0, 0);
    *kc += 2;
    if (train) {
        // the backward needs x1 = the residual layer's output as well as z = c x1
        e = layer_fwd(d, w, nb, w.x0, wt_of(d, d.L), d.fx, P + d.loc_r, nullptr, 0, nullptr, w.x1, st, kc);
        if (e != cudaSuccess) return e;
        k_mul<<<grid_of((long long)nb * C * np), 256, 0, st>>>((long long)nb * C * np, cf, w.x1, w.z);
        *kc += 1;
    } else {
        e = layer_fwd(d, w, nb, w.x0, wt_of(d, d.L), d.fx, P + d.loc_r, nullptr, 0, nullptr, w.z, st, kc, cf);
        if (e != cudaSuccess) return e;
    }
    e = layer_fwd(d, w, nb, w.z, wt_of(d, d.L + 1), d.m, P + d.loc_f, nullptr, 0, nullptr, w.z1, st, kc);
    if (e != cudaSuccess) return e;
    if (!out) return cudaSuccess;  // a recomputation for the backward needs the activations only
    k_proj<<<grid_of((long long)nb * np), 256, 0, st>>>(sd, w.z1, C, P + d.proj, out, add, d.skip ? r : nullptr);
    *kc += 1;
    return cudaGetLastError();
}

// kernel attributes of the current device: the FFT kernels' and the mixing
// kernel's shared-memory limits
cudaError_t set_fft_attrs() {
    cudaError_t e = fft2d::set_attrs();
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mix_modes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mix_smem(kMaxC));
}

}  // namespace

npbs_status fno_prepare(npbs_ctx* ctx, const Net& net, const Plan& pl, const std::vector<int>& which, bool train,
                        NetRun* run, cudaStream_t st, const float* a) {
    const FnoDef& d = *net.fno;
    run->groups.clear();
    run->train = train;
    std::vector<long long> off;
    for (int j : which) {
        const InstDev& in = pl.inst_h[j];
        if (in.nx != d.n || in.ny != d.n) {
            char buf[128];
            snprintf(buf, sizeof buf, "FNO network: instance %d is %d x %d, the network's grid is %d x %d", j, in.ny,
                     in.nx, d.n, d.n);
            return set_err(ctx, NPBS_ERR_UNSUPPORTED_SIZE, buf);
        }
        off.push_back(in.offset);
    }
    if (off.empty()) return NPBS_OK;
    NPBS_CK(ctx, set_fft_attrs());
    NPBS_CK(ctx, ensure_wt(d, net.params, net.version, st));
    NPBS_CK(ctx, ctx->net_ws.ensure(ws_layout(d, (int)off.size(), train, nullptr, nullptr)));
    NPBS_CK(ctx, ctx->work[5].ensure(sizeof(long long) * off.size()));
    long long* doff = static_cast<long long*>(ctx->work[5].p);
    NPBS_CK(ctx, cudaMemcpyAsync(doff, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
    NPBS_CK(ctx, cudaStreamSynchronize(st));
    NetGroup g;
    g.H = g.W = d.n;
    g.sd.nb = (int)off.size();
    g.sd.np = (long long)d.n * d.n;
    g.sd.off = doff;
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the offsets
    for (long long o : off) {
        for (int b = 0; b < 8; ++b) {
            h ^= (unsigned long long)((o >> (8 * b)) & 0xff);
            h *= 1099511628211ull;
        }
    }
    g.key = h;
    g.astride = pl.extent;
    run->groups.push_back(g);
    // inference: compute the coefficient branch once for this instance set,
    // outside any capture, so that the runs (and graphs captured from them)
    // only evaluate the residual path
    if (!train && a) {
        const size_t need = sizeof(float) * (size_t)g.sd.nb * d.C * g.sd.np;
        if (d.cache_bytes < need) {
            cudaFree(d.cache);
            d.cache = nullptr;
            d.cache_bytes = 0;
            NPBS_CK(ctx, cudaMalloc(&d.cache, need));
            d.cache_bytes = need;
        }
        FnoWS w;
        ws_layout(d, g.sd.nb, false, &w, static_cast<char*>(ctx->net_ws.p));
        long long kc = 0;
        NPBS_CK(ctx, coefficient_branch(d, net.params, w, g.sd, a, g.astride, false, st, &kc));
        NPBS_CK(ctx, cudaMemcpyAsync(d.cache, coef(w, d, d.L, false), need, cudaMemcpyDeviceToDevice, st));
        ctx->count(st, kc);
        d.cache_a = a;
        d.cache_key = g.key;
        d.cache_version = net.version;
    }
    return NPBS_OK;
}

npbs_status fno_run_forward(npbs_ctx* ctx, const Net& net, const NetRun& run, const float2* r, const float* a,
                            float2* out, int add, cudaStream_t st) {
    const FnoDef& d = *net.fno;
    if (!run.groups.empty()) NPBS_CK(ctx, ensure_wt(d, net.params, net.version, st));
    for (const NetGroup& g : run.groups) {
        FnoWS w;
        ws_layout(d, g.sd.nb, run.train, &w, static_cast<char*>(ctx->net_ws.p));
        long long kc = 0;
        const bool cached = !run.train && d.cache && d.cache_a == a && d.cache_key == g.key &&
                            d.cache_version == net.version;
        NPBS_CK(ctx, forward_group(d, net.params, w, g, r, a, out, add, run.train, st, &kc,
                                   cached ? d.cache : nullptr));
        ctx->count(st, kc);
    }
    return NPBS_OK;
}

// Backward of out = M(r; a): recomputes the forward keeping every activation,
// accumulates d<gc, M(r; a)>/dtheta into net.grads and writes (or adds) gr.
npbs_status fno_run_backward(npbs_ctx* ctx, Net& net, const NetRun& run, const float2* r, const float* a,
                             const float2* gc, float2* gr, int add, cudaStream_t st) {
    const FnoDef& d = *net.fno;
    const int C = d.C;
    const float* P = net.params;
    float* dP = net.grads;
    if (!run.groups.empty()) NPBS_CK(ctx, ensure_wt(d, P, net.version, st));
    for (const NetGroup& g : run.groups) {
        FnoWS w;
        ws_layout(d, g.sd.nb, true, &w, static_cast<char*>(ctx->net_ws.p));
        const SlotDev sd = g.sd;
        const int nb = sd.nb;
        const long long np = sd.np, cnt = (long long)nb * C * np;
        long long kc = 0;
        NPBS_CK(ctx, forward_group(d, P, w, g, r, a, nullptr, 0, true, st, &kc));
        // projection
        k_complex_planes<<<grid_of((long long)nb * np), 256, 0, st>>>(sd, gc, w.gp);
        k_wgrad_points<<<304, 256, 0, st>>>(nb, np, w.gp, 2, w.z1, C, dP + d.proj, nullptr);
        k_proj_back<<<grid_of((long long)nb * np), 256, 0, st>>>(sd, gc, C, P + d.proj, w.g1);
        kc += 3;
        NPBS_CK(ctx, cudaGetLastError());
        // fusion layer, then the product
        NPBS_CK(ctx, layer_bwd(d, w, nb, w.z, wt_of(d, d.L + 1), dP + d.spec_f, d.m, P + d.loc_f, dP + d.loc_f, nullptr,
                               w.g1, w.g2, st, &kc));
        k_mul_back<<<grid_of(cnt), 256, 0, st>>>(cnt, w.g2, w.c[d.L], w.x1, w.g1, w.dc);
        kc += 1;
        // residual layer and the lifting of r
        NPBS_CK(ctx, layer_bwd(d, w, nb, w.x0, wt_of(d, d.L), dP + d.spec_r, d.fx, P + d.loc_r, dP + d.loc_r,
                               nullptr, w.g1, w.g3, st, &kc));
        k_wgrad_points<<<304, 256, 0, st>>>(nb, np, w.g3, C, w.rp, 2, dP + d.lift_r, nullptr);
        k_lift_r_back<<<grid_of((long long)nb * np), 256, 0, st>>>(sd, w.g3, C, P + d.lift_r, gr, add,
                                                                   d.skip ? gc : nullptr);
        kc += 2;
        NPBS_CK(ctx, cudaGetLastError());
        // coefficient branch, last NLFL first
        for (int l = d.L - 1; l >= 0; --l) {
            k_gelu_back<<<grid_of(cnt), 256, 0, st>>>(cnt, w.dc, w.pre[l], w.g1);
            kc += 1;
            NPBS_CK(ctx, layer_bwd(d, w, nb, w.c[l], wt_of(d, l), dP + d.spec[l], d.m, P + d.loc_w[l],
                                   dP + d.loc_w[l], dP + d.loc_b[l], w.g1, w.dc, st, &kc));
        }
        k_wgrad_points<<<304, 256, 0, st>>>(nb, np, w.dc, C, w.lnp, d.ca, dP + d.lift_a_w, dP + d.lift_a_b);
        kc += 1;
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(st, kc);
    }
    return NPBS_OK;
}

}  // namespace npbs

using namespace npbs;

extern "C" {

npbs_status npbs_net_create_fno(npbs_net** out, int device, int n, int width, int modes, int layers,
                                int coef_channels, uint64_t seed) {
    if (!out) return NPBS_ERR_INVALID_ARG;
    *out = nullptr;
    RadixPlan plan;
    if (n < 4 || n % 2 || !fno_radix_plan(n, &plan) || width < 1 || width > kMaxC || layers < 0 || layers > 8 ||
        modes < 1 || modes > n / 2 + 1 || coef_channels < 1 || coef_channels > kMaxC)
        return NPBS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return NPBS_ERR_INVALID_ARG;
    Net* net = new (std::nothrow) Net();
    if (!net) return NPBS_ERR_OOM;
    net->device = device;
    net->fno = new (std::nothrow) FnoDef(fno_def(n, width, modes, layers, coef_channels));
    if (!net->fno || net->fno->count <= 0) {
        delete net;
        return NPBS_ERR_OOM;
    }
    FnoDef& d = *net->fno;
    d.plan = plan;
    const long long P = d.count;
    std::vector<float2> tw(n);
    for (int k = 0; k < n; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)n;
        tw[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    bool ok = cudaMalloc(&net->params, sizeof(float) * P) == cudaSuccess &&
              cudaMalloc(&net->grads, sizeof(float) * P) == cudaSuccess &&
              cudaMalloc(&net->m1, sizeof(float) * P) == cudaSuccess &&
              cudaMalloc(&net->m2, sizeof(float) * P) == cudaSuccess &&
              cudaMalloc(&d.tw, sizeof(float2) * n) == cudaSuccess;
    if (!ok) {
        delete net;
        return NPBS_ERR_OOM;
    }
    // seeded initial parameters: 1x1 weights uniform in +-1/sqrt(fan_in),
    // spectral weights uniform in [0, 1/C^2) for both parts, biases zero
    std::vector<float> h(P, 0.f);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto uni = [&]() {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return (double)(s >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill_w = [&](long long o, long long cnt, int fan_in) {
        const double b = 1.0 / std::sqrt((double)fan_in);
        for (long long i = 0; i < cnt; ++i) h[o + i] = (float)((2.0 * uni() - 1.0) * b);
    };
    auto fill_s = [&](long long o, long long cnt) {
        for (long long i = 0; i < cnt; ++i) h[o + i] = (float)(uni() / (double)(width * width));
    };
    const long long spec = 2LL * width * width * d.ky * d.kx, full = 2LL * width * width * d.fy * d.fx;
    fill_w(d.lift_a_w, (long long)width * coef_channels, coef_channels);
    for (int l = 0; l < layers; ++l) {
        fill_s(d.spec[l], spec);
        fill_w(d.loc_w[l], (long long)width * width, width);
    }
    fill_w(d.lift_r, 2LL * width, 2);
    fill_s(d.spec_r, full);
    fill_w(d.loc_r, (long long)width * width, width);
    fill_s(d.spec_f, spec);
    fill_w(d.loc_f, (long long)width * width, width);
    fill_w(d.proj, 2LL * width, width);
    ok = cudaMemcpy(net->params, h.data(), sizeof(float) * P, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(net->grads, 0, sizeof(float) * P) == cudaSuccess &&
         cudaMemset(net->m1, 0, sizeof(float) * P) == cudaSuccess &&
         cudaMemset(net->m2, 0, sizeof(float) * P) == cudaSuccess &&
         cudaMemcpy(d.tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        delete net;
        return NPBS_ERR_CUDA;
    }
    *out = reinterpret_cast<npbs_net*>(net);
    return NPBS_OK;
}

int64_t npbs_net_param_count(const npbs_net* net) {
    if (!net) return -1;
    const Net* N = reinterpret_cast<const Net*>(net);
    return N->fno ? (int64_t)N->fno->count : (int64_t)canon_param_count();
}

npbs_status npbs_net_fno_set_skip(npbs_net* net, int32_t on) {
    if (!net) return NPBS_ERR_INVALID_ARG;
    Net* N = reinterpret_cast<Net*>(net);
    if (!N->fno) return NPBS_ERR_UNSUPPORTED_SIZE;
    if (cudaSetDevice(N->device) != cudaSuccess) return NPBS_ERR_CUDA;
    FnoDef& d = *N->fno;
    if (on && !d.skip) {
        // the network starts as the identity: zero projection (2 x C weights)
        if (cudaMemset(N->params + d.proj, 0, sizeof(float) * 2 * d.C) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return NPBS_ERR_CUDA;
    }
    d.skip = on ? 1 : 0;
    N->version += 1;
    return NPBS_OK;
}

}  // extern "C"
