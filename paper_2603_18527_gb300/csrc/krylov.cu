// Batched restarted flexible GMRES on the Lippmann-Schwinger system
// B delta = G rho (Eq. LS_discrete), B = I - G V, after Saad 1993 (the FGMRES
// comparison of Sec. 5.1.3), one independent Krylov process per instance.
//
// Every restart cycle is also a mixed-precision refinement cycle: the float64
// residual rho = f - A u is recomputed (folding the previous correction into
// the complex128 solution), b = G rho is formed by one apply, and the cycle
// runs up to `restart` Arnoldi steps on complex64 vectors:
//   z_j = P(v_j)                       (none / CBS sweeps / network)
//   w   = B z_j                        (OP_B apply)
//   two classical Gram-Schmidt passes against v_0..v_j, dots in float64
//   h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
//   Givens rotation of the new Hessenberg column, residual estimate |g_{j+1}|
// and ends with delta = Z y (triangular solve on the device).
#include <algorithm>
#include <cmath>
#include <vector>

#include "krylov.cuh"
#include "net.cuh"
#include "solve.cuh"

namespace npbs {

constexpr int kVecThreads = 256;
constexpr int kMaxRestart = 64;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// h[inst][i] += <V_i, w> for i < nv (V_i rows of length `stride` elements).
// The basis vectors are taken kDotGroup at a time: each thread reads its
// elements of w once per group and accumulates kDotGroup products, so w is
// read ceil(nv / kDotGroup) times instead of nv times and the block reduces
// once per group.  Each thread sums its (at most kVecChunk / blockDim)
// products in float32 and the block and instance sums are float64: float64
// arithmetic per element would bound the kernel by the FP64 pipe, whose rate
// on GB300 is a small fraction of the FP32 rate (the vectors are float32).
constexpr int kDotGroup = 8;
__global__ void k_dots(const VecItem* items, const InstDev* inst, const int* active, const float2* __restrict__ Vb,
                       long long stride, int nv, const float2* __restrict__ w, double2* h, int ldh) {
    const VecItem it = items[blockIdx.x];
    if (active && !active[it.inst]) return;
    const long long base = inst[it.inst].offset + it.start;
    __shared__ double red[2 * kDotGroup][kVecThreads / 32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int i0 = 0; i0 < nv; i0 += kDotGroup) {
        float pr[kDotGroup], pi[kDotGroup];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) pr[q] = pi[q] = 0.f;
        for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
            const float2 b = w[base + e];
#pragma unroll
            for (int q = 0; q < kDotGroup; ++q) {
                if (i0 + q < nv) {
                    const float2 a = Vb[(long long)(i0 + q) * stride + base + e];
                    pr[q] = fmaf(a.x, b.x, fmaf(a.y, b.y, pr[q]));  // conj(a) b
                    pi[q] = fmaf(a.x, b.y, fmaf(-a.y, b.x, pi[q]));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) {
            const double sr = warp_sum((double)pr[q]);
            const double si = warp_sum((double)pi[q]);
            if (lane == 0) {
                red[2 * q][wp] = sr;
                red[2 * q + 1][wp] = si;
            }
        }
        __syncthreads();
        if (threadIdx.x < 2 * kDotGroup) {
            const int q = threadIdx.x >> 1, part = threadIdx.x & 1;
            if (i0 + q < nv) {
                double a = 0;
                for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a += red[threadIdx.x][k];
                double2* hp = &h[(long long)it.inst * ldh + i0 + q];
                atomicAdd(part ? &hp->y : &hp->x, a);
            }
        }
        __syncthreads();
    }
}

// w -= sum_i c[inst][i] V_i; optionally norm2[inst] += ||w||^2 of the result
// (per-thread float32 partial sums, float64 across threads, as in k_dots).
__global__ void k_update(const VecItem* items, const InstDev* inst, const int* active, const float2* __restrict__ Vb,
                         long long stride, int nv, float2* w, const double2* c, int ldc, double* norm2,
                         const int* nv_inst) {
    const VecItem it = items[blockIdx.x];
    if (active && !active[it.inst]) return;
    if (nv_inst) nv = min(nv, nv_inst[it.inst]);
    const long long base = inst[it.inst].offset + it.start;
    __shared__ float2 cs[kMaxRestart + 1];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        const double2 t = c[(long long)it.inst * ldc + i];
        cs[i] = make_float2((float)t.x, (float)t.y);
    }
    __syncthreads();
    float accf = 0.f;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        float2 x = w[base + e];
        for (int i = 0; i < nv; ++i) {
            const float2 v = Vb[(long long)i * stride + base + e];
            const float2 a = cs[i];
            x.x -= a.x * v.x - a.y * v.y;
            x.y -= a.x * v.y + a.y * v.x;
        }
        w[base + e] = x;
        accf = fmaf(x.x, x.x, fmaf(x.y, x.y, accf));
    }
    if (norm2) {
        __shared__ double red[kVecThreads / 32];
        const double acc = warp_sum((double)accf);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
            atomicAdd(norm2 + it.inst, s);
        }
    }
}

// out = x * scale[inst] where scale = 1/sqrt(norm2) (0 if the norm vanishes).
__global__ void k_normalize(const VecItem* items, const InstDev* inst, const int* active, const float2* x, float2* out,
                            const double* norm2) {
    const VecItem it = items[blockIdx.x];
    if (active && !active[it.inst]) return;
    const long long base = inst[it.inst].offset + it.start;
    const double n2 = norm2[it.inst];
    const float s = n2 > 0.0 ? (float)(1.0 / sqrt(n2)) : 0.f;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 a = x[base + e];
        out[base + e] = make_float2(a.x * s, a.y * s);
    }
}

// Per instance (one thread each): finish Hessenberg column j (h1 + h2 from the
// two Gram-Schmidt passes, h_{j+1,j} = sqrt(norm2)), apply the previous Givens
// rotations, form the new one, update g and the residual estimate.
__global__ void k_givens(int count, int j, const int* active, double2* H, int ldh, const double2* h1, const double2* h2,
                         int ldv, const double* wnorm2, double2* cs, double2* sn, double2* g, double* est) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count || (active && !active[q])) return;
    double2* col = H + (long long)q * ldh * (ldh - 1) + (long long)j * ldh;  // column j, ldh = restart + 1 rows
    for (int i = 0; i <= j; ++i) {
        col[i].x = h1[(long long)q * ldv + i].x + h2[(long long)q * ldv + i].x;
        col[i].y = h1[(long long)q * ldv + i].y + h2[(long long)q * ldv + i].y;
    }
    const double hn = sqrt(fmax(wnorm2[q], 0.0));
    col[j + 1] = make_double2(hn, 0.0);
    double2* c = cs + (long long)q * (ldh - 1);
    double2* s = sn + (long long)q * (ldh - 1);
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], b = col[i + 1];
        // [conj(c) conj(s); -s c] (a, b)
        const double2 ci = c[i], si = s[i];
        col[i] = make_double2(ci.x * a.x + ci.y * a.y + si.x * b.x + si.y * b.y,
                              ci.x * a.y - ci.y * a.x + si.x * b.y - si.y * b.x);
        col[i + 1] = make_double2(-(si.x * a.x - si.y * a.y) + (ci.x * b.x - ci.y * b.y),
                                  -(si.x * a.y + si.y * a.x) + (ci.x * b.y + ci.y * b.x));
    }
    const double2 a = col[j], b = col[j + 1];
    const double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
    double2 cj = make_double2(1.0, 0.0), sj = make_double2(0.0, 0.0);
    if (den > 0) {
        cj = make_double2(a.x / den, a.y / den);
        sj = make_double2(b.x / den, b.y / den);
    }
    c[j] = cj;
    s[j] = sj;
    col[j] = make_double2(den, 0.0);
    col[j + 1] = make_double2(0.0, 0.0);
    double2* gq = g + (long long)q * ldh;
    const double2 gj = gq[j];
    gq[j + 1] = make_double2(-(sj.x * gj.x - sj.y * gj.y), -(sj.x * gj.y + sj.y * gj.x));
    gq[j] = make_double2(cj.x * gj.x + cj.y * gj.y, cj.x * gj.y - cj.y * gj.x);
    est[q] = sqrt(gq[j + 1].x * gq[j + 1].x + gq[j + 1].y * gq[j + 1].y);
}

// y = R^{-1} g over the first k[inst] columns (upper-triangular back solve).
__global__ void k_backsolve(int count, const int* ksteps, const double2* H, int ldh, const double2* g, double2* y) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const int k = ksteps[q];
    const double2* Hq = H + (long long)q * ldh * (ldh - 1);
    double2* yq = y + (long long)q * (ldh - 1);
    const double2* gq = g + (long long)q * ldh;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = gq[i];
        for (int l = i + 1; l < k; ++l) {
            const double2 r = Hq[(long long)l * ldh + i], t = yq[l];
            acc.x -= r.x * t.x - r.y * t.y;
            acc.y -= r.x * t.y + r.y * t.x;
        }
        const double2 d = Hq[(long long)i * ldh + i];
        const double dd = d.x * d.x + d.y * d.y;
        yq[i] = dd > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                       : make_double2(0.0, 0.0);
    }
    for (int i = k; i < ldh - 1; ++i) yq[i] = make_double2(0.0, 0.0);
}

__global__ void k_negate(double2* y, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_double2(-y[i].x, -y[i].y);
}

}  // namespace npbs

using namespace npbs;

namespace {

struct Fg {
    npbs_ctx* ctx;
    const Plan* pl;
    cudaStream_t st;
    int count;
    long long ext;
    int vgrid;
};

}  // namespace

extern "C" npbs_status fgmres_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const void* k2,
                                    const void* f, const float* n, void* u, int32_t restart, int32_t precond,
                                    int32_t cbs_sweeps, const npbs_solve_opts* opts, npbs_report* report,
                                    npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    if (pl->count == 0) return NPBS_OK;
    st = check_solve_args(ctx, opts, k2, f, u);
    if (st != NPBS_OK) return st;
    if (restart < 1 || restart > kMaxRestart)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "fgmres_solve: restart must be in [1, 64]");
    if (precond < 0 || precond > 2 || (precond == 1 && cbs_sweeps < 1) || (precond == 2 && (!net || !n)))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "fgmres_solve: precond 0 (none), 1 (cbs_sweeps >= 1) or 2 (net, n)");
    cudaStream_t s = nullptr;
    st = solve_stream_begin(ctx, reinterpret_cast<cudaStream_t>(stream), &s);
    if (st != NPBS_OK) return st;
    const int cnt = pl->count;
    const int m = restart;
    const int ldh = m + 1;
    const long long ext = std::max<long long>(pl->extent, 1);
    const float2* K2 = static_cast<const float2*>(k2);
    const float2* Vp = nullptr;
    st = solver_potential(ctx, *pl, K2, s, &Vp);
    if (st != NPBS_OK) return st;
    const float2* fp = static_cast<const float2*>(f);
    double2* up = static_cast<double2*>(u);

    // workspaces: basis V (m+1), Z (m, if preconditioned), w, delta, rho
    const int nz = precond == 0 ? 0 : m;
    NPBS_CK(ctx, ctx->work[3].ensure(sizeof(float2) * ext * (size_t)(m + 1 + nz + 1)));
    NPBS_CK(ctx, ctx->work[0].ensure(ext * sizeof(float2)));
    NPBS_CK(ctx, ctx->work[1].ensure(ext * sizeof(float2)));
    // small per-instance arrays carved from one buffer (each rounded to 256 bytes)
    const size_t small_sizes[] = {sizeof(double2) * cnt * ldh * m, sizeof(double2) * cnt * ldh,
                                  sizeof(double2) * cnt * ldh,     sizeof(double2) * cnt * m,
                                  sizeof(double2) * cnt * m,       sizeof(double2) * cnt * m,
                                  sizeof(double2) * cnt * ldh,     sizeof(double) * cnt,
                                  sizeof(double) * cnt,            sizeof(double) * cnt,
                                  sizeof(double) * cnt,            sizeof(double) * cnt,
                                  sizeof(int) * cnt,               sizeof(int) * cnt,
                                  sizeof(int) * cnt};
    size_t small = 0;
    for (size_t b : small_sizes) small += (b + 255) / 256 * 256;
    NPBS_CK(ctx, ctx->work[4].ensure(small));
    NPBS_CK(ctx, ctx->scratch.ensure(ext * 16));
    float2* Vb = static_cast<float2*>(ctx->work[3].p);
    float2* Zb = nz ? Vb + ext * (m + 1) : Vb;
    float2* w = Vb + ext * (m + 1 + nz);
    float2* delta = static_cast<float2*>(ctx->work[0].p);
    float2* rho = static_cast<float2*>(ctx->work[1].p);
    char* sp = static_cast<char*>(ctx->work[4].p);
    char* const sp_end = sp + small;
    auto take = [&](size_t bytes) { char* p = sp; sp += (bytes + 255) / 256 * 256; return p; };
    double2* H = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * ldh * m));
    double2* h1 = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * ldh));
    double2* h2 = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * ldh));
    double2* cs = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * m));
    double2* sn = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * m));
    double2* y = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * m));
    double2* g = reinterpret_cast<double2*>(take(sizeof(double2) * cnt * ldh));
    double* rho2 = reinterpret_cast<double*>(take(sizeof(double) * cnt));
    double* f2 = reinterpret_cast<double*>(take(sizeof(double) * cnt));
    double* bn2 = reinterpret_cast<double*>(take(sizeof(double) * cnt));
    double* wn2 = reinterpret_cast<double*>(take(sizeof(double) * cnt));
    double* est = reinterpret_cast<double*>(take(sizeof(double) * cnt));
    int* act_run = reinterpret_cast<int*>(take(sizeof(int) * cnt));   // instances still solving
    int* act_cyc = reinterpret_cast<int*>(take(sizeof(int) * cnt));   // instances still in this cycle
    int* ksteps = reinterpret_cast<int*>(take(sizeof(int) * cnt));
    if (sp > sp_end) return set_err(ctx, NPBS_ERR_INVALID_ARG, "fgmres_solve: internal workspace layout error");

    const int vb = pl->nvec;
    const VecItem* vi = pl->vitems;

    std::vector<int> iters(cnt, 0), run(cnt, 1), cyc(cnt, 0), ks(cnt, 0);
    std::vector<double> rt(cnt, 0.0), hr(cnt), hf(cnt), hb(cnt), he(cnt);
    std::vector<npbs_status> stat(cnt, NPBS_OK);

    auto refresh = [&](bool fold) -> npbs_status {
        ApplyArgs a{};
        a.V = Vp;
        a.f = fp;
        a.out = rho;
        a.norm2 = rho2;
        a.norm2b = f2;
        a.uhi = up;
        a.k2 = K2;
        a.delta = fold ? delta : nullptr;
        npbs_status s2 = run_apply(ctx, *pl, kTrueRes64, a, fold ? act_run : nullptr, s);
        if (s2 != NPBS_OK) return s2;
        NPBS_CK(ctx, cudaMemcpyAsync(hr.data(), rho2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        NPBS_CK(ctx, cudaMemcpyAsync(hf.data(), f2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        NPBS_CK(ctx, cudaStreamSynchronize(s));
        for (int j = 0; j < cnt; ++j) {
            if (fold && !run[j]) continue;
            const double fn = std::sqrt(hf[j]), rn = std::sqrt(hr[j]);
            rt[j] = fn > 0 ? rn / fn : rn;
            if (!std::isfinite(rt[j])) { stat[j] = NPBS_ERR_NONFINITE; run[j] = 0; }
            else if (rt[j] <= opts->rtol) { stat[j] = NPBS_OK; run[j] = 0; }
            else if (iters[j] >= opts->max_iter) { stat[j] = NPBS_NOT_CONVERGED; run[j] = 0; }
            else run[j] = 1;
        }
        NPBS_CK(ctx, cudaMemcpyAsync(act_run, run.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        return NPBS_OK;
    };

    auto precondition = [&](const float2* v, float2* z) -> npbs_status {
        if (precond == 1) {
            NPBS_CK(ctx, cudaMemsetAsync(z, 0, sizeof(float2) * ext, s));
            // all sweeps fused into one launch per grid side
            ApplyArgs a{};
            a.V = Vp;
            a.f = v;
            a.x = z;
            a.out = z;
            a.steps = cbs_sweeps;
            return run_apply(ctx, *pl, NPBS_PREC_SWEEP, a, act_cyc, s);
        }
        std::vector<int> which;
        for (int q = 0; q < cnt; ++q)
            if (cyc[q]) which.push_back(q);
        NetRun runp;
        npbs_status s2 = net_prepare(ctx, *reinterpret_cast<const Net*>(net), *pl, which, false, &runp, s, n);
        if (s2 != NPBS_OK) return s2;
        return net_run_forward(ctx, *reinterpret_cast<const Net*>(net), runp, v, n, z, 0, s);
    };

    npbs_status r = refresh(false);
    if (r != NPBS_OK) return r;
    while (true) {
        bool any = false;
        for (int j = 0; j < cnt; ++j) any |= run[j] != 0;
        if (!any) break;
        // b = G rho (RESIDUAL apply at delta = 0 with source rho), v_0 = b / ||b||
        NPBS_CK(ctx, cudaMemsetAsync(delta, 0, sizeof(float2) * ext, s));
        {
            ApplyArgs a{};
            a.V = Vp;
            a.f = rho;
            a.x = delta;
            a.out = w;
            a.norm2 = bn2;
            r = run_apply(ctx, *pl, NPBS_RESIDUAL, a, act_run, s);
            if (r != NPBS_OK) return r;
        }
        k_normalize<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_run, w, Vb, bn2);
        NPBS_CK(ctx, cudaMemcpyAsync(hb.data(), bn2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        NPBS_CK(ctx, cudaMemsetAsync(g, 0, sizeof(double2) * cnt * ldh, s));
        NPBS_CK(ctx, cudaStreamSynchronize(s));
        std::vector<double2> g0(cnt * ldh, make_double2(0, 0));
        std::vector<double> target(cnt, 0.0);
        for (int j = 0; j < cnt; ++j) {
            cyc[j] = run[j];
            ks[j] = 0;
            g0[(size_t)j * ldh] = make_double2(std::sqrt(hb[j]), 0.0);
            // stop the cycle once the B-residual fell by the factor still needed (with margin)
            target[j] = std::sqrt(hb[j]) * std::min(1.0, 0.5 * opts->rtol / std::max(rt[j], 1e-300));
        }
        NPBS_CK(ctx, cudaMemcpyAsync(g, g0.data(), sizeof(double2) * cnt * ldh, cudaMemcpyHostToDevice, s));
        NPBS_CK(ctx, cudaMemcpyAsync(act_cyc, cyc.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        NPBS_CK(ctx, cudaStreamSynchronize(s));
        r = set_active_lists(ctx, *pl, cyc, act_cyc);
        if (r != NPBS_OK) return r;
        for (int j = 0; j < m; ++j) {
            float2* vj = Vb + ext * j;
            float2* zj = nz ? Zb + ext * j : vj;
            if (precond != 0) {
                r = precondition(vj, zj);
                if (r != NPBS_OK) return r;
            }
            {
                ApplyArgs a{};
                a.V = Vp;
                a.x = zj;
                a.out = w;
                r = run_apply(ctx, *pl, NPBS_OP_B, a, act_cyc, s);
                if (r != NPBS_OK) return r;
            }
            // CGS2 against v_0..v_j
            NPBS_CK(ctx, cudaMemsetAsync(h1, 0, sizeof(double2) * cnt * ldh, s));
            NPBS_CK(ctx, cudaMemsetAsync(h2, 0, sizeof(double2) * cnt * ldh, s));
            NPBS_CK(ctx, cudaMemsetAsync(wn2, 0, sizeof(double) * cnt, s));
            k_dots<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_cyc, Vb, ext, j + 1, w, h1, ldh);
            k_update<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_cyc, Vb, ext, j + 1, w, h1, ldh, nullptr, nullptr);
            k_dots<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_cyc, Vb, ext, j + 1, w, h2, ldh);
            k_update<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_cyc, Vb, ext, j + 1, w, h2, ldh, wn2, nullptr);
            k_normalize<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_cyc, w, Vb + ext * (j + 1), wn2);
            k_givens<<<(cnt + 127) / 128, 128, 0, s>>>(cnt, j, act_cyc, H, ldh, h1, h2, ldh, wn2, cs, sn, g, est);
            NPBS_CK(ctx, cudaGetLastError());
            ctx->count(s, 7);
            NPBS_CK(ctx, cudaMemcpyAsync(he.data(), est, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
            NPBS_CK(ctx, cudaStreamSynchronize(s));
            bool any_c = false;
            for (int q = 0; q < cnt; ++q) {
                if (!cyc[q]) continue;
                ks[q] = j + 1;
                iters[q] += 1;
                if (he[q] <= target[q] || !std::isfinite(he[q]) || iters[q] >= opts->max_iter) cyc[q] = 0;
                any_c |= cyc[q] != 0;
            }
            if (!any_c) break;
            NPBS_CK(ctx, cudaMemcpyAsync(act_cyc, cyc.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
            NPBS_CK(ctx, cudaStreamSynchronize(s));
            r = set_active_lists(ctx, *pl, cyc, act_cyc);
            if (r != NPBS_OK) return r;
        }
        // delta = Z y
        NPBS_CK(ctx, cudaMemcpyAsync(ksteps, ks.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        k_backsolve<<<(cnt + 127) / 128, 128, 0, s>>>(cnt, ksteps, H, ldh, g, y);
        // delta = 0 - sum (-y_i) z_i: reuse the update kernel with negated coefficients
        NPBS_CK(ctx, cudaMemsetAsync(delta, 0, sizeof(float2) * ext, s));
        k_negate<<<(cnt * m + 255) / 256, 256, 0, s>>>(y, cnt * m);
        k_update<<<vb, kVecThreads, 0, s>>>(vi, pl->inst, act_run, nz ? Zb : Vb, ext, m, delta, y, m, nullptr, ksteps);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(s, 3);
        r = refresh(true);
        if (r != NPBS_OK) return r;
    }
    npbs_status ret = NPBS_OK;
    for (int j = 0; j < cnt; ++j) {
        if (report) {
            if (report->iters) report->iters[j] = iters[j];
            if (report->rtol) report->rtol[j] = rt[j];
            if (report->status) report->status[j] = stat[j];
        }
        if (stat[j] == NPBS_ERR_NONFINITE) ret = NPBS_ERR_NONFINITE;
        else if (stat[j] != NPBS_OK && ret == NPBS_OK) ret = NPBS_NOT_CONVERGED;
    }
    return ret;
}
