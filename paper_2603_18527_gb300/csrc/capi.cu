// C ABI: context, batch plans, potential set-up and the fused apply entry.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>

#include "conv.cuh"
#include "ctx.cuh"

namespace npbs {

Plan::~Plan() {
    cudaFree(inst);
    cudaFree(plans);
    cudaFree(tw32);
    cudaFree(twds);
    cudaFree(rows32);
    cudaFree(cols32);
    cudaFree(rows64);
    cudaFree(cols64);
    cudaFree(vitems);
    cudaFree(rows32s);
    cudaFree(cols32s);
    for (auto& g : fast) {
        cudaFree(g.list);
        cudaFree(g.alist);
    }
}

cudaError_t DevBuf::ensure(size_t need) {
    if (need <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e == cudaSuccess) bytes = need;
    return e;
}

DevBuf::~DevBuf() {
    if (p) cudaFree(p);
}

npbs_status set_err(npbs_ctx* ctx, npbs_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

npbs_status cuda_err(npbs_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") at " + where;
    return set_err(ctx, e == cudaErrorMemoryAllocation ? NPBS_ERR_OOM : NPBS_ERR_CUDA, m);
}

// 2^a 3^b with 2 <= n <= 1024; radices 8, 4, 2 then 3.
static bool radix_plan(int n, RadixPlan* p) {
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

template <typename T> static cudaError_t upload(T** dst, const std::vector<T>& v) {
    if (v.empty()) { *dst = nullptr; return cudaSuccess; }
    cudaError_t e = cudaMalloc(dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

const Plan* get_plan(npbs_ctx* ctx, const npbs_batch* batch, npbs_status* st) {
    *st = NPBS_OK;
    if (!batch || batch->count < 0 || (batch->count > 0 && !batch->inst)) {
        *st = set_err(ctx, NPBS_ERR_INVALID_ARG, "batch is NULL, has a negative count or a NULL instance array");
        return nullptr;
    }
    std::string key(reinterpret_cast<const char*>(batch->inst), sizeof(npbs_instance) * batch->count);
    auto itp = ctx->plans.find(key);
    if (itp != ctx->plans.end()) {
        itp->second->last_use = ++ctx->plan_clock;
        return itp->second.get();
    }

    auto pl = std::make_unique<Plan>();
    pl->count = batch->count;
    std::map<int, int> plan_of, tw_of;
    std::vector<RadixPlan> plans;
    std::vector<float2> tw32;
    std::vector<float4> twds;
    auto add_n = [&](int n) -> bool {
        if (plan_of.count(n)) return true;
        RadixPlan rp;
        if (!radix_plan(n, &rp)) return false;
        plan_of[n] = (int)plans.size();
        plans.push_back(rp);
        tw_of[n] = (int)tw32.size();
        for (int k = 0; k < n; ++k) {
            const double a = -2.0 * M_PI * (double)k / (double)n;
            const double c = std::cos(a), s = std::sin(a);
            const float ch = (float)c, sh = (float)s;
            twds.push_back(make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh)));
            tw32.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
        return true;
    };
    std::vector<RowItem> r32, r64;
    std::vector<ColItem> c32, c64;
    std::vector<VecItem> vit;
    std::vector<RowItem> r32s;
    std::vector<ColItem> c32s;
    std::map<int, std::vector<int>> fastlists;
    for (int j = 0; j < batch->count; ++j) {
        const npbs_instance& s = batch->inst[j];
        char buf[256];
        if (!(s.h > 0.0) || !std::isfinite(s.h) || !std::isfinite(s.k0sq) || !(s.eps > 0.0) ||
            !std::isfinite(s.eps) || s.offset < 0 || (s.offset % 32) != 0) {
            snprintf(buf, sizeof buf, "instance %d: need h > 0, eps > 0, finite k0sq and offset >= 0, multiple of 32", j);
            *st = set_err(ctx, NPBS_ERR_INVALID_ARG, buf);
            return nullptr;
        }
        if (!add_n(s.nx) || !add_n(s.ny)) {
            snprintf(buf, sizeof buf, "instance %d: grid %d x %d is not 2^a 3^b in [2, %d]", j, s.ny, s.nx, kMaxN);
            *st = set_err(ctx, NPBS_ERR_UNSUPPORTED_SIZE, buf);
            return nullptr;
        }
        InstDev d;
        d.nx = s.nx;
        d.ny = s.ny;
        d.plan_x = plan_of[s.nx];
        d.plan_y = plan_of[s.ny];
        d.tw_x = tw_of[s.nx];
        d.tw_y = tw_of[s.ny];
        d.h = s.h;
        d.k0sq = s.k0sq;
        d.eps = s.eps;
        d.offset = s.offset;
        pl->inst_h.push_back(d);
        pl->extent = std::max<long long>(pl->extent, s.offset + (long long)s.nx * s.ny);
        pl->points += (long long)s.nx * s.ny;
        for (long long st0 = 0; st0 < (long long)s.nx * s.ny; st0 += kVecChunk) {
            VecItem v{j, (int)st0, (int)std::min<long long>(kVecChunk, (long long)s.nx * s.ny - st0), 0};
            vit.push_back(v);
        }
        const bool fast = ctx->use_fast && s.nx == s.ny && fast_supported(s.nx);
        if (fast) fastlists[s.nx].push_back(j);
        for (int f64 = 0; f64 < 2; ++f64) {
            const int tile = f64 ? kTileElems<double>() : kTileElems<float>();
            const int rp = std::max(1, std::min(s.ny, tile / s.nx));
            for (int r0 = 0; r0 < s.ny; r0 += rp) {
                RowItem it{j, r0, std::min(rp, s.ny - r0), 0};
                (f64 ? r64 : r32).push_back(it);
                if (!f64 && !fast) r32s.push_back(it);
            }
            const int cp = std::max(1, std::min(16, tile / s.ny));
            for (int c0 = 0; c0 < s.nx; c0 += cp) {
                ColItem it{j, c0, std::min(cp, s.nx - c0), 0};
                (f64 ? c64 : c32).push_back(it);
                if (!f64 && !fast) c32s.push_back(it);
            }
        }
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = upload(&pl->inst, pl->inst_h);
    if (e == cudaSuccess) e = upload(&pl->plans, plans);
    if (e == cudaSuccess) e = upload(&pl->tw32, tw32);
    if (e == cudaSuccess) e = upload(&pl->twds, twds);
    if (e == cudaSuccess) e = upload(&pl->rows32, r32);
    if (e == cudaSuccess) e = upload(&pl->cols32, c32);
    if (e == cudaSuccess) e = upload(&pl->rows64, r64);
    if (e == cudaSuccess) e = upload(&pl->cols64, c64);
    if (e == cudaSuccess) e = upload(&pl->vitems, vit);
    if (e == cudaSuccess) e = upload(&pl->rows32s, r32s);
    if (e == cudaSuccess) e = upload(&pl->cols32s, c32s);
    for (auto& kv : fastlists) {
        if (e != cudaSuccess) break;
        Plan::FastGroup g;
        g.n = kv.first;
        g.count = (int)kv.second.size();
        g.list_h = kv.second;
        e = upload(&g.list, kv.second);
        if (e == cudaSuccess) e = upload(&g.alist, kv.second);
        g.acount = g.count;
        pl->fast.push_back(g);
    }
    if (e != cudaSuccess) {
        *st = cuda_err(ctx, e, "plan upload");
        return nullptr;
    }
    pl->nrow32 = (int)r32.size();
    pl->ncol32 = (int)c32.size();
    pl->nrow64 = (int)r64.size();
    pl->ncol64 = (int)c64.size();
    pl->nvec = (int)vit.size();
    pl->nrow32s = (int)r32s.size();
    pl->ncol32s = (int)c32s.size();
    // bounded cache: evict the least recently used plan (no call is in flight
    // across this point, and captured graphs never outlive the call that made them)
    if (ctx->plans.size() >= 256) {
        auto victim = ctx->plans.begin();
        for (auto it = ctx->plans.begin(); it != ctx->plans.end(); ++it)
            if (it->second->last_use < victim->second->last_use) victim = it;
        ctx->plans.erase(victim);
    }
    pl->last_use = ++ctx->plan_clock;
    const Plan* out = pl.get();
    ctx->plans[key] = std::move(pl);
    return out;
}

npbs_status run_apply(npbs_ctx* ctx, const Plan& pl, int mode, const ApplyArgs& a0, const int* active,
                      cudaStream_t st) {
    const bool f64 = (mode == kTrueRes64);
    ApplyArgs a = a0;
    NPBS_CK(ctx, ctx->scratch.ensure((size_t)std::max<long long>(pl.extent, 1) * (f64 ? 16 : 8)));
    a.scratch = ctx->scratch.p;
    if (a.norm2) NPBS_CK(ctx, cudaMemsetAsync(a.norm2, 0, sizeof(double) * pl.count, st));
    if (a.norm2b) NPBS_CK(ctx, cudaMemsetAsync(a.norm2b, 0, sizeof(double) * pl.count, st));
    BatchDev bd = pl.bd(f64, active);
    if (f64) {
        NPBS_CK(ctx, launch_apply(mode, bd, pl.nrow64, pl.ncol64, a, st));
        ctx->count(st, 3);
        return NPBS_OK;
    }
    const bool compact = active && active == pl.alist_mask;
    // grid sides with work, largest first: each side is one cluster launch
    // (three band launches for 1024);
    // with several sides the larger ones go to side streams so that the
    // few-wave launches of the large grids overlap the others
    std::vector<std::pair<int, FastDev>> todo;
    for (const auto& g : pl.fast) {
        FastDev fd{compact ? g.alist : g.list, compact ? g.acount : g.count};
        if (fd.count > 0) todo.emplace_back(g.n, fd);
    }
    std::sort(todo.begin(), todo.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    const int nside = (int)todo.size() > 1 && ctx->fork_ev ? std::min<int>((int)todo.size() - 1, npbs_ctx::kAux) : 0;
    if (nside > 0) NPBS_CK(ctx, cudaEventRecord(ctx->fork_ev, st));
    for (int i = 0; i < (int)todo.size(); ++i) {
        const int n = todo[i].first;
        auto itv = ctx->fast_variant.find(n);
        int var = itv == ctx->fast_variant.end() ? 0 : itv->second;
        auto itt = ctx->fast_tail.find(n);
        if (itt != ctx->fast_tail.end() && todo[i].second.count <= itt->second.second) var = itt->second.first;
        cudaStream_t s = i < nside ? ctx->aux[i] : st;
        if (i < nside) NPBS_CK(ctx, cudaStreamWaitEvent(s, ctx->fork_ev, 0));
        // fused steps pay off while a group is a single latency-bound wave;
        // larger groups run one launch per step
        const bool iter = mode == NPBS_CBS_STEP || mode == NPBS_PREC_SWEEP;
        auto itf = ctx->fast_fused_max.find(n);
        const int fmax = itf == ctx->fast_fused_max.end() ? npbs_ctx::kDefaultFusedMax : itf->second;
        if (iter && a.steps > 1 && todo[i].second.count > fmax) {
            for (int k = 0; k < a.steps; ++k) {
                ApplyArgs ak = a;
                ak.steps = 1;
                if (k > 0) ak.x = a.out;
                if (k < a.steps - 1) ak.norm2 = nullptr;
                NPBS_CK(ctx, launch_apply_fast(n, var, mode, todo[i].second, bd, ak, s));
            }
            ctx->count(st, (long long)a.steps * fast_kernel_launches(n, mode, 1));
        } else {
            NPBS_CK(ctx, launch_apply_fast(n, var, mode, todo[i].second, bd, a, s));
            ctx->count(st, fast_kernel_launches(n, mode, a.steps));
        }
        if (i < nside) NPBS_CK(ctx, cudaEventRecord(ctx->join_ev[i], s));
    }
    for (int i = 0; i < nside; ++i) NPBS_CK(ctx, cudaStreamWaitEvent(st, ctx->join_ev[i], 0));
    if (pl.nrow32s > 0) {
        bd.rows = pl.rows32s;
        bd.cols = pl.cols32s;
        // the three-launch path takes fused steps one apply at a time
        const bool iter = mode == NPBS_CBS_STEP || mode == NPBS_PREC_SWEEP;
        const int nsteps = iter ? std::max(1, a.steps) : 1;
        for (int k = 0; k < nsteps; ++k) {
            ApplyArgs ak = a;
            if (k > 0) ak.x = a.out;
            if (k < nsteps - 1) ak.norm2 = nullptr;
            NPBS_CK(ctx, launch_apply(mode, bd, pl.nrow32s, pl.ncol32s, ak, st));
            ctx->count(st, 3);
        }
    }
    return NPBS_OK;
}

npbs_status set_active_lists(npbs_ctx* ctx, const Plan& pl, const std::vector<int>& act, const int* active_dev) {
    for (const auto& g : pl.fast) {
        std::vector<int> l;
        for (int j : g.list_h)
            if (act[j]) l.push_back(j);
        if (!l.empty()) NPBS_CK(ctx, cudaMemcpy(g.alist, l.data(), sizeof(int) * l.size(), cudaMemcpyHostToDevice));
        g.acount = (int)l.size();
    }
    pl.alist_mask = active_dev;
    return NPBS_OK;
}

// k0^2 = (min Re k^2 + max Re k^2)/2, eps = max |k^2 - k0^2|, V = k^2 - k0^2 - i eps.
__global__ void k_potential(const InstDev* inst, const float2* k2, float2* V, double* consts) {
    __shared__ float smin[32], smax[32];
    __shared__ double sd[32];
    __shared__ double c0, c1;
    const InstDev in = inst[blockIdx.x];
    const long long n = (long long)in.nx * in.ny;
    const float2* p = k2 + in.offset;
    float mn = 3.0e38f, mx = -3.0e38f;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const float v = p[e].x;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { smin[w] = mn; smax[w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = smin[0], b = smax[0];
        for (int i = 1; i < nw; ++i) { a = fminf(a, smin[i]); b = fmaxf(b, smax[i]); }
        c0 = 0.5 * ((double)a + (double)b);
    }
    __syncthreads();
    const double k0sq = c0;
    double m = 0.0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const double dr = (double)p[e].x - k0sq, di = (double)p[e].y;
        m = fmax(m, dr * dr + di * di);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sd[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = sd[0];
        for (int i = 1; i < nw; ++i) a = fmax(a, sd[i]);
        c1 = sqrt(a);
        consts[2 * blockIdx.x] = k0sq;
        consts[2 * blockIdx.x + 1] = c1;
    }
    __syncthreads();
    const double eps = c1;
    if (V) {
        float2* q = V + in.offset;
        for (long long e = threadIdx.x; e < n; e += blockDim.x)
            q[e] = make_float2((float)((double)p[e].x - k0sq), (float)((double)p[e].y - eps));
    }
}

// Depth (cells, 1..w) of index j into a w-cell absorbing layer at both ends
// of a line of n cells; 0 in the interior.  The upper end wins where the two
// layers overlap (w > n / 2).
__device__ __forceinline__ int layer_depth(int j, int n, int w) {
    int d = j < w ? w - j : 0;
    if (j >= n - w) d = j - (n - w) + 1;
    return d;
}

// k^2 = omega^2 n^2 + i a omega^2 rho^2 with rho = max(depth_x, depth_y) / w
// (quadratic imaginary ramp, the larger depth in the corners), in float64,
// stored as complex64.  One block row of the grid per instance.
__global__ void k_medium(const InstDev* inst, const float* n, const double* omega, int w, double amp,
                         float2* k2) {
    const InstDev in = inst[blockIdx.y];
    const double om = omega[blockIdx.y];
    const long long np = (long long)in.nx * in.ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < np; e += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(e / in.nx), x = (int)(e - (long long)y * in.nx);
        double rho = 0.0;
        if (w > 0) {
            const int d = max(layer_depth(y, in.ny, w), layer_depth(x, in.nx, w));
            rho = (double)d / (double)w;
        }
        const double nn = (double)n[in.offset + e];
        const double re = (om * om) * (nn * nn);
        const double im = amp * om * om * (rho * rho);
        k2[in.offset + e] = make_float2((float)re, (float)im);
    }
}

}  // namespace npbs

using namespace npbs;

extern "C" {

const char* npbs_version(void) { return "npbs-gb300 0.1 (sm_103a)"; }

npbs_status npbs_create(npbs_ctx** out, int device) {
    if (!out) return NPBS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NPBS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return NPBS_ERR_CUDA;
    if (prepare_apply() != cudaSuccess) return NPBS_ERR_CUDA;
    if (prepare_apply_fast() != cudaSuccess) return NPBS_ERR_CUDA;
    if (prepare_conv_tc() != cudaSuccess) return NPBS_ERR_CUDA;
    npbs_ctx* c = new (std::nothrow) npbs_ctx();
    if (!c) return NPBS_ERR_OOM;
    c->device = device;
    {
        bool ok = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < npbs_ctx::kAux && ok; ++i)
            ok = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            npbs_destroy(c);
            return NPBS_ERR_CUDA;
        }
    }
    const char* env = getenv("NPBS_APPLY_PATH");
    c->use_fast = !(env && strcmp(env, "three_pass") == 0);
    // NPBS_FAST_VARIANT="256:1,512:0" pins cluster-kernel variants
    if (const char* fv = getenv("NPBS_FAST_VARIANT")) {
        int n = 0, v = 0, used = 0;
        while (sscanf(fv, "%d:%d%n", &n, &v, &used) == 2) {
            if (v >= 0 && v < fast_variants(n)) c->fast_variant[n] = v;
            fv += used;
            if (*fv != ',') break;
            ++fv;
        }
    }
    *out = c;
    return NPBS_OK;
}

npbs_status npbs_destroy(npbs_ctx* ctx) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->solve_stream) {
        cudaStreamSynchronize(ctx->solve_stream);
        cudaStreamDestroy(ctx->solve_stream);
    }
    if (ctx->solve_event) cudaEventDestroy(ctx->solve_event);
    for (int i = 0; i < npbs_ctx::kAux; ++i) {
        if (ctx->aux[i]) {
            cudaStreamSynchronize(ctx->aux[i]);
            cudaStreamDestroy(ctx->aux[i]);
        }
        if (ctx->join_ev[i]) cudaEventDestroy(ctx->join_ev[i]);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    delete ctx;
    return NPBS_OK;
}

const char* npbs_last_error(const npbs_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int64_t npbs_launch_count(const npbs_ctx* ctx) { return ctx ? (int64_t)ctx->launches : -1; }

npbs_status npbs_potential_from_k2(npbs_ctx* ctx, const npbs_batch* batch, const void* k2, void* V_out,
                                   double* k0sq_out, double* eps_out, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!batch || batch->count < 0 || (batch->count > 0 && (!batch->inst || !k2 || !k0sq_out || !eps_out)))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_potential_from_k2: NULL argument");
    if (batch->count == 0) return NPBS_OK;
    // the constants are outputs here: plan with placeholders that pass validation
    std::vector<npbs_instance> tmp(batch->inst, batch->inst + batch->count);
    for (auto& t : tmp) { t.k0sq = 0.0; t.eps = 1.0; }
    npbs_batch b2{batch->count, tmp.data()};
    npbs_status st;
    const Plan* pl = get_plan(ctx, &b2, &st);
    if (!pl) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NPBS_CK(ctx, ctx->work[7].ensure(sizeof(double) * 2 * batch->count));
    double* dc = static_cast<double*>(ctx->work[7].p);
    k_potential<<<batch->count, 1024, 0, s>>>(pl->inst, static_cast<const float2*>(k2), static_cast<float2*>(V_out), dc);
    NPBS_CK(ctx, cudaGetLastError());
    ctx->count(s, 1);
    std::vector<double> hc(2 * batch->count);
    NPBS_CK(ctx, cudaMemcpyAsync(hc.data(), dc, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaStreamSynchronize(s));
    for (int j = 0; j < batch->count; ++j) {
        k0sq_out[j] = hc[2 * j];
        eps_out[j] = hc[2 * j + 1];
    }
    return NPBS_OK;
}

npbs_status npbs_build_potential(npbs_ctx* ctx, const npbs_batch* batch, const float* n, const double* omega,
                                 int32_t layer_cells, double ramp_amp_over_omega2, void* k2_out, void* V_out,
                                 double* k0sq_out, double* eps_out, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!batch || batch->count < 0 || (batch->count > 0 && (!batch->inst || !n || !omega || !k0sq_out || !eps_out)))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_build_potential: NULL argument");
    if (layer_cells < 0 || !(ramp_amp_over_omega2 >= 0.0) || !std::isfinite(ramp_amp_over_omega2))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_build_potential: need layer_cells >= 0 and a finite ramp >= 0");
    if (batch->count == 0) return NPBS_OK;
    if (batch->count > 65535) return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_build_potential: more than 65535 instances");
    for (int j = 0; j < batch->count; ++j)
        if (!(omega[j] > 0.0) || !std::isfinite(omega[j])) {
            char buf[128];
            snprintf(buf, sizeof buf, "npbs_build_potential: instance %d: need a finite omega > 0", j);
            return set_err(ctx, NPBS_ERR_INVALID_ARG, buf);
        }
    std::vector<npbs_instance> tmp(batch->inst, batch->inst + batch->count);
    for (auto& t : tmp) { t.k0sq = 0.0; t.eps = 1.0; }
    npbs_batch b2{batch->count, tmp.data()};
    npbs_status st;
    const Plan* pl = get_plan(ctx, &b2, &st);
    if (!pl) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float2* k2 = static_cast<float2*>(k2_out);
    if (!k2) {
        NPBS_CK(ctx, ctx->work[10].ensure(sizeof(float2) * (size_t)std::max<long long>(pl->extent, 1)));
        k2 = static_cast<float2*>(ctx->work[10].p);
    }
    NPBS_CK(ctx, ctx->work[11].ensure(sizeof(double) * batch->count));
    double* dom = static_cast<double*>(ctx->work[11].p);
    NPBS_CK(ctx, cudaMemcpyAsync(dom, omega, sizeof(double) * batch->count, cudaMemcpyHostToDevice, s));
    dim3 grid(64, (unsigned)batch->count);
    k_medium<<<grid, 256, 0, s>>>(pl->inst, n, dom, layer_cells, ramp_amp_over_omega2, k2);
    NPBS_CK(ctx, cudaGetLastError());
    ctx->count(s, 1);
    return npbs_potential_from_k2(ctx, batch, k2, V_out, k0sq_out, eps_out, stream);
}

npbs_status npbs_autotune_apply(npbs_ctx* ctx, const npbs_batch* batch, const void* V, const void* f, void* x,
                                int32_t reps, int32_t* chosen, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    if (!V || !f || !x || reps < 1) return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_autotune_apply: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NPBS_CK(ctx, ctx->scratch.ensure((size_t)std::max<long long>(pl->extent, 1) * 8));
    ApplyArgs a{};
    a.V = static_cast<const float2*>(V);
    a.f = static_cast<const float2*>(f);
    a.x = static_cast<const float2*>(x);
    a.out = static_cast<float2*>(x);
    a.scratch = ctx->scratch.p;
    const BatchDev bd = pl->bd(false, nullptr);
    cudaEvent_t e0, e1;
    NPBS_CK(ctx, cudaEventCreate(&e0));
    NPBS_CK(ctx, cudaEventCreate(&e1));
    // milliseconds per launch of variant v over the first cnt instances of g
    // (`steps` fused CBS steps per launch)
    auto time_v = [&](const Plan::FastGroup& g, int v, int cnt, int nrep, float* ms, int steps = 1) -> cudaError_t {
        FastDev fd{g.list, cnt};
        ApplyArgs as = a;
        as.steps = steps;
        cudaError_t e = launch_apply_fast(g.n, v, NPBS_CBS_STEP, fd, bd, as, s);  // warm-up
        for (int r = 0; r < nrep && e == cudaSuccess; ++r) {
            if (r == 0) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_apply_fast(g.n, v, NPBS_CBS_STEP, fd, bd, as, s);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        ctx->count(s, (long long)(nrep + 1) * fast_kernel_launches(g.n, NPBS_CBS_STEP, steps));
        *ms /= (float)nrep;
        return e;
    };
    int gi = 0;
    cudaError_t e = cudaSuccess;
    for (const auto& g : pl->fast) {
        // throughput: the whole group
        float best = 1e30f, ms = 0.f;
        int bestv = 0;
        for (int v = 0; v < fast_variants(g.n) && e == cudaSuccess; ++v) {
            e = time_v(g, v, g.count, reps, &ms);
            if (e == cudaSuccess && ms < best) { best = ms; bestv = v; }
        }
        // latency: one instance; then the largest power-of-two count up to
        // which the lowest-latency variant still beats the throughput one
        const int lreps = std::max(reps, 20);
        float lbest = 1e30f;
        int tailv = bestv, tailmax = 0;
        for (int v = 0; v < fast_variants(g.n) && e == cudaSuccess; ++v) {
            e = time_v(g, v, 1, lreps, &ms);
            if (e == cudaSuccess && ms < lbest) { lbest = ms; tailv = v; }
        }
        if (tailv != bestv) {
            for (int k = 1; k < g.count && e == cudaSuccess; k *= 2) {
                float mt = 0.f, mb = 0.f;
                e = time_v(g, tailv, k, lreps, &mt);
                if (e == cudaSuccess) e = time_v(g, bestv, k, lreps, &mb);
                if (e != cudaSuccess || mt >= mb) break;
                tailmax = k;
            }
        }
        // fused steps: the largest power-of-two count (or the whole group) for
        // which one launch of kFs fused steps beats kFs launches
        constexpr int kFs = 8;
        int fusedmax = 0;
        for (int k = 1; e == cudaSuccess; k = std::min(2 * k, g.count)) {
            const int v = k <= tailmax ? tailv : bestv;
            float mf = 0.f, ms1 = 0.f;
            e = time_v(g, v, k, std::max(reps, 4), &mf, kFs);
            if (e == cudaSuccess) e = time_v(g, v, k, kFs * std::max(reps, 4), &ms1, 1);
            if (e != cudaSuccess || mf >= kFs * ms1) break;
            fusedmax = k;
            if (k == g.count) break;
        }
        if (e != cudaSuccess) break;
        ctx->fast_variant[g.n] = bestv;
        if (tailmax > 0) ctx->fast_tail[g.n] = {tailv, tailmax};
        else ctx->fast_tail.erase(g.n);
        ctx->fast_fused_max[g.n] = fusedmax;
        if (chosen) chosen[gi] = g.n * 16 + bestv;
        ++gi;
    }
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_err(ctx, e, "npbs_autotune_apply");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return NPBS_OK;
}

npbs_status cbs_apply(npbs_ctx* ctx, const npbs_batch* batch, const void* V, const void* f, const void* x,
                      void* out, npbs_mode mode, double* norm2, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if ((int)mode < 0 || (int)mode > NPBS_PREC_SWEEP) return set_err(ctx, NPBS_ERR_INVALID_ARG, "cbs_apply: bad mode");
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    if (pl->count == 0) return NPBS_OK;
    const bool need_f = mode == NPBS_RESIDUAL || mode == NPBS_CBS_STEP || mode == NPBS_TRUE_RESIDUAL ||
                        mode == NPBS_PREC_SWEEP;
    if (!V || !x || !out || (need_f && !f))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cbs_apply: NULL field pointer");
    ApplyArgs a{};
    a.V = static_cast<const float2*>(V);
    a.f = static_cast<const float2*>(f);
    a.x = static_cast<const float2*>(x);
    a.out = static_cast<float2*>(out);
    a.norm2 = norm2;
    return run_apply(ctx, *pl, (int)mode, a, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

npbs_status npbs_device_status(npbs_ctx* ctx) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    NPBS_CK(ctx, cudaSetDevice(ctx->device));
    NPBS_CK(ctx, cudaDeviceSynchronize());
    if (conv_tc_timeout_flag() || newton_tc_timeout_flag()) {
        conv_tc_clear_timeout();
        newton_tc_clear_timeout();
        return set_err(ctx, NPBS_ERR_DEVICE_TIMEOUT,
                       "a bounded device wait gave up (a TMA or tensor-core stage never completed); the kernel "
                       "returned early and its results are invalid");
    }
    return NPBS_OK;
}

npbs_status npbs_test_device_timeout(npbs_ctx* ctx, double seconds, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!(seconds > 0.0 && seconds <= 2.0))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_test_device_timeout: need 0 < seconds <= 2");
    NPBS_CK(ctx, wait_selftest(seconds, reinterpret_cast<cudaStream_t>(stream)));
    ctx->count(reinterpret_cast<cudaStream_t>(stream), 1);
    return NPBS_OK;
}

npbs_status cbs_steps(npbs_ctx* ctx, const npbs_batch* batch, const void* V, const void* f, const void* x,
                      void* out, npbs_mode mode, int32_t steps, double* norm2, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (mode != NPBS_CBS_STEP && mode != NPBS_PREC_SWEEP)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "cbs_steps: mode must be CBS_STEP or PREC_SWEEP");
    if (steps < 0) return set_err(ctx, NPBS_ERR_INVALID_ARG, "cbs_steps: steps < 0");
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    if (pl->count == 0 || steps == 0) return NPBS_OK;
    if (!V || !f || !x || !out) return set_err(ctx, NPBS_ERR_INVALID_ARG, "cbs_steps: NULL field pointer");
    ApplyArgs a{};
    a.V = static_cast<const float2*>(V);
    a.f = static_cast<const float2*>(f);
    a.x = static_cast<const float2*>(x);
    a.out = static_cast<float2*>(out);
    a.norm2 = norm2;
    a.steps = steps;
    return run_apply(ctx, *pl, (int)mode, a, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
