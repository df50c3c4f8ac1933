// Solvers: stationary CBS (Eq. CBS) and the shared mixed-precision refinement
// driver used by the NPBS solve.
//
// The solution u is kept in complex128.  A refinement cycle
//   1. computes rho = f - A u in float64 (kTrueRes64 apply; this also folds the
//      previous cycle's correction delta into u) and rTol = ||rho|| / ||f||;
//   2. runs the complex64 iteration on the correction equation A delta = rho
//      from delta = 0 (source term rho in place of f),
// in chunks of `check_every` iterations, each chunk a captured CUDA graph.
// Because CBS/NPBS restarted from delta = 0 on the correction equation see the
// same Born residuals as the uninterrupted iteration, the iteration count is
// that of the method; the float64 residual removes the float32 floor.
#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "solve.cuh"

namespace npbs {

struct GraphGuard {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~GraphGuard() {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
    }
};

__global__ void k_build_V(const VecItem* items, const InstDev* inst, const float2* k2, float2* V) {
    const VecItem it = items[blockIdx.x];
    const InstDev in = inst[it.inst];
    const long long base = in.offset + it.start;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 k = k2[base + e];
        V[base + e] = make_float2((float)((double)k.x - in.k0sq), (float)((double)k.y - in.eps));
    }
}

// delta = 0 on the instances with mask[inst] set
__global__ void k_zero_masked(const VecItem* items, const InstDev* inst, const int* mask, float2* delta) {
    const VecItem it = items[blockIdx.x];
    if (!mask[it.inst]) return;
    const long long base = inst[it.inst].offset + it.start;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) delta[base + e] = make_float2(0.f, 0.f);
}

npbs_status solver_potential(npbs_ctx* ctx, const Plan& pl, const float2* k2, cudaStream_t st, const float2** V) {
    NPBS_CK(ctx, ctx->work[8].ensure(sizeof(float2) * (size_t)std::max<long long>(pl.extent, 1)));
    float2* v = static_cast<float2*>(ctx->work[8].p);
    k_build_V<<<pl.nvec, 256, 0, st>>>(pl.vitems, pl.inst, k2, v);
    NPBS_CK(ctx, cudaGetLastError());
    ctx->count(st, 1);
    *V = v;
    return NPBS_OK;
}

npbs_status refine_driver(npbs_ctx* ctx, const Plan& pl, const float2* k2, const float2* V, const float2* f, double2* u,
                          const npbs_solve_opts& o, npbs_report* rep, cudaStream_t st, const InnerStep& step,
                          RefineWork& w) {
    const int n = pl.count;
    const size_t ext = (size_t)std::max<long long>(pl.extent, 1);
    NPBS_CK(ctx, ctx->work[0].ensure(ext * sizeof(float2)));  // delta
    NPBS_CK(ctx, ctx->work[1].ensure(ext * sizeof(float2)));  // rho
    NPBS_CK(ctx, ctx->work[2].ensure(sizeof(double) * 4 * n + sizeof(int) * 2 * n + 64));
    w.delta = static_cast<float2*>(ctx->work[0].p);
    w.rho = static_cast<float2*>(ctx->work[1].p);
    double* rho2 = static_cast<double*>(ctx->work[2].p);
    double* f2 = rho2 + n;
    w.nb = f2 + n;            // inner Born residual norms^2 (written by the inner step)
    int* active = reinterpret_cast<int*>(w.nb + 2 * n);
    int* rmask = active + n;  // instances refreshed by the current float64 apply
    w.active = active;
    NPBS_CK(ctx, ctx->scratch.ensure(ext * 16));

    // Every instance runs its own refinement cycles: the inner iteration of one
    // instance never reads another's correction, so an instance whose cycle
    // ends (its estimate reached the tolerance, its residual fell by
    // max_reduction or grew, or max_cycle iterations passed) is refreshed in
    // float64 and restarted alone while the others keep iterating.
    std::vector<int> iters(n, 0), act(n, 0), need(n, 0), cycle_its(n, 0);
    std::vector<double> rt(n, 0.0), hrho2(n), hf2(n), hnb(n), nb_first(n, -1.0), rt_cycle(n, 0.0);
    std::vector<npbs_status> stat(n, NPBS_OK);

    // float64 refresh of the instances with need[j] (all of them when !fold)
    auto refresh = [&](bool fold) -> npbs_status {
        NPBS_CK(ctx, cudaMemcpyAsync(rmask, need.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        ApplyArgs a{};
        a.V = V;
        a.f = f;
        a.out = w.rho;
        a.norm2 = rho2;
        a.norm2b = f2;
        a.uhi = u;
        a.k2 = k2;
        a.delta = fold ? w.delta : nullptr;
        npbs_status s = run_apply(ctx, pl, kTrueRes64, a, rmask, st);
        if (s != NPBS_OK) return s;
        if (fold) {
            // the folded corrections restart from zero
            k_zero_masked<<<pl.nvec, 256, 0, st>>>(pl.vitems, pl.inst, rmask, w.delta);
            NPBS_CK(ctx, cudaGetLastError());
            ctx->count(st, 1);
        }
        NPBS_CK(ctx, cudaMemcpyAsync(hrho2.data(), rho2, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        NPBS_CK(ctx, cudaMemcpyAsync(hf2.data(), f2, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        NPBS_CK(ctx, cudaStreamSynchronize(st));
        for (int j = 0; j < n; ++j) {
            if (!need[j]) continue;
            const double fn = std::sqrt(hf2[j]);
            const double rn = std::sqrt(hrho2[j]);
            rt[j] = fn > 0 ? rn / fn : rn;
            if (!std::isfinite(rt[j])) {
                stat[j] = NPBS_ERR_NONFINITE;
                act[j] = 0;
            } else if (rt[j] <= o.rtol) {
                stat[j] = NPBS_OK;
                act[j] = 0;
            } else if (iters[j] >= o.max_iter) {
                stat[j] = NPBS_NOT_CONVERGED;
                act[j] = 0;
            } else {
                act[j] = 1;
            }
            nb_first[j] = -1.0;
            rt_cycle[j] = rt[j];
            cycle_its[j] = 0;
        }
        NPBS_CK(ctx, cudaMemcpyAsync(active, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        return NPBS_OK;
    };

    for (int j = 0; j < n; ++j) need[j] = 1;
    NPBS_CK(ctx, cudaMemsetAsync(w.delta, 0, ext * sizeof(float2), st));
    npbs_status s = refresh(false);
    if (s != NPBS_OK) return s;
    std::vector<int> act_prev;
    bool first_notify = true;
    // after every refresh: tell the solver which instances were refreshed;
    // returns whether the inner step's launch shapes changed
    auto notify = [&](bool* changed) -> npbs_status {
        std::vector<int> list;
        for (int j = 0; j < n; ++j)
            if (act[j]) list.push_back(j);
        const bool shape = w.on_refresh ? w.on_refresh(rt, act, need) : false;
        *changed = false;
        if (list == act_prev && !shape && !first_notify) return NPBS_OK;
        first_notify = false;
        act_prev = list;
        *changed = true;
        // the device mask was just uploaded by the refresh: compact the
        // per-size launch lists to the instances still iterating
        npbs_status s2 = set_active_lists(ctx, pl, act, active);
        if (s2 != NPBS_OK) return s2;
        return w.on_active ? w.on_active(list) : NPBS_OK;
    };

    const int chunk = std::max(1, o.check_every);
    GraphGuard graph;
    bool graph_ready = false;
    long long graph_kernels = 0;
    auto run_chunk = [&]() -> npbs_status {
        if (o.use_graph) {
            if (!graph_ready) {
                ctx->capture_kernels = 0;
                NPBS_CK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                npbs_status s2 = NPBS_OK;
                if (w.fused) s2 = w.fused(chunk);
                else
                    for (int i = 0; i < chunk && s2 == NPBS_OK; ++i) s2 = step(i == chunk - 1);
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamEndCapture(st, &g);
                if (s2 != NPBS_OK) {
                    if (g) cudaGraphDestroy(g);
                    return s2;
                }
                NPBS_CK(ctx, e);
                graph.g = g;
                graph_kernels = ctx->capture_kernels;
                NPBS_CK(ctx, cudaGraphInstantiate(&graph.e, g, 0));
                graph_ready = true;
            }
            NPBS_CK(ctx, cudaGraphLaunch(graph.e, st));
            ctx->launches += graph_kernels;
            return NPBS_OK;
        }
        if (w.fused) return w.fused(chunk);
        for (int i = 0; i < chunk; ++i) {
            npbs_status s2 = step(i == chunk - 1);
            if (s2 != NPBS_OK) return s2;
        }
        return NPBS_OK;
    };

    while (true) {
        bool any = false;
        for (int j = 0; j < n; ++j) any |= act[j] != 0;
        if (!any) break;
        bool changed = false;
        s = notify(&changed);
        if (s != NPBS_OK) return s;
        if (changed && graph_ready) {
            // the active set changed: launch shapes of the inner step may differ
            if (graph.e) cudaGraphExecDestroy(graph.e);
            if (graph.g) cudaGraphDestroy(graph.g);
            graph.e = nullptr;
            graph.g = nullptr;
            graph_ready = false;
        }
        // inner chunks until at least one instance ends its cycle
        bool go = false;
        while (!go) {
            s = run_chunk();
            if (s != NPBS_OK) return s;
            NPBS_CK(ctx, cudaMemcpyAsync(hnb.data(), w.nb, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            NPBS_CK(ctx, cudaStreamSynchronize(st));
            for (int j = 0; j < n; ++j) {
                need[j] = 0;
                if (!act[j]) continue;
                iters[j] += chunk;
                cycle_its[j] += chunk;
                if (nb_first[j] < 0) {
                    // the reported norm precedes the last update of the chunk; scale
                    // from the first chunk's value (the cycle's starting residual
                    // is about that of the first step)
                    nb_first[j] = std::max(hnb[j], 1e-300);
                }
                const double red = std::sqrt(hnb[j] / nb_first[j]);
                const double est = rt_cycle[j] * red;
                if (!std::isfinite(hnb[j]) || est <= o.rtol || red <= w.max_reduction || red > 2.0 ||
                    iters[j] >= o.max_iter || cycle_its[j] >= w.max_cycle) {
                    need[j] = 1;
                    go = true;
                }
            }
        }
        s = refresh(true);
        if (s != NPBS_OK) return s;
    }
    npbs_status ret = NPBS_OK;
    for (int j = 0; j < n; ++j) {
        if (rep) {
            if (rep->iters) rep->iters[j] = iters[j];
            if (rep->rtol) rep->rtol[j] = rt[j];
            if (rep->status) rep->status[j] = stat[j];
            if (rep->flags) rep->flags[j] = j < (int)w.flags.size() ? w.flags[j] : 0;
        }
        if (stat[j] == NPBS_ERR_NONFINITE) ret = NPBS_ERR_NONFINITE;
        else if (stat[j] != NPBS_OK && ret == NPBS_OK) ret = NPBS_NOT_CONVERGED;
    }
    return ret;
}

npbs_status solve_stream_begin(npbs_ctx* ctx, cudaStream_t user, cudaStream_t* work) {
    if (!ctx->solve_stream) {
        NPBS_CK(ctx, cudaStreamCreateWithFlags(&ctx->solve_stream, cudaStreamNonBlocking));
        NPBS_CK(ctx, cudaEventCreateWithFlags(&ctx->solve_event, cudaEventDisableTiming));
    }
    NPBS_CK(ctx, cudaEventRecord(ctx->solve_event, user));
    NPBS_CK(ctx, cudaStreamWaitEvent(ctx->solve_stream, ctx->solve_event, 0));
    *work = ctx->solve_stream;
    return NPBS_OK;
}

npbs_status check_solve_args(npbs_ctx* ctx, const npbs_solve_opts* o, const void* k2, const void* f, const void* u) {
    if (!o || !(o->rtol >= 0.0) || o->max_iter < 0 || o->check_every < 1)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "solve options: need rtol >= 0, max_iter >= 0, check_every >= 1");
    if (!k2 || !f || !u) return set_err(ctx, NPBS_ERR_INVALID_ARG, "solve: NULL field pointer");
    return NPBS_OK;
}

}  // namespace npbs

using namespace npbs;

extern "C" npbs_status cbs_solve(npbs_ctx* ctx, const npbs_batch* batch, const void* k2, const void* f, void* u,
                                 const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    if (pl->count == 0) return NPBS_OK;
    st = check_solve_args(ctx, opts, k2, f, u);
    if (st != NPBS_OK) return st;
    cudaStream_t s = nullptr;
    st = solve_stream_begin(ctx, reinterpret_cast<cudaStream_t>(stream), &s);
    if (st != NPBS_OK) return st;
    RefineWork w;
    const float2* K2 = static_cast<const float2*>(k2);
    const float2* Vp = nullptr;
    st = solver_potential(ctx, *pl, K2, s, &Vp);
    if (st != NPBS_OK) return st;
    // inner step: delta <- delta + gamma (G(V delta + rho) - delta), in place
    InnerStep step = [&](bool last) -> npbs_status {
        ApplyArgs a{};
        a.V = Vp;
        a.f = w.rho;
        a.x = w.delta;
        a.out = w.delta;
        a.norm2 = last ? w.nb : nullptr;
        return run_apply(ctx, *pl, NPBS_CBS_STEP, a, w.active, s);
    };
    // a chunk of inner iterations as one fused launch per grid side
    w.fused = [&](int steps) -> npbs_status {
        ApplyArgs a{};
        a.V = Vp;
        a.f = w.rho;
        a.x = w.delta;
        a.out = w.delta;
        a.norm2 = w.nb;
        a.steps = steps;
        return run_apply(ctx, *pl, NPBS_CBS_STEP, a, w.active, s);
    };
    return refine_driver(ctx, *pl, K2, Vp, static_cast<const float2*>(f), static_cast<double2*>(u), *opts, report,
                         s, step, w);
}

#include "net.cuh"

namespace npbs {
// delta += gamma r (gamma = i V / eps) for active instances in CBS fallback mode
__global__ void k_cbs_fallback(const VecItem* items, const InstDev* inst, const int* active, const int* cbs_mode,
                               const float2* V, const float2* r, float2* delta) {
    const VecItem it = items[blockIdx.x];
    if ((active && !active[it.inst]) || !cbs_mode[it.inst]) return;
    const InstDev in = inst[it.inst];
    const float ie = (float)(1.0 / in.eps);
    const long long base = in.offset + it.start;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 v = V[base + e], q = r[base + e];
        const float gr = -v.y * ie, gi = v.x * ie;
        float2 d = delta[base + e];
        d.x += gr * q.x - gi * q.y;
        d.y += gr * q.y + gi * q.x;
        delta[base + e] = d;
    }
}
}  // namespace npbs

// Stationary NPBS (Eq. npbs_integral) with the network as M_theta:
//   delta <- delta + M(G(V delta + rho) - delta)
// on the correction equation; r = G(V delta + rho) - delta equals the Born
// residual of u + delta for the original problem.
// Learned stationary iteration in either format: Born (Eq. npbs_integral,
// with the CBS guard) or direct (Eq. direct_iter: r = rho - A delta from the
// TRUE_RESIDUAL apply, no guard).
static npbs_status learned_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const void* k2,
                                 const void* f, const float* n, void* u, const npbs_solve_opts* opts,
                                 npbs_report* report, npbs_stream stream, bool direct) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!net || !n) return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_solve: NULL network or refractive index");
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    if (pl->count == 0) return NPBS_OK;
    st = check_solve_args(ctx, opts, k2, f, u);
    if (st != NPBS_OK) return st;
    cudaStream_t s = nullptr;
    st = solve_stream_begin(ctx, reinterpret_cast<cudaStream_t>(stream), &s);
    if (st != NPBS_OK) return st;
    const float2* K2 = static_cast<const float2*>(k2);
    const float2* Vp = nullptr;
    st = solver_potential(ctx, *pl, K2, s, &Vp);
    if (st != NPBS_OK) return st;
    const size_t ext = (size_t)std::max<long long>(pl->extent, 1);
    NPBS_CK(ctx, ctx->work[6].ensure(ext * sizeof(float2)));
    float2* r = static_cast<float2*>(ctx->work[6].p);
    const Net& N = *reinterpret_cast<const Net*>(net);
    NPBS_CK(ctx, ctx->work[2].ensure(sizeof(double) * 4 * pl->count + sizeof(int) * pl->count + 64));
    NPBS_CK(ctx, ctx->work[7].ensure(sizeof(int) * pl->count + 64));
    int* cbs_mode = static_cast<int*>(ctx->work[7].p);
    RefineWork w;
    NetRun run;
    const int cnt = pl->count;
    std::vector<int> mode(cnt, 0);          // 0: network correction, 1: CBS fallback
    std::vector<double> last_rt(cnt, -1.0);
    w.flags.assign(cnt, 0);
    // divergence guard: an instance whose float64 rTol grew since the previous
    // refresh continues with plain CBS steps (and is flagged in the report)
    w.on_refresh = [&](const std::vector<double>& rt, const std::vector<int>& act,
                       const std::vector<int>& refreshed) -> bool {
        if (direct) return false;
        bool changed = false;
        for (int j = 0; j < cnt; ++j) {
            if (!refreshed[j]) continue;
            if (act[j] && mode[j] == 0 && last_rt[j] >= 0.0 && !(rt[j] < last_rt[j])) {
                mode[j] = 1;
                w.flags[j] = 1;
                changed = true;
            }
            last_rt[j] = rt[j];
        }
        return changed;
    };
    w.on_active = [&](const std::vector<int>& list) -> npbs_status {
        std::vector<int> netl;
        for (int j : list)
            if (mode[j] == 0) netl.push_back(j);
        NPBS_CK(ctx, cudaMemcpyAsync(cbs_mode, mode.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        return net_prepare(ctx, N, *pl, netl, false, &run, s, n);
    };
    InnerStep step = [&](bool last) -> npbs_status {
        ApplyArgs a{};
        a.V = Vp;
        a.f = w.rho;
        a.x = w.delta;
        a.out = r;
        a.norm2 = last ? w.nb : nullptr;
        npbs_status s2 = run_apply(ctx, *pl, direct ? NPBS_TRUE_RESIDUAL : NPBS_RESIDUAL, a, w.active, s);
        if (s2 != NPBS_OK) return s2;
        s2 = net_run_forward(ctx, N, run, r, n, w.delta, 1, s);
        if (s2 != NPBS_OK) return s2;
        if (direct) return NPBS_OK;
        k_cbs_fallback<<<pl->nvec, 256, 0, s>>>(pl->vitems, pl->inst, w.active, cbs_mode, Vp, r, w.delta);
        NPBS_CK(ctx, cudaGetLastError());
        ctx->count(s, 1);
        return NPBS_OK;
    };
    return refine_driver(ctx, *pl, K2, Vp, static_cast<const float2*>(f), static_cast<double2*>(u), *opts, report,
                         s, step, w);
}

extern "C" npbs_status npbs_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const void* k2,
                                  const void* f, const float* n, void* u, const npbs_solve_opts* opts,
                                  npbs_report* report, npbs_stream stream) {
    return learned_solve(ctx, net, batch, k2, f, n, u, opts, report, stream, false);
}

extern "C" npbs_status npbs_solve_direct(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const void* k2,
                                         const void* f, const float* n, void* u, const npbs_solve_opts* opts,
                                         npbs_report* report, npbs_stream stream) {
    return learned_solve(ctx, net, batch, k2, f, n, u, opts, report, stream, true);
}
