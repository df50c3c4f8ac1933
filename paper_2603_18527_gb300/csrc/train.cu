// Training step over unrolled learned iterations with activation
// checkpointing, for the three objectives of Sec. 4.
//
// Metric-matched (Eq. L_bs_Reta_integral), in Born-residual coordinates:
//   r_0 = G(V u + f) - u,  c_k = M(r_k),  r_{k+1} = r_k - (I - G V) c_k,
//   loss = mean over instances of (1/U) sum_{k=1..U} ||r_k||^2 / ||r_0||^2,
// backward with the hand-written adjoints in reverse:
//   g_{r_U} = 2 w r_U,  g_{c_k} = -(I - G V)^* g_{r_{k+1}}  (ADJ_B apply),
//   g_{r_k} = g_{r_{k+1}} + J_M(r_k)^* g_{c_k} + 2 w r_k (k >= 1),
// with w = 1 / (U * count * ||r_0||^2).
//
// Euclidean objectives (Eq. L_bs_l2 and Eq. L_dir), in true-residual
// coordinates t = f - A u:
//   x_k = P t_k (P = G for L_bs_l2, I for L_dir), c_k = M(x_k),
//   t_{k+1} = t_k - A c_k,  loss = mean of (1/U) sum ||t_k||^2 / ||t_0||^2,
//   g_{t_U} = 2 w t_U,  g_{c_k} = -A^* g_{t_{k+1}},
//   g_{t_k} = g_{t_{k+1}} + P^* J_M(x_k)^* g_{c_k} + 2 w t_k (k >= 1).
// A x is minus the TRUE_RESIDUAL apply with f = 0, G x the RESIDUAL apply
// with x = 0 and f = x; A and G are complex symmetric (their symbols are even
// in xi and their potentials diagonal), so A^* y = conj(A conj(y)) and
// likewise for G.  Only the states (and for L_bs_l2 the network inputs) are
// kept; the network activations are recomputed in the backward sweep.  One
// AdamW update ends the step.
#include <algorithm>
#include <cmath>
#include <vector>

#include "net.cuh"

namespace npbs {

// out = a + sb * b and norm2[inst] += ||out||^2
__global__ void k_sub_norm(const VecItem* items, const InstDev* inst, const float2* a, const float2* b, float2* out,
                           double* norm2, float sb = -1.f) {
    const VecItem it = items[blockIdx.x];
    const long long base = inst[it.inst].offset + it.start;
    double acc = 0.0;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 x = a[base + e], y = b[base + e];
        const float2 o = make_float2(x.x + sb * y.x, x.y + sb * y.y);
        out[base + e] = o;
        acc += (double)o.x * o.x + (double)o.y * o.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(norm2 + it.inst, t);
    }
}

// out = coef * w[inst] * x (+ base if non-null; + extra if non-null)
__global__ void k_axpby_inst(const VecItem* items, const InstDev* inst, const float2* x, const double* w, float coef,
                             const float2* base_in, const float2* extra, float2* out) {
    const VecItem it = items[blockIdx.x];
    const long long base = inst[it.inst].offset + it.start;
    const float k = w ? (float)(coef * w[it.inst]) : coef;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 v = x[base + e];
        float2 o = make_float2(k * v.x, k * v.y);
        if (base_in) {
            const float2 b = base_in[base + e];
            o.x += b.x;
            o.y += b.y;
        }
        if (extra) {
            const float2 b = extra[base + e];
            o.x += b.x;
            o.y += b.y;
        }
        out[base + e] = o;
    }
}

// out = conj(x)
__global__ void k_conj(const VecItem* items, const InstDev* inst, const float2* x, float2* out) {
    const VecItem it = items[blockIdx.x];
    const long long base = inst[it.inst].offset + it.start;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 v = x[base + e];
        out[base + e] = make_float2(v.x, -v.y);
    }
}

npbs_status train_step_reta(npbs_ctx* ctx, Net& N, const Plan* pl, const float* n, int unroll, float lr,
                            float weight_decay, float* loss_host, cudaStream_t s, const BornOp& op) {
    npbs_status st;
    const int cnt = pl->count;
    const int U = unroll;
    const size_t ext = (size_t)std::max<long long>(pl->extent, 1);
    NPBS_CK(ctx, ctx->work[6].ensure(ext * sizeof(float2) * (size_t)(U + 1 + 4)));
    NPBS_CK(ctx, ctx->work[7].ensure(sizeof(double) * (size_t)cnt * (U + 3) + 256));
    float2* R = static_cast<float2*>(ctx->work[6].p);
    float2* c = R + ext * (U + 1);
    float2* wv = c + ext;
    float2* gr = wv + ext;
    float2* gn = gr + ext;
    double* r0n2 = static_cast<double*>(ctx->work[7].p);
    double* nk2 = r0n2 + cnt;
    double* wgt = nk2 + (size_t)cnt * U;
    const VecItem* vi = pl->vitems;
    const int vb = pl->nvec;
    auto Rk = [&](int k) { return R + ext * k; };

    std::vector<int> which(cnt);
    for (int j = 0; j < cnt; ++j) which[j] = j;
    NetRun run;
    st = net_prepare(ctx, N, *pl, which, true, &run, s);
    if (st != NPBS_OK) return st;
    NPBS_CK(ctx, cudaMemsetAsync(N.grads, 0, sizeof(float) * N.count(), s));
    NPBS_CK(ctx, cudaMemsetAsync(nk2, 0, sizeof(double) * cnt * U, s));

    // forward: r_0 and the unrolled residuals
    st = op(NPBS_RESIDUAL, nullptr, Rk(0), r0n2);
    if (st != NPBS_OK) return st;
    for (int k = 0; k < U; ++k) {
        st = net_run_forward(ctx, N, run, Rk(k), n, c, 0, s);
        if (st != NPBS_OK) return st;
        st = op(NPBS_OP_B, c, wv, nullptr);
        if (st != NPBS_OK) return st;
        k_sub_norm<<<vb, 256, 0, s>>>(vi, pl->inst, Rk(k), wv, Rk(k + 1), nk2 + (size_t)k * cnt);
        ctx->count(s, 1);
    }
    std::vector<double> h0(cnt), hk((size_t)cnt * U), hw(cnt);
    NPBS_CK(ctx, cudaMemcpyAsync(h0.data(), r0n2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaMemcpyAsync(hk.data(), nk2, sizeof(double) * cnt * U, cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaStreamSynchronize(s));
    double loss = 0.0;
    for (int j = 0; j < cnt; ++j) {
        hw[j] = h0[j] > 0 ? 1.0 / ((double)U * cnt * h0[j]) : 0.0;
        for (int k = 0; k < U; ++k) loss += hk[(size_t)k * cnt + j] * hw[j];
    }
    if (!std::isfinite(loss)) return set_err(ctx, NPBS_ERR_NONFINITE, "npbs_train_step: non-finite loss");
    *loss_host = (float)loss;
    NPBS_CK(ctx, cudaMemcpyAsync(wgt, hw.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, s));

    // backward sweep
    k_axpby_inst<<<vb, 256, 0, s>>>(vi, pl->inst, Rk(U), wgt, 2.f, nullptr, nullptr, gr);
    ctx->count(s, 1);
    for (int k = U - 1; k >= 0; --k) {
        st = op(NPBS_ADJ_B, gr, c, nullptr);  // B^* g_r
        if (st != NPBS_OK) return st;
        k_axpby_inst<<<vb, 256, 0, s>>>(vi, pl->inst, c, nullptr, -1.f, nullptr, nullptr, c);  // g_c = -B^* g_r
        ctx->count(s, 1);
        st = net_run_backward(ctx, N, run, Rk(k), n, c, gn, 0, s);
        if (st != NPBS_OK) return st;
        if (k > 0) {
            // g_r <- g_r + J^* g_c + 2 w r_k
            k_axpby_inst<<<vb, 256, 0, s>>>(vi, pl->inst, Rk(k), wgt, 2.f, gr, gn, gr);
            ctx->count(s, 1);
        }
    }
    NPBS_CK(ctx, cudaGetLastError());
    return net_adamw(ctx, N, lr, weight_decay, s);
}

}  // namespace npbs

using namespace npbs;

extern "C" npbs_status npbs_train_step_loss(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* V,
                                            const void* f, const float* n, const void* u_snap, int32_t unroll,
                                            npbs_loss kind, float lr, float weight_decay, float* loss_host,
                                            npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!net || !V || !f || !n || !u_snap || !loss_host)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_train_step: NULL argument");
    if (unroll < 1 || unroll > 16 || !(lr >= 0.f) || !(weight_decay >= 0.f))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_train_step: need 1 <= unroll <= 16, lr >= 0, weight_decay >= 0");
    if (kind != NPBS_LOSS_BS_RETA && kind != NPBS_LOSS_BS_L2 && kind != NPBS_LOSS_DIR)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_train_step: unknown loss");
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    const int cnt = pl->count;
    *loss_host = 0.f;
    if (cnt == 0) return NPBS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Net& N = *reinterpret_cast<Net*>(net);
    const float2* Vp = static_cast<const float2*>(V);
    const float2* fp = static_cast<const float2*>(f);
    const float2* usnap = static_cast<const float2*>(u_snap);
    if (kind != NPBS_LOSS_BS_RETA) {
        // A and G are complex symmetric (even symbols, diagonal potential), so
        // A^* y = conj(A conj(y)) and likewise for G; scratch: zero, t1, t2
        const size_t ext = (size_t)std::max<long long>(pl->extent, 1);
        NPBS_CK(ctx, ctx->work[9].ensure(3 * ext * sizeof(float2)));
        float2* zero = static_cast<float2*>(ctx->work[9].p);
        float2* t1 = zero + ext;
        float2* t2 = t1 + ext;
        NPBS_CK(ctx, cudaMemsetAsync(zero, 0, ext * sizeof(float2), s));
        const VecItem* vi = pl->vitems;
        const int vb = pl->nvec;
        auto conj = [&](const float2* x, float2* out) {
            k_conj<<<vb, 256, 0, s>>>(vi, pl->inst, x, out);
            ctx->count(s, 1);
        };
        EuclidOps op;
        op.minus_a = [&](const float2* x, const float2* f_in, float2* out, double* norm2) -> npbs_status {
            ApplyArgs a{};
            a.V = Vp;
            a.f = f_in;
            a.x = x;
            a.out = out;
            a.norm2 = norm2;
            return run_apply(ctx, *pl, NPBS_TRUE_RESIDUAL, a, nullptr, s);
        };
        op.green = [&](const float2* x, float2* out) -> npbs_status {
            ApplyArgs a{};  // RESIDUAL with x = 0 and f = x: G x
            a.V = Vp;
            a.f = x;
            a.x = zero;
            a.out = out;
            return run_apply(ctx, *pl, NPBS_RESIDUAL, a, nullptr, s);
        };
        op.minus_a_adj = [&](const float2* y, float2* out) -> npbs_status {
            conj(y, t1);
            npbs_status r = op.minus_a(t1, zero, t2, nullptr);
            if (r != NPBS_OK) return r;
            conj(t2, out);
            return NPBS_OK;
        };
        op.green_adj = [&](const float2* y, float2* out) -> npbs_status {
            conj(y, t1);
            npbs_status r = op.green(t1, t2);
            if (r != NPBS_OK) return r;
            conj(t2, out);
            return NPBS_OK;
        };
        return train_step_euclid(ctx, N, pl, n, fp, usnap, unroll, kind == NPBS_LOSS_BS_L2, lr, weight_decay,
                                 loss_host, s, op);
    }
    BornOp op = [&](int mode, const float2* x, float2* out, double* norm2) -> npbs_status {
        ApplyArgs a{};
        a.V = Vp;
        a.f = mode == NPBS_RESIDUAL ? fp : nullptr;
        a.x = mode == NPBS_RESIDUAL ? usnap : x;
        a.out = out;
        a.norm2 = norm2;
        return run_apply(ctx, *pl, mode, a, nullptr, s);
    };
    return train_step_reta(ctx, N, pl, n, unroll, lr, weight_decay, loss_host, s, op);
}

extern "C" npbs_status npbs_train_step(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* V,
                                       const void* f, const float* n, const void* u_snap, int32_t unroll, float lr,
                                       float weight_decay, float* loss_host, npbs_stream stream) {
    return npbs_train_step_loss(ctx, net, batch, V, f, n, u_snap, unroll, NPBS_LOSS_BS_RETA, lr, weight_decay,
                                loss_host, stream);
}

namespace npbs {

// Eq. L_bs_l2 (green_input) and Eq. L_dir in true-residual coordinates.
npbs_status train_step_euclid(npbs_ctx* ctx, Net& N, const Plan* pl, const float* n, const float2* f,
                              const float2* u_snap, int U, bool green_input, float lr, float weight_decay,
                              float* loss_host, cudaStream_t s, const EuclidOps& op) {
    const int cnt = pl->count;
    const size_t ext = (size_t)std::max<long long>(pl->extent, 1);
    // states t_0..t_U, network inputs x_0..x_{U-1} (green_input only), c, wv, gr, gn, zero
    const size_t nbuf = (size_t)(U + 1) + (green_input ? (size_t)U : 0) + 5;
    NPBS_CK(ctx, ctx->work[6].ensure(ext * sizeof(float2) * nbuf));
    NPBS_CK(ctx, ctx->work[7].ensure(sizeof(double) * (size_t)cnt * (U + 3) + 256));
    float2* T = static_cast<float2*>(ctx->work[6].p);
    float2* X = T + ext * (U + 1);
    float2* c = X + (green_input ? ext * U : 0);
    float2* wv = c + ext;
    float2* gr = wv + ext;
    float2* gn = gr + ext;
    float2* zero = gn + ext;
    double* t0n2 = static_cast<double*>(ctx->work[7].p);
    double* nk2 = t0n2 + cnt;
    double* wgt = nk2 + (size_t)cnt * U;
    const VecItem* vi = pl->vitems;
    const int vb = pl->nvec;
    auto Tk = [&](int k) { return T + ext * k; };
    auto Xk = [&](int k) { return green_input ? X + ext * k : Tk(k); };
    npbs_status st;
    std::vector<int> which(cnt);
    for (int j = 0; j < cnt; ++j) which[j] = j;
    NetRun run;
    st = net_prepare(ctx, N, *pl, which, true, &run, s, n);
    if (st != NPBS_OK) return st;
    NPBS_CK(ctx, cudaMemsetAsync(N.grads, 0, sizeof(float) * N.count(), s));
    NPBS_CK(ctx, cudaMemsetAsync(nk2, 0, sizeof(double) * cnt * U, s));
    NPBS_CK(ctx, cudaMemsetAsync(zero, 0, sizeof(float2) * ext, s));

    // forward
    st = op.minus_a(u_snap, f, Tk(0), t0n2);  // t_0 = f - A u
    if (st != NPBS_OK) return st;
    for (int k = 0; k < U; ++k) {
        if (green_input) {
            st = op.green(Tk(k), Xk(k));
            if (st != NPBS_OK) return st;
        }
        st = net_run_forward(ctx, N, run, Xk(k), n, c, 0, s);
        if (st != NPBS_OK) return st;
        st = op.minus_a(c, zero, wv, nullptr);  // -A c
        if (st != NPBS_OK) return st;
        k_sub_norm<<<vb, 256, 0, s>>>(vi, pl->inst, Tk(k), wv, Tk(k + 1), nk2 + (size_t)k * cnt, 1.f);
        ctx->count(s, 1);
    }
    std::vector<double> h0(cnt), hk((size_t)cnt * U), hw(cnt);
    NPBS_CK(ctx, cudaMemcpyAsync(h0.data(), t0n2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaMemcpyAsync(hk.data(), nk2, sizeof(double) * cnt * U, cudaMemcpyDeviceToHost, s));
    NPBS_CK(ctx, cudaStreamSynchronize(s));
    double loss = 0.0;
    for (int j = 0; j < cnt; ++j) {
        hw[j] = h0[j] > 0 ? 1.0 / ((double)U * cnt * h0[j]) : 0.0;
        for (int k = 0; k < U; ++k) loss += hk[(size_t)k * cnt + j] * hw[j];
    }
    if (!std::isfinite(loss)) return set_err(ctx, NPBS_ERR_NONFINITE, "npbs_train_step: non-finite loss");
    *loss_host = (float)loss;
    NPBS_CK(ctx, cudaMemcpyAsync(wgt, hw.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, s));

    // backward sweep
    k_axpby_inst<<<vb, 256, 0, s>>>(vi, pl->inst, Tk(U), wgt, 2.f, nullptr, nullptr, gr);
    ctx->count(s, 1);
    for (int k = U - 1; k >= 0; --k) {
        st = op.minus_a_adj(gr, c);  // g_c = -A^* g_t
        if (st != NPBS_OK) return st;
        st = net_run_backward(ctx, N, run, Xk(k), n, c, gn, 0, s);
        if (st != NPBS_OK) return st;
        if (green_input) {
            st = op.green_adj(gn, gn);  // P^* = G^*
            if (st != NPBS_OK) return st;
        }
        if (k > 0) {
            // g_t <- g_t + P^* J^* g_c + 2 w t_k
            k_axpby_inst<<<vb, 256, 0, s>>>(vi, pl->inst, Tk(k), wgt, 2.f, gr, gn, gr);
            ctx->count(s, 1);
        }
    }
    NPBS_CK(ctx, cudaGetLastError());
    return net_adamw(ctx, N, lr, weight_decay, s);
}

}  // namespace npbs
