// Metric-matched training step (Eq. L_bs_Reta_integral) over unrolled NPBS
// steps with activation checkpointing:
//   r_0 = G(V u + f) - u,  c_k = M(r_k),  r_{k+1} = r_k - (I - G V) c_k,
//   loss = mean over instances of (1/U) sum_{k=1..U} ||r_k||^2 / ||r_0||^2.
// Only r_0..r_U are kept; the network activations are recomputed during the
// backward sweep, which runs the hand-written adjoints in reverse:
//   g_{r_U} = 2 w r_U,  g_{c_k} = -(I - G V)^* g_{r_{k+1}}  (ADJ_B apply),
//   g_{r_k} = g_{r_{k+1}} + J_M(r_k)^* g_{c_k} + 2 w r_k (k >= 1),
// with w = 1 / (U * count * ||r_0||^2), then one AdamW update.
#include <algorithm>
#include <cmath>
#include <vector>

#include "net.cuh"

namespace npbs {

__global__ void k_sub_norm(const VecItem* items, const InstDev* inst, const float2* a, const float2* b, float2* out,
                           double* norm2) {
    const VecItem it = items[blockIdx.x];
    const long long base = inst[it.inst].offset + it.start;
    double acc = 0.0;
    for (int e = threadIdx.x; e < it.len; e += blockDim.x) {
        const float2 x = a[base + e], y = b[base + e];
        const float2 o = make_float2(x.x - y.x, x.y - y.y);
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

}  // namespace npbs

using namespace npbs;

extern "C" npbs_status npbs_train_step(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* V,
                                       const void* f, const float* n, const void* u_snap, int32_t unroll, float lr,
                                       float weight_decay, float* loss_host, npbs_stream stream) {
    if (!ctx) return NPBS_ERR_INVALID_ARG;
    if (!net || !V || !f || !n || !u_snap || !loss_host)
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_train_step: NULL argument");
    if (unroll < 1 || unroll > 16 || !(lr >= 0.f) || !(weight_decay >= 0.f))
        return set_err(ctx, NPBS_ERR_INVALID_ARG, "npbs_train_step: need 1 <= unroll <= 16, lr >= 0, weight_decay >= 0");
    npbs_status st;
    const Plan* pl = get_plan(ctx, batch, &st);
    if (!pl) return st;
    const int cnt = pl->count;
    *loss_host = 0.f;
    if (cnt == 0) return NPBS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Net& N = *reinterpret_cast<Net*>(net);
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
    st = net_prepare(ctx, *pl, which, true, &run, s);
    if (st != NPBS_OK) return st;
    NPBS_CK(ctx, cudaMemsetAsync(N.grads, 0, sizeof(float) * dev_param_count(), s));
    NPBS_CK(ctx, cudaMemsetAsync(nk2, 0, sizeof(double) * cnt * U, s));

    // forward: r_0 and the unrolled residuals
    {
        ApplyArgs a{};
        a.V = static_cast<const float2*>(V);
        a.f = static_cast<const float2*>(f);
        a.x = static_cast<const float2*>(u_snap);
        a.out = Rk(0);
        a.norm2 = r0n2;
        st = run_apply(ctx, *pl, NPBS_RESIDUAL, a, nullptr, s);
        if (st != NPBS_OK) return st;
    }
    for (int k = 0; k < U; ++k) {
        st = net_run_forward(ctx, N, run, Rk(k), n, c, 0, s);
        if (st != NPBS_OK) return st;
        ApplyArgs a{};
        a.V = static_cast<const float2*>(V);
        a.x = c;
        a.out = wv;
        st = run_apply(ctx, *pl, NPBS_OP_B, a, nullptr, s);
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
        {
            ApplyArgs a{};
            a.V = static_cast<const float2*>(V);
            a.x = gr;
            a.out = c;  // B^* g_r
            st = run_apply(ctx, *pl, NPBS_ADJ_B, a, nullptr, s);
            if (st != NPBS_OK) return st;
        }
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
