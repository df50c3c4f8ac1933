// cbs_apply_static: the fused Born apply for callers that must not allocate
// device memory.
//
// cbs_apply keeps its spectrum scratch and its device copy of the batch plan
// in buffers the context allocates on first use (cudaMalloc).  Some callers
// cannot allow that: applications whose memory manager has reserved the whole
// device for its own pool (a cudaMalloc behind its back fails or fragments
// the pool), and latency-sensitive code that must not pay for cudaMalloc /
// cudaFree, which can synchronise the whole device.  This entry point runs the
// same kernels with the scratch and the plan in file-scope static device
// arrays of fixed size that the library reserves when it is loaded; every GPU
// that loads the library holds them (about 8.3 MiB) until the process exits.
//
// Limits: at most kStaticMaxPoints elements of batch extent (max offset + nx*ny),
// kStaticMaxInstances instances, kStaticMaxSizes distinct transform lengths
// and kStaticMaxItems row / column work items; larger batches are rejected with
// NPBS_ERR_UNSUPPORTED_SIZE and a message.  All calls share the static arrays
// and keep the last call's contents, so calls that overlap on the GPU (two
// streams, two host threads) race; calls on one stream are ordered and safe.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "apply.cuh"

namespace npbs {
namespace {

constexpr long long kStaticMaxPoints = 1LL << 20;  // complex64 spectrum elements (8 MiB)
constexpr int kStaticMaxInstances = 64;
constexpr int kStaticMaxSizes = 8;
constexpr int kStaticMaxItems = 8192;

struct StaticPlan {
    InstDev inst[kStaticMaxInstances];
    RadixPlan plans[kStaticMaxSizes];
    float2 tw32[kStaticMaxSizes * kMaxN];
    RowItem rows[kStaticMaxItems];
    ColItem cols[kStaticMaxItems];
};

// The static device memory.  In host code these names are host-side shadows,
// not device addresses: the device addresses come from cudaGetSymbolAddress.
static __device__ __align__(256) float2 g_static_scratch[kStaticMaxPoints];
static __device__ __align__(256) StaticPlan g_static_plan;

constexpr int kMaxDevices = 64;
struct DeviceState {
    bool ready = false;
    float2* scratch = nullptr;
    StaticPlan* plan = nullptr;
};
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

// Once per device, with that device current: resolve the device addresses of
// the static arrays and opt the apply kernels into their shared memory.
// Called with g_mutex held.
npbs_status setup_current_device(int dev, char* err, int errlen) {
    DeviceState& s = g_state[dev];
    if (s.ready) return NPBS_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
        if (err && errlen > 0) snprintf(err, errlen, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    s.scratch = static_cast<float2*>(p);
    e = cudaGetSymbolAddress(&p, g_static_plan);
    if (e != cudaSuccess) {
        if (err && errlen > 0) snprintf(err, errlen, "cudaGetSymbolAddress(plan): %s", cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    s.plan = static_cast<StaticPlan*>(p);
    e = prepare_apply();
    if (e != cudaSuccess) {
        if (err && errlen > 0) snprintf(err, errlen, "kernel set-up: %s", cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    s.ready = true;
    return NPBS_OK;
}

npbs_status fail(char* err, int errlen, npbs_status st, const char* msg) {
    if (err && errlen > 0) snprintf(err, errlen, "%s", msg);
    return st;
}

bool radix_plan_of(int n, RadixPlan* p) {
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

// Host-side staging of the plan (static storage, guarded by g_mutex; the
// pageable copies below are staged by the driver before they return, so the
// buffer may be reused by the next call at once).
StaticPlan g_host_plan;

}  // namespace
}  // namespace npbs

using namespace npbs;

extern "C" npbs_status cbs_apply_static(const npbs_batch* batch, const void* V, const void* f, const void* x,
                                        void* out, npbs_mode mode, double* norm2, npbs_stream stream, char* err,
                                        int32_t errlen) {
    if (err && errlen > 0) err[0] = '\0';
    if ((int)mode < 0 || (int)mode > NPBS_PREC_SWEEP) return fail(err, errlen, NPBS_ERR_INVALID_ARG, "bad mode");
    if (!batch || batch->count < 0 || (batch->count > 0 && !batch->inst))
        return fail(err, errlen, NPBS_ERR_INVALID_ARG, "batch is NULL or malformed");
    const int count = batch->count;
    if (count == 0) return NPBS_OK;
    const bool need_f = mode == NPBS_RESIDUAL || mode == NPBS_CBS_STEP || mode == NPBS_TRUE_RESIDUAL ||
                        mode == NPBS_PREC_SWEEP;
    if (!V || !x || !out || (need_f && !f)) return fail(err, errlen, NPBS_ERR_INVALID_ARG, "NULL field pointer");
    if (count > kStaticMaxInstances) {
        char m[160];
        snprintf(m, sizeof m, "cbs_apply_static: %d instances exceed the static limit of %d", count,
                 kStaticMaxInstances);
        return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, m);
    }

    // Plan on the host, in the staging copy (one call at a time on the host).
    std::lock_guard<std::mutex> lock(g_mutex);
    StaticPlan& hp = g_host_plan;
    int nsizes = 0, sizes[kStaticMaxSizes];
    int nrows = 0, ncols = 0;
    long long extent = 0;
    constexpr int tile = kTileElems<float>();
    for (int j = 0; j < count; ++j) {
        const npbs_instance& s = batch->inst[j];
        if (!(s.h > 0.0) || !std::isfinite(s.h) || !std::isfinite(s.k0sq) || !(s.eps > 0.0) || !std::isfinite(s.eps) ||
            s.offset < 0 || (s.offset % 32) != 0)
            return fail(err, errlen, NPBS_ERR_INVALID_ARG,
                        "need h > 0, eps > 0, finite k0sq and offsets >= 0 that are multiples of 32");
        int idx[2];
        const int dims[2] = {s.nx, s.ny};
        for (int d = 0; d < 2; ++d) {
            int k = 0;
            while (k < nsizes && sizes[k] != dims[d]) ++k;
            if (k == nsizes) {
                if (nsizes == kStaticMaxSizes)
                    return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE,
                                "cbs_apply_static: more distinct grid sizes than the static limit of 8");
                if (!radix_plan_of(dims[d], &hp.plans[k]))
                    return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, "grid side is not 2^a 3^b in [2, 1024]");
                for (int q = 0; q < dims[d]; ++q) {
                    const double a = -2.0 * M_PI * (double)q / (double)dims[d];
                    hp.tw32[k * kMaxN + q] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
                sizes[nsizes++] = dims[d];
            }
            idx[d] = k;
        }
        InstDev& d = hp.inst[j];
        d.nx = s.nx;
        d.ny = s.ny;
        d.plan_x = idx[0];
        d.plan_y = idx[1];
        d.tw_x = idx[0] * kMaxN;
        d.tw_y = idx[1] * kMaxN;
        d.h = s.h;
        d.k0sq = s.k0sq;
        d.eps = s.eps;
        d.offset = s.offset;
        extent = std::max<long long>(extent, s.offset + (long long)s.nx * s.ny);
        if (extent > kStaticMaxPoints) {
            char m[200];
            snprintf(m, sizeof m,
                     "cbs_apply_static: batch extent %lld elements exceeds the static scratch of %lld elements",
                     extent, kStaticMaxPoints);
            return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, m);
        }
        const int rp = std::max(1, std::min(s.ny, tile / s.nx));
        for (int r0 = 0; r0 < s.ny; r0 += rp) {
            if (nrows == kStaticMaxItems)
                return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, "cbs_apply_static: too many row work items");
            hp.rows[nrows++] = RowItem{j, r0, std::min(rp, s.ny - r0), 0};
        }
        const int cp = std::max(1, std::min(16, tile / s.ny));
        for (int c0 = 0; c0 < s.nx; c0 += cp) {
            if (ncols == kStaticMaxItems)
                return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, "cbs_apply_static: too many column work items");
            hp.cols[ncols++] = ColItem{j, c0, std::min(cp, s.nx - c0), 0};
        }
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(err, errlen, NPBS_ERR_CUDA, "no current CUDA device");
    npbs_status st = setup_current_device(dev, err, errlen);
    if (st != NPBS_OK) return st;
    StaticPlan* dp = g_state[dev].plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // Upload the used parts of the plan (pageable source: staged before return).
    cudaError_t e = cudaMemcpyAsync(dp->inst, hp.inst, sizeof(InstDev) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp->plans, hp.plans, sizeof(RadixPlan) * nsizes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp->tw32, hp.tw32, sizeof(float2) * kMaxN * nsizes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp->rows, hp.rows, sizeof(RowItem) * nrows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp->cols, hp.cols, sizeof(ColItem) * ncols, cudaMemcpyHostToDevice, s);
    // the reductions accumulate: norm2 must start at zero
    if (e == cudaSuccess && norm2) e = cudaMemsetAsync(norm2, 0, sizeof(double) * count, s);
    if (e != cudaSuccess) {
        if (err && errlen > 0) snprintf(err, errlen, "plan upload: %s", cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    BatchDev bd;
    bd.inst = dp->inst;
    bd.plans = dp->plans;
    bd.tw32 = dp->tw32;
    bd.tw64 = nullptr;
    bd.rows = dp->rows;
    bd.cols = dp->cols;
    bd.active = nullptr;
    bd.count = count;
    ApplyArgs a{};
    a.V = static_cast<const float2*>(V);
    a.f = static_cast<const float2*>(f);
    a.x = static_cast<const float2*>(x);
    a.out = static_cast<float2*>(out);
    a.norm2 = norm2;
    a.scratch = g_state[dev].scratch;
    e = launch_apply((int)mode, bd, nrows, ncols, a, s);
    if (e != cudaSuccess) {
        if (err && errlen > 0) snprintf(err, errlen, "launch: %s", cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    return NPBS_OK;
}
