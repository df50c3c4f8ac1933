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
// arrays of fixed size (about 8.3 MiB).  The CUDA runtime places them on a
// device when the library's module is loaded there: under lazy module loading
// (the default) that happens in the first call on the device, which therefore
// must come before the caller's own pool takes the device's memory (or the
// process runs with CUDA_MODULE_LOADING=EAGER).  From then on the device holds
// them until the process exits.
//
// The plan (instance table, radix plans, twiddles, row / column work items)
// is written on the device by a small set-up kernel from its launch
// parameters, in stream order before the apply kernels; no host buffer is
// read after the call returns.
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
        if (err && errlen > 0)
            snprintf(err, errlen,
                     "loading the static scratch on device %d failed (%s): the first call on a device must come "
                     "before other allocators take its memory",
                     dev, cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    s.scratch = static_cast<float2*>(p);
    e = cudaGetSymbolAddress(&p, g_static_plan);
    if (e != cudaSuccess) {
        if (err && errlen > 0)
            snprintf(err, errlen, "loading the static plan on device %d failed (%s)", dev, cudaGetErrorString(e));
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

// Everything the set-up kernel needs, passed by value as its launch parameter
// (about 4.5 KB): the instance table with each instance's first row and
// column work item, and the distinct transform lengths.
struct StaticParams {
    InstDev inst[kStaticMaxInstances];
    int row0[kStaticMaxInstances + 1];  // first row item of instance j; row0[count] = number of row items
    int col0[kStaticMaxInstances + 1];
    int sizes[kStaticMaxSizes];
    int count, nsizes;
};

// Radix schedule 8, 4, 2 then 3 (the same rule as the context's plans).
__host__ __device__ inline bool radix_plan_of(int n, RadixPlan* p) {
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

// Rows per row item and columns per column item of an nx x ny instance (the
// tiling of the three-launch apply).
__host__ __device__ inline int rows_per_item(int nx, int ny) {
    const int t = kTileElems<float>() / nx;
    return t < 1 ? 1 : (t < ny ? t : ny);
}
__host__ __device__ inline int cols_per_item(int ny) {
    const int t = kTileElems<float>() / ny;
    return t < 1 ? 1 : (t < 16 ? t : 16);
}

// Writes the plan of one call into the static plan array.  Grid-stride over
// the instance table, the twiddle tables and the work items.
__global__ void k_static_plan(const __grid_constant__ StaticParams p, StaticPlan* dp) {
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int j = t0; j < p.count; j += nt) dp->inst[j] = p.inst[j];
    for (int k = t0; k < p.nsizes; k += nt) radix_plan_of(p.sizes[k], &dp->plans[k]);
    for (int e = t0; e < p.nsizes * kMaxN; e += nt) {
        const int k = e / kMaxN, q = e - k * kMaxN, n = p.sizes[k];
        if (q < n) {
            double sn, cs;
            sincospi(-2.0 * (double)q / (double)n, &sn, &cs);
            dp->tw32[e] = make_float2((float)cs, (float)sn);
        }
    }
    for (int i = t0; i < p.row0[p.count]; i += nt) {
        int j = 0;
        while (p.row0[j + 1] <= i) ++j;
        const InstDev& d = p.inst[j];
        const int rp = rows_per_item(d.nx, d.ny), r0 = (i - p.row0[j]) * rp;
        dp->rows[i] = RowItem{j, r0, rp < d.ny - r0 ? rp : d.ny - r0, 0};
    }
    for (int i = t0; i < p.col0[p.count]; i += nt) {
        int j = 0;
        while (p.col0[j + 1] <= i) ++j;
        const InstDev& d = p.inst[j];
        const int cp = cols_per_item(d.ny), c0 = (i - p.col0[j]) * cp;
        dp->cols[i] = ColItem{j, c0, cp < d.nx - c0 ? cp : d.nx - c0, 0};
    }
}

// Parameter block of the call in progress (guarded by g_mutex).
StaticParams g_params;

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

    // Plan on the host into the parameter block (one call at a time on the host).
    std::lock_guard<std::mutex> lock(g_mutex);
    StaticParams& hp = g_params;
    int nsizes = 0;
    int nrows = 0, ncols = 0;
    long long extent = 0;
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
            while (k < nsizes && hp.sizes[k] != dims[d]) ++k;
            if (k == nsizes) {
                if (nsizes == kStaticMaxSizes)
                    return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE,
                                "cbs_apply_static: more distinct grid sizes than the static limit of 8");
                RadixPlan rp;
                if (!radix_plan_of(dims[d], &rp))
                    return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, "grid side is not 2^a 3^b in [2, 1024]");
                hp.sizes[nsizes++] = dims[d];
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
        const int rp = rows_per_item(s.nx, s.ny), cp = cols_per_item(s.ny);
        hp.row0[j] = nrows;
        hp.col0[j] = ncols;
        nrows += (s.ny + rp - 1) / rp;
        ncols += (s.nx + cp - 1) / cp;
        if (nrows > kStaticMaxItems)
            return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, "cbs_apply_static: too many row work items");
        if (ncols > kStaticMaxItems)
            return fail(err, errlen, NPBS_ERR_UNSUPPORTED_SIZE, "cbs_apply_static: too many column work items");
    }
    hp.row0[count] = nrows;
    hp.col0[count] = ncols;
    hp.count = count;
    hp.nsizes = nsizes;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(err, errlen, NPBS_ERR_CUDA, "no current CUDA device");
    npbs_status st = setup_current_device(dev, err, errlen);
    if (st != NPBS_OK) return st;
    StaticPlan* dp = g_state[dev].plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // The plan is written on the device, in stream order, from the launch
    // parameters (captured by value at launch).
    k_static_plan<<<32, 256, 0, s>>>(hp, dp);
    cudaError_t e = cudaGetLastError();
    // the reductions accumulate: norm2 must start at zero
    if (e == cudaSuccess && norm2) e = cudaMemsetAsync(norm2, 0, sizeof(double) * count, s);
    if (e != cudaSuccess) {
        if (err && errlen > 0) snprintf(err, errlen, "plan set-up: %s", cudaGetErrorString(e));
        return NPBS_ERR_CUDA;
    }
    BatchDev bd;
    bd.inst = dp->inst;
    bd.plans = dp->plans;
    bd.tw32 = dp->tw32;
    bd.twds = nullptr;
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
