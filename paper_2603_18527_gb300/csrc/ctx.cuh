// Context internals shared by the C ABI implementation files.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "apply.cuh"
#include "apply_fast.cuh"
#include "common.cuh"

namespace npbs {

// Device copy of a batch description: instances, radix plans, twiddles and
// the row / column work items for float32 and float64 tiles.
struct Plan {
    int count = 0;
    long long extent = 0;         // one past the last element used by any instance
    long long points = 0;         // sum of nx * ny
    std::vector<InstDev> inst_h;
    InstDev* inst = nullptr;
    RadixPlan* plans = nullptr;
    float2* tw32 = nullptr;
    float4* twds = nullptr;
    RowItem* rows32 = nullptr;
    ColItem* cols32 = nullptr;
    RowItem* rows64 = nullptr;
    ColItem* cols64 = nullptr;
    int nrow32 = 0, ncol32 = 0, nrow64 = 0, ncol64 = 0;
    VecItem* vitems = nullptr;
    int nvec = 0;
    // float32 modes: square instances of a cluster-kernel size (or 1024) go
    // to one group per size; the rest use the generic three-launch path
    // (rows32s / cols32s)
    struct FastGroup {
        int n = 0;
        int* list = nullptr;
        int count = 0;
        std::vector<int> list_h;
        // compacted active subset for the mask `alist_mask` (set_active_lists)
        int* alist = nullptr;
        mutable int acount = 0;
    };
    mutable const int* alist_mask = nullptr;
    std::vector<FastGroup> fast;
    RowItem* rows32s = nullptr;
    ColItem* cols32s = nullptr;
    int nrow32s = 0, ncol32s = 0;
    long long last_use = 0;  // LRU stamp in the context's plan cache
    BatchDev bd(bool f64, const int* active) const {
        BatchDev b;
        b.inst = inst;
        b.plans = plans;
        b.tw32 = tw32;
        b.twds = twds;
        b.rows = f64 ? rows64 : rows32;
        b.cols = f64 ? cols64 : cols32;
        b.active = active;
        b.count = count;
        return b;
    }
    ~Plan();
};

// Growable device buffer owned by a context.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need);
    ~DevBuf();
};

}  // namespace npbs

struct npbs_ctx {
    int device = 0;
    std::string err;
    std::map<std::string, std::unique_ptr<npbs::Plan>> plans;
    long long plan_clock = 0;
    npbs::DevBuf scratch;   // spectrum between apply passes
    npbs::DevBuf work[21];  // solver workspaces (12-17: the CDR operators, 18-20: Newton)
    // the last prepared CDR / Newton batch (its device tables stay in work[12] /
    // work[18]): reused while a call describes exactly the same batch
    std::shared_ptr<void> cdr_prep, nt_prep;
    npbs::DevBuf net_ws;    // network activations
    bool use_fast = true;  // cluster apply for square 128..512 grids, band kernels for 1024
                           // (NPBS_APPLY_PATH=three_pass disables both)
    std::map<int, int> fast_variant;  // grid side -> chosen cluster-kernel variant (autotuned; default 0)
    // grid side -> (variant, max count): the lowest-latency variant, used
    // instead when at most `max count` instances of that side are launched
    // (the few-instance tail of a solve); autotuned
    std::map<int, std::pair<int, int>> fast_tail;
    // grid side -> largest instance count for which a chunk of fused steps
    // (cbs_steps, the solvers' inner chunks) runs as one launch; larger groups
    // take one launch per step.  Autotuned; kDefaultFusedMax until then.
    std::map<int, int> fast_fused_max;
    static constexpr int kDefaultFusedMax = 8;
    cudaStream_t solve_stream = nullptr;  // capturable stream the solvers run on
    cudaEvent_t solve_event = nullptr;
    // side streams on which the cluster applies of different grid sides run
    // concurrently (fork / join by events, so they also work under capture)
    static constexpr int kAux = 4;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kAux] = {};
    long long launches = 0;         // kernels launched (graph launches count their kernels)
    long long capture_kernels = 0;  // kernels recorded into the graph being captured
    void count(cudaStream_t st, long long k) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusActive) capture_kernels += k;
        else launches += k;
    }
};

namespace npbs {

npbs_status set_err(npbs_ctx* ctx, npbs_status st, const std::string& msg);
npbs_status cuda_err(npbs_ctx* ctx, cudaError_t e, const char* where);
// Validate the batch and return its (cached) device plan; nullptr on error
// with the status in *st.
const Plan* get_plan(npbs_ctx* ctx, const npbs_batch* batch, npbs_status* st);
// Launch one apply of `mode` on the plan (float32 modes or kTrueRes64).
npbs_status run_apply(npbs_ctx* ctx, const Plan& pl, int mode, const ApplyArgs& a, const int* active,
                      cudaStream_t st);
// Record which instances the device mask `active_dev` currently enables (host
// copy `act`): cluster-kernel launches under that mask then cover only those
// instances and skip empty size groups.  Call outside stream capture whenever
// an instance becomes active again; deactivations only make the lists loose
// (the kernels still check the mask).  Synchronous.
npbs_status set_active_lists(npbs_ctx* ctx, const Plan& pl, const std::vector<int>& act, const int* active_dev);

}  // namespace npbs

#define NPBS_CK(ctx, call)                                                   \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) return npbs::cuda_err((ctx), _e, #call);      \
    } while (0)
