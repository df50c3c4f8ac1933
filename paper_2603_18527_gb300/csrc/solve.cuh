// Mixed-precision refinement driver shared by the stationary solvers.
#pragma once

#include <functional>
#include <vector>

#include "ctx.cuh"

namespace npbs {

// Buffers of one refined solve.  delta: complex64 correction; rho: complex64
// copy of the float64 residual (the inner source term); nb: per-instance
// squared inner Born residual written by the last step of a chunk; active:
// per-instance mask.
struct RefineWork {
    float2* delta = nullptr;
    float2* rho = nullptr;
    double* nb = nullptr;
    int* active = nullptr;
    double max_reduction = 1e-3;   // refresh once the inner residual fell by this factor
    int max_cycle = 1 << 30;       // refresh at least every this many iterations
    // called (outside any capture) with the active instances whenever the set
    // changes; the captured inner-chunk graph is rebuilt afterwards
    std::function<npbs_status(const std::vector<int>&)> on_active;
    // called after every float64 refresh with the per-instance rTol, the
    // active mask and the mask of instances this refresh updated; returns true
    // when the inner step changed shape (forces the graph and on_active to be
    // redone)
    std::function<bool(const std::vector<double>&, const std::vector<int>&, const std::vector<int>&)> on_refresh;
    std::vector<int> flags;  // per-instance flags reported to the caller
    // optional: a whole chunk of `steps` inner iterations in one call (the last
    // writes nb), used instead of `steps` InnerStep calls when set
    std::function<npbs_status(int steps)> fused;
};

// One inner iteration on delta; `last` asks it to write the squared Born
// residual norms into RefineWork::nb.
using InnerStep = std::function<npbs_status(bool last)>;

// Solvers run on a context-owned, capturable stream that first waits for the
// caller's stream (which may be the legacy default stream, not capturable).
npbs_status solve_stream_begin(npbs_ctx* ctx, cudaStream_t user, cudaStream_t* work);

// V = k^2 - k0^2 - i eps (float32) for every instance, into a context buffer.
npbs_status solver_potential(npbs_ctx* ctx, const Plan& pl, const float2* k2, cudaStream_t st, const float2** V);

npbs_status refine_driver(npbs_ctx* ctx, const Plan& pl, const float2* k2, const float2* V, const float2* f, double2* u,
                          const npbs_solve_opts& o, npbs_report* rep, cudaStream_t st, const InnerStep& step,
                          RefineWork& w);
npbs_status check_solve_args(npbs_ctx* ctx, const npbs_solve_opts* o, const void* k2, const void* f,
                             const void* u);

}  // namespace npbs
