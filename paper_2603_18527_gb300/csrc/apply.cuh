// Launch interface of the fused Born apply (apply.cu).
#pragma once

#include "common.cuh"

namespace npbs {

constexpr int kThreads = 256;
// Elements of one shared-memory tile buffer (two buffers per block, 64 KB).
template <typename R> constexpr int kTileElems() { return sizeof(R) == 4 ? 4096 : 2048; }

// Internal mode: float64 true residual f - A u on the complex128 solution,
// after folding the complex64 correction into it (mixed-precision refinement).
constexpr int kTrueRes64 = 100;

struct ApplyArgs {
    const float2* V;
    const float2* f;
    const float2* x;
    float2* out;
    double* norm2;      // per-instance squared norm (atomically accumulated; zero before)
    double* norm2b;     // kTrueRes64: per-instance ||f||^2
    void* scratch;      // spectrum between passes (complex64 or complex128 per point)
    double2* uhi;       // kTrueRes64: complex128 solution (updated in place)
    const float2* delta;  // kTrueRes64: complex64 correction folded into uhi (nullable)
    const float2* k2;     // kTrueRes64: k^2 (nullable: then k^2 = V + k0^2 + i eps)
    int steps;            // CBS_STEP / PREC_SWEEP: consecutive in-place steps (0 or 1: one); step
                          // k >= 1 reads x from out; norm2 is the last step's
};

// Opt the apply kernels into their dynamic shared memory (once per device).
cudaError_t prepare_apply();
cudaError_t launch_apply(int mode, const BatchDev& bd, int nrow_items, int ncol_items, const ApplyArgs& a,
                         cudaStream_t st);

}  // namespace npbs
