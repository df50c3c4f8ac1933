// Launch interface of the single-launch cluster apply (apply_fast.cu).
#pragma once

#include "apply.cuh"

namespace npbs {

// Instances of one square size handled by the cluster kernel.
struct FastDev {
    const int* list;  // device [count]: instance indices
    int count;
};

bool fast_supported(int n);
// number of compiled (N1, N2, cluster, threads) variants for grid side n
int fast_variants(int n);
cudaError_t prepare_apply_fast();
cudaError_t launch_apply_fast(int n, int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st);

}  // namespace npbs
