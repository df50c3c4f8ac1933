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
cudaError_t prepare_apply_fast();
cudaError_t launch_apply_fast(int n, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st);

}  // namespace npbs
