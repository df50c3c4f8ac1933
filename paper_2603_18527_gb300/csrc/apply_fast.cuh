// Launch interface of the square-grid apply (apply_fast.cu): the single-launch
// cluster kernel for sides 128..512, the three-launch band kernels for 1024.
#pragma once

#include "apply.cuh"

namespace npbs {

// Instances of one square size handled by the cluster (or band) kernels.
struct FastDev {
    const int* list;  // device [count]: instance indices
    int count;
    int ahead;        // > 0: after its loads, cluster c prefetches into L2 the rows of list[c + ahead]
                      // (the launcher sets a third of the resident cluster count)
};

bool fast_supported(int n);
// number of variants V for grid side n: every compiled (N1, N2, cluster,
// threads, min CTAs) configuration, without (variant < V/2) and with
// (variant >= V/2) the L2 prefetch of the instance each cluster slot runs next;
// for 1024 every compiled band configuration (rows and columns per block)
int fast_variants(int n);
// kernel launches issued by one launch_apply_fast call
int fast_kernel_launches(int n, int mode, int steps);
cudaError_t prepare_apply_fast();
cudaError_t launch_apply_fast(int n, int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st);

}  // namespace npbs
