// Cluster-apply variants for 192 x 192 grids: (N1, N2, cluster size, threads, min CTAs per SM[, 1 = row -> column exchange through L2]).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

int fast_variants_192() { return 4; }

cudaError_t prepare_fast_192() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 12, 4, 384, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 12, 8, 192, 3>();
    if (e == cudaSuccess) e = set_attr_size<16, 12, 16, 192, 3>();
    if (e == cudaSuccess) e = set_attr_size<16, 12, 8, 192, 3, 1>();
    return e;
}

cudaError_t launch_fast_192(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 12, 4, 384, 1>(mode, fd, bd, a, st);
        case 1: return launch_size<16, 12, 8, 192, 3>(mode, fd, bd, a, st);
        case 2: return launch_size<16, 12, 16, 192, 3>(mode, fd, bd, a, st);
        case 3: return launch_size<16, 12, 8, 192, 3, 1>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
