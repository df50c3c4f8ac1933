// Cluster-apply variants for 256 x 256 grids: (N1, N2, cluster size, threads, min CTAs per SM).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

int fast_variants_256() { return 4; }

cudaError_t prepare_fast_256() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 16, 8, 256, 3>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 8, 256, 2>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 16, 128, 4>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 16, 256, 2>();
    return e;
}

cudaError_t launch_fast_256(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 16, 8, 256, 3>(mode, fd, bd, a, st);
        case 1: return launch_size<16, 16, 8, 256, 2>(mode, fd, bd, a, st);
        case 2: return launch_size<16, 16, 16, 128, 4>(mode, fd, bd, a, st);
        case 3: return launch_size<16, 16, 16, 256, 2>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
