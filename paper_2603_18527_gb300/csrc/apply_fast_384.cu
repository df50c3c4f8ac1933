// Cluster-apply variants for 384 x 384 grids: (N1, N2, cluster size, threads, min CTAs per SM).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

int fast_variants_384() { return 4; }

cudaError_t prepare_fast_384() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 384, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 192, 2>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 8, 384, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 576, 1>();
    return e;
}

cudaError_t launch_fast_384(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 24, 16, 384, 1>(mode, fd, bd, a, st);
        case 1: return launch_size<16, 24, 16, 192, 2>(mode, fd, bd, a, st);
        case 2: return launch_size<16, 24, 8, 384, 1>(mode, fd, bd, a, st);
        case 3: return launch_size<16, 24, 16, 576, 1>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
