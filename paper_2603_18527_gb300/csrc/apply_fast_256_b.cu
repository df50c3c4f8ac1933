// Cluster-apply variants 4-5 for 256 x 256 grids (see apply_fast_256.cu).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

cudaError_t prepare_fast_256_b() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 16, 8, 256, 2, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 16, 128, 4, 1>();
    return e;
}

cudaError_t launch_fast_256_b(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st) {
    switch (variant) {
        case 4: return launch_size<16, 16, 8, 256, 2, 1>(mode, fd, bd, a, st);
        case 5: return launch_size<16, 16, 16, 128, 4, 1>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
