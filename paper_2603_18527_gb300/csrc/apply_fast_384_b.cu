// Cluster-apply variants 3-5 for 384 x 384 grids (see apply_fast_384.cu).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

cudaError_t prepare_fast_384_b() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 576, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 384, 1, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 576, 1, 1>();
    return e;
}

cudaError_t launch_fast_384_b(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st) {
    switch (variant) {
        case 3: return launch_size<16, 24, 16, 576, 1>(mode, fd, bd, a, st);
        case 4: return launch_size<16, 24, 16, 384, 1, 1>(mode, fd, bd, a, st);
        case 5: return launch_size<16, 24, 16, 576, 1, 1>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
