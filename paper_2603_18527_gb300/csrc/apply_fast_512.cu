// Cluster-apply variants for 512 x 512 grids: (N1, N2, cluster size, threads, min CTAs per SM[, 1 = row -> column exchange through L2]).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

int fast_variants_512() { return 3; }

cudaError_t prepare_fast_512() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 32, 16, 512, 1>();
    if (e == cudaSuccess) e = set_attr_size<32, 16, 16, 512, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 32, 16, 512, 1, 1>();
    return e;
}

cudaError_t launch_fast_512(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 32, 16, 512, 1>(mode, fd, bd, a, st);
        case 1: return launch_size<32, 16, 16, 512, 1>(mode, fd, bd, a, st);
        case 2: return launch_size<16, 32, 16, 512, 1, 1>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
