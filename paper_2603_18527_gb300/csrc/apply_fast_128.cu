// Cluster-apply variants for 128 x 128 grids: (N1, N2, cluster size, threads, min CTAs per SM[, 1 = row -> column exchange through L2]).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

int fast_variants_128() { return 5; }

cudaError_t prepare_fast_128() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 8, 4, 256, 3>();
    if (e == cudaSuccess) e = set_attr_size<16, 8, 8, 128, 4>();
    if (e == cudaSuccess) e = set_attr_size<8, 16, 8, 128, 4>();
    if (e == cudaSuccess) e = set_attr_size<16, 8, 4, 256, 3, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 8, 8, 128, 4, 1>();
    return e;
}

cudaError_t launch_fast_128(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 8, 4, 256, 3>(mode, fd, bd, a, st);
        case 1: return launch_size<16, 8, 8, 128, 4>(mode, fd, bd, a, st);
        case 2: return launch_size<8, 16, 8, 128, 4>(mode, fd, bd, a, st);
        case 3: return launch_size<16, 8, 4, 256, 3, 1>(mode, fd, bd, a, st);
        case 4: return launch_size<16, 8, 8, 128, 4, 1>(mode, fd, bd, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
