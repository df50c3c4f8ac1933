// Cluster-apply variants for 256 x 256 grids: (N1, N2, cluster size, threads, min CTAs per SM[, 1 = row -> column exchange through L2]).
// Variants 0-3 here, 4-5 in apply_fast_256_b.cu (two translation units compile in parallel).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

cudaError_t prepare_fast_256_b();
cudaError_t launch_fast_256_b(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st);

int fast_variants_256() { return 6; }

cudaError_t prepare_fast_256() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 16, 8, 256, 3>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 8, 256, 2>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 16, 128, 4>();
    if (e == cudaSuccess) e = set_attr_size<16, 16, 16, 256, 2>();
    if (e == cudaSuccess) e = prepare_fast_256_b();
    return e;
}

cudaError_t launch_fast_256(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 16, 8, 256, 3>(mode, fd, bd, a, st);
        case 1: return launch_size<16, 16, 8, 256, 2>(mode, fd, bd, a, st);
        case 2: return launch_size<16, 16, 16, 128, 4>(mode, fd, bd, a, st);
        case 3: return launch_size<16, 16, 16, 256, 2>(mode, fd, bd, a, st);
        default: return launch_fast_256_b(variant, mode, fd, bd, a, st);
    }
}

}  // namespace npbs
