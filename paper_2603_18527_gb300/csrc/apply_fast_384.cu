// Cluster-apply variants for 384 x 384 grids: (N1, N2, cluster size, threads, min CTAs per SM[, 1 = row -> column exchange through L2]).
// Variants 0-2 here, 3-5 in apply_fast_384_b.cu (two translation units compile in parallel).
#include "apply_fast_impl.cuh"

namespace npbs {
using namespace fastimpl;

cudaError_t prepare_fast_384_b();
cudaError_t launch_fast_384_b(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st);

int fast_variants_384() { return 6; }

cudaError_t prepare_fast_384() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 384, 1>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 16, 192, 2>();
    if (e == cudaSuccess) e = set_attr_size<16, 24, 8, 384, 1>();
    if (e == cudaSuccess) e = prepare_fast_384_b();
    return e;
}

cudaError_t launch_fast_384(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                          cudaStream_t st) {
    switch (variant) {
        case 0: return launch_size<16, 24, 16, 384, 1>(mode, fd, bd, a, st);
        case 1: return launch_size<16, 24, 16, 192, 2>(mode, fd, bd, a, st);
        case 2: return launch_size<16, 24, 8, 384, 1>(mode, fd, bd, a, st);
        default: return launch_fast_384_b(variant, mode, fd, bd, a, st);
    }
}

}  // namespace npbs
