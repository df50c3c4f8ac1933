// Single-launch cluster apply: size dispatch and the per-size variant tables
// (the kernel itself is in apply_fast_impl.cuh, instantiated per grid size in
// apply_fast_<N>.cu so the sizes compile in parallel).
#include "apply_fast.cuh"

namespace npbs {

#define NPBS_FAST_SIZES(X) X(128) X(192) X(256) X(384) X(512)
#define NPBS_DECL(n)                                                                                        \
    int fast_variants_##n();                                                                              \
    cudaError_t prepare_fast_##n();                                                                       \
    cudaError_t launch_fast_##n(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a, \
                                cudaStream_t st);
NPBS_FAST_SIZES(NPBS_DECL)
#undef NPBS_DECL

bool fast_supported(int n) { return n == 128 || n == 192 || n == 256 || n == 384 || n == 512; }

static int kernel_variants(int n) {
    switch (n) {
        case 128: return fast_variants_128();
        case 192: return fast_variants_192();
        case 256: return fast_variants_256();
        case 384: return fast_variants_384();
        case 512: return fast_variants_512();
        default: return 0;
    }
}

int fast_variants(int n) { return 2 * kernel_variants(n); }

cudaError_t prepare_apply_fast() {
    cudaError_t e = cudaSuccess;
#define NPBS_PREP(n) \
    if (e == cudaSuccess) e = prepare_fast_##n();
    NPBS_FAST_SIZES(NPBS_PREP)
#undef NPBS_PREP
    return e;
}

cudaError_t launch_apply_fast(int n, int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st) {
    if (fd.count == 0) return cudaSuccess;
    const int nv = kernel_variants(n);
    if (variant < 0 || variant >= 2 * nv) return cudaErrorInvalidValue;
    FastDev f2 = fd;
    f2.ahead = variant >= nv ? 1 : 0;  // launch_one replaces 1 by the resident cluster count
    variant %= nv;
    switch (n) {
#define NPBS_CASE(n) \
    case n: return launch_fast_##n(variant, mode, f2, bd, a, st);
        NPBS_FAST_SIZES(NPBS_CASE)
#undef NPBS_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npbs
