// Square-grid apply: size dispatch and the per-size variant tables.  Sides
// 128..512 run the single-launch cluster kernel (apply_fast_impl.cuh,
// instantiated per grid size in apply_fast_<N>.cu so the sizes compile in
// parallel); side 1024 runs the three-launch band kernels (apply_band.cu).
#include "apply_fast.cuh"

#include <algorithm>

namespace npbs {

#define NPBS_FAST_SIZES(X) X(128) X(192) X(256) X(384) X(512)
#define NPBS_DECL(n)                                                                                        \
    int fast_variants_##n();                                                                              \
    cudaError_t prepare_fast_##n();                                                                       \
    cudaError_t launch_fast_##n(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a, \
                                cudaStream_t st);
NPBS_FAST_SIZES(NPBS_DECL)
#undef NPBS_DECL
int band_variants_1024();
cudaError_t prepare_band_1024();
cudaError_t launch_band_1024(int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                             cudaStream_t st);

bool fast_supported(int n) { return n == 128 || n == 192 || n == 256 || n == 384 || n == 512 || n == 1024; }

static int kernel_variants(int n) {
    switch (n) {
        case 128: return fast_variants_128();
        case 192: return fast_variants_192();
        case 256: return fast_variants_256();
        case 384: return fast_variants_384();
        case 512: return fast_variants_512();
        case 1024: return band_variants_1024();
        default: return 0;
    }
}

// the band kernels have no prefetch twin: they stream whole bands
int fast_variants(int n) { return n == 1024 ? kernel_variants(n) : 2 * kernel_variants(n); }

int fast_kernel_launches(int n, int mode, int steps) {
    if (n != 1024) return 1;
    const bool iter = mode == NPBS_CBS_STEP || mode == NPBS_PREC_SWEEP;
    return 3 * (iter ? std::max(1, steps) : 1);
}

cudaError_t prepare_apply_fast() {
    cudaError_t e = cudaSuccess;
#define NPBS_PREP(n) \
    if (e == cudaSuccess) e = prepare_fast_##n();
    NPBS_FAST_SIZES(NPBS_PREP)
#undef NPBS_PREP
    if (e == cudaSuccess) e = prepare_band_1024();
    return e;
}

cudaError_t launch_apply_fast(int n, int variant, int mode, const FastDev& fd, const BatchDev& bd, const ApplyArgs& a,
                              cudaStream_t st) {
    if (fd.count == 0) return cudaSuccess;
    if (n == 1024) {
        if (variant < 0 || variant >= band_variants_1024()) return cudaErrorInvalidValue;
        return launch_band_1024(variant, mode, fd, bd, a, st);
    }
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
