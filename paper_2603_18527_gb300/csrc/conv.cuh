// Convolution and elementwise kernels of the residual-to-correction U-Net.
// Activations are NHWC bfloat16 with an explicit pixel stride (channels of a
// concatenation share one buffer); accumulation is float32.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace npbs {

using bf16 = __nv_bfloat16;

// One 3x3 (zero padding 1) convolution as an implicit GEMM:
//   out[p, n] = sum_{tap, c} in[nbr(p, tap), c] * w[n, tap, c]   (+ bias, GELU)
// M = B*H*W output pixels, N = Cout, K = 9*Cin.
struct ConvFwd {
    const bf16* x;      // input [B][Hin][Win][xs], channels [xo, xo + Cin) read
    int xs, xo;
    int B, H, W;        // output spatial size; input is H x W, or H/2 x W/2 when ups
    int ups;            // 1: nearest-neighbour x2 upsampling folded into the gather
    int Cin, Cout;      // Cin multiple of 16, Cout multiple of 8
    const bf16* w;      // [Cout][9][Cin]
    const bf16* w_sub;  // ups only (nullable): [parity py*2+px][Cout][4][Cin], 2x2 sub-pixel weights
    const float* bias;  // [Cout] or null
    int act;            // 1: GELU (erf form)
    bf16* y;            // output [B][H][W][ys] at channel offset yo (bf16) ...
    int ys, yo;
    bf16* z;            // ... and optionally the pre-activation in the same layout
    float* yf;          // or float32 output [B][H][W][ys] at yo (no activation)
};

// Weight gradient dW[n, tap, c] += sum_p dz[p, n] * in[nbr(p, tap), c], split
// over pixel ranges with float32 atomics.
struct ConvWgrad {
    const bf16* x;
    int xs, xo;
    int B, H, W, ups;
    int Cin, Cout;
    const bf16* dz;     // [B][H][W][Cout]
    float* dw;          // [Cout][9][Cin], accumulated
    int pix_per_cta;
};

cudaError_t conv_fwd(const ConvFwd& a, cudaStream_t st);
cudaError_t conv_wgrad(const ConvWgrad& a, cudaStream_t st);

// tcgen05 path (conv_tc.cu): used by conv_fwd when the geometry allows TMA
// tiling (no upsampling, W a multiple of 128 or a divisor of 128 with H*W a
// multiple of 128, Cout a multiple of 16 up to 256).
bool conv_tc_supported(const ConvFwd& a);
cudaError_t conv_fwd_tc(const ConvFwd& a, cudaStream_t st);
// tcgen05 weight gradient (conv_tc.cu): used by conv_wgrad when there is no
// upsampling in the gather, the grid splits into 64-pixel runs (W a multiple
// of 64, or whole rows), Cin is 16, 32 or a multiple of 64 and Cout 32 or a
// multiple of 64 up to 256.  NPBS_WGRAD=mma forces the warp-level kernel.
bool conv_wgrad_tc_supported(const ConvWgrad& a);
cudaError_t conv_wgrad_tc(const ConvWgrad& a, cudaStream_t st);
cudaError_t prepare_conv_tc();
int conv_tc_timeout_flag();   // 1 once a bounded device wait gave up (synchronous read)
void conv_tc_clear_timeout();
int newton_tc_timeout_flag();  // the same for the tensor-core Newton apply (newton.cu)
void newton_tc_clear_timeout();
// One CTA waits on an mbarrier nothing arrives at for `seconds`, then gives up.
cudaError_t wait_selftest(double seconds, cudaStream_t st);

}  // namespace npbs
