// Network internals shared by the network, solver and training files.
#pragma once

#include <functional>
#include <vector>

#include "conv.cuh"
#include "ctx.cuh"

namespace npbs {

struct LayerDef {
    const char* kind;  // enc_a, enc_b, up, dec_a, dec_b
    int level, cin, cout, ups;
    int cin_pad = 0;                 // input channels padded to a multiple of 16
    long long w_off = 0, b_off = 0;  // device layout offsets (float32 master copy)
    long long cw_off = 0, cb_off = 0;  // canonical (OIHW) offsets
};

const std::vector<LayerDef>& layer_defs();
long long dev_param_count();
long long canon_param_count();

// Shape and canonical parameter offsets of an FNO map (fno.cu): square N x N
// grids, C hidden channels, m retained modes of the NLFL and fusion layers
// (Ky x Kx of them), the full-bandwidth residual layer (Fy x Fx modes).
struct FnoDef {
    int n = 0, C = 0, m = 0, L = 0;
    int ca = 1;  // coefficient channels (planes of the batch extent, one after another)
    int skip = 0;  // 1: M = I + N (the output adds the residual input)
    int ky = 0, kx = 0, fy = 0, fx = 0;
    long long lift_a_w = 0, lift_a_b = 0;
    long long spec[8] = {}, loc_w[8] = {}, loc_b[8] = {};
    long long lift_r = 0, spec_r = 0, loc_r = 0, spec_f = 0, loc_f = 0, proj = 0;
    long long count = 0;
    float2* tw = nullptr;  // device W_N^k = exp(-2 pi i k / N), k < N
    RadixPlan plan{};
    // Coefficient-branch cache for inference: NLFL_L(...Phi(a)) of the last
    // prepared instance set, valid while the coefficient field, the instances
    // and the parameters (Net::version) stay the same.
    mutable float* cache = nullptr;
    mutable size_t cache_bytes = 0;
    mutable const float* cache_a = nullptr;
    mutable unsigned long long cache_key = 0;
    mutable long long cache_version = -1;
    // Mode-major copy of every spectral weight block, Wt[k][i][o] (complex;
    // each mode's C x C block padded to an even length), layers in the order
    // spec[0..L), spec_r, spec_f; valid for Net::version
    // == wt_version (refreshed when a network run is prepared).
    mutable float2* wt = nullptr;
    mutable long long wt_version = -1;
};
FnoDef fno_def(int n, int C, int m, int L, int ca = 1);

// Weights, gradients and AdamW moments on one device (U-Net device layout: per
// conv [Cout][9][Cin_pad] then bias, then the 2 x 32 head; an FNO keeps the
// canonical order of its parameters).
struct Net {
    int device = 0;
    long long step = 0;
    FnoDef* fno = nullptr;  // non-null: this network is the FNO map of fno.cu
    long long version = 0;  // bumped whenever the parameters change
    long long count() const { return fno ? fno->count : dev_param_count(); }
    float* params = nullptr;
    float* grads = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    bf16* wb = nullptr;  // bfloat16 copy, [Cout][9][Cin_pad]
    bf16* wt = nullptr;  // flipped transpose for data gradients, [Cin_pad][9][Cout]
    bf16* wsub = nullptr;  // upsampling convs: 2x2 sub-pixel weights [4 parities][Cout][4][Cin_pad]
    std::vector<long long> wb_off;
    std::vector<long long> wsub_off;  // -1 for convs without upsampling
    npbs_status alloc(int dev);
    cudaError_t refresh_bf16(cudaStream_t st) const;
    ~Net();
};

// Instances the network runs on: nb slots of one grid size, element offsets.
struct SlotDev {
    int nb;
    long long np;           // points per instance
    const long long* off;   // device [nb]
};

// A prepared network launch over a set of instances (grouped by size): all
// allocations and host-to-device copies happen in net_prepare, so the run
// functions only launch kernels and can be captured in a CUDA graph.
struct NetGroup {
    int H, W;
    SlotDev sd;
    unsigned long long key = 0;  // hash of the instance offsets (host side)
    long long astride = 0;       // elements between coefficient channels (the batch extent)
};
struct NetRun {
    std::vector<NetGroup> groups;
    bool train = false;
};

// a: the coefficient channel the runs will read (the FNO precomputes its
// coefficient branch here for inference runs; nullable: no precomputation)
npbs_status net_prepare(npbs_ctx* ctx, const Net& net, const Plan& pl, const std::vector<int>& which, bool train,
                        NetRun* run, cudaStream_t st, const float* a = nullptr);

// The FNO counterparts (fno.cu), called by the net_* functions for an FNO network.
npbs_status fno_prepare(npbs_ctx* ctx, const Net& net, const Plan& pl, const std::vector<int>& which, bool train,
                        NetRun* run, cudaStream_t st, const float* a);
npbs_status fno_run_forward(npbs_ctx* ctx, const Net& net, const NetRun& run, const float2* r, const float* a,
                            float2* out, int add, cudaStream_t st);
npbs_status fno_run_backward(npbs_ctx* ctx, Net& net, const NetRun& run, const float2* r, const float* a,
                             const float2* gc, float2* gr, int add, cudaStream_t st);
// out = M(r) (add = 0) or out += M(r) (add = 1)
npbs_status net_run_forward(npbs_ctx* ctx, const Net& net, const NetRun& run, const float2* r, const float* n,
                            float2* out, int add, cudaStream_t st);
// weight gradients += d/dtheta <gc, M(r)>, gr = (or +=) d/dr; run must be prepared with train = true
npbs_status net_run_backward(npbs_ctx* ctx, Net& net, const NetRun& run, const float2* r, const float* n,
                             const float2* gc, float2* gr, int add, cudaStream_t st);
npbs_status net_adamw(npbs_ctx* ctx, Net& net, float lr, float wd, cudaStream_t st);

// The Born-type operator of a training step: mode RESIDUAL writes r_0 of the
// snapshots (x unused), OP_B applies B = I - G V to x, ADJ_B its adjoint;
// norm2 (nullable) receives ||out||^2 per instance.
using BornOp = std::function<npbs_status(int mode, const float2* x, float2* out, double* norm2)>;
// One metric-matched training step (Eq. L_bs_Reta_integral, unrolled, squared)
// for any Born operator over the instances of pl, then one AdamW update.
npbs_status train_step_reta(npbs_ctx* ctx, Net& N, const Plan* pl, const float* n, int unroll, float lr,
                            float weight_decay, float* loss_host, cudaStream_t s, const BornOp& op);

// The operators of the Euclidean objectives (Eqs. L_bs_l2, L_dir):
//   minus_a(x, f_in, out, norm2): out = f_in - A x, norm2 (nullable) += ||out||^2
//   minus_a_adj(y, out):          out = -A^* y
//   green(x, out), green_adj(y, out): G x, G^* y
// out may alias the input of minus_a_adj, green and green_adj.
struct EuclidOps {
    std::function<npbs_status(const float2* x, const float2* f_in, float2* out, double* norm2)> minus_a;
    std::function<npbs_status(const float2* y, float2* out)> minus_a_adj;
    std::function<npbs_status(const float2* x, float2* out)> green;
    std::function<npbs_status(const float2* y, float2* out)> green_adj;
};
// One training step of L_bs_l2 (green_input: the network sees G t) or L_dir
// (the network sees t = f - A u), unrolled from the snapshots, then AdamW.
npbs_status train_step_euclid(npbs_ctx* ctx, Net& N, const Plan* pl, const float* n, const float2* f,
                              const float2* u_snap, int U, bool green_input, float lr, float weight_decay,
                              float* loss_host, cudaStream_t s, const EuclidOps& op);

}  // namespace npbs
