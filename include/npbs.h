/*
 * npbs.h - C ABI of the GB300 (sm_103a) Born-preconditioned Helmholtz library.
 *
 * The library implements the hot path of Neural Preconditioned Born Series
 * (NPBS): the Born-preconditioned residual apply r = G_eta(V_eta u + f) - u,
 * the CBS and NPBS iterations built on it, FGMRES on the Lippmann-Schwinger
 * system, and the learned residual-to-correction U-Net with its training step.
 *
 * Discretisation (App. Fourier Pseudospectral Discretization): every instance
 * lives on a periodic ny x nx grid with spacing h (absorbing layer included),
 * row-major [ny][nx]; modes n in {-N/2..N/2-1}, xi = 2 pi n/(N h), forward DFT
 * unnormalised, inverse scaled by 1/(nx ny).  Supported sizes: nx, ny of the
 * form 2^a 3^b with 2 <= n <= 1024 (anything else is NPBS_ERR_UNSUPPORTED_SIZE;
 * there is no fallback path).
 *
 * Operators (Sec. 3.1):
 *   lambda(xi) = |xi|^2 - k0^2 - i eps          symbol of L_eta
 *   G q        = F^{-1}(F q / lambda)          Green operator, G = L_eta^{-1}
 *   V          = k^2 - k0^2 - i eps             perturbation (pointwise)
 *   A u        = F^{-1}(|xi|^2 F u) - k^2 u     Helmholtz operator, A = L_eta - V
 *   gamma      = i V / eps                      CBS diagonal preconditioner
 *   B          = I - G V                        Lippmann-Schwinger operator (Eq. LS_discrete)
 *
 * Memory.  Every field argument is caller-owned DEVICE memory holding the whole
 * batch: instance j occupies elements [offset_j, offset_j + nx_j ny_j) of each
 * buffer.  Complex fields are interleaved (re, im): complex64 (8 bytes) unless
 * a parameter says complex128.  Real per-point fields (the refractive index n)
 * use the same offsets in float32 elements.  Offsets must be multiples of 32
 * elements.  The library never frees or retains caller buffers past a call.
 * It owns only the internals of npbs_ctx and npbs_net (workspace, plans,
 * captured graphs, weights, moments).
 *
 * Errors.  Every call returns a status; nothing aborts or traps.  Device waits
 * are bounded.  npbs_last_error() gives a one-line message for the last failure
 * on a context.
 *
 * Streams.  Calls taking a stream are asynchronous on it except where noted
 * ("synchronises"): the solvers synchronise before filling their report.
 * Threads.  A context (and a network) is used by one host thread at a time:
 * its plan cache, workspaces, autotuned choices and side streams are not
 * locked.  Separate contexts may be used from separate threads.
 * cbs_apply and cbs_steps may be captured into a CUDA graph on the caller's
 * stream once a call with the same batch has run outside capture (that call
 * builds the batch plan and workspace; later calls only enqueue work, forking
 * side streams by events for concurrent grid sides).
 */
#ifndef NPBS_H
#define NPBS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* npbs_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    NPBS_OK = 0,
    NPBS_ERR_INVALID_ARG = 1,
    NPBS_ERR_UNSUPPORTED_SIZE = 2,
    NPBS_ERR_NONFINITE = 3,
    NPBS_NOT_CONVERGED = 4,
    NPBS_ERR_DEVICE_TIMEOUT = 5,
    NPBS_ERR_CUDA = 6,
    NPBS_ERR_OOM = 7
} npbs_status;

typedef struct npbs_ctx npbs_ctx;
typedef struct npbs_net npbs_net;

/* One instance.  nx, ny: full grid including the absorbing layer.  h: grid
 * spacing.  k0sq, eps: k0^2 and eta of L_eta (eps > 0).  offset: first element
 * of this instance in every field buffer (multiple of 32). */
typedef struct {
    int32_t nx, ny;
    double h, k0sq, eps;
    int64_t offset;
} npbs_instance;

typedef struct {
    int32_t count;              /* number of instances, >= 0 */
    const npbs_instance* inst;  /* HOST array [count] */
} npbs_batch;

/* Apply modes of cbs_apply.  x is the field operated on, out the result.
 *   NPBS_RESIDUAL      out = G(V x + f) - x                      (Eq. npbs_integral)
 *   NPBS_CBS_STEP      out = x + gamma (G(V x + f) - x)          (Eq. CBS); out may alias x
 *   NPBS_OP_B          out = x - G(V x)                          (Eq. LS_discrete)
 *   NPBS_ADJ_B         out = x - conj(V) G^*(x), G^* symbol 1/conj(lambda)
 *   NPBS_TRUE_RESIDUAL out = f - A x                             (Sec. 5 stopping rule)
 *   NPBS_PREC_SWEEP    out = x + gamma (f - B x): one CBS Richardson sweep for
 *                      B z = f with f in preconditioned coordinates
 * norm2 (nullable, DEVICE double[count]) receives, per instance, the squared
 * 2-norm of G(Vx+f)-x for RESIDUAL / CBS_STEP (before the update), of out for
 * OP_B, ADJ_B, TRUE_RESIDUAL, and of f - B x for PREC_SWEEP.  It is
 * overwritten, not accumulated. */
typedef enum {
    NPBS_RESIDUAL = 0,
    NPBS_CBS_STEP = 1,
    NPBS_OP_B = 2,
    NPBS_ADJ_B = 3,
    NPBS_TRUE_RESIDUAL = 4,
    NPBS_PREC_SWEEP = 5
} npbs_mode;

typedef struct {
    double rtol;          /* target ||f - A u|| / ||f|| (Sec. 5) */
    int32_t max_iter;     /* cap on iterations (CBS/NPBS updates or FGMRES steps) */
    int32_t check_every;  /* iterations between convergence checks (>= 1) */
    int32_t use_graph;    /* capture the inner loop in a CUDA graph (0/1) */
} npbs_solve_opts;

typedef struct {
    int32_t* iters;        /* HOST [count]: iterations at the passing check (or at the cap) */
    double* rtol;          /* HOST [count]: final ||f - A u|| / ||f|| in float64 */
    npbs_status* status;   /* HOST [count]: NPBS_OK or NPBS_NOT_CONVERGED / NPBS_ERR_NONFINITE */
    int32_t* flags;        /* HOST [count], nullable: npbs_solve sets 1 where the divergence
                            * guard switched the instance to plain CBS steps */
} npbs_report;

/* ---- context ------------------------------------------------------------ */

/* Device-side failures.  Every wait inside the library's kernels (TMA and
 * tensor-core pipeline barriers) is bounded (about 2 s); a wait that gives up
 * records it in a device flag, and the kernel cleans up and returns, leaving
 * its outputs invalid.  npbs_device_status synchronises the device and
 * returns NPBS_ERR_DEVICE_TIMEOUT (clearing the flag) if that happened since
 * the last call, else NPBS_OK. */
npbs_status npbs_device_status(npbs_ctx* ctx);
/* Exercises that path without harm: one thread waits `seconds` (0 < s <= 2)
 * on a barrier that nothing completes, gives up and sets the flag; the next
 * npbs_device_status returns NPBS_ERR_DEVICE_TIMEOUT.  Asynchronous. */
npbs_status npbs_test_device_timeout(npbs_ctx* ctx, double seconds, npbs_stream stream);

/* Create a context on CUDA device `device` (made current for the call). */
npbs_status npbs_create(npbs_ctx** out, int device);
npbs_status npbs_destroy(npbs_ctx* ctx);
/* One-line description of the last error on ctx ("" if none).  Owned by ctx. */
const char* npbs_last_error(const npbs_ctx* ctx);
/* Library version string, static storage. */
const char* npbs_version(void);
/* Number of kernels launched through ctx so far (graph launches count the
 * kernels they contain); -1 for a NULL ctx.  For benchmarks. */
int64_t npbs_launch_count(const npbs_ctx* ctx);

/* Process-wide counts of network convolution calls (forward, input gradient
 * and weight gradient) by engine: the tcgen05 tensor-core kernels (TMA-fed,
 * TMEM accumulators) and the warp-level MMA kernels used where TMA cannot
 * tile the geometry (grids whose 128- or 64-pixel runs do not tile the image)
 * or when NPBS_CONV=mma / NPBS_WGRAD=mma force them.  For benchmarks. */
void npbs_conv_stats(int64_t* tensor_core_launches, int64_t* warp_mma_launches);

/* ---- problem set-up ----------------------------------------------------- */

/* The medium, its absorbing layer and the potential (Sec. 3.1: the Helmholtz
 * problem with k = omega n(x), truncated by an absorbing layer folded into the
 * operator; App. Dataset Illustration: a padded grid around the interior).
 * For every instance j:
 *   k^2(x) = omega_j^2 n(x)^2 + i a omega_j^2 rho(x)^2,  a = ramp_amp_over_omega2,
 *   rho = max(d_x, d_y) / W, W = layer_cells, d = depth in cells into the W-cell
 *   layer along each side (1 .. W at the outermost cell, 0 inside; the larger
 *   of the two in the corners),
 * computed in float64 and stored as complex64 in k2_out; then the reference
 * constants and potential as npbs_potential_from_k2.  The paper describes the
 * layer only as a sponge / PML; this quadratic ramp up to a omega^2 is the
 * library's reading.
 * n: DEVICE float32 refractive index with the batch layout.  omega: HOST
 * double[count], > 0.  layer_cells >= 0 (0: no layer), the same for every
 * instance of the call (call once per layer width).  ramp_amp_over_omega2 >= 0.
 * k2_out: DEVICE complex64 (nullable: then a context buffer holds k^2 for the
 * call only); V_out: DEVICE complex64 (nullable); k0sq_out, eps_out: HOST
 * double[count].  At most 65535 instances.  Synchronises the stream. */
npbs_status npbs_build_potential(npbs_ctx* ctx, const npbs_batch* batch, const float* n,
                                 const double* omega, int32_t layer_cells,
                                 double ramp_amp_over_omega2, void* k2_out, void* V_out,
                                 double* k0sq_out, double* eps_out, npbs_stream stream);

/* Reference constants and potential from a given k^2 (Sec. 3.1; the paper
 * leaves k0 and eta free, this library takes k0^2 = (min Re k^2 + max Re k^2)/2
 * and eps = max |k^2 - k0^2| over each instance's full grid).
 * k2: DEVICE complex64 k(x)^2 (Im k^2 >= 0 carries the absorbing layer).
 * V_out: DEVICE complex64, receives V = k^2 - k0^2 - i eps (may be NULL).
 * k0sq_out, eps_out: HOST double[count].  The k0sq / eps fields of `batch`
 * are ignored.  Synchronises the stream. */
npbs_status npbs_potential_from_k2(npbs_ctx* ctx, const npbs_batch* batch, const void* k2,
                                   void* V_out, double* k0sq_out, double* eps_out,
                                   npbs_stream stream);

/* ---- the apply (Eq. CBS / Eq. npbs_integral / Eq. LS_discrete) ------------ */

/* One fused Born apply over the batch in the given mode (see npbs_mode).
 * V, f, x, out: DEVICE complex64.  f may be NULL for OP_B and ADJ_B.  Inputs
 * other than x may not alias out.  Asynchronous. */
npbs_status cbs_apply(npbs_ctx* ctx, const npbs_batch* batch, const void* V, const void* f,
                      const void* x, void* out, npbs_mode mode, double* norm2,
                      npbs_stream stream);

/* `steps` consecutive in-place CBS steps (Eq. CBS: u <- u + gamma (G(V u + f)
 * - u)) or preconditioner sweeps (PREC_SWEEP: z <- z + gamma (v - B z), with v
 * in f) on every instance: the same arithmetic as `steps` cbs_apply calls
 * whose output feeds the next call's x (bit-identical results).  For the
 * square sides 128..512 a grid side with few instances (at most an
 * autotuned count, 8 before npbs_autotune_apply) runs all steps in one
 * cluster launch, so that after the first step the operands come from L2 and
 * no launch gaps remain; larger groups, which fill the GPU, run one launch
 * per step.  Side 1024 and the other grids run three launches per step.
 * Step 0 reads x, later steps read out; x may alias out.  mode: CBS_STEP or
 * PREC_SWEEP (anything else: NPBS_ERR_INVALID_ARG); steps >= 0 (0: nothing).
 * norm2 (nullable, DEVICE float64 [count], zeroed by the call) receives the
 * squared norm of the last step's residual G(V x + f) - x (PREC_SWEEP: v - B x).
 * V, f, x, out: DEVICE complex64 with the batch layout.  Asynchronous. */
npbs_status cbs_steps(npbs_ctx* ctx, const npbs_batch* batch, const void* V, const void* f,
                      const void* x, void* out, npbs_mode mode, int32_t steps, double* norm2,
                      npbs_stream stream);

/* Autotuner for the square-grid apply: for every square grid side of the
 * batch that has a cluster kernel (128, 192, 256, 384, 512), time each
 * compiled (N1 x N2 factorisation, cluster size, threads, with or without the
 * L2 prefetch of the next instance) variant over `reps` CBS_STEP applies on
 * the caller's data and keep the fastest for later calls on ctx; side 1024
 * (three-launch band kernels) likewise over its compiled band shapes (rows
 * and columns per block).  It also
 * times one instance per variant and keeps the lowest-latency variant for
 * launches of at most the largest power-of-two count of instances for which
 * it stays faster (the few unconverged instances late in a solve), and the
 * largest instance count for which a launch of fused steps (cbs_steps and
 * the solvers' inner chunks) beats one launch per step.  x is
 * overwritten (it is iterated in place).  chosen (nullable, HOST int32 per
 * grid side present, in increasing side order) receives side * 16 + variant
 * of the throughput choice.  Synchronises the stream. */
npbs_status npbs_autotune_apply(npbs_ctx* ctx, const npbs_batch* batch, const void* V, const void* f,
                                void* x, int32_t reps, int32_t* chosen, npbs_stream stream);

/* The same apply as cbs_apply for callers that cannot allocate device memory
 * (the paper has no counterpart; this is a deployment variant).  cbs_apply
 * allocates its spectrum scratch and batch plan through the context on first
 * use; an application whose memory manager has reserved the whole device for
 * its own pool, or latency-critical code that must not pay for (possibly
 * device-synchronising) cudaMalloc / cudaFree, cannot allow that.  This entry
 * point takes no context and allocates nothing: the scratch (2^20 complex64
 * elements, 8 MiB) and the plan live in static device arrays of the library.
 * The CUDA runtime places them on a device when it loads the library's module
 * there; under lazy module loading (the default) that is the first call on the
 * device, so make that call before the caller's own pool takes the device's
 * memory (or run with CUDA_MODULE_LOADING=EAGER); if they cannot be placed the
 * call returns NPBS_ERR_CUDA with a message.  The device then holds them until
 * the process exits.  Each call writes its plan on the device with a small
 * set-up kernel from its launch parameters, in stream order before the apply.
 * The caller still passes inputs and outputs (same meaning and layout as
 * cbs_apply) on the current device.  Limits: batch extent (max offset + nx*ny)
 * <= 2^20 elements, <= 64 instances, <= 8 distinct grid sides; larger batches
 * return NPBS_ERR_UNSUPPORTED_SIZE.  The first call on a device resolves the
 * static arrays' device addresses and sets kernel attributes; make that first
 * call before any stream capture.  All calls share the static arrays: calls that
 * overlap on the GPU (different streams or host threads) race; calls on one
 * stream are ordered.  err (nullable, errlen bytes) receives a one-line
 * message on failure.  Asynchronous on `stream`. */
npbs_status cbs_apply_static(const npbs_batch* batch, const void* V, const void* f, const void* x,
                             void* out, npbs_mode mode, double* norm2, npbs_stream stream,
                             char* err, int32_t errlen);

/* ---- solvers --------------------------------------------------------------
 * All solvers iterate in complex64 on a correction delta and fold it into the
 * solution u held in complex128 every refinement cycle, where the true
 * residual f - A u is recomputed in float64 (mixed-precision iterative
 * refinement; the transforms of that residual run in double-single
 * arithmetic, pairs of floats with about 48 significant bits, and its
 * pointwise terms and norms in float64).  Linear stationary iterations restarted from delta = 0 on the
 * correction equation A delta = f - A u produce the same iterates as the
 * uninterrupted iteration, so iteration counts are those of the method; the
 * float64 residual removes the float32 floor (about 1e-5 for complex64 CBS).
 * k2: DEVICE complex64 k(x)^2 of every instance (the problem data; the solver
 * forms V = k^2 - k0^2 - i eps from it with the batch's k0sq / eps, and uses
 * k^2 itself, exactly, in the float64 residual f - A u).
 * u: DEVICE complex128, initial guess on entry, solution on exit.
 * Converged instances are masked out of later launches.  Synchronise. */

/* Stationary CBS (Eq. CBS) to opts->rtol. */
npbs_status cbs_solve(npbs_ctx* ctx, const npbs_batch* batch, const void* k2, const void* f,
                      void* u, const npbs_solve_opts* opts, npbs_report* report,
                      npbs_stream stream);

/* Stationary NPBS (Eq. npbs_integral) with the network of `net` as M_theta:
 * u <- u + M(G(V u + f) - u), M(r) = s N([Re r/s, Im r/s, n]), s = rms(r).
 * n: DEVICE float32 refractive index (network input channel).  Divergence
 * guard: an instance whose float64 rTol did not decrease between two refresh
 * points continues with plain CBS steps (report->flags). */
npbs_status npbs_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch,
                       const void* k2, const void* f, const float* n, void* u,
                       const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream);

/* The Direct format (Eq. direct_iter), the baseline of Sec. 4: u <- u + M(f - A u)
 * with the network fed the unpreconditioned residual (scale wrapper as in
 * npbs_solve).  Same mixed-precision refinement, arguments and report as
 * npbs_solve; no CBS guard (this format has no Born residual to step with). */
npbs_status npbs_solve_direct(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch,
                              const void* k2, const void* f, const float* n, void* u,
                              const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream);

/* Restarted flexible GMRES on B u = G f (Eq. LS_discrete), restart length
 * `restart` (1..64), right preconditioner precond: 0 none, 1 `cbs_sweeps`
 * CBS Richardson sweeps, 2 the network of `net` (may be NULL unless precond = 2). */
npbs_status fgmres_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch,
                         const void* k2, const void* f, const float* n, void* u,
                         int32_t restart, int32_t precond, int32_t cbs_sweeps,
                         const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream);


/* ---- convection-diffusion-reaction (App. Full Derivations, CDR) ------------
 * The paper's CDR extension on the same periodic pseudospectral grid:
 *   A u  = -div(kappa grad u) + v . grad u + sigma u            (Eq. cdr_pde)
 *   L0   = -kappa0 Lap + v0 . grad + sigma0, G = L0^{-1}         (Eqs. cdr_L0, cdr_G_symbol)
 *   V    = L0 - A, so I - G V = G A and G(V u + f) - u = G(f - A u)  (Eqs. cdr_V, cdr_identity)
 * First derivatives are i xi on the mode set of the Helmholtz operators.
 * kappa, vx (along x, the row direction), vy, sigma: DEVICE float32 with the
 * batch layout; fields complex64.  Instances: square grids whose side is a
 * multiple of 16 and 2^a 3^b <= 1024; h > 0; the k0sq / eps fields of the
 * batch are ignored.  Background constants per instance (HOST array). */
typedef struct {
    double kappa0, v0x, v0y, sigma0;  /* kappa0 > 0 */
} npbs_cdr_consts;

/* The library's reading of the background constants, per instance: kappa0 and
 * sigma0 the midpoints of the ranges of kappa and sigma (so that the diffusion
 * and reaction parts of G V contract, as the midpoint k0^2 does for Helmholtz),
 * v0 the grid mean of v.  out: HOST [count].  Synchronises the stream. */
npbs_status npbs_cdr_background(npbs_ctx* ctx, const npbs_batch* batch, const float* kappa, const float* vx,
                                const float* vy, const float* sigma, npbs_cdr_consts* out, npbs_stream stream);

/* One CDR apply: mode RESIDUAL out = G(V x + f) - x = G(f - A x); OP_B out = G A x
 * (= x - G V x); TRUE_RESIDUAL out = f - A x; ADJ_B out = (G A)^* x = A^* G^* x
 * (G^* of symbol 1/conj(lambda0), A^* g = -div(kappa grad g + v g) + sigma g).
 * f may be NULL for OP_B and ADJ_B; out may alias x.  norm2 (nullable, DEVICE
 * double [count]) receives ||out||^2 per instance.  Asynchronous. */
npbs_status cdr_apply(npbs_ctx* ctx, const npbs_batch* batch, const npbs_cdr_consts* consts, const float* kappa,
                      const float* vx, const float* vy, const float* sigma, const void* f, const void* x, void* out,
                      npbs_mode mode, double* norm2, npbs_stream stream);

/* NPBS for CDR (the template of Eq. npbs_integral with the CDR operators):
 * u <- u + M(G(V u + f) - u), M the network `net` fed the coefficient field
 * `a` (DEVICE float32: the FNO's coef_channels planes of the batch extent one
 * after another, e.g. kappa, vx, vy, sigma; one plane for a U-Net), or the
 * identity when net is NULL (the Born series, which converges when
 * ||G V|| < 1).  u: DEVICE complex128, initial guess in, iterate out.  The
 * iteration runs in complex64 on the correction equation A delta = f - A u;
 * every opts->check_every iterations delta is folded into u and rTol =
 * ||f - A u|| / ||f|| is evaluated in float64 (so tolerances below the float32
 * floor of about 1e-5 are reached, with the iteration count of the
 * uninterrupted method).  Every instance iterates until all have passed or
 * opts->max_iter; an instance's u and report are those of its first passing
 * check.  Synchronises. */
npbs_status cdr_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const npbs_cdr_consts* consts,
                      const float* kappa, const float* vx, const float* vy, const float* sigma, const void* f,
                      const float* a, void* u, const npbs_solve_opts* opts, npbs_report* report, npbs_stream stream);

/* The metric-matched training step for CDR (Eq. cdr_bs_loss, the template of
 * npbs_train_step with (G, A, V) the CDR operators): r_0 = G(V u + f) - u of the
 * snapshots u_snap, r_{k+1} = r_k - (I - G V) M(r_k), loss = mean_j (1/U)
 * sum_k ||r_k||^2 / ||r_0||^2, gradients by the CDR adjoint and the network
 * backward, one AdamW update.  a: the network's coefficient field, laid out
 * as for cdr_solve.
 * Synchronises the stream once (to read the loss). */
npbs_status cdr_train_step(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const npbs_cdr_consts* consts,
                           const float* kappa, const float* vx, const float* vy, const float* sigma, const void* f,
                           const float* a, const void* u_snap, int32_t unroll, float lr, float weight_decay,
                           float* loss_host, npbs_stream stream);

/* ---- the learned correction M_theta (App. Experimental Setup, U-Net) -------
 * M(r; n) = s N([Re r / s, Im r / s, n]), s = ||r||_2 / sqrt(nx ny) per
 * instance, N a 4-level U-Net (32/64/128/256 channels, two 3x3 conv + GELU per
 * level, 2x2 average pooling, nearest x2 upsampling + 3x3 conv + GELU,
 * concatenated skips, bias-free 1x1 head to 2 channels), BF16 weights and
 * activations with FP32 accumulation on the tensor cores.  Grid sides must be
 * multiples of 8.  Parameters are exchanged in the canonical order: for each of
 * the 17 convolutions (enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, enc3a, enc3b,
 * up2, dec2a, dec2b, up1, dec1a, dec1b, up0, dec0a, dec0b) a float32 weight
 * [Cout][Cin][3][3] then a bias [Cout]; then the head weight [2][32]. */

/* Total number of parameters of the U-Net in the canonical order. */
int64_t npbs_net_num_params(void);
/* Parameters of a network of either kind in its canonical order (U-Net or
 * FNO); -1 for NULL. */
int64_t npbs_net_param_count(const npbs_net* net);

/* The FNO map (App. Architectural Instantiations, Eqs. fno_impl, fno_lift,
 * fno_proj, lfl, nlfl), the paper's primary backbone, as a network of the
 * same object type: every entry taking an npbs_net (forward, backward, AdamW,
 * save / load, npbs_solve, fgmres_solve, the training steps) accepts it.
 *   M(r; a) = P( LFL_f[ NLFL_L(...NLFL_1(Phi(a))) * LFL_r(Psi(r)) ] ),
 *   Phi(a) = W_a LayerNorm(a) + b_a, Psi(r) = W_r [Re r, Im r], P(z) = W_p z,
 *   LFL(x) = irfft2(W^F * R(rfft2(x))) + W^loc x (+ b), NLFL = GELU(LFL);
 * a is the network's coefficient field (the `n` argument of the entries):
 * coef_channels planes one after another, plane c starting at element
 * c * E with E = max_j (offset_j + nx_j ny_j) the batch extent (1 plane for
 * Helmholtz; the CDR problems pass kappa, vx, vy, sigma), each plane
 * LayerNorm-ed over the grid of each instance.
 * M is linear in r (no bias on the residual path, no scale wrapper).  The
 * NLFL and fusion layers keep the modes with min(ky, N - ky) < modes and
 * kx < modes of the half plane, the residual layer all of them (N/2 + 1
 * columns).  The paper's configuration is width 25, modes 45, layers 3.  The
 * network is tied to one grid: every instance must be n x n.  n: even,
 * 2^a 3^b, 4..1024; width 1..32; modes 1..n/2+1; layers 0..8;
 * coef_channels 1..32.  Float32
 * throughout.  Canonical parameter order: lift_a.w [C][coef], lift_a.b [C]; per
 * layer spec [C][C][Ky][Kx][2 = re, im], loc.w [C out][C in], loc.b [C];
 * lift_r.w [C][2]; spec_r [C][C][n][n/2+1][2]; loc_r.w [C][C];
 * spec_f [C][C][Ky][Kx][2]; loc_f.w [C][C]; proj.w [2][C].  Seeded initial
 * weights. */
npbs_status npbs_net_create_fno(npbs_net** out, int device, int n, int width, int modes, int layers,
                                int coef_channels, uint64_t seed);

/* Switches the FNO's identity skip: on, M(r) = r + N(r) with N the network
 * above, so that zero weights give the Born series (NPBS leaves the form of
 * M open, Eq. npbs_integral); turning it on zeroes the projection weights,
 * so the network starts as the identity (call it before training or loading
 * parameters).  Saved with the network.  NPBS_ERR_UNSUPPORTED_SIZE for a
 * U-Net. */
npbs_status npbs_net_fno_set_skip(npbs_net* net, int32_t on);
/* Create a network on `device` with seeded He-normal weights. */
npbs_status npbs_net_create(npbs_net** out, int device, uint64_t seed);
npbs_status npbs_net_destroy(npbs_net* net);
/* Copy parameters / accumulated gradients in the canonical order (HOST float[n],
 * n = npbs_net_num_params()).  Synchronous. */
npbs_status npbs_net_set_params(npbs_net* net, const float* host, int64_t n);
npbs_status npbs_net_get_params(const npbs_net* net, float* host, int64_t n);
npbs_status npbs_net_get_grads(const npbs_net* net, float* host, int64_t n);
npbs_status npbs_net_zero_grad(npbs_net* net, npbs_stream stream);
/* One AdamW update (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay) with
 * the accumulated gradients. */
npbs_status npbs_net_adamw(npbs_ctx* ctx, npbs_net* net, float lr, float weight_decay, npbs_stream stream);
/* Checkpoint: parameters, AdamW moments and step count to a binary file. */
npbs_status npbs_net_save(const npbs_net* net, const char* path);
npbs_status npbs_net_load(npbs_net** out, int device, const char* path);

/* c_out = M(r; n) per instance (Eq. npbs_integral, learned map).  r, c_out:
 * DEVICE complex64; n: DEVICE float32. */
npbs_status npbs_net_forward(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const void* r,
                             const float* n, void* c_out, npbs_stream stream);
/* Hand-written adjoint of c = M(r; n): accumulates d<grad_c, c>/dtheta into the
 * network gradients and writes grad_r = (J_M(r))^* grad_c (gradients of real
 * losses in the convention dL/dRe + i dL/dIm).  Recomputes the forward. */
npbs_status npbs_net_backward(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* r,
                              const float* n, const void* grad_c, void* grad_r, npbs_stream stream);

/* Metric-matched training step (Eq. L_bs_Reta_integral, squared, over `unroll`
 * NPBS steps from the snapshots u_snap): r_0 = G(V u + f) - u,
 * r_{k+1} = r_k - (I - G V) M(r_k), loss = mean_j (1/U) sum_k ||r_k||^2/||r_0||^2;
 * gradients by the adjoint apply and network backward with activation
 * checkpointing (only r_0..r_U stored), then one AdamW update.  u_snap:
 * DEVICE complex64.  loss_host receives the loss before the update.
 * Synchronises the stream once (to read the loss). */
npbs_status npbs_train_step(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* V,
                            const void* f, const float* n, const void* u_snap, int32_t unroll, float lr,
                            float weight_decay, float* loss_host, npbs_stream stream);

/* Training objectives of Sec. 4 (the format/loss ablation). */
typedef enum {
    NPBS_LOSS_BS_RETA = 0, /* Eq. L_bs_Reta_integral: NPBS input G r, residual measured with G (npbs_train_step) */
    NPBS_LOSS_BS_L2 = 1,   /* Eq. L_bs_l2: NPBS input G r, Euclidean residual of A */
    NPBS_LOSS_DIR = 2      /* Eq. L_dir: Direct-format input r = f - A u, Euclidean residual */
} npbs_loss;

/* npbs_train_step with a choice of objective, each in the squared unrolled
 * form: for BS_L2 and DIR the state is the true residual t_0 = f - A u_snap,
 * x_k = G t_k (BS_L2) or t_k (DIR), t_{k+1} = t_k - A M(x_k), loss =
 * mean_j (1/U) sum_k ||t_k||^2/||t_0||^2, with the adjoints A^* and G^*
 * (A and G are complex symmetric: A^* y = conj(A conj(y))).  BS_RETA is
 * npbs_train_step.  Other arguments as there; an unknown kind returns
 * NPBS_ERR_INVALID_ARG. */
npbs_status npbs_train_step_loss(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const void* V,
                                 const void* f, const float* n, const void* u_snap, int32_t unroll,
                                 npbs_loss kind, float lr, float weight_decay, float* loss_host,
                                 npbs_stream stream);

/* The CDR counterparts of the format/loss comparison (the CDR column of the
 * comparison across other PDEs): cdr_train_step with a choice of objective
 * (BS_L2 and DIR use the explicit adjoints A^* g = -div(kappa grad g + v g)
 * + sigma g and G^* of symbol 1/conj(lambda0), since convection makes A not
 * complex symmetric), and the Direct format u <- u + M(f - A u) with the
 * float64 stopping test of cdr_solve (net required).  Arguments as in
 * cdr_train_step and cdr_solve. */
npbs_status cdr_train_step_loss(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch,
                                const npbs_cdr_consts* consts, const float* kappa, const float* vx, const float* vy,
                                const float* sigma, const void* f, const float* a, const void* u_snap,
                                int32_t unroll, npbs_loss kind, float lr, float weight_decay, float* loss_host,
                                npbs_stream stream);
npbs_status cdr_solve_direct(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch,
                             const npbs_cdr_consts* consts, const float* kappa, const float* vx, const float* vy,
                             const float* sigma, const void* f, const float* a, void* u, const npbs_solve_opts* opts,
                             npbs_report* report, npbs_stream stream);


/* ---- Newton-Born linearisation with a DST-I Green operator ------------------
 * (App. Full Derivations, Nonlinear PDE via Newton-Born Linearization; Eqs.
 * nonlinear_residual, newton_linear_system, newton_ref, newton_vm,
 * newton_born_identity, newton_inner_iter; App. Verification, Newton linear
 * systems; Sec. 5.2):
 *   F(u) = L_D u - u^2 - f on the N x N interior unknowns of [0, 1]^2,
 *          homogeneous Dirichlet, L_D the five-point negative Laplacian / h^2,
 *          h = 1/(N + 1)  (the batch's h is ignored)
 *   J = L_D - 2 diag(u_m), J0 = L_D + c I (c = alpha - 2 mean(u_m)),
 *   V = J0 - J = c + 2 u_m, G = J0^{-1} by the 2D DST-I, I - G V = G J.
 * Instances: square, N a multiple of 4 in 8..96 (else UNSUPPORTED_SIZE);
 * offsets multiples of 32.  Fields use the batch layout. */

/* One apply at linearisation points u (DEVICE float32) with shifts c (HOST
 * double [count]): RESIDUAL out = G(r - J x); OP_B out = G J x = (I - G V) x;
 * TRUE_RESIDUAL out = r - J x (r nullable: -J x); ADJ_B out = (G J)^* x =
 * J G x (J and G are real symmetric).  r, x, out: DEVICE complex64 (out may
 * alias x); norm2 (nullable, DEVICE double [count]) receives ||out||^2.
 * Side 64 runs its sine-matrix products on the tensor cores (TF32 with a
 * three-term split, float32-class accuracy); other sides, TRUE_RESIDUAL and
 * the environment setting NPBS_NEWTON_TC=0 use the CUDA-core kernel.  A
 * bounded wait of the tensor-core kernel that gives up is reported by
 * npbs_device_status.  Asynchronous. */
npbs_status newton_apply(npbs_ctx* ctx, const npbs_batch* batch, const double* shift, const float* u,
                         const void* r, const void* x, void* out, npbs_mode mode, double* norm2,
                         npbs_stream stream);

typedef struct {
    double tol;             /* outer: ||F(u)|| / ||f|| <= tol */
    int32_t max_steps;      /* Newton steps */
    double inner_rtol;      /* inner: ||r - J delta|| / ||r|| <= inner_rtol (1e-4 in the paper) */
    int32_t inner_max_iter; /* inner iterations per Newton step */
    int32_t check_every;    /* inner iterations between float64 checks */
    int32_t direct_format;  /* 0: NPBS (network input G(r - J delta)); 1: the Direct format (input
                               r - J delta, Eq. direct_iter's template; net required) */
} npbs_newton_opts;

typedef struct {            /* HOST arrays [count], each nullable */
    int32_t* steps;         /* Newton steps taken */
    int32_t* inner_iters;   /* inner iterations summed over the steps */
    double* residual;       /* final ||F(u)|| / ||f|| (float64) */
    npbs_status* status;    /* OK, NOT_CONVERGED or ERR_NONFINITE */
} npbs_newton_report;

/* Newton's method with inner Born (net NULL) or NPBS solves (Eq.
 * newton_inner_iter: delta <- delta + M(G(r - J delta)), M the network fed the
 * linearisation point u_m as its coefficient channel).  f, u: DEVICE float64
 * (u: initial guess in, solution out).  Each Newton step linearises at u in
 * float64 (r = -F(u), c = alpha - 2 mean(u)); the inner iteration runs in
 * complex64 on the correction of delta, which is folded into a complex128
 * delta at every check where r - J delta is evaluated in float64; an instance
 * leaves the inner loop at its first passing check (or inner_max_iter) and u
 * += Re delta.  Instances stop at ||F(u)|| / ||f|| <= tol (u is left at that
 * iterate) or after max_steps.  Synchronises. */
npbs_status newton_solve(npbs_ctx* ctx, const npbs_net* net, const npbs_batch* batch, const double* f, double* u,
                         double alpha, const npbs_newton_opts* opts, npbs_newton_report* report,
                         npbs_stream stream);

/* One linearisation per instance at u (DEVICE float64): shift_out (HOST double
 * [count]) = alpha - 2 mean(u), u32_out (DEVICE float32) = u rounded, r_out
 * (DEVICE complex64) = -F(u) = f - L_D u + u^2 evaluated in float64 and
 * rounded: the state (u_m, c_m, r_m) of a Newton trajectory for
 * newton_apply and newton_train_step_loss.  Synchronises. */
npbs_status newton_linearise(npbs_ctx* ctx, const npbs_batch* batch, const double* u, const double* f, double alpha,
                             double* shift_out, float* u32_out, void* r_out, npbs_stream stream);

/* The training step for the Newton inner systems (Eq. nl_bs_loss for BS_RETA,
 * the template of npbs_train_step_loss with (G, J, V) of each state): u
 * (DEVICE float32) the linearisation points and network coefficient channel,
 * shift (HOST double [count]) their c, r (DEVICE complex64) the right-hand
 * sides -F(u_m), d_snap (DEVICE complex64) the inner iterates the unrolled
 * loss starts from (r_0 = G(r - J d)).  BS_L2 and DIR use J^* = J, G^* = G.
 * Synchronises once (to read the loss). */
npbs_status newton_train_step_loss(npbs_ctx* ctx, npbs_net* net, const npbs_batch* batch, const double* shift,
                                   const float* u, const void* r, const void* d_snap, int32_t unroll,
                                   npbs_loss kind, float lr, float weight_decay, float* loss_host,
                                   npbs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* NPBS_H */
