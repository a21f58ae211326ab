/*
 * mca.h — C ABI of the GB300 steady-state memristor-crossbar (MCA) solver.
 *
 * The library computes the steady state of a memristor crossbar array: two resistive
 * wire grids (top rows = word lines, bottom columns = bit lines) coupled at every cross
 * point (i, j) by a memristor, driven at the left end of every top row.  It solves the
 * modified-nodal-analysis system of Xie et al., "A Fast Method for Steady-State
 * Memristor Crossbar Array Circuit Simulation" (arXiv 2109.07929):
 *
 *   Section 2, eq. (MNA) / eq. (F):  G_t V_t + I(V_t - V_b) - Y_t = 0,
 *                                    G_b V_b - I(V_t - V_b) - Y_b = 0,
 *   eqs. (Gt), (Gb):                 G_t = I (x) G_r,  G_b = G_c (x) I,
 *   eq. (Newton3), eq. (J):          Newton's method on F with the MNA Jacobian,
 *   Section 3, eqs. (P), (block), (M):  each Newton system is solved by GMRES,
 *                                    preconditioned with P = [[G_t + a1 I, -a1 I],
 *                                    [-a2 I, G_b + a2 I]], a1 = a2 = mean device
 *                                    conductance, inverted through the Kronecker
 *                                    structure of G_t and G_b.
 *
 * Device model: i = (g_ij / b) sinh(b * dV) (b = 0 selects the linear device i = g dV).
 *
 * Conventions for every array argument:
 *   - node voltages are row-major m x n (cell (i, j) at i*n + j), one block per input
 *     vector: v_top[v][i][j], v_bot[v][i][j];
 *   - input vectors are v_in[v][i] (volts at the left end of top row i);
 *   - output currents are i_out[v][j] (amperes into the sense amplifier of column j).
 *   - pointers may be host or device memory (CUDA unified addressing tells them apart);
 *     the caller owns every buffer it passes in and may free it when the call returns.
 *
 * Errors: every int-returning call returns MCA_OK (0) or a negative MCA_ERR_* code and
 * never throws.  mca_last_error_message() gives a human-readable detail of the most
 * recent failure in the calling thread.  One handle must not be used from two threads at
 * the same time.
 */
#ifndef MCA_H_
#define MCA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------------- */
#define MCA_OK 0
#define MCA_ERR_INVALID_ARG (-1)   /* bad size, NULL pointer, non-positive conductance  */
#define MCA_ERR_CUDA (-2)          /* a CUDA runtime call failed                        */
#define MCA_ERR_NONFINITE (-3)     /* NaN/Inf in the inputs or in the residual          */
#define MCA_ERR_NOT_CONVERGED (-4) /* Newton stopped at max_newton; outputs still valid */
#define MCA_ERR_TIMEOUT (-5)       /* a bounded device-side wait gave up                */
#define MCA_ERR_OOM (-6)           /* device memory allocation failed                   */
#define MCA_ERR_UNSUPPORTED (-7)   /* precision mode not available on this device       */

/* ---- precision of the preconditioner apply (Section 3.2) -------------------------- */
#define MCA_PREC_FP64 0        /* all four eigenbasis transforms in FP64 (CUDA cores)     */
#define MCA_PREC_BF16 1        /* all four transforms on tcgen05 tensor cores, BF16 in,
                                  FP32 accumulate                                        */
#define MCA_PREC_BF16_SPLIT 2  /* forward transforms BF16; back transforms with the
                                  eigenvectors split as hi+lo BF16 pairs: transform 3
                                  Y_hat (hi) x Q_r (hi+lo), 2 tensor-core products;
                                  transform 4 E (hi+lo) x Q_c (hi+lo), 3 products
                                  (hi*hi + lo*hi + hi*lo); FP32 accumulate               */
#define MCA_PREC_MHAT 3        /* the paper's own evaluation: eq. (block) with the
                                  approximate Schur complement M_hat of eq. (Mhat), applied
                                  by tridiagonal solves (eq. 2matrix4), FP64              */
#define MCA_PREC_JACOBI 4      /* comparison preconditioner of Table 1: diag(J)^-1      */
#define MCA_PREC_NONE 5        /* no preconditioner (Table 1, "before preconditioned")  */

typedef struct mca_params {
  int32_t rows;              /* m >= 1: number of top-layer rows (word lines)            */
  int32_t cols;              /* n >= 1: number of bottom-layer columns (bit lines)       */
  double g_wire_top;         /* S, top-layer segment conductance (Section 2)             */
  double g_wire_bot;         /* S, bottom-layer segment conductance                      */
  double g_src;              /* S, driver conductance at the left end of each top row    */
  double g_term_top_right;   /* S, right end of each top row to ground                   */
  double g_term_bot_top;     /* S, row-0 end of each bottom column to ground             */
  double g_sense;            /* S, row-(m-1) end of each bottom column to virtual ground */
  double b;                  /* 1/V, memristor sinh nonlinearity (0 = linear)            */
  int32_t precision;         /* MCA_PREC_*                                               */
  int32_t gmres_restart;     /* 1..30 (flexible GMRES restart length)                    */
  int32_t max_newton;        /* Newton iteration limit (>= 1)                            */
  int32_t max_batch;         /* input vectors solved together per pass (>= 1)            */
  double newton_rtol;        /* stop when ||F||_2 / ||Y||_2 <= newton_rtol               */
  double eta0;               /* relative tolerance of the first linear solve             */
  double eta_max;            /* upper bound of later forcing terms                       */
  int32_t flags;             /* MCA_FLAG_* bit set                                       */
  int32_t device_model;      /* MCA_DEVICE_* (memristor I-V law)                         */
  double neg_ratio;          /* MCA_DEVICE_YAKOPCIC: current amplitude for dV < 0 over the
                                one for dV >= 0 (a2/a1, finite and > 0); else ignored    */
} mca_params;

/* ---- memristor I-V law (Section 2; Section 4 uses Yakopcic's model at programmed
 * states).  g is each device's small-signal conductance (the conductance map), dV the
 * top-minus-bottom node voltage:
 *   MCA_DEVICE_SINH      i = (g/b) sinh(b dV)   (b = 0: i = g dV)
 *   MCA_DEVICE_YAKOPCIC  the same for dV >= 0 and neg_ratio times it for dV < 0: the
 *                        Yakopcic form a1 x sinh(b V) / a2 x sinh(b V) with the state x
 *                        fixed, g = a1 x b and neg_ratio = a2 / a1.  The Jacobian uses the
 *                        derivative on the side of dV the device is on. */
#define MCA_DEVICE_SINH 0
#define MCA_DEVICE_YAKOPCIC 1

/* ---- flags --------------------------------------------------------------------------- */
#define MCA_FLAG_GRAPHS 1      /* replay each GMRES iteration as a captured CUDA graph      */
#define MCA_FLAG_AUTOTUNE 2    /* time the tensor-core tile widths at create, keep the best */
#define MCA_FLAG_PAIR_GEMM 4   /* the two-SM form of the persistent GEMM (CTA pairs,        */
                               /* cta_group::2 MMAs, 256 x 256 tiles) for transforms 1, 3    */
                               /* and 4 where rows and columns are multiples of 256: with    */
                               /* AUTOTUNE one more timed candidate, without it always used  */

typedef struct mca_stats {
  int32_t status;            /* MCA_OK, MCA_ERR_NOT_CONVERGED or MCA_ERR_NONFINITE       */
  int32_t newton_iters;      /* Jacobian solves performed                                */
  int32_t gmres_iters;       /* GMRES iterations summed over the Newton steps            */
  int32_t fallback;          /* mca_solve_from: 1 when the guess was rejected            */
  double rel_residual;       /* ||F||_2 / ||Y||_2 at the returned voltages               */
  double kcl_rel_error;      /* |sum I_in - sum I_out - sum leaks| / sum |I_in|          */
} mca_stats;

typedef struct mca_handle mca_handle;

/* Fill *p with the defaults: 1 S wires, 10 ohm driver and sense, 1 kohm terminations,
 * b = 2, MCA_PREC_BF16_SPLIT, restart 30, max_newton 20, max_batch 4, newton_rtol 1e-8,
 * eta0 1e-3, eta_max 1e-2, flags MCA_FLAG_GRAPHS | MCA_FLAG_AUTOTUNE | MCA_FLAG_PAIR_GEMM.
 * rows/cols are left at 0 and must be set. */
void mca_default_params(mca_params* p);

/* Create a solver for one crossbar.
 *   p     : circuit and solver parameters (copied).
 *   g_map : m*n memristor conductances g_ij in siemens, row-major, host or device,
 *           every entry > 0 and finite (copied; the caller keeps ownership).
 *   out   : receives the handle.
 * Builds the 1-D wire operators G_r (n x n) and G_c (m x m) of eq. (G) with the end
 * terminations, and their FP64 eigendecompositions on the GPU (separability of eqs.
 * (Gt)/(Gb), Section 3.1).  Allocates the device workspace for max_batch vectors.
 * Returns MCA_ERR_INVALID_ARG for bad sizes or values, MCA_ERR_OOM, MCA_ERR_CUDA. */
int mca_create(const mca_params* p, const double* g_map, mca_handle** out);

/* Solve the steady state for nvec input vectors (Newton, eq. (Newton3), from V = 0).
 *   v_in  : nvec*m input voltages, row vector per input (host or device).
 *   v_top : nvec*m*n top-layer node voltages out, or NULL.
 *   v_bot : nvec*m*n bottom-layer node voltages out, or NULL.
 *   i_out : nvec*n sensed column currents g_sense * V_b[m-1, j] out, or NULL.
 *   stats : nvec entries out, or NULL.
 *   stream: cudaStream_t to run on (NULL = the handle's own stream, ordered with the
 *           legacy default stream).  The call returns after the results are written.
 * More than max_batch vectors run as passes of max_batch; the output copies of a pass run
 * on an internal stream while the next pass computes (the handle double-buffers its state),
 * so a call over several batches hides most of the device-to-host traffic.
 * Returns MCA_OK when every vector met newton_rtol, else the first failing status
 * (MCA_ERR_NOT_CONVERGED / MCA_ERR_NONFINITE; outputs are still written), or
 * MCA_ERR_INVALID_ARG / MCA_ERR_CUDA / MCA_ERR_TIMEOUT. */
int mca_solve(mca_handle* h, const double* v_in, int32_t nvec, double* v_top, double* v_bot,
              double* i_out, mca_stats* stats, void* stream);

/* Several crossbars of one shape and wiring in one handle (the statistical-
 * characterisation workload): n_maps conductance maps share the eigenbasis and the
 * tensor-core operands, and every input vector picks its map, so vectors of different
 * crossbars run in the same batched kernels.
 *   g_maps : n_maps * m*n conductances (host or device), map k at k*m*n.
 * mca_create(p, g, out) equals mca_create_multi(p, g, 1, out). */
int mca_create_multi(const mca_params* p, const double* g_maps, int32_t n_maps,
                     mca_handle** out);

/* mca_solve for a handle with several maps: map_index (host, nvec entries, each in
 * 0..n_maps-1) selects vector v's crossbar; NULL means map 0 for every vector.  Output
 * layouts as in mca_solve. */
int mca_solve_multi(mca_handle* h, const double* v_in, const int32_t* map_index, int32_t nvec,
                    double* v_top, double* v_bot, double* i_out, mca_stats* stats,
                    void* stream);

/* Solve nh handles concurrently: worker k of n_threads host threads takes handles in turn
 * and runs mca_solve_multi on a stream of its own, so crossbars of different shapes
 * overlap on the GPU.  Arrays are indexed by handle; entries of the output arrays may be
 * NULL.  Returns MCA_OK or the first failing status. */
int mca_solve_many(mca_handle* const* hs, int32_t nh, const double* const* v_in,
                   const int32_t* const* map_index, const int32_t* nvec,
                   double* const* v_top, double* const* v_bot, double* const* i_out,
                   mca_stats* const* stats, int32_t n_threads);

/* ---- persistent batched solve: one launch for many independent solves ---------------
 * A batch object binds handles of several shapes (each MCA_PREC_BF16_SPLIT, all on one
 * device, all with the same device model) to one persistent kernel: every CTA runs the
 * whole Newton / flexible-GMRES solve of one (crossbar, input vector) item (eqs. (F), (J),
 * (Newton3), the preconditioner of eq. (P) in the Kronecker eigenbasis of Section 3.2 on
 * the tensor cores) and then takes the next item from a device-side queue, largest items
 * first, until the batch is done.  Each handle's own settings (wires, b, newton_rtol, eta0,
 * eta_max, max_newton, restart) apply to its items; every Newton residual is the FP64 one.
 * The batch owns one scratch slot per CTA sized for the largest shape and restart:
 * about 8 * 2mn * (2 * restart + 4) bytes each, 2 CTAs per SM by default. */
typedef struct mca_batch mca_batch;

typedef struct mca_item {
  int32_t handle;            /* index into the handles given to mca_batch_create          */
  int32_t map;               /* conductance map of that handle (0..n_maps-1)              */
  const double* v_in;        /* device: m input voltages                                  */
  double* v_top;             /* device: m*n top-layer voltages out, or NULL               */
  double* v_bot;             /* device: m*n bottom-layer voltages out, or NULL            */
  double* i_out;             /* device: n sensed column currents out, or NULL             */
} mca_item;

/* Create a batch over nh handles (the handles must outlive it; their conductance maps are
 * read at solve time).  max_ctas: CTAs (= scratch slots) of a launch, 0 for 2 per SM.
 * Returns MCA_ERR_INVALID_ARG, MCA_ERR_UNSUPPORTED (a handle not in MCA_PREC_BF16_SPLIT),
 * MCA_ERR_OOM or MCA_ERR_CUDA. */
int mca_batch_create(mca_handle* const* hs, int32_t nh, int32_t max_ctas, mca_batch** out);

/* Solve n items in one kernel launch.  items (host array) point at device buffers; stats
 * (host, n entries, or NULL) in item order.  The call returns after the results are
 * written.  Returns MCA_OK when every item met its newton_rtol, else the first failing
 * status (outputs still written), MCA_ERR_INVALID_ARG for an index out of range or a NULL
 * v_in, MCA_ERR_TIMEOUT when a bounded device wait gave up, MCA_ERR_OOM, MCA_ERR_CUDA. */
int mca_batch_solve(mca_batch* b, const mca_item* items, int32_t n, mca_stats* stats,
                    void* stream);

/* The persistent kernel's preconditioner alone (for testing): for each item, v_top / v_bot
 * (device, m*n each) hold r on entry and z = P^-1 r on return, with a1 = a2 = a[k] (host,
 * n entries) in eq. (P); v_in and i_out are ignored. */
int mca_batch_precond(mca_batch* b, const mca_item* items, const double* a, int32_t n,
                      void* stream);

/* Per-phase timing of the persistent kernel.  mca_batch_profile(b, 1) zeroes and enables
 * it (0 disables); mca_batch_profile_read fills ms[MCA_BATCH_PHASES] with the time each
 * phase took, summed over the CTAs (CTA-milliseconds) since it was enabled, in the order
 * residual, transform 1, transform 2 (with the modes), transform 3, transform 4, Jacobian
 * apply + dots, update pass, second Gram-Schmidt pass, least squares + solution update,
 * other (queue, setup, outputs). */
#define MCA_BATCH_PHASES 10
int mca_batch_profile(mca_batch* b, int32_t enable);
int mca_batch_profile_read(mca_batch* b, double* ms);

void mca_batch_destroy(mca_batch* b);

/* Reprogram the crossbars of a handle: replace its n_maps conductance maps (host or
 * device, n_maps*m*n, every entry finite and > 0) without redoing the eigen setup,
 * which depends only on the wires and terminations. */
int mca_set_conductances(mca_handle* h, const double* g_maps);

/* Newton from a caller's initial guess instead of V = 0 (warm start).
 *   guess    : device, nvec * 2*m*n states [V_t ; V_b] (e.g. V_lin + the CNN's correction).
 *   fallback : device, nvec * 2*m*n states, or NULL for V = 0.
 * The residual of the guess and of the fallback state are evaluated; a guess is rejected
 * (stats.fallback = 1) when its residual is not finite or not smaller than the
 * fallback's (||F(guess)|| >= ||F(fallback)||, with ||F(0)|| = ||Y|| for NULL), and that
 * vector starts from the fallback state instead.  The Newton solve is the judge of the
 * guess: the returned voltages meet newton_rtol either way, and stats.newton_iters counts
 * the steps taken from the starting state.  Other arguments as in mca_solve_multi. */
int mca_solve_from(mca_handle* h, const double* v_in, const double* guess,
                   const double* fallback, const int32_t* map_index, int32_t nvec,
                   double* v_top, double* v_bot, double* i_out, mca_stats* stats, void* stream);

/* ---- learned warm start: the network's kernels (not part of the paper) -------------
 * The network maps a crossbar's conductances, its input vector and the state V_lin after
 * the first Newton step to the correction V* - V_lin.  Activations and gradients are NHWC
 * BF16 device tensors with 32 channels ([n][y][x][c], uint16_t bit patterns, channels
 * beyond a layer's count zero); FP32 master weights w[cout][cin][K][K] live with the
 * optimiser and mca_cnn_prep_weights turns them into the BF16 operand tiles.  A layer is
 * a K x K convolution (K odd, <= 15) with dilation d and zero padding d (K - 1) / 2
 * (output size = input size), bias and act (0 none, 1 leaky ReLU with slope 0.1).  The
 * convolutions run on the tcgen05 tensor cores (BF16 operands, FP32 accumulation).  All
 * calls only enqueue work on the stream; the caller owns every buffer.  Returns
 * MCA_ERR_INVALID_ARG for bad sizes or NULL buffers. */

/* Convolution as an implicit GEMM over 128-pixel row tiles.
 *   x       : NHWC32, n x h x w pixels.
 *   wt      : BF16 tiles [K*K][cout_mma][32] (forward) or [K*K][32][32] (backward data),
 *             from mca_cnn_prep_weights.
 *   cout_mma: 16 or 32 (32 for backward); cout <= cout_mma channels are written.
 *   backward = 0: out = act(conv(x) + bias) (bias may be NULL);
 *   backward = 1: x is the output gradient dL/dz of a layer, wt its backward tile, and
 *             out = dL/dx, times act'(y_prev) when act = 1 (y_prev: NHWC32 output of the
 *             layer below, i.e. the layer's input), the gradient dL/dz of that layer.
 *   out     : NHWC32 BF16 output (may be NULL); out32: [n][h][w][cout] FP32 (may be NULL). */
int mca_cnn_conv(const uint16_t* x, int32_t n, int32_t h, int32_t w, const uint16_t* wt,
                 int32_t ksize, int32_t dilation, int32_t cout_mma, int32_t cout,
                 const float* bias, int32_t act, int32_t backward, const uint16_t* y_prev,
                 uint16_t* out, float* out32, void* stream);

/* Floats of scratch mca_cnn_conv_wgrad needs for n x h x w pixels and K x K kernels
 * (-1 for bad sizes). */
int64_t mca_cnn_wgrad_scratch(int32_t n, int32_t h, int32_t w, int32_t ksize);

/* Parameter gradients of a layer from its input x and output gradient gz (both NHWC32):
 * gw[cout][cin][K][K] = sum_p gz[p][co] x[p + d (ky - r, kx - r)][ci] (FP32, written), and
 * gb[cout] = sum_p gz[p][co] (may be NULL).  scratch: mca_cnn_wgrad_scratch floats. */
int mca_cnn_conv_wgrad(const uint16_t* x, const uint16_t* gz, int32_t n, int32_t h, int32_t w,
                       int32_t ksize, int32_t dilation, int32_t cin, int32_t cout,
                       float* scratch, float* gw, float* gb, void* stream);

/* BF16 operand tiles of one layer from its FP32 master weights w[cout][cin][K][K]:
 * wf[K*K][cout_mma][32] = w[co][ci][t] (forward; may be NULL) and wb[K*K][32][32] =
 * w[co][ci][K*K - 1 - t] at [t][ci][co] (backward data: flipped taps; may be NULL). */
int mca_cnn_prep_weights(const float* w, int32_t cout, int32_t cin, int32_t ksize,
                         int32_t cout_mma, uint16_t* wf, uint16_t* wb, void* stream);

/* Network input x (NHWC32, nvec x m x n) of nvec vectors: channel 0 = log10(g) + 5,
 * 1 = V_in[i] / vscale along row i, 2 = V_lin,t / vscale, 3 = V_lin,b * bscale / vscale.
 *   g_maps: device FP64 maps (m*n each); map_index: device int32 per vector (NULL: map 0);
 *   v_in: device nvec * m; vlin_t, vlin_b: device nvec * m*n voltages of each layer (the
 *   layout of mca_solve's v_top and v_bot). */
int mca_cnn_features(const double* g_maps, const int32_t* map_index, const double* v_in,
                     const double* vlin_t, const double* vlin_b, int32_t nvec, int32_t m,
                     int32_t n, float vscale, float bscale, uint16_t* x, void* stream);

/* Training target target[v][node][2] = (V* - V_lin) * (dscale_t, dscale_b) (FP32), from
 * the two layers of V* and of V_lin (nvec * m*n each). */
int mca_cnn_target(const double* vstar_t, const double* vstar_b, const double* vlin_t,
                   const double* vlin_b, int32_t nvec, int32_t m, int32_t n, float dscale_t,
                   float dscale_b, float* target, void* stream);

/* Warm-start state guess = V_lin + pred / (dscale_t, dscale_b) as FP64 states [V_t ; V_b]
 * (nvec * 2*m*n) from the network's FP32 output pred[v][node][2]; pred = NULL writes V_lin
 * itself (the fallback state of mca_solve_from). */
int mca_cnn_guess(const float* pred, const double* vlin_t, const double* vlin_b, int32_t nvec,
                  int32_t m, int32_t n, float dscale_t, float dscale_b, double* guess,
                  void* stream);

/* Mean squared error of pred against target over npix pixels x 2 channels (loss: device,
 * 1 float; part: 256 floats) and its gradient gz = 2 (pred - target) / (2 npix) as NHWC32
 * BF16 (may be NULL). */
int mca_cnn_loss(const float* pred, const float* target, int64_t npix, uint16_t* gz,
                 float* part, float* loss, void* stream);

/* One Adam step (bias-corrected, step >= 1) on FP32 master weights w. */
int mca_cnn_adam(float* w, const float* g, float* m1, float* m2, int64_t count, float lr,
                 float beta1, float beta2, float eps, int32_t step, void* stream);

/* Synchronise the stream and report whether a bounded wait of a network kernel expired
 * since the last check (MCA_ERR_TIMEOUT, flag cleared) or MCA_OK. */
int mca_cnn_check(void* stream);

/* Release the handle and its device memory.  NULL is ignored. */
void mca_destroy(mca_handle* h);

/* Static description of a status code. */
const char* mca_strerror(int code);

/* Detail of the most recent failure in this thread ("" if none). */
const char* mca_last_error_message(void);

/* ---- single-operation entry points (device pointers only; used by tests/bench) ----- */

/* Residual and Jacobian diagonal (eq. (F), eq. (J)) at nvec states.
 *   x     : device, nvec * 2*m*n, [V_t ; V_b] per vector.
 *   v_in  : device, nvec * m.
 *   F     : device out, nvec * 2*m*n, [F_t ; F_b] per vector.
 *   D     : device out, nvec * m*n, g_ij cosh(b (V_t - V_b)).
 *   fnorm : host out, nvec values of ||F||_2 (may be NULL).
 *   dmean : host out, nvec values of mean(D) = a1 = a2 of eq. (P) (may be NULL). */
int mca_residual(mca_handle* h, const double* x, const double* v_in, int32_t nvec,
                 double* F, double* D, double* fnorm, double* dmean, void* stream);

/* The same residual in FP32 pairs, the form the solver uses, with the BF16 and BF16_SPLIT
 * preconditioners, for states far from convergence (eq. (F), eq. (J)).  Each FP64
 * voltage is split into two FP32 halves, products and sums are formed error-free in FP32
 * and each F entry is rounded once to FP64; D is the FP32 conductance as in mca_residual.
 *   ferr : host out, nvec bounds on | ||F computed|| - ||F exact|| | (may be NULL):
 *          2^-40 times the 2-norm of the per-entry term sizes (|wire diagonal x| +
 *          |wire couplings| + |device current| + |source current|).  The solver uses
 *          this residual only for iterates whose ||F|| - ferr stays more than 10 times
 *          above the target (there it is the right-hand side of the next inexact Newton
 *          step); every convergence decision is made on the FP64 residual.
 * Other arguments as mca_residual.  Returns MCA_ERR_UNSUPPORTED when b lies outside about
 * [0.021, 2000] (the device polynomial's tail leaves the FP32 range). */
int mca_residual_pair(mca_handle* h, const double* x, const double* v_in, int32_t nvec,
                      double* F, double* D, double* fnorm, double* dmean, double* ferr,
                      void* stream);

/* Jacobian apply w = J z with J = [[G_t + D, -D], [-D, G_b + D]] (eq. (J)).
 *   D : device, nvec * m*n;  z, w : device, nvec * 2*m*n. */
int mca_jacobian_apply(mca_handle* h, const double* D, const double* z, double* w,
                       int32_t nvec, void* stream);

/* The same apply with z in FP32, as the solver takes it from the tensor-core
 * preconditioner (eq. (J); Section 3.1 for the operator).  mode picks the arithmetic:
 *   MCA_APPLY_PAIR : FP32 pairs, the solver's form for the BF16 and BF16_SPLIT
 *                    preconditioners: z and the neighbours enter error-free FP32 products
 *                    with the wire conductances and D (each split into two FP32 halves)
 *                    and error-free FP32 sums; the low parts are summed in FP32 and the
 *                    result is rounded once to FP64.  Error within about 2^-45 of the
 *                    sum of |diag z|, |g_wire (z_left + z_right)|, |D (z_t - z_b)|.
 *   MCA_APPLY_F64  : FP64 arithmetic on z widened exactly (error within about 2^-51).
 *   MCA_APPLY_F32  : FP32 arithmetic, w rounded to FP32 (the solver's first Newton step
 *                    when eta0 >= 1e-4).
 *   D : device, nvec * m*n (FP64);  z : device, nvec * 2*m*n (FP32);  w : device out,
 *   nvec * 2*m*n (FP64).  Returns MCA_ERR_INVALID_ARG for a null pointer, nvec outside
 *   1..max_batch or an unknown mode. */
#define MCA_APPLY_PAIR 0
#define MCA_APPLY_F64 1
#define MCA_APPLY_F32 2
int mca_jacobian_apply_f32(mca_handle* h, const double* D, const float* z, double* w,
                           int32_t nvec, int32_t mode, void* stream);

/* Preconditioner apply z = P^-1 r (eqs. (P), (block), (M)) with a1 = a2 = a[v] per
 * vector, in the given MCA_PREC_* precision (FP64, BF16, BF16_SPLIT or MHAT; the
 * tensor-core forms need a handle created with one of them).
 *   a : host, nvec values (> 0);  r, z : device, nvec * 2*m*n. */
int mca_precond_apply(mca_handle* h, const double* a, const double* r, double* z,
                      int32_t nvec, int32_t precision, void* stream);

/* Copy out the FP64 eigenpairs of the wire operators (host or device buffers):
 * mu[n], Q_r[n*n] (column k is eigenvector k, row-major storage Q_r[j*n + k]) for G_r;
 * nu[m], Q_c[m*m] for G_c.  Eigenvalues ascending.  NULL outputs are skipped. */
int mca_eigenpairs(mca_handle* h, double* mu, double* q_r, double* nu, double* q_c);

/* Restarted flexible GMRES(restart) for J dx = rhs (Section 4) with the handle's
 * preconditioner (a1 = a2 = a[v]), at the Jacobian diagonal D, from dx = 0.  Stops when
 * the residual reaches rtol * ||rhs|| or after max_iters iterations (max_iters <= 0:
 * one cycle of gmres_restart iterations).
 *   D : device nvec*m*n;  a : host nvec (> 0);  rhs, dx : device nvec*2*m*n;
 *   iters : host out, nvec iteration counts (may be NULL);
 *   res   : host out, nvec final residual estimates ||rhs - J dx|| (may be NULL). */
int mca_gmres_solve(mca_handle* h, const double* D, const double* a, const double* rhs,
                    double* dx, int32_t nvec, double rtol, int32_t max_iters, int32_t* iters,
                    double* res, void* stream);

/* ---- per-kernel-family timing (measurement support) -------------------------------- */
#define MCA_FAM_RESIDUAL 0      /* residual + Jacobian diagonal (eq. F, eq. J)              */
#define MCA_FAM_SPMV_DOTS 1     /* Jacobian apply fused with the first Gram-Schmidt pass    */
#define MCA_FAM_UPDATE_DOTS 2   /* reorthogonalisation (dots, then update + norm), only for
                                   the vectors whose orthogonality estimate asks for it      */
#define MCA_FAM_UPDATE_NORM 3   /* Gram-Schmidt update with the norm; writes the next
                                   (unnormalised) basis vector and its BF16 copy            */
#define MCA_FAM_NORMALIZE 4     /* reserved: no separate normalisation pass (the basis is
                                   kept unnormalised with per-vector scales); reads 0       */
#define MCA_FAM_SMALL 5         /* reductions, Givens, Newton control, least squares        */
#define MCA_FAM_UPDATE_X 6      /* x += Z y                                                 */
#define MCA_FAM_PRECOND_1 7     /* preconditioner transform 1 (X Q_r)                       */
#define MCA_FAM_PRECOND_2 8     /* transform 2 (Q_c^T T1) + per-mode 2x2 inverse            */
#define MCA_FAM_PRECOND_3 9     /* transform 3 (Y_hat Q_r^T)                                */
#define MCA_FAM_PRECOND_4 10    /* transform 4 (Q_c E), FP64 output                         */
#define MCA_NUM_FAMILIES 11

/* Enable (1) or disable (0) timing of the handle's kernel launches with CUDA events on
 * the solve stream; enabling resets the counters.  Timing adds host synchronisation per
 * GMRES cycle, so timed throughput runs keep it off. */
int mca_profile(mca_handle* h, int32_t enable);

/* Totals of one family since the last enable: launches that did work, their summed
 * device time in ms, and their algorithmic DRAM bytes and FLOPs (counting only the
 * vectors still iterating in each launch; the tensor-core transforms count the MMA
 * FLOPs they execute: 2 products in split transform 3, 3 in split transform 4).  Any output may be NULL. */
int mca_profile_read(mca_handle* h, int32_t family, int64_t* launches, double* ms,
                     double* bytes, double* flops);

/* GEMM configuration of the four tensor-core transforms (after autotuning, if enabled):
 * cfg[3 s + 0] = 1 persistent warp-specialised kernel, 0 one CTA per tile, -1 no
 * tensor-core form; cfg[3 s + 1] = tile columns; cfg[3 s + 2] = layers per tile, for
 * transform s = 0..3.  cfg: host, 12 int32.  Diagnostic only. */
int mca_tile_config(const mca_handle* h, int32_t* cfg);

/* ---- residual without device allocation ------------------------------------------- */

/* Residual, Jacobian diagonal and their norms for callers that cannot allocate device
 * memory: services that forbid allocator calls after start-up (fixed memory budgets,
 * real-time loops), and hosts whose device memory is owned by another framework's pool.
 * The paper has no counterpart; this is a usage variant of mca_residual() that needs no
 * handle and makes no cudaMalloc/cudaFree.  Parameters are checked as in mca_create()
 * (circuit part only: sizes, conductances, b, device model).
 *   p      : circuit parameters (rows, cols, wire/termination conductances, b).
 *   g_map  : device, m*n memristor conductances.
 *   x      : device, nvec * 2*m*n states [V_t ; V_b].
 *   v_in   : device, nvec * m input voltages.
 *   F, D   : device outputs as in mca_residual().
 *   fnorm  : device output, nvec values ||F||_2 (may be NULL).
 *   dmean  : device output, nvec values mean(D) (may be NULL).
 *   stream : the call only enqueues work on it (no synchronisation).
 * Limits: 1 <= nvec <= 8, else MCA_ERR_INVALID_ARG.  Scratch lives in a fixed 1.2 MiB
 * device array that every GPU loading the library keeps until exit; all calls on a
 * device share it, so calls that overlap on the GPU race (order them on one stream).
 * The first call on a device looks up that array's address; make it before any stream
 * capture. */
int mca_residual_noalloc(const mca_params* p, const double* g_map, const double* x,
                         const double* v_in, int32_t nvec, double* F, double* D,
                         double* fnorm, double* dmean, void* stream);

/* Self-test of the bounded device waits that guard every mbarrier wait of the
 * tensor-core kernels: launches one thread that waits on a barrier nothing completes,
 * with a limit of limit_ns nanoseconds.  Returns MCA_ERR_TIMEOUT (the expected result)
 * with the CUDA context still usable, or MCA_ERR_CUDA. */
int mca_wait_selftest(mca_handle* h, int64_t limit_ns);

/* Number of CUDA kernel launches this library has made in the calling process. */
int64_t mca_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* MCA_H_ */
