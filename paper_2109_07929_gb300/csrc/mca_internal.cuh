// Internal declarations shared by the CUDA translation units of the crossbar solver.
//
// Data layout (device, FP64 unless noted):
//   one solve vector  x = [V_t ; V_b], each layer m x n row-major (cell (i,j) at i*n+j),
//   so a vector holds N2 = 2*m*n doubles; a batch of B vectors is contiguous [b][N2].
//   D (device conductance g*cosh(b dV), the diagonal of the Jacobian's device blocks)
//   is [b][m*n].
// Krylov storage for flexible GMRES(restart): V[b][j][N2] (j = 0..restart) and
// Z[b][j][N2] (j = 0..restart-1).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "../../include/mca.h"

#define MCA_KMAX 30            // largest GMRES restart length
#define MCA_NPART 1024         // max per-vector partial sums of a reduction kernel

namespace mca {

// Per-vector solver control block, written by the control kernels and read by every
// iteration kernel (vectors whose flags are cleared skip their work).
struct VecCtl {
  double ynorm;        // ||Y||_2
  double fnorm;        // ||F||_2 at the current Newton iterate
  double fnorm_prev;   // ||F||_2 at the previous Newton iterate
  double a;            // a1 = a2 = mean(D)
  double eta;          // forcing term of the current linear solve
  double tol_abs;      // GMRES stop: ||r|| <= tol_abs
  double inv_h;        // 1 / h_{k+1,k} for the basis normalisation
  double res_est;      // Givens residual estimate |g_{k+1}|
  int32_t newton_active;
  int32_t status;
  int32_t newton_iters;
  int32_t gmres_iters;
  int32_t gm_active;   // GMRES cycle running
  int32_t k_done;      // columns finished in this cycle
  int32_t reorth;      // the current iteration needs the second Gram-Schmidt pass
  uint32_t reorth_mask;  // bit k: iteration k of this cycle took the second pass
  int32_t need_fp64;   // the FP32-pair residual could not decide convergence
  int32_t d64;         // some entry of D is not an FP32 number (the pair apply splits D)
  int32_t d64_next;    // the same, gathered by the blocks of the running residual launch
  int32_t pad_;
  double orth;         // running estimate of the basis' loss of orthogonality
  double orth1;        // estimate for the new vector after the first pass (when reorth)
  double wn2;          // its squared norm after the first pass (when reorth)
  double H[(MCA_KMAX + 1) * MCA_KMAX];   // column k at H[k*(KMAX+1) + row]
  double cs[MCA_KMAX];
  double sn[MCA_KMAX];
  double g[MCA_KMAX + 1];
  double y[MCA_KMAX];
  // The basis is stored unnormalised: v_j = s[j] * V[j] (s[0] = 1; s[j+1] = 1/h_{j+1,j}
  // is set with the Givens column, saving a separate normalisation pass over the vector).
  double s[MCA_KMAX + 1];
};

// Per-vector results of a solve pass, written by a kernel into mapped pinned host memory
// so the host reads them without a copy (a small device-to-host copy would queue behind
// the large output copies of the previous pass on the copy engine).
struct HostReport {
  int32_t status, newton_iters, gmres_iters, k_done;
  double fnorm, ynorm, kcl, res_est;
};
// rep[b] for b < B from ctl[b] and kcl[b] (kcl may be NULL); rep[B].status = *err.
void launch_report(const VecCtl* ctl, const double* kcl, const int* err, HostReport* rep,
                   int B, cudaStream_t s);

// Scalars of one crossbar needed by the stencil kernels.
struct Grid {
  int m, n;                 // rows, cols
  double gt, gb;            // wire segment conductances (top rows, bottom columns)
  double g_src, g_tr;       // top-row ends: source (j = 0), termination (j = n-1)
  double g_bt, g_sense;     // bottom-column ends: termination (i = 0), sense (i = m-1)
  double b;                 // sinh nonlinearity (0 = linear device)
  double inv_b;             // 1 / b (0 when b = 0)
  // sinh(b dV) / (b dV) = sum_k pc[k] (dV^2)^k for |dV| below the limit whose FP64 high
  // word (sign cleared) is dv_lim_hi: the polynomial of the memristor current with b
  // folded into its coefficients
  double pc[7];
  uint32_t dv_lim_hi;
  // the tail pc[3] + pc[4] t + pc[5] t^2 + pc[6] t^3 in FP32 (pcf) when tail32: at most
  // 3.5e-5 of the polynomial, so FP32 rounding there costs below 1e-11 relative; tail32
  // is off when a folded coefficient leaves [1e-30, 1e30] (b outside about [0.021, 2000])
  float pcf[7];
  int tail32;
  // for the FP32-pair residual: low halves of pc[1], pc[2] (pcf holds the high halves),
  // the polynomial's range in FP32, the source conductance and rneg as FP32 pairs
  float pc1l, pc2l, dv_limf, gsrcf, gsrcl, rnegl;
  float bf;                 // b in FP32 (for the FP32 conductance)
  // Yakopcic-form device: currents and conductances of devices with dV < 0 are scaled by
  // rneg (yak = 0: the symmetric sinh device, rneg = 1)
  int yak;
  double rneg;
  float rnegf;
  // FP32 copies of the wire operators for the FP32 Jacobian apply (each rounded to
  // nearest), and the FP32 remainders x - (double)xf for the pair apply
  float gtf, gbf, dt0f, dtmf, dtlf, db0f, dbmf, dblf;
  float gtl, gbl, dt0l, dtml, dtll, db0l, dbml, dbll;
  // diagonals of the wire operators (eq. G with terminations): first / inside / last node
  double dt0, dtm, dtl;     // top row, along j
  double db0, dbm, dbl;     // bottom column, along i
};

// Fill a Grid from the circuit parameters.
Grid make_grid(const mca_params& p);

struct SolverCfg {
  double newton_rtol;
  double eta0;
  double eta_max;
  int max_newton;
  int restart;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of KP accumulators at once by recursive halving (reduce-scatter): at each of
// the first log2(KP) butterfly levels a lane keeps half of its accumulators and sends the
// other half to its partner, so the whole reduction takes KP - 1 + 5 - log2(KP) FP64
// additions instead of 5 KP (FP64 additions are the scarce resource).  Returns, in every
// lane, the warp total of accumulator warp_scatter_index<KP>(lane); acc is overwritten.
// KP is a power of two <= 32.
template <int KP>
__device__ __forceinline__ double warp_sum_scatter(double (&acc)[KP]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int L = 0; L < 5; ++L) {
    const int o = 16 >> L;
    const int h = KP >> (L + 1);
    if (h >= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < KP / 2; ++i) {
        if (i < h) {
          const double send = up ? acc[i] : acc[i + h];
          const double keep = up ? acc[i + h] : acc[i];
          acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
    } else {
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
    }
  }
  return acc[0];
}

template <int KP>
__device__ __forceinline__ int warp_scatter_index(int lane) {
  int j = 0;
#pragma unroll
  for (int L = 0; L < 5; ++L) {
    const int h = KP >> (L + 1);
    if (h >= 1 && (lane & (16 >> L))) j += h;
  }
  return j;
}

// True in the one lane per accumulator that stores the result of warp_sum_scatter.
template <int KP>
__device__ __forceinline__ bool warp_scatter_writer(int lane) {
  return (lane & (32 / KP - 1)) == 0;
}

// ---------------------------------------------------------------- kernels (launchers)
// stencil / residual / Jacobian (k_stencil.cu)
// warm: the states are a caller's guess (the first forcing term then follows
// Eisenstat-Walker with ||F(0)|| = ||Y|| as the previous residual)
void launch_setup_vectors(const Grid& gr, const double* vin, int B, VecCtl* ctl, bool warm,
                          cudaStream_t s);
// pair: the residual in FP32 pairs (requires gr.tail32), which also leaves the squared
// term sizes' partial sums in part row 2; pair_err_bound turns their total into the bound
// on the error of ||F||
void launch_residual(const Grid& gr, const double* gmap, const double* vin, const double* x,
                     double* F, double* D, double* part, int nblk, int B, const VecCtl* ctl,
                     cudaStream_t s, bool pair = false);
double pair_err_bound(double size2_sum);
// Residual of the solver loop: zero_state skips the device model at x = 0 (F = -Y,
// D = g); the last block of each vector runs the Newton control (convergence test,
// forcing term, start of the GMRES cycle).
// gmaps: conductance maps of the crossbars sharing this shape (m*n each); map_of[b] picks
// vector b's map (NULL: map 0 for all).
// F[b] at F + b*fstride, with its BF16 copy in xbf (may be NULL); the Newton control
// sets the scale -1/||F|| that turns the stored F into the first GMRES basis vector.
// pair (not with zero_state; requires gr.tail32): the FP32-pair residual for vectors whose
// last linear solve ended more than 10 times above the target; its Newton control accepts
// ||F|| only when, within its error bound, it is still more than 10 times above the target,
// and otherwise leaves the vector undecided (host flag 2, need_fp64); confirm: the FP64
// residual for exactly those vectors.
// sparse_f (zero_state only): F = -Y is stored in the first column of the top layer only
// (its other entries are zero and left unwritten); the step's kernels must then read v_0
// there only (kApplyF32Zero, the update passes' zs).
void launch_residual_newton(const Grid& gr, const double* gmaps, const int* map_of,
                            const double* vin, const double* x, bool zero_state, double* F,
                            size_t fstride, __nv_bfloat16* xbf, int mp, int np, double* D,
                            double* part, int nblk, int B, VecCtl* ctl, SolverCfg cfg,
                            unsigned int* cnt, int32_t* host_flags, cudaStream_t s,
                            bool pair = false, bool confirm = false, bool sparse_f = false);
void launch_init_basis(const double* F, double sign, double* V0, size_t vstride,
                       __nv_bfloat16* xbf, int mp, int np, int m, int n, const VecCtl* ctl,
                       int B, cudaStream_t s);
// w = J z fused with the partial dots <V_j, w> (j < nk); with cnt != NULL the last block
// of each vector also reduces them into h[b][j].
void launch_spmv_dots(const Grid& gr, const double* D, const double* z, size_t zstride,
                      double* w, const double* V, size_t vstride, int nk, double* part,
                      int nblk, int B, const VecCtl* ctl, unsigned int* cnt, double* h,
                      cudaStream_t s);
// The same with z in FP32 (the tensor-core preconditioner's output).  apply picks the
// arithmetic of w = J z; the dots stay FP64 in every mode:
//   kApplyPair: FP32 pairs (error-free products and sums of the FP32 z with the wire
//     constants and D split into FP32 pairs), rounded once to FP64; the error stays
//     within about 2^-45 of the size of the terms, against 2^-51 for kApplyF64, and the FP64
//     pipe only splits D and forms the two results (3 operations per cell instead of 8);
//   kApplyF64: FP64 on z widened exactly;
//   kApplyF32: plain FP32 (w rounded to FP32, then widened), for linear solves whose
//     forcing term is loose (kF32ApplyMinEta).
//   kApplyF32Zero: kApplyF32 in the Newton step from V = 0 whose v_0 is stored in the first
//     column of the top layer only (the residual's sparse_f): the dots read it there only.
enum ApplyMode { kApplyF64 = 0, kApplyF32 = 1, kApplyPair = 2, kApplyF32Zero = 3 };
void launch_spmv_dots(const Grid& gr, const double* D, const float* z, size_t zstride,
                      double* w, const double* V, size_t vstride, int nk, double* part,
                      int nblk, int B, const VecCtl* ctl, unsigned int* cnt, double* h,
                      cudaStream_t s, int apply);
// Smallest forcing term at which a Newton step's Jacobian applies run in FP32.  FP32
// rounding of J z is relative to the wire terms, which cancel heavily, so it leaves a
// floor on the linear residual (near 1e-5 relative in an FP32 model of the solver); the
// first Newton step, solved to eta0 = 1e-3, stays well above it.
constexpr double kF32ApplyMinEta = 1e-4;
void launch_outputs(const Grid& gr, const double* vin, const double* x, double* i_out,
                    double* kcl, int B, cudaStream_t s);
// Blocks per vector of the grid-stride stencil / vector kernels for B vectors: about
// kGridBlocks blocks in all (several waves of 256-thread blocks on 152 SMs, so the tail
// is short) but never more than one element per thread or 608 blocks per vector; fewer
// blocks per vector at large B leave each thread more elements, which shrinks the share
// of the per-thread FP64 reduction work.
int residual_nblk(int mn, int B = 1);
// Upper bound of residual_nblk() for every mn and B (sizes the partial-sum buffers).
constexpr int kResidualMaxBlocks = 608;
// Krylov (k_krylov.cu)
int vec_nblk(size_t n2, int B = 1);
void launch_reduce_dots(const double* part, int nblk, int nk, double* h, int B,
                        const VecCtl* ctl, cudaStream_t s);
// pass 2: w -= V h1, partial dots <V_j, w>; the last block reduces them into h2.
// Update passes of the Gram-Schmidt step (phase of launch_update_norm):
//   UPD_PLAIN  out = w - V hc and ||out||^2 partials only (cnt, ctl unused)
//   UPD_FIRST  out = w - V h1 (hc = h1); the last block of each vector estimates the loss
//              of orthogonality of out and either finishes Hessenberg column nk-1 (Givens
//              rotation, scale of the new basis vector, flags) or marks the vector for the
//              second pass
//   UPD_REORTH only for marked vectors: out = w - V h2 (hc = h2, w = out in place), then
//              column nk-1 = h1 + h2 is finished as above
enum UpdPhase { UPD_PLAIN = 0, UPD_FIRST = 1, UPD_REORTH = 2 };
// second-pass dots h2 = V^T u (j < nk) of the new vector u (u[b] at u + b*vstride), only
// for the vectors marked by UPD_FIRST
// zs: the Newton step from V = 0 with a sparse v_0 (see launch_residual_newton), ncols = n
void launch_reorth_dots(const double* u, const double* V, size_t vstride, size_t n2, int nk,
                        double* part, int nblk, int B, const VecCtl* ctl, unsigned int* cnt,
                        double* h2, cudaStream_t s, bool zs = false, int ncols = 1);
// out[b] at out + b*ostride, w[b] at w + b*wstride; BF16 copy of out in xbf (may be NULL)
void launch_update_norm(int phase, const double* w, size_t wstride, const double* V,
                        size_t vstride, size_t n2, int nk, const double* hc, double* part,
                        int nblk, int B, VecCtl* ctl, unsigned int* cnt, const double* h1,
                        int restart, int32_t* host_flags, double* out, size_t ostride,
                        __nv_bfloat16* xbf, int mp, int np, int m, int n, cudaStream_t s,
                        bool zs = false);
void launch_lsq_update(double* x, const double* Z, size_t zstride, size_t n2, VecCtl* ctl,
                       int B, cudaStream_t s);
void launch_lsq_update(double* x, const float* Z, size_t zstride, size_t n2, VecCtl* ctl,
                       int B, cudaStream_t s);
// first = 1: remember beta = ||rhs|| and stop at rtol * beta; first = 0 (a restart): keep
// the tolerance of the first cycle.
void launch_gmres_init(const double* part_norm, int nblk, VecCtl* ctl, int B, double rtol,
                       int first, cudaStream_t s);
// eigen setup (k_eig.cu)
void launch_eig_tridiag(int n, double g, double g_first, double g_last, double* lam,
                        double* Q, double* scratch, cudaStream_t s);
void launch_pack_q_bf16(const double* Q, int n, int npad, __nv_bfloat16* out_q,
                        __nv_bfloat16* out_q_lo, __nv_bfloat16* out_qt, cudaStream_t s);
void launch_transpose64(const double* Q, int n, double* QT, cudaStream_t s);
// paper-literal M_hat, Jacobi and identity preconditioners (k_precond_mhat.cu); fac holds
// 4 * ld doubles per vector, ld = max(m, n)
// (the outputs carry the scale s[kidx] of the input basis vector)
int precond_mhat(const Grid& gr, const double* r, size_t rstride, double* z, size_t zstride,
                 int B, const VecCtl* ctl, double* fac, int ld, int kidx, cudaStream_t s);
int precond_jacobi(const Grid& gr, const double* D, const double* r, size_t rstride, double* z,
                   size_t zstride, int B, bool none, const VecCtl* ctl, int kidx,
                   cudaStream_t s);
// element-wise out = a - b on nvec vectors of n2 doubles (k_krylov.cu)
void launch_sub(const double* a, const double* b, double* out, size_t n2, int B, cudaStream_t s);
// FP64 preconditioner (k_precond64.cu)
// Block-transposed GEMM used by all four eigenbasis transforms:
//   O[blk][c][r] = sum_k A[blk][r][k] * Bm[c][k]   (r < R, c < C, k < K)
// with blk = 2*b + layer; A block blk starts at A + b*a.bs + layer*a.ls (row stride K),
// O block blk starts at O + b*o.bs + layer*o.ls (row stride o.ld along c).
struct BlkAddr {
  size_t bs;   // elements between batch entries
  size_t ls;   // elements between the two layers of one entry
  size_t ld;   // leading dimension (A: row stride; O: stride between c)
};
void launch_gemm64_tstore(const double* A, BlkAddr a, const double* Bm, double* O, BlkAddr o,
                          int B, int R, int K, int C, const VecCtl* ctl, cudaStream_t s);
// Per-mode 2x2 inverse of eq. (P) in place on X_hat[b][layer][i'][k'] (m x n), times the
// scale s[kidx] of the (unnormalised) input basis vector.
void launch_modes_2x2_f64(double* Xh, const double* mu, const double* nu, int m, int n,
                          const VecCtl* ctl, int B, int kidx, cudaStream_t s);

// ---- persistent batched solve (k_persist.cu) ---------------------------------------------
// One shape class of the batch (one handle): stencil constants, solver settings,
// conductance maps, FP32 eigenvalues and the preconditioner's eigenvector operands in the
// tiled layout of k_persist.cu (padded extents mp, np: multiples of 128).
struct PersistShape {
  Grid gr;
  SolverCfg cfg;
  int mp, np;
  const double* gmaps;                  // n_maps * m*n
  const float* mu_f;                    // np
  const float* nu_f;                    // mp
  const __nv_bfloat16* qrt;             // Q_r^T  [np x np]  (transform 1)
  const __nv_bfloat16* qct;             // Q_c^T  [mp x mp]  (transform 2)
  const __nv_bfloat16* qr_hi;           // Q_r    [np x np]  hi / lo words (transform 3)
  const __nv_bfloat16* qr_lo;
  const __nv_bfloat16* qc_hi;           // Q_c    [mp x mp]  hi / lo words (transform 4)
  const __nv_bfloat16* qc_lo;
};

// One work item: an input vector of one crossbar of one shape.
struct PersistItem {
  int32_t shape, map;
  const double* vin;                    // m
  double* vt;                           // m*n or NULL (preconditioner test: r in, z out)
  double* vb;                           // m*n or NULL
  double* iout;                         // n or NULL
  double a;                             // preconditioner test only: a1 = a2 = a
};

struct PersistResult {
  int32_t status, newton_iters, gmres_iters, pad_;
  double fnorm, ynorm, kcl;
};

// Per-CTA scratch ("slot"): the state, D, J z, the Krylov bases and the BF16 operands of one
// solve, for the largest shape of the batch; slot b at base + b * slot_bytes.
struct PersistSlots {
  uint8_t* base;
  size_t slot_bytes;
  size_t off_x, off_d, off_w, off_v, off_z, off_ctl;
  size_t off_bf[5];                     // X, T1, Y_hat, E hi, E lo
  int restart;
};
// Fills the offsets for vectors of up to n2max doubles (two layers of m n entries, each
// padded to a multiple of 4), BF16 operands of up to bfmax
// elements and the given restart length; returns slot_bytes.
size_t persist_slot_layout(PersistSlots& sl, size_t n2max, size_t bfmax, int restart);
// Dynamic shared memory of the kernel and its one-time attribute setup.
int persist_smem_bytes();
cudaError_t persist_configure();
// mode 0: solve every item; mode 1: only z = P^-1 r for each item (r, z in vt / vb).
// prof (device, MCA_BATCH_PHASES entries, or NULL): CTA-nanoseconds per phase are added.
void launch_persist(const PersistShape* shapes, const PersistItem* items, int n_items,
                    PersistResult* res, int* queue, int* err, const PersistSlots& sl,
                    int grid, int mode, bool yak, unsigned long long* prof, cudaStream_t s);
// dst (tiled, R x K) from the row-major BF16 matrix src (R x K); R % 8 == 0, K % 64 == 0;
// k32: the 32-wide K chunks of the split GEMMs' operands, else 64-wide.
void launch_retile_bf16(const __nv_bfloat16* src, int R, int K, __nv_bfloat16* dst, bool k32,
                        cudaStream_t s);

}  // namespace mca

// Report the first CUDA error of a call chain as MCA_ERR_CUDA.
#define MCA_CUDA_TRY(expr)                                 \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) {                               \
      mca::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return MCA_ERR_CUDA;                                 \
    }                                                      \
  } while (0)

namespace mca {
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void set_error_message(const char* msg);
void clear_error_message();
void count_launches(int n);
// Checks of the circuit part of mca_params (sizes, conductances, b, device model); sets
// the error message and returns MCA_ERR_INVALID_ARG on the first failure.
int validate_circuit(const mca_params* p);
}
