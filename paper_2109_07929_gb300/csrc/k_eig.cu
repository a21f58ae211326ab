// FP64 eigendecomposition of the 1-D wire operators G_r (n x n) and G_c (m x m).
//
// The separability of eqs. (Gt)/(Gb) (Section 3.1) makes the preconditioner of eq. (P)
// block-diagonal in the Kronecker eigenbasis Q_c (x) Q_r, so only the two tridiagonal
// chains need eigenpairs.  A chain of n nodes with segment conductance g, tied at node 0
// through g_first and at node n-1 through g_last, is T = tridiag(-g, d, -g) with
// d_0 = g_first + g, d_{n-1} = g + g_last, d_j = 2g inside (eq. G with terminations;
// n = 1 gives d_0 = g_first + g_last).
//
// Eigenvalue k (ascending) is found by bisection on the Sturm count of T/g (one thread
// per eigenvalue; the count uses the three-term recurrence of the characteristic
// polynomials, which needs one FMA per node because every off-diagonal is -1 after the
// scaling, with power-of-two rescaling to stay in range).  Its eigenvector comes from the
// twisted factorisation (forward LDL^T and backward UDU^T pivots, twist index r where
// |gamma_r| is smallest, then the two one-sided recurrences from x_r = 1), again one
// thread per eigenvector.
#include "mca_internal.cuh"

namespace mca {

namespace {

__device__ __forceinline__ double diag_entry(int i, int n, double d0, double dl, double dm) {
  return (i == 0) ? d0 : ((i == n - 1) ? dl : dm);
}

// Number of eigenvalues of S = T/g below sigma.  S has diagonal s0, sm (inside), sl and
// off-diagonal -1.
__device__ int sturm_count(int n, double s0, double sm, double sl, double sigma) {
  if (n == 1) return (s0 - sigma < 0.0) ? 1 : 0;
  const double kBig = 0x1p+500, kSmall = 0x1p-500;
  double pp = 1.0;                 // p_{i-1}
  double p = s0 - sigma;           // p_i
  if (p == 0.0) p = -0x1p-60;
  int cnt = (p < 0.0) ? 1 : 0;
  const double c = sm - sigma;
  for (int i = 1; i < n - 1; ++i) {
    double pn = fma(c, p, -pp);
    if (pn == 0.0) pn = -p * 0x1p-60;
    cnt += ((pn < 0.0) != (p < 0.0)) ? 1 : 0;
    pp = p;
    p = pn;
    if ((i & 7) == 0) {
      const double ap = fabs(p);
      if (ap > kBig) {
        p *= kSmall;
        pp *= kSmall;
      } else if (ap < kSmall && fabs(pp) < kSmall) {
        p *= kBig;
        pp *= kBig;
      }
    }
  }
  double pn = fma(sl - sigma, p, -pp);
  if (pn == 0.0) pn = -p * 0x1p-60;
  cnt += ((pn < 0.0) != (p < 0.0)) ? 1 : 0;
  return cnt;
}

__global__ void k_eig_values(int n, double g, double d0, double dl, double dm,
                             double* __restrict__ lam) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double s0 = d0 / g, sl = dl / g, sm = dm / g;
  // Gershgorin bounds of S
  double lo = fmin(fmin(s0, sl), sm) - 2.0;
  double hi = fmax(fmax(s0, sl), sm) + 2.0;
  lo -= 1e-12 * fabs(lo) + 1e-300;
  hi += 1e-12 * fabs(hi) + 1e-300;
  // The Sturm count is exact only to about eps * ||S||; stop bisecting below that.
  const double width = 2.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi));
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi || hi - lo <= width) break;
    if (sturm_count(n, s0, sm, sl, mid) >= k + 1)
      hi = mid;
    else
      lo = mid;
  }
  lam[k] = 0.5 * (lo + hi) * g;
}

// Twisted-factorisation eigenvector for lam[k]; DP pivots are kept in Q's column k,
// DM pivots in scratch, both stored [i][k] so a warp touches consecutive addresses.
__global__ void k_eig_vectors(int n, double g, double d0, double dl, double dm,
                              const double* __restrict__ lam, double* __restrict__ Q,
                              double* __restrict__ DM) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (n == 1) {
    Q[0] = 1.0;
    return;
  }
  const double L = lam[k];
  const double g2 = g * g;
  const double tiny = 1e-290;
  double dp = diag_entry(0, n, d0, dl, dm) - L;
  if (dp == 0.0) dp = tiny;
  Q[k] = dp;
  for (int i = 1; i < n; ++i) {
    dp = (diag_entry(i, n, d0, dl, dm) - L) - g2 / dp;
    if (dp == 0.0) dp = tiny;
    Q[(size_t)i * n + k] = dp;
  }
  double dmv = diag_entry(n - 1, n, d0, dl, dm) - L;
  if (dmv == 0.0) dmv = tiny;
  DM[(size_t)(n - 1) * n + k] = dmv;
  int r = n - 1;
  double best = fabs(Q[(size_t)(n - 1) * n + k]);
  for (int i = n - 2; i >= 0; --i) {
    const double di = diag_entry(i, n, d0, dl, dm) - L;
    dmv = di - g2 / dmv;
    if (dmv == 0.0) dmv = tiny;
    DM[(size_t)i * n + k] = dmv;
    const double gam = fabs(Q[(size_t)i * n + k] + dmv - di);
    if (gam < best) {
      best = gam;
      r = i;
    }
  }
  // x_r = 1; x_i = g x_{i+1} / dp_i (i < r); x_{i+1} = g x_i / dm_{i+1} (i >= r)
  double nrm = 1.0;
  double xv = 1.0;
  for (int i = r - 1; i >= 0; --i) {
    xv = g * xv / Q[(size_t)i * n + k];
    Q[(size_t)i * n + k] = xv;
    nrm = fma(xv, xv, nrm);
  }
  Q[(size_t)r * n + k] = 1.0;
  xv = 1.0;
  for (int i = r + 1; i < n; ++i) {
    xv = g * xv / DM[(size_t)i * n + k];
    Q[(size_t)i * n + k] = xv;
    nrm = fma(xv, xv, nrm);
  }
  const double s = 1.0 / sqrt(nrm);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + k] *= s;
}

// hi = bf16(Q), lo = bf16(Q - hi) in [j][k] order and QT = bf16(Q^T) in [k][j] order,
// zero-padded to npad x npad.
__global__ void k_pack_q(const double* __restrict__ Q, int n, int npad,
                         __nv_bfloat16* __restrict__ qh, __nv_bfloat16* __restrict__ ql,
                         __nv_bfloat16* __restrict__ qt) {
  const size_t tot = (size_t)npad * npad;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / npad), c = (int)(e % npad);
    const double v = (r < n && c < n) ? Q[(size_t)r * n + c] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(v);
    if (qh) qh[e] = h;
    if (ql) ql[e] = __double2bfloat16(v - (double)__bfloat162float(h));
    // transposed: element (c, r) of Q^T
    const double vt = (r < n && c < n) ? Q[(size_t)c * n + r] : 0.0;
    if (qt) qt[e] = __double2bfloat16(vt);
  }
}

__global__ void k_transpose64(const double* __restrict__ Q, int n, double* __restrict__ QT) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int r = by + yy, c = bx + threadIdx.x;
    if (r < n && c < n) tile[yy][threadIdx.x] = Q[(size_t)r * n + c];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int r = bx + yy, c = by + threadIdx.x;
    if (r < n && c < n) QT[(size_t)r * n + c] = tile[threadIdx.x][yy];
  }
}

}  // namespace

void launch_eig_tridiag(int n, double g, double g_first, double g_last, double* lam,
                        double* Q, double* scratch, cudaStream_t s) {
  const double d0 = (n == 1) ? g_first + g_last : g_first + g;
  const double dl = (n == 1) ? d0 : g + g_last;
  const double dm = 2.0 * g;
  const int th = 128;
  const int nb = (n + th - 1) / th;
  k_eig_values<<<nb, th, 0, s>>>(n, g, d0, dl, dm, lam);
  k_eig_vectors<<<nb, th, 0, s>>>(n, g, d0, dl, dm, lam, Q, scratch);
}

void launch_pack_q_bf16(const double* Q, int n, int npad, __nv_bfloat16* out_q,
                        __nv_bfloat16* out_q_lo, __nv_bfloat16* out_qt, cudaStream_t s) {
  const size_t tot = (size_t)npad * npad;
  int nb = (int)((tot + 255) / 256);
  if (nb > 4096) nb = 4096;
  k_pack_q<<<nb, 256, 0, s>>>(Q, n, npad, out_q, out_q_lo, out_qt);
}

void launch_transpose64(const double* Q, int n, double* QT, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32);
  k_transpose64<<<grid, dim3(32, 8), 0, s>>>(Q, n, QT);
}

}  // namespace mca
