// The paper's own evaluation of the preconditioner (Section 3.2, eqs. block, Mhat,
// G2hat, M-1hat, 2matrix1-4) and the two comparison preconditioners of its Table 1
// (Jacobi, none), all in FP64 on CUDA cores.
//
// Block inversion with B = -a1 I (eq. block):
//   z_t = M^-1 (r_b + (G_b + a2 I) r_t / a1),   z_b = ((G_t + a1 I) z_t - r_t) / a1,
// with the Schur complement approximated as M_hat = (G_2 / a1) (x) G_1 (eq. Mhat, the
// whole G_2 divided by a1), so M_hat^-1 W = a1 G_2^-1 W G_1^-1 on the row-major m x n grid
// W (eq. 2matrix4): tridiagonal solves along every column (G_2 = G_c + a2 I) and then
// along every row (G_1 = G_r + a1 I).  The tridiagonal factors (Thomas algorithm: pivots
// and the eliminated upper diagonal) depend only on a and are built once per apply for
// each vector; the solves are O(m n) and memory bound.
#include "mca_internal.cuh"

namespace mca {

namespace {

constexpr int kT = 256;

// Thomas factors of tridiag(-g, d + a, -g) (d: first/inside/last diagonal classes):
// ip[j] = 1 / pivot_j, cp[j] = -g / pivot_j.  One thread per (vector, operator).
__global__ void k_mhat_factor(int m, int n, Grid gr, const VecCtl* __restrict__ ctl,
                              double* __restrict__ fac, int ld) {
  const int b = blockIdx.x;
  const int which = threadIdx.x;  // 0: G_1 over j (n), 1: G_2 over i (m)
  if (which > 1 || (ctl && !ctl[b].gm_active)) return;
  const double a = ctl ? ctl[b].a : 0.0;
  const int len = which == 0 ? n : m;
  const double g = which == 0 ? gr.gt : gr.gb;
  const double d0 = which == 0 ? gr.dt0 : gr.db0;
  const double dm = which == 0 ? gr.dtm : gr.dbm;
  const double dl = which == 0 ? gr.dtl : gr.dbl;
  double* ip = fac + ((size_t)b * 4 + which * 2) * ld;
  double* cp = ip + ld;
  double prev_cp = 0.0;
  for (int j = 0; j < len; ++j) {
    const double d = ((j == 0) ? d0 : ((j == len - 1) ? dl : dm)) + a;
    const double piv = d + g * prev_cp;     // d - (-g) * cp[j-1]
    ip[j] = 1.0 / piv;
    prev_cp = -g / piv;
    cp[j] = prev_cp;
  }
}

// w = r_b + (G_b r_t + a2 r_t) / a1  (G_b acts along columns: neighbours i +- 1)
// (times the scale sc of the unnormalised input basis vector; the whole apply is linear)
__global__ void k_mhat_rhs(Grid gr, const double* __restrict__ r, size_t rstride,
                           double* __restrict__ z, size_t zstride,
                           const VecCtl* __restrict__ ctl, int kidx) {
  const int b = blockIdx.y;
  if (!ctl[b].gm_active) return;
  const double a = ctl[b].a, inv_a = 1.0 / a;
  const double sc = (kidx >= 0) ? ctl[b].s[kidx] : 1.0;
  const int m = gr.m, n = gr.n, mn = m * n;
  const double* rt = r + (size_t)b * rstride;
  const double* rb = rt + mn;
  double* w = z + (size_t)b * zstride;     // z_t slot
  for (int c = blockIdx.x * kT + threadIdx.x; c < mn; c += gridDim.x * kT) {
    const int i = c / n;
    const double db = ((i == 0) ? gr.db0 : ((i == m - 1) ? gr.dbl : gr.dbm)) + a;
    double s = db * rt[c];
    if (i > 0) s -= gr.gb * rt[c - n];
    if (i < m - 1) s -= gr.gb * rt[c + n];
    w[c] = sc * fma(s, inv_a, rb[c]);
  }
}

// In-place tridiagonal solve G_2 U = W along every column (one thread per column j).
__global__ void k_mhat_cols(int m, int n, double* __restrict__ z, size_t zstride,
                            const double* __restrict__ fac, int ld, double g,
                            const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  if (!ctl[b].gm_active) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double* ip = fac + ((size_t)b * 4 + 2) * ld;
  const double* cp = ip + ld;
  double* w = z + (size_t)b * zstride + j;
  double y = 0.0;
  for (int i = 0; i < m; ++i) {           // forward: y_i = (w_i + g y_{i-1}) / piv_i
    y = (w[(size_t)i * n] + g * y) * ip[i];
    w[(size_t)i * n] = y;
  }
  double x = 0.0;
  for (int i = m - 1; i >= 0; --i) {      // back: x_i = y_i - cp_i x_{i+1}
    x = w[(size_t)i * n] - ((i < m - 1) ? cp[i] * x : 0.0);
    w[(size_t)i * n] = x;
  }
}

// In-place tridiagonal solve along every row with G_1, then scale by a1 (M_hat^-1 =
// a1 G_2^-1 (.) G_1^-1).  32 rows per block; 32 x 32 tiles staged in shared memory so the
// global accesses stay coalesced while one thread walks each row.
__global__ void k_mhat_rows(int m, int n, double* __restrict__ z, size_t zstride,
                            const double* __restrict__ fac, int ld, double g,
                            const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  if (!ctl[b].gm_active) return;
  const double a = ctl[b].a;
  __shared__ double tile[32][33];
  const double* ip = fac + ((size_t)b * 4 + 0) * ld;
  const double* cp = ip + ld;
  double* w = z + (size_t)b * zstride;
  const int r0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 warps
  const int ntile = (n + 31) / 32;
  double y = 0.0;                       // carried recurrence of row r0 + tx (warp 0)
  for (int t = 0; t < ntile; ++t) {
    const int c0 = t * 32;
    for (int rr = ty; rr < 32; rr += 8) {
      const int i = r0 + rr, j = c0 + tx;
      tile[rr][tx] = (i < m && j < n) ? w[(size_t)i * n + j] : 0.0;
    }
    __syncthreads();
    if (ty == 0 && r0 + tx < m) {
      for (int jj = 0; jj < 32 && c0 + jj < n; ++jj) {
        y = (tile[tx][jj] + g * y) * ip[c0 + jj];
        tile[tx][jj] = y;
      }
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
      const int i = r0 + rr, j = c0 + tx;
      if (i < m && j < n) w[(size_t)i * n + j] = tile[rr][tx];
    }
    __syncthreads();
  }
  double x = 0.0;
  for (int t = ntile - 1; t >= 0; --t) {
    const int c0 = t * 32;
    for (int rr = ty; rr < 32; rr += 8) {
      const int i = r0 + rr, j = c0 + tx;
      tile[rr][tx] = (i < m && j < n) ? w[(size_t)i * n + j] : 0.0;
    }
    __syncthreads();
    if (ty == 0 && r0 + tx < m) {
      for (int jj = 31; jj >= 0; --jj) {
        const int j = c0 + jj;
        if (j >= n) continue;
        x = tile[tx][jj] - ((j < n - 1) ? cp[j] * x : 0.0);
        tile[tx][jj] = x;
      }
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
      const int i = r0 + rr, j = c0 + tx;
      if (i < m && j < n) w[(size_t)i * n + j] = a * tile[rr][tx];
    }
    __syncthreads();
  }
}

// z_b = ((G_t + a1 I) z_t - r_t) / a1  (G_t acts along rows: neighbours j +- 1)
__global__ void k_mhat_back(Grid gr, const double* __restrict__ r, size_t rstride,
                            double* __restrict__ z, size_t zstride,
                            const VecCtl* __restrict__ ctl, int kidx) {
  const int b = blockIdx.y;
  if (!ctl[b].gm_active) return;
  const double a = ctl[b].a, inv_a = 1.0 / a;
  const double sc = (kidx >= 0) ? ctl[b].s[kidx] : 1.0;
  const int m = gr.m, n = gr.n, mn = m * n;
  const double* rt = r + (size_t)b * rstride;
  double* zt = z + (size_t)b * zstride;
  double* zb = zt + mn;
  for (int c = blockIdx.x * kT + threadIdx.x; c < mn; c += gridDim.x * kT) {
    const int j = c % n;
    const double dt = ((j == 0) ? gr.dt0 : ((j == n - 1) ? gr.dtl : gr.dtm)) + a;
    double s = dt * zt[c];
    if (j > 0) s -= gr.gt * zt[c - 1];
    if (j < n - 1) s -= gr.gt * zt[c + 1];
    zb[c] = fma(-sc, rt[c], s) * inv_a;
  }
}

// Jacobi: z = r / diag(J), diag(J) = wire diagonal + D; none: z = r.
__global__ void k_jacobi(Grid gr, const double* __restrict__ D, const double* __restrict__ r,
                         size_t rstride, double* __restrict__ z, size_t zstride, int none,
                         const VecCtl* __restrict__ ctl, int kidx) {
  const int b = blockIdx.y;
  if (ctl && !ctl[b].gm_active) return;
  const double sc = (ctl && kidx >= 0) ? ctl[b].s[kidx] : 1.0;
  const int m = gr.m, n = gr.n, mn = m * n;
  const double* rb = r + (size_t)b * rstride;
  double* zb = z + (size_t)b * zstride;
  const double* Db = D + (size_t)b * mn;
  for (int c = blockIdx.x * kT + threadIdx.x; c < mn; c += gridDim.x * kT) {
    if (none) {
      zb[c] = sc * rb[c];
      zb[mn + c] = sc * rb[mn + c];
      continue;
    }
    const int i = c / n, j = c - i * n;
    const double dt = (j == 0) ? gr.dt0 : ((j == n - 1) ? gr.dtl : gr.dtm);
    const double db = (i == 0) ? gr.db0 : ((i == m - 1) ? gr.dbl : gr.dbm);
    zb[c] = sc * rb[c] / (dt + Db[c]);
    zb[mn + c] = sc * rb[mn + c] / (db + Db[c]);
  }
}

int nblocks(size_t count) {
  size_t nb = (count + kT - 1) / kT;
  if (nb > 1216) nb = 1216;
  return nb < 1 ? 1 : (int)nb;
}

}  // namespace

int precond_mhat(const Grid& gr, const double* r, size_t rstride, double* z, size_t zstride,
                 int B, const VecCtl* ctl, double* fac, int ld, int kidx, cudaStream_t s) {
  const int m = gr.m, n = gr.n;
  const size_t mn = (size_t)m * n;
  k_mhat_factor<<<B, 32, 0, s>>>(m, n, gr, ctl, fac, ld);
  k_mhat_rhs<<<dim3(nblocks(mn), B), kT, 0, s>>>(gr, r, rstride, z, zstride, ctl, kidx);
  k_mhat_cols<<<dim3((n + 127) / 128, B), 128, 0, s>>>(m, n, z, zstride, fac, ld, gr.gb, ctl);
  k_mhat_rows<<<dim3((m + 31) / 32, B), 256, 0, s>>>(m, n, z, zstride, fac, ld, gr.gt, ctl);
  k_mhat_back<<<dim3(nblocks(mn), B), kT, 0, s>>>(gr, r, rstride, z, zstride, ctl, kidx);
  count_launches(5);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

int precond_jacobi(const Grid& gr, const double* D, const double* r, size_t rstride, double* z,
                   size_t zstride, int B, bool none, const VecCtl* ctl, int kidx,
                   cudaStream_t s) {
  const size_t mn = (size_t)gr.m * gr.n;
  k_jacobi<<<dim3(nblocks(mn), B), kT, 0, s>>>(gr, D, r, rstride, z, zstride, none ? 1 : 0, ctl,
                                               kidx);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

}  // namespace mca
