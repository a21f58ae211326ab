// Stencil kernels: the KCL residual with the Jacobian diagonal (eq. F, eq. J), the
// Jacobian apply fused with the first Gram-Schmidt dot pass, Newton control and the
// output currents.
//
// Wire operators (eq. G with terminations): along top row i, node j has diagonal
//   (j > 0 ? g_t : g_src) + (j < n-1 ? g_t : g_term_right) and couplings -g_t to j +- 1;
// along bottom column j, node i has diagonal (i > 0 ? g_b : g_term_top) +
//   (i < m-1 ? g_b : g_sense) and couplings -g_b to i +- 1 (eqs. Gt, Gb: G_t = I (x) G_r,
//   G_b = G_c (x) I in the row-major node order shared by both layers, Section 3.1).
#include "mca_internal.cuh"

namespace mca {

namespace {

constexpr int kThreads = 256;

// Block-wide sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = (l < kThreads / 32) ? sa[l] : 0.0;
    b = (l < kThreads / 32) ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

__global__ void k_setup_vectors(Grid gr, const double* __restrict__ vin, VecCtl* ctl) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < gr.m; i += blockDim.x) {
    const double v = vin[(size_t)b * gr.m + i];
    s += v * v;
  }
  double dummy = 0.0;
  block_sum2(s, dummy);
  if (threadIdx.x == 0) {
    VecCtl& c = ctl[b];
    const double yn = gr.g_src * sqrt(s);
    c.ynorm = yn;
    c.fnorm = 0.0;
    c.fnorm_prev = 0.0;
    c.a = 0.0;
    c.eta = 0.0;
    c.tol_abs = 0.0;
    c.newton_iters = 0;
    c.gmres_iters = 0;
    c.gm_active = 0;
    c.k_done = 0;
    if (!isfinite(yn)) {
      c.status = MCA_ERR_NONFINITE;
      c.newton_active = 0;
    } else if (yn == 0.0) {          // V_in = 0: the solution is V = 0
      c.status = MCA_OK;
      c.newton_active = 0;
    } else {
      c.status = MCA_OK;
      c.newton_active = 1;
    }
  }
}

// K1: F = blockdiag(G_t, G_b) x + [i; -i] - [Y_t; 0] and D = g cosh(b dV) per cell, with
// per-block partial sums of ||F||^2 and sum(D).
__global__ void __launch_bounds__(kThreads)
k_residual(Grid gr, const double* __restrict__ gmap, const double* __restrict__ vin,
           const double* __restrict__ x, double* __restrict__ F, double* __restrict__ D,
           double* __restrict__ part, int nblk, const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  if (ctl != nullptr && !ctl[b].newton_active) return;
  const int m = gr.m, n = gr.n;
  const int mn = m * n;
  const double* Vt = x + (size_t)b * 2 * mn;
  const double* Vb = Vt + mn;
  double* Ft = F + (size_t)b * 2 * mn;
  double* Fb = Ft + mn;
  double* Db = D + (size_t)b * mn;
  const double* vinb = vin + (size_t)b * m;
  double sf = 0.0, sd = 0.0;
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < mn; c += nblk * kThreads) {
    const int i = c / n;
    const int j = c - i * n;
    const double vt = Vt[c], vb = Vb[c];
    double ft = ((j > 0 ? gr.gt : gr.g_src) + (j < n - 1 ? gr.gt : gr.g_tr)) * vt;
    if (j > 0) ft -= gr.gt * Vt[c - 1];
    if (j < n - 1) ft -= gr.gt * Vt[c + 1];
    if (j == 0) ft -= gr.g_src * vinb[i];
    double fb = ((i > 0 ? gr.gb : gr.g_bt) + (i < m - 1 ? gr.gb : gr.g_sense)) * vb;
    if (i > 0) fb -= gr.gb * Vb[c - n];
    if (i < m - 1) fb -= gr.gb * Vb[c + n];
    const double g = gmap[c];
    const double dv = vt - vb;
    double cur, dg;
    if (gr.b != 0.0) {
      const double zz = gr.b * dv;
      cur = (g / gr.b) * sinh(zz);
      dg = g * cosh(zz);
    } else {
      cur = g * dv;
      dg = g;
    }
    ft += cur;
    fb -= cur;
    Ft[c] = ft;
    Fb[c] = fb;
    Db[c] = dg;
    sf += ft * ft + fb * fb;
    sd += dg;
  }
  block_sum2(sf, sd);
  if (threadIdx.x == 0) {
    part[((size_t)b * 32 + 0) * nblk + blockIdx.x] = sf;
    part[((size_t)b * 32 + 1) * nblk + blockIdx.x] = sd;
  }
}

// Newton control (eq. Newton3): ||F||, a = mean(D), convergence test, forcing term of
// the next linear solve (first: eta0; then Eisenstat-Walker 0.9 (|F_k|/|F_k-1|)^2 capped
// by eta_max, and never tighter than needed to reach the target), GMRES cycle start.
__global__ void k_newton_control(const double* __restrict__ part, int nblk, int mn,
                                 VecCtl* ctl, SolverCfg cfg, int32_t* host_flags) {
  const int b = blockIdx.x;
  VecCtl& c = ctl[b];
  if (!c.newton_active) {
    if (threadIdx.x == 0 && host_flags) host_flags[b] = 0;
    return;
  }
  double sf = 0.0, sd = 0.0;
  for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
    sf += part[((size_t)b * 32 + 0) * nblk + t];
    sd += part[((size_t)b * 32 + 1) * nblk + t];
  }
  block_sum2(sf, sd);
  if (threadIdx.x == 0) {
    const double fn = sqrt(sf);
    const double a = sd / (double)mn;
    c.fnorm_prev = c.fnorm;
    c.fnorm = fn;
    c.a = a;
    c.gm_active = 0;
    c.k_done = 0;
    if (!isfinite(fn) || !isfinite(a)) {
      c.status = MCA_ERR_NONFINITE;
      c.newton_active = 0;
    } else if (fn <= cfg.newton_rtol * c.ynorm) {
      c.status = MCA_OK;
      c.newton_active = 0;
    } else if (c.newton_iters >= cfg.max_newton) {
      c.status = MCA_ERR_NOT_CONVERGED;
      c.newton_active = 0;
    } else {
      double eta;
      if (c.newton_iters == 0 || c.fnorm_prev <= 0.0) {
        eta = cfg.eta0;
      } else {
        const double r = fn / c.fnorm_prev;
        eta = fmin(cfg.eta_max, 0.9 * r * r);
      }
      eta = fmax(eta, 0.5 * cfg.newton_rtol * c.ynorm / fn);
      eta = fmin(eta, 0.5);
      c.eta = eta;
      c.tol_abs = eta * fn;
      c.g[0] = fn;
      c.res_est = fn;
      c.gm_active = 1;
      c.newton_iters += 1;
    }
    if (host_flags) host_flags[b] = c.newton_active;
    __threadfence_system();
  }
}

// v_0 = sign * F / ||F|| (GMRES from dx = 0; sign = -1 for the Newton system J dx = -F) and its BF16 copy in the padded [layer][mp][np]
// layout read by the tensor-core preconditioner.
__global__ void k_init_basis(const double* __restrict__ F, double sign, double* __restrict__ V0,
                             size_t vstride, __nv_bfloat16* __restrict__ xbf, int mp, int np,
                             int m, int n, const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  const VecCtl& c = ctl[b];
  if (!c.gm_active) return;
  const int mn = m * n;
  const size_t n2 = 2 * (size_t)mn;
  const double s = sign / c.g[0];
  const double* f = F + (size_t)b * n2;
  double* v = V0 + (size_t)b * vstride;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n2;
       e += (size_t)gridDim.x * blockDim.x) {
    const double val = f[e] * s;
    v[e] = val;
    if (xbf != nullptr) {
      const int l = (int)(e / mn);
      const int cell = (int)(e - (size_t)l * mn);
      const int i = cell / n, j = cell - (cell / n) * n;
      xbf[(((size_t)b * 2 + l) * mp + i) * np + j] = __double2bfloat16(val);
    }
  }
}

// K2 fused with the first classical Gram-Schmidt pass: w = J z for one cell (both
// layers), then partial dots <V_j, w> for j < nk.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_spmv_dots(Grid gr, const double* __restrict__ D, const double* __restrict__ z,
            size_t zstride, double* __restrict__ w, const double* __restrict__ V,
            size_t vstride, int nk, double* __restrict__ part, int nblk,
            const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  if (ctl != nullptr && !ctl[b].gm_active) return;
  const int m = gr.m, n = gr.n, mn = m * n;
  const size_t n2 = 2 * (size_t)mn;
  const double* zt = z + (size_t)b * zstride;
  const double* zb = zt + mn;
  const double* Db = D + (size_t)b * mn;
  double* wt = w + (size_t)b * n2;
  double* wb = wt + mn;
  const double* Vb_ = V + (size_t)b * vstride;
  double acc[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) acc[j] = 0.0;
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < mn; c += nblk * kThreads) {
    const int i = c / n;
    const int jj = c - i * n;
    const double a = zt[c], bb = zb[c];
    const double cpl = Db[c] * (a - bb);
    double ot = ((jj > 0 ? gr.gt : gr.g_src) + (jj < n - 1 ? gr.gt : gr.g_tr)) * a;
    if (jj > 0) ot -= gr.gt * zt[c - 1];
    if (jj < n - 1) ot -= gr.gt * zt[c + 1];
    ot += cpl;
    double ob = ((i > 0 ? gr.gb : gr.g_bt) + (i < m - 1 ? gr.gb : gr.g_sense)) * bb;
    if (i > 0) ob -= gr.gb * zb[c - n];
    if (i < m - 1) ob -= gr.gb * zb[c + n];
    ob -= cpl;
    wt[c] = ot;
    wb[c] = ob;
    if (V != nullptr) {
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        if (j < nk) {
          const double* vj = Vb_ + (size_t)j * n2;
          acc[j] = fma(vj[c], ot, acc[j]);
          acc[j] = fma(vj[mn + c], ob, acc[j]);
        }
      }
    }
  }
  if (V == nullptr) return;
  __shared__ double red[kThreads / 32][KP];
  const int wv = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    const double s = warp_sum(acc[j]);
    if (l == 0) red[wv][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < nk && threadIdx.x < KP) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) s += red[q][threadIdx.x];
    part[((size_t)b * 32 + threadIdx.x) * nblk + blockIdx.x] = s;
  }
}

// Output currents and the Kirchhoff balance per vector.
__global__ void k_outputs(Grid gr, const double* __restrict__ vin, const double* __restrict__ x,
                          double* __restrict__ i_out, double* __restrict__ kcl) {
  const int b = blockIdx.x;
  const int m = gr.m, n = gr.n, mn = m * n;
  const double* Vt = x + (size_t)b * 2 * mn;
  const double* Vb = Vt + mn;
  double s_in = 0.0, s_abs = 0.0, s_out = 0.0, s_leak = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double iin = gr.g_src * (vin[(size_t)b * m + i] - Vt[(size_t)i * n]);
    s_in += iin;
    s_abs += fabs(iin);
    s_leak += gr.g_tr * Vt[(size_t)i * n + n - 1];
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double io = gr.g_sense * Vb[(size_t)(m - 1) * n + j];
    if (i_out) i_out[(size_t)b * n + j] = io;
    s_out += io;
    s_leak += gr.g_bt * Vb[j];
  }
  block_sum2(s_in, s_abs);
  __syncthreads();
  block_sum2(s_out, s_leak);
  if (threadIdx.x == 0) {
    const double bal = s_in - s_out - s_leak;
    kcl[b] = (s_abs > 0.0) ? fabs(bal) / s_abs : 0.0;
  }
}

}  // namespace

int residual_nblk(int mn) {
  int nb = (mn + kThreads - 1) / kThreads;
  return nb < 608 ? (nb < 1 ? 1 : nb) : 608;
}

void launch_setup_vectors(const Grid& gr, const double* vin, int B, VecCtl* ctl,
                          cudaStream_t s) {
  k_setup_vectors<<<B, kThreads, 0, s>>>(gr, vin, ctl);
}

void launch_residual(const Grid& gr, const double* gmap, const double* vin, const double* x,
                     double* F, double* D, double* part, int nblk, int B, const VecCtl* ctl,
                     cudaStream_t s) {
  k_residual<<<dim3(nblk, B), kThreads, 0, s>>>(gr, gmap, vin, x, F, D, part, nblk, ctl);
}

void launch_newton_control(const double* part, int nblk, int mn, VecCtl* ctl, int B,
                           SolverCfg cfg, int32_t* host_flags, cudaStream_t s) {
  k_newton_control<<<B, kThreads, 0, s>>>(part, nblk, mn, ctl, cfg, host_flags);
}

void launch_init_basis(const double* F, double sign, double* V0, size_t vstride,
                       __nv_bfloat16* xbf, int mp, int np, int m, int n, const VecCtl* ctl,
                       int B, cudaStream_t s) {
  const size_t n2 = 2 * (size_t)m * n;
  int nb = (int)((n2 + kThreads - 1) / kThreads);
  if (nb > 1216) nb = 1216;
  k_init_basis<<<dim3(nb, B), kThreads, 0, s>>>(F, sign, V0, vstride, xbf, mp, np, m, n, ctl);
}

void launch_spmv_dots(const Grid& gr, const double* D, const double* z, size_t zstride,
                      double* w, const double* V, size_t vstride, int nk, double* part,
                      int nblk, int B, const VecCtl* ctl, cudaStream_t s) {
  // z: the vector of batch entry 0, later entries zstride doubles apart; V: basis vector
  // 0 of batch entry 0 (nk vectors N2 apart, entries vstride apart), or NULL.
  dim3 grid(nblk, B);
  if (nk <= 1)
    k_spmv_dots<1><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, ctl);
  else if (nk <= 2)
    k_spmv_dots<2><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, ctl);
  else if (nk <= 4)
    k_spmv_dots<4><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, ctl);
  else if (nk <= 8)
    k_spmv_dots<8><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, ctl);
  else if (nk <= 16)
    k_spmv_dots<16><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, ctl);
  else
    k_spmv_dots<32><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, ctl);
}

void launch_outputs(const Grid& gr, const double* vin, const double* x, double* i_out,
                    double* kcl, int B, cudaStream_t s) {
  k_outputs<<<B, kThreads, 0, s>>>(gr, vin, x, i_out, kcl);
}

}  // namespace mca
