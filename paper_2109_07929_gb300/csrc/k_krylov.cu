// Flexible GMRES kernels (Section 4: GMRES on each Newton system; right preconditioned,
// Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.6): classical Gram-Schmidt
// with one reorthogonalisation (CGS2) in FP64, Givens rotations on the Hessenberg column,
// back substitution and the solution update dx = Z y.
//
// Per iteration k the orthogonalisation runs as
//   pass 1 (fused into the Jacobian apply): h1 = V^T w
//   pass 2: w <- w - V h1, and h2 = V^T w in the same sweep
//   pass 3: w <- w - V h2, and ||w||^2 in the same sweep
// so the nk = k+1 basis vectors are read three times.  All reductions are two-level
// (per-block partials, then one fixed-order sum per vector), hence deterministic.
#include "bits.cuh"
#include "mca_internal.cuh"

namespace mca {

namespace {

constexpr int kThreads = 256;

template <int KP>
__device__ __forceinline__ void block_store_partials(double (&acc)[KP], int nk,
                                                     double* __restrict__ part, int b,
                                                     int nblk) {
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
    __threadfence();
  }
}

// True in every thread of the block that finished last among the nblk blocks of vector b
// (its partial sums are then all visible); the counter is reset by the caller.
__device__ __forceinline__ bool last_block(unsigned int* cnt, int b, int nblk) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&cnt[b], 1u) == (unsigned)nblk - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Fixed-order reduction of part[b][j][0..nblk) into h[b][j] = scale[j] * sum (j < nk),
// warp w taking rows w, w + 8, ...
__device__ __forceinline__ void block_reduce_rows(const double* __restrict__ part, int b,
                                                  int nblk, int nk, double* __restrict__ h,
                                                  const double* scale) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int j = w; j < nk; j += kThreads / 32) {
    double s = 0.0;
    for (int t = l; t < nblk; t += 32) s += __ldcg(&part[((size_t)b * 32 + j) * nblk + t]);
    s = warp_sum(s);
    if (l == 0) h[(size_t)b * 32 + j] = scale ? s * scale[j] : s;
  }
}

// Givens rotation of Hessenberg column k (h = h1 + h2, h_{k+1,k} = sqrt(hn2)), residual
// estimate |g_{k+1}| and the stop test of the GMRES cycle.  One thread.
__device__ void givens_column(VecCtl& c, int b, double hn2, const double* __restrict__ h1,
                              const double* __restrict__ h2, int k, int restart,
                              int32_t* host_flags) {
  const int ld = MCA_KMAX + 1;
  double* col = c.H + (size_t)k * ld;
  for (int j = 0; j <= k; ++j) col[j] = __ldcg(&h1[(size_t)b * 32 + j]) + __ldcg(&h2[(size_t)b * 32 + j]);
  const double hk1 = sqrt(hn2);
  col[k + 1] = hk1;
  for (int j = 0; j < k; ++j) {
    const double t = c.cs[j] * col[j] + c.sn[j] * col[j + 1];
    col[j + 1] = -c.sn[j] * col[j] + c.cs[j] * col[j + 1];
    col[j] = t;
  }
  const double rho = hypot(col[k], col[k + 1]);
  double cs = 1.0, sn = 0.0;
  if (rho > 0.0) {
    cs = col[k] / rho;
    sn = col[k + 1] / rho;
  }
  c.cs[k] = cs;
  c.sn[k] = sn;
  col[k] = rho;
  col[k + 1] = 0.0;
  c.g[k + 1] = -sn * c.g[k];
  c.g[k] = cs * c.g[k];
  const double res = fabs(c.g[k + 1]);
  c.res_est = res;
  c.k_done = k + 1;
  c.gmres_iters += 1;
  c.inv_h = (hk1 > 0.0) ? 1.0 / hk1 : 0.0;
  c.s[k + 1] = c.inv_h;
  const bool stop = !(res > c.tol_abs) || (k + 1 >= restart) || !(hk1 > 0.0) ||
                    !(rho > 0.0) || !isfinite(res);
  if (stop) c.gm_active = 0;
  if (host_flags) host_flags[b] = c.gm_active;
  __threadfence_system();
}

// h[b][j] = sum over blocks of part[b][j][:] for j < nk.
__global__ void k_reduce_dots(const double* __restrict__ part, int nblk, int nk,
                              double* __restrict__ h, const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.x;
  if (ctl != nullptr && !ctl[b].gm_active) return;
  const int wv = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int j = wv; j < nk; j += kThreads / 32) {
    double s = 0.0;
    for (int t = l; t < nblk; t += 32) s += part[((size_t)b * 32 + j) * nblk + t];
    s = warp_sum(s);
    if (l == 0) h[(size_t)b * 32 + j] = s;
  }
}

// pass 2: w <- w - sum_j h_j v_j, then partial dots <v_j, w>.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_update_dots(double* __restrict__ w, const double* __restrict__ V, size_t vstride, size_t n2,
              int nk, const double* __restrict__ h, double* __restrict__ part, int nblk,
              const VecCtl* __restrict__ ctl, unsigned int* cnt, double* h2) {
  const int b = blockIdx.y;
  if (ctl != nullptr && !ctl[b].gm_active) return;
  double hj[KP], acc[KP];
  const double* sc = ctl ? ctl[b].s : nullptr;
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    hj[j] = (j < nk) ? h[(size_t)b * 32 + j] * (sc ? sc[j] : 1.0) : 0.0;
    acc[j] = 0.0;
  }
  double* wb = w + (size_t)b * n2;
  const double* Vb = V + (size_t)b * vstride;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n2;
       e += (size_t)nblk * kThreads) {
    double v[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) v[j] = (j < nk) ? Vb[(size_t)j * n2 + e] : 0.0;
    double x = wb[e];
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < nk) x = fma(-hj[j], v[j], x);
    wb[e] = x;
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < nk) acc[j] = fma(v[j], x, acc[j]);
  }
  block_store_partials<KP>(acc, nk, part, b, nblk);
  if (cnt != nullptr && last_block(cnt, b, nblk)) {
    block_reduce_rows(part, b, nblk, nk, h2, sc);
    if (threadIdx.x == 0) cnt[b] = 0;
  }
}

// pass 3: out <- w - sum_j h_j v_j (the next, unnormalised basis vector, with its BF16
// copy for the tensor-core preconditioner), then the partial ||out||^2; the last block
// of each vector turns the norm into h_{k+1,k}, the Givens column and the new scale.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_update_norm(const double* w, const double* __restrict__ V, size_t vstride, size_t n2,
              int nk, const double* __restrict__ h, double* __restrict__ part, int nblk,
              VecCtl* ctl, unsigned int* cnt, const double* __restrict__ h1, int restart,
              int32_t* host_flags, double* out, size_t ostride,
              __nv_bfloat16* __restrict__ xbf, int mp, int np, int m, int n) {
  const int b = blockIdx.y;
  if (ctl != nullptr && !ctl[b].gm_active) return;
  const double* sc = ctl ? ctl[b].s : nullptr;
  double hj[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j)
    hj[j] = (j < nk) ? h[(size_t)b * 32 + j] * (sc ? sc[j] : 1.0) : 0.0;
  const double* wb = w + (size_t)b * n2;
  double* ob = out + (size_t)b * ostride;
  const double* Vb = V + (size_t)b * vstride;
  const size_t mn = n2 / 2;
  double acc[1] = {0.0};
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n2;
       e += (size_t)nblk * kThreads) {
    double x = wb[e];
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < nk) x = fma(-hj[j], Vb[(size_t)j * n2 + e], x);
    ob[e] = x;
    if (xbf != nullptr) {
      const int l = (e >= mn) ? 1 : 0;
      const int cell = (int)(e - (size_t)l * mn);
      const int i = cell / n, jj = cell - i * n;
      xbf[(((size_t)b * 2 + l) * mp + i) * np + jj] = d2bf16_bits(x);
    }
    acc[0] = fma(x, x, acc[0]);
  }
  block_store_partials<1>(acc, 1, part, b, nblk);
  if (cnt == nullptr) return;
  if (last_block(cnt, b, nblk)) {
    __shared__ double hn2;
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int t = threadIdx.x; t < nblk; t += 32) s += __ldcg(&part[((size_t)b * 32) * nblk + t]);
      s = warp_sum(s);
      if (threadIdx.x == 0) hn2 = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cnt[b] = 0;
      givens_column(ctl[b], b, hn2, h1, h, nk - 1, restart, host_flags);
    }
  }
}

// y = R^-1 g (upper triangular back substitution of the rotated Hessenberg matrix).
__global__ void k_lsq(VecCtl* ctl) {
  const int b = blockIdx.x;
  VecCtl& c = ctl[b];
  if (threadIdx.x != 0 || !c.newton_active) return;
  const int kd = c.k_done;
  const int ld = MCA_KMAX + 1;
  for (int i = kd - 1; i >= 0; --i) {
    double s = c.g[i];
    for (int j = i + 1; j < kd; ++j) s -= c.H[(size_t)j * ld + i] * c.y[j];
    const double d = c.H[(size_t)i * ld + i];
    c.y[i] = (d != 0.0) ? s / d : 0.0;
  }
}

// x <- x + sum_j y_j z_j over the finished cycle.
__global__ void k_update_x(double* __restrict__ x, const double* __restrict__ Z,
                           size_t zstride, size_t n2, const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  const VecCtl& c = ctl[b];
  if (!c.newton_active) return;
  const int kd = c.k_done;
  __shared__ double ys[MCA_KMAX];
  if (threadIdx.x < MCA_KMAX) ys[threadIdx.x] = (threadIdx.x < kd) ? c.y[threadIdx.x] : 0.0;
  __syncthreads();
  double* xb = x + (size_t)b * n2;
  const double* Zb = Z + (size_t)b * zstride;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n2;
       e += (size_t)gridDim.x * blockDim.x) {
    double s = xb[e];
    for (int j = 0; j < kd; ++j) s = fma(ys[j], Zb[(size_t)j * n2 + e], s);
    xb[e] = s;
  }
}

// Start of a stand-alone linear solve: beta = ||rhs|| from the norm partials, stop at
// rtol * beta.
__global__ void k_gmres_init(const double* __restrict__ part_norm, int nblk, VecCtl* ctl,
                             double rtol, int first) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int t = threadIdx.x; t < nblk; t += 32) s += part_norm[((size_t)b * 32) * nblk + t];
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    VecCtl& c = ctl[b];
    const double beta = sqrt(s);
    if (first) {
      c.ynorm = beta;                      // ||rhs|| of the linear system
      c.tol_abs = rtol * beta;
      c.gmres_iters = 0;
    }
    c.g[0] = beta;
    c.s[0] = 1.0;
    c.res_est = beta;
    c.k_done = 0;
    c.newton_active = 1;
    c.status = MCA_OK;
    c.gm_active = (beta > c.tol_abs && beta > 0.0) ? 1 : 0;
  }
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ out, size_t n2) {
  const size_t off = (size_t)blockIdx.y * n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n2;
       e += (size_t)gridDim.x * blockDim.x)
    out[off + e] = a[off + e] - b[off + e];
}

}  // namespace

void launch_gmres_init(const double* part_norm, int nblk, VecCtl* ctl, int B, double rtol,
                       int first, cudaStream_t s) {
  k_gmres_init<<<B, 32, 0, s>>>(part_norm, nblk, ctl, rtol, first);
}

void launch_sub(const double* a, const double* b, double* out, size_t n2, int B,
                cudaStream_t s) {
  int nb = (int)((n2 + kThreads - 1) / kThreads);
  if (nb > 1216) nb = 1216;
  k_sub<<<dim3(nb, B), kThreads, 0, s>>>(a, b, out, n2);
}

int vec_nblk(size_t n2) {
  size_t nb = (n2 + kThreads - 1) / kThreads;
  if (nb > 608) nb = 608;
  return nb < 1 ? 1 : (int)nb;
}

void launch_reduce_dots(const double* part, int nblk, int nk, double* h, int B,
                        const VecCtl* ctl, cudaStream_t s) {
  k_reduce_dots<<<B, kThreads, 0, s>>>(part, nblk, nk, h, ctl);
}

#define MCA_KP_DISPATCH(KERN, nk, grid, ...)                                  \
  do {                                                                        \
    if ((nk) <= 1) KERN<1><<<grid, kThreads, 0, s>>>(__VA_ARGS__);            \
    else if ((nk) <= 2) KERN<2><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
    else if ((nk) <= 4) KERN<4><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
    else if ((nk) <= 8) KERN<8><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
    else if ((nk) <= 16) KERN<16><<<grid, kThreads, 0, s>>>(__VA_ARGS__);     \
    else KERN<32><<<grid, kThreads, 0, s>>>(__VA_ARGS__);                     \
  } while (0)

void launch_update_dots(double* w, const double* V, size_t vstride, size_t n2, int nk,
                        const double* h1, double* part, int nblk, int B, const VecCtl* ctl,
                        unsigned int* cnt, double* h2, cudaStream_t s) {
  dim3 grid(nblk, B);
  MCA_KP_DISPATCH(k_update_dots, nk, grid, w, V, vstride, n2, nk, h1, part, nblk, ctl, cnt, h2);
}

void launch_update_norm(double* w, const double* V, size_t vstride, size_t n2, int nk,
                        const double* h2, double* part, int nblk, int B, VecCtl* ctl,
                        unsigned int* cnt, const double* h1, int restart,
                        int32_t* host_flags, double* out, size_t ostride,
                        __nv_bfloat16* xbf, int mp, int np, int m, int n, cudaStream_t s) {
  dim3 grid(nblk, B);
  MCA_KP_DISPATCH(k_update_norm, nk, grid, w, V, vstride, n2, nk, h2, part, nblk, ctl, cnt,
                  h1, restart, host_flags, out, ostride, xbf, mp, np, m, n);
}

void launch_lsq_update(double* x, const double* Z, size_t zstride, size_t n2, VecCtl* ctl,
                       int B, cudaStream_t s) {
  k_lsq<<<B, 32, 0, s>>>(ctl);
  int nb = (int)((n2 + kThreads - 1) / kThreads);
  if (nb > 1216) nb = 1216;
  k_update_x<<<dim3(nb, B), kThreads, 0, s>>>(x, Z, zstride, n2, ctl);
}

}  // namespace mca
