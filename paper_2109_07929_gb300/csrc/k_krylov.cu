// Flexible GMRES kernels (Section 4: GMRES on each Newton system; right preconditioned,
// Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.6): classical Gram-Schmidt in
// FP64 with a second pass when a running estimate of the loss of orthogonality asks for
// it (the Daniel-Gragg-Kaufman-Stewart selective reorthogonalisation), Givens rotations
// on the Hessenberg column, back substitution and the solution update dx = Z y.
//
// Per iteration k the orthogonalisation runs as
//   pass 1 (fused into the Jacobian apply): h1 = V^T w
//   pass 2: u = w - V h1 (the next basis vector) and ||u||^2 in the same sweep
//   only when the estimate asks for it:
//   pass 3: h2 = V^T u;  pass 4: u <- u - V h2 and ||u||^2
// The estimate follows u = (I - V V^T) w: if V^T V = I + E with |E| <= delta, then
// |V^T u| <= delta |V^T w| plus rounding of order nk eps |w|, so the new vector keeps a
// loss of about (sqrt(nk) delta + c nk eps) / rho with rho = |u| / |w| (the cancellation
// of the pass, |w|^2 = |u|^2 + |h1|^2).  While that stays below kOrthTol the second pass
// is skipped; the GMRES residual estimate is then exact up to a factor 1 + O(k kOrthTol).
// All reductions are two-level (per-block partials, then one fixed-order sum per vector),
// hence deterministic.
#include "bits.cuh"
#include "mca_internal.cuh"
#include "solver_dev.cuh"

namespace mca {

namespace {

constexpr int kThreads = 256;

template <int KP>
__device__ __forceinline__ void block_store_partials(double (&acc)[KP], int nk,
                                                     double* __restrict__ part, int b,
                                                     int nblk) {
  __shared__ double red[kThreads / 32][KP];
  const int wv = threadIdx.x >> 5, l = threadIdx.x & 31;
  const double tot = warp_sum_scatter<KP>(acc);
  if (warp_scatter_writer<KP>(l)) red[wv][warp_scatter_index<KP>(l)] = tot;
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

// pass 3 (marked vectors only): partial dots <V_j, u> of the new vector u, reduced by the
// last block into h2_j = s_j <V_j, u>.
// ZS: the Newton step from V = 0, whose v_0 is stored in the first column of the top layer
// only (the residual's sparse_f); its other entries are not read.
template <int KP, bool ZS = false>
__global__ void __launch_bounds__(kThreads)
k_reorth_dots(const double* __restrict__ u, const double* __restrict__ V, size_t vstride,
              size_t n2, int nk, double* __restrict__ part, int nblk,
              const VecCtl* __restrict__ ctl, unsigned int* cnt, double* h2, int ncols) {
  const int b = blockIdx.y;
  if (!ctl[b].gm_active || !ctl[b].reorth) return;
  double acc[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) acc[j] = 0.0;
  const double* ub = u + (size_t)b * vstride;
  const double* Vb = V + (size_t)b * vstride;
  const int N2 = (int)n2;
  const int mn = N2 / 2, n = ncols;
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < N2; e += nblk * kThreads) {
    const double x = ub[e];
    const bool v0 = !ZS || (e < mn && e % n == 0);
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < nk && (!ZS || j > 0 || v0)) acc[j] = fma(Vb[(size_t)j * n2 + e], x, acc[j]);
  }
  block_store_partials<KP>(acc, nk, part, b, nblk);
  if (last_block(cnt, b, nblk)) {
    block_reduce_rows(part, b, nblk, nk, h2, ctl[b].s);
    if (threadIdx.x == 0) cnt[b] = 0;
  }
}

// Passes 2 and 4: out <- w - sum_j hc_j v_j (the next, unnormalised basis vector, with
// its BF16 copy for the tensor-core preconditioner), then the partial ||out||^2; the last
// block of each vector runs the phase's control step (UpdPhase).
template <int KP, bool ZS = false>
__global__ void __launch_bounds__(kThreads)
k_update_norm(int phase, const double* w, size_t wstride, const double* __restrict__ V,
              size_t vstride, size_t n2, int nk, const double* __restrict__ hc,
              double* __restrict__ part, int nblk, VecCtl* ctl, unsigned int* cnt,
              const double* __restrict__ h1, int restart, int32_t* host_flags, double* out,
              size_t ostride, __nv_bfloat16* __restrict__ xbf, int mp, int np, int m, int n) {
  const int b = blockIdx.y;
  if (phase != UPD_PLAIN && (!ctl[b].gm_active || (phase == UPD_REORTH && !ctl[b].reorth)))
    return;
  const double* sc = (phase != UPD_PLAIN) ? ctl[b].s : nullptr;
  double hj[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j)
    hj[j] = (j < nk) ? hc[(size_t)b * 32 + j] * (sc ? sc[j] : 1.0) : 0.0;
  const double* wb = w + (size_t)b * wstride;
  double* ob = out + (size_t)b * ostride;
  const double* Vb = V + (size_t)b * vstride;
  const size_t mn = n2 / 2;
  double acc[1] = {0.0};
  auto finish = [&](size_t e, double x) {
    ob[e] = x;
    if (xbf != nullptr) {
      const int l = (e >= mn) ? 1 : 0;
      const int cell = (int)(e - (size_t)l * mn);
      const int i = cell / n, jj = cell - i * n;
      xbf[(((size_t)b * 2 + l) * mp + i) * np + jj] = d2bf16_bits(x);
    }
    acc[0] = fma(x, x, acc[0]);
  };
  // four elements per trip with all their loads issued before the first store (out may
  // alias w, so the compiler cannot move loads of the next trip above the stores)
  const size_t st = (size_t)nblk * kThreads;
  size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x;
  // ZS: v_0 is stored (and nonzero) in the first column of the top layer only
  auto v0 = [&](size_t e) { return !ZS || (e < mn && e % (size_t)n == 0); };
  for (; e + 3 * st < n2; e += 4 * st) {
    double x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = wb[e + u * st];
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < nk) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (!ZS || j > 0 || v0(e + u * st))
            x[u] = fma(-hj[j], Vb[(size_t)j * n2 + e + u * st], x[u]);
      }
#pragma unroll
    for (int u = 0; u < 4; ++u) finish(e + u * st, x[u]);
  }
  for (; e < n2; e += st) {
    double x = wb[e];
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < nk && (!ZS || j > 0 || v0(e))) x = fma(-hj[j], Vb[(size_t)j * n2 + e], x);
    finish(e, x);
  }
  block_store_partials<1>(acc, 1, part, b, nblk);
  if (phase == UPD_PLAIN) return;
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
      gram_schmidt_control(ctl[b], b, phase, hn2, hc, h1, nk, restart, host_flags);
    }
  }
}

// y = R^-1 g (upper triangular back substitution of the rotated Hessenberg matrix).
__global__ void k_lsq(VecCtl* ctl) {
  const int b = blockIdx.x;
  VecCtl& c = ctl[b];
  if (threadIdx.x != 0 || !c.newton_active) return;
  lsq_solve(c);
}

__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f2d_bits(x); }

// x <- x + sum_j y_j z_j over the finished cycle (Z in FP64 or FP32).
template <typename ZT>
__global__ void k_update_x(double* __restrict__ x, const ZT* __restrict__ Z,
                           size_t zstride, size_t n2, const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.y;
  const VecCtl& c = ctl[b];
  if (!c.newton_active) return;
  const int kd = c.k_done;
  __shared__ double ys[MCA_KMAX];
  if (threadIdx.x < MCA_KMAX) ys[threadIdx.x] = (threadIdx.x < kd) ? c.y[threadIdx.x] : 0.0;
  __syncthreads();
  double* xb = x + (size_t)b * n2;
  const ZT* Zb = Z + (size_t)b * zstride;
  // 32-bit element indices (n2 < 2^31), as in k_update_norm
  const int N2 = (int)n2;
  const int st = gridDim.x * blockDim.x;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * st < N2; e += 4 * st) {     // four independent elements per trip
    double s[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] = xb[e + u * st];
    const ZT* zj = Zb;
    for (int j = 0; j < kd; ++j, zj += n2) {
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] = fma(ys[j], widen(zj[e + u * st]), s[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) xb[e + u * st] = s[u];
  }
  for (; e < N2; e += st) {
    double s = xb[e];
    const ZT* zj = Zb;
    for (int j = 0; j < kd; ++j, zj += n2) s = fma(ys[j], widen(zj[e]), s);
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
    c.orth = 0.0;
    c.reorth = 0;
    c.reorth_mask = 0u;
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

__global__ void k_report(const VecCtl* __restrict__ ctl, const double* __restrict__ kcl,
                         const int* __restrict__ err, HostReport* rep, int B) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const VecCtl& c = ctl[b];
    HostReport r;
    r.status = c.status;
    r.newton_iters = c.newton_iters;
    r.gmres_iters = c.gmres_iters;
    r.k_done = c.k_done;
    r.fnorm = c.fnorm;
    r.ynorm = c.ynorm;
    r.kcl = kcl ? kcl[b] : 0.0;
    r.res_est = c.res_est;
    rep[b] = r;
  }
  if (threadIdx.x == 0) rep[B].status = *err;
  __threadfence_system();
}

}  // namespace

void launch_report(const VecCtl* ctl, const double* kcl, const int* err, HostReport* rep,
                   int B, cudaStream_t s) {
  k_report<<<1, 128, 0, s>>>(ctl, kcl, err, rep, B);
}

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

int vec_nblk(size_t n2, int B) {
  constexpr size_t kGridBlocks = 152 * 32;
  size_t nb = (n2 + kThreads - 1) / kThreads;
  const size_t want = (kGridBlocks + B - 1) / (size_t)(B < 1 ? 1 : B);
  if (nb > want) nb = want;
  if (nb > 608) nb = 608;
  return nb < 1 ? 1 : (int)nb;
}

void launch_reduce_dots(const double* part, int nblk, int nk, double* h, int B,
                        const VecCtl* ctl, cudaStream_t s) {
  k_reduce_dots<<<B, kThreads, 0, s>>>(part, nblk, nk, h, ctl);
}

#define MCA_KP_DISPATCH1(KERN, ZS_, nk, grid, ...)                             \
  do {                                                                        \
    if ((nk) <= 1) KERN<1, ZS_><<<grid, kThreads, 0, s>>>(__VA_ARGS__);       \
    else if ((nk) <= 2) KERN<2, ZS_><<<grid, kThreads, 0, s>>>(__VA_ARGS__);  \
    else if ((nk) <= 4) KERN<4, ZS_><<<grid, kThreads, 0, s>>>(__VA_ARGS__);  \
    else if ((nk) <= 8) KERN<8, ZS_><<<grid, kThreads, 0, s>>>(__VA_ARGS__);  \
    else if ((nk) <= 16) KERN<16, ZS_><<<grid, kThreads, 0, s>>>(__VA_ARGS__); \
    else KERN<32, ZS_><<<grid, kThreads, 0, s>>>(__VA_ARGS__);                \
  } while (0)
#define MCA_KP_DISPATCH(KERN, zs, nk, grid, ...)                              \
  do {                                                                        \
    if (zs) MCA_KP_DISPATCH1(KERN, true, nk, grid, __VA_ARGS__);              \
    else MCA_KP_DISPATCH1(KERN, false, nk, grid, __VA_ARGS__);                \
  } while (0)

void launch_reorth_dots(const double* u, const double* V, size_t vstride, size_t n2, int nk,
                        double* part, int nblk, int B, const VecCtl* ctl, unsigned int* cnt,
                        double* h2, cudaStream_t s, bool zs, int ncols) {
  dim3 grid(nblk, B);
  MCA_KP_DISPATCH(k_reorth_dots, zs, nk, grid, u, V, vstride, n2, nk, part, nblk, ctl, cnt, h2,
                  ncols);
}

void launch_update_norm(int phase, const double* w, size_t wstride, const double* V,
                        size_t vstride, size_t n2, int nk, const double* hc, double* part,
                        int nblk, int B, VecCtl* ctl, unsigned int* cnt, const double* h1,
                        int restart, int32_t* host_flags, double* out, size_t ostride,
                        __nv_bfloat16* xbf, int mp, int np, int m, int n, cudaStream_t s,
                        bool zs) {
  dim3 grid(nblk, B);
  MCA_KP_DISPATCH(k_update_norm, zs, nk, grid, phase, w, wstride, V, vstride, n2, nk, hc, part,
                  nblk, ctl, cnt, h1, restart, host_flags, out, ostride, xbf, mp, np, m, n);
}

template <typename ZT>
void lsq_update(double* x, const ZT* Z, size_t zstride, size_t n2, VecCtl* ctl, int B,
                cudaStream_t s) {
  k_lsq<<<B, 32, 0, s>>>(ctl);
  int nb = (int)((n2 + kThreads - 1) / kThreads);
  if (nb > 608) nb = 608;
  k_update_x<ZT><<<dim3(nb, B), kThreads, 0, s>>>(x, Z, zstride, n2, ctl);
}

void launch_lsq_update(double* x, const double* Z, size_t zstride, size_t n2, VecCtl* ctl,
                       int B, cudaStream_t s) {
  lsq_update(x, Z, zstride, n2, ctl, B, s);
}

void launch_lsq_update(double* x, const float* Z, size_t zstride, size_t n2, VecCtl* ctl,
                       int B, cudaStream_t s) {
  lsq_update(x, Z, zstride, n2, ctl, B, s);
}

}  // namespace mca
