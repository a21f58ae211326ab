// FP64 form of the preconditioner apply z = P^-1 r (eqs. P, block, M; Section 3.2).
//
// In the Kronecker eigenbasis of G_t = I (x) G_r and G_b = G_c (x) I the operator P is a
// 2x2 block per mode (i', k'): [[mu_k' + a1, -a1], [-a2, nu_i' + a2]].  The apply is four
// dense transforms per layer with a per-mode 2x2 inverse in the middle:
//   T1^T = (X Q_r)^T,  X_hat = Q_c^T X Q_r,  Y_hat = modes^-1 X_hat,
//   E^T = (Y_hat Q_r^T)^T,  Z = Q_c Y_hat Q_r^T,
// each one the block-transposed GEMM below.  This is the plain FP64 form (CUDA-core DFMA);
// the tensor-core form lives in k_precond_tc.cu.
#include "mca_internal.cuh"

namespace mca {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256)
k_gemm64_tstore(const double* __restrict__ A, BlkAddr a, const double* __restrict__ Bm,
                double* __restrict__ O, BlkAddr o, int R, int K, int C,
                const VecCtl* __restrict__ ctl) {
  const int b = blockIdx.z >> 1, layer = blockIdx.z & 1;
  if (ctl != nullptr && !ctl[b].gm_active) return;
  const double* Ab = A + b * a.bs + layer * a.ls;
  double* Ob = O + b * o.bs + layer * o.ls;
  const int r0 = blockIdx.x * TM, c0 = blockIdx.y * TN;
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int t = threadIdx.x;
  const int tr = t & 15, tc = t >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += TK) {
    // 64 x 16 tiles of A and Bm, 4 elements per thread, coalesced along k
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * 256;
      const int rr = e >> 4, kk = e & 15;
      const int gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < R && gk < K) ? Ab[(size_t)gr * a.ld + gk] : 0.0;
      const int gc = c0 + rr;
      Bs[kk][rr] = (gc < C && gk < K) ? Bm[(size_t)gc * K + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + tc + 16 * j;
    if (c >= C) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tr + 16 * i;
      if (r < R) Ob[(size_t)c * o.ld + r] = acc[i][j];
    }
  }
}

// [y_t; y_b] = (1/det) [[nu + a2, a1], [a2, mu + a1]] [x_t; x_b],
// det = mu nu + mu a2 + nu a1 = (mu + a1)(nu + a2) - a1 a2, with a1 = a2 = a.
__global__ void k_modes_2x2(double* __restrict__ Xh, const double* __restrict__ mu,
                            const double* __restrict__ nu, int m, int n,
                            const VecCtl* __restrict__ ctl, int kidx) {
  const int b = blockIdx.y;
  if (!ctl[b].gm_active) return;
  const double a = ctl[b].a;
  // scale of the unnormalised input basis vector (kidx < 0: none)
  const double sc = (kidx >= 0) ? ctl[b].s[kidx] : 1.0;
  const size_t mn = (size_t)m * n;
  double* xt = Xh + (size_t)b * 2 * mn;
  double* xb = xt + mn;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < mn;
       e += (size_t)gridDim.x * blockDim.x) {
    const int ip = (int)(e / n), kp = (int)(e - (size_t)ip * n);
    const double M = mu[kp], N = nu[ip];
    const double f = sc / (M * N + M * a + N * a);
    const double u = xt[e], v = xb[e];
    xt[e] = ((N + a) * u + a * v) * f;
    xb[e] = (a * u + (M + a) * v) * f;
  }
}

}  // namespace

void launch_gemm64_tstore(const double* A, BlkAddr a, const double* Bm, double* O, BlkAddr o,
                          int B, int R, int K, int C, const VecCtl* ctl, cudaStream_t s) {
  dim3 grid((R + TM - 1) / TM, (C + TN - 1) / TN, 2 * B);
  k_gemm64_tstore<<<grid, 256, 0, s>>>(A, a, Bm, O, o, R, K, C, ctl);
}

void launch_modes_2x2_f64(double* Xh, const double* mu, const double* nu, int m, int n,
                          const VecCtl* ctl, int B, int kidx, cudaStream_t s) {
  const size_t mn = (size_t)m * n;
  int nb = (int)((mn + 255) / 256);
  if (nb > 1216) nb = 1216;
  k_modes_2x2<<<dim3(nb, B), 256, 0, s>>>(Xh, mu, nu, m, n, ctl, kidx);
}

}  // namespace mca
