// Learned warm start: kernels of a small dilated CNN that maps a crossbar's conductance
// map and input vector to a guess of both layers' node voltages, trained on solves the
// method itself produces.  Not part of the paper (a throughput pattern layered on top of
// the Newton solve, which remains the judge of the guess: mca_solve_from).
//
// Layout: activations NCHW FP32; weights [cout][cin][3][3] in BF16 (the FP32 master copy
// lives with the optimiser); FP32 accumulation.  Every layer is a 3x3 convolution with
// dilation d and zero padding d (output size = input size), plus bias and an optional
// leaky ReLU (slope 0.1) whose derivative is read back from the output's sign.
//
// These are CUDA-core kernels: the network is tiny next to the solve, and a direct
// convolution with the weights of one output-channel group staged in shared memory keeps
// every tap in registers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "mca_internal.cuh"

namespace mca {

namespace {

constexpr int kCoGroup = 8;    // output channels per thread in the forward pass
constexpr int kMaxCin = 64;

__device__ __forceinline__ float act_fwd(float z, int act) {
  return (act == 1) ? (z > 0.f ? z : 0.1f * z) : z;
}
__device__ __forceinline__ float act_grad(float y, int act) {
  return (act == 1) ? (y > 0.f ? 1.f : 0.1f) : 1.f;
}

// y[n][co][p] = act(b[co] + sum_ci sum_k w[co][ci][k] x[n][ci][p + d*(k - 1)])
__global__ void k_conv_fwd(const float* __restrict__ x, int N, int Cin, int H, int W,
                           const __nv_bfloat16* __restrict__ wt, const float* __restrict__ bias,
                           int Cout, int d, int act, float* __restrict__ y) {
  __shared__ float ws[kCoGroup][kMaxCin * 9];
  const int co0 = blockIdx.y * kCoGroup;
  const int n = blockIdx.z;
  for (int t = threadIdx.x; t < kCoGroup * Cin * 9; t += blockDim.x) {
    const int g = t / (Cin * 9), r = t - g * (Cin * 9);
    ws[g][r] = (co0 + g < Cout) ? __bfloat162float(wt[(size_t)(co0 + g) * Cin * 9 + r]) : 0.f;
  }
  __syncthreads();
  const int HW = H * W;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  const int yy = p / W, xx = p - yy * W;
  float acc[kCoGroup];
#pragma unroll
  for (int g = 0; g < kCoGroup; ++g) acc[g] = (co0 + g < Cout) ? bias[co0 + g] : 0.f;
  const float* xn = x + (size_t)n * Cin * HW;
  for (int ci = 0; ci < Cin; ++ci) {
    const float* xc = xn + (size_t)ci * HW;
    float v[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int sy = yy + d * (ky - 1);
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int sx = xx + d * (kx - 1);
        v[ky * 3 + kx] = (sy >= 0 && sy < H && sx >= 0 && sx < W) ? xc[sy * W + sx] : 0.f;
      }
    }
#pragma unroll
    for (int g = 0; g < kCoGroup; ++g) {
      const float* wg = &ws[g][ci * 9];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[g] = fmaf(wg[k], v[k], acc[g]);
    }
  }
#pragma unroll
  for (int g = 0; g < kCoGroup; ++g)
    if (co0 + g < Cout) y[((size_t)n * Cout + co0 + g) * HW + p] = act_fwd(acc[g], act);
}

// gz = gy * act'(y), in place into gz (may alias gy).
__global__ void k_act_back(const float* __restrict__ y, const float* gy, float* gz, size_t count,
                           int act) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    gz[e] = gy[e] * act_grad(y[e], act);
}

// gx[n][ci][p] = sum_co sum_k w[co][ci][k] gz[n][co][p - d*(k - 1)]
__global__ void k_conv_bwd_data(const float* __restrict__ gz, int N, int Cin, int H, int W,
                                const __nv_bfloat16* __restrict__ wt, int Cout, int d,
                                float* __restrict__ gx) {
  __shared__ float ws[kCoGroup][kMaxCin * 9];   // here: [ci group][co * 9 + k]
  const int ci0 = blockIdx.y * kCoGroup;
  const int n = blockIdx.z;
  for (int t = threadIdx.x; t < kCoGroup * Cout * 9; t += blockDim.x) {
    const int g = t / (Cout * 9), r = t - g * (Cout * 9);
    const int co = r / 9, k = r - co * 9;
    ws[g][r] = (ci0 + g < Cin) ? __bfloat162float(wt[((size_t)co * Cin + ci0 + g) * 9 + k]) : 0.f;
  }
  __syncthreads();
  const int HW = H * W;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW) return;
  const int yy = p / W, xx = p - yy * W;
  float acc[kCoGroup];
#pragma unroll
  for (int g = 0; g < kCoGroup; ++g) acc[g] = 0.f;
  const float* gn = gz + (size_t)n * Cout * HW;
  for (int co = 0; co < Cout; ++co) {
    const float* gc = gn + (size_t)co * HW;
    float v[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int sy = yy - d * (ky - 1);
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int sx = xx - d * (kx - 1);
        v[ky * 3 + kx] = (sy >= 0 && sy < H && sx >= 0 && sx < W) ? gc[sy * W + sx] : 0.f;
      }
    }
#pragma unroll
    for (int g = 0; g < kCoGroup; ++g) {
      const float* wg = &ws[g][co * 9];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[g] = fmaf(wg[k], v[k], acc[g]);
    }
  }
#pragma unroll
  for (int g = 0; g < kCoGroup; ++g)
    if (ci0 + g < Cin) gx[((size_t)n * Cin + ci0 + g) * HW + p] = acc[g];
}

// Partial weight/bias gradients over a chunk of pixels of all images:
//   part[chunk][co][ci][k] = sum_{n,p in chunk} gz[n][co][p] x[n][ci][p + d*(k - 1)]
//   part_b[chunk][co]      = sum gz[n][co][p]
// one block per (co, chunk), threads over pixels, fixed-order block reduction.
__global__ void k_conv_bwd_weight(const float* __restrict__ x, const float* __restrict__ gz,
                                  int N, int Cin, int H, int W, int Cout, int d, int chunk,
                                  float* __restrict__ part, float* __restrict__ part_b) {
  const int co = blockIdx.x;
  const int ch = blockIdx.y;
  const int HW = H * W;
  const size_t total = (size_t)N * HW;
  const size_t beg = (size_t)ch * chunk;
  const size_t end = (beg + chunk < total) ? beg + chunk : total;
  __shared__ float red[256 / 32];
  for (int ci = 0; ci < Cin; ++ci) {
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    float accb = 0.f;
    for (size_t q = beg + threadIdx.x; q < end; q += blockDim.x) {
      const int n = (int)(q / HW);
      const int p = (int)(q - (size_t)n * HW);
      const int yy = p / W, xx = p - yy * W;
      const float g = gz[((size_t)n * Cout + co) * HW + p];
      if (ci == 0) accb += g;
      const float* xc = x + ((size_t)n * Cin + ci) * HW;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const int sy = yy + d * (ky - 1);
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int sx = xx + d * (kx - 1);
          if (sy >= 0 && sy < H && sx >= 0 && sx < W) acc[ky * 3 + kx] = fmaf(g, xc[sy * W + sx], acc[ky * 3 + kx]);
        }
      }
    }
    for (int k = 0; k < 10; ++k) {
      float v = (k < 9) ? acc[k] : accb;
      if (k == 9 && ci != 0) break;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        if (k < 9)
          part[(((size_t)ch * Cout + co) * Cin + ci) * 9 + k] = s;
        else
          part_b[(size_t)ch * Cout + co] = s;
      }
      __syncthreads();
    }
  }
}

// gw[i] = sum over chunks of part[chunk][i] (fixed order).
__global__ void k_sum_chunks(const float* __restrict__ part, int nchunk, size_t count,
                             float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * count + i];
    out[i] = s;
  }
}

// Mean squared error and its gradient: loss_part[block] partial sums, gp = 2 (p - t) / count.
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ tgt, size_t count,
                      float* __restrict__ gp, float* __restrict__ loss_part) {
  float s = 0.f;
  const float sc = 2.0f / (float)count;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const float r = pred[e] - tgt[e];
    s = fmaf(r, r, s);
    if (gp) gp[e] = sc * r;
  }
  __shared__ float red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    loss_part[blockIdx.x] = t;
  }
}

__global__ void k_mse_finish(const float* __restrict__ part, int nb, size_t count,
                             float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *loss = (float)(s / (double)count);
  }
}

// Adam on the FP32 master weights, then the BF16 copy used by the convolutions.
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                       const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, size_t count, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float upd = (a / bc1) / (sqrtf(b / bc2) + eps);
    const float nw = w[i] - lr * upd;
    w[i] = nw;
    if (wb) wb[i] = __float2bfloat16(nw);
  }
}

// Network input of one crossbar and input vector: channel 0 = log10(g) + 5 (log-uniform
// [1e-6, 1e-4] S maps to [-1, 1]), channel 1 = V_in[i] / vscale along row i, and with
// four channels the node position j/(n-1), i/(m-1).
__global__ void k_features(const double* __restrict__ gmap, const double* __restrict__ vin,
                           int m, int n, float vscale, int nchan, float* __restrict__ x) {
  const int b = blockIdx.y;
  const int mn = m * n;
  float* xb = x + (size_t)b * nchan * mn;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < mn; c += gridDim.x * blockDim.x) {
    const int i = c / n, j = c - i * n;
    xb[c] = (float)(log10(gmap[c]) + 5.0);
    xb[mn + c] = (float)(vin[(size_t)b * m + i] / vscale);
    if (nchan == 4) {
      xb[2 * mn + c] = (n > 1) ? (float)j / (float)(n - 1) : 0.f;
      xb[3 * mn + c] = (m > 1) ? (float)i / (float)(m - 1) : 0.f;
    }
  }
}

// Network output (2 channels) to an FP64 solver state [V_t ; V_b] (scales undone).
__global__ void k_to_state(const float* __restrict__ y, int mn, float vscale, float bscale,
                           double* __restrict__ x) {
  const int b = blockIdx.y;
  const float* yb = y + (size_t)b * 2 * mn;
  double* xs = x + (size_t)b * 2 * mn;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < mn; c += gridDim.x * blockDim.x) {
    xs[c] = (double)yb[c] * vscale;
    xs[mn + c] = (double)yb[mn + c] * (vscale / bscale);
  }
}

// FP64 solver state to the network's 2-channel target (training data).
__global__ void k_from_state(const double* __restrict__ x, int mn, float vscale, float bscale,
                             float* __restrict__ y) {
  const int b = blockIdx.y;
  const double* xs = x + (size_t)b * 2 * mn;
  float* yb = y + (size_t)b * 2 * mn;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < mn; c += gridDim.x * blockDim.x) {
    yb[c] = (float)(xs[c] / vscale);
    yb[mn + c] = (float)(xs[mn + c] * bscale / vscale);
  }
}

int grid1d(size_t count, int th) {
  size_t nb = (count + th - 1) / th;
  if (nb > 4096) nb = 4096;
  return nb < 1 ? 1 : (int)nb;
}

}  // namespace

}  // namespace mca

using namespace mca;

extern "C" {

int mca_cnn_conv_forward(const float* x, int32_t n, int32_t cin, int32_t h, int32_t w,
                         const uint16_t* wt, const float* bias, int32_t cout, int32_t dilation,
                         int32_t act, float* y, void* stream) {
  if (!x || !wt || !bias || !y || n < 1 || cin < 1 || cin > kMaxCin || cout < 1 || h < 1 ||
      w < 1 || dilation < 1 || (act != 0 && act != 1))
    return MCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int th = 128;
  dim3 grid((h * w + th - 1) / th, (cout + kCoGroup - 1) / kCoGroup, n);
  k_conv_fwd<<<grid, th, 0, s>>>(x, n, cin, h, w, reinterpret_cast<const __nv_bfloat16*>(wt),
                                 bias, cout, dilation, act, y);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

int mca_cnn_conv_backward(const float* x, const float* y, const float* gy, int32_t n,
                          int32_t cin, int32_t h, int32_t w, const uint16_t* wt, int32_t cout,
                          int32_t dilation, int32_t act, float* gz_scratch, float* gx,
                          float* gw, float* gb, float* part, int32_t nchunk, void* stream) {
  if (!x || !y || !gy || !wt || !gz_scratch || !gw || !gb || !part || n < 1 || cin < 1 ||
      cin > kMaxCin || cout < 1 || cout > kMaxCin || h < 1 || w < 1 || dilation < 1 ||
      nchunk < 1)
    return MCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ycount = (size_t)n * cout * h * w;
  k_act_back<<<grid1d(ycount, 256), 256, 0, s>>>(y, gy, gz_scratch, ycount, act);
  count_launches(1);
  const int th = 128;
  if (gx) {
    dim3 grid((h * w + th - 1) / th, (cin + kCoGroup - 1) / kCoGroup, n);
    k_conv_bwd_data<<<grid, th, 0, s>>>(gz_scratch, n, cin, h, w,
                                        reinterpret_cast<const __nv_bfloat16*>(wt), cout,
                                        dilation, gx);
    count_launches(1);
  }
  const size_t total = (size_t)n * h * w;
  const int chunk = (int)((total + nchunk - 1) / nchunk);
  float* part_b = part + (size_t)nchunk * cout * cin * 9;
  k_conv_bwd_weight<<<dim3(cout, nchunk), 256, 0, s>>>(x, gz_scratch, n, cin, h, w, cout,
                                                       dilation, chunk, part, part_b);
  const size_t wcount = (size_t)cout * cin * 9;
  k_sum_chunks<<<grid1d(wcount, 256), 256, 0, s>>>(part, nchunk, wcount, gw);
  k_sum_chunks<<<grid1d(cout, 256), 256, 0, s>>>(part_b, nchunk, cout, gb);
  count_launches(4);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

int mca_cnn_mse(const float* pred, const float* target, int64_t count, float* gpred,
                float* part, float* loss, void* stream) {
  if (!pred || !target || !part || !loss || count < 1) return MCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = 256;
  k_mse<<<nb, 256, 0, s>>>(pred, target, (size_t)count, gpred, part);
  k_mse_finish<<<1, 32, 0, s>>>(part, nb, (size_t)count, loss);
  count_launches(2);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

int mca_cnn_adam(float* w, uint16_t* w_bf16, const float* g, float* m1, float* m2, int64_t count,
                 float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
  if (!w || !g || !m1 || !m2 || count < 1 || step < 1) return MCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid1d((size_t)count, 256), 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16*>(w_bf16),
                                                    g, m1, m2, (size_t)count, lr, beta1, beta2,
                                                    eps, bc1, bc2);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

int mca_cnn_features(const double* gmap, const double* vin, int32_t nvec, int32_t m, int32_t n,
                     float vscale, int32_t nchan, float* x, void* stream) {
  if (!gmap || !vin || !x || nvec < 1 || m < 1 || n < 1 || !(vscale > 0.f) ||
      (nchan != 2 && nchan != 4))
    return MCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_features<<<dim3(grid1d((size_t)m * n, 256), nvec), 256, 0, s>>>(gmap, vin, m, n, vscale,
                                                                      nchan, x);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

int mca_cnn_state(const float* y, double* x, int32_t nvec, int32_t m, int32_t n, float vscale,
                  float bscale, int32_t to_state, float* y_out, void* stream) {
  if (nvec < 1 || m < 1 || n < 1 || !(vscale > 0.f) || !(bscale > 0.f)) return MCA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid(grid1d((size_t)m * n, 256), nvec);
  if (to_state) {
    if (!y || !x) return MCA_ERR_INVALID_ARG;
    k_to_state<<<grid, 256, 0, s>>>(y, m * n, vscale, bscale, x);
  } else {
    if (!x || !y_out) return MCA_ERR_INVALID_ARG;
    k_from_state<<<grid, 256, 0, s>>>(x, m * n, vscale, bscale, y_out);
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? MCA_OK : MCA_ERR_CUDA;
}

}  // extern "C"
