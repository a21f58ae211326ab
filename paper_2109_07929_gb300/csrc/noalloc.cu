// Residual evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the KCL residual:
// services that must not touch the device allocator after start-up (fixed memory
// budgets, real-time control loops), and hosts whose device memory belongs to another
// framework's pool, which hands out no raw allocations.  mca_create() allocates the whole
// solver workspace, so those callers get this one entry point instead: it needs no
// handle, takes every input and output from the caller, and keeps its only scratch -- the
// per-block partial sums of ||F||^2 and sum(D) -- in the fixed array below, which every
// GPU that loads the library holds until the process exits.
//
// Rules of use:
//   * at most kMaxVec input vectors per call (larger calls return MCA_ERR_INVALID_ARG);
//   * every call on a device shares the one array; it keeps the previous call's
//     partials, but each call writes every slot it reads before reading it, so nothing
//     has to be cleared.  Calls whose kernels overlap on the GPU (different streams
//     without ordering between them) race on the array and give wrong norms;
//   * the first call on a device looks up the array's device address (once per device,
//     with that device current); make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mca_internal.cuh"

namespace mca {

namespace {

constexpr int kMaxVec = 8;                        // vectors per call
constexpr int kMaxBlocks = kResidualMaxBlocks;    // residual_nblk() never exceeds this
constexpr int kMaxDevices = 64;

// Partial sums of the residual kernel: [vector][32 rows][block] (rows 0 and 1 used).
static __device__ __align__(256) double g_noalloc_part[kMaxVec * 32 * kMaxBlocks];

std::mutex g_mu;
double* g_part_addr[kMaxDevices] = {};

// ||F||_2 and mean(D) per vector from the two partial rows of the residual kernel.
__global__ void k_noalloc_finish(const double* __restrict__ part, int nblk, int mn,
                                 double* __restrict__ fnorm, double* __restrict__ dmean) {
  const int b = blockIdx.x;
  double sf = 0.0, sd = 0.0;
  for (int t = threadIdx.x; t < nblk; t += 32) {
    sf += part[((size_t)b * 32 + 0) * nblk + t];
    sd += part[((size_t)b * 32 + 1) * nblk + t];
  }
  sf = warp_sum(sf);
  sd = warp_sum(sd);
  if (threadIdx.x == 0) {
    if (fnorm) fnorm[b] = sqrt(sf);
    if (dmean) dmean[b] = sd / (double)mn;
  }
}

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MCA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_part_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
    if (e != cudaSuccess || p == nullptr) {
      set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_part)", __FILE__, __LINE__);
      return MCA_ERR_CUDA;
    }
    g_part_addr[dev] = static_cast<double*>(p);
  }
  *out = g_part_addr[dev];
  return MCA_OK;
}

}  // namespace

}  // namespace mca

using namespace mca;

extern "C" int mca_residual_noalloc(const mca_params* p, const double* g_map, const double* x,
                                    const double* v_in, int32_t nvec, double* F, double* D,
                                    double* fnorm, double* dmean, void* stream) {
  clear_error_message();
  if (!p || !g_map || !x || !v_in || !F || !D) {
    set_error_message("mca_residual_noalloc: NULL argument");
    return MCA_ERR_INVALID_ARG;
  }
  // the same circuit checks as mca_create (sizes, conductances, b, device model)
  if (validate_circuit(p) != MCA_OK) return MCA_ERR_INVALID_ARG;
  if (nvec < 1 || nvec > kMaxVec) {
    set_error_message("mca_residual_noalloc: nvec must be in 1..8 (size of the fixed scratch)");
    return MCA_ERR_INVALID_ARG;
  }
  double* part = nullptr;
  int rc = scratch_address(&part);
  if (rc != MCA_OK) return rc;
  const Grid gr = make_grid(*p);
  const int mn = gr.m * gr.n;
  const int nblk = residual_nblk(mn);
  if (nblk > kMaxBlocks) {   // the partial sums would not fit the fixed array
    set_error_message("mca_residual_noalloc: residual grid exceeds the fixed scratch");
    return MCA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_residual(gr, g_map, v_in, x, F, D, part, nblk, nvec, nullptr, s);
  count_launches(1);
  if (fnorm || dmean) {
    k_noalloc_finish<<<nvec, 32, 0, s>>>(part, nblk, mn, fnorm, dmean);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "mca_residual_noalloc launch", __FILE__, __LINE__);
    return MCA_ERR_CUDA;
  }
  return MCA_OK;
}
