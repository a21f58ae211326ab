// Host interface of the tcgen05 preconditioner GEMM (k_precond_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "mca_internal.cuh"

namespace mca {
namespace tc {

enum Epi {
  EPI_BF16 = 0,         // out = bf16(acc)
  EPI_MODES = 1,        // out = bf16(per-mode 2x2 inverse of eq. P applied to (acc_t, acc_b))
  EPI_SPLIT = 2,        // out = bf16(acc), out_lo = bf16(acc - out)
  EPI_F64 = 3,          // out = (double)acc for r < R_valid, c < C_valid (unpadded)
  EPI_F32 = 5,          // out = acc (float) for r < R_valid, c < C_valid (unpadded)
};

// Operand words of a GEMM: one BF16 word each (SPLIT_NONE); A and B both hi + lo, three
// products hi*hi + lo*hi + hi*lo (SPLIT_AB); only B hi + lo, two products A*hi + A*lo
// (SPLIT_B).
enum Split { SPLIT_NONE = 0, SPLIT_AB = 1, SPLIT_B = 2 };

// Output addressing: element (blk = 2b + layer, c, r) is written to
//   out[b*o_bs + layer*o_ls + c*o_ld + r].
struct GemmEpi {
  int R, K, C;              // padded extents: rows per block (x128), K (x64), cols (xBN)
  int R_valid, C_valid;     // logical extents
  void* out;
  void* out_lo;
  size_t o_bs, o_ls, o_ld;
  const double* mu;         // eigenvalue per r (EPI_MODES*)
  const double* nu;         // eigenvalue per c (EPI_MODES*)
  const float* mu_f;        // the same in FP32 (the epilogue arithmetic is FP32)
  const float* nu_f;
  const VecCtl* ctl;        // per-vector a and activity flag (NULL: all active)
  int kidx;                 // EPI_MODES*: scale the modes by ctl[b].s[kidx] (-1: none)
  int* err;                 // device status flag (MCA_ERR_TIMEOUT on an expired wait)
};

bool encode_available();
// box_k: 64 (single-word GEMMs) or 32 (split GEMMs)
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
              uint32_t box_rows, uint32_t box_k);
// 4-D map over an NHWC BF16 tensor with 32 channels, box = box_px pixels of one row
// (64-byte swizzle; out-of-range elements read zero)
bool make_map_nhwc32(CUtensorMap* map, const void* base, uint64_t W, uint64_t H, uint64_t N,
                     uint32_t box_px);
// The same tensor with a box of 8 channels x box_px pixels and no swizzle: each box lands as
// box_px consecutive 16-byte rows (one K chunk of a K-major operand without swizzling)
bool make_map_nhwc32_k8(CUtensorMap* map, const void* base, uint64_t W, uint64_t H, uint64_t N,
                        uint32_t box_px);
cudaError_t gemm(int bn, int split, int epi, const CUtensorMap& a, const CUtensorMap& al,
                 const CUtensorMap& bm, const CUtensorMap& bml, const GemmEpi& ep, int B,
                 cudaStream_t s);
// Persistent warp-specialised form: one CTA per SM over tiles of 128 x bn with lp layers
// (lp = 2 for the modes epilogues, which need both layers of a mode in one CTA); cg = 2:
// pairs of CTAs on two SMs over tiles of 256 x bn (bn = 256, lp = 1), B's maps with boxes
// of bn / 2 rows.
cudaError_t gemm_ws(int bn, int lp, int cg, int split, int epi, const CUtensorMap& a,
                    const CUtensorMap& al, const CUtensorMap& bm, const CUtensorMap& bml,
                    const GemmEpi& ep, int B, cudaStream_t s);
cudaError_t configure_all();
// After configure_all on this device: every two-SM instantiation can be launched.
bool pair_available();
cudaError_t wait_selftest(unsigned long long limit_ns, int* err, cudaStream_t s);
void cast_pad(const double* x, size_t xstride, __nv_bfloat16* xbf, int m, int n, int mp,
              int np, int B, cudaStream_t s);

}  // namespace tc
}  // namespace mca
