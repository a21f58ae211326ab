// Tensor-core form of the preconditioner apply z = P^-1 r (eqs. P, block, M; the
// tensor-product evaluation of Section 3.2 done in the exact Kronecker eigenbasis).
//
// Four block-transposed GEMMs O[blk][c][r] = sum_k A[blk][r][k] B[c][k] on tcgen05
// (kind::f16, BF16 operands, FP32 accumulators in TMEM), blk = 2*b + layer:
//   1: T1^T  = (X Q_r)^T            A = X      [blk][i][j]    B = Q_r^T  [k'][j]
//   2: Y_hat = modes^-1 (Q_c^T T1)  A = T1^T   [blk][k'][i]   B = Q_c^T  [i'][i]
//      (stored [blk][i'][k']; the per-mode 2x2 inverse of eq. P is the epilogue, which
//       needs both layers of one mode, so each CTA owns the two layers' tiles)
//   3: E^T   = (Y_hat Q_r^T)^T      A = Y_hat  [blk][i'][k']  B = Q_r    [j][k']
//   4: Z     = (E^T Q_c^T)^T        A = E^T    [blk][j][i']   B = Q_c    [i][i']
// Every operand is K-major, so TMA tiles land in the canonical 128-byte-swizzled layout
// the MMA descriptors expect, and every epilogue writes its tile transposed, which makes
// the TMEM lane = output row mapping store coalesced.
//
// Precision: the back transforms (3, 4) multiply the large amplified low modes of Y_hat.
// With MCA_PREC_BF16_SPLIT the eigenvector operands of both are split as hi + lo BF16
// pairs, so the rounding of Q does not leak the amplified low modes into the high ones.
// Transform 3's data operand Y_hat stays one BF16 word (its rounding changes each mode by
// 2^-9 of itself: two products, A*hi + A*lo), while transform 4's data operand E (modes
// along rows only) is split as well: three products hi*hi + lo*hi + hi*lo in one FP32
// tile.
//
// All device-side waits are bounded by a wall-clock limit; on expiry the CTA records
// MCA_ERR_TIMEOUT in a device flag, frees its TMEM and returns.
#include <atomic>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>

#include "bits.cuh"
#include "mca_internal.cuh"
#include "precond_tc.h"
#include "tc_ptx.cuh"

namespace mca {
namespace tc {

namespace {

constexpr int BM = 128;          // accumulator rows (TMEM lanes)
constexpr int BK = 64;           // K elements per stage with 128-byte swizzling
constexpr int BK_SPLIT = 32;     // split GEMMs: 64-byte swizzle rows, half-size stages
constexpr int kThreads = 128;    // 4 warps: TMA producer, MMA issuer, all 4 run the epilogue

template <int BKT>
__device__ __forceinline__ uint64_t tile_desc(const void* p) {
  return BKT == 64 ? sw128_desc(p) : sw64_desc(p);
}

// Shared-memory plan.  A configuration that fits two CTAs per SM (<= 110 KB) keeps two
// stages so one CTA's epilogue overlaps the other's main loop; otherwise one CTA uses up
// to ~200 KB of stages.  A staged BF16 epilogue reuses the stage buffers (2 or 4 output
// tiles of 128 x BN), which sets the floor on their size.  Split GEMMs use 32-wide K
// tiles (64-byte swizzle) to make their stages small enough to pair up.
template <int BN, int SPLIT, int EPI>
struct Layout {
  static constexpr int BKT = SPLIT ? BK_SPLIT : BK;
  static constexpr int A_BYTES = BM * BKT * 2;
  static constexpr int B_BYTES = BN * BKT * 2;
  static constexpr int HALF = 2 * A_BYTES + B_BYTES;       // hi words: 2 layers of A, B
  static constexpr int STAGE = SPLIT == SPLIT_AB ? 2 * HALF :
                               (SPLIT == SPLIT_B ? HALF + B_BYTES : HALF);
  static constexpr int STAGE_OUT = (EPI == EPI_F64 || EPI == EPI_F32) ? 0 :
      (EPI == EPI_SPLIT ? 4 : 2) * BN * BM * 2;
  static constexpr int STAGES_MIN = (STAGE_OUT + STAGE - 1) / STAGE;
  static constexpr int STAGES_2 = STAGES_MIN > 2 ? STAGES_MIN : 2;
  static constexpr int CTAS = (STAGES_2 * STAGE <= 110 * 1024) ? 2 : 1;
  static constexpr int STAGES_1 = (200 * 1024) / STAGE;
  static constexpr int STAGES = (CTAS == 2) ? STAGES_2 : (STAGES_1 > STAGES_MIN ? STAGES_1 : STAGES_MIN);
  static constexpr int BAR_OFF = STAGES * STAGE;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;  // barriers + TMEM slot + alignment
  static constexpr int TMEM_COLS = (2 * BN < 32) ? 32 : 2 * BN;
};

// Instantiations of the persistent kernel (BN, SPLIT, EPI, LP).
#define MCA_WS_LIST(X)                    \
  X(128, SPLIT_NONE, EPI_BF16, 1, 1)      \
  X(256, SPLIT_NONE, EPI_BF16, 1, 1)      \
  X(64, SPLIT_NONE, EPI_MODES, 2, 1)      \
  X(128, SPLIT_NONE, EPI_MODES, 2, 1)     \
  X(128, SPLIT_B, EPI_SPLIT, 1, 1)        \
  X(256, SPLIT_B, EPI_SPLIT, 1, 1)        \
  X(128, SPLIT_NONE, EPI_F64, 1, 1)       \
  X(256, SPLIT_NONE, EPI_F64, 1, 1)       \
  X(128, SPLIT_AB, EPI_F64, 1, 1)         \
  X(256, SPLIT_AB, EPI_F64, 1, 1)         \
  X(128, SPLIT_NONE, EPI_F32, 1, 1)       \
  X(256, SPLIT_NONE, EPI_F32, 1, 1)       \
  X(128, SPLIT_AB, EPI_F32, 1, 1)         \
  X(256, SPLIT_AB, EPI_F32, 1, 1)         \
  X(256, SPLIT_NONE, EPI_BF16, 1, 2)      \
  X(256, SPLIT_B, EPI_SPLIT, 1, 2)        \
  X(256, SPLIT_NONE, EPI_F64, 1, 2)       \
  X(256, SPLIT_AB, EPI_F64, 1, 2)         \
  X(256, SPLIT_NONE, EPI_F32, 1, 2)       \
  X(256, SPLIT_AB, EPI_F32, 1, 2)

// Instantiations of the one-CTA-per-tile kernel (BN, SPLIT, EPI).
#define MCA_TC_LIST(X)                 \
  X(128, SPLIT_NONE, EPI_BF16)         \
  X(64, SPLIT_NONE, EPI_BF16)          \
  X(128, SPLIT_NONE, EPI_MODES)        \
  X(64, SPLIT_NONE, EPI_MODES)         \
  X(128, SPLIT_NONE, EPI_F64)          \
  X(64, SPLIT_NONE, EPI_F64)           \
  X(128, SPLIT_B, EPI_SPLIT)           \
  X(64, SPLIT_B, EPI_SPLIT)            \
  X(128, SPLIT_AB, EPI_F64)            \
  X(64, SPLIT_AB, EPI_F64)             \
  X(128, SPLIT_NONE, EPI_F32)          \
  X(64, SPLIT_NONE, EPI_F32)           \
  X(128, SPLIT_AB, EPI_F32)            \
  X(64, SPLIT_AB, EPI_F32)

template <int BN, int SPLIT, int EPI>
__global__ void __launch_bounds__(kThreads, Layout<BN, SPLIT, EPI>::CTAS)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAl,
          const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBl,
          GemmEpi ep) {
  using L = Layout<BN, SPLIT, EPI>;
  const int rt = blockIdx.x, ct = blockIdx.y, b = blockIdx.z;
  if (ep.ctl != nullptr && !ep.ctl[b].gm_active) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + L::STAGES;
  uint64_t* accum = empty + L::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = rt * BM, c0 = ct * BN;
  const int blk0 = 2 * b, blk1 = 2 * b + 1;
  constexpr int BKT = L::BKT;
  const int nkb = ep.K / BKT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < L::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % L::STAGES;
      const uint32_t ph = (uint32_t)(kb / L::STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        record_error(ep.err, MCA_ERR_TIMEOUT);
        break;
      }
      uint8_t* st = smem + s * L::STAGE;
      mbar_expect_tx(&full[s], (uint32_t)L::STAGE);
      const int k0 = kb * BKT;
      tma_load_2d(st, &tmA, k0, blk0 * ep.R + r0, &full[s]);
      tma_load_2d(st + L::A_BYTES, &tmA, k0, blk1 * ep.R + r0, &full[s]);
      tma_load_2d(st + 2 * L::A_BYTES, &tmB, k0, c0, &full[s]);
      if (SPLIT == SPLIT_AB) {
        uint8_t* sl = st + L::HALF;
        tma_load_2d(sl, &tmAl, k0, blk0 * ep.R + r0, &full[s]);
        tma_load_2d(sl + L::A_BYTES, &tmAl, k0, blk1 * ep.R + r0, &full[s]);
        tma_load_2d(sl + 2 * L::A_BYTES, &tmBl, k0, c0, &full[s]);
      } else if (SPLIT == SPLIT_B) {
        tma_load_2d(st + L::HALF, &tmBl, k0, c0, &full[s]);
      }
    }
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer (one thread)
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % L::STAGES;
      const uint32_t ph = (uint32_t)(kb / L::STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        record_error(ep.err, MCA_ERR_TIMEOUT);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint8_t* st = smem + s * L::STAGE;
#pragma unroll
      for (int kk = 0; kk < BKT / 16; ++kk) {
        const int off = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzle row
        const uint64_t a0 = tile_desc<BKT>(st + off);
        const uint64_t a1 = tile_desc<BKT>(st + L::A_BYTES + off);
        const uint64_t bd = tile_desc<BKT>(st + 2 * L::A_BYTES + off);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        umma(tmem, a0, bd, idesc, acc);
        umma(tmem + BN, a1, bd, idesc, acc);
        if (SPLIT == SPLIT_AB) {
          const uint8_t* sl = st + L::HALF;
          const uint64_t a0l = tile_desc<BKT>(sl + off);
          const uint64_t a1l = tile_desc<BKT>(sl + L::A_BYTES + off);
          const uint64_t bdl = tile_desc<BKT>(sl + 2 * L::A_BYTES + off);
          umma(tmem, a0l, bd, idesc, 1u);
          umma(tmem, a0, bdl, idesc, 1u);
          umma(tmem + BN, a1l, bd, idesc, 1u);
          umma(tmem + BN, a1, bdl, idesc, 1u);
        } else if (SPLIT == SPLIT_B) {
          const uint64_t bdl = tile_desc<BKT>(st + L::HALF + off);
          umma(tmem, a0, bdl, idesc, 1u);
          umma(tmem + BN, a1, bdl, idesc, 1u);
        }
      }
      umma_commit(&empty[s]);
    }
    if (ok) umma_commit(accum);
  }
  __syncwarp();

  // ---------------- epilogue: thread = TMEM lane = output row r0 + 32*warp + lane
  // (the vote makes a timed-out wait uniform, so every thread meets the same barriers)
  const bool have = __syncthreads_and(mbar_wait(accum, 0) ? 1 : 0) != 0;
  if (!have && threadIdx.x == 0) record_error(ep.err, MCA_ERR_TIMEOUT);
  constexpr bool kBf16Out = (EPI != EPI_F64 && EPI != EPI_F32);
  constexpr bool kLo = (EPI == EPI_SPLIT);
  constexpr int kOuts = kLo ? 4 : 2;            // [hi t, hi b, lo t, lo b]
  // BF16 outputs are staged transposed in the (now idle) pipeline buffers as
  // stage[o][c][r] and leave in 16-byte chunks along r; FP64 outputs go straight out
  // (one 8-byte store per thread and column is already a full 256-byte warp segment).
  __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(smem);
  static_assert(!kBf16Out || kOuts * BN * BM * 2 <= L::BAR_OFF, "staging exceeds smem");
  if (have) {
    tc_fence_after();
    const int rl = warp * 32 + lane;             // row inside the tile
    const int r = r0 + rl;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float a_mode = 0.f, mu_r = 0.f;
    const bool r_ok = r < ep.R_valid;
    float sc = 1.f;          // scale of the unnormalised input basis vector
    if (EPI == EPI_MODES) {
      a_mode = (float)ep.ctl[b].a;
      mu_r = r_ok ? ep.mu_f[r] : 0.f;
      if (ep.kidx >= 0) sc = (float)ep.ctl[b].s[ep.kidx];
    }
#pragma unroll 1
    for (int cc = 0; cc < BN / 32; ++cc) {
      uint32_t v0[32], v1[32];
      tmem_ld32(lane_base + cc * 32, v0);
      tmem_ld32(lane_base + BN + cc * 32, v1);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int cl = cc * 32 + q;
        const int c = c0 + cl;
        float x0 = __uint_as_float(v0[q]);
        float x1 = __uint_as_float(v1[q]);
        if (EPI == EPI_MODES) {
          // [y_t; y_b] = (1/det) [[nu + a, a], [a, mu + a]] [x_t; x_b]
          float y0 = 0.f, y1 = 0.f;
          if (r_ok && c < ep.C_valid) {
            const float nu_c = ep.nu_f[c];
            const float det = mu_r * nu_c + mu_r * a_mode + nu_c * a_mode;
            const float inv = sc * __frcp_rn(det);
            y0 = ((nu_c + a_mode) * x0 + a_mode * x1) * inv;
            y1 = (a_mode * x0 + (mu_r + a_mode) * x1) * inv;
          }
          x0 = y0;
          x1 = y1;
        }
        if (EPI == EPI_F64) {
          if (r_ok && c < ep.C_valid) {
            const size_t o0 = (size_t)b * ep.o_bs + (size_t)c * ep.o_ld + r;
            double* out = static_cast<double*>(ep.out);
            out[o0] = f2d_bits(x0);
            out[o0 + ep.o_ls] = f2d_bits(x1);
          }
        } else if (EPI == EPI_F32) {
          if (r_ok && c < ep.C_valid) {
            const size_t o0 = (size_t)b * ep.o_bs + (size_t)c * ep.o_ld + r;
            float* out = static_cast<float*>(ep.out);
            out[o0] = x0;
            out[o0 + ep.o_ls] = x1;
          }
        } else {
          const __nv_bfloat16 h0 = __float2bfloat16(x0);
          const __nv_bfloat16 h1 = __float2bfloat16(x1);
          stage[((size_t)0 * BN + cl) * BM + rl] = h0;
          stage[((size_t)1 * BN + cl) * BM + rl] = h1;
          if (kLo) {
            stage[((size_t)2 * BN + cl) * BM + rl] = __float2bfloat16(x0 - __bfloat162float(h0));
            stage[((size_t)3 * BN + cl) * BM + rl] = __float2bfloat16(x1 - __bfloat162float(h1));
          }
        }
      }
    }
  }
  if (kBf16Out) {
    __syncthreads();
    if (have) {
      // 16-byte chunks: 16 per staged column of 128 rows; thread t takes t, t + 128, ...
      constexpr int kChunks = BN * (BM / 8);
#pragma unroll 1
      for (int o = 0; o < kOuts; ++o) {
        __nv_bfloat16* out = static_cast<__nv_bfloat16*>((o < 2) ? ep.out : ep.out_lo);
        const size_t base = (size_t)b * ep.o_bs + (size_t)(o & 1) * ep.o_ls + r0;
        for (int q = threadIdx.x; q < kChunks; q += kThreads) {
          const int cl = q >> 4, rc = (q & 15) * 8;
          const uint4 v = *reinterpret_cast<const uint4*>(&stage[((size_t)o * BN + cl) * BM + rc]);
          *reinterpret_cast<uint4*>(&out[base + (size_t)(c0 + cl) * ep.o_ld + rc]) = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)L::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------------------
// Persistent, warp-specialised form of the same GEMMs.  One CTA per SM walks a static
// round-robin list of output tiles; warp 0 streams A/B stages with TMA, warp 1 issues the
// MMAs into one of two TMEM accumulators, and the epilogue warps drain the other
// accumulator (the epilogue of tile i overlaps the main loop of tile i + 1).  There are 8
// epilogue warps (16 for the two-layer tiles, whose modes epilogue does the most work per
// element): 2 or 4 per TMEM lane quarter, each taking every 2nd or 4th column chunk.  A tile is 128 rows x BN
// columns of LP layers: LP = 2 keeps both layers of a mode in one CTA (required by the
// per-mode 2x2 epilogue), LP = 1 makes twice as many single-layer tiles (better balance
// of the tiles over the SMs).  BF16 outputs are transposed through a small staging tile per
// epilogue warp, one output at a time, and leave in 16-byte chunks.
//
// CG = 2: a cluster of two CTAs on two SMs computes one 256 x BN tile of one layer with
// pair MMAs (cta_group::2).  Each CTA loads its 128 rows of A and half of B's BN rows, so a
// stage carries a third fewer bytes per MMA than with CG = 1 and more stages fit; each
// CTA's TMEM holds its 128 output rows.  Both CTAs' TMA loads of a stage complete on the
// even CTA's stage barrier, which expects the bytes of both; the even CTA's thread issues
// the MMAs; their completions arrive at both CTAs' barriers (multicast commit); the odd
// CTA's epilogue warps report a drained accumulator to the even CTA.
constexpr int kWsSmemMax = 227 * 1024;

template <int BN, int SPLIT, int EPI, int LP, int CG = 1>
struct WsLayout {
  static_assert(CG == 1 || (CG == 2 && LP == 1), "CTA pairs take single-layer tiles");
  static constexpr int BKT = SPLIT ? BK_SPLIT : BK;
  static constexpr int A_BYTES = BM * BKT * 2;
  static constexpr int B_BYTES = (BN / CG) * BKT * 2;      // this CTA's rows of B
  static constexpr int HALF = LP * A_BYTES + B_BYTES;      // hi words: LP layers of A, B
  static constexpr int STAGE = SPLIT == SPLIT_AB ? 2 * HALF :
                               (SPLIT == SPLIT_B ? HALF + B_BYTES : HALF);
  static constexpr bool LO = (EPI == EPI_SPLIT);
  static constexpr int NOUT = (EPI == EPI_F64 || EPI == EPI_F32) ? 0 : (LO ? 2 : 1) * LP;
  static constexpr int EW = (LP == 2) ? 16 : 8;                           // epilogue warps
  static constexpr int THREADS = 64 + 32 * EW;
  static constexpr int CW = (LP == 2) ? 16 : 32;            // columns per TMEM load/chunk
  static constexpr int STG_WARP = NOUT > 0 ? CW * 32 * 2 : 0;             // bytes per warp
  static constexpr int FIXED = EW * STG_WARP + 512 + 1024;                // + barriers, align
  static constexpr int STAGES_FIT = (kWsSmemMax - FIXED) / STAGE;
  static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
  static constexpr int STG_OFF = STAGES * STAGE;
  static constexpr int BAR_OFF = STG_OFF + EW * STG_WARP;
  static constexpr int SMEM = BAR_OFF + 512 + 1024;
  static constexpr int ACC_COLS = LP * BN;                                // one accumulator
  static constexpr int TMEM_COLS = 2 * ACC_COLS < 32 ? 32 : 2 * ACC_COLS;
  static_assert(STAGES >= 2, "not enough shared memory for two stages");
  static_assert(2 * ACC_COLS <= 512, "two accumulators must fit in TMEM");
  static_assert(SMEM <= kWsSmemMax, "shared memory plan too large");
};

template <int CG>
__device__ __forceinline__ void umma_cg(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  if constexpr (CG == 2) umma_pair(d, a, b, idesc, acc); else umma(d, a, b, idesc, acc);
}

template <int CG>
__device__ __forceinline__ void commit_cg(uint64_t* bar) {
  if constexpr (CG == 2) umma_commit_pair(bar); else umma_commit(bar);
}

template <int BN, int SPLIT, int EPI, int LP, int CG>
__global__ void __launch_bounds__(WsLayout<BN, SPLIT, EPI, LP, CG>::THREADS, 1)
k_gemm_ws(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAl,
          const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBl,
          GemmEpi ep, int B) {
  using L = WsLayout<BN, SPLIT, EPI, LP, CG>;
  static_assert(LP == 2 || EPI != EPI_MODES, "the modes epilogue needs both layers in one tile");
  constexpr int BKT = L::BKT;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* empty = full + L::STAGES;
  uint64_t* tfull = empty + L::STAGES;           // [2] accumulator ready
  uint64_t* tempty = tfull + 2;                  // [2] accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CG = 2: this CTA's rank in the pair; the even CTA issues the MMAs
  const uint32_t rank = (CG == 2) ? cluster_ctarank() : 0u;
  const bool issuer = (rank == 0);
  const int first = (CG == 2) ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int step = (CG == 2) ? (int)(gridDim.x >> 1) : (int)gridDim.x;

  // tiles (of BM * CG rows): column tile fastest (neighbouring CTAs share their A rows in
  // L2), then row tile, then layer (LP = 1), then vector
  const int tr = ep.R / (BM * CG), tc = ep.C / BN;
  const int per_vec = tr * tc * (LP == 1 ? 2 : 1);
  const int ntiles = per_vec * B;
  const int nkb = ep.K / BKT;
  auto decode = [&](int t, int& b, int& layer, int& r0, int& c0) {
    b = t / per_vec;
    int u = t - b * per_vec;
    layer = 0;
    if (LP == 1) {
      layer = u / (tr * tc);
      u -= layer * tr * tc;
    }
    r0 = (u / tc) * (BM * CG);
    c0 = (u % tc) * BN;
  };
  auto active = [&](int b) { return ep.ctl == nullptr || ep.ctl[b].gm_active; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < L::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], L::EW * CG);        // CG = 2: both CTAs' epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // CG = 2: one warp of each CTA allocates the same columns in both
    if (CG == 2) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"((uint32_t)L::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"((uint32_t)L::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (CG == 2) cluster_sync();      // both CTAs' barriers initialised before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer (one thread)
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = first; t < ntiles && ok; t += step) {
        int b, layer, r0, c0;
        decode(t, b, layer, r0, c0);
        if (!active(b)) continue;
        // first A row (layer 0 of LP = 2; this CTA's half of a pair tile)
        const int row0 = (2 * b + layer) * ep.R + r0 + (int)rank * BM;
        const int cb = c0 + (int)rank * (BN / CG);        // this CTA's rows of B
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % L::STAGES;
          const uint32_t ph = (uint32_t)(it / L::STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u)) {
            record_error(ep.err, MCA_ERR_TIMEOUT);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * L::STAGE;
          const int k0 = kb * BKT;
          if (CG == 2) {
            // both CTAs' bytes complete on the even CTA's barrier, which expects them all
            if (issuer) mbar_expect_tx(&full[s], (uint32_t)(2 * L::STAGE));
            const uint32_t bar = peer_addr(&full[s], 0);
            tma_load_2d_pair(st, &tmA, k0, row0, bar);
            tma_load_2d_pair(st + L::A_BYTES, &tmB, k0, cb, bar);
            if (SPLIT == SPLIT_AB) {
              tma_load_2d_pair(st + L::HALF, &tmAl, k0, row0, bar);
              tma_load_2d_pair(st + L::HALF + L::A_BYTES, &tmBl, k0, cb, bar);
            } else if (SPLIT == SPLIT_B) {
              tma_load_2d_pair(st + L::HALF, &tmBl, k0, cb, bar);
            }
            continue;
          }
          mbar_expect_tx(&full[s], (uint32_t)L::STAGE);
#pragma unroll
          for (int l = 0; l < LP; ++l)
            tma_load_2d(st + l * L::A_BYTES, &tmA, k0, row0 + l * ep.R, &full[s]);
          tma_load_2d(st + LP * L::A_BYTES, &tmB, k0, cb, &full[s]);
          if (SPLIT == SPLIT_AB) {
            uint8_t* sl = st + L::HALF;
#pragma unroll
            for (int l = 0; l < LP; ++l)
              tma_load_2d(sl + l * L::A_BYTES, &tmAl, k0, row0 + l * ep.R, &full[s]);
            tma_load_2d(sl + LP * L::A_BYTES, &tmBl, k0, cb, &full[s]);
          } else if (SPLIT == SPLIT_B) {
            tma_load_2d(st + L::HALF, &tmBl, k0, cb, &full[s]);
          }
        }
      }
      if (CG == 2 && ok) {
        // the pair MMAs' completions still due to arrive at this CTA's stage barriers: wait
        // for them, so that no arrive reaches a CTA that has exited
        for (int i = 0; i < L::STAGES; ++i, ++it) {
          if (!mbar_wait(&empty[it % L::STAGES], ((uint32_t)(it / L::STAGES) & 1u) ^ 1u)) {
            record_error(ep.err, MCA_ERR_TIMEOUT);
            break;
          }
        }
      }
    }
  } else if (warp == 1 && !issuer) {
    // CG = 2, odd CTA: the even CTA's thread issues the pair's MMAs
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM * CG, BN);
      int it = 0, tl = 0;
      bool ok = true;
      for (int t = first; t < ntiles && ok; t += step) {
        int b, layer, r0, c0;
        decode(t, b, layer, r0, c0);
        if (!active(b)) continue;
        const int acc = tl & 1;
        const uint32_t aph = (uint32_t)(tl >> 1) & 1u;
        if (!(CG == 2 ? mbar_wait_cluster(&tempty[acc], aph ^ 1u)
                      : mbar_wait(&tempty[acc], aph ^ 1u))) {
          record_error(ep.err, MCA_ERR_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(acc * L::ACC_COLS);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % L::STAGES;
          const uint32_t ph = (uint32_t)(it / L::STAGES) & 1u;
          if (!mbar_wait(&full[s], ph)) {
            record_error(ep.err, MCA_ERR_TIMEOUT);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint8_t* st = smem + s * L::STAGE;
#pragma unroll
          for (int kk = 0; kk < BKT / 16; ++kk) {
            const int off = kk * 32;
            const uint64_t bd = tile_desc<BKT>(st + LP * L::A_BYTES + off);
            const uint32_t accf = (kb > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
            for (int l = 0; l < LP; ++l) {
              const uint64_t ad = tile_desc<BKT>(st + l * L::A_BYTES + off);
              umma_cg<CG>(dacc + l * BN, ad, bd, idesc, accf);
              if (SPLIT == SPLIT_AB) {
                const uint8_t* sl = st + L::HALF;
                const uint64_t adl = tile_desc<BKT>(sl + l * L::A_BYTES + off);
                const uint64_t bdl = tile_desc<BKT>(sl + LP * L::A_BYTES + off);
                umma_cg<CG>(dacc + l * BN, adl, bd, idesc, 1u);
                umma_cg<CG>(dacc + l * BN, ad, bdl, idesc, 1u);
              } else if (SPLIT == SPLIT_B) {
                umma_cg<CG>(dacc + l * BN, ad, tile_desc<BKT>(st + L::HALF + off), idesc, 1u);
              }
            }
          }
          commit_cg<CG>(&empty[s]);
        }
        if (!ok) break;
        commit_cg<CG>(&tfull[acc]);
        ++tl;
      }
    }
  } else {
    // ---------------- epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 and
    // the CW-column chunks cc with cc % NG == (w - 2) / 4, NG = EW / 4
    constexpr int NG = L::EW / 4;
    constexpr int CW = L::CW;
    const int q = warp & 3;
    const int grp = (warp - 2) >> 2;
    const int rl = q * 32 + lane;                    // row inside the tile
    __nv_bfloat16* stg =
        reinterpret_cast<__nv_bfloat16*>(smem + L::STG_OFF + (warp - 2) * L::STG_WARP);
    int tl = 0;
    for (int t = first; t < ntiles; t += step) {
      int b, layer, r0, c0;
      decode(t, b, layer, r0, c0);
      if (!active(b)) continue;
      const int acc = tl & 1;
      const uint32_t aph = (uint32_t)(tl >> 1) & 1u;
      const bool have = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], aph) ? 1 : 0) != 0;
      if (!have) {
        if (lane == 0) record_error(ep.err, MCA_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const int r = r0 + (int)rank * BM + rl;
      const bool r_ok = r < ep.R_valid;
      const uint32_t lane_base =
          tmem + (uint32_t)(acc * L::ACC_COLS) + ((uint32_t)(q * 32) << 16);
      float a_mode = 0.f, mu_a = 0.f, a2 = 0.f, sc = 1.f;
      if (EPI == EPI_MODES) {
        a_mode = (float)ep.ctl[b].a;
        mu_a = (r_ok ? ep.mu_f[r] : 0.f) + a_mode;
        a2 = a_mode * a_mode;
        if (ep.kidx >= 0) sc = (float)ep.ctl[b].s[ep.kidx];
      }
#pragma unroll 1
      for (int cc = grp; cc < BN / CW; cc += NG) {
        uint32_t v0[CW], v1[CW];
        tmem_ld<CW>(lane_base + cc * CW, v0);
        if (LP == 2) tmem_ld<CW>(lane_base + BN + cc * CW, v1);
        if (EPI == EPI_F64 || EPI == EPI_F32) {
          // unpadded FP64 or FP32 output: one full warp segment per column
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            const int c = c0 + cc * CW + j;
            if (r_ok && c < ep.C_valid) {
#pragma unroll
              for (int l = 0; l < LP; ++l) {
                const size_t o = (size_t)b * ep.o_bs + (size_t)(layer + l) * ep.o_ls +
                                 (size_t)c * ep.o_ld + r;
                const uint32_t v = (l == 0) ? v0[j] : v1[j];
                if (EPI == EPI_F64)
                  static_cast<double*>(ep.out)[o] = f2d_bits(__uint_as_float(v));
                else
                  static_cast<float*>(ep.out)[o] = __uint_as_float(v);
              }
            }
          }
        } else {
          if (EPI == EPI_MODES) {
            // [y_t; y_b] = (sc / det) [[nu + a, a], [a, mu + a]] [x_t; x_b] in place,
            // det = (mu + a)(nu + a) - a^2; the column eigenvalues come in with one
            // coalesced load and a shuffle per column
            const int cl = c0 + cc * CW + lane;
            const float nu_l = (lane < CW && cl < ep.C_valid) ? ep.nu_f[cl] : 0.f;
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int c = c0 + cc * CW + j;
              const float nu_a = __shfl_sync(0xffffffffu, nu_l, j) + a_mode;
              float y0 = 0.f, y1 = 0.f;
              if (r_ok && c < ep.C_valid) {
                const float x0 = __uint_as_float(v0[j]), x1 = __uint_as_float(v1[j]);
                // (approximate reciprocal: a few FP32 ulps, far below the BF16 outputs)
                const float inv = __fdividef(sc, fmaf(mu_a, nu_a, -a2));
                y0 = fmaf(nu_a, x0, a_mode * x1) * inv;
                y1 = fmaf(mu_a, x1, a_mode * x0) * inv;
              }
              v0[j] = __float_as_uint(y0);
              v1[j] = __float_as_uint(y1);
            }
          }
          // one output at a time through this warp's [CW columns][32 rows] staging tile,
          // then 4 chunks of 16 bytes per column (64 bytes of rows)
#pragma unroll 1
          for (int o = 0; o < L::NOUT; ++o) {
            const int l = o % LP;
            const bool lo = o >= LP;
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const float x = __uint_as_float((LP == 2 && l == 1) ? v1[j] : v0[j]);
              const __nv_bfloat16 hi = __float2bfloat16(x);
              stg[j * 32 + lane] = lo ? __float2bfloat16(x - __bfloat162float(hi)) : hi;
            }
            __syncwarp();
            __nv_bfloat16* out = static_cast<__nv_bfloat16*>(lo ? ep.out_lo : ep.out);
            const size_t base = (size_t)b * ep.o_bs + (size_t)(layer + l) * ep.o_ls + r0 +
                                (int)rank * BM + q * 32;
#pragma unroll
            for (int i = 0; i < CW / 8; ++i) {
              const int id = lane + 32 * i;
              const int col = id >> 2, part = id & 3;
              const uint4 v = *reinterpret_cast<const uint4*>(&stg[col * 32 + part * 8]);
              *reinterpret_cast<uint4*>(
                  &out[base + (size_t)(c0 + cc * CW + col) * ep.o_ld + part * 8]) = v;
            }
            __syncwarp();
          }
        }
      }
      // accumulator drained: the MMA warp may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (CG == 2 && !issuer)
          mbar_arrive_cluster(peer_addr(&tempty[acc], 0));
        else
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc]))
                       : "memory");
      }
      ++tl;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (CG == 2) cluster_sync();      // no remote arrive or pair MMA still due at either CTA
  if (warp == 1) {
    tc_fence_after();
    if (CG == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"((uint32_t)L::TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"((uint32_t)L::TMEM_COLS)
                   : "memory");
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives at,
// with a limit of limit_ns, and records MCA_ERR_TIMEOUT when the wait gives up.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    bool ok = false;
    while (!(ok = mbar_try_wait(&bar, 0))) {
      if (global_ns() - t0 > limit_ns) break;
    }
    if (!ok) record_error(err, MCA_ERR_TIMEOUT);
  }
}

// FP64 [b][layer][m][n] -> BF16 padded [b][layer][mp][np] (the pads stay zero).
__global__ void k_cast_pad(const double* __restrict__ x, size_t xstride,
                           __nv_bfloat16* __restrict__ xbf, int m, int n, int mp, int np) {
  const int b = blockIdx.y;
  const size_t mn = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * mn;
       e += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(e / mn);
    const size_t cell = e - l * mn;
    const int i = (int)(cell / n), j = (int)(cell - (size_t)i * n);
    xbf[(((size_t)b * 2 + l) * mp + i) * np + j] = __double2bfloat16(x[b * xstride + e]);
  }
}

template <int BN, int SPLIT, int EPI>
cudaError_t launch_one(const CUtensorMap& a, const CUtensorMap& al, const CUtensorMap& bm,
                       const CUtensorMap& bml, const GemmEpi& ep, int B, cudaStream_t s) {
  using L = Layout<BN, SPLIT, EPI>;
  auto kern = k_gemm_tc<BN, SPLIT, EPI>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L::SMEM);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(ep.R / BM, ep.C / BN, B);
  kern<<<grid, kThreads, L::SMEM, s>>>(a, al, bm, bml, ep);
  return cudaGetLastError();
}

// SM count per device ordinal, set on first use there; atomic because handles may be
// used from several host threads
constexpr int kMaxDevices = 64;
std::atomic<int> g_num_sms[kMaxDevices] = {};

// Co-resident two-CTA clusters of each pair instantiation per device ordinal (set by
// configure_all before any launch, 0 = not known: the launch is refused).
template <int BN, int SPLIT, int EPI, int LP, int CG>
std::atomic<int> g_pair_clusters[kMaxDevices] = {};

template <int BN, int SPLIT, int EPI, int LP, int CG>
cudaLaunchConfig_t pair_config(int grid, cudaStream_t s, cudaLaunchAttribute* at) {
  using L = WsLayout<BN, SPLIT, EPI, LP, CG>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(L::THREADS, 1, 1);
  cfg.dynamicSmemBytes = L::SMEM;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <int BN, int SPLIT, int EPI, int LP, int CG>
cudaError_t launch_ws(const CUtensorMap& a, const CUtensorMap& al, const CUtensorMap& bm,
                      const CUtensorMap& bml, const GemmEpi& ep, int B, cudaStream_t s) {
  using L = WsLayout<BN, SPLIT, EPI, LP, CG>;
  if (ep.R % (BM * CG) != 0 || ep.C % BN != 0 || ep.K % L::BKT != 0)
    return cudaErrorInvalidValue;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return cudaErrorInvalidValue;
  int nsm = g_num_sms[dev].load(std::memory_order_relaxed);
  if (nsm <= 0) {
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm <= 0)
      return cudaErrorInvalidValue;
    g_num_sms[dev].store(nsm, std::memory_order_relaxed);
  }
  const int ntiles = (ep.R / (BM * CG)) * (ep.C / BN) * (LP == 1 ? 2 : 1) * B;
  if (CG == 2) {
    // one cluster per co-resident pair of SMs, each walking the pair tiles
    const int ncl = g_pair_clusters<BN, SPLIT, EPI, LP, CG>[dev].load(std::memory_order_relaxed);
    if (ncl <= 0) return cudaErrorInvalidValue;
    const int grid = 2 * (ntiles < ncl ? ntiles : ncl);
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = pair_config<BN, SPLIT, EPI, LP, CG>(grid, s, at);
    return cudaLaunchKernelEx(&cfg, k_gemm_ws<BN, SPLIT, EPI, LP, CG>, a, al, bm, bml, ep, B);
  }
  const int grid = ntiles < nsm ? ntiles : nsm;
  k_gemm_ws<BN, SPLIT, EPI, LP, CG><<<grid, L::THREADS, L::SMEM, s>>>(a, al, bm, bml, ep, B);
  return cudaGetLastError();
}

std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

}  // namespace

bool encode_available() {
  if (g_encode.load()) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr)
    return false;
  g_encode.store(reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn));
  return true;
}

// 2-D BF16 map over a row-major [rows][cols] matrix with a box of box_rows x box_k
// elements: box_k = 64 with 128-byte swizzle, box_k = 32 with 64-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
              uint32_t box_rows, uint32_t box_k) {
  if (!encode_available()) return false;
  if (box_k != (uint32_t)BK && box_k != (uint32_t)BK_SPLIT) return false;
  cuuint64_t gdim[2] = {cols, rows};
  cuuint64_t gstride[1] = {cols * 2};
  cuuint32_t box[2] = {box_k, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode.load()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim,
                        gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_k == (uint32_t)BK ? CU_TENSOR_MAP_SWIZZLE_128B
                                              : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 4-D BF16 map over an NHWC activation tensor with 32 channels ([n][y][x][c], 64 bytes per
// pixel) and a box of box_px pixels of one row of one image, 64-byte swizzle (one pixel
// = one swizzle row).  Out-of-range boxes read zeros (the convolutions' padding).
bool make_map_nhwc32(CUtensorMap* map, const void* base, uint64_t W, uint64_t H, uint64_t N,
                     uint32_t box_px) {
  if (!encode_available() || box_px < 1 || box_px > 256) return false;
  cuuint64_t gdim[4] = {32, W, H, N};
  cuuint64_t gstride[3] = {64, 64 * W, 64 * W * H};
  cuuint32_t box[4] = {32, box_px, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode.load()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base),
                               gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_map_nhwc32_k8(CUtensorMap* map, const void* base, uint64_t W, uint64_t H, uint64_t N,
                        uint32_t box_px) {
  if (!encode_available() || box_px < 1 || box_px > 256) return false;
  cuuint64_t gdim[4] = {32, W, H, N};
  cuuint64_t gstride[3] = {64, 64 * W, 64 * W * H};
  cuuint32_t box[4] = {8, box_px, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode.load()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base),
                               gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t gemm(int bn, int split, int epi, const CUtensorMap& a, const CUtensorMap& al,
                 const CUtensorMap& bm, const CUtensorMap& bml, const GemmEpi& ep, int B,
                 cudaStream_t s) {
#define MCA_TC_CASE(BN_, SPLIT_, EPI_)                                       \
  if (bn == BN_ && split == SPLIT_ && epi == EPI_)                           \
    return launch_one<BN_, SPLIT_, EPI_>(a, al, bm, bml, ep, B, s);
  MCA_TC_LIST(MCA_TC_CASE)
#undef MCA_TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t gemm_ws(int bn, int lp, int cg, int split, int epi, const CUtensorMap& a,
                    const CUtensorMap& al, const CUtensorMap& bm, const CUtensorMap& bml,
                    const GemmEpi& ep, int B, cudaStream_t s) {
#define MCA_WS_CASE(BN_, SPLIT_, EPI_, LP_, CG_)                                  \
  if (bn == BN_ && split == SPLIT_ && epi == EPI_ && lp == LP_ && cg == CG_)      \
    return launch_ws<BN_, SPLIT_, EPI_, LP_, CG_>(a, al, bm, bml, ep, B, s);
  MCA_WS_LIST(MCA_WS_CASE)
#undef MCA_WS_CASE
  return cudaErrorInvalidValue;
}

// Set the dynamic shared-memory limit of every GEMM instantiation up front, so no
// attribute call happens later inside a stream capture.
cudaError_t configure_all() {
#define MCA_TC_CFG(BN_, SPLIT_, EPI_)                                                   \
  {                                                                                     \
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN_, SPLIT_, EPI_>,                  \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                         Layout<BN_, SPLIT_, EPI_>::SMEM);              \
    if (e != cudaSuccess) return e;                                                     \
  }
  MCA_TC_LIST(MCA_TC_CFG)
#undef MCA_TC_CFG
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return cudaErrorInvalidValue;
#define MCA_WS_CFG(BN_, SPLIT_, EPI_, LP_, CG_)                                        \
  {                                                                                    \
    auto kern = k_gemm_ws<BN_, SPLIT_, EPI_, LP_, CG_>;                                \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         WsLayout<BN_, SPLIT_, EPI_, LP_, CG_>::SMEM); \
    if (e != cudaSuccess) return e;                                                    \
    if (CG_ == 2) {                                                                    \
      cudaLaunchAttribute at[1];                                                       \
      const cudaLaunchConfig_t cfg = pair_config<BN_, SPLIT_, EPI_, LP_, CG_>(2, 0, at); \
      int ncl = 0;                                                                     \
      if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) {           \
        (void)cudaGetLastError();   /* no pair form on this device */                  \
        ncl = 0;                                                                       \
      }                                                                                \
      g_pair_clusters<BN_, SPLIT_, EPI_, LP_, CG_>[dev].store(ncl);                    \
    }                                                                                  \
  }
  MCA_WS_LIST(MCA_WS_CFG)
#undef MCA_WS_CFG
  return cudaSuccess;
}

bool pair_available() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  bool ok = true;
#define MCA_WS_PAIR_OK(BN_, SPLIT_, EPI_, LP_, CG_) \
  if (CG_ == 2) ok = ok && g_pair_clusters<BN_, SPLIT_, EPI_, LP_, CG_>[dev].load() > 0;
  MCA_WS_LIST(MCA_WS_PAIR_OK)
#undef MCA_WS_PAIR_OK
  return ok;
}

cudaError_t wait_selftest(unsigned long long limit_ns, int* err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, err);
  return cudaGetLastError();
}

void cast_pad(const double* x, size_t xstride, __nv_bfloat16* xbf, int m, int n, int mp,
              int np, int B, cudaStream_t s) {
  const size_t n2 = 2 * (size_t)m * n;
  int nb = (int)((n2 + 255) / 256);
  if (nb > 1216) nb = 1216;
  k_cast_pad<<<dim3(nb, B), 256, 0, s>>>(x, xstride, xbf, m, n, mp, np);
}

}  // namespace tc
}  // namespace mca
