// Persistent whole-solve kernel for batches of independent crossbar solves (the
// statistical-characterisation workload: many crossbars of several shapes, several input
// vectors each).  One CTA runs the complete solve of one (crossbar, input vector) work item:
// Newton on eq. (F) with the Eisenstat-Walker forcing terms of eq. (Newton3), one flexible
// GMRES cycle per Newton step (classical Gram-Schmidt with selective reorthogonalisation,
// Givens rotations), right-preconditioned by eq. (P) applied in the Kronecker eigenbasis of
// Section 3.2 on the tensor cores; then it takes the next item from a device-side queue.
// Items are queued largest first, so one launch covers the whole batch with no grid-wide
// synchronisation: CTAs never wait on each other, and every reduction is a CTA reduction in
// a fixed order (deterministic).
//
// Phases of one GMRES iteration k inside the CTA (256 threads, two CTAs per SM so that one
// CTA's memory-bound phases overlap the other's tensor-core phases):
//   preconditioner z_k = P^-1 v_k: four GEMMs on tcgen05 (BF16 operands, FP32 accumulators
//     in TMEM), operands brought in by bulk copies from pre-tiled global buffers:
//       1  T1^T  = (X Q_r)^T                    one product
//       2  Y_hat = modes^-1 (Q_c^T T1)          one product, the 2x2 inverse per mode as
//                                               the epilogue (both layers in one tile)
//       3  E^T   = (Y_hat Q_r^T)^T              Q_r as hi + lo: two products
//       4  Z     = (E^T Q_c^T)^T                E and Q_c as hi + lo: three products
//     every epilogue writes its output straight into the next GEMM's tiled operand layout;
//   w = J z_k (eq. J; FP32 for the first Newton step, FP32 pairs after it) fused with the
//     first Gram-Schmidt dots; the update pass writing v_{k+1} (FP64 and its tiled BF16
//     copy); the optional second pass; the Givens column (one thread).
// The residual is the FP64 cell of eq. (F) for every Newton iterate.
//
// Tiled BF16 operand layout (tix, tix32 below): a K-major matrix of R rows is stored as
// column chunks of R rows in the swizzled order of the MMA's shared-memory operands, so a
// 128-row tile of one chunk is one contiguous bulk copy: transform 1 takes K/64 chunks of
// 128-byte rows (128-byte swizzle), transforms 2-4 K/32 chunks of 64-byte rows (64-byte
// swizzle), so that one stage holds every word its products need.
//
// Every wait is bounded (2 s of %globaltimer); on expiry the CTA records MCA_ERR_TIMEOUT,
// stops taking items, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "bits.cuh"
#include "mca_internal.cuh"
#include "solver_dev.cuh"
#include "tc_ptx.cuh"

namespace mca {

namespace {

using tc::bulk_load;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::proxy_fence_global;
using tc::sw128_desc;
using tc::tc_fence_after;
using tc::tc_fence_before;
using tc::tmem_ld32;
using tc::umma;
using tc::umma_commit;

constexpr int kPT = 256;                  // threads per CTA
constexpr int kWarps = kPT / 32;
constexpr int kChunk = 128 * 128;         // bytes of one 128-row x 64-K BF16 chunk
constexpr int kStageRegion = 6 * kChunk;  // 3 stages of (A, B) or 2 of (A, A', B)
constexpr uint32_t kTmemCols = 256;       // two 128-column accumulators
constexpr int kU = 4;                     // entries per trip of the register-unrolled phases
constexpr int kUR = 4;                    // the same for the residual
constexpr int kUS = 4;                    // the same for the Jacobian apply

constexpr int kMaxStages = 4;             // GEMM stages: 4 of 24 KB down to 2 of 48 KB

struct PSmem {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t accb;
  uint64_t sfull[3];                      // streamed phases: chunk s landed
  uint64_t accb2[2];                      // overlapped GEMMs: accumulator a complete
  uint64_t tempty2[2];                    // overlapped GEMMs: accumulator a drained
  uint32_t tmem_slot;
  uint32_t g1;                            // overlapped-GEMM tiles so far
  int item;
  int err;
  uint32_t full_par, empty_par, pending;  // thread 0's pipeline state (bit s: stage s)
  double red[kWarps][32];
  double h1[32];
  double h2[32];
  double sc[4];
};

constexpr int kSmemBytes = 1024 + kStageRegion + (int)((sizeof(PSmem) + 127) / 128 * 128);

// Element offset of (row, k) in the tiled layout of a K-major BF16 matrix with R rows.
__device__ __forceinline__ size_t tix(int row, int k, int R) {
  return ((size_t)(k >> 6) * R + row) * 64 +
         (size_t)(((((k >> 3) & 7) ^ (row & 7)) << 3) | (k & 7));
}

// The same for the 32-wide K chunks of the split GEMMs' operands: K/32 chunks of R rows x
// 64 bytes in the 64-byte-swizzled order (16-byte unit u of row r at u ^ ((r / 2) % 4)).
__device__ __forceinline__ size_t tix32(int row, int k, int R) {
  return ((size_t)(k >> 5) * R + row) * 32 +
         (size_t)(((((k >> 3) & 3) ^ ((row >> 1) & 3)) << 3) | (k & 7));
}

// Optional per-phase timing (prof != NULL): thread 0 adds the %globaltimer time of each
// phase, which ends at a CTA barrier, to prof[phase] (CTA-nanoseconds summed over CTAs).
enum Phase {
  PH_RESIDUAL = 0, PH_T1, PH_T2, PH_T3, PH_T4, PH_SPMV, PH_UPDATE, PH_REORTH, PH_XUPDATE,
  PH_OTHER, PH_COUNT
};
static_assert(PH_COUNT == MCA_BATCH_PHASES, "phase count");

struct Clock {
  unsigned long long* prof;
  unsigned long long t;
  __device__ __forceinline__ void lap(int ph) {
    if (prof != nullptr && threadIdx.x == 0) {
      const unsigned long long now = tc::global_ns();
      atomicAdd(&prof[ph], now - t);
      t = now;
    }
  }
};

// ---------------------------------------------------------------- tensor-core GEMMs
// O[r][c] = sum_p sum_k A_p[r][k] B_p[c][k] over 128 x 128 output tiles (r < mrows,
// c < ncols); lp = 2: each tile also accumulates A rows r + loff into a second accumulator.
struct Job {
  const __nv_bfloat16* A[3];
  const __nv_bfloat16* B[3];
  int npass;
  int RA, RB;         // rows of the tiled A and B operands
  int K;              // contraction length (multiple of 64)
  int mrows, ncols;   // output extent (multiples of 128)
  int lp, loff;
};

// Thread 0: bring chunk g (tile, pass, 64-wide K chunk) into stage g % nst.
__device__ __forceinline__ bool produce(const Job& J, int g, int nst, int stage_bytes,
                                        uint8_t* stg, PSmem& S, int per_tile, int nkc,
                                        int ntc) {
  const int s = g % nst;
  if (S.pending & (1u << s)) {          // still read by the MMAs of chunk g - nst
    if (!mbar_wait(&S.empty[s], (S.empty_par >> s) & 1u)) return false;
    S.empty_par ^= 1u << s;
    S.pending &= ~(1u << s);
  }
  const int t = g / per_tile, w = g - t * per_tile;
  const int p = w / nkc, kc = w - p * nkc;
  const int r0 = (t / ntc) * 128, c0 = (t % ntc) * 128;
  uint8_t* st = stg + s * stage_bytes;
  mbar_expect_tx(&S.full[s], (uint32_t)stage_bytes);
  const __nv_bfloat16* a = J.A[p] + ((size_t)kc * J.RA + r0) * 64;
  bulk_load(st, a, kChunk, &S.full[s]);
  if (J.lp == 2) bulk_load(st + kChunk, a + (size_t)J.loff * 64, kChunk, &S.full[s]);
  bulk_load(st + J.lp * kChunk, J.B[p] + ((size_t)kc * J.RB + c0) * 64, kChunk, &S.full[s]);
  return true;
}

// Thread 0: the MMAs of chunk g (four K = 16 steps per layer), then release its stage.
__device__ __forceinline__ bool consume(const Job& J, int g, int nst, int stage_bytes,
                                        uint8_t* stg, PSmem& S, uint32_t tmem, bool first) {
  const int s = g % nst;
  if (!mbar_wait(&S.full[s], (S.full_par >> s) & 1u)) return false;
  S.full_par ^= 1u << s;
  tc_fence_after();
  const uint8_t* st = stg + s * stage_bytes;
  constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint64_t bd = sw128_desc(st + J.lp * kChunk + kk * 32);
    const uint32_t accf = (first && kk == 0) ? 0u : 1u;
    umma(tmem, sw128_desc(st + kk * 32), bd, idesc, accf);
    if (J.lp == 2) umma(tmem + 128, sw128_desc(st + kChunk + kk * 32), bd, idesc, accf);
  }
  umma_commit(&S.empty[s]);
  S.pending |= 1u << s;
  return true;
}

// GEMM in one pass over 32-wide K chunks (64-byte swizzle, 8 KB per 128 rows): a stage holds
// the NA A words and NB B words of one K chunk, and each product of the table P (KIND) reads
// them from the same stage into its accumulator:
//   KIND 2 (transform 2): A = both layers' rows of T1, one B: A0 B -> acc 0, A1 B -> acc 128
//   KIND 3 (transform 3): A = Y_hat, B = Q_r hi, lo:       A Bh + A Bl           -> acc 0
//   KIND 4 (transform 4): A = E hi, lo, B = Q_c hi, lo:    Ah Bh + Al Bh + Ah Bl -> acc 0
constexpr int kChunk32 = 128 * 64;
template <int KIND>
struct Prod;
template <>
struct Prod<2> {
  static constexpr int NA = 2, NB = 1, NP = 2;
  __device__ static constexpr int pa(int p) { return p; }
  __device__ static constexpr int pb(int) { return 0; }
  __device__ static constexpr int acc(int p) { return 128 * p; }
};
template <>
struct Prod<3> {
  static constexpr int NA = 1, NB = 2, NP = 2;
  __device__ static constexpr int pa(int) { return 0; }
  __device__ static constexpr int pb(int p) { return p; }
  __device__ static constexpr int acc(int) { return 0; }
};
template <>
struct Prod<4> {
  static constexpr int NA = 2, NB = 2, NP = 3;
  __device__ static constexpr int pa(int p) { return p == 1 ? 1 : 0; }
  __device__ static constexpr int pb(int p) { return p == 2 ? 1 : 0; }
  __device__ static constexpr int acc(int) { return 0; }
};

template <int KIND>
struct Job32 {
  using P = Prod<KIND>;
  const __nv_bfloat16* A[2];
  const __nv_bfloat16* B[2];
  int RA, RB, K;
  __device__ __forceinline__ int stage_bytes() const { return (P::NA + P::NB) * kChunk32; }
  __device__ __forceinline__ int chunks_per_tile() const { return K >> 5; }
  __device__ __forceinline__ bool produce(int g, int nst, uint8_t* stg, PSmem& S,
                                          int ntc) const {
    const int s = g % nst;
    if (S.pending & (1u << s)) {
      if (!mbar_wait(&S.empty[s], (S.empty_par >> s) & 1u)) return false;
      S.empty_par ^= 1u << s;
      S.pending &= ~(1u << s);
    }
    const int nkc = K >> 5;
    const int t = g / nkc, kc = g - t * nkc;
    const int r0 = (t / ntc) * 128, c0 = (t % ntc) * 128;
    uint8_t* st = stg + s * stage_bytes();
    mbar_expect_tx(&S.full[s], (uint32_t)stage_bytes());
#pragma unroll
    for (int a = 0; a < P::NA; ++a)
      bulk_load(st + a * kChunk32, A[a] + ((size_t)kc * RA + r0) * 32, kChunk32, &S.full[s]);
#pragma unroll
    for (int b = 0; b < P::NB; ++b)
      bulk_load(st + (P::NA + b) * kChunk32, B[b] + ((size_t)kc * RB + c0) * 32, kChunk32,
                &S.full[s]);
    return true;
  }
  __device__ __forceinline__ bool consume(int g, int nst, uint8_t* stg, PSmem& S,
                                          uint32_t tmem, bool first) const {
    const int s = g % nst;
    if (!mbar_wait(&S.full[s], (S.full_par >> s) & 1u)) return false;
    S.full_par ^= 1u << s;
    tc_fence_after();
    const uint8_t* st = stg + s * stage_bytes();
    constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
      for (int p = 0; p < P::NP; ++p) {
        const uint64_t ad = tc::sw64_desc(st + P::pa(p) * kChunk32 + kk * 32);
        const uint64_t bd = tc::sw64_desc(st + (P::NA + P::pb(p)) * kChunk32 + kk * 32);
        // the first product into each accumulator overwrites it
        const bool opens = first && kk == 0 && (p == 0 || P::acc(p) != P::acc(0));
        umma(tmem + (uint32_t)P::acc(p), ad, bd, idesc, opens ? 0u : 1u);
      }
    }
    umma_commit(&S.empty[s]);
    S.pending |= 1u << s;
    return true;
  }
};

// The single-pass K64 jobs of the overlapped path (lp = 1) through the same interface.
struct Job64 {
  Job J;
  __device__ __forceinline__ int stage_bytes() const { return 2 * kChunk; }
  __device__ __forceinline__ int chunks_per_tile() const { return J.npass * (J.K >> 6); }
  __device__ __forceinline__ bool produce(int g, int nst, uint8_t* stg, PSmem& S,
                                          int ntc) const {
    return mca::produce(J, g, nst, stage_bytes(), stg, S, chunks_per_tile(), J.K >> 6, ntc);
  }
  __device__ __forceinline__ bool consume(int g, int nst, uint8_t* stg, PSmem& S,
                                          uint32_t tmem, bool first) const {
    return mca::consume(J, g, nst, stage_bytes(), stg, S, tmem, first);
  }
};

// The whole GEMM by the CTA: thread 0 streams the chunks (up to nst in flight, running ahead
// across tiles) and issues the MMAs; all 8 warps drain each finished tile (warp w: TMEM lanes
// 32 (w % 4) .., columns 64 (w / 4) ..) through epi(r, c, x0, x1).  Returns false after a
// timeout (S.err set).
template <class JobT, class Epi>
__device__ bool run_gemm(const JobT& J, int mrows, int ncols, uint8_t* stg, PSmem& S,
                         uint32_t tmem, uint32_t& acc_ctr, const Epi& epi) {
  const int nst = min(kMaxStages, kStageRegion / J.stage_bytes());
  const int ntc = ncols >> 7;
  const int ntile = (mrows >> 7) * ntc;
  const int per_tile = J.chunks_per_tile();
  const int total = ntile * per_tile;
  int prod = 0;
  if (threadIdx.x == 0) {
    bool ok = true;
    for (; prod < total && prod < nst && ok; ++prod) ok = J.produce(prod, nst, stg, S, ntc);
    if (!ok) S.err = MCA_ERR_TIMEOUT;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, hc = warp >> 2;
  for (int t = 0; t < ntile; ++t) {
    if (threadIdx.x == 0 && S.err == 0) {
      tc_fence_after();
      bool ok = true;
      for (int c = 0; c < per_tile && ok; ++c) {
        const int g = t * per_tile + c;
        ok = J.consume(g, nst, stg, S, tmem, c == 0);
        if (ok && g >= 1 && prod < total) {
          ok = J.produce(prod, nst, stg, S, ntc);
          ++prod;
        }
      }
      if (ok)
        umma_commit(&S.accb);
      else
        S.err = MCA_ERR_TIMEOUT;
    }
    __syncthreads();
    if (S.err) return false;
    const bool have = mbar_wait(&S.accb, acc_ctr & 1u);
    ++acc_ctr;
    if (__syncthreads_or(have ? 0 : 1)) {
      if (threadIdx.x == 0) S.err = MCA_ERR_TIMEOUT;
      return false;
    }
    tc_fence_after();
    const int r = (t / ntc) * 128 + q * 32 + lane;
    const int c0 = (t % ntc) * 128 + hc * 64;
    const uint32_t lbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hc * 64);
#pragma unroll 1
    for (int cc = 0; cc < 2; ++cc) {
      uint32_t v0[32], v1[32];
      tmem_ld32(lbase + cc * 32, v0);
      tmem_ld32(lbase + 128 + cc * 32, v1);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        epi(r, c0 + cc * 32 + j, __uint_as_float(v0[j]), __uint_as_float(v1[j]));
    }
    tc_fence_before();
    proxy_fence_global();          // the epilogue's stores feed the next GEMM's bulk copies
    __syncthreads();
  }
  if (threadIdx.x == 0) {          // every stage's last MMAs are done: consume their phases
    for (int s = 0; s < nst; ++s) {
      if (S.pending & (1u << s)) {
        if (!mbar_wait(&S.empty[s], (S.empty_par >> s) & 1u)) S.err = MCA_ERR_TIMEOUT;
        S.empty_par ^= 1u << s;
        S.pending &= ~(1u << s);
      }
    }
  }
  __syncthreads();
  return S.err == 0;
}

// Single-layer GEMMs (lp = 1) with the epilogue overlapped: two 128-column accumulators in
// TMEM; thread 0 issues tile t + 1 into one while warps 4..7 drain tile t from the other
// (warp 4 + q: TMEM lanes 32 q .., all 128 columns) and release it on tempty2.  Tiles are
// counted over the CTA's lifetime in S.g1 (tile g uses accumulator g & 1; its accb2
// completion has parity (g >> 1) & 1, and it waits for the drain of tile g - 2).
template <class JobT, class Epi>
__device__ bool run_gemm_ws(const JobT& J, int mrows, int ncols, uint8_t* stg, PSmem& S,
                            uint32_t tmem, const Epi& epi) {
  const int nst = min(kMaxStages, kStageRegion / J.stage_bytes());
  const int ntc = ncols >> 7;
  const int ntile = (mrows >> 7) * ntc;
  const int per_tile = J.chunks_per_tile();
  const int total = ntile * per_tile;
  const uint32_t g1 = S.g1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    bool ok = true;
    int prod = 0;
    for (; prod < total && prod < nst && ok; ++prod) ok = J.produce(prod, nst, stg, S, ntc);
    for (int t = 0; t < ntile && ok; ++t) {
      const uint32_t g = g1 + (uint32_t)t;
      const uint32_t acc = g & 1u;
      if (g >= 2u && !mbar_wait(&S.tempty2[acc], ((g >> 1) - 1u) & 1u)) {
        ok = false;
        break;
      }
      tc_fence_after();
      for (int c = 0; c < per_tile && ok; ++c) {
        const int gc = t * per_tile + c;
        ok = J.consume(gc, nst, stg, S, tmem + acc * 128u, c == 0);
        if (ok && gc >= 1 && prod < total) {
          ok = J.produce(prod, nst, stg, S, ntc);
          ++prod;
        }
      }
      if (ok) umma_commit(&S.accb2[acc]);
    }
    if (!ok) S.err = MCA_ERR_TIMEOUT;
  } else if (warp >= 4) {
    const int q = warp - 4;
    for (int t = 0; t < ntile; ++t) {
      const uint32_t g = g1 + (uint32_t)t;
      const uint32_t acc = g & 1u;
      const bool have = __all_sync(0xffffffffu, mbar_wait(&S.accb2[acc], (g >> 1) & 1u)) != 0;
      if (!have) {
        if (lane == 0) S.err = MCA_ERR_TIMEOUT;
        break;
      }
      tc_fence_after();
      const int r = (t / ntc) * 128 + q * 32 + lane;
      const int c0 = (t % ntc) * 128;
      const uint32_t lbase = tmem + acc * 128u + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        uint32_t v0[32];
        tmem_ld32(lbase + cc * 32, v0);
#pragma unroll
        for (int j = 0; j < 32; ++j) epi(r, c0 + cc * 32 + j, __uint_as_float(v0[j]), 0.f);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(
                         &S.tempty2[acc]))
                     : "memory");
    }
    proxy_fence_global();          // the epilogue's stores feed the next GEMM's bulk copies
  }
  __syncthreads();
  if (threadIdx.x == 0) {          // every stage's last MMAs are done: consume their phases
    for (int s = 0; s < nst; ++s) {
      if (S.pending & (1u << s)) {
        if (!mbar_wait(&S.empty[s], (S.empty_par >> s) & 1u)) S.err = MCA_ERR_TIMEOUT;
        S.empty_par ^= 1u << s;
        S.pending &= ~(1u << s);
      }
    }
    S.g1 = g1 + (uint32_t)ntile;
  }
  __syncthreads();
  return S.err == 0;
}

// Per-item buffers inside the CTA's slot.  Vectors of 2 m n unknowns are stored as two
// layers of mnp = round_up(m n, 4) entries (v_j at V + j n2s, n2s = 2 mnp), so every layer and
// every 4-entry group starts on a 16-byte boundary (the bulk copies of the streamed phases);
// the padding entries are never read as data.
struct Work {
  double* x;           // state [2][mnp]
  double* D;           // Jacobian diagonal [mnp]
  double* W;           // J z
  double* V;           // basis, v_j at V + j n2s (unnormalised, scale ctl.s[j])
  float* Z;            // preconditioned basis, z_j at Z + j n2s
  __nv_bfloat16* xbf;  // tiled BF16 copy of the current basis vector, [np/64][2 mp][64]
  __nv_bfloat16* t1;   // [mp/64][2 np][64]
  __nv_bfloat16* yh;   // [np/64][2 mp][64]
  __nv_bfloat16* eh;   // [mp/64][2 np][64]
  __nv_bfloat16* el;
  VecCtl* ctl;
  int mnp, n2s;        // of the current item
};

// z = P^-1 (sc * X) with X the BF16 vector in w.xbf, a1 = a2 = a (eq. P, Section 3.2).
__device__ bool precond(const PersistShape& sh, const Work& w, float* z, float a, float sc,
                        uint8_t* stg, PSmem& S, uint32_t tmem, uint32_t& acc_ctr,
                        Clock& clk) {
  const int m = sh.gr.m, n = sh.gr.n, mp = sh.mp, np = sh.np;
  const int mnp = w.mnp;
  {
    __nv_bfloat16* t1 = w.t1;
    const Job64 j{{{w.xbf}, {sh.qrt}, 1, 2 * mp, np, np, 2 * mp, np, 1, 0}};
    if (!run_gemm_ws(j, 2 * mp, np, stg, S, tmem, [=](int r, int c, float x0, float) {
          const int l = r >= mp ? 1 : 0;
          t1[tix32(l * np + c, r - l * mp, 2 * np)] = __float2bfloat16(x0);
        }))
      return false;
    clk.lap(PH_T1);
  }
  {
    __nv_bfloat16* yh = w.yh;
    const float* mu_f = sh.mu_f;
    const float* nu_f = sh.nu_f;
    // both layers of a mode in one tile: A rows r (layer 0) and np + r (layer 1), one B
    const Job32<2> j{{w.t1, w.t1 + (size_t)np * 32}, {sh.qct, nullptr}, 2 * np, mp, mp};
    if (!run_gemm(j, np, mp, stg, S, tmem, acc_ctr, [=](int r, int c, float x0, float x1) {
          // [y_t; y_b] = (1/det) [[nu + a, a], [a, mu + a]] [x_t; x_b] for mode (r, c)
          float y0 = 0.f, y1 = 0.f;
          if (r < n && c < m) {
            const float mu = mu_f[r], nu = nu_f[c];
            const float det = mu * nu + mu * a + nu * a;
            const float inv = sc * __frcp_rn(det);
            y0 = ((nu + a) * x0 + a * x1) * inv;
            y1 = (a * x0 + (mu + a) * x1) * inv;
          }
          yh[tix32(c, r, 2 * mp)] = __float2bfloat16(y0);
          yh[tix32(mp + c, r, 2 * mp)] = __float2bfloat16(y1);
        }))
      return false;
    clk.lap(PH_T2);
  }
  {
    __nv_bfloat16* eh = w.eh;
    __nv_bfloat16* el = w.el;
    // A = Y_hat (one word), B = Q_r hi, lo: products A Bh + A Bl
    const Job32<3> j{{w.yh, nullptr}, {sh.qr_hi, sh.qr_lo}, 2 * mp, np, np};
    if (!run_gemm_ws(j, 2 * mp, np, stg, S, tmem, [=](int r, int c, float x0, float) {
          const int l = r >= mp ? 1 : 0;
          const size_t o = tix32(l * np + c, r - l * mp, 2 * np);
          const __nv_bfloat16 hi = __float2bfloat16(x0);
          eh[o] = hi;
          el[o] = __float2bfloat16(x0 - __bfloat162float(hi));
        }))
      return false;
    clk.lap(PH_T3);
  }
  {
    // A = E hi, lo and B = Q_c hi, lo: products Eh Qh + El Qh + Eh Ql
    const Job32<4> j{{w.eh, w.el}, {sh.qc_hi, sh.qc_lo}, 2 * np, mp, mp};
    if (!run_gemm_ws(j, 2 * np, mp, stg, S, tmem, [=](int r, int c, float x0, float) {
          const int l = r >= np ? 1 : 0;
          const int jj = r - l * np;
          if (jj < n && c < m) z[(size_t)l * mnp + (size_t)c * n + jj] = x0;
        }))
      return false;
    clk.lap(PH_T4);
  }
  return true;
}

// ---------------------------------------------------------------- CTA reductions
// out[j] = (scale ? scale[j] : 1) * (block total of acc[j]) for j < nk; ends synchronised.
template <int KP>
__device__ __forceinline__ void block_reduce(double (&acc)[KP], int nk, double* out,
                                             const double* scale, PSmem& S) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const double tot = warp_sum_scatter<KP>(acc);
  if (warp_scatter_writer<KP>(l)) S.red[w][warp_scatter_index<KP>(l)] = tot;
  __syncthreads();
  if (threadIdx.x < nk) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) s += S.red[q][threadIdx.x];
    out[threadIdx.x] = scale ? s * scale[threadIdx.x] : s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- memory-bound phases
// Two forms, chosen per phase by measurement.  Register-unrolled: kU entries per thread and
// trip, all loads of a trip issued before its arithmetic (residual, Jacobian apply, update
// passes).  Streamed (the solution update): operands go through the operand stages, idle
// outside the GEMMs, as a ring of kSStages chunks of at most kSStageBytes, each chunk one
// bulk copy per stream completing on one mbarrier, two chunks in flight while the CTA works
// on the third from shared memory.  Every streamed window starts and ends on a 16-byte
// boundary.
constexpr int kSStages = 3;
constexpr int kSStageBytes = kStageRegion / kSStages;

__device__ __forceinline__ int align4_dn(int v) { return v & ~3; }

// Runs nchunks chunks: issue(c, stage) (thread 0) starts the bulk copies of chunk c and
// returns their byte count; body(c, stage) consumes chunk c.  sctr counts the chunks the
// CTA has streamed (stage sctr % kSStages, phase parity (sctr / kSStages) & 1).
template <class Issue, class Body>
__device__ bool stream_run(int nchunks, const Issue& issue, const Body& body, uint8_t* stg,
                           PSmem& S, uint32_t& sctr) {
  if (threadIdx.x == 0) {
    for (int c = 0; c < nchunks && c < kSStages - 1; ++c) {
      const int s = (int)((sctr + c) % kSStages);
      uint8_t* st = stg + s * kSStageBytes;
      tc::mbar_expect_tx(&S.sfull[s], (uint32_t)issue(c, st, &S.sfull[s], true));
      issue(c, st, &S.sfull[s], false);
    }
  }
  for (int c = 0; c < nchunks; ++c) {
    const int s = (int)(sctr % kSStages);
    if (!mbar_wait(&S.sfull[s], (sctr / kSStages) & 1u)) S.err = MCA_ERR_TIMEOUT;
    body(c, stg + s * kSStageBytes);
    __syncthreads();
    if (threadIdx.x == 0 && c + kSStages - 1 < nchunks) {
      const int s2 = (int)((sctr + kSStages - 1) % kSStages);
      uint8_t* st = stg + s2 * kSStageBytes;
      tc::mbar_expect_tx(&S.sfull[s2], (uint32_t)issue(c + kSStages - 1, st, &S.sfull[s2], true));
      issue(c + kSStages - 1, st, &S.sfull[s2], false);
    }
    ++sctr;
  }
  return S.err == 0;
}

// One stream window: copy entries [lo, hi) of src (esz bytes each) to dst; dry: only the
// byte count.
__device__ __forceinline__ int window(bool dry, uint8_t*& dst, const void* src, int esz, int lo,
                                      int hi, uint64_t* bar) {
  const int bytes = (hi - lo) * esz;
  if (!dry && bytes > 0)
    bulk_load(dst, static_cast<const uint8_t*>(src) + (size_t)lo * esz, (uint32_t)bytes, bar);
  dst += bytes;
  return bytes;
}

// Residual of eq. (F) (FP64 cell) into v_0 = F (with its tiled BF16 copy), D, and the Newton
// control.  ZERO: the state is V = 0 (F = -Y, D = g).  kU cells per trip with all their loads
// issued before the first cell's arithmetic (the stores may alias the loads, so the compiler
// cannot hoist them itself); each thread still visits its cells in increasing order.
template <bool ZERO, bool YAK>
__device__ bool residual_phase(const PersistShape& sh, const double* gmap, const double* vin,
                               const Work& w, PSmem& S) {
  const Grid& gr = sh.gr;
  const int m = gr.m, n = gr.n, mn = m * n, mp = sh.mp, mnp = w.mnp;
  const double* Vt = w.x;
  const double* Vb = w.x + mnp;
  double* Ft = w.V;
  double* Fb = w.V + mnp;
  VecCtl& ctl = *w.ctl;
  const bool lin = (gr.b == 0.0);
  const bool norm32 = sh.cfg.newton_rtol * ctl.ynorm > kNorm32Min;
  double sf = 0.0, sd = 0.0;
  float sdf = 0.f, sfh = 0.f, sfl = 0.f;
  bool dnot32 = false;
  for (int base = threadIdx.x; base < mn; base += kUR * kPT) {
    int iu[kUR], ju[kUR];
    double vt[kUR], vb[kUR], tl[kUR], tr[kUR], bu[kUR], bd[kUR], g[kUR], vi[kUR];
#pragma unroll
    for (int u = 0; u < kUR; ++u) {
      const int c = base + u * kPT;
      const int cc = c < mn ? c : base;
      iu[u] = cc / n;
      ju[u] = cc - iu[u] * n;
      g[u] = gmap[cc];
      vi[u] = (ju[u] == 0) ? vin[iu[u]] : 0.0;
      if (!ZERO) {
        vt[u] = Vt[cc];
        vb[u] = Vb[cc];
        tl[u] = (ju[u] > 0) ? Vt[cc - 1] : 0.0;
        tr[u] = (ju[u] < n - 1) ? Vt[cc + 1] : 0.0;
        bu[u] = (iu[u] > 0) ? Vb[cc - n] : 0.0;
        bd[u] = (iu[u] < m - 1) ? Vb[cc + n] : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < kUR; ++u) {
      const int c = base + u * kPT;
      if (c >= mn) break;
      const int i = iu[u], j = ju[u];
      double ft, fb, dg;
      float dgf = 0.f;
      if (ZERO) {
        ft = (j == 0) ? -gr.g_src * vi[u] : 0.0;
        fb = 0.0;
        dg = g[u];
        dgf = d2f_round(dg);
      } else {
        cell_residual_vals<YAK>(gr, i, j, vt[u], vb[u], tl[u], tr[u], bu[u], bd[u], g[u],
                                vi[u], ft, fb, dg, dgf);
      }
      Ft[c] = ft;
      Fb[c] = fb;
      if (!ZERO) w.D[c] = dg;        // (the zero state's D is g: the apply reads the map)
      {
        const uint32_t dh = (uint32_t)__double2hiint(dg), dlw = (uint32_t)__double2loint(dg);
        const uint32_t de = (dh >> 20) & 0x7FFu;
        dnot32 |= ((dlw & 0x1FFFFFFFu) != 0u) ||
                  (de - 897u > 253u && ((dh & 0x7FFFFFFFu) | dlw));
      }
      if (!ZERO || j == 0) {         // the zero state's F is zero off the first column, and
        w.xbf[tix(i, j, 2 * mp)] = d2bf16_bits(ft);   // the BF16 copy starts zeroed
        if (!ZERO) w.xbf[tix(mp + i, j, 2 * mp)] = d2bf16_bits(fb);
      }
      if (!ZERO) {
        if (!norm32) {
          sf = fma(ft, ft, sf);
          sf = fma(fb, fb, sf);
        } else {
          const float a = d2f_round(ft), bb = d2f_round(fb);
          float e;
          sfh = two_sum(sfh, fmaf(a, a, bb * bb), e);
          sfl += e;
        }
      }
      if (lin) sd += dg; else sdf += dgf;
    }
  }
  sd += f2d_bits(sdf);
  sf += f2d_bits(sfh) + f2d_bits(sfl);
  const int any64 = __syncthreads_or(dnot32 ? 1 : 0);
  double acc[2] = {sf, sd};
  block_reduce<2>(acc, 2, S.sc, nullptr, S);
  if (threadIdx.x == 0) {
    ctl.d64_next = any64 ? 1 : 0;
    const double f2 = ZERO ? ctl.ynorm * ctl.ynorm : S.sc[0];
    newton_control(ctl, f2, S.sc[1], mn, sh.cfg, nullptr);
  }
  proxy_fence_global();
  __syncthreads();
  return true;
}

// w = J z (eq. J; AM: kApplyF32 or kApplyPair) and h1_j = s_j <V_j, w> for j < nk, kU cells
// per trip with their loads first.
template <int KP, int AM>
__device__ bool spmv_phase(const Grid& gr, const Work& w, const double* D, const float* z,
                           int nk, PSmem& S) {
  const int m = gr.m, n = gr.n, mn = m * n, mnp = w.mnp, n2s = w.n2s;
  const float* zt = z;
  const float* zb = z + mnp;
  const bool dsplit = w.ctl->d64 != 0;
  double acc[KP];
#pragma unroll
  for (int jv = 0; jv < KP; ++jv) acc[jv] = 0.0;
  for (int base = threadIdx.x; base < mn; base += kUS * kPT) {
    float za[kUS], zbv[kUS], tl[kUS], tr[kUS], bu[kUS], bd[kUS];
    double Dv[kUS], ot[kUS], ob[kUS];
    int iu[kUS], ju[kUS];
#pragma unroll
    for (int u = 0; u < kUS; ++u) {
      const int c = base + u * kPT;
      const int cc = c < mn ? c : base;
      const int i = cc / n, jj = cc - (cc / n) * n;
      iu[u] = i;
      ju[u] = jj;
      za[u] = zt[cc];
      zbv[u] = zb[cc];
      tl[u] = (jj > 0) ? zt[cc - 1] : 0.f;
      tr[u] = (jj < n - 1) ? zt[cc + 1] : 0.f;
      bu[u] = (i > 0) ? zb[cc - n] : 0.f;
      bd[u] = (i < m - 1) ? zb[cc + n] : 0.f;
      Dv[u] = D[cc];
    }
#pragma unroll
    for (int u = 0; u < kUS; ++u) {
      const int i = iu[u], jj = ju[u];
      if constexpr (AM == kApplyPair) {
        const bool f = (jj == 0), l = (jj == n - 1), up = (i == 0), dn = (i == m - 1);
        apply_pair(za[u], zbv[u], tl[u], tr[u], bu[u], bd[u], Dv[u],
                   f ? gr.dt0f : (l ? gr.dtlf : gr.dtmf), f ? gr.dt0l : (l ? gr.dtll : gr.dtml),
                   up ? gr.db0f : (dn ? gr.dblf : gr.dbmf),
                   up ? gr.db0l : (dn ? gr.dbll : gr.dbml), gr, ot[u], ob[u], dsplit);
      } else {
        const float a = za[u], bb = zbv[u];
        const float cpl = d2f_round(Dv[u]) * (a - bb);
        const float dt = (jj == 0) ? gr.dt0f : ((jj == n - 1) ? gr.dtlf : gr.dtmf);
        const float db = (i == 0) ? gr.db0f : ((i == m - 1) ? gr.dblf : gr.dbmf);
        ot[u] = f2d_bits(fmaf(dt, a, fmaf(-gr.gtf, tl[u] + tr[u], cpl)));
        ob[u] = f2d_bits(fmaf(db, bb, fmaf(-gr.gbf, bu[u] + bd[u], -cpl)));
      }
    }
    // the dots' loads before the stores of w (which may alias them for the compiler)
#pragma unroll
    for (int jv = 0; jv < KP; ++jv) {
      if (jv < nk) {
        const double* vj = w.V + (size_t)jv * n2s;
#pragma unroll
        for (int u = 0; u < kUS; ++u) {
          const int c = base + u * kPT;
          if (c < mn) {
            acc[jv] = fma(vj[c], ot[u], acc[jv]);
            acc[jv] = fma(vj[mnp + c], ob[u], acc[jv]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUS; ++u) {
      const int c = base + u * kPT;
      if (c < mn) {
        w.W[c] = ot[u];
        w.W[mnp + c] = ob[u];
      }
    }
  }
  block_reduce<KP>(acc, nk, S.h1, w.ctl->s, S);
  proxy_fence_global();
  __syncthreads();
  return true;
}

// Entries e of a vector in the padded layout that hold data (not layer padding).
__device__ __forceinline__ bool live(int e, int mn, int mnp) {
  return e < mn || (e >= mnp && e - mnp < mn);
}

// out = src - sum_j hc_j s_j V_j (j < nk) with its tiled BF16 copy; ||out||^2 into *hn2
// (out may alias src).  Each layer's m n entries in turn, kU per trip with all their loads
// first (the stores may alias the loads of the next trip).
template <int KP>
__device__ bool update_phase(const PersistShape& sh, const Work& w, const double* src,
                             double* out, int nk, const double* hc, PSmem& S, double* hn2) {
  const int n = sh.gr.n, mn = sh.gr.m * n, mp = sh.mp, mnp = w.mnp, n2s = w.n2s;
  double hj[KP];
#pragma unroll
  for (int jv = 0; jv < KP; ++jv) hj[jv] = (jv < nk) ? hc[jv] * w.ctl->s[jv] : 0.0;
  double acc[1] = {0.0};
  auto finish = [&](int l, int cell, double x) {
    out[l * mnp + cell] = x;
    const int i = cell / n, j = cell - i * n;
    w.xbf[tix(l * mp + i, j, 2 * mp)] = d2bf16_bits(x);
    acc[0] = fma(x, x, acc[0]);
  };
  for (int l = 0; l < 2; ++l) {
    const double* sl = src + l * mnp;
    const double* Vl = w.V + l * mnp;
    int c = threadIdx.x;
    for (; c + (kU - 1) * kPT < mn; c += kU * kPT) {
      double x[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) x[u] = sl[c + u * kPT];
#pragma unroll
      for (int jv = 0; jv < KP; ++jv)
        if (jv < nk) {
#pragma unroll
          for (int u = 0; u < kU; ++u)
            x[u] = fma(-hj[jv], Vl[(size_t)jv * n2s + c + u * kPT], x[u]);
        }
#pragma unroll
      for (int u = 0; u < kU; ++u) finish(l, c + u * kPT, x[u]);
    }
    for (; c < mn; c += kPT) {
      double x = sl[c];
#pragma unroll
      for (int jv = 0; jv < KP; ++jv)
        if (jv < nk) x = fma(-hj[jv], Vl[(size_t)jv * n2s + c], x);
      finish(l, c, x);
    }
  }
  block_reduce<1>(acc, 1, S.sc, nullptr, S);
  *hn2 = S.sc[0];
  return true;
}

// h2_j = s_j <V_j, u> for j < nk (second Gram-Schmidt pass).
template <int KP>
__device__ bool dots_phase(const PersistShape& sh, const Work& w, const double* u, int nk,
                           PSmem& S) {
  const int mn = sh.gr.m * sh.gr.n, mnp = w.mnp, n2s = w.n2s;
  double acc[KP];
#pragma unroll
  for (int jv = 0; jv < KP; ++jv) acc[jv] = 0.0;
  for (int e = threadIdx.x; e < n2s; e += kPT) {
    if (!live(e, mn, mnp)) continue;
    const double x = u[e];
#pragma unroll
    for (int jv = 0; jv < KP; ++jv)
      if (jv < nk) acc[jv] = fma(w.V[(size_t)jv * n2s + e], x, acc[jv]);
  }
  block_reduce<KP>(acc, nk, S.h2, w.ctl->s, S);
  return true;
}

// x += sum_j y_j z_j (j < kd <= KP).  Streams: x and z_j over the whole padded vector.
template <int KP>
__device__ bool xupdate_phase(const PersistShape& sh, const Work& w, int kd, const double* y,
                              uint8_t* stg, PSmem& S, uint32_t& sctr) {
  const int mn = sh.gr.m * sh.gr.n, mnp = w.mnp, n2s = w.n2s;
  double yj[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) yj[j] = (j < kd) ? y[j] : 0.0;
  int len = align4_dn(kSStageBytes / (8 + 4 * kd));
  if (len > n2s) len = n2s;
  const int nchunks = (n2s + len - 1) / len;
  auto issue = [&](int c, uint8_t* st, uint64_t* bar, bool dry) {
    const int e0 = c * len, e1 = min(e0 + len, n2s);
    int bytes = window(dry, st, w.x, 8, e0, e1, bar);
    for (int j = 0; j < kd; ++j) bytes += window(dry, st, w.Z + (size_t)j * n2s, 4, e0, e1, bar);
    return bytes;
  };
  auto body = [&](int c, uint8_t* st) {
    const int e0 = c * len, e1 = min(e0 + len, n2s), L = e1 - e0;
    const double* s_x = reinterpret_cast<const double*>(st);
    const float* s_z = reinterpret_cast<const float*>(s_x + L);
    for (int e = e0 + (int)threadIdx.x; e < e1; e += kPT) {
      if (!live(e, mn, mnp)) continue;
      double s = s_x[e - e0];
#pragma unroll
      for (int j = 0; j < KP; ++j)
        if (j < kd) s = fma(yj[j], f2d_bits(s_z[(size_t)j * L + e - e0]), s);
      w.x[e] = s;
    }
  };
  const bool ok = stream_run(nchunks, issue, body, stg, S, sctr);
  proxy_fence_global();
  __syncthreads();
  return ok;
}

#define MCA_PKP(F, nk, ...)                       \
  do {                                            \
    if ((nk) <= 1) ok = F<1>(__VA_ARGS__);        \
    else if ((nk) <= 2) ok = F<2>(__VA_ARGS__);   \
    else if ((nk) <= 4) ok = F<4>(__VA_ARGS__);   \
    else if ((nk) <= 8) ok = F<8>(__VA_ARGS__);   \
    else if ((nk) <= 16) ok = F<16>(__VA_ARGS__); \
    else ok = F<32>(__VA_ARGS__);                 \
  } while (0)

template <int KP>
__device__ bool spmv_f32(const Grid& gr, const Work& w, const double* D, const float* z,
                         int nk, PSmem& S) {
  return spmv_phase<KP, kApplyF32>(gr, w, D, z, nk, S);
}
template <int KP>
__device__ bool spmv_pair(const Grid& gr, const Work& w, const double* D, const float* z,
                          int nk, PSmem& S) {
  return spmv_phase<KP, kApplyPair>(gr, w, D, z, nk, S);
}

// Output currents and the Kirchhoff balance (as k_outputs); copies the state out.
__device__ void outputs_phase(const PersistShape& sh, const PersistItem& it, const Work& w,
                              PersistResult* res, PSmem& S) {
  const Grid& gr = sh.gr;
  const int m = gr.m, n = gr.n, mn = m * n;
  const double* Vt = w.x;
  const double* Vb = w.x + w.mnp;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};   // in, |in|, out, leaks
  for (int i = threadIdx.x; i < m; i += kPT) {
    const double iin = gr.g_src * (it.vin[i] - Vt[(size_t)i * n]);
    acc[0] += iin;
    acc[1] += fabs(iin);
    acc[3] += gr.g_tr * Vt[(size_t)i * n + n - 1];
  }
  for (int j = threadIdx.x; j < n; j += kPT) {
    const double io = gr.g_sense * Vb[(size_t)(m - 1) * n + j];
    if (it.iout) it.iout[j] = io;
    acc[2] += io;
    acc[3] += gr.g_bt * Vb[j];
  }
  for (int c = threadIdx.x; c < mn; c += kPT) {
    if (it.vt) it.vt[c] = Vt[c];
    if (it.vb) it.vb[c] = Vb[c];
  }
  block_reduce<4>(acc, 4, S.sc, nullptr, S);
  if (threadIdx.x == 0) {
    const VecCtl& c = *w.ctl;
    const double bal = S.sc[0] - S.sc[2] - S.sc[3];
    PersistResult r;
    r.status = c.status;
    r.newton_iters = c.newton_iters;
    r.gmres_iters = c.gmres_iters;
    r.pad_ = 0;
    r.fnorm = c.fnorm;
    r.ynorm = c.ynorm;
    r.kcl = (S.sc[1] > 0.0) ? fabs(bal) / S.sc[1] : 0.0;
    *res = r;
  }
}

// Zero the tiled BF16 copy of the basis vector (its padding must read zero).
__device__ void zero_xbf(const PersistShape& sh, const Work& w) {
  const size_t n16 = (size_t)2 * sh.mp * sh.np / 8;
  uint4* p = reinterpret_cast<uint4*>(w.xbf);
  for (size_t e = threadIdx.x; e < n16; e += kPT) p[e] = make_uint4(0u, 0u, 0u, 0u);
}

template <bool YAK>
__device__ bool solve_item(const PersistShape& sh, const PersistItem& it, Work& w,
                           PersistResult* res, uint8_t* stg, PSmem& S, uint32_t tmem,
                           uint32_t& acc_ctr, uint32_t& sctr, int restart, Clock& clk) {
  const Grid& gr = sh.gr;
  const int m = gr.m, n = gr.n, mn = m * n;
  w.mnp = (mn + 3) & ~3;
  w.n2s = 2 * w.mnp;
  const int n2s = w.n2s;
  VecCtl& ctl = *w.ctl;
  const double* gmap = sh.gmaps + (size_t)it.map * mn;
  zero_xbf(sh, w);
  for (int e = threadIdx.x; e < n2s; e += kPT) w.x[e] = 0.0;
  {
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < m; i += kPT) acc[0] = fma(it.vin[i], it.vin[i], acc[0]);
    block_reduce<1>(acc, 1, S.sc, nullptr, S);
    if (threadIdx.x == 0) init_ctl(ctl, gr.g_src * sqrt(S.sc[0]), false);
    proxy_fence_global();
    __syncthreads();
  }
  clk.lap(PH_OTHER);
  bool ok = true;
  for (int itn = 0; itn <= sh.cfg.max_newton; ++itn) {
    if (!ctl.newton_active) break;
    if (itn == 0)
      ok = residual_phase<true, false>(sh, gmap, it.vin, w, S);
    else
      ok = residual_phase<false, YAK>(sh, gmap, it.vin, w, S);
    if (!ok) return false;
    clk.lap(PH_RESIDUAL);
    if (!ctl.newton_active) break;
    const bool f32 = (itn == 0) && sh.cfg.eta0 >= kF32ApplyMinEta;
    for (int k = 0; k < restart; ++k) {
      float* zk = w.Z + (size_t)k * n2s;
      if (!precond(sh, w, zk, (float)ctl.a, (float)ctl.s[k], stg, S, tmem, acc_ctr, clk))
        return false;
      const int nk = k + 1;
      // D of the zero state is the conductance map itself
      const double* D = (itn == 0) ? gmap : w.D;
      if (f32)
        MCA_PKP(spmv_f32, nk, gr, w, D, zk, nk, S);
      else
        MCA_PKP(spmv_pair, nk, gr, w, D, zk, nk, S);
      if (!ok) return false;
      clk.lap(PH_SPMV);
      double* vnext = w.V + (size_t)(k + 1) * n2s;
      double hn2 = 0.0;
      MCA_PKP(update_phase, nk, sh, w, w.W, vnext, nk, S.h1, S, &hn2);
      if (!ok) return false;
      if (threadIdx.x == 0)
        gram_schmidt_control<false>(ctl, 0, UPD_FIRST, hn2, S.h1, S.h1, nk, restart, nullptr);
      proxy_fence_global();
      __syncthreads();
      clk.lap(PH_UPDATE);
      if (ctl.reorth) {
        MCA_PKP(dots_phase, nk, sh, w, vnext, nk, S);
        if (!ok) return false;
        MCA_PKP(update_phase, nk, sh, w, vnext, vnext, nk, S.h2, S, &hn2);
        if (!ok) return false;
        if (threadIdx.x == 0)
          gram_schmidt_control<false>(ctl, 0, UPD_REORTH, hn2, S.h2, S.h1, nk, restart,
                                      nullptr);
        proxy_fence_global();
        __syncthreads();
        clk.lap(PH_REORTH);
      }
      if (!ctl.gm_active) break;
    }
    if (threadIdx.x == 0) lsq_solve(ctl);
    __syncthreads();
    {
      const int kd = ctl.k_done;
      if (threadIdx.x < 32) S.h2[threadIdx.x] = (threadIdx.x < kd) ? ctl.y[threadIdx.x] : 0.0;
      __syncthreads();
      if (kd > 0) {
        MCA_PKP(xupdate_phase, kd, sh, w, kd, S.h2, stg, S, sctr);
        if (!ok) return false;
      }
    }
    clk.lap(PH_XUPDATE);
  }
  outputs_phase(sh, it, w, res, S);
  __syncthreads();
  clk.lap(PH_OTHER);
  return true;
}

// Preconditioner test: z = P^-1 r for r in (vt, vb), written back there.
__device__ bool precond_item(const PersistShape& sh, const PersistItem& it, Work& w,
                             uint8_t* stg, PSmem& S, uint32_t tmem, uint32_t& acc_ctr,
                             Clock& clk) {
  const int m = sh.gr.m, n = sh.gr.n, mn = m * n, mp = sh.mp;
  w.mnp = (mn + 3) & ~3;
  w.n2s = 2 * w.mnp;
  zero_xbf(sh, w);
  __syncthreads();
  for (int c = threadIdx.x; c < mn; c += kPT) {
    const int i = c / n, j = c - i * n;
    w.xbf[tix(i, j, 2 * mp)] = d2bf16_bits(it.vt[c]);
    w.xbf[tix(mp + i, j, 2 * mp)] = d2bf16_bits(it.vb[c]);
  }
  proxy_fence_global();
  __syncthreads();
  if (!precond(sh, w, w.Z, (float)it.a, 1.f, stg, S, tmem, acc_ctr, clk)) return false;
  for (int c = threadIdx.x; c < mn; c += kPT) {
    it.vt[c] = f2d_bits(w.Z[c]);
    it.vb[c] = f2d_bits(w.Z[w.mnp + c]);
  }
  __syncthreads();
  return true;
}

template <bool YAK>
__global__ void __launch_bounds__(kPT, 2)
k_persist(const PersistShape* __restrict__ shapes, const PersistItem* __restrict__ items,
          int n_items, PersistResult* res, int* queue, int* err, PersistSlots sl, int mode,
          unsigned long long* prof) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* stg = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  PSmem& S = *reinterpret_cast<PSmem*>(stg + kStageRegion);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int s = 0; s < kSStages; ++s) mbar_init(&S.sfull[s], 1);
    mbar_init(&S.accb, 1);
    for (int a = 0; a < 2; ++a) {
      mbar_init(&S.accb2[a], 1);
      mbar_init(&S.tempty2[a], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.full_par = S.empty_par = S.pending = 0u;
    S.g1 = 0u;
    S.err = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&S.tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_slot;
  uint8_t* slot = sl.base + (size_t)blockIdx.x * sl.slot_bytes;
  Work w;
  w.x = reinterpret_cast<double*>(slot + sl.off_x);
  w.D = reinterpret_cast<double*>(slot + sl.off_d);
  w.W = reinterpret_cast<double*>(slot + sl.off_w);
  w.V = reinterpret_cast<double*>(slot + sl.off_v);
  w.Z = reinterpret_cast<float*>(slot + sl.off_z);
  w.xbf = reinterpret_cast<__nv_bfloat16*>(slot + sl.off_bf[0]);
  w.t1 = reinterpret_cast<__nv_bfloat16*>(slot + sl.off_bf[1]);
  w.yh = reinterpret_cast<__nv_bfloat16*>(slot + sl.off_bf[2]);
  w.eh = reinterpret_cast<__nv_bfloat16*>(slot + sl.off_bf[3]);
  w.el = reinterpret_cast<__nv_bfloat16*>(slot + sl.off_bf[4]);
  w.ctl = reinterpret_cast<VecCtl*>(slot + sl.off_ctl);
  w.mnp = w.n2s = 0;
  uint32_t acc_ctr = 0, sctr = 0;
  Clock clk{prof, prof ? tc::global_ns() : 0ull};
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(queue, 1);
    __syncthreads();
    const int k = S.item;
    if (k >= n_items || S.err) break;
    const PersistItem it = items[k];
    const PersistShape& sh = shapes[it.shape];
    clk.lap(PH_OTHER);
    const bool ok = (mode == 1) ? precond_item(sh, it, w, stg, S, tmem, acc_ctr, clk)
                                : solve_item<YAK>(sh, it, w, res + k, stg, S, tmem, acc_ctr,
                                                  sctr, sh.cfg.restart, clk);
    __syncthreads();
    if (!ok || S.err) break;
  }
  if (threadIdx.x == 0 && S.err) tc::record_error(err, S.err);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

__global__ void k_retile(const __nv_bfloat16* __restrict__ src, int R, int K,
                         __nv_bfloat16* __restrict__ dst, int k32) {
  const size_t total = (size_t)R * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / K), k = (int)(e - (size_t)r * K);
    dst[k32 ? tix32(r, k, R) : tix(r, k, R)] = src[e];
  }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

size_t persist_slot_layout(PersistSlots& sl, size_t n2max, size_t bfmax, int restart) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 1024);
    return at;
  };
  sl.off_x = take(n2max * sizeof(double));
  sl.off_d = take(n2max / 2 * sizeof(double));
  sl.off_w = take(n2max * sizeof(double));
  sl.off_v = take((size_t)(restart + 1) * n2max * sizeof(double));
  sl.off_z = take((size_t)restart * n2max * sizeof(float));
  for (int b = 0; b < 5; ++b) sl.off_bf[b] = take(bfmax * sizeof(__nv_bfloat16));
  sl.off_ctl = take(sizeof(VecCtl));
  sl.restart = restart;
  sl.slot_bytes = o;
  return o;
}

int persist_smem_bytes() { return kSmemBytes; }

cudaError_t persist_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_persist<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_persist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemBytes);
}

void launch_persist(const PersistShape* shapes, const PersistItem* items, int n_items,
                    PersistResult* res, int* queue, int* err, const PersistSlots& sl,
                    int grid, int mode, bool yak, unsigned long long* prof, cudaStream_t s) {
  if (yak)
    k_persist<true><<<grid, kPT, kSmemBytes, s>>>(shapes, items, n_items, res, queue, err, sl,
                                                  mode, prof);
  else
    k_persist<false><<<grid, kPT, kSmemBytes, s>>>(shapes, items, n_items, res, queue, err, sl,
                                                   mode, prof);
}

void launch_retile_bf16(const __nv_bfloat16* src, int R, int K, __nv_bfloat16* dst, bool k32,
                        cudaStream_t s) {
  const size_t total = (size_t)R * K;
  int nb = (int)((total + 255) / 256);
  if (nb > 1216) nb = 1216;
  k_retile<<<nb, 256, 0, s>>>(src, R, K, dst, k32 ? 1 : 0);
}

}  // namespace mca
