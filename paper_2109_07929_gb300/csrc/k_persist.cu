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
// Tiled BF16 operand layout (tix below): a K-major matrix of R rows is stored as
// K/64 column chunks of R rows x 128 bytes in the 128-byte-swizzled order of the MMA's
// shared-memory operands (16-byte unit u of row r at position u ^ (r % 8)), so a 128-row
// tile of one chunk is one contiguous 16 KB bulk copy.
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

struct PSmem {
  uint64_t full[3];
  uint64_t empty[3];
  uint64_t accb;
  uint32_t tmem_slot;
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

// The whole GEMM by the CTA: thread 0 streams the chunks (up to nst in flight, running ahead
// across tiles) and issues the MMAs; all 8 warps drain each finished tile (warp w: TMEM lanes
// 32 (w % 4) .., columns 64 (w / 4) ..) through epi(r, c, x0, x1).  Returns false after a
// timeout (S.err set).
template <class Epi>
__device__ bool run_gemm(const Job& J, uint8_t* stg, PSmem& S, uint32_t tmem,
                         uint32_t& acc_ctr, const Epi& epi) {
  const int stage_bytes = (J.lp + 1) * kChunk;
  const int nst = kStageRegion / stage_bytes;
  const int nkc = J.K >> 6;
  const int ntc = J.ncols >> 7;
  const int ntile = (J.mrows >> 7) * ntc;
  const int per_tile = J.npass * nkc;
  const int total = ntile * per_tile;
  int prod = 0;
  if (threadIdx.x == 0) {
    bool ok = true;
    for (; prod < total && prod < nst && ok; ++prod)
      ok = produce(J, prod, nst, stage_bytes, stg, S, per_tile, nkc, ntc);
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
        ok = consume(J, g, nst, stage_bytes, stg, S, tmem, c == 0);
        if (ok && g >= 1 && prod < total) {
          ok = produce(J, prod, nst, stage_bytes, stg, S, per_tile, nkc, ntc);
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
      if (J.lp == 2) {
        tmem_ld32(lbase + 128 + cc * 32, v1);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v1[j] = 0u;
      }
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

// Per-item buffers inside the CTA's slot.
struct Work {
  double* x;           // state [2][m][n]
  double* D;           // Jacobian diagonal [m][n]
  double* W;           // J z
  double* V;           // basis, v_j at V + j n2 (unnormalised, scale ctl.s[j])
  float* Z;            // preconditioned basis, z_j at Z + j n2
  __nv_bfloat16* xbf;  // tiled BF16 copy of the current basis vector, [np/64][2 mp][64]
  __nv_bfloat16* t1;   // [mp/64][2 np][64]
  __nv_bfloat16* yh;   // [np/64][2 mp][64]
  __nv_bfloat16* eh;   // [mp/64][2 np][64]
  __nv_bfloat16* el;
  VecCtl* ctl;
};

// z = P^-1 (sc * X) with X the BF16 vector in w.xbf, a1 = a2 = a (eq. P, Section 3.2).
__device__ bool precond(const PersistShape& sh, const Work& w, float* z, float a, float sc,
                        uint8_t* stg, PSmem& S, uint32_t tmem, uint32_t& acc_ctr) {
  const int m = sh.gr.m, n = sh.gr.n, mp = sh.mp, np = sh.np;
  const int mn = m * n;
  {
    __nv_bfloat16* t1 = w.t1;
    const Job j{{w.xbf}, {sh.qrt}, 1, 2 * mp, np, np, 2 * mp, np, 1, 0};
    if (!run_gemm(j, stg, S, tmem, acc_ctr, [=](int r, int c, float x0, float) {
          const int l = r >= mp ? 1 : 0;
          t1[tix(l * np + c, r - l * mp, 2 * np)] = __float2bfloat16(x0);
        }))
      return false;
  }
  {
    __nv_bfloat16* yh = w.yh;
    const float* mu_f = sh.mu_f;
    const float* nu_f = sh.nu_f;
    const Job j{{w.t1}, {sh.qct}, 1, 2 * np, mp, mp, np, mp, 2, np};
    if (!run_gemm(j, stg, S, tmem, acc_ctr, [=](int r, int c, float x0, float x1) {
          // [y_t; y_b] = (1/det) [[nu + a, a], [a, mu + a]] [x_t; x_b] for mode (r, c)
          float y0 = 0.f, y1 = 0.f;
          if (r < n && c < m) {
            const float mu = mu_f[r], nu = nu_f[c];
            const float det = mu * nu + mu * a + nu * a;
            const float inv = sc * __frcp_rn(det);
            y0 = ((nu + a) * x0 + a * x1) * inv;
            y1 = (a * x0 + (mu + a) * x1) * inv;
          }
          yh[tix(c, r, 2 * mp)] = __float2bfloat16(y0);
          yh[tix(mp + c, r, 2 * mp)] = __float2bfloat16(y1);
        }))
      return false;
  }
  {
    __nv_bfloat16* eh = w.eh;
    __nv_bfloat16* el = w.el;
    const Job j{{w.yh, w.yh}, {sh.qr_hi, sh.qr_lo}, 2, 2 * mp, np, np, 2 * mp, np, 1, 0};
    if (!run_gemm(j, stg, S, tmem, acc_ctr, [=](int r, int c, float x0, float) {
          const int l = r >= mp ? 1 : 0;
          const size_t o = tix(l * np + c, r - l * mp, 2 * np);
          const __nv_bfloat16 hi = __float2bfloat16(x0);
          eh[o] = hi;
          el[o] = __float2bfloat16(x0 - __bfloat162float(hi));
        }))
      return false;
  }
  {
    const Job j{{w.eh, w.el, w.eh}, {sh.qc_hi, sh.qc_hi, sh.qc_lo}, 3, 2 * np, mp, mp,
                2 * np, mp, 1, 0};
    if (!run_gemm(j, stg, S, tmem, acc_ctr, [=](int r, int c, float x0, float) {
          const int l = r >= np ? 1 : 0;
          const int jj = r - l * np;
          if (jj < n && c < m) z[(size_t)l * mn + (size_t)c * n + jj] = x0;
        }))
      return false;
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
// Residual of eq. (F) (FP64 cell) into v_0 = F (with its tiled BF16 copy), D, and the Newton
// control.  ZERO: the state is V = 0 (F = -Y, D = g).
template <bool ZERO, bool YAK>
__device__ void residual_phase(const PersistShape& sh, const double* gmap, const double* vin,
                               const Work& w, PSmem& S) {
  const Grid& gr = sh.gr;
  const int m = gr.m, n = gr.n, mn = m * n, mp = sh.mp;
  const double* Vt = w.x;
  const double* Vb = w.x + mn;
  double* Ft = w.V;
  double* Fb = w.V + mn;
  VecCtl& ctl = *w.ctl;
  const bool lin = (gr.b == 0.0);
  const bool norm32 = sh.cfg.newton_rtol * ctl.ynorm > kNorm32Min;
  double sf = 0.0, sd = 0.0;
  float sdf = 0.f, sfh = 0.f, sfl = 0.f;
  bool dnot32 = false;
  const int Si = kPT / n, Sj = kPT - Si * n;
  int i = threadIdx.x / n, j = threadIdx.x - (threadIdx.x / n) * n;
  for (int c = threadIdx.x; c < mn; c += kPT) {
    double ft, fb, dg;
    float dgf = 0.f;
    if (ZERO) {
      ft = (j == 0) ? -gr.g_src * vin[i] : 0.0;
      fb = 0.0;
      dg = gmap[c];
      dgf = d2f_round(dg);
    } else {
      cell_residual<YAK>(gr, i, j, c, Vt, Vb, gmap[c], (j == 0) ? vin[i] : 0.0, ft, fb, dg,
                         dgf);
    }
    Ft[c] = ft;
    Fb[c] = fb;
    w.D[c] = dg;
    {
      const uint32_t dh = (uint32_t)__double2hiint(dg), dlw = (uint32_t)__double2loint(dg);
      const uint32_t de = (dh >> 20) & 0x7FFu;
      dnot32 |= ((dlw & 0x1FFFFFFFu) != 0u) || (de - 897u > 253u && ((dh & 0x7FFFFFFFu) | dlw));
    }
    w.xbf[tix(i, j, 2 * mp)] = d2bf16_bits(ft);
    w.xbf[tix(mp + i, j, 2 * mp)] = d2bf16_bits(fb);
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
    j += Sj;
    i += Si;
    if (j >= n) {
      j -= n;
      ++i;
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
}

// w = J z (eq. J; AM: kApplyF32 or kApplyPair) and h1_j = s_j <V_j, w> for j < nk.
template <int KP, int AM>
__device__ void spmv_phase(const Grid& gr, const Work& w, const float* z, int nk, PSmem& S) {
  const int m = gr.m, n = gr.n, mn = m * n;
  const size_t n2 = 2 * (size_t)mn;
  const float* zt = z;
  const float* zb = z + mn;
  const bool dsplit = w.ctl->d64 != 0;
  double acc[KP];
#pragma unroll
  for (int jv = 0; jv < KP; ++jv) acc[jv] = 0.0;
  const int Si = kPT / n, Sj = kPT - Si * n;
  int i = threadIdx.x / n, jj = threadIdx.x - (threadIdx.x / n) * n;
  for (int c = threadIdx.x; c < mn; c += kPT) {
    double ot, ob;
    if constexpr (AM == kApplyPair) {
      const bool f = (jj == 0), l = (jj == n - 1), u = (i == 0), dn = (i == m - 1);
      apply_pair(zt[c], zb[c], f ? 0.f : zt[c - 1], l ? 0.f : zt[c + 1],
                 u ? 0.f : zb[c - n], dn ? 0.f : zb[c + n], w.D[c],
                 f ? gr.dt0f : (l ? gr.dtlf : gr.dtmf), f ? gr.dt0l : (l ? gr.dtll : gr.dtml),
                 u ? gr.db0f : (dn ? gr.dblf : gr.dbmf), u ? gr.db0l : (dn ? gr.dbll : gr.dbml),
                 gr, ot, ob, dsplit);
    } else {
      const float a = zt[c], bb = zb[c];
      const float cpl = d2f_round(w.D[c]) * (a - bb);
      const float dt = (jj == 0) ? gr.dt0f : ((jj == n - 1) ? gr.dtlf : gr.dtmf);
      const float db = (i == 0) ? gr.db0f : ((i == m - 1) ? gr.dblf : gr.dbmf);
      const float tl = (jj > 0) ? zt[c - 1] : 0.f;
      const float tr = (jj < n - 1) ? zt[c + 1] : 0.f;
      const float bu = (i > 0) ? zb[c - n] : 0.f;
      const float bd = (i < m - 1) ? zb[c + n] : 0.f;
      ot = f2d_bits(fmaf(dt, a, fmaf(-gr.gtf, tl + tr, cpl)));
      ob = f2d_bits(fmaf(db, bb, fmaf(-gr.gbf, bu + bd, -cpl)));
    }
    w.W[c] = ot;
    w.W[mn + c] = ob;
#pragma unroll
    for (int jv = 0; jv < KP; ++jv) {
      if (jv < nk) {
        const double* vj = w.V + (size_t)jv * n2;
        acc[jv] = fma(vj[c], ot, acc[jv]);
        acc[jv] = fma(vj[mn + c], ob, acc[jv]);
      }
    }
    jj += Sj;
    i += Si;
    if (jj >= n) {
      jj -= n;
      ++i;
    }
  }
  block_reduce<KP>(acc, nk, S.h1, w.ctl->s, S);
}

// out = src - sum_j hc_j s_j V_j (j < nk) with its tiled BF16 copy; returns ||out||^2
// (out may alias src).
template <int KP>
__device__ double update_phase(const PersistShape& sh, const Work& w, const double* src,
                               double* out, int nk, const double* hc, PSmem& S) {
  const int n = sh.gr.n, mn = sh.gr.m * n, mp = sh.mp;
  const int n2 = 2 * mn;
  double hj[KP];
#pragma unroll
  for (int jv = 0; jv < KP; ++jv) hj[jv] = (jv < nk) ? hc[jv] * w.ctl->s[jv] : 0.0;
  double acc[1] = {0.0};
  auto finish = [&](int e, double x) {
    out[e] = x;
    const int l = (e >= mn) ? 1 : 0;
    const int cell = e - l * mn;
    const int i = cell / n, j = cell - i * n;
    w.xbf[tix(l * mp + i, j, 2 * mp)] = d2bf16_bits(x);
    acc[0] = fma(x, x, acc[0]);
  };
  int e = threadIdx.x;
  for (; e + 3 * kPT < n2; e += 4 * kPT) {
    double x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = src[e + u * kPT];
#pragma unroll
    for (int jv = 0; jv < KP; ++jv)
      if (jv < nk) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          x[u] = fma(-hj[jv], w.V[(size_t)jv * n2 + e + u * kPT], x[u]);
      }
#pragma unroll
    for (int u = 0; u < 4; ++u) finish(e + u * kPT, x[u]);
  }
  for (; e < n2; e += kPT) {
    double x = src[e];
#pragma unroll
    for (int jv = 0; jv < KP; ++jv)
      if (jv < nk) x = fma(-hj[jv], w.V[(size_t)jv * n2 + e], x);
    finish(e, x);
  }
  block_reduce<1>(acc, 1, S.sc, nullptr, S);
  return S.sc[0];
}

// h2_j = s_j <V_j, u> for j < nk (second Gram-Schmidt pass).
template <int KP>
__device__ void dots_phase(const Work& w, const double* u, int n2, int nk, PSmem& S) {
  double acc[KP];
#pragma unroll
  for (int jv = 0; jv < KP; ++jv) acc[jv] = 0.0;
  for (int e = threadIdx.x; e < n2; e += kPT) {
    const double x = u[e];
#pragma unroll
    for (int jv = 0; jv < KP; ++jv)
      if (jv < nk) acc[jv] = fma(w.V[(size_t)jv * n2 + e], x, acc[jv]);
  }
  block_reduce<KP>(acc, nk, S.h2, w.ctl->s, S);
}

#define MCA_PKP(F, nk, ...)                       \
  do {                                            \
    if ((nk) <= 1) F<1>(__VA_ARGS__);             \
    else if ((nk) <= 2) F<2>(__VA_ARGS__);        \
    else if ((nk) <= 4) F<4>(__VA_ARGS__);        \
    else if ((nk) <= 8) F<8>(__VA_ARGS__);        \
    else if ((nk) <= 16) F<16>(__VA_ARGS__);      \
    else F<32>(__VA_ARGS__);                      \
  } while (0)

template <int KP>
__device__ void spmv_f32(const Grid& gr, const Work& w, const float* z, int nk, PSmem& S) {
  spmv_phase<KP, kApplyF32>(gr, w, z, nk, S);
}
template <int KP>
__device__ void spmv_pair(const Grid& gr, const Work& w, const float* z, int nk, PSmem& S) {
  spmv_phase<KP, kApplyPair>(gr, w, z, nk, S);
}
template <int KP>
__device__ void update_kp(const PersistShape& sh, const Work& w, const double* src, double* out,
                          int nk, const double* hc, PSmem& S, double* hn2) {
  *hn2 = update_phase<KP>(sh, w, src, out, nk, hc, S);
}

// Output currents and the Kirchhoff balance (as k_outputs); copies the state out.
__device__ void outputs_phase(const PersistShape& sh, const PersistItem& it, const Work& w,
                              PersistResult* res, PSmem& S) {
  const Grid& gr = sh.gr;
  const int m = gr.m, n = gr.n, mn = m * n;
  const double* Vt = w.x;
  const double* Vb = w.x + mn;
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
__device__ bool solve_item(const PersistShape& sh, const PersistItem& it, const Work& w,
                           PersistResult* res, uint8_t* stg, PSmem& S, uint32_t tmem,
                           uint32_t& acc_ctr, int restart) {
  const Grid& gr = sh.gr;
  const int m = gr.m, n = gr.n, mn = m * n;
  const int n2 = 2 * mn;
  VecCtl& ctl = *w.ctl;
  const double* gmap = sh.gmaps + (size_t)it.map * mn;
  zero_xbf(sh, w);
  for (int e = threadIdx.x; e < n2; e += kPT) w.x[e] = 0.0;
  {
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < m; i += kPT) acc[0] = fma(it.vin[i], it.vin[i], acc[0]);
    block_reduce<1>(acc, 1, S.sc, nullptr, S);
    if (threadIdx.x == 0) init_ctl(ctl, gr.g_src * sqrt(S.sc[0]), false);
    __syncthreads();
  }
  for (int itn = 0; itn <= sh.cfg.max_newton; ++itn) {
    if (!ctl.newton_active) break;
    if (itn == 0)
      residual_phase<true, false>(sh, gmap, it.vin, w, S);
    else
      residual_phase<false, YAK>(sh, gmap, it.vin, w, S);
    if (!ctl.newton_active) break;
    const bool f32 = (itn == 0) && sh.cfg.eta0 >= kF32ApplyMinEta;
    for (int k = 0; k < restart; ++k) {
      float* zk = w.Z + (size_t)k * n2;
      if (!precond(sh, w, zk, (float)ctl.a, (float)ctl.s[k], stg, S, tmem, acc_ctr))
        return false;
      const int nk = k + 1;
      if (f32)
        MCA_PKP(spmv_f32, nk, gr, w, zk, nk, S);
      else
        MCA_PKP(spmv_pair, nk, gr, w, zk, nk, S);
      double* vnext = w.V + (size_t)(k + 1) * n2;
      double hn2 = 0.0;
      MCA_PKP(update_kp, nk, sh, w, w.W, vnext, nk, S.h1, S, &hn2);
      if (threadIdx.x == 0)
        gram_schmidt_control<false>(ctl, 0, UPD_FIRST, hn2, S.h1, S.h1, nk, restart, nullptr);
      proxy_fence_global();
      __syncthreads();
      if (ctl.reorth) {
        MCA_PKP(dots_phase, nk, w, vnext, n2, nk, S);
        MCA_PKP(update_kp, nk, sh, w, vnext, vnext, nk, S.h2, S, &hn2);
        if (threadIdx.x == 0)
          gram_schmidt_control<false>(ctl, 0, UPD_REORTH, hn2, S.h2, S.h1, nk, restart,
                                      nullptr);
        proxy_fence_global();
        __syncthreads();
      }
      if (!ctl.gm_active) break;
    }
    if (threadIdx.x == 0) lsq_solve(ctl);
    __syncthreads();
    {
      const int kd = ctl.k_done;
      if (threadIdx.x < 32) S.h2[threadIdx.x] = (threadIdx.x < kd) ? ctl.y[threadIdx.x] : 0.0;
      __syncthreads();
      for (int e = threadIdx.x; e < n2; e += kPT) {
        double s = w.x[e];
        const float* zj = w.Z + e;
        for (int j = 0; j < kd; ++j, zj += n2) s = fma(S.h2[j], f2d_bits(*zj), s);
        w.x[e] = s;
      }
      __syncthreads();
    }
  }
  outputs_phase(sh, it, w, res, S);
  __syncthreads();
  return true;
}

// Preconditioner test: z = P^-1 r for r in (vt, vb), written back there.
__device__ bool precond_item(const PersistShape& sh, const PersistItem& it, const Work& w,
                             uint8_t* stg, PSmem& S, uint32_t tmem, uint32_t& acc_ctr) {
  const int m = sh.gr.m, n = sh.gr.n, mn = m * n, mp = sh.mp;
  zero_xbf(sh, w);
  __syncthreads();
  for (int c = threadIdx.x; c < mn; c += kPT) {
    const int i = c / n, j = c - i * n;
    w.xbf[tix(i, j, 2 * mp)] = d2bf16_bits(it.vt[c]);
    w.xbf[tix(mp + i, j, 2 * mp)] = d2bf16_bits(it.vb[c]);
  }
  proxy_fence_global();
  __syncthreads();
  if (!precond(sh, w, w.Z, (float)it.a, 1.f, stg, S, tmem, acc_ctr)) return false;
  for (int c = threadIdx.x; c < mn; c += kPT) {
    it.vt[c] = f2d_bits(w.Z[c]);
    it.vb[c] = f2d_bits(w.Z[mn + c]);
  }
  __syncthreads();
  return true;
}

template <bool YAK>
__global__ void __launch_bounds__(kPT, 2)
k_persist(const PersistShape* __restrict__ shapes, const PersistItem* __restrict__ items,
          int n_items, PersistResult* res, int* queue, int* err, PersistSlots sl, int mode) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* stg = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  PSmem& S = *reinterpret_cast<PSmem*>(stg + kStageRegion);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 3; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.full_par = S.empty_par = S.pending = 0u;
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
  uint32_t acc_ctr = 0;
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(queue, 1);
    __syncthreads();
    const int k = S.item;
    if (k >= n_items || S.err) break;
    const PersistItem it = items[k];
    const PersistShape& sh = shapes[it.shape];
    const bool ok = (mode == 1) ? precond_item(sh, it, w, stg, S, tmem, acc_ctr)
                                : solve_item<YAK>(sh, it, w, res + k, stg, S, tmem, acc_ctr,
                                                  sh.cfg.restart);
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
                         __nv_bfloat16* __restrict__ dst) {
  const size_t total = (size_t)R * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / K), k = (int)(e - (size_t)r * K);
    dst[tix(r, k, R)] = src[e];
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
                    int grid, int mode, bool yak, cudaStream_t s) {
  if (yak)
    k_persist<true><<<grid, kPT, kSmemBytes, s>>>(shapes, items, n_items, res, queue, err, sl,
                                                  mode);
  else
    k_persist<false><<<grid, kPT, kSmemBytes, s>>>(shapes, items, n_items, res, queue, err, sl,
                                                   mode);
}

void launch_retile_bf16(const __nv_bfloat16* src, int R, int K, __nv_bfloat16* dst,
                        cudaStream_t s) {
  const size_t total = (size_t)R * K;
  int nb = (int)((total + 255) / 256);
  if (nb > 1216) nb = 1216;
  k_retile<<<nb, 256, 0, s>>>(src, R, K, dst);
}

}  // namespace mca
