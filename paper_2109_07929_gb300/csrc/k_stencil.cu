// Stencil kernels: the KCL residual with the Jacobian diagonal (eq. F, eq. J), the
// Jacobian apply fused with the first Gram-Schmidt dot pass, Newton control and the
// output currents.
//
// Wire operators (eq. G with terminations): along top row i, node j has diagonal
//   (j > 0 ? g_t : g_src) + (j < n-1 ? g_t : g_term_right) and couplings -g_t to j +- 1;
// along bottom column j, node i has diagonal (i > 0 ? g_b : g_term_top) +
//   (i < m-1 ? g_b : g_sense) and couplings -g_b to i +- 1 (eqs. Gt, Gb: G_t = I (x) G_r,
//   G_b = G_c (x) I in the row-major node order shared by both layers, Section 3.1).
//
// FP64 arithmetic is the scarce resource on this GPU (about 1/64 of the FP32 rate), so the
// kernels keep FP64 instructions per cell low: diagonals are precomputed per position
// class, and the device model uses a short economised polynomial for sinh and FP32 cosh
// instead of the FP64 library functions.
#include <cmath>
#include <cstring>

#include "bits.cuh"
#include "mca_internal.cuh"
#include "twofloat.cuh"
#include "solver_dev.cuh"

namespace mca {

namespace {

// sinh(x) / x ~ sum_k kSinhPoly[k] t^k, t = x^2, on |x| <= kSinhPolyX: the degree-6
// Chebyshev-economised Taylor polynomial (coefficients from gen_sinh_poly.py; truncation
// error below 2e-18 relative).
constexpr double kSinhPolyX = 0.75;
constexpr double kSinhPoly[7] = {
  1.0,                          // t^0
  1.66666666666666380e-01,      // t^1
  8.33333333334163734e-03,      // t^2
  1.98412698324150781e-04,      // t^3
  2.75573237196537609e-06,      // t^4
  2.50509370460377762e-08,      // t^5
  1.62102664139390868e-10,      // t^6
};

// x - (double)(float)x rounded to FP32: the low half of x as an FP32 pair
float low_part(double x) { return (float)(x - (double)(float)x); }

}  // namespace

Grid make_grid(const mca_params& p) {
  Grid g;
  g.m = p.rows;
  g.n = p.cols;
  g.gt = p.g_wire_top;
  g.gb = p.g_wire_bot;
  g.g_src = p.g_src;
  g.g_tr = p.g_term_top_right;
  g.g_bt = p.g_term_bot_top;
  g.g_sense = p.g_sense;
  g.b = p.b;
  g.inv_b = (p.b != 0.0) ? 1.0 / p.b : 0.0;
  g.dt0 = (g.n == 1) ? g.g_src + g.g_tr : g.g_src + g.gt;
  g.dtm = 2.0 * g.gt;
  g.dtl = g.gt + g.g_tr;
  g.db0 = (g.m == 1) ? g.g_bt + g.g_sense : g.g_bt + g.gb;
  g.dbm = 2.0 * g.gb;
  g.dbl = g.gb + g.g_sense;
  // fold b into the polynomial: x = b dV, t = x^2 = b^2 dV^2
  double b2k = 1.0;
  g.tail32 = 1;
  for (int k = 0; k < 7; ++k) {
    g.pc[k] = kSinhPoly[k] * b2k;
    g.pcf[k] = (float)g.pc[k];
    if (k >= 3 && !(g.pc[k] >= 1e-30 && g.pc[k] <= 1e30)) g.tail32 = 0;
    b2k *= p.b * p.b;
  }
  const double lim = (p.b != 0.0) ? kSinhPolyX / fabs(p.b) : 0.0;
  unsigned long long bits;
  memcpy(&bits, &lim, sizeof(bits));
  g.dv_lim_hi = (uint32_t)(bits >> 32);
  g.bf = (float)p.b;
  g.pc1l = low_part(g.pc[1]);
  g.pc2l = low_part(g.pc[2]);
  g.dv_limf = (float)lim;
  g.gsrcf = (float)g.g_src;
  g.gsrcl = low_part(g.g_src);
  g.rneg = (p.device_model == MCA_DEVICE_YAKOPCIC) ? p.neg_ratio : 1.0;
  g.rnegf = (float)g.rneg;
  g.rnegl = low_part(g.rneg);
  g.yak = (g.rneg != 1.0) ? 1 : 0;
  g.gtf = (float)g.gt;
  g.gbf = (float)g.gb;
  g.dt0f = (float)g.dt0;
  g.dtmf = (float)g.dtm;
  g.dtlf = (float)g.dtl;
  g.db0f = (float)g.db0;
  g.dbmf = (float)g.dbm;
  g.dblf = (float)g.dbl;
  g.gtl = low_part(g.gt);
  g.gbl = low_part(g.gb);
  g.dt0l = low_part(g.dt0);
  g.dtml = low_part(g.dtm);
  g.dtll = low_part(g.dtl);
  g.db0l = low_part(g.db0);
  g.dbml = low_part(g.dbm);
  g.dbll = low_part(g.dbl);
  return g;
}

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

// Block-wide sum of three values; result valid in thread 0.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32], sc[kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; sc[w] = c; }
  __syncthreads();
  if (w == 0) {
    a = (l < kThreads / 32) ? sa[l] : 0.0;
    b = (l < kThreads / 32) ? sb[l] : 0.0;
    c = (l < kThreads / 32) ? sc[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
  }
}

// ---- the residual in FP32 pairs ------------------------------------------------------
//
// For Newton iterates far from convergence, whose residual only becomes the right-hand side
// of the next inexact linear solve (every convergence decision is made on the FP64
// residual).  The same cell as cell_residual with every FP64 operand split into an FP32 pair
// (d2f_round / d2f_low, integer pipe) and every product and sum formed error-free
// (two_prod, two_sum); the low parts are summed in FP32 and each result is rounded once to
// FP64.  Besides F and D the cell returns the size of its terms (|wire diagonal x| +
// |wire coupling sum| + |current| + |source|, per layer), from which the Newton control
// bounds the error of ||F||: kPairErrScale times the 2-norm of those sizes.  The exact
// difference is a few 2^-48 of the sizes (the split of each voltage is good to 2^-48, and
// every low part is within 2^-24 of a term that is within 2^-24 of a size); the scale
// leaves a factor of 16 over 2^-44.
//
// FP64 work per cell: the two final additions (the norm then takes two FMAs); the device
// current's polynomial runs in pairs up to t^2 and in FP32 beyond (tail32 is required).

constexpr double kPairErrScale = 1.0 / (double)(1ull << 40);

// BF16 (round to nearest even) of a float; Inf / NaN kept
__device__ __forceinline__ __nv_bfloat16 f2bf16_bits(float x) {
  const uint32_t f = __float_as_uint(x);
  uint32_t r;
  if ((f & 0x7F800000u) == 0x7F800000u)
    r = (f >> 16) | ((f & 0xFFFFu) ? 0x40u : 0u);
  else
    r = (f + 0x7FFFu + ((f >> 16) & 1u)) >> 16;
  __nv_bfloat16_raw raw;
  raw.x = (unsigned short)r;
  return __nv_bfloat16(raw);
}

// current / g of one device, (1 / b) sinh(b dV) for dV = d + dl, as a pair; for
// |b dV| < 3/4: dV P(dV^2) with P - 1 = t (pc1 + t (pc2 + t r)), r the FP32 tail
__device__ __forceinline__ F2 current_pair(const Grid& gr, float d, float dl) {
  if (fabsf(d) < gr.dv_limf) {
    const F2 pm1 = poly_m1_pair(gr, d, dl);                  // P - 1
    const F2 c = mul2(F2{d, dl}, pm1);                       // dV (P - 1)
    float eg;
    const float h = two_sum(d, c.h, eg);
    return F2{h, dl + (c.l + eg)};
  }
  const double x = gr.b * (f2d_bits(d) + f2d_bits(dl));
  return split2(sinh(x) * gr.inv_b);
}

// The pair cell from its voltages already split: vt, vb at (i, j), tl, tr the top layer at
// j - 1, j + 1 and bu, bd the bottom layer at i - 1, i + 1 (zero pairs off the grid).
template <bool YAK>
__device__ __forceinline__ void cell_residual_pair_split(const Grid& gr, int i, int j, F2 vt,
                                                         F2 vb, F2 tl, F2 tr, F2 bu, F2 bd,
                                                         double g64, double vin_i, double& ft,
                                                         double& fb, double& dg, float& dgf,
                                                         float& size2, float& ft32,
                                                         float& fb32) {
  const int m = gr.m, n = gr.n;
  const bool jf = (j == 0), jl = (j == n - 1), iu = (i == 0), il = (i == m - 1);
  const F2 dt{jf ? gr.dt0f : (jl ? gr.dtlf : gr.dtmf), jf ? gr.dt0l : (jl ? gr.dtll : gr.dtml)};
  const F2 db{iu ? gr.db0f : (il ? gr.dblf : gr.dbmf), iu ? gr.db0l : (il ? gr.dbll : gr.dbml)};
  // device voltage dV = d + dl and current g * cg
  float ed;
  const float d = two_sum(vt.h, -vb.h, ed);
  const float dl = ed + (vt.l - vb.l);
  F2 cg = current_pair(gr, d, dl);
  const bool big = !(fabsf(d) < gr.dv_limf);
  if (big) {
    const double dgd = g64 * cosh(gr.b * (f2d_bits(d) + f2d_bits(dl)));
    dg = dgd;
    dgf = d2f_round(dgd);
  } else {
    dgf = d2f_round(g64) * coshf(d * gr.bf);
  }
  if (YAK && (d < 0.f || (d == 0.f && dl < 0.f))) {     // dV < 0
    cg = mul2(cg, F2{gr.rnegf, gr.rnegl});
    dgf *= gr.rnegf;
    if (big) dg *= gr.rneg;
  }
  if (!big) dg = f2d_bits(dgf);
  const F2 cur = mul2(split2(g64), cg);
  // top: dt vt - gt (tl + tr) + cur [- g_src vin]
  const F2 a1 = mul2(vt, dt);
  float es;
  const float st = two_sum(tl.h, tr.h, es);
  const F2 a2 = mul2(F2{st, es + (tl.l + tr.l)}, F2{gr.gtf, gr.gtl});
  float eu, ev;
  const float u = two_sum(a1.h, -a2.h, eu);
  float v = two_sum(u, cur.h, ev);
  float lt = (a1.l - a2.l) + (cur.l + (eu + ev));
  float szt = fabsf(a1.h) + fabsf(a2.h) + fabsf(cur.h);
  if (jf) {
    const F2 a3 = mul2(split2(vin_i), F2{gr.gsrcf, gr.gsrcl});
    float ew;
    v = two_sum(v, -a3.h, ew);
    lt += ew - a3.l;
    szt += fabsf(a3.h);
  }
  // bottom: db vb - gb (bu + bd) - cur
  const F2 b1 = mul2(vb, db);
  float fs;
  const float sb = two_sum(bu.h, bd.h, fs);
  const F2 b2 = mul2(F2{sb, fs + (bu.l + bd.l)}, F2{gr.gbf, gr.gbl});
  float fu, fv;
  const float ub = two_sum(b1.h, -b2.h, fu);
  const float wb = two_sum(ub, -cur.h, fv);
  const float lb = (b1.l - b2.l) + ((fu + fv) - cur.l);
  const float szb = fabsf(b1.h) + fabsf(b2.h) + fabsf(cur.h);
  ft = f2d_bits(v) + f2d_bits(lt);
  fb = f2d_bits(wb) + f2d_bits(lb);
  ft32 = v + lt;
  fb32 = wb + lb;
  size2 = fmaf(szt, szt, fmaf(szb, szb, size2));
}

// The pair cell at c = i n + j, loading and splitting its own six voltages.
template <bool YAK>
__device__ __forceinline__ void cell_residual_pair(const Grid& gr, int i, int j, int c,
                                                   const double* __restrict__ Vt,
                                                   const double* __restrict__ Vb, double g64,
                                                   double vin_i, double& ft, double& fb,
                                                   double& dg, float& dgf, float& size2,
                                                   float& ft32, float& fb32) {
  const int m = gr.m, n = gr.n;
  const F2 z0{0.f, 0.f};
  const F2 vt = split2(Vt[c]), vb = split2(Vb[c]);
  const F2 tl = (j > 0) ? split2(Vt[c - 1]) : z0;
  const F2 tr = (j < n - 1) ? split2(Vt[c + 1]) : z0;
  const F2 bu = (i > 0) ? split2(Vb[c - n]) : z0;
  const F2 bd = (i < m - 1) ? split2(Vb[c + n]) : z0;
  cell_residual_pair_split<YAK>(gr, i, j, vt, vb, tl, tr, bu, bd, g64, vin_i, ft, fb, dg, dgf,
                                size2, ft32, fb32);
}

// Column-strip walk of the pair cells with shared-memory halo staging.  The top layer
// couples a node to j - 1 and j + 1 in its row, the bottom layer to i - 1 and i + 1 in its
// column, and a pair cell needs all six voltages as FP32 pairs.  A split takes a few dozen
// integer instructions, and a cell that splits its own neighbours splits every voltage three
// times (those splits were a third of the pair cell's instructions).  Here the block's cells
// are columns of strips kThreads wide: block bx of nblk owns the units
// [U bx / nblk, U (bx + 1) / nblk) of the strip-major list of U = m * strips (strip, row)
// units, and each thread walks down its column of each strip segment.  The bottom layer's rows i - 1, i, i + 1 stay split in
// registers; the top layer's row is split once into shared memory, with one halo entry on
// each side of the strip (threads 0 and kThreads - 1); the next row's voltages are loaded
// before the current row is evaluated.  Each voltage is split about once (twice per segment
// start for the bottom layer).  fn(i, j, c, vt, vb, tl, tr, bu, bd) evaluates cell
// c = i n + j from its pairs.  Every thread of the block calls this: it synchronises once
// per row (the row buffer alternates, so a row's writes never meet the previous row's
// reads).
__device__ __forceinline__ bool strip_walk_fits(int n) {
  // lanes past n in the last strip idle: walk only when at least 3/4 of them work
  const int strips = (n + kThreads - 1) / kThreads;
  return 4 * n >= 3 * strips * kThreads;
}

template <typename Fn>
__device__ __forceinline__ void pair_strip_walk(int m, int n, const double* __restrict__ Vt,
                                                const double* __restrict__ Vb, int nblk,
                                                Fn&& fn) {
  __shared__ F2 row[2][kThreads + 2];
  const F2 z0{0.f, 0.f};
  const int strips = (n + kThreads - 1) / kThreads;
  const long long U = (long long)m * strips;
  long long u = U * blockIdx.x / nblk;
  const long long u1 = U * (blockIdx.x + 1) / nblk;
  const int t = threadIdx.x;
  int buf = 0;
  while (u < u1) {
    const int st = (int)(u / m);
    const int i0 = (int)(u - (long long)st * m);
    const int i1 = (int)min((long long)m, (long long)i0 + (u1 - u));
    const int j0 = st * kThreads;
    const int j = j0 + t;
    const bool col = j < n;
    // halo columns of the top row: j0 - 1 (thread 0) and j0 + kThreads (the last thread)
    const int jh = (t == 0) ? j0 - 1 : j0 + kThreads;
    const bool halo = (t == 0 && j0 > 0) || (t == kThreads - 1 && jh < n);
    const int hs = (t == 0) ? 0 : kThreads + 1;          // its shared-memory slot
    F2 bu = z0, bc = z0;
    // raw voltages of the current row: Vt[i][j], Vb[i + 1][j] and the halo Vt[i][jh]
    double rt = 0.0, rb = 0.0, rh = 0.0;
    if (col) {
      if (i0 > 0) bu = split2(Vb[(size_t)(i0 - 1) * n + j]);
      bc = split2(Vb[(size_t)i0 * n + j]);
      rt = Vt[(size_t)i0 * n + j];
      if (i0 < m - 1) rb = Vb[(size_t)(i0 + 1) * n + j];
    }
    if (halo) rh = Vt[(size_t)i0 * n + jh];
    for (int i = i0; i < i1; ++i) {
      const F2 vt = split2(rt);
      const F2 bd = (i < m - 1) ? split2(rb) : z0;
      const F2 hv = halo ? split2(rh) : z0;
      if (i + 1 < i1) {
        if (col) {
          rt = Vt[(size_t)(i + 1) * n + j];
          rb = (i + 1 < m - 1) ? Vb[(size_t)(i + 2) * n + j] : 0.0;
        }
        if (halo) rh = Vt[(size_t)(i + 1) * n + jh];
      }
      row[buf][t + 1] = vt;
      if (halo) row[buf][hs] = hv;
      __syncthreads();
      if (col) {
        const F2 tl = (j > 0) ? row[buf][t] : z0;
        const F2 tr = (j < n - 1) ? row[buf][t + 2] : z0;
        fn(i, j, i * n + j, vt, bc, tl, tr, bu, bd);
      }
      bu = bc;
      bc = bd;
      buf ^= 1;
    }
    u += i1 - i0;
  }
}

__global__ void k_setup_vectors(Grid gr, const double* __restrict__ vin, VecCtl* ctl,
                                int warm) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < gr.m; i += blockDim.x) {
    const double v = vin[(size_t)b * gr.m + i];
    s += v * v;
  }
  double dummy = 0.0;
  block_sum2(s, dummy);
  if (threadIdx.x == 0) {
    init_ctl(ctl[b], gr.g_src * sqrt(s), warm != 0);
  }
}

// K1: F = blockdiag(G_t, G_b) x + [i; -i] - [Y_t; 0] and D = g cosh(b dV) per cell, with
// per-block partial sums of ||F||^2 and sum(D) (PAIR: the FP32-pair cell, and a third
// partial sum, of the squared term sizes).
template <bool YAK, bool PAIR>
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
  // sum(D): FP64 for linear devices, where a = mean(D) must equal a uniform D to FP64
  // rounding for the preconditioner to be exact (one GMRES iteration); otherwise D itself
  // is FP32 and so is its sum within a thread
  const bool lin = (gr.b == 0.0);
  double sf = 0.0, sd = 0.0;
  float sdf = 0.f, ss = 0.f;
  auto emit = [&](int c, double ft, double fb, double dg, float dgf) {
    Ft[c] = ft;
    Fb[c] = fb;
    Db[c] = dg;
    sf = fma(ft, ft, sf);
    sf = fma(fb, fb, sf);
    if (lin) sd += dg; else sdf += dgf;
  };
  bool walked = false;
  if constexpr (PAIR) {
    if (strip_walk_fits(n)) {
      pair_strip_walk(m, n, Vt, Vb, nblk,
                      [&](int i, int j, int c, F2 vt, F2 vb, F2 tl, F2 tr, F2 bu, F2 bd) {
                        double ft, fb, dg;
                        float dgf, f32a, f32b;
                        cell_residual_pair_split<YAK>(gr, i, j, vt, vb, tl, tr, bu, bd, gmap[c],
                                                      (j == 0) ? vinb[i] : 0.0, ft, fb, dg,
                                                      dgf, ss, f32a, f32b);
                        emit(c, ft, fb, dg, dgf);
                      });
      walked = true;
    }
  }
  if (!walked) {
    for (int c = blockIdx.x * kThreads + threadIdx.x; c < mn; c += nblk * kThreads) {
      const int i = c / n;
      const int j = c - i * n;
      double ft, fb, dg;
      float dgf;
      float f32a, f32b;
      if constexpr (PAIR)
        cell_residual_pair<YAK>(gr, i, j, c, Vt, Vb, gmap[c], (j == 0) ? vinb[i] : 0.0, ft, fb,
                                dg, dgf, ss, f32a, f32b);
      else
        cell_residual<YAK>(gr, i, j, c, Vt, Vb, gmap[c], (j == 0) ? vinb[i] : 0.0, ft, fb, dg,
                           dgf);
      emit(c, ft, fb, dg, dgf);
    }
  }
  sd += f2d_bits(sdf);
  double sz = f2d_bits(ss);
  block_sum3(sf, sd, sz);
  if (threadIdx.x == 0) {
    part[((size_t)b * 32 + 0) * nblk + blockIdx.x] = sf;
    part[((size_t)b * 32 + 1) * nblk + blockIdx.x] = sd;
    if (PAIR) part[((size_t)b * 32 + 2) * nblk + blockIdx.x] = sz;
  }
}

// Residual of the solver loop with the Newton control in the last block of each vector.
// ZERO: the state is x = 0 (first Newton step from V = 0), where F = -Y and D = g.
// PAIR: the FP32-pair cell for vectors far from convergence, whose ||F|| comes with an
// error bound (see newton_control), the FP64 cell for the others.
// confirm: only vectors flagged need_fp64 by a PAIR launch run (the FP64 decision).
// F[b] is written at F + b*fstride: the solver points it at the first Krylov basis vector,
// which GMRES keeps unnormalised (v_0 = -F / ||F||, the scale set by the Newton control),
// and xbf (may be NULL) receives its BF16 copy for the tensor-core preconditioner.
template <bool ZERO, bool YAK, bool PAIR>
__global__ void __launch_bounds__(kThreads, 4)
k_residual_newton(Grid gr, const double* __restrict__ gmaps, const int* __restrict__ map_of,
                  const double* __restrict__ vin,
                  const double* __restrict__ x, double* __restrict__ F, size_t fstride,
                  __nv_bfloat16* __restrict__ xbf, int mp, int np,
                  double* __restrict__ D, double* __restrict__ part, int nblk, VecCtl* ctl,
                  SolverCfg cfg, unsigned int* cnt, int32_t* host_flags, int opts) {
  const int b = blockIdx.y;
  const bool confirm = (opts & 1) != 0;
  // the zero state's F = -Y is zero off the first column of the top layer; with sparse_f
  // only that column is stored (the first Newton step's kernels read v_0 there only)
  const bool sparse_f = ZERO && (opts & 2) != 0;
  if (confirm ? !ctl[b].need_fp64 : !ctl[b].newton_active) return;
  // PAIR: a vector whose last linear solve ended within kPairMinRatio of the target (its
  // new residual may decide convergence) takes the FP64 cell right away
  const bool use_pair =
      PAIR && !(ctl[b].res_est <= kPairMinRatio * cfg.newton_rtol * ctl[b].ynorm);
  const int m = gr.m, n = gr.n;
  const int mn = m * n;
  // conductance map of this vector's crossbar (several crossbars of one shape share a batch)
  const double* gmap = gmaps + (map_of ? (size_t)map_of[b] * mn : (size_t)0);
  const double* Vt = x + (size_t)b * 2 * mn;
  const double* Vb = Vt + mn;
  double* Ft = F + (size_t)b * fstride;
  double* Fb = Ft + mn;
  __nv_bfloat16* xt = xbf ? xbf + (size_t)b * 2 * mp * np : nullptr;
  double* Db = D + (size_t)b * mn;
  const double* vinb = vin + (size_t)b * m;
  // sum(D): FP64 for linear devices, where a = mean(D) must equal a uniform D to FP64
  // rounding for the preconditioner to be exact (one GMRES iteration); otherwise D itself
  // is FP32 and so is its sum within a thread
  const bool lin = (gr.b == 0.0);
  // ||F||^2 of the FP64 cell: the squares of the FP32-rounded entries summed in FP32 with
  // compensation (TwoSum), within about 1e-7 relative, when the convergence threshold
  // newton_rtol ||Y|| exceeds kNorm32Min: every entry that can matter for the test is
  // then far inside the FP32 range.  Otherwise FP64 FMAs.  The zero state needs no sum:
  // F(0) = -Y, so ||F|| = ||Y||.
  const bool norm32 = cfg.newton_rtol * ctl[b].ynorm > kNorm32Min;
  double sf = 0.0, sd = 0.0;
  float sdf = 0.f, ss = 0.f, sfh = 0.f, sfl = 0.f;
  bool dnot32 = false;
  // grid-stride walk over the cells with (i, j) advanced incrementally (no division per
  // cell); the BF16 copy sits in the padded [layer][mp][np] layout at row offset i * np
  // the stores and sums of one cell (both cell forms and both walks)
  auto emit = [&](int i, int j, int c, double ft, double fb, double dg, float dgf, float ft32,
                  float fb32) {
    if (!sparse_f || j == 0) Ft[c] = ft;
    if (!sparse_f) Fb[c] = fb;
    Db[c] = dg;
    {
      // D is an FP32 number when its low 29 mantissa bits are clear and its exponent is
      // in the FP32 normal range (or D = 0)
      const uint32_t dh = (uint32_t)__double2hiint(dg), dlw = (uint32_t)__double2loint(dg);
      const uint32_t de = (dh >> 20) & 0x7FFu;
      dnot32 |= ((dlw & 0x1FFFFFFFu) != 0u) || (de - 897u > 253u && ((dh & 0x7FFFFFFFu) | dlw));
    }
    if (xt != nullptr) {
      const int o = i * np + j;
      if (PAIR && use_pair) {
        xt[o] = f2bf16_bits(ft32);
        xt[o + mp * np] = f2bf16_bits(fb32);
      } else {
        xt[o] = d2bf16_bits(ft);
        xt[o + mp * np] = d2bf16_bits(fb);
      }
    }
    if (!ZERO) {
      if ((PAIR && use_pair) || !norm32) {
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
  };
  bool walked = false;
  if constexpr (PAIR && !ZERO) {
    // pair cells of a grid whose columns fill the strips: split each voltage once
    if (use_pair && strip_walk_fits(n)) {
      pair_strip_walk(m, n, Vt, Vb, nblk,
                      [&](int i, int j, int c, F2 vt, F2 vb, F2 tl, F2 tr, F2 bu, F2 bd) {
                        double ft, fb, dg;
                        float dgf, ft32, fb32;
                        cell_residual_pair_split<YAK>(gr, i, j, vt, vb, tl, tr, bu, bd, gmap[c],
                                                      (j == 0) ? vinb[i] : 0.0, ft, fb, dg,
                                                      dgf, ss, ft32, fb32);
                        emit(i, j, c, ft, fb, dg, dgf, ft32, fb32);
                      });
      walked = true;
    }
  }
  if (!walked) {
    const int S = nblk * kThreads;
    const int Si = S / n, Sj = S - Si * n;
    int c = blockIdx.x * kThreads + threadIdx.x;
    int i = c / n, j = c - (c / n) * n;
    for (; c < mn; c += S) {
      double ft, fb, dg;
      float dgf = 0.f, ft32 = 0.f, fb32 = 0.f;
      if (ZERO) {
        ft = (j == 0) ? -gr.g_src * vinb[i] : 0.0;
        fb = 0.0;
        dg = gmap[c];
        dgf = d2f_round(dg);
      } else if (PAIR && use_pair) {
        cell_residual_pair<YAK>(gr, i, j, c, Vt, Vb, gmap[c], (j == 0) ? vinb[i] : 0.0, ft, fb,
                                dg, dgf, ss, ft32, fb32);
      } else {
        cell_residual<YAK>(gr, i, j, c, Vt, Vb, gmap[c], (j == 0) ? vinb[i] : 0.0, ft, fb, dg,
                           dgf);
      }
      emit(i, j, c, ft, fb, dg, dgf, ft32, fb32);
      j += Sj;
      i += Si;
      if (j >= n) {
        j -= n;
        ++i;
      }
    }
  }
  sd += f2d_bits(sdf);
  sf += f2d_bits(sfh) + f2d_bits(sfl);
  double sz = f2d_bits(ss);
  if (__syncthreads_or(dnot32) && threadIdx.x == 0) atomicOr(&ctl[b].d64_next, 1);
  if (PAIR)
    block_sum3(sf, sd, sz);
  else
    block_sum2(sf, sd);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[((size_t)b * 32 + 0) * nblk + blockIdx.x] = sf;
    part[((size_t)b * 32 + 1) * nblk + blockIdx.x] = sd;
    if (PAIR) part[((size_t)b * 32 + 2) * nblk + blockIdx.x] = sz;
    __threadfence();
    last = (atomicAdd(&cnt[b], 1u) == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order sum over blocks: warp 0 -> ||F||^2, warp 1 -> sum(D), warp 2 -> the
  // squared term sizes (PAIR)
  constexpr int kRows = PAIR ? 3 : 2;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __shared__ double tot[3];
  if (w < kRows) {
    double s = 0.0;
    for (int t = l; t < nblk; t += 32) s += __ldcg(&part[((size_t)b * 32 + w) * nblk + t]);
    s = warp_sum(s);
    if (l == 0) tot[w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cnt[b] = 0;
    const double f2 = ZERO ? ctl[b].ynorm * ctl[b].ynorm : tot[0];
    newton_control(ctl[b], f2, tot[1], mn, cfg, host_flags ? &host_flags[b] : nullptr,
                   use_pair ? kPairErrScale * sqrt(tot[2]) : -1.0);
  }
}

// v_0 = sign * F / ||F|| (GMRES from dx = 0; sign = -1 for the Newton system J dx = -F)
// and its BF16 copy in the padded [layer][mp][np] layout read by the tensor-core
// preconditioner.
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
      xbf[(((size_t)b * 2 + l) * mp + i) * np + j] = d2bf16_bits(val);
    }
  }
}

// Deterministic reduction of part[b][j][0..nblk) (j < nk) into h[b][j] by the whole
// block (warp w sums rows w, w + 8, ...).
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

// K2 fused with the first classical Gram-Schmidt pass: w = J z for one cell (both
// layers), then partial dots <V_j, w> for j < nk; the last block of each vector reduces
// the partials into h.
// z is FP64, or FP32 (the tensor-core preconditioner's accumulators, widened exactly).
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f2d_bits(x); }

template <int KP, typename ZT, int AM, bool ZS = false>
__global__ void __launch_bounds__(kThreads)
k_spmv_dots(Grid gr, const double* __restrict__ D, const ZT* __restrict__ z,
            size_t zstride, double* __restrict__ w, const double* __restrict__ V,
            size_t vstride, int nk, double* __restrict__ part, int nblk,
            const VecCtl* __restrict__ ctl, unsigned int* cnt, double* h) {
  const int b = blockIdx.y;
  if (ctl != nullptr && !ctl[b].gm_active) return;
  // the pair apply skips the split of D when every entry is an FP32 number
  const bool dsplit = (ctl == nullptr) || ctl[b].d64;
  const int m = gr.m, n = gr.n, mn = m * n;
  const size_t n2 = 2 * (size_t)mn;
  const ZT* zt = z + (size_t)b * zstride;
  const ZT* zb = zt + mn;
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
    double ot, ob;
    if constexpr (AM == kApplyPair) {
      const bool f = (jj == 0), l = (jj == n - 1), u = (i == 0), dn = (i == m - 1);
      apply_pair(zt[c], zb[c], f ? 0.f : (float)zt[c - 1], l ? 0.f : (float)zt[c + 1],
                 u ? 0.f : (float)zb[c - n], dn ? 0.f : (float)zb[c + n], Db[c],
                 f ? gr.dt0f : (l ? gr.dtlf : gr.dtmf), f ? gr.dt0l : (l ? gr.dtll : gr.dtml),
                 u ? gr.db0f : (dn ? gr.dblf : gr.dbmf), u ? gr.db0l : (dn ? gr.dbll : gr.dbml),
                 gr, ot, ob, dsplit);
    } else if constexpr (AM == kApplyF32) {
      // FP32 apply (z is FP32 here): the same formula, rounded to FP32, widened exactly
      const float a = zt[c], bb = zb[c];
      const float cpl = d2f_round(Db[c]) * (a - bb);
      const float dt = (jj == 0) ? gr.dt0f : ((jj == n - 1) ? gr.dtlf : gr.dtmf);
      const float db = (i == 0) ? gr.db0f : ((i == m - 1) ? gr.dblf : gr.dbmf);
      const float tl = (jj > 0) ? (float)zt[c - 1] : 0.f;
      const float tr = (jj < n - 1) ? (float)zt[c + 1] : 0.f;
      const float bu = (i > 0) ? (float)zb[c - n] : 0.f;
      const float bd = (i < m - 1) ? (float)zb[c + n] : 0.f;
      ot = f2d_bits(fmaf(dt, a, fmaf(-gr.gtf, tl + tr, cpl)));
      ob = f2d_bits(fmaf(db, bb, fmaf(-gr.gbf, bu + bd, -cpl)));
    } else {
      const double a = widen(zt[c]), bb = widen(zb[c]);
      const double cpl = Db[c] * (a - bb);
      const double dt = (jj == 0) ? gr.dt0 : ((jj == n - 1) ? gr.dtl : gr.dtm);
      const double db = (i == 0) ? gr.db0 : ((i == m - 1) ? gr.dbl : gr.dbm);
      const double tl = (jj > 0) ? widen(zt[c - 1]) : 0.0;
      const double tr = (jj < n - 1) ? widen(zt[c + 1]) : 0.0;
      const double bu = (i > 0) ? widen(zb[c - n]) : 0.0;
      const double bd = (i < m - 1) ? widen(zb[c + n]) : 0.0;
      ot = fma(dt, a, fma(-gr.gt, tl + tr, cpl));
      ob = fma(db, bb, fma(-gr.gb, bu + bd, -cpl));
    }
    wt[c] = ot;
    wb[c] = ob;
    if (V != nullptr) {
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        if (j < nk) {
          const double* vj = Vb_ + (size_t)j * n2;
          if (ZS && j == 0) {            // v_0 of the zero state: first top column only
            if (jj == 0) acc[0] = fma(vj[c], ot, acc[0]);
          } else {
            acc[j] = fma(vj[c], ot, acc[j]);
            acc[j] = fma(vj[mn + c], ob, acc[j]);
          }
        }
      }
    }
  }
  if (V == nullptr) return;
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
  if (cnt == nullptr) return;
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&cnt[b], 1u) == (unsigned)nblk - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the stored basis is unnormalised: <v_j, w> = s_j <V_j, w>
  block_reduce_rows(part, b, nblk, nk, h, ctl ? ctl[b].s : nullptr);
  if (threadIdx.x == 0) cnt[b] = 0;
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

int residual_nblk(int mn, int B) {
  constexpr int kGridBlocks = 152 * 32;
  int nb = (mn + kThreads - 1) / kThreads;
  const int want = (kGridBlocks + B - 1) / (B < 1 ? 1 : B);
  if (nb > want) nb = want;
  if (nb > kResidualMaxBlocks) nb = kResidualMaxBlocks;
  return nb < 1 ? 1 : nb;
}

void launch_setup_vectors(const Grid& gr, const double* vin, int B, VecCtl* ctl, bool warm,
                          cudaStream_t s) {
  k_setup_vectors<<<B, kThreads, 0, s>>>(gr, vin, ctl, warm ? 1 : 0);
}

void launch_residual(const Grid& gr, const double* gmap, const double* vin, const double* x,
                     double* F, double* D, double* part, int nblk, int B, const VecCtl* ctl,
                     cudaStream_t s, bool pair) {
  const dim3 grid(nblk, B);
#define MCA_RES(Y_, P_) \
  k_residual<Y_, P_><<<grid, kThreads, 0, s>>>(gr, gmap, vin, x, F, D, part, nblk, ctl)
  if (gr.yak) {
    if (pair) MCA_RES(true, true); else MCA_RES(true, false);
  } else {
    if (pair) MCA_RES(false, true); else MCA_RES(false, false);
  }
#undef MCA_RES
}

double pair_err_bound(double size2_sum) { return kPairErrScale * std::sqrt(size2_sum); }

void launch_residual_newton(const Grid& gr, const double* gmaps, const int* map_of,
                            const double* vin, const double* x, bool zero_state, double* F,
                            size_t fstride, __nv_bfloat16* xbf, int mp, int np, double* D,
                            double* part, int nblk, int B, VecCtl* ctl, SolverCfg cfg,
                            unsigned int* cnt, int32_t* host_flags, cudaStream_t s, bool pair,
                            bool confirm, bool sparse_f) {
  dim3 grid(nblk, B);
  const int opts = (confirm ? 1 : 0) | (sparse_f ? 2 : 0);
#define MCA_RESN(Z_, Y_, P_)                                                                \
  k_residual_newton<Z_, Y_, P_><<<grid, kThreads, 0, s>>>(gr, gmaps, map_of, vin, x, F,      \
                                                          fstride, xbf, mp, np, D, part,     \
                                                          nblk, ctl, cfg, cnt, host_flags,   \
                                                          opts)
  // (the zero state has dV = 0 everywhere: no device is under negative bias)
  if (zero_state)
    MCA_RESN(true, false, false);
  else if (gr.yak)
    if (pair) MCA_RESN(false, true, true); else MCA_RESN(false, true, false);
  else
    if (pair) MCA_RESN(false, false, true); else MCA_RESN(false, false, false);
#undef MCA_RESN
}

void launch_init_basis(const double* F, double sign, double* V0, size_t vstride,
                       __nv_bfloat16* xbf, int mp, int np, int m, int n, const VecCtl* ctl,
                       int B, cudaStream_t s) {
  const size_t n2 = 2 * (size_t)m * n;
  int nb = (int)((n2 + kThreads - 1) / kThreads);
  if (nb > 1216) nb = 1216;
  k_init_basis<<<dim3(nb, B), kThreads, 0, s>>>(F, sign, V0, vstride, xbf, mp, np, m, n, ctl);
}

template <typename ZT, int AM, bool ZS = false>
void spmv_dots(const Grid& gr, const double* D, const ZT* z, size_t zstride, double* w,
               const double* V, size_t vstride, int nk, double* part, int nblk, int B,
               const VecCtl* ctl, unsigned int* cnt, double* h, cudaStream_t s) {
  // z: the vector of batch entry 0, later entries zstride doubles apart; V: basis vector
  // 0 of batch entry 0 (nk vectors N2 apart, entries vstride apart), or NULL.
  dim3 grid(nblk, B);
#define MCA_SPMV(KP_)                                                                      \
  k_spmv_dots<KP_, ZT, AM, ZS><<<grid, kThreads, 0, s>>>(gr, D, z, zstride, w, V, vstride, nk, \
                                                      part, nblk, ctl, cnt, h)
  if (nk <= 1) MCA_SPMV(1);
  else if (nk <= 2) MCA_SPMV(2);
  else if (nk <= 4) MCA_SPMV(4);
  else if (nk <= 8) MCA_SPMV(8);
  else if (nk <= 16) MCA_SPMV(16);
  else MCA_SPMV(32);
#undef MCA_SPMV
}

void launch_spmv_dots(const Grid& gr, const double* D, const double* z, size_t zstride,
                      double* w, const double* V, size_t vstride, int nk, double* part,
                      int nblk, int B, const VecCtl* ctl, unsigned int* cnt, double* h,
                      cudaStream_t s) {
  spmv_dots<double, kApplyF64>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, B, ctl, cnt, h,
                           s);
}

void launch_spmv_dots(const Grid& gr, const double* D, const float* z, size_t zstride,
                      double* w, const double* V, size_t vstride, int nk, double* part,
                      int nblk, int B, const VecCtl* ctl, unsigned int* cnt, double* h,
                      cudaStream_t s, int apply) {
  if (apply == kApplyF32Zero)
    spmv_dots<float, kApplyF32, true>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, B, ctl,
                                      cnt, h, s);
  else if (apply == kApplyF32)
    spmv_dots<float, kApplyF32>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, B, ctl, cnt,
                                h, s);
  else if (apply == kApplyF64)
    spmv_dots<float, kApplyF64>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, B, ctl, cnt,
                                h, s);
  else
    spmv_dots<float, kApplyPair>(gr, D, z, zstride, w, V, vstride, nk, part, nblk, B, ctl, cnt,
                                 h, s);
}

void launch_outputs(const Grid& gr, const double* vin, const double* x, double* i_out,
                    double* kcl, int B, cudaStream_t s) {
  k_outputs<<<B, kThreads, 0, s>>>(gr, vin, x, i_out, kcl);
}

}  // namespace mca
