// Device-side pieces of the solver shared by the batched kernels (one vector per grid
// row of blocks) and the persistent whole-solve kernel (one solve per CTA): FP32-pair
// arithmetic, the memristor current, one cell of the KCL residual (eq. F) and of the
// Jacobian apply (eq. J), the Newton control (eq. Newton3) and the Givens column of
// flexible GMRES.  Included inside namespace mca; every definition has internal linkage.
#pragma once
#include "bits.cuh"
#include "mca_internal.cuh"
#include "twofloat.cuh"

namespace mca {
namespace {

constexpr double kEps = 1.1102230246251565e-16;   // 2^-53, unit roundoff of FP64
constexpr double kOrthTol = 1e-8;                 // largest accepted loss of orthogonality

// smallest convergence threshold newton_rtol ||Y|| for which the FP64 residual's ||F||^2 is
// summed in FP32: entries that matter against it are above 1e-13 / sqrt(2 m n), whose
// squares are normal FP32 numbers for any size this library takes
constexpr double kNorm32Min = 1e-13;
// the pair residual is used only for iterates more than this factor above the target
constexpr double kPairMinRatio = 10.0;

// ---- FP32 pairs: a value held as the unevaluated sum h + l of two floats -------------

struct F2 {
  float h, l;   // unevaluated sum h + l
};

// x as an FP32 pair (d2f_round(x), d2f_low(x)); one range test selects the common case
// 2^-74 <= |x| < 2^128, where both halves come from the two 32-bit words directly.
__device__ __forceinline__ F2 split2(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t ex = (hi >> 20) & 0x7FFu;
  if (ex - 949u <= 201u) {
    const uint32_t lo2 = lo + (1u << 28);                       // round at mantissa bit 29
    const uint32_t hi2 = hi + (lo2 < lo ? 1u : 0u);
    const uint32_t hb = ((((hi2 & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lo2 >> 29)) |
                        (hi & 0x80000000u);                      // exponent rebiased by 896
    const int32_t dl = (int32_t)(lo - (lo2 & 0xE0000000u));      // x - hi in ulps of x
    const float mag = u29_to_float((uint32_t)(dl < 0 ? -dl : dl)) *
                      __int_as_float((int)(ex - 948u) << 23);
    const uint32_t sg = (hi & 0x80000000u) ^ (dl < 0 ? 0x80000000u : 0u);
    return F2{__uint_as_float(hb), __uint_as_float(__float_as_uint(mag) ^ sg)};
  }
  return F2{d2f_round(x), d2f_low(x)};
}

// a * b for a pair a and an FP32 pair b, as a pair (not renormalised)
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  float e;
  const float p = two_prod(a.h, b.h, e);
  return F2{p, fmaf(a.h, b.l, fmaf(a.l, b.h, e))};
}

// P(dV^2) - 1 = t (pc1 + t (pc2 + t r)), t = dV^2, for dV = d + dl as an FP32 pair, with the
// polynomial's tail r = pc3 + pc4 t + pc5 t^2 + pc6 t^3 in FP32 (at most x^6 / 5040 < 3.5e-5
// of P for x = b dV, |x| < 3/4): error-free FP32 products and sums (two_prod, two_sum), the
// low parts added in FP32.  The result carries the FP32 tail's relative error (below
// 3e-11 of P - 1) and a few 2^-44 from the pair arithmetic.
__device__ __forceinline__ F2 poly_m1_pair(const Grid& gr, float d, float dl) {
  float et;
  const float t = two_prod(d, d, et);
  const float tl = fmaf(2.f * d, dl, et);                   // dV^2 = t + tl
  float r = fmaf(gr.pcf[6], t, gr.pcf[5]);
  r = fmaf(r, t, gr.pcf[4]);
  r = fmaf(r, t, gr.pcf[3]);
  float ea, eb, ec, ed;
  const float a = two_prod(t, r, ea);
  const float q2 = two_sum(gr.pcf[2], a, eb);
  const float q2l = (gr.pc2l + fmaf(tl, r, ea)) + eb;        // pc2 + t r
  const float bq = two_prod(t, q2, ec);
  const float bql = fmaf(t, q2l, fmaf(tl, q2, ec));
  const float q1 = two_sum(gr.pcf[1], bq, ed);
  const float q1l = (gr.pc1l + bql) + ed;                    // pc1 + t q2
  return mul2(F2{t, tl}, F2{q1, q1l});                       // P - 1
}

// Memristor current and conductance for the FP64 residual.  The current
// (g / b) sinh(b dV) = g dV P(dV^2) with P(dV^2) = sinh(x) / x, x = b dV, enters the KCL
// residual at FP64 accuracy: for |x| < 3/4 (range test on the high word, integer pipe),
// P - 1 comes from the FP32-pair polynomial above (b folded into its coefficients), is
// rounded once to FP64, and cur = fma(g dV, P - 1, g dV): three FP64 instructions where a
// Horner evaluation in FP64 takes seven.  Outside that range the CUDA math library.  The
// conductance g cosh(x) only shapes the Newton matrix (the Jacobian diagonal and
// a = mean(D)), so it is evaluated in FP32 (relative error below 3e-7, which changes the
// inexact Newton steps but not the solution the FP64 residual drives them to) and returned
// both as float and widened.
__device__ __forceinline__ void device_current(const Grid& gr, double g, double dv,
                                               double& cur, double& dg, float& dgf) {
  if (((uint32_t)__double2hiint(dv) & 0x7FFFFFFFu) < gr.dv_lim_hi && gr.tail32) {
    const F2 d = split2(dv);
    const F2 q = poly_m1_pair(gr, d.h, d.l);
    const double gd = g * dv;
    cur = fma(gd, f2d_bits(q.h) + f2d_bits(q.l), gd);
    dgf = d2f_round(g) * coshf(d.h * gr.bf);
    dg = f2d_bits(dgf);
  } else if (((uint32_t)__double2hiint(dv) & 0x7FFFFFFFu) < gr.dv_lim_hi) {
    // b outside the FP32 tail's range: Horner in FP64
    const double t = dv * dv;
    double ps = gr.pc[6];
    ps = fma(ps, t, gr.pc[5]);
    ps = fma(ps, t, gr.pc[4]);
    ps = fma(ps, t, gr.pc[3]);
    ps = fma(ps, t, gr.pc[2]);
    ps = fma(ps, t, gr.pc[1]);
    ps = fma(ps, t, gr.pc[0]);
    cur = g * (dv * ps);
    dgf = d2f_round(g) * coshf(d2f_round(dv) * gr.bf);
    dg = f2d_bits(dgf);
  } else {
    const double x = gr.b * dv;
    cur = g * (sinh(x) * gr.inv_b);
    dg = g * cosh(x);
    dgf = d2f_round(dg);
  }
}

// Yakopcic-form device: scale the current and the conductance of a device under negative
// bias (sign read from the bit pattern, on the integer pipe).
__device__ __forceinline__ void negative_bias(const Grid& gr, double dv, double& cur,
                                              double& dg, float& dgf) {
  const uint32_t hi = (uint32_t)__double2hiint(dv), lo = (uint32_t)__double2loint(dv);
  if ((hi >> 31) && ((hi & 0x7FFFFFFFu) | lo)) {   // dV < 0, not -0
    cur *= gr.rneg;
    dg *= gr.rneg;
    dgf *= gr.rnegf;
  }
}

// One cell of eq. (F) and the Jacobian diagonal; returns (F_t, F_b, D).  YAK: the
// Yakopcic-form device (a compile-time choice, so the sinh device pays nothing for it).
// FP64 instructions: the device voltage 1, the current 3 (device_current), and per layer
// the neighbour sum and two FMAs that add the wire diagonal term and the coupling term to
// the current (10 in all; the source term adds one on the first column).
// The arithmetic of cell_residual on the cell's loaded voltages (vt, vb), its neighbours
// (tl, tr along the top row, bu, bd along the bottom column; 0 outside the array) and g.
template <bool YAK>
__device__ __forceinline__ void cell_residual_vals(const Grid& gr, int i, int j, double vt,
                                                   double vb, double tl, double tr,
                                                   double bu, double bd, double g,
                                                   double vin_i, double& ft, double& fb,
                                                   double& dg, float& dgf) {
  const int m = gr.m, n = gr.n;
  const double dt = (j == 0) ? gr.dt0 : ((j == n - 1) ? gr.dtl : gr.dtm);
  const double db = (i == 0) ? gr.db0 : ((i == m - 1) ? gr.dbl : gr.dbm);
  const double dv = vt - vb;
  double cur;                                    // device current, top to bottom
  if (gr.b != 0.0) {
    device_current(gr, g, dv, cur, dg, dgf);
  } else {
    cur = g * dv;
    dg = g;
    dgf = 0.f;
  }
  if (YAK) negative_bias(gr, dv, cur, dg, dgf);
  ft = fma(-gr.gt, tl + tr, fma(dt, vt, cur));
  if (j == 0) ft = fma(-gr.g_src, vin_i, ft);
  fb = fma(-gr.gb, bu + bd, fma(db, vb, -cur));
}

template <bool YAK>
__device__ __forceinline__ void cell_residual(const Grid& gr, int i, int j, int c,
                                              const double* __restrict__ Vt,
                                              const double* __restrict__ Vb, double g,
                                              double vin_i, double& ft, double& fb,
                                              double& dg, float& dgf) {
  const int m = gr.m, n = gr.n;
  const double vt = Vt[c], vb = Vb[c];
  const double tl = (j > 0) ? Vt[c - 1] : 0.0;
  const double tr = (j < n - 1) ? Vt[c + 1] : 0.0;
  const double bu = (i > 0) ? Vb[c - n] : 0.0;
  const double bd = (i < m - 1) ? Vb[c + n] : 0.0;
  cell_residual_vals<YAK>(gr, i, j, vt, vb, tl, tr, bu, bd, g, vin_i, ft, fb, dg, dgf);
}

// One cell of w = J z in FP32 pairs (ApplyMode kApplyPair).  The FP32 inputs a = z_t,
// bb = z_b and the neighbours enter error-free products with the FP32 halves of the wire
// constants and of D, and error-free sums; the low parts (each within 2^-24 of its term)
// are added in FP32 and the pair is rounded once to FP64.  D (a - bb) is shared by the
// two layers.  FP64 work: splitting D and the two final additions.
__device__ __forceinline__ void apply_pair(float a, float bb, float tl, float tr, float bu,
                                           float bd, double Dd, float dth, float dtl,
                                           float dbh, float dbl, const Grid& gr, double& ot,
                                           double& ob, bool dsplit) {
  const float dh = d2f_round(Dd);
  const float dl = dsplit ? d2f_round(Dd - f2d_bits(dh)) : 0.f;
  float ed, e3;
  const float d = two_sum(a, -bb, ed);
  const float p3 = two_prod(dh, d, e3);
  const float t3 = fmaf(dl, d, fmaf(dh, ed, e3));           // D (a - bb) = p3 + t3
  // top: dt a - gt (tl + tr) + D (a - bb)
  float es, e1, e2, eu, ev;
  const float st = two_sum(tl, tr, es);
  const float p1 = two_prod(dth, a, e1);
  const float p2 = two_prod(gr.gtf, st, e2);
  const float u = two_sum(p1, -p2, eu);
  const float v = two_sum(u, p3, ev);
  const float lt = (fmaf(dtl, a, e1) - fmaf(gr.gtl, st, fmaf(gr.gtf, es, e2))) + (t3 + (eu + ev));
  // bottom: db bb - gb (bu + bd) - D (a - bb)
  float fs, f1, f2, fu, fv;
  const float sb = two_sum(bu, bd, fs);
  const float q1 = two_prod(dbh, bb, f1);
  const float q2 = two_prod(gr.gbf, sb, f2);
  const float ub = two_sum(q1, -q2, fu);
  const float vb = two_sum(ub, -p3, fv);
  const float lb = (fmaf(dbl, bb, f1) - fmaf(gr.gbl, sb, fmaf(gr.gbf, fs, f2))) + ((fu + fv) - t3);
  ot = f2d_bits(v) + f2d_bits(lt);
  ob = f2d_bits(vb) + f2d_bits(lb);
}

// Newton control (eq. Newton3) for one vector from the reduced sums: ||F||, a = mean(D),
// convergence test, forcing term of the next linear solve (first: eta0; then
// Eisenstat-Walker 0.9 (|F_k|/|F_k-1|)^2 capped by eta_max, and never tighter than needed
// to reach the target), GMRES cycle start.  Runs in one thread.
// err >= 0 (the FP32-pair residual): ||F|| is known to within err.  The pair residual
// only serves iterates that are certainly more than kPairMinRatio times the target
// newton_rtol ||Y|| away from convergence (there it is the right-hand side of the next
// inexact Newton step); for any other vector nothing is decided or changed here: it is
// flagged (need_fp64, host flag 2) for the FP64 residual, which makes every convergence
// decision.
__device__ void newton_control(VecCtl& c, double sf, double sd, int mn, const SolverCfg& cfg,
                               int32_t* host_flag, double err = -1.0) {
  const double fn = sqrt(sf);
  const double a = sd / (double)mn;
  if (err >= 0.0 && isfinite(fn) && isfinite(a) &&
      fn - err <= kPairMinRatio * cfg.newton_rtol * c.ynorm) {
    c.d64_next = 0;                // the FP64 residual rewrites D
    c.need_fp64 = 1;
    c.gm_active = 0;
    if (host_flag) *host_flag = 2;
    __threadfence_system();
    return;
  }
  c.need_fp64 = 0;
  c.d64 = c.d64_next;
  c.d64_next = 0;
  c.fnorm_prev = c.fnorm;
  c.fnorm = fn;
  c.a = a;
  c.gm_active = 0;
  c.k_done = 0;
  if (!isfinite(fn) || !isfinite(a)) {
    c.status = MCA_ERR_NONFINITE;
    c.newton_active = 0;
  } else if (fn <= cfg.newton_rtol * c.ynorm) {
    c.status = MCA_OK;
    c.newton_active = 0;
  } else if (c.newton_iters >= cfg.max_newton) {
    c.status = MCA_ERR_NOT_CONVERGED;
    c.newton_active = 0;
  } else {
    double eta;
    if (c.fnorm_prev <= 0.0) {
      eta = cfg.eta0;
    } else {
      const double r = fn / c.fnorm_prev;
      eta = fmin(cfg.eta_max, 0.9 * r * r);
    }
    eta = fmax(eta, 0.5 * cfg.newton_rtol * c.ynorm / fn);
    eta = fmin(eta, 0.5);
    c.eta = eta;
    c.tol_abs = eta * fn;
    c.g[0] = fn;
    c.s[0] = -1.0 / fn;            // v_0 = -F / ||F|| from the stored residual
    c.orth = 0.0;
    c.reorth = 0;
    c.reorth_mask = 0u;
    c.res_est = fn;
    c.gm_active = 1;
    c.newton_iters += 1;
  }
  if (host_flag) *host_flag = c.newton_active;
  __threadfence_system();
}

// Givens rotation of Hessenberg column k (h = h1 + h2, h2 may be NULL; h_{k+1,k} =
// sqrt(hn2)), residual
// estimate |g_{k+1}| and the stop test of the GMRES cycle.  One thread.
// kL2: the h arrays were written by other blocks (read through L2); otherwise plain loads
// (the persistent kernel keeps them in its own CTA's shared memory).
template <bool kL2 = true>
__device__ void givens_column(VecCtl& c, int b, double hn2, const double* __restrict__ h1,
                              const double* __restrict__ h2, int k, int restart,
                              int32_t* host_flags) {
  auto ldh = [](const double* p) { return kL2 ? __ldcg(p) : *p; };
  const int ld = MCA_KMAX + 1;
  double* col = c.H + (size_t)k * ld;
  for (int j = 0; j <= k; ++j)
    col[j] = ldh(&h1[(size_t)b * 32 + j]) + (h2 ? ldh(&h2[(size_t)b * 32 + j]) : 0.0);
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

// Control block of one vector at the start of a solve: ||Y|| = yn and the counters; a
// zero or non-finite input ends the solve at once.
__device__ __forceinline__ void init_ctl(VecCtl& c, double yn, bool warm) {
  c.ynorm = yn;
  // a warm start treats V = 0, with ||F(0)|| = ||Y||, as its previous iterate, so its first
  // forcing term follows Eisenstat-Walker instead of the cold start's eta0
  c.fnorm = warm ? yn : 0.0;
  c.fnorm_prev = 0.0;
  c.a = 0.0;
  c.eta = 0.0;
  c.tol_abs = 0.0;
  c.newton_iters = 0;
  c.gmres_iters = 0;
  c.gm_active = 0;
  c.k_done = 0;
  c.need_fp64 = 0;
  c.d64 = 1;
  c.d64_next = 0;
  c.res_est = INFINITY;          // no linear solve yet
  if (!isfinite(yn)) {
    c.status = MCA_ERR_NONFINITE;
    c.newton_active = 0;
  } else if (yn == 0.0) {          // V_in = 0: the solution is V = 0
    c.status = MCA_OK;
    c.newton_active = 0;
  } else {
    c.status = MCA_OK;
    c.newton_active = 1;
  }
}

// Gram-Schmidt step control of one vector after an update pass (phase UPD_FIRST or
// UPD_REORTH, see k_krylov.cu) for the new vector of squared norm hn2.  hc: the pass's
// coefficients (h1 after the first pass, h2 after the second), h1: the first pass's.
// UPD_FIRST estimates the loss of orthogonality of the new vector and either marks the
// vector for the second pass or finishes Hessenberg column nk-1; UPD_REORTH finishes it with
// h1 + h2.  One thread.  kL2: the coefficients were written by other blocks.
template <bool kL2 = true>
__device__ void gram_schmidt_control(VecCtl& c, int b, int phase, double hn2,
                                     const double* __restrict__ hc,
                                     const double* __restrict__ h1, int nk, int restart,
                                     int32_t* host_flags) {
  const int k = nk - 1;
  const double grow = sqrt((double)nk) * c.orth;
  if (phase == UPD_FIRST) {
    double proj = 0.0;                      // |h1|^2 = |w|^2 - |u|^2
    for (int j = 0; j < nk; ++j) {
      const double t = kL2 ? __ldcg(&hc[(size_t)b * 32 + j]) : hc[(size_t)b * 32 + j];
      proj = fma(t, t, proj);
    }
    const double rho = (hn2 > 0.0) ? sqrt(hn2 / (hn2 + proj)) : 0.0;
    const double est = (grow + 4.0 * nk * kEps) / rho;
    if (hn2 > 0.0 && !(est <= kOrthTol)) {
      c.reorth = 1;
      c.reorth_mask |= 1u << k;
      c.orth1 = est;
      c.wn2 = hn2;
      __threadfence();
    } else {
      if (hn2 > 0.0) c.orth = est;
      givens_column<kL2>(c, b, hn2, hc, nullptr, k, restart, host_flags);
    }
  } else {
    // after the second pass: what is left of the first pass' loss orth1 is scaled by
    // the basis' own loss, plus rounding, relative to the new norm
    const double rho2 = (c.wn2 > 0.0 && hn2 > 0.0) ? sqrt(hn2 / c.wn2) : 0.0;
    if (rho2 > 0.0) c.orth = fmax(c.orth, (grow * c.orth1 + 4.0 * nk * kEps) / rho2);
    c.reorth = 0;
    givens_column<kL2>(c, b, hn2, h1, hc, k, restart, host_flags);
  }
}

// y = R^-1 g: back substitution of the rotated Hessenberg matrix of the finished cycle.
// One thread.
__device__ __forceinline__ void lsq_solve(VecCtl& c) {
  const int kd = c.k_done;
  const int ld = MCA_KMAX + 1;
  for (int i = kd - 1; i >= 0; --i) {
    double s = c.g[i];
    for (int j = i + 1; j < kd; ++j) s -= c.H[(size_t)j * ld + i] * c.y[j];
    const double d = c.H[(size_t)i * ld + i];
    c.y[i] = (d != 0.0) ? s / d : 0.0;
  }
}

}  // namespace
}  // namespace mca
