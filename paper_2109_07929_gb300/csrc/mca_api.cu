// C ABI and host orchestration of the steady-state crossbar solve.
//
//   mca_create : 1-D wire operators of eq. (G) with terminations, FP64 eigenpairs on the
//                GPU, BF16 operand copies and TMA maps for the tensor-core transforms,
//                device workspace for max_batch vectors.
//   mca_solve  : Newton (eq. Newton3) from V = 0; every Newton system J dx = -F (eq. J)
//                is solved by one flexible GMRES(restart) cycle right-preconditioned with
//                P^-1 of eq. (P) (Section 3), inexact-Newton forcing terms.
//
// The host only enqueues kernels; the iteration state lives on the device (VecCtl).  The
// host reads one small flag array per Newton step and polls the GMRES stop flags one
// iteration behind the launches, so the GPU queue never drains inside a cycle.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <utility>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mca_internal.cuh"
#include "precond_tc.h"

namespace mca {

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
thread_local bool g_capturing = false;   // launches recorded into a graph are counted on replay
}

// Every kernel launch of the library goes through one of the launch_* wrappers; their
// call sites add to this counter.
void count_launches(int n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

static void set_error(const char* msg) { g_last_error = msg; }
void set_error_message(const char* msg) { g_last_error = msg; }
void clear_error_message() { g_last_error.clear(); }

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Tensor-core preconditioner forms (need the BF16 operands and TMA maps).
static bool is_tc(int prec) { return prec == MCA_PREC_BF16 || prec == MCA_PREC_BF16_SPLIT; }

}  // namespace mca

using namespace mca;

struct mca_handle {
  mca_params p;
  Grid gr;
  int m = 0, n = 0, mp = 0, np = 0;
  size_t mn = 0, n2 = 0;
  int restart = 30;
  int Bmax = 1;
  int device = 0;
  // crossbars + eigenbasis (FP64): n_maps conductance maps of this shape
  int n_maps = 1;
  double* g = nullptr;
  int* map_of = nullptr;               // device: map of each vector of the current pass
  float* Z32 = nullptr;                // FP32 preconditioned vectors (tensor-core forms)
  std::vector<int> map_host;
  double *mu = nullptr, *nu = nullptr, *Qr = nullptr, *Qc = nullptr, *QrT = nullptr,
         *QcT = nullptr;
  float *mu_f = nullptr, *nu_f = nullptr;   // FP32 eigenvalues for the GEMM epilogue
  // BF16 copies (padded)
  __nv_bfloat16 *QrT_bf = nullptr, *QcT_bf = nullptr, *Qr_hi = nullptr, *Qr_lo = nullptr,
                *Qc_hi = nullptr, *Qc_lo = nullptr;
  // workspace
  double *x = nullptr, *F = nullptr, *D = nullptr, *V = nullptr, *Z = nullptr, *W = nullptr;
  double *part = nullptr, *h1 = nullptr, *h2 = nullptr;
  double *vin = nullptr, *iout = nullptr, *kcl = nullptr;
  VecCtl* ctl = nullptr;
  unsigned int* cnt = nullptr;    // per-vector block counters of the fused reductions
  int32_t* hflags = nullptr;      // pinned, mapped
  HostReport* report = nullptr;   // pinned, mapped: Bmax + 1 entries
  HostReport* report_dev = nullptr;
  int32_t* hflags_dev = nullptr;
  int* err = nullptr;
  double *T1_64 = nullptr, *Xh_64 = nullptr, *E_64 = nullptr;
  double* fac = nullptr;          // tridiagonal factors of the paper-literal M_hat
  int fac_ld = 0;
  __nv_bfloat16 *Xbf = nullptr, *T1bf = nullptr, *Yh = nullptr, *Eh = nullptr,
                *El = nullptr;
  bool tc_ok = false;
  CUtensorMap mA1, mA2, mA3, mA4h, mA4l;                 // A operands
  // B operands for 128-, 64- and 256-column tiles
  CUtensorMap mB1[3], mB2[3], mB3h[3], mB3l[3], mB4h[3], mB4l[3];
  // GEMM form of each transform: ws = 1 persistent warp-specialised kernel (tiles of
  // 128 x bn with lp layers), ws = 2 its two-SM form (CTA pairs over 256 x bn tiles of one
  // layer), ws = 0 one CTA per 128 x bn two-layer tile
  int bn[4] = {128, 128, 128, 128};
  int ws[4] = {0, 0, 0, 0};
  int lp[4] = {2, 2, 2, 2};
  std::vector<void*> allocs;
  cudaEvent_t ev[MCA_KMAX + 1];
  bool ev_ok = false;
  // Work requested on the legacy default stream runs on this blocking stream instead
  // (same ordering with the legacy stream, and legal to capture into graphs).
  cudaStream_t own_stream = nullptr;
  // Output copies of a pass run on copy_stream while the next pass computes: the state and
  // output currents are double-buffered (x and iout point at the current pass' buffers).
  cudaStream_t copy_stream = nullptr;
  double* xbuf[2] = {nullptr, nullptr};
  double* ioutbuf[2] = {nullptr, nullptr};
  cudaEvent_t ev_solved = nullptr;
  cudaEvent_t copy_done[2] = {nullptr, nullptr};
  bool copy_pending[2] = {false, false};
  // inputs of a pass are staged one pass ahead (before the previous pass' output copies
  // are queued, so they never wait behind them on the copy engine)
  double* vinbuf[2] = {nullptr, nullptr};
  int* mapbuf[2] = {nullptr, nullptr};
  // statistics of the last solve pass (host copies)
  std::vector<VecCtl> ctl_host;
  // captured GMRES iterations, keyed by (iteration k, batch size B)
  std::map<std::pair<int, int>, std::pair<cudaGraphExec_t, int>> graphs;
  // kernel-family timing
  struct ProfRec {
    int fam, k;
    bool reorth;                // second Gram-Schmidt pass: only the vectors that took it
    cudaEvent_t a, b;
    double bytes_pv, flops_pv;  // per vector still iterating
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_next = 0;
  std::vector<ProfRec> prof_pending;
  int64_t prof_launches[MCA_NUM_FAMILIES] = {};
  double prof_ms[MCA_NUM_FAMILIES] = {}, prof_bytes[MCA_NUM_FAMILIES] = {},
         prof_flops[MCA_NUM_FAMILIES] = {};
};

// Persistent batched solve over the shapes of several handles (k_persist.cu).
struct mca_batch {
  int device = 0;
  std::vector<mca_handle*> hs;
  std::vector<void*> allocs;
  PersistShape* shapes = nullptr;        // device, one per handle
  PersistSlots slots{};
  int grid = 0;                          // CTAs (= slots)
  bool yak = false;
  cudaStream_t own_stream = nullptr;
  PersistItem* items = nullptr;          // device
  PersistItem* items_host = nullptr;     // pinned
  PersistResult* res = nullptr;          // device
  PersistResult* res_host = nullptr;     // pinned
  int cap = 0;                           // items the buffers hold
  int* flags = nullptr;                  // device: [0] queue head, [1] error flag
  unsigned long long* prof = nullptr;    // device: CTA-ns per phase (NULL: off)
};

namespace {

template <typename T>
int dalloc(mca_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return MCA_OK;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation failed");
    return MCA_ERR_OOM;
  }
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return MCA_OK;
}

#define MCA_TRY(expr)               \
  do {                              \
    int _rc = (expr);               \
    if (_rc != MCA_OK) return _rc;  \
  } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

int mca::validate_circuit(const mca_params* p) {
  if (!p) {
    set_error("NULL parameters");
    return MCA_ERR_INVALID_ARG;
  }
  if (p->rows < 1 || p->cols < 1 || p->rows > 16384 || p->cols > 16384) {
    set_error("rows/cols must be in 1..16384");
    return MCA_ERR_INVALID_ARG;
  }
  if (!finite_pos(p->g_wire_top) || !finite_pos(p->g_wire_bot) || !finite_pos(p->g_src) ||
      !finite_pos(p->g_term_top_right) || !finite_pos(p->g_term_bot_top) ||
      !finite_pos(p->g_sense)) {
    set_error("wire and termination conductances must be finite and > 0");
    return MCA_ERR_INVALID_ARG;
  }
  if (!std::isfinite(p->b) || p->b < 0.0) {
    set_error("b must be finite and >= 0");
    return MCA_ERR_INVALID_ARG;
  }
  if (p->device_model != MCA_DEVICE_SINH && p->device_model != MCA_DEVICE_YAKOPCIC) {
    set_error("unknown device_model");
    return MCA_ERR_INVALID_ARG;
  }
  if (p->device_model == MCA_DEVICE_YAKOPCIC && !finite_pos(p->neg_ratio)) {
    set_error("neg_ratio must be finite and > 0");
    return MCA_ERR_INVALID_ARG;
  }
  return MCA_OK;
}

namespace {

int validate(const mca_params* p) {
  const int rc = validate_circuit(p);
  if (rc != MCA_OK) return rc;
  if (p->precision < MCA_PREC_FP64 || p->precision > MCA_PREC_NONE) {
    set_error("unknown precision");
    return MCA_ERR_INVALID_ARG;
  }
  if (p->gmres_restart < 1 || p->gmres_restart > MCA_KMAX || p->max_newton < 1 ||
      p->max_batch < 1 || p->max_batch > 64) {
    set_error("gmres_restart in 1..30, max_newton >= 1, max_batch in 1..64");
    return MCA_ERR_INVALID_ARG;
  }
  if (p->flags & ~(MCA_FLAG_GRAPHS | MCA_FLAG_AUTOTUNE | MCA_FLAG_PAIR_GEMM)) {
    set_error("unknown flag bits");
    return MCA_ERR_INVALID_ARG;
  }
  if (!(p->newton_rtol > 0.0) || !(p->eta0 > 0.0) || !(p->eta_max > 0.0)) {
    set_error("tolerances must be > 0");
    return MCA_ERR_INVALID_ARG;
  }
  return MCA_OK;
}

int setup_tc(mca_handle* h) {
  if (!tc::encode_available()) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return MCA_ERR_UNSUPPORTED;
  }
  MCA_CUDA_TRY(tc::configure_all());
  const size_t B = h->Bmax, mp = h->mp, np = h->np;
  MCA_TRY(dalloc(h, &h->Xbf, B * 2 * mp * np));
  MCA_TRY(dalloc(h, &h->T1bf, B * 2 * np * mp));
  MCA_TRY(dalloc(h, &h->Yh, B * 2 * mp * np));
  MCA_TRY(dalloc(h, &h->Eh, B * 2 * np * mp));
  MCA_TRY(dalloc(h, &h->El, B * 2 * np * mp));
  MCA_CUDA_TRY(cudaMemset(h->Xbf, 0, B * 2 * mp * np * sizeof(__nv_bfloat16)));
  bool ok = true;
  // K tiles: 64 wide for the single-word transforms, 32 wide for the split back
  // transforms (split precision: transform 3 holds Q_r as a hi/lo pair, transform 4 both
  // of its operands)
  const bool split = h->p.precision == MCA_PREC_BF16_SPLIT;
  const uint32_t kb = split ? 32u : 64u;
  ok &= tc::make_map(&h->mA1, h->Xbf, B * 2 * mp, np, 128, 64);
  ok &= tc::make_map(&h->mA2, h->T1bf, B * 2 * np, mp, 128, 64);
  ok &= tc::make_map(&h->mA3, h->Yh, B * 2 * mp, np, 128, kb);
  ok &= tc::make_map(&h->mA4h, h->Eh, B * 2 * np, mp, 128, kb);
  ok &= tc::make_map(&h->mA4l, h->El, B * 2 * np, mp, 128, kb);
  const uint32_t bns[3] = {128, 64, 256};
  for (int q = 0; q < 3; ++q) {
    ok &= tc::make_map(&h->mB1[q], h->QrT_bf, np, np, bns[q], 64);
    ok &= tc::make_map(&h->mB2[q], h->QcT_bf, mp, mp, bns[q], 64);
    ok &= tc::make_map(&h->mB3h[q], h->Qr_hi, np, np, bns[q], kb);
    ok &= tc::make_map(&h->mB3l[q], h->Qr_lo, np, np, bns[q], kb);
    ok &= tc::make_map(&h->mB4h[q], h->Qc_hi, mp, mp, bns[q], kb);
    ok &= tc::make_map(&h->mB4l[q], h->Qc_lo, mp, mp, bns[q], kb);
  }
  if (!ok) {
    set_error("tensor map encoding failed");
    return MCA_ERR_UNSUPPORTED;
  }
  // tile width: 64 columns when 128 would leave most SMs idle
  const int R[4] = {h->mp, h->np, h->mp, h->np};
  const int C[4] = {h->np, h->mp, h->np, h->mp};
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  for (int s = 0; s < 4; ++s) {
    const long ctas128 = (long)(R[s] / 128) * (C[s] / 128) * h->Bmax;
    h->bn[s] = (ctas128 < sms) ? 64 : 128;
    // persistent form by default: two-layer tiles for the modes transform, single-layer
    // 128-column tiles for the others
    h->ws[s] = 1;
    h->lp[s] = (s == 1) ? 2 : 1;
    if (s != 1) h->bn[s] = 128;
    // two-SM form asked for without the autotuner: wherever the tile fits
    if (s != 1 && (h->p.flags & MCA_FLAG_PAIR_GEMM) && !(h->p.flags & MCA_FLAG_AUTOTUNE) &&
        R[s] % 256 == 0 && C[s] % 256 == 0 && tc::pair_available()) {
      h->ws[s] = 2;
      h->bn[s] = 256;
    }
  }
  h->tc_ok = true;
  return MCA_OK;
}

int alloc_workspace(mca_handle* h) {
  const size_t B = h->Bmax, n2 = h->n2, mn = h->mn;
  const size_t kv = h->restart + 1;
  MCA_TRY(dalloc(h, &h->xbuf[0], B * n2));
  MCA_TRY(dalloc(h, &h->xbuf[1], B * n2));
  h->x = h->xbuf[0];
  MCA_TRY(dalloc(h, &h->F, B * n2));
  MCA_TRY(dalloc(h, &h->D, B * mn));
  MCA_TRY(dalloc(h, &h->V, B * kv * n2));
  // preconditioned vectors: FP32 for the tensor-core forms (their FP32 accumulators,
  // widened exactly where FP64 work reads them), FP64 otherwise
  if (is_tc(h->p.precision))
    MCA_TRY(dalloc(h, &h->Z32, B * h->restart * n2));
  else
    MCA_TRY(dalloc(h, &h->Z, B * h->restart * n2));
  MCA_TRY(dalloc(h, &h->W, B * n2));
  MCA_TRY(dalloc(h, &h->part, B * 32 * MCA_NPART));
  MCA_TRY(dalloc(h, &h->h1, B * 32));
  MCA_TRY(dalloc(h, &h->h2, B * 32));
  MCA_TRY(dalloc(h, &h->vinbuf[0], B * h->m));
  MCA_TRY(dalloc(h, &h->vinbuf[1], B * h->m));
  h->vin = h->vinbuf[0];
  MCA_TRY(dalloc(h, &h->ioutbuf[0], B * h->n));
  MCA_TRY(dalloc(h, &h->ioutbuf[1], B * h->n));
  h->iout = h->ioutbuf[0];
  MCA_TRY(dalloc(h, &h->kcl, B));
  MCA_TRY(dalloc(h, &h->ctl, B));
  MCA_TRY(dalloc(h, &h->err, 1));
  MCA_TRY(dalloc(h, &h->cnt, B));
  MCA_TRY(dalloc(h, &h->mapbuf[0], B));
  MCA_TRY(dalloc(h, &h->mapbuf[1], B));
  h->map_of = h->mapbuf[0];
  h->fac_ld = std::max(h->m, h->n);
  MCA_TRY(dalloc(h, &h->fac, B * 4 * (size_t)h->fac_ld));
  MCA_CUDA_TRY(cudaMemset(h->mapbuf[0], 0, B * sizeof(int)));
  MCA_CUDA_TRY(cudaMemset(h->mapbuf[1], 0, B * sizeof(int)));
  h->map_host.assign(B, 0);
  MCA_CUDA_TRY(cudaMemset(h->err, 0, sizeof(int)));
  MCA_CUDA_TRY(cudaMemset(h->cnt, 0, B * sizeof(unsigned int)));
  MCA_CUDA_TRY(cudaMemset(h->ctl, 0, B * sizeof(VecCtl)));
  if (h->p.precision == MCA_PREC_FP64) {
    MCA_TRY(dalloc(h, &h->T1_64, B * n2));
    MCA_TRY(dalloc(h, &h->Xh_64, B * n2));
    MCA_TRY(dalloc(h, &h->E_64, B * n2));
  }
  MCA_CUDA_TRY(cudaHostAlloc(&h->hflags, 64 * sizeof(int32_t), cudaHostAllocMapped));
  MCA_CUDA_TRY(cudaHostGetDevicePointer(&h->hflags_dev, h->hflags, 0));
  MCA_CUDA_TRY(cudaHostAlloc(&h->report, (B + 1) * sizeof(HostReport), cudaHostAllocMapped));
  MCA_CUDA_TRY(cudaHostGetDevicePointer(&h->report_dev, h->report, 0));
  for (int k = 0; k <= MCA_KMAX; ++k)
    MCA_CUDA_TRY(cudaEventCreateWithFlags(&h->ev[k], cudaEventDisableTiming));
  h->ev_ok = true;
  MCA_CUDA_TRY(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamDefault));
  MCA_CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  MCA_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_solved, cudaEventDisableTiming));
  for (int q = 0; q < 2; ++q)
    MCA_CUDA_TRY(cudaEventCreateWithFlags(&h->copy_done[q], cudaEventDisableTiming));
  h->ctl_host.resize(B);
  return MCA_OK;
}

// ---- kernel-family timing -------------------------------------------------------------
cudaEvent_t prof_event(mca_handle* h) {
  if (h->prof_next == h->prof_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->prof_pool.push_back(e);
  }
  return h->prof_pool[h->prof_next++];
}

// Record a start event when timing is on; returns it (or NULL).
cudaEvent_t prof_begin(mca_handle* h, cudaStream_t s) {
  if (!h->prof_on) return nullptr;
  cudaEvent_t a = prof_event(h);
  if (a) cudaEventRecord(a, s);
  return a;
}

void prof_end(mca_handle* h, cudaEvent_t a, int fam, int k, double bytes_pv, double flops_pv,
              cudaStream_t s, bool reorth = false) {
  if (!h->prof_on || !a) return;
  cudaEvent_t b = prof_event(h);
  if (!b) return;
  cudaEventRecord(b, s);
  h->prof_pending.push_back({fam, k, reorth, a, b, bytes_pv, flops_pv});
}

// Fold the pending records into the family totals.  active(k, reorth) is the number of
// vectors that did work in GMRES iteration k (k < 0: launches outside the Krylov loop;
// reorth: the conditional second Gram-Schmidt pass).
template <typename F>
void prof_flush(mca_handle* h, F active) {
  if (!h->prof_on) return;
  for (auto& r : h->prof_pending) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) continue;
    const int act = active(r.k, r.reorth);
    if (act <= 0) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    h->prof_launches[r.fam] += 1;
    h->prof_ms[r.fam] += ms;
    h->prof_bytes[r.fam] += r.bytes_pv * act;
    h->prof_flops[r.fam] += r.flops_pv * act;
  }
  h->prof_pending.clear();
  h->prof_next = 0;
}

// Results of the pass' B vectors into h->ctl_host (status, iteration counts, norms) and,
// if kcl_out is given, the KCL balances; returns the device error flag as a status.  Only
// kernel work on s is waited for (no copy-engine transfer).
int read_report(mca_handle* h, int B, const double* kcl_dev, double* kcl_out, cudaStream_t s) {
  launch_report(h->ctl, kcl_dev, h->err, h->report_dev, B, s);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  const volatile HostReport* r = h->report;
  for (int b = 0; b < B; ++b) {
    VecCtl& c = h->ctl_host[b];
    c.status = r[b].status;
    c.newton_iters = r[b].newton_iters;
    c.gmres_iters = r[b].gmres_iters;
    c.k_done = r[b].k_done;
    c.fnorm = r[b].fnorm;
    c.ynorm = r[b].ynorm;
    c.res_est = r[b].res_est;
    if (kcl_out) kcl_out[b] = r[b].kcl;
  }
  const int e = r[B].status;
  if (e != 0) {
    cudaMemsetAsync(h->err, 0, sizeof(int), s);
    set_error("a bounded device wait expired");
    return e;
  }
  return MCA_OK;
}

int check_device_error(mca_handle* h) {
  int e = 0;
  MCA_CUDA_TRY(cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    cudaMemset(h->err, 0, sizeof(int));
    set_error("a bounded device wait expired");
    return e;
  }
  return MCA_OK;
}

// Tensor-core transform `step` (0..3) of the preconditioner for B vectors; the input of
// step 0 is the BF16 copy in h->Xbf, the output of step 3 goes to zout (FP64).
int tc_step(mca_handle* h, int step, bool split, void* zout, size_t zstride, int B,
            const VecCtl* ctl, cudaStream_t s, int prof_k, int kidx = -1, bool z32 = false) {
  const int m = h->m, n = h->n;
  const size_t mn = h->mn, mp = h->mp, np = h->np;
  const int bn = h->bn[step];
  // B maps by box rows (the two-SM form loads bn / 2 rows of B per CTA)
  const int boxb = (h->ws[step] == 2) ? bn / 2 : bn;
  auto q = [boxb](int) { return boxb == 128 ? 0 : (boxb == 64 ? 1 : 2); };
  auto run = [&](int sp_, int epi, const CUtensorMap& a, const CUtensorMap& al,
                 const CUtensorMap& bm, const CUtensorMap& bml, const tc::GemmEpi& ep) {
    return h->ws[step] ? tc::gemm_ws(bn, h->lp[step], h->ws[step], sp_, epi, a, al, bm, bml,
                                     ep, B, s)
                       : tc::gemm(bn, sp_, epi, a, al, bm, bml, ep, B, s);
  };
  // executed MMA FLOPs per vector: 2 layers x 2 M N K; when split, two products in
  // transform 3 (Q_r as hi + lo) and three in transform 4 (E and Q_c as hi + lo)
  const double f_r = 4.0 * m * (double)n * n, f_c = 4.0 * n * (double)m * m;
  const int sp3 = split ? tc::SPLIT_B : tc::SPLIT_NONE;
  const int sp4 = split ? tc::SPLIT_AB : tc::SPLIT_NONE;
  tc::GemmEpi e{};
  e.ctl = ctl;
  e.kidx = kidx;
  e.err = h->err;
  e.mu = h->mu;
  e.nu = h->nu;
  e.mu_f = h->mu_f;
  e.nu_f = h->nu_f;
  cudaEvent_t t0 = prof_begin(h, s);
  switch (step) {
    case 0:  // T1^T = (X Q_r)^T
      e.R = h->mp; e.K = h->np; e.C = h->np; e.R_valid = m; e.C_valid = n;
      e.out = h->T1bf; e.o_bs = 2 * np * mp; e.o_ls = np * mp; e.o_ld = mp;
      MCA_CUDA_TRY(run(tc::SPLIT_NONE, tc::EPI_BF16, h->mA1, h->mA1, h->mB1[q(bn)],
                       h->mB1[q(bn)], e));
      prof_end(h, t0, MCA_FAM_PRECOND_1, prof_k, 8.0 * mn, f_r, s);
      break;
    case 1:  // Y_hat = modes^-1 (Q_c^T T1), stored [i'][k'] (one BF16 word)
      e.R = h->np; e.K = h->mp; e.C = h->mp; e.R_valid = n; e.C_valid = m;
      e.out = h->Yh; e.o_bs = 2 * mp * np; e.o_ls = mp * np; e.o_ld = np;
      MCA_CUDA_TRY(run(tc::SPLIT_NONE, tc::EPI_MODES, h->mA2, h->mA2, h->mB2[q(bn)],
                       h->mB2[q(bn)], e));
      prof_end(h, t0, MCA_FAM_PRECOND_2, prof_k, 8.0 * mn, f_c, s);
      break;
    case 2:  // E^T = (Y_hat Q_r^T)^T
      e.R = h->mp; e.K = h->np; e.C = h->np; e.R_valid = m; e.C_valid = n;
      e.out = h->Eh; e.out_lo = h->El; e.o_bs = 2 * np * mp; e.o_ls = np * mp; e.o_ld = mp;
      MCA_CUDA_TRY(run(sp3, split ? tc::EPI_SPLIT : tc::EPI_BF16, h->mA3, h->mA3,
                       h->mB3h[q(bn)], h->mB3l[q(bn)], e));
      prof_end(h, t0, MCA_FAM_PRECOND_3, prof_k, (split ? 12.0 : 8.0) * mn,
               (split ? 2.0 : 1.0) * f_r, s);
      break;
    default:  // Z = (E^T Q_c^T)^T, FP64 unpadded
      e.R = h->np; e.K = h->mp; e.C = h->mp; e.R_valid = n; e.C_valid = m;
      e.out = zout; e.o_bs = zstride; e.o_ls = mn; e.o_ld = n;
      MCA_CUDA_TRY(run(sp4, z32 ? tc::EPI_F32 : tc::EPI_F64, h->mA4h, h->mA4l, h->mB4h[q(bn)],
                       h->mB4l[q(bn)], e));
      prof_end(h, t0, MCA_FAM_PRECOND_4, prof_k,
               (split ? 8.0 : 4.0) * mn + (z32 ? 8.0 : 16.0) * mn, (split ? 3.0 : 1.0) * f_c, s);
      break;
  }
  count_launches(1);
  return MCA_OK;
}

// Tile-width autotuner: time each transform with 128- and 64-column tiles at the handle's
// batch size and keep the faster one (the best width depends on how many CTAs a shape
// gives against the SM count).
int autotune_tiles(mca_handle* h) {
  const int B = h->Bmax;
  for (int b = 0; b < B; ++b) {
    VecCtl& c = h->ctl_host[b];
    memset(&c, 0, sizeof(VecCtl));
    c.a = 2e-5;
    c.gm_active = 1;
    c.newton_active = 1;
    c.d64 = 1;
  }
  MCA_CUDA_TRY(cudaMemcpy(h->ctl, h->ctl_host.data(), (size_t)B * sizeof(VecCtl),
                          cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  MCA_CUDA_TRY(cudaEventCreate(&e0));
  MCA_CUDA_TRY(cudaEventCreate(&e1));
  const bool split = h->p.precision == MCA_PREC_BF16_SPLIT;
  const size_t zstride = (size_t)h->restart * h->n2;
  int rc = MCA_OK;
  for (int step = 0; step < 4 && rc == MCA_OK; ++step) {
    float best = 1e30f;
    int best_bn = h->bn[step], best_ws = h->ws[step], best_lp = h->lp[step];
    const int Cs = (step == 0 || step == 2) ? h->np : h->mp;
    // candidates (ws, bn, lp): the one-CTA-per-tile kernel with 128 / 64 columns, the
    // persistent kernel with its instantiated tile shapes, its two-SM form (256-row tiles)
    const int cands[][3] = {{0, 128, 2}, {0, 64, 2}, {1, 128, 1}, {1, 256, 1},
                            {1, 64, 2}, {1, 128, 2}, {2, 256, 1}};
    const int Rs = (step == 0 || step == 2) ? h->mp : h->np;
    for (const auto& cd : cands) {
      const int ws = cd[0], bn = cd[1], lp = cd[2];
      if (Cs % bn != 0) continue;
      if (ws >= 1 && ((step == 1) != (lp == 2))) continue;   // modes: 2 layers; others: 1
      if (ws == 2 && (Rs % 256 != 0 || !(h->p.flags & MCA_FLAG_PAIR_GEMM) ||
                      !tc::pair_available()))
        continue;
      h->ws[step] = ws;
      h->bn[step] = bn;
      h->lp[step] = lp;
      rc = tc_step(h, step, split, h->Z32, zstride, B, h->ctl, 0, -1, -1, true);
      if (rc != MCA_OK) break;
      cudaEventRecord(e0, 0);
      for (int r = 0; r < 3 && rc == MCA_OK; ++r)
        rc = tc_step(h, step, split, h->Z32, zstride, B, h->ctl, 0, -1, -1, true);
      cudaEventRecord(e1, 0);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = MCA_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_bn = bn;
        best_ws = ws;
        best_lp = lp;
      }
    }
    h->bn[step] = best_bn;
    h->ws[step] = best_ws;
    h->lp[step] = best_lp;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaMemset(h->ctl, 0, (size_t)B * sizeof(VecCtl));
  if (rc == MCA_OK) rc = check_device_error(h);
  return rc;
}

// z = P^-1 r for B vectors: r at rin + b*rstride, z at zout + b*zstride.  For the
// tensor-core forms the BF16 copy of r must already be in h->Xbf.  kidx >= 0: r is the
// unnormalised basis vector k, and z = P^-1 (ctl[b].s[kidx] r).
// zout is double*, or float* when z32 (tensor-core forms only).
int precond_apply(mca_handle* h, int precision, const double* rin, size_t rstride,
                  void* zout_v, size_t zstride, int B, const VecCtl* ctl, cudaStream_t s,
                  int prof_k = -1, const double* D = nullptr, int kidx = -1,
                  bool z32 = false) {
  double* zout = static_cast<double*>(zout_v);
  if (precision == MCA_PREC_MHAT) {
    cudaEvent_t t0 = prof_begin(h, s);
    MCA_TRY(precond_mhat(h->gr, rin, rstride, zout, zstride, B, ctl, h->fac, h->fac_ld, kidx,
                         s));
    prof_end(h, t0, MCA_FAM_PRECOND_1, prof_k, 112.0 * (double)h->mn, 40.0 * (double)h->mn, s);
    return MCA_OK;
  }
  if (precision == MCA_PREC_JACOBI || precision == MCA_PREC_NONE) {
    if (precision == MCA_PREC_JACOBI && D == nullptr) return MCA_ERR_UNSUPPORTED;
    cudaEvent_t t0 = prof_begin(h, s);
    MCA_TRY(precond_jacobi(h->gr, D, rin, rstride, zout, zstride, B,
                           precision == MCA_PREC_NONE, ctl, kidx, s));
    prof_end(h, t0, MCA_FAM_PRECOND_1, prof_k, 40.0 * (double)h->mn, 4.0 * (double)h->mn, s);
    return MCA_OK;
  }
  const int m = h->m, n = h->n;
  const size_t mn = h->mn;
  if (precision == MCA_PREC_FP64) {
    if (!h->T1_64) return MCA_ERR_UNSUPPORTED;
    const double f_r = 4.0 * m * (double)n * n, f_c = 4.0 * n * (double)m * m;
    BlkAddr a1{rstride, mn, (size_t)n}, o1{2 * mn, mn, (size_t)m};
    cudaEvent_t t0 = prof_begin(h, s);
    launch_gemm64_tstore(rin, a1, h->QrT, h->T1_64, o1, B, m, n, n, ctl, s);
    count_launches(1);
    prof_end(h, t0, MCA_FAM_PRECOND_1, prof_k, 32.0 * mn, f_r, s);
    BlkAddr a2{2 * mn, mn, (size_t)m}, o2{2 * mn, mn, (size_t)n};
    t0 = prof_begin(h, s);
    launch_gemm64_tstore(h->T1_64, a2, h->QcT, h->Xh_64, o2, B, n, m, m, ctl, s);
    count_launches(1);
    launch_modes_2x2_f64(h->Xh_64, h->mu, h->nu, m, n, ctl, B, kidx, s);
    count_launches(1);
    prof_end(h, t0, MCA_FAM_PRECOND_2, prof_k, 64.0 * mn, f_c, s);
    BlkAddr a3{2 * mn, mn, (size_t)n}, o3{2 * mn, mn, (size_t)m};
    t0 = prof_begin(h, s);
    launch_gemm64_tstore(h->Xh_64, a3, h->Qr, h->E_64, o3, B, m, n, n, ctl, s);
    count_launches(1);
    prof_end(h, t0, MCA_FAM_PRECOND_3, prof_k, 32.0 * mn, f_r, s);
    BlkAddr a4{2 * mn, mn, (size_t)m}, o4{zstride, mn, (size_t)n};
    t0 = prof_begin(h, s);
    launch_gemm64_tstore(h->E_64, a4, h->Qc, zout, o4, B, n, m, m, ctl, s);
    count_launches(1);
    prof_end(h, t0, MCA_FAM_PRECOND_4, prof_k, 32.0 * mn, f_c, s);
    MCA_CUDA_TRY(cudaGetLastError());
    return MCA_OK;
  }
  if (!h->tc_ok) return MCA_ERR_UNSUPPORTED;
  const bool split = (precision == MCA_PREC_BF16_SPLIT);
  for (int step = 0; step < 4; ++step)
    MCA_TRY(tc_step(h, step, split, zout_v, zstride, B, ctl, s, prof_k, kidx, z32));
  return MCA_OK;
}

SolverCfg make_cfg(const mca_handle* h) {
  SolverCfg c;
  c.newton_rtol = h->p.newton_rtol;
  c.eta0 = h->p.eta0;
  c.eta_max = h->p.eta_max;
  c.max_newton = h->p.max_newton;
  c.restart = h->restart;
  return c;
}

bool any_flag(const mca_handle* h, int B) {
  for (int b = 0; b < B; ++b)
    if (reinterpret_cast<volatile int32_t*>(h->hflags)[b]) return true;
  return false;
}

// Enqueue GMRES iteration k (preconditioner, Jacobian apply + classical Gram-Schmidt with
// the fused reductions, the conditional second pass and the Givens column) for the vectors
// still iterating.  The basis vectors after v_0 are kept unnormalised with their scales in
// VecCtl::s, so the update pass writes v_{k+1} (and its BF16 copy) directly.
int enqueue_iteration(mca_handle* h, const double* D, int B, int k, cudaStream_t s,
                      bool f32 = false) {
  const size_t n2 = h->n2;
  const double cells = (double)h->mn;
  const size_t vstride = (size_t)(h->restart + 1) * n2;
  const size_t zstride = (size_t)h->restart * n2;
  const int nbS = residual_nblk((int)h->mn, B);
  const int nbV = vec_nblk(n2, B);
  const bool tc = is_tc(h->p.precision);
  const double* vk = h->V + (size_t)k * n2;
  const double nk = k + 1;
  cudaEvent_t t0 = nullptr;
  // (tensor-core forms read the BF16 copy of v_k written by the kernel that made v_k)
  if (tc) {
    float* zk = h->Z32 + (size_t)k * n2;
    MCA_TRY(precond_apply(h, h->p.precision, vk, vstride, zk, zstride, B, h->ctl, s, k, D, k,
                          true));
    t0 = prof_begin(h, s);
    // the FP32 apply runs in the Newton step from V = 0, whose v_0 the residual stored in
    // the first column of the top layer only (sparse_f): its dots read v_0 there only
    launch_spmv_dots(h->gr, D, zk, zstride, h->W, h->V, vstride, k + 1, h->part, nbS, B,
                     h->ctl, h->cnt, h->h1, s, f32 ? kApplyF32Zero : kApplyPair);
  } else {
    double* zk = h->Z + (size_t)k * n2;
    MCA_TRY(precond_apply(h, h->p.precision, vk, vstride, zk, zstride, B, h->ctl, s, k, D, k));
    t0 = prof_begin(h, s);
    launch_spmv_dots(h->gr, D, zk, zstride, h->W, h->V, vstride, k + 1, h->part, nbS, B,
                     h->ctl, h->cnt, h->h1, s);
  }
  count_launches(1);
  // FP64 flops per cell: the stencil's 12 when the apply runs in FP64 (FP64 z), 3 in the
  // FP32-pair apply (splitting D, forming the two results), none in the FP32 apply; the
  // sparse v_0 of the zero-state step counts neither bytes nor flops
  const double nkd = f32 ? nk - 1.0 : nk;     // basis vectors read in full
  prof_end(h, t0, MCA_FAM_SPMV_DOTS, k, cells * ((tc ? 32.0 : 40.0) + 16.0 * nkd),
           cells * ((tc ? (f32 ? 0.0 : 3.0) : 12.0) + 4.0 * nkd), s);
  double* vnext = h->V + (size_t)(k + 1) * n2;
  __nv_bfloat16* xbf = tc ? h->Xbf : nullptr;
  t0 = prof_begin(h, s);
  launch_update_norm(UPD_FIRST, h->W, n2, h->V, vstride, n2, k + 1, h->h1, h->part, nbV, B,
                     h->ctl, h->cnt, h->h1, h->restart, h->hflags_dev, vnext, vstride, xbf,
                     h->mp, h->np, h->m, h->n, s, f32);
  count_launches(1);
  prof_end(h, t0, MCA_FAM_UPDATE_NORM, k, cells * (32.0 + 16.0 * nkd + (tc ? 4.0 : 0.0)),
           cells * (4.0 * nkd + 4.0), s);
  // second pass, a no-op for the vectors whose orthogonality estimate did not ask for it
  t0 = prof_begin(h, s);
  launch_reorth_dots(vnext, h->V, vstride, n2, k + 1, h->part, nbV, B, h->ctl, h->cnt, h->h2,
                     s, f32, h->n);
  launch_update_norm(UPD_REORTH, vnext, vstride, h->V, vstride, n2, k + 1, h->h2, h->part,
                     nbV, B, h->ctl, h->cnt, h->h1, h->restart, h->hflags_dev, vnext, vstride,
                     xbf, h->mp, h->np, h->m, h->n, s, f32);
  count_launches(2);
  prof_end(h, t0, MCA_FAM_UPDATE_DOTS, k,
           cells * (48.0 + 32.0 * nkd + (tc ? 4.0 : 0.0)),
           cells * (8.0 * nkd + 4.0), s, true);
  MCA_CUDA_TRY(cudaGetLastError());
  return MCA_OK;
}

// Capture iteration k for batch size B once and replay it as one graph launch.
int launch_iteration_graph(mca_handle* h, const double* D, int B, int k, cudaStream_t s,
                           bool f32) {
  auto key = std::make_pair(k + (f32 ? MCA_KMAX + 1 : 0), B);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaGraph_t graph = nullptr;
    MCA_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    int rc = enqueue_iteration(h, D, B, k, s, f32);
    g_capturing = false;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != MCA_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    MCA_CUDA_TRY(e);
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    MCA_CUDA_TRY(e);
    it = h->graphs.emplace(key, std::make_pair(exec, (int)nodes)).first;
  }
  MCA_CUDA_TRY(cudaGraphLaunch(it->second.first, s));
  count_launches(it->second.second);
  return MCA_OK;
}

// One flexible GMRES cycle on the vectors whose gm_active flag is set; V[b][0] and its
// BF16 copy are already in place.  D is the Jacobian diagonal (graphs only for the
// handle's own D).
int gmres_cycle(mca_handle* h, const double* D, int B, cudaStream_t s, bool f32 = false) {
  const bool graphs = (h->p.flags & MCA_FLAG_GRAPHS) && !h->prof_on && D == h->D;
  for (int k = 0; k < h->restart; ++k) {
    if (graphs) {
      MCA_TRY(launch_iteration_graph(h, D, B, k, s, f32));
    } else {
      MCA_TRY(enqueue_iteration(h, D, B, k, s, f32));
    }
    MCA_CUDA_TRY(cudaEventRecord(h->ev[k], s));
    if (k >= 1) {
      MCA_CUDA_TRY(cudaEventSynchronize(h->ev[k - 1]));
      if (!any_flag(h, B)) break;
    }
  }
  if (h->prof_on) {
    // iterations done per vector in this cycle decide which launches did work
    MCA_CUDA_TRY(cudaMemcpyAsync(h->ctl_host.data(), h->ctl, (size_t)B * sizeof(VecCtl),
                                 cudaMemcpyDeviceToHost, s));
    MCA_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> kd(B);
    std::vector<uint32_t> rm(B);
    for (int b = 0; b < B; ++b) {
      kd[b] = h->ctl_host[b].k_done;
      rm[b] = h->ctl_host[b].reorth_mask;
    }
    prof_flush(h, [&](int k, bool reorth) {
      int c = 0;
      for (int b = 0; b < B; ++b)
        c += (k < kd[b] && (!reorth || ((rm[b] >> k) & 1u))) ? 1 : 0;
      return c;
    });
  }
  return MCA_OK;
}


// Solve B <= Bmax vectors whose inputs are in h->vin; results stay in h->x / h->iout.
// from_guess: h->x already holds the initial states (otherwise Newton starts at x = 0).
int solve_pass(mca_handle* h, int B, cudaStream_t s, bool from_guess = false) {
  const SolverCfg cfg = make_cfg(h);
  const int nbR = residual_nblk((int)h->mn, B);
  const bool tc = is_tc(h->p.precision);
  const size_t vstride = (size_t)(h->restart + 1) * h->n2;
  const size_t zstride = (size_t)h->restart * h->n2;
  launch_setup_vectors(h->gr, h->vin, B, h->ctl, from_guess, s);
  count_launches(1);
  if (!from_guess)
    MCA_CUDA_TRY(cudaMemsetAsync(h->x, 0, (size_t)B * h->n2 * sizeof(double), s));
  const double cells = (double)h->mn;
  int n_active = B;  // vectors entering the current Newton step
  for (int it = 0; it <= h->p.max_newton; ++it) {
    cudaEvent_t t0 = prof_begin(h, s);
    const bool zero_state = (it == 0) && !from_guess;
    // F goes straight into the first Krylov basis vector (kept unnormalised) and its BF16
    // copy, so no separate pass builds v_0
    // with the tensor-core forms, states after the first whose last linear solve ended far
    // above the target take the residual in FP32 pairs; a vector whose pair ||F|| is not
    // certainly far above the target gets the FP64 residual, which decides convergence
    const bool pair = tc && !zero_state && h->gr.tail32;
    // the first step from V = 0 solves to the loosest forcing term, eta0: with the
    // tensor-core forms its Jacobian applies run in FP32 when eta0 allows it, and that step's
    // kernels read v_0 only where F(0) = -Y is nonzero (the first column of the top layer),
    // so the residual stores only that column of F
    const bool f32 = tc && zero_state && h->p.eta0 >= kF32ApplyMinEta;
    launch_residual_newton(h->gr, h->g, h->n_maps > 1 ? h->map_of : nullptr, h->vin, h->x,
                           zero_state, h->V, vstride, tc ? h->Xbf : nullptr, h->mp, h->np,
                           h->D, h->part, nbR, B, h->ctl, cfg, h->cnt, h->hflags_dev, s, pair,
                           false, f32);
    count_launches(1);
    // FP64 flops per cell (an FMA counts 2): the FP64 cell 15 in 10 instructions (device
    // voltage, current, two stencil rows; ||F||^2 and the conductance cosh are FP32); the
    // pair form 6 (its two final additions and the FP64 norm); the zero state none
    prof_end(h, t0, MCA_FAM_RESIDUAL, -1,
             cells * ((zero_state ? (f32 ? 20.0 : 36.0) : 48.0) + (tc ? 4.0 : 0.0)),
             cells * (zero_state ? 0.0 : (pair ? 6.0 : 15.0)), s);
    MCA_CUDA_TRY(cudaGetLastError());
    MCA_CUDA_TRY(cudaStreamSynchronize(s));
    const int entering = n_active;
    volatile int32_t* hf = reinterpret_cast<volatile int32_t*>(h->hflags);
    int undecided = 0;
    for (int b = 0; b < B; ++b) undecided += (hf[b] == 2) ? 1 : 0;
    if (undecided > 0) {
      t0 = prof_begin(h, s);
      launch_residual_newton(h->gr, h->g, h->n_maps > 1 ? h->map_of : nullptr, h->vin, h->x,
                             false, h->V, vstride, tc ? h->Xbf : nullptr, h->mp, h->np, h->D,
                             h->part, nbR, B, h->ctl, cfg, h->cnt, h->hflags_dev, s, false,
                             true);
      count_launches(1);
      prof_end(h, t0, MCA_FAM_RESIDUAL, -2, cells * (48.0 + 4.0), cells * 15.0, s);
      MCA_CUDA_TRY(cudaGetLastError());
      MCA_CUDA_TRY(cudaStreamSynchronize(s));
    }
    n_active = 0;
    for (int b = 0; b < B; ++b) n_active += hf[b] ? 1 : 0;
    prof_flush(h, [&](int k, bool) { return k == -2 ? undecided : entering; });
    if (n_active == 0) break;
    MCA_TRY(gmres_cycle(h, h->D, B, s, f32));
    t0 = prof_begin(h, s);
    if (tc)
      launch_lsq_update(h->x, h->Z32, zstride, h->n2, h->ctl, B, s);
    else
      launch_lsq_update(h->x, h->Z, zstride, h->n2, h->ctl, B, s);
    count_launches(2);
    double kbar = 0.0;
    if (h->prof_on) {
      int c = 0;
      for (int b = 0; b < B; ++b)
        if (h->ctl_host[b].k_done > 0) { kbar += h->ctl_host[b].k_done; ++c; }
      kbar = c ? kbar / c : 0.0;
    }
    prof_end(h, t0, MCA_FAM_UPDATE_X, -1, cells * (32.0 + (tc ? 8.0 : 16.0) * kbar),
             cells * 4.0 * kbar, s);
    prof_flush(h, [&](int, bool) { return n_active; });
    MCA_CUDA_TRY(cudaGetLastError());
  }
  launch_outputs(h->gr, h->vin, h->x, h->iout, h->kcl, B, s);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  return MCA_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst || bytes == 0) return MCA_OK;
  MCA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return MCA_OK;
}

}  // namespace

extern "C" {

void mca_default_params(mca_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->g_wire_top = 1.0;
  p->g_wire_bot = 1.0;
  p->g_src = 0.1;
  p->g_term_top_right = 1e-3;
  p->g_term_bot_top = 1e-3;
  p->g_sense = 0.1;
  p->b = 2.0;
  p->device_model = MCA_DEVICE_SINH;
  p->neg_ratio = 1.0;
  p->precision = MCA_PREC_BF16_SPLIT;
  p->gmres_restart = 30;
  p->max_newton = 20;
  p->max_batch = 4;
  p->newton_rtol = 1e-8;
  p->eta0 = 1e-3;
  p->eta_max = 1e-2;
  p->flags = MCA_FLAG_GRAPHS | MCA_FLAG_AUTOTUNE | MCA_FLAG_PAIR_GEMM;
}

const char* mca_strerror(int code) {
  switch (code) {
    case MCA_OK: return "ok";
    case MCA_ERR_INVALID_ARG: return "invalid argument";
    case MCA_ERR_CUDA: return "CUDA runtime error";
    case MCA_ERR_NONFINITE: return "non-finite value in inputs or residual";
    case MCA_ERR_NOT_CONVERGED: return "Newton did not reach the tolerance";
    case MCA_ERR_TIMEOUT: return "bounded device wait expired";
    case MCA_ERR_OOM: return "device memory allocation failed";
    case MCA_ERR_UNSUPPORTED: return "unsupported on this device";
    default: return "unknown status";
  }
}

const char* mca_last_error_message(void) { return g_last_error.c_str(); }

void mca_destroy(mca_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (void* q : h->allocs) cudaFree(q);
  if (h->hflags) cudaFreeHost(h->hflags);
  if (h->report) cudaFreeHost(h->report);
  if (h->ev_ok)
    for (int k = 0; k <= MCA_KMAX; ++k) cudaEventDestroy(h->ev[k]);
  for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.first);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->ev_solved) cudaEventDestroy(h->ev_solved);
  for (int q = 0; q < 2; ++q)
    if (h->copy_done[q]) cudaEventDestroy(h->copy_done[q]);
  delete h;
}

int mca_create(const mca_params* p, const double* g_map, mca_handle** out) {
  return mca_create_multi(p, g_map, 1, out);
}

int mca_create_multi(const mca_params* p, const double* g_map, int32_t n_maps,
                     mca_handle** out) {
  g_last_error.clear();
  if (!out || !g_map || n_maps < 1) {
    set_error("NULL argument or n_maps < 1");
    return MCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int rc = validate(p);
  if (rc != MCA_OK) return rc;
  mca_handle* h = new mca_handle();
  h->p = *p;
  h->n_maps = n_maps;
  cudaGetDevice(&h->device);
  h->m = p->rows;
  h->n = p->cols;
  h->mp = (int)round_up(h->m, 128);
  h->np = (int)round_up(h->n, 128);
  h->mn = (size_t)h->m * h->n;
  h->n2 = 2 * h->mn;
  h->restart = p->gmres_restart;
  h->Bmax = p->max_batch;
  h->gr = make_grid(*p);
  auto fail = [&](int code) {
    mca_destroy(h);
    return code;
  };
  // conductance maps: copy and validate on the host
  const size_t gtot = h->mn * (size_t)n_maps;
  std::vector<double> gh(gtot);
  if (cudaMemcpy(gh.data(), g_map, gtot * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot read g_map");
    return fail(MCA_ERR_INVALID_ARG);
  }
  for (size_t i = 0; i < gtot; ++i) {
    if (!std::isfinite(gh[i])) {
      set_error("g_map has a non-finite entry");
      return fail(MCA_ERR_NONFINITE);
    }
    if (!(gh[i] > 0.0)) {
      set_error("g_map entries must be > 0");
      return fail(MCA_ERR_INVALID_ARG);
    }
  }
  if ((rc = dalloc(h, &h->g, gtot)) != MCA_OK) return fail(rc);
  if (cudaMemcpy(h->g, gh.data(), gtot * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(MCA_ERR_CUDA);
  // eigenpairs of the two wire operators
  const size_t nn = (size_t)h->n * h->n, mm = (size_t)h->m * h->m;
  double* scratch = nullptr;
  if ((rc = dalloc(h, &h->mu, h->n)) || (rc = dalloc(h, &h->nu, h->m)) ||
      (rc = dalloc(h, &h->Qr, nn)) || (rc = dalloc(h, &h->Qc, mm)) ||
      (rc = dalloc(h, &h->QrT, nn)) || (rc = dalloc(h, &h->QcT, mm)) ||
      (rc = dalloc(h, &scratch, std::max(nn, mm))))
    return fail(rc);
  cudaStream_t s = 0;
  launch_eig_tridiag(h->n, p->g_wire_top, p->g_src, p->g_term_top_right, h->mu, h->Qr,
                     scratch, s);
  count_launches(2);
  launch_eig_tridiag(h->m, p->g_wire_bot, p->g_term_bot_top, p->g_sense, h->nu, h->Qc,
                     scratch, s);
  count_launches(2);
  launch_transpose64(h->Qr, h->n, h->QrT, s);
  count_launches(1);
  launch_transpose64(h->Qc, h->m, h->QcT, s);
  count_launches(1);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    set_error("eigen setup kernels failed");
    return fail(MCA_ERR_CUDA);
  }
  if (is_tc(p->precision)) {
    const size_t npp = (size_t)h->np * h->np, mpp = (size_t)h->mp * h->mp;
    if ((rc = dalloc(h, &h->QrT_bf, npp)) || (rc = dalloc(h, &h->QcT_bf, mpp)) ||
        (rc = dalloc(h, &h->Qr_hi, npp)) || (rc = dalloc(h, &h->Qr_lo, npp)) ||
        (rc = dalloc(h, &h->Qc_hi, mpp)) || (rc = dalloc(h, &h->Qc_lo, mpp)))
      return fail(rc);
    // FP32 copies of the eigenvalues (host-side rounding of n + m values)
    std::vector<double> ev(std::max(h->m, h->n));
    std::vector<float> evf(ev.size());
    if ((rc = dalloc(h, &h->mu_f, h->n)) || (rc = dalloc(h, &h->nu_f, h->m))) return fail(rc);
    if (cudaMemcpy(ev.data(), h->mu, h->n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(MCA_ERR_CUDA);
    for (int i = 0; i < h->n; ++i) evf[i] = (float)ev[i];
    cudaMemcpy(h->mu_f, evf.data(), h->n * sizeof(float), cudaMemcpyHostToDevice);
    if (cudaMemcpy(ev.data(), h->nu, h->m * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(MCA_ERR_CUDA);
    for (int i = 0; i < h->m; ++i) evf[i] = (float)ev[i];
    cudaMemcpy(h->nu_f, evf.data(), h->m * sizeof(float), cudaMemcpyHostToDevice);
    launch_pack_q_bf16(h->Qr, h->n, h->np, h->Qr_hi, h->Qr_lo, h->QrT_bf, s);
    count_launches(1);
    launch_pack_q_bf16(h->Qc, h->m, h->mp, h->Qc_hi, h->Qc_lo, h->QcT_bf, s);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return fail(MCA_ERR_CUDA);
  }
  if ((rc = alloc_workspace(h)) != MCA_OK) return fail(rc);
  if (is_tc(p->precision)) {
    if ((rc = setup_tc(h)) != MCA_OK) return fail(rc);
    if ((p->flags & MCA_FLAG_AUTOTUNE) && (rc = autotune_tiles(h)) != MCA_OK) return fail(rc);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("create failed");
    return fail(MCA_ERR_CUDA);
  }
  *out = h;
  return MCA_OK;
}

int mca_solve(mca_handle* h, const double* v_in, int32_t nvec, double* v_top, double* v_bot,
              double* i_out, mca_stats* stats, void* stream) {
  return mca_solve_multi(h, v_in, nullptr, nvec, v_top, v_bot, i_out, stats, stream);
}

static int solve_impl(mca_handle* h, const double* v_in, const double* guess,
                      const double* fallback, const int32_t* map_index, int32_t nvec,
                      double* v_top, double* v_bot, double* i_out, mca_stats* stats,
                      void* stream);

int mca_solve_multi(mca_handle* h, const double* v_in, const int32_t* map_index, int32_t nvec,
                    double* v_top, double* v_bot, double* i_out, mca_stats* stats,
                    void* stream) {
  return solve_impl(h, v_in, nullptr, nullptr, map_index, nvec, v_top, v_bot, i_out, stats,
                    stream);
}

int mca_set_conductances(mca_handle* h, const double* g_maps) {
  g_last_error.clear();
  if (!h || !g_maps) {
    set_error("NULL argument");
    return MCA_ERR_INVALID_ARG;
  }
  const size_t gtot = h->mn * (size_t)h->n_maps;
  std::vector<double> gh(gtot);
  MCA_CUDA_TRY(cudaMemcpy(gh.data(), g_maps, gtot * sizeof(double), cudaMemcpyDefault));
  for (size_t i = 0; i < gtot; ++i) {
    if (!std::isfinite(gh[i])) {
      set_error("g_maps has a non-finite entry");
      return MCA_ERR_NONFINITE;
    }
    if (!(gh[i] > 0.0)) {
      set_error("g_maps entries must be > 0");
      return MCA_ERR_INVALID_ARG;
    }
  }
  MCA_CUDA_TRY(cudaMemcpy(h->g, gh.data(), gtot * sizeof(double), cudaMemcpyHostToDevice));
  return MCA_OK;
}

int mca_solve_from(mca_handle* h, const double* v_in, const double* guess,
                   const double* fallback, const int32_t* map_index, int32_t nvec,
                   double* v_top, double* v_bot, double* i_out, mca_stats* stats, void* stream) {
  if (!guess) {
    set_error("NULL guess");
    return MCA_ERR_INVALID_ARG;
  }
  return solve_impl(h, v_in, guess, fallback, map_index, nvec, v_top, v_bot, i_out, stats,
                    stream);
}

static int solve_passes(mca_handle* h, const double* v_in, const double* guess,
                        const double* fallback,
                        const int32_t* map_index, int32_t nvec, double* v_top, double* v_bot,
                        double* i_out, mca_stats* stats, cudaStream_t s);

static int solve_impl(mca_handle* h, const double* v_in, const double* guess,
                      const double* fallback, const int32_t* map_index, int32_t nvec,
                      double* v_top, double* v_bot, double* i_out, mca_stats* stats,
                      void* stream) {
  g_last_error.clear();
  if (!h || !v_in || nvec < 0) {
    set_error("NULL handle/input or negative nvec");
    return MCA_ERR_INVALID_ARG;
  }
  if (map_index) {
    for (int v = 0; v < nvec; ++v) {
      if (map_index[v] < 0 || map_index[v] >= h->n_maps) {
        set_error("map_index out of range");
        return MCA_ERR_INVALID_ARG;
      }
    }
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
  int rc = solve_passes(h, v_in, guess, fallback, map_index, nvec, v_top, v_bot, i_out, stats,
                        s);
  // the outputs of every pass are in place when the call returns
  for (int q = 0; q < 2; ++q) {
    if (!h->copy_pending[q]) continue;
    const cudaError_t e = cudaEventSynchronize(h->copy_done[q]);
    h->copy_pending[q] = false;
    if (e != cudaSuccess && (rc == MCA_OK || rc == MCA_ERR_NOT_CONVERGED ||
                             rc == MCA_ERR_NONFINITE)) {
      set_last_cuda_error(e, "output copy", __FILE__, __LINE__);
      rc = MCA_ERR_CUDA;
    }
  }
  return rc;
}

// The passes of a solve call: batches of up to max_batch vectors.  Pass p works in state
// buffer p % 2; its output copies go on the copy stream and overlap pass p + 1, which only
// has to wait for the copies of pass p - 1 (same buffer) before it overwrites the state.
// Inputs of the pass starting at vector v0 into staging buffer q (on s).
static int stage_inputs(mca_handle* h, const double* v_in, const int32_t* map_index, int v0,
                        int B, int q, cudaStream_t s) {
  MCA_CUDA_TRY(cudaMemcpyAsync(h->vinbuf[q], v_in + (size_t)v0 * h->m,
                               (size_t)B * h->m * sizeof(double), cudaMemcpyDefault, s));
  if (h->n_maps > 1) {
    for (int b = 0; b < B; ++b) h->map_host[b] = map_index ? map_index[v0 + b] : 0;
    MCA_CUDA_TRY(cudaMemcpyAsync(h->mapbuf[q], h->map_host.data(), (size_t)B * sizeof(int),
                                 cudaMemcpyHostToDevice, s));
  }
  return MCA_OK;
}

static int solve_passes(mca_handle* h, const double* v_in, const double* guess,
                        const double* fallback, const int32_t* map_index, int32_t nvec,
                        double* v_top, double* v_bot, double* i_out, mca_stats* stats,
                        cudaStream_t s) {
  const size_t m = h->m, n = h->n, mn = h->mn;
  (void)m;
  int worst = MCA_OK;
  int pass = 0;
  if (nvec > 0) MCA_TRY(stage_inputs(h, v_in, map_index, 0, std::min(h->Bmax, nvec), 0, s));
  for (int v0 = 0; v0 < nvec; v0 += h->Bmax, ++pass) {
    const int B = std::min(h->Bmax, nvec - v0);
    const int q = pass & 1;
    if (h->copy_pending[q]) MCA_CUDA_TRY(cudaStreamWaitEvent(s, h->copy_done[q], 0));
    h->x = h->xbuf[q];
    h->iout = h->ioutbuf[q];
    h->vin = h->vinbuf[q];
    h->map_of = h->mapbuf[q];
    std::vector<int> fell(B, 0);
    if (guess) {
      // judge the guess: keep it only if its residual is finite and below that of the
      // fallback state (||F(0)|| = ||Y|| when there is none)
      const int nb = residual_nblk((int)h->mn, B);
      SolverCfg probe = make_cfg(h);
      probe.max_newton = 0;
      probe.newton_rtol = 0.0;
      // ||F|| of the states now in h->x (map-aware through the Newton kernel with
      // max_newton = 0), into fn[b]
      auto probe_norms = [&](std::vector<double>& fn) -> int {
        launch_setup_vectors(h->gr, h->vin, B, h->ctl, false, s);
        count_launches(1);
        launch_residual_newton(h->gr, h->g, h->n_maps > 1 ? h->map_of : nullptr, h->vin, h->x,
                               false, h->F, h->n2, nullptr, 0, 0, h->D, h->part, nb, B, h->ctl,
                               probe, h->cnt, nullptr, s);
        count_launches(1);
        MCA_TRY(read_report(h, B, nullptr, nullptr, s));
        for (int b = 0; b < B; ++b)
          fn[b] = (h->ctl_host[b].ynorm > 0.0) ? h->ctl_host[b].fnorm : 0.0;
        return MCA_OK;
      };
      std::vector<double> fref(B), fg(B);
      if (fallback) {
        MCA_CUDA_TRY(cudaMemcpyAsync(h->x, fallback + (size_t)v0 * h->n2,
                                     (size_t)B * h->n2 * sizeof(double), cudaMemcpyDefault, s));
        MCA_TRY(probe_norms(fref));
      }
      MCA_CUDA_TRY(cudaMemcpyAsync(h->x, guess + (size_t)v0 * h->n2,
                                   (size_t)B * h->n2 * sizeof(double), cudaMemcpyDefault, s));
      MCA_TRY(probe_norms(fg));
      for (int b = 0; b < B; ++b) {
        const double yn = h->ctl_host[b].ynorm;
        const double ref = fallback ? fref[b] : yn;
        const bool ok = std::isfinite(fg[b]) && fg[b] < ref;
        if (!ok && yn > 0.0) {
          fell[b] = 1;
          double* xb = h->x + (size_t)b * h->n2;
          if (fallback)
            MCA_CUDA_TRY(cudaMemcpyAsync(xb, fallback + (size_t)(v0 + b) * h->n2,
                                         h->n2 * sizeof(double), cudaMemcpyDefault, s));
          else
            MCA_CUDA_TRY(cudaMemsetAsync(xb, 0, h->n2 * sizeof(double), s));
        }
      }
    }
    int rc = solve_pass(h, B, s, guess != nullptr);
    if (rc != MCA_OK) return rc;
    // the next pass' inputs, then this pass' output copies on the copy stream
    const int v1 = v0 + h->Bmax;
    if (v1 < nvec)
      MCA_TRY(stage_inputs(h, v_in, map_index, v1, std::min(h->Bmax, nvec - v1), q ^ 1, s));
    cudaStream_t cs = h->copy_stream;
    MCA_CUDA_TRY(cudaEventRecord(h->ev_solved, s));
    MCA_CUDA_TRY(cudaStreamWaitEvent(cs, h->ev_solved, 0));
    // one strided copy per layer: state rows of 2 m n doubles into output rows of m n
    if (v_top)
      MCA_CUDA_TRY(cudaMemcpy2DAsync(v_top + (size_t)v0 * mn, mn * sizeof(double), h->x,
                                     h->n2 * sizeof(double), mn * sizeof(double), B,
                                     cudaMemcpyDefault, cs));
    if (v_bot)
      MCA_CUDA_TRY(cudaMemcpy2DAsync(v_bot + (size_t)v0 * mn, mn * sizeof(double), h->x + mn,
                                     h->n2 * sizeof(double), mn * sizeof(double), B,
                                     cudaMemcpyDefault, cs));
    MCA_TRY(copy_out(i_out ? i_out + (size_t)v0 * n : nullptr, h->iout,
                     (size_t)B * n * sizeof(double), cs));
    MCA_CUDA_TRY(cudaEventRecord(h->copy_done[q], cs));
    h->copy_pending[q] = true;
    std::vector<double> kcl(B);
    MCA_TRY(read_report(h, B, h->kcl, kcl.data(), s));
    for (int b = 0; b < B; ++b) {
      const VecCtl& c = h->ctl_host[b];
      if (c.status != MCA_OK && worst == MCA_OK) worst = c.status;
      if (stats) {
        mca_stats& st = stats[v0 + b];
        st.status = c.status;
        st.newton_iters = c.newton_iters;
        st.gmres_iters = c.gmres_iters;
        st.fallback = fell[b];
        st.rel_residual = (c.ynorm > 0.0) ? c.fnorm / c.ynorm : 0.0;
        st.kcl_rel_error = kcl[b];
      }
    }
  }
  return worst;
}

int mca_solve_many(mca_handle* const* hs, int32_t nh, const double* const* v_in,
                   const int32_t* const* map_index, const int32_t* nvec,
                   double* const* v_top, double* const* v_bot, double* const* i_out,
                   mca_stats* const* stats, int32_t n_threads) {
  g_last_error.clear();
  if (!hs || !v_in || !nvec || nh < 0 || n_threads < 1) {
    set_error("bad arguments");
    return MCA_ERR_INVALID_ARG;
  }
  std::atomic<int> next{0};
  std::mutex mu;
  int worst = MCA_OK;
  std::string first_msg;
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(mu);
      if (worst == MCA_OK) worst = MCA_ERR_CUDA;
      return;
    }
    for (int i = next++; i < nh; i = next++) {
      int rc = mca_solve_multi(hs[i], v_in[i], map_index ? map_index[i] : nullptr, nvec[i],
                               v_top ? v_top[i] : nullptr, v_bot ? v_bot[i] : nullptr,
                               i_out ? i_out[i] : nullptr, stats ? stats[i] : nullptr, s);
      if (rc != MCA_OK) {
        std::lock_guard<std::mutex> lock(mu);
        if (worst == MCA_OK) {
          worst = rc;
          first_msg = g_last_error;
        }
      }
    }
    cudaStreamDestroy(s);
  };
  const int nt = std::min<int>(n_threads, std::max(1, nh));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  g_last_error = first_msg;
  return worst;
}

void mca_batch_destroy(mca_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  for (void* q : b->allocs) cudaFree(q);
  if (b->items_host) cudaFreeHost(b->items_host);
  if (b->res_host) cudaFreeHost(b->res_host);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

int mca_batch_create(mca_handle* const* hs, int32_t nh, int32_t max_ctas, mca_batch** out) {
  g_last_error.clear();
  if (!out || !hs || nh < 1 || max_ctas < 0) {
    set_error("bad arguments");
    return MCA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int k = 0; k < nh; ++k) {
    const mca_handle* h = hs[k];
    if (!h) {
      set_error("null handle");
      return MCA_ERR_INVALID_ARG;
    }
    if (h->device != hs[0]->device) {
      set_error("handles on different devices");
      return MCA_ERR_INVALID_ARG;
    }
    if (h->p.precision != MCA_PREC_BF16_SPLIT || !h->tc_ok) {
      set_error("the persistent solve needs MCA_PREC_BF16_SPLIT handles");
      return MCA_ERR_UNSUPPORTED;
    }
    if (h->gr.yak != hs[0]->gr.yak) {
      set_error("handles with different device models");
      return MCA_ERR_INVALID_ARG;
    }
  }
  std::unique_ptr<mca_batch> b(new mca_batch);
  b->device = hs[0]->device;
  MCA_CUDA_TRY(cudaSetDevice(b->device));
  b->hs.assign(hs, hs + nh);
  b->yak = hs[0]->gr.yak != 0;
  auto alloc = [&](void** q, size_t bytes) -> int {
    *q = nullptr;
    if (cudaMalloc(q, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation failed");
      return MCA_ERR_OOM;
    }
    b->allocs.push_back(*q);
    return MCA_OK;
  };
  MCA_CUDA_TRY(cudaStreamCreate(&b->own_stream));
  MCA_CUDA_TRY(persist_configure());
  // eigenvector operands of each shape in the tiled layout of the persistent kernel
  std::vector<PersistShape> shp(nh);
  size_t n2max = 0, bfmax = 0;
  int rmax = 1;
  for (int k = 0; k < nh; ++k) {
    mca_handle* h = hs[k];
    const size_t mp = h->mp, np = h->np;
    __nv_bfloat16* t[6];
    const __nv_bfloat16* src[6] = {h->QrT_bf, h->QcT_bf, h->Qr_hi, h->Qr_lo, h->Qc_hi, h->Qc_lo};
    const size_t dim[6] = {np, mp, np, np, mp, mp};
    for (int q = 0; q < 6; ++q) {
      MCA_TRY(alloc(reinterpret_cast<void**>(&t[q]), dim[q] * dim[q] * sizeof(__nv_bfloat16)));
      // transforms 2, 3 and 4 take 32-wide K chunks, transform 1 64-wide
      launch_retile_bf16(src[q], (int)dim[q], (int)dim[q], t[q], q >= 1, b->own_stream);
      count_launches(1);
    }
    PersistShape& ps = shp[k];
    ps.gr = h->gr;
    ps.cfg = make_cfg(h);
    ps.mp = h->mp;
    ps.np = h->np;
    ps.gmaps = h->g;
    ps.mu_f = h->mu_f;
    ps.nu_f = h->nu_f;
    ps.qrt = t[0];
    ps.qct = t[1];
    ps.qr_hi = t[2];
    ps.qr_lo = t[3];
    ps.qc_hi = t[4];
    ps.qc_lo = t[5];
    n2max = std::max(n2max, 2 * ((h->mn + 3) / 4 * 4));   // two layers padded to 4 entries
    bfmax = std::max(bfmax, 2 * mp * np);
    rmax = std::max(rmax, h->restart);
  }
  MCA_TRY(alloc(reinterpret_cast<void**>(&b->shapes), nh * sizeof(PersistShape)));
  MCA_CUDA_TRY(cudaMemcpyAsync(b->shapes, shp.data(), nh * sizeof(PersistShape),
                               cudaMemcpyHostToDevice, b->own_stream));
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->grid = max_ctas > 0 ? max_ctas : 2 * sms;
  const size_t slot = persist_slot_layout(b->slots, n2max, bfmax, rmax);
  void* base = nullptr;
  MCA_TRY(alloc(&base, slot * (size_t)b->grid));
  b->slots.base = static_cast<uint8_t*>(base);
  MCA_TRY(alloc(reinterpret_cast<void**>(&b->flags), 2 * sizeof(int)));
  MCA_CUDA_TRY(cudaGetLastError());
  MCA_CUDA_TRY(cudaStreamSynchronize(b->own_stream));
  *out = b.release();
  return MCA_OK;
}

namespace {
// Grow the item and result buffers of a batch to hold n items.
int batch_reserve(mca_batch* b, int n) {
  if (n <= b->cap) return MCA_OK;
  if (b->items_host) cudaFreeHost(b->items_host);
  if (b->res_host) cudaFreeHost(b->res_host);
  b->items_host = nullptr;
  b->res_host = nullptr;
  for (void* q : {static_cast<void*>(b->items), static_cast<void*>(b->res)}) {
    if (!q) continue;
    cudaFree(q);
    b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), q));
  }
  b->items = nullptr;
  b->res = nullptr;
  b->cap = 0;
  void *pi = nullptr, *pr = nullptr;
  if (cudaMalloc(&pi, n * sizeof(PersistItem)) != cudaSuccess ||
      cudaMalloc(&pr, n * sizeof(PersistResult)) != cudaSuccess) {
    cudaGetLastError();
    if (pi) cudaFree(pi);
    set_error("device allocation failed");
    return MCA_ERR_OOM;
  }
  b->allocs.push_back(pi);
  b->allocs.push_back(pr);
  b->items = static_cast<PersistItem*>(pi);
  b->res = static_cast<PersistResult*>(pr);
  MCA_CUDA_TRY(cudaMallocHost(&b->items_host, n * sizeof(PersistItem)));
  MCA_CUDA_TRY(cudaMallocHost(&b->res_host, n * sizeof(PersistResult)));
  b->cap = n;
  return MCA_OK;
}

// One launch of the persistent kernel over n items (mode 0: solve, 1: preconditioner).
// Items are queued largest first (tensor-core work ~ m n (m + n), memory work ~ m n).
int batch_run(mca_batch* b, const mca_item* items, const double* a, int n, int mode,
              mca_stats* stats, cudaStream_t s) {
  for (int k = 0; k < n; ++k) {
    const mca_item& it = items[k];
    if (it.handle < 0 || it.handle >= (int)b->hs.size()) {
      set_error("item handle index out of range");
      return MCA_ERR_INVALID_ARG;
    }
    const mca_handle* h = b->hs[it.handle];
    if (it.map < 0 || it.map >= h->n_maps) {
      set_error("item map index out of range");
      return MCA_ERR_INVALID_ARG;
    }
    if (mode == 0 && !it.v_in) {
      set_error("item without input vector");
      return MCA_ERR_INVALID_ARG;
    }
    if (mode == 1 && (!it.v_top || !it.v_bot)) {
      set_error("preconditioner item without vectors");
      return MCA_ERR_INVALID_ARG;
    }
  }
  if (n == 0) return MCA_OK;
  MCA_TRY(batch_reserve(b, n));
  std::vector<int> order(n);
  std::vector<double> cost(n);
  for (int k = 0; k < n; ++k) {
    const mca_handle* h = b->hs[items[k].handle];
    order[k] = k;
    cost[k] = (double)h->mp * h->np * (1.0 + (h->mp + h->np) / 4096.0);
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return cost[x] > cost[y]; });
  for (int q = 0; q < n; ++q) {
    const mca_item& it = items[order[q]];
    PersistItem& pi = b->items_host[q];
    pi.shape = it.handle;
    pi.map = it.map;
    pi.vin = it.v_in;
    pi.vt = it.v_top;
    pi.vb = it.v_bot;
    pi.iout = it.i_out;
    pi.a = a ? a[order[q]] : 0.0;
  }
  MCA_CUDA_TRY(cudaMemcpyAsync(b->items, b->items_host, n * sizeof(PersistItem),
                               cudaMemcpyHostToDevice, s));
  MCA_CUDA_TRY(cudaMemsetAsync(b->flags, 0, 2 * sizeof(int), s));
  launch_persist(b->shapes, b->items, n, b->res, b->flags, b->flags + 1, b->slots,
                 std::min(b->grid, n), mode, b->yak, b->prof, s);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  int err = 0;
  MCA_CUDA_TRY(cudaMemcpyAsync(b->res_host, b->res, n * sizeof(PersistResult),
                               cudaMemcpyDeviceToHost, s));
  MCA_CUDA_TRY(cudaMemcpyAsync(&err, b->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  if (err != 0) {
    set_error("a bounded wait in the persistent kernel gave up");
    return MCA_ERR_TIMEOUT;
  }
  if (mode != 0) return MCA_OK;
  int worst = MCA_OK;
  for (int q = 0; q < n; ++q) {
    const PersistResult& r = b->res_host[q];
    if (stats) {
      mca_stats& st = stats[order[q]];
      st.status = r.status;
      st.newton_iters = r.newton_iters;
      st.gmres_iters = r.gmres_iters;
      st.fallback = 0;
      st.rel_residual = (r.ynorm > 0.0) ? r.fnorm / r.ynorm : 0.0;
      st.kcl_rel_error = r.kcl;
    }
    if (r.status != MCA_OK && worst == MCA_OK) worst = r.status;
  }
  return worst;
}
}  // namespace

int mca_batch_solve(mca_batch* b, const mca_item* items, int32_t n, mca_stats* stats,
                    void* stream) {
  g_last_error.clear();
  if (!b || (n > 0 && !items) || n < 0) {
    set_error("bad arguments");
    return MCA_ERR_INVALID_ARG;
  }
  MCA_CUDA_TRY(cudaSetDevice(b->device));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->own_stream;
  return batch_run(b, items, nullptr, n, 0, stats, s);
}

int mca_batch_profile(mca_batch* b, int32_t enable) {
  g_last_error.clear();
  if (!b) {
    set_error("bad arguments");
    return MCA_ERR_INVALID_ARG;
  }
  MCA_CUDA_TRY(cudaSetDevice(b->device));
  if (!enable) {
    b->prof = nullptr;
    return MCA_OK;
  }
  static_assert(MCA_BATCH_PHASES <= 16, "profile buffer");
  if (!b->prof) {
    void* q = nullptr;
    if (cudaMalloc(&q, 16 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation failed");
      return MCA_ERR_OOM;
    }
    b->allocs.push_back(q);
    b->prof = static_cast<unsigned long long*>(q);
  }
  MCA_CUDA_TRY(cudaMemset(b->prof, 0, 16 * sizeof(unsigned long long)));
  return MCA_OK;
}

int mca_batch_profile_read(mca_batch* b, double* ms) {
  g_last_error.clear();
  if (!b || !ms || !b->prof) {
    set_error(b && !b->prof ? "profiling is not enabled" : "bad arguments");
    return MCA_ERR_INVALID_ARG;
  }
  MCA_CUDA_TRY(cudaSetDevice(b->device));
  unsigned long long ns[MCA_BATCH_PHASES];
  MCA_CUDA_TRY(cudaMemcpy(ns, b->prof, sizeof(ns), cudaMemcpyDeviceToHost));
  for (int k = 0; k < MCA_BATCH_PHASES; ++k) ms[k] = (double)ns[k] * 1e-6;
  return MCA_OK;
}

int mca_batch_precond(mca_batch* b, const mca_item* items, const double* a, int32_t n,
                      void* stream) {
  g_last_error.clear();
  if (!b || (n > 0 && (!items || !a)) || n < 0) {
    set_error("bad arguments");
    return MCA_ERR_INVALID_ARG;
  }
  MCA_CUDA_TRY(cudaSetDevice(b->device));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->own_stream;
  return batch_run(b, items, a, n, 1, nullptr, s);
}

int mca_residual(mca_handle* h, const double* x, const double* v_in, int32_t nvec, double* F,
                 double* D, double* fnorm, double* dmean, void* stream) {
  g_last_error.clear();
  if (!h || !x || !v_in || !F || !D || nvec < 1 || nvec > h->Bmax) {
    set_error("bad arguments (nvec must be in 1..max_batch)");
    return MCA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = residual_nblk((int)h->mn);
  launch_residual(h->gr, h->g, v_in, x, F, D, h->part, nb, nvec, nullptr, s);
  count_launches(1);
  launch_reduce_dots(h->part, nb, 2, h->h1, nvec, nullptr, s);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  std::vector<double> hh((size_t)nvec * 32);
  MCA_CUDA_TRY(cudaMemcpyAsync(hh.data(), h->h1, hh.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  for (int b = 0; b < nvec; ++b) {
    if (fnorm) fnorm[b] = std::sqrt(hh[(size_t)b * 32]);
    if (dmean) dmean[b] = hh[(size_t)b * 32 + 1] / (double)h->mn;
  }
  return MCA_OK;
}

int mca_residual_pair(mca_handle* h, const double* x, const double* v_in, int32_t nvec,
                      double* F, double* D, double* fnorm, double* dmean, double* ferr,
                      void* stream) {
  g_last_error.clear();
  if (!h || !x || !v_in || !F || !D || nvec < 1 || nvec > h->Bmax) {
    set_error("bad arguments (nvec must be in 1..max_batch)");
    return MCA_ERR_INVALID_ARG;
  }
  if (!h->gr.tail32) {
    set_error("the FP32-pair residual needs b in about [0.021, 2000] (FP32 polynomial tail)");
    return MCA_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = residual_nblk((int)h->mn);
  launch_residual(h->gr, h->g, v_in, x, F, D, h->part, nb, nvec, nullptr, s, true);
  count_launches(1);
  launch_reduce_dots(h->part, nb, 3, h->h1, nvec, nullptr, s);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  std::vector<double> hh((size_t)nvec * 32);
  MCA_CUDA_TRY(cudaMemcpyAsync(hh.data(), h->h1, hh.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  for (int b = 0; b < nvec; ++b) {
    if (fnorm) fnorm[b] = std::sqrt(hh[(size_t)b * 32]);
    if (dmean) dmean[b] = hh[(size_t)b * 32 + 1] / (double)h->mn;
    if (ferr) ferr[b] = pair_err_bound(hh[(size_t)b * 32 + 2]);
  }
  return MCA_OK;
}

int mca_jacobian_apply(mca_handle* h, const double* D, const double* z, double* w, int32_t nvec,
                       void* stream) {
  g_last_error.clear();
  if (!h || !D || !z || !w || nvec < 1 || nvec > h->Bmax) {
    set_error("bad arguments (nvec must be in 1..max_batch)");
    return MCA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_spmv_dots(h->gr, D, z, h->n2, w, nullptr, 0, 0, h->part, residual_nblk((int)h->mn),
                   nvec, nullptr, nullptr, nullptr, s);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  return MCA_OK;
}

int mca_jacobian_apply_f32(mca_handle* h, const double* D, const float* z, double* w,
                           int32_t nvec, int32_t mode, void* stream) {
  g_last_error.clear();
  if (!h || !D || !z || !w || nvec < 1 || nvec > h->Bmax) {
    set_error("bad arguments (nvec must be in 1..max_batch)");
    return MCA_ERR_INVALID_ARG;
  }
  int apply;
  switch (mode) {
    case MCA_APPLY_PAIR: apply = kApplyPair; break;
    case MCA_APPLY_F64: apply = kApplyF64; break;
    case MCA_APPLY_F32: apply = kApplyF32; break;
    default:
      set_error("mode must be MCA_APPLY_PAIR, MCA_APPLY_F64 or MCA_APPLY_F32");
      return MCA_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_spmv_dots(h->gr, D, z, h->n2, w, nullptr, 0, 0, h->part, residual_nblk((int)h->mn),
                   nvec, nullptr, nullptr, nullptr, s, apply);
  count_launches(1);
  MCA_CUDA_TRY(cudaGetLastError());
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  return MCA_OK;
}

static int load_ctl_a(mca_handle* h, const double* a, int nvec, cudaStream_t s) {
  for (int b = 0; b < nvec; ++b) {
    if (!finite_pos(a[b])) {
      set_error("a must be finite and > 0");
      return MCA_ERR_INVALID_ARG;
    }
    VecCtl& c = h->ctl_host[b];
    memset(&c, 0, sizeof(VecCtl));
    c.a = a[b];
    c.gm_active = 1;
    c.newton_active = 1;
    c.d64 = 1;                     // D is the caller's: split it in the pair apply
  }
  MCA_CUDA_TRY(cudaMemcpyAsync(h->ctl, h->ctl_host.data(), (size_t)nvec * sizeof(VecCtl),
                               cudaMemcpyHostToDevice, s));
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  return MCA_OK;
}

int mca_precond_apply(mca_handle* h, const double* a, const double* r, double* z, int32_t nvec,
                      int32_t precision, void* stream) {
  g_last_error.clear();
  if (!h || !a || !r || !z || nvec < 1 || nvec > h->Bmax) {
    set_error("bad arguments (nvec must be in 1..max_batch)");
    return MCA_ERR_INVALID_ARG;
  }
  const bool ok = (precision == MCA_PREC_MHAT) ||
                  (precision == MCA_PREC_FP64 && h->p.precision == MCA_PREC_FP64) ||
                  (is_tc(precision) && is_tc(h->p.precision));
  if (!ok) {
    set_error("precision not prepared by this handle");
    return MCA_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MCA_TRY(load_ctl_a(h, a, nvec, s));
  if (is_tc(precision)) {
    tc::cast_pad(r, h->n2, h->Xbf, h->m, h->n, h->mp, h->np, nvec, s);
    count_launches(1);
  }
  MCA_TRY(precond_apply(h, precision, r, h->n2, z, h->n2, nvec, h->ctl, s));
  MCA_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(h);
}

int mca_eigenpairs(mca_handle* h, double* mu, double* q_r, double* nu, double* q_c) {
  g_last_error.clear();
  if (!h) return MCA_ERR_INVALID_ARG;
  const size_t nn = (size_t)h->n * h->n, mm = (size_t)h->m * h->m;
  if (mu) MCA_CUDA_TRY(cudaMemcpy(mu, h->mu, h->n * sizeof(double), cudaMemcpyDefault));
  if (q_r) MCA_CUDA_TRY(cudaMemcpy(q_r, h->Qr, nn * sizeof(double), cudaMemcpyDefault));
  if (nu) MCA_CUDA_TRY(cudaMemcpy(nu, h->nu, h->m * sizeof(double), cudaMemcpyDefault));
  if (q_c) MCA_CUDA_TRY(cudaMemcpy(q_c, h->Qc, mm * sizeof(double), cudaMemcpyDefault));
  return MCA_OK;
}

int mca_gmres_solve(mca_handle* h, const double* D, const double* a, const double* rhs,
                    double* dx, int32_t nvec, double rtol, int32_t max_iters, int32_t* iters,
                    double* res, void* stream) {
  g_last_error.clear();
  if (!h || !D || !a || !rhs || !dx || nvec < 1 || nvec > h->Bmax || !(rtol > 0.0)) {
    set_error("bad arguments (nvec must be in 1..max_batch, rtol > 0)");
    return MCA_ERR_INVALID_ARG;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
  const size_t n2 = h->n2;
  const size_t vstride = (size_t)(h->restart + 1) * n2;
  const size_t zstride = (size_t)h->restart * n2;
  const bool tc = is_tc(h->p.precision);
  const int nbV = vec_nblk(n2, nvec);
  const int nbS = residual_nblk((int)h->mn, nvec);
  const int cap = (max_iters > 0) ? max_iters : h->restart;
  MCA_TRY(load_ctl_a(h, a, nvec, s));
  MCA_CUDA_TRY(cudaMemsetAsync(dx, 0, (size_t)nvec * n2 * sizeof(double), s));
  // r = rhs (dx = 0)
  MCA_CUDA_TRY(cudaMemcpyAsync(h->F, rhs, (size_t)nvec * n2 * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
  std::vector<int> total(nvec, 0);
  for (int cycle = 0;; ++cycle) {
    // beta = ||r||, v_0 = r / beta
    MCA_CUDA_TRY(cudaMemcpyAsync(h->W, h->F, (size_t)nvec * n2 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
    launch_update_norm(UPD_PLAIN, h->W, n2, h->V, vstride, n2, 0, h->h2, h->part, nbV, nvec,
                       nullptr, nullptr, nullptr, h->restart, nullptr, h->W, n2, nullptr, 0, 0,
                       h->m, h->n, s);
    launch_gmres_init(h->part, nbV, h->ctl, nvec, rtol, cycle == 0 ? 1 : 0, s);
    launch_init_basis(h->F, 1.0, h->V, vstride, tc ? h->Xbf : nullptr, h->mp, h->np, h->m,
                      h->n, h->ctl, nvec, s);
    count_launches(3);
    MCA_TRY(gmres_cycle(h, D, nvec, s));
    if (tc)
      launch_lsq_update(dx, h->Z32, zstride, n2, h->ctl, nvec, s);
    else
      launch_lsq_update(dx, h->Z, zstride, n2, h->ctl, nvec, s);
    count_launches(2);
    MCA_CUDA_TRY(cudaGetLastError());
    MCA_CUDA_TRY(cudaMemcpyAsync(h->ctl_host.data(), h->ctl, (size_t)nvec * sizeof(VecCtl),
                                 cudaMemcpyDeviceToHost, s));
    MCA_CUDA_TRY(cudaStreamSynchronize(s));
    bool more = false;
    for (int b = 0; b < nvec; ++b) {
      const VecCtl& c = h->ctl_host[b];
      total[b] += c.k_done;
      if (c.res_est > c.tol_abs && total[b] < cap) more = true;
    }
    if (!more || max_iters <= 0) break;
    // restart from the true residual r = rhs - J dx (vectors already converged restart
    // with a residual below their tolerance and do no further work)
    launch_spmv_dots(h->gr, D, dx, n2, h->W, nullptr, 0, 0, h->part, nbS, nvec, nullptr,
                     nullptr, nullptr, s);
    launch_sub(rhs, h->W, h->F, n2, nvec, s);
    count_launches(2);
  }
  for (int b = 0; b < nvec; ++b) {
    if (iters) iters[b] = total[b];
    if (res) res[b] = h->ctl_host[b].res_est;
  }
  return check_device_error(h);
}

int64_t mca_kernel_launches(void) { return g_launches.load(); }

int mca_tile_config(const mca_handle* h, int32_t* cfg) {
  if (!h || !cfg) return MCA_ERR_INVALID_ARG;
  for (int s = 0; s < 4; ++s) {
    cfg[3 * s + 0] = h->tc_ok ? h->ws[s] : -1;
    cfg[3 * s + 1] = h->tc_ok ? h->bn[s] : 0;
    cfg[3 * s + 2] = h->tc_ok ? (h->ws[s] ? h->lp[s] : 2) : 0;
  }
  return MCA_OK;
}

int mca_wait_selftest(mca_handle* h, int64_t limit_ns) {
  g_last_error.clear();
  if (!h || limit_ns < 0) return MCA_ERR_INVALID_ARG;
  MCA_CUDA_TRY(cudaMemset(h->err, 0, sizeof(int)));
  MCA_CUDA_TRY(tc::wait_selftest((unsigned long long)limit_ns, h->err, h->own_stream));
  count_launches(1);
  MCA_CUDA_TRY(cudaStreamSynchronize(h->own_stream));
  return check_device_error(h);
}

int mca_profile(mca_handle* h, int32_t enable) {
  if (!h) return MCA_ERR_INVALID_ARG;
  h->prof_on = enable != 0;
  h->prof_pending.clear();
  h->prof_next = 0;
  for (int f = 0; f < MCA_NUM_FAMILIES; ++f) {
    h->prof_launches[f] = 0;
    h->prof_ms[f] = h->prof_bytes[f] = h->prof_flops[f] = 0.0;
  }
  return MCA_OK;
}

int mca_profile_read(mca_handle* h, int32_t family, int64_t* launches, double* ms,
                     double* bytes, double* flops) {
  if (!h || family < 0 || family >= MCA_NUM_FAMILIES) return MCA_ERR_INVALID_ARG;
  if (launches) *launches = h->prof_launches[family];
  if (ms) *ms = h->prof_ms[family];
  if (bytes) *bytes = h->prof_bytes[family];
  if (flops) *flops = h->prof_flops[family];
  return MCA_OK;
}

}  // extern "C"
