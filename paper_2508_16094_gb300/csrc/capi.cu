// C ABI of the solver (declared in include/gb300_ipm.h): context, workspace,
// assembly/factor/solve drivers with FP64 refinement and PCG, and the
// interior-point iteration.
#include <algorithm>
#include <functional>
#include <chrono>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <mutex>
#include <stdexcept>

#include "../../include/gb300_ipm.h"
#include "forms.h"
#include "ipm_kernels.h"
#include "launch.h"
#include "learned.h"
#include "nlp.h"
#include "oz.h"
#include "tc.h"

using namespace gipm;

struct ipm_ctx {
  Problem P;
  Symbolic S;
  Plan plan;
  ipm_options opts;
  cudaStream_t st = nullptr;
  int device = -1;  // the GPU current at ipm_set_workspace (the workspace's device)
  int state = 0;  // 0 created, 1 analysed, 2 workspace, 3 assembled, 4 factored
  std::string err;
  // workspace
  char *ws = nullptr;
  size_t ws_bytes = 0, ws_need = 0;
  int storage_bytes = 8;  // bytes per stored factor entry
  DevPlan dp{};
  double *kval = nullptr;
  void *L = nullptr, *U = nullptr;
  double *yv = nullptr, *tv = nullptr;  // solve scratch (doubles; float views)
  double *vx = nullptr, *vr = nullptr, *vc = nullptr, *vz = nullptr, *vp = nullptr,
         *vq = nullptr, *vb = nullptr, *vdx = nullptr, *vrd = nullptr, *vwx = nullptr;
  double *vg = nullptr, *vD = nullptr, *vw = nullptr, *vds = nullptr, *vdl = nullptr,
         *vt = nullptr, *vjd = nullptr, *vjx = nullptr, *vtA = nullptr;
  double *dl_ = nullptr, *du_ = nullptr;
  double *jv_copy = nullptr, *D_copy = nullptr, *wv_copy = nullptr;  // inputs kept for refinement
  float *Llo = nullptr;  // low parts of the split-TF32 factor
  float *dinv = nullptr, *fsa = nullptr, *fsb = nullptr, *fsx = nullptr;  // persistent FP32 solve
  unsigned *psflags = nullptr;  // its tickets, flags and counters
  float *pspart = nullptr;    // its partial sums
  // learned correction of a stale factor
  LearnedBufs lb;
  bool learned_active = false;  // PCG preconditioner = corrected stale factor
  bool lb_on = false;           // learned buffers sized for n (fixed by the layout)
  bool nlp_grad = false;        // direction(): cc is the whole gradient (no W x term)
  bool bwd_measure = false;     // do_solve: normwise backward error instead of ||r|| / ||b||
  bool warm_x = false;          // do_solve: start from the incoming x (x + M^-1 (b - K x))
  double knorm = 0.0;           // ||K||_inf of the assembled matrix (when bwd_measure)
  bool have_stale = false;      // lb.D_old / diag_old / mu[0] describe the held factor
  int refine_override = -1, pcg_override = -1;
  unsigned test_spins = 0;   // next persistent solve launch only: barrier poll limit
  int test_withhold = -1;    // ... and the ticket of the task it abandons
  double *lb_loss = nullptr;
  double *scal = nullptr, *partial = nullptr;
  IpmScalars *sc = nullptr;
  int32_t *status = nullptr, *col2s = nullptr;
  TcPlan tcp;
  OzPlan ozp;          // FP64 factor on tensor cores (Ozaki slices), with options.fp64_tc
  bool oz_on = false;  // its task lists and slice storage were sized by kkt_analyze
  int64_t oz_rechecks = 0;  // its failed pivots redone on the FMA pipe
  // formulations (4) and (6): `sys` is the context of that system's matrix
  // (its pattern, symbolic analysis, factor and solves); this context keeps
  // the interior-point vectors and builds sys's inputs with the map kernels
  // of forms.cu
  int form = IPM_FORM_PRIMAL;
  ipm_ctx *sys = nullptr;
  std::vector<int8_t> sign_orig;  // pivot signs of a quasi-definite system (original numbering)
  std::vector<int64_t> wdiag_h;   // per variable: index of W_jj in W's values, or -1
  std::vector<int32_t> aug_kind_h;
  std::vector<int64_t> aug_idx_h;
  int64_t *wdiag = nullptr, *aug_idx = nullptr;
  int32_t *aug_kind = nullptr;
  double *hdiag = nullptr, *rtil = nullptr, *qv = nullptr, *sysb = nullptr, *sysx = nullptr,
         *sysw = nullptr, *sysD = nullptr, *sysj = nullptr;
  size_t outer_need = 0;  // bytes of this context's own part of the workspace
  // inputs of the last assembly (device pointers, used by the residual)
  const double *cur_jvals = nullptr, *cur_D = nullptr, *cur_wvals = nullptr;
  double cur_delta_p = 0.0;
  int factor_prec = -1;
  int32_t last_perturbed = 0;
  int64_t refine_steps = 0, pcg_steps = 0;
  double last_rel = 0.0;
  VecOps vec() const { return VecOps{dp, st, partial}; }
  ~ipm_ctx() { delete sys; }
};

namespace gipm {
int64_t &launch_counter() {
  static int64_t count = 0;
  return count;
}
}  // namespace gipm

namespace {

struct Fail {
  ipm_status code;
  std::string msg;
};

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw Fail{IPM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};       \
  } while (0)

template <typename F>
ipm_status guarded(ipm_ctx *ctx, F &&f) {
  try {
    return f();
  } catch (const Fail &e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    if (ctx) ctx->err = "host allocation failed";
    return IPM_ERR_NOMEM;
  } catch (const std::exception &e) {
    if (ctx) ctx->err = e.what();
    return IPM_ERR_ARG;
  }
}

template <typename T>
const T *upload(Carve &cv, const std::vector<T> &v, cudaStream_t st) {
  T *p = cv.take<T>(std::max<size_t>(v.size(), 1));
  if (cv.base && !v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

// Full symmetric W in CSR with the index of each entry's value in the caller's lower CSC.
void w_full(const Problem &P, std::vector<int64_t> &fp, std::vector<int32_t> &fi,
            std::vector<int64_t> &src) {
  const int32_t n = P.n;
  fp.assign(n + 1, 0);
  fi.clear();
  src.clear();
  if (P.wp.empty()) return;
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++) {
      fp[P.wi[e] + 1]++;
      if (P.wi[e] != j) fp[j + 1]++;
    }
  for (int32_t j = 0; j < n; j++) fp[j + 1] += fp[j];
  fi.resize(fp[n]);
  src.resize(fp[n]);
  std::vector<int64_t> f(fp.begin(), fp.end() - 1);
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++) {
      const int32_t i = P.wi[e];
      fi[f[i]] = j; src[f[i]++] = e;
      if (i != j) { fi[f[j]] = i; src[f[j]++] = e; }
    }
}

// Assign every device pointer of the context inside the workspace.
void layout(ipm_ctx *c, char *base) {
  Carve cv{base};
  const Plan &pl = c->plan;
  const Problem &P = c->P;
  const cudaStream_t st = c->st;
  DevPlan &d = c->dp;
  d.fronts = upload(cv, pl.fronts, st);
  d.children = upload(cv, pl.children, st);
  d.inv = upload(cv, pl.inv, st);
  d.relpos = upload(cv, pl.relpos, st);
  d.sri = upload(cv, c->S.sri, st);
  d.build = upload(cv, pl.build_tasks, st);
  d.gemm = upload(cv, pl.gemm_tasks, st);
  d.potrf = upload(cv, pl.potrf_tasks, st);
  d.trsm = upload(cv, pl.trsm_tasks, st);
  d.syrk = upload(cv, pl.syrk_tasks, st);
  d.gath = upload(cv, pl.gath_tasks, st);
  d.sdiag = upload(cv, pl.sdiag_tasks, st);
  d.sgemv = upload(cv, pl.sgemv_tasks, st);
  d.rgemv = upload(cv, pl.rgemv_tasks, st);
  d.toff = upload(cv, pl.toff, st);
  d.fs_inv = upload(cv, pl.fs_inv, st);
  d.fs_first_slot = upload(cv, pl.fs_first_slot, st);
  d.ps_tasks = upload(cv, pl.ps_tasks, st);
  d.ps_pbase = upload(cv, pl.ps_pbase, st);
  d.ps_kid_chunks = upload(cv, pl.ps_kid_chunks, st);
  d.ps_recs = upload(cv, pl.ps_recs, st);
  d.ps_parent_blocks = upload(cv, pl.ps_parent_blocks, st);
  d.fs_dinv_off = upload(cv, pl.fs_dinv_off, st);
  d.k_slot = upload(cv, pl.k_slot, st);
  d.k_poff = upload(cv, pl.k_poff, st);
  d.k_w = upload(cv, pl.k_w, st);
  d.k_orig = upload(cv, pl.k_orig, st);
  d.k_pa = upload(cv, pl.k_pa, st);
  d.k_pb = upload(cv, pl.k_pb, st);
  d.k_diag = upload(cv, pl.k_diag, st);
  d.perm = upload(cv, c->S.perm, st);
  d.jp = upload(cv, P.jp, st);
  d.jtp = upload(cv, P.jtp, st);
  d.ji = upload(cv, P.ji, st);
  d.jrow = upload(cv, P.jrow, st);
  d.jtpos = upload(cv, P.jtpos, st);
  {
    std::vector<int64_t> fp, src;
    std::vector<int32_t> fi;
    w_full(P, fp, fi, src);
    if (fp.empty()) fp.assign(P.n + 1, 0);
    d.wfp = upload(cv, fp, st);
    d.wfi = upload(cv, fi, st);
    d.wfsrc = upload(cv, src, st);
  }
  d.lpos = upload(cv, P.lpos, st);
  d.upos = upload(cv, P.upos, st);
  d.lidx = upload(cv, P.lidx, st);
  d.uidx = upload(cv, P.uidx, st);
  {
    std::vector<int32_t> col2s(P.n);
    for (int32_t s = 0; s < c->S.nsuper; s++)
      for (int32_t j = c->S.super[s]; j < c->S.super[s + 1]; j++) col2s[j] = s;
    c->col2s = const_cast<int32_t *>(upload(cv, col2s, st));
  }
  c->dl_ = const_cast<double *>(upload(cv, P.l, st));
  c->du_ = const_cast<double *>(upload(cv, P.u, st));
  if (!c->sign_orig.empty()) {  // pivot signs of a quasi-definite system, final numbering
    std::vector<int8_t> sg(P.n);
    for (int32_t k = 0; k < P.n; k++) sg[k] = c->sign_orig[c->S.perm[k]];
    d.sgn = upload(cv, sg, st);
  } else {
    d.sgn = nullptr;
  }
  if (c->form != IPM_FORM_PRIMAL) {  // inputs of the formulation's system
    const size_t nsys = c->form == IPM_FORM_DUAL ? (size_t)std::max<int32_t>(P.m, 1)
                                                 : (size_t)P.n + (size_t)P.m;
    c->wdiag = const_cast<int64_t *>(upload(cv, c->wdiag_h, st));
    c->aug_kind = const_cast<int32_t *>(upload(cv, c->aug_kind_h, st));
    c->aug_idx = const_cast<int64_t *>(upload(cv, c->aug_idx_h, st));
    c->hdiag = cv.take<double>(std::max<int32_t>(P.n, 1));
    c->rtil = cv.take<double>(std::max<int32_t>(P.n, 1));
    c->qv = cv.take<double>(std::max<int32_t>(P.m, 1));
    c->sysb = cv.take<double>(std::max<size_t>(nsys, 1));
    c->sysx = cv.take<double>(std::max<size_t>(nsys, 1));
    c->sysw = cv.take<double>(std::max<size_t>(c->form == IPM_FORM_DUAL ? (size_t)P.m
                                                                         : c->aug_kind_h.size(), 1));
    c->sysD = cv.take<double>(std::max<int32_t>(P.n, 1));
    c->sysj = cv.take<double>(std::max<int64_t>(P.jp.back(), 1));
  }
  c->tcp.layout(cv, st);
  if (c->oz_on) c->ozp.layout(cv, st, true);
  d.n = P.n;
  d.m = P.m;
  d.nl = P.nl;
  d.nu = P.nu;
  d.mt = P.mt;
  d.nk = (int64_t)pl.k_slot.size();
  const size_t n = std::max<int64_t>(P.n, 1), mt = std::max<int64_t>(P.mt, 1),
               m = std::max<int32_t>(P.m, 1);
  c->kval = cv.take<double>(std::max<int64_t>(d.nk, 1));
  c->yv = cv.take<double>(n);
  c->tv = cv.take<double>(pl.t_entries);
  for (double **v : {&c->vx, &c->vr, &c->vc, &c->vz, &c->vp, &c->vq, &c->vb, &c->vdx, &c->vrd,
                     &c->vwx})
    *v = cv.take<double>(n);
  for (double **v : {&c->vg, &c->vD, &c->vw, &c->vds, &c->vdl, &c->vt, &c->vjd})
    *v = cv.take<double>(mt);
  c->jv_copy = cv.take<double>(std::max<int64_t>(P.jp.back(), 1));
  c->D_copy = cv.take<double>(mt);
  c->wv_copy = cv.take<double>(std::max<int64_t>(P.wp.empty() ? 0 : P.wp.back(), 1));
  c->vjx = cv.take<double>(m);
  c->vtA = cv.take<double>(m);
  c->dinv = cv.take<float>(pl.fs_dinv_entries);
  c->fsa = cv.take<float>(n);
  c->fsb = cv.take<float>(n);
  c->fsx = cv.take<float>(n);
  c->psflags = cv.take<unsigned>(std::max<int64_t>(pl.ps_flag_words, 32));
  c->pspart = cv.take<float>(std::max<int64_t>(pl.ps_part_entries, 1));
  {  // learned-correction buffers (only when enabled)
    LearnedBufs &B = c->lb;
    const bool on = c->opts.learned != 0 || c->opts.learned_probes > 0;
    c->lb_on = on;
    B.n = P.n;
    B.mt = P.mt;
    B.P = std::min(8, std::max(1, c->opts.learned_probes));
    const size_t nn = on ? n : 1, mm = on ? mt : 1;
    B.w = cv.take<float>(kNParams);
    B.m = cv.take<float>(kNParams);
    B.v = cv.take<float>(kNParams);
    B.grad = cv.take<float>(kNParams);
    B.feat = cv.take<float>(nn * kNF);
    B.h1 = cv.take<float>(nn * kNH);
    B.h2 = cv.take<float>(nn * kNH);
    B.out = cv.take<float>(nn * kNO);
    B.gout = cv.take<float>(nn * (kNO + 2 * kNH));
    B.delta = cv.take<float>(nn);
    B.U = cv.take<float>(nn * kNR);
    B.diag_old = cv.take<double>(nn);
    B.diag_new = cv.take<double>(nn);
    B.D_old = cv.take<double>(mm);
    B.mu = cv.take<double>(2);
    B.partial = cv.take<float>((size_t)kLRedBlocks * kNParams);
    B.dpart = cv.take<double>((size_t)kLRedBlocks * 256);
    B.probe_t = cv.take<float>(8 * kNR);
    B.probe_q = cv.take<float>(8 * kNR);
    B.cap = cv.take<double>(kNR * kNR);
    B.ts = cv.take<float>(kNR);
    c->lb_loss = cv.take<double>(2);
  }
  c->scal = cv.take<double>(64);
  c->partial = cv.take<double>(kRedBlocks * 8);
  c->sc = cv.take<IpmScalars>(1);
  c->status = cv.take<int32_t>(ST_COUNT);
  c->L = cv.take<char>((size_t)pl.l_entries * c->storage_bytes);
  // low parts of the split-TF32 factor: the second half of an FP64-sized
  // buffer, else their own array
  c->Llo = c->storage_bytes == 8 ? (c->L ? reinterpret_cast<float *>(c->L) + pl.l_entries : nullptr)
                                 : cv.take<float>((size_t)pl.l_entries);
  c->U = cv.take<char>((size_t)pl.u_entries * c->storage_bytes);
  c->ws_need = cv.off + 256;
}

double d2h_scalar(ipm_ctx *c, const double *p) {
  double v = 0;
  CK(cudaMemcpyAsync(&v, p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return v;
}

// ---- factor ----------------------------------------------------------------
ipm_status do_factor(ipm_ctx *c, int prec, int32_t *bad_col) {
  if (c->state < 3) throw Fail{IPM_ERR_STATE, "kkt_factor before kkt_assemble"};
  if (prec < IPM_FP64 || prec > IPM_TF32X3) throw Fail{IPM_ERR_ARG, "unknown precision"};
  if (prec == IPM_FP64 && c->storage_bytes < 8)
    throw Fail{IPM_ERR_NOMEM, "factor storage sized for FP32; FP64 factor needs storage_fp64"};
  if (c->dp.sgn && prec != IPM_FP64 && prec != IPM_FP32)
    throw Fail{IPM_ERR_UNSUPPORTED, "the signed factorisation of a quasi-definite system runs in FP64 or FP32"};
  int32_t init[ST_COUNT] = {INT32_MAX, 0, 0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(c->status, init, sizeof(init), cudaMemcpyHostToDevice, c->st));
  if (prec == IPM_FP64 && c->opts.fp64_tc && !c->dp.sgn) {
    if (!c->ozp.ready())
      throw Fail{IPM_ERR_UNSUPPORTED,
                 "FP64 tensor-core factor not prepared (fp64_tc must be set before kkt_analyze)"};
    c->ozp.factor(c->dp, c->plan, c->kval, (double *)c->L, (double *)c->U, c->status, c->st);
  } else if (prec == IPM_FP64) {
    launch_factor_simt<double>(c->dp, c->plan, c->kval, (double *)c->L, (double *)c->U, c->status,
                               false, c->st);
  } else if (prec == IPM_FP32) {
    launch_factor_simt<float>(c->dp, c->plan, c->kval, (float *)c->L, (float *)c->U, c->status,
                              true, c->st);
  } else {
    if (!c->tcp.ready()) throw Fail{IPM_ERR_UNSUPPORTED, "tensor-core factor not prepared"};
    c->tcp.factor(c->dp, c->plan, c->kval, (float *)c->L, (float *)c->U, c->dinv, c->status,
                  prec == IPM_TF32X3 ? 3 : (prec == IPM_BF16 ? 16 : 1), c->st);
  }
  if (prec == IPM_FP32)  // explicit inverses of the diagonal blocks for the persistent solve
    launch_dinv(c->dp, c->plan, (const float *)c->L, c->dinv, c->st);  // (the TF32 paths write them)
  CK(cudaGetLastError());
  int32_t out[ST_COUNT];
  CK(cudaMemcpyAsync(out, c->status, sizeof(out), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (prec == IPM_FP64 && c->opts.fp64_tc && !c->dp.sgn && out[ST_FAIL_COL] != INT32_MAX &&
      !out[ST_TIMEOUT]) {
    // The slices keep each 128-column window to 56 bits of its largest entry:
    // where a row's entries span many decades within a window, a pivot that
    // cancels to a small positive value can come out non-positive. The FMA-pipe
    // FP64 factor of the same matrix decides before the caller regularises.
    CK(cudaMemcpyAsync(c->status, init, sizeof(init), cudaMemcpyHostToDevice, c->st));
    launch_factor_simt<double>(c->dp, c->plan, c->kval, (double *)c->L, (double *)c->U, c->status,
                               false, c->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, c->status, sizeof(out), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->oz_rechecks++;
  }
  c->last_perturbed = out[ST_PERTURBED];
  c->factor_prec = prec;
  c->have_stale = false;  // ipm_solve re-records what a new factor was computed from
  c->state = 4;
  if (out[ST_TIMEOUT]) {
    c->state = 3;
    throw Fail{IPM_ERR_TIMEOUT, "a bounded wait of the tensor-core factorisation ran out"};
  }
  if (bad_col) *bad_col = out[ST_FAIL_COL] == INT32_MAX ? -1 : out[ST_FAIL_COL];
  if (out[ST_FAIL_COL] != INT32_MAX) {
    c->err = "non-positive pivot at column " + std::to_string(out[ST_FAIL_COL]);
    return IPM_ERR_NOT_SPD;
  }
  return IPM_OK;
}

// One persistent FP32 solve launch over the workspace vectors: which = 0 both
// sweeps (fsa -> fsx), 1 forward only (fsa -> fsb), 2 backward only (fsb -> fsx)
void launch_fp32_solve(ipm_ctx *c, int which) {
  launch_psolve(c->dp, c->plan, (const float *)c->L, c->dinv, c->fsa, c->fsb, c->fsx,
                reinterpret_cast<float *>(c->tv), c->pspart, c->psflags, c->status, which != 2, which != 1,
                c->st, c->test_spins, c->test_withhold);
  c->test_spins = 0;
  c->test_withhold = -1;
}

// out = M^{-1} b with the current factor (b, out: original numbering, device)
void apply_factor(ipm_ctx *c, const double *b, double *out, bool accumulate) {
  VecOps V = c->vec();
  if (c->learned_active) {  // P^T L_s^{-T} (Delta + U U^T)^{-1} L_s^{-1} P b
    double *scale = c->scal + 8, *amax = c->scal + 9;
    V.absmax(c->P.n, b, amax);
    V.inv_scale(amax, scale);
    V.permute_in<float>(b, scale, c->fsa);
    launch_fp32_solve(c, 1);
    learned_apply(c->lb, c->fsb, c->st);
    launch_fp32_solve(c, 2);
    V.permute_out<float>(c->fsx, scale, out, accumulate);
    return;
  }
  if (c->storage_bytes == 8 && c->factor_prec == IPM_FP64) {
    V.permute_in<double>(b, nullptr, c->yv);
    launch_solve<double, double>(c->dp, c->plan, (const double *)c->L, c->yv, c->tv, c->st);
    V.permute_out<double>(c->yv, nullptr, out, accumulate);
  } else {
    double *scale = c->scal + 8, *amax = c->scal + 9;
    V.absmax(c->P.n, b, amax);
    V.inv_scale(amax, scale);
    V.permute_in<float>(b, scale, c->fsa);
    if (c->dp.sgn) {  // K = L S L^T: forward sweep, S, backward sweep
      launch_fp32_solve(c, 1);
      launch_sign<float>(c->dp, c->fsb, c->st);
      launch_fp32_solve(c, 2);
    } else {
      launch_fp32_solve(c, 0);
    }
    V.permute_out<float>(c->fsx, scale, out, accumulate);
  }
}

// A wait of the persistent solve that ran out of time: the launch drained and
// its result is invalid; clear the word (each launch zeroes its own flags) and
// report the timeout.
void check_solve_barrier(ipm_ctx *c) {
  int32_t flag = 0;
  CK(cudaMemcpyAsync(&flag, c->status + ST_SOLVE_TIMEOUT, sizeof(flag), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (flag) {
    CK(cudaMemsetAsync(c->status + ST_SOLVE_TIMEOUT, 0, sizeof(int32_t), c->st));
    throw Fail{IPM_ERR_TIMEOUT, "a bounded wait of the persistent solve ran out of time"};
  }
}

// ---- solve with refinement / PCG ----------------------------------------------
ipm_status do_solve(ipm_ctx *c, const double *b, double *x, int refine, ipm_solve_info *info) {
  if (c->state < 4) throw Fail{IPM_ERR_STATE, "kkt_solve before kkt_factor"};
  VecOps V = c->vec();
  const int64_t n = c->P.n;
  const ipm_options &o = c->opts;
  double *bb = c->vb, *r = c->vr, *z = c->vz, *p = c->vp, *q = c->vq, *xx = c->vx;
  CK(cudaMemcpyAsync(bb, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  double *sN = c->scal;  // scalars: 0 |b|, 1 |r|, 2 rz, 3 pq, 4 rz_new
  const int pcg_max = c->pcg_override >= 0 ? c->pcg_override : o.pcg_max;
  V.absmax(n, bb, sN + 0);
  const double bn = d2h_scalar(c, sN + 0);
  if (info) *info = ipm_solve_info{0, 0, 0.0};
  if (bn == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->st));
    c->last_rel = 0.0;
    return IPM_OK;
  }
  // ||b - K x|| / ||b|| drives refinement. For a badly scaled matrix (the grid
  // NLP: entries up to (nx+1)^4 times D) its floor is about eps ||K|| ||x|| / ||b||,
  // so with bwd_measure the solve is accepted on the normwise backward error
  // ||b - K x|| / (||K|| ||x|| + ||b||) instead (refinement still runs until it stalls).
  double bwd = 0.0;
  auto residual = [&](const double *xv) {
    V.residual(c->cur_jvals, c->cur_D, c->cur_wvals, c->cur_delta_p, xv, bb, r, c->vtA);
    V.absmax(n, r, sN + 1);
    if (!c->bwd_measure) return d2h_scalar(c, sN + 1) / bn;
    V.absmax(n, xv, sN + 5);
    double h2[5];
    CK(cudaMemcpyAsync(h2, sN + 1, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    bwd = h2[0] / (c->knorm * h2[4] + bn);
    return h2[0] / bn;
  };
  double rel;
  if (c->warm_x) {  // x holds a nearby solution (the predictor's direction)
    CK(cudaMemcpyAsync(xx, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    residual(xx);
    apply_factor(c, r, xx, true);
  } else {
    apply_factor(c, bb, xx, false);
  }
  rel = residual(xx);
  int iters = 0, used_pcg = 0;
  if (refine != IPM_REFINE_NONE && refine != IPM_REFINE_PCG) {
    double prev = rel;
    int slow = 0;
    while (rel > o.ir_tol && iters < o.ir_max) {
      apply_factor(c, r, xx, true);
      iters++;
      rel = residual(xx);
      if (!(rel < 0.5 * prev)) slow++;
      else slow = 0;
      prev = std::min(prev, rel);
      if (slow >= 2 || !std::isfinite(rel)) break;
    }
    c->refine_steps += iters;
  }
  if ((refine == IPM_REFINE_PCG || refine == IPM_REFINE_IR) && (rel > o.ir_tol || !std::isfinite(rel)) &&
      !(c->bwd_measure && bwd <= o.ir_tol && std::isfinite(rel))) {
    // PCG on K x = b preconditioned by the factor, from the current x
    if (!std::isfinite(rel)) {
      CK(cudaMemsetAsync(xx, 0, n * sizeof(double), c->st));
      rel = residual(xx);
    }
    used_pcg = 1;
    CK(cudaMemsetAsync(c->vc, 0, n * sizeof(double), c->st));  // zero right-hand side for q = K p
    apply_factor(c, r, z, false);
    CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    V.dot(n, r, z, sN + 2);
    const double rel0 = rel;
    int k = 0;
    for (; k < pcg_max && rel > o.ir_tol; k++) {
      // q = K p  (residual of b = 0 gives -K p)
      V.residual(c->cur_jvals, c->cur_D, c->cur_wvals, c->cur_delta_p, p, c->vc, q, c->vtA);
      V.negate(n, q);
      V.dot(n, p, q, sN + 3);
      V.axpy_ratio(n, sN + 2, sN + 3, +1, p, xx);
      V.axpy_ratio(n, sN + 2, sN + 3, -1, q, r);
      V.absmax(n, r, sN + 1);
      rel = d2h_scalar(c, sN + 1) / bn;
      if (rel <= o.ir_tol || !std::isfinite(rel)) { k++; break; }
      // a corrected stale factor is only worth keeping if PCG converges
      // within the budget: from the fifth iteration on, give up once the mean
      // contraction so far projects past pcg_max
      if (c->learned_active && k + 1 >= 5) {
        if (!(rel < rel0)) { k++; break; }
        const double rate = std::log(rel / rel0) / (k + 1);  // < 0
        const double need = (k + 1) + std::log(o.ir_tol / rel) / rate;
        if (need > pcg_max) { k++; break; }
      }
      apply_factor(c, r, z, false);
      V.dot(n, r, z, sN + 4);
      V.xpby_ratio(n, sN + 4, sN + 2, z, p);
      CK(cudaMemcpyAsync(sN + 2, sN + 4, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    }
    c->pcg_steps += k;
    iters += k;
    rel = residual(xx);  // true residual of the returned iterate
  }
  CK(cudaMemcpyAsync(x, xx, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaGetLastError());
  if (c->factor_prec != IPM_FP64) check_solve_barrier(c);
  if (c->bwd_measure) rel = bwd;
  c->last_rel = rel;
  if (info) *info = ipm_solve_info{iters, used_pcg, rel};
  if (!(rel <= o.accept_tol)) {
    c->err = "linear solve residual " + std::to_string(rel) + " above accept_tol";
    return IPM_ERR_NUMERIC;
  }
  return IPM_OK;
}

void set_assembly(ipm_ctx *c, const double *wv, const double *jv, const double *D, double dp) {
  c->cur_jvals = jv;
  c->cur_D = D;
  c->cur_wvals = wv;
  c->cur_delta_p = dp;
  launch_assemble(c->dp, jv, D, wv, dp, c->kval, c->st);
  CK(cudaGetLastError());
  if (c->bwd_measure) {  // ||K||_inf for the backward error of the solves
    VecOps V = c->vec();
    V.abs_rowsum(jv, D, wv, dp, c->vz, c->vtA);
    V.absmax(c->P.n, c->vz, c->scal + 7);
    c->knorm = d2h_scalar(c, c->scal + 7);
  }
  if (c->state < 3) c->state = 3;
}

// ---- formulations (4) and (6) ------------------------------------------------
// The formulation's matrix from W, J, D and delta_p (device pointers that stay
// valid while the system is in use): H, then the system's own inputs, then the
// system context's assembly.
void form_assemble(ipm_ctx *c, const double *wv, const double *jv, const double *D, double dp) {
  FormOps F{c->dp, c->st};
  F.hdiag(wv, c->wdiag, D, dp, c->hdiag);
  ipm_status st;
  if (c->form == IPM_FORM_DUAL) {
    F.dual_values((int64_t)c->P.ji.size(), jv, D, c->hdiag, c->sysD, c->sysj, c->sysw);
    st = kkt_assemble(c->sys, c->sysw, c->sysj, c->sysD, 0.0);
  } else {
    F.aug_values((int64_t)c->aug_kind_h.size(), c->aug_kind, c->aug_idx, c->hdiag, wv, jv, D,
                 c->sysw);
    st = kkt_assemble(c->sys, c->sysw, nullptr, nullptr, 0.0);
  }
  if (st != IPM_OK) throw Fail{st, c->sys->err};
  c->cur_jvals = jv;
  c->cur_D = D;
  c->cur_wvals = wv;
  c->cur_delta_p = dp;
  if (c->state < 3) c->state = 3;
}

void assemble_any(ipm_ctx *c, const double *wv, const double *jv, const double *D, double dp) {
  if (c->sys) form_assemble(c, wv, jv, D, dp);
  else set_assembly(c, wv, jv, D, dp);
}

// Factor the context's system (the formulation's, if any).
ipm_status factor_any(ipm_ctx *c, int prec, int32_t *bad) {
  if (!c->sys) return do_factor(c, prec, bad);
  if (c->state < 3) throw Fail{IPM_ERR_STATE, "kkt_factor before kkt_assemble"};
  const ipm_status st = do_factor(c->sys, prec, bad);
  c->factor_prec = prec;
  c->last_perturbed = c->sys->last_perturbed;
  c->state = c->sys->state;
  if (st != IPM_OK) c->err = c->sys->err;
  return st;
}

// Newton direction through (6) or (4) (see forms.h), then rows 2-3 of (3).
ipm_status form_direction(ipm_ctx *c, const double *jvals, const double *cc, const double *wvals,
                          const double *x, const double *s, const double *lam, const double *w,
                          double *dx, double *ds, double *dl, ipm_solve_info *si) {
  VecOps V = c->vec();
  FormOps F{c->dp, c->st};
  const int64_t n = c->P.n, m = c->P.m;
  F.rhs_rows(c->vD, c->vg, w, lam, c->vt, c->qv);
  V.jtv(jvals, c->vt, 1.0, wvals, x, cc, c->rtil);  // r~ = c + W x + J^T t
  int refine = c->refine_override >= 0 ? c->refine_override : c->opts.refine;
  ipm_status stt;
  if (c->form == IPM_FORM_DUAL) {
    F.div(c->rtil, c->hdiag, 1.0, c->vz);  // u = H^{-1} r~
    V.jv(jvals, c->vz, c->vjx);            // A u
    F.sub(m, c->qv, c->vjx, c->sysb);      // q - A u
    stt = do_solve(c->sys, c->sysb, c->sysx, refine, si);
    F.pad_rows(c->sysx, c->vt);            // [y; 0]
    V.jtv(jvals, c->vt, 1.0, nullptr, nullptr, c->rtil, c->vrd);  // r~ + A^T y
    F.div(c->vrd, c->hdiag, -1.0, dx);
    // Recovering d_x through H^{-1} amplifies the reduced solve's error where
    // H is near delta_p (H^{-1} up to 1 / delta_p), so (d_x, y) is refined on
    // the augmented system (4), FP64 residuals, with the factor of (6):
    //   K6 dy = A H^{-1} r1 - r2,  dx = H^{-1} (r1 - A^T dy).
    double *sN = c->scal + 56;  // scalars: |r1|, |r2|, |r~|, |q|
    V.absmax(n, c->rtil, sN + 2);
    V.absmax(m, c->qv, sN + 3);
    for (int r = 0; r < 3 && stt == IPM_OK; r++) {
      F.pad_rows(c->sysx, c->vt);
      V.jtv(jvals, c->vt, 1.0, nullptr, nullptr, nullptr, c->vp);  // A^T y
      F.aug_res_n(c->rtil, c->hdiag, dx, c->vp, c->vc);            // r1
      V.jv(jvals, dx, c->vjx);                                     // A d_x
      F.aug_res_m(c->qv, c->vjx, c->vD, c->sysx, c->vtA);          // r2
      V.absmax(n, c->vc, sN + 0);
      V.absmax(m, c->vtA, sN + 1);
      double h4[4];
      CK(cudaMemcpyAsync(h4, sN, sizeof(h4), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (!(std::max(h4[0], h4[1]) > c->opts.ir_tol * std::max(h4[2], h4[3]))) break;
      F.div(c->vc, c->hdiag, 1.0, c->vz);                 // H^{-1} r1
      V.jv(jvals, c->vz, c->vjx);                         // A H^{-1} r1
      F.lincomb(m, 1.0, c->vjx, -1.0, c->vtA, c->sysb);   // - r2
      ipm_solve_info s2{};
      stt = do_solve(c->sys, c->sysb, c->sysb, refine, &s2);  // dy (in place)
      F.pad_rows(c->sysb, c->vt);
      V.jtv(jvals, c->vt, -1.0, nullptr, nullptr, c->vc, c->vp);  // r1 - A^T dy
      F.div(c->vp, c->hdiag, 1.0, c->vz);                         // dx correction
      F.lincomb(n, 1.0, dx, 1.0, c->vz, dx);
      F.lincomb(m, 1.0, c->sysx, 1.0, c->sysb, c->sysx);
      c->refine_steps++;
    }
  } else {
    if (refine == IPM_REFINE_PCG) refine = IPM_REFINE_IR;  // indefinite: no conjugate gradients
    F.neg_concat(c->rtil, n, c->qv, m, c->sysb);  // -[r~; q]
    stt = do_solve(c->sys, c->sysb, c->sysx, refine, si);
    CK(cudaMemcpyAsync(dx, c->sysx, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  }
  c->last_rel = c->sys->last_rel;
  V.jv(jvals, dx, c->vjx);
  V.jfull(c->vjx, dx, c->vjd);
  V.recover(c->vD, c->vg, w, s, lam, c->vjd, ds, dl);
  return stt;
}

// Newton direction at (x, s, lambda) with target w (w == nullptr: zero), reusing
// the factor held by the context (assembled with D = (delta_d + s/lambda)^{-1}).
ipm_status direction(ipm_ctx *c, const double *jvals, const double *b, const double *cc,
                     const double *wvals, const double *x, const double *s, const double *lam,
                     const double *w, double *dx, double *ds, double *dl, ipm_solve_info *si) {
  if (c->sys) return form_direction(c, jvals, cc, wvals, x, s, lam, w, dx, ds, dl, si);
  VecOps V = c->vec();
  V.rhs_rows(c->vD, c->vg, w, lam, c->vt);
  // r_p = c + W x + J^T (D (g - w/lam) - lam); for the NLP, cc is grad f itself
  V.jtv(jvals, c->vt, 1.0, wvals, c->nlp_grad ? nullptr : x, cc, c->vrd);
  V.negate(c->P.n, c->vrd);
  ipm_status stt = do_solve(c, c->vrd, dx,
                            c->refine_override >= 0 ? c->refine_override : c->opts.refine, si);
  V.jv(jvals, dx, c->vjx);
  V.jfull(c->vjx, dx, c->vjd);
  V.recover(c->vD, c->vg, w, s, lam, c->vjd, ds, dl);
  (void)b;
  return stt;
}

void eval_g(ipm_ctx *c, const double *jvals, const double *b, const double *x) {
  VecOps V = c->vec();
  V.jv(jvals, x, c->vjx);
  V.g(c->vjx, x, b, c->dl_, c->du_, c->vg);
}

// Factor with the regularisation raised after a non-positive pivot (inertia
// correction reduced to "Cholesky succeeds" for the SPD condensed system), at
// most max_tries times.
ipm_status factor_with_retry(ipm_ctx *c, const double *wvals, const double *jvals, int prec,
                             double &delta_p, ipm_result *res, int max_tries = 12) {
  for (int tries = 0;; tries++) {
    assemble_any(c, wvals, jvals, c->vD, delta_p);
    int32_t bad = -1;
    ipm_ctx *fc = c->sys ? c->sys : c;  // the context that factors
    const int64_t rechecks = fc->oz_rechecks;
    ipm_status stt = factor_any(c, prec, &bad);
    if (res) {
      res->factorizations++;
      res->perturbed_pivots += c->last_perturbed;
      res->fp64_tc_rechecks += (int32_t)(fc->oz_rechecks - rechecks);
    }
    if (stt == IPM_OK) return IPM_OK;
    if (stt != IPM_ERR_NOT_SPD || tries >= max_tries) return stt;
    delta_p = delta_p > 0 ? delta_p * 100.0 : 1e-8;
    if (res) res->regularizations++;
  }
}

// After a fresh factorisation: remember what it was computed from (features of
// later iterations compare against it).
void save_stale(ipm_ctx *c, const double *jv) {
  LearnedBufs &B = c->lb;
  if (!c->lb_on || !(c->opts.learned != 0 || c->opts.learned_probes > 0)) return;
  CK(cudaMemcpyAsync(B.D_old, c->cur_D, c->P.mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  learned_diag(c->dp, jv, c->cur_D, c->cur_delta_p, B.diag_old, c->st);
  CK(cudaMemcpyAsync(B.mu, &c->sc->mu, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  c->have_stale = true;
}

// Features of the current D against the held factor, network forward (or the
// E = 0 ablation) and the Woodbury capacitance.
void learned_prepare(ipm_ctx *c, const double *jv, const double *x, double delta_p, bool ablate) {
  LearnedBufs &B = c->lb;
  CK(cudaMemcpyAsync(B.mu + 1, &c->sc->mu, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  learned_diag(c->dp, jv, c->vD, delta_p, B.diag_new, c->st);
  learned_features(c->dp, B, jv, c->vD, x, c->st);
  learned_forward(B, ablate, c->st);
  learned_capacitance(B, c->st);
}

// Deterministic initial weights: uniform Glorot ranges for the hidden layers
// (SplitMix64 stream), zero output layer, so the untrained network is the
// E = 0 correction (Delta = 1, U = 0).
void learned_init_weights(ipm_ctx *c) {
  std::vector<float> w(kNParams, 0.f);
  uint64_t st = 0x9E3779B97F4A7C15ull * 77u;
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  const float a1 = std::sqrt(6.f / (kNF + kNH)), a2 = std::sqrt(6.f / (kNH + kNH));
  for (int p = kW1; p < kB1; p++) w[p] = (float)((2 * next() - 1) * a1);
  for (int p = kW2; p < kB2; p++) w[p] = (float)((2 * next() - 1) * a2);
  CK(cudaMemcpyAsync(c->lb.w, w.data(), kNParams * sizeof(float), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->lb.m, 0, kNParams * sizeof(float), c->st));
  CK(cudaMemsetAsync(c->lb.v, 0, kNParams * sizeof(float), c->st));
  CK(cudaStreamSynchronize(c->st));
  c->lb.step = 0;
}

// Device address of the allocation-free solve's static array on `dev`, looked
// up (and the array committed) on the first call for that device.
double *noalloc_scratch(int dev);

// Symbolic analysis for the formulations (6) and (4): the pattern of the
// system's matrix, a context `sys` that analyses and later factors it, and
// this context's own (small) layout of interior-point vectors.
//  (6): order m, sys's Jacobian J' = A^T (rows = variables, CSR of A^T), its
//       W' = diag(D_G^{-1}) and its D' = 1 / H: K' = W' + J'^T D' J'.
//  (4): order n + m, no Jacobian, sys's W' = the lower triangle of
//       [H, A^T; A, -D_G^{-1}] (columns j < n: W's rows with the diagonal,
//       then n + i for A_ij != 0; column n + i: its diagonal), pivot signs +1
//       on the first n and -1 on the last m variables.
ipm_status analyze_form(ipm_ctx *c, const int32_t *perm, ipm_symbolic_info *info) {
  const Problem &P = c->P;
  const int32_t n = P.n, m = P.m;
  const int64_t nnz = (int64_t)P.ji.size();
  if (c->opts.learned != 0 || c->opts.learned_probes > 0)
    throw Fail{IPM_ERR_UNSUPPORTED, "the learned correction uses the primal condensed formulation"};
  if (c->form == IPM_FORM_DUAL && m == 0)
    throw Fail{IPM_ERR_ARG, "the dual condensed formulation needs general rows (m >= 1)"};
  c->wdiag_h.assign(n, -1);
  if (!P.wp.empty())
    for (int32_t j = 0; j < n; j++)
      for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++) {
        if (P.wi[e] == j) c->wdiag_h[j] = e;
        else if (c->form == IPM_FORM_DUAL)
          throw Fail{IPM_ERR_UNSUPPORTED, "the dual condensed formulation needs a diagonal W"};
      }
  std::vector<int64_t> sp(1, 0), swp;
  std::vector<int32_t> si, swi;
  int32_t ns, ms;
  c->aug_kind_h.clear();
  c->aug_idx_h.clear();
  if (c->form == IPM_FORM_DUAL) {
    ns = m;
    ms = n;
    sp = P.jtp;
    si.resize(nnz);
    for (int64_t e = 0; e < nnz; e++) si[e] = P.jrow[P.jtpos[e]];
    swp.resize((size_t)m + 1);
    swi.resize(m);
    for (int32_t i = 0; i <= m; i++) swp[i] = i;
    for (int32_t i = 0; i < m; i++) swi[i] = i;
  } else {
    ns = n + m;
    ms = 0;
    swp.assign((size_t)ns + 1, 0);
    for (int32_t j = 0; j < n; j++) {
      c->aug_kind_h.push_back(AUG_HDIAG);  // the diagonal first (W's rows are >= j)
      c->aug_idx_h.push_back(j);
      swi.push_back(j);
      if (!P.wp.empty())
        for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++)
          if (P.wi[e] != j) {
            c->aug_kind_h.push_back(AUG_W);
            c->aug_idx_h.push_back(e);
            swi.push_back(P.wi[e]);
          }
      for (int64_t t = P.jtp[j]; t < P.jtp[j + 1]; t++) {  // rows of J in ascending order
        c->aug_kind_h.push_back(AUG_J);
        c->aug_idx_h.push_back(P.jtpos[t]);
        swi.push_back(n + P.jrow[P.jtpos[t]]);
      }
      swp[j + 1] = (int64_t)swi.size();
    }
    for (int32_t i = 0; i < m; i++) {
      c->aug_kind_h.push_back(AUG_DINV);
      c->aug_idx_h.push_back(i);
      swi.push_back(n + i);
      swp[(size_t)n + i + 1] = (int64_t)swi.size();
    }
    // W's rows of a column must ascend (checked again by ipm_create)
    for (int32_t j = 0; j < n; j++)
      for (int64_t e = swp[j] + 1; e < swp[j + 1]; e++)
        if (swi[e] <= swi[e - 1]) throw Fail{IPM_ERR_ARG, "W rows must be ascending within a column"};
  }
  ipm_options so = c->opts;
  so.formulation = IPM_FORM_PRIMAL;
  so.learned = 0;
  so.learned_probes = 0;
  if (c->form == IPM_FORM_AUGMENTED && so.refine == IPM_REFINE_PCG) so.refine = IPM_REFINE_IR;
  ipm_ctx *sys = nullptr;
  ipm_status st = ipm_create(ns, ms, sp.data(), si.empty() ? nullptr : si.data(), swp.data(),
                             swi.empty() ? nullptr : swi.data(), nullptr, nullptr, &so, c->st, &sys);
  if (st != IPM_OK) throw Fail{st, "system context of the formulation"};
  delete c->sys;
  c->sys = sys;
  if (c->form == IPM_FORM_AUGMENTED) {
    sys->sign_orig.assign((size_t)ns, 1);
    for (int32_t i = 0; i < m; i++) sys->sign_orig[(size_t)n + i] = -1;
  }
  st = kkt_analyze(sys, perm, info);
  if (st != IPM_OK) throw Fail{st, sys->err};
  c->S = Symbolic{};  // this context factors nothing itself
  c->plan = Plan{};
  c->storage_bytes = sys->storage_bytes;
  layout(c, nullptr);
  c->outer_need = c->ws_need;
  c->ws_need = ((c->outer_need + 255) & ~size_t(255)) + sys->ws_need + 256;
  c->state = 1;
  if (info) {
    info->m_tot = P.mt;
    info->workspace_bytes = (int64_t)c->ws_need;
  }
  return IPM_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

void ipm_default_options(ipm_options *o) {
  if (!o) return;
  o->max_iter = 500;
  o->tol = 1e-8;
  o->delta_p = 1e-8;
  o->delta_d = 1e-8;
  o->precision = IPM_FP64;
  o->storage_fp64 = -1;
  o->refine = IPM_REFINE_PCG;
  o->ir_max = 10;
  o->ir_tol = 1e-10;
  o->pcg_max = 100;
  o->fallback_fp64 = 0;
  o->accept_tol = 1e-6;
  o->verbose = 0;
  o->warm_start = 0;
  o->learned = 0;
  o->learned_probes = 0;
  o->learned_pcg_max = 30;
  o->formulation = IPM_FORM_PRIMAL;
  o->cg_escalate = 0;
  o->fp64_tc = 0;
}

ipm_status ipm_create_pattern(int32_t n, int32_t m, const ipm_pattern *p, const ipm_options *opts,
                              void *stream, ipm_ctx **out) {
  if (!p) return IPM_ERR_ARG;
  return ipm_create(n, m, p->j_rowptr, p->j_col, p->w_colptr, p->w_row, p->l, p->u, opts, stream, out);
}

ipm_status ipm_create(int32_t n, int32_t m, const int64_t *jp, const int32_t *ji,
                      const int64_t *wp, const int32_t *wi, const double *l, const double *u,
                      const ipm_options *opts, void *stream, ipm_ctx **out) {
  if (!out || n < 0 || m < 0 || (m > 0 && (!jp || !ji)) || ((wp == nullptr) != (wi == nullptr)))
    return IPM_ERR_ARG;
  *out = nullptr;
  ipm_ctx *c = new (std::nothrow) ipm_ctx();
  if (!c) return IPM_ERR_NOMEM;
  ipm_status st = guarded(c, [&]() -> ipm_status {
    if (opts) c->opts = *opts;
    else ipm_default_options(&c->opts);
    c->st = (cudaStream_t)stream;
    Problem &P = c->P;
    P.n = n;
    P.m = m;
    P.jp.assign(jp ? jp : nullptr, jp ? jp + m + 1 : nullptr);
    if (m == 0) P.jp.assign(1, 0);
    if (P.jp[0] != 0) throw Fail{IPM_ERR_ARG, "J row pointer must start at 0"};
    const int64_t nnz = P.jp[m];
    P.ji.assign(ji ? ji : nullptr, ji ? ji + nnz : nullptr);
    P.jrow.resize(nnz);
    for (int32_t r = 0; r < m; r++) {
      if (P.jp[r + 1] < P.jp[r]) throw Fail{IPM_ERR_ARG, "J row pointer not monotone"};
      for (int64_t e = P.jp[r]; e < P.jp[r + 1]; e++) {
        if (P.ji[e] < 0 || P.ji[e] >= n) throw Fail{IPM_ERR_ARG, "J column index out of range"};
        if (e > P.jp[r] && P.ji[e] <= P.ji[e - 1])
          throw Fail{IPM_ERR_ARG, "J columns must be strictly ascending within a row"};
        P.jrow[e] = r;
      }
    }
    P.jtp.assign(n + 1, 0);
    for (int64_t e = 0; e < nnz; e++) P.jtp[P.ji[e] + 1]++;
    for (int32_t j = 0; j < n; j++) P.jtp[j + 1] += P.jtp[j];
    P.jtpos.resize(nnz);
    {
      std::vector<int64_t> f(P.jtp.begin(), P.jtp.end() - 1);
      for (int64_t e = 0; e < nnz; e++) P.jtpos[f[P.ji[e]]++] = (int32_t)e;
    }
    if (wp) {
      P.wp.assign(wp, wp + n + 1);
      P.wi.assign(wi, wi + wp[n]);
      for (int32_t j = 0; j < n; j++)
        for (int64_t e = wp[j]; e < wp[j + 1]; e++)
          if (wi[e] < j || wi[e] >= n) throw Fail{IPM_ERR_ARG, "W must be lower CSC"};
    }
    P.l.assign(n, -INFINITY);
    P.u.assign(n, INFINITY);
    if (l) P.l.assign(l, l + n);
    if (u) P.u.assign(u, u + n);
    P.lpos.assign(n, -1);
    P.upos.assign(n, -1);
    P.lidx.clear();
    P.uidx.clear();
    for (int32_t i = 0; i < n; i++) if (std::isfinite(P.l[i])) P.lidx.push_back(i);
    for (int32_t i = 0; i < n; i++) if (std::isfinite(P.u[i])) P.uidx.push_back(i);
    P.nl = (int32_t)P.lidx.size();
    P.nu = (int32_t)P.uidx.size();
    P.mt = (int64_t)m + P.nl + P.nu;
    for (int32_t k = 0; k < P.nl; k++) P.lpos[P.lidx[k]] = m + k;
    for (int32_t k = 0; k < P.nu; k++) P.upos[P.uidx[k]] = m + P.nl + k;
    c->state = 0;
    return IPM_OK;
  });
  if (st != IPM_OK) {
    delete c;
    return st;
  }
  *out = c;
  return IPM_OK;
}

ipm_status ipm_set_options(ipm_ctx *c, const ipm_options *o) {
  if (!c || !o) return IPM_ERR_ARG;
  // the learned buffers are sized when the workspace is laid out: they cannot
  // be switched on afterwards
  if (c->state >= 1 && !c->lb_on && (o->learned != 0 || o->learned_probes > 0)) {
    c->err = "learned options must be set before kkt_analyze";
    return IPM_ERR_STATE;
  }
  c->opts = *o;
  return IPM_OK;
}

ipm_status kkt_analyze(ipm_ctx *c, const int32_t *perm, ipm_symbolic_info *info) {
  if (!c) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    const int32_t n = c->P.n;
    c->form = c->opts.formulation;
    if (c->form < IPM_FORM_PRIMAL || c->form > IPM_FORM_AUGMENTED)
      throw Fail{IPM_ERR_ARG, "unknown formulation"};
    c->oz_on = false;
    if (c->form != IPM_FORM_PRIMAL) return analyze_form(c, perm, info);
    delete c->sys;
    c->sys = nullptr;
    if (perm) {
      std::vector<char> seen(n, 0);
      for (int32_t k = 0; k < n; k++) {
        if (perm[k] < 0 || perm[k] >= n || seen[perm[k]]) throw Fail{IPM_ERR_ARG, "perm is not a permutation"};
        seen[perm[k]] = 1;
      }
    }
    analyze_symbolic(c->P, perm, c->S);
    build_plan(c->P, c->S, c->plan, 64, 64);
    validate_plan(c->P, c->S, c->plan);
    build_fused_solve(c->plan);
    c->tcp.build(c->plan);
    c->oz_on = c->opts.fp64_tc != 0 && c->sign_orig.empty();
    if (c->oz_on) c->ozp.build(c->plan);
    const int so = c->opts.storage_fp64;
    c->storage_bytes = (so == 1 || c->oz_on ||
                        (so < 0 && (c->opts.precision == IPM_FP64 || c->opts.fallback_fp64))) ? 8 : 4;
    layout(c, nullptr);
    c->state = 1;
    if (info) {
      info->n = n;
      info->m_tot = c->P.mt;
      info->nnz_k = (int64_t)c->S.koi.size();
      info->nnz_l = c->S.nnz_l;
      info->nsuper = c->S.nsuper;
      info->nlevels = c->S.nlevels;
      info->max_front = c->plan.max_front;
      info->max_ncol = c->plan.max_ncol;
      info->flops = c->S.flops;
      info->factor_entries = c->plan.l_entries;
      info->update_entries = c->plan.u_entries;
      info->workspace_bytes = (int64_t)c->ws_need;
    }
    return IPM_OK;
  });
}

ipm_status ipm_set_workspace(ipm_ctx *c, void *buf, size_t bytes) {
  if (!c || !buf) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 1) throw Fail{IPM_ERR_STATE, "ipm_set_workspace before kkt_analyze"};
    if (bytes < c->ws_need)
      throw Fail{IPM_ERR_NOMEM, "workspace of " + std::to_string(bytes) + " bytes, need " +
                                    std::to_string(c->ws_need)};
    char *base = (char *)(((uintptr_t)buf + 255) & ~uintptr_t(255));
    if ((size_t)(base - (char *)buf) + c->ws_need - 256 > bytes) throw Fail{IPM_ERR_NOMEM, "workspace misaligned"};
    c->ws = base;
    c->ws_bytes = bytes;
    CK(cudaGetDevice(&c->device));
    const size_t total = c->ws_need;
    layout(c, base);
    CK(cudaStreamSynchronize(c->st));
    if (c->sys) {  // the formulation's system takes the rest of the buffer
      c->ws_need = total;
      char *sub = base + ((c->outer_need + 255) & ~size_t(255));
      const ipm_status st = ipm_set_workspace(c->sys, sub, bytes - (size_t)(sub - (char *)buf));
      if (st != IPM_OK) throw Fail{st, c->sys->err};
    }
    // Commit the allocation-free solve's static array on this device now,
    // while the caller is handing over memory anyway: a later
    // kkt_solve_noalloc then loads no module and commits nothing.
    noalloc_scratch(c->device);
    CK(preload_level_solve());
    CK(preload_vec_kernels());
    c->have_stale = false;
    if (c->lb_on) learned_init_weights(c);
    try {  // tensor maps of the FP32 panels for the tensor-core path
      if (!c->sys) c->tcp.encode(c->plan, (float *)c->L, c->Llo, (float *)c->U, c->st);
    } catch (const std::exception &e) {
      c->err = std::string("tensor-core path unavailable: ") + e.what();
    }
    try {  // tensor maps of the slice planes of the FP64 tensor-core factor
      if (c->oz_on) c->ozp.encode(c->plan, c->st);
    } catch (const std::exception &e) {
      c->err = std::string("FP64 tensor-core path unavailable: ") + e.what();
    }
    c->state = 2;
    return IPM_OK;
  });
}

ipm_status kkt_assemble(ipm_ctx *c, const double *wv, const double *jv, const double *D,
                        double delta_p) {
  if (!c) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 2) throw Fail{IPM_ERR_STATE, "kkt_assemble before ipm_set_workspace"};
    if ((!jv && c->P.jp.back() > 0) || (!D && c->P.mt > 0)) throw Fail{IPM_ERR_ARG, "null values"};
    // keep copies: refinement in kkt_solve evaluates K x from J, D and W
    const int64_t nj = c->P.jp.back(), nw = c->P.wp.empty() ? 0 : c->P.wp.back();
    if (nj > 0) CK(cudaMemcpyAsync(c->jv_copy, jv, nj * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (c->P.mt > 0) CK(cudaMemcpyAsync(c->D_copy, D, c->P.mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (wv && nw > 0) CK(cudaMemcpyAsync(c->wv_copy, wv, nw * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    assemble_any(c, wv ? c->wv_copy : nullptr, c->jv_copy, c->D_copy, delta_p);
    c->state = 3;
    return IPM_OK;
  });
}

ipm_status kkt_factor(ipm_ctx *c, int32_t precision, int32_t *bad_col) {
  if (!c) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status { return factor_any(c, precision, bad_col); });
}

ipm_status kkt_solve(ipm_ctx *c, const double *b, double *x, int32_t nrhs, int32_t refine,
                     ipm_solve_info *info) {
  if (!c || !b || !x || nrhs < 1) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    // right-hand side k occupies b[k n .. (k+1) n); each is solved (and
    // refined) on its own, the info reports the totals and the worst residual
    // (with a formulation (4) or (6), n is the order of its system)
    ipm_ctx *t = c->sys ? c->sys : c;
    if (c->sys && c->state < 4) throw Fail{IPM_ERR_STATE, "kkt_solve before kkt_factor"};
    const int64_t n = t->P.n;
    ipm_solve_info all{0, 0, 0.0};
    ipm_status worst = IPM_OK;
    for (int32_t k = 0; k < nrhs; k++) {
      ipm_solve_info one{};
      const ipm_status st = do_solve(t, b + k * n, x + k * n, refine, &one);
      if (st != IPM_OK && t != c) c->err = t->err;
      all.iterations += one.iterations;
      all.used_pcg = std::max(all.used_pcg, one.used_pcg);
      all.rel_residual = std::max(all.rel_residual, one.rel_residual);
      if (st != IPM_OK && worst == IPM_OK) worst = st;
    }
    if (info) *info = all;
    return worst;
  });
}

ipm_status ipm_newton_direction(ipm_ctx *c, const double *jv, const double *b, const double *cc,
                                const double *wv, const double *x, const double *s,
                                const double *lam, const double *w, double *dx, double *ds,
                                double *dl) {
  if (!c) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 2) throw Fail{IPM_ERR_STATE, "ipm_newton_direction before ipm_set_workspace"};
    VecOps V = c->vec();
    eval_g(c, jv, b, x);
    V.scaling(s, lam, c->opts.delta_d, c->vD);
    double delta_p = c->opts.delta_p;
    ipm_status stt = factor_with_retry(c, wv, jv, c->opts.precision, delta_p, nullptr);
    if (stt != IPM_OK) return stt;
    return direction(c, jv, b, cc, wv, x, s, lam, w, dx, ds, dl, nullptr);
  });
}

ipm_status ipm_solve(ipm_ctx *c, const double *jv, const double *b, const double *cc,
                     const double *wv, double *x, double *s, double *lam, ipm_result *res_out) {
  if (!c || !x || !s || !lam || !cc) return IPM_ERR_ARG;
  ipm_result res{};
  ipm_status rs = guarded(c, [&]() -> ipm_status {
    if (c->state < 2) throw Fail{IPM_ERR_STATE, "ipm_solve before ipm_set_workspace"};
    const auto t_start = std::chrono::steady_clock::now();
    const Problem &P = c->P;
    const ipm_options &o = c->opts;
    VecOps V = c->vec();
    c->refine_steps = c->pcg_steps = 0;
    if (c->sys) c->sys->refine_steps = c->sys->pcg_steps = 0;
    // starting point (unless warm-started from the caller's x, s, lambda)
    if (!o.warm_start) {
      c->have_stale = false;  // a held factor belongs to another run
      std::vector<double> x0(P.n);
      for (int32_t i = 0; i < P.n; i++) {
        const bool fl = std::isfinite(P.l[i]), fu = std::isfinite(P.u[i]);
        if (fl && fu) x0[i] = 0.5 * (P.l[i] + P.u[i]);
        else if (fl) x0[i] = std::max(0.0, P.l[i] + 1.0);
        else if (fu) x0[i] = std::min(0.0, P.u[i] - 1.0);
        else x0[i] = 0.0;
      }
      CK(cudaMemcpyAsync(x, x0.data(), P.n * sizeof(double), cudaMemcpyHostToDevice, c->st));
      eval_g(c, jv, b, x);
      V.init_slack(c->vg, s, lam);
    }
    // scales of the KKT residual
    double bscale = 1.0, cscale = 1.0;
    {
      V.absmax(P.m, b, c->scal + 20);
      V.absmax(P.n, cc, c->scal + 21);
      double bm = P.m > 0 ? d2h_scalar(c, c->scal + 20) : 0.0, cm = d2h_scalar(c, c->scal + 21);
      for (int32_t k = 0; k < P.nl; k++) bm = std::max(bm, std::fabs(P.l[P.lidx[k]]));
      for (int32_t k = 0; k < P.nu; k++) bm = std::max(bm, std::fabs(P.u[P.uidx[k]]));
      bscale = std::max(1.0, bm);
      cscale = std::max(1.0, cm);
    }
    cudaEvent_t ev[6];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    double delta_p = o.delta_p;
    res.status = IPM_ERR_MAXITER;
    ipm_status stt = IPM_OK;
    // Arithmetic of the factor: starts at o.precision; after an escalation
    // (fallback_fp64) it stays at the fallback arithmetic for the rest of the
    // solve, since the condensed matrix only gets worse conditioned as mu -> 0.
    int prec_now = o.precision;
    const int fb_prec = c->storage_bytes == 8 ? IPM_FP64 : IPM_TF32X3;
    const ipm_ctx *fac = c->sys ? c->sys : c;  // the context that holds the factor
    auto can_escalate = [&]() {
      return o.fallback_fp64 && c->factor_prec != fb_prec && c->factor_prec != IPM_FP64 &&
             (fb_prec == IPM_FP64 || (fac->tcp.ready() && !fac->dp.sgn));
    };
    // The iterate before a step taken with a low-precision factor: a step
    // that made the KKT residual grow tenfold is taken back and the iteration
    // redone in the fallback arithmetic (the direction's error, not the
    // method, made it grow).
    double *keep = nullptr;
    double prev_kkt = 0.0;
    bool low_step = false;
    const int64_t nkeep = P.n + 2 * P.mt;
    if (o.fallback_fp64 && o.precision != IPM_FP64 && o.precision != fb_prec)
      CK(cudaMallocAsync(&keep, nkeep * sizeof(double), c->st));
    struct KeepFree {
      double *&p;
      cudaStream_t st;
      ~KeepFree() {
        if (p) cudaFreeAsync(p, st);
      }
    } keep_free{keep, c->st};
    int it = 0;
    for (it = 0; it <= o.max_iter; it++) {
      eval_g(c, jv, b, x);
      V.jtv(jv, lam, -1.0, wv, x, cc, c->vrd);  // rd = c + W x - J^T lambda
      if (wv) V.jtv(jv, lam, 0.0, wv, x, nullptr, c->vwx);  // W x
      V.kkt(c->vg, s, lam, c->vrd, cc, wv ? c->vwx : nullptr, x, c->scal + 24, c->sc);
      IpmScalars h;
      CK(cudaMemcpyAsync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      const double fs = std::max(1.0, std::fabs(h.fx));
      res.primal_res = h.primal_inf / bscale;
      res.dual_res = h.dual_inf / cscale;
      res.compl_res = h.compl_inf / fs;
      res.kkt = std::max(res.primal_res, std::max(res.dual_res, res.compl_res));
      res.objective = h.fx;
      res.mu = h.mu;
      if (o.verbose)
        std::fprintf(stderr, "ipm it %3d f % .10e kkt %.3e (p %.2e d %.2e c %.2e) mu %.2e\n", it,
                     h.fx, res.kkt, res.primal_res, res.dual_res, res.compl_res, h.mu);
      // the maxima skip NaN, the sums (mu, f) do not
      if (!std::isfinite(res.kkt) || !std::isfinite(h.mu) || !std::isfinite(h.fx)) {
        res.status = IPM_ERR_NUMERIC;
        break;
      }
      if (keep && low_step && res.kkt > 10.0 * prev_kkt && can_escalate()) {
        CK(cudaMemcpyAsync(x, keep, P.n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(s, keep + P.n, P.mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(lam, keep + P.n + P.mt, P.mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        if (o.verbose)
          std::fprintf(stderr, "ipm it %3d: KKT grew from %.3e, step taken back, fallback arithmetic\n", it,
                       prev_kkt);
        res.fp64_fallbacks++;
        prec_now = fb_prec;
        low_step = false;
        c->have_stale = false;
        it--;
        continue;
      }
      if (res.kkt <= o.tol) { res.status = IPM_OK; break; }
      if (it == o.max_iter) break;
      const int64_t cg_iter0 = c->pcg_steps + (c->sys ? c->sys->pcg_steps : 0);
      CK(cudaEventRecord(ev[0], c->st));
      V.scaling(s, lam, o.delta_d, c->vD);
      CK(cudaEventRecord(ev[1], c->st));
      // Learned skip: keep the held (stale) factor, correct it with the
      // network's Delta + U U^T and solve both directions by PCG; any solve
      // that misses ir_tol within learned_pcg_max iterations falls back to
      // the exact refactorisation.
      const bool try_skip = o.learned != 0 && c->lb_on && c->have_stale && c->factor_prec != IPM_FP64 &&
                            c->tcp.ready();
      bool factored = false;
      auto refactor = [&]() -> ipm_status {
        c->learned_active = false;
        c->refine_override = c->pcg_override = -1;
        // a low-precision factor that had to perturb pivots, or met a pivot
        // of the wrong sign, has broken down by rounding: redo it in the
        // fallback arithmetic before solving with it (and raise delta_p only
        // for a breakdown in that arithmetic)
        const bool esc = can_escalate();
        ipm_status f = factor_with_retry(c, wv, jv, prec_now, delta_p, &res, esc ? 0 : 12);
        if (esc && (f == IPM_ERR_NOT_SPD || (f == IPM_OK && c->last_perturbed > 0))) {
          res.fp64_fallbacks++;
          prec_now = fb_prec;
          f = factor_with_retry(c, wv, jv, prec_now, delta_p, &res);
        }
        if (f == IPM_OK) {
          factored = true;
          save_stale(c, jv);
        }
        return f;
      };
      ipm_solve_info si{};
      if (try_skip) {
        learned_prepare(c, jv, x, delta_p, o.learned == 2);
        c->cur_jvals = jv;
        c->cur_D = c->vD;
        c->cur_wvals = wv;
        c->cur_delta_p = delta_p;
        c->learned_active = true;
        c->refine_override = IPM_REFINE_PCG;
        c->pcg_override = o.learned_pcg_max;
        const int64_t pcg0 = c->pcg_steps;
        stt = direction(c, jv, b, cc, wv, x, s, lam, nullptr, c->vdx, c->vds, c->vdl, &si);
        res.learned_pcg_steps += (int32_t)(c->pcg_steps - pcg0);
        if (o.verbose)
          std::fprintf(stderr, "ipm it %3d stale-factor PCG: %d iterations, residual %.2e -> %s\n",
                       it, (int)(c->pcg_steps - pcg0), c->last_rel,
                       c->last_rel <= o.ir_tol ? "kept" : "refactor");
        if (stt != IPM_OK || !(c->last_rel <= o.ir_tol)) {
          stt = refactor();
          if (stt == IPM_OK)
            stt = direction(c, jv, b, cc, wv, x, s, lam, nullptr, c->vdx, c->vds, c->vdl, &si);
        }
      } else {
        stt = refactor();
        if (stt == IPM_OK)
          stt = direction(c, jv, b, cc, wv, x, s, lam, nullptr, c->vdx, c->vds, c->vdl, &si);
      }
      CK(cudaEventRecord(ev[2], c->st));
      res.worst_rel_residual = std::max(res.worst_rel_residual, si.rel_residual);
      // A solve that missed accept_tol with a low-precision factor: refactor in
      // the most accurate arithmetic the storage allows and solve again.
      if (stt != IPM_OK && can_escalate()) {
        res.fp64_fallbacks++;
        prec_now = fb_prec;
        c->learned_active = false;
        c->refine_override = c->pcg_override = -1;
        stt = factor_with_retry(c, wv, jv, fb_prec, delta_p, &res);
        if (stt == IPM_OK)
          stt = direction(c, jv, b, cc, wv, x, s, lam, nullptr, c->vdx, c->vds, c->vdl, &si);
      }
      if (stt != IPM_OK) { res.status = stt; c->learned_active = false; break; }
      V.ftb(s, c->vds, lam, c->vdl, c->scal + 32, c->sc, true);
      V.muaff(s, c->vds, lam, c->vdl, c->scal + 34, c->sc);
      // corrector: w = sigma mu - ds_aff .* dl_aff
      V.corrector_target(c->vds, c->vdl, c->sc, c->vw);
      {
        const int64_t pcg0 = c->pcg_steps;
        const bool with_stale = c->learned_active;
        // the corrector's system differs from the predictor's only in its
        // right-hand side: its solve starts from the predictor's d_x
        struct Reset {
          bool &f;
          ~Reset() { f = false; }  // also when the direction throws
        } reset{c->warm_x};
        c->warm_x = !c->sys && !with_stale;
        stt = direction(c, jv, b, cc, wv, x, s, lam, c->vw, c->vdx, c->vds, c->vdl, &si);
        c->warm_x = false;
        if (with_stale) res.learned_pcg_steps += (int32_t)(c->pcg_steps - pcg0);
        if (with_stale && (stt != IPM_OK || !(c->last_rel <= o.ir_tol))) {
          stt = refactor();
          if (stt == IPM_OK)
            stt = direction(c, jv, b, cc, wv, x, s, lam, c->vw, c->vdx, c->vds, c->vdl, &si);
        }
        if (stt != IPM_OK && can_escalate()) {  // the corrector missed accept_tol
          res.fp64_fallbacks++;
          prec_now = fb_prec;
          c->learned_active = false;
          c->refine_override = c->pcg_override = -1;
          stt = factor_with_retry(c, wv, jv, fb_prec, delta_p, &res);
          if (stt == IPM_OK)
            stt = direction(c, jv, b, cc, wv, x, s, lam, c->vw, c->vdx, c->vds, c->vdl, &si);
        }
      }
      c->learned_active = false;
      c->refine_override = c->pcg_override = -1;
      if (try_skip && !factored) res.learned_skips++;
      res.worst_rel_residual = std::max(res.worst_rel_residual, si.rel_residual);
      if (stt != IPM_OK) { res.status = stt; break; }
      CK(cudaEventRecord(ev[3], c->st));
      if (keep) {
        CK(cudaMemcpyAsync(keep, x, P.n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(keep + P.n, s, P.mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(keep + P.n + P.mt, lam, P.mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        low_step = c->factor_prec != IPM_FP64 && c->factor_prec != fb_prec;
        prev_kkt = res.kkt;
      }
      V.ftb(s, c->vds, lam, c->vdl, c->scal + 32, c->sc, false);
      V.update(c->sc, x, c->vdx, s, c->vds, lam, c->vdl);
      {  // cost-driven escalation (cg_escalate): CG steps of this iteration's two solves
        const int64_t cg_now = c->pcg_steps + (c->sys ? c->sys->pcg_steps : 0);
        if (o.cg_escalate > 0 && cg_now - cg_iter0 > o.cg_escalate && can_escalate()) {
          if (o.verbose)
            std::fprintf(stderr, "ipm it %3d: %lld CG steps, fallback arithmetic from here\n", it,
                         (long long)(cg_now - cg_iter0));
          res.fp64_fallbacks++;
          prec_now = fb_prec;
          c->have_stale = false;
        }
      }
      CK(cudaEventRecord(ev[4], c->st));
      CK(cudaEventSynchronize(ev[4]));
      float ms[4];
      for (int k = 0; k < 4; k++) CK(cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]));
      res.time_assemble_ms += ms[0];
      res.time_factor_ms += ms[1];
      res.time_solve_ms += ms[2];
      res.time_other_ms += ms[3];
    }
    for (auto &e : ev) cudaEventDestroy(e);
    CK(cudaStreamSynchronize(c->st));
    res.iterations = it;
    res.refine_steps = (int32_t)(c->refine_steps + (c->sys ? c->sys->refine_steps : 0));
    res.pcg_steps = (int32_t)(c->pcg_steps + (c->sys ? c->sys->pcg_steps : 0));
    res.time_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return (ipm_status)res.status;
  });
  res.status = rs;  // also the status of an error that ended the call early
  if (res_out) *res_out = res;
  return rs;
}

ipm_status kkt_symbolic_export(const ipm_ctx *c, int32_t *perm, int32_t *parent, int32_t *colcount,
                               int32_t *super, int32_t *sparent, int32_t *slevel, int64_t *srp,
                               int32_t *sri) {
  if (!c || c->state < 1) return c ? IPM_ERR_STATE : IPM_ERR_ARG;
  if (c->sys)  // the formulation's system
    return kkt_symbolic_export(c->sys, perm, parent, colcount, super, sparent, slevel, srp, sri);
  const Symbolic &S = c->S;
  auto cp = [](auto *dst, const auto &v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(perm, S.perm);
  cp(parent, S.parent);
  cp(colcount, S.colcount);
  cp(super, S.super);
  cp(sparent, S.sparent);
  cp(slevel, S.slevel);
  cp(srp, S.srp);
  cp(sri, S.sri);
  return IPM_OK;
}

ipm_status kkt_export_assembled(ipm_ctx *c, double *h_out) {
  if (!c || !h_out) return IPM_ERR_ARG;
  if (c->sys) {
    const ipm_status st = kkt_export_assembled(c->sys, h_out);
    if (st != IPM_OK) c->err = c->sys->err;
    return st;
  }
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 3) throw Fail{IPM_ERR_STATE, "nothing assembled"};
    const int64_t nk = c->dp.nk;
    std::vector<double> tmp(nk);
    CK(cudaMemcpyAsync(tmp.data(), c->kval, nk * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int64_t q = 0; q < nk; q++) h_out[c->plan.k_orig[q]] = tmp[q];
    return IPM_OK;
  });
}

ipm_status kkt_factor_entries(ipm_ctx *c, int64_t count, const int32_t *rows, const int32_t *cols,
                              double *out) {
  if (!c || count < 0 || (count > 0 && (!rows || !cols || !out))) return IPM_ERR_ARG;
  if (c->sys) {
    const ipm_status st = kkt_factor_entries(c->sys, count, rows, cols, out);
    if (st != IPM_OK) c->err = c->sys->err;
    return st;
  }
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 4) throw Fail{IPM_ERR_STATE, "no factor"};
    if (count == 0) return IPM_OK;
    int32_t *dr = nullptr, *dc = nullptr;
    double *dout = nullptr;
    CK(cudaMallocAsync(&dr, count * sizeof(int32_t), c->st));
    CK(cudaMallocAsync(&dc, count * sizeof(int32_t), c->st));
    CK(cudaMallocAsync(&dout, count * sizeof(double), c->st));
    CK(cudaMemcpyAsync(dr, rows, count * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(dc, cols, count * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    if (c->factor_prec == IPM_FP64)
      launch_factor_entries<double>(c->dp, (const double *)c->L, c->col2s, count, dr, dc, dout, c->st);
    else
      launch_factor_entries<float>(c->dp, (const float *)c->L, c->col2s, count, dr, dc, dout, c->st);
    CK(cudaMemcpyAsync(out, dout, count * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaFreeAsync(dr, c->st));
    CK(cudaFreeAsync(dc, c->st));
    CK(cudaFreeAsync(dout, c->st));
    CK(cudaStreamSynchronize(c->st));
    return IPM_OK;
  });
}

int32_t ipm_last_perturbed(const ipm_ctx *c) { return c ? c->last_perturbed : 0; }

ipm_status kkt_test_solve_timeout(ipm_ctx *c, uint32_t spins, int32_t withheld_task) {
  if (!c || spins == 0 || withheld_task < 0) return IPM_ERR_ARG;
  if (c->sys) return kkt_test_solve_timeout(c->sys, spins, withheld_task);
  c->test_spins = spins;
  c->test_withhold = withheld_task;
  return IPM_OK;
}

ipm_status kkt_time_kernel(ipm_ctx *c, int32_t kernel, int32_t reps, double *ms) {
  if (!c || !ms || reps < 1) return IPM_ERR_ARG;
  if (c->sys) {
    const ipm_status st = kkt_time_kernel(c->sys, kernel, reps, ms);
    if (st != IPM_OK) c->err = c->sys->err;
    return st;
  }
  return guarded(c, [&]() -> ipm_status {
    if (kernel == 0 && c->state < 3) throw Fail{IPM_ERR_STATE, "nothing assembled"};
    if (kernel != 0 && c->state < 4) throw Fail{IPM_ERR_STATE, "no factor"};
    if ((kernel == 1 || kernel == 3 || kernel == 4) && c->factor_prec == IPM_FP64)
      throw Fail{IPM_ERR_STATE, "the persistent solve needs an FP32-storage factor"};
    if (kernel == 2 && c->factor_prec != IPM_FP64)
      throw Fail{IPM_ERR_STATE, "the level solve is timed on an FP64 factor"};
    if (kernel < 0 || kernel > 4) throw Fail{IPM_ERR_ARG, "unknown kernel id"};
    // the solves' work does not depend on the values: zero right-hand sides
    if (kernel == 1 || kernel == 3) CK(cudaMemsetAsync(c->fsa, 0, c->P.n * sizeof(float), c->st));
    if (kernel == 4) CK(cudaMemsetAsync(c->fsb, 0, c->P.n * sizeof(float), c->st));
    if (kernel == 2) CK(cudaMemsetAsync(c->yv, 0, c->P.n * sizeof(double), c->st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, c->st));
    for (int r = 0; r < reps; r++) {
      if (kernel == 0)
        launch_assemble(c->dp, c->cur_jvals, c->cur_D, c->cur_wvals, c->cur_delta_p, c->kval, c->st);
      else if (kernel == 1)
        launch_fp32_solve(c, 0);
      else if (kernel == 3 || kernel == 4)
        launch_fp32_solve(c, kernel == 3 ? 1 : 2);
      else
        launch_solve<double, double>(c->dp, c->plan, (const double *)c->L, c->yv, c->tv, c->st);
    }
    CK(cudaEventRecord(e1, c->st));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    if (kernel == 1 || kernel >= 3) check_solve_barrier(c);
    *ms = (double)t / reps;
    return IPM_OK;
  });
}

int32_t ipm_learned_param_count(void) { return kNParams; }

static bool learned_on(const ipm_ctx *c) {
  return c->lb_on && (c->opts.learned != 0 || c->opts.learned_probes > 0);
}

ipm_status ipm_learned_weights(ipm_ctx *c, float *h_get, const float *h_set) {
  if (!c) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 2 || !learned_on(c)) throw Fail{IPM_ERR_STATE, "learned buffers not set up"};
    if (h_get) CK(cudaMemcpyAsync(h_get, c->lb.w, kNParams * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    if (h_set) {
      CK(cudaMemcpyAsync(c->lb.w, h_set, kNParams * sizeof(float), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemsetAsync(c->lb.m, 0, kNParams * sizeof(float), c->st));
      CK(cudaMemsetAsync(c->lb.v, 0, kNParams * sizeof(float), c->st));
      c->lb.step = 0;
    }
    CK(cudaStreamSynchronize(c->st));
    return IPM_OK;
  });
}

ipm_status ipm_learned_sample(ipm_ctx *c, const double *jv, const double *x, const double *s,
                              const double *lam, const float *z, float *feat, float *w) {
  if (!c || !s || !lam || !z || !feat || !w) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (!learned_on(c) || !c->have_stale || c->factor_prec == IPM_FP64 || c->state < 4)
      throw Fail{IPM_ERR_STATE, "needs a held FP32-storage factor and learned buffers"};
    LearnedBufs &B = c->lb;
    VecOps V = c->vec();
    const int64_t n = c->P.n, mt = c->P.mt;
    V.scaling(s, lam, c->opts.delta_d, c->vD);
    V.dot(mt, s, lam, c->scal + 40);
    const double mu = d2h_scalar(c, c->scal + 40) / (double)std::max<int64_t>(mt, 1);
    CK(cudaMemcpyAsync(B.mu + 1, &mu, sizeof(double), cudaMemcpyHostToDevice, c->st));
    learned_diag(c->dp, jv, c->vD, c->cur_delta_p, B.diag_new, c->st);
    learned_features(c->dp, B, jv, c->vD, x, c->st);
    CK(cudaMemcpyAsync(feat, B.feat, n * kNF * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemsetAsync(c->vc, 0, n * sizeof(double), c->st));
    for (int p = 0; p < B.P; p++) {  // w_p = L^{-1} P K P^T L^{-T} z_p
      CK(cudaMemcpyAsync(c->fsb, z + (int64_t)p * n, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
      launch_fp32_solve(c, 2);
      V.permute_out<float>(c->fsx, nullptr, c->vz, false);
      V.residual(jv, c->vD, c->cur_wvals, c->cur_delta_p, c->vz, c->vc, c->vq, c->vtA);
      V.negate(n, c->vq);
      V.permute_in<float>(c->vq, nullptr, c->fsa);
      launch_fp32_solve(c, 1);
      CK(cudaMemcpyAsync(w + (int64_t)p * n, c->fsb, n * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    }
    check_solve_barrier(c);
    return IPM_OK;
  });
}

ipm_status ipm_learned_loss_grad(ipm_ctx *c, const float *feat, const float *z, const float *w,
                                 double *h_loss, float *h_grad) {
  if (!c || !feat || !z || !w) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (!learned_on(c) || c->state < 2) throw Fail{IPM_ERR_STATE, "learned buffers not set up"};
    LearnedBufs &B = c->lb;
    CK(cudaMemcpyAsync(B.feat, feat, c->P.n * kNF * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    learned_forward(B, false, c->st);
    learned_loss_grad(B, z, w, c->lb_loss, c->st);
    if (h_loss) CK(cudaMemcpyAsync(h_loss, c->lb_loss, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (h_grad) CK(cudaMemcpyAsync(h_grad, B.grad, kNParams * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return IPM_OK;
  });
}

ipm_status ipm_learned_train(ipm_ctx *c, const float *feat, const float *z, const float *w,
                             float lr, int32_t steps, double *h_loss) {
  if (!c || !feat || !z || !w || steps < 0) return IPM_ERR_ARG;
  return guarded(c, [&]() -> ipm_status {
    if (!learned_on(c) || c->state < 2) throw Fail{IPM_ERR_STATE, "learned buffers not set up"};
    LearnedBufs &B = c->lb;
    CK(cudaMemcpyAsync(B.feat, feat, c->P.n * kNF * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    for (int k = 0; k < steps; k++) {
      learned_forward(B, false, c->st);
      learned_loss_grad(B, z, w, c->lb_loss, c->st);
      learned_adam(B, lr, c->st);
    }
    if (h_loss) CK(cudaMemcpyAsync(h_loss, c->lb_loss, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return IPM_OK;
  });
}

static bool grid_from(const ipm_grid_nlp *pp, GridNlp &p) {
  if (!pp || pp->nx < 2 || pp->nx > 16384 || !(pp->alpha >= 0.0)) return false;
  if (pp->v_bounded && !(pp->v_lo < pp->v_hi)) return false;
  p.N = pp->nx;
  p.alpha = pp->alpha;
  p.v_lo = pp->v_lo;
  p.v_hi = pp->v_hi;
  p.cubic = pp->cubic ? 1 : 0;
  p.v_bounded = pp->v_bounded ? 1 : 0;
  return true;
}

ipm_status ipm_grid_nlp_sizes(const ipm_grid_nlp *pp, int32_t *n, int32_t *m, int64_t *nnz_j) {
  GridNlp p;
  if (!grid_from(pp, p)) return IPM_ERR_ARG;
  const int64_t NN = p.NN();
  if (n) *n = (int32_t)(2 * NN);
  if (m) *m = (int32_t)(2 * NN);
  if (nnz_j) *nnz_j = 2 * (5 * NN - 4 * (int64_t)p.N + NN);
  return IPM_OK;
}

ipm_status ipm_grid_nlp_pattern(const ipm_grid_nlp *pp, int64_t *h_jrowptr, int32_t *h_jcol,
                                int64_t *h_wcolptr, int32_t *h_wrow, double *h_l, double *h_u) {
  GridNlp p;
  if (!grid_from(pp, p)) return IPM_ERR_ARG;
  try {
    std::vector<int64_t> rp;
    std::vector<int32_t> cl;
    grid_nlp_pattern(p, rp, cl);
    const int64_t NN = p.NN(), n = 2 * NN;
    if (h_jrowptr) std::memcpy(h_jrowptr, rp.data(), rp.size() * sizeof(int64_t));
    if (h_jcol) std::memcpy(h_jcol, cl.data(), cl.size() * sizeof(int32_t));
    for (int64_t j = 0; j <= n && h_wcolptr; j++) h_wcolptr[j] = j;
    for (int64_t j = 0; j < n && h_wrow; j++) h_wrow[j] = (int32_t)j;
    for (int64_t j = 0; j < n; j++) {
      const bool bv = p.v_bounded && j >= NN;
      if (h_l) h_l[j] = bv ? p.v_lo : -INFINITY;
      if (h_u) h_u[j] = bv ? p.v_hi : INFINITY;
    }
  } catch (const std::bad_alloc &) {
    return IPM_ERR_NOMEM;
  }
  return IPM_OK;
}

ipm_status ipm_solve_problem(ipm_ctx *c, const ipm_problem *p, double *x, double *s, double *lam,
                             ipm_result *res) {
  if (!c || !p) return IPM_ERR_ARG;
  switch (p->kind) {
    case IPM_PROBLEM_LPQP: return ipm_solve(c, p->d_jvals, p->d_b, p->d_c, p->d_wvals, x, s, lam, res);
    case IPM_PROBLEM_GRID_NLP: return ipm_solve_grid_nlp(c, p->nlp, p->d_ut, x, s, lam, res);
    case IPM_PROBLEM_NLP: return ipm_solve_nlp(c, p->fns, x, s, lam, res);
    default: return IPM_ERR_ARG;
  }
}

}  // extern "C"

// The nonlinear interior-point loop (Sec. 3 rules for a general problem; see
// the header's ipm_solve_nlp) over evaluation callbacks: F.eval(x) writes f
// (device scalar), grad f (n), the m general rows g_G(x) and J's values in the
// context's pattern order; F.hess(x, lambda) the values of W (the Hessian of
// f - lambda_G^T g_G) in the context's W pattern.
struct NlpFns {
  std::function<void(const double *x, double *d_f, double *grad, double *grows, double *jv)> eval;
  std::function<void(const double *x, const double *lam, double *wv)> hess;
};

ipm_status nlp_solve(ipm_ctx *c, const NlpFns &F, double *x, double *s, double *lam,
                     ipm_result *res_out, const char *who) {
  ipm_result res{};
  double *scratch = nullptr;
  ipm_status rs = guarded(c, [&]() -> ipm_status {
    if (c->state < 2) throw Fail{IPM_ERR_STATE, std::string(who) + " before ipm_set_workspace"};
    if (c->sys) throw Fail{IPM_ERR_UNSUPPORTED, "the nonlinear solver uses the primal condensed formulation"};
    const Problem &P = c->P;
    const int64_t n = P.n, m = P.m, mt = P.mt;
    (void)m;
    const auto t_start = std::chrono::steady_clock::now();
    const ipm_options &o = c->opts;
    VecOps V = c->vec();
    c->refine_steps = c->pcg_steps = 0;
    const int64_t nnz = (int64_t)P.ji.size();
    c->bwd_measure = true;
    const int64_t nw = std::max<int64_t>((int64_t)P.wi.size(), 1);
    const size_t words = (size_t)(3 * n + 6 * mt + nnz + nw);
    CK(cudaMallocAsync(&scratch, words * sizeof(double), c->st));
    double *jv = scratch, *hrows = jv + nnz, *grad = hrows + mt, *wv = grad + n, *zero = wv + nw,
           *xt = zero + mt, *stv = xt + n, *gt = stv + mt, *keep = gt + mt;  // keep: x, s, lambda
    CK(cudaMemsetAsync(zero, 0, mt * sizeof(double), c->st));
    double *d_f = c->scal + 44, *terms = c->scal + 48;
    auto d2h = [&](const double *d, double *h, int cnt) {
      CK(cudaMemcpyAsync(h, d, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
    };
    auto eval_at = [&](const double *xx, double *gout) {  // f (returned), g_G, J, grad, g
      F.eval(xx, d_f, grad, hrows, jv);
      V.g(hrows, xx, zero, c->dl_, c->du_, gout);
      double f;
      d2h(d_f, &f, 1);
      return f;
    };
    auto set_sc = [&](size_t off, double v) {
      CK(cudaMemcpyAsync(reinterpret_cast<char *>(c->sc) + off, &v, sizeof(double),
                         cudaMemcpyHostToDevice, c->st));
    };
    // starting point: the box midpoint, 1 inside a one-sided bound, else 0
    {
      std::vector<double> x0(n);
      for (int64_t i = 0; i < n; i++) {
        const bool fl = std::isfinite(P.l[i]), fu = std::isfinite(P.u[i]);
        x0[i] = fl && fu ? 0.5 * (P.l[i] + P.u[i])
                         : (fl ? std::max(0.0, P.l[i] + 1.0) : (fu ? std::min(0.0, P.u[i] - 1.0) : 0.0));
      }
      CK(cudaMemcpyAsync(x, x0.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->st));
      CK(cudaStreamSynchronize(c->st));
    }
    eval_at(x, c->vg);
    V.init_slack(c->vg, s, lam);
    double mu = 0.1, nu = 0.0;
    double bscale = 1.0;  // largest finite bound (at least 1)
    for (int64_t i = 0; i < n; i++) {
      if (std::isfinite(P.l[i])) bscale = std::max(bscale, std::fabs(P.l[i]));
      if (std::isfinite(P.u[i])) bscale = std::max(bscale, std::fabs(P.u[i]));
    }
    V.absmax(n, grad, c->scal + 20);
    const double cscale = std::max(1.0, d2h_scalar(c, c->scal + 20));
    res.status = IPM_ERR_MAXITER;
    ipm_status stt = IPM_OK;
    // arithmetic of the factor: o.precision until a low-precision factor has
    // to be redone in FP64, FP64 from then on (K only gets worse conditioned)
    int prec_now = o.precision;
    // the iterate (and mu, nu) before a step taken with a low-precision factor:
    // a step after which the KKT residual is more than 10x the previous one is
    // taken back and redone in FP64, as in ipm_solve
    double prev_kkt = 0.0, keep_mu = 0.0, keep_nu = 0.0;
    bool low_step = false;
    int it = 0;
    for (it = 0; it <= o.max_iter; it++) {
      const double f = eval_at(x, c->vg);
      V.jtv(jv, lam, -1.0, nullptr, nullptr, grad, c->vrd);  // grad f - J^T lambda
      V.kkt(c->vg, s, lam, c->vrd, zero, nullptr, x, c->scal + 24, c->sc);
      IpmScalars h;
      CK(cudaMemcpyAsync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      const double fs = std::max(1.0, std::fabs(f));
      res.primal_res = h.primal_inf / bscale;
      res.dual_res = h.dual_inf / cscale;
      res.compl_res = h.compl_inf / fs;
      res.kkt = std::max(res.primal_res, std::max(res.dual_res, res.compl_res));
      res.objective = f;
      res.mu = mu;
      if (o.verbose)
        std::fprintf(stderr, "nlp it %3d f % .10e kkt %.3e (p %.2e d %.2e c %.2e) mu %.2e\n", it, f,
                     res.kkt, res.primal_res, res.dual_res, res.compl_res, mu);
      if (low_step && res.kkt > 10.0 * prev_kkt && o.fallback_fp64 && c->storage_bytes == 8) {
        CK(cudaMemcpyAsync(x, keep, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(s, keep + n, mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(lam, keep + n + mt, mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        if (o.verbose)
          std::fprintf(stderr, "nlp it %3d: KKT grew from %.3e, step taken back, FP64 from here\n", it,
                       prev_kkt);
        mu = keep_mu;
        nu = keep_nu;
        res.fp64_fallbacks++;
        prec_now = IPM_FP64;
        low_step = false;
        it--;
        continue;
      }
      if (!std::isfinite(res.kkt) || !std::isfinite(h.mu) || !std::isfinite(f)) {
        res.status = IPM_ERR_NUMERIC;
        break;
      }
      if (res.kkt <= o.tol) { res.status = IPM_OK; break; }
      if (it == o.max_iter) break;
      if (prec_now != IPM_FP64) {
        CK(cudaMemcpyAsync(keep, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(keep + n, s, mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(keep + n + mt, lam, mt * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        keep_mu = mu;
        keep_nu = nu;
        prev_kkt = res.kkt;
      }
      // monotone barrier update once the barrier problem is solved to 10 mu
      nlp_barrier_err(mt, s, lam, mu, terms, c->partial, c->st);
      double berr;
      d2h(terms, &berr, 1);
      if (std::max(res.primal_res, std::max(res.dual_res, berr / fs)) <= 10.0 * mu)
        mu = std::max(o.tol / 10.0, std::min(0.2 * mu, std::pow(mu, 1.5)));
      // Newton direction with target mu; inertia by regularisation
      F.hess(x, lam, wv);
      V.scaling(s, lam, o.delta_d, c->vD);
      double delta_p = o.delta_p;
      for (int tries = 0; tries < 12; tries++) {
        stt = factor_with_retry(c, wv, jv, prec_now, delta_p, &res);
        if (stt != IPM_OK || c->factor_prec == IPM_FP64 || c->last_perturbed == 0) break;
        // the FP32 factor met a non-positive pivot: an FP64 factor tells a
        // rounding breakdown from true indefiniteness (which it regularises)
        if (o.fallback_fp64 && c->storage_bytes == 8) {
          res.fp64_fallbacks++;
          prec_now = IPM_FP64;
          stt = factor_with_retry(c, wv, jv, IPM_FP64, delta_p, &res);
          break;
        }
        delta_p = delta_p > 0 ? delta_p * 100.0 : 1e-8;
        res.regularizations++;
      }
      ipm_solve_info si{};
      if (stt == IPM_OK) {
        nlp_fill(mt, mu, c->vw, c->st);
        c->nlp_grad = true;
        // K may be indefinite away from a local minimum (W is the Hessian of
        // the Lagrangian): refine without conjugate gradients
        if (o.refine == IPM_REFINE_PCG) c->refine_override = IPM_REFINE_IR;
        stt = direction(c, jv, nullptr, grad, wv, x, s, lam, c->vw, c->vdx, c->vds, c->vdl, &si);
        c->nlp_grad = false;
        if (stt != IPM_OK && o.fallback_fp64 && c->factor_prec != IPM_FP64 && c->storage_bytes == 8) {
          res.fp64_fallbacks++;
          prec_now = IPM_FP64;
          stt = factor_with_retry(c, wv, jv, IPM_FP64, delta_p, &res);
          if (stt == IPM_OK) {
            c->nlp_grad = true;
            stt = direction(c, jv, nullptr, grad, wv, x, s, lam, c->vw, c->vdx, c->vds, c->vdl, &si);
            c->nlp_grad = false;
          }
        }
        c->refine_override = -1;
      }
      res.worst_rel_residual = std::max(res.worst_rel_residual, si.rel_residual);
      if (stt != IPM_OK) { res.status = stt; break; }
      // common step from the fraction to the boundary, then backtracking on the merit
      set_sc(offsetof(IpmScalars, mu), mu);
      V.ftb(s, c->vds, lam, c->vdl, c->scal + 32, c->sc, false);
      CK(cudaMemcpyAsync(&h, c->sc, sizeof(h), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      double alpha = std::min(h.alpha_p, h.alpha_d);
      double dt[3], mt2[2];
      nlp_dir_terms(n, mt, grad, c->vdx, s, c->vds, lam, c->vdl, terms, c->partial, c->st);
      d2h(terms, dt, 3);
      nu = std::max(nu, dt[2] + 1.0);
      nlp_merit_terms(mt, s, c->vg, terms, c->partial, c->st);
      d2h(terms, mt2, 2);
      // derivative of nu ||g - s||_1 along the step actually solved: the
      // regularised system (3) leaves O(delta_d d_lambda) in g - s, which is
      // all there is on the rows of an equality pair (both slacks stay
      // positive), so -nu ||g - s||_1 would promise a decrease no step can give
      double dth;
      nlp_dtheta(mt, c->vg, s, c->vjd, c->vds, terms + 2, c->partial, c->st);
      d2h(terms + 2, &dth, 1);
      const double phi0 = f - mu * mt2[0] + nu * mt2[1];
      const double dphi = dt[0] - mu * dt[1] + nu * dth;
      if (dphi < 0.0) {
        for (int hv = 0; hv < 10; hv++) {
          nlp_trial(n, mt, x, c->vdx, s, c->vds, alpha, xt, stv, c->st);
          const double ft = eval_at(xt, gt);
          nlp_merit_terms(mt, stv, gt, terms, c->partial, c->st);
          d2h(terms, mt2, 2);
          // Armijo, allowing for the rounding of phi (10 eps |phi|)
          if (ft - mu * mt2[0] + nu * mt2[1] <= phi0 + 1e-4 * alpha * dphi + 10.0 * DBL_EPSILON * std::fabs(phi0))
            break;
          alpha *= 0.5;
        }
      }
      set_sc(offsetof(IpmScalars, alpha_p), alpha);
      set_sc(offsetof(IpmScalars, alpha_d), alpha);
      V.update(c->sc, x, c->vdx, s, c->vds, lam, c->vdl);
      low_step = c->factor_prec != IPM_FP64;
    }
    res.iterations = it;
    CK(cudaStreamSynchronize(c->st));
    res.time_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    res.refine_steps = (int32_t)c->refine_steps;
    res.pcg_steps = (int32_t)c->pcg_steps;
    return (ipm_status)res.status;
  });
  c->nlp_grad = false;
  c->bwd_measure = false;
  if (scratch) {
    cudaFreeAsync(scratch, c->st);
    cudaStreamSynchronize(c->st);
  }
  if (res_out) {
    res.status = rs;
    *res_out = res;
  }
  return rs;
}

extern "C" {

ipm_status ipm_solve_grid_nlp(ipm_ctx *c, const ipm_grid_nlp *pp, const double *ut, double *x,
                              double *s, double *lam, ipm_result *res_out) {
  if (!c || !pp || !ut || !x || !s || !lam) return IPM_ERR_ARG;
  GridNlp p;
  ipm_status chk = guarded(c, [&]() -> ipm_status {
    if (!grid_from(pp, p)) throw Fail{IPM_ERR_ARG, "invalid grid NLP parameters"};
    const Problem &P = c->P;
    const int64_t NN = p.NN(), n = P.n, m = P.m;
    std::vector<int64_t> rp;  // the context must carry this problem's patterns
    std::vector<int32_t> cl;
    grid_nlp_pattern(p, rp, cl);
    bool ok = n == 2 * NN && m == 2 * NN && P.jp.size() == rp.size() && P.ji.size() == cl.size() &&
              std::equal(rp.begin(), rp.end(), P.jp.begin()) &&
              std::equal(cl.begin(), cl.end(), P.ji.begin()) && (int64_t)P.wp.size() == n + 1;
    for (int64_t j = 0; ok && j < n; j++)
      ok = P.wp[j] == j && P.wi[j] == (int32_t)j &&
           std::isfinite(P.l[j]) == (p.v_bounded && j >= NN) &&
           std::isfinite(P.u[j]) == (p.v_bounded && j >= NN);
    if (!ok) throw Fail{IPM_ERR_ARG, "context pattern is not the grid NLP's"};
    return IPM_OK;
  });
  if (chk != IPM_OK) return chk;
  NlpFns F;
  F.eval = [&](const double *xx, double *d_f, double *grad, double *grows, double *jv) {
    nlp_eval(p, c->dp.jp, xx, ut, grows, jv, grad, d_f, c->partial, c->st);
  };
  F.hess = [&](const double *xx, const double *lm, double *wv) { nlp_hess(p, xx, lm, wv, c->st); };
  return nlp_solve(c, F, x, s, lam, res_out, "ipm_solve_grid_nlp");
}

ipm_status ipm_solve_nlp(ipm_ctx *c, const ipm_nlp *p, double *x, double *s, double *lam,
                         ipm_result *res_out) {
  if (!c || !p || !p->eval || !p->hess || !x || !s || !lam) return IPM_ERR_ARG;
  NlpFns F;
  F.eval = [&](const double *xx, double *d_f, double *grad, double *grows, double *jv) {
    if (p->eval(p->user, xx, d_f, grad, grows, jv, c->st) != 0)
      throw Fail{IPM_ERR_NUMERIC, "the problem's evaluation callback failed"};
  };
  F.hess = [&](const double *xx, const double *lm, double *wv) {
    if (p->hess(p->user, xx, lm, wv, c->st) != 0)
      throw Fail{IPM_ERR_NUMERIC, "the problem's Hessian callback failed"};
  };
  return nlp_solve(c, F, x, s, lam, res_out, "ipm_solve_nlp");
}

int64_t ipm_kernel_launches(void) { return gipm::launch_counter(); }

const char *ipm_last_error(const ipm_ctx *c) { return c ? c->err.c_str() : "null context"; }

void ipm_destroy(ipm_ctx *c) {
  delete c;
}

}  // extern "C"

// ===========================================================================
// Solve without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code running while a memory pool is locked or exhausted, code inside
// another library's allocation-free callback, or a process whose allocator
// belongs to a framework it must not re-enter. kkt_solve_noalloc gives them
// the factor-only solve x = P^T L^{-T} L^{-1} P b with its working vectors
// (the permuted right-hand side, the children's update vectors, a scale and
// the reduction partials) in the file-scope array below instead of the
// context workspace. The caller still passes b and x.
// ===========================================================================
namespace {

constexpr size_t kNoAllocDoubles = size_t(1) << 20;  // 8 MiB per device, held until exit
__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {};

}  // namespace

namespace {

// The lookup runs with `dev` current; cudaGetSymbolAddress loads this file's
// module on that device (under lazy module loading, the first use of the
// array is what commits it).
double *noalloc_scratch(int dev) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) throw Fail{IPM_ERR_UNSUPPORTED, "device index too large"};
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != dev) throw Fail{IPM_ERR_ARG, "static scratch looked up with another device current"};
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  return g_noalloc_addr[dev];
}

size_t noalloc_need(const ipm_ctx *c) {
  // partials + 32 scalars + y (n) + update vectors (plan.t_entries), in doubles
  return (size_t)kRedBlocks * 8 + 32 + (size_t)std::max<int32_t>(c->P.n, 1) +
         (size_t)c->plan.t_entries;
}

}  // namespace

extern "C" {

int64_t kkt_solve_noalloc_capacity(void) { return (int64_t)kNoAllocDoubles; }

ipm_status kkt_solve_noalloc(ipm_ctx *c, const double *b, double *x) {
  if (!c || !b || !x) return IPM_ERR_ARG;
  if (c->sys) {  // the formulation's system (b, x: its order)
    const ipm_status st = kkt_solve_noalloc(c->sys, b, x);
    if (st != IPM_OK) c->err = c->sys->err;
    return st;
  }
  return guarded(c, [&]() -> ipm_status {
    if (c->state < 1) throw Fail{IPM_ERR_STATE, "kkt_solve_noalloc before kkt_analyze"};
    const size_t need = noalloc_need(c);
    if (need > kNoAllocDoubles)
      throw Fail{IPM_ERR_NOMEM, "kkt_solve_noalloc needs " + std::to_string(need) +
                                    " doubles of static scratch (n + update-vector entries + " +
                                    std::to_string(kRedBlocks * 8 + 32) + "); the limit is " +
                                    std::to_string(kNoAllocDoubles)};
    if (c->state < 4) throw Fail{IPM_ERR_STATE, "kkt_solve_noalloc before kkt_factor"};
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != c->device)
      throw Fail{IPM_ERR_ARG, "kkt_solve_noalloc called with device " + std::to_string(cur) +
                                  " current; the context's workspace is on device " +
                                  std::to_string(c->device)};
    double *base = noalloc_scratch(c->device);  // resolved by ipm_set_workspace
    double *partial = base;
    double *scal = base + (size_t)kRedBlocks * 8;
    double *y = scal + 32;
    double *t = y + std::max<int32_t>(c->P.n, 1);
    // every entry of y and t is written before it is read (permutation in,
    // then the gathers initialise each front's update vector): nothing to clear
    VecOps V{c->dp, c->st, partial};
    if (c->factor_prec == IPM_FP64) {
      V.permute_in<double>(b, nullptr, y);
      launch_solve<double, double>(c->dp, c->plan, (const double *)c->L, y, t, c->st);
      V.permute_out<double>(y, nullptr, x, false);
    } else {
      V.absmax(c->P.n, b, scal + 1);
      V.inv_scale(scal + 1, scal);
      float *yf = reinterpret_cast<float *>(y), *tf = reinterpret_cast<float *>(t);
      V.permute_in<float>(b, scal, yf);
      launch_solve<float, float>(c->dp, c->plan, (const float *)c->L, yf, tf, c->st);
      V.permute_out<float>(yf, scal, x, false);
    }
    CK(cudaGetLastError());
    return IPM_OK;
  });
}

}  // extern "C"
