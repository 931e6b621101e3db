// FP64 map/reduce kernels of the interior-point iteration (Sec. 1: line search
// and barrier updates are map or reduce operations) and of the matrix-free
// residual used by iterative refinement. Reductions are two-pass with a fixed
// grid, so every result is bit-reproducible.
#include <cfloat>

#include "ipm_kernels.h"

namespace gipm {

namespace {

constexpr int kRedBlock = 256;

__device__ __forceinline__ double red_combine(double a, double b, int op) {
  return op == RED_SUM ? a + b : (op == RED_MAX ? fmax(a, b) : fmin(a, b));
}
__device__ __forceinline__ double red_identity(int op) {
  return op == RED_SUM ? 0.0 : (op == RED_MAX ? -DBL_MAX : DBL_MAX);
}

// Block-level reduction of NS slots; thread 0 writes partial[blockIdx.x * NS + k].
template <int NS>
__device__ void block_reduce_store(double (&v)[NS], const RedOps &ops, double *partial) {
  __shared__ double sh[NS][kRedBlock / 32];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int k = 0; k < NS; k++) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = red_combine(x, __shfl_xor_sync(0xffffffffu, x, o), ops.op[k]);
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NS; k++) {
      double x = sh[k][0];
      for (int w = 1; w < kRedBlock / 32; w++) x = red_combine(x, sh[k][w], ops.op[k]);
      partial[blockIdx.x * NS + k] = x;
    }
  }
}

template <int NS>
__global__ void final_reduce_kernel(const double *partial, int nblocks, RedOps ops, double *out) {
  double v[NS];
#pragma unroll
  for (int k = 0; k < NS; k++) v[k] = red_identity(ops.op[k]);
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NS; k++) v[k] = red_combine(v[k], partial[b * NS + k], ops.op[k]);
  __shared__ double sh[NS][kRedBlock];
#pragma unroll
  for (int k = 0; k < NS; k++) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NS; k++) {
      double x = sh[k][0];
      for (int t = 1; t < kRedBlock; t++) x = red_combine(x, sh[k][t], ops.op[k]);
      out[k] = x;
    }
  }
}

#define GRID_STRIDE(i, n)                                                              \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n);             \
       i += (int64_t)gridDim.x * blockDim.x)

inline int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

// ---------------------------------------------------------------------------
__global__ void jv_kernel(DevPlan dp, const double *__restrict__ jv, const double *__restrict__ x,
                          double *__restrict__ out) {
  GRID_STRIDE(r, dp.m) {
    double a = 0.0;
    for (int64_t e = dp.jp[r]; e < dp.jp[r + 1]; e++) a = fma(jv[e], x[dp.ji[e]], a);
    out[r] = a;
  }
}

// out[j] = base_j + sgn * (J^T v)_j + (W x)_j  (v has length m_tot: general rows,
// then lower-bound rows (+e_i), then upper-bound rows (-e_i))
__global__ void jtv_kernel(DevPlan dp, const double *__restrict__ jv, const double *__restrict__ v,
                           double sgn, const double *__restrict__ wv, const double *__restrict__ x,
                           const double *__restrict__ base, double *__restrict__ out) {
  GRID_STRIDE(j, dp.n) {
    double a = 0.0;
    for (int64_t t = dp.jtp[j]; t < dp.jtp[j + 1]; t++) {
      const int32_t e = dp.jtpos[t];
      a = fma(jv[e], v[dp.jrow[e]], a);
    }
    if (dp.lpos[j] >= 0) a += v[dp.lpos[j]];
    if (dp.upos[j] >= 0) a -= v[dp.upos[j]];
    a = sgn * a + (base ? base[j] : 0.0);
    if (wv && x)
      for (int64_t e = dp.wfp[j]; e < dp.wfp[j + 1]; e++) a = fma(wv[dp.wfsrc[e]], x[dp.wfi[e]], a);
    out[j] = a;
  }
}
__global__ void init_slack_kernel(int64_t mt, const double *__restrict__ g, double *__restrict__ s,
                                  double *__restrict__ lam) {
  GRID_STRIDE(k, mt) {
    s[k] = fmax(g[k], 1.0);
    lam[k] = 1.0;
  }
}

// (J x) for all m_tot rows: general rows from jx, bound rows +-x
__global__ void jfull_kernel(DevPlan dp, const double *__restrict__ jx, const double *__restrict__ x,
                             double *__restrict__ out) {
  GRID_STRIDE(k, dp.mt) {
    double v;
    if (k < dp.m) v = jx[k];
    else if (k < dp.m + dp.nl) v = x[dp.lidx[k - dp.m]];
    else v = -x[dp.uidx[k - dp.m - dp.nl]];
    out[k] = v;
  }
}

// residual r = b - K x with K = W + J_A^T D_A J_A + diag(D_l + D_u) + delta_p I
__global__ void resid_rows_kernel(DevPlan dp, const double *__restrict__ jv,
                                  const double *__restrict__ D, const double *__restrict__ x,
                                  double *__restrict__ tA) {
  GRID_STRIDE(r, dp.m) {
    double a = 0.0;
    for (int64_t e = dp.jp[r]; e < dp.jp[r + 1]; e++) a = fma(jv[e], x[dp.ji[e]], a);
    tA[r] = D[r] * a;
  }
}
__global__ void resid_cols_kernel(DevPlan dp, const double *__restrict__ jv,
                                  const double *__restrict__ D, const double *__restrict__ wv,
                                  double delta_p, const double *__restrict__ tA,
                                  const double *__restrict__ x, const double *__restrict__ b,
                                  double *__restrict__ r) {
  GRID_STRIDE(j, dp.n) {
    double a = 0.0;
    for (int64_t t = dp.jtp[j]; t < dp.jtp[j + 1]; t++) {
      const int32_t e = dp.jtpos[t];
      a = fma(jv[e], tA[dp.jrow[e]], a);
    }
    double d = delta_p;
    if (dp.lpos[j] >= 0) d += D[dp.lpos[j]];
    if (dp.upos[j] >= 0) d += D[dp.upos[j]];
    a = fma(d, x[j], a);
    if (wv)
      for (int64_t e = dp.wfp[j]; e < dp.wfp[j + 1]; e++) a = fma(wv[dp.wfsrc[e]], x[dp.wfi[e]], a);
    r[j] = b[j] - a;
  }
}

// row sums of |K|: |W| 1 + |J_A|^T D_A |J_A| 1 + D_l + D_u + delta_p (D >= 0)
__global__ void absk_rows_kernel(DevPlan dp, const double *__restrict__ jv,
                                 const double *__restrict__ D, double *__restrict__ tA) {
  GRID_STRIDE(r, dp.m) {
    double a = 0.0;
    for (int64_t e = dp.jp[r]; e < dp.jp[r + 1]; e++) a += fabs(jv[e]);
    tA[r] = D[r] * a;
  }
}
__global__ void absk_cols_kernel(DevPlan dp, const double *__restrict__ jv,
                                 const double *__restrict__ D, const double *__restrict__ wv,
                                 double delta_p, const double *__restrict__ tA,
                                 double *__restrict__ out) {
  GRID_STRIDE(j, dp.n) {
    double a = 0.0;
    for (int64_t t = dp.jtp[j]; t < dp.jtp[j + 1]; t++) {
      const int32_t e = dp.jtpos[t];
      a = fma(fabs(jv[e]), tA[dp.jrow[e]], a);
    }
    double d = fabs(delta_p);
    if (dp.lpos[j] >= 0) d += D[dp.lpos[j]];
    if (dp.upos[j] >= 0) d += D[dp.upos[j]];
    a += d;
    if (wv)
      for (int64_t e = dp.wfp[j]; e < dp.wfp[j + 1]; e++) a += fabs(wv[dp.wfsrc[e]]);
    out[j] = a;
  }
}
template <typename V>
__global__ void permute_in_kernel(int32_t n, const int32_t *__restrict__ perm,
                                  const double *__restrict__ b, const double *__restrict__ scale,
                                  V *__restrict__ y) {
  const double s = scale ? scale[0] : 1.0;
  GRID_STRIDE(k, n) y[k] = (V)(b[perm[k]] * s);
}
template <typename V>
__global__ void permute_out_kernel(int32_t n, const int32_t *__restrict__ perm,
                                   const V *__restrict__ y, const double *__restrict__ scale,
                                   double *__restrict__ x, int accumulate) {
  const double s = scale ? 1.0 / scale[0] : 1.0;
  GRID_STRIDE(k, n) {
    const double v = (double)y[k] * s;
    if (accumulate) x[perm[k]] += v;
    else x[perm[k]] = v;
  }
}

// ---- reductions -----------------------------------------------------------
__global__ void absmax_kernel(int64_t n, const double *__restrict__ v, double *partial) {
  double a[1] = {0.0};
  GRID_STRIDE(i, n) a[0] = fmax(a[0], fabs(v[i]));
  RedOps ops{{RED_MAX}};
  block_reduce_store<1>(a, ops, partial);
}
__global__ void dot_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                           double *partial) {
  double v[1] = {0.0};
  GRID_STRIDE(i, n) v[0] = fma(a[i], b[i], v[0]);
  RedOps ops{{RED_SUM}};
  block_reduce_store<1>(v, ops, partial);
}
__global__ void inv_scale_kernel(const double *absmax, double *scale) {
  // scale = 1 / max|v| (1 if zero): keeps low-precision right-hand sides in range
  const double m = absmax[0];
  scale[0] = (m > 0.0 && m < DBL_MAX) ? 1.0 / m : 1.0;
}

// KKT quantities: slots 0 sum s.lambda, 1 max|g - s|, 2 max|s.lambda|, 3 max|rd|, 4 f(x)
__global__ void kkt_reduce_kernel(DevPlan dp, const double *__restrict__ g,
                                  const double *__restrict__ s, const double *__restrict__ lam,
                                  const double *__restrict__ rd, const double *__restrict__ c,
                                  const double *__restrict__ wx, const double *__restrict__ x,
                                  double *partial) {
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  GRID_STRIDE(i, dp.mt + dp.n) {
    if (i < dp.mt) {
      const double sl = s[i] * lam[i];
      v[0] += sl;
      v[1] = fmax(v[1], fabs(g[i] - s[i]));
      v[2] = fmax(v[2], fabs(sl));
    } else {
      const int64_t j = i - dp.mt;
      v[3] = fmax(v[3], fabs(rd[j]));
      v[4] = fma(c[j] + (wx ? 0.5 * wx[j] : 0.0), x[j], v[4]);
    }
  }
  RedOps ops{{RED_SUM, RED_MAX, RED_MAX, RED_MAX, RED_SUM}};
  block_reduce_store<5>(v, ops, partial);
}

// fraction to the boundary: slot 0 min over ds<0 of -s/ds, slot 1 min over dl<0 of -lam/dl
__global__ void ftb_kernel(int64_t mt, const double *__restrict__ s, const double *__restrict__ ds,
                           const double *__restrict__ lam, const double *__restrict__ dl,
                           double *partial) {
  double v[2] = {DBL_MAX, DBL_MAX};
  GRID_STRIDE(i, mt) {
    if (ds[i] < 0.0) v[0] = fmin(v[0], -s[i] / ds[i]);
    if (dl[i] < 0.0) v[1] = fmin(v[1], -lam[i] / dl[i]);
  }
  RedOps ops{{RED_MIN, RED_MIN}};
  block_reduce_store<2>(v, ops, partial);
}

__global__ void muaff_kernel(int64_t mt, const double *__restrict__ s, const double *__restrict__ ds,
                             const double *__restrict__ lam, const double *__restrict__ dl,
                             const IpmScalars *sc, double *partial) {
  const double ap = sc->alpha_aff_p, ad = sc->alpha_aff_d;
  double v[1] = {0.0};
  GRID_STRIDE(i, mt) v[0] = fma(fma(ap, ds[i], s[i]), fma(ad, dl[i], lam[i]), v[0]);
  RedOps ops{{RED_SUM}};
  block_reduce_store<1>(v, ops, partial);
}

// ---- elementwise steps ---------------------------------------------------
// g = J x - bfull from (J x) of the general rows
__global__ void g_kernel(DevPlan dp, const double *__restrict__ jx, const double *__restrict__ x,
                         const double *__restrict__ b, const double *__restrict__ l,
                         const double *__restrict__ u, double *__restrict__ g) {
  GRID_STRIDE(k, dp.mt) {
    double v;
    if (k < dp.m) v = jx[k] - b[k];
    else if (k < dp.m + dp.nl) { const int32_t i = dp.lidx[k - dp.m]; v = x[i] - l[i]; }
    else { const int32_t i = dp.uidx[k - dp.m - dp.nl]; v = u[i] - x[i]; }
    g[k] = v;
  }
}
__global__ void scaling_kernel(int64_t mt, const double *__restrict__ s,
                               const double *__restrict__ lam, double delta_d,
                               double *__restrict__ D) {
  GRID_STRIDE(k, mt) D[k] = 1.0 / (delta_d + s[k] / lam[k]);
}
// t = D (g - w/lambda) - lambda   (w may be NULL: zero)
__global__ void rhs_rows_kernel(int64_t mt, const double *__restrict__ D, const double *__restrict__ g,
                                const double *__restrict__ w, const double *__restrict__ lam,
                                double *__restrict__ t) {
  GRID_STRIDE(k, mt) {
    const double wl = w ? w[k] / lam[k] : 0.0;
    t[k] = D[k] * (g[k] - wl) - lam[k];
  }
}
__global__ void negate_kernel(int64_t n, double *__restrict__ v) {
  GRID_STRIDE(i, n) v[i] = -v[i];
}
// d_lambda = D (w/lambda - g - J d_x);  d_s = -s + w/lambda - (s/lambda) d_lambda
__global__ void recover_kernel(int64_t mt, const double *__restrict__ D, const double *__restrict__ g,
                               const double *__restrict__ w, const double *__restrict__ s,
                               const double *__restrict__ lam, const double *__restrict__ jdx,
                               double *__restrict__ ds, double *__restrict__ dl) {
  GRID_STRIDE(k, mt) {
    const double wl = w ? w[k] / lam[k] : 0.0;
    const double d = D[k] * (wl - g[k] - jdx[k]);
    dl[k] = d;
    ds[k] = -s[k] + wl - (s[k] / lam[k]) * d;
  }
}
// w = sigma mu - ds_aff .* dl_aff, with sigma = (mu_aff / mu)^3 computed here
__global__ void corrector_target_kernel(int64_t mt, const double *__restrict__ ds,
                                        const double *__restrict__ dl, IpmScalars *sc,
                                        double *__restrict__ w) {
  const double mu = sc->mu, ratio = sc->mu_aff / mu;
  const double sm = ratio * ratio * ratio * mu;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->sigma = ratio * ratio * ratio;
  GRID_STRIDE(k, mt) w[k] = sm - ds[k] * dl[k];
}
__global__ void update_kernel(int64_t n, int64_t mt, const IpmScalars *sc, double *__restrict__ x,
                              const double *__restrict__ dx, double *__restrict__ s,
                              const double *__restrict__ ds, double *__restrict__ lam,
                              const double *__restrict__ dl) {
  const double ap = sc->alpha_p, ad = sc->alpha_d;
  GRID_STRIDE(i, n + mt) {
    if (i < n) x[i] = fma(ap, dx[i], x[i]);
    else {
      const int64_t k = i - n;
      s[k] = fma(ap, ds[k], s[k]);
      lam[k] = fma(ad, dl[k], lam[k]);
    }
  }
}
// scalar bookkeeping after reductions
__global__ void finish_kkt_kernel(const double *red, int64_t mt, IpmScalars *sc) {
  sc->mu = red[0] / (double)(mt > 0 ? mt : 1);
  sc->primal_inf = red[1];
  sc->compl_inf = red[2];
  sc->dual_inf = red[3];
  sc->fx = red[4];
}
__global__ void finish_ftb_kernel(const double *red, IpmScalars *sc, int affine) {
  if (affine) {
    sc->alpha_aff_p = fmin(1.0, red[0]);
    sc->alpha_aff_d = fmin(1.0, red[1]);
  } else {
    const double tau = fmax(0.99, 1.0 - sc->mu);
    sc->alpha_p = fmin(1.0, tau * red[0]);
    sc->alpha_d = fmin(1.0, tau * red[1]);
  }
}
__global__ void finish_muaff_kernel(const double *red, int64_t mt, IpmScalars *sc) {
  sc->mu_aff = red[0] / (double)(mt > 0 ? mt : 1);
}

// ---- vector updates used by refinement / PCG ------------------------------
__global__ void axpy_dev_kernel(int64_t n, const double *alpha_num, const double *alpha_den,
                                int sign, const double *__restrict__ xv, double *__restrict__ yv) {
  const double a = (alpha_den[0] != 0.0) ? sign * alpha_num[0] / alpha_den[0] : 0.0;
  GRID_STRIDE(i, n) yv[i] = fma(a, xv[i], yv[i]);
}
__global__ void xpby_dev_kernel(int64_t n, const double *num, const double *den,
                                const double *__restrict__ xv, double *__restrict__ p) {
  const double b = (den[0] != 0.0) ? num[0] / den[0] : 0.0;
  GRID_STRIDE(i, n) p[i] = fma(b, p[i], xv[i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Load the kernels of the allocation-free solve now (a function query loads a
// lazily loaded kernel), so that its later launches commit no device memory.
cudaError_t preload_vec_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess;
  auto q = [&](const void *f) { if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, f); };
  q((const void *)permute_in_kernel<double>);
  q((const void *)permute_in_kernel<float>);
  q((const void *)permute_out_kernel<double>);
  q((const void *)permute_out_kernel<float>);
  q((const void *)absmax_kernel);
  q((const void *)inv_scale_kernel);
  q((const void *)final_reduce_kernel<1>);
  return e;
}

void VecOps::reduce_final(int ns, const RedOps &ops, double *out) const {
  switch (ns) {
    case 1: { note_launch(); final_reduce_kernel<1><<<1, kRedBlock, 0, st>>>(partial, kRedBlocks, ops, out); } break;
    case 2: { note_launch(); final_reduce_kernel<2><<<1, kRedBlock, 0, st>>>(partial, kRedBlocks, ops, out); } break;
    case 5: { note_launch(); final_reduce_kernel<5><<<1, kRedBlock, 0, st>>>(partial, kRedBlocks, ops, out); } break;
    default: break;
  }
}
void VecOps::absmax(int64_t n, const double *v, double *out) const {
  { note_launch(); absmax_kernel<<<kRedBlocks, kRedBlock, 0, st>>>(n, v, partial); }
  reduce_final(1, RedOps{{RED_MAX}}, out);
}
void VecOps::dot(int64_t n, const double *a, const double *b, double *out) const {
  { note_launch(); dot_kernel<<<kRedBlocks, kRedBlock, 0, st>>>(n, a, b, partial); }
  reduce_final(1, RedOps{{RED_SUM}}, out);
}
void VecOps::inv_scale(const double *absmax_v, double *scale) const {
  { note_launch(); inv_scale_kernel<<<1, 1, 0, st>>>(absmax_v, scale); }
}
void VecOps::jv(const double *jvals, const double *x, double *out) const {
  if (dp.m > 0) { note_launch(); jv_kernel<<<grid_of(dp.m), 256, 0, st>>>(dp, jvals, x, out); }
}
void VecOps::jfull(const double *jx, const double *x, double *out) const {
  if (dp.mt > 0) { note_launch(); jfull_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp, jx, x, out); }
}
void VecOps::jtv(const double *jvals, const double *v, double sgn, const double *wv,
                 const double *x, const double *base, double *out) const {
  { note_launch(); jtv_kernel<<<grid_of(dp.n), 256, 0, st>>>(dp, jvals, v, sgn, wv, x, base, out); }
}
void VecOps::init_slack(const double *gv, double *s, double *lam) const {
  if (dp.mt > 0) { note_launch(); init_slack_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp.mt, gv, s, lam); }
}
void VecOps::residual(const double *jvals, const double *D, const double *wv, double delta_p,
                      const double *x, const double *b, double *r, double *tA) const {
  if (dp.m > 0) { note_launch(); resid_rows_kernel<<<grid_of(dp.m), 256, 0, st>>>(dp, jvals, D, x, tA); }
  { note_launch(); resid_cols_kernel<<<grid_of(dp.n), 256, 0, st>>>(dp, jvals, D, wv, delta_p, tA, x, b, r); }
}
void VecOps::abs_rowsum(const double *jvals, const double *D, const double *wv, double delta_p,
                        double *out, double *tA) const {
  if (dp.m > 0) { note_launch(); absk_rows_kernel<<<grid_of(dp.m), 256, 0, st>>>(dp, jvals, D, tA); }
  { note_launch(); absk_cols_kernel<<<grid_of(dp.n), 256, 0, st>>>(dp, jvals, D, wv, delta_p, tA, out); }
}
template <typename V>
void VecOps::permute_in(const double *b, const double *scale, V *y) const {
  { note_launch(); permute_in_kernel<V><<<grid_of(dp.n), 256, 0, st>>>(dp.n, dp.perm, b, scale, y); }
}
template <typename V>
void VecOps::permute_out(const V *y, const double *scale, double *x, bool accumulate) const {
  { note_launch(); permute_out_kernel<V><<<grid_of(dp.n), 256, 0, st>>>(dp.n, dp.perm, y, scale, x, accumulate); }
}
template void VecOps::permute_in<double>(const double *, const double *, double *) const;
template void VecOps::permute_in<float>(const double *, const double *, float *) const;
template void VecOps::permute_out<double>(const double *, const double *, double *, bool) const;
template void VecOps::permute_out<float>(const float *, const double *, double *, bool) const;

void VecOps::kkt(const double *g, const double *s, const double *lam, const double *rd,
                 const double *c, const double *wx, const double *x, double *red5,
                 IpmScalars *sc) const {
  { note_launch(); kkt_reduce_kernel<<<kRedBlocks, kRedBlock, 0, st>>>(dp, g, s, lam, rd, c, wx, x, partial); }
  reduce_final(5, RedOps{{RED_SUM, RED_MAX, RED_MAX, RED_MAX, RED_SUM}}, red5);
  { note_launch(); finish_kkt_kernel<<<1, 1, 0, st>>>(red5, dp.mt, sc); }
}
void VecOps::g(const double *jx, const double *x, const double *b, const double *l,
               const double *u, double *gout) const {
  if (dp.mt > 0) { note_launch(); g_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp, jx, x, b, l, u, gout); }
}
void VecOps::scaling(const double *s, const double *lam, double delta_d, double *D) const {
  if (dp.mt > 0) { note_launch(); scaling_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp.mt, s, lam, delta_d, D); }
}
void VecOps::rhs_rows(const double *D, const double *gv, const double *w, const double *lam,
                      double *t) const {
  if (dp.mt > 0) { note_launch(); rhs_rows_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp.mt, D, gv, w, lam, t); }
}
void VecOps::negate(int64_t n, double *v) const {
  { note_launch(); negate_kernel<<<grid_of(n), 256, 0, st>>>(n, v); }
}
void VecOps::recover(const double *D, const double *gv, const double *w, const double *s,
                     const double *lam, const double *jdx, double *ds, double *dl) const {
  if (dp.mt > 0)
    { note_launch(); recover_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp.mt, D, gv, w, s, lam, jdx, ds, dl); }
}
void VecOps::ftb(const double *s, const double *ds, const double *lam, const double *dl,
                 double *red2, IpmScalars *sc, bool affine) const {
  { note_launch(); ftb_kernel<<<kRedBlocks, kRedBlock, 0, st>>>(dp.mt, s, ds, lam, dl, partial); }
  reduce_final(2, RedOps{{RED_MIN, RED_MIN}}, red2);
  { note_launch(); finish_ftb_kernel<<<1, 1, 0, st>>>(red2, sc, affine ? 1 : 0); }
}
void VecOps::muaff(const double *s, const double *ds, const double *lam, const double *dl,
                   double *red1, IpmScalars *sc) const {
  { note_launch(); muaff_kernel<<<kRedBlocks, kRedBlock, 0, st>>>(dp.mt, s, ds, lam, dl, sc, partial); }
  reduce_final(1, RedOps{{RED_SUM}}, red1);
  { note_launch(); finish_muaff_kernel<<<1, 1, 0, st>>>(red1, dp.mt, sc); }
}
void VecOps::corrector_target(const double *ds, const double *dl, IpmScalars *sc,
                              double *w) const {
  { note_launch(); corrector_target_kernel<<<grid_of(dp.mt), 256, 0, st>>>(dp.mt, ds, dl, sc, w); }
}
void VecOps::update(const IpmScalars *sc, double *x, const double *dx, double *s,
                    const double *ds, double *lam, const double *dl) const {
  { note_launch(); update_kernel<<<grid_of(dp.n + dp.mt), 256, 0, st>>>(dp.n, dp.mt, sc, x, dx, s, ds, lam, dl); }
}
void VecOps::axpy_ratio(int64_t n, const double *num, const double *den, int sign,
                        const double *x, double *y) const {
  { note_launch(); axpy_dev_kernel<<<grid_of(n), 256, 0, st>>>(n, num, den, sign, x, y); }
}
void VecOps::xpby_ratio(int64_t n, const double *num, const double *den, const double *x,
                        double *p) const {
  { note_launch(); xpby_dev_kernel<<<grid_of(n), 256, 0, st>>>(n, num, den, x, p); }
}

}  // namespace gipm
