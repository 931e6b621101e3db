// Map kernels of the augmented (4) and dual condensed (6) formulations (see
// forms.h): the diagonal H, the values of the two systems' matrices and their
// right-hand sides. Every kernel is a grid-stride map over HBM-resident FP64
// vectors (coalesced except the gathers through J's CSC order and the bound
// rows).
#include <algorithm>

#include "forms.h"

namespace gipm {

namespace {

#define FORM_STRIDE(i, n)                                                              \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n);             \
       i += (int64_t)gridDim.x * blockDim.x)

inline int blocks_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

__global__ void hdiag_kernel(DevPlan dp, const double *__restrict__ wv,
                             const int64_t *__restrict__ wdiag, const double *__restrict__ D,
                             double delta_p, double *__restrict__ h) {
  FORM_STRIDE(j, dp.n) {
    double v = delta_p;
    if (dp.lpos[j] >= 0) v += D[dp.lpos[j]];
    if (dp.upos[j] >= 0) v += D[dp.upos[j]];
    if (wv && wdiag && wdiag[j] >= 0) v += wv[wdiag[j]];
    h[j] = v;
  }
}

__global__ void dual_values_kernel(DevPlan dp, int64_t nnz, const double *__restrict__ jv,
                                   const double *__restrict__ D, const double *__restrict__ h,
                                   double *__restrict__ Dp, double *__restrict__ jt,
                                   double *__restrict__ wd) {
  FORM_STRIDE(e, nnz) jt[e] = jv[dp.jtpos[e]];
  FORM_STRIDE(j, dp.n) Dp[j] = 1.0 / h[j];
  FORM_STRIDE(i, dp.m) wd[i] = 1.0 / D[i];
}

__global__ void aug_values_kernel(int64_t nnz, const int32_t *__restrict__ kind,
                                  const int64_t *__restrict__ idx, const double *__restrict__ h,
                                  const double *__restrict__ wv, const double *__restrict__ jv,
                                  const double *__restrict__ D, double *__restrict__ out) {
  FORM_STRIDE(k, nnz) {
    const int64_t e = idx[k];
    double v;
    switch (kind[k]) {
      case AUG_HDIAG: v = h[e]; break;
      case AUG_W: v = wv[e]; break;
      case AUG_J: v = jv[e]; break;
      default: v = -1.0 / D[e]; break;
    }
    out[k] = v;
  }
}

__global__ void rhs_rows_kernel(int64_t mt, int32_t m, const double *__restrict__ D,
                                const double *__restrict__ g, const double *__restrict__ w,
                                const double *__restrict__ lam, double *__restrict__ t,
                                double *__restrict__ q) {
  FORM_STRIDE(i, mt) {
    const double wl = w ? w[i] / lam[i] : 0.0;
    if (i < m) {
      t[i] = -lam[i];
      q[i] = g[i] - wl;
    } else {
      t[i] = D[i] * (g[i] - wl) - lam[i];
    }
  }
}

__global__ void div_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ h,
                           double sgn, double *__restrict__ out) {
  FORM_STRIDE(j, n) out[j] = sgn * a[j] / h[j];
}

__global__ void sub_kernel(int64_t k, const double *__restrict__ q, const double *__restrict__ ju,
                           double *__restrict__ out) {
  FORM_STRIDE(i, k) out[i] = q[i] - ju[i];
}

__global__ void neg_concat_kernel(const double *__restrict__ a, int64_t na,
                                  const double *__restrict__ b, int64_t nb,
                                  double *__restrict__ out) {
  FORM_STRIDE(i, na + nb) out[i] = i < na ? -a[i] : -b[i - na];
}

__global__ void pad_rows_kernel(int64_t mt, int32_t m, const double *__restrict__ y,
                                double *__restrict__ out) {
  FORM_STRIDE(i, mt) out[i] = i < m ? y[i] : 0.0;
}

// Residual of the augmented system (4) at (d_x, y): the first n rows and the
// last m rows.
__global__ void aug_res_n_kernel(int64_t n, const double *__restrict__ rt, const double *__restrict__ h,
                                 const double *__restrict__ dx, const double *__restrict__ aty,
                                 double *__restrict__ r1) {
  FORM_STRIDE(j, n) r1[j] = -rt[j] - h[j] * dx[j] - aty[j];
}
__global__ void aug_res_m_kernel(int64_t m, const double *__restrict__ q, const double *__restrict__ adx,
                                 const double *__restrict__ D, const double *__restrict__ y,
                                 double *__restrict__ r2) {
  FORM_STRIDE(i, m) r2[i] = -q[i] - adx[i] + y[i] / D[i];
}
__global__ void lincomb_kernel(int64_t k, double a, const double *__restrict__ x, double b,
                               const double *__restrict__ y, double *__restrict__ out) {
  FORM_STRIDE(i, k) out[i] = a * x[i] + b * y[i];
}

}  // namespace

void FormOps::aug_res_n(const double *rt, const double *h, const double *dx, const double *aty,
                        double *r1) const {
  note_launch();
  aug_res_n_kernel<<<blocks_for(dp.n), 256, 0, st>>>(dp.n, rt, h, dx, aty, r1);
}
void FormOps::aug_res_m(const double *q, const double *adx, const double *D, const double *y,
                        double *r2) const {
  if (dp.m <= 0) return;
  note_launch();
  aug_res_m_kernel<<<blocks_for(dp.m), 256, 0, st>>>(dp.m, q, adx, D, y, r2);
}
void FormOps::lincomb(int64_t k, double a, const double *x, double b, const double *y,
                      double *out) const {
  if (k <= 0) return;
  note_launch();
  lincomb_kernel<<<blocks_for(k), 256, 0, st>>>(k, a, x, b, y, out);
}

void FormOps::hdiag(const double *wv, const int64_t *wdiag, const double *D, double delta_p,
                    double *h) const {
  note_launch();
  hdiag_kernel<<<blocks_for(dp.n), 256, 0, st>>>(dp, wv, wdiag, D, delta_p, h);
}

void FormOps::dual_values(int64_t nnz, const double *jv, const double *D, const double *h,
                          double *Dp, double *jt, double *wd) const {
  const int64_t work = std::max<int64_t>({nnz, (int64_t)dp.n, (int64_t)dp.m, (int64_t)1});
  note_launch();
  dual_values_kernel<<<blocks_for(work), 256, 0, st>>>(dp, nnz, jv, D, h, Dp, jt, wd);
}

void FormOps::aug_values(int64_t nnz, const int32_t *kind, const int64_t *idx, const double *h,
                         const double *wv, const double *jv, const double *D, double *out) const {
  if (nnz <= 0) return;
  note_launch();
  aug_values_kernel<<<blocks_for(nnz), 256, 0, st>>>(nnz, kind, idx, h, wv, jv, D, out);
}

void FormOps::rhs_rows(const double *D, const double *g, const double *w, const double *lam,
                       double *t, double *q) const {
  if (dp.mt <= 0) return;
  note_launch();
  rhs_rows_kernel<<<blocks_for(dp.mt), 256, 0, st>>>(dp.mt, dp.m, D, g, w, lam, t, q);
}

void FormOps::div(const double *a, const double *h, double sgn, double *out) const {
  note_launch();
  div_kernel<<<blocks_for(dp.n), 256, 0, st>>>(dp.n, a, h, sgn, out);
}

void FormOps::sub(int64_t k, const double *q, const double *ju, double *out) const {
  if (k <= 0) return;
  note_launch();
  sub_kernel<<<blocks_for(k), 256, 0, st>>>(k, q, ju, out);
}

void FormOps::neg_concat(const double *a, int64_t na, const double *b, int64_t nb,
                         double *out) const {
  if (na + nb <= 0) return;
  note_launch();
  neg_concat_kernel<<<blocks_for(na + nb), 256, 0, st>>>(a, na, b, nb, out);
}

void FormOps::pad_rows(const double *y, double *out) const {
  if (dp.mt <= 0) return;
  note_launch();
  pad_rows_kernel<<<blocks_for(dp.mt), 256, 0, st>>>(dp.mt, dp.m, y, out);
}

}  // namespace gipm
