// Map kernels of the augmented (4) and dual condensed (6) formulations of the
// Newton system (3) (Sec. 3, "Condensed KKT Systems"). The bound rows (Jacobian
// rows +-e_i) are folded into the (1,1) block H = W + delta_p I + D_l + D_u; the
// m general rows keep a multiplier block:
//   (4)  [H, A^T; A, -D_G^{-1}] [d_x; y] = -[r~; q]
//   (6)  (D_G^{-1} + A H^{-1} A^T) y = q - A H^{-1} r~,  d_x = -H^{-1} (r~ + A^T y)
// with y = -d_lambda_G, q = g_G - w_G / lambda_G and
//   r~ = grad f - J^T lambda + J_B^T D_B (g_B - w_B / lambda_B).
// Both give the d_x of the primal condensed system (5).
#pragma once

#include "dev.cuh"

namespace gipm {

// Source of one value of the augmented matrix (lower CSC of order n + m).
enum AugSource : int32_t {
  AUG_HDIAG = 0,  // (j, j), j < n: H_jj (W_jj included)
  AUG_W = 1,      // an off-diagonal entry of W (index into W's values)
  AUG_J = 2,      // (n + i, j): A_ij (index into J's CSR values)
  AUG_DINV = 3    // (n + i, n + i): -1 / D_i
};

struct FormOps {
  DevPlan dp;  // the outer problem's structure (J, W, bounds)
  cudaStream_t st;

  // H_jj = delta_p + D_l + D_u (+ W_jj at wdiag[j] >= 0), length n.
  void hdiag(const double *wv, const int64_t *wdiag, const double *D, double delta_p,
             double *h) const;
  // Dual system inputs: Dp = 1 / H (n), jt = J's nnz values in the CSC order
  // of J (the CSR order of J^T), wd = 1 / D_G (m).
  void dual_values(int64_t nnz, const double *jv, const double *D, const double *h, double *Dp,
                   double *jt, double *wd) const;
  // Augmented values: out[k] from (kind[k], idx[k]).
  void aug_values(int64_t nnz, const int32_t *kind, const int64_t *idx, const double *h,
                  const double *wv, const double *jv, const double *D, double *out) const;
  // t (m_tot) = -lambda on the general rows, D (g - w / lambda) - lambda on the
  // bound rows; q (m) = g - w / lambda on the general rows (w may be null).
  void rhs_rows(const double *D, const double *g, const double *w, const double *lam, double *t,
                double *q) const;
  // out = sgn * a / h (n)
  void div(const double *a, const double *h, double sgn, double *out) const;
  // out (m) = q - ju
  void sub(int64_t k, const double *q, const double *ju, double *out) const;
  // out = [-a (n); -b (m)]
  void neg_concat(const double *a, int64_t na, const double *b, int64_t nb, double *out) const;
  // out (m_tot) = [y (m); 0]
  void pad_rows(const double *y, double *out) const;
  // residual of (4) at (d_x, y): r1 = -r~ - H d_x - A^T y (n), r2 = -q - A d_x +
  // D_G^{-1} y (m)
  void aug_res_n(const double *rt, const double *h, const double *dx, const double *aty,
                 double *r1) const;
  void aug_res_m(const double *q, const double *adx, const double *D, const double *y,
                 double *r2) const;
  // out = a x + b y (k entries; out may alias x or y)
  void lincomb(int64_t k, double a, const double *x, double b, const double *y,
               double *out) const;
};

}  // namespace gipm
