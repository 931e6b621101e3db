// Launchers of the FP64 vector kernels (interior-point step, residuals, reductions).
#pragma once

#include "dev.cuh"

namespace gipm {

enum RedOp : int { RED_SUM = 0, RED_MAX = 1, RED_MIN = 2 };
struct RedOps {
  int op[8];
};

// Scalars of one interior-point iteration, kept in device memory so that the
// iteration needs no host round trip except the convergence test.
struct IpmScalars {
  double mu, mu_aff, sigma;
  double alpha_aff_p, alpha_aff_d, alpha_p, alpha_d;
  double primal_inf, dual_inf, compl_inf, fx;
  double pad[5];
};

// Loads the vector kernels the allocation-free solve launches (see capi.cu).
cudaError_t preload_vec_kernels();

constexpr int kRedBlocks = 304;  // fixed grid of the first reduction pass (2 per SM)

struct VecOps {
  DevPlan dp;
  cudaStream_t st;
  double *partial;  // kRedBlocks * 8 doubles

  void reduce_final(int ns, const RedOps &ops, double *out) const;
  void absmax(int64_t n, const double *v, double *out) const;
  void dot(int64_t n, const double *a, const double *b, double *out) const;
  void inv_scale(const double *absmax_v, double *scale) const;
  void jv(const double *jvals, const double *x, double *out) const;
  void jfull(const double *jx, const double *x, double *out) const;
  // out = base + sgn J^T v (+ W x)
  void jtv(const double *jvals, const double *v, double sgn, const double *wv, const double *x,
           const double *base, double *out) const;
  // s = max(g, 1), lambda = 1
  void init_slack(const double *gv, double *s, double *lam) const;
  // r = b - K x (matrix-free); tA: scratch of length m
  void residual(const double *jvals, const double *D, const double *wv, double delta_p,
                const double *x, const double *b, double *r, double *tA) const;
  // out_j = sum_i |K_ji| (matrix-free, D >= 0); tA: scratch of length m
  void abs_rowsum(const double *jvals, const double *D, const double *wv, double delta_p,
                  double *out, double *tA) const;
  template <typename V> void permute_in(const double *b, const double *scale, V *y) const;
  template <typename V>
  void permute_out(const V *y, const double *scale, double *x, bool accumulate) const;
  void kkt(const double *g, const double *s, const double *lam, const double *rd, const double *c,
           const double *wx, const double *x, double *red5, IpmScalars *sc) const;
  void g(const double *jx, const double *x, const double *b, const double *l, const double *u,
         double *gout) const;
  void scaling(const double *s, const double *lam, double delta_d, double *D) const;
  void rhs_rows(const double *D, const double *gv, const double *w, const double *lam,
                double *t) const;
  void negate(int64_t n, double *v) const;
  void recover(const double *D, const double *gv, const double *w, const double *s,
               const double *lam, const double *jdx, double *ds, double *dl) const;
  void ftb(const double *s, const double *ds, const double *lam, const double *dl, double *red2,
           IpmScalars *sc, bool affine) const;
  void muaff(const double *s, const double *ds, const double *lam, const double *dl,
             double *red1, IpmScalars *sc) const;
  void corrector_target(const double *ds, const double *dl, IpmScalars *sc, double *w) const;
  void update(const IpmScalars *sc, double *x, const double *dx, double *s, const double *ds,
              double *lam, const double *dl) const;
  // y += sign * (num/den) * x ;  p = x + (num/den) * p
  void axpy_ratio(int64_t n, const double *num, const double *den, int sign, const double *x,
                  double *y) const;
  void xpby_ratio(int64_t n, const double *num, const double *den, const double *x,
                  double *p) const;
};

}  // namespace gipm
