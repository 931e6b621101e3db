// Grid NLP: problem evaluation (f, h, J values, grad f, Hessian of the
// Lagrangian) and the map/reduce pieces of its line search, all FP64.
#pragma once

#include <vector>

#include "dev.cuh"

namespace gipm {

struct GridNlp {
  int N = 0;
  double alpha = 0.0, v_lo = -1.0, v_hi = 1.0;
  int cubic = 1, v_bounded = 1;
  __host__ __device__ int64_t NN() const { return (int64_t)N * N; }
};

// J pattern of [h; -h]: per grid point (ix, iy) the u columns of the five-point
// stencil inside the grid in ascending order, then its v column; rows NN..
// repeat rows 0..NN-1.
void grid_nlp_pattern(const GridNlp &p, std::vector<int64_t> &rowptr, std::vector<int32_t> &col);

constexpr int kNlpRedBlocks = 304;

// hrows (2 NN) = [h; -h], jv (pattern order), grad (2 NN) and f (device scalar)
void nlp_eval(const GridNlp &p, const int64_t *jp, const double *x, const double *ut,
              double *hrows, double *jv, double *grad, double *d_f, double *partial,
              cudaStream_t st);
// wv (2 NN): diag(1 - 6 c3 u (lambda+ - lambda-), alpha)
void nlp_hess(const GridNlp &p, const double *x, const double *lam, double *wv, cudaStream_t st);
// out[0] = sum ln s, out[1] = sum |g - s|
void nlp_merit_terms(int64_t mt, const double *s, const double *g, double *out, double *partial,
                     cudaStream_t st);
// out[0] = grad . dx, out[1] = sum ds / s, out[2] = max |lambda + dlambda|
void nlp_dir_terms(int64_t n, int64_t mt, const double *grad, const double *dx, const double *s,
                   const double *ds, const double *lam, const double *dl, double *out,
                   double *partial, cudaStream_t st);
// out[0] = one-sided derivative of sum |g - s| along (J dx - ds): sum of
// sign(g - s) (J dx - ds) over rows with g != s plus |J dx - ds| over the rest
void nlp_dtheta(int64_t mt, const double *g, const double *s, const double *jdx, const double *ds,
                double *out, double *partial, cudaStream_t st);
// out[0] = max |s lambda - mu|
void nlp_barrier_err(int64_t mt, const double *s, const double *lam, double mu, double *out,
                     double *partial, cudaStream_t st);
// xt = x + alpha dx, st = s + alpha ds
void nlp_trial(int64_t n, int64_t mt, const double *x, const double *dx, const double *s,
               const double *ds, double alpha, double *xt, double *stv, cudaStream_t st);
void nlp_fill(int64_t n, double v, double *out, cudaStream_t st);

}  // namespace gipm
