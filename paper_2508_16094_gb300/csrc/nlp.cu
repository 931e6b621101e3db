// Grid-NLP evaluation and line-search reductions (FP64). Reductions use a
// fixed grid and a fixed final order, so results are bit-reproducible.
#include <cfloat>

#include "nlp.h"

namespace gipm {

namespace {

constexpr int kT = 256;

#define NLP_GRID(i, n)                                                                   \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n);             \
       i += (int64_t)gridDim.x * blockDim.x)

inline int grid_for(int64_t n) {
  const int64_t g = (n + kT - 1) / kT;
  return (int)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

// block sums/maxes of NS slots -> partial[blockIdx.x * NS + k]
template <int NS>
__device__ void block_store(double (&v)[NS], const int (&ismax)[NS], double *partial) {
  __shared__ double sh[NS][kT / 32];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int k = 0; k < NS; k++) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = ismax[k] ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NS; k++) {
      double x = sh[k][0];
      for (int w = 1; w < kT / 32; w++) x = ismax[k] ? fmax(x, sh[k][w]) : x + sh[k][w];
      partial[blockIdx.x * NS + k] = x;
    }
}

template <int NS>
__global__ void final_kernel(const double *partial, int nb, int3 maxmask, double *out) {
  if (threadIdx.x != 0) return;
  const int mm[3] = {maxmask.x, maxmask.y, maxmask.z};
  for (int k = 0; k < NS; k++) {
    double x = mm[k] ? -DBL_MAX : 0.0;
    for (int b = 0; b < nb; b++) x = mm[k] ? fmax(x, partial[b * NS + k]) : x + partial[b * NS + k];
    out[k] = x;
  }
}

__global__ void eval_kernel(GridNlp p, const int64_t *__restrict__ jp, const double *__restrict__ x,
                            const double *__restrict__ ut, double *__restrict__ hrows,
                            double *__restrict__ jv, double *__restrict__ grad, double *partial) {
  const int N = p.N;
  const int64_t NN = p.NN();
  const double hinv2 = (double)(N + 1) * (double)(N + 1);
  double fsum[1] = {0.0};
  NLP_GRID(idx, NN) {
    const int ix = (int)(idx % N), iy = (int)(idx / N);
    const double u = x[idx], v = x[NN + idx];
    double nb = 0.0;
    if (iy > 0) nb += x[idx - N];
    if (ix > 0) nb += x[idx - 1];
    if (ix < N - 1) nb += x[idx + 1];
    if (iy < N - 1) nb += x[idx + N];
    const double hv = (4.0 * u - nb) * hinv2 + p.cubic * u * u * u - v;
    hrows[idx] = hv;
    hrows[NN + idx] = -hv;
    int64_t e = jp[idx], e2 = jp[NN + idx];
    auto put = [&](double w) {
      jv[e++] = w;
      jv[e2++] = -w;
    };
    if (iy > 0) put(-hinv2);
    if (ix > 0) put(-hinv2);
    put(4.0 * hinv2 + 3.0 * p.cubic * u * u);
    if (ix < N - 1) put(-hinv2);
    if (iy < N - 1) put(-hinv2);
    put(-1.0);
    const double du = u - ut[idx];
    grad[idx] = du;
    grad[NN + idx] = p.alpha * v;
    fsum[0] += 0.5 * du * du + 0.5 * p.alpha * v * v;
  }
  const int mx[1] = {0};
  block_store<1>(fsum, mx, partial);
}

__global__ void hess_kernel(GridNlp p, const double *__restrict__ x, const double *__restrict__ lam,
                            double *__restrict__ wv) {
  const int64_t NN = p.NN();
  NLP_GRID(idx, NN) {
    wv[idx] = 1.0 - 6.0 * p.cubic * x[idx] * (lam[idx] - lam[NN + idx]);
    wv[NN + idx] = p.alpha;
  }
}

__global__ void merit_kernel(int64_t mt, const double *__restrict__ s, const double *__restrict__ g,
                             double *partial) {
  double v[2] = {0.0, 0.0};
  NLP_GRID(k, mt) {
    v[0] += log(s[k]);
    v[1] += fabs(g[k] - s[k]);
  }
  const int mx[2] = {0, 0};
  block_store<2>(v, mx, partial);
}

// One-sided derivative of sum |g - s| along t = J dx - ds: sign(g - s) t where
// g != s, |t| where g == s.
__global__ void dtheta_kernel(int64_t mt, const double *__restrict__ g, const double *__restrict__ s,
                              const double *__restrict__ jdx, const double *__restrict__ ds,
                              double *partial) {
  double v[1] = {0.0};
  NLP_GRID(k, mt) {
    const double r = g[k] - s[k], t = jdx[k] - ds[k];
    v[0] += r > 0.0 ? t : (r < 0.0 ? -t : fabs(t));
  }
  const int mx[1] = {0};
  block_store<1>(v, mx, partial);
}

__global__ void dir_kernel(int64_t n, int64_t mt, const double *__restrict__ grad,
                           const double *__restrict__ dx, const double *__restrict__ s,
                           const double *__restrict__ ds, const double *__restrict__ lam,
                           const double *__restrict__ dl, double *partial) {
  double v[3] = {0.0, 0.0, 0.0};
  NLP_GRID(i, n + mt) {
    if (i < n) {
      v[0] = fma(grad[i], dx[i], v[0]);
    } else {
      const int64_t k = i - n;
      v[1] += ds[k] / s[k];
      v[2] = fmax(v[2], fabs(lam[k] + dl[k]));
    }
  }
  const int mx[3] = {0, 0, 1};
  block_store<3>(v, mx, partial);
}

__global__ void berr_kernel(int64_t mt, const double *__restrict__ s, const double *__restrict__ lam,
                            double mu, double *partial) {
  double v[1] = {0.0};
  NLP_GRID(k, mt) v[0] = fmax(v[0], fabs(s[k] * lam[k] - mu));
  const int mx[1] = {1};
  block_store<1>(v, mx, partial);
}

__global__ void trial_kernel(int64_t n, int64_t mt, const double *__restrict__ x,
                             const double *__restrict__ dx, const double *__restrict__ s,
                             const double *__restrict__ ds, double alpha, double *__restrict__ xt,
                             double *__restrict__ stv) {
  NLP_GRID(i, n + mt) {
    if (i < n) xt[i] = fma(alpha, dx[i], x[i]);
    else stv[i - n] = fma(alpha, ds[i - n], s[i - n]);
  }
}

__global__ void fill_kernel(int64_t n, double v, double *out) {
  NLP_GRID(i, n) out[i] = v;
}

}  // namespace

void grid_nlp_pattern(const GridNlp &p, std::vector<int64_t> &rowptr, std::vector<int32_t> &col) {
  const int N = p.N;
  const int64_t NN = p.NN();
  rowptr.assign(2 * NN + 1, 0);
  col.clear();
  col.reserve(12 * NN);
  for (int half = 0; half < 2; half++)
    for (int64_t idx = 0; idx < NN; idx++) {
      const int ix = (int)(idx % N), iy = (int)(idx / N);
      if (iy > 0) col.push_back((int32_t)(idx - N));
      if (ix > 0) col.push_back((int32_t)(idx - 1));
      col.push_back((int32_t)idx);
      if (ix < N - 1) col.push_back((int32_t)(idx + 1));
      if (iy < N - 1) col.push_back((int32_t)(idx + N));
      col.push_back((int32_t)(NN + idx));
      rowptr[half * NN + idx + 1] = (int64_t)col.size();
    }
}

void nlp_eval(const GridNlp &p, const int64_t *jp, const double *x, const double *ut,
              double *hrows, double *jv, double *grad, double *d_f, double *partial,
              cudaStream_t st) {
  note_launch();
  eval_kernel<<<kNlpRedBlocks, kT, 0, st>>>(p, jp, x, ut, hrows, jv, grad, partial);
  note_launch();
  final_kernel<1><<<1, 32, 0, st>>>(partial, kNlpRedBlocks, make_int3(0, 0, 0), d_f);
}

void nlp_hess(const GridNlp &p, const double *x, const double *lam, double *wv, cudaStream_t st) {
  note_launch();
  hess_kernel<<<grid_for(p.NN()), kT, 0, st>>>(p, x, lam, wv);
}

void nlp_merit_terms(int64_t mt, const double *s, const double *g, double *out, double *partial,
                     cudaStream_t st) {
  note_launch();
  merit_kernel<<<kNlpRedBlocks, kT, 0, st>>>(mt, s, g, partial);
  note_launch();
  final_kernel<2><<<1, 32, 0, st>>>(partial, kNlpRedBlocks, make_int3(0, 0, 0), out);
}

void nlp_dir_terms(int64_t n, int64_t mt, const double *grad, const double *dx, const double *s,
                   const double *ds, const double *lam, const double *dl, double *out,
                   double *partial, cudaStream_t st) {
  note_launch();
  dir_kernel<<<kNlpRedBlocks, kT, 0, st>>>(n, mt, grad, dx, s, ds, lam, dl, partial);
  note_launch();
  final_kernel<3><<<1, 32, 0, st>>>(partial, kNlpRedBlocks, make_int3(0, 0, 1), out);
}

void nlp_dtheta(int64_t mt, const double *g, const double *s, const double *jdx, const double *ds,
                double *out, double *partial, cudaStream_t st) {
  note_launch();
  dtheta_kernel<<<kNlpRedBlocks, kT, 0, st>>>(mt, g, s, jdx, ds, partial);
  note_launch();
  final_kernel<1><<<1, 32, 0, st>>>(partial, kNlpRedBlocks, make_int3(0, 0, 0), out);
}

void nlp_barrier_err(int64_t mt, const double *s, const double *lam, double mu, double *out,
                     double *partial, cudaStream_t st) {
  note_launch();
  berr_kernel<<<kNlpRedBlocks, kT, 0, st>>>(mt, s, lam, mu, partial);
  note_launch();
  final_kernel<1><<<1, 32, 0, st>>>(partial, kNlpRedBlocks, make_int3(1, 0, 0), out);
}

void nlp_trial(int64_t n, int64_t mt, const double *x, const double *dx, const double *s,
               const double *ds, double alpha, double *xt, double *stv, cudaStream_t st) {
  note_launch();
  trial_kernel<<<grid_for(n + mt), kT, 0, st>>>(n, mt, x, dx, s, ds, alpha, xt, stv);
}

void nlp_fill(int64_t n, double v, double *out, cudaStream_t st) {
  note_launch();
  fill_kernel<<<grid_for(n), kT, 0, st>>>(n, v, out);
}

}  // namespace gipm
