// Supernodal triangular solves with the multifrontal factor (Sec. 2: once
// pivoting is gone, the triangular solves run on the GPU; level scheduling
// over the elimination tree, Naumov's parallel sparse triangular solve).
//
// Forward (L y = b), levels ascending. Each front first gathers its children's
// update vectors (entries on its own columns are subtracted from y, entries on
// its rows below are summed into its own update vector), then block column by
// block column: solve the diagonal block, then warp-cooperative dot products
// with the rows below (its own later columns -> y, rows below -> update vector).
// Backward (L^T x = y), levels descending: subtract L21^T x(rows below) with a
// fixed-order reduction, then block columns from last to first: solve the
// transposed diagonal block and update the columns to its left.
#include <algorithm>

#include "launch.h"

namespace gipm {

namespace {

// Substitution with one diagonal block (jb <= 64, lower triangle in Lb) on one
// warp: lane l holds y_l and y_{l+32}; each step finishes y_c on its lane,
// broadcasts it by shuffle and updates the rows still open (forward: rows
// below c with L_ic; backward, L^T: rows above c with L_ci). With `recip`
// (FP64 without pivot signs) y_c is multiplied by 1 / L_cc formed before the
// chain, otherwise divided by L_cc, keeping the FP32 and signed solves' rounding.
template <typename V, bool FWD>
__device__ __forceinline__ void diag_chain(const V (*Lb)[65], V *yb, int jb, int lane, bool recip) {
  V y0 = lane < jb ? yb[lane] : V(0), y1 = lane + 32 < jb ? yb[lane + 32] : V(0);
  V d0 = lane < jb ? Lb[lane][lane] : V(1), d1 = lane + 32 < jb ? Lb[lane + 32][lane + 32] : V(1);
  if (recip) {
    d0 = V(1) / d0;
    d1 = V(1) / d1;
  }
  for (int s = 0; s < jb; s++) {
    const int c = FWD ? s : jb - 1 - s, src = c & 31;
    const bool hi = c >= 32;
    if (lane == src) {
      if (hi) y1 = recip ? y1 * d1 : y1 / d1;
      else y0 = recip ? y0 * d0 : y0 / d0;
    }
    const V yc = __shfl_sync(0xFFFFFFFFu, hi ? y1 : y0, src);
    if (FWD) {
      if (lane > c && lane < jb) y0 = fma(-Lb[lane][c], yc, y0);
      if (lane + 32 > c && lane + 32 < jb) y1 = fma(-Lb[lane + 32][c], yc, y1);
    } else {
      if (lane < c) y0 = fma(-Lb[c][lane], yc, y0);
      if (lane + 32 < c) y1 = fma(-Lb[c][lane + 32], yc, y1);
    }
  }
  if (lane < jb) yb[lane] = y0;
  if (lane + 32 < jb) yb[lane + 32] = y1;
}

template <typename V>
__global__ void __launch_bounds__(kGathPos) gather_fwd_kernel(DevPlan dp, int32_t task0,
                                                              V *__restrict__ y,
                                                              V *__restrict__ t) {
  const Task tk = dp.gath[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int p = tk.a + threadIdx.x;
  if (p >= F.ncol + F.nrow) return;
  V v = V(0);
  for (int ci = F.child_begin; ci < F.child_end; ci++) {
    const int32_t c = dp.children[ci];
    const int32_t a = dp.inv[dp.fronts[c].inv_off + p];
    if (a >= 0) v += t[dp.toff[c] + a];
  }
  if (p < F.ncol) y[F.first + p] -= v;
  else t[dp.toff[tk.front] + p - F.ncol] = v;
}

template <typename T, typename V>
__global__ void __launch_bounds__(64) diag_fwd_kernel(DevPlan dp, int32_t task0, int nbs,
                                                      const T *__restrict__ L,
                                                      V *__restrict__ y) {
  const Task tk = dp.sdiag[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int j = tk.a, jb = min(nbs, F.ncol - j), tid = threadIdx.x;
  __shared__ V Lb[64][65];
  __shared__ V yb[64];
  const T *A = L + F.loff + (int64_t)j * F.ld + j;
  for (int e = tid; e < jb * jb; e += 64) {
    const int r = e / jb, c = e % jb;
    if (r >= c) Lb[r][c] = (V)A[(int64_t)r * F.ld + c];
  }
  if (tid < jb) yb[tid] = y[F.first + j + tid];
  __syncthreads();
  if (tid < 32) diag_chain<V, true>(Lb, yb, jb, tid, sizeof(V) == 8 && !dp.sgn);
  __syncthreads();
  if (tid < jb) y[F.first + j + tid] = yb[tid];
}

template <typename T, typename V>
__global__ void __launch_bounds__(256) upd_fwd_kernel(DevPlan dp, int32_t task0, int nbs,
                                                      const T *__restrict__ L,
                                                      V *__restrict__ y, V *__restrict__ t) {
  const Task tk = dp.sgemv[task0 + blockIdx.x];
  if (tk.c != 0) return;
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow, i0 = tk.a, j = tk.b, jb = min(nbs, F.ncol - j);
  __shared__ V yj[64];
  if (threadIdx.x < jb) yj[threadIdx.x] = y[F.first + j + threadIdx.x];
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int r1 = min(i0 + kSolveRows, nf);
  for (int r = i0 + warp; r < r1; r += 8) {
    const T *row = L + F.loff + (int64_t)r * F.ld + j;
    V v = V(0);
    for (int c = lane; c < jb; c += 32) v = fma((V)row[c], yj[c], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      if (r < F.ncol) y[F.first + r] -= v;
      else t[dp.toff[tk.front] + r - F.ncol] += v;
    }
  }
}

template <typename T, typename V>
__global__ void __launch_bounds__(256) rows_bwd_kernel(DevPlan dp, int32_t task0,
                                                       const T *__restrict__ L,
                                                       V *__restrict__ y) {
  const Task tk = dp.rgemv[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int c0 = tk.a, warp = threadIdx.x / 32, lane = threadIdx.x % 32, c = c0 + lane;
  __shared__ V part[8][33];
  V acc = V(0);
  if (c < F.ncol) {
    const T *P = L + F.loff + (int64_t)F.ncol * F.ld + c;
    const int32_t *rs = dp.sri + F.rows_off;
    for (int r = warp; r < F.nrow; r += 8) acc = fma((V)P[(int64_t)r * F.ld], y[rs[r]], acc);
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < F.ncol) {
    V s = part[0][lane];
    for (int w = 1; w < 8; w++) s += part[w][lane];
    y[F.first + c] -= s;
  }
}

template <typename T, typename V>
__global__ void __launch_bounds__(64) diag_bwd_kernel(DevPlan dp, int32_t task0, int nbs,
                                                      const T *__restrict__ L,
                                                      V *__restrict__ y) {
  const Task tk = dp.sdiag[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int j = tk.a, jb = min(nbs, F.ncol - j), tid = threadIdx.x;
  __shared__ V Lb[64][65];
  __shared__ V yb[64];
  const T *A = L + F.loff + (int64_t)j * F.ld + j;
  for (int e = tid; e < jb * jb; e += 64) {
    const int r = e / jb, c = e % jb;
    if (r >= c) Lb[r][c] = (V)A[(int64_t)r * F.ld + c];
  }
  if (tid < jb) yb[tid] = y[F.first + j + tid];
  __syncthreads();
  if (tid < 32) diag_chain<V, false>(Lb, yb, jb, tid, sizeof(V) == 8 && !dp.sgn);
  __syncthreads();
  if (tid < jb) y[F.first + j + tid] = yb[tid];
}

template <typename T, typename V>
__global__ void __launch_bounds__(256) upd_bwd_kernel(DevPlan dp, int32_t task0, int nbs,
                                                      const T *__restrict__ L,
                                                      V *__restrict__ y) {
  const Task tk = dp.sgemv[task0 + blockIdx.x];
  if (tk.c != 1) return;
  const FrontInfo F = dp.fronts[tk.front];
  const int c0 = tk.a, j = tk.b, jb = min(nbs, F.ncol - j);
  __shared__ V xj[64];
  if (threadIdx.x < jb) xj[threadIdx.x] = y[F.first + j + threadIdx.x];
  __syncthreads();
  const int c = c0 + threadIdx.x;
  if (c >= j) return;
  const T *P = L + F.loff + (int64_t)j * F.ld + c;
  V v = V(0);
  for (int r = 0; r < jb; r++) v = fma((V)P[(int64_t)r * F.ld], xj[r], v);
  y[F.first + c] -= v;
}

// y <- S y between the sweeps of a signed factor K = L S L^T (final numbering).
template <typename V>
__global__ void sign_kernel(int32_t n, const int8_t *__restrict__ sgn, V *__restrict__ y) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    if (sgn[k] < 0) y[k] = -y[k];
}

}  // namespace

template <typename V>
void launch_sign(const DevPlan &dp, V *y, cudaStream_t st) {
  if (!dp.sgn || dp.n <= 0) return;
  const int g = (int)std::min<int64_t>((dp.n + 255) / 256, 152 * 16);
  note_launch();
  sign_kernel<V><<<g, 256, 0, st>>>(dp.n, dp.sgn, y);
}
template void launch_sign<float>(const DevPlan &, float *, cudaStream_t);
template void launch_sign<double>(const DevPlan &, double *, cudaStream_t);

template <typename T, typename V>
void launch_solve(const DevPlan &dp, const Plan &plan, const T *L, V *y, V *t, cudaStream_t st) {
  const int nbs = plan.nbs;
  const int nlev = (int)plan.levels.size();
  for (int li = 0; li < nlev; li++) {
    const LevelPlan &LP = plan.levels[li];
    if (LP.gath_e > LP.gath_b)
      { note_launch(); gather_fwd_kernel<V><<<LP.gath_e - LP.gath_b, kGathPos, 0, st>>>(dp, LP.gath_b, y, t); }
    for (size_t si = 0; si + 1 < LP.sstep_b.size(); si++) {
      const int d0 = LP.sstep_b[si], d1 = LP.sstep_b[si + 1];
      const int g0 = LP.sgemv_b[si], g1 = LP.sgemv_b[si + 1];
      if (d1 > d0) { note_launch(); diag_fwd_kernel<T, V><<<d1 - d0, 64, 0, st>>>(dp, d0, nbs, L, y); }
      if (g1 > g0) { note_launch(); upd_fwd_kernel<T, V><<<g1 - g0, 256, 0, st>>>(dp, g0, nbs, L, y, t); }
    }
  }
  launch_sign<V>(dp, y, st);  // K = L S L^T: y <- S L^{-1} b before the backward sweep
  for (int li = nlev - 1; li >= 0; li--) {
    const LevelPlan &LP = plan.levels[li];
    if (LP.rg_e > LP.rg_b)
      { note_launch(); rows_bwd_kernel<T, V><<<LP.rg_e - LP.rg_b, 256, 0, st>>>(dp, LP.rg_b, L, y); }
    for (int si = (int)LP.sstep_b.size() - 2; si >= 0; si--) {
      const int d0 = LP.sstep_b[si], d1 = LP.sstep_b[si + 1];
      const int g0 = LP.sgemv_b[si], g1 = LP.sgemv_b[si + 1];
      if (d1 > d0) { note_launch(); diag_bwd_kernel<T, V><<<d1 - d0, 64, 0, st>>>(dp, d0, nbs, L, y); }
      if (g1 > g0) { note_launch(); upd_bwd_kernel<T, V><<<g1 - g0, 256, 0, st>>>(dp, g0, nbs, L, y); }
    }
  }
}

template <typename T, typename V>
static cudaError_t preload_one() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, (const void *)gather_fwd_kernel<V>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)diag_fwd_kernel<T, V>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)upd_fwd_kernel<T, V>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)rows_bwd_kernel<T, V>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)diag_bwd_kernel<T, V>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)upd_bwd_kernel<T, V>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, (const void *)sign_kernel<V>);
  return e;
}

cudaError_t preload_level_solve() {
  cudaError_t e = preload_one<double, double>();
  return e == cudaSuccess ? preload_one<float, float>() : e;
}

template void launch_solve<double, double>(const DevPlan &, const Plan &, const double *,
                                           double *, double *, cudaStream_t);
template void launch_solve<float, float>(const DevPlan &, const Plan &, const float *, float *,
                                         float *, cudaStream_t);
template void launch_solve<float, double>(const DevPlan &, const Plan &, const float *, double *,
                                          double *, cudaStream_t);

}  // namespace gipm
