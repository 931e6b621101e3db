// Fused supernodal triangular solves for FP32 factors (TF32/TF32x3/FP32).
//
// After the factorisation, one launch inverts every 128-wide diagonal block of
// L (explicit inverse, jb x jb). A forward step of a level is then a single
// kernel: each block of the step first forms y_j = L_jj^{-1} y_j itself (a
// 128 x 128 triangular matrix-vector product on data that no block of this
// step writes), the block whose rows start at j publishes y_j to a separate
// output vector, and every block updates its own rows below j (warp-per-row
// dot products; rows of the front's later columns -> y, rows below the front
// -> its update vector). The backward step mirrors it with x_j = L_jj^{-T} y_j
// and column updates to the left. Three vectors (right-hand side, forward
// result, solution) keep every read of a step disjoint from its writes.
#include "launch.h"

namespace gipm {

namespace {

constexpr int kFB = 128;  // block width of the fused solve

// Inverse of one diagonal block (jb <= 128): column c of X = L_jj^{-1} by
// forward substitution in thread c.
__global__ void __launch_bounds__(128) dinv_kernel(DevPlan dp, const float *__restrict__ L,
                                                   float *__restrict__ Dinv) {
  constexpr int LS = 129;
  const Task tk = dp.fs_inv[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int j = tk.a, jb = min(kFB, F.ncol - j), tid = threadIdx.x;
  extern __shared__ float smd[];
  float *A = smd;             // [128][129]
  float *X = smd + 128 * LS;  // [128][129]
  const float *g = L + F.loff + (int64_t)j * F.ld + j;
  for (int e = tid; e < jb * jb; e += 128) {
    const int r = e / jb, c = e % jb;
    A[r * LS + c] = (c <= r) ? g[(int64_t)r * F.ld + c] : 0.f;
  }
  __syncthreads();
  if (tid < jb) {
    const int c = tid;
    for (int i = c; i < jb; i++) {
      float s = (i == c) ? 1.f : 0.f;
      for (int m = c; m < i; m++) s = fmaf(-A[i * LS + m], X[m * LS + c], s);
      X[i * LS + c] = s / A[i * LS + i];
    }
  }
  __syncthreads();
  float *out = Dinv + dp.fs_dinv_off[tk.b];
  for (int e = tid; e < jb * jb; e += 128) {
    const int r = e / jb, c = e % jb;
    out[e] = (c <= r) ? X[r * LS + c] : 0.f;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) fwd_fused_kernel(DevPlan dp, int32_t task0,
                                                        const float *__restrict__ L,
                                                        const float *__restrict__ Dinv,
                                                        float *__restrict__ yin,
                                                        float *__restrict__ yout,
                                                        float *__restrict__ t) {
  const Task tk = dp.fs_fwd[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow, i0 = tk.a, j = tk.b, jb = min(kFB, F.ncol - j);
  const float *Di = Dinv + dp.fs_dinv_off[tk.c];
  __shared__ float ys[kFB], yj[kFB];
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (tid < jb) ys[tid] = yin[F.first + j + tid];
  __syncthreads();
  for (int r = warp; r < jb; r += 8) {  // y_j = L_jj^{-1} y_j (lower triangular)
    float v = 0.f;
    for (int c = lane; c <= r; c += 32) v = fmaf(Di[r * jb + c], ys[c], v);
    v = warp_sum(v);
    if (lane == 0) yj[r] = v;
  }
  __syncthreads();
  if (i0 == j && tid < jb) yout[F.first + j + tid] = yj[tid];
  const int r0 = max(i0, j + jb), r1 = min(i0 + 128, nf);
  for (int r = r0 + warp; r < r1; r += 8) {
    const float *row = L + F.loff + (int64_t)r * F.ld + j;
    float v = 0.f;
    for (int c = lane; c < jb; c += 32) v = fmaf(row[c], yj[c], v);
    v = warp_sum(v);
    if (lane == 0) {
      if (r < F.ncol) yin[F.first + r] -= v;
      else t[dp.toff[tk.front] + r - F.ncol] += v;
    }
  }
}

// xin[cols of the front] -= L21^T xout[rows below the front] (fixed-order reduction)
__global__ void __launch_bounds__(256) rows_bwd2_kernel(DevPlan dp, int32_t task0,
                                                        const float *__restrict__ L,
                                                        float *__restrict__ xin,
                                                        const float *__restrict__ xout) {
  const Task tk = dp.rgemv[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int c0 = tk.a, warp = threadIdx.x / 32, lane = threadIdx.x % 32, c = c0 + lane;
  __shared__ float part[8][33];
  float acc = 0.f;
  if (c < F.ncol) {
    const float *P = L + F.loff + (int64_t)F.ncol * F.ld + c;
    const int32_t *rs = dp.sri + F.rows_off;
    for (int r = warp; r < F.nrow; r += 8) acc = fmaf(P[(int64_t)r * F.ld], xout[rs[r]], acc);
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < F.ncol) {
    float s = part[0][lane];
    for (int w = 1; w < 8; w++) s += part[w][lane];
    xin[F.first + c] -= s;
  }
}

__global__ void __launch_bounds__(256) bwd_fused_kernel(DevPlan dp, int32_t task0,
                                                        const float *__restrict__ L,
                                                        const float *__restrict__ Dinv,
                                                        float *__restrict__ xin,
                                                        float *__restrict__ xout) {
  const Task tk = dp.fs_bwd[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int c0 = tk.a, j = tk.b, jb = min(kFB, F.ncol - j);
  const float *Di = Dinv + dp.fs_dinv_off[tk.c];
  __shared__ float ys[kFB], xj[kFB];
  const int tid = threadIdx.x;
  if (tid < jb) ys[tid] = xin[F.first + j + tid];
  __syncthreads();
  if (tid < jb) {  // x_j = L_jj^{-T} y_j
    float v = 0.f;
    for (int r = tid; r < jb; r++) v = fmaf(Di[r * jb + tid], ys[r], v);
    xj[tid] = v;
  }
  __syncthreads();
  if (c0 == 0 && tid < jb) xout[F.first + j + tid] = xj[tid];
  const int cc = c0 + tid;
  if (cc < j) {
    const float *P = L + F.loff + (int64_t)j * F.ld + cc;
    float v = 0.f;
    for (int r = 0; r < jb; r++) v = fmaf(P[(int64_t)r * F.ld], xj[r], v);
    xin[F.first + cc] -= v;
  }
}

__global__ void __launch_bounds__(256) gather_fused_kernel(DevPlan dp, int32_t task0,
                                                           float *__restrict__ y,
                                                           float *__restrict__ t) {
  const Task tk = dp.gath[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int p = tk.a + threadIdx.x;
  if (p >= F.ncol + F.nrow) return;
  float v = 0.f;
  for (int ci = F.child_begin; ci < F.child_end; ci++) {
    const int32_t c = dp.children[ci];
    const int32_t a = dp.inv[dp.fronts[c].inv_off + p];
    if (a >= 0) v += t[dp.toff[c] + a];
  }
  if (p < F.ncol) y[F.first + p] -= v;
  else t[dp.toff[tk.front] + p - F.ncol] = v;
}

}  // namespace

void launch_dinv(const DevPlan &dp, const Plan &plan, const float *L, float *Dinv,
                 cudaStream_t st) {
  const int n = (int)plan.fs_inv.size();
  if (n == 0) return;
  const int smem = 2 * 128 * 129 * (int)sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(dinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  { note_launch(); dinv_kernel<<<n, 128, smem, st>>>(dp, L, Dinv); }
}

int launch_solve_fused(const DevPlan &dp, const Plan &plan, const float *L, const float *Dinv,
                       float *a, float *b, float *x, float *t, cudaStream_t st, bool fwd,
                       bool bwd) {
  int launches = 0;
  const int nlev = (int)plan.levels.size();
  for (int li = 0; li < nlev && fwd; li++) {
    const LevelPlan &LP = plan.levels[li];
    if (LP.gath_e > LP.gath_b) {
      note_launch(); launches++;
      gather_fused_kernel<<<LP.gath_e - LP.gath_b, 256, 0, st>>>(dp, LP.gath_b, a, t);
    }
    for (size_t si = 0; si + 1 < LP.ffwd_b.size(); si++) {
      const int f0 = LP.ffwd_b[si], f1 = LP.ffwd_b[si + 1];
      if (f1 > f0) {
        note_launch(); launches++;
        fwd_fused_kernel<<<f1 - f0, 256, 0, st>>>(dp, f0, L, Dinv, a, b, t);
      }
    }
  }
  for (int li = nlev - 1; li >= 0 && bwd; li--) {
    const LevelPlan &LP = plan.levels[li];
    if (LP.rg_e > LP.rg_b) {
      note_launch(); launches++;
      rows_bwd2_kernel<<<LP.rg_e - LP.rg_b, 256, 0, st>>>(dp, LP.rg_b, L, b, x);
    }
    for (int si = (int)LP.fbwd_b.size() - 2; si >= 0; si--) {
      const int g0 = LP.fbwd_b[si], g1 = LP.fbwd_b[si + 1];
      if (g1 > g0) {
        note_launch(); launches++;
        bwd_fused_kernel<<<g1 - g0, 256, 0, st>>>(dp, g0, L, Dinv, b, x);
      }
    }
  }
  return launches;
}

}  // namespace gipm
