// Kernels of the learned stale-factor correction: features, the per-variable
// network (forward and backward), the probe loss, deterministic weight-gradient
// reductions, Adam, and the Woodbury application of (Delta + U U^T)^{-1}.
// All reductions use fixed grids and fixed summation orders.
#include <cfloat>
#include <cmath>

#include "learned.h"

namespace gipm {

namespace {

#define LGRID(i, n)                                                                      \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n);             \
       i += (int64_t)gridDim.x * blockDim.x)

inline int lgrid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

__global__ void diag_kernel(DevPlan dp, const double *__restrict__ jv, const double *__restrict__ D,
                            double delta_p, double *__restrict__ diag) {
  LGRID(i, dp.n) {
    double a = delta_p;
    for (int64_t t = dp.jtp[i]; t < dp.jtp[i + 1]; t++) {
      const int32_t e = dp.jtpos[t];
      a = fma(jv[e] * jv[e], D[dp.jrow[e]], a);
    }
    if (dp.lpos[i] >= 0) a += D[dp.lpos[i]];
    if (dp.upos[i] >= 0) a += D[dp.upos[i]];
    diag[i] = a;
  }
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}

__global__ void feat_kernel(DevPlan dp, LearnedBufs B, const double *__restrict__ jv,
                            const double *__restrict__ D, const double *__restrict__ x) {
  const double mu_old = B.mu[0], mu_new = B.mu[1];
  LGRID(j, dp.n) {
    const int32_t i = dp.perm[j];
    const double kn = B.diag_new[i], ko = B.diag_old[i];
    double bn = 0.0, bo = 0.0;
    if (dp.lpos[i] >= 0) { bn += D[dp.lpos[i]]; bo += B.D_old[dp.lpos[i]]; }
    if (dp.upos[i] >= 0) { bn += D[dp.upos[i]]; bo += B.D_old[dp.upos[i]]; }
    double ss = 0.0, sa = 0.0;
    for (int64_t t = dp.jtp[i]; t < dp.jtp[i + 1]; t++) {
      const int32_t e = dp.jtpos[t];
      const int32_t r = dp.jrow[e];
      const double d = (D[r] - B.D_old[r]) * jv[e] * jv[e];
      ss += d;
      sa += fabs(d);
    }
    float *f = B.feat + j * kNF;
    f[0] = clampf((float)log(kn / ko), -30.f, 30.f);
    f[1] = clampf((float)(log((bn + 1e-300) / (bo + 1e-300)) / 10.0), -5.f, 5.f);
    f[2] = (float)asinh(ss / ko);
    f[3] = (float)asinh(sa / ko);
    f[4] = (float)(log10(fmax(mu_new, 1e-300)) / 10.0);
    f[5] = clampf((float)(log(fmax(mu_new, 1e-300) / fmax(mu_old, 1e-300)) / 10.0), -5.f, 5.f);
    f[6] = clampf((float)(log(bn / kn + 1e-30) / 10.0), -7.f, 1.f);
    f[7] = (float)(x ? x[i] / 10.0 : 0.0);
  }
}

__global__ void __launch_bounds__(256) fwd_kernel(LearnedBufs B, int ablate) {
  __shared__ float w[kNParams];
  for (int p = threadIdx.x; p < kNParams; p += blockDim.x) w[p] = B.w[p];
  __syncthreads();
  LGRID(j, B.n) {
    if (ablate) {
      B.delta[j] = 1.f;
      for (int a = 0; a < kNR; a++) B.U[j * kNR + a] = 0.f;
      continue;
    }
    float f[kNF], h1[kNH], h2[kNH];
    for (int q = 0; q < kNF; q++) f[q] = B.feat[j * kNF + q];
    for (int a = 0; a < kNH; a++) {
      float s = w[kB1 + a];
      for (int q = 0; q < kNF; q++) s = fmaf(w[kW1 + a * kNF + q], f[q], s);
      h1[a] = tanhf(s);
      B.h1[j * kNH + a] = h1[a];
    }
    for (int a = 0; a < kNH; a++) {
      float s = w[kB2 + a];
      for (int q = 0; q < kNH; q++) s = fmaf(w[kW2 + a * kNH + q], h1[q], s);
      h2[a] = tanhf(s);
      B.h2[j * kNH + a] = h2[a];
    }
    for (int a = 0; a < kNO; a++) {
      float s = w[kB3 + a];
      for (int q = 0; q < kNH; q++) s = fmaf(w[kW3 + a * kNH + q], h2[q], s);
      B.out[j * kNO + a] = s;
      if (a == 0) B.delta[j] = expf(clampf(s, -20.f, 20.f));
      else B.U[j * kNR + a - 1] = kUScale * s;
    }
  }
}

// capacitance partials: C_ab = sum_j U_ja U_jb / Delta_j over a chunk of j per block
__global__ void __launch_bounds__(256) cap_partial_kernel(LearnedBufs B) {
  __shared__ float us[64][kNR + 1];
  const int a = threadIdx.x / kNR, b = threadIdx.x % kNR;
  double acc = 0.0;
  for (int64_t j0 = (int64_t)blockIdx.x * 64; j0 < B.n; j0 += (int64_t)gridDim.x * 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * kNR; e += 256) {
      const int jj = e / kNR, c = e % kNR;
      const int64_t j = j0 + jj;
      us[jj][c] = j < B.n ? B.U[j * kNR + c] * rsqrtf(B.delta[j]) : 0.f;
    }
    __syncthreads();
    for (int jj = 0; jj < 64; jj++) acc += (double)us[jj][a] * (double)us[jj][b];
  }
  B.dpart[blockIdx.x * 256 + threadIdx.x] = acc;
}

__global__ void cap_final_kernel(LearnedBufs B, int nblocks) {
  __shared__ double C[kNR][kNR];
  const int t = threadIdx.x, a = t / kNR, b = t % kNR;
  double s = (a == b) ? 1.0 : 0.0;
  for (int k = 0; k < nblocks; k++) s += B.dpart[k * 256 + t];
  C[a][b] = s;
  __syncthreads();
  if (t == 0) {  // Cholesky of the (SPD) capacitance
    for (int j = 0; j < kNR; j++) {
      double d = C[j][j];
      for (int k = 0; k < j; k++) d -= C[j][k] * C[j][k];
      d = sqrt(fmax(d, 1e-300));
      C[j][j] = d;
      for (int i = j + 1; i < kNR; i++) {
        double v = C[i][j];
        for (int k = 0; k < j; k++) v -= C[i][k] * C[j][k];
        C[i][j] = v / d;
      }
    }
  }
  __syncthreads();
  B.cap[t] = C[a][b];
}

// y = v / Delta (in place) and per-block partials of U^T y
__global__ void __launch_bounds__(256) wood_scale_kernel(LearnedBufs B, float *v) {
  __shared__ float red[256 / 32][kNR];
  float acc[kNR];
  for (int a = 0; a < kNR; a++) acc[a] = 0.f;
  LGRID(j, B.n) {
    const float y = v[j] / B.delta[j];
    v[j] = y;
    for (int a = 0; a < kNR; a++) acc[a] = fmaf(B.U[j * kNR + a], y, acc[a]);
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int a = 0; a < kNR; a++) {
    float s = acc[a];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][a] = s;
  }
  __syncthreads();
  if (threadIdx.x < kNR) {
    float s = 0.f;
    for (int w = 0; w < 256 / 32; w++) s += red[w][threadIdx.x];
    B.partial[blockIdx.x * kNR + threadIdx.x] = s;
  }
}

// ts = C^{-1} (sum of partials), C given by its Cholesky factor
__global__ void wood_solve_kernel(LearnedBufs B, int nblocks) {
  if (threadIdx.x != 0) return;
  double t[kNR];
  for (int a = 0; a < kNR; a++) {
    double s = 0.0;
    for (int k = 0; k < nblocks; k++) s += B.partial[k * kNR + a];
    t[a] = s;
  }
  for (int i = 0; i < kNR; i++) {
    double v = t[i];
    for (int k = 0; k < i; k++) v -= B.cap[i * kNR + k] * t[k];
    t[i] = v / B.cap[i * kNR + i];
  }
  for (int i = kNR - 1; i >= 0; i--) {
    double v = t[i];
    for (int k = i + 1; k < kNR; k++) v -= B.cap[k * kNR + i] * t[k];
    t[i] = v / B.cap[i * kNR + i];
  }
  for (int a = 0; a < kNR; a++) B.ts[a] = (float)t[a];
}

__global__ void wood_update_kernel(LearnedBufs B, float *v) {
  LGRID(j, B.n) {
    float s = 0.f;
    for (int a = 0; a < kNR; a++) s = fmaf(B.U[j * kNR + a], B.ts[a], s);
    v[j] -= s / B.delta[j];
  }
}

// ---- training ----------------------------------------------------------------
constexpr int kMaxP = 8;

// per-block partials of t_p = U^T z_p (P x 16)
__global__ void __launch_bounds__(256) probe_t_kernel(LearnedBufs B, const float *z) {
  __shared__ float red[256 / 32][kMaxP * kNR];
  float acc[kMaxP * kNR];
  for (int a = 0; a < B.P * kNR; a++) acc[a] = 0.f;
  LGRID(j, B.n) {
    for (int p = 0; p < B.P; p++) {
      const float zv = z[(int64_t)p * B.n + j];
      for (int a = 0; a < kNR; a++) acc[p * kNR + a] = fmaf(B.U[j * kNR + a], zv, acc[p * kNR + a]);
    }
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int a = 0; a < B.P * kNR; a++) {
    float s = acc[a];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][a] = s;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < B.P * kNR; a += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < 256 / 32; w++) s += red[w][a];
    B.partial[blockIdx.x * kMaxP * kNR + a] = s;
  }
}

__global__ void sum_partials_kernel(const float *partial, int nblocks, int width, int stride,
                                    float *out) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < width; a += blockDim.x * gridDim.x) {
    float s = 0.f;
    for (int k = 0; k < nblocks; k++) s += partial[k * stride + a];
    out[a] = s;
  }
}

// relative residual r_p = Delta^{-1} (w_p - Delta z_p - U t_p): loss partials (FP64)
// and partials of q_p = U^T Delta^{-1} r_p
__global__ void __launch_bounds__(256) resid_kernel(LearnedBufs B, const float *z, const float *wt) {
  __shared__ float red[256 / 32][kMaxP * kNR];
  __shared__ double lred[256 / 32];
  float acc[kMaxP * kNR];
  for (int a = 0; a < B.P * kNR; a++) acc[a] = 0.f;
  double loss = 0.0;
  LGRID(j, B.n) {
    for (int p = 0; p < B.P; p++) {
      const float zv = z[(int64_t)p * B.n + j];
      float ut = 0.f;
      for (int a = 0; a < kNR; a++) ut = fmaf(B.U[j * kNR + a], B.probe_t[p * kNR + a], ut);
      const float dj = B.delta[j];
      const float r = (wt[(int64_t)p * B.n + j] - dj * zv - ut) / dj;
      loss += (double)r * (double)r;
      const float rd = r / dj;
      for (int a = 0; a < kNR; a++) acc[p * kNR + a] = fmaf(B.U[j * kNR + a], rd, acc[p * kNR + a]);
    }
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (int a = 0; a < B.P * kNR; a++) {
    float s = acc[a];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][a] = s;
  }
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0) lred[warp] = loss;
  __syncthreads();
  for (int a = threadIdx.x; a < B.P * kNR; a += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < 256 / 32; w++) s += red[w][a];
    B.partial[blockIdx.x * kMaxP * kNR + a] = s;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 256 / 32; w++) s += lred[w];
    B.dpart[blockIdx.x] = s;
  }
}

__global__ void loss_final_kernel(LearnedBufs B, int nblocks, double *loss) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < nblocks; k++) s += B.dpart[k];
  *loss = s / ((double)B.P * (double)B.n);
}

// gradient w.r.t. the raw outputs, then back through the two tanh layers
__global__ void __launch_bounds__(256) outgrad_bwd_kernel(LearnedBufs B, const float *z,
                                                          const float *wt) {
  __shared__ float w[kNParams];
  for (int p = threadIdx.x; p < kNParams; p += blockDim.x) w[p] = B.w[p];
  __syncthreads();
  const float scale = 1.f / ((float)B.P * (float)B.n);
  LGRID(j, B.n) {
    float go[kNO];
    float gd = 0.f, gu[kNR];
    for (int a = 0; a < kNR; a++) gu[a] = 0.f;
    const float dj = B.delta[j];
    for (int p = 0; p < B.P; p++) {
      const float zv = z[(int64_t)p * B.n + j];
      float ut = 0.f;
      for (int a = 0; a < kNR; a++) ut = fmaf(B.U[j * kNR + a], B.probe_t[p * kNR + a], ut);
      const float r = (wt[(int64_t)p * B.n + j] - dj * zv - ut) / dj;
      // d r / d Delta_j = -(r + z_j) / Delta_j; d loss / d log Delta_j = Delta_j d loss / d Delta_j
      gd += -2.f * r * (r + zv);
      const float rd = r / dj;
      for (int a = 0; a < kNR; a++)
        gu[a] += -2.f * (rd * B.probe_t[p * kNR + a] + zv * B.probe_q[p * kNR + a]);
    }
    const float o0 = B.out[j * kNO];
    go[0] = (o0 > -20.f && o0 < 20.f) ? gd * scale : 0.f;
    for (int a = 0; a < kNR; a++) go[1 + a] = gu[a] * kUScale * scale;
    float *g = B.gout + j * (kNO + 2 * kNH);
    for (int a = 0; a < kNO; a++) g[a] = go[a];
    float gh2[kNH];
    for (int q = 0; q < kNH; q++) {
      float s = 0.f;
      for (int a = 0; a < kNO; a++) s = fmaf(w[kW3 + a * kNH + q], go[a], s);
      const float h = B.h2[j * kNH + q];
      gh2[q] = s * (1.f - h * h);
      g[kNO + q] = gh2[q];
    }
    for (int q = 0; q < kNH; q++) {
      float s = 0.f;
      for (int a = 0; a < kNH; a++) s = fmaf(w[kW2 + a * kNH + q], gh2[a], s);
      const float h = B.h1[j * kNH + q];
      g[kNO + kNH + q] = s * (1.f - h * h);
    }
  }
}

// weight gradient partials: sum over a chunk of variables of the outer
// products (gout h2^T, gh2 h1^T, gh1 f^T and the bias terms); parameter p is
// owned by threads p, p+256, ... so every sum has a fixed order
__global__ void __launch_bounds__(256) wgrad_partial_kernel(LearnedBufs B) {
  constexpr int CH = 32, GW = kNO + 2 * kNH;
  __shared__ float sg[CH][GW], sh1[CH][kNH], sh2[CH][kNH], sf[CH][kNF];
  float acc[(kNParams + 255) / 256];
  for (int k = 0; k < (kNParams + 255) / 256; k++) acc[k] = 0.f;
  for (int64_t j0 = (int64_t)blockIdx.x * CH; j0 < B.n; j0 += (int64_t)gridDim.x * CH) {
    __syncthreads();
    for (int e = threadIdx.x; e < CH * GW; e += 256) {
      const int jj = e / GW, c = e % GW;
      const int64_t j = j0 + jj;
      sg[jj][c] = j < B.n ? B.gout[j * GW + c] : 0.f;
    }
    for (int e = threadIdx.x; e < CH * kNH; e += 256) {
      const int jj = e / kNH, c = e % kNH;
      const int64_t j = j0 + jj;
      sh1[jj][c] = j < B.n ? B.h1[j * kNH + c] : 0.f;
      sh2[jj][c] = j < B.n ? B.h2[j * kNH + c] : 0.f;
    }
    for (int e = threadIdx.x; e < CH * kNF; e += 256) {
      const int jj = e / kNF, c = e % kNF;
      const int64_t j = j0 + jj;
      sf[jj][c] = j < B.n ? B.feat[j * kNF + c] : 0.f;
    }
    __syncthreads();
    for (int k = 0, p = threadIdx.x; p < kNParams; k++, p += 256) {
      float s = acc[k];
      for (int jj = 0; jj < CH; jj++) {
        float v;
        if (p < kB1) { const int a = p / kNF, q = p % kNF; v = sg[jj][kNO + kNH + a] * sf[jj][q]; }
        else if (p < kW2) { v = sg[jj][kNO + kNH + (p - kB1)]; }
        else if (p < kB2) { const int a = (p - kW2) / kNH, q = (p - kW2) % kNH; v = sg[jj][kNO + a] * sh1[jj][q]; }
        else if (p < kW3) { v = sg[jj][kNO + (p - kB2)]; }
        else if (p < kB3) { const int a = (p - kW3) / kNH, q = (p - kW3) % kNH; v = sg[jj][a] * sh2[jj][q]; }
        else { v = sg[jj][p - kB3]; }
        s += v;
      }
      acc[k] = s;
    }
  }
  for (int k = 0, p = threadIdx.x; p < kNParams; k++, p += 256)
    B.partial[(int64_t)blockIdx.x * kNParams + p] = acc[k];
}

__global__ void adam_kernel(LearnedBufs B, float lr, float b1t, float b2t) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int p = threadIdx.x + blockIdx.x * blockDim.x; p < kNParams; p += blockDim.x * gridDim.x) {
    const float g = B.grad[p];
    const float m = b1 * B.m[p] + (1.f - b1) * g;
    const float v = b2 * B.v[p] + (1.f - b2) * g * g;
    B.m[p] = m;
    B.v[p] = v;
    B.w[p] -= lr * (m / (1.f - b1t)) / (sqrtf(v / (1.f - b2t)) + eps);
  }
}

}  // namespace

void learned_diag(const DevPlan &dp, const double *jv, const double *D, double delta_p,
                  double *diag, cudaStream_t st) {
  note_launch();
  diag_kernel<<<lgrid(dp.n), 256, 0, st>>>(dp, jv, D, delta_p, diag);
}

void learned_features(const DevPlan &dp, const LearnedBufs &B, const double *jv, const double *D,
                      const double *x, cudaStream_t st) {
  note_launch();
  feat_kernel<<<lgrid(dp.n), 256, 0, st>>>(dp, B, jv, D, x);
}

void learned_forward(const LearnedBufs &B, bool ablate, cudaStream_t st) {
  note_launch();
  fwd_kernel<<<lgrid(B.n), 256, 0, st>>>(B, ablate ? 1 : 0);
}

void learned_capacitance(const LearnedBufs &B, cudaStream_t st) {
  note_launch();
  cap_partial_kernel<<<kLRedBlocks, 256, 0, st>>>(B);
  note_launch();
  cap_final_kernel<<<1, 256, 0, st>>>(B, kLRedBlocks);
}

void learned_apply(const LearnedBufs &B, float *v, cudaStream_t st) {
  note_launch();
  wood_scale_kernel<<<kLRedBlocks, 256, 0, st>>>(B, v);
  note_launch();
  wood_solve_kernel<<<1, 32, 0, st>>>(B, kLRedBlocks);
  note_launch();
  wood_update_kernel<<<lgrid(B.n), 256, 0, st>>>(B, v);
}

void learned_loss_grad(const LearnedBufs &B, const float *z, const float *wt, double *d_loss,
                       cudaStream_t st) {
  const int W = kMaxP * kNR;
  note_launch();
  probe_t_kernel<<<kLRedBlocks, 256, 0, st>>>(B, z);
  note_launch();
  sum_partials_kernel<<<1, 256, 0, st>>>(B.partial, kLRedBlocks, B.P * kNR, W, B.probe_t);
  note_launch();
  resid_kernel<<<kLRedBlocks, 256, 0, st>>>(B, z, wt);
  note_launch();
  sum_partials_kernel<<<1, 256, 0, st>>>(B.partial, kLRedBlocks, B.P * kNR, W, B.probe_q);
  note_launch();
  loss_final_kernel<<<1, 32, 0, st>>>(B, kLRedBlocks, d_loss);
  note_launch();
  outgrad_bwd_kernel<<<lgrid(B.n), 256, 0, st>>>(B, z, wt);
  note_launch();
  wgrad_partial_kernel<<<kLRedBlocks, 256, 0, st>>>(B);
  note_launch();
  sum_partials_kernel<<<(kNParams + 255) / 256, 256, 0, st>>>(B.partial, kLRedBlocks, kNParams,
                                                              kNParams, B.grad);
}

void learned_adam(LearnedBufs &B, float lr, cudaStream_t st) {
  B.step++;
  const float b1t = powf(0.9f, (float)B.step), b2t = powf(0.999f, (float)B.step);
  note_launch();
  adam_kernel<<<(kNParams + 255) / 256, 256, 0, st>>>(B, lr, b1t, b2t);
}

}  // namespace gipm
