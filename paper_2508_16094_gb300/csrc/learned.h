// Learned diagonal-plus-low-rank correction of a stale factor (not in the
// paper): a per-variable network maps local features of the change between the
// factored and the current condensed matrix to Delta (diagonal, > 0) and U
// (rank 16) so that M^{-1} = P^T L_s^{-T} (Delta + U U^T)^{-1} L_s^{-1} P
// preconditions conjugate gradients on the current K.
#pragma once

#include "ipm_kernels.h"

namespace gipm {

constexpr int kNF = 8;            // features per variable
constexpr int kNH = 32;           // hidden width (two tanh layers)
constexpr int kNR = 16;           // rank of U
constexpr int kNO = 1 + kNR;      // outputs: log Delta, U row
constexpr int kW1 = 0, kB1 = kW1 + kNH * kNF, kW2 = kB1 + kNH, kB2 = kW2 + kNH * kNH,
              kW3 = kB2 + kNH, kB3 = kW3 + kNO * kNH, kNParams = kB3 + kNO;
constexpr float kUScale = 0.1f;   // U = kUScale * raw outputs
constexpr int kLRedBlocks = 152;  // fixed grid of the first pass of learned reductions

struct LearnedBufs {
  int64_t n = 0, mt = 0;
  int P = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // kNParams each
  float *feat = nullptr, *h1 = nullptr, *h2 = nullptr, *out = nullptr, *gout = nullptr;
  float *delta = nullptr, *U = nullptr;
  double *diag_old = nullptr, *diag_new = nullptr, *D_old = nullptr;
  double *mu = nullptr;          // [0] mu at the factored iterate, [1] current mu
  float *partial = nullptr;      // kLRedBlocks * (kNParams + kNR*kNR) floats
  double *dpart = nullptr;       // kLRedBlocks * 8 doubles
  float *probe_t = nullptr, *probe_q = nullptr;  // P * kNR
  double *cap = nullptr;         // 16x16 capacitance, then its Cholesky factor
  float *ts = nullptr;           // kNR (Woodbury scratch)
  int64_t step = 0;              // Adam step
};

// diag(K) = sum_r J_ri^2 D_r + D_l + D_u + delta_p (original numbering)
void learned_diag(const DevPlan &dp, const double *jv, const double *D, double delta_p,
                  double *diag, cudaStream_t st);
// features of every permuted index (current D, diag vs the factored ones)
void learned_features(const DevPlan &dp, const LearnedBufs &B, const double *jv, const double *D,
                      const double *x, cudaStream_t st);
// network forward: Delta, U (and activations for training); ablation: Delta = 1, U = 0
void learned_forward(const LearnedBufs &B, bool ablate, cudaStream_t st);
// capacitance I + U^T Delta^{-1} U and its Cholesky factor (device)
void learned_capacitance(const LearnedBufs &B, cudaStream_t st);
// v <- (Delta + U U^T)^{-1} v (permuted index, FP32) by the Woodbury identity
void learned_apply(const LearnedBufs &B, float *v, cudaStream_t st);
// loss sum_z ||Delta^{-1} (w_z - Delta z - U U^T z)||^2 / (P n) and its gradient
// w.r.t. the weights (into B.grad); the loss goes to d_loss (device)
void learned_loss_grad(const LearnedBufs &B, const float *z, const float *wt, double *d_loss,
                       cudaStream_t st);
void learned_adam(LearnedBufs &B, float lr, cudaStream_t st);

}  // namespace gipm
