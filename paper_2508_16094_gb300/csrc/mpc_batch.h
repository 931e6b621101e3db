// Batched MPC interior-point solver: kernel arguments and launcher.
#pragma once

#include "dev.cuh"

namespace gipm {

// Workspace doubles per stage: 6 vectors x 16, 7 row arrays x 64 slots, two
// FP64 16x16 blocks (K) and two 16x16 blocks of the factor (sized for FP64).
constexpr int64_t kMpcStageDoubles = 6 * 16 + 8 * 64 + 2 * 256 + 2 * 256;

struct MpcArgs {
  int count;
  const int32_t *T;      // horizons (device)
  const int64_t *soff;   // first stage of each instance (device)
  const int32_t *order;  // instance queue, longest horizon first (device)
  const double *A, *B, *Q, *R, *x0;
  double umax, xmax;
  double tol, delta_p, delta_d;
  int max_iter;
  double *work;  // total_stages * kMpcStageDoubles
  int *counter;
  double *zout;  // (sum T) x 16 or nullptr
  double *obj, *kkt;
  int32_t *iters, *status;
  int32_t *fp64_used;  // per instance: 1 if the FP32 factor was replaced by FP64 (or nullptr)
};

// precision 0: FP64 factor and solves; 1: FP32 factor/solves + 2 FP64
// refinement steps per solve. instances_per_cta in {2, 4, 8, 16}.
void launch_mpc(const MpcArgs &a, int precision, int instances_per_cta, int ctas, cudaStream_t st);

}  // namespace gipm
