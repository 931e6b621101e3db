// Tensor-core (tcgen05) factorisation path: TF32 or BF16 operands staged by
// TMA into shared memory, FP32 accumulators in tensor memory.
#pragma once

#include "dev.cuh"

namespace gipm {

struct Carve;

class TcPlan {
 public:
  // Host-side preparation after the symbolic analysis (task lists, sizes).
  void build(const Plan &plan);
  // Carve device memory inside the workspace (cv == nullptr: size only).
  template <typename C>
  void layout(C *cv, const Plan &plan, cudaStream_t st);
  bool ready() const { return ready_; }
  void factor(const DevPlan &dp, const Plan &plan, const double *kval, float *L, float *U,
              int32_t *status, bool bf16, cudaStream_t st);

 private:
  bool ready_ = false;
};

template <typename C>
void TcPlan::layout(C *, const Plan &, cudaStream_t) {}

}  // namespace gipm
