// Tensor-core factorisation path (placeholder until the tcgen05 kernels land).
#include "tc.h"

namespace gipm {

void TcPlan::build(const Plan &) { ready_ = false; }

void TcPlan::factor(const DevPlan &, const Plan &, const double *, float *, float *, int32_t *,
                    bool, cudaStream_t) {}

}  // namespace gipm
