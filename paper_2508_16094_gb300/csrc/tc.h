// Tensor-core (tcgen05) factorisation path: TF32 operands staged by TMA into
// 128B-swizzled shared memory, FP32 accumulators in tensor memory. The GEMM-
// shaped work of the factorisation (left-looking panel updates, the triangular
// solve of the rows below a diagonal block as a product with its inverse, and
// the update-matrix SYRK) runs on the tensor cores; the diagonal-block
// Cholesky and its inverse run on the FP32 FMA pipe.
#pragma once

#include <vector>

#include "dev.cuh"

namespace gipm {

class TcPlan {
 public:
  static constexpr int kNb = 128;  // block-column width of the tensor-core path
  // CTAs left to the main stream's panel steps while the side stream runs the
  // look-ahead update of the next super-step on the other SMs.
  static constexpr int kMainCtas = 24;
  TcPlan() = default;
  TcPlan(const TcPlan &) = delete;
  TcPlan &operator=(const TcPlan &) = delete;
  ~TcPlan();
  // Host task lists (after the symbolic analysis and plan).
  void build(const Plan &plan);
  // Carve device memory for tasks and tensor maps (cv.base == nullptr: size only).
  void layout(Carve &cv, cudaStream_t st);
  // Encode one TMA tensor map per front panel of the FP32 factor storage L and
  // of Llo (low parts x - tf32(x) of the finished entries, same layout), and
  // one per update matrix in U; also creates the side stream and events of
  // the look-ahead (once).
  void encode(const Plan &plan, float *L, float *Llo, float *U, cudaStream_t st);
  bool ready() const { return ready_; }
  // split = 1: plain TF32 products; split = 3: A_lo B + A B_lo + A B
  // (FP32-accurate products on tensor cores); split = 16: BF16 products
  // (kind::f16) for every update by finished entries, read from their BF16
  // copy, with the panel solves in TF32 (L must be the encoded buffer)
  // Dinv (may be null): also write the diagonal-block inverses in the layout of
  // the persistent solve. Work forks onto the side stream and joins back into
  // st before the call's last launch, so st alone orders the result.
  void factor(const DevPlan &dp, const Plan &plan, const double *kval, float *L, float *U,
              float *Dinv, int32_t *status, int split, cudaStream_t st);

 private:
  struct Step { int gemm_b, gemm_e, potrf_b, potrf_e, trsm_b, trsm_e; };
  // A super-step: the update of its columns by the previous super-step's
  // (now_*), the look-ahead update of the next super-step's columns by all
  // columns before this one (ahead_*, side stream), and its block steps.
  struct Super { int k0, now_b, now_e, ahead_b, ahead_e, step_b, step_e; };  // k0: first column
  struct Level {
    std::vector<Step> steps;
    std::vector<Super> supers;
    int pair_b = 0, pair_e = 0;  // the level's update-matrix SYRK
  };
  std::vector<Task> gemm_, potrf_, trsm_, pairs_;
  std::vector<Level> levels_;
  int nfronts_ = 0, max_slots_ = 1;
  float *d_inv_ = nullptr;  // inverses of the diagonal blocks of one step (max_slots_ x 128 x 128)
  Task *d_gemm_ = nullptr, *d_potrf_ = nullptr, *d_trsm_ = nullptr, *d_pairs_ = nullptr;
  void *d_maps_ = nullptr;  // 7 nfronts_ + 1 CUtensorMap (128 bytes each)
  float *L_ = nullptr, *Llo_ = nullptr, *U_ = nullptr;
  cudaStream_t side_ = nullptr;                              // look-ahead stream (low priority)
  cudaEvent_t ev_main_ = nullptr, ev_side_ = nullptr;        // fork / join
  bool ready_ = false;
};

}  // namespace gipm
