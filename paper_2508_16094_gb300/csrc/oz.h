// FP64-accurate tensor-core factorisation: the dense updates of the FP64
// multifrontal Cholesky as error-free sums of BF16 slice products (Ozaki
// scheme) on tcgen05, the diagonal blocks and their triangular solves in FP64
// on the FMA pipe.
#pragma once

#include <vector>

#include "dev.cuh"

namespace gipm {

// Per front: where its slice planes and exponent table live.
struct OzFront {
  int64_t soff;  // first element of plane 0 (7 planes of nf x lds BF16 values)
  int64_t eoff;  // first exponent (nf rows x nblk int16)
  int32_t lds;   // row stride of a plane (elements, a multiple of 8)
  int32_t nblk;  // 64-column blocks of the panel
  int32_t pad[2];
};
static_assert(sizeof(OzFront) == 32, "OzFront layout");

class OzPlan {
 public:
  static constexpr int kPlanes = 7;  // BF16 slices per FP64 value
  static constexpr int kBlk = 64;    // the plan's block width; windows are 1 or 2 blocks
  OzPlan() = default;
  OzPlan(const OzPlan &) = delete;
  OzPlan &operator=(const OzPlan &) = delete;
  // Task lists and slice layout from the FP64 plan (block width kBlk).
  void build(const Plan &plan);
  // Carve device memory: tasks, per-front records and tensor maps, and (when
  // `storage` is set) the slice planes and exponent tables.
  void layout(Carve &cv, cudaStream_t st, bool storage);
  // Tensor maps of every front's slice planes (needs the carved storage).
  void encode(const Plan &plan, cudaStream_t st);
  bool ready() const { return ready_; }
  bool sized() const { return sized_; }
  int64_t slice_bytes() const { return slice_elems_ * 2 + exp_elems_ * 2; }
  // Factor the assembled K (kval) into the FP64 storage L, U.
  void factor(const DevPlan &dp, const Plan &plan, const double *kval, double *L, double *U,
              int32_t *status, cudaStream_t st);

 private:
  void validate(const Plan &plan) const;
  struct Step { int gemm_b, gemm_e, slice_b, slice_e; };
  struct Level { std::vector<Step> steps; int syrk_b = 0, syrk_e = 0; };
  std::vector<Task> gemm_, slice_;
  std::vector<OzFront> fr_;
  std::vector<Level> levels_;
  int64_t slice_elems_ = 0, exp_elems_ = 0;
  Task *d_gemm_ = nullptr, *d_slice_ = nullptr;
  OzFront *d_fr_ = nullptr;
  void *d_maps_ = nullptr;  // 2 CUtensorMap per front: 128-row and 64-row boxes
  uint16_t *S_ = nullptr;   // slice planes (BF16 bits)
  int16_t *E_ = nullptr;    // exponent tables
  bool sized_ = false, ready_ = false;
};

}  // namespace gipm
