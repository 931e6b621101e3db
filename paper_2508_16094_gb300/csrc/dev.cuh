// Device-side views shared by the kernels and the host launchers.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"

namespace gipm {

// Device pointers of the plan and problem structure (all inside the caller's workspace).
struct DevPlan {
  const FrontInfo *fronts;
  const int32_t *children, *inv, *relpos, *sri;
  const Task *build, *gemm, *potrf, *trsm, *syrk, *gath, *sdiag, *sgemv, *rgemv;
  const int64_t *toff;
  const Task *fs_inv, *ps_tasks;  // persistent FP32 solve
  const int64_t *ps_pbase;        // per front: first partial-sum row of its backward tasks
  const int32_t *ps_kid_chunks;   // per front: below-front chunks of all its children
  const SolveRec *ps_recs;        // per task: the task with its front's data
  const int32_t *ps_parent_blocks;  // per front: diagonal blocks of its parent
  const int64_t *fs_dinv_off;
  const int32_t *fs_first_slot;  // per front: slot of its first diagonal block
  const int64_t *k_slot, *k_poff, *k_w, *k_orig;
  const int32_t *k_pa, *k_pb, *k_diag;
  const int32_t *perm;  // final new -> old
  // Pivot signs (final numbering) of a signed factorisation K = L S L^T of a
  // quasi-definite matrix (S = diag(sgn)); nullptr for Cholesky (S = I).
  const int8_t *sgn;
  // problem structure
  const int64_t *jp, *jtp;
  const int32_t *ji, *jrow, *jtpos;
  const int64_t *wfp;    // W, both triangles, CSR (for matrix-free products)
  const int32_t *wfi;
  const int64_t *wfsrc;  // index of each full-W entry in the caller's lower-CSC values
  const int32_t *lpos, *upos;  // per variable: row of its bound in g, or -1
  const int32_t *lidx, *uidx;  // per bound row: its variable
  int32_t n, m, nl, nu;
  int64_t mt, nk;
};

// Status words written by kernels (one int32 array in device memory).
enum StatusWord : int {
  ST_FAIL_COL = 0,   // smallest column with a non-positive pivot (INT32_MAX if none)
  ST_PERTURBED = 1,  // pivots replaced by the low-precision factorisation
  ST_TIMEOUT = 2,    // a bounded device-side wait of the factorisation ran out
  ST_SOLVE_TIMEOUT = 3,  // a grid barrier of the persistent solve ran out
  ST_COUNT = 8
};

// Bump allocator over the caller's workspace (base == nullptr: size only).
struct Carve {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

constexpr int kGemmTile = 64;
constexpr int kTrsmRows = 128;
constexpr int kGathPos = 256;
constexpr int kSolveRows = 128;
constexpr int kSolveCols = 256;

// Kernel launches issued by this library (host-side count, single stream of work).
int64_t &launch_counter();
inline void note_launch() { launch_counter() += 1; }

template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

}  // namespace gipm
