// Host launchers of the device kernels (one stream, no synchronisation inside).
#pragma once

#include "dev.cuh"

namespace gipm {

// K = W + J^T diag(D_J) J + diag(D_bounds) + delta_p I into the compact FP64
// array kval (level-major order of the plan).
void launch_assemble(const DevPlan &dp, const double *jv, const double *D, const double *wv,
                     double delta_p, double *kval, cudaStream_t st);

// Multifrontal factorisation of all levels with SIMT FMA kernels. status must
// be initialised by the caller (ST_FAIL_COL = INT32_MAX, ST_PERTURBED = 0).
template <typename T>
void launch_factor_simt(const DevPlan &dp, const Plan &plan, const double *kval, T *L, T *U,
                        int32_t *status, bool perturb, cudaStream_t st);

// Pieces of a level of the factorisation, shared with the tensor-core path:
// front assembly (+ K entries), diagonal-block Cholesky (nb <= 128) and the
// triangular solve of the rows below (nb <= 128).
template <typename T>
void launch_build_level(const DevPlan &dp, const LevelPlan &LP, const double *kval, T *L, T *U,
                        cudaStream_t st);
template <typename T>
void launch_potrf(const DevPlan &dp, const Task *tasks, int ntasks, int nb, T *L, int32_t *status,
                  bool perturb, cudaStream_t st);
template <typename T>
void launch_trsm(const DevPlan &dp, const Task *tasks, int ntasks, int nb, T *L, cudaStream_t st);
// FP64 without pivot signs, 64-wide blocks: the panel solve with each row in registers.
void launch_trsm_f64(const DevPlan &dp, const Task *tasks, int ntasks, double *L, cudaStream_t st);

// Triangular solves with the factor: y (final numbering, length n) is
// overwritten by L^{-T} L^{-1} y (L^{-T} S L^{-1} y for a signed factor,
// dp.sgn). t: update-vector scratch (plan.t_entries).
template <typename T, typename V>
void launch_solve(const DevPlan &dp, const Plan &plan, const T *L, V *y, V *t, cudaStream_t st);

// y <- S y with the pivot signs of a signed factor (no-op without dp.sgn).
template <typename V>
void launch_sign(const DevPlan &dp, V *y, cudaStream_t st);

// Loads the level-solve kernels (FP64 and FP32) so that a later first launch
// commits no device memory (lazy module loading); used by the allocation-free solve.
cudaError_t preload_level_solve();

// Persistent FP32 solve: inverses of the 128-wide diagonal blocks (after each
// FP32 factorisation), then x = L^{-T} L^{-1} a in one launch, with b the
// forward result and t the update vectors. fwd/bwd select the sweeps: forward
// only maps a to b = L^{-1} a; backward only maps b to x = L^{-T} b. part:
// plan.ps_part_entries floats of scratch; flags: plan.ps_flag_words words
// (zeroed by the launch). A wait that runs out sets status[ST_SOLVE_TIMEOUT]
// and the launch drains. test_spins (0: the default of seconds) bounds each
// wait; test_withhold >= 0 abandons the task of that ticket (tests of
// the bounded wait).
void launch_dinv(const DevPlan &dp, const Plan &plan, const float *L, float *Dinv, cudaStream_t st);
void launch_psolve(const DevPlan &dp, const Plan &plan, const float *L, const float *Dinv, float *a,
                   float *b, float *x, float *t, float *part, unsigned *bar, int32_t *status, bool fwd,
                   bool bwd, cudaStream_t st, unsigned test_spins = 0, int test_withhold = -1);

// Sampled entries of L (final numbering).
template <typename T>
void launch_factor_entries(const DevPlan &dp, const T *L, const int32_t *col2s, int64_t count,
                           const int32_t *rows, const int32_t *cols, double *out,
                           cudaStream_t st);

}  // namespace gipm
