// Internal data structures of the solver library (host + device).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace gipm {

// ---------------------------------------------------------------------------
// Symbolic analysis (host). Final numbering = given ordering + etree postorder.
// ---------------------------------------------------------------------------
struct Symbolic {
  int32_t n = 0;
  std::vector<int32_t> perm, iperm;       // final new->old, old->new
  std::vector<int32_t> parent, colcount;  // elimination tree, column counts (incl. diagonal)
  // lower CSC pattern of K in the ORIGINAL numbering (export order)
  std::vector<int64_t> kop;
  std::vector<int32_t> koi;
  // supernodes
  int32_t nsuper = 0, nlevels = 0;
  std::vector<int32_t> super, sparent, slevel;
  std::vector<int64_t> srp;  // row structure of each supernode (rows below its columns)
  std::vector<int32_t> sri;
  int64_t nnz_l = 0;
  double flops = 0.0;
};

// Per-supernode layout of the frontal matrices (device-visible, 64 bytes).
// Front of supernode s: order nf = ncol + nrow; local index p < ncol is column
// first + p, p >= ncol is row sri[rows_off + p - ncol]. The first ncol columns
// live in the panel (row-major, nf rows x ld), the trailing nrow x nrow block
// (the update matrix handed to the parent) lives in U storage (row-major, uld).
// Front assembly tiles: kBuildTile rows x at most kBuildTile columns.
constexpr int kBuildTile = 64;

struct FrontInfo {
  int64_t loff;      // panel offset in the factor storage (elements)
  int64_t uoff;      // update matrix offset in the update storage (elements)
  int64_t rows_off;  // offset of the row structure in sri
  int64_t inv_off;   // offset of this front's map into its parent's front (length nf(parent))
  int32_t first, ncol, nrow, ld;
  int32_t uld, child_begin, child_end, parent;
};
static_assert(sizeof(FrontInfo) == 64, "FrontInfo layout");

// A unit of work of a batched kernel: meaning of a/b depends on the kernel.
struct Task {
  int32_t front, a, b, c;
};

// One task of the persistent FP32 solve with everything it reads of its front,
// so a CTA fetches what its next task needs in a single 112-byte copy.
struct SolveRec {
  Task task;
  FrontInfo front;
  int64_t toff;   // the front's update vector
  int64_t pbase;  // its first partial-sum row of the backward sweep
  int32_t slot0;  // slot of its first diagonal block
  int32_t kid_chunks;     // below-front chunks of all its children
  int32_t parent_blocks;  // diagonal blocks of its parent (0 at a root)
  int32_t pad;
};
static_assert(sizeof(SolveRec) == 112 && sizeof(SolveRec) % 16 == 0, "SolveRec layout");

// A task of the persistent FP32 solve. Tasks run in the order of the plan
// (a ticket taken from a global counter), and a task waits only for tasks
// earlier in that order (flags and counters in device memory), so the solve
// needs no grid barrier and cannot deadlock. Blocks are 128 wide.
enum SolveTaskKind : int32_t {
  WS_FWD_DIAG = 0,   // (front, a = block i): gather the children's update entries for
                     // the block's rows, subtract L_ij y_j for j < i as each y_j is
                     // published, y_i = L_ii^{-1} (.) (explicit inverse), publish y_i
  WS_FWD_BELOW = 1,  // (front, a = first row below the front of a 128-row chunk): gather,
                     // add L_rj y_j for every block j, store the front's update vector
  WS_BWD_PART = 2,   // (front, b = first row below of a 128-row chunk): partial sums
                     // L_{r,cb}^T x_r of every column block cb, last first, once the
                     // parent front is done
  WS_BWD_DIAG = 3    // (front, a = column block cb): the partial sums, L_{i,cb}^T x_i for
                     // i > cb as each x_i is published, x_cb = L_cc^{-T} (.), publish x_cb
};

// Work of one level of the supernodal tree, as ranges into the task arrays.
struct StepRange {
  int32_t gemm_b, gemm_e, potrf_b, potrf_e, trsm_b, trsm_e;
};
struct LevelPlan {
  int32_t front_b = 0, front_e = 0;  // into the level-ordered front list
  int32_t build_b = 0, build_e = 0;  // front-assembly tiles
  int64_t k_b = 0, k_e = 0;          // K entries of this level's fronts
  int32_t syrk_b = 0, syrk_e = 0;    // update-matrix tiles
  int32_t gath_b = 0, gath_e = 0;    // solve gather tasks
  int32_t rg_b = 0, rg_e = 0;        // backward-solve tasks on the rows below the block
  int32_t sdiag_b = 0, sdiag_e = 0;  // solve diagonal-block tasks, by step: see solve_steps
  std::vector<StepRange> steps;      // factor steps (block columns)
  std::vector<int32_t> sstep_b;      // solve steps: [sstep_b[j], sstep_b[j+1]) in stasks
  std::vector<int32_t> sgemv_b;      // solve update tasks per step
  int32_t max_ncol = 0;
};

// Numeric plan: everything the kernels need, built on the host by analysis.
struct Plan {
  int nb = 64;                       // factor block width
  int nbs = 64;                      // solve block width
  std::vector<FrontInfo> fronts;     // by supernode index
  std::vector<int32_t> sched;        // schedule level of each supernode (parent = child + 1)
  std::vector<int32_t> level_fronts; // supernodes sorted by (schedule level, index)
  std::vector<int32_t> children;     // child lists (ascending), ranges in FrontInfo
  std::vector<int32_t> inv;          // child -> parent-front inverse maps
  std::vector<int32_t> relpos;       // child row -> position in parent's front (by sri offset)
  std::vector<LevelPlan> levels;
  std::vector<Task> build_tasks, gemm_tasks, potrf_tasks, trsm_tasks, syrk_tasks;
  std::vector<Task> gath_tasks, sdiag_tasks, sgemv_tasks, rgemv_tasks;
  std::vector<int64_t> toff;         // per front: offset of its solve update vector (length nrow)
  int64_t t_entries = 0;
  // persistent FP32 solve: inverses of the 128-wide diagonal blocks (slot s:
  // jb rows of round_up(jb, 4) floats at fs_dinv_off[s]; the slots of a front
  // are consecutive from fs_first_slot[front]) and its task list, forward
  // tasks first. Flags (32-bit words): [0, 32) tickets, then per slot "y
  // published", "x published", "partial sums done", per front "update-vector
  // chunks of its children done", "column blocks done".
  std::vector<Task> fs_inv;                  // (front, first column, slot)
  std::vector<int32_t> fs_first_slot;        // per front: slot of block 0
  std::vector<int64_t> fs_dinv_off;
  int64_t fs_dinv_entries = 0;
  std::vector<Task> ps_tasks;                // (front, a, b, kind)
  int32_t ps_fwd_tasks = 0;
  std::vector<int64_t> ps_pbase;             // per front: first partial-sum row (128 floats each)
  std::vector<SolveRec> ps_recs;             // per task: the task and its front's data
  std::vector<int32_t> ps_kid_chunks;        // per front: below-front chunks of all its children
  std::vector<int32_t> ps_parent_blocks;     // per front: diagonal blocks of its parent (0 at roots)
  int64_t ps_part_entries = 0;               // floats of partial sums
  int64_t ps_flag_words = 0;
  // K entries in level-major order
  std::vector<int64_t> k_slot;   // element offset of L(i, j) in the factor storage
  std::vector<int64_t> k_poff;   // products [k_poff[q], k_poff[q+1])
  std::vector<int32_t> k_pa, k_pb;  // CSR positions of the two J factors of each product
  std::vector<int64_t> k_w;      // W value index or -1
  std::vector<int32_t> k_diag;   // original variable index for a diagonal entry, else -1
  std::vector<int64_t> k_orig;   // original lower-CSC entry index (export order)
  int64_t l_entries = 0, u_entries = 0;
  int32_t max_front = 0, max_ncol = 0;
};

// Problem description kept by the context (host copies).
struct Problem {
  int32_t n = 0, m = 0;
  std::vector<int64_t> jp;
  std::vector<int32_t> ji;
  std::vector<int32_t> jrow;         // row of each CSR position
  std::vector<int64_t> jtp;          // CSC of J: column pointers
  std::vector<int32_t> jtpos;        // CSR position of each CSC entry
  std::vector<int64_t> wp;
  std::vector<int32_t> wi;
  std::vector<double> l, u;
  int32_t nl = 0, nu = 0;
  int64_t mt = 0;
  std::vector<int32_t> lidx, uidx;   // variables with a finite lower/upper bound
  std::vector<int32_t> lpos, upos;   // per variable: row of its bound in g (or -1)
};

void analyze_symbolic(const Problem &P, const int32_t *perm, Symbolic &S);
void build_plan(const Problem &P, const Symbolic &S, Plan &plan, int nb, int nbs);
void validate_plan(const Problem &P, const Symbolic &S, const Plan &plan);
// Task lists of the fused FP32 solve (128-wide blocks), appended to the plan.
void build_fused_solve(Plan &plan);

}  // namespace gipm
