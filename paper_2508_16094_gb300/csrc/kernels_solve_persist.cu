// Persistent supernodal triangular solves for FP32 factors (TF32/TF32x3/BF16/FP32).
//
// After each factorisation one launch inverts every 128-wide diagonal block of
// L (explicit inverse, rows padded to a multiple of 4 floats). A solve is then
// ONE launch of a persistent kernel whose CTAs take the tasks of the plan in
// order from a global ticket counter (forward sweep leaves -> root, backward
// sweep root -> leaves). Instead of grid barriers between phases, each task
// waits only for the results it reads, published through flags and counters
// in device memory: a diagonal block of the forward sweep subtracts
// L_ij y_j as each y_j of its front appears (a wavefront down the front's
// blocks), rows below a front take every y_j and then count towards the
// front's update vector, which the parent's gathers wait for; the backward
// sweep mirrors this with partial sums over the rows below a front (waiting
// for the parent front) and x_i published block by block. A task waits only
// for earlier tasks, so the schedule cannot deadlock, and every wait is
// bounded: on expiry the status word is set and the whole launch drains.
// Three vectors keep reads disjoint from writes: a (right-hand side), b
// (forward result) and x (solution); t holds the fronts' update vectors.
// Vectors written inside the launch are read through L2 (ld.global.cg), and
// the loads of L for a block are issued before its wait.
#include <algorithm>
#include <stdexcept>
#include <string>

#include "launch.h"

namespace gipm {

namespace {

constexpr int kB = 128;                     // block width of the solve
constexpr int kT = 256;                     // threads per CTA
constexpr unsigned kBarrierSpins = 1u << 24;  // polls of >= 0.3 us each: seconds before giving up

void ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}

// Inverse of one diagonal block (jb <= 128): column c of X = L_jj^{-1} by
// forward substitution in thread c; stored as jb rows of ldi = round_up(jb, 4)
// floats with zeros above the diagonal and in the padding.
__global__ void __launch_bounds__(128) dinv_kernel(DevPlan dp, const float *__restrict__ L,
                                                   float *__restrict__ Dinv) {
  constexpr int LS = 129;
  const Task tk = dp.fs_inv[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int j = tk.a, jb = min(kB, F.ncol - j), ldi = (jb + 3) & ~3, tid = threadIdx.x;
  extern __shared__ float smd[];
  float *A = smd;             // [128][129]
  float *X = smd + 128 * LS;  // [128][129]
  const float *g = L + F.loff + (int64_t)j * F.ld + j;
  for (int e = tid; e < jb * jb; e += 128) {
    const int r = e / jb, c = e % jb;
    A[r * LS + c] = (c <= r) ? g[(int64_t)r * F.ld + c] : 0.f;
  }
  __syncthreads();
  if (tid < jb) {
    const int c = tid;
    for (int i = c; i < jb; i++) {
      float s = (i == c) ? 1.f : 0.f;
      for (int m = c; m < i; m++) s = fmaf(-A[i * LS + m], X[m * LS + c], s);
      X[i * LS + c] = s / A[i * LS + i];
    }
  }
  __syncthreads();
  float *out = Dinv + dp.fs_dinv_off[tk.b];
  for (int e = tid; e < jb * ldi; e += 128) {
    const int r = e / ldi, c = e % ldi;
    out[e] = (c <= r && c < jb) ? X[r * LS + c] : 0.f;
  }
}

struct PsArgs {
  DevPlan dp;
  const float *L, *Dinv;
  float *a, *b, *x, *t, *part;
  int32_t q0, q1;    // tasks [q0, q1) of the plan
  unsigned *flags;   // plan.ps_flag_words words, zeroed before the launch
  int32_t *status;   // ST_SOLVE_TIMEOUT
  unsigned spins;    // polls before a wait gives up
  int32_t withhold;  // test of the bounded wait: the task of this ticket is abandoned (-1: none)
  int32_t nslot, nfr;
  int32_t fwd_here;  // the forward sweep runs in this launch: backward blocks wait for their y
};

constexpr int kRC = 128;  // rows below a front per task
constexpr int kMaxKids = 32;  // children staged in shared memory for the gathers
constexpr long long kCopySpinCycles = 2000000000ll;  // bounded wait on a staging copy (~1 s)

__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }

__device__ __forceinline__ float4 fma4(const float4 l, float y, float4 acc) {
  acc.x = fmaf(l.x, y, acc.x);
  acc.y = fmaf(l.y, y, acc.y);
  acc.z = fmaf(l.z, y, acc.z);
  acc.w = fmaf(l.w, y, acc.w);
  return acc;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Flag words (see Plan): tickets, then per slot y / x published and partial
// sums done, per front update-vector chunks and column blocks done.
__device__ __forceinline__ unsigned *f_ticket(const PsArgs &A) { return A.flags; }
__device__ __forceinline__ unsigned *f_y(const PsArgs &A, int slot) { return A.flags + 32 + slot; }
__device__ __forceinline__ unsigned *f_x(const PsArgs &A, int slot) { return A.flags + 32 + A.nslot + slot; }
__device__ __forceinline__ unsigned *f_part(const PsArgs &A, int slot) {
  return A.flags + 32 + 2 * A.nslot + slot;
}
// per front: chunks of rows below its children that are done (the children's
// update vectors are complete once it reaches ps_kid_chunks[front])
__device__ __forceinline__ unsigned *f_tvec(const PsArgs &A, int front) {
  return A.flags + 32 + 3 * A.nslot + front;
}
__device__ __forceinline__ unsigned *f_front(const PsArgs &A, int front) {
  return A.flags + 32 + 3 * A.nslot + A.nfr + front;
}

// Shared scratch of one CTA (dynamic shared memory).
struct PsShared {
  float di[kB * kB];            // staged inverse of a diagonal block (TMA bulk copy)
  float sv[kB];                 // values handed to the diagonal-block solve
  float xs[kRC];                // solution entries of the rows below a front
  float red[kT / 32][16][33];   // per-warp transpose reduction of 16 row sums
  float4 red4[kT / 32][32];     // per-row-group column sums
  unsigned long long mbar;      // completion of the staging copy
  uint32_t parity;              // its phase
  int tk;                       // this CTA's current task
  int ok;                       // outcome of the last wait
  int ready;                    // blocks of the running chain known to be published
  int nkids;                    // children of the task's front staged below
  int64_t kid_inv[kMaxKids];    // their child -> front map offsets
  int64_t kid_toff[kMaxKids];   // their update-vector offsets
  alignas(16) SolveRec rec[2];  // the running task's record and the next one's
};

// Thread 0: start the bulk copy of a diagonal-block inverse into S.di.
__device__ __forceinline__ void stage_dinv(const PsArgs &A, PsShared &S, int slot, int jb) {
  const uint32_t bytes = (uint32_t)(jb * ((jb + 3) & ~3) * (int)sizeof(float));
  const float *src = A.Dinv + A.dp.fs_dinv_off[slot];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.mbar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(S.di)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(&S.mbar))
      : "memory");
}

// All threads: bounded wait for the staging copy; false after a timeout (the
// status word is set, and a second bounded wait lets the copy land first).
__device__ bool wait_dinv(const PsArgs &A, PsShared &S) {
  const uint32_t par = S.parity;
  auto try_wait = [&]() {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(&S.mbar)), "r"(par)
        : "memory");
    return done != 0;
  };
  bool ok = true;
  long long t0 = clock64();
  while (!try_wait()) {
    if (clock64() - t0 > kCopySpinCycles) {
      ok = false;
      atomicExch(A.status + ST_SOLVE_TIMEOUT, 1);
      t0 = clock64();
      while (!try_wait() && clock64() - t0 < kCopySpinCycles) {
      }
      break;
    }
  }
  ok = __syncthreads_and(ok) != 0;  // one outcome for the whole CTA
  if (threadIdx.x == 0) S.parity = par ^ 1u;
  return ok;
}

// Row sums of 16 consecutive rows per warp: p[k] = <row k, v> for the lane's 4
// columns; returns the full sum of row `lane` in lanes 0..15.
__device__ __forceinline__ float rows16_reduce(PsShared &S, const float (&p)[16]) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int k = 0; k < 16; k++) S.red[warp][k][lane] = p[k];
  __syncwarp();
  float s = 0.f;
  if (lane < 16) {
#pragma unroll 8
    for (int q = 0; q < 32; q++) s += S.red[warp][lane][q];
  }
  __syncwarp();
  return s;
}

// b[first + j + r] = sum_c Dinv[r][c] v[c]  (Dinv staged in S.di, v = S.sv
// zero past jb); warp w takes rows 16w .. 16w + 15
__device__ void diag_fwd(const PsArgs &A, PsShared &S, const FrontInfo &F, int j) {
  const int jb = min(kB, F.ncol - j), ldi = (jb + 3) & ~3;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, c = 4 * lane, rw = 16 * warp;
  if (rw >= jb) return;  // whole warp idle (uniform per warp)
  const float4 v4 = *reinterpret_cast<const float4 *>(S.sv + c);
  float p[16];
#pragma unroll
  for (int k = 0; k < 16; k++) {
    p[k] = 0.f;
    if (c < ldi && rw + k < jb) {
      const float4 d = *reinterpret_cast<const float4 *>(S.di + (rw + k) * ldi + c);
      p[k] = d.x * v4.x + d.y * v4.y + d.z * v4.z + d.w * v4.w;
    }
  }
  const float s = rows16_reduce(S, p);
  if (lane < 16 && rw + lane < jb) A.b[F.first + j + rw + lane] = s;
}

// x[first + j + c] = sum_{r >= c} Dinv[r][c] v[r]  (Dinv staged in S.di, zero
// above the diagonal; v = S.sv); thread (g, q): columns 4q .. 4q + 3, rows
// 16g .. 16g + 15
__device__ void diag_bwd(const PsArgs &A, PsShared &S, const FrontInfo &F, int j) {
  const int jb = min(kB, F.ncol - j), ldi = (jb + 3) & ~3;
  const int q = threadIdx.x % 32, g = threadIdx.x / 32, c = 4 * q;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c < ldi) {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int r = 16 * g + k;
      if (r < jb) acc = fma4(*reinterpret_cast<const float4 *>(S.di + r * ldi + c), S.sv[r], acc);
    }
  }
  S.red4[g][q] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float4 s = S.red4[0][q];
#pragma unroll
    for (int h = 1; h < kT / 32; h++) {
      const float4 o = S.red4[h][q];
      s.x += o.x; s.y += o.y; s.z += o.z; s.w += o.w;
    }
    float *xo = A.x + F.first + j;
    if (c + 0 < jb) xo[c + 0] = s.x;
    if (c + 1 < jb) xo[c + 1] = s.y;
    if (c + 2 < jb) xo[c + 2] = s.z;
    if (c + 3 < jb) xo[c + 3] = s.w;
  }
}

// Thread 0 polls *w until it reaches target (acquire), at most A.spins times
// and only while no other wait of the launch has run out; the CTA then shares
// the outcome (and, on success, S.ready = ready unless ready < -1). On expiry
// the status word is set, and every later wait of the launch gives up at once.
__device__ bool wait_flag(const PsArgs &A, PsShared &S, const unsigned *w, unsigned target,
                          int ready = -2) {
  __syncthreads();  // every thread has read the previous outcome
  if (threadIdx.x == 0) {
    unsigned v, spins = 0;
    int ok = 1;
    while (true) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(w) : "memory");
      if (v >= target) break;
      if ((spins & 63u) == 0 && *(volatile int32_t *)(A.status + ST_SOLVE_TIMEOUT) != 0) {
        ok = 0;
        break;
      }
      if (++spins > A.spins) {
        atomicExch(A.status + ST_SOLVE_TIMEOUT, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    S.ok = ok;
    if (ok && ready >= -1) S.ready = ready;
  }
  __syncthreads();
  return S.ok != 0;
}

// Wait for block j of a chain whose flags are published in order (each
// producer acquired its predecessor's flag before releasing its own), with
// `last` the last block this task needs: one acquire of the last flag makes
// every earlier block visible, so a task behind the chain waits once and then
// streams its blocks without polling. S.ready holds the highest block known
// published (reset by the caller to -1).
__device__ bool wait_chain(const PsArgs &A, PsShared &S, const unsigned *flags, int j, int last,
                           int step) {
  if ((step > 0 ? j <= S.ready : j >= S.ready) && S.ready >= 0) return true;
  __syncthreads();  // every thread has read S.ready and the previous outcome
  if (threadIdx.x == 0) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flags + last) : "memory");
    if (v >= 1u) S.ready = last;
  }
  __syncthreads();
  if (S.ready == last) return true;
  return wait_flag(A, S, flags + j, 1, j);
}

// After this CTA's writes: count one more on *w. The barrier orders every
// thread's writes before thread 0's release add, and a release is cumulative,
// so a consumer that acquires the count sees all of them.
__device__ void signal(unsigned *w) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(w) : "memory");
}

// Wait until the update vectors of all children of front s are complete (one
// counter per front), and stage the children's map and vector offsets.
__device__ bool wait_children(const PsArgs &A, PsShared &S, const FrontInfo &F, const SolveRec &R) {
  const DevPlan &dp = A.dp;
  const int nk = F.child_end - F.child_begin;
  if (threadIdx.x < min(nk, kMaxKids)) {
    const int32_t ch = dp.children[F.child_begin + threadIdx.x];
    S.kid_inv[threadIdx.x] = dp.fronts[ch].inv_off;
    S.kid_toff[threadIdx.x] = dp.toff[ch];
  }
  if (threadIdx.x == 0) S.nkids = nk;
  if (nk == 0) {
    __syncthreads();
    return true;
  }
  return wait_flag(A, S, f_tvec(A, R.task.front), (unsigned)R.kid_chunks);  // (syncs first)
}

// Sum of the children's update entries at front position p (after
// wait_children), in child order; the map entries of two children are loaded
// together, then their update entries.
__device__ __forceinline__ float gather_children(const PsArgs &A, const PsShared &S,
                                                 const FrontInfo &F, int p) {
  const DevPlan &dp = A.dp;
  auto offs = [&](int k, int64_t &io, int64_t &to) {
    if (k < kMaxKids) {
      io = S.kid_inv[k];
      to = S.kid_toff[k];
    } else {
      const int32_t ch = dp.children[F.child_begin + k];
      io = dp.fronts[ch].inv_off;
      to = dp.toff[ch];
    }
  };
  float v = 0.f;
  const int nk = S.nkids;
  int k = 0;
  for (; k + 1 < nk; k += 2) {
    int64_t io0, to0, io1, to1;
    offs(k, io0, to0);
    offs(k + 1, io1, to1);
    const int32_t q0 = dp.inv[io0 + p], q1 = dp.inv[io1 + p];
    const float t0 = q0 >= 0 ? ldcg(A.t + to0 + q0) : 0.f;
    const float t1 = q1 >= 0 ? ldcg(A.t + to1 + q1) : 0.f;
    if (q0 >= 0) v += t0;
    if (q1 >= 0) v += t1;
  }
  if (k < nk) {
    int64_t io, to;
    offs(k, io, to);
    const int32_t q = dp.inv[io + p];
    if (q >= 0) v += ldcg(A.t + to + q);
  }
  return v;
}

// The CTA's next ticket and its task record (registers of thread 32), taken
// once the running task has passed its last wait: the atomic and the load of
// the record then overlap the task's remaining work, and no CTA ever holds a
// ticket while it waits, so the smallest unfinished ticket is always running.
struct Next {
  int q;
  bool have;
};

__device__ __forceinline__ void take_next(const PsArgs &A, Next &N) {
  if (threadIdx.x == 32 && !N.have) {
    N.q = (int)atomicAdd(f_ticket(A), 1u) + A.q0;  // the result is first read after the task
    N.have = true;
  }
}

// Thread 32: start the asynchronous copy of record q into S.rec[buf], and
// warm L2 with the record one grid further on.
__device__ __forceinline__ void fetch_rec(const PsArgs &A, PsShared &S, int q, int buf) {
  if (q >= A.q1) return;
  const char *src = reinterpret_cast<const char *>(A.dp.ps_recs + q);
  const uint32_t dst = smem_u32(&S.rec[buf]);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(SolveRec) / 16); k++)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * k), "l"(src + 16 * k)
                 : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  const int ahead = min(q + (int)gridDim.x, A.q1 - 1);
  asm volatile("prefetch.global.L2 [%0];" ::"l"(A.dp.ps_recs + ahead));
}

// Forward, diagonal block i of front s: rows j0 .. j0 + jb of the front.
// warp w: rows 16w .. 16w + 15, lane: columns 4 lane .. 4 lane + 3 of block j
// (the loads of block j are issued before y_j is waited for).
__device__ void fwd_diag(const PsArgs &A, PsShared &S, const SolveRec &R, Next &N) {
  const Task &tk = R.task;
  const FrontInfo &F = R.front;
  const DevPlan &dp = A.dp;
  const int i = tk.a, j0 = kB * i, jb = min(kB, F.ncol - j0), slot0 = R.slot0;
  if (threadIdx.x == 0) stage_dinv(A, S, slot0 + i, jb);
  bool ok = wait_children(A, S, F, R);
  if (ok && threadIdx.x < kB)
    S.sv[threadIdx.x] = threadIdx.x < jb
                            ? ldcg(A.a + F.first + j0 + threadIdx.x) - gather_children(A, S, F, j0 + threadIdx.x)
                            : 0.f;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, c = 4 * lane, rw = 16 * warp;
  // per-thread partial row sums over the lane's 4 columns of every block,
  // reduced across the warp once after the last block
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; k++) acc[k] = 0.f;
  if (threadIdx.x == 0) S.ready = -1;
  __syncthreads();  // no thread reads the previous task's value
  for (int j = 0; j < i && ok; j++) {
    float4 l[16];
    const float *P = A.L + F.loff + (int64_t)(j0 + rw) * F.ld + kB * j + c;
#pragma unroll
    for (int k = 0; k < 16; k++)
      l[k] = rw + k < jb ? __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    ok = wait_chain(A, S, f_y(A, slot0), j, i - 1, 1);
    if (!ok) break;
    const float *yb = A.b + F.first + kB * j + c;  // block j < i is a full block
    const float4 y4 = make_float4(ldcg(yb), ldcg(yb + 1), ldcg(yb + 2), ldcg(yb + 3));
#pragma unroll
    for (int k = 0; k < 16; k++)
      acc[k] = fmaf(l[k].x, y4.x, fmaf(l[k].y, y4.y, fmaf(l[k].z, y4.z, fmaf(l[k].w, y4.w, acc[k]))));
  }
  take_next(A, N);
  const float racc = rows16_reduce(S, acc);  // rows of this warp only
  if (ok && lane < 16 && rw + lane < jb) S.sv[rw + lane] -= racc;
  // the staged copy always lands before S.di is reused; the wait ends with a
  // barrier, after which every row of S.sv is final
  const bool got = wait_dinv(A, S);
  if (ok && got) {
    diag_fwd(A, S, F, j0);
    signal(f_y(A, slot0 + i));
  }
}

// Forward, rows r0 .. r0 + nr below front s: the children's entries plus
// L_rj y_j over every block j of the front, into the front's update vector.
__device__ void fwd_below(const PsArgs &A, PsShared &S, const SolveRec &R, Next &N) {
  const Task &tk = R.task;
  const FrontInfo &F = R.front;
  const DevPlan &dp = A.dp;
  const int r0 = tk.a, nr = min(kRC, F.nrow - r0), nb = (F.ncol + kB - 1) / kB;
  const int slot0 = R.slot0;
  bool ok = wait_children(A, S, F, R);
  if (ok && threadIdx.x < nr) S.xs[threadIdx.x] = gather_children(A, S, F, F.ncol + r0 + threadIdx.x);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, c = 4 * lane, rw = 16 * warp;
  float acc[16];  // partial row sums, reduced once after the last block
#pragma unroll
  for (int k = 0; k < 16; k++) acc[k] = 0.f;
  if (threadIdx.x == 0) S.ready = -1;
  __syncthreads();  // no thread reads the previous task's value
  for (int j = 0; j < nb && ok; j++) {
    const int jbj = min(kB, F.ncol - kB * j);
    float4 l[16];
    const float *P = A.L + F.loff + (int64_t)(F.ncol + r0 + rw) * F.ld + kB * j + c;
#pragma unroll
    for (int k = 0; k < 16; k++)
      l[k] = (c < jbj && rw + k < nr) ? __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    ok = wait_chain(A, S, f_y(A, slot0), j, nb - 1, 1);
    if (!ok) break;
    // columns past ncol (the padding of the last block) never enter the sums
    const float *yb = A.b + F.first + kB * j + c;
    const float4 y4 = make_float4(c < jbj ? ldcg(yb) : 0.f, c + 1 < jbj ? ldcg(yb + 1) : 0.f,
                                  c + 2 < jbj ? ldcg(yb + 2) : 0.f, c + 3 < jbj ? ldcg(yb + 3) : 0.f);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      float4 v = l[k];
      if (c + 1 >= jbj) v.y = 0.f;
      if (c + 2 >= jbj) v.z = 0.f;
      if (c + 3 >= jbj) v.w = 0.f;
      acc[k] = fmaf(v.x, y4.x, fmaf(v.y, y4.y, fmaf(v.z, y4.z, fmaf(v.w, y4.w, acc[k]))));
    }
  }
  take_next(A, N);
  const float racc = rows16_reduce(S, acc);
  __syncthreads();
  if (ok) {
    if (lane < 16 && rw + lane < nr) A.t[R.toff + r0 + rw + lane] = S.xs[rw + lane] + racc;
    signal(f_tvec(A, F.parent));  // rows below a front exist only below a parent
  }
}

// Backward, rows r0 .. r0 + nr below front s: once the parent front (and so
// every ancestor holding those rows) is solved, the partial sums
// part[cb][c] = sum_r L[ncol + r0 + r, 128 cb + c] x[row r] of every column
// block, last block first (the order of the front's backward chain), each
// published as it is written. Thread (g, q): columns 4q .. 4q + 3, rows
// 16g .. 16g + 15; the loads of the next block are issued before the
// reduction of the current one.
__device__ void bwd_part(const PsArgs &A, PsShared &S, const SolveRec &R, Next &N) {
  const Task &tk = R.task;
  const FrontInfo &F = R.front;
  const DevPlan &dp = A.dp;
  const int r0 = tk.b, nr = min(kRC, F.nrow - r0), nb = (F.ncol + kB - 1) / kB;
  const int nbl = (F.nrow + kRC - 1) / kRC;
  const int q = threadIdx.x % 32, g = threadIdx.x / 32;
  const float *P = A.L + F.loff + (int64_t)(F.ncol + r0 + 16 * g) * F.ld + 4 * q;
  float4 l[16];
  auto load = [&](int cb) {
    const int c = kB * cb + 4 * q;
#pragma unroll
    for (int k = 0; k < 16; k++)
      l[k] = (c < F.ncol && 16 * g + k < nr)
                 ? __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld + kB * cb))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  load(nb - 1);
  const int32_t xrow = threadIdx.x < nr ? dp.sri[F.rows_off + r0 + threadIdx.x] : 0;
  if (F.parent >= 0 && !wait_flag(A, S, f_front(A, F.parent), (unsigned)R.parent_blocks))
    return;
  take_next(A, N);
  if (threadIdx.x < nr) S.xs[threadIdx.x] = ldcg(A.x + xrow);
  __syncthreads();
  for (int cb = nb - 1; cb >= 0; cb--) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 16; k++)
      if (16 * g + k < nr) acc = fma4(l[k], S.xs[16 * g + k], acc);
    if (cb > 0) load(cb - 1);
    S.red4[g][q] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      float4 sm = S.red4[0][q];
#pragma unroll
      for (int h = 1; h < kT / 32; h++) {
        const float4 o = S.red4[h][q];
        sm.x += o.x; sm.y += o.y; sm.z += o.z; sm.w += o.w;
      }
      const int64_t row = R.pbase + (int64_t)cb * nbl + r0 / kRC;
      reinterpret_cast<float4 *>(A.part + row * kB)[q] = sm;
    }
    signal(f_part(A, R.slot0 + cb));  // (its barrier also frees S.red4)
  }
}

// Backward, column block cb of front s: the partial sums in chunk order, then
// L[block i, block cb]^T x_i for i > cb as each x_i is published, then
// x_cb = L_cc^{-T} (.) with the staged inverse.
__device__ void bwd_diag(const PsArgs &A, PsShared &S, const SolveRec &R, Next &N) {
  const Task &tk = R.task;
  const FrontInfo &F = R.front;
  const DevPlan &dp = A.dp;
  const int cb = tk.a, c0 = kB * cb, jb = min(kB, F.ncol - c0), nb = (F.ncol + kB - 1) / kB;
  const int nbl = (F.nrow + kRC - 1) / kRC, slot0 = R.slot0;
  if (threadIdx.x == 0) stage_dinv(A, S, slot0 + cb, jb);
  // b of this block is the forward result: published by this launch's forward
  // task of the block, or complete before a backward-only launch
  bool ok = !A.fwd_here || wait_flag(A, S, f_y(A, slot0 + cb), 1);
  if (ok && nbl > 0) ok = wait_flag(A, S, f_part(A, slot0 + cb), nbl);  // implies the parent is done
  else if (ok && F.parent >= 0)
    ok = wait_flag(A, S, f_front(A, F.parent), (unsigned)R.parent_blocks);
  if (ok && threadIdx.x < kB) {
    float v = 0.f;
    if (threadIdx.x < jb) {
      const float *pp = A.part + (R.pbase + (int64_t)cb * nbl) * kB + threadIdx.x;
      float ps = 0.f;
      for (int k = 0; k < nbl; k++) ps += ldcg(pp + (int64_t)k * kB);
      v = ldcg(A.b + F.first + c0 + threadIdx.x) - ps;
    }
    S.sv[threadIdx.x] = v;
  }
  const int q = threadIdx.x % 32, g = threadIdx.x / 32, c = c0 + 4 * q;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) S.ready = -1;
  __syncthreads();  // no thread reads the previous task's value
  for (int i = nb - 1; i > cb && ok; i--) {
    const int jbi = min(kB, F.ncol - kB * i);
    float4 l[16];
    const float *P = A.L + F.loff + (int64_t)(kB * i + 16 * g) * F.ld + c;
#pragma unroll
    for (int k = 0; k < 16; k++)
      l[k] = (c < F.ncol && 16 * g + k < jbi) ? __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
    ok = wait_chain(A, S, f_x(A, slot0), i, cb + 1, -1);
    if (!ok) break;
    // lane k < 16 loads x of row 16 g + k of block i; the warp shares them
    const float xv = (q < 16 && 16 * g + q < jbi) ? ldcg(A.x + F.first + kB * i + 16 * g + q) : 0.f;
#pragma unroll
    for (int k = 0; k < 16; k++) acc = fma4(l[k], __shfl_sync(0xffffffffu, xv, k), acc);
  }
  take_next(A, N);
  S.red4[g][q] = acc;
  __syncthreads();
  if (ok && threadIdx.x < 32) {
    float4 sm = S.red4[0][q];
#pragma unroll
    for (int h = 1; h < kT / 32; h++) {
      const float4 o = S.red4[h][q];
      sm.x += o.x; sm.y += o.y; sm.z += o.z; sm.w += o.w;
    }
    const float d[4] = {sm.x, sm.y, sm.z, sm.w};
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (4 * q + k < jb) S.sv[4 * q + k] -= d[k];
  }
  const bool got = wait_dinv(A, S);  // (ends with a barrier)
  if (ok && got) {
    diag_bwd(A, S, F, c0);
    signal(f_x(A, slot0 + cb));
    if (threadIdx.x == 0)  // the release of signal() above already ordered the writes
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(f_front(A, tk.front)) : "memory");
  }
}

// Persistent solve: every CTA takes tasks in plan order from the global ticket
// counter until the range is exhausted.
__global__ void __launch_bounds__(kT, 2) psolve_kernel(PsArgs A) {
  extern __shared__ __align__(128) unsigned char ps_smem[];
  PsShared &S = *reinterpret_cast<PsShared *>(ps_smem);
  // Thread 32 takes the tickets: the first here, each next one inside the
  // running task once it has passed its last wait (take_next), or right after
  // a task that ended early; the next task's record is copied into the other
  // shared buffer while the CTA finishes the current one.
  Next N{0, false};
  int cur = 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar)), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.parity = 0;
  }
  if (threadIdx.x == 32) {
    const int q = (int)atomicAdd(f_ticket(A), 1u) + A.q0;
    fetch_rec(A, S, q, 0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    S.tk = q;
  }
  __syncthreads();
  while (true) {
    const int qt = S.tk;
    if (qt >= A.q1) break;
    const SolveRec &R = S.rec[cur];
    N.have = false;
    if (qt == A.withhold) {
      // abandoned (test of the bounded waits): the tasks that need its result
      // run out of time
    } else switch (R.task.c) {
      case WS_FWD_DIAG: fwd_diag(A, S, R, N); break;
      case WS_FWD_BELOW: fwd_below(A, S, R, N); break;
      case WS_BWD_PART: bwd_part(A, S, R, N); break;
      default: bwd_diag(A, S, R, N); break;
    }
    take_next(A, N);  // a task that gave up early
    if (threadIdx.x == 32) {
      fetch_rec(A, S, N.q, cur ^ 1);
      asm volatile("cp.async.wait_all;" ::: "memory");
      S.tk = N.q;
    }
    __syncthreads();  // the next record has landed; the shared scratch is free
    cur ^= 1;
  }
}

int psolve_grid(int ntask) {
  static int per_device[64] = {0};
  int dev = 0;
  ck(cudaGetDevice(&dev), "cudaGetDevice");
  int &g = per_device[dev & 63];
  if (g == 0) {
    int sms = 0, nb = 0;
    ck(cudaFuncSetAttribute(psolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sizeof(PsShared)),
       "solve shared-memory attribute");
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, psolve_kernel, kT, sizeof(PsShared)),
       "occupancy");
    g = std::max(1, sms * std::min(nb, 2));
  }
  return std::max(1, std::min(g, ntask));
}

}  // namespace

void launch_dinv(const DevPlan &dp, const Plan &plan, const float *L, float *Dinv,
                 cudaStream_t st) {
  const int n = (int)plan.fs_inv.size();
  if (n == 0) return;
  const int smem = 2 * 128 * 129 * (int)sizeof(float);
  static bool attr = false;
  if (!attr) {
    ck(cudaFuncSetAttribute(dinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "dinv attribute");
    attr = true;
  }
  note_launch();
  dinv_kernel<<<n, 128, smem, st>>>(dp, L, Dinv);
}

void launch_psolve(const DevPlan &dp, const Plan &plan, const float *L, const float *Dinv, float *a,
                   float *b, float *x, float *t, float *part, unsigned *flags, int32_t *status,
                   bool fwd, bool bwd, cudaStream_t st, unsigned test_spins, int test_withhold) {
  const int32_t q0 = fwd ? 0 : plan.ps_fwd_tasks;
  const int32_t q1 = bwd ? (int32_t)plan.ps_tasks.size() : plan.ps_fwd_tasks;
  if (q1 <= q0) return;
  ck(cudaMemsetAsync(flags, 0, (size_t)plan.ps_flag_words * sizeof(unsigned), st), "solve flags");
  const int grid = psolve_grid(q1 - q0);
  PsArgs A{dp, L, Dinv, a, b, x, t, part, q0, q1, flags, status,
           test_spins ? test_spins : kBarrierSpins, test_withhold,
           (int32_t)plan.fs_dinv_off.size(), (int32_t)plan.fronts.size(), fwd && bwd ? 1 : 0};
  note_launch();
  psolve_kernel<<<grid, kT, sizeof(PsShared), st>>>(A);
  ck(cudaGetLastError(), "solve launch");
}

}  // namespace gipm
