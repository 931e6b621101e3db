// Persistent supernodal triangular solves for FP32 factors (TF32/TF32x3/FP32).
//
// After each factorisation one launch inverts every 128-wide diagonal block of
// L (explicit inverse, rows padded to a multiple of 4 floats). A solve is then
// ONE cooperative launch that walks the phases of the plan (forward sweep
// leaves -> root, backward sweep root -> leaves) with a grid barrier between
// phases. Per block step only the update of the rows (forward) or columns
// (backward) outside the diagonal block is spread over the grid; the block that
// owns the next diagonal block finishes its own update and then applies that
// block's inverse, so each step costs one barrier and the inverse is read once.
// Three vectors keep every read of a phase disjoint from its writes: a (right-
// hand side, updated in place), b (forward result, then updated in place by the
// backward sweep) and x (solution); t holds the update vectors of the fronts.
// Vectors written inside the launch are read through L2 (ld.global.cg).
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
  int32_t p0, p1;   // phases [p0, p1)
  unsigned *bar;    // [2..3] 64-bit arrival counter of the grid barrier
  int32_t *status;  // ST_SOLVE_TIMEOUT
  unsigned spins;   // polls before a barrier wait gives up
  int32_t withhold; // test of the bounded wait: this CTA leaves at its first barrier (-1: none)
};

constexpr int kMaxGrid = 1024;  // CTAs of one cooperative solve launch
constexpr int kRC = 128;  // rows below a front per partial-sum task
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

// Grid-wide barrier of a cooperative launch (all CTAs co-resident): one
// 64-bit arrival counter (words 2-3 of the barrier state) that only grows. A
// CTA adds 1 (release) and waits (acquire) until the counter reaches the next
// multiple of the grid size above the value it found, so launches need no
// reset as long as every barrier of the previous one completed (after a
// timeout the host zeroes the state). Every wait is bounded (max_spins polls);
// on a timeout the status word is set and all CTAs return false; a CTA that
// sees the word set by another one stops waiting too. The CTA `withhold`
// (tests of the bounded wait) returns false at once without arriving, so the
// other CTAs' waits run out.
__device__ bool grid_barrier(unsigned *bar, int32_t *status, unsigned max_spins, int withhold) {
  __shared__ int ok;
  __syncthreads();
  if ((int)blockIdx.x == withhold) return false;
  if (threadIdx.x == 0) {
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(bar + 2);
    unsigned long long old, v;
    __threadfence();
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(ctr) : "memory");
    const unsigned long long G = gridDim.x, target = (old / G + 1) * G;
    unsigned spins = 0;
    while (true) {
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (++spins > max_spins) {
        atomicExch(status + ST_SOLVE_TIMEOUT, 1);
        break;
      }
      if ((spins & 63u) == 0 && *(volatile int32_t *)(status + ST_SOLVE_TIMEOUT) != 0) break;
      __nanosleep(16);
    }
    __threadfence();
    ok = *(volatile int32_t *)(status + ST_SOLVE_TIMEOUT) == 0;
  }
  __syncthreads();
  return ok != 0;
}

// Shared scratch of one CTA (dynamic shared memory).
struct PsShared {
  float di[kB * kB];            // staged inverse of a diagonal block (TMA bulk copy)
  float sy[kB];                 // block vector of a step
  float sv[kB];                 // values handed to the diagonal-block solve
  float xs[kRC];                // solution entries of the rows below a front
  float red[kT / 32][16][33];   // per-warp transpose reduction of 16 row sums
  float4 red4[kT / 32][32];     // per-row-group column sums
  unsigned long long mbar;      // completion of the staging copy
  uint32_t parity;              // its phase
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
  ok = __syncthreads_and(ok) != 0;  // one verdict for the whole CTA
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

// forward gather: a[cols] -= sum of the children's update entries, t[rows] =
// that sum; the chunk holding block 0 then solves it
__device__ void fwd_gather(const PsArgs &A, PsShared &S, const Task &tk, const FrontInfo &F) {
  const DevPlan &dp = A.dp;
  const bool owner = tk.b >= 0;
  if (owner && threadIdx.x == 0) stage_dinv(A, S, tk.b, min(kB, F.ncol));
  const int nf = F.ncol + F.nrow, p = tk.a + threadIdx.x;
  if (p < nf) {
    float v = 0.f;
    for (int ci = F.child_begin; ci < F.child_end; ci++) {
      const int32_t ch = dp.children[ci];
      const int32_t q = dp.inv[dp.fronts[ch].inv_off + p];
      if (q >= 0) v += ldcg(A.t + dp.toff[ch] + q);
    }
    if (p < F.ncol) {
      const float y = ldcg(A.a + F.first + p) - v;
      A.a[F.first + p] = y;
      if (p < kB) S.sv[p] = y;
    } else {
      A.t[dp.toff[tk.front] + p - F.ncol] = v;
    }
  }
  if (owner) {
    if (threadIdx.x < kB && threadIdx.x >= min(kB, F.ncol)) S.sv[threadIdx.x] = 0.f;
    if (wait_dinv(A, S)) diag_fwd(A, S, F, 0);
  }
}

// forward step of block column j: rows [i0, i0 + 128) below the block take
// L[r, j:j+jb] y_j (warp w: rows i0 + 16w .. + 15, every load issued before
// y_j arrives); the chunk right below the block then solves the next one
__device__ void fwd_step(const PsArgs &A, PsShared &S, const Task &tk, const FrontInfo &F) {
  const DevPlan &dp = A.dp;
  const int nf = F.ncol + F.nrow, i0 = tk.a, j = tk.b, jb = min(kB, F.ncol - j);
  const bool owner = tk.c >= 0;
  if (owner && threadIdx.x == 0) stage_dinv(A, S, tk.c, min(kB, F.ncol - (j + kB)));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, c = 4 * lane;
  const int rw = i0 + 16 * warp, r1 = min(i0 + kB, nf), r = rw + lane;
  float4 l[16];
  const float *P = A.L + F.loff + (int64_t)rw * F.ld + j + c;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    l[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < jb && rw + k < r1) l[k] = __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld));
  }
  float *dst = nullptr;
  float old = 0.f;
  if (lane < 16 && r < r1) {
    dst = r < F.ncol ? A.a + F.first + r : A.t + dp.toff[tk.front] + r - F.ncol;
    old = ldcg(dst);
  }
  if (threadIdx.x < kB) S.sy[threadIdx.x] = threadIdx.x < jb ? ldcg(A.b + F.first + j + threadIdx.x) : 0.f;
  __syncthreads();
  if (rw < r1) {
    const float4 y4 = *reinterpret_cast<const float4 *>(S.sy + c);
    float p[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      float4 v = l[k];
      if (c + 1 >= jb) v.y = 0.f;
      if (c + 2 >= jb) v.z = 0.f;
      if (c + 3 >= jb) v.w = 0.f;
      p[k] = v.x * y4.x + v.y * y4.y + v.z * y4.z + v.w * y4.w;
    }
    const float s = rows16_reduce(S, p);
    if (dst) {
      if (r < F.ncol) {
        const float y = old - s;
        *dst = y;
        if (owner) S.sv[r - i0] = y;
      } else {
        *dst = old + s;
      }
    }
  }
  if (owner) {
    const int jbn = min(kB, F.ncol - (j + kB));
    __syncthreads();
    if (threadIdx.x < kB && threadIdx.x >= jbn) S.sv[threadIdx.x] = 0.f;
    if (wait_dinv(A, S)) diag_fwd(A, S, F, j + kB);
  }
}

// backward, rows below the front, one 128-row chunk: partial sums
// part[slot][c] = sum_r L[ncol + r0 + r, c0 + c] x[row r]; thread (g, q):
// columns 4q .. 4q + 3, rows 16g .. 16g + 15 (loads issued before x arrives)
__device__ void bwd_part(const PsArgs &A, PsShared &S, const Task &tk, const FrontInfo &F) {
  const DevPlan &dp = A.dp;
  const int c0 = tk.a, r0 = tk.b, nr = min(kRC, F.nrow - r0);
  const int q = threadIdx.x % 32, g = threadIdx.x / 32, c = c0 + 4 * q;
  float4 l[16];
  const float *P = A.L + F.loff + (int64_t)(F.ncol + r0 + 16 * g) * F.ld + c;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    l[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < F.ncol && 16 * g + k < nr) l[k] = __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld));
  }
  if (threadIdx.x < nr) S.xs[threadIdx.x] = ldcg(A.x + dp.sri[F.rows_off + r0 + threadIdx.x]);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 16; k++)
    if (16 * g + k < nr) acc = fma4(l[k], S.xs[16 * g + k], acc);
  S.red4[g][q] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float4 s = S.red4[0][q];
#pragma unroll
    for (int h = 1; h < kT / 32; h++) {
      const float4 o = S.red4[h][q];
      s.x += o.x; s.y += o.y; s.z += o.z; s.w += o.w;
    }
    reinterpret_cast<float4 *>(A.part + (int64_t)tk.c * kB)[q] = s;
  }
}

// backward, rows below the front, final: b[cols] -= the partial sums of the
// block in chunk order; the last block of the front is then solved. Padding
// columns past ncol carry products of padding entries and are never stored.
__device__ void bwd_rows(const PsArgs &A, PsShared &S, const Task &tk, const FrontInfo &F) {
  const int c0 = tk.a, nparts = (F.nrow + kRC - 1) / kRC;
  const bool owner = tk.b >= 0;
  if (owner && threadIdx.x == 0) stage_dinv(A, S, tk.b, min(kB, F.ncol - c0));
  if (threadIdx.x < kB) {
    const int c = c0 + threadIdx.x;
    float s = 0.f;
    for (int k = 0; k < nparts; k++) s += ldcg(A.part + (int64_t)(tk.c + k) * kB + threadIdx.x);
    if (c < F.ncol) {
      const float v = ldcg(A.b + F.first + c) - s;
      A.b[F.first + c] = v;
      S.sv[threadIdx.x] = v;
    }
  }
  if (owner && wait_dinv(A, S)) diag_bwd(A, S, F, c0);
}

// backward step of block row j: columns [c0, c0 + 128) left of the block take
// L[j:j+jb, c]^T x_j (loads issued before x_j arrives); the chunk holding the
// block left of j then solves it
__device__ void bwd_step(const PsArgs &A, PsShared &S, const Task &tk, const FrontInfo &F) {
  const int c0 = tk.a, j = tk.b, jb = min(kB, F.ncol - j);
  const bool owner = tk.c >= 0;
  if (owner && threadIdx.x == 0) stage_dinv(A, S, tk.c, kB);
  const int q = threadIdx.x % 32, g = threadIdx.x / 32, c = c0 + 4 * q;
  const float *P = A.L + F.loff + (int64_t)(j + 16 * g) * F.ld + c;
  float4 l[16];
#pragma unroll
  for (int k = 0; k < 16; k++) {
    l[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (16 * g + k < jb) l[k] = __ldg(reinterpret_cast<const float4 *>(P + (int64_t)k * F.ld));
  }
  float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
  float *bp = A.b + F.first + c;
  if (threadIdx.x < 32) old = make_float4(ldcg(bp), ldcg(bp + 1), ldcg(bp + 2), ldcg(bp + 3));
  if (threadIdx.x < kB) S.sy[threadIdx.x] = threadIdx.x < jb ? ldcg(A.x + F.first + j + threadIdx.x) : 0.f;
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 16; k++) acc = fma4(l[k], S.sy[16 * g + k], acc);
  S.red4[g][q] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float4 s = S.red4[0][q];
#pragma unroll
    for (int h = 1; h < kT / 32; h++) {
      const float4 o = S.red4[h][q];
      s.x += o.x; s.y += o.y; s.z += o.z; s.w += o.w;
    }
    const float v0 = old.x - s.x, v1 = old.y - s.y, v2 = old.z - s.z, v3 = old.w - s.w;
    bp[0] = v0; bp[1] = v1; bp[2] = v2; bp[3] = v3;
    S.sv[4 * q] = v0; S.sv[4 * q + 1] = v1; S.sv[4 * q + 2] = v2; S.sv[4 * q + 3] = v3;
  }
  if (owner && wait_dinv(A, S)) diag_bwd(A, S, F, j - kB);
}

__global__ void __launch_bounds__(kT, 2) psolve_kernel(PsArgs A) {
  extern __shared__ __align__(128) unsigned char ps_smem[];
  PsShared &S = *reinterpret_cast<PsShared *>(ps_smem);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar)), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.parity = 0;
  }
  __syncthreads();
  for (int p = A.p0; p < A.p1; p++) {
    const SolvePhase ph = A.dp.ps_phases[p];
    int q = ph.begin + blockIdx.x;
    Task tk{};
    FrontInfo F{};
    if (q < ph.end) {
      tk = A.dp.ps_tasks[q];
      F = A.dp.fronts[tk.front];
    }
    while (q < ph.end) {
      const int qn = q + gridDim.x;  // prefetch the next task of this CTA
      Task tkn{};
      FrontInfo Fn{};
      if (qn < ph.end) {
        tkn = A.dp.ps_tasks[qn];
        Fn = A.dp.fronts[tkn.front];
      }
      switch (ph.kind) {
        case PS_FWD_GATHER: fwd_gather(A, S, tk, F); break;
        case PS_FWD_STEP: fwd_step(A, S, tk, F); break;
        case PS_BWD_PART: bwd_part(A, S, tk, F); break;
        case PS_BWD_ROWS: bwd_rows(A, S, tk, F); break;
        default: bwd_step(A, S, tk, F); break;
      }
      __syncthreads();  // shared scratch is reused by the next task
      tk = tkn;
      F = Fn;
      q = qn;
    }
    if (p + 1 < A.p1 && !grid_barrier(A.bar, A.status, A.spins, A.withhold)) return;
  }
}

int psolve_grid(int max_tasks) {
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
  return std::max(1, std::min(g, max_tasks));
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
                   float *b, float *x, float *t, float *part, unsigned *bar, int32_t *status, bool fwd,
                   bool bwd, cudaStream_t st, unsigned test_spins, int test_withhold) {
  const int32_t p0 = fwd ? 0 : plan.ps_fwd_phases;
  const int32_t p1 = bwd ? (int32_t)plan.ps_phases.size() : plan.ps_fwd_phases;
  if (p1 <= p0) return;
  const int grid = psolve_grid(plan.ps_max_tasks);
  if (grid > kMaxGrid) throw std::runtime_error("persistent solve: grid above the barrier's capacity");
  PsArgs A{dp, L, Dinv, a, b, x, t, part, p0, p1, bar, status,
           test_spins ? test_spins : kBarrierSpins, test_withhold};
  void *args[] = {&A};
  note_launch();
  ck(cudaLaunchCooperativeKernel((const void *)psolve_kernel, dim3(grid), dim3(kT), args,
                                 sizeof(PsShared), st),
     "cooperative solve launch");
}

}  // namespace gipm
