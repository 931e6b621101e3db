// FP64-accurate dense updates of the supernodal Cholesky on tcgen05 tensor
// cores by the Ozaki scheme (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012; run on
// tensor cores by Mukunoki, Ozaki, Ogita and Imamura, ICCS 2020).
//
// Splitting. The panel's columns are taken in windows of two 64-column blocks
// (the last one of a range may be a single block): once a block is finished
// its row segments are sliced, and when the second block of a window is, the
// window's rows are sliced again as one. Each row segment of a window gets
// one exponent e (all its |x| < 2^e); every x of it is rounded to the integer
// X = round(x 2^(55-e)) and written in balanced base 256,
//   X = sum_{i<7} D_i 256^(6-i),  D_1..D_6 in [-128, 127], |D_0| <= 129,
// stored as the BF16 slices s_i = D_i 2^(-8i) (exact: at most 8 significant
// bits). Then x = 2^(e-7) sum_i s_i up to 2^(e-56).
//
// Products. For a 128 x 64 tile of C -= A B^T and one window, the products
// s_i t_j with i + j = d <= 4 are summed over the window's (at most 128)
// columns into their own FP32 accumulator in tensor memory: every term is an
// integer multiple of 2^(-8d) and the sum stays below 2^24 of those units, so
// the accumulation is exact whatever its order. Diagonals 5 and 6 share one
// accumulator, rounded in FP32. The epilogue turns the five exact sums and
// the tail into one 64-bit fixed-point integer W per entry and adds
// W 2^(e_a + e_b - 54) in FP64. Relative to K max|a| max|b| of the window
// (K = 128), the tail's rounding costs at most about 2^-50 and the dropped
// terms i + j >= 7 at most 2^-53: both below the worst-case rounding bound of
// an FP64 dot product of that length (K u = 2^-46 relative to sum |a||b|),
// and far below it for digits of mixed signs. The bound is normwise per
// window: an entry far below its window's largest keeps fewer significant
// bits (the caller redoes a factorisation on the FMA pipe when that turns a
// pivot non-positive).
//
// Long K ranges of one tile are split over several CTAs whose results are
// added with FP64 atomics (the sum of a few FP64 partials in any order).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <stdexcept>
#include <string>

#include "launch.h"
#include "oz.h"
#include "ptx.cuh"
#include "tmap.h"

namespace gipm {

namespace {

using namespace ptx;

constexpr int kP = OzPlan::kPlanes, kBlk = OzPlan::kBlk;
constexpr int kM = 128, kN = 64;   // tile rows and columns
constexpr int kKs = 32;            // K per stage: 64-byte operand rows
constexpr int kStages = 2;
constexpr int kAPlane = kM * kKs * 2, kBPlane = kN * kKs * 2;  // bytes of one slice tile
constexpr int kABytes = kP * kAPlane, kBBytes = kP * kBPlane;
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kSlots = 6;  // exact diagonals 0..4, then diagonals 5 and 6
constexpr int kTmemCols = 512;
constexpr int kSmem = kStages * kStageBytes + 1024 /*barriers*/ + 1024 /*alignment*/;
constexpr int kThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kEpiWarps = 8;
constexpr int kTargetCtas = 2 * 152;  // split long K ranges until a launch has about this many CTAs
constexpr int kMinSplitWin = 4;       // windows per CTA at least
constexpr int16_t kZeroExp = -32768;  // window of zeros (or rows past the front)
constexpr int16_t kNanExp = 32767;    // window holding an Inf or NaN
static_assert(kSlots * kN <= kTmemCols, "tensor memory");
static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(kAPlane % 1024 == 0 && kBPlane % 1024 == 0 && kStageBytes % 1024 == 0, "alignment");

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 bytes, 8-row groups 512 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;            // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)4 << 61;                     // 64-byte swizzle
  return d;
}

// tcgen05.mma kind::f16: BF16 A and B (format 1), FP32 accumulator, both
// K-major, N = 64, M = 128.
constexpr uint32_t kIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, uint64_t *bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// 8 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// The integer n held exactly by an FP32 accumulator as n / scale, |n| < 2^22:
// adding 1.5 * 2^23 puts n in the low mantissa bits.
__device__ __forceinline__ int exact_int(uint32_t bits, float scale) {
  return __float_as_int(fmaf(__uint_as_float(bits), scale, 12582912.0f)) - 0x4B400000;
}
// The same for |n| < 2^31 (a conversion instruction).
__device__ __forceinline__ int wide_int(uint32_t bits, float scale) {
  return __float2int_rn(__uint_as_float(bits) * scale);
}

// W 2^(ea + eb - 54) as an FP64 value built from W's bits (rounded to 53
// bits, ties away from zero; a carry out of the mantissa moves into the
// exponent field); 0 below the normal range, NaN if either window held an
// Inf or NaN.
__device__ __forceinline__ double scaled_double(long long W, int ea, int eb) {
  const unsigned long long a = W < 0 ? (unsigned long long)(-W) : (unsigned long long)W;
  const int lz = __clzll(a);
  const int ex = 63 - lz + ea + eb - 54 + 1023;
  const unsigned long long n = a << (lz & 63);  // leading one at bit 63
  const unsigned long long bits = (W < 0 ? (1ull << 63) : 0ull) |
                                  (((unsigned long long)min(ex, 2045) << 52) +
                                   ((n >> 11) & 0xFFFFFFFFFFFFFull) + ((n >> 10) & 1ull));
  if (ea == kNanExp || eb == kNanExp) return __longlong_as_double(0x7FF8000000000000LL);
  return (a == 0 || ex <= 0) ? 0.0 : __longlong_as_double((long long)bits);
}

// X = round(x 2^(55 - e)) for the window exponent e = mx - 1022 (mx: the
// window's largest biased exponent), from the bits of x.
__device__ __forceinline__ long long scaled_int(unsigned long long b, int mx) {
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - mx + 2;  // <= 2
  const unsigned long long X =
      sh >= 0 ? mant << sh : (-sh >= 60 ? 0ull : (mant + (1ull << (-sh - 1))) >> -sh);
  return (b >> 63) ? -(long long)X : (long long)X;
}

// Slices of one window of a front: columns [b, b + c) (a finished 64-column
// block, or that block and the one before it, sliced again with one
// exponent), rows [a, a + 128) below the window's last diagonal block: one
// warp per row.
__global__ void __launch_bounds__(256) oz_slice_kernel(DevPlan dp, const OzFront *__restrict__ ozf,
                                                       const Task *__restrict__ tasks,
                                                       const double *__restrict__ L,
                                                       uint16_t *__restrict__ S,
                                                       int16_t *__restrict__ E) {
  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const OzFront Z = ozf[tk.front];
  const int nf = F.ncol + F.nrow, c0 = tk.b, width = tk.c, blk = c0 / kBlk;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t plane = (int64_t)nf * Z.lds;
  const int rend = min(nf, tk.a + 128);
  const float pw[kP] = {1.f, 0x1p-8f, 0x1p-16f, 0x1p-24f, 0x1p-32f, 0x1p-40f, 0x1p-48f};
  for (int row = tk.a + warp; row < rend; row += 8) {
    const double *xr = L + F.loff + (int64_t)row * F.ld + c0;
    unsigned long long b[4];
    int mx = 0;
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const int col = lane + 32 * h;
      b[h] = col < width ? (unsigned long long)__double_as_longlong(xr[col]) : 0ull;
      mx = max(mx, (int)((b[h] >> 52) & 0x7FF));
    }
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    const bool normal = mx > 0 && mx < 0x7FF;
    uint16_t *out = S + Z.soff + (int64_t)row * Z.lds + c0;
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const int col = lane + 32 * h;
      if (col >= width) continue;
      long long X = normal ? scaled_int(b[h], mx) : 0ll;
      int D[kP];
#pragma unroll
      for (int i = kP - 1; i >= 1; i--) {
        const int d = (int)(signed char)(X & 0xFF);
        D[i] = d;
        X = (X - d) >> 8;
      }
      D[0] = (int)X;
#pragma unroll
      for (int i = 0; i < kP; i++)
        out[i * plane + col] = __bfloat16_as_ushort(__float2bfloat16_rn((float)D[i] * pw[i]));
    }
    if (lane < (width > kBlk ? 2 : 1))
      E[Z.eoff + (int64_t)row * Z.nblk + blk + lane] =
          normal ? (int16_t)(mx - 1022) : (mx == 0 ? kZeroExp : kNanExp);
  }
}

// One task: a 128 x 64 tile of C -= A B^T over the windows [wb, we).
//  Mode 0 (left-looking update of block column k = b): C = panel rows a..,
//    columns k..k+64; A = panel rows a.., B = panel rows k.., K = columns [0, k).
//  Mode 1 (update-matrix SYRK): C = U rows a.., columns b..; A = panel rows
//    ncol + a.., B = panel rows ncol + b.., K = all ncol columns.
// Window w of the K range covers columns [128 w, 128 w + 128), the last one
// only 64 when the range has an odd number of blocks; its exponent is that of
// block 2 w. c = mode | wb << 2 | we << 17.
__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(DevPlan dp, const OzFront *__restrict__ ozf, const Task *__restrict__ tasks,
                   const CUtensorMap *__restrict__ maps, const int16_t *__restrict__ E,
                   double *__restrict__ L, double *__restrict__ U, int32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(base + kStages * kStageBytes);
  uint64_t *empty = full + kStages;
  uint64_t *accfull = empty + kStages;  // the window's sums are in tensor memory
  uint64_t *accempty = accfull + 1;     // the epilogue has read them
  uint64_t *drain = accempty + 1;       // all products issued by this CTA complete
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int mode = tk.c & 3;
  const int wb = (tk.c >> 2) & 0x7FFF, we = (tk.c >> 17) & 0x7FFF;
  const int nf = F.ncol + F.nrow;
  const int arow = mode == 0 ? tk.a : F.ncol + tk.a;  // operand rows (front-local)
  const int brow = mode == 0 ? tk.b : F.ncol + tk.b;
  const int nblk = mode == 0 ? tk.b / kBlk : (F.ncol + kBlk - 1) / kBlk;  // blocks of K
  const int npair = nblk / 2;  // windows of two blocks

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, kEpiWarps);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer: all 7 slices of a 32-column step of A and B
      const CUtensorMap *ma = maps + 2 * tk.front, *mb = ma + 1;
      uint32_t g = 0;
      for (int w = wb; w < we && !*abort_flag; w++)
        for (int sub = 0; sub < (w < npair ? 4 : 2); sub++, g++) {
          const int s = g % kStages;
          const uint32_t round = g / kStages;
          if (!mbar_wait(&empty[s], (round & 1) ^ 1, status)) { *abort_flag = 1; break; }
          mbar_arrive_expect_tx(&full[s], kStageBytes);
          uint8_t *st = base + s * kStageBytes;
          const int x = w * 2 * kBlk + sub * kKs;
          tma_load_3d(st, ma, &full[s], x, arow, 0);
          tma_load_3d(st + kABytes, mb, &full[s], x, brow, 0);
        }
      if (*abort_flag)  // let the copies already issued land before the CTA exits
        for (uint32_t q = g > (uint32_t)kStages ? g - kStages : 0; q < g; q++)
          mbar_wait(&full[q % kStages], (q / kStages) & 1, status);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t g = 0;
      int wi = 0;
      for (int w = wb; w < we && !*abort_flag; w++, wi++) {
        if (!mbar_wait(accempty, (wi & 1) ^ 1, status)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool fail = false;
        for (int sub = 0; sub < (w < npair ? 4 : 2); sub++, g++) {
          const int s = g % kStages;
          const uint32_t round = g / kStages;
          if (!mbar_wait(&full[s], round & 1, status)) { *abort_flag = 1; fail = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(base + s * kStageBytes), b0 = a0 + kABytes;
#pragma unroll
          for (int d = 0; d <= 6; d++) {
            const uint32_t acc = tmem + (uint32_t)((d < 5 ? d : 5) * kN);
#pragma unroll
            for (int i = 0; i <= d; i++) {
              const uint64_t ad = sw64_desc(a0 + i * kAPlane), bd = sw64_desc(b0 + (d - i) * kBPlane);
#pragma unroll
              for (int kk = 0; kk < 2; kk++) {  // 16 BF16 (32 bytes) of K per product
                const bool first = sub == 0 && kk == 0 && i == 0 && d <= 5;
                mma_bf16(acc, ad + 2 * kk, bd + 2 * kk, kIdesc, first ? 0u : 1u);
              }
            }
          }
          mma_commit(&empty[s]);
        }
        if (fail) break;
        mma_commit(accfull);
      }
      mma_commit(drain);  // tensor memory is released only after every product landed
      mbar_wait(drain, 0, status);
    }
  } else {  // warps 2-9: per window, W from the six sums, accumulated in FP64
    const int q = warp & 3;         // tensor-memory lane quarter this warp may access
    const int c0 = 32 * ((warp - 2) >> 2);  // this thread's 32 columns of the tile
    const int r = 32 * q + lane;    // its row of the tile
    const OzFront Z = ozf[tk.front];
    const bool arow_ok = arow + r < nf;
    const int16_t *ea_row = E + Z.eoff + (int64_t)(arow + r) * Z.nblk;
    const int16_t *eb_col = E + Z.eoff + (int64_t)(brow + c0) * Z.nblk;
    const int nb_rows = nf - (brow + c0);  // B rows of this thread's columns inside the front
    double acc[32];
#pragma unroll
    for (int c = 0; c < 32; c++) acc[c] = 0.0;
    int wi = 0;
    for (int w = wb; w < we && !*abort_flag; w++, wi++) {
      const int ea = arow_ok ? ea_row[2 * w] : kZeroExp;
      // lane c holds the exponent of this thread's column c0 + c (one load per
      // lane; the additions below take it by shuffle)
      const int eb_lane = lane < nb_rows ? eb_col[(int64_t)lane * Z.nblk + 2 * w] : kZeroExp;
      if (!mbar_wait(accfull, wi & 1, status)) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // W of all 32 entries first (cheap FP32/INT work), then free the
      // accumulators for the next window, then the FP64 additions
      long long Wv[32];
#pragma unroll
      for (int sub = 0; sub < 4; sub++) {  // 8 columns at a time, one sum at a time
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c0 + 8 * sub);
        uint32_t v[8];
        int hi[8];
        tmem_ld8(ta, v);  // diagonal 0
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++) hi[c] = exact_int(v[c], 1.f) * 256;
        tmem_ld8(ta + kN, v);  // diagonal 1
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++) Wv[8 * sub + c] = (long long)(hi[c] + wide_int(v[c], 0x1p8f)) << 32;
        tmem_ld8(ta + 2 * kN, v);  // diagonal 2
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++) Wv[8 * sub + c] += (long long)wide_int(v[c], 0x1p16f) << 24;
        tmem_ld8(ta + 3 * kN, v);  // diagonal 3
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++) hi[c] = wide_int(v[c], 0x1p24f);
        tmem_ld8(ta + 4 * kN, v);  // diagonal 4
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++)
          Wv[8 * sub + c] += ((long long)hi[c] << 16) + ((long long)wide_int(v[c], 0x1p32f) << 8);
        tmem_ld8(ta + 5 * kN, v);  // diagonals 5 and 6 (rounded), |.| < 2^24 units
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++) Wv[8 * sub + c] += wide_int(v[c], 0x1p40f);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty);
#pragma unroll
      for (int c = 0; c < 32; c++) {
        const int eb = __shfl_sync(0xFFFFFFFFu, eb_lane, c);
        acc[c] += scaled_double(Wv[c], ea, eb);
      }
    }
    if (!*abort_flag) {
      int M, N;
      double *C;
      int64_t ldc;
      if (mode == 0) {
        M = min(kM, nf - tk.a);
        N = min(kBlk, F.ncol - tk.b);
        C = L + F.loff + (int64_t)tk.a * F.ld + tk.b;
        ldc = F.ld;
      } else {
        M = min(kM, F.nrow - tk.a);
        N = min(kN, F.nrow - tk.b);
        C = U + F.uoff + (int64_t)tk.a * F.uld + tk.b;
        ldc = F.uld;
      }
      if (r < M) {
        double *crow = C + (int64_t)r * ldc + c0;
#pragma unroll
        for (int c = 0; c < 32; c++)
          if (c0 + c < N) atomicAdd(crow + c, -acc[c]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
}

// Chunks of the K range of each tile: enough CTAs for the launch, at least
// kMinSplitWin windows each.
int split_for(int64_t tiles, int nwin) {
  if (tiles <= 0 || tiles >= kTargetCtas) return 1;
  const int64_t want = (kTargetCtas + tiles - 1) / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, nwin / kMinSplitWin));
}

void push_split(std::vector<Task> &out, int32_t front, int32_t a, int32_t b, int mode, int nwin,
                int split) {
  for (int c = 0; c < split; c++) {
    const int w0 = (int)((int64_t)nwin * c / split), w1 = (int)((int64_t)nwin * (c + 1) / split);
    if (w1 > w0) out.push_back({front, a, b, mode | (w0 << 2) | (w1 << 17)});
  }
}

// Windows of a K range of nblk blocks: pairs, and a last single block.
int windows(int nblk) { return nblk / 2 + nblk % 2; }

}  // namespace

void OzPlan::build(const Plan &plan) {
  if (plan.nb != kBlk) throw std::runtime_error("the FP64 tensor-core factor needs 64-wide blocks");
  gemm_.clear();
  slice_.clear();
  levels_.clear();
  const size_t nfr = plan.fronts.size();
  fr_.assign(nfr, OzFront{});
  int64_t so = 0, eo = 0;
  for (size_t f = 0; f < nfr; f++) {
    const FrontInfo &F = plan.fronts[f];
    const int nf = F.ncol + F.nrow;
    const int lds = (std::max(F.ncol, 1) + 7) / 8 * 8;
    const int nblk = (F.ncol + kBlk - 1) / kBlk;
    if (windows(nblk) >= 0x7FFF) throw std::runtime_error("front too wide for the FP64 tensor-core factor");
    fr_[f] = OzFront{so, eo, lds, nblk, {0, 0}};
    so += (int64_t)kP * nf * lds;
    eo += (int64_t)nf * nblk;
  }
  slice_elems_ = so;
  exp_elems_ = eo;
  levels_.resize(plan.levels.size());
  for (size_t l = 0; l < plan.levels.size(); l++) {
    const LevelPlan &LP = plan.levels[l];
    Level &V = levels_[l];
    for (int32_t k = 0; k < LP.max_ncol; k += kBlk) {
      Step st{};
      st.gemm_b = (int)gemm_.size();
      if (k > 0) {
        int64_t tiles = 0;
        for (int32_t t = LP.front_b; t < LP.front_e; t++) {
          const FrontInfo &F = plan.fronts[plan.level_fronts[t]];
          if (F.ncol > k) tiles += (F.ncol + F.nrow - k + kM - 1) / kM;
        }
        const int nw = windows(k / kBlk);
        const int split = split_for(tiles, nw);
        for (int32_t t = LP.front_b; t < LP.front_e; t++) {
          const int32_t s = plan.level_fronts[t];
          const FrontInfo &F = plan.fronts[s];
          if (F.ncol <= k) continue;
          for (int32_t i0 = k; i0 < F.ncol + F.nrow; i0 += kM) push_split(gemm_, s, i0, k, 0, nw, split);
        }
      }
      st.gemm_e = (int)gemm_.size();
      // the finished block (an even block alone, an odd block with the one
      // before it), rows below it
      st.slice_b = (int)slice_.size();
      const bool odd = (k / kBlk) % 2 == 1;
      for (int32_t t = LP.front_b; t < LP.front_e; t++) {
        const int32_t s = plan.level_fronts[t];
        const FrontInfo &F = plan.fronts[s];
        if (F.ncol <= k) continue;
        const int32_t kb = std::min(kBlk, F.ncol - k);
        const int32_t c0 = odd ? k - kBlk : k, width = odd ? kBlk + kb : kb;
        for (int32_t r0 = k + kb; r0 < F.ncol + F.nrow; r0 += 128) slice_.push_back({s, r0, c0, width});
      }
      st.slice_e = (int)slice_.size();
      V.steps.push_back(st);
    }
    if (V.steps.size() != LP.steps.size()) throw std::runtime_error("FP64 tensor-core plan: step count");
    V.syrk_b = (int)gemm_.size();
    int64_t tiles = 0;
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const FrontInfo &F = plan.fronts[plan.level_fronts[t]];
      for (int32_t i0 = 0; i0 < F.nrow; i0 += kM) tiles += (std::min(F.nrow, i0 + kM) + kN - 1) / kN;
    }
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const FrontInfo &F = plan.fronts[s];
      if (F.nrow == 0) continue;
      const int nw = windows((F.ncol + kBlk - 1) / kBlk);
      const int split = split_for(tiles, nw);
      for (int32_t i0 = 0; i0 < F.nrow; i0 += kM)
        for (int32_t j0 = 0; j0 < F.nrow && j0 < i0 + kM; j0 += kN)
          push_split(gemm_, s, i0, j0, 1, nw, split);
    }
    V.syrk_e = (int)gemm_.size();
  }
  validate(plan);
}

// Every task against the buffers it indexes, and the K chunks of each tile
// against its window range (consecutive, no gap, no overlap): a violation is a
// planning bug, reported before any launch.
void OzPlan::validate(const Plan &plan) const {
  auto need = [](bool ok, const char *what) {
    if (!ok) throw std::runtime_error(std::string("FP64 tensor-core plan: ") + what);
  };
  const int nfr = (int)plan.fronts.size();
  for (int f = 0; f < nfr; f++) {
    const FrontInfo &F = plan.fronts[f];
    const OzFront &Z = fr_[f];
    const int64_t nf = F.ncol + F.nrow;
    need(Z.lds >= F.ncol && Z.lds % 8 == 0 && Z.soff % 8 == 0, "slice row stride");
    need(Z.soff + (int64_t)kP * nf * Z.lds <= slice_elems_, "slice planes past the storage");
    need(Z.eoff + nf * Z.nblk <= exp_elems_, "exponents past the storage");
  }
  int cur_f = -1, cur_a = -1, cur_b = -1, cur_mode = -1, next_w = 0, cur_W = 0;
  auto close_tile = [&]() { need(cur_f < 0 || next_w == cur_W, "a tile's chunks miss windows"); };
  for (const Task &t : gemm_) {
    need(t.front >= 0 && t.front < nfr, "task front");
    const FrontInfo &F = plan.fronts[t.front];
    const int mode = t.c & 3, w0 = (t.c >> 2) & 0x7FFF, w1 = (t.c >> 17) & 0x7FFF;
    int W;
    if (mode == 0) {
      need(t.b > 0 && t.b % kBlk == 0 && t.b < F.ncol, "update: block column");
      need(t.a >= t.b && t.a < F.ncol + F.nrow && (t.a - t.b) % kM == 0, "update: row tile");
      W = windows(t.b / kBlk);
    } else {
      need(mode == 1 && F.nrow > 0, "task mode");
      need(t.a >= 0 && t.a < F.nrow && t.a % kM == 0, "SYRK: row tile");
      need(t.b >= 0 && t.b < F.nrow && t.b % kN == 0 && t.b < t.a + kM, "SYRK: column tile");
      W = windows((F.ncol + kBlk - 1) / kBlk);
    }
    need(0 <= w0 && w0 < w1 && w1 <= W, "window range");
    if (t.front != cur_f || t.a != cur_a || t.b != cur_b || mode != cur_mode || w0 == 0) {
      close_tile();
      need(w0 == 0, "a tile's first chunk starts past window 0");
      cur_f = t.front, cur_a = t.a, cur_b = t.b, cur_mode = mode, cur_W = W, next_w = 0;
    }
    need(w0 == next_w, "a tile's chunks are not consecutive");
    next_w = w1;
  }
  close_tile();
  for (const Task &t : slice_) {
    need(t.front >= 0 && t.front < nfr, "slice front");
    const FrontInfo &F = plan.fronts[t.front];
    need(t.b % kBlk == 0 && t.c > 0 && t.c <= 2 * kBlk && t.b + t.c <= F.ncol, "slice columns");
    need(t.a >= t.b + t.c && t.a < F.ncol + F.nrow, "slice rows");
  }
}

void OzPlan::layout(Carve &cv, cudaStream_t st, bool storage) {
  auto up = [&](const std::vector<Task> &v) {
    Task *p = cv.take<Task>(std::max<size_t>(v.size(), 1));
    if (cv.base && !v.empty())
      cudaMemcpyAsync(p, v.data(), v.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    return p;
  };
  d_gemm_ = up(gemm_);
  d_slice_ = up(slice_);
  d_fr_ = cv.take<OzFront>(std::max<size_t>(fr_.size(), 1));
  if (cv.base && !fr_.empty())
    cudaMemcpyAsync(d_fr_, fr_.data(), fr_.size() * sizeof(OzFront), cudaMemcpyHostToDevice, st);
  d_maps_ = cv.take<CUtensorMap>(2 * std::max<size_t>(fr_.size(), 1));
  S_ = storage ? cv.take<uint16_t>((size_t)std::max<int64_t>(slice_elems_, 1)) : nullptr;
  E_ = storage ? cv.take<int16_t>((size_t)std::max<int64_t>(exp_elems_, 1)) : nullptr;
  sized_ = storage;
  ready_ = false;
}

void OzPlan::encode(const Plan &plan, cudaStream_t st) {
  ready_ = false;
  if (!sized_ || !S_) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  const size_t nfr = plan.fronts.size();
  std::vector<CUtensorMap> maps(2 * nfr);
  for (size_t f = 0; f < nfr; f++) {
    const FrontInfo &F = plan.fronts[f];
    const OzFront &Z = fr_[f];
    const int nf = F.ncol + F.nrow;
    for (int h = 0; h < 2; h++) {
      CUtensorMap &m = maps[2 * f + h];
      std::memset(&m, 0, sizeof(m));
      if (F.ncol <= 0 || nf <= 0) continue;
      cuuint64_t dims[3] = {(cuuint64_t)F.ncol, (cuuint64_t)nf, (cuuint64_t)kP};
      cuuint64_t strides[2] = {(cuuint64_t)Z.lds * 2, (cuuint64_t)nf * Z.lds * 2};
      cuuint32_t box[3] = {(cuuint32_t)kKs, (cuuint32_t)(h == 0 ? kM : kN), (cuuint32_t)kP};
      cuuint32_t estr[3] = {1, 1, 1};
      CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)(S_ + Z.soff), dims, strides,
                       box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        throw std::runtime_error("cuTensorMapEncodeTiled failed for the slices of front " +
                                 std::to_string(f));
    }
  }
  if (!maps.empty() && cudaMemcpyAsync(d_maps_, maps.data(), maps.size() * sizeof(CUtensorMap),
                                       cudaMemcpyHostToDevice, st) != cudaSuccess)
    throw std::runtime_error("tensor map upload failed");
  if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("tensor map upload failed");
  if (cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) !=
      cudaSuccess)
    throw std::runtime_error("FP64 tensor-core kernel: shared memory");
  ready_ = true;
}

void OzPlan::factor(const DevPlan &dp, const Plan &plan, const double *kval, double *L, double *U,
                    int32_t *status, cudaStream_t st) {
  if (!ready_) throw std::runtime_error("FP64 tensor-core factor not prepared");
  const CUtensorMap *maps = reinterpret_cast<const CUtensorMap *>(d_maps_);
  auto gemm = [&](int b, int e) {
    if (e > b) {
      note_launch();
      oz_gemm_kernel<<<e - b, kThreads, kSmem, st>>>(dp, d_fr_, d_gemm_ + b, maps, E_, L, U, status);
    }
  };
  for (size_t l = 0; l < plan.levels.size(); l++) {
    const LevelPlan &LP = plan.levels[l];
    const Level &V = levels_[l];
    launch_build_level<double>(dp, LP, kval, L, U, st);
    for (size_t s = 0; s < LP.steps.size(); s++) {
      const StepRange &R = LP.steps[s];
      const Step &Z = V.steps[s];
      gemm(Z.gemm_b, Z.gemm_e);
      launch_potrf<double>(dp, dp.potrf + R.potrf_b, R.potrf_e - R.potrf_b, plan.nb, L, status,
                           false, st);
      launch_trsm_f64(dp, dp.trsm + R.trsm_b, R.trsm_e - R.trsm_b, L, st);
      if (Z.slice_e > Z.slice_b) {
        note_launch();
        oz_slice_kernel<<<Z.slice_e - Z.slice_b, 256, 0, st>>>(dp, d_fr_, d_slice_ + Z.slice_b, L,
                                                              S_, E_);
      }
    }
    gemm(V.syrk_b, V.syrk_e);
  }
}

}  // namespace gipm
