// Tensor-core kernels of the supernodal factorisation on sm_103a (tcgen05,
// TMA, thread-block clusters).
//
// Two persistent GEMM kernels compute C -= A B^T (or C = A B^T) where A and B
// are row blocks of a front's panel (row-major, K contiguous: "K-major"):
//  - tc_pair_kernel: 128 x 256 tiles in clusters of two CTAs that share their
//    B rows by TMA multicast; the update-matrix SYRK and the left-looking
//    super-step updates of the panel;
//  - tc_gemm_kernel: 128 x 128 tiles; the short per-block-step updates and the
//    triangular solve of the rows below a diagonal block as a product with its
//    inverse.
// In both, warp 0 streams 128 x 32 FP32 tiles (and, for the 3-term split, their
// low parts) through a ring of 128B-swizzled shared memory with TMA, warp 1
// issues tcgen05.mma kind::tf32 into one of two FP32 accumulators in tensor
// memory, and warps 2-5 read the other accumulator back with tcgen05.ld and
// hand it to TMA through shared memory (reduce-add or store). potrf_inv_kernel
// factors and inverts the 128 x 128 diagonal blocks on the FMA pipe. Every wait
// on an mbarrier is bounded by a clock limit; on expiry the CTA records
// ST_TIMEOUT, skips the rest of its work and still releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <stdexcept>
#include <string>

#include "launch.h"
#include "ptx.cuh"
#include "tc.h"
#include "tmap.h"

#include <cstring>

namespace gipm {

namespace {

using namespace ptx;

constexpr int kTileM = 128, kTileN = 128, kTileK = 32, kSyrkN = 256;
// Operand arithmetic of a kernel instantiation ("SPLIT"): 1 TF32, 3 the
// 3-term split TF32, kBf16 BF16 operands (kind::f16) for the updates of
// finished entries, read from their BF16 copy, with the panel solve in TF32.
constexpr int kBf16 = 16;
constexpr int kTileKBf = 64;  // BF16 elements per 128-byte operand row
constexpr int kMaxClusters = 76;  // CTA pairs of the persistent SYRK (152 SMs)
constexpr int kSuper = 512;  // columns per super-step of the left-looking panel updates
constexpr int kAheadFronts = 2;  // levels with at most this many fronts run the look-ahead
constexpr int kBandGroup = 16;   // row bands per group of the SYRK's tile order
constexpr int kTileBytes = kTileM * kTileK * 4;  // 16 KB per 128-row operand tile
// Ring depth: as many stages as fit in ~200 KB (each stage: A and B tiles, and
// their low parts when SPLIT == 3). BN = 256 tiles (SYRK) halve the operand
// bytes per product of the B side.
// After the ring and its barriers: the epilogue's staging, 4 warps x 2 x 4 KB
// (1024-byte aligned for the 128-byte swizzle).
template <int SPLIT, int BN> struct Cfg {
  static constexpr int kB = BN / 128;                            // 128-row B tiles per stage
  static constexpr int kStage = (SPLIT == 3 ? 2 : 1) * (1 + kB) * kTileBytes;
  static constexpr int S = (200 * 1024) / kStage > 4 ? 4 : (200 * 1024) / kStage;
  static constexpr int stage_off = S * kStage + 1024 /*barriers*/;
  static constexpr int smem = stage_off + 4 * 8192 + 1024 /*alignment*/;
  static_assert(smem <= 227 * 1024, "tensor-core kernel shared memory");
};

// x - tf32(x): what the tensor core drops from an FP32 operand (low 13 mantissa bits)
__device__ __forceinline__ float lo1(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}
__device__ __forceinline__ float4 lo_part(float4 v) {
  return make_float4(lo1(v.x), lo1(v.y), lo1(v.z), lo1(v.w));
}

__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// The same box written to this CTA's and its cluster peer's shared memory at
// the same offset; each destination's mbarrier at the same offset receives its bytes.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const void *tmap, uint64_t *bar, int x,
                                               int y, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(mask)
      : "memory");
}

// C[box at (x, y)] += the box in shared memory (128-byte swizzled rows), done
// in L2 by the TMA unit; the issuing thread tracks it as a bulk group.
__device__ __forceinline__ void tma_reduce_add_2d(const void *tmap, const void *src, int x, int y) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3}], [%1];"
      ::"l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(src)), "r"(x), "r"(y)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// C[box at (x, y)] = the box in shared memory (128-byte swizzled rows).
__device__ __forceinline__ void tma_store_2d(const void *tmap, const void *src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];"
               ::"l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Writes 32 floats (one row of a 32 x 32 box, `row` = lane) in the 128-byte
// swizzled layout: 16-byte chunk j of row r sits at chunk j ^ (r % 8).
template <typename F>
__device__ __forceinline__ void stage_row(uint8_t *buf, int row, const float (&v)[32], F f) {
  uint8_t *rowp = buf + row * 128;
#pragma unroll
  for (int j = 0; j < 8; j++)
    *reinterpret_cast<float4 *>(rowp + ((j ^ (row & 7)) << 4)) =
        make_float4(f(v[4 * j]), f(v[4 * j + 1]), f(v[4 * j + 2]), f(v[4 * j + 3]));
}
// Writes 32 values of one row of a 32 x 32 BF16 box (64-byte rows, no swizzle),
// rounded to nearest even.
__device__ __forceinline__ void stage_row_bf16(uint8_t *buf, int row, const float (&v)[32]) {
  uint8_t *rowp = buf + row * 64;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * j + 2 * h], v[8 * j + 2 * h + 1]);
      w[h] = *reinterpret_cast<const uint32_t *>(&b2);
    }
    *reinterpret_cast<uint4 *>(rowp + 16 * j) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}
// Wait until at most N of this thread's bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator, TF32 A
// and B, both K-major, N = 128, M = 128.
template <int BN>
__host__ __device__ constexpr uint32_t tf32_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(kTileM >> 4) << 24);
}

// Instruction descriptor of tcgen05.mma kind::f16 with BF16 A and B (format 1),
// FP32 accumulator, both K-major, N = BN, M = 128.
template <int BN>
__host__ __device__ constexpr uint32_t bf16_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Completion of this CTA's issued products, signalled to the mbarrier at the
// same offset in every CTA of the mask.
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Task of the 128 x 128 kernel: front, a = first row of the A tile
// (front-local), b = k, c = mode | slot << 2 (mode 2) or mode | kbeg / 128 << 2
// | kend / 128 << 17 (mode 0).
//  Mode 0 (left-looking update of block column k by the columns [kbeg, kend)):
//    C = panel[a:a+128, k:k+kb] -= A B^T with A = panel rows a.., B = panel
//    rows k.., K = kend - kbeg.
//  Mode 2 (triangular solve of the rows below a diagonal block, as a product
//    with its inverse): C = panel[a:a+128, k:k+kb] = A B^T with A = the same
//    panel rows and columns, B = L_kk^{-1} from scratch slot `slot`, K = kb.
//    The tile's rows are read completely before its epilogue overwrites them.
// (The update-matrix SYRK and the super-step updates run in the pair kernel.)
//
// SPLIT == 3: mode 0 reads finished panel entries, whose low parts the mode-2
// epilogue stored in Llo: all four tiles (A, A_lo, B, B_lo) arrive by TMA.
// Mode 2 reads entries that are still being updated and the inverse, so warps
// 2-5 form their low parts in shared memory.
// Geometry of one task (see the task encoding above).
struct Geo {
  int mode, arow, brow, K, M, N, ax0, bx0, nk, kstep;
  bool bf;  // BF16 operands (kind::f16) from the BF16 copy of the panel
  const CUtensorMap *amap, *bmap, *lomap;
};

template <int SPLIT>
__device__ __forceinline__ Geo task_geo(const DevPlan &dp, const Task &tk, const CUtensorMap *maps,
                                        const CUtensorMap *maps_lo, const CUtensorMap *inv_map,
                                        const CUtensorMap *maps_bf, int nb) {
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow;
  Geo g;
  g.mode = tk.c & 3;
  g.amap = maps + tk.front;
  g.bmap = g.amap;
  g.lomap = maps_lo + tk.front;
  const int k = tk.b;
  g.arow = tk.a;
  g.M = min(kTileM, nf - tk.a);
  g.N = min(nb, F.ncol - k);
  g.bf = false;
  if (g.mode == 0) {  // K range [kbeg, kend) of the update of block column k
    const int kbeg = ((tk.c >> 2) & 0x7FFF) * kTileN, kend = ((tk.c >> 17) & 0x7FFF) * kTileN;
    g.brow = k;
    g.ax0 = g.bx0 = kbeg;
    g.K = kend - kbeg;
    if (SPLIT == kBf16) {  // finished entries: their BF16 copy
      g.bf = true;
      g.amap = g.bmap = maps_bf + tk.front;
    }
  } else {
    g.ax0 = k;
    g.bx0 = 0;
    g.brow = (tk.c >> 2) * kTileN;
    g.bmap = inv_map;
    g.K = g.N;
  }
  g.kstep = g.bf ? kTileKBf : kTileK;
  g.nk = (g.K + g.kstep - 1) / g.kstep;
  return g;
}

// Persistent: each CTA takes tasks blockIdx.x, blockIdx.x + gridDim.x, ...
// The k-steps of all its tasks flow through one ring of shared-memory stages;
// two accumulators in tensor memory let the epilogue of one tile overlap the
// main loop of the next.
template <int SPLIT, int BN>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(DevPlan dp, const Task *__restrict__ tasks, int ntask,
                   const CUtensorMap *__restrict__ maps, const CUtensorMap *__restrict__ maps_lo,
                   const CUtensorMap *__restrict__ inv_map, const CUtensorMap *__restrict__ lmaps,
                   const CUtensorMap *__restrict__ llomaps, const CUtensorMap *__restrict__ maps_bf,
                   const CUtensorMap *__restrict__ lbfmaps, int nb, int32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  using CF = Cfg<SPLIT, BN>;
  constexpr int S = CF::S, kBB = CF::kB * kTileBytes;  // bytes of a B tile
  uint8_t *sA = base;                          // S x A tiles
  uint8_t *sB = sA + S * kTileBytes;           // S x B tiles
  uint8_t *sAl = sB + S * kBB;                 // low parts (SPLIT == 3 only)
  uint8_t *sBl = sAl + (SPLIT == 3 ? S * kTileBytes : 0);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + S * CF::kStage);
  uint64_t *empty = full + S;
  uint64_t *lofull = empty + S;
  uint64_t *accfull = lofull + S;   // [2] accumulator ready for the epilogue
  uint64_t *accempty = accfull + 2; // [2] accumulator free for the next tile
  uint64_t *drain = accempty + 2;   // all products issued by this CTA complete
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&lofull[s], 4);  // one arrival per converting warp
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&accfull[a], 1);
      mbar_init(&accempty[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      uint32_t g = 0;
      for (int t = blockIdx.x; t < ntask && !*abort_flag; t += gridDim.x) {
        const Geo G = task_geo<SPLIT>(dp, tasks[t], maps, maps_lo, inv_map, maps_bf, nb);
        const bool pre = SPLIT == 3 && G.mode != 2;  // low parts loaded with the tiles
        for (int kt = 0; kt < G.nk; kt++, g++) {
          const int s = g % S;
          const uint32_t round = g / S;
          if (!mbar_wait(&empty[s], (round & 1) ^ 1, status)) { *abort_flag = 1; break; }
          mbar_arrive_expect_tx(&full[s], (pre ? 2 : 1) * (kTileBytes + kBB));
          tma_load_2d(sA + s * kTileBytes, G.amap, &full[s], G.ax0 + kt * G.kstep, G.arow);
          for (int h = 0; h < CF::kB; h++)  // a 256-row B tile is two 128-row boxes
            tma_load_2d(sB + s * kBB + h * kTileBytes, G.bmap, &full[s], G.bx0 + kt * G.kstep,
                        G.brow + 128 * h);
          if (pre) {
            tma_load_2d(sAl + s * kTileBytes, G.lomap, &full[s], G.ax0 + kt * kTileK, G.arow);
            for (int h = 0; h < CF::kB; h++)
              tma_load_2d(sBl + s * kBB + h * kTileBytes, G.lomap, &full[s], G.bx0 + kt * kTileK,
                          G.brow + 128 * h);
          }
        }
      }
      if (*abort_flag)  // let the copies already issued land before the CTA exits
        for (uint32_t q = g > (uint32_t)S ? g - S : 0; q < g; q++)
          mbar_wait(&full[q % S], (q / S) & 1, status);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = tf32_idesc<BN>();
      constexpr uint32_t idesc_bf = bf16_idesc<BN>();
      uint32_t g = 0;
      int i = 0;
      for (int t = blockIdx.x; t < ntask && !*abort_flag; t += gridDim.x, i++) {
        const Geo G = task_geo<SPLIT>(dp, tasks[t], maps, maps_lo, inv_map, maps_bf, nb);
        const bool conv = SPLIT == 3 && G.mode == 2;
        const int a = i & 1;
        if (!mbar_wait(&accempty[a], ((i >> 1) & 1) ^ 1, status)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(a * BN);
        for (int kt = 0; kt < G.nk; kt++, g++) {
          const int s = g % S;
          const uint32_t round = g / S;
          if (!mbar_wait(&full[s], round & 1, status)) { *abort_flag = 1; break; }
          if (conv && !mbar_wait(&lofull[s], round & 1, status)) { *abort_flag = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t ad = sw128_desc(smem_u32(sA + s * kTileBytes));
          const uint64_t bd = sw128_desc(smem_u32(sB + s * kBB));
          const uint64_t ald = sw128_desc(smem_u32(sAl + s * kTileBytes));
          const uint64_t bld = sw128_desc(smem_u32(sBl + s * kBB));
#pragma unroll
          for (int k4 = 0; k4 < kTileK / 8; k4++) {  // 8 TF32 (16 BF16) = 32 bytes per MMA along K
            if (SPLIT == kBf16 && G.bf) {
              mma_bf16(acc, ad + 2 * k4, bd + 2 * k4, idesc_bf, (kt | k4) != 0);
            } else if (SPLIT == 3) {  // small terms first: A_lo B + A B_lo, then A B
              mma_tf32(acc, ald + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
              mma_tf32(acc, ad + 2 * k4, bld + 2 * k4, idesc, 1);
              mma_tf32(acc, ad + 2 * k4, bd + 2 * k4, idesc, 1);
            } else {
              mma_tf32(acc, ad + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
            }
          }
          mma_commit(&empty[s]);
        }
        if (*abort_flag) break;
        mma_commit(&accfull[a]);
      }
      mma_commit(drain);  // tensor memory is released only after every product landed
      mbar_wait(drain, 0, status);
    }
  } else {  // warps 2-5: low parts (mode 2) and the epilogue
    const int q = warp % 4;  // tensor-memory lane quarter this warp may access
    uint8_t *stg = base + CF::stage_off + q * 8192;  // this warp's two 4 KB staging buffers
    uint32_t nissued = 0;
    uint32_t g = 0;
    int i = 0;
    for (int t = blockIdx.x; t < ntask && !*abort_flag; t += gridDim.x, i++) {
      const Geo G = task_geo<SPLIT>(dp, tasks[t], maps, maps_lo, inv_map, maps_bf, nb);
      if (SPLIT == 3 && G.mode == 2) {
        // low parts x - tf32(x) of both operand tiles (tf32 keeps the top 19 bits)
        const int tt = threadIdx.x - 64;
        for (int kt = 0; kt < G.nk; kt++, g++) {
          const int s = g % S;
          const uint32_t round = g / S;
          if (!mbar_wait(&full[s], round & 1, status)) { *abort_flag = 1; break; }
          const float4 *av = reinterpret_cast<const float4 *>(sA + s * kTileBytes);
          const float4 *bv = reinterpret_cast<const float4 *>(sB + s * kBB);
          float4 *al = reinterpret_cast<float4 *>(sAl + s * kTileBytes);
          float4 *bl = reinterpret_cast<float4 *>(sBl + s * kBB);
          for (int e = tt; e < kTileBytes / 16; e += 128) al[e] = lo_part(av[e]);
          for (int e = tt; e < kBB / 16; e += 128) bl[e] = lo_part(bv[e]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&lofull[s]);
        }
        if (*abort_flag) break;
      } else {
        g += G.nk;
      }
      const int a = i & 1;
      if (!mbar_wait(&accfull[a], (i >> 1) & 1, status)) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // 32 x 32 blocks through shared memory to TMA: mode 0 adds the negated
      // block in L2 (C -= A B^T), mode 2 stores it and its low parts.
      if (32 * q < G.M) {
        const Task tk = tasks[t];
        const int y = tk.a + 32 * q, x0 = tk.b;  // panel rows and columns
        const CUtensorMap *cm = lmaps + tk.front;
        for (int cb = 0; cb < (G.N + 31) / 32; cb++) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN + cb * 32), v);
          if (G.mode == 2) {
            if (lane == 0) bulk_wait_read<0>();
            __syncwarp();
            stage_row(stg, lane, v, [](float x) { return x; });
            if (SPLIT == 3) stage_row(stg + 4096, lane, v, [](float x) { return lo1(x); });
            if (SPLIT == kBf16) stage_row_bf16(stg + 4096, lane, v);  // the entries' BF16 copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(cm, stg, x0 + 32 * cb, y);
              if (SPLIT == 3) tma_store_2d(llomaps + tk.front, stg + 4096, x0 + 32 * cb, y);
              if (SPLIT == kBf16) tma_store_2d(lbfmaps + tk.front, stg + 4096, x0 + 32 * cb, y);
            }
            nissued = 0;  // a later reduction stages into the buffer read first
          } else {
            uint8_t *buf = stg + (nissued & 1) * 4096;
            if (lane == 0) bulk_wait_read<1>();
            __syncwarp();
            stage_row(buf, lane, v, [](float x) { return -x; });
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) tma_reduce_add_2d(cm, buf, x0 + 32 * cb, y);
            nissued++;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[a]);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
}

// Geometry of a pair task {front, a = i0, b = j0 or c, mode}: CTA `rank` of the
// pair computes the 128 x 256 tile whose rows start 128 * rank below i0.
//  Mode 1 (update-matrix SYRK): U[i0.., j0..j0+256) -= A B^T, A = panel rows
//    ncol + i0 + 128 rank.., B = panel rows ncol + j0.., K = ncol.
//  Mode 0 (super-step update): panel[i0.., c..c+256) -= A B^T over the columns
//    [kbeg, kend) (encoded as in the 128 x 128 tasks), A = panel rows
//    i0 + 128 rank.., B = panel rows c.., i0 >= c.
// Rows and columns past the target matrix are cut off by the stores' tensor
// maps (and read as zeros by the loads).
struct PairGeo {
  int arow, brow, x0, nk;  // operand rows (this CTA's A, this CTA's half of B), first column, k-steps
  int cy, cx, rows, N;     // target origin (rows, columns), its row count, columns of the tile
  bool panel;              // target is the panel (mode 0), else the update matrix
};
__device__ __forceinline__ PairGeo pair_geo(const FrontInfo &F, const Task &tk, int rank,
                                            int kstep) {
  PairGeo g;
  int K;
  if ((tk.c & 3) == 1) {
    g.arow = F.ncol + tk.a + 128 * rank;
    g.brow = F.ncol + tk.b + 128 * rank;
    g.x0 = 0;
    K = F.ncol;
    g.cy = tk.a + 128 * rank;
    g.rows = F.nrow;
    g.N = min(256, F.nrow - tk.b);
    g.panel = false;
  } else {
    const int kbeg = ((tk.c >> 2) & 0x7FFF) * kTileN, kend = ((tk.c >> 17) & 0x7FFF) * kTileN;
    g.arow = tk.a + 128 * rank;
    g.brow = tk.b + 128 * rank;
    g.x0 = kbeg;
    K = kend - kbeg;
    g.cy = g.arow;
    g.rows = F.ncol + F.nrow;
    g.N = min(256, F.ncol - tk.b);
    g.panel = true;
  }
  g.cx = tk.b;
  g.nk = (K + kstep - 1) / kstep;
  return g;
}

// 128 x 256 tiles in clusters of two CTAs: a task is the pair of tiles whose
// rows start at i0 and i0 + 128 and which share their B operand (256 rows of
// the panel). CTA r loads its own A rows and the r-th 128-row half of B with
// TMA multicast into both CTAs' shared memory, so each CTA reads 2/3 of the
// operand bytes of an unpaired tile. A stage is free again when the products
// of both CTAs have read it (each MMA commit is multicast to both CTAs' empty
// barriers, which count two arrivals). The second tile of a pair past the end
// of the target reads zeros and stores nothing.
template <int SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
    tc_pair_kernel(DevPlan dp, const Task *__restrict__ pairs, int npair,
                   const CUtensorMap *__restrict__ maps, const CUtensorMap *__restrict__ maps_lo,
                   const CUtensorMap *__restrict__ umaps, const CUtensorMap *__restrict__ lmaps,
                   const CUtensorMap *__restrict__ maps_bf, int32_t *status) {
  constexpr int BN = 256;
  constexpr int KS = SPLIT == kBf16 ? kTileKBf : kTileK;  // elements per k-step
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  using CF = Cfg<SPLIT, BN>;
  constexpr int S = CF::S, kBB = CF::kB * kTileBytes;
  uint8_t *sA = base;
  uint8_t *sB = sA + S * kTileBytes;
  uint8_t *sAl = sB + S * kBB;
  uint8_t *sBl = sAl + (SPLIT == 3 ? S * kTileBytes : 0);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + S * CF::kStage);
  uint64_t *empty = full + S;
  uint64_t *accfull = empty + S;
  uint64_t *accempty = accfull + 2;
  uint64_t *drain = accempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = cluster_rank();
  const int cid = blockIdx.x / 2, ncl = gridDim.x / 2;
  constexpr uint16_t kBoth = 0x3;

  if (threadIdx.x == 0) {
    for (int st = 0; st < S; st++) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 2);  // the products of both CTAs
    }
    for (int a = 0; a < 2; a++) {
      mbar_init(&accfull[a], 1);
      mbar_init(&accempty[a], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // the peer's barriers exist before anything is multicast to them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer: own A rows, this CTA's half of B for both CTAs
      uint32_t g = 0;
      for (int p = cid; p < npair && !*abort_flag; p += ncl) {
        const Task tk = pairs[p];
        const FrontInfo F = dp.fronts[tk.front];
        const CUtensorMap *amap = (SPLIT == kBf16 ? maps_bf : maps) + tk.front,
                          *lomap = maps_lo + tk.front;
        const PairGeo G = pair_geo(F, tk, (int)rank, KS);
        for (int kt = 0; kt < G.nk; kt++, g++) {
          const int st = g % S;
          const uint32_t round = g / S;
          const int x = G.x0 + kt * KS;
          if (!mbar_wait(&empty[st], (round & 1) ^ 1, status)) { *abort_flag = 1; break; }
          mbar_arrive_expect_tx(&full[st], (SPLIT == 3 ? 2 : 1) * (kTileBytes + kBB));
          tma_load_2d(sA + st * kTileBytes, amap, &full[st], x, G.arow);
          tma_load_2d_mc(sB + st * kBB + rank * kTileBytes, amap, &full[st], x, G.brow, kBoth);
          if (SPLIT == 3) {
            tma_load_2d(sAl + st * kTileBytes, lomap, &full[st], x, G.arow);
            tma_load_2d_mc(sBl + st * kBB + rank * kTileBytes, lomap, &full[st], x, G.brow, kBoth);
          }
        }
      }
      if (*abort_flag)
        for (uint32_t q = g > (uint32_t)S ? g - S : 0; q < g; q++)
          mbar_wait(&full[q % S], (q / S) & 1, status);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = SPLIT == kBf16 ? bf16_idesc<BN>() : tf32_idesc<BN>();
      uint32_t g = 0;
      int i = 0;
      for (int p = cid; p < npair && !*abort_flag; p += ncl, i++) {
        const Task tk = pairs[p];
        const FrontInfo F = dp.fronts[tk.front];
        const int nk = pair_geo(F, tk, (int)rank, KS).nk;
        const int a = i & 1;
        if (!mbar_wait(&accempty[a], ((i >> 1) & 1) ^ 1, status)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(a * BN);
        for (int kt = 0; kt < nk; kt++, g++) {
          const int st = g % S;
          const uint32_t round = g / S;
          if (!mbar_wait(&full[st], round & 1, status)) { *abort_flag = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t ad = sw128_desc(smem_u32(sA + st * kTileBytes));
          const uint64_t bd = sw128_desc(smem_u32(sB + st * kBB));
          const uint64_t ald = sw128_desc(smem_u32(sAl + st * kTileBytes));
          const uint64_t bld = sw128_desc(smem_u32(sBl + st * kBB));
#pragma unroll
          for (int k4 = 0; k4 < kTileK / 8; k4++) {
            if (SPLIT == kBf16) {
              mma_bf16(acc, ad + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
            } else if (SPLIT == 3) {
              mma_tf32(acc, ald + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
              mma_tf32(acc, ad + 2 * k4, bld + 2 * k4, idesc, 1);
              mma_tf32(acc, ad + 2 * k4, bd + 2 * k4, idesc, 1);
            } else {
              mma_tf32(acc, ad + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
            }
          }
          mma_commit_mc(&empty[st], kBoth);
        }
        if (*abort_flag) break;
        mma_commit(&accfull[a]);
      }
      mma_commit(drain);
      mbar_wait(drain, 0, status);
    }
  } else {  // warps 2-5: epilogue of this CTA's tile, 32 rows per warp
    // Each 32 x 32 block of the accumulator goes (negated) through this warp's
    // two 4 KB staging buffers in the 128-byte swizzled layout of the 32 x 32
    // tensor maps, and is added to the target by a TMA reduction in L2:
    // C -= A B^T without reading C into the SM, whole 128-byte rows per transfer.
    const int q = warp % 4;
    uint8_t *stg = base + CF::stage_off + q * 8192;
    uint32_t nissued = 0;
    int i = 0;
    for (int p = cid; p < npair && !*abort_flag; p += ncl, i++) {
      const Task tk = pairs[p];
      const FrontInfo F = dp.fronts[tk.front];
      const PairGeo G = pair_geo(F, tk, (int)rank, KS);
      const int a = i & 1;
      if (!mbar_wait(&accfull[a], (i >> 1) & 1, status)) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (G.cy + 32 * q < G.rows) {
        const CUtensorMap *um = (G.panel ? lmaps : umaps) + tk.front;
        for (int cb = 0; cb < (G.N + 31) / 32; cb++) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN + cb * 32), v);
          uint8_t *buf = stg + (nissued & 1) * 4096;
          if (lane == 0) bulk_wait_read<1>();  // the reduction that last read buf is done
          __syncwarp();
          stage_row(buf, lane, v, [](float x) { return -x; });
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) tma_reduce_add_2d(um, buf, G.cx + 32 * cb, G.cy + 32 * q);
          nissued++;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[a]);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync_all();  // no multicast can still target this CTA's shared memory
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
}

// Cholesky of one diagonal block (kb <= 128) in FP32 and the explicit inverse
// of its factor, written row-major (128 x 128, zero outside the lower kb x kb
// triangle) to scratch slot `b` for the triangular solve of the rows below as
// a tensor-core product, and (when Dinv is given) in the layout of the
// persistent solve. One right-looking step per column j does both: the rank-1
// update of the trailing block with column j of the factor, and the update of
// Y (which starts as I and ends as L^{-1} up to row scaling) with the same
// column and row j of the inverse, Y_j / L_jj. Thread (ty, tx) of a 16 x 16
// grid holds rows ty + 16a and columns tx + 16b of the lower tiles a >= b of
// both matrices in registers; the column of the factor, the row of Y and the
// next pivot's 1 / L_jj (computed by its owner before the barrier) are
// published in shared memory, double-buffered, so a step costs one barrier.
// The loop over the 16 columns of a tile column stays rolled, which keeps the
// code that runs once per launch small. A non-positive pivot is replaced by a
// large value (static pivoting) and counted.
__global__ void __launch_bounds__(256, 1) potrf_inv_kernel(DevPlan dp, const Task *__restrict__ tasks,
                                                        float *__restrict__ L,
                                                        float *__restrict__ Linv,
                                                        float *__restrict__ Dinv, int32_t *status) {
  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int k = tk.a, slot = tk.b, kb = min(TcPlan::kNb, F.ncol - k);
  __shared__ float cbuf[2][128];  // column j of the factor (unscaled, updated through step j - 1)
  __shared__ float ybuf[2][128];  // row j of Y
  __shared__ float rdv[128];      // 1 / L_jj
  __shared__ float sqv[128];      // L_jj
  float *g = L + F.loff + (int64_t)k * F.ld + k;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  // the pivot of column j, owned by the thread holding entry (j, j)
  auto pivot = [&](int j, float d) {
    const bool bad = !(d > 0.f) || !(d < 3.0e38f);
    if (bad) {
      d = 1e30f;
      atomicAdd(&status[ST_PERTURBED], 1);
    }
    // 1 / sqrt(d) from the hardware estimate and one Newton step for
    // r^-2 = d (r' = r + r (1 - d r^2) / 2, error ~1 ulp), instead of a
    // correctly rounded square root and division on the step's critical path
    float r = d >= 1e-30f ? rsqrtf(d) : 1.f / sqrtf(d);
    r = fmaf(0.5f * r, fmaf(-d * r, r, 1.f), r);
    sqv[j] = d * r;
    rdv[j] = r;
  };
  float acc[8][8], y[8][8];  // entries a >= b only
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int b = 0; b <= a; b++) {
      const int r = ty + 16 * a, c = tx + 16 * b;
      acc[a][b] = (r < kb && c <= r) ? g[(int64_t)r * F.ld + c] : 0.f;
      y[a][b] = (a == b && tx == ty) ? 1.f : 0.f;
    }
  if (tx == 0)
#pragma unroll
    for (int a = 0; a < 8; a++) cbuf[0][ty + 16 * a] = acc[a][0];
  if (ty == 0) ybuf[0][tx] = y[0][0];
  if (tid == 0) pivot(0, acc[0][0]);
  __syncthreads();
#pragma unroll
  for (int jb = 0; jb < 8; jb++) {
    if (16 * jb < kb) {
#pragma unroll 1
      for (int jj = 0; jj < 16; jj++) {
        const int j = 16 * jb + jj;
        if (j >= kb) break;
        const float *cb = cbuf[j & 1], *yb = ybuf[j & 1];
        const float rs = rdv[j];
        float u[8], v[8], x[8];
#pragma unroll
        for (int a = jb; a < 8; a++) {
          const int r = ty + 16 * a, c = tx + 16 * a;
          u[a] = r > j ? cb[r] * rs : 0.f;  // L_rj below the diagonal
          v[a] = c > j ? cb[c] * rs : 0.f;
        }
#pragma unroll
        for (int b = 0; b <= jb; b++) x[b] = yb[tx + 16 * b] * rs;  // row j of L^{-1}
#pragma unroll
        for (int a = jb; a < 8; a++)
#pragma unroll
          for (int b = jb; b <= a; b++) acc[a][b] = fmaf(-u[a], v[b], acc[a][b]);
#pragma unroll
        for (int a = jb; a < 8; a++)
#pragma unroll
          for (int b = 0; b <= jb && b <= a; b++) y[a][b] = fmaf(-u[a], x[b], y[a][b]);
        const int jn = j + 1;
        if (jn < kb) {
          float *nc = cbuf[jn & 1], *ny = ybuf[jn & 1];
          if (jj < 15) {
            if (tx == jj + 1) {
#pragma unroll
              for (int a = jb; a < 8; a++) nc[ty + 16 * a] = acc[a][jb];
              if (ty == jj + 1) pivot(jn, acc[jb][jb]);
            }
            if (ty == jj + 1)
#pragma unroll
              for (int b = 0; b <= jb; b++) ny[tx + 16 * b] = y[jb][b];
          } else if (jb < 7) {
            if (tx == 0) {
#pragma unroll
              for (int a = jb + 1; a < 8; a++) nc[ty + 16 * a] = acc[a][jb + 1];
              if (ty == 0) pivot(jn, acc[jb + 1][jb + 1]);
            }
            if (ty == 0)
#pragma unroll
              for (int b = 0; b <= jb + 1; b++) ny[tx + 16 * b] = y[jb + 1][b];
          }
        }
        __syncthreads();
      }
    }
  }
  float *out = Linv + (int64_t)slot * 128 * 128;
  const int ldi = (kb + 3) & ~3;
  float *o2 = Dinv ? Dinv + dp.fs_dinv_off[dp.fs_first_slot[tk.front] + k / TcPlan::kNb] : nullptr;
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int b = 0; b < 8; b++) {
      const int r = ty + 16 * a, c = tx + 16 * b;
      float xv = 0.f;
      if (b <= a) {
        if (r < kb && c < r) g[(int64_t)r * F.ld + c] = acc[a][b] * rdv[c];
        if (r < kb && c == r) g[(int64_t)r * F.ld + c] = sqv[c];
        if (r < kb && c <= r) xv = y[a][b] * rdv[r];
      }
      out[r * 128 + c] = xv;
      if (o2 && r < kb && c < ldi) o2[r * ldi + c] = xv;
    }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      throw std::runtime_error("cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

void TcPlan::build(const Plan &plan) {
  gemm_.clear();
  potrf_.clear();
  trsm_.clear();
  pairs_.clear();
  levels_.assign(plan.levels.size(), Level{});
  nfronts_ = (int)plan.fronts.size();
  max_slots_ = 1;
  for (size_t li = 0; li < plan.levels.size(); li++) {
    const LevelPlan &LP = plan.levels[li];
    Level &lv = levels_[li];
    // Left-looking in super-steps of kSuper columns. Super-step s (columns
    // [K0, K0 + kSuper)) starts with the update of its columns by the columns
    // before it; then each 128-wide block column takes the columns of its own
    // super-step before it (short K), is factored and solved below. On a level
    // of at most kAheadFronts fronts that chain of block steps is latency-bound,
    // so the update of super-step s + 1 by the columns before K0 runs ahead on
    // the side stream meanwhile, and super-step s + 1 starts with the update by
    // super-step s's columns only (K in [K0, K0 + kSuper)).
    auto enc = [](int32_t kbeg, int32_t kend) { return 0 | (kbeg / kNb) << 2 | (kend / kNb) << 17; };
    // columns [c0, c0 + kSuper) of all fronts: 256-wide tiles in row pairs,
    // rows outermost so that the column tiles of a row band run back to back
    // (one read of the band's A rows serves both)
    auto span = [&](int32_t c0, int32_t kbeg, int32_t kend) {
      for (int32_t t = LP.front_b; t < LP.front_e; t++) {
        const int32_t s = plan.level_fronts[t];
        const FrontInfo &F = plan.fronts[s];
        for (int32_t i0 = c0; i0 < F.ncol + F.nrow; i0 += 2 * kTileM)
          for (int32_t c = c0; c < std::min(F.ncol, c0 + kSuper) && c <= i0; c += kSyrkN)
            pairs_.push_back({s, i0, c, enc(kbeg, kend)});
      }
    };
    bool ahead_done = false;  // the previous super-step ran this one's update ahead
    for (int32_t K0 = 0; K0 < LP.max_ncol; K0 += kSuper) {
      Super sp{};
      sp.k0 = K0;
      sp.now_b = (int)pairs_.size();
      if (K0 > 0) span(K0, ahead_done ? K0 - kSuper : 0, K0);
      sp.now_e = (int)pairs_.size();
      sp.ahead_b = (int)pairs_.size();
      if (K0 > 0 && K0 + kSuper < LP.max_ncol && LP.front_e - LP.front_b <= kAheadFronts)
        span(K0 + kSuper, 0, K0);
      sp.ahead_e = (int)pairs_.size();
      ahead_done = sp.ahead_e > sp.ahead_b;
      sp.step_b = (int)lv.steps.size();
      for (int32_t k = K0; k < std::min(LP.max_ncol, K0 + kSuper); k += kNb) {
        Step st{};
        st.gemm_b = (int)gemm_.size();
        for (int32_t t = LP.front_b; t < LP.front_e && k > K0; t++) {
          const int32_t s = plan.level_fronts[t];
          const FrontInfo &F = plan.fronts[s];
          if (F.ncol <= k) continue;
          for (int32_t i0 = k; i0 < F.ncol + F.nrow; i0 += kTileM) gemm_.push_back({s, i0, k, enc(K0, k)});
        }
        st.gemm_e = (int)gemm_.size();
        st.potrf_b = (int)potrf_.size();
        int32_t slot = 0;
        for (int32_t t = LP.front_b; t < LP.front_e; t++) {
          const int32_t s = plan.level_fronts[t];
          if (plan.fronts[s].ncol > k) potrf_.push_back({s, k, slot++, 0});
        }
        st.potrf_e = (int)potrf_.size();
        max_slots_ = std::max(max_slots_, slot);
        st.trsm_b = (int)trsm_.size();
        slot = 0;
        for (int32_t t = LP.front_b; t < LP.front_e; t++) {
          const int32_t s = plan.level_fronts[t];
          const FrontInfo &F = plan.fronts[s];
          if (F.ncol <= k) continue;
          const int32_t kb = std::min(kNb, F.ncol - k);
          for (int32_t i0 = k + kb; i0 < F.ncol + F.nrow; i0 += kTileM) trsm_.push_back({s, i0, k, 2 | (slot << 2)});
          slot++;
        }
        st.trsm_e = (int)trsm_.size();
        lv.steps.push_back(st);
      }
      sp.step_e = (int)lv.steps.size();
      lv.supers.push_back(sp);
    }
    // SYRK: 128 x 256 tiles (i0, j0), (i0 + 128, j0) of the lower triangle,
    // ordered in groups of kBandGroup row bands with the column outermost, so
    // that the pairs running at the same time share a few A bands and B panels
    lv.pair_b = (int)pairs_.size();
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const FrontInfo &F = plan.fronts[s];
      constexpr int32_t band = 2 * kTileM;
      for (int32_t g0 = 0; g0 < F.nrow; g0 += kBandGroup * band) {
        const int32_t g1 = std::min(F.nrow, g0 + kBandGroup * band);
        for (int32_t j0 = 0; j0 < g1; j0 += kSyrkN)
          for (int32_t i0 = g0; i0 < g1; i0 += band)
            if (j0 <= i0) pairs_.push_back({s, i0, j0, 1});
      }
    }
    lv.pair_e = (int)pairs_.size();
  }
  // range checks of the tasks against the fronts (the kernel masks only the tile edges)
  auto fail = [](const char *w) { throw std::runtime_error(std::string("tc plan check: ") + w); };
  for (const Task &t : gemm_) {
    const FrontInfo &F = plan.fronts[t.front];
    const int32_t kbeg = ((t.c >> 2) & 0x7FFF) * kNb, kend = ((t.c >> 17) & 0x7FFF) * kNb;
    if (!(t.b > 0 && t.b < F.ncol && t.b % kNb == 0 && t.a >= t.b && t.a < F.ncol + F.nrow &&
          (t.c & 3) == 0 && kbeg >= 0 && kbeg < kend && kend <= t.b))
      fail("gemm");
  }
  for (const Task &t : pairs_) {
    const FrontInfo &F = plan.fronts[t.front];
    if ((t.c & 3) == 1) {
      if (!(t.a >= 0 && t.a < F.nrow && t.a % (2 * kTileM) == 0 && t.b >= 0 && t.b <= t.a &&
            t.b % kSyrkN == 0 && t.c == 1))
        fail("syrk pair");
    } else {
      const int32_t kbeg = ((t.c >> 2) & 0x7FFF) * kNb, kend = ((t.c >> 17) & 0x7FFF) * kNb;
      if (!(t.b > 0 && t.b < F.ncol && t.b % kSyrkN == 0 && t.a >= t.b && t.a < F.ncol + F.nrow &&
            (t.c & 3) == 0 && kbeg >= 0 && kbeg < kend && kend <= t.b))
        fail("update pair");
    }
  }
  for (const Task &t : trsm_) {
    const FrontInfo &F = plan.fronts[t.front];
    const int kb = std::min(kNb, F.ncol - t.b);
    if (!(t.b >= 0 && t.b < F.ncol && t.a >= t.b + kb && t.a < F.ncol + F.nrow && (t.c & 3) == 2 &&
          (t.c >> 2) < max_slots_))
      fail("trsm");
  }
  for (const Task &t : potrf_)
    if (!(t.a >= 0 && t.a < plan.fronts[t.front].ncol && t.b >= 0 && t.b < max_slots_)) fail("potrf");
  // The look-ahead runs concurrently with the block steps of its super-step:
  // it may only read columns before k0 and write columns from k0 + kSuper on,
  // while everything on the main stream stays inside [k0, k0 + kSuper).
  auto kend_of = [](const Task &t) { return ((t.c >> 17) & 0x7FFF) * kNb; };
  auto kbeg_of = [](const Task &t) { return ((t.c >> 2) & 0x7FFF) * kNb; };
  for (const Level &lv : levels_)
    for (const Super &sp : lv.supers) {
      const int32_t lo = sp.k0, hi = sp.k0 + kSuper;
      for (int i = sp.ahead_b; i < sp.ahead_e; i++)
        if (!(kend_of(pairs_[i]) <= lo && pairs_[i].b >= hi)) fail("look-ahead columns");
      for (int i = sp.now_b; i < sp.now_e; i++)
        if (!(pairs_[i].b >= lo && pairs_[i].b < hi && kend_of(pairs_[i]) <= lo)) fail("super-step update");
      for (int i = sp.step_b; i < sp.step_e; i++) {
        const Step &st = lv.steps[i];
        for (int q = st.gemm_b; q < st.gemm_e; q++)
          if (!(gemm_[q].b >= lo && gemm_[q].b < hi && kbeg_of(gemm_[q]) >= lo)) fail("block-step update");
        for (int q = st.potrf_b; q < st.potrf_e; q++)
          if (!(potrf_[q].a >= lo && potrf_[q].a < hi)) fail("block-step factor");
        for (int q = st.trsm_b; q < st.trsm_e; q++)
          if (!(trsm_[q].b >= lo && trsm_[q].b < hi)) fail("block-step solve");
      }
    }
  ready_ = false;
}

void TcPlan::layout(Carve &cv, cudaStream_t st) {
  auto up = [&](const std::vector<Task> &v) {
    Task *p = cv.take<Task>(std::max<size_t>(v.size(), 1));
    if (cv.base && !v.empty())
      cudaMemcpyAsync(p, v.data(), v.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    return p;
  };
  d_gemm_ = up(gemm_);
  d_potrf_ = up(potrf_);
  d_trsm_ = up(trsm_);
  d_pairs_ = up(pairs_);
  // L, Llo (32 x 128 boxes), the inverse scratch, U, L, Llo (32 x 32 boxes),
  // the BF16 copy (64 x 128 boxes, then 32 x 32 boxes)
  d_maps_ = cv.take<CUtensorMap>(7 * std::max(nfronts_, 1) + 1);
  d_inv_ = cv.take<float>((size_t)max_slots_ * kTileM * kTileN);
  ready_ = false;
}

void TcPlan::encode(const Plan &plan, float *L, float *Llo, float *U, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!side_) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&side_, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_main_, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_side_, cudaEventDisableTiming) != cudaSuccess)
      throw std::runtime_error("cannot create the look-ahead stream");
  }
  L_ = L;
  Llo_ = Llo;
  U_ = U;
  const size_t nfr = plan.fronts.size();
  std::vector<CUtensorMap> maps(2 * nfr);  // panels of L, then of Llo
  for (size_t s = 0; s < 2 * nfr; s++) {
    const FrontInfo &F = plan.fronts[s % nfr];
    float *base = (s < nfr ? L : Llo) + F.loff;
    cuuint64_t dims[2] = {(cuuint64_t)F.ncol, (cuuint64_t)(F.ncol + F.nrow)};
    cuuint64_t strides[1] = {(cuuint64_t)F.ld * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      throw std::runtime_error("cuTensorMapEncodeTiled failed for front " + std::to_string(s % nfr));
  }
  {
    CUtensorMap im;
    cuuint64_t dims[2] = {(cuuint64_t)kTileN, (cuuint64_t)max_slots_ * kTileM};
    cuuint64_t strides[1] = {(cuuint64_t)kTileN * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileN};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&im, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d_inv_, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed for the inverse scratch");
    maps.push_back(im);
  }
  auto box32 = [&](float *ptr, const char *what, size_t s, uint64_t cols, uint64_t rows, int64_t ld) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    if (cols > 0 && rows > 0) {
      cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
      cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
      cuuint32_t box[2] = {32, 32};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        throw std::runtime_error(std::string("cuTensorMapEncodeTiled failed for ") + what + " " +
                                 std::to_string(s));
    }
    maps.push_back(m);
  };
  // 32 x 32 boxes for the epilogues' stores and reductions: update matrices,
  // then panels of L and of Llo
  for (size_t s = 0; s < nfr; s++) {
    const FrontInfo &F = plan.fronts[s];
    box32(U + F.uoff, "update matrix", s, F.nrow, F.nrow, F.uld);
  }
  for (size_t s = 0; s < nfr; s++) {
    const FrontInfo &F = plan.fronts[s];
    box32(L + F.loff, "panel", s, F.ncol, F.ncol + F.nrow, F.ld);
  }
  for (size_t s = 0; s < nfr; s++) {
    const FrontInfo &F = plan.fronts[s];
    box32(Llo + F.loff, "low-part panel", s, F.ncol, F.ncol + F.nrow, F.ld);
  }
  // The BF16 copy of the finished panel entries lives in the low-part buffer
  // (the two are never needed by the same factorisation), each panel at the
  // same element offset and row stride as in L: operand loads in 64 x 128
  // boxes (128-byte swizzled rows), epilogue stores in 32 x 32 boxes.
  __nv_bfloat16 *Lbf = reinterpret_cast<__nv_bfloat16 *>(Llo);
  auto bfmap = [&](size_t s, uint32_t bx, uint32_t by, CUtensorMapSwizzle sw) {
    const FrontInfo &F = plan.fronts[s];
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)F.ncol, (cuuint64_t)(F.ncol + F.nrow)};
    cuuint64_t strides[1] = {(cuuint64_t)F.ld * sizeof(__nv_bfloat16)};
    cuuint32_t box[2] = {bx, by};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)(Lbf + F.loff), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                     by == 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      throw std::runtime_error("cuTensorMapEncodeTiled failed for the BF16 panel " + std::to_string(s));
    maps.push_back(m);
  };
  for (size_t s = 0; s < nfr; s++) bfmap(s, kTileKBf, kTileM, CU_TENSOR_MAP_SWIZZLE_128B);
  for (size_t s = 0; s < nfr; s++) bfmap(s, 32, 32, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!maps.empty())
    if (cudaMemcpyAsync(d_maps_, maps.data(), maps.size() * sizeof(CUtensorMap),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
      throw std::runtime_error("tensor map upload failed");
  if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("tensor map upload failed");
  cudaFuncSetAttribute(tc_gemm_kernel<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<1, 128>::smem);
  cudaFuncSetAttribute(tc_gemm_kernel<3, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<3, 128>::smem);
  cudaFuncSetAttribute(tc_pair_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<1, kSyrkN>::smem);
  cudaFuncSetAttribute(tc_pair_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<3, kSyrkN>::smem);
  cudaFuncSetAttribute(tc_gemm_kernel<kBf16, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Cfg<kBf16, 128>::smem);
  cudaFuncSetAttribute(tc_pair_kernel<kBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Cfg<kBf16, kSyrkN>::smem);
  ready_ = true;
}

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Persistent launch: at most ctas CTAs (one per SM), each taking tiles ctas apart.
template <int SPLIT, int BN>
static void gemm_launch(int ntask, int ctas, const DevPlan &dp, const Task *tasks,
                        const CUtensorMap *maps, int nfronts, int32_t *status, cudaStream_t st) {
  const CUtensorMap *maps_lo = maps + nfronts, *inv_map = maps + 2 * nfronts;
  const CUtensorMap *lmaps = inv_map + 1 + nfronts, *llomaps = lmaps + nfronts;
  const CUtensorMap *maps_bf = llomaps + nfronts, *lbfmaps = maps_bf + nfronts;
  note_launch();
  tc_gemm_kernel<SPLIT, BN><<<std::min(ntask, std::max(ctas, 1)), 192, Cfg<SPLIT, BN>::smem, st>>>(
      dp, tasks, ntask, maps, maps_lo, inv_map, lmaps, llomaps, maps_bf, lbfmaps, TcPlan::kNb,
      status);
}

// Pair kernel on at most ctas CTAs (clusters of two, each pair of tiles ncl apart).
template <int SPLIT>
static void pair_launch(int npair, int ctas, const DevPlan &dp, const Task *pairs,
                        const CUtensorMap *maps, int nfronts, int32_t *status, cudaStream_t st) {
  const CUtensorMap *maps_lo = maps + nfronts, *umaps = maps + 2 * nfronts + 1;
  const CUtensorMap *lmaps = umaps + nfronts, *maps_bf = lmaps + 2 * nfronts;
  const int ncl = std::max(1, std::min({npair, ctas / 2, kMaxClusters}));
  note_launch();
  tc_pair_kernel<SPLIT><<<2 * ncl, 192, Cfg<SPLIT, kSyrkN>::smem, st>>>(
      dp, pairs, npair, maps, maps_lo, umaps, lmaps, maps_bf, status);
}

TcPlan::~TcPlan() {
  if (ev_main_) cudaEventDestroy(ev_main_);
  if (ev_side_) cudaEventDestroy(ev_side_);
  if (side_) cudaStreamDestroy(side_);
}

void TcPlan::factor(const DevPlan &dp, const Plan &plan, const double *kval, float *L, float *U,
                    float *Dinv, int32_t *status, int split, cudaStream_t st) {
  auto gemm3 = split == 3 ? gemm_launch<3, 128>
                          : (split == kBf16 ? gemm_launch<kBf16, 128> : gemm_launch<1, 128>);
  auto pair3 = split == 3 ? pair_launch<3> : (split == kBf16 ? pair_launch<kBf16> : pair_launch<1>);
  const CUtensorMap *maps = static_cast<const CUtensorMap *>(d_maps_);
  if (L != L_ || U != U_) throw std::runtime_error("tensor maps were encoded for other factor buffers");
  if (!side_) throw std::runtime_error("tensor-core factor streams not created");
  const int sms = sm_count();
  const int main_ctas = std::min(kMainCtas, sms / 2), side_ctas = sms - main_ctas;
  auto gemm = [&](const Task *t, int n, int ctas, cudaStream_t s) {
    gemm3(n, ctas, dp, t, maps, nfronts_, status, s);
  };
  auto pair = [&](int b, int e, int ctas, cudaStream_t s) {
    if (e > b) pair3(e - b, ctas, dp, d_pairs_ + b, maps, nfronts_, status, s);
  };
  bool pending = false;  // look-ahead work on the side stream not yet joined
  for (size_t li = 0; li < levels_.size(); li++) {
    const Level &lv = levels_[li];
    launch_build_level<float>(dp, plan.levels[li], kval, L, U, st);
    for (const Super &sp : lv.supers) {
      if (pending) {  // this super-step's columns took the look-ahead update
        cudaStreamWaitEvent(st, ev_side_, 0);
        pending = false;
      }
      const bool ahead = sp.ahead_e > sp.ahead_b;
      if (ahead) {  // the columns before this super-step are final: fork
        cudaEventRecord(ev_main_, st);
        cudaStreamWaitEvent(side_, ev_main_, 0);
      }
      pair(sp.now_b, sp.now_e, sms, st);
      const int ctas = ahead ? main_ctas : sms;
      if (ahead) {
        pair(sp.ahead_b, sp.ahead_e, side_ctas, side_);
        cudaEventRecord(ev_side_, side_);
        pending = true;
      }
      for (int i = sp.step_b; i < sp.step_e; i++) {
        const Step &s = lv.steps[i];
        if (s.gemm_e > s.gemm_b) gemm(d_gemm_ + s.gemm_b, s.gemm_e - s.gemm_b, ctas, st);
        if (s.potrf_e > s.potrf_b)
          { note_launch(); potrf_inv_kernel<<<s.potrf_e - s.potrf_b, 256, 0, st>>>(dp, d_potrf_ + s.potrf_b, L, d_inv_, Dinv, status); }
        if (s.trsm_e > s.trsm_b) gemm(d_trsm_ + s.trsm_b, s.trsm_e - s.trsm_b, ctas, st);
      }
    }
    if (pending) {
      cudaStreamWaitEvent(st, ev_side_, 0);
      pending = false;
    }
    pair(lv.pair_b, lv.pair_e, sms, st);  // the level's update matrices
  }
}

}  // namespace gipm
