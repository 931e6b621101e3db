// Tensor-core GEMM for the supernodal factorisation on sm_103a (tcgen05 + TMA).
//
// One CTA computes one 128 x 128 tile of C -= A B^T, where A and B are row
// blocks of a front's panel (row-major, K contiguous: "K-major") and C is
// either the panel itself (left-looking update of a block column) or the
// front's update matrix (SYRK). Warp 0 streams 128 x 32 FP32 tiles of A and B
// through a 4-stage ring of 128B-swizzled shared memory with TMA, warp 1
// issues tcgen05.mma kind::tf32 (M=128, N=128, K=8) into a 128-column FP32
// accumulator in tensor memory, warps 2-5 read the accumulator back with
// tcgen05.ld and subtract it from C. Every wait on an mbarrier is bounded by a
// clock limit; on expiry the CTA records ST_TIMEOUT, skips the epilogue and
// still releases its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdexcept>
#include <string>

#include "launch.h"
#include "tc.h"

namespace gipm {

namespace {

constexpr int kTileM = 128, kTileN = 128, kTileK = 32, kStages = 4;
constexpr int kTileBytes = kTileM * kTileK * 4;  // 16 KB per operand tile
constexpr long long kSpinCycles = 2000000000LL;  // ~1 s at 2 GHz
template <int SPLIT> struct StagesOf { static constexpr int value = SPLIT == 3 ? 3 : kStages; };
template <int SPLIT>
constexpr int smem_bytes() {
  return (SPLIT == 3 ? 4 : 2) * StagesOf<SPLIT>::value * kTileBytes + 1024 /*barriers*/ +
         1024 /*alignment*/;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// x - tf32(x): what the tensor core drops from an FP32 operand (low 13 mantissa bits)
__device__ __forceinline__ float lo1(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}
__device__ __forceinline__ float4 lo_part(float4 v) {
  return make_float4(lo1(v.x), lo1(v.y), lo1(v.z), lo1(v.w));
}

// Bounded wait on an mbarrier phase; false (and ST_TIMEOUT recorded) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kSpinCycles) {
      atomicExch(&status[ST_TIMEOUT], 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
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
__host__ __device__ constexpr uint32_t tf32_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
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

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
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

// Task: front, a = first row of the A tile (front-local), b = k (modes 0, 2) or
// j0 (mode 1), c = mode | slot << 2.
//  Mode 0 (left-looking update): C = panel[a:a+128, k:k+kb] -= A B^T with
//    A = panel rows a.., B = panel rows k.., K = k.
//  Mode 1 (update matrix): C = U[a:a+128, b:b+128] -= A B^T with
//    A = panel rows ncol+a.., B = panel rows ncol+b.., K = ncol.
//  Mode 2 (triangular solve of the rows below a diagonal block, as a product
//    with its inverse): C = panel[a:a+128, k:k+kb] = A B^T with A = the same
//    panel rows and columns, B = L_kk^{-1} from scratch slot `slot`, K = kb.
//    The tile's rows are read completely before its epilogue overwrites them.
template <int SPLIT>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(DevPlan dp, const Task *__restrict__ tasks, const CUtensorMap *__restrict__ maps,
                   const CUtensorMap *__restrict__ inv_map, float *__restrict__ L,
                   float *__restrict__ U, int nb, int32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  constexpr int S = StagesOf<SPLIT>::value;
  uint8_t *sA = base;
  uint8_t *sB = base + S * kTileBytes;
  uint8_t *sAl = base + 2 * S * kTileBytes;  // low parts (SPLIT == 3 only)
  uint8_t *sBl = base + 3 * S * kTileBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(base + (SPLIT == 3 ? 4 : 2) * S * kTileBytes);
  uint64_t *empty = full + S;
  uint64_t *lofull = empty + S;
  uint64_t *accum = lofull + S;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow;
  const int mode = tk.c & 3;
  int arow, brow, K, M, N, ax0 = 0;
  float *C;
  int64_t ldc;
  const CUtensorMap *amap = maps + tk.front, *bmap = amap;
  if (mode == 0) {
    const int k = tk.b;
    arow = tk.a;
    brow = k;
    K = k;
    M = min(kTileM, nf - tk.a);
    N = min(nb, F.ncol - k);
    C = L + F.loff + (int64_t)tk.a * F.ld + k;
    ldc = F.ld;
  } else if (mode == 2) {
    const int k = tk.b;
    arow = tk.a;
    ax0 = k;
    brow = (tk.c >> 2) * kTileN;
    bmap = inv_map;
    N = min(nb, F.ncol - k);
    K = N;
    M = min(kTileM, nf - tk.a);
    C = L + F.loff + (int64_t)tk.a * F.ld + k;
    ldc = F.ld;
  } else {
    arow = F.ncol + tk.a;
    brow = F.ncol + tk.b;
    K = F.ncol;
    M = min(kTileM, F.nrow - tk.a);
    N = min(kTileN, F.nrow - tk.b);
    C = U + F.uoff + (int64_t)tk.a * F.uld + tk.b;
    ldc = F.uld;
  }
  const int nk = (K + kTileK - 1) / kTileK;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&lofull[s], 4);  // one arrival per converting warp
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTileN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int kt = 0; kt < nk; kt++) {
        const int s = kt % S, round = kt / S;
        if (!mbar_wait(&empty[s], (round & 1) ^ 1, status)) { *abort_flag = 1; break; }
        mbar_arrive_expect_tx(&full[s], 2 * kTileBytes);
        tma_load_2d(sA + s * kTileBytes, amap, &full[s], ax0 + kt * kTileK, arow);
        tma_load_2d(sB + s * kTileBytes, bmap, &full[s], kt * kTileK, brow);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc();
      for (int kt = 0; kt < nk; kt++) {
        const int s = kt % S, round = kt / S;
        if (!mbar_wait(&full[s], round & 1, status)) { *abort_flag = 1; break; }
        if (SPLIT == 3 && !mbar_wait(&lofull[s], round & 1, status)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ad = sw128_desc(smem_u32(sA + s * kTileBytes));
        const uint64_t bd = sw128_desc(smem_u32(sB + s * kTileBytes));
        const uint64_t ald = sw128_desc(smem_u32(sAl + s * kTileBytes));
        const uint64_t bld = sw128_desc(smem_u32(sBl + s * kTileBytes));
#pragma unroll
        for (int k4 = 0; k4 < kTileK / 8; k4++) {  // 8 TF32 = 32 bytes per MMA along K
          if (SPLIT == 3) {  // small terms first: A_lo B + A B_lo, then A B
            mma_tf32(tmem, ald + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
            mma_tf32(tmem, ad + 2 * k4, bld + 2 * k4, idesc, 1);
            mma_tf32(tmem, ad + 2 * k4, bd + 2 * k4, idesc, 1);
          } else {
            mma_tf32(tmem, ad + 2 * k4, bd + 2 * k4, idesc, (kt | k4) != 0);
          }
        }
        mma_commit(&empty[s]);
      }
      mma_commit(accum);
    }
  } else {
    if (SPLIT == 3) {
      // low parts x - tf32(x) of both operand tiles (tf32 keeps the top 19 bits)
      const int t = threadIdx.x - 64;
      for (int kt = 0; kt < nk && !*abort_flag; kt++) {
        const int s = kt % S, round = kt / S;
        if (!mbar_wait(&full[s], round & 1, status)) { *abort_flag = 1; break; }
        const float4 *a = reinterpret_cast<const float4 *>(sA + s * kTileBytes);
        const float4 *b = reinterpret_cast<const float4 *>(sB + s * kTileBytes);
        float4 *al = reinterpret_cast<float4 *>(sAl + s * kTileBytes);
        float4 *bl = reinterpret_cast<float4 *>(sBl + s * kTileBytes);
        for (int i = t; i < kTileBytes / 16; i += 128) {
          al[i] = lo_part(a[i]);
          bl[i] = lo_part(b[i]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&lofull[s]);
      }
    }
    const bool ok = mbar_wait(accum, 0, status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp % 4;  // tensor-memory lane quarter this warp may access
    const int row = q * 32 + lane;
    if (ok && !*abort_flag) {
      for (int cb = 0; cb < (N + 31) / 32; cb++) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32), v);
        if (row < M) {
          float *crow = C + (int64_t)row * ldc + cb * 32;
          const int nc = min(32, N - cb * 32);
          if (mode == 2) {
#pragma unroll
            for (int c = 0; c < 32; c++)
              if (c < nc) crow[c] = v[c];
          } else {
#pragma unroll
            for (int c = 0; c < 32; c++)
              if (c < nc) crow[c] -= v[c];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTileN));
}

// Cholesky of one diagonal block (kb <= 128) in FP32 and the explicit inverse
// of its factor, written row-major (128 x 128, zero outside the lower kb x kb
// triangle) to scratch slot `b` for the triangular solve of the rows below as
// a tensor-core product. Division-free 2D thread mapping for the trailing
// update; a non-positive pivot is replaced by a large value (static pivoting)
// and counted.
__global__ void __launch_bounds__(256) potrf_inv_kernel(DevPlan dp, const Task *__restrict__ tasks,
                                                        float *__restrict__ L,
                                                        float *__restrict__ Linv,
                                                        int32_t *status) {
  constexpr int LS = 129;
  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int k = tk.a, slot = tk.b, kb = min(TcPlan::kNb, F.ncol - k);
  extern __shared__ float smf[];
  float *A = smf;            // [128][129]
  float *X = smf + 128 * LS;  // [128][129]
  float *g = L + F.loff + (int64_t)k * F.ld + k;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int e = tid; e < 128 * 128; e += 256) {
    const int r = e >> 7, c = e & 127;
    A[r * LS + c] = (r < kb && c <= r) ? g[(int64_t)r * F.ld + c] : 0.f;
  }
  __syncthreads();
  for (int j = 0; j < kb; j++) {
    if (tid == 0) {
      float d = A[j * LS + j];
      if (!(d > 0.f) || !(d < 3.0e38f)) {
        d = 1e30f;
        atomicAdd(&status[ST_PERTURBED], 1);
      }
      A[j * LS + j] = sqrtf(d);
    }
    __syncthreads();
    const float ljj = A[j * LS + j];
    if (tid > j && tid < kb) A[tid * LS + j] /= ljj;
    __syncthreads();
    for (int r = j + 1 + ty; r < kb; r += 16) {
      const float arj = A[r * LS + j];
      for (int c = j + 1 + tx; c <= r; c += 16) A[r * LS + c] = fmaf(-arj, A[c * LS + j], A[r * LS + c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += 256) {
    const int r = e / kb, c = e % kb;
    if (c <= r) g[(int64_t)r * F.ld + c] = A[r * LS + c];
  }
  if (tid < 128) {  // column c of the inverse by forward substitution
    const int c = tid;
    for (int i = 0; i < 128; i++) X[i * LS + c] = 0.f;
    if (c < kb)
      for (int i = c; i < kb; i++) {
        float s = (i == c) ? 1.f : 0.f;
        for (int m = c; m < i; m++) s = fmaf(-A[i * LS + m], X[m * LS + c], s);
        X[i * LS + c] = s / A[i * LS + i];
      }
  }
  __syncthreads();
  float *out = Linv + (int64_t)slot * 128 * 128;
  for (int e = tid; e < 128 * 128; e += 256) out[e] = X[(e >> 7) * LS + (e & 127)];
}

constexpr int kPotrfInvSmem = 2 * 128 * 129 * 4;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

}  // namespace

void TcPlan::build(const Plan &plan) {
  gemm_.clear();
  potrf_.clear();
  trsm_.clear();
  syrk_.clear();
  levels_.assign(plan.levels.size(), Level{});
  nfronts_ = (int)plan.fronts.size();
  max_slots_ = 1;
  for (size_t li = 0; li < plan.levels.size(); li++) {
    const LevelPlan &LP = plan.levels[li];
    Level &lv = levels_[li];
    for (int32_t k = 0; k < LP.max_ncol; k += kNb) {
      Step st{};
      st.gemm_b = (int)gemm_.size();
      for (int32_t t = LP.front_b; t < LP.front_e && k > 0; t++) {
        const int32_t s = plan.level_fronts[t];
        const FrontInfo &F = plan.fronts[s];
        if (F.ncol <= k) continue;
        for (int32_t i0 = k; i0 < F.ncol + F.nrow; i0 += kTileM) gemm_.push_back({s, i0, k, 0});
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
    lv.syrk_b = (int)syrk_.size();
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const FrontInfo &F = plan.fronts[s];
      for (int32_t i0 = 0; i0 < F.nrow; i0 += kTileM)
        for (int32_t j0 = 0; j0 <= i0; j0 += kTileN) syrk_.push_back({s, i0, j0, 1});
    }
    lv.syrk_e = (int)syrk_.size();
  }
  // range checks of the tasks against the fronts (the kernel masks only the tile edges)
  auto fail = [](const char *w) { throw std::runtime_error(std::string("tc plan check: ") + w); };
  for (const Task &t : gemm_) {
    const FrontInfo &F = plan.fronts[t.front];
    if (!(t.b > 0 && t.b < F.ncol && t.a >= t.b && t.a < F.ncol + F.nrow && t.c == 0)) fail("gemm");
  }
  for (const Task &t : syrk_) {
    const FrontInfo &F = plan.fronts[t.front];
    if (!(t.a >= 0 && t.a < F.nrow && t.b >= 0 && t.b <= t.a && t.c == 1)) fail("syrk");
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
  d_syrk_ = up(syrk_);
  d_maps_ = cv.take<CUtensorMap>(std::max(nfronts_, 1) + 1);  // + the inverse-scratch map
  d_inv_ = cv.take<float>((size_t)max_slots_ * kTileM * kTileN);
  ready_ = false;
}

void TcPlan::encode(const Plan &plan, float *L, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  std::vector<CUtensorMap> maps(plan.fronts.size());
  for (size_t s = 0; s < plan.fronts.size(); s++) {
    const FrontInfo &F = plan.fronts[s];
    cuuint64_t dims[2] = {(cuuint64_t)F.ncol, (cuuint64_t)(F.ncol + F.nrow)};
    cuuint64_t strides[1] = {(cuuint64_t)F.ld * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)kTileM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(L + F.loff), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      throw std::runtime_error("cuTensorMapEncodeTiled failed for front " + std::to_string(s));
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
  if (!maps.empty())
    if (cudaMemcpyAsync(d_maps_, maps.data(), maps.size() * sizeof(CUtensorMap),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
      throw std::runtime_error("tensor map upload failed");
  if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("tensor map upload failed");
  cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<1>());
  cudaFuncSetAttribute(tc_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<3>());
  cudaFuncSetAttribute(potrf_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPotrfInvSmem);
  ready_ = true;
}

template <int SPLIT>
static void gemm_launch(int ntask, const DevPlan &dp, const Task *tasks, const CUtensorMap *maps,
                        const CUtensorMap *inv_map, float *L, float *U, int32_t *status,
                        cudaStream_t st) {
  note_launch();
  tc_gemm_kernel<SPLIT><<<ntask, 192, smem_bytes<SPLIT>(), st>>>(dp, tasks, maps, inv_map, L, U,
                                                                 TcPlan::kNb, status);
}

void TcPlan::factor(const DevPlan &dp, const Plan &plan, const double *kval, float *L, float *U,
                    int32_t *status, int split, cudaStream_t st) {
  auto gemm = split == 3 ? gemm_launch<3> : gemm_launch<1>;
  const CUtensorMap *maps = static_cast<const CUtensorMap *>(d_maps_);
  const CUtensorMap *inv_map = maps + nfronts_;
  for (size_t li = 0; li < levels_.size(); li++) {
    launch_build_level<float>(dp, plan.levels[li], kval, L, U, st);
    for (const Step &s : levels_[li].steps) {
      if (s.gemm_e > s.gemm_b)
        gemm(s.gemm_e - s.gemm_b, dp, d_gemm_ + s.gemm_b, maps, inv_map, L, U, status, st);
      if (s.potrf_e > s.potrf_b)
        { note_launch(); potrf_inv_kernel<<<s.potrf_e - s.potrf_b, 256, kPotrfInvSmem, st>>>(dp, d_potrf_ + s.potrf_b, L, d_inv_, status); }
      if (s.trsm_e > s.trsm_b)
        gemm(s.trsm_e - s.trsm_b, dp, d_trsm_ + s.trsm_b, maps, inv_map, L, U, status, st);
    }
    const Level &lv = levels_[li];
    if (lv.syrk_e > lv.syrk_b)
      gemm(lv.syrk_e - lv.syrk_b, dp, d_syrk_ + lv.syrk_b, maps, inv_map, L, U, status, st);
  }
}

}  // namespace gipm
