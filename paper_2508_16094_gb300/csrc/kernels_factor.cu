// Assembly of the primal condensed matrix (Eq. 5) and the level-scheduled
// multifrontal supernodal Cholesky (Sec. 2: pivoting-free factorisation with
// elimination-tree parallelism), SIMT FMA path for FP64 and FP32.
//
// Per level of the supernodal tree: build every frontal matrix of the level
// (gather of the children's update matrices, each entry written once), add the
// K entries owned by the level, then factor the fronts' panels block column by
// block column (left-looking GEMM update, Cholesky of the diagonal block,
// triangular solve of the rows below) and form their update matrices
// U = F22 - L21 L21^T (SYRK). No atomics on values: results are bit-reproducible.
#include <cfloat>
#include <climits>

#include "launch.h"

namespace gipm {

namespace {

__global__ void assemble_kernel(DevPlan dp, const double *__restrict__ jv,
                                const double *__restrict__ D, const double *__restrict__ wv,
                                double delta_p, double *__restrict__ kval) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < dp.nk;
       q += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    const int64_t p1 = dp.k_poff[q + 1];
    for (int64_t p = dp.k_poff[q]; p < p1; p++) {
      const int32_t a = dp.k_pa[p], b = dp.k_pb[p];
      v = fma(jv[a] * D[dp.jrow[a]], jv[b], v);
    }
    const int64_t w = dp.k_w[q];
    if (w >= 0 && wv) v += wv[w];
    const int32_t i = dp.k_diag[q];
    if (i >= 0) {
      double d = delta_p;
      if (dp.lpos[i] >= 0) d += D[dp.lpos[i]];
      if (dp.upos[i] >= 0) d += D[dp.upos[i]];
      v += d;
    }
    kval[q] = v;
  }
}

// Four consecutive entries at a 16-byte aligned address.
__device__ __forceinline__ void store4(float *p, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double *p, double a, double b, double c, double d) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}

// Front assembly: one tile of 64 rows x (at most) 64 columns of a front's
// lower triangle per block of 128 threads; thread (row group g, column group
// q) owns rows r0 + g + 8i (i < 8) and columns c0 + 4q .. c0 + 4q + 3. Each
// entry is the sum, over the children in ascending order, of the matching
// entry of the child's update matrix (through the child->front inverse map).
// The maps of up to four children are staged together (one memory round
// trip), and a child none of whose rows or none of whose columns fall in the
// tile is skipped by the whole block. Panel tiles start at multiples of 64
// columns and update-matrix tiles at ncol + multiples of 64, so every
// 4-column group is one aligned vector store (entries above the diagonal and
// padding past ncol or nf are written as zeros). 32 entries per thread keep
// enough bytes in flight per block for the chain of dependent loads
// (task, front, children, maps) a tile starts with.
constexpr int kBuildThreads = 128, kBuildGroup = 4;
template <typename T>
__global__ void __launch_bounds__(kBuildThreads) build_front_kernel(DevPlan dp, int32_t task0,
                                                                    T *__restrict__ L,
                                                                    T *__restrict__ U) {
  constexpr int BT = kBuildTile, RS = kBuildThreads / (BT / 4), NR = BT / RS;  // 8 row groups, 8 rows each
  const Task tk = dp.build[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow;
  const int r0 = tk.a, c0 = tk.b, w = tk.c;
  __shared__ __align__(16) int32_t map[kBuildGroup][2 * BT];  // row maps, then column maps
  __shared__ int32_t hit[kBuildGroup][2 * BT / 32];  // per 32 maps: some entry maps into the child
  __shared__ int64_t uoff[kBuildGroup];
  __shared__ int32_t uld[kBuildGroup];
  const int tid = threadIdx.x, lane = tid % 32, g = tid / (BT / 4), q4 = 4 * (tid % (BT / 4));
  T acc[NR][4];
#pragma unroll
  for (int i = 0; i < NR; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = T(0);
  for (int cg = F.child_begin; cg < F.child_end; cg += kBuildGroup) {
    const int nc = min(kBuildGroup, F.child_end - cg);
    __syncthreads();
    // a warp's 32 entries are half of one child's row maps or column maps
    for (int e = tid; e < nc * 2 * BT; e += kBuildThreads) {
      const int q = e / (2 * BT), m = e % (2 * BT);
      const FrontInfo C = dp.fronts[dp.children[cg + q]];
      const int idx = m < BT ? r0 + m : c0 + m - BT;
      const bool inside = m < BT ? idx < nf : m - BT < w;
      const int32_t t = inside ? dp.inv[C.inv_off + idx] : -1;
      map[q][m] = t;
      const unsigned any = __ballot_sync(0xffffffffu, t >= 0);
      if (lane == 0) hit[q][m / 32] = any != 0u;
      if (m == 0) {
        uoff[q] = C.uoff;
        uld[q] = C.uld;
      }
    }
    __syncthreads();
    for (int q = 0; q < nc; q++) {
      if (!(hit[q][0] | hit[q][1]) || !(hit[q][2] | hit[q][3])) continue;
      const int4 b = *reinterpret_cast<const int4 *>(&map[q][BT + q4]);
      const int bb[4] = {b.x, b.y, b.z, b.w};
      const T *Uc = U + uoff[q];
      const int64_t ldq = uld[q];
#pragma unroll
      for (int i = 0; i < NR; i++) {
        const int rr = g + RS * i;
        const int a = map[q][rr];
        const T *row = Uc + a * ldq;
        T v[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
          v[j] = (a >= 0 && bb[j] >= 0 && r0 + rr >= c0 + q4 + j) ? row[bb[j]] : T(0);
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] += v[j];
      }
    }
  }
  if (q4 >= w) return;
  const int c = c0 + q4;
  const bool panel = c0 < F.ncol;
  const int lim = panel ? F.ncol : nf;  // columns past lim are padding
#pragma unroll
  for (int i = 0; i < NR; i++) {
    const int r = r0 + g + RS * i;
    if (r >= nf) continue;
    T o[4];
#pragma unroll
    for (int j = 0; j < 4; j++) o[j] = (c + j <= r && c + j < lim) ? acc[i][j] : T(0);
    T *dst = panel ? L + F.loff + (int64_t)r * F.ld + c
                   : U + F.uoff + (int64_t)(r - F.ncol) * F.uld + (c - F.ncol);
    if (panel || r >= F.ncol) store4(dst, o[0], o[1], o[2], o[3]);
  }
}

template <typename T>
__global__ void kadd_kernel(DevPlan dp, int64_t q0, int64_t q1, const double *__restrict__ kval,
                            T *__restrict__ L) {
  for (int64_t q = q0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < q1;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = dp.k_slot[q];
    L[s] = T((double)L[s] + kval[q]);
  }
}

// C[M x N] -= A[M x K] * S * B[N x K]^T for one 64x64 tile (rows of A and B
// are contiguous along K), 256 threads, 4x4 outputs per thread; S = diag(sk)
// holds the pivot signs of the K columns of a signed factorisation (sk ==
// nullptr: S = I).
template <typename T>
__device__ __forceinline__ void gemm_nt_tile(T *C, int64_t ldc, const T *A, int64_t lda,
                                             const T *B, int64_t ldb, int M, int N, int K,
                                             const int8_t *sk) {
  constexpr int BK = 16;
  __shared__ T As[BK][kGemmTile + 4], Bs[BK][kGemmTile + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int e = tid + 256 * q, r = e / BK, kk = e % BK;
      As[kk][r] = (r < M && k0 + kk < K) ? A[(int64_t)r * lda + k0 + kk] : T(0);
      T bv = (r < N && k0 + kk < K) ? B[(int64_t)r * ldb + k0 + kk] : T(0);
      if (sk && k0 + kk < K && sk[k0 + kk] < 0) bv = -bv;
      Bs[kk][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int r = ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int c = tx + 16 * j;
      if (c < N) C[(int64_t)r * ldc + c] -= acc[i][j];
    }
  }
}

// Left-looking update of block column k of a panel: rows i0..i0+63 of
// F[:, k:k+kb] -= L[:, 0:k] * L[k:k+kb, 0:k]^T.
template <typename T>
__global__ void __launch_bounds__(256) gemm_ll_kernel(DevPlan dp, int32_t task0, int nb,
                                                      T *__restrict__ L) {
  const Task tk = dp.gemm[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow, i0 = tk.a, k = tk.b;
  const int kb = min(nb, F.ncol - k), M = min(kGemmTile, nf - i0);
  T *P = L + F.loff;
  gemm_nt_tile<T>(P + (int64_t)i0 * F.ld + k, F.ld, P + (int64_t)i0 * F.ld, F.ld,
                  P + (int64_t)k * F.ld, F.ld, M, kb, k, dp.sgn ? dp.sgn + F.first : nullptr);
}

// Update matrix U = F22 - L21 L21^T, one 64x64 lower tile per block.
template <typename T>
__global__ void __launch_bounds__(256) syrk_kernel(DevPlan dp, int32_t task0,
                                                   const T *__restrict__ L, T *__restrict__ U) {
  const Task tk = dp.syrk[task0 + blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int i0 = tk.a, j0 = tk.b;
  const int M = min(kGemmTile, F.nrow - i0), N = min(kGemmTile, F.nrow - j0);
  const T *P = L + F.loff + (int64_t)F.ncol * F.ld;
  gemm_nt_tile<T>(U + F.uoff + (int64_t)i0 * F.uld + j0, F.uld, P + (int64_t)i0 * F.ld, F.ld,
                  P + (int64_t)j0 * F.ld, F.ld, M, N, F.ncol, dp.sgn ? dp.sgn + F.first : nullptr);
}

template <typename T> __device__ __forceinline__ T big_pivot();
template <> __device__ __forceinline__ float big_pivot<float>() { return 1e30f; }
template <> __device__ __forceinline__ double big_pivot<double>() { return 1e64; }

// Cholesky of one diagonal block (kb <= nb <= 128) in shared memory. A pivot
// that is not positive is either reported (smallest failing column kept) or
// replaced by a large value (static pivoting) and counted. With pivot signs
// (dp.sgn, a quasi-definite matrix) the block is factored as L S L^T: the
// pivot d_j must have the sign s_j, L_jj = sqrt(s_j d_j), the column below is
// divided by s_j L_jj and the trailing update is -= L_ij s_j L_cj.
template <typename T>
__global__ void __launch_bounds__(256) potrf_kernel(DevPlan dp, const Task *__restrict__ tasks,
                                                    int nb, T *__restrict__ L, int32_t *status,
                                                    int perturb) {
  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int k = tk.a, kb = min(nb, F.ncol - k), ls = nb + 1;
  T *A = L + F.loff + (int64_t)k * F.ld + k;
  const int8_t *sg = dp.sgn ? dp.sgn + F.first + k : nullptr;
  extern __shared__ unsigned char smem_raw[];
  T *Ad = reinterpret_cast<T *>(smem_raw);  // [nb][nb + 1]
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    if (r >= c) Ad[r * ls + c] = A[(int64_t)r * F.ld + c];
  }
  __syncthreads();
  // FP64 Cholesky (no signs): the column below the pivot is multiplied by one
  // reciprocal instead of divided entry by entry (an FP64 division is a long
  // sequence on the FP64 pipe); FP32 and signed factors keep the division.
  const bool recip = sizeof(T) == 8 && !sg;
  __shared__ T rl;  // 1 / (s_j L_jj) of the current column
  const int tx = tid % 16, ty = tid / 16;  // 16 x 16 grid over the trailing block
  for (int j = 0; j < kb; j++) {
    const T sj = (sg && sg[j] < 0) ? T(-1) : T(1);
    if (tid == 0) {
      T d = sj * Ad[j * ls + j];
      if (!(d > T(0)) || !(d < big_pivot<T>() * big_pivot<T>())) {
        if (perturb) {
          d = big_pivot<T>();
          atomicAdd(&status[ST_PERTURBED], 1);
        } else {
          atomicMin(&status[ST_FAIL_COL], F.first + k + j);
          d = T(1);
        }
      }
      const T l = sqrt(d);
      Ad[j * ls + j] = l;
      if (recip) rl = T(1) / l;
    }
    __syncthreads();
    if (recip) {
      const T r = rl;
      for (int i = j + 1 + tid; i < kb; i += blockDim.x) Ad[i * ls + j] *= r;
    } else {
      const T ljj = sj * Ad[j * ls + j];
      for (int i = j + 1 + tid; i < kb; i += blockDim.x) Ad[i * ls + j] /= ljj;
    }
    __syncthreads();
    for (int i = j + 1 + ty; i < kb; i += 16) {
      const T lij = -sj * Ad[i * ls + j];
      for (int c = j + 1 + tx; c <= i; c += 16) Ad[i * ls + c] = fma(lij, Ad[c * ls + j], Ad[i * ls + c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    if (r >= c) A[(int64_t)r * F.ld + c] = Ad[r * ls + c];
  }
}

// Rows below the diagonal block: X <- X L_kk^{-T} (row-wise forward
// substitution), kTrsmRows rows per block, kb <= nb <= 128; with pivot signs
// X <- X L_kk^{-T} S_k.
template <typename T>
__global__ void __launch_bounds__(kTrsmRows) trsm_kernel(DevPlan dp, const Task *__restrict__ tasks,
                                                         int nb, T *__restrict__ L) {
  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow, i0 = tk.a, k = tk.b, ls = nb + 1;
  const int kb = min(nb, F.ncol - k), rows = min(kTrsmRows, nf - i0);
  extern __shared__ unsigned char smem_raw[];
  T *Lk = reinterpret_cast<T *>(smem_raw);  // [nb][nb + 1]
  T *X = Lk + nb * ls;                      // [kTrsmRows][nb + 1]
  const T *A = L + F.loff + (int64_t)k * F.ld + k;
  T *Xg = L + F.loff + (int64_t)i0 * F.ld + k;
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    Lk[r * ls + c] = (r >= c) ? A[(int64_t)r * F.ld + c] : T(0);
  }
  for (int e = tid; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    X[r * ls + c] = Xg[(int64_t)r * F.ld + c];
  }
  const int8_t *sg = dp.sgn ? dp.sgn + F.first + k : nullptr;
  // FP64 without signs: the diagonal replaced by its reciprocal (no FP64
  // division on the substitution's critical path); otherwise s_c L_cc, the
  // signs also folded into the entries below the diagonal (s_c2 L_c,c2)
  const bool recip = sizeof(T) == 8 && !sg;
  __syncthreads();
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    if (r == c) {
      const T d = (sg && sg[c] < 0) ? -Lk[r * ls + c] : Lk[r * ls + c];
      Lk[r * ls + c] = recip ? T(1) / d : d;
    } else if (r > c && sg && sg[c] < 0) {
      Lk[r * ls + c] = -Lk[r * ls + c];
    }
  }
  __syncthreads();
  if (tid < rows) {  // column by column: the updates of one step are independent
    T *x = X + tid * ls;
    for (int c = 0; c < kb; c++) {
      const T xc = recip ? x[c] * Lk[c * ls + c] : x[c] / Lk[c * ls + c];
      x[c] = xc;
      for (int c2 = c + 1; c2 < kb; c2++) x[c2] = fma(-xc, Lk[c2 * ls + c], x[c2]);
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    Xg[(int64_t)r * F.ld + c] = X[r * ls + c];
  }
}

// FP64 rows below a diagonal block without pivot signs: X <- X L_kk^{-T}. A
// full 64-wide block keeps each thread's row in registers (64 values) and
// reads the block by broadcast from shared memory, its diagonal replaced by
// reciprocals; the 2080 multiply-adds of a row then issue back to back on the
// FP64 pipe. A narrower last block takes the shared-memory loop of trsm_kernel.
// Same arithmetic, in the same order, as trsm_kernel<double> on such a block.
__global__ void __launch_bounds__(kTrsmRows) trsm_f64_kernel(DevPlan dp, const Task *__restrict__ tasks,
                                                             double *__restrict__ L) {
  constexpr int NB = 64, LS = NB + 1;
  const Task tk = tasks[blockIdx.x];
  const FrontInfo F = dp.fronts[tk.front];
  const int nf = F.ncol + F.nrow, i0 = tk.a, k = tk.b;
  const int kb = min(NB, F.ncol - k), rows = min(kTrsmRows, nf - i0);
  extern __shared__ unsigned char smem_raw[];
  double *Lk = reinterpret_cast<double *>(smem_raw);  // [NB][LS]
  double *X = Lk + NB * LS;                           // [kTrsmRows][LS]
  const double *A = L + F.loff + (int64_t)k * F.ld + k;
  double *Xg = L + F.loff + (int64_t)i0 * F.ld + k;
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    const double v = A[(int64_t)r * F.ld + c];
    Lk[r * LS + c] = r > c ? v : (r == c ? 1.0 / v : 0.0);
  }
  for (int e = tid; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    X[r * LS + c] = Xg[(int64_t)r * F.ld + c];
  }
  __syncthreads();
  if (tid < rows) {
    double *xs = X + tid * LS;
    if (kb == NB) {
      double x[NB];
#pragma unroll
      for (int c = 0; c < NB; c++) x[c] = xs[c];
#pragma unroll
      for (int c = 0; c < NB; c++) {
        x[c] *= Lk[c * LS + c];
#pragma unroll
        for (int c2 = c + 1; c2 < NB; c2++) x[c2] = fma(-x[c], Lk[c2 * LS + c], x[c2]);
      }
#pragma unroll
      for (int c = 0; c < NB; c++) xs[c] = x[c];
    } else {
      for (int c = 0; c < kb; c++) {
        const double xc = xs[c] * Lk[c * LS + c];
        xs[c] = xc;
        for (int c2 = c + 1; c2 < kb; c2++) xs[c2] = fma(-xc, Lk[c2 * LS + c], xs[c2]);
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * kb; e += blockDim.x) {
    const int r = e / kb, c = e % kb;
    Xg[(int64_t)r * F.ld + c] = X[r * LS + c];
  }
}

template <typename T>
__global__ void entries_kernel(DevPlan dp, const T *__restrict__ L, const int32_t *col2s,
                               int64_t count, const int32_t *rows, const int32_t *cols,
                               double *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = rows[e], j = cols[e];
    double v = 0.0;
    if (i >= j && j >= 0 && i < dp.n) {
      const FrontInfo F = dp.fronts[col2s[j]];
      int32_t p = -1;
      if (i < F.first + F.ncol) {
        p = i - F.first;
      } else {
        int lo = 0, hi = F.nrow;  // binary search in the row structure
        const int32_t *rs = dp.sri + F.rows_off;
        while (lo < hi) {
          int mid = (lo + hi) / 2;
          if (rs[mid] < i) lo = mid + 1; else hi = mid;
        }
        if (lo < F.nrow && rs[lo] == i) p = F.ncol + lo;
      }
      if (p >= 0) v = (double)L[F.loff + (int64_t)p * F.ld + (j - F.first)];
    }
    out[e] = v;
  }
}

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

void launch_assemble(const DevPlan &dp, const double *jv, const double *D, const double *wv,
                     double delta_p, double *kval, cudaStream_t st) {
  if (dp.nk == 0) return;
  { note_launch(); assemble_kernel<<<grid_for(dp.nk, 256), 256, 0, st>>>(dp, jv, D, wv, delta_p, kval); }
}

template <typename T>
void launch_build_level(const DevPlan &dp, const LevelPlan &LP, const double *kval, T *L, T *U,
                        cudaStream_t st) {
  if (LP.build_e > LP.build_b)
    { note_launch(); build_front_kernel<T><<<LP.build_e - LP.build_b, kBuildThreads, 0, st>>>(dp, LP.build_b, L, U); }
  if (LP.k_e > LP.k_b)
    { note_launch(); kadd_kernel<T><<<grid_for(LP.k_e - LP.k_b, 256), 256, 0, st>>>(dp, LP.k_b, LP.k_e, kval, L); }
}

template <typename T>
void launch_potrf(const DevPlan &dp, const Task *tasks, int ntasks, int nb, T *L, int32_t *status,
                  bool perturb, cudaStream_t st) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)nb * (nb + 1) * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(potrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { note_launch(); potrf_kernel<T><<<ntasks, 256, smem, st>>>(dp, tasks, nb, L, status, perturb ? 1 : 0); }
}

template <typename T>
void launch_trsm(const DevPlan &dp, const Task *tasks, int ntasks, int nb, T *L, cudaStream_t st) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)(nb + kTrsmRows) * (nb + 1) * sizeof(T);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { note_launch(); trsm_kernel<T><<<ntasks, kTrsmRows, smem, st>>>(dp, tasks, nb, L); }
}

void launch_trsm_f64(const DevPlan &dp, const Task *tasks, int ntasks, double *L, cudaStream_t st) {
  if (ntasks <= 0) return;
  const size_t smem = (size_t)(64 + kTrsmRows) * 65 * sizeof(double);
  cudaFuncSetAttribute(trsm_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { note_launch(); trsm_f64_kernel<<<ntasks, kTrsmRows, smem, st>>>(dp, tasks, L); }
}

template <typename T>
void launch_factor_simt(const DevPlan &dp, const Plan &plan, const double *kval, T *L, T *U,
                        int32_t *status, bool perturb, cudaStream_t st) {
  const int nb = plan.nb;
  for (const LevelPlan &LP : plan.levels) {
    launch_build_level<T>(dp, LP, kval, L, U, st);
    for (const StepRange &S : LP.steps) {
      if (S.gemm_e > S.gemm_b)
        { note_launch(); gemm_ll_kernel<T><<<S.gemm_e - S.gemm_b, 256, 0, st>>>(dp, S.gemm_b, nb, L); }
      launch_potrf<T>(dp, dp.potrf + S.potrf_b, S.potrf_e - S.potrf_b, nb, L, status, perturb, st);
      launch_trsm<T>(dp, dp.trsm + S.trsm_b, S.trsm_e - S.trsm_b, nb, L, st);
    }
    if (LP.syrk_e > LP.syrk_b)
      { note_launch(); syrk_kernel<T><<<LP.syrk_e - LP.syrk_b, 256, 0, st>>>(dp, LP.syrk_b, L, U); }
  }
}

template <typename T>
void launch_factor_entries(const DevPlan &dp, const T *L, const int32_t *col2s, int64_t count,
                           const int32_t *rows, const int32_t *cols, double *out,
                           cudaStream_t st) {
  if (count <= 0) return;
  { note_launch(); entries_kernel<T><<<grid_for(count, 256), 256, 0, st>>>(dp, L, col2s, count, rows, cols, out); }
}

template void launch_build_level<float>(const DevPlan &, const LevelPlan &, const double *,
                                        float *, float *, cudaStream_t);
template void launch_build_level<double>(const DevPlan &, const LevelPlan &, const double *,
                                         double *, double *, cudaStream_t);
template void launch_potrf<double>(const DevPlan &, const Task *, int, int, double *, int32_t *,
                                   bool, cudaStream_t);
template void launch_trsm<double>(const DevPlan &, const Task *, int, int, double *, cudaStream_t);
template void launch_potrf<float>(const DevPlan &, const Task *, int, int, float *, int32_t *, bool,
                                  cudaStream_t);
template void launch_trsm<float>(const DevPlan &, const Task *, int, int, float *, cudaStream_t);
template void launch_factor_simt<double>(const DevPlan &, const Plan &, const double *, double *,
                                         double *, int32_t *, bool, cudaStream_t);
template void launch_factor_simt<float>(const DevPlan &, const Plan &, const double *, float *,
                                        float *, int32_t *, bool, cudaStream_t);
template void launch_factor_entries<double>(const DevPlan &, const double *, const int32_t *,
                                            int64_t, const int32_t *, const int32_t *, double *,
                                            cudaStream_t);
template void launch_factor_entries<float>(const DevPlan &, const float *, const int32_t *,
                                           int64_t, const int32_t *, const int32_t *, double *,
                                           cudaStream_t);

}  // namespace gipm
