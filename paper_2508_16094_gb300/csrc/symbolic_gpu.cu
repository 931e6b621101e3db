// Symbolic analysis of many small patterns on the GPU (Sec. 6: batch solvers
// for many problems of one family; Sec. 2: the analysis itself is serial,
// computed once per pattern and reused).
//
// For a batch of constraint-Jacobian patterns J_b (m_b x n_b, CSR) with
// orderings P_b, each CTA analyses one pattern of K_b = J_b^T J_b + I:
//  - the elimination tree of P K P^T, straight from the rows of J (each row of
//    J is a clique of K; the previous column seen in a row links the columns
//    of that row, and ancestor links with path compression give the tree);
//  - its postorder (children ascending, roots ascending), which fixes the
//    final numbering;
//  - the column counts of L: the nonzeros of row i of L are the nodes of the
//    row subtree of i, the union over the rows r of J containing i of the
//    tree path from first(r) (the smallest final index in row r: every column
//    of r lies on that path) up to i, walked with per-row marks;
//  - the starts of the fundamental supernodes (j joins j - 1 when parent(j-1)
//    = j, j has that one child and count(j) = count(j-1) - 1).
// The tree and postorder are serial (thread 0); the row subtrees are walked by
// four warps. Results are the same bits as a host analysis of the same
// pattern: the tree, postorder and counts are unique.
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gb300_ipm.h"
#include "dev.cuh"

namespace gipm {
namespace {

constexpr int kSymThreads = 128, kWalkers = 4;

struct SymArgs {
  int32_t count;
  const int64_t *n_off, *m_off, *w_off;  // prefix sums (count + 1)
  const int64_t *rowptr;                 // pattern b: m_b + 1 offsets into col at m_off[b] + b
  const int32_t *col;
  const int32_t *perm;                   // new -> old per pattern, or nullptr
  int32_t *work;
  int32_t *post, *parent, *colcount, *sstart;
  int32_t *status;                       // [0]: first pattern with an invalid index, INT_MAX if none
};

// ints of workspace per pattern
__host__ __device__ inline int64_t sym_words(int64_t n, int64_t m, int64_t nnz) {
  return 13 * n + 2 + 2 * m + nnz + (int64_t)kWalkers * n;
}

__global__ void __launch_bounds__(kSymThreads) sym_batch_kernel(SymArgs A) {
  const int tid = threadIdx.x;
  for (int b = blockIdx.x; b < A.count; b += gridDim.x) {
    const int64_t n = A.n_off[b + 1] - A.n_off[b], m = A.m_off[b + 1] - A.m_off[b];
    const int64_t *rp = A.rowptr + A.m_off[b] + b;
    const int64_t base = rp[0], nnz = rp[m] - base;
    const int32_t *perm = A.perm ? A.perm + A.n_off[b] : nullptr;
    int32_t *w = A.work + A.w_off[b];
    int32_t *iperm = w, *colptr = iperm + n, *crow = colptr + n + 1, *prev = crow + nnz;
    int32_t *anc = prev + m, *par = anc + n, *head = par + n, *nxt = head + n, *stk = nxt + n;
    int32_t *post = stk + n, *ipost = post + n, *pfin = ipost + n, *first = pfin + n;
    int32_t *nchild = first + m, *marks = nchild + n;  // marks: kWalkers x n
    int32_t *out_post = A.post + A.n_off[b], *out_par = A.parent + A.n_off[b];
    int32_t *cc = A.colcount + A.n_off[b], *out_start = A.sstart + A.n_off[b];
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int64_t k = tid; k < n; k += kSymThreads) {
      iperm[k] = -1;
      colptr[k + 1] = 0;
      nchild[k] = 0;
      cc[k] = 0;
    }
    if (tid == 0) colptr[0] = 0;
    for (int64_t k = tid; k < kWalkers * n; k += kSymThreads) marks[k] = -1;
    for (int64_t r = tid; r < m; r += kSymThreads) prev[r] = -1;
    __syncthreads();
    // inverse ordering (an index outside [0, n) or a repeated one is an error)
    for (int64_t k = tid; k < n; k += kSymThreads) {
      const int32_t p = perm ? perm[k] : (int32_t)k;
      if (p < 0 || p >= n || atomicExch(&iperm[p], (int32_t)k) != -1) bad = 1;
    }
    for (int64_t e = tid; e < nnz; e += kSymThreads) {
      const int32_t c = A.col[base + e];
      if (c < 0 || c >= n) bad = 1;
    }
    __syncthreads();
    const int skip = bad;
    __syncthreads();  // every thread has read the flag before the next pattern resets it
    if (skip) {
      if (tid == 0) atomicMin(&A.status[0], b);
      continue;
    }
    // CSC of J by new column index (entry order within a column is free)
    for (int64_t e = tid; e < nnz; e += kSymThreads) atomicAdd(&colptr[iperm[A.col[base + e]] + 1], 1);
    __syncthreads();
    if (tid == 0)
      for (int64_t k = 0; k < n; k++) colptr[k + 1] += colptr[k];
    __syncthreads();
    for (int64_t k = tid; k < n; k += kSymThreads) head[k] = colptr[k];
    __syncthreads();
    for (int64_t r = tid; r < m; r += kSymThreads)
      for (int64_t e = rp[r]; e < rp[r + 1]; e++) {
        const int32_t j = iperm[A.col[e]];
        crow[atomicAdd(&head[j], 1)] = (int32_t)r;
      }
    __syncthreads();
    if (tid == 0) {
      // elimination tree of J^T J, column by column: every row r of column k
      // links its previously seen column prev[r] (and that column's root
      // path, compressed to point at k) under k
      for (int32_t k = 0; k < n; k++) {
        par[k] = -1;
        anc[k] = -1;
        for (int32_t p = colptr[k]; p < colptr[k + 1]; p++) {
          const int32_t r = crow[p];
          int32_t i = prev[r];
          while (i != -1 && i < k) {
            const int32_t inext = anc[i];
            anc[i] = k;
            if (inext == -1) par[i] = k;
            i = inext;
          }
          prev[r] = k;
        }
      }
      // postorder: children ascending (lists built from the back), roots ascending
      for (int32_t i = 0; i < n; i++) head[i] = -1;
      for (int32_t j = n - 1; j >= 0; j--)
        if (par[j] != -1) {
          nxt[j] = head[par[j]];
          head[par[j]] = j;
        }
      int32_t k = 0;
      for (int32_t r = 0; r < n; r++) {
        if (par[r] != -1) continue;
        int32_t top = 0;
        stk[0] = r;
        while (top >= 0) {
          const int32_t v = stk[top], ch = head[v];
          if (ch == -1) {
            post[k++] = v;
            top--;
          } else {
            head[v] = nxt[ch];
            stk[++top] = ch;
          }
        }
      }
    }
    __syncthreads();
    for (int64_t k = tid; k < n; k += kSymThreads) ipost[post[k]] = (int32_t)k;
    __syncthreads();
    for (int64_t k = tid; k < n; k += kSymThreads) {
      const int32_t v = post[k];
      pfin[k] = par[v] == -1 ? -1 : ipost[par[v]];
      out_par[k] = pfin[k];
      out_post[k] = perm ? perm[v] : v;
      if (pfin[k] >= 0) atomicAdd(&nchild[pfin[k]], 1);
    }
    // first column of every row of J in the final numbering
    for (int64_t r = tid; r < m; r += kSymThreads) {
      int32_t f = INT_MAX;
      for (int64_t e = rp[r]; e < rp[r + 1]; e++) f = min(f, ipost[iperm[A.col[e]]]);
      first[r] = f;
    }
    __syncthreads();
    // row subtrees: lane 0 of each warp walks rows i = warp, warp + 4, ...
    const int warp = tid / 32;
    if (tid % 32 == 0) {
      int32_t *mk = marks + (int64_t)warp * n;
      for (int32_t i = warp; i < n; i += kWalkers) {
        const int32_t jn = post[i];  // column of final index i before the postorder
        for (int32_t p = colptr[jn]; p < colptr[jn + 1]; p++) {
          int32_t v = first[crow[p]];
          while (v != -1 && v < i && mk[v] != i) {
            mk[v] = i;
            atomicAdd(&cc[v], 1);
            v = pfin[v];
          }
        }
      }
    }
    __syncthreads();
    for (int64_t j = tid; j < n; j += kSymThreads) cc[j] += 1;  // the diagonal
    __syncthreads();
    for (int64_t j = tid; j < n; j += kSymThreads)
      out_start[j] = (j == 0 || !(pfin[j - 1] == j && nchild[j] == 1 && cc[j] == cc[j - 1] - 1)) ? 1 : 0;
    __syncthreads();
  }
}

}  // namespace
}  // namespace gipm

using namespace gipm;

extern "C" {

ipm_status ipm_symbolic_batched_workspace(const ipm_pattern_batch *b, size_t *bytes) {
  if (!b || !bytes || b->count < 0 || (b->count > 0 && (!b->h_n || !b->h_m || !b->h_nnz)))
    return IPM_ERR_ARG;
  int64_t words = 0;
  for (int32_t i = 0; i < b->count; i++) {
    if (b->h_n[i] < 0 || b->h_m[i] < 0 || b->h_nnz[i] < 0) return IPM_ERR_ARG;
    words += sym_words(b->h_n[i], b->h_m[i], b->h_nnz[i]);
  }
  *bytes = (size_t)(3 * ((int64_t)b->count + 1)) * sizeof(int64_t) + 256 + (size_t)words * sizeof(int32_t) + 256;
  return IPM_OK;
}

ipm_status ipm_symbolic_batched(const ipm_pattern_batch *b, void *d_work, size_t bytes, void *stream,
                                int32_t *d_post, int32_t *d_parent, int32_t *d_colcount,
                                int32_t *d_sstart, int32_t *h_bad) {
  if (!b || !d_work || !d_post || !d_parent || !d_colcount || !d_sstart) return IPM_ERR_ARG;
  size_t need = 0;
  ipm_status st = ipm_symbolic_batched_workspace(b, &need);
  if (st != IPM_OK) return st;
  if (bytes < need || ((uintptr_t)d_work & 255) != 0) return IPM_ERR_NOMEM;
  if (b->count == 0) return IPM_OK;
  if (!b->d_rowptr || !b->d_col) return IPM_ERR_ARG;
  const int32_t cnt = b->count;
  std::vector<int64_t> offs(3 * ((size_t)cnt + 1), 0);
  int64_t *n_off = offs.data(), *m_off = n_off + cnt + 1, *w_off = m_off + cnt + 1;
  for (int32_t i = 0; i < cnt; i++) {
    n_off[i + 1] = n_off[i] + b->h_n[i];
    m_off[i + 1] = m_off[i] + b->h_m[i];
    w_off[i + 1] = w_off[i] + sym_words(b->h_n[i], b->h_m[i], b->h_nnz[i]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  char *base = (char *)d_work;
  int64_t *d_offs = (int64_t *)base;
  int32_t *d_status = (int32_t *)(base + ((offs.size() * sizeof(int64_t) + 255) & ~size_t(255)));
  int32_t *d_words = d_status + 64;
  const int32_t init = INT_MAX;
  if (cudaMemcpyAsync(d_offs, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(d_status, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return IPM_ERR_CUDA;
  SymArgs A{cnt, d_offs, d_offs + cnt + 1, d_offs + 2 * ((int64_t)cnt + 1), b->d_rowptr, b->d_col,
            b->d_perm, d_words, d_post, d_parent, d_colcount, d_sstart, d_status};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min<int>(cnt, std::max(1, sms) * 8);
  note_launch();
  sym_batch_kernel<<<grid, kSymThreads, 0, s>>>(A);
  int32_t badv = INT_MAX;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&badv, d_status, sizeof(badv), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return IPM_ERR_CUDA;
  if (h_bad) *h_bad = badv == INT_MAX ? -1 : badv;
  return badv == INT_MAX ? IPM_OK : IPM_ERR_ARG;
}

}  // extern "C"
