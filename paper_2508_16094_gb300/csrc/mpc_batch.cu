// Batched interior-point solver for thousands of small MPC QPs in one
// persistent launch (Sec. 6, batch solvers; the same pivoting-free method as
// the sparse path: KKT conditions (2), Newton system (3) condensed to (5)).
//
// Instance: z = (u_0, x_1, u_1, x_2, ...), stage k owns z_k = (u_k, x_{k+1})
// (16 variables). Constraints g(z) >= 0 per stage: the dynamics as the pair
// h_k >= 0, -h_k >= 0 with h_k = x_{k+1} - A_k x_k - B_k u_k (x_0 given), and
// the box bounds on u_k and x_{k+1}. The condensed matrix K = W + J^T D J +
// delta_p I is block tridiagonal with 16 x 16 blocks; it is factored by a
// sequential block Cholesky over the stages.
//
// Execution: 16 lanes (half a warp) per instance; lane i holds row i of every
// 16 x 16 block and the rows of g tied to variable i of the stage (dynamics row
// i for i < 12, lower and upper bound of variable i). Rows of L blocks move
// between lanes with width-16 shuffles. Instances come from an atomic queue
// ordered by horizon (longest first) so a persistent grid stays balanced.
// The FP32 variant assembles, factors and solves in FP32 and refines in FP64
// on a residual evaluated matrix-free from A, B and D (J v, scaled by D, J^T),
// so the FP64 pipe only carries the refinement.
#include <cfloat>
#include <cmath>
#include <stdexcept>

#include "mpc_batch.h"

namespace gipm {

namespace {

constexpr int NX = 12, NU = 4, NS = 16, NSLOT = 64;  // row slots per stage: 4 kinds x 16 lanes
constexpr int KIND_DP = 0, KIND_DM = 1, KIND_LO = 2, KIND_HI = 3;

struct Group {
  unsigned mask;
  int lane;
};

__device__ __forceinline__ double sum16(const Group &G, double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(G.mask, v, o, 16);
  return v;
}
__device__ __forceinline__ double max16(const Group &G, double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(G.mask, v, o, 16));
  return v;
}
__device__ __forceinline__ double min16(const Group &G, double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(G.mask, v, o, 16));
  return v;
}
template <typename T>
__device__ __forceinline__ T bcast(const Group &G, T v, int src) {
  return __shfl_sync(G.mask, v, src, 16);
}

__device__ __forceinline__ bool row_valid(int kind, int lane) {
  return kind >= KIND_LO || lane < NX;
}

// Per-instance views into the batch arrays and the workspace.
template <typename TF>
struct Inst {
  int T;
  const double *A, *B, *Q, *R, *x0;
  double *z, *dz, *rhs, *tv, *corr, *res;  // 16 per stage
  double *s, *lam, *D, *g, *w, *ds, *dl;   // NSLOT per stage
  double *il;                              // NSLOT per stage: 1 / lambda of the iteration
  double *Kd, *Ko;                         // 256 per stage (row-major)
  TF *Kf, *Kof;                            // the same storage as K blocks of type TF
  TF *Ld, *Lo;                             // 256 per stage (row-major; Ld keeps 1 / L_ii on its diagonal)
};

template <typename TF>
__device__ Inst<TF> make_inst(const MpcArgs &a, int inst) {
  Inst<TF> I;
  const int64_t s0 = a.soff[inst];
  I.T = a.T[inst];
  I.A = a.A + s0 * NX * NX;
  I.B = a.B + s0 * NX * NU;
  I.Q = a.Q + (int64_t)inst * NX;
  I.R = a.R + (int64_t)inst * NU;
  I.x0 = a.x0 + (int64_t)inst * NX;
  double *base = a.work + s0 * kMpcStageDoubles;
  const int64_t T = I.T;
  I.z = base;
  I.dz = I.z + T * NS;
  I.rhs = I.dz + T * NS;
  I.tv = I.rhs + T * NS;
  I.corr = I.tv + T * NS;
  I.res = I.corr + T * NS;
  I.s = I.res + T * NS;
  I.lam = I.s + T * NSLOT;
  I.D = I.lam + T * NSLOT;
  I.g = I.D + T * NSLOT;
  I.w = I.g + T * NSLOT;
  I.ds = I.w + T * NSLOT;
  I.dl = I.ds + T * NSLOT;
  I.il = I.dl + T * NSLOT;
  I.Kd = I.il + T * NSLOT;
  I.Ko = I.Kd + T * 256;
  I.Kf = reinterpret_cast<TF *>(I.Kd);
  I.Kof = reinterpret_cast<TF *>(I.Ko);
  I.Ld = reinterpret_cast<TF *>(I.Ko + T * 256);
  I.Lo = I.Ld + T * 256;
  return I;
}

__device__ __forceinline__ double wdiag(const double *Q, const double *R, int i) {
  return i < NU ? R[i] : Q[i - NU];
}

// x_k entry j (j < 12) of a stage vector family v (z or dz): x_0 is data (zero
// for a direction), x_k for k >= 1 is the x-part of stage k-1.
__device__ __forceinline__ double xprev(const double *v, const double *x0, int k, int j) {
  return k == 0 ? (x0 ? x0[j] : 0.0) : v[(k - 1) * NS + NU + j];
}

// out[slot] = J v (linear part) for every valid row; with x0 != nullptr and
// lb/ub the constant parts of g are included (out = g(v)).
template <typename TF>
__device__ __noinline__ void eval_rows(const Group &G, const Inst<TF> &I, const double *v, const double *x0,
                          double umax, double xmax, double *out, bool constant) {
  const int i = G.lane;
  for (int k = 0; k < I.T; k++) {
    const double *vk = v + k * NS;
    if (i < NX) {
      const double *Ar = I.A + (int64_t)k * NX * NX + i * NX;
      const double *Br = I.B + (int64_t)k * NX * NU + i * NU;
      double h = vk[NU + i];
      for (int j = 0; j < NX; j++) h -= Ar[j] * xprev(v, constant ? x0 : nullptr, k, j);
      for (int j = 0; j < NU; j++) h -= Br[j] * vk[j];
      out[k * NSLOT + KIND_DP * 16 + i] = h;
      out[k * NSLOT + KIND_DM * 16 + i] = -h;
    }
    const double lim = i < NU ? umax : xmax;
    out[k * NSLOT + KIND_LO * 16 + i] = vk[i] + (constant ? lim : 0.0);
    out[k * NSLOT + KIND_HI * 16 + i] = (constant ? lim : 0.0) - vk[i];
  }
}

// out (16 per stage) = base + sgn * J^T rowv + (W z if z)
template <typename TF>
__device__ __noinline__ void jt_rows(const Group &G, const Inst<TF> &I, const double *rowv, double sgn,
                        const double *z, const double *base, double *out) {
  const int i = G.lane;
  for (int k = 0; k < I.T; k++) {
    const double *rk = rowv + k * NSLOT;
    double a = rk[KIND_LO * 16 + i] - rk[KIND_HI * 16 + i];
    if (i < NU) {
      const double *Bk = I.B + (int64_t)k * NX * NU;
      for (int r = 0; r < NX; r++) a -= Bk[r * NU + i] * (rk[r] - rk[16 + r]);
    } else {
      const int xi = i - NU;
      a += rk[xi] - rk[16 + xi];
      if (k + 1 < I.T) {
        const double *A1 = I.A + (int64_t)(k + 1) * NX * NX;
        const double *r1 = rowv + (k + 1) * NSLOT;
        for (int r = 0; r < NX; r++) a -= A1[r * NX + xi] * (r1[r] - r1[16 + r]);
      }
    }
    a *= sgn;
    if (base) a += base[k * NS + i];
    if (z) a += wdiag(I.Q, I.R, i) * z[k * NS + i];
    out[k * NS + i] = a;
  }
}

// K = W + J^T D J + diag(bounds) + delta_p I as diagonal (Kf) and sub-diagonal
// (Kof) blocks, computed and stored in the arithmetic TF.
template <typename TF>
__device__ __noinline__ void assemble(const Group &G, const Inst<TF> &I, double delta_p) {
  const int i = G.lane;
  for (int k = 0; k < I.T; k++) {
    const double *Dk = I.D + k * NSLOT;
    const double *Bk = I.B + (int64_t)k * NX * NU;
    const double *Ak = I.A + (int64_t)k * NX * NX;
    TF *kd = I.Kf + (int64_t)k * 256 + i * NS;
    TF dsum[NX];  // D of the dynamics pair of each row of stage k
    for (int r = 0; r < NX; r++) dsum[r] = TF(Dk[r] + Dk[16 + r]);
    for (int c = 0; c < NS; c++) {
      TF v = TF(0);
      if (i < NU && c < NU) {
        for (int r = 0; r < NX; r++) v += TF(Bk[r * NU + i]) * dsum[r] * TF(Bk[r * NU + c]);
      } else if (i < NU) {
        v = -TF(Bk[(c - NU) * NU + i]) * dsum[c - NU];
      } else if (c < NU) {
        v = -dsum[i - NU] * TF(Bk[(i - NU) * NU + c]);
      } else if (i == c) {
        v = dsum[i - NU];
      }
      if (i >= NU && c >= NU && k + 1 < I.T) {
        const double *A1 = I.A + (int64_t)(k + 1) * NX * NX;
        const double *D1 = I.D + (k + 1) * NSLOT;
        for (int r = 0; r < NX; r++)
          v += TF(A1[r * NX + i - NU]) * TF(D1[r] + D1[16 + r]) * TF(A1[r * NX + c - NU]);
      }
      if (i == c) v += TF(wdiag(I.Q, I.R, i) + delta_p + Dk[32 + i] + Dk[48 + i]);
      kd[c] = v;
    }
    if (k > 0) {
      TF *ko = I.Kof + (int64_t)k * 256 + i * NS;
      for (int c = 0; c < NS; c++) {
        TF v = TF(0);
        if (c >= NU) {
          if (i < NU) {
            for (int r = 0; r < NX; r++) v += TF(Bk[r * NU + i]) * dsum[r] * TF(Ak[r * NX + c - NU]);
          } else {
            v = -dsum[i - NU] * TF(Ak[(i - NU) * NX + c - NU]);
          }
        }
        ko[c] = v;
      }
    }
  }
}

template <typename TF> __device__ __forceinline__ TF big_piv();
template <> __device__ __forceinline__ float big_piv<float>() { return 1e30f; }
template <> __device__ __forceinline__ double big_piv<double>() { return 1e64; }

// Block Cholesky of the block-tridiagonal K. Returns false on a non-positive
// pivot in FP64 (caller raises delta_p); FP32 replaces such pivots.
template <typename TF>
__device__ __noinline__ bool factor(const Group &G, const Inst<TF> &I, int &perturbed) {
  const int i = G.lane;
  TF lo[NS];  // row i of L_{k,k-1}
#pragma unroll
  for (int c = 0; c < NS; c++) lo[c] = TF(0);
  bool ok = true;
  for (int k = 0; k < I.T; k++) {
    TF srow[NS];
    const TF *kd = I.Kf + (int64_t)k * 256 + i * NS;
#pragma unroll
    for (int c = 0; c < NS; c++) srow[c] = TF(kd[c]);
    if (k > 0) {  // S = Kd - Lo Lo^T
#pragma unroll
      for (int c = 0; c < NS; c++) {
        TF acc = TF(0);
#pragma unroll
        for (int m = 0; m < NS; m++) acc += lo[m] * bcast(G, lo[m], c);
        srow[c] -= acc;
      }
    }
    // Cholesky of S, rows in registers; lane i keeps 1 / L_ii (rdg)
    TF rdg = TF(0);
#pragma unroll
    for (int j = 0; j < NS; j++) {
      TF piv = bcast(G, srow[j], j);
      if (!(piv > TF(0)) || !(piv < big_piv<TF>())) {
        if (sizeof(TF) == 8) ok = false;
        else perturbed++;
        piv = sizeof(TF) == 8 ? TF(1) : big_piv<TF>();
      }
      const TF ljj = sqrt(piv), rjj = TF(1) / ljj;
      if (i == j) {
        srow[j] = ljj;
        rdg = rjj;
      }
      if (i > j) srow[j] *= rjj;
      const TF lij = srow[j];
#pragma unroll
      for (int c = j + 1; c < NS; c++) {
        const TF lcj = bcast(G, lij, c);
        if (i >= c) srow[c] -= lij * lcj;
      }
    }
    TF *ld = I.Ld + (int64_t)k * 256 + i * NS;
#pragma unroll
    for (int c = 0; c < NS; c++) ld[c] = c < i ? srow[c] : (c == i ? rdg : TF(0));  // diagonal: 1 / L_ii
    if (k + 1 < I.T) {  // L_{k+1,k} = Ko_{k+1} L_kk^{-T}: row i by forward substitution
      const TF *ko = I.Kof + (int64_t)(k + 1) * 256 + i * NS;
      TF x[NS];
#pragma unroll
      for (int c = 0; c < NS; c++) {
        TF v = TF(ko[c]);
#pragma unroll
        for (int m = 0; m < c; m++) v -= x[m] * bcast(G, srow[m], c);
        x[c] = v * bcast(G, rdg, c);
      }
      TF *lop = I.Lo + (int64_t)(k + 1) * 256 + i * NS;
#pragma unroll
      for (int c = 0; c < NS; c++) {
        lo[c] = x[c];
        lop[c] = x[c];
      }
    }
  }
  return ok;
}

// out = K^{-1} in via the block factor (arithmetic in TF); work: 16 per stage.
template <typename TF>
__device__ __noinline__ void block_solve(const Group &G, const Inst<TF> &I, const double *in, double *out,
                            double *work) {
  const int i = G.lane;
  TF yprev = TF(0);
  for (int k = 0; k < I.T; k++) {  // forward: y_k = L_kk^{-1}(r_k - L_{k,k-1} y_{k-1})
    TF t = TF(in[k * NS + i]);
    if (k > 0) {
      const TF *lo = I.Lo + (int64_t)k * 256 + i * NS;
#pragma unroll
      for (int m = 0; m < NS; m++) t -= lo[m] * bcast(G, yprev, m);
    }
    const TF *ld = I.Ld + (int64_t)k * 256 + i * NS;
    TF lrow[NS];
#pragma unroll
    for (int m = 0; m < NS; m++) lrow[m] = ld[m];
    TF y = TF(0);
#pragma unroll
    for (int j = 0; j < NS; j++) {
      const TF yj = bcast(G, t * lrow[j], j);  // lane j: t_j / L_jj (the diagonal holds 1 / L_jj)
      if (i == j) y = yj;
      if (i > j) t -= lrow[j] * yj;
    }
    work[k * NS + i] = (double)y;
    yprev = y;
  }
  TF xnext = TF(0);
  for (int k = I.T - 1; k >= 0; k--) {  // backward: x_k = L_kk^{-T}(y_k - L_{k+1,k}^T x_{k+1})
    TF t = TF(work[k * NS + i]);
    if (k + 1 < I.T) {
      const TF *lo = I.Lo + (int64_t)(k + 1) * 256;
#pragma unroll
      for (int m = 0; m < NS; m++) t -= lo[m * NS + i] * bcast(G, xnext, m);
    }
    const TF *ld = I.Ld + (int64_t)k * 256;
    TF lcol[NS];
#pragma unroll
    for (int m = 0; m < NS; m++) lcol[m] = ld[m * NS + i];
    TF x = TF(0);
#pragma unroll
    for (int j = NS - 1; j >= 0; j--) {
      const TF xj = bcast(G, t * lcol[j], j);  // lane j: t_j / L_jj (the diagonal holds 1 / L_jj)
      if (i == j) x = xj;
      if (i < j) t -= lcol[j] * xj;
    }
    out[k * NS + i] = (double)x;
    xnext = x;
  }
}

// res = in - K v in FP64, matrix-free: K v = W v + J^T D J v + delta_p v over
// every row of g (dynamics pairs and bounds). rows: NSLOT per stage of scratch.
__device__ __noinline__ void kresid(const Group &G, const Inst<double> &I, const double *in, const double *v,
                       double *res, double *rows, double delta_p) {
  const int i = G.lane;
  eval_rows<double>(G, I, v, nullptr, 0.0, 0.0, rows, false);  // J v
  for (int k = 0; k < I.T; k++)
    for (int kind = 0; kind < 4; kind++) {
      const int q = k * NSLOT + kind * 16 + i;
      rows[q] = row_valid(kind, i) ? I.D[q] * rows[q] : 0.0;
    }
  __syncwarp(G.mask);
  jt_rows<double>(G, I, rows, 1.0, v, nullptr, res);  // J^T D J v + W v
  for (int k = 0; k < I.T; k++) {
    const int q = k * NS + i;
    res[q] = in[q] - res[q] - delta_p * v[q];
  }
}

// Views of one instance's workspace as FP64 and FP32 factor storage.
struct Views {
  Inst<double> d;
  Inst<float> f;
};

__device__ bool kfactor(const Group &G, const Views &V, bool f32, int &perturbed) {
  return f32 ? factor<float>(G, V.f, perturbed) : factor<double>(G, V.d, perturbed);
}

// Solve K out = in. FP64 factor: one block solve. FP32 factor: block solve plus
// FP64 refinement on the residual in - K out; returns false when that does not
// reach 1e-8 relative (the caller then refactors this instance in FP64).
__device__ bool ksolve(const Group &G, const Views &V, bool f32, const double *in, double *out,
                       double delta_p) {
  const Inst<double> &I = V.d;
  const int i = G.lane;
  if (!f32) {
    block_solve<double>(G, I, in, out, I.tv);
    __syncwarp(G.mask);
    return true;
  }
  block_solve<float>(G, V.f, in, out, I.tv);
  double bn = 0.0;
  for (int k = 0; k < I.T; k++) bn = fmax(bn, fabs(in[k * NS + i]));
  bn = max16(G, bn);
  double rn = 0.0;
  for (int step = 0; step < 4; step++) {
    __syncwarp(G.mask);
    kresid(G, I, in, out, I.res, I.dl, delta_p);  // dl is free during a solve
    __syncwarp(G.mask);
    rn = 0.0;
    for (int k = 0; k < I.T; k++) {
      const double r = fabs(I.res[k * NS + i]);
      rn = (r > rn || r != r) ? r : rn;  // NaN propagates
    }
    for (int o = 8; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(G.mask, rn, o, 16);
      rn = (other > rn || other != other) ? other : rn;
    }
    if (rn <= 1e-10 * bn) break;
    if (!(rn == rn) || step == 3) break;
    block_solve<float>(G, V.f, I.res, I.corr, I.tv);
    for (int k = 0; k < I.T; k++) out[k * NS + i] += I.corr[k * NS + i];
  }
  __syncwarp(G.mask);
  return rn <= 1e-8 * bn;
}

// One Newton direction with complementarity target w (nullptr: zero); returns
// false when an FP32 solve missed its tolerance.
__device__ __noinline__ bool direction(const Group &G, const Views &V, const double *w, bool f32,
                          double delta_p) {
  const Inst<double> &I = V.d;
  const int i = G.lane;
  // row values D (g - w/lam) - lam, then rhs = -(W z + J^T(...))
  for (int k = 0; k < I.T; k++)
    for (int kind = 0; kind < 4; kind++) {
      const int q = k * NSLOT + kind * 16 + i;
      if (!row_valid(kind, i)) { I.ds[q] = 0.0; continue; }
      const double wl = w ? w[q] * I.il[q] : 0.0;
      I.ds[q] = I.D[q] * (I.g[q] - wl) - I.lam[q];
    }
  __syncwarp(G.mask);
  jt_rows<double>(G, I, I.ds, 1.0, I.z, nullptr, I.rhs);
  for (int k = 0; k < I.T; k++) I.rhs[k * NS + i] = -I.rhs[k * NS + i];
  __syncwarp(G.mask);
  const bool ok = __all_sync(G.mask, ksolve(G, V, f32, I.rhs, I.dz, delta_p));
  if (!ok) return false;
  eval_rows<double>(G, I, I.dz, nullptr, 0.0, 0.0, I.dl, false);  // J dz into dl (temporarily)
  __syncwarp(G.mask);
  for (int k = 0; k < I.T; k++)
    for (int kind = 0; kind < 4; kind++) {
      const int q = k * NSLOT + kind * 16 + i;
      if (!row_valid(kind, i)) { I.dl[q] = 0.0; I.ds[q] = 0.0; continue; }
      const double wl = w ? w[q] * I.il[q] : 0.0;
      const double d = I.D[q] * (wl - I.g[q] - I.dl[q]);
      I.dl[q] = d;
      I.ds[q] = -I.s[q] + wl - (I.s[q] * I.il[q]) * d;
    }
  __syncwarp(G.mask);
  return true;
}

// largest step in (0, 1] keeping v + alpha dv >= (1 - tau) v, for s and lambda.
// The smallest ratio v / (-dv) of each lane is tracked as a fraction (n, d),
// compared by cross products (all factors positive), and divided out once.
__device__ void step_lengths(const Group &G, const Inst<double> &I, double tau, double &ap,
                             double &ad) {
  double pn = 1.0, pd = 0.0, dn = 1.0, dd = 0.0;  // (1, 0): no bound yet
  const int i = G.lane;
  for (int k = 0; k < I.T; k++)
    for (int kind = 0; kind < 4; kind++) {
      if (!row_valid(kind, i)) continue;
      const int q = k * NSLOT + kind * 16 + i;
      const double ds = I.ds[q], dl = I.dl[q];
      if (ds < 0.0 && I.s[q] * pd < pn * -ds) { pn = I.s[q]; pd = -ds; }
      if (dl < 0.0 && I.lam[q] * dd < dn * -dl) { dn = I.lam[q]; dd = -dl; }
    }
  double mp = pd > 0.0 ? pn / pd : DBL_MAX, md = dd > 0.0 ? dn / dd : DBL_MAX;
  mp = min16(G, mp);
  md = min16(G, md);
  ap = fmin(1.0, tau * mp);
  ad = fmin(1.0, tau * md);
}

__device__ void solve_instance(const Group &G, const MpcArgs &a, int inst, bool mixed) {
  Views V{make_inst<double>(a, inst), make_inst<float>(a, inst)};
  const Inst<double> &I = V.d;
  const int i = G.lane;
  const int T = I.T;
  const double mt = (double)T * 56.0;
  bool f32 = mixed;
  // starting point: z at the middle of its box (0), s = max(g, 1), lambda = 1
  for (int k = 0; k < T; k++) I.z[k * NS + i] = 0.0;
  __syncwarp(G.mask);
  eval_rows<double>(G, I, I.z, I.x0, a.umax, a.xmax, I.g, true);
  for (int k = 0; k < T; k++)
    for (int kind = 0; kind < 4; kind++) {
      const int q = k * NSLOT + kind * 16 + i;
      const bool v = row_valid(kind, i);
      I.s[q] = v ? fmax(I.g[q], 1.0) : 1.0;
      I.lam[q] = v ? 1.0 : 0.0;
    }
  __syncwarp(G.mask);
  // scale of the primal residual: bfull = [A_0 x_0 (dynamics), bounds]
  double bs = fmax(a.umax, a.xmax);
  if (i < NX) {
    double h = 0.0;
    for (int j = 0; j < NX; j++) h += I.A[i * NX + j] * I.x0[j];
    bs = fmax(bs, fabs(h));
  }
  bs = fmax(1.0, max16(G, bs));
  double delta_p = a.delta_p;
  int status = 7, it = 0, perturbed = 0;
  double kkt = 0.0, fx = 0.0;
  for (it = 0; it <= a.max_iter; it++) {
    eval_rows<double>(G, I, I.z, I.x0, a.umax, a.xmax, I.g, true);
    __syncwarp(G.mask);
    jt_rows<double>(G, I, I.lam, -1.0, I.z, nullptr, I.rhs);  // rd = W z - J^T lambda
    double slam = 0.0, pinf = 0.0, cinf = 0.0, dinf = 0.0, f = 0.0;
    for (int k = 0; k < T; k++) {
      for (int kind = 0; kind < 4; kind++) {
        if (!row_valid(kind, i)) continue;
        const int q = k * NSLOT + kind * 16 + i;
        const double sl = I.s[q] * I.lam[q];
        slam += sl;
        pinf = fmax(pinf, fabs(I.g[q] - I.s[q]));
        cinf = fmax(cinf, fabs(sl));
      }
      dinf = fmax(dinf, fabs(I.rhs[k * NS + i]));
      const double zi = I.z[k * NS + i];
      f += 0.5 * wdiag(I.Q, I.R, i) * zi * zi;
    }
    slam = sum16(G, slam);  // sums propagate NaN; the max reductions below may not
    pinf = max16(G, pinf);
    cinf = max16(G, cinf);
    dinf = max16(G, dinf);
    fx = sum16(G, f);
    const double mu = slam / mt;
    kkt = fmax(pinf / bs, fmax(dinf, cinf / fmax(1.0, fabs(fx))));
    if (!(kkt == kkt) || !(fx == fx) || !(mu == mu)) { status = 6; break; }
    if (kkt <= a.tol) { status = 0; break; }
    if (it == a.max_iter) break;
    for (int k = 0; k < T; k++)
      for (int kind = 0; kind < 4; kind++) {
        const int q = k * NSLOT + kind * 16 + i;
        // one division per row and iteration: with t = delta_d lambda + s and
        // r = 1 / (lambda t), 1 / lambda = t r (kept for the directions) and
        // D = 1 / (delta_d + s / lambda) = lambda^2 r
        if (row_valid(kind, i)) {
          const double lm = I.lam[q], t = fma(a.delta_d, lm, I.s[q]), r = 1.0 / (lm * t);
          I.il[q] = t * r;
          I.D[q] = (lm * lm) * r;
        } else {
          I.il[q] = 0.0;
          I.D[q] = 0.0;
        }
      }
    __syncwarp(G.mask);
    bool fok = false;
    for (int tries = 0; tries < 12 && !fok; tries++) {
      if (f32) assemble<float>(G, V.f, delta_p);
      else assemble<double>(G, I, delta_p);
      __syncwarp(G.mask);
      fok = __all_sync(G.mask, kfactor(G, V, f32, perturbed));
      if (!fok) delta_p *= 100.0;
      __syncwarp(G.mask);
    }
    if (!fok) { status = 5; break; }
    // predictor; an FP32 solve that misses its tolerance switches this instance to FP64
    if (!direction(G, V, nullptr, f32, delta_p)) {
      f32 = false;
      assemble<double>(G, I, delta_p);
      __syncwarp(G.mask);
      kfactor(G, V, false, perturbed);
      __syncwarp(G.mask);
      direction(G, V, nullptr, false, delta_p);
    }
    double apa, ada;
    step_lengths(G, I, 1.0, apa, ada);
    double mua = 0.0;
    for (int k = 0; k < T; k++)
      for (int kind = 0; kind < 4; kind++) {
        if (!row_valid(kind, i)) continue;
        const int q = k * NSLOT + kind * 16 + i;
        mua += (I.s[q] + apa * I.ds[q]) * (I.lam[q] + ada * I.dl[q]);
      }
    mua = sum16(G, mua) / mt;
    const double ratio = mua / mu, sig = ratio * ratio * ratio;
    for (int k = 0; k < T; k++)
      for (int kind = 0; kind < 4; kind++) {
        const int q = k * NSLOT + kind * 16 + i;
        I.w[q] = row_valid(kind, i) ? sig * mu - I.ds[q] * I.dl[q] : 0.0;
      }
    __syncwarp(G.mask);
    // corrector
    if (!direction(G, V, I.w, f32, delta_p)) {
      f32 = false;
      assemble<double>(G, I, delta_p);
      __syncwarp(G.mask);
      kfactor(G, V, false, perturbed);
      __syncwarp(G.mask);
      direction(G, V, I.w, false, delta_p);
    }
    double ap, ad;
    step_lengths(G, I, fmax(0.99, 1.0 - mu), ap, ad);
    for (int k = 0; k < T; k++) {
      I.z[k * NS + i] += ap * I.dz[k * NS + i];
      for (int kind = 0; kind < 4; kind++) {
        if (!row_valid(kind, i)) continue;
        const int q = k * NSLOT + kind * 16 + i;
        I.s[q] += ap * I.ds[q];
        I.lam[q] += ad * I.dl[q];
      }
    }
    __syncwarp(G.mask);
  }
  if (i == 0) {
    a.obj[inst] = fx;
    a.kkt[inst] = kkt;
    a.iters[inst] = it;
    a.status[inst] = status;
    if (a.fp64_used) a.fp64_used[inst] = (mixed && !f32) ? 1 : 0;
  }
  if (a.zout)
    for (int k = 0; k < T; k++) a.zout[(a.soff[inst] + k) * NS + i] = I.z[k * NS + i];
}

__global__ void __launch_bounds__(256) mpc_ipm_kernel(MpcArgs a, int mixed) {
  Group G;
  G.lane = threadIdx.x % 16;
  G.mask = 0xFFFFu << (((threadIdx.x % 32) / 16) * 16);
  for (;;) {
    int q = 0;
    if (G.lane == 0) q = atomicAdd(a.counter, 1);
    q = __shfl_sync(G.mask, q, 0, 16);
    if (q >= a.count) break;
    solve_instance(G, a, a.order[q], mixed != 0);
  }
}

__global__ void reset_counter_kernel(int *c) { *c = 0; }

}  // namespace

void launch_mpc(const MpcArgs &a, int precision, int instances_per_cta, int ctas, cudaStream_t st) {
  const int threads = 16 * instances_per_cta;
  { note_launch(); reset_counter_kernel<<<1, 1, 0, st>>>(a.counter); }
  note_launch();
  mpc_ipm_kernel<<<ctas, threads, 0, st>>>(a, precision == 0 ? 0 : 1);
}

}  // namespace gipm
