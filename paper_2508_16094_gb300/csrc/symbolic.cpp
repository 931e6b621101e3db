// Host symbolic analysis and numeric plan of the supernodal multifrontal
// Cholesky (Sec. 2: the fill-reducing ordering is computed once on the host
// and reused across iterations; elimination-tree parallelism drives the GPU
// factorisation).
//
// Steps: pattern of K = W + J^T J + I -> elimination tree of the permuted
// pattern -> postorder (children ascending) -> column counts (sum over each
// subtree of row-subtree leaf/LCA weights, Gilbert-Ng-Peyton 1994) ->
// fundamental supernodes -> relaxed amalgamation (fixed rule below) ->
// supernode row structures by merging children -> levels -> layout of the
// frontal matrices and the batched task lists of every level.
#include <algorithm>
#include <numeric>
#include <stdexcept>

#include "internal.h"

namespace gipm {

namespace {

// Symmetric adjacency of K = W + J^T J (diagonal excluded), original numbering.
void k_adjacency(const Problem &P, std::vector<int64_t> &adjp, std::vector<int32_t> &adji) {
  const int32_t n = P.n;
  // W as a symmetric list of neighbours
  std::vector<int64_t> wsp(n + 1, 0);
  if (!P.wp.empty()) {
    for (int32_t j = 0; j < n; j++)
      for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++)
        if (P.wi[e] != j) { wsp[j + 1]++; wsp[P.wi[e] + 1]++; }
  }
  for (int32_t j = 0; j < n; j++) wsp[j + 1] += wsp[j];
  std::vector<int32_t> wsi(wsp[n]);
  {
    std::vector<int64_t> fill(wsp.begin(), wsp.end() - 1);
    if (!P.wp.empty())
      for (int32_t j = 0; j < n; j++)
        for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++)
          if (P.wi[e] != j) { wsi[fill[j]++] = P.wi[e]; wsi[fill[P.wi[e]]++] = j; }
  }
  std::vector<int32_t> mark(n, -1), buf;
  buf.reserve(64);
  adjp.assign(n + 1, 0);
  adji.clear();
  for (int32_t j = 0; j < n; j++) {
    buf.clear();
    mark[j] = j;
    for (int64_t t = P.jtp[j]; t < P.jtp[j + 1]; t++) {
      int32_t r = P.jrow[P.jtpos[t]];
      for (int64_t e = P.jp[r]; e < P.jp[r + 1]; e++) {
        int32_t i = P.ji[e];
        if (mark[i] != j) { mark[i] = j; buf.push_back(i); }
      }
    }
    for (int64_t e = wsp[j]; e < wsp[j + 1]; e++) {
      int32_t i = wsi[e];
      if (mark[i] != j) { mark[i] = j; buf.push_back(i); }
    }
    std::sort(buf.begin(), buf.end());
    adji.insert(adji.end(), buf.begin(), buf.end());
    adjp[j + 1] = (int64_t)adji.size();
  }
}

// Elimination tree of the matrix permuted by p (new->old), ip = inverse.
// Each node k links its lower neighbours' current roots to k (ancestor links
// compressed towards k as they are walked).
void etree_of(int32_t n, const std::vector<int64_t> &adjp, const std::vector<int32_t> &adji,
              const std::vector<int32_t> &p, const std::vector<int32_t> &ip,
              std::vector<int32_t> &parent) {
  parent.assign(n, -1);
  std::vector<int32_t> anc(n, -1);
  for (int32_t k = 0; k < n; k++) {
    int32_t o = p[k];
    for (int64_t e = adjp[o]; e < adjp[o + 1]; e++) {
      int32_t i = ip[adji[e]];
      if (i >= k) continue;
      while (i != k) {
        int32_t up = anc[i];
        anc[i] = k;
        if (up < 0) { parent[i] = k; break; }
        i = up;
      }
    }
  }
}

// Postorder of a forest (children ascending, roots ascending).
std::vector<int32_t> postorder_of(const std::vector<int32_t> &parent) {
  const int32_t n = (int32_t)parent.size();
  std::vector<int32_t> kidp(n + 1, 0), kids;
  for (int32_t j = 0; j < n; j++) if (parent[j] >= 0) kidp[parent[j] + 1]++;
  for (int32_t j = 0; j < n; j++) kidp[j + 1] += kidp[j];
  kids.resize(kidp[n]);
  {
    std::vector<int32_t> f(kidp.begin(), kidp.end() - 1);
    for (int32_t j = 0; j < n; j++) if (parent[j] >= 0) kids[f[parent[j]]++] = j;  // ascending
  }
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<std::pair<int32_t, int32_t>> st;  // (node, next child slot)
  for (int32_t r = 0; r < n; r++) {
    if (parent[r] >= 0) continue;
    st.emplace_back(r, kidp[r]);
    while (!st.empty()) {
      auto &top = st.back();
      if (top.second < kidp[top.first + 1]) {
        int32_t c = kids[top.second++];
        st.emplace_back(c, kidp[c]);
      } else {
        order.push_back(top.first);
        st.pop_back();
      }
    }
  }
  return order;
}

// Amalgamation rule: a child group may merge into its parent when the explicit
// zeros z of the merged block (relative to the merged trapezoid nz) satisfy:
// ncol <= 4, or ncol <= 16 and z <= 0.8 nz, or ncol <= 48 and z <= 0.1 nz, or
// z <= 0.05 nz. No width cap: a separator whose column counts shrink by more
// than one per column still becomes one wide supernode, not a chain of narrow
// ones each handing a full update matrix to the next.
bool may_merge(int64_t ncol, int64_t nrow, int64_t true_nnz) {
  const int64_t nz = ncol * (ncol + 1) / 2 + ncol * nrow;
  const int64_t z = nz - true_nnz;
  return ncol <= 4 || (ncol <= 16 && 10 * z <= 8 * nz) || (ncol <= 48 && 10 * z <= nz) ||
         20 * z <= nz;
}

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace

void analyze_symbolic(const Problem &P, const int32_t *perm_in, Symbolic &S) {
  const int32_t n = P.n;
  S.n = n;
  std::vector<int64_t> adjp;
  std::vector<int32_t> adji;
  k_adjacency(P, adjp, adji);

  // lower CSC pattern of K in the original numbering (export order)
  S.kop.assign(n + 1, 0);
  S.koi.clear();
  for (int32_t j = 0; j < n; j++) {
    S.koi.push_back(j);
    for (int64_t e = adjp[j]; e < adjp[j + 1]; e++)
      if (adji[e] > j) S.koi.push_back(adji[e]);
    S.kop[j + 1] = (int64_t)S.koi.size();
  }

  std::vector<int32_t> p0(n), ip0(n);
  for (int32_t k = 0; k < n; k++) p0[k] = perm_in ? perm_in[k] : k;
  for (int32_t k = 0; k < n; k++) ip0[p0[k]] = k;
  std::vector<int32_t> par0;
  etree_of(n, adjp, adji, p0, ip0, par0);
  std::vector<int32_t> post = postorder_of(par0);

  S.perm.resize(n);
  S.iperm.resize(n);
  for (int32_t k = 0; k < n; k++) S.perm[k] = p0[post[k]];
  for (int32_t k = 0; k < n; k++) S.iperm[S.perm[k]] = k;
  etree_of(n, adjp, adji, S.perm, S.iperm, S.parent);

  // ---- column counts: cc(j) = number of row subtrees containing j -------
  // Weight w: +1 at every leaf of a row subtree, -1 at the LCA of two
  // consecutive leaves (postorder), -1 at the parent of every row's root;
  // cc(j) = sum of w over the subtree of j.
  std::vector<int32_t> first(n), w(n, 0), prevk(n, -1), prevleaf(n, -1), anc(n);
  for (int32_t j = 0; j < n; j++) first[j] = j;
  for (int32_t j = 0; j < n; j++)  // postordered: descendants precede j
    if (S.parent[j] >= 0) first[S.parent[j]] = std::min(first[S.parent[j]], first[j]);
  for (int32_t j = 0; j < n; j++) {
    anc[j] = j;
    if (S.parent[j] >= 0) w[S.parent[j]] -= 1;
  }
  auto find_root = [&](int32_t x) {
    int32_t r = x;
    while (anc[r] != r) r = anc[r];
    while (anc[x] != r) { int32_t nx = anc[x]; anc[x] = r; x = nx; }
    return r;
  };
  for (int32_t j = 0; j < n; j++) {
    const int32_t o = S.perm[j];
    auto visit = [&](int32_t i) {  // entry (i, j) of the lower triangle, i >= j
      if (first[j] > prevk[i]) {
        w[j] += 1;
        if (prevleaf[i] >= 0) w[find_root(prevleaf[i])] -= 1;
        prevleaf[i] = j;
      }
      prevk[i] = j;
    };
    visit(j);
    for (int64_t e = adjp[o]; e < adjp[o + 1]; e++) {
      int32_t i = S.iperm[adji[e]];
      if (i > j) visit(i);
    }
    if (S.parent[j] >= 0) anc[j] = S.parent[j];
  }
  S.colcount.assign(w.begin(), w.end());
  for (int32_t j = 0; j < n; j++)
    if (S.parent[j] >= 0) S.colcount[S.parent[j]] += S.colcount[j];
  S.nnz_l = 0;
  S.flops = 0.0;
  for (int32_t j = 0; j < n; j++) {
    S.nnz_l += S.colcount[j];
    S.flops += (double)S.colcount[j] * (double)S.colcount[j];
  }

  // ---- fundamental supernodes ---------------------------------------------
  std::vector<int32_t> nkids(n, 0);
  for (int32_t j = 0; j < n; j++) if (S.parent[j] >= 0) nkids[S.parent[j]]++;
  std::vector<int32_t> fs;  // first column of each fundamental supernode
  for (int32_t j = 0; j < n; j++) {
    bool chain = j > 0 && S.parent[j - 1] == j && nkids[j] == 1 &&
                 S.colcount[j] + 1 == S.colcount[j - 1];
    if (!chain) fs.push_back(j);
  }
  const int32_t nf = (int32_t)fs.size();
  fs.push_back(n);
  std::vector<int32_t> col2f(n);
  for (int32_t f = 0; f < nf; f++)
    for (int32_t j = fs[f]; j < fs[f + 1]; j++) col2f[j] = f;

  // ---- relaxed amalgamation (child right before its parent only) ----------
  std::vector<int32_t> gfirst(fs.begin(), fs.end() - 1);
  std::vector<int64_t> gtrue(nf, 0);
  std::vector<char> gone(nf, 0);
  for (int32_t f = 0; f < nf; f++)
    for (int32_t j = fs[f]; j < fs[f + 1]; j++) gtrue[f] += S.colcount[j];
  for (int32_t f = 0; f < nf; f++) {
    const int32_t last = fs[f + 1] - 1;
    const int32_t pc = S.parent[last];
    if (pc < 0) continue;
    const int32_t q = col2f[pc];
    if (fs[q] != last + 1) continue;
    const int64_t ncol = (int64_t)(fs[f + 1] - gfirst[f]) + (fs[q + 1] - fs[q]);
    const int64_t nrow = (int64_t)S.colcount[fs[q + 1] - 1] - 1;
    if (may_merge(ncol, nrow, gtrue[f] + gtrue[q])) {
      gfirst[q] = gfirst[f];
      gtrue[q] += gtrue[f];
      gone[f] = 1;
    }
  }
  S.super.clear();
  for (int32_t f = 0; f < nf; f++) if (!gone[f]) S.super.push_back(gfirst[f]);
  S.nsuper = (int32_t)S.super.size();
  S.super.push_back(n);
  std::vector<int32_t> col2s(n);
  for (int32_t s = 0; s < S.nsuper; s++)
    for (int32_t j = S.super[s]; j < S.super[s + 1]; j++) col2s[j] = s;
  S.sparent.assign(S.nsuper, -1);
  for (int32_t s = 0; s < S.nsuper; s++) {
    int32_t pc = S.parent[S.super[s + 1] - 1];
    if (pc >= 0) S.sparent[s] = col2s[pc];
  }
  S.slevel.assign(S.nsuper, 0);
  S.nlevels = S.nsuper ? 1 : 0;
  for (int32_t s = 0; s < S.nsuper; s++) {
    int32_t p = S.sparent[s];
    if (p >= 0) S.slevel[p] = std::max(S.slevel[p], S.slevel[s] + 1);
    S.nlevels = std::max(S.nlevels, S.slevel[s] + 1);
  }

  // ---- row structures: merge the block's K rows and the children's rows ---
  std::vector<int32_t> skp(S.nsuper + 1, 0), skids;
  for (int32_t s = 0; s < S.nsuper; s++) if (S.sparent[s] >= 0) skp[S.sparent[s] + 1]++;
  for (int32_t s = 0; s < S.nsuper; s++) skp[s + 1] += skp[s];
  skids.resize(skp[S.nsuper]);
  {
    std::vector<int32_t> f(skp.begin(), skp.end() - 1);
    for (int32_t s = 0; s < S.nsuper; s++) if (S.sparent[s] >= 0) skids[f[S.sparent[s]]++] = s;
  }
  S.srp.assign(S.nsuper + 1, 0);
  S.sri.clear();
  std::vector<int32_t> mark(n, -1), buf;
  for (int32_t s = 0; s < S.nsuper; s++) {
    const int32_t c0 = S.super[s], c1 = S.super[s + 1];
    buf.clear();
    for (int32_t j = c0; j < c1; j++) {
      const int32_t o = S.perm[j];
      for (int64_t e = adjp[o]; e < adjp[o + 1]; e++) {
        int32_t i = S.iperm[adji[e]];
        if (i >= c1 && mark[i] != s) { mark[i] = s; buf.push_back(i); }
      }
    }
    for (int32_t t = skp[s]; t < skp[s + 1]; t++) {
      const int32_t c = skids[t];
      for (int64_t e = S.srp[c]; e < S.srp[c + 1]; e++) {
        int32_t i = S.sri[e];
        if (i >= c1 && mark[i] != s) { mark[i] = s; buf.push_back(i); }
      }
    }
    std::sort(buf.begin(), buf.end());
    if ((int64_t)buf.size() != (int64_t)S.colcount[c1 - 1] - 1)
      throw std::runtime_error("symbolic: supernode structure disagrees with column count");
    S.sri.insert(S.sri.end(), buf.begin(), buf.end());
    S.srp[s + 1] = (int64_t)S.sri.size();
  }
}

void build_plan(const Problem &P, const Symbolic &S, Plan &plan, int nb, int nbs) {
  const int32_t ns = S.nsuper;
  plan.nb = nb;
  plan.nbs = nbs;
  plan.fronts.assign(ns, FrontInfo{});
  plan.max_front = plan.max_ncol = 0;
  plan.levels.clear();
  // children lists
  std::vector<int32_t> kp(ns + 1, 0);
  for (int32_t s = 0; s < ns; s++) if (S.sparent[s] >= 0) kp[S.sparent[s] + 1]++;
  for (int32_t s = 0; s < ns; s++) kp[s + 1] += kp[s];
  plan.children.assign(kp[ns], 0);
  {
    std::vector<int32_t> f(kp.begin(), kp.end() - 1);
    for (int32_t s = 0; s < ns; s++) if (S.sparent[s] >= 0) plan.children[f[S.sparent[s]]++] = s;
  }
  // Schedule level: as late as possible (depth below the root counted from the
  // deepest front), so every child sits exactly one level below its parent and
  // an update matrix lives from its own level to the next one only.
  std::vector<int32_t> depth(ns, 0);
  int32_t maxdepth = 0;
  for (int32_t s = ns - 1; s >= 0; s--) {  // parents have larger indices
    if (S.sparent[s] >= 0) depth[s] = depth[S.sparent[s]] + 1;
    maxdepth = std::max(maxdepth, depth[s]);
  }
  plan.sched.assign(ns, 0);
  for (int32_t s = 0; s < ns; s++) plan.sched[s] = maxdepth - depth[s];
  const int32_t nlev = ns ? maxdepth + 1 : 0;
  // update matrices: two pools alternating by level parity
  std::vector<int64_t> lev_u(nlev + 1, 0);
  int64_t loff = 0;
  for (int32_t s = 0; s < ns; s++) {
    FrontInfo &F = plan.fronts[s];
    F.first = S.super[s];
    F.ncol = S.super[s + 1] - S.super[s];
    F.nrow = (int32_t)(S.srp[s + 1] - S.srp[s]);
    F.ld = (int32_t)round_up(F.ncol, 8);  // 16-byte rows for TMA in FP32 and in BF16
    F.uld = (int32_t)round_up(std::max(F.nrow, 1), 4);
    F.loff = loff;
    loff += round_up((int64_t)(F.ncol + F.nrow) * F.ld, 32);
    F.rows_off = S.srp[s];
    F.child_begin = kp[s];
    F.child_end = kp[s + 1];
    F.parent = S.sparent[s];
    F.inv_off = -1;
    F.uoff = 0;
    if (F.nrow > 0) {
      F.uoff = lev_u[plan.sched[s]];
      lev_u[plan.sched[s]] += round_up((int64_t)F.nrow * F.uld, 32);
    }
    plan.max_front = std::max(plan.max_front, F.ncol + F.nrow);
    plan.max_ncol = std::max(plan.max_ncol, F.ncol);
  }
  int64_t pool[2] = {0, 0};
  for (int32_t L = 0; L < nlev; L++) pool[L & 1] = std::max(pool[L & 1], lev_u[L]);
  for (int32_t s = 0; s < ns; s++)
    if (plan.sched[s] & 1) plan.fronts[s].uoff += pool[0];
  plan.l_entries = loff;
  plan.u_entries = std::max<int64_t>(pool[0] + pool[1], 32);

  // child -> parent maps (relative positions and their inverses)
  plan.relpos.assign(S.sri.size(), -1);
  int64_t inv_total = 0;
  for (int32_t s = 0; s < ns; s++) {
    if (S.sparent[s] < 0) continue;
    const FrontInfo &Pf = plan.fronts[S.sparent[s]];
    plan.fronts[s].inv_off = inv_total;
    inv_total += Pf.ncol + Pf.nrow;
  }
  plan.inv.assign(inv_total, -1);
  for (int32_t s = 0; s < ns; s++) {
    const int32_t p = S.sparent[s];
    if (p < 0) continue;
    const FrontInfo &C = plan.fronts[s];
    const FrontInfo &Pf = plan.fronts[p];
    const int32_t *prow = S.sri.data() + Pf.rows_off;
    int32_t q = 0;  // walk the parent's sorted rows alongside the child's sorted rows
    for (int32_t t = 0; t < C.nrow; t++) {
      const int32_t r = S.sri[C.rows_off + t];
      int32_t pos;
      if (r < Pf.first + Pf.ncol) {
        pos = r - Pf.first;
        if (pos < 0) throw std::runtime_error("plan: child row below parent block");
      } else {
        while (q < Pf.nrow && prow[q] < r) q++;
        if (q >= Pf.nrow || prow[q] != r) throw std::runtime_error("plan: child row not in parent");
        pos = Pf.ncol + q;
      }
      plan.relpos[C.rows_off + t] = pos;
      plan.inv[C.inv_off + pos] = t;
    }
  }

  // fronts ordered by schedule level
  plan.level_fronts.resize(ns);
  std::iota(plan.level_fronts.begin(), plan.level_fronts.end(), 0);
  std::stable_sort(plan.level_fronts.begin(), plan.level_fronts.end(),
                   [&](int32_t a, int32_t b) { return plan.sched[a] < plan.sched[b]; });
  plan.levels.assign(nlev, LevelPlan{});
  {
    int32_t i = 0;
    for (int32_t L = 0; L < nlev; L++) {
      plan.levels[L].front_b = i;
      while (i < ns && plan.sched[plan.level_fronts[i]] == L) i++;
      plan.levels[L].front_e = i;
    }
  }

  // ---- K entries, level-major, with their product lists ------------------
  const int32_t n = S.n;
  const int64_t nk = S.kop[n];
  std::vector<int32_t> col2s(n);
  for (int32_t s = 0; s < ns; s++)
    for (int32_t j = S.super[s]; j < S.super[s + 1]; j++) col2s[j] = s;
  std::vector<int64_t> slot(nk);
  std::vector<int32_t> elev(nk);
  for (int32_t oj = 0; oj < n; oj++)
    for (int64_t e = S.kop[oj]; e < S.kop[oj + 1]; e++) {
      int32_t a = S.iperm[S.koi[e]], b = S.iperm[oj];
      int32_t i = std::max(a, b), j = std::min(a, b);
      int32_t s = col2s[j];
      const FrontInfo &F = plan.fronts[s];
      int32_t prow;
      if (i < F.first + F.ncol) {
        prow = i - F.first;
      } else {
        const int32_t *rb = S.sri.data() + F.rows_off;
        const int32_t *it = std::lower_bound(rb, rb + F.nrow, i);
        if (it == rb + F.nrow || *it != i) throw std::runtime_error("plan: K entry outside L");
        prow = F.ncol + (int32_t)(it - rb);
      }
      slot[e] = F.loff + (int64_t)prow * F.ld + (j - F.first);
      elev[e] = plan.sched[s];
    }
  std::vector<int64_t> order(nk);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return elev[x] != elev[y] ? elev[x] < elev[y] : slot[x] < slot[y];
  });
  std::vector<int64_t> pos_of(nk);
  for (int64_t q = 0; q < nk; q++) pos_of[order[q]] = q;
  for (int32_t L = 0, q = 0; L < nlev; L++) {
    plan.levels[L].k_b = q;
    while (q < nk && elev[order[q]] == L) q++;
    plan.levels[L].k_e = q;
  }
  // entry index of K(i, j) (original numbering, i >= j) in the export order
  auto kindex = [&](int32_t i, int32_t j) -> int64_t {
    const int32_t *b = S.koi.data() + S.kop[j], *e = S.koi.data() + S.kop[j + 1];
    const int32_t *it = std::lower_bound(b, e, i);
    if (it == e || *it != i) throw std::runtime_error("plan: product outside K pattern");
    return S.kop[j] + (it - b);
  };
  // products: every pair of positions in one J row contributes to one entry
  std::vector<int64_t> cnt(nk + 1, 0);
  for (int32_t r = 0; r < P.m; r++)
    for (int64_t a = P.jp[r]; a < P.jp[r + 1]; a++)
      for (int64_t b = P.jp[r]; b <= a; b++) {
        int32_t i = std::max(P.ji[a], P.ji[b]), j = std::min(P.ji[a], P.ji[b]);
        cnt[pos_of[kindex(i, j)] + 1]++;
      }
  for (int64_t q = 0; q < nk; q++) cnt[q + 1] += cnt[q];
  plan.k_poff = cnt;
  plan.k_pa.assign(cnt[nk], 0);
  plan.k_pb.assign(cnt[nk], 0);
  {
    std::vector<int64_t> f(cnt.begin(), cnt.end() - 1);
    for (int32_t r = 0; r < P.m; r++)  // ascending row: products of an entry stay row-sorted
      for (int64_t a = P.jp[r]; a < P.jp[r + 1]; a++)
        for (int64_t b = P.jp[r]; b <= a; b++) {
          int32_t i = std::max(P.ji[a], P.ji[b]), j = std::min(P.ji[a], P.ji[b]);
          int64_t q = pos_of[kindex(i, j)];
          plan.k_pa[f[q]] = (int32_t)a;
          plan.k_pb[f[q]] = (int32_t)b;
          f[q]++;
        }
  }
  plan.k_slot.resize(nk);
  plan.k_orig.resize(nk);
  plan.k_diag.assign(nk, -1);
  plan.k_w.assign(nk, -1);
  for (int64_t q = 0; q < nk; q++) {
    plan.k_slot[q] = slot[order[q]];
    plan.k_orig[q] = order[q];
  }
  for (int32_t j = 0; j < n; j++) plan.k_diag[pos_of[S.kop[j]]] = j;  // first entry of a column
  if (!P.wp.empty())
    for (int32_t j = 0; j < n; j++)
      for (int64_t e = P.wp[j]; e < P.wp[j + 1]; e++) {
        int32_t i = std::max(P.wi[e], j), jj = std::min(P.wi[e], j);
        plan.k_w[pos_of[kindex(i, jj)]] = e;
      }

  // ---- task lists of every level -----------------------------------------
  const int BT = kBuildTile;  // front-assembly tile
  const int GM = 64;        // GEMM / SYRK tile rows
  const int TR = 128;       // TRSM rows per task
  const int GR = 256;       // solve gather positions per task
  const int SR = 128;       // solve forward-update rows per task
  const int SC = 256;       // solve backward-update columns per task
  plan.build_tasks.clear(); plan.gemm_tasks.clear(); plan.potrf_tasks.clear();
  plan.trsm_tasks.clear(); plan.syrk_tasks.clear(); plan.gath_tasks.clear();
  plan.sdiag_tasks.clear(); plan.sgemv_tasks.clear(); plan.rgemv_tasks.clear();
  plan.toff.assign(ns, 0);
  plan.t_entries = 0;
  for (int32_t s = 0; s < ns; s++) {
    plan.toff[s] = plan.t_entries;
    plan.t_entries += plan.fronts[s].nrow;
  }
  plan.t_entries = std::max<int64_t>(plan.t_entries, 1);
  for (int32_t L = 0; L < nlev; L++) {
    LevelPlan &LP = plan.levels[L];
    LP.max_ncol = 0;
    for (int32_t t = LP.front_b; t < LP.front_e; t++)
      LP.max_ncol = std::max(LP.max_ncol, plan.fronts[plan.level_fronts[t]].ncol);
    LP.build_b = (int32_t)plan.build_tasks.size();
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const int32_t nfr = plan.fronts[s].ncol + plan.fronts[s].nrow;
      const int32_t ncol = plan.fronts[s].ncol;
      // BT x BT tiles of the lower triangle; column tiles start at multiples
      // of BT in the panel and at ncol + multiples of BT in the update matrix,
      // so both take aligned 4-wide stores (c = tile width)
      for (int32_t r0 = 0; r0 < nfr; r0 += BT) {
        for (int32_t c0 = 0; c0 < ncol && c0 <= r0 + BT - 1; c0 += BT)
          plan.build_tasks.push_back({s, r0, c0, std::min(BT, ncol - c0)});
        for (int32_t c0 = ncol; c0 < nfr && c0 <= r0 + BT - 1; c0 += BT)
          plan.build_tasks.push_back({s, r0, c0, std::min(BT, nfr - c0)});
      }
    }
    LP.build_e = (int32_t)plan.build_tasks.size();
    LP.steps.clear();
    for (int32_t k = 0; k < LP.max_ncol; k += nb) {
      StepRange st{};
      st.gemm_b = (int32_t)plan.gemm_tasks.size();
      if (k > 0)
        for (int32_t t = LP.front_b; t < LP.front_e; t++) {
          const int32_t s = plan.level_fronts[t];
          const FrontInfo &F = plan.fronts[s];
          if (F.ncol <= k) continue;
          for (int32_t i0 = k; i0 < F.ncol + F.nrow; i0 += GM) plan.gemm_tasks.push_back({s, i0, k, 0});
        }
      st.gemm_e = (int32_t)plan.gemm_tasks.size();
      st.potrf_b = (int32_t)plan.potrf_tasks.size();
      for (int32_t t = LP.front_b; t < LP.front_e; t++) {
        const int32_t s = plan.level_fronts[t];
        if (plan.fronts[s].ncol > k) plan.potrf_tasks.push_back({s, k, 0, 0});
      }
      st.potrf_e = (int32_t)plan.potrf_tasks.size();
      st.trsm_b = (int32_t)plan.trsm_tasks.size();
      for (int32_t t = LP.front_b; t < LP.front_e; t++) {
        const int32_t s = plan.level_fronts[t];
        const FrontInfo &F = plan.fronts[s];
        if (F.ncol <= k) continue;
        const int32_t kb = std::min(nb, F.ncol - k);
        for (int32_t i0 = k + kb; i0 < F.ncol + F.nrow; i0 += TR) plan.trsm_tasks.push_back({s, i0, k, 0});
      }
      st.trsm_e = (int32_t)plan.trsm_tasks.size();
      LP.steps.push_back(st);
    }
    LP.syrk_b = (int32_t)plan.syrk_tasks.size();
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const FrontInfo &F = plan.fronts[s];
      for (int32_t i0 = 0; i0 < F.nrow; i0 += GM)
        for (int32_t j0 = 0; j0 <= i0; j0 += GM) plan.syrk_tasks.push_back({s, i0, j0, 0});
    }
    LP.syrk_e = (int32_t)plan.syrk_tasks.size();
    // solve: gather tasks cover every front (they also initialise its update vector)
    LP.gath_b = (int32_t)plan.gath_tasks.size();
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const FrontInfo &F = plan.fronts[s];
      for (int32_t p0 = 0; p0 < F.ncol + F.nrow; p0 += GR) plan.gath_tasks.push_back({s, p0, 0, 0});
    }
    LP.gath_e = (int32_t)plan.gath_tasks.size();
    LP.rg_b = (int32_t)plan.rgemv_tasks.size();
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = plan.level_fronts[t];
      const FrontInfo &F = plan.fronts[s];
      if (F.nrow == 0) continue;
      for (int32_t c0 = 0; c0 < F.ncol; c0 += 32) plan.rgemv_tasks.push_back({s, c0, 0, 0});
    }
    LP.rg_e = (int32_t)plan.rgemv_tasks.size();
    // solve steps over block columns of width nbs: diagonal tasks and update tasks
    LP.sstep_b.clear();
    LP.sgemv_b.clear();
    LP.sdiag_b = (int32_t)plan.sdiag_tasks.size();
    for (int32_t j = 0; j < LP.max_ncol; j += nbs) {
      LP.sstep_b.push_back((int32_t)plan.sdiag_tasks.size());
      LP.sgemv_b.push_back((int32_t)plan.sgemv_tasks.size());
      for (int32_t t = LP.front_b; t < LP.front_e; t++) {
        const int32_t s = plan.level_fronts[t];
        const FrontInfo &F = plan.fronts[s];
        if (F.ncol <= j) continue;
        plan.sdiag_tasks.push_back({s, j, 0, 0});
      }
      // forward update rows below the block (SR rows per task); the backward
      // update of columns left of the block (SC columns per task) uses the
      // same list with c = 1
      for (int32_t t = LP.front_b; t < LP.front_e; t++) {
        const int32_t s = plan.level_fronts[t];
        const FrontInfo &F = plan.fronts[s];
        if (F.ncol <= j) continue;
        const int32_t jb = std::min(nbs, F.ncol - j);
        for (int32_t i0 = j + jb; i0 < F.ncol + F.nrow; i0 += SR) plan.sgemv_tasks.push_back({s, i0, j, 0});
        for (int32_t c0 = 0; c0 < j; c0 += SC) plan.sgemv_tasks.push_back({s, c0, j, 1});
      }
    }
    LP.sstep_b.push_back((int32_t)plan.sdiag_tasks.size());
    LP.sgemv_b.push_back((int32_t)plan.sgemv_tasks.size());
    LP.sdiag_e = (int32_t)plan.sdiag_tasks.size();
  }
}

}  // namespace gipm

namespace gipm {

// Range checks of every task against the buffers its kernel indexes (the
// kernels mask rows/columns past a front's order; everything else must hold
// here). Throws std::runtime_error naming the first violation.
void validate_plan(const Problem &P, const Symbolic &S, const Plan &pl) {
  auto need = [](bool ok, const char *what) {
    if (!ok) throw std::runtime_error(std::string("plan check failed: ") + what);
  };
  const int32_t ns = (int32_t)pl.fronts.size();
  need(pl.nb <= 64 && pl.nbs <= 64, "block widths above the kernels' 64-wide shared tiles");
  auto nf = [&](int32_t s) { return (int64_t)pl.fronts[s].ncol + pl.fronts[s].nrow; };
  for (int32_t s = 0; s < ns; s++) {
    const FrontInfo &F = pl.fronts[s];
    need(F.ncol > 0 && F.nrow >= 0 && F.ld >= F.ncol && F.ld % 8 == 0, "front shape");
    need(F.loff >= 0 && F.loff + nf(s) * F.ld <= pl.l_entries, "panel inside factor storage");
    need(F.nrow == 0 || (F.uoff >= 0 && F.uoff + (int64_t)F.nrow * F.uld <= pl.u_entries),
         "update matrix inside update storage");
    need(F.uld >= F.nrow, "update stride");
    need(F.rows_off + F.nrow <= (int64_t)S.sri.size(), "row structure range");
    need(pl.toff[s] + F.nrow <= pl.t_entries, "solve update vector range");
    need(F.child_begin >= 0 && F.child_end <= (int32_t)pl.children.size() &&
             F.child_begin <= F.child_end, "child range");
    for (int32_t ci = F.child_begin; ci < F.child_end; ci++) {
      const int32_t c = pl.children[ci];
      need(c >= 0 && c < s && pl.fronts[c].parent == s, "child link");
      need(pl.sched[c] + 1 == pl.sched[s], "child one level below its parent");
      const FrontInfo &Cf = pl.fronts[c];
      need(Cf.inv_off >= 0 && Cf.inv_off + nf(s) <= (int64_t)pl.inv.size(), "inverse map range");
      for (int64_t p = 0; p < nf(s); p++) {
        const int32_t a = pl.inv[Cf.inv_off + p];
        need(a >= -1 && a < Cf.nrow, "inverse map entry");
      }
      for (int32_t t = 0; t < Cf.nrow; t++) {
        const int32_t r = pl.relpos[Cf.rows_off + t];
        need(r >= 0 && r < nf(s) && pl.inv[Cf.inv_off + r] == t, "relative position");
      }
    }
    for (int32_t t = 0; t < F.nrow; t++) {
      const int32_t r = S.sri[F.rows_off + t];
      need(r >= F.first + F.ncol && r < P.n, "row index");
    }
  }
  // update pools: fronts of one level must not overlap
  for (const LevelPlan &LP : pl.levels) {
    std::vector<std::pair<int64_t, int64_t>> iv;
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const FrontInfo &F = pl.fronts[pl.level_fronts[t]];
      if (F.nrow > 0) iv.emplace_back(F.uoff, F.uoff + (int64_t)F.nrow * F.uld);
    }
    std::sort(iv.begin(), iv.end());
    for (size_t i = 1; i < iv.size(); i++) need(iv[i].first >= iv[i - 1].second, "update overlap");
  }
  auto in_front = [&](const Task &t) { return t.front >= 0 && t.front < ns; };
  // build tiles: in range, and together covering every lower-triangle entry of
  // each front exactly once (tiles of a front in strictly increasing (row,
  // column) order, entry counts adding up to nf (nf + 1) / 2)
  {
    int32_t cur = -1, pa = -1, pb = -1;
    int64_t covered = 0;
    auto close_front = [&]() {
      if (cur >= 0) need(covered == (int64_t)nf(cur) * (nf(cur) + 1) / 2, "build tiles cover the front");
    };
    for (const Task &t : pl.build_tasks) {
      need(in_front(t), "build task");
      const int32_t nc = pl.fronts[t.front].ncol, n = nf(t.front), lim = t.b < nc ? nc : n;
      need(t.a >= 0 && t.a < n && t.a % kBuildTile == 0 && t.b >= 0 &&
               t.b <= t.a + kBuildTile - 1 && t.c >= 1 && t.c <= kBuildTile && t.b + t.c <= lim &&
               (t.b < nc ? t.b : t.b - nc) % kBuildTile == 0,
           "build task");
      if (t.front != cur) {
        close_front();
        cur = t.front;
        covered = 0;
        pa = pb = -1;
      } else {
        need(t.a > pa || (t.a == pa && t.b > pb), "build tiles in order");
      }
      pa = t.a;
      pb = t.b;
      // entries (r, c) with c <= r, r in [a, min(a + tile, n)), c in [b, b + w)
      const int64_t lo = t.a, hi = std::min<int64_t>(t.a + kBuildTile, n) - 1, b = t.b, w = t.c;
      const int64_t s0 = std::max(lo, b), s1 = std::min(hi, b + w - 2);
      if (s1 >= s0) {
        const int64_t u0 = s0 - b + 1, u1 = s1 - b + 1;
        covered += (u0 + u1) * (u1 - u0 + 1) / 2;
      }
      covered += w * std::max<int64_t>(0, hi - std::max(lo, b + w - 1) + 1);
    }
    close_front();
  }
  for (const Task &t : pl.gemm_tasks)
    need(in_front(t) && t.b > 0 && t.b < pl.fronts[t.front].ncol && t.a >= t.b &&
             t.a < nf(t.front), "gemm task");
  for (const Task &t : pl.potrf_tasks)
    need(in_front(t) && t.a >= 0 && t.a < pl.fronts[t.front].ncol, "potrf task");
  for (const Task &t : pl.trsm_tasks) {
    need(in_front(t) && t.b >= 0 && t.b < pl.fronts[t.front].ncol, "trsm task block");
    const int32_t kb = std::min(pl.nb, pl.fronts[t.front].ncol - t.b);
    need(t.a >= t.b + kb && t.a < nf(t.front), "trsm task rows");
  }
  for (const Task &t : pl.syrk_tasks)
    need(in_front(t) && t.a >= 0 && t.a < pl.fronts[t.front].nrow && t.b >= 0 && t.b <= t.a,
         "syrk task");
  for (const Task &t : pl.gath_tasks)
    need(in_front(t) && t.a >= 0 && t.a < nf(t.front), "gather task");
  for (const Task &t : pl.sdiag_tasks)
    need(in_front(t) && t.a >= 0 && t.a < pl.fronts[t.front].ncol, "solve diagonal task");
  for (const Task &t : pl.sgemv_tasks) {
    need(in_front(t) && t.b >= 0 && t.b < pl.fronts[t.front].ncol, "solve update block");
    const int32_t jb = std::min(pl.nbs, pl.fronts[t.front].ncol - t.b);
    if (t.c == 0) need(t.a >= t.b + jb && t.a < nf(t.front), "solve forward rows");
    else need(t.c == 1 && t.a >= 0 && t.a < t.b, "solve backward columns");
  }
  for (const Task &t : pl.rgemv_tasks)
    need(in_front(t) && t.a >= 0 && t.a < pl.fronts[t.front].ncol && pl.fronts[t.front].nrow > 0,
         "solve rows-below task");
  const int64_t nnzj = P.jp.empty() ? 0 : P.jp.back();
  for (size_t q = 0; q < pl.k_slot.size(); q++) {
    need(pl.k_slot[q] >= 0 && pl.k_slot[q] < pl.l_entries, "K slot");
    need(pl.k_poff[q] <= pl.k_poff[q + 1], "K product range");
    need(pl.k_diag[q] >= -1 && pl.k_diag[q] < P.n, "K diagonal index");
  }
  for (size_t p = 0; p < pl.k_pa.size(); p++)
    need(pl.k_pa[p] >= 0 && pl.k_pa[p] < nnzj && pl.k_pb[p] >= 0 && pl.k_pb[p] < nnzj,
         "K product operands");
  for (const LevelPlan &LP : pl.levels) {
    need(LP.build_b <= LP.build_e && LP.build_e <= (int32_t)pl.build_tasks.size(), "build range");
    need(LP.k_b <= LP.k_e && LP.k_e <= (int64_t)pl.k_slot.size(), "K range");
    need(LP.syrk_e <= (int32_t)pl.syrk_tasks.size() && LP.gath_e <= (int32_t)pl.gath_tasks.size() &&
             LP.rg_e <= (int32_t)pl.rgemv_tasks.size(), "level ranges");
  }
}

}  // namespace gipm

namespace gipm {

// Fused FP32 solve: for every front and 128-wide block column j, one inverse
// task (the diagonal block's inverse, jb x jb, at fs_dinv_off[slot]), forward
// tasks over the rows [j, nf) in chunks of 128 (the chunk starting at j also
// publishes the solved block), backward tasks over the columns [0, j) in
// chunks of 256 (at least one, which publishes the solved block).
void build_fused_solve(Plan &pl) {
  constexpr int B = 128, RC = 128;
  const int32_t nfr = (int32_t)pl.fronts.size();
  pl.fs_inv.clear();
  pl.fs_dinv_off.clear();
  pl.fs_dinv_entries = 0;
  pl.ps_tasks.clear();
  pl.fs_first_slot.assign(nfr, 0);
  for (int32_t s = 0; s < nfr; s++) {
    const FrontInfo &F = pl.fronts[s];
    pl.fs_first_slot[s] = (int32_t)pl.fs_dinv_off.size();
    for (int32_t j = 0; j < F.ncol; j += B) {
      const int32_t jb = std::min(B, F.ncol - j);
      const int32_t slot = (int32_t)pl.fs_dinv_off.size();
      pl.fs_dinv_off.push_back(pl.fs_dinv_entries);
      pl.fs_dinv_entries += (int64_t)jb * round_up(jb, 4);  // keeps every slot 16-byte aligned
      pl.fs_inv.push_back({s, j, slot, 0});
    }
  }
  pl.fs_dinv_entries = std::max<int64_t>(pl.fs_dinv_entries, 4);
  auto nblk = [&](int32_t s) { return (pl.fronts[s].ncol + B - 1) / B; };
  // forward, leaves to root, level by level: the diagonal chunks of every front
  // of the level (ascending), then the chunks of rows below the fronts
  for (const LevelPlan &LP : pl.levels) {
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = pl.level_fronts[t];
      for (int32_t i = 0; i < nblk(s); i++) pl.ps_tasks.push_back({s, i, 0, WS_FWD_DIAG});
    }
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = pl.level_fronts[t];
      for (int32_t r0 = 0; r0 < pl.fronts[s].nrow; r0 += RC) pl.ps_tasks.push_back({s, r0, 0, WS_FWD_BELOW});
    }
  }
  pl.ps_fwd_tasks = (int32_t)pl.ps_tasks.size();
  // backward, root to leaves, level by level: the partial sums of every
  // 128-row chunk below every front of the level (one task per chunk, all
  // column blocks), then the column blocks (last to first)
  pl.ps_pbase.assign(nfr, 0);
  int64_t prow = 0;
  for (int32_t s = 0; s < nfr; s++) {
    pl.ps_pbase[s] = prow;
    prow += (int64_t)nblk(s) * ((pl.fronts[s].nrow + RC - 1) / RC);
  }
  pl.ps_part_entries = std::max<int64_t>(prow, 1) * B;
  for (int32_t li = (int32_t)pl.levels.size() - 1; li >= 0; li--) {
    const LevelPlan &LP = pl.levels[li];
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = pl.level_fronts[t];
      for (int32_t r0 = 0; r0 < pl.fronts[s].nrow; r0 += RC) pl.ps_tasks.push_back({s, 0, r0, WS_BWD_PART});
    }
    for (int32_t t = LP.front_b; t < LP.front_e; t++) {
      const int32_t s = pl.level_fronts[t];
      for (int32_t cb = nblk(s) - 1; cb >= 0; cb--) pl.ps_tasks.push_back({s, cb, 0, WS_BWD_DIAG});
    }
  }
  pl.ps_kid_chunks.assign(nfr, 0);
  pl.ps_parent_blocks.assign(nfr, 0);
  for (int32_t s = 0; s < nfr; s++) {
    const int32_t par = pl.fronts[s].parent;
    if (par >= 0) {
      pl.ps_kid_chunks[par] += (pl.fronts[s].nrow + RC - 1) / RC;
      pl.ps_parent_blocks[s] = nblk(par);
    }
  }
  const int64_t nslot = (int64_t)pl.fs_dinv_off.size();
  pl.ps_flag_words = 32 + 3 * nslot + 2 * (int64_t)nfr;
  // range checks (the kernel masks only the chunk edges), and the order every
  // wait of the kernel relies on: a task waits only for earlier tasks
  auto need = [](bool ok, const char *w) {
    if (!ok) throw std::runtime_error(std::string("solve plan check failed: ") + w);
  };
  for (const Task &t : pl.fs_inv)
    need(t.b >= 0 && t.b < nslot && t.b == pl.fs_first_slot[t.front] + t.a / B &&
             pl.fs_dinv_off[t.b] % 4 == 0,
         "inverse task");
  std::vector<int32_t> fwd_diag_seen(nfr, 0), fwd_below_seen(nfr, 0), bwd_diag_seen(nfr, 0);
  std::vector<int32_t> bwd_part_seen(nfr, 0), level_of(nfr, -1);
  for (size_t li = 0; li < pl.levels.size(); li++)
    for (int32_t t = pl.levels[li].front_b; t < pl.levels[li].front_e; t++) level_of[pl.level_fronts[t]] = (int32_t)li;
  auto nbelow = [&](int32_t s) { return (pl.fronts[s].nrow + RC - 1) / RC; };
  for (size_t q = 0; q < pl.ps_tasks.size(); q++) {
    const Task &t = pl.ps_tasks[q];
    need(t.front >= 0 && t.front < nfr, "task front");
    const FrontInfo &F = pl.fronts[t.front];
    need(F.ld % 4 == 0 && F.loff % 4 == 0, "panel alignment");
    need((q < (size_t)pl.ps_fwd_tasks) == (t.c <= WS_FWD_BELOW) && t.c >= 0 && t.c <= WS_BWD_DIAG,
         "task order");
    const int32_t s = t.front;
    switch (t.c) {
      case WS_FWD_DIAG:
        need(t.a == fwd_diag_seen[s]++ && t.a < nblk(s), "forward diagonal task");
        for (int32_t ci = F.child_begin; ci < F.child_end; ci++)  // children complete before
          need(fwd_below_seen[pl.children[ci]] == nbelow(pl.children[ci]), "forward child order");
        break;
      case WS_FWD_BELOW:
        need(t.a == RC * fwd_below_seen[s]++ && t.a < F.nrow && fwd_diag_seen[s] == nblk(s),
             "forward below task");
        for (int32_t ci = F.child_begin; ci < F.child_end; ci++)
          need(fwd_below_seen[pl.children[ci]] == nbelow(pl.children[ci]), "forward child order");
        break;
      case WS_BWD_PART:
        need(t.a == 0 && t.b == RC * bwd_part_seen[s] && t.b < F.nrow &&
                 (F.parent < 0 || bwd_diag_seen[F.parent] == nblk(F.parent)) &&
                 pl.ps_pbase[s] + (int64_t)(nblk(s) - 1) * nbelow(s) + t.b / RC < pl.ps_part_entries / B,
             "backward partial task");
        bwd_part_seen[s]++;
        break;
      default:
        need(t.a == nblk(s) - 1 - bwd_diag_seen[s]++ && t.a >= 0 &&
                 bwd_part_seen[s] == nbelow(s) &&
                 (F.parent < 0 || bwd_diag_seen[F.parent] == nblk(F.parent)),
             "backward diagonal task");
    }
  }
  for (int32_t s = 0; s < nfr; s++) {
    need(fwd_diag_seen[s] == nblk(s) && fwd_below_seen[s] == nbelow(s) && bwd_diag_seen[s] == nblk(s),
         "every block solved once per sweep");
    int32_t kids = 0;  // the chunk counter a front waits for covers exactly its children
    for (int32_t ci = pl.fronts[s].child_begin; ci < pl.fronts[s].child_end; ci++) {
      need(pl.fronts[pl.children[ci]].parent == s, "child list");
      kids += nbelow(pl.children[ci]);
    }
    need(kids == pl.ps_kid_chunks[s], "children's chunk count");
  }
  pl.ps_recs.resize(pl.ps_tasks.size());
  for (size_t q = 0; q < pl.ps_tasks.size(); q++) {
    const int32_t s = pl.ps_tasks[q].front;
    pl.ps_recs[q] = SolveRec{pl.ps_tasks[q], pl.fronts[s], pl.toff[s], pl.ps_pbase[s],
                             pl.fs_first_slot[s], pl.ps_kid_chunks[s], pl.ps_parent_blocks[s], 0};
  }
}

}  // namespace gipm
