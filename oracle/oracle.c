/*
 * CPU oracle for the pivoting-free interior-point method (test infrastructure).
 *
 * Plain, slow, single-threaded FP64 C. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it; the product library never links it and
 * shares no code with it.
 *
 * What it computes, in the paper's order and notation:
 *   - Problem (1):  min f(x) s.t. g(x) >= 0, here the LP  min c^T x,
 *     g = [A x - b ; x - l ; u - x]  (bounds are rows of g with J = [A; I; -I]).
 *   - KKT conditions (2) with slack s and multipliers lambda.
 *   - Regularised Newton system (3); eliminating d_s gives the augmented form
 *     (4), eliminating d_lambda gives the primal condensed system (5):
 *       K = W + delta_p I + J^T D J,   D = (delta_d I + Lambda^{-1} S)^{-1},
 *       K d_x = -r_p,  r_p = grad f - J^T lambda + J^T D (g - w ./ lambda),
 *     with d_lambda = D (w ./ lambda - g - J d_x),
 *          d_s      = -s + w ./ lambda - (s ./ lambda) .* d_lambda,
 *     where w = mu e for the pure barrier step (the "mu S^{-1} e" term of (3)).
 *   - K is SPD, so it is factored by Cholesky without pivoting after a given
 *     fill-reducing ordering (Sec. 2, Sec. 3 "Pivoting-Free IPM").
 *
 * Symbolic analysis (ordering given, Sec. 2): elimination tree (Liu's
 * algorithm with path compression), postorder (children ascending), explicit
 * column structures by merging children's structures, fundamental supernodes
 * and a fixed relaxed-amalgamation rule, supernode row structures as explicit
 * unions, supernode levels (height above the leaves).
 *
 * Numeric: textbook left-looking column Cholesky on the column structures,
 * forward/backward substitution, FP64 iterative refinement (Sec. 2, pivot
 * perturbation "corrected through iterative refinements").
 *
 * Where the paper is silent (barrier/step rule, starting point, residual
 * scaling), this file follows Mehrotra's predictor-corrector and the
 * definitions stated at orc_ipm_lp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

static void *xmalloc(size_t n) {
  void *p = malloc((size_t)(n > 0 ? n : 1));
  return p;
}
static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------- */
/* Result of the symbolic analysis.                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  /* pattern of K (lower, incl. diagonal) in ORIGINAL numbering, CSC */
  int64_t *kop;
  int32_t *koi;
  /* final ordering (given permutation followed by the etree postorder): new->old */
  int32_t *perm;
  int32_t *iperm;
  /* pattern of K in FINAL numbering, lower CSC, and the map original entry -> final entry */
  int64_t *kp;
  int32_t *ki;
  int64_t *kmap;
  /* elimination tree and column structure of L (final numbering) */
  int32_t *parent;
  int32_t *colcount; /* including the diagonal */
  int64_t *lp;       /* strictly-below-diagonal structure of column j: li[lp[j] .. lp[j+1]) */
  int32_t *li;
  /* supernodes */
  int32_t nsuper;
  int32_t *super;   /* nsuper+1 first columns */
  int32_t *sparent; /* -1 for a root */
  int32_t *slevel;  /* 0 for a leaf, else 1 + max over children */
  int64_t *srp;     /* rows below each supernode's column block */
  int32_t *sri;
  int64_t nnz_l;    /* sum of column counts */
  double flops;     /* sum of colcount^2 (algorithmic factor flop count) */
} orc_sym;

ORC_EXPORT void orc_sym_free(orc_sym *s) {
  if (!s) return;
  free(s->kop); free(s->koi); free(s->perm); free(s->iperm); free(s->kp); free(s->ki);
  free(s->kmap); free(s->parent); free(s->colcount); free(s->lp); free(s->li);
  free(s->super); free(s->sparent); free(s->slevel); free(s->srp); free(s->sri);
  free(s);
}

/* Pattern of K = W + J^T J + I (lower triangle), original numbering.
 * Entry (i, j), i >= j, is present iff i == j, W has (i, j), or some row r of J
 * holds both columns i and j. Built by listing all pairs, sorting, deduplicating. */
static int build_k_pattern(int32_t n, int32_t m, const int64_t *jp, const int32_t *ji,
                           const int64_t *wp, const int32_t *wi, int64_t **kp_out,
                           int32_t **ki_out) {
  int64_t cnt = n;
  for (int32_t r = 0; r < m; r++) {
    int64_t k = jp[r + 1] - jp[r];
    cnt += k * (k + 1) / 2;
  }
  if (wp) cnt += wp[n];
  /* pairs encoded as (col * n + row) in int64 */
  int64_t *pairs = (int64_t *)xmalloc(sizeof(int64_t) * cnt);
  int64_t t = 0;
  for (int32_t j = 0; j < n; j++) pairs[t++] = (int64_t)j * n + j;
  for (int32_t r = 0; r < m; r++)
    for (int64_t a = jp[r]; a < jp[r + 1]; a++)
      for (int64_t b = jp[r]; b <= a; b++) {
        int32_t i = ji[a], j = ji[b];
        if (i < j) { int32_t tmp = i; i = j; j = tmp; }
        pairs[t++] = (int64_t)j * n + i;
      }
  if (wp)
    for (int32_t j = 0; j < n; j++)
      for (int64_t a = wp[j]; a < wp[j + 1]; a++) {
        int32_t i = wi[a], jj = j;
        if (i < jj) { int32_t tmp = i; i = jj; jj = tmp; }
        pairs[t++] = (int64_t)jj * n + i;
      }
  /* sort (simple qsort on int64) */
  int cmp64(const void *x, const void *y);
  qsort(pairs, (size_t)t, sizeof(int64_t), cmp64);
  int64_t u = 0;
  for (int64_t q = 0; q < t; q++)
    if (u == 0 || pairs[q] != pairs[u - 1]) pairs[u++] = pairs[q];
  int64_t *kp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  int32_t *ki = (int32_t *)xmalloc(sizeof(int32_t) * u);
  for (int64_t q = 0; q < u; q++) {
    int32_t j = (int32_t)(pairs[q] / n), i = (int32_t)(pairs[q] % n);
    kp[j + 1]++;
    ki[q] = i;
  }
  for (int32_t j = 0; j < n; j++) kp[j + 1] += kp[j];
  free(pairs);
  *kp_out = kp;
  *ki_out = ki;
  return 0;
}
int cmp64(const void *x, const void *y) {
  int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
  return (a > b) - (a < b);
}

/* Permute a lower CSC pattern: entry (i, j) of the original goes to
 * (max(ip[i], ip[j]), min(...)) of the result. Returns the result pattern
 * (rows sorted) and map[e] = position of original entry e in the result. */
static void permute_lower(int32_t n, const int64_t *p, const int32_t *ix, const int32_t *ip,
                          int64_t **pp_out, int32_t **pi_out, int64_t *map) {
  int64_t nz = p[n];
  int64_t *pp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = p[j]; e < p[j + 1]; e++) {
      int32_t a = ip[ix[e]], b = ip[j];
      int32_t col = a < b ? a : b;
      pp[col + 1]++;
    }
  for (int32_t j = 0; j < n; j++) pp[j + 1] += pp[j];
  int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)n + 1));
  memcpy(fill, pp, sizeof(int64_t) * ((size_t)n + 1));
  int32_t *pi = (int32_t *)xmalloc(sizeof(int32_t) * (nz ? nz : 1));
  int64_t *tmpmap = (int64_t *)xmalloc(sizeof(int64_t) * (nz ? nz : 1));
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = p[j]; e < p[j + 1]; e++) {
      int32_t a = ip[ix[e]], b = ip[j];
      int32_t col = a < b ? a : b, row = a < b ? b : a;
      int64_t q = fill[col]++;
      pi[q] = row;
      tmpmap[q] = e;
    }
  /* sort each column by row, carrying the map (insertion sort: columns are short) */
  for (int32_t j = 0; j < n; j++)
    for (int64_t q = pp[j] + 1; q < pp[j + 1]; q++) {
      int32_t r = pi[q];
      int64_t mm = tmpmap[q];
      int64_t z = q - 1;
      while (z >= pp[j] && pi[z] > r) { pi[z + 1] = pi[z]; tmpmap[z + 1] = tmpmap[z]; z--; }
      pi[z + 1] = r;
      tmpmap[z + 1] = mm;
    }
  if (map)
    for (int64_t q = 0; q < nz; q++) map[tmpmap[q]] = q;
  free(tmpmap);
  free(fill);
  *pp_out = pp;
  *pi_out = pi;
}

/* Elimination tree by Liu's algorithm with path compression, on a lower CSC
 * pattern. For each row i, every k < i with K(i, k) != 0 is walked up to its
 * current root r through the ancestor links (compressed to point at i); if
 * r != i then parent(r) = i. */
static void etree_liu(int32_t n, const int64_t *p, const int32_t *ix, int32_t *parent) {
  /* row lists of the strictly-lower part: for each row i, the columns k < i */
  int64_t *rp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = p[j]; e < p[j + 1]; e++)
      if (ix[e] > j) rp[ix[e] + 1]++;
  for (int32_t i = 0; i < n; i++) rp[i + 1] += rp[i];
  int32_t *rc = (int32_t *)xmalloc(sizeof(int32_t) * (rp[n] ? rp[n] : 1));
  int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)n + 1));
  memcpy(fill, rp, sizeof(int64_t) * ((size_t)n + 1));
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = p[j]; e < p[j + 1]; e++)
      if (ix[e] > j) rc[fill[ix[e]]++] = j;
  int32_t *anc = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t i = 0; i < n; i++) {
    parent[i] = -1;
    anc[i] = -1;
    for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
      int32_t k = rc[e];
      while (k != -1 && k != i) {
        int32_t next = anc[k];
        anc[k] = i;
        if (next == -1) { parent[k] = i; break; }
        k = next;
      }
    }
  }
  free(anc); free(fill); free(rc); free(rp);
}

/* Postorder of a forest: depth-first, children visited in ascending index,
 * roots in ascending index. post[k] = k-th node in postorder. */
static void postorder(int32_t n, const int32_t *parent, int32_t *post) {
  int32_t *head = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  int32_t *next = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  int32_t *stack = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t i = 0; i < n; i++) head[i] = -1;
  /* insert children in descending order so each list reads ascending */
  for (int32_t j = n - 1; j >= 0; j--)
    if (parent[j] != -1) { next[j] = head[parent[j]]; head[parent[j]] = j; }
  int32_t k = 0;
  for (int32_t r = 0; r < n; r++) {
    if (parent[r] != -1) continue;
    int32_t top = 0;
    stack[0] = r;
    while (top >= 0) {
      int32_t v = stack[top];
      int32_t c = head[v];
      if (c == -1) {
        post[k++] = v;
        top--;
      } else {
        head[v] = next[c];
        stack[++top] = c;
      }
    }
  }
  free(head); free(next); free(stack);
}

/* Relaxed amalgamation test for merging a child group into its parent.
 * ncol: merged column count; nrow: rows below the merged block;
 * ztrue: sum of the true column counts of both groups. */
static int amalgamate_ok(int64_t ncol, int64_t nrow, int64_t ztrue) {
  int64_t nz = ncol * (ncol + 1) / 2 + ncol * nrow;
  int64_t z = nz - ztrue;
  if (ncol <= 4) return 1;
  if (ncol <= 16 && 10 * z <= 8 * nz) return 1;
  if (ncol <= 48 && 10 * z <= nz) return 1;
  if (20 * z <= nz) return 1;
  return 0;
}

/* Full symbolic analysis. perm: new->old (NULL = identity). */
ORC_EXPORT orc_sym *orc_analyze(int32_t n, int32_t m, const int64_t *jp, const int32_t *ji,
                                const int64_t *wp, const int32_t *wi, const int32_t *perm_in) {
  orc_sym *S = (orc_sym *)xcalloc(1, sizeof(orc_sym));
  S->n = n;
  build_k_pattern(n, m, jp, ji, wp, wi, &S->kop, &S->koi);

  /* 1. permute by the given ordering and build the etree */
  int32_t *ip0 = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t k = 0; k < n; k++) ip0[perm_in ? perm_in[k] : k] = k;
  int64_t *p1; int32_t *i1;
  permute_lower(n, S->kop, S->koi, ip0, &p1, &i1, NULL);
  int32_t *par1 = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  etree_liu(n, p1, i1, par1);
  int32_t *post = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  postorder(n, par1, post);
  free(p1); free(i1); free(par1);

  /* 2. final ordering = given ordering followed by the postorder */
  S->perm = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  S->iperm = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t k = 0; k < n; k++) {
    int32_t mid = post[k];
    S->perm[k] = perm_in ? perm_in[mid] : mid;
  }
  for (int32_t k = 0; k < n; k++) S->iperm[S->perm[k]] = k;
  free(post); free(ip0);
  S->kmap = (int64_t *)xmalloc(sizeof(int64_t) * (S->kop[n] ? S->kop[n] : 1));
  permute_lower(n, S->kop, S->koi, S->iperm, &S->kp, &S->ki, S->kmap);
  S->parent = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  etree_liu(n, S->kp, S->ki, S->parent);

  /* 3. explicit column structures: struct(j) = {i > j : K(i,j)} U (U_children struct(c) \ {j}) */
  int32_t *mark = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t i = 0; i < n; i++) mark[i] = -1;
  int32_t *chead = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  int32_t *cnext = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  int32_t *nchild = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  for (int32_t i = 0; i < n; i++) chead[i] = -1;
  for (int32_t j = n - 1; j >= 0; j--)
    if (S->parent[j] != -1) {
      cnext[j] = chead[S->parent[j]];
      chead[S->parent[j]] = j;
      nchild[S->parent[j]]++;
    }
  S->lp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  int64_t cap = S->kp[n] + 16, used = 0;
  S->li = (int32_t *)xmalloc(sizeof(int32_t) * cap);
  int32_t *buf = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  S->colcount = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t j = 0; j < n; j++) {
    int32_t cnt = 0;
    mark[j] = j;
    for (int64_t e = S->kp[j]; e < S->kp[j + 1]; e++) {
      int32_t i = S->ki[e];
      if (mark[i] != j) { mark[i] = j; buf[cnt++] = i; }
    }
    for (int32_t c = chead[j]; c != -1; c = cnext[c])
      for (int64_t e = S->lp[c]; e < S->lp[c + 1]; e++) {
        int32_t i = S->li[e];
        if (mark[i] != j) { mark[i] = j; buf[cnt++] = i; }
      }
    qsort(buf, (size_t)cnt, sizeof(int32_t), cmp_i32);
    if (used + cnt > cap) {
      while (used + cnt > cap) cap *= 2;
      S->li = (int32_t *)realloc(S->li, sizeof(int32_t) * cap);
    }
    memcpy(S->li + used, buf, sizeof(int32_t) * cnt);
    used += cnt;
    S->lp[j + 1] = used;
    S->colcount[j] = cnt + 1;
  }
  free(buf);
  S->nnz_l = 0;
  S->flops = 0.0;
  for (int32_t j = 0; j < n; j++) {
    S->nnz_l += S->colcount[j];
    S->flops += (double)S->colcount[j] * (double)S->colcount[j];
  }

  /* 4. fundamental supernodes: j+1 joins j's supernode iff parent(j) = j+1,
   *    j is the only child of j+1, and count(j+1) = count(j) - 1 */
  int32_t *fstart = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t nf = 0;
  for (int32_t j = 0; j < n; j++) {
    int join = j > 0 && S->parent[j - 1] == j && nchild[j] == 1 &&
               S->colcount[j] == S->colcount[j - 1] - 1;
    if (!join) fstart[nf++] = j;
  }
  fstart[nf] = n;
  int32_t *fof = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1))); /* column -> fundamental sn */
  for (int32_t f = 0; f < nf; f++)
    for (int32_t j = fstart[f]; j < fstart[f + 1]; j++) fof[j] = f;

  /* 5. relaxed amalgamation over fundamental supernodes in column order */
  int32_t *gfirst = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(nf > 0 ? nf : 1)));
  int64_t *gtrue = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)(nf > 0 ? nf : 1)));
  int32_t *absorbed = (int32_t *)xcalloc((size_t)nf, sizeof(int32_t));
  for (int32_t f = 0; f < nf; f++) {
    gfirst[f] = fstart[f];
    gtrue[f] = 0;
    for (int32_t j = fstart[f]; j < fstart[f + 1]; j++) gtrue[f] += S->colcount[j];
  }
  for (int32_t f = 0; f < nf; f++) {
    int32_t last = fstart[f + 1] - 1;
    int32_t pc = S->parent[last];
    if (pc == -1) continue;
    int32_t P = fof[pc];
    if (last + 1 != fstart[P]) continue; /* only the child right before the parent is contiguous */
    int64_t ncol = (int64_t)(fstart[f + 1] - gfirst[f]) + (fstart[P + 1] - fstart[P]);
    int64_t nrow = S->colcount[fstart[P + 1] - 1] - 1;
    if (amalgamate_ok(ncol, nrow, gtrue[f] + gtrue[P])) {
      gfirst[P] = gfirst[f];
      gtrue[P] += gtrue[f];
      absorbed[f] = 1;
    }
  }
  S->nsuper = 0;
  for (int32_t f = 0; f < nf; f++) if (!absorbed[f]) S->nsuper++;
  S->super = (int32_t *)xmalloc(sizeof(int32_t) * (S->nsuper + 1));
  int32_t q = 0;
  for (int32_t f = 0; f < nf; f++) if (!absorbed[f]) S->super[q++] = gfirst[f];
  S->super[S->nsuper] = n;
  free(gfirst); free(gtrue); free(absorbed); free(fof); free(fstart);

  /* 6. supernode of each column, supernode parent and level */
  int32_t *sof = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t s = 0; s < S->nsuper; s++)
    for (int32_t j = S->super[s]; j < S->super[s + 1]; j++) sof[j] = s;
  S->sparent = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(S->nsuper > 0 ? S->nsuper : 1)));
  S->slevel = (int32_t *)xcalloc((size_t)S->nsuper, sizeof(int32_t));
  for (int32_t s = 0; s < S->nsuper; s++) {
    int32_t pc = S->parent[S->super[s + 1] - 1];
    S->sparent[s] = pc == -1 ? -1 : sof[pc];
  }
  for (int32_t s = 0; s < S->nsuper; s++) /* children precede parents */
    if (S->sparent[s] != -1 && S->slevel[S->sparent[s]] < S->slevel[s] + 1)
      S->slevel[S->sparent[s]] = S->slevel[s] + 1;

  /* 7. supernode row structure: explicit union of the column structures of its
   *    columns, minus its own columns */
  S->srp = (int64_t *)xcalloc((size_t)S->nsuper + 1, sizeof(int64_t));
  int64_t scap = 1024, sused = 0;
  S->sri = (int32_t *)xmalloc(sizeof(int32_t) * scap);
  int32_t *ubuf = (int32_t *)xmalloc(sizeof(int32_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t i = 0; i < n; i++) mark[i] = -1;
  for (int32_t s = 0; s < S->nsuper; s++) {
    int32_t c0 = S->super[s], c1 = S->super[s + 1], cnt = 0;
    for (int32_t j = c0; j < c1; j++)
      for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) {
        int32_t i = S->li[e];
        if (i >= c1 && mark[i] != s) { mark[i] = s; ubuf[cnt++] = i; }
      }
    qsort(ubuf, (size_t)cnt, sizeof(int32_t), cmp_i32);
    if (sused + cnt > scap) {
      while (sused + cnt > scap) scap *= 2;
      S->sri = (int32_t *)realloc(S->sri, sizeof(int32_t) * scap);
    }
    memcpy(S->sri + sused, ubuf, sizeof(int32_t) * cnt);
    sused += cnt;
    S->srp[s + 1] = sused;
  }
  free(ubuf); free(sof); free(mark); free(chead); free(cnext); free(nchild);
  return S;
}

/* accessors for the Python wrapper */
ORC_EXPORT int32_t orc_sym_n(const orc_sym *S) { return S->n; }
ORC_EXPORT int32_t orc_sym_nsuper(const orc_sym *S) { return S->nsuper; }
ORC_EXPORT int64_t orc_sym_nnz_korig(const orc_sym *S) { return S->kop[S->n]; }
ORC_EXPORT int64_t orc_sym_nnz_lstruct(const orc_sym *S) { return S->lp[S->n]; }
ORC_EXPORT int64_t orc_sym_nnz_srows(const orc_sym *S) { return S->srp[S->nsuper]; }
ORC_EXPORT int64_t orc_sym_nnz_l(const orc_sym *S) { return S->nnz_l; }
ORC_EXPORT double orc_sym_flops(const orc_sym *S) { return S->flops; }
ORC_EXPORT void orc_sym_export(const orc_sym *S, int64_t *kop, int32_t *koi, int32_t *perm,
                               int32_t *parent, int32_t *colcount, int64_t *lp, int32_t *li,
                               int32_t *super, int32_t *sparent, int32_t *slevel, int64_t *srp,
                               int32_t *sri) {
  int32_t n = S->n;
  if (kop) memcpy(kop, S->kop, sizeof(int64_t) * ((size_t)n + 1));
  if (koi) memcpy(koi, S->koi, sizeof(int32_t) * S->kop[n]);
  if (perm) memcpy(perm, S->perm, sizeof(int32_t) * n);
  if (parent) memcpy(parent, S->parent, sizeof(int32_t) * n);
  if (colcount) memcpy(colcount, S->colcount, sizeof(int32_t) * n);
  if (lp) memcpy(lp, S->lp, sizeof(int64_t) * ((size_t)n + 1));
  if (li) memcpy(li, S->li, sizeof(int32_t) * S->lp[n]);
  if (super) memcpy(super, S->super, sizeof(int32_t) * (S->nsuper + 1));
  if (sparent) memcpy(sparent, S->sparent, sizeof(int32_t) * S->nsuper);
  if (slevel) memcpy(slevel, S->slevel, sizeof(int32_t) * S->nsuper);
  if (srp) memcpy(srp, S->srp, sizeof(int64_t) * (S->nsuper + 1));
  if (sri) memcpy(sri, S->sri, sizeof(int32_t) * S->srp[S->nsuper]);
}

/* ------------------------------------------------------------------------- */
/* Numeric phase.                                                             */
/* ------------------------------------------------------------------------- */

/* Assembly of the primal condensed matrix (5):
 *   K = W + J^T diag(D) J + diag(dextra) + delta_p I
 * on the original lower pattern (kval[e] for entry e of kop/koi). J is m x n
 * CSR; dextra holds bound terms that act only on the diagonal. Products are
 * summed in ascending J row. Returns 0. */
ORC_EXPORT int orc_assemble(const orc_sym *S, int32_t m, const int64_t *jp, const int32_t *ji,
                            const double *jv, const double *D, const int64_t *wp,
                            const int32_t *wi, const double *wv, const double *dextra,
                            double delta_p, double *kval) {
  int32_t n = S->n;
  memset(kval, 0, sizeof(double) * S->kop[n]);
  /* locate entry (i, j) (i >= j) in column j by binary search */
#define KPOS(i_, j_, out_)                                     \
  do {                                                         \
    int64_t lo_ = S->kop[j_], hi_ = S->kop[(j_) + 1] - 1;      \
    while (lo_ < hi_) {                                        \
      int64_t mid_ = (lo_ + hi_) / 2;                          \
      if (S->koi[mid_] < (i_)) lo_ = mid_ + 1; else hi_ = mid_; \
    }                                                          \
    out_ = lo_;                                                \
  } while (0)
  if (wp)
    for (int32_t j = 0; j < n; j++)
      for (int64_t e = wp[j]; e < wp[j + 1]; e++) {
        int32_t i = wi[e], jj = j;
        if (i < jj) { int32_t t = i; i = jj; jj = t; }
        int64_t pos; KPOS(i, jj, pos);
        kval[pos] += wv[e];
      }
  for (int32_t r = 0; r < m; r++)
    for (int64_t a = jp[r]; a < jp[r + 1]; a++)
      for (int64_t b = jp[r]; b < jp[r + 1]; b++) {
        int32_t i = ji[a], j = ji[b];
        if (i < j) continue; /* lower triangle only */
        int64_t pos; KPOS(i, j, pos);
        kval[pos] += jv[a] * D[r] * jv[b];
      }
  for (int32_t j = 0; j < n; j++) {
    int64_t pos; KPOS(j, j, pos);
    kval[pos] += (dextra ? dextra[j] : 0.0) + delta_p;
  }
#undef KPOS
  return 0;
}

/* Left-looking column Cholesky K = L L^T in the final numbering.
 * L is stored by column: column j at lval[lp[j] + j] (diagonal first), then its
 * strictly-lower structure li[lp[j] .. lp[j+1]).
 * For j = 0..n-1: w = K(j:, j); for every k < j with L(j, k) != 0:
 * w -= L(j:, k) * L(j, k); then L(j, j) = sqrt(w_j), L(i, j) = w_i / L(j, j).
 * Returns 0, or 1 + the first column whose pivot is not positive. */
ORC_EXPORT int32_t orc_factor(const orc_sym *S, const double *kval_orig, double *lval) {
  int32_t n = S->n;
  /* K values in the final numbering */
  double *kf = (double *)xmalloc(sizeof(double) * (S->kp[n] ? S->kp[n] : 1));
  for (int64_t e = 0; e < S->kop[n]; e++) kf[S->kmap[e]] = kval_orig[e];
  /* row lists of L: for each row j, the columns k < j with L(j, k) != 0 */
  int64_t *rp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t e = 0; e < S->lp[n]; e++) rp[S->li[e] + 1]++;
  for (int32_t i = 0; i < n; i++) rp[i + 1] += rp[i];
  int32_t *rk = (int32_t *)xmalloc(sizeof(int32_t) * (S->lp[n] ? S->lp[n] : 1));
  int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)n + 1));
  memcpy(fill, rp, sizeof(int64_t) * ((size_t)n + 1));
  for (int32_t k = 0; k < n; k++)
    for (int64_t e = S->lp[k]; e < S->lp[k + 1]; e++) rk[fill[S->li[e]]++] = k;
  /* next[k]: position in column k's structure of the next row to be used */
  int64_t *next = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t k = 0; k < n; k++) next[k] = S->lp[k];
  double *w = (double *)xcalloc((size_t)n, sizeof(double));
  int32_t bad = 0;
  for (int32_t j = 0; j < n && !bad; j++) {
    for (int64_t e = S->kp[j]; e < S->kp[j + 1]; e++) w[S->ki[e]] = kf[e];
    for (int64_t t = rp[j]; t < rp[j + 1]; t++) {
      int32_t k = rk[t];
      int64_t pos = next[k]; /* li[pos] == j */
      double ljk = lval[S->lp[k] + k + 1 + (pos - S->lp[k])];
      w[j] -= ljk * ljk;
      for (int64_t e = pos + 1; e < S->lp[k + 1]; e++)
        w[S->li[e]] -= lval[S->lp[k] + k + 1 + (e - S->lp[k])] * ljk;
      next[k] = pos + 1;
    }
    double d = w[j];
    if (!(d > 0.0) || !isfinite(d)) { bad = j + 1; break; }
    double ljj = sqrt(d);
    double *col = lval + S->lp[j] + j;
    col[0] = ljj;
    w[j] = 0.0;
    for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) {
      col[1 + (e - S->lp[j])] = w[S->li[e]] / ljj;
      w[S->li[e]] = 0.0;
    }
  }
  free(w); free(next); free(fill); free(rk); free(rp); free(kf);
  return bad;
}

/* Left-looking LDL^T factorisation K = L D L^T (L unit lower) without pivoting,
 * for symmetric quasi-definite matrices such as the augmented system (4):
 * a quasi-definite matrix has such a factorisation for every symmetric
 * permutation, with the sign of each pivot fixed by the block its variable
 * belongs to (strong factorizability, Sec. 2). sign_orig[i] (original
 * numbering) is that expected sign (+1 or -1).
 * For j = 0..n-1: w = K(j:, j); for every k < j with L(j, k) != 0:
 * w -= L(j:, k) * L(j, k) * d_k; then d_j = w_j, L(i, j) = w_i / d_j.
 * L is stored like the Cholesky factor (unit diagonal in the diagonal slot),
 * d in dval (final numbering). Returns 0, or 1 + the first column whose pivot
 * is zero, not finite or of the wrong sign. */
ORC_EXPORT int32_t orc_factor_ldlt(const orc_sym *S, const double *kval_orig,
                                   const int8_t *sign_orig, double *lval, double *dval) {
  int32_t n = S->n;
  double *kf = (double *)xmalloc(sizeof(double) * (S->kp[n] ? S->kp[n] : 1));
  for (int64_t e = 0; e < S->kop[n]; e++) kf[S->kmap[e]] = kval_orig[e];
  int64_t *rp = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t e = 0; e < S->lp[n]; e++) rp[S->li[e] + 1]++;
  for (int32_t i = 0; i < n; i++) rp[i + 1] += rp[i];
  int32_t *rk = (int32_t *)xmalloc(sizeof(int32_t) * (S->lp[n] ? S->lp[n] : 1));
  int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)n + 1));
  memcpy(fill, rp, sizeof(int64_t) * ((size_t)n + 1));
  for (int32_t k = 0; k < n; k++)
    for (int64_t e = S->lp[k]; e < S->lp[k + 1]; e++) rk[fill[S->li[e]]++] = k;
  int64_t *next = (int64_t *)xmalloc(sizeof(int64_t) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t k = 0; k < n; k++) next[k] = S->lp[k];
  double *w = (double *)xcalloc((size_t)n, sizeof(double));
  int32_t bad = 0;
  for (int32_t j = 0; j < n && !bad; j++) {
    for (int64_t e = S->kp[j]; e < S->kp[j + 1]; e++) w[S->ki[e]] = kf[e];
    for (int64_t t = rp[j]; t < rp[j + 1]; t++) {
      int32_t k = rk[t];
      int64_t pos = next[k]; /* li[pos] == j */
      double ljk = lval[S->lp[k] + k + 1 + (pos - S->lp[k])];
      double f = ljk * dval[k];
      w[j] -= ljk * f;
      for (int64_t e = pos + 1; e < S->lp[k + 1]; e++)
        w[S->li[e]] -= lval[S->lp[k] + k + 1 + (e - S->lp[k])] * f;
      next[k] = pos + 1;
    }
    double d = w[j];
    int8_t sg = sign_orig[S->perm[j]];
    if (!isfinite(d) || !(sg > 0 ? d > 0.0 : d < 0.0)) { bad = j + 1; break; }
    dval[j] = d;
    double *col = lval + S->lp[j] + j;
    col[0] = 1.0;
    w[j] = 0.0;
    for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) {
      col[1 + (e - S->lp[j])] = w[S->li[e]] / d;
      w[S->li[e]] = 0.0;
    }
  }
  free(w); free(next); free(fill); free(rk); free(rp); free(kf);
  return bad;
}

/* Solve K x = b with K = P^T L D L^T P: y = L^{-1} P b, y ./= d, z = L^{-T} y,
 * x = P^T z (b, x in the ORIGINAL numbering). */
ORC_EXPORT void orc_solve_ldlt(const orc_sym *S, const double *lval, const double *dval,
                               const double *b, double *x) {
  int32_t n = S->n;
  double *y = (double *)xmalloc(sizeof(double) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t k = 0; k < n; k++) y[k] = b[S->perm[k]];
  for (int32_t j = 0; j < n; j++) {
    const double *col = lval + S->lp[j] + j;
    for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) y[S->li[e]] -= col[1 + (e - S->lp[j])] * y[j];
  }
  for (int32_t j = 0; j < n; j++) y[j] /= dval[j];
  for (int32_t j = n - 1; j >= 0; j--) {
    const double *col = lval + S->lp[j] + j;
    double t = y[j];
    for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) t -= col[1 + (e - S->lp[j])] * y[S->li[e]];
    y[j] = t;
  }
  for (int32_t k = 0; k < n; k++) x[S->perm[k]] = y[k];
  free(y);
}

/* Solve K x = b with the factor: b, x in the ORIGINAL numbering.
 * y = L^{-1} P b (forward), z = L^{-T} y (backward), x = P^T z. */
ORC_EXPORT void orc_solve(const orc_sym *S, const double *lval, const double *b, double *x) {
  int32_t n = S->n;
  double *y = (double *)xmalloc(sizeof(double) * ((size_t)(n > 0 ? n : 1)));
  for (int32_t k = 0; k < n; k++) y[k] = b[S->perm[k]];
  for (int32_t j = 0; j < n; j++) {
    const double *col = lval + S->lp[j] + j;
    y[j] /= col[0];
    for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) y[S->li[e]] -= col[1 + (e - S->lp[j])] * y[j];
  }
  for (int32_t j = n - 1; j >= 0; j--) {
    const double *col = lval + S->lp[j] + j;
    double t = y[j];
    for (int64_t e = S->lp[j]; e < S->lp[j + 1]; e++) t -= col[1 + (e - S->lp[j])] * y[S->li[e]];
    y[j] = t / col[0];
  }
  for (int32_t k = 0; k < n; k++) x[S->perm[k]] = y[k];
  free(y);
}

/* y = K x with K given by its lower pattern values (original numbering). */
ORC_EXPORT void orc_kmatvec(const orc_sym *S, const double *kval, const double *x, double *y) {
  int32_t n = S->n;
  for (int32_t i = 0; i < n; i++) y[i] = 0.0;
  for (int32_t j = 0; j < n; j++)
    for (int64_t e = S->kop[j]; e < S->kop[j + 1]; e++) {
      int32_t i = S->koi[e];
      y[i] += kval[e] * x[j];
      if (i != j) y[j] += kval[e] * x[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Interior-point method for the LP  min c^T x  s.t.  A x >= b,  l <= x <= u.  */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t max_iter;
  int32_t ir_max;      /* iterative-refinement steps per solve (at most) */
  double tol;          /* KKT residual tolerance */
  double delta_p;      /* primal regularisation of (3) */
  double delta_d;      /* dual regularisation of (3) */
  double ir_tol;       /* stop refining once ||b - K x|| <= ir_tol ||b|| */
} orc_ipm_opts;

typedef struct {
  int32_t status;      /* 0 converged, 1 iteration limit, 2 factorisation failure, 3 non-finite iterate */
  int32_t iterations;
  int32_t refactorizations;
  double objective;
  double kkt;          /* final scaled KKT residual */
  double primal_res, dual_res, compl_res, mu;
} orc_ipm_result;

/* The LP's constraint function g = J x - bfull with J = [A; I_l; -I_u]:
 * rows 0..m-1 are A x - b, rows m..m+nl-1 are x_i - l_i for the finite l_i
 * (ascending i), rows m+nl..mt-1 are u_i - x_i for the finite u_i. */
typedef struct {
  int32_t n, m, nl, nu;
  int64_t mt;
  const int64_t *ap;
  const int32_t *ai;
  const double *av, *b, *c, *l, *u;
  const int64_t *wp;  /* Hessian W of f (lower CSC), NULL for an LP */
  const int32_t *wi;
  const double *wv;
  int32_t *lidx, *uidx;
} lp_rows;

static void lp_rows_init(lp_rows *P, int32_t n, int32_t m, const int64_t *ap, const int32_t *ai,
                         const double *av, const double *b, const double *c, const double *l,
                         const double *u) {
  P->n = n; P->m = m; P->ap = ap; P->ai = ai; P->av = av; P->b = b; P->c = c; P->l = l; P->u = u;
  P->wp = NULL; P->wi = NULL; P->wv = NULL;
  P->nl = P->nu = 0;
  for (int32_t i = 0; i < n; i++) { if (isfinite(l[i])) P->nl++; if (isfinite(u[i])) P->nu++; }
  P->mt = (int64_t)m + P->nl + P->nu;
  P->lidx = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(P->nl > 0 ? P->nl : 1));
  P->uidx = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(P->nu > 0 ? P->nu : 1));
  int32_t a = 0, q = 0;
  for (int32_t i = 0; i < n; i++) { if (isfinite(l[i])) P->lidx[a++] = i; if (isfinite(u[i])) P->uidx[q++] = i; }
}
static void lp_rows_free(lp_rows *P) { free(P->lidx); free(P->uidx); }

/* out (length mt) = J v */
static void lp_jv(const lp_rows *P, const double *v, double *out) {
  for (int32_t r = 0; r < P->m; r++) {
    double a = 0.0;
    for (int64_t e = P->ap[r]; e < P->ap[r + 1]; e++) a += P->av[e] * v[P->ai[e]];
    out[r] = a;
  }
  for (int32_t k = 0; k < P->nl; k++) out[P->m + k] = v[P->lidx[k]];
  for (int32_t k = 0; k < P->nu; k++) out[P->m + P->nl + k] = -v[P->uidx[k]];
}
/* out (length n) = J^T v */
static void lp_jtv(const lp_rows *P, const double *v, double *out) {
  for (int32_t i = 0; i < P->n; i++) out[i] = 0.0;
  for (int32_t r = 0; r < P->m; r++)
    for (int64_t e = P->ap[r]; e < P->ap[r + 1]; e++) out[P->ai[e]] += P->av[e] * v[r];
  for (int32_t k = 0; k < P->nl; k++) out[P->lidx[k]] += v[P->m + k];
  for (int32_t k = 0; k < P->nu; k++) out[P->uidx[k]] -= v[P->m + P->nl + k];
}
/* out (length n) = W x for the symmetric W given by its lower triangle (0 without W) */
static void lp_wx(const lp_rows *P, const double *x, double *out) {
  for (int32_t i = 0; i < P->n; i++) out[i] = 0.0;
  if (!P->wp) return;
  for (int32_t j = 0; j < P->n; j++)
    for (int64_t e = P->wp[j]; e < P->wp[j + 1]; e++) {
      const int32_t i = P->wi[e];
      out[i] += P->wv[e] * x[j];
      if (i != j) out[j] += P->wv[e] * x[i];
    }
}

/* g(x) = J x - bfull */
static void lp_g(const lp_rows *P, const double *x, double *g) {
  lp_jv(P, x, g);
  for (int32_t r = 0; r < P->m; r++) g[r] -= P->b[r];
  for (int32_t k = 0; k < P->nl; k++) g[P->m + k] -= P->l[P->lidx[k]];
  for (int32_t k = 0; k < P->nu; k++) g[P->m + P->nl + k] += P->u[P->uidx[k]];
}

static double inf_norm(const double *v, int64_t k) {
  double r = 0.0;
  for (int64_t i = 0; i < k; i++) { double a = fabs(v[i]); if (a > r) r = a; }
  return r;
}

/* Largest alpha in (0, 1] with v + alpha * dv >= (1 - tau) v  (fraction to the
 * boundary): min over dv_i < 0 of -tau v_i / dv_i, capped at 1. */
static double step_to_boundary(const double *v, const double *dv, int64_t k, double tau) {
  double a = 1.0;
  for (int64_t i = 0; i < k; i++)
    if (dv[i] < 0.0) { double t = -tau * v[i] / dv[i]; if (t < a) a = t; }
  return a;
}

/* D = (delta_d + s ./ lambda)^{-1}, and the bound rows' share of J^T D J,
 * which acts on the diagonal only. */
static void lp_scaling(const lp_rows *P, const double *s, const double *lam, double delta_d,
                       double *D, double *dextra) {
  for (int64_t k = 0; k < P->mt; k++) D[k] = 1.0 / (delta_d + s[k] / lam[k]);
  for (int32_t i = 0; i < P->n; i++) dextra[i] = 0.0;
  for (int32_t k = 0; k < P->nl; k++) dextra[P->lidx[k]] += D[P->m + k];
  for (int32_t k = 0; k < P->nu; k++) dextra[P->uidx[k]] += D[P->m + P->nl + k];
}

/* One Newton direction of (3) through the condensed system (5), with the
 * factor of K already computed:
 *   r_p = (c - J^T lambda) + J^T D (g - w ./ lambda),   K d_x = -r_p  (+ FP64 refinement),
 *   d_lambda = D (w ./ lambda - g - J d_x),
 *   d_s = -s + w ./ lambda - (s ./ lambda) .* d_lambda. */
static void lp_direction(const orc_sym *S, const lp_rows *P, const double *kval,
                         const double *lval, const double *xcur, const double *g, const double *s,
                         const double *lam, const double *D, const double *w, int32_t ir_max,
                         double ir_tol, double *dx, double *ds, double *dl, double *work_n3,
                         double *work_mt) {
  int32_t n = P->n;
  int64_t mt = P->mt;
  double *rp = work_n3, *r = work_n3 + n, *cx = work_n3 + 2 * (int64_t)n;
  for (int64_t k = 0; k < mt; k++) work_mt[k] = D[k] * (g[k] - w[k] / lam[k]) - lam[k];
  lp_jtv(P, work_mt, rp); /* J^T (D (g - w/lambda) - lambda) */
  lp_wx(P, xcur, r);      /* grad f = c + W x */
  for (int32_t i = 0; i < n; i++) rp[i] = -(P->c[i] + r[i] + rp[i]);
  orc_solve(S, lval, rp, dx);
  double bn = inf_norm(rp, n);
  for (int32_t ir = 0; ir < ir_max; ir++) {
    orc_kmatvec(S, kval, dx, cx);
    for (int32_t i = 0; i < n; i++) r[i] = rp[i] - cx[i];
    if (inf_norm(r, n) <= ir_tol * bn) break;
    orc_solve(S, lval, r, cx);
    for (int32_t i = 0; i < n; i++) dx[i] += cx[i];
  }
  lp_jv(P, dx, work_mt);
  for (int64_t k = 0; k < mt; k++) {
    dl[k] = D[k] * (w[k] / lam[k] - g[k] - work_mt[k]);
    ds[k] = -s[k] + w[k] / lam[k] - (s[k] / lam[k]) * dl[k];
  }
}

/* Exported for the tests: the Newton direction at (x, s, lambda) with the
 * complementarity target w (length mt). Returns 0, or 1 + the failing column. */
ORC_EXPORT int32_t orc_lp_direction(const orc_sym *S, int32_t m, const int64_t *ap,
                                    const int32_t *ai, const double *av, const double *b,
                                    const double *c, const double *l, const double *u,
                                    const double *x, const double *s, const double *lam,
                                    const double *w, double delta_p, double delta_d,
                                    int32_t ir_max, const int64_t *wp, const int32_t *wi,
                                    const double *wv, double *dx, double *ds, double *dl) {
  lp_rows P;
  lp_rows_init(&P, S->n, m, ap, ai, av, b, c, l, u);
  P.wp = wp; P.wi = wi; P.wv = wv;
  int32_t n = S->n;
  double *g = (double *)xmalloc(sizeof(double) * (size_t)P.mt);
  double *D = (double *)xmalloc(sizeof(double) * (size_t)P.mt);
  double *wmt = (double *)xmalloc(sizeof(double) * (size_t)P.mt);
  double *dextra = (double *)xmalloc(sizeof(double) * (size_t)n);
  double *wn3 = (double *)xmalloc(sizeof(double) * 3 * (size_t)n);
  double *kval = (double *)xmalloc(sizeof(double) * (size_t)S->kop[n]);
  double *lval = (double *)xmalloc(sizeof(double) * (size_t)S->nnz_l);
  lp_g(&P, x, g);
  lp_scaling(&P, s, lam, delta_d, D, dextra);
  orc_assemble(S, m, ap, ai, av, D, wp, wi, wv, dextra, delta_p, kval);
  int32_t bad = orc_factor(S, kval, lval);
  if (!bad) lp_direction(S, &P, kval, lval, x, g, s, lam, D, w, ir_max, 1e-14, dx, ds, dl, wn3, wmt);
  free(g); free(D); free(wmt); free(dextra); free(wn3); free(kval); free(lval);
  lp_rows_free(&P);
  return bad;
}

/* Mehrotra predictor-corrector IPM on the primal condensed system (5).
 *
 * Starting point: x_i = (l_i+u_i)/2 if both bounds are finite, max(0, l_i+1)
 * if only l_i is, min(0, u_i-1) if only u_i is, else 0; s = max(g(x), 1);
 * lambda = 1.
 * Scaled KKT residual (from the conditions (2)):
 *   max( ||g - s||_inf / max(1, ||bfull||_inf),
 *        ||c - J^T lambda||_inf / max(1, ||c||_inf),
 *        ||s .* lambda||_inf / max(1, |c^T x|) ),
 * where bfull = [b; l_finite; -u_finite] so that g = J x - bfull.
 * Each iteration: D = (delta_d + s ./ lambda)^{-1}; factor K; predictor with
 * w = 0; mu_aff from the affine step lengths; sigma = (mu_aff / mu)^3;
 * corrector with w = sigma mu - d_s_aff .* d_lambda_aff; step lengths with
 * tau = max(0.99, 1 - mu), separately for (x, s) and lambda.
 * A non-positive pivot multiplies delta_p by 100 and refactors (at most 12
 * times per iteration). */
ORC_EXPORT int orc_ipm_lp(const orc_sym *S, int32_t m, const int64_t *ap, const int32_t *ai,
                          const double *av, const double *b, const double *c, const double *l,
                          const double *u, const int64_t *wp, const int32_t *wi,
                          const double *wv, const orc_ipm_opts *o, double *x, double *s_out,
                          double *lam_out, orc_ipm_result *res, double *log_mu,
                          double *log_kkt) {
  int32_t n = S->n;
  lp_rows P;
  lp_rows_init(&P, n, m, ap, ai, av, b, c, l, u);
  P.wp = wp; P.wi = wi; P.wv = wv;
  int64_t mt = P.mt;
  size_t zmt = (size_t)(mt > 0 ? mt : 1), zn = (size_t)(n > 0 ? n : 1);
  double *s = (double *)xmalloc(sizeof(double) * zmt), *lam = (double *)xmalloc(sizeof(double) * zmt);
  double *g = (double *)xmalloc(sizeof(double) * zmt), *D = (double *)xmalloc(sizeof(double) * zmt);
  double *w = (double *)xmalloc(sizeof(double) * zmt), *wmt = (double *)xmalloc(sizeof(double) * zmt);
  double *dl = (double *)xmalloc(sizeof(double) * zmt), *ds = (double *)xmalloc(sizeof(double) * zmt);
  double *rd = (double *)xmalloc(sizeof(double) * zn), *dx = (double *)xmalloc(sizeof(double) * zn);
  double *dextra = (double *)xmalloc(sizeof(double) * zn);
  double *wn3 = (double *)xmalloc(sizeof(double) * 3 * zn);
  double *kval = (double *)xmalloc(sizeof(double) * (size_t)S->kop[n]);
  double *lval = (double *)xmalloc(sizeof(double) * (size_t)(S->nnz_l ? S->nnz_l : 1));

  double bscale = inf_norm(b, m);
  for (int32_t k = 0; k < P.nl; k++) if (fabs(l[P.lidx[k]]) > bscale) bscale = fabs(l[P.lidx[k]]);
  for (int32_t k = 0; k < P.nu; k++) if (fabs(u[P.uidx[k]]) > bscale) bscale = fabs(u[P.uidx[k]]);
  bscale = bscale > 1.0 ? bscale : 1.0;
  double cscale = inf_norm(c, n);
  cscale = cscale > 1.0 ? cscale : 1.0;

  for (int32_t i = 0; i < n; i++) {
    int fl = isfinite(l[i]), fu = isfinite(u[i]);
    if (fl && fu) x[i] = 0.5 * (l[i] + u[i]);
    else if (fl) x[i] = l[i] + 1.0 > 0.0 ? l[i] + 1.0 : 0.0;
    else if (fu) x[i] = u[i] - 1.0 < 0.0 ? u[i] - 1.0 : 0.0;
    else x[i] = 0.0;
  }
  lp_g(&P, x, g);
  for (int64_t k = 0; k < mt; k++) { s[k] = g[k] > 1.0 ? g[k] : 1.0; lam[k] = 1.0; }

  double delta_p = o->delta_p;
  res->status = 1;
  res->refactorizations = 0;
  int32_t it;
  for (it = 0; it <= o->max_iter; it++) {
    lp_g(&P, x, g);
    lp_jtv(&P, lam, rd);
    lp_wx(&P, x, dx); /* dx used as scratch for W x here */
    for (int32_t i = 0; i < n; i++) rd[i] = c[i] + dx[i] - rd[i];
    double mu = 0.0, fx = 0.0, pr = 0.0, cr = 0.0;
    for (int64_t k = 0; k < mt; k++) {
      mu += s[k] * lam[k];
      double a = fabs(g[k] - s[k]); if (a > pr) pr = a;
      double q = fabs(s[k] * lam[k]); if (q > cr) cr = q;
    }
    mu /= (double)(mt ? mt : 1);
    for (int32_t i = 0; i < n; i++) fx += (c[i] + 0.5 * dx[i]) * x[i]; /* c^T x + x^T W x / 2 */
    double dr = inf_norm(rd, n);
    double fs = fabs(fx) > 1.0 ? fabs(fx) : 1.0;
    double kkt = pr / bscale;
    if (dr / cscale > kkt) kkt = dr / cscale;
    if (cr / fs > kkt) kkt = cr / fs;
    res->objective = fx; res->kkt = kkt; res->mu = mu;
    res->primal_res = pr / bscale; res->dual_res = dr / cscale; res->compl_res = cr / fs;
    if (log_mu) log_mu[it] = mu;
    if (log_kkt) log_kkt[it] = kkt;
    /* the maxima above skip NaN, the sums do not: a non-finite iterate cannot
       satisfy the KKT conditions (2) */
    if (!isfinite(fx) || !isfinite(mu)) { res->status = 3; break; }
    if (kkt <= o->tol) { res->status = 0; break; }
    if (it == o->max_iter) break;

    lp_scaling(&P, s, lam, o->delta_d, D, dextra);
    int32_t bad = 1, tries = 0;
    while (bad) {
      orc_assemble(S, m, ap, ai, av, D, wp, wi, wv, dextra, delta_p, kval);
      bad = orc_factor(S, kval, lval);
      if (bad) {
        res->refactorizations++;
        delta_p *= 100.0;
        if (++tries > 12) { res->status = 2; goto done; }
      }
    }
    /* predictor: w = 0 */
    for (int64_t k = 0; k < mt; k++) w[k] = 0.0;
    lp_direction(S, &P, kval, lval, x, g, s, lam, D, w, o->ir_max, o->ir_tol, dx, ds, dl, wn3, wmt);
    double apa = step_to_boundary(s, ds, mt, 1.0), ada = step_to_boundary(lam, dl, mt, 1.0);
    double mua = 0.0;
    for (int64_t k = 0; k < mt; k++) mua += (s[k] + apa * ds[k]) * (lam[k] + ada * dl[k]);
    mua /= (double)mt;
    double sigma = mua / mu;
    sigma = sigma * sigma * sigma;
    /* corrector: w = sigma mu - d_s_aff .* d_lambda_aff */
    for (int64_t k = 0; k < mt; k++) w[k] = sigma * mu - ds[k] * dl[k];
    lp_direction(S, &P, kval, lval, x, g, s, lam, D, w, o->ir_max, o->ir_tol, dx, ds, dl, wn3, wmt);
    double tau = 1.0 - mu > 0.99 ? 1.0 - mu : 0.99;
    double alpha_p = step_to_boundary(s, ds, mt, tau), alpha_d = step_to_boundary(lam, dl, mt, tau);
    for (int32_t i = 0; i < n; i++) x[i] += alpha_p * dx[i];
    for (int64_t k = 0; k < mt; k++) { s[k] += alpha_p * ds[k]; lam[k] += alpha_d * dl[k]; }
  }
done:
  res->iterations = it;
  if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)mt);
  if (lam_out) memcpy(lam_out, lam, sizeof(double) * (size_t)mt);
  free(s); free(lam); free(g); free(D); free(w); free(wmt); free(dl); free(ds); free(rd);
  free(dx); free(dextra); free(wn3); free(kval); free(lval);
  lp_rows_free(&P);
  return res->status;
}
