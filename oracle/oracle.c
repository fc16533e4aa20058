/*
 * oracle.c -- plain, slow, obviously correct CPU reference for sparse Cholesky.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the bench's CPU-baseline
 * leg call this file through oracle/__init__.py; the library (include/chol.h and the
 * package) never includes, links or calls it, and it shares no code with them.
 *
 * Everything is IEEE double, one thread, no blocking and no reordering beyond what the
 * definitions below state.  What it computes is fixed by the paper:
 *   - A = L L^T with L lower triangular (Sec. 1), for the symmetrically permuted
 *     matrix B = P^T A P (the analysis phase reorders rows and columns, Sec. 2);
 *   - the solve phase solves L y = b then L^T x = y (Sec. 1, Sec. 2);
 *   - the analysis phase builds the elimination tree and merges adjacent columns into
 *     supernodes (Sec. 2); the parallel factorization runs supernodes whose subtrees
 *     are done at the same time (Sec. 3, Fig. 1), which gives the level sets below;
 *   - the factorization is left-looking: a column first receives the updates of the
 *     columns to its left, then is factored (Sec. 3, Listing 1).
 * Where the paper gives no formula the textbook definition is written out:
 *   struct(L_j) = struct(B_{j:n,j}) U  union over children k of (struct(L_k) \ {k}),
 *   parent(j)   = min { i > j : i in struct(L_j) }                (elimination tree)
 *   L_jj = sqrt(b_jj - sum_{k<j} L_jk^2),
 *   L_ij = (b_ij - sum_{k<j} L_ik L_jk) / L_jj                      (column Cholesky)
 * Every function returns 0 on success and a negative code on invalid input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

typedef struct { int32_t row; double val; } orc_entry;

static int orc_cmp_entry(const void* a, const void* b) {
  int32_t x = ((const orc_entry*)a)->row, y = ((const orc_entry*)b)->row;
  return (x > y) - (x < y);
}
static int orc_cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* B = P^T A P, both as lower CSC; perm[new] = old, so B[i][j] = A[perm[i]][perm[j]].
 * Rejects upper-triangle entries, out-of-range or duplicate rows, and a perm that is
 * not a permutation. */
int orc_permute(int64_t n, const int64_t* Ap, const int32_t* Ai, const double* Ax,
                const int32_t* perm, int64_t* Bp, int32_t* Bi, double* Bx) {
  int64_t nnz = Ap[n];
  int32_t* iperm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  orc_entry* tmp = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)(nnz > 0 ? nnz : 1));
  int rc = 0;
  if (!iperm || !cnt || !tmp) { rc = ORC_ENOMEM; goto done; }
  for (int64_t i = 0; i < n; i++) iperm[i] = -1;
  for (int64_t i = 0; i < n; i++) {
    if (perm[i] < 0 || perm[i] >= n || iperm[perm[i]] != -1) { rc = ORC_EINVAL; goto done; }
    iperm[perm[i]] = (int32_t)i;
  }
  for (int64_t j = 0; j < n; j++) {
    for (int64_t p = Ap[j]; p < Ap[j + 1]; p++) {
      int64_t i = Ai[p];
      if (i < j || i >= n) { rc = ORC_EINVAL; goto done; }
      if (p > Ap[j] && Ai[p - 1] >= i) { rc = ORC_EINVAL; goto done; }
      int32_t a = iperm[i], b = iperm[j];
      cnt[(a < b ? a : b) + 1]++;
    }
  }
  for (int64_t j = 0; j < n; j++) cnt[j + 1] += cnt[j];
  memcpy(Bp, cnt, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t j = 0; j < n; j++) {
    for (int64_t p = Ap[j]; p < Ap[j + 1]; p++) {
      int32_t a = iperm[Ai[p]], b = iperm[j];
      int32_t c = a < b ? a : b, r = a < b ? b : a;
      tmp[cnt[c]].row = r;
      tmp[cnt[c]].val = Ax[p];
      cnt[c]++;
    }
  }
  for (int64_t j = 0; j < n; j++) {
    qsort(tmp + Bp[j], (size_t)(Bp[j + 1] - Bp[j]), sizeof(orc_entry), orc_cmp_entry);
    for (int64_t p = Bp[j]; p < Bp[j + 1]; p++) { Bi[p] = tmp[p].row; Bx[p] = tmp[p].val; }
  }
done:
  free(iperm); free(cnt); free(tmp);
  return rc;
}

/* Symbolic factorization by the column-union rule (header).  Allocates the pattern
 * Li (sorted rows, diagonal first) with malloc; the caller frees it with orc_free.
 * parent[j] = -1 for a root.  colcount[j] = |struct(L_j)| including the diagonal. */
int orc_symbolic(int64_t n, const int64_t* Bp, const int32_t* Bi, int32_t* parent,
                 int64_t* colcount, int64_t* Lp, int32_t** Li_out) {
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t cap = Bp[n] + n + 16, len = 0;
  int32_t* Li = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  if (!mark || !head || !next || !Li) { free(mark); free(head); free(next); free(Li); return ORC_ENOMEM; }
  for (int64_t i = 0; i < n; i++) { mark[i] = -1; head[i] = -1; next[i] = -1; }
  Lp[0] = 0;
  for (int64_t j = 0; j < n; j++) {
    /* column j can hold at most n - j rows */
    if (len + (n - j) > cap) {
      int64_t ncap = cap * 2 > len + (n - j) ? cap * 2 : len + (n - j);
      int32_t* t = (int32_t*)realloc(Li, sizeof(int32_t) * (size_t)ncap);
      if (!t) { free(mark); free(head); free(next); free(Li); return ORC_ENOMEM; }
      Li = t; cap = ncap;
    }
    int64_t start = len;
    Li[len++] = (int32_t)j;
    mark[j] = (int32_t)j;
    for (int64_t p = Bp[j]; p < Bp[j + 1]; p++) {
      int32_t i = Bi[p];
      if (mark[i] != j) { mark[i] = (int32_t)j; Li[len++] = i; }
    }
    for (int32_t k = head[j]; k != -1; k = next[k]) {
      for (int64_t p = Lp[k]; p < Lp[k + 1]; p++) {
        int32_t i = Li[p];
        if (i != k && mark[i] != j) { mark[i] = (int32_t)j; Li[len++] = i; }
      }
    }
    qsort(Li + start, (size_t)(len - start), sizeof(int32_t), orc_cmp_i32);
    Lp[j + 1] = len;
    colcount[j] = len - start;
    parent[j] = (len - start > 1) ? Li[start + 1] : -1;
    if (parent[j] != -1) { next[j] = head[parent[j]]; head[parent[j]] = (int32_t)j; }
  }
  free(mark); free(head); free(next);
  *Li_out = Li;
  return 0;
}

void orc_free(void* p) { free(p); }

/* Supernode partition.  Column j+1 joins the supernode of j iff parent(j) = j+1,
 * colcount(j+1) = colcount(j) - 1 and j+1 has exactly one child (fundamental
 * supernodes); each is then cut from the left into pieces of at most W columns.
 * Writes sn_start[0..ns] and returns ns through *ns_out.  sn_parent[s] is the
 * supernode holding parent(last column of s) (-1 at a root).  level[s] = 0 for a
 * supernode with no children, else 1 + the largest level of its children: the level
 * sets are the groups that may run at the same time (Sec. 3, Fig. 1). */
int orc_supernodes(int64_t n, const int32_t* parent, const int64_t* colcount, int64_t W,
                   int32_t* sn_start, int32_t* sn_parent, int32_t* level, int64_t* ns_out) {
  if (W < 1) return ORC_EINVAL;
  int32_t* nchild = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  int32_t* sn_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!nchild || !sn_of) { free(nchild); free(sn_of); return ORC_ENOMEM; }
  for (int64_t j = 0; j < n; j++) if (parent[j] >= 0) nchild[parent[j]]++;
  int64_t ns = 0, width = 0;
  for (int64_t j = 0; j < n; j++) {
    int joins = j > 0 && parent[j - 1] == j && colcount[j] == colcount[j - 1] - 1 &&
                nchild[j] == 1;
    if (!joins || width == W) { sn_start[ns++] = (int32_t)j; width = 0; }
    sn_of[j] = (int32_t)(ns - 1);
    width++;
  }
  sn_start[ns] = (int32_t)n;
  for (int64_t s = 0; s < ns; s++) {
    int32_t last = sn_start[s + 1] - 1;
    sn_parent[s] = parent[last] >= 0 ? sn_of[parent[last]] : -1;
    level[s] = 0;
  }
  for (int64_t s = 0; s < ns; s++)
    if (sn_parent[s] >= 0 && level[sn_parent[s]] < level[s] + 1) level[sn_parent[s]] = level[s] + 1;
  *ns_out = ns;
  free(nchild); free(sn_of);
  return 0;
}

/* Row lists of L: for every row i, the (column k < i, position of L_ik) pairs, k
 * ascending.  Used by the left-looking loop to visit the columns that update j. */
static int orc_rowlists(int64_t n, const int64_t* Lp, const int32_t* Li, int64_t** Rp_out,
                        int64_t** Rq_out, int32_t** Rk_out) {
  int64_t* Rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t m = Lp[n] - n;
  int64_t* Rq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  int32_t* Rk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!Rp || !Rq || !Rk || !fill) { free(Rp); free(Rq); free(Rk); free(fill); return ORC_ENOMEM; }
  for (int64_t k = 0; k < n; k++)
    for (int64_t p = Lp[k] + 1; p < Lp[k + 1]; p++) Rp[Li[p] + 1]++;
  for (int64_t i = 0; i < n; i++) Rp[i + 1] += Rp[i];
  memcpy(fill, Rp, sizeof(int64_t) * (size_t)n);
  for (int64_t k = 0; k < n; k++)
    for (int64_t p = Lp[k] + 1; p < Lp[k + 1]; p++) {
      int64_t i = Li[p];
      Rq[fill[i]] = p; Rk[fill[i]] = (int32_t)k; fill[i]++;
    }
  free(fill);
  *Rp_out = Rp; *Rq_out = Rq; *Rk_out = Rk;
  return 0;
}

/* Left-looking column Cholesky of B on the pattern (Lp, Li) from orc_symbolic.
 * For each column j: w <- B(j:n, j); for every k < j with L_jk != 0 (row list of j),
 * w(i) -= L_ik L_jk for i in struct(L_k), i >= j; then L_jj = sqrt(w_j) and
 * L_ij = w_i / L_jj.  Returns -1 on success, or the first column j whose pivot w_j is
 * not > 0 (or NaN).  *flops counts every multiply, subtract, divide and sqrt done. */
int64_t orc_factor(int64_t n, const int64_t* Bp, const int32_t* Bi, const double* Bx,
                   const int64_t* Lp, const int32_t* Li, double* Lx, double* flops) {
  int64_t *Rp, *Rq; int32_t* Rk;
  if (orc_rowlists(n, Lp, Li, &Rp, &Rq, &Rk)) return -2;
  double* w = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!w) { free(Rp); free(Rq); free(Rk); return -2; }
  double fl = 0.0;
  int64_t bad = -1;
  for (int64_t j = 0; j < n && bad < 0; j++) {
    for (int64_t p = Bp[j]; p < Bp[j + 1]; p++) w[Bi[p]] += Bx[p];
    for (int64_t r = Rp[j]; r < Rp[j + 1]; r++) {
      int64_t pos = Rq[r], k = Rk[r];
      double ljk = Lx[pos];
      for (int64_t q = pos; q < Lp[k + 1]; q++) { w[Li[q]] -= Lx[q] * ljk; fl += 2.0; }
    }
    double d = w[j];
    if (!(d > 0.0)) { bad = j; break; }
    double ljj = sqrt(d);
    fl += 1.0;
    Lx[Lp[j]] = ljj;
    w[j] = 0.0;
    for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; p++) {
      Lx[p] = w[Li[p]] / ljj;
      w[Li[p]] = 0.0;
      fl += 1.0;
    }
  }
  free(w); free(Rp); free(Rq); free(Rk);
  if (flops) *flops = fl;
  return bad;
}

/* Solve A X = Bm through B = P^T A P = L L^T: z = P^T b (z_i = b_{perm[i]}),
 * L y = z by forward substitution, L^T u = y by back substitution, x_{perm[i]} = u_i.
 * Bm and X are n x nrhs column-major with leading dimensions ldb, ldx. */
int orc_solve(int64_t n, const int64_t* Lp, const int32_t* Li, const double* Lx,
              const int32_t* perm, int64_t nrhs, const double* Bm, int64_t ldb, double* X,
              int64_t ldx) {
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!y) return ORC_ENOMEM;
  for (int64_t c = 0; c < nrhs; c++) {
    for (int64_t i = 0; i < n; i++) y[i] = Bm[c * ldb + perm[i]];
    for (int64_t j = 0; j < n; j++) {
      y[j] /= Lx[Lp[j]];
      for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; p++) y[Li[p]] -= Lx[p] * y[j];
    }
    for (int64_t j = n - 1; j >= 0; j--) {
      double s = y[j];
      for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; p++) s -= Lx[p] * y[Li[p]];
      y[j] = s / Lx[Lp[j]];
    }
    for (int64_t i = 0; i < n; i++) X[c * ldx + perm[i]] = y[i];
  }
  free(y);
  return 0;
}

/* y = A x for the full symmetric A stored as its lower CSC. */
int orc_spmv(int64_t n, const int64_t* Ap, const int32_t* Ai, const double* Ax,
             const double* x, double* y) {
  for (int64_t i = 0; i < n; i++) y[i] = 0.0;
  for (int64_t j = 0; j < n; j++)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; p++) {
      int64_t i = Ai[p];
      y[i] += Ax[p] * x[j];
      if (i != j) y[j] += Ax[p] * x[i];
    }
  return 0;
}

/* Relative residual max_c ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf), ||A||_inf the
 * largest absolute row sum of the full symmetric A. */
int orc_residual(int64_t n, const int64_t* Ap, const int32_t* Ai, const double* Ax,
                 int64_t nrhs, const double* Bm, int64_t ldb, const double* X, int64_t ldx,
                 double* rel) {
  double* rs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!rs || !y) { free(rs); free(y); return ORC_ENOMEM; }
  for (int64_t j = 0; j < n; j++)
    for (int64_t p = Ap[j]; p < Ap[j + 1]; p++) {
      rs[Ai[p]] += fabs(Ax[p]);
      if (Ai[p] != j) rs[j] += fabs(Ax[p]);
    }
  double anorm = 0.0;
  for (int64_t i = 0; i < n; i++) if (rs[i] > anorm) anorm = rs[i];
  double worst = 0.0;
  for (int64_t c = 0; c < nrhs; c++) {
    orc_spmv(n, Ap, Ai, Ax, X + c * ldx, y);
    double rn = 0.0, xn = 0.0;
    for (int64_t i = 0; i < n; i++) {
      double r = fabs(Bm[c * ldb + i] - y[i]);
      if (r > rn) rn = r;
      if (fabs(X[c * ldx + i]) > xn) xn = fabs(X[c * ldx + i]);
    }
    double v = (anorm > 0 && xn > 0) ? rn / (anorm * xn) : rn;
    if (v > worst) worst = v;
  }
  *rel = worst;
  free(rs); free(y);
  return 0;
}

/* ||B - L L^T||_F and ||B||_F over the full symmetric matrices.  (L L^T)_ij for
 * i >= j is sum over k <= j of L_ik L_jk; its lower pattern lies inside struct(L). */
int orc_llt_error(int64_t n, const int64_t* Bp, const int32_t* Bi, const double* Bx,
                  const int64_t* Lp, const int32_t* Li, const double* Lx, double* err_f,
                  double* b_f) {
  int64_t *Rp, *Rq; int32_t* Rk;
  if (orc_rowlists(n, Lp, Li, &Rp, &Rq, &Rk)) return ORC_ENOMEM;
  double* w = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!w) { free(Rp); free(Rq); free(Rk); return ORC_ENOMEM; }
  double e2 = 0.0, b2 = 0.0;
  for (int64_t j = 0; j < n; j++) {
    for (int64_t r = Rp[j]; r < Rp[j + 1]; r++) {
      int64_t pos = Rq[r], k = Rk[r];
      double ljk = Lx[pos];
      for (int64_t q = pos; q < Lp[k + 1]; q++) w[Li[q]] += Lx[q] * ljk;
    }
    double ljj = Lx[Lp[j]];
    for (int64_t q = Lp[j]; q < Lp[j + 1]; q++) w[Li[q]] += Lx[q] * ljj;
    for (int64_t p = Bp[j]; p < Bp[j + 1]; p++) {
      w[Bi[p]] -= Bx[p];
      b2 += (Bi[p] == j ? 1.0 : 2.0) * Bx[p] * Bx[p];
    }
    for (int64_t q = Lp[j]; q < Lp[j + 1]; q++) {
      double d = w[Li[q]];
      e2 += (Li[q] == j ? 1.0 : 2.0) * d * d;
      w[Li[q]] = 0.0;
    }
  }
  free(w); free(Rp); free(Rq); free(Rk);
  *err_f = sqrt(e2);
  *b_f = sqrt(b2);
  return 0;
}

/*
 * Task-granularity threshold D of the OPT-D heuristic (Sec. 4.1, Algorithm 1), in the
 * paper's order and names:
 *   goalTasks = max(1.1 nsuper, n / 14);
 *   maxChildren = max_i C[i];  T[k] = number of outer tasks with exactly k inner tasks
 *   (a bucket count);
 *   D = maxChildren + 1, numOuterTasks = 0, numTasks = nsuper; then, while
 *   (numTasks < goalTasks or D > 0.3 maxChildren or numOuterTasks < nsuper / 1000) and
 *   D > 0: D = D - 1, numOuterTasks += T[D], numTasks += D T[D].
 * C[i] >= 0 is the number of inner tasks of outer task i.  Returns 0 and D in *D_out, or
 * ORC_EINVAL (negative count, nsuper < 0) / ORC_ENOMEM.
 */
int orc_opt_d(int64_t n, int32_t nsuper, const int32_t* C, int32_t* D_out) {
  if (nsuper < 0 || n < 0 || (nsuper > 0 && !C) || !D_out) return ORC_EINVAL;
  int32_t maxc = 0;
  for (int32_t i = 0; i < nsuper; i++) {
    if (C[i] < 0) return ORC_EINVAL;
    if (C[i] > maxc) maxc = C[i];
  }
  int64_t* T = (int64_t*)calloc((size_t)maxc + 1, sizeof(int64_t));
  if (!T) return ORC_ENOMEM;
  for (int32_t i = 0; i < nsuper; i++) T[C[i]]++;
  const double goal = fmax(1.1 * (double)nsuper, (double)n / 14.0);
  int64_t D = (int64_t)maxc + 1, outer = 0;
  double tasks = (double)nsuper;
  while ((tasks < goal || (double)D > 0.3 * (double)maxc || (double)outer < (double)nsuper / 1000.0) &&
         D > 0) {
    D--;
    outer += T[D];
    tasks += (double)D * (double)T[D];
  }
  free(T);
  *D_out = (int32_t)D;
  return 0;
}

/*
 * The hybrid switch of Sec. 4.3: multi-threaded BLAS on each supernode (returns 1) when the
 * average supernode size n / nsuper exceeds 50, or exceeds 20 while the density
 * nnz / (n n) of the matrix is below 1e-4; otherwise the nested-task heuristic (returns 0).
 */
int orc_hybrid_uses_blas(int64_t n, int32_t nsuper, int64_t nnz) {
  if (n <= 0 || nsuper <= 0) return 0;
  const double avg = (double)n / (double)nsuper;
  const double density = (double)nnz / ((double)n * (double)n);
  return avg > 50.0 || (avg > 20.0 && density < 1e-4);
}
