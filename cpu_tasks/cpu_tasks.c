/*
 * cpu_tasks.c -- multi-core CPU baseline of the paper's own method.
 *
 * CHOLMOD-style left-looking supernodal Cholesky run as OpenMP tasks (Sec. 3, Listing 1):
 * the task of supernode s first applies the update of every descendant d that touches s
 * (the SYRK and GEMM of Listing 1: the product of d's rows at and below s's first column
 * with d's rows inside s's columns), then factors s's panel (POTRF of the diagonal block,
 * TRSM of the rows below).  A supernode's task is started when the tasks of all its
 * children in the supernodal elimination tree are done (Sec. 3, Fig. 1).  The updates
 * follow one of the task-granularity policies of Sec. 4:
 *   CT_NONESTED   every update runs inside its supernode's task;
 *   CT_NESTED     every update is a task of its own (inner task), its result is
 *                 subtracted from the panel under a per-supernode lock;
 *   CT_OPTD       nested only for supernodes with at least D updates, D from the OPT-D
 *                 heuristic (Sec. 4.1, Algorithm 1);
 *   CT_OPTD_COST  as CT_OPTD, and an update of fewer than 50,000 flops stays inside its
 *                 supernode's task (Sec. 4.2).
 * It is a comparison point measured on the host cores beside the single-thread oracle;
 * it shares no code with the library or the oracle (the supernode partition and panel row
 * lists come in as plain arrays).  Dense kernels are plain loops (no BLAS in this image).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CT_NONESTED 0
#define CT_NESTED 1
#define CT_OPTD 2
#define CT_OPTD_COST 3

#define CT_EINVAL (-1)
#define CT_ENOMEM (-2)
#define CT_ENOTSPD (-3)

typedef struct {
  int64_t n;
  int32_t ns;
  const int32_t* start;   /* ns + 1: first column of each supernode (permuted numbering) */
  const int64_t* rowptr;  /* ns + 1: offsets into rows */
  const int32_t* rows;    /* sorted rows of each panel; the first n_s are its own columns */
  const int64_t* valptr;  /* ns + 1: offsets into Lx (m_s x n_s, column-major, ld m_s) */
  double* Lx;
  /* updates into supernode t: desc_ptr[t] .. desc_ptr[t+1]: source d, first row position
     p1 of d at or after t's first column, end p2 of d's rows inside t's columns */
  const int64_t* desc_ptr;
  const int32_t* desc_d;
  const int32_t* desc_p1;
  const int32_t* desc_p2;
  const int32_t* parent;  /* supernodal elimination tree */
  int32_t* pending;       /* unfinished children */
  omp_lock_t* locks;      /* one per supernode: the lock of the paper's assembly */
  int policy;
  int32_t D;
  int64_t inner_tasks;    /* inner tasks created (atomic) */
  int32_t bad_col;        /* first failing column (atomic min), or INT32_MAX */
} ct_problem;

static int32_t ct_m(const ct_problem* P, int32_t s) {
  return (int32_t)(P->rowptr[s + 1] - P->rowptr[s]);
}
static int32_t ct_w(const ct_problem* P, int32_t s) { return P->start[s + 1] - P->start[s]; }

/* Threshold D of OPT-D (Sec. 4.1, Algorithm 1), restated: outer tasks by number of inner
 * tasks (counting sort); D walks down from the largest count, splitting the outer tasks with
 * D inner tasks at each step, until the task total reaches max(1.1 ns, n/14), D is at most
 * 30 % of the largest count and at least ns/1000 outer tasks are split. */
static int32_t ct_opt_d(int64_t n, int32_t ns, const int32_t* C) {
  int32_t top = 0;
  for (int32_t i = 0; i < ns; i++)
    if (C[i] > top) top = C[i];
  int64_t* bucket = (int64_t*)calloc((size_t)top + 1, sizeof(int64_t));
  if (!bucket) return 0;
  for (int32_t i = 0; i < ns; i++) bucket[C[i]]++;
  const double goal = fmax(1.1 * ns, (double)n / 14.0);
  int64_t d = (int64_t)top + 1, split = 0;
  double total = ns;
  while (d > 0 && (total < goal || (double)d > 0.3 * top || (double)split < ns / 1000.0)) {
    d--;
    split += bucket[d];
    total += (double)d * (double)bucket[d];
  }
  free(bucket);
  return (int32_t)d;
}

/* The update of supernode t by descendant d (rows p1 .. m_d-1 of d against rows p1 .. p2-1):
 * U[jj][ii] = sum_k L_d[p1+ii][k] L_d[p1+jj][k], into U (R x J column-major, R = m_d - p1,
 * J = p2 - p1). */
static void ct_update_block(const ct_problem* P, int32_t d, int32_t p1, int32_t p2, double* U) {
  const int32_t md = ct_m(P, d), nd = ct_w(P, d);
  const int32_t R = md - p1, J = p2 - p1;
  const double* Ld = P->Lx + P->valptr[d];
  memset(U, 0, sizeof(double) * (size_t)R * J);
  for (int32_t k = 0; k < nd; k++) {
    const double* col = Ld + (int64_t)k * md + p1;
    for (int32_t jj = 0; jj < J; jj++) {
      const double b = col[jj];
      if (b == 0.0) continue;
      double* u = U + (int64_t)jj * R;
      for (int32_t ii = jj; ii < R; ii++) u[ii] += col[ii] * b;
    }
  }
}

/* Subtracts U from the panel of t: row p1+ii of d goes to its position in t's row list
 * (both lists sorted: one merge), column p1+jj to t's column rows_d[p1+jj] - start[t]. */
static void ct_scatter(const ct_problem* P, int32_t t, int32_t d, int32_t p1, int32_t p2,
                       const double* U, int32_t* pos) {
  const int32_t md = ct_m(P, d), mt = ct_m(P, t);
  const int32_t* rd = P->rows + P->rowptr[d];
  const int32_t* rt = P->rows + P->rowptr[t];
  const int32_t R = md - p1, J = p2 - p1;
  int32_t q = 0;
  for (int32_t ii = 0; ii < R; ii++) {
    while (rt[q] != rd[p1 + ii]) q++; /* every row of d from p1 on is a row of t */
    pos[ii] = q;
  }
  double* Lt = P->Lx + P->valptr[t];
  for (int32_t jj = 0; jj < J; jj++) {
    double* col = Lt + (int64_t)(rd[p1 + jj] - P->start[t]) * mt;
    const double* u = U + (int64_t)jj * R;
    for (int32_t ii = jj; ii < R; ii++) col[pos[ii]] -= u[ii];
  }
}

/* One update as a unit of work; locked when other updates of t may run at the same time. */
static void ct_apply(ct_problem* P, int32_t t, int32_t d, int32_t p1, int32_t p2, int locked) {
  const int32_t R = ct_m(P, d) - p1, J = p2 - p1;
  double* U = (double*)malloc(sizeof(double) * (size_t)R * J + sizeof(int32_t) * (size_t)R);
  if (!U) { /* out of memory inside a task: report as a failed column */
#pragma omp atomic write
    P->bad_col = -1;
    return;
  }
  int32_t* pos = (int32_t*)(U + (size_t)R * J);
  ct_update_block(P, d, p1, p2, U);
  if (locked) omp_set_lock(&P->locks[t]);
  ct_scatter(P, t, d, p1, p2, U, pos);
  if (locked) omp_unset_lock(&P->locks[t]);
  free(U);
}

/* POTRF of the diagonal block and TRSM of the rows below, right-looking over the panel's
 * columns (column-major, ld m). */
static int32_t ct_panel_factor(double* A, int32_t m, int32_t w) {
  for (int32_t j = 0; j < w; j++) {
    double* cj = A + (int64_t)j * m;
    const double p = cj[j];
    if (!(p > 0.0)) return j;
    const double l = sqrt(p);
    cj[j] = l;
    for (int32_t r = j + 1; r < m; r++) cj[r] /= l;
    for (int32_t c = j + 1; c < w; c++) {
      double* cc = A + (int64_t)c * m;
      const double lc = cj[c];
      for (int32_t r = c; r < m; r++) cc[r] -= cj[r] * lc;
    }
  }
  return w;
}

static void ct_run(ct_problem* P, int32_t t);

static void ct_factor_supernode(ct_problem* P, int32_t t) {
  const int64_t b = P->desc_ptr[t], e = P->desc_ptr[t + 1];
  /* OPT-D: nested when the supernode receives at least D updates (Sec. 4.1) */
  const int nested_sn = P->policy == CT_NESTED ||
                        ((P->policy == CT_OPTD || P->policy == CT_OPTD_COST) && e > b &&
                         e - b >= P->D);
  if (nested_sn) {
    for (int64_t q = b; q < e; q++) {
      const int32_t d = P->desc_d[q], p1 = P->desc_p1[q], p2 = P->desc_p2[q];
      const double flops = 2.0 * (double)(ct_m(P, d) - p1) * (p2 - p1) * ct_w(P, d);
      if (P->policy == CT_OPTD_COST && flops < 50000.0) {
        ct_apply(P, t, d, p1, p2, 1);  /* too small for a task of its own */
      } else {
#pragma omp atomic
        P->inner_tasks++;
#pragma omp task firstprivate(t, d, p1, p2)
        ct_apply(P, t, d, p1, p2, 1);
      }
    }
#pragma omp taskwait
  } else {
    for (int64_t q = b; q < e; q++) ct_apply(P, t, P->desc_d[q], P->desc_p1[q], P->desc_p2[q], 0);
  }
  const int32_t bad = ct_panel_factor(P->Lx + P->valptr[t], ct_m(P, t), ct_w(P, t));
  if (bad < ct_w(P, t)) {
    const int32_t col = P->start[t] + bad;
    int32_t cur;
#pragma omp atomic read
    cur = P->bad_col;
    while (col < cur && !__atomic_compare_exchange_n(&P->bad_col, &cur, col, 0, __ATOMIC_ACQ_REL,
                                                     __ATOMIC_ACQUIRE)) {
    }
  }
}

/* The task of supernode t; when it is its parent's last child, it starts the parent's. */
static void ct_run(ct_problem* P, int32_t t) {
  ct_factor_supernode(P, t);
  const int32_t p = P->parent[t];
  if (p >= 0 && __atomic_sub_fetch(&P->pending[p], 1, __ATOMIC_ACQ_REL) == 0) {
#pragma omp task firstprivate(p)
    ct_run(P, p);
  }
}

/* Factors A (lower CSC in the original numbering, perm[i] = original index of row/column i
 * of the permuted matrix) into the panels Lx of the given supernode partition (panel s:
 * rows rows[rowptr[s] .. rowptr[s+1]), sorted, the first n_s being its own columns; values
 * column-major with leading dimension m_s, panels one after another in order of s) with
 * `threads` OpenMP threads under the given policy.  *D_out: the OPT-D threshold (-1 for
 * CT_NONESTED / CT_NESTED); *inner_out: inner tasks created.  Returns 0, CT_EINVAL,
 * CT_ENOMEM, or CT_ENOTSPD with the failing column in *bad_col. */
int ct_factor(int64_t n, const int64_t* Ap, const int32_t* Ai, const double* Ax,
              const int32_t* perm, int32_t ns, const int32_t* start, const int64_t* rowptr,
              const int32_t* rows, int policy, int threads, double* Lx, int32_t* D_out,
              int64_t* inner_out, int32_t* bad_col) {
  if (n < 0 || ns < 0 || policy < CT_NONESTED || policy > CT_OPTD_COST || threads < 1 || !Lx)
    return CT_EINVAL;
  int rc = CT_ENOMEM;
  int32_t *iperm = NULL, *col2sn = NULL, *parent = NULL, *pending = NULL, *count = NULL;
  int32_t *desc_d = NULL, *desc_p1 = NULL, *desc_p2 = NULL;
  int64_t *valptr = NULL, *desc_ptr = NULL;
  omp_lock_t* locks = NULL;
  iperm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  col2sn = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns + 1));
  pending = (int32_t*)calloc((size_t)ns + 1, sizeof(int32_t));
  count = (int32_t*)calloc((size_t)ns + 1, sizeof(int32_t));
  valptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  desc_ptr = (int64_t*)calloc((size_t)ns + 2, sizeof(int64_t));
  locks = (omp_lock_t*)malloc(sizeof(omp_lock_t) * (size_t)(ns + 1));
  if (!iperm || !col2sn || !parent || !pending || !count || !valptr || !desc_ptr || !locks)
    goto done;
  for (int64_t i = 0; i < n; i++) iperm[perm[i]] = (int32_t)i;
  valptr[0] = 0;
  for (int32_t s = 0; s < ns; s++) {
    for (int32_t j = start[s]; j < start[s + 1]; j++) col2sn[j] = s;
    valptr[s + 1] = valptr[s] + (rowptr[s + 1] - rowptr[s]) * (int64_t)(start[s + 1] - start[s]);
  }
  /* targets of every supernode: runs of its off-diagonal rows by owning supernode */
  int64_t nupd = 0;
  for (int32_t d = 0; d < ns; d++) {
    const int32_t w = start[d + 1] - start[d], m = (int32_t)(rowptr[d + 1] - rowptr[d]);
    const int32_t* r = rows + rowptr[d];
    parent[d] = m > w ? col2sn[r[w]] : -1;
    for (int32_t i = w; i < m; i++)
      if (i == w || col2sn[r[i]] != col2sn[r[i - 1]]) {
        count[col2sn[r[i]]]++;
        nupd++;
      }
  }
  for (int32_t s = 0; s < ns; s++) desc_ptr[s + 1] = desc_ptr[s] + count[s];
  desc_d = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nupd + 1));
  desc_p1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nupd + 1));
  desc_p2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nupd + 1));
  if (!desc_d || !desc_p1 || !desc_p2) goto done;
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
    if (!fill) goto done;
    memcpy(fill, desc_ptr, sizeof(int64_t) * (size_t)ns);
    for (int32_t d = 0; d < ns; d++) {  /* ascending d: each target's list in source order */
      const int32_t w = start[d + 1] - start[d], m = (int32_t)(rowptr[d + 1] - rowptr[d]);
      const int32_t* r = rows + rowptr[d];
      for (int32_t i = w; i < m;) {
        const int32_t t = col2sn[r[i]];
        int32_t e = i;
        while (e < m && col2sn[r[e]] == t) e++;
        const int64_t q = fill[t]++;
        desc_d[q] = d;
        desc_p1[q] = i;
        desc_p2[q] = e;
        i = e;
      }
    }
    free(fill);
  }
  /* assembly of the permuted lower triangle into the zeroed panels */
  memset(Lx, 0, sizeof(double) * (size_t)valptr[ns]);
  for (int64_t jo = 0; jo < n; jo++)
    for (int64_t p = Ap[jo]; p < Ap[jo + 1]; p++) {
      const int32_t a = iperm[Ai[p]], b = iperm[jo];
      const int32_t r = a > b ? a : b, c = a > b ? b : a;
      const int32_t s = col2sn[c];
      const int32_t* rs = rows + rowptr[s];
      int32_t lo = 0, hi = (int32_t)(rowptr[s + 1] - rowptr[s]) - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (rs[mid] < r) lo = mid + 1; else hi = mid;
      }
      if (rs[lo] != r) { rc = CT_EINVAL; goto done; }
      Lx[valptr[s] + (int64_t)(c - start[s]) * (rowptr[s + 1] - rowptr[s]) + lo] += Ax[p];
    }
  for (int32_t s = 0; s < ns; s++) {
    if (parent[s] >= 0) pending[parent[s]]++;
    omp_init_lock(&locks[s]);
  }
  ct_problem P;
  P.n = n; P.ns = ns; P.start = start; P.rowptr = rowptr; P.rows = rows; P.valptr = valptr;
  P.Lx = Lx; P.desc_ptr = desc_ptr; P.desc_d = desc_d; P.desc_p1 = desc_p1; P.desc_p2 = desc_p2;
  P.parent = parent; P.pending = pending; P.locks = locks; P.policy = policy;
  P.D = (policy == CT_OPTD || policy == CT_OPTD_COST) ? ct_opt_d(n, ns, count) : -1;
  P.inner_tasks = 0;
  P.bad_col = INT32_MAX;
  {
    int32_t* leaves = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns + 1));
    if (!leaves) goto done_locks;
    int32_t nl = 0;
    for (int32_t s = 0; s < ns; s++)
      if (pending[s] == 0) leaves[nl++] = s;
#pragma omp parallel num_threads(threads)
#pragma omp single
    for (int32_t q = 0; q < nl; q++) {
      const int32_t s = leaves[q];
#pragma omp task firstprivate(s)
      ct_run(&P, s);
    }
    free(leaves);
  }
  if (D_out) *D_out = P.D;
  if (inner_out) *inner_out = P.inner_tasks;
  if (bad_col) *bad_col = P.bad_col;
  rc = P.bad_col == INT32_MAX ? 0 : (P.bad_col < 0 ? CT_ENOMEM : CT_ENOTSPD);
done_locks:
  for (int32_t s = 0; s < ns; s++) omp_destroy_lock(&locks[s]);
done:
  free(iperm); free(col2sn); free(parent); free(pending); free(count); free(valptr);
  free(desc_ptr); free(locks); free(desc_d); free(desc_p1); free(desc_p2);
  return rc;
}
