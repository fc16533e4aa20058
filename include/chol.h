/*
 * chol.h -- C ABI of a GB300 (sm_103a) supernodal sparse Cholesky library.
 *
 * The library factors a sparse symmetric positive definite matrix A = L L^T and solves
 * A X = B with the two triangular solves L Y = B, L^T X = Y.  This is the computation the
 * paper ("Optimization of the Sparse Multi-Threaded Cholesky Factorization for A64FX")
 * names as the bulk of the solver: Sec. 1 states A = L L^T and the three phases
 * analyze / factorize / solve, Sec. 2 describes the analysis (reordering, elimination
 * tree, supernodes), Sec. 3 and Listing 1 the supernodal factorization (SYRK and GEMM
 * updates from earlier supernodes, then POTRF and TRSM of the supernode, with a
 * serialized assembly of the updates), and Fig. 1 the elimination-tree parallelism.
 *
 * Conventions that hold for every entry point:
 *  - Matrices enter as the LOWER triangle, diagonal included, in compressed sparse column
 *    form: colptr int64[n+1], rowind int32[nnz] (rows strictly increasing inside a
 *    column, every row >= its column), values float64[nnz] in the same order.
 *  - perm is int32[n] with perm[new] = old; the library factors B = P^T A P, i.e.
 *    B[i][j] = A[perm[i]][perm[j]].  Solves take and return vectors in A's numbering.
 *  - Dense blocks (B, X) are column-major n x nrhs with a leading dimension >= n.
 *  - Every function returns an int status: CHOL_OK (0), CHOL_PENDING (1), or a negative
 *    CHOL_E_* code; chol_strerror() names it.  No exception crosses the ABI and the
 *    library never aborts the process.
 *  - "where" arguments say whether a pointer is host memory (CHOL_HOST) or device memory
 *    of the context's GPU (CHOL_DEVICE).  Device work is ordered on the context stream.
 *    Host-pointer calls copy in, compute and copy out before returning; device-pointer
 *    calls return after enqueueing, and a device-side failure (a non-positive pivot) is
 *    reported by the next chol_factor_status() call.
 *  - Ownership: the caller owns every array it passes and may free it once the call
 *    returns (device arrays: once the stream has passed the call).  Handles returned by
 *    the library are owned by it until the matching chol_free_* / chol_destroy.  A factor
 *    refers to the analysis it was made from: free factors before that analysis.
 *    Destroying a context releases the device memory of every handle bound to it; those
 *    handles must then only be passed to chol_free_*.
 *  - Threading: a context and its handles must not be used from two threads at once.
 */
#ifndef CHOL_H
#define CHOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHOL_OK 0
#define CHOL_PENDING 1
#define CHOL_E_INVALID (-1)   /* malformed input or argument */
#define CHOL_E_NOT_SPD (-2)   /* a pivot was <= 0 or NaN: A is not positive definite */
#define CHOL_E_OOM (-3)       /* device allocation failed or the HBM budget is exceeded */
#define CHOL_E_CUDA (-4)      /* a CUDA runtime call failed */
#define CHOL_E_TIMEOUT (-5)   /* a bounded device-side wait expired */
#define CHOL_E_NODEVICE (-6)  /* no usable CUDA device for a call that needs one */
#define CHOL_E_STALL (-7)     /* iterative refinement did not converge */
#define CHOL_E_SCRATCH (-8)   /* chol_solve_noalloc: the solve needs more than the fixed
                                 scratch area holds */

#define CHOL_HOST 0
#define CHOL_DEVICE 1

/* Scatter of the Schur updates into ancestor supernodes (Sec. 3: the paper serializes
 * this assembly with a lock).  ATOMIC adds each update with device atomics (fast, run-to-
 * run rounding differences).  OWNER stages each level's updates and lets every target
 * pull them in a fixed order (bitwise reproducible). */
#define CHOL_ASSEMBLY_ATOMIC 0
#define CHOL_ASSEMBLY_OWNER 1

#define CHOL_FP64 0   /* FP64 factor */
#define CHOL_MIXED 1  /* FP32 panels with TF32 tensor-core Schur updates; FP64 refinement */

typedef struct chol_ctx chol_ctx;
typedef struct chol_sym chol_sym;
typedef struct chol_num chol_num;

typedef struct chol_opts {
  int device;         /* CUDA device ordinal */
  void* stream;       /* cudaStream_t for all device work; NULL: the context makes one */
  int width_cap;      /* largest supernode width W in columns (1..128); 0 = default 64 */
  int assembly;       /* CHOL_ASSEMBLY_ATOMIC or CHOL_ASSEMBLY_OWNER */
  size_t hbm_budget;  /* bytes of device memory the context may hold; 0 = no limit */
  double pivot_tau;   /* CHOL_MIXED: a pivot below pivot_tau * a_jj redoes the supernode's
                         diagonal block in FP64; 0 = default 1e-5 */
  double relax;       /* relaxed amalgamation (Sec. 2): a fundamental supernode joins the
                         one before it when that one's last column is its child and the
                         merged panel stays mostly nonzero -- explicit zeros at most 1/2 of
                         it for merged widths <= 16, 1/5 for widths <= 64, else `relax`.
                         0 = default 0.05; negative = fundamental supernodes only.  The
                         factor's pattern, export and flop count stay those of the exact L */
  int fp64_schur;     /* CHOL_FP64 factors: how the 128x128 Schur tiles are computed.
                         CHOL_SCHUR_OZAKI (default): on the bf16 tensor cores (tcgen05) by
                         splitting every L21 row into 8 exact 7-bit slices scaled by a power
                         of two; slice products accumulate exactly, so the tile carries FP64
                         accuracy (representation error < 2^-57 of the row maximum).  Needs
                         W <= 64 (else DMMA).  CHOL_SCHUR_DMMA: FP64 mma.sync tiles. */
} chol_opts;

#define CHOL_SCHUR_OZAKI 0
#define CHOL_SCHUR_DMMA 1

typedef struct chol_sym_stats {
  int64_t n;          /* order of A */
  int64_t nnz_a;      /* stored lower entries of A */
  int64_t nnz_l;      /* entries of L (diagonal included), exact, no padding */
  int64_t l_storage;  /* values held by the supernode panels (incl. unused upper
                         triangles of diagonal blocks) */
  int64_t nsuper;     /* supernodes after the width cap */
  int64_t nlevels;    /* elimination-tree levels of the supernodal tree */
  double flops;       /* sum_j c_j^2, c_j = entries of column j of L */
  int64_t max_width;  /* widest supernode */
  int64_t max_rows;   /* most rows in a supernode */
  double flops_panel; /* sum of c^2 over the columns of the (padded) panels: the operations
                         the factorization performs, >= flops under relaxed amalgamation */
  int64_t nfundamental; /* fundamental supernodes (before amalgamation and the width cap) */
  int64_t ntrsm_tc;     /* supernodes whose TRSM runs on the tensor cores in an FP64 factor with
                           the tensor-core tiles (under the current tile policy) */
} chol_sym_stats;

/* Fills *opts with the defaults (device 0, own stream, W = 64, atomic assembly,
 * pivot_tau 1e-5, relax 0.05). */
void chol_default_opts(chol_opts* opts);

/* Library version as major*10000 + minor*100 + patch. */
int chol_version(void);

/* Human-readable name of a status code (static storage). */
const char* chol_strerror(int status);

/* Creates a context bound to opts->device.  Fails with CHOL_E_NODEVICE when the device
 * cannot be opened.  opts may be NULL for the defaults. */
int chol_create(const chol_opts* opts, chol_ctx** out);
void chol_destroy(chol_ctx* ctx);

/* Symbolic analysis (Sec. 2): permutes the pattern, builds the elimination tree
 * (parent(j) = smallest off-diagonal row of column j of L), the column counts, the
 * fundamental supernodes cut to at most W columns, their row structures, the level sets
 * of the supernodal tree (Sec. 3, Fig. 1) and the per-level task lists of the device
 * factorization.  Host work only (no device is touched): only opts->width_cap is read,
 * opts may be NULL for W = 64, and the result is uploaded to the device of the first
 * context that factors with it.  Errors: CHOL_E_INVALID for n < 0, n >= 2^31,
 * a row out of range, above the diagonal, unsorted or duplicated, a perm that is not a
 * permutation.  The caller keeps ownership of colptr, rowind and perm. */
int chol_analyze(const chol_opts* opts, int64_t n, const int64_t* colptr,
                 const int32_t* rowind, const int32_t* perm, chol_sym** out);
int chol_sym_info(const chol_sym* sym, chol_sym_stats* stats);

/* Copies symbolic results to host arrays; each pointer may be NULL.  parent and colcount
 * have n entries (column elimination tree, -1 at a root; column counts incl. diagonal);
 * sn_start has nsuper+1 entries (first column of each supernode, then n); sn_level has
 * nsuper entries (0 for supernodes without children, else 1 + the children's maximum). */
int chol_sym_export(const chol_sym* sym, int32_t* parent, int64_t* colcount,
                    int32_t* sn_start, int32_t* sn_level);
/* Copies the row lists of the supernode panels: supernode s holds rows[rowptr[s] ..
 * rowptr[s+1]) in ascending order, its own columns first (rowptr: nsuper+1 entries).  Under
 * relaxed amalgamation a column's rows in L are a subset of its panel's rows from its own
 * position on; otherwise they are equal. */
int chol_sym_rows(const chol_sym* sym, int64_t* rowptr, int32_t* rows);
void chol_free_sym(chol_sym* sym);

/* Numeric factorization of B = P^T A P (Sec. 3, Listing 1, reorganized per level).
 * vals holds A's lower values in the order of the colptr/rowind given to chol_analyze
 * (copied into the factor).  precision is CHOL_FP64, or CHOL_MIXED: FP32 panels of the
 * equilibrated matrix S B S, S = diag(B)^{-1/2}, with a diagonal block refactored in FP64
 * whenever one of its FP32 pivots falls below opts.pivot_tau; use chol_refine to reach
 * FP64 accuracy with it.  Allocates the factor on the device and enqueues the
 * factorization; *out is valid at once.  Errors: CHOL_E_INVALID, CHOL_E_OOM,
 * CHOL_E_CUDA; a non-positive pivot surfaces through chol_factor_status(). */
int chol_factorize(chol_ctx* ctx, const chol_sym* sym, const double* vals, int where,
                   int precision, chol_num** out);

/* Re-runs the numeric factorization in the storage of an existing factor with new values
 * on the same pattern (no allocation). */
int chol_refactorize(chol_ctx* ctx, chol_num* num, const double* vals, int where);

/* Waits for the factorization to finish.  Returns CHOL_OK or CHOL_E_NOT_SPD; in the
 * latter case *bad_col (if not NULL) receives a column of B whose pivot failed (the
 * smallest one this run saw). */
int chol_factor_status(chol_ctx* ctx, const chol_num* num, int64_t* bad_col);

/* Copies L to host CSC arrays in B's numbering: Lp int64[n+1], Li int32[nnz_l],
 * Lx float64[nnz_l], rows sorted, diagonal first.  Any pointer may be NULL. */
int chol_factor_export(chol_ctx* ctx, const chol_num* num, int64_t* Lp, int32_t* Li,
                       double* Lx);

/* Copies the raw supernode panels of supernodes first .. first+count-1 (Sec. 2: a supernode
 * stores its columns as one dense block over the rows of its row list) to out, as float64
 * (FP32 panels of a CHOL_MIXED factor are widened): panel s is the m_s x n_s column-major
 * block of L[rows_s, sn_start[s] .. sn_start[s+1]) (m_s and rows_s from chol_sym_rows, n_s
 * from chol_sym_export's sn_start), the panels one after another in supernode order, so out
 * holds sum_s m_s n_s doubles.  Entries above the diagonal of a panel's leading n_s x n_s
 * block are unspecified; under relaxed amalgamation a panel also holds explicit zeros of L.
 * where: CHOL_HOST (returns once copied) or CHOL_DEVICE (device memory of the context's GPU,
 * stream-ordered).  Errors: CHOL_E_INVALID for a range outside 0 .. nsuper. */
int chol_factor_panels(chol_ctx* ctx, const chol_num* num, int64_t first, int64_t count,
                       double* out, int where);
void chol_free_num(chol_num* num);

/* Solves A X = B (Sec. 1: L Y = P^T B, then L^T Z = Y, X = P Z) for nrhs right-hand
 * sides with the device forward and back substitution over the supernodal levels.
 * X may equal B (in place) only when ldx == ldb.  where: CHOL_HOST (copy in, solve, copy
 * out, synchronize) or CHOL_DEVICE (stream-ordered, returns after enqueue). */
int chol_solve(chol_ctx* ctx, const chol_num* num, int64_t nrhs, const double* B,
               int64_t ldb, double* X, int64_t ldx, int where);

/* Result of chol_refine. */
typedef struct chol_refine_info {
  int iterations;       /* refinement steps taken, over all passes and column blocks */
  int fell_back;        /* 1 if refinement with a CHOL_MIXED factor stalled and the FP64
                           factor (made once, kept with the factor) was used */
  double residual;      /* final max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf) */
  int64_t pivot_redos;  /* diagonal blocks of a CHOL_MIXED factor refactored in FP64 */
} chol_refine_info;

/* Solves A X = B to a relative residual <= tol by iterative refinement (FP64 residual
 * r = b - A x with the original A, correction d from the factor, x += d).  With a
 * CHOL_FP64 factor this polishes the direct solution; with a CHOL_MIXED factor (FP32
 * panels of the equilibrated matrix diag(A)^{-1/2} A diag(A)^{-1/2}) it recovers FP64
 * accuracy.  Refinement stops when the residual meets tol, or stalls when the largest
 * residual norm fails to halve twice in a row or after maxit steps; a stalled CHOL_MIXED
 * factor falls back once to an FP64 factor of the same values (kept until the values
 * change) and refines again.  B and X must not alias.  where as in chol_solve; the call
 * synchronizes with the stream (it reads residual norms every step).  Returns CHOL_OK,
 * CHOL_E_STALL (X holds the last iterate, info->residual its residual), or an error. */
int chol_refine(chol_ctx* ctx, chol_num* num, int64_t nrhs, const double* B, int64_t ldb,
                double* X, int64_t ldx, int where, double tol, int maxit,
                chol_refine_info* info);

/* Iterative refinement whose correction equations are solved by GMRES (GMRES-IR; not in the
 * paper, whose factor is FP64 only): each step forms the FP64 residual r = b - A x with the
 * original A and solves A d = r by flexible GMRES(restart) right-preconditioned with the
 * factor (z = M^-1 v by the factor's triangular solves: an FP32 factor of the equilibrated
 * matrix for CHOL_MIXED), orthonormalizing the Krylov basis in FP64 (classical Gram-Schmidt
 * with one reorthogonalization), until the correction residual fell by 1e-6, then x += d.
 * Plain refinement (chol_refine) contracts the error by about kappa(A) times the factor's
 * accuracy per step and stalls for kappa(A) beyond ~1e7 with an FP32 factor; this converges
 * for kappa(A) up to about the inverse square of the factor's accuracy.  Same arguments as
 * chol_refine plus restart (Krylov vectors per GMRES cycle, 1..64; 0 = 30); maxit bounds the
 * GMRES iterations of a right-hand side (0 = 10 restart).  Stops when the relative residual
 * meets tol, or stalls when two refinement steps in a row fail to halve the residual or
 * after maxit iterations; a stalled CHOL_MIXED factor falls back once to an FP64 factor of
 * the same values (kept with the factor, as in chol_refine).  info->iterations counts GMRES
 * iterations (each one factor solve and one SpMV).  Right-hand sides are done one after
 * another; the call synchronizes.  Device workspace: (2 restart + 1) n doubles, kept with
 * the factor.  Returns CHOL_OK, CHOL_E_STALL or an error. */
int chol_refine_gmres(chol_ctx* ctx, chol_num* num, int64_t nrhs, const double* B, int64_t ldb,
                      double* X, int64_t ldx, int where, double tol, int restart, int maxit,
                      chol_refine_info* info);

/* Device-pointer solve that allocates nothing (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they solve, e.g. code
 * capturing a stream in global capture mode, where cudaMalloc is an error, or a runtime
 * that owns all device memory).  Same arguments and result as chol_solve with
 * where = CHOL_DEVICE: B and X are device pointers, the work is enqueued on the context
 * stream and the call returns without waiting.  The workspace is one fixed array of
 * chol_noalloc_scratch_bytes() (32 MiB) compiled into the library; every GPU that loads
 * the library holds it until the process exits.  A solve of k = min(nrhs, 32) columns
 * needs about 8 * (2 n k + per-level partial sums) bytes; larger requests fail with
 * CHOL_E_SCRATCH before any work is enqueued.  The first call on a device looks up the
 * array's device address (with that device current); make that first call before any
 * stream capture.  All calls share the array and leave its contents behind; each call
 * clears the work-queue counters at its head (all that must start at zero).  Calls whose
 * device work overlaps (other streams or contexts on the same device) race on it and must
 * be ordered by the caller.  The array's address is kept for the life of the process: after
 * a cudaDeviceReset of a device (which destroys the context it was looked up in) the entry
 * point must not be used on that device again.  The call leaves the calling thread's
 * current device as it found it. */
int chol_solve_noalloc(chol_ctx* ctx, const chol_num* num, int64_t nrhs, const double* B,
                       int64_t ldb, double* X, int64_t ldx);
size_t chol_noalloc_scratch_bytes(void);

/* ---- batching ----------------------------------------------------------------------
 * A batch packs existing factors (same context, precision and assembly mode; any
 * patterns) so that level l of the batch -- level l, counted from the leaves, of every
 * member (Sec. 3, Fig. 1 applied across matrices) -- runs as one launch per kernel kind.
 * A launch has one CTA per task of its list (the hardware block scheduler refills SMs as
 * CTAs finish; measured faster than a single resident wave of CTAs taking tasks from a
 * queue); the 128 x 128 tensor-core Schur launches are the exception, with one resident
 * CTA per SM taking tasks from a work queue.  With use_graph, the first chol_batch_factorize captures the whole launch
 * sequence into a CUDA graph and later calls replay it.  Members stay usable on their own
 * (chol_solve, chol_refine, chol_factor_status); free the batch before its members. */
typedef struct chol_batch chol_batch;
int chol_batch_create(chol_ctx* ctx, int count, chol_num* const* nums, chol_batch** out);
/* Re-factors every member.  vals[i] (may be NULL, as may vals itself: keep member i's
 * current values) are new values of member i on its pattern, host or device per where.
 * Stream-ordered; check each member with chol_factor_status. */
int chol_batch_factorize(chol_ctx* ctx, chol_batch* batch, const double* const* vals,
                         int where, int use_graph);
void chol_batch_free(chol_batch* batch);

/* Schur tile sizes per supernode size class: 128x128 tiles for supernodes with at least
 * min_rows_tile128 off-diagonal rows on levels holding at least min_level_tiles128 such
 * tiles, else 64x64 tiles from min_rows_tile64 rows on levels holding at least
 * min_level_tiles64 such tiles, else 32x32 from min_rows_tile32 rows, else 16x16.
 * A 128x128 tile is one tcgen05 tensor-core task: 3xTF32 for an FP32 (mixed-precision)
 * factor, exact bf16 operand slices for an FP64 factor (four 64x64 DMMA tasks under
 * CHOL_SCHUR_DMMA).
 * granularity (Sec. 4 of the paper, re-targeted to tiles): CHOL_GRAN_TILES uses the size
 * thresholds alone.  Otherwise a supernode's Schur update is an outer task and the tiles
 * the thresholds give it are its inner tasks; an outer task with at least D inner tasks
 * (D by the OPT-D heuristic, Algorithm 1, over all supernodes) is split into those tiles,
 * the others are done whole (the coarsest tile that covers the update in one task, 128
 * wide above 64 rows).  CHOL_GRAN_OPTD_COST also keeps whole an outer task whose tiles
 * would carry fewer than 50,000 flops each (OPT-D-COST); CHOL_GRAN_HYBRID takes
 * CHOL_GRAN_TILES when the average supernode size is above 50, or above 20 with density
 * nnz(A) / n^2 below 1e-4, and CHOL_GRAN_OPTD_COST otherwise.
 * Default {64, 17, 304, 128, 0, CHOL_GRAN_TILES, 8192}.  All thresholds >= 1 except the two
 * level thresholds (>= 0), granularity one of the four; anything else is CHOL_E_INVALID. */
#define CHOL_GRAN_TILES 0
#define CHOL_GRAN_OPTD 1
#define CHOL_GRAN_OPTD_COST 2
#define CHOL_GRAN_HYBRID 3
typedef struct chol_tile_policy {
  int min_rows_tile64;
  int min_rows_tile32;
  int min_level_tiles64;
  int min_rows_tile128;
  int min_level_tiles128;
  int granularity;
  /* FP64 factors with the tensor-core tiles: a level's 128-tile supernodes take the
   * tensor-core TRSM (L21 = A21 L11^-T with the explicit inverse, slices on the bf16 tensor
   * cores) when their off-diagonal rows add up to at least this many; >= 1 */
  int min_rows_trsm_tc;
} chol_tile_policy;
int chol_sym_get_tile_policy(const chol_sym* sym, chol_tile_policy* policy);
/* Rebuilds the Schur task lists of sym (and its device copy); factors made from sym use
 * the new lists from their next factorization; existing batches keep their own copy. */
int chol_sym_set_tile_policy(chol_sym* sym, const chol_tile_policy* policy);
/* The threshold D of the OPT-D heuristic (Sec. 4.1, Algorithm 1) for nsuper outer tasks
 * with counts[i] inner tasks each (host array, counts[i] >= 0; NULL allowed when nsuper
 * is 0) and matrix size n: the outer tasks with at least D (and at least one) inner tasks
 * are the ones to split.  CHOL_E_INVALID on n < 0, nsuper < 0 or a negative count. */
int chol_opt_d(int64_t n, int32_t nsuper, const int32_t* counts, int32_t* D);
/* The granularity rule of sym's current task lists: *rule the CHOL_GRAN_* value applied
 * (CHOL_GRAN_HYBRID resolved to the rule it chose), *D its threshold (-1 under
 * CHOL_GRAN_TILES), *nsplit the number of supernodes whose Schur update is split. */
int chol_sym_granularity(const chol_sym* sym, int* rule, int32_t* D, int32_t* nsplit);
/* The Schur tile tasks of sym's current task lists, all levels and tile sizes: task q
 * updates the tile of supernode s[q]'s Schur complement with rows i0[q] .. and columns
 * k0[q] .. of its off-diagonal rows, tile[q] wide (128, 64, 32 or 16; clipped at the
 * update's order).  With s == NULL only *count is set; otherwise the four host arrays must
 * hold *count entries (the value a first call returned). */
int chol_sym_schur_tiles(const chol_sym* sym, int32_t* s, int32_t* i0, int32_t* k0,
                         int32_t* tile, int64_t* count);
/* ---- subtree-to-device partition (multi-GPU layout; measured on one GPU only) ----------
 * The supernodal elimination tree splits into independent subtrees: supernodes of
 * different subtrees never update one another (Sec. 3, Fig. 1), so each subtree can be
 * factored on its own device with no communication, and only the supernodes above them
 * (the top separators) need the update blocks of several devices, summed into the device
 * that owns the top part (the layer idea of Geist and Ng that the paper's related work
 * cites).  chol_partition_tree partitions a forest of nv vertices (parent[v] = -1 at a root,
 * work[v] >= 0): starting from the roots, the heaviest subtree that has children is replaced
 * by its children (its own vertex joins the top part) until the current subtrees, dealt
 * largest first to the least loaded of nparts parts, give every part at most (1 + tol) of
 * an even share -- or only single vertices remain.  owner[v] (nv entries) receives the part
 * 0 .. nparts-1 of v's subtree, or -1 for the top part; *imbalance (may be NULL) the largest
 * part's work over the mean.  CHOL_E_INVALID on a malformed forest (cycle, parent out of
 * range), negative work, nparts < 1 or tol < 0. */
int chol_partition_tree(int32_t nv, const int32_t* parent, const double* work, int nparts,
                        double tol, int32_t* owner, double* imbalance);
/* The same on sym's supernodal elimination tree with work = the flops of each supernode's
 * columns (sum of c_j^2): owner has nsuper entries; *top_flops (may be NULL) receives the
 * work left to the top part. */
int chol_sym_partition(const chol_sym* sym, int nparts, double tol, int32_t* owner,
                       double* imbalance, double* top_flops);

/* Autotuner: times refactorizations of num (reps each) under candidate tile policies by
 * coordinate descent over the five thresholds, keeps the fastest in num's analysis,
 * stores it in *best (and its time in *best_ms) and leaves num factored under it. */
int chol_autotune(chol_ctx* ctx, chol_num* num, int reps, chol_tile_policy* best,
                  double* best_ms);

/* ---- serving -----------------------------------------------------------------------
 * A server takes SPD systems as they arrive and answers each with a solution refined to
 * its residual target (the paper has no serving layer).  Worker slots -- each a thread
 * with its own context and stream on opts.device -- take the oldest queued requests that
 * fit the HBM budget (up to max_batch at a time), factor them together as one batch,
 * refine every request and complete it; a request that arrives while other groups are on
 * the GPU starts as soon as a slot and memory are free (continuous batching).  Symbolic
 * analyses run on host analyzer threads ahead of the slots, are shared by pattern, and
 * their device copies stay resident per slot.  The budget is split: each slot may
 * keep analyses worth budget / (4 slots) resident, the groups in flight share the rest;
 * a request larger than that share alone completes with CHOL_E_OOM. */
typedef struct chol_server chol_server;
typedef struct chol_server_opts {
  int device;
  int slots;          /* worker slots (concurrent groups); 0 = 2 */
  int max_batch;      /* requests factored together; 0 = 16 */
  size_t hbm_budget;  /* device bytes the server may hold; 0 = no limit */
  int width_cap;      /* as chol_opts; 0 = 64 */
  int assembly;       /* as chol_opts */
  int sym_cache;      /* device copies of analyses cached per slot; 0 = 64 (the shared
                         host cache keeps 4x as many) */
  int analyzers;      /* host threads running symbolic analyses ahead of the slots; 0 = 4 */
} chol_server_opts;

typedef struct chol_request {
  int64_t n;
  const int64_t* colptr;  /* lower CSC of A, host (copied by chol_submit) */
  const int32_t* rowind;
  const double* vals;
  const int32_t* perm;    /* ordering, perm[new] = old (copied) */
  int64_t nrhs;           /* >= 1 */
  const double* B;        /* n x nrhs column-major, host (copied) */
  int64_t ldb;
  double* X;              /* n x nrhs host output; must stay valid until the request ends */
  int64_t ldx;
  int precision;          /* CHOL_FP64 or CHOL_MIXED */
  double tol;             /* residual target; 0 = 1e-12 */
} chol_request;

typedef struct chol_result {
  int status;             /* CHOL_OK, or the error of the request */
  int iterations;         /* refinement steps */
  int fell_back;          /* a CHOL_MIXED request needed the FP64 factor */
  double residual;        /* max_c ||b - A x||_inf / (||A||_inf ||x||_inf) */
  double t_submit, t_start, t_done;  /* seconds on the server clock */
  int batch_size;         /* requests factored in the same group */
} chol_result;

void chol_default_server_opts(chol_server_opts* opts);
int chol_server_create(const chol_server_opts* opts, chol_server** out);
/* Queues a request and returns at once with its ticket. */
int chol_submit(chol_server* srv, const chol_request* req, uint64_t* ticket);
/* CHOL_PENDING while the request runs; CHOL_OK with *result once it has ended (X then
 * holds the solution); a ticket is reported once. */
int chol_poll(chol_server* srv, uint64_t ticket, chol_result* result);
/* Blocks until the request has ended, then as chol_poll. */
int chol_wait(chol_server* srv, uint64_t ticket, chol_result* result);
/* Seconds since the server was created (the clock of chol_result's times). */
double chol_server_clock(chol_server* srv);
/* Stops the slots (requests still queued are dropped) and frees the server. */
void chol_server_destroy(chol_server* srv);

/* Test hook for the failure path of the bounded device waits (not a tuning knob).  Every wait
 * inside the 128 x 128 tensor-core Schur kernels gives up after 2^31 SM clock cycles (about a
 * second; a working wait lasts microseconds).  With cycles > 0 the kernels' consumer warps
 * wait, for at most that many cycles, on a barrier that nothing completes (standing in for an
 * accumulator that never finishes), then give up: the kernel's other waits expire in turn,
 * each role waits (bounded) for its own copies and MMAs in flight, the tensor memory is
 * freed, every launch ends, later launches of the same factorization skip their work, and
 * chol_factor_status reports CHOL_E_TIMEOUT; the context stays usable.  0 turns the hook off.
 * CHOL_E_INVALID for cycles < 0. */
int chol_set_device_wait(chol_ctx* ctx, long long cycles);

/* ---- tracing ------------------------------------------------------------------------
 * Per-kernel-kind accounting of the device work a context enqueues: the launch count is
 * always kept; with profiling on, every launch is bracketed by CUDA events on the context
 * stream and its duration is added to its kind.  flops and bytes are the algorithmic work
 * of the launches (Schur tiles: u(u+1)n per supernode of u off-diagonal rows and n
 * columns; POTRF: n^3/3 + n^2/2; TRSM: u n^2; solves: bytes of L and the vectors read). */
typedef struct chol_prof_entry {
  char name[32];      /* kernel kind, e.g. "schur64_f64" */
  int64_t launches;   /* launches since the last reset */
  double ms;          /* summed event time of the timed launches (profiling on) */
  int64_t timed;      /* launches that were bracketed by events */
  double flops;       /* algorithmic flops of those launches */
  double bytes;       /* algorithmic bytes of those launches */
} chol_prof_entry;

/* Turns event bracketing on (1) or off (0).  Events are recorded on the context stream;
 * do not enable while the stream is being captured into a CUDA graph. */
int chol_profile_enable(chol_ctx* ctx, int on);
/* Restricts event bracketing to the launches of one kernel kind (name as in
 * chol_prof_entry.name, e.g. "schur128_oz"); NULL or "" brackets every kind again.  Launch
 * counts are kept for every kind either way.  Bracketing one kind keeps the event overhead
 * off the other launches of a timed region.  CHOL_E_INVALID for an unknown name. */
int chol_profile_only(chol_ctx* ctx, const char* name);
/* Synchronizes the stream, folds finished events in, and copies up to max entries; the
 * number of kinds is stored in *count.  Entries with zero launches are included. */
int chol_profile_read(chol_ctx* ctx, chol_prof_entry* out, int max, int* count);
int chol_profile_reset(chol_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CHOL_H */
