// chol_internal.h -- data structures shared by the host analysis, the runtime and the
// device kernels of the supernodal Cholesky library.  Not part of the public ABI.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/chol.h"

namespace chol {

// Row blocks and tile shapes of the device task lists.
constexpr int kTrsmRows = 32;    // off-diagonal rows per TRSM task (one row per lane)
constexpr int kSolveRows = 128;  // off-diagonal rows per solve task
constexpr int kMaxWidth = 128;   // hard limit on the width cap W (diagonal block in smem)

// Schur tile classes: the update U = L21 L21^T of a supernode is cut into lower-triangular
// T x T tiles, T in {128, 64, 32, 16}.  128-tiles run on tcgen05 tensor cores: 3xTF32 in
// the mixed-precision factor, bf16 operand slices in FP64 (or, with the DMMA option, as
// four 64 x 64 FP64 tiles).
//
// FP64 on bf16 tensor cores (operand splitting): a row r of L21 is scaled by 2^-e_r
// (max |L21[r,:]| < 2^e_r) and cut into kOzSlices integer slices of 7 bits,
//   L21[r,k] 2^-e_r = sum_p s_p[r,k] 2^(-7(p+1)),  |s_0| <= 128, |s_p| <= 64 (p > 0),
// each exact in bf16.  Slice products are accumulated exactly in FP32 (every partial sum
// of one diagonal p+q stays below 2^24 for K <= 128), and
//   U[i,k] = 2^(e_i+e_k) sum_{p+q < kOzSlices} 2^(-7(p+q+2)) sum_kk s_p[i,kk] s_q[k,kk].
// The representation error is below 2^-57 of the row maximum.
constexpr int kOzSlices = 8;
constexpr int kOzRowBytes = 128;  // one slice row: 64 bf16 (K <= 64), 128-byte swizzled
constexpr int kOzInvRows = 64;    // slice rows of a diagonal-block inverse (n <= 64, zero-padded)
enum SchurClass { kTile64 = 0, kTile32 = 1, kTile16 = 2, kTile128 = 3, kNumTileClasses = 4 };
inline int tile_of_class(int c) {
  return c == kTile128 ? 128 : (c == kTile64 ? 64 : (c == kTile32 ? 32 : 16));
}

// Task kinds of the per-level schedule.  Every task is an int4 {s, a, b, c}.
enum TaskKind {
  kTaskPotrf = 0,   // {s, first_bwd, nbwd, y}: diagonal block of s; its backward tasks; y: the
                    //   first row of its inverse's slices (128-tile supernodes) or -1
  kTaskTrsm = 1,    // {s, r0, -, -}: L21 rows r0 .. r0+kTrsmRows of s
  kTaskSchur64 = 2, // {s, i0, k0, -}: tile of U_s (rows i0.., cols k0.., offsets into L21)
  kTaskSchur32 = 3,
  kTaskSchur16 = 4,
  kTaskFwd = 5,     // {s, r0, -, -}: forward-solve block
  kTaskBwd = 6,     // {s, r0, -, -}: backward-solve partial block
  kTaskAsm = 7,     // {t, cb, first, end}: owner assembly group (see Sym::asm_src)
  kTaskSchur128 = 8,  // {s, i0, k0, oz}: 128 x 128 tile of U_s; oz = first slice row of s
  kTaskOzSlice = 9,   // {s, r0, oz, y}: slices of rows r0 .. r0+127 of s's A21 or L21 (FP64
                      //   only); the same rows' tensor-core TRSM with the inverse's slices at y
                      //   (y = -1: s keeps the FP64 TRSM)
  kTaskTrsmRest = 10, // {s, r0, -, -}: kTaskTrsm without the 128-tile supernodes
  kNumTaskKinds = 11
};
inline int schur_kind(int cls) { return cls == kTile128 ? kTaskSchur128 : kTaskSchur64 + cls; }

// Device descriptor of one supernode (absolute device pointers: descriptors of several
// matrices can be concatenated into one batch).
struct alignas(16) SnDev {
  void* L;              // panel, m x n column-major, ld = m (double or float)
  const int32_t* rows;  // m row indices (matrix numbering), ascending; first n = own columns
  int32_t n, m;         // columns, rows
  int32_t col0;         // first column
  int32_t mat;          // index into the MatDev array
  int64_t ustage;       // owner assembly: offset of U_s in the level staging buffer (-1 none)
  int32_t run0, nrun;   // target runs of the off-diagonal rows (MatDev::run_a / run_base)
  void* dinv;           // inverse of the diagonal block L11, n x n column-major (lower
                        // triangle; the panel's precision), or null (not kept)
};

struct alignas(16) MatDev {
  const int32_t* col2sn;          // column -> supernode index (matrix-local)
  int32_t sn_base;                // index of supernode 0 of this matrix in the SnDev array
  int32_t pad0;
  void* stage;                    // owner assembly: the level staging buffer of this matrix
  // relative map: the off-diagonal rows of supernode s fall into runs of one target each;
  // run r starts at row position run_a[r] (0-based among the u off-diagonal rows) and the
  // position inside the target's row list of off-diagonal row i >= run_a[r] is
  // relmap[run_base[r] + i] (run_base already has run_a subtracted)
  const int32_t* run_a;
  const int64_t* run_base;
  const int32_t* relmap;
  unsigned long long* err;        // err[0]: smallest failing column + 1 (all ones = none),
                                  // kept by atomicMin;
                                  // err[1]: relative-map misses (internal check, 0 expected)
                                  // err[2]: FP64 pivot redos of the mixed factor
                                  // err[3]: tensor-core waits that gave up (0 expected)
};

// Which Schur tile size a supernode gets (autotuned per matrix family): 128x128 tiles when
// it has at least min_rows_tile128 off-diagonal rows and its level holds at least
// min_level_tiles128 such tiles, else 64x64 under the same rule with the 64 thresholds, else
// 32x32 from min_rows_tile32 rows, else 16x16.
// granularity: kGranTiles uses the size thresholds alone; the other rules apply the
// paper's task-granularity heuristics (Sec. 4) to GPU tiles: a supernode's Schur update is
// the outer task, its tiles under the size thresholds the inner tasks it would create; an
// outer task with more than D inner tasks (D from OPT-D, Sec. 4.1, Algorithm 1) is split
// into those tiles, the others are kept whole (the coarsest tile class that covers the
// update in one task, 128 wide above 64 rows); kGranOptDCost also keeps whole any outer
// task whose inner tasks would each carry fewer than 50,000 flops (OPT-D-COST, Sec. 4.2);
// kGranHybrid takes the size thresholds when the average supernode size is above 50, or
// above 20 with density below 1e-4, and OPT-D-COST otherwise (the hybrid rule, Sec. 4.3).
enum Granularity { kGranTiles = 0, kGranOptD = 1, kGranOptDCost = 2, kGranHybrid = 3 };

struct TilePolicy {
  int min_rows_tile64 = 64;
  int min_rows_tile32 = 17;
  int min_level_tiles64 = 2 * 152;
  int min_rows_tile128 = 128;
  int min_level_tiles128 = 0;
  int granularity = kGranTiles;
  // FP64: a level's 128-tile supernodes take the tensor-core TRSM when their off-diagonal rows
  // add up to at least this many (below, the inverse's FP64 latency on one SM per supernode
  // outweighs the FP64 TRSM it replaces)
  int min_rows_trsm_tc = 8192;
};

// Host-side symbolic analysis result.
struct Sym {
  TilePolicy policy;
  int64_t n = 0, nnz_a = 0;
  int width_cap = 64;
  std::vector<int32_t> perm, iperm;
  std::vector<int64_t> a_colptr;   // A's lower CSC as given (original numbering)
  std::vector<int32_t> a_rowind;
  // full symmetric A in CSR form for the FP64 residual: row i holds columns csr_col[e]
  // with values vals[csr_src[e]] for e in [csr_ptr[i], csr_ptr[i+1])
  std::vector<int64_t> csr_ptr;
  std::vector<int32_t> csr_col, csr_src;
  std::vector<int32_t> parent;
  std::vector<int64_t> colcount;
  int32_t ns = 0;
  std::vector<int32_t> sn_start;   // ns + 1
  std::vector<int32_t> sn_m;       // rows of each supernode
  std::vector<int64_t> sn_rowptr;  // ns + 1 offsets into rows
  std::vector<int32_t> rows;
  std::vector<int64_t> sn_valptr;  // ns + 1 offsets into panel storage
  std::vector<int64_t> sn_dinvptr; // ns + 1 offsets of the diagonal-block inverses (n_s^2 each)
  std::vector<int32_t> sn_parent, sn_level;
  std::vector<int32_t> col2sn;     // n
  std::vector<int64_t> amap;       // nnz_a: panel offset of every stored entry of A
  int32_t nlev = 0;
  std::vector<int32_t> lvl_ptr, lvl_sn;
  std::vector<int32_t> lvl_maxw;  // widest supernode of each level (launch sizes of the solves)
  // task lists: tasks[k] holds all tasks of kind k, level l occupies
  // [task_off[k][l], task_off[k][l+1])
  std::vector<int32_t> tasks[kNumTaskKinds];      // 4 ints per task
  std::vector<int64_t> task_off[kNumTaskKinds];   // nlev + 1
  // owner assembly: staging offsets of U_s inside its level's buffer, and the size
  int64_t stage_elems = 0;
  // relative map (see MatDev): runs of each supernode's off-diagonal rows by target,
  // sn_run0[s] .. sn_run0[s+1]; run_a / run_t / run_base per run; relmap_size entries
  std::vector<int32_t> sn_run0, run_a, run_t;
  std::vector<int64_t> run_base;
  int64_t relmap_size = 0;
  // slice rows of the 128-tile supernodes of each level (rounded up to 8 per supernode),
  // and the largest level's count plus one tile of slack (rows a tile may read past u)
  std::vector<int64_t> lvl_ozrows;
  int64_t oz_rows = 0;
  // slice rows of the diagonal-block inverses of the supernodes whose TRSM runs on the tensor
  // cores (64 per supernode), and those supernodes' count, per level
  std::vector<int64_t> lvl_oyrows;
  std::vector<int32_t> lvl_trsmoz;
  int64_t oy_rows = 0;
  std::vector<int64_t> sn_ustage;  // ns
  // sources of the owner-assembly groups: {s, kb, ke, 0}, columns [kb, ke) of U_s
  std::vector<int32_t> asm_src;
  // owner-ordered forward solve: the rows updated by level l are fg_row[fg_lvl[l] ..
  // fg_lvl[l+1]); row i sums the staged contributions fg_ent[fg_ptr[i] .. fg_ptr[i+1])
  // (level-local slots q * kSolveRows + ii of forward task q), in ascending source order
  std::vector<int64_t> fg_lvl, fg_ptr;
  std::vector<int32_t> fg_row, fg_ent;
  int64_t max_fwd_per_level = 0;
  bool owner_lists = false;  // asm groups and gather lists built (build_owner_lists)
  // algorithmic flops of each task kind per level (POTRF n(n+1)(2n+1)/6, TRSM u n^2,
  // Schur u(u+1)n per supernode; they add up to sum_j c_j^2) and panel bytes per level
  std::vector<double> lvl_flops[kNumTaskKinds];
  std::vector<double> lvl_panel_bytes;
  double flops = 0.0;        // sum of c_j^2 over the exact factor
  double flops_panel = 0.0;  // the same over the padded panels (relaxed amalgamation)
  int64_t nnz_l = 0, l_storage = 0, max_width = 0, max_rows = 0;
  int64_t l_dinv = 0;  // values of all diagonal-block inverses (sum of n_s^2)
  int64_t n_fundamental = 0;  // fundamental supernodes before amalgamation and the cap
  // the granularity rule applied by the last build_schur_tasks (kGranHybrid resolved), its
  // threshold D (-1 under kGranTiles) and the number of outer tasks split
  int gran_rule = kGranTiles;
  int32_t gran_D = -1, gran_split = 0;
};

// Host analysis (analyze.cpp).  relax > 0 enables relaxed amalgamation with that largest
// share of explicit zeros for wide merges; relax <= 0 keeps the fundamental supernodes.
// Returns CHOL_OK or CHOL_E_INVALID.
int analyze(int64_t n, const int64_t* colptr, const int32_t* rowind, const int32_t* perm,
            int width_cap, double relax, Sym* out);
// Builds the owner-assembly groups (kTaskAsm, asm_src) and the owner-ordered forward-solve
// gather lists; only factors with owner-ordered assembly need them.
void build_owner_lists(Sym* S);
// (Re)builds the Schur tile task lists of every level under a tile policy.
void build_schur_tasks(Sym* S, const TilePolicy& policy);
// Threshold D of OPT-D (Sec. 4.1, Algorithm 1) for nsuper outer tasks with counts[i] >= 0
// inner tasks each, n the matrix size.
int32_t opt_d_threshold(int64_t n, int32_t nsuper, const int32_t* counts);
// Subtree-to-device partition of a forest (parent[v] = -1 at a root, work[v] >= 0): see
// chol_partition_tree.  Returns the imbalance of the chosen layer (max part / mean part).
double partition_tree(int32_t nv, const int32_t* parent, const double* work, int nparts,
                      double tol, int32_t* owner);

}  // namespace chol
