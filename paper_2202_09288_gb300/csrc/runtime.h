// runtime.h -- internal runtime state shared by the translation units of the library:
// the handle structures behind the C ABI, device allocation, tracing and launch helpers.
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <set>
#include <unordered_map>
#include <vector>

#include "../../include/chol.h"
#include "chol_internal.h"

using chol::MatDev;
using chol::SnDev;
using chol::Sym;

// Kernel kinds of the tracing counters.
enum ProfKindId {
  kProfAssemble, kProfPotrf, kProfTrsm, kProfSchur64, kProfSchur32, kProfSchur16,
  kProfAsmOwner, kProfFwd, kProfBwd, kProfPerm, kProfScale, kProfPotrfF32, kProfTrsmF32,
  kProfSchur64F32, kProfSchur32F32, kProfSchur16F32, kProfRefine, kProfGraph, kProfSchur128,
  kProfSchur128Tc, kProfOzSlice, kProfSchur128Oz, kProfDinv, kProfTrsmOz, kNumProf
};
inline const char* const kProfNames[kNumProf] = {
    "assemble",    "potrf_f64",   "trsm_f64",    "schur64_f64",  "schur32_f64",
    "schur16_f64", "assemble_owner", "solve_fwd", "solve_bwd",   "solve_perm",
    "equilibrate", "potrf_f32",   "trsm_f32",    "schur64_f32",  "schur32_f32",
    "schur16_f32", "refine",      "batch_graph", "schur128_f64", "schur128_tc",
    "oz_slice",    "schur128_oz", "diag_inverse", "trsm_oz"};

// Tracing kind of a Schur tile class (oz: FP64 128-tiles on the bf16 tensor cores).
inline int prof_schur_kind(int cls, bool f32, bool oz = false) {
  if (cls == chol::kTile128) return f32 ? kProfSchur128Tc : (oz ? kProfSchur128Oz : kProfSchur128);
  return (f32 ? kProfSchur64F32 : kProfSchur64) + cls;
}

struct ProfPending {
  int kind;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct chol_ctx {
  chol_opts opts;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaMemPool_t pool = nullptr;
  size_t held = 0;
  bool attrs_set = false;
  long long acc_wait = 0;  // tensor-core Schur consumers' accumulator wait bound (0: default)
  // tracing
  bool prof_on = false;
  int prof_only = -1;  // kind whose launches alone are bracketed (-1: every kind)
  chol_prof_entry prof[kNumProf];
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> spare_events;
  cudaEvent_t open_event = nullptr;
  // handles holding device memory of this context; chol_destroy detaches them
  std::set<chol_sym*> syms;
  std::set<chol_num*> nums;
  std::set<chol_batch*> batches;
  std::unordered_map<void*, size_t> sizes;  // live allocations (budget accounting)
};

struct DevSym {
  int device = -1;
  int32_t* rows = nullptr;
  int32_t* col2sn = nullptr;
  int64_t* amap = nullptr;
  int32_t* perm = nullptr;
  int32_t* iperm = nullptr;
  int64_t* a_colptr = nullptr;
  int32_t* a_rowind = nullptr;
  int64_t* csr_ptr = nullptr;
  int32_t* csr_col = nullptr;
  int32_t* csr_src = nullptr;
  int4* tasks[chol::kNumTaskKinds] = {};
  int4* asm_src = nullptr;
  int64_t* fg_ptr = nullptr;
  int32_t* fg_row = nullptr;
  int32_t* fg_ent = nullptr;
  // relative map (MatDev::relmap) and the arrays it is built from
  int32_t* sn_start = nullptr;
  int64_t* sn_rowptr = nullptr;
  int32_t* sn_run0 = nullptr;
  int32_t* run_a = nullptr;
  int32_t* run_t = nullptr;
  int64_t* run_base = nullptr;
  int32_t* relmap = nullptr;
  size_t bytes = 0;
};

struct chol_sym {
  Sym S;
  DevSym dev;
  chol_ctx* ctx = nullptr;  // context that holds dev (set at upload)
  int64_t max_bwd_per_level = 0;
};

struct chol_num {
  chol_ctx* ctx = nullptr;
  const chol_sym* sym = nullptr;
  int precision = CHOL_FP64;
  int assembly = CHOL_ASSEMBLY_ATOMIC;
  void* L = nullptr;           // panels (double, or float for CHOL_MIXED)
  SnDev* d_sn = nullptr;
  MatDev* d_mat = nullptr;
  int* d_ctr = nullptr;        // work-queue counters: factor launches, then solve launches
  unsigned long long* d_err = nullptr;  // [0] failing column + 1, [1] map misses,
                                        // [2] FP64 pivot redos
  double* d_vals = nullptr;    // device copy of A's values (assembly and residual)
  double* d_stage = nullptr;   // owner assembly staging
  double* d_scale = nullptr;   // CHOL_MIXED: equilibration a_jj^{-1/2}
  void* d_oz = nullptr;        // FP64 tensor-core Schur: operand slices (zeroed scratch)
  void* d_dinv = nullptr;      // inverses of the diagonal blocks (W <= 64; panel precision)
  int64_t oz_cap = 0;          // slice rows d_oz holds
  void* d_oy = nullptr;        // FP64 tensor-core TRSM: slices of the diagonal-block inverses
  int64_t oy_cap = 0;          // slice rows d_oy holds
  // solve workspace, grown on demand
  int64_t ws_nrhs = 0;
  double* d_y = nullptr;
  double* d_w = nullptr;
  double* d_part = nullptr;
  double* d_bx = nullptr;      // host-call staging of B / X
  double* d_fstage = nullptr;  // owner-ordered forward-solve staging
  // refinement workspace
  int64_t rws_nrhs = 0;
  double* d_rr = nullptr;      // residual
  double* d_rd = nullptr;      // correction
  double* d_rb = nullptr;      // host-call staging of B
  unsigned long long* d_norm = nullptr;  // per-column max |r|, max |x|, and ||A||_inf
  double anorm = -1.0;         // ||A||_inf of the current values (-1: not computed)
  chol_num* fb = nullptr;      // FP64 factor made when refinement of a mixed one stalls
  // flexible-GMRES refinement workspace (chol_refine_gmres), grown on demand
  int gm_cap = 0;              // Krylov vectors the workspace holds (restart length)
  double* d_gv = nullptr;      // V: n x (cap + 1), orthonormal basis
  double* d_gz = nullptr;      // Z: n x cap, preconditioned basis vectors
  double* d_gw = nullptr;      // w: n
  double* d_gpart = nullptr;   // dot-product partial sums
  double* d_gh = nullptr;      // dot products / coefficients of one step
};


namespace chol {
namespace rt {

// Per-level task lists of one matrix or of a batch: kind k at level l is
// d[k][off[k][l] .. off[k][l+1]) (device), with algorithmic flops flops[k][l] (host).
struct TaskView {
  const int4* d[kNumTaskKinds] = {};
  const int64_t* off[kNumTaskKinds] = {};
  const double* flops[kNumTaskKinds] = {};
  const int4* asm_src = nullptr;
  const int32_t* trsmoz = nullptr;  // per level: supernodes whose TRSM runs on the tensor cores
  int32_t nlev = 0;
  int max_width = 0;
  const int4* level(int k, int32_t l, int* count) const {
    *count = (int)(off[k][l + 1] - off[k][l]);
    return d[k] + off[k][l];
  }
};

int enqueue_assembly(chol_num* f);
int enqueue_factor(chol_num* f);
// Releases the device memory of every batch of c (called by chol_destroy).
void detach_batches(chol_ctx* c);
TaskView sym_view(const chol_sym* sym);
// Work-queue counters (one int per task launch): 7 per level for a factorization (POTRF,
// TRSM, four Schur tile classes, owner assembly), 3 per level for a solve.
constexpr int kFactorCountersPerLevel = 3 + chol::kNumTileClasses;
inline size_t factor_counters(int32_t nlev) { return kFactorCountersPerLevel * (size_t)nlev + 8; }
// Counters of a solve, zeroed at its start: 3 work-queue counters per level, then (from
// solve_arrive_offset) one arrival counter per supernode for the backward step.
inline size_t solve_arrive_offset(const Sym& S) { return 3 * (size_t)S.nlev + 8; }
inline size_t solve_counters(const Sym& S) { return solve_arrive_offset(S) + (size_t)S.ns; }
// oz / oz_rows: slice scratch of FP64 128-tiles on the bf16 tensor cores (null: those
// tiles run as 64 x 64 DMMA tiles)
// oz: the slice scratch of the tensor-core Schur tiles (FP64 slices or TF32 parts); oy (FP64
// only): the scratch of the diagonal-block inverses' slices, which also selects the
// tensor-core TRSM of the 128-tile supernodes.
// One request of a group refinement (refine_group): host right-hand sides B (n x k, ld ldb)
// and solution X (ld ldx); info and status are outputs.
struct GroupItem {
  chol_num* f = nullptr;
  int k = 0;
  const double* B = nullptr;
  int64_t ldb = 0;
  double* X = nullptr;
  int64_t ldx = 0;
  double tol = 0.0;
  int maxit = 10;
  chol_refine_info info{};
  int status = CHOL_OK;
};
int refine_group(chol_ctx* c, std::vector<GroupItem>& g);
int enqueue_levels(chol_ctx* c, const TaskView& v, const SnDev* sns, const MatDev* mats,
                   bool f32, bool owner, int* ctr, void* oz = nullptr, int64_t oz_rows = 0,
                   void* oy = nullptr, int64_t oy_rows = 0);
// Grows a zeroed slice scratch to at least `rows` rows (oz_scratch_bytes, or oy_scratch_bytes
// for the inverses' slices), freeing the old one only after the stream drains.
int grow_scratch(chol_ctx* c, void** buf, int64_t* cap, int64_t rows, bool inverses);
// Whether FP64 factors of sym under c's options use the bf16 tensor-core Schur tiles.
bool use_oz(const chol_ctx* c, const chol_sym* sym);
void fill_descriptors(const chol_num* f, int mat, int32_t sn_base, std::vector<SnDev>* sn,
                      MatDev* md);

int dev_alloc(chol_ctx* c, void** p, size_t bytes);
void dev_free(chol_ctx* c, void* p);
void prof_begin(chol_ctx* c, int kind);
void prof_end(chol_ctx* c, int k, double flops, double bytes);
const int4* task_ptr(const chol_sym* s, int kind, int32_t level, int* count);
int ensure_uploaded(chol_ctx* c, chol_sym* s);
int ensure_attrs(chol_ctx* c);
int ensure_solve_ws(chol_num* f, int64_t nrhs);
int ensure_refine_ws(chol_num* f, int64_t k);
// ||A||_inf of f's values, computed once per set of values.
int compute_anorm(chol_num* f);
// R = B - A X into f's residual buffer (k <= 32 columns); *rel = max_c ||r_c||_inf /
// (||A||_inf ||x_c||_inf), *rmax = max_c ||r_c||_inf (synchronizes).
int residual_norms(chol_num* f, int k, const double* B, int64_t ldb, const double* X,
                   int64_t ldx, double* rel, double* rmax);
int enqueue_solve(chol_num* f, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx);
// Allocates a factor of sym and copies vals into it; with factor_now it also enqueues the
// factorization (otherwise a batch will factor it).
int make_factor(chol_ctx* c, chol_sym* sym, const double* vals, int where, int precision,
                int assembly, chol_num** out, bool factor_now);
// Bytes of device memory a factor of sym holds (panels, values, descriptors, staging).
size_t factor_bytes(const chol_sym* sym, int precision, int assembly);
// A copy of the host analysis of src, not bound to any device (nullptr when out of memory).
chol_sym* clone_sym(const chol_sym* src);
// Bytes of the device copy of sym, and of the solve + refinement workspace for k columns.
size_t sym_upload_bytes(const chol_sym* sym);
size_t solve_ws_bytes(const chol_sym* sym, int64_t k, int assembly);

}  // namespace rt
}  // namespace chol
