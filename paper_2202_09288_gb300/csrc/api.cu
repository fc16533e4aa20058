// api.cu -- the C ABI (include/chol.h): contexts, device memory, upload of the symbolic
// analysis, the per-level launch sequences of the factorization and the solves, and the
// iterative-refinement driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "chol_internal.h"
#include "kernels.h"
#include "runtime.h"

using namespace chol::rt;

namespace chol {
namespace rt {

constexpr int kNormSlots = 2 * 32 + 1;

cudaEvent_t prof_event(chol_ctx* c) {
  cudaEvent_t e = nullptr;
  if (!c->spare_events.empty()) {
    e = c->spare_events.back();
    c->spare_events.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}

// Brackets one launch of kind k (the launch count is always kept).  With a kind selected
// by chol_profile_only, only launches of that kind are bracketed: prof_begin(c, k) of
// another kind records nothing.
void prof_begin(chol_ctx* c, int k) {
  if (!c->prof_on || (c->prof_only >= 0 && k != c->prof_only)) return;
  c->open_event = prof_event(c);
  if (c->open_event) cudaEventRecord(c->open_event, c->stream);
}

void prof_end(chol_ctx* c, int k, double flops, double bytes) {
  c->prof[k].launches++;
  if (!c->prof_on || !c->open_event) return;
  cudaEvent_t b = prof_event(c);
  if (!b) return;
  cudaEventRecord(b, c->stream);
  c->pending.push_back({k, c->open_event, b, flops, bytes});
  c->open_event = nullptr;
}

void prof_fold(chol_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof[p.kind].ms += ms;
      c->prof[p.kind].timed++;
      c->prof[p.kind].flops += p.flops;
      c->prof[p.kind].bytes += p.bytes;
    } else {
      cudaGetLastError();
    }
    c->spare_events.push_back(p.a);
    c->spare_events.push_back(p.b);
  }
  c->pending.clear();
}

void prof_reset(chol_ctx* c) {
  for (int k = 0; k < kNumProf; k++) {
    memset(&c->prof[k], 0, sizeof(chol_prof_entry));
    snprintf(c->prof[k].name, sizeof(c->prof[k].name), "%s", kProfNames[k]);
  }
}

#define CK(call)                                   \
  do {                                             \
    if ((call) != cudaSuccess) {                   \
      cudaGetLastError();                          \
      return CHOL_E_CUDA;                          \
    }                                              \
  } while (0)

int dev_alloc(chol_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->opts.hbm_budget && c->held + bytes > c->opts.hbm_budget) return CHOL_E_OOM;
  if (cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return CHOL_E_OOM;
  }
  c->held += bytes;
  c->sizes[*p] = bytes;
  return CHOL_OK;
}

void dev_free(chol_ctx* c, void* p) {
  if (!p) return;
  cudaFreeAsync(p, c->stream);
  auto it = c->sizes.find(p);
  if (it != c->sizes.end()) {
    c->held -= std::min(c->held, it->second);
    c->sizes.erase(it);
  }
}

template <typename T>
int upload(chol_ctx* c, T** dst, const std::vector<T>& v, size_t* acc) {
  size_t bytes = v.size() * sizeof(T);
  int rc = dev_alloc(c, (void**)dst, bytes);
  if (rc) return rc;
  *acc += bytes ? bytes : 16;
  if (bytes) CK(cudaMemcpyAsync(*dst, v.data(), bytes, cudaMemcpyHostToDevice, c->stream));
  return CHOL_OK;
}

void free_devsym(chol_sym* s) {
  if (!s->ctx) return;
  chol_ctx* c = s->ctx;
  DevSym& d = s->dev;
  void* ptrs[] = {d.rows,     d.col2sn,   d.amap,   d.perm,    d.iperm,  d.a_colptr,
                  d.a_rowind, d.csr_ptr,  d.csr_col, d.csr_src, d.asm_src, d.fg_ptr,
                  d.fg_row,   d.fg_ent,   d.sn_start, d.sn_rowptr, d.sn_run0, d.run_a,
                  d.run_t,    d.run_base, d.relmap};
  for (void* p : ptrs) dev_free(c, p);
  for (int k = 0; k < chol::kNumTaskKinds; k++) dev_free(c, d.tasks[k]);
  d = DevSym();
  c->syms.erase(s);
  s->ctx = nullptr;
}

int ensure_uploaded(chol_ctx* c, chol_sym* s) {
  if (s->ctx == c) return CHOL_OK;
  if (s->ctx) return CHOL_E_INVALID;  // bound to another context
  const Sym& S = s->S;
  DevSym& d = s->dev;
  size_t acc = 0;
  int rc;
  s->ctx = c;
  c->syms.insert(s);
  if ((rc = upload(c, &d.rows, S.rows, &acc)) || (rc = upload(c, &d.col2sn, S.col2sn, &acc)) ||
      (rc = upload(c, &d.amap, S.amap, &acc)) || (rc = upload(c, &d.perm, S.perm, &acc)) ||
      (rc = upload(c, &d.iperm, S.iperm, &acc)) ||
      (rc = upload(c, &d.a_colptr, S.a_colptr, &acc)) ||
      (rc = upload(c, &d.a_rowind, S.a_rowind, &acc)) ||
      (rc = upload(c, &d.csr_ptr, S.csr_ptr, &acc)) ||
      (rc = upload(c, &d.csr_col, S.csr_col, &acc)) ||
      (rc = upload(c, &d.csr_src, S.csr_src, &acc)) ||
      (rc = upload(c, reinterpret_cast<int32_t**>(&d.asm_src), S.asm_src, &acc)) ||
      (rc = upload(c, &d.fg_ptr, S.fg_ptr, &acc)) || (rc = upload(c, &d.fg_row, S.fg_row, &acc)) ||
      (rc = upload(c, &d.fg_ent, S.fg_ent, &acc))) {
    free_devsym(s);
    return rc;
  }
  for (int k = 0; k < chol::kNumTaskKinds; k++)
    if ((rc = upload(c, reinterpret_cast<int32_t**>(&d.tasks[k]), S.tasks[k], &acc))) {
      free_devsym(s);
      return rc;
    }
  // the relative map, built once per pattern on the device
  unsigned long long* miss = nullptr;
  if ((rc = upload(c, &d.sn_start, S.sn_start, &acc)) ||
      (rc = upload(c, &d.sn_rowptr, S.sn_rowptr, &acc)) ||
      (rc = upload(c, &d.sn_run0, S.sn_run0, &acc)) || (rc = upload(c, &d.run_a, S.run_a, &acc)) ||
      (rc = upload(c, &d.run_t, S.run_t, &acc)) ||
      (rc = upload(c, &d.run_base, S.run_base, &acc)) ||
      (rc = dev_alloc(c, (void**)&d.relmap, (size_t)S.relmap_size * sizeof(int32_t))) ||
      (rc = dev_alloc(c, (void**)&miss, sizeof(unsigned long long)))) {
    dev_free(c, miss);
    free_devsym(s);
    return rc;
  }
  acc += (size_t)S.relmap_size * sizeof(int32_t);
  unsigned long long hmiss = 0;
  if (cudaMemsetAsync(miss, 0, sizeof(hmiss), c->stream) != cudaSuccess) rc = CHOL_E_CUDA;
  if (!rc) {
    chol::launch_build_relmap(S.ns, d.sn_start, d.sn_rowptr, d.rows, d.sn_run0, d.run_a, d.run_t,
                              d.run_base, d.relmap, miss, c->stream);
    if (cudaMemcpyAsync(&hmiss, miss, sizeof(hmiss), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      rc = CHOL_E_CUDA;
    else if (hmiss)
      rc = CHOL_E_INVALID;  // rows missing from an ancestor: an inconsistent analysis
  }
  dev_free(c, miss);
  if (rc) {
    cudaGetLastError();
    free_devsym(s);
    return rc;
  }
  d.bytes = acc;
  d.device = c->opts.device;
  int64_t mb = 0;
  for (int32_t l = 0; l < S.nlev; l++)
    mb = std::max(mb, S.task_off[chol::kTaskBwd][l + 1] - S.task_off[chol::kTaskBwd][l]);
  s->max_bwd_per_level = mb;
  return CHOL_OK;
}

chol_sym* clone_sym(const chol_sym* src) {
  chol_sym* s = new (std::nothrow) chol_sym();
  if (!s) return nullptr;
  try {
    s->S = src->S;
  } catch (...) {
    delete s;
    return nullptr;
  }
  return s;
}

// Builds the owner-assembly lists of sym on first use by an owner-mode factor and, if sym
// is already on the device, uploads them.
int ensure_owner_lists(chol_ctx* c, chol_sym* s) {
  if (s->S.owner_lists) return CHOL_OK;
  try {
    chol::build_owner_lists(&s->S);
  } catch (...) {
    return CHOL_E_OOM;
  }
  if (s->ctx != c) return CHOL_OK;  // uploaded with everything else later
  DevSym& d = s->dev;
  const Sym& S = s->S;
  dev_free(c, d.asm_src);
  dev_free(c, d.fg_ptr);
  dev_free(c, d.fg_row);
  dev_free(c, d.fg_ent);
  dev_free(c, d.tasks[chol::kTaskAsm]);
  d.asm_src = nullptr;
  d.fg_ptr = nullptr;
  d.fg_row = d.fg_ent = nullptr;
  d.tasks[chol::kTaskAsm] = nullptr;
  size_t acc = 0;
  int rc;
  if ((rc = upload(c, reinterpret_cast<int32_t**>(&d.asm_src), S.asm_src, &acc)) ||
      (rc = upload(c, &d.fg_ptr, S.fg_ptr, &acc)) || (rc = upload(c, &d.fg_row, S.fg_row, &acc)) ||
      (rc = upload(c, &d.fg_ent, S.fg_ent, &acc)) ||
      (rc = upload(c, reinterpret_cast<int32_t**>(&d.tasks[chol::kTaskAsm]), S.tasks[chol::kTaskAsm],
                   &acc)))
    return rc;
  d.bytes += acc;
  return CHOL_OK;
}

int ensure_attrs(chol_ctx* c) {
  if (c->attrs_set) return CHOL_OK;
  int rc = chol::set_factor_kernel_attrs(chol::kMaxWidth);
  if (rc) return rc;
  rc = chol::set_solve_kernel_attrs(chol::kMaxWidth, 32);
  if (rc) return rc;
  rc = chol::set_tc_kernel_attrs();
  if (rc) return rc;
  rc = chol::set_oz_kernel_attrs();
  if (rc) return rc;
  c->attrs_set = true;
  return CHOL_OK;
}

const int4* task_ptr(const chol_sym* s, int kind, int32_t level, int* count) {
  const Sym& S = s->S;
  int64_t a = S.task_off[kind][level], b = S.task_off[kind][level + 1];
  *count = (int)(b - a);
  return s->dev.tasks[kind] + a;
}

// Zeroes the panels and error words of f and assembles its values (f->d_vals) into them
// (FP64), or equilibrates and assembles them (CHOL_MIXED).
int enqueue_assembly(chol_num* f) {
  chol_ctx* c = f->ctx;
  const chol_sym* sym = f->sym;
  const Sym& S = sym->S;
  cudaStream_t st = c->stream;
  const bool f32 = f->precision == CHOL_MIXED;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  // err[0] = smallest failing column + 1, kept by atomicMin: starts at all ones (none);
  // err[1] = relative-map misses, err[2] = FP64 pivot redos, err[3] = tensor-core wait
  // timeouts: start at 0
  CK(cudaMemsetAsync(f->d_err, 0xff, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(f->d_err + 1, 0, 3 * sizeof(unsigned long long), st));
  f->anorm = -1.0;
  prof_begin(c, f32 ? kProfScale : kProfAssemble);
  CK(cudaMemsetAsync(f->L, 0, (size_t)S.l_storage * esz, st));
  if (f32) {
    chol::launch_diag_scale(sym->dev.a_colptr, sym->dev.a_rowind, f->d_vals, sym->dev.iperm,
                            S.n, f->d_scale, f->d_err, st);
    chol::launch_assemble_scaled(sym->dev.a_colptr, sym->dev.a_rowind, f->d_vals,
                                 sym->dev.amap, f->d_scale, S.n, (float*)f->L, st);
    prof_end(c, kProfScale, 0.0, (double)S.l_storage * esz + 24.0 * S.nnz_a);
  } else {
    chol::launch_assemble(f->d_vals, sym->dev.amap, S.nnz_a, f->L, false, st);
    prof_end(c, kProfAssemble, 0.0, (double)S.l_storage * esz + 16.0 * S.nnz_a + 8.0 * S.nnz_a);
  }
  return CHOL_OK;
}

// The task lists of one matrix, as a view for enqueue_levels.
TaskView sym_view(const chol_sym* sym) {
  const Sym& S = sym->S;
  TaskView v;
  for (int k = 0; k < chol::kNumTaskKinds; k++) {
    v.d[k] = sym->dev.tasks[k];
    v.off[k] = S.task_off[k].data();
    v.flops[k] = S.lvl_flops[k].data();
  }
  v.asm_src = sym->dev.asm_src;
  v.trsmoz = S.lvl_trsmoz.data();
  v.nlev = S.nlev;
  v.max_width = (int)S.max_width;
  return v;
}

// Per level: POTRF, TRSM, the Schur tile classes and (owner mode) the ordered assembly,
// each one launch over the level's tasks of every matrix in the view.
bool use_oz(const chol_ctx* c, const chol_sym* sym) {
  return c->opts.fp64_schur == CHOL_SCHUR_OZAKI && sym->S.max_width <= 64;
}

int enqueue_levels(chol_ctx* c, const TaskView& v, const SnDev* sns, const MatDev* mats,
                   bool f32, bool owner, int* ctr, void* oz, int64_t oz_rows, void* oy,
                   int64_t oy_rows) {
  // FP64 factors with the slice scratches: 128-tile supernodes take the tensor-core TRSM
  const bool trsm_oz = oz && oy && !f32;
  cudaStream_t st = c->stream;
  CK(cudaMemsetAsync(ctr, 0, factor_counters(v.nlev) * sizeof(int), st));
  const float tau = (float)(c->opts.pivot_tau > 0 ? c->opts.pivot_tau : 1e-5);
  const int kp = f32 ? kProfPotrfF32 : kProfPotrf, kt = f32 ? kProfTrsmF32 : kProfTrsm;
  for (int32_t l = 0; l < v.nlev; l++) {
    int cnt;
    int* q = ctr + kFactorCountersPerLevel * l;  // this level's work-queue counters
    const int4* t = v.level(chol::kTaskPotrf, l, &cnt);
    if (cnt > 0) {
      prof_begin(c, kp);
      chol::launch_potrf(t, cnt, q, sns, mats, v.max_width, f32, tau, trsm_oz ? oy : nullptr,
                         oy_rows, st);
      prof_end(c, kp, v.flops[chol::kTaskPotrf][l], 0.0);
    }
    t = v.level(trsm_oz ? chol::kTaskTrsmRest : chol::kTaskTrsm, l, &cnt);
    if (cnt > 0) {
      prof_begin(c, kt);
      chol::launch_trsm(t, cnt, q + 1, sns, v.max_width, f32, st);
      prof_end(c, kt, v.flops[trsm_oz ? chol::kTaskTrsmRest : chol::kTaskTrsm][l], 0.0);
    }
    // the 128-tile supernodes' TRSM: slices of A21 S^-1, then L21 = A21 Y^T on the tensor
    // cores
    if (trsm_oz && v.trsmoz[l] > 0) {
      t = v.level(chol::kTaskOzSlice, l, &cnt);
      if (cnt > 0) {
        prof_begin(c, kProfOzSlice);
        chol::launch_oz_slice(t, cnt, sns, oz, oz_rows, oy, oy_rows, st);
        prof_end(c, kProfOzSlice, 0.0, 0.0);
        prof_begin(c, kProfTrsmOz);
        chol::launch_trsm_oz(t, cnt, sns, mats, oz, oz_rows, oy, oy_rows, st);
        prof_end(c, kProfTrsmOz,
                 v.flops[chol::kTaskTrsm][l] - v.flops[chol::kTaskTrsmRest][l], 0.0);
      }
    }
    // 128-tiles on the tensor cores: FP64 by bf16 slices, FP32 by TF32 hi/lo parts; their
    // operands are prepared per level after TRSM
    if (oz) {
      t = v.level(chol::kTaskOzSlice, l, &cnt);
      if (cnt > 0) {
        prof_begin(c, kProfOzSlice);
        if (f32) chol::launch_tf32_split(t, cnt, sns, v.max_width, oz, oz_rows, st);
        else chol::launch_oz_slice(t, cnt, sns, oz, oz_rows, nullptr, 0, st);
        prof_end(c, kProfOzSlice, 0.0, 0.0);
      }
    }
    for (int cls = 0; cls < chol::kNumTileClasses; cls++) {
      const int kind = chol::schur_kind(cls);
      t = v.level(kind, l, &cnt);
      if (cnt <= 0) continue;
      const bool tcc = oz && cls == chol::kTile128;
      const int pk = prof_schur_kind(cls, f32, tcc && !f32);
      prof_begin(c, pk);
      if (tcc && f32)
        chol::launch_schur_tc(t, cnt, q + 2 + cls, sns, mats, owner, oz, oz_rows, c->acc_wait, st);
      else if (tcc)
        chol::launch_schur_oz(t, cnt, q + 2 + cls, sns, mats, owner, oz, oz_rows, c->acc_wait, st);
      else chol::launch_schur(cls, t, cnt, q + 2 + cls, sns, mats, owner, f32, st);
      prof_end(c, pk, v.flops[kind][l], 0.0);
    }
    if (owner) {
      t = v.level(chol::kTaskAsm, l, &cnt);
      if (cnt > 0) {
        prof_begin(c, kProfAsmOwner);
        chol::launch_assemble_owner(t, cnt, q + 2 + chol::kNumTileClasses, v.asm_src, sns, mats, f32, st);
        prof_end(c, kProfAsmOwner, 0.0, 0.0);
      }
    }
  }
  // the inverses of all finished diagonal blocks, for the solves (supernodes of factors that
  // keep them), in one launch over every POTRF task: nothing in the factorization needs
  // them, and per level the top of the tree would serialize their n-step chains
  {
    const int64_t* o = v.off[chol::kTaskPotrf];
    const int cnt = (int)(o[v.nlev] - o[0]);
    if (cnt > 0) {
      prof_begin(c, kProfDinv);
      chol::launch_diag_inverse(v.d[chol::kTaskPotrf] + o[0], cnt, sns, f32, trsm_oz, st);
      prof_end(c, kProfDinv, 0.0, 0.0);
    }
  }
  CK(cudaGetLastError());
  return CHOL_OK;
}

// Enqueues the numeric factorization of the values in f->d_vals.
// Slice scratch of a factor's FP64 tensor-core Schur tiles, grown to the analysis' need
// (a new tile policy can raise it) and zeroed when allocated.
int grow_scratch(chol_ctx* c, void** buf, int64_t* cap, int64_t rows, bool inverses) {
  if (*cap >= rows) return CHOL_OK;
  // the stream may still use the old scratch: free it only after the stream drains
  if (*buf) {
    CK(cudaStreamSynchronize(c->stream));
    dev_free(c, *buf);
    *buf = nullptr;
    *cap = 0;
  }
  const size_t bytes = inverses ? chol::oy_scratch_bytes(rows) : chol::oz_scratch_bytes(rows);
  int rc = dev_alloc(c, buf, bytes);
  if (rc) return rc;
  CK(cudaMemsetAsync(*buf, 0, bytes, c->stream));
  *cap = rows;
  return CHOL_OK;
}

int ensure_oz(chol_num* f, void** oz, int64_t* rows, void** oy, int64_t* oy_rows) {
  *oz = nullptr;
  *rows = 0;
  *oy = nullptr;
  *oy_rows = 0;
  const Sym& S = f->sym->S;
  // FP64: bf16 slices (W <= 64, unless the DMMA tiles are asked for); FP32: TF32 parts
  const bool need = f->precision == CHOL_MIXED ? true : use_oz(f->ctx, f->sym);
  if (!need || S.oz_rows <= 0) return CHOL_OK;
  int rc = grow_scratch(f->ctx, &f->d_oz, &f->oz_cap, S.oz_rows, false);
  if (rc) return rc;
  *oz = f->d_oz;
  *rows = f->oz_cap;
  // FP64: the slices of the 128-tile supernodes' diagonal-block inverses (tensor-core TRSM)
  if (f->precision != CHOL_MIXED && S.oy_rows > 0 && f->d_dinv) {
    if ((rc = grow_scratch(f->ctx, &f->d_oy, &f->oy_cap, S.oy_rows, true))) return rc;
    *oy = f->d_oy;
    *oy_rows = f->oy_cap;
  }
  return CHOL_OK;
}

int enqueue_factor(chol_num* f) {
  int rc = enqueue_assembly(f);
  if (rc) return rc;
  void *oz, *oy;
  int64_t oz_rows, oy_rows;
  if ((rc = ensure_oz(f, &oz, &oz_rows, &oy, &oy_rows))) return rc;
  return enqueue_levels(f->ctx, sym_view(f->sym), f->d_sn, f->d_mat,
                        f->precision == CHOL_MIXED, f->assembly == CHOL_ASSEMBLY_OWNER, f->d_ctr,
                        oz, oz_rows, oy, oy_rows);
}

// Device descriptors of f's supernodes (matrix slot `mat`) and of f itself.
void fill_descriptors(const chol_num* f, int mat, int32_t sn_base, std::vector<SnDev>* sn,
                      MatDev* md) {
  const chol_sym* sym = f->sym;
  const Sym& S = sym->S;
  const size_t esz = f->precision == CHOL_MIXED ? sizeof(float) : sizeof(double);
  const size_t first = sn->size();
  sn->resize(first + S.ns);
  for (int32_t s = 0; s < S.ns; s++) {
    SnDev& d = (*sn)[first + s];
    d.L = (char*)f->L + (size_t)S.sn_valptr[s] * esz;
    d.rows = sym->dev.rows + S.sn_rowptr[s];
    d.n = S.sn_start[s + 1] - S.sn_start[s];
    d.m = S.sn_m[s];
    d.col0 = S.sn_start[s];
    d.mat = mat;
    d.ustage = S.sn_ustage[s];
    d.run0 = S.sn_run0[s];
    d.nrun = S.sn_run0[s + 1] - S.sn_run0[s];
    d.dinv = f->d_dinv ? (char*)f->d_dinv + (size_t)S.sn_dinvptr[s] * esz : nullptr;
  }
  md->col2sn = sym->dev.col2sn;
  md->run_a = sym->dev.run_a;
  md->run_base = sym->dev.run_base;
  md->relmap = sym->dev.relmap;
  md->sn_base = sn_base;
  md->pad0 = 0;
  md->stage = f->d_stage;
  md->err = f->d_err;
}

int ensure_solve_ws(chol_num* f, int64_t nrhs) {
  if (f->ws_nrhs >= nrhs) return CHOL_OK;
  chol_ctx* c = f->ctx;
  const Sym& S = f->sym->S;
  const int64_t n = S.n;
  dev_free(c, f->d_y);
  dev_free(c, f->d_w);
  dev_free(c, f->d_bx);
  dev_free(c, f->d_part);
  dev_free(c, f->d_fstage);
  f->d_y = f->d_w = f->d_bx = f->d_part = f->d_fstage = nullptr;
  f->ws_nrhs = 0;
  int rc;
  if (f->assembly == CHOL_ASSEMBLY_OWNER &&
      (rc = dev_alloc(c, (void**)&f->d_fstage,
                      (size_t)S.max_fwd_per_level * chol::kSolveRows * nrhs * 8)))
    return rc;
  if ((rc = dev_alloc(c, (void**)&f->d_y, (size_t)n * nrhs * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_w, (size_t)n * nrhs * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_bx, (size_t)n * nrhs * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_part,
                      (size_t)f->sym->max_bwd_per_level * S.width_cap * nrhs * 8)))
    return rc;
  f->ws_nrhs = nrhs;
  return CHOL_OK;
}

// Work buffers of one device solve of k <= 32 right-hand sides: the work-queue counters
// (3 per level, zeroed by the solve), y and w (n x k each), the backward partial sums (the
// most backward tasks of a level x W x k) and, for owner assembly, the forward staging (the
// most forward tasks of a level x kSolveRows x k; null otherwise).
struct SolveBufs {
  int* sq;
  double* y;
  double* w;
  double* part;
  double* fstage;
};

// Tracing of one launch of the solve sequence: with trace, event brackets when profiling is
// on (prof_begin / prof_end); without, only the launch count (no event is created).
struct SolveTrace {
  chol_ctx* c;
  bool trace;
  void begin(int kind) const {
    if (trace) prof_begin(c, kind);
  }
  void end(int kind, double bytes) const {
    if (trace) prof_end(c, kind, 0.0, bytes);
    else c->prof[kind].launches++;
  }
};

// The launch sequence of a device-pointer solve of k <= 32 columns (Sec. 1: L y = P^T b
// over the levels from the leaves up, then L^T z = y from the root down, x = P z).
int enqueue_solve_seq(chol_ctx* c, const chol_num* f, int k, const double* B, int64_t ldb,
                      double* X, int64_t ldx, const SolveBufs& bf, bool trace) {
  const chol_sym* sym = f->sym;
  const Sym& S = sym->S;
  cudaStream_t st = c->stream;
  const int64_t n = S.n;
  const int W = S.width_cap;
  const bool f32 = f->precision == CHOL_MIXED;
  const double* scale = f32 ? f->d_scale : nullptr;
  const bool inv = f->d_dinv != nullptr;
  const double vec = 8.0 * n * k;
  const SolveTrace tr{c, trace};
  CK(cudaMemsetAsync(bf.sq, 0, solve_counters(S) * sizeof(int), st));
  tr.begin(kProfPerm);
  chol::launch_gather_perm(B, ldb, sym->dev.perm, scale, n, k, bf.y, st);
  tr.end(kProfPerm, 2 * vec + 4.0 * n);
  for (int32_t l = 0; l < S.nlev; l++) {
    int cnt;
    const int4* t = task_ptr(sym, chol::kTaskFwd, l, &cnt);
    tr.begin(kProfFwd);
    chol::launch_fwd(t, cnt, bf.sq + 3 * l, f->d_sn, n, k, S.lvl_maxw[l], bf.y, bf.w, bf.fstage,
                     inv, f32, st);
    if (bf.fstage)
      chol::launch_fwd_gather(sym->dev.fg_row + S.fg_lvl[l], sym->dev.fg_ptr + S.fg_lvl[l],
                              sym->dev.fg_ent, S.fg_lvl[l + 1] - S.fg_lvl[l], n, k, bf.fstage,
                              bf.y, st);
    tr.end(kProfFwd, S.lvl_panel_bytes[l] * (f32 ? 0.5 : 1.0));
  }
  int* arrive = bf.sq + solve_arrive_offset(S);
  for (int32_t l = S.nlev - 1; l >= 0; l--) {
    int nb;
    const int4* tb = task_ptr(sym, chol::kTaskBwd, l, &nb);
    tr.begin(kProfBwd);
    chol::launch_bwd(tb, nb, bf.sq + 3 * l + 1, f->d_sn, n, k, W, S.lvl_maxw[l], bf.w, bf.part,
                     arrive, inv, f32, st);
    tr.end(kProfBwd, S.lvl_panel_bytes[l] * (f32 ? 0.5 : 1.0));
  }
  tr.begin(kProfPerm);
  chol::launch_scatter_perm(bf.w, sym->dev.perm, scale, n, k, X, ldx, st);
  tr.end(kProfPerm, 2 * vec + 4.0 * n);
  CK(cudaGetLastError());
  return CHOL_OK;
}

// Device-pointer solve of nrhs <= 32 columns in the factor's own workspace.
int enqueue_solve(chol_num* f, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx) {
  const SolveBufs bf{f->d_ctr + factor_counters(f->sym->S.nlev), f->d_y, f->d_w, f->d_part,
                     f->d_fstage};
  return enqueue_solve_seq(f->ctx, f, nrhs, B, ldb, X, ldx, bf, true);
}

void free_num_buffers(chol_num* f) {
  chol_ctx* c = f->ctx;
  if (!c) return;
  void* ptrs[] = {f->L, f->d_sn, f->d_mat, f->d_err, f->d_ctr, f->d_vals, f->d_stage, f->d_scale,
                  f->d_y, f->d_w, f->d_bx, f->d_part, f->d_fstage, f->d_rr, f->d_rd,
                  f->d_rb, f->d_norm, f->d_oz, f->d_oy, f->d_gv, f->d_gz, f->d_gw, f->d_gpart,
                  f->d_gh, f->d_dinv};
  for (void* p : ptrs) dev_free(c, p);
  c->nums.erase(f);
  f->ctx = nullptr;
}

// Allocates a factor and enqueues its numeric factorization of vals.
int make_factor(chol_ctx* c, chol_sym* sym, const double* vals, int where, int precision,
                int assembly, chol_num** out, bool factor_now) {
  const Sym& S = sym->S;
  if (assembly == CHOL_ASSEMBLY_OWNER) {
    int rc0 = ensure_owner_lists(c, sym);
    if (rc0) return rc0;
  }
  chol_num* f = new (std::nothrow) chol_num();
  if (!f) return CHOL_E_OOM;
  f->ctx = c;
  c->nums.insert(f);
  f->sym = sym;
  f->precision = precision;
  f->assembly = assembly;
  const bool f32 = precision == CHOL_MIXED;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  int rc;
  if ((rc = dev_alloc(c, &f->L, (size_t)S.l_storage * esz)) ||
      (rc = dev_alloc(c, (void**)&f->d_sn, (size_t)S.ns * sizeof(SnDev))) ||
      (rc = dev_alloc(c, (void**)&f->d_mat, sizeof(MatDev))) ||
      (rc = dev_alloc(c, (void**)&f->d_err, 4 * sizeof(unsigned long long))) ||
      (rc = dev_alloc(c, (void**)&f->d_ctr,
                      (factor_counters(S.nlev) + solve_counters(S)) * sizeof(int))) ||
      (rc = dev_alloc(c, (void**)&f->d_vals, (size_t)S.nnz_a * 8)) ||
      (f32 && (rc = dev_alloc(c, (void**)&f->d_scale, (size_t)S.n * 8))) ||
      (assembly == CHOL_ASSEMBLY_OWNER &&
       (rc = dev_alloc(c, (void**)&f->d_stage, (size_t)S.stage_elems * 8))) ||
      (S.max_width <= chol::kDinvMaxWidth &&
       (rc = dev_alloc(c, &f->d_dinv, (size_t)S.l_dinv * esz)))) {
    free_num_buffers(f);
    delete f;
    return rc;
  }
  std::vector<SnDev> sn;
  MatDev md;
  fill_descriptors(f, 0, 0, &sn, &md);
  if (cudaMemcpyAsync(f->d_sn, sn.data(), sn.size() * sizeof(SnDev), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(f->d_mat, &md, sizeof(md), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    free_num_buffers(f);
    delete f;
    return CHOL_E_CUDA;
  }
  *out = f;
  if (factor_now) return chol_refactorize(c, f, vals, where);
  if (S.nnz_a > 0 && vals)
    CK(cudaMemcpyAsync(f->d_vals, vals, (size_t)S.nnz_a * 8,
                       where == CHOL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       c->stream));
  return CHOL_OK;
}

size_t sym_upload_bytes(const chol_sym* sym) {
  const Sym& S = sym->S;
  size_t b = S.rows.size() * 4 + S.col2sn.size() * 4 + S.amap.size() * 8 + S.perm.size() * 4 +
             S.iperm.size() * 4 + S.a_colptr.size() * 8 + S.a_rowind.size() * 4 +
             S.csr_ptr.size() * 8 + S.csr_col.size() * 4 + S.csr_src.size() * 4 +
             S.asm_src.size() * 4 + S.fg_ptr.size() * 8 + S.fg_row.size() * 4 +
             S.fg_ent.size() * 4;
  for (int k = 0; k < chol::kNumTaskKinds; k++) b += S.tasks[k].size() * 4;
  b += (size_t)S.relmap_size * 4 + S.run_a.size() * 16 + S.sn_run0.size() * 4 +
       S.sn_start.size() * 4 + S.sn_rowptr.size() * 8;
  return b + 64 * 16;
}

size_t solve_ws_bytes(const chol_sym* sym, int64_t k, int assembly) {
  const Sym& S = sym->S;
  int64_t mb = 0;
  for (int32_t l = 0; l < S.nlev; l++)
    mb = std::max(mb, S.task_off[chol::kTaskBwd][l + 1] - S.task_off[chol::kTaskBwd][l]);
  size_t b = 3 * (size_t)S.n * k * 8 + (size_t)mb * S.width_cap * k * 8;
  if (assembly == CHOL_ASSEMBLY_OWNER) b += (size_t)S.max_fwd_per_level * chol::kSolveRows * k * 8;
  return b + 3 * (size_t)S.n * k * 8 + kNormSlots * 8;  // + refinement workspace
}

size_t factor_bytes(const chol_sym* sym, int precision, int assembly) {
  const Sym& S = sym->S;
  const size_t esz = precision == CHOL_MIXED ? 4 : 8;
  size_t b = (size_t)S.l_storage * esz + (size_t)S.ns * sizeof(SnDev) + sizeof(MatDev) + 32 +
             (size_t)S.nnz_a * 8;
  if (precision == CHOL_MIXED) b += (size_t)S.n * 8;
  if (assembly == CHOL_ASSEMBLY_OWNER) b += (size_t)S.stage_elems * 8;
  if (precision != CHOL_MIXED && S.oz_rows > 0) b += chol::oz_scratch_bytes(S.oz_rows);
  if (precision != CHOL_MIXED && S.oy_rows > 0 && S.max_width <= chol::kDinvMaxWidth)
    b += chol::oy_scratch_bytes(S.oy_rows);
  if (S.max_width <= chol::kDinvMaxWidth) b += (size_t)S.l_dinv * esz;
  return b;
}

int ensure_refine_ws(chol_num* f, int64_t k) {
  if (f->rws_nrhs >= k) return CHOL_OK;
  chol_ctx* c = f->ctx;
  const int64_t n = f->sym->S.n;
  dev_free(c, f->d_rr);
  dev_free(c, f->d_rd);
  dev_free(c, f->d_rb);
  f->d_rr = f->d_rd = f->d_rb = nullptr;
  f->rws_nrhs = 0;
  int rc;
  if (!f->d_norm && (rc = dev_alloc(c, (void**)&f->d_norm, kNormSlots * 8))) return rc;
  if ((rc = dev_alloc(c, (void**)&f->d_rr, (size_t)n * k * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_rd, (size_t)n * k * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_rb, (size_t)n * k * 8)))
    return rc;
  f->rws_nrhs = k;
  return CHOL_OK;
}

int compute_anorm(chol_num* f) {
  if (f->anorm >= 0.0) return CHOL_OK;
  chol_ctx* c = f->ctx;
  const chol_sym* sym = f->sym;
  unsigned long long* slot = f->d_norm + 2 * 32;
  CK(cudaMemsetAsync(slot, 0, 8, c->stream));
  prof_begin(c, kProfRefine);
  chol::launch_anorm(sym->dev.csr_ptr, sym->dev.csr_src, f->d_vals, sym->S.n, slot, c->stream);
  prof_end(c, kProfRefine, 0.0, 0.0);
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, slot, 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double a;
  memcpy(&a, &v, 8);
  f->anorm = a;
  return CHOL_OK;
}

// Residual R = B - A X of k columns, and its relative size; *rmax = max_c ||r_c||_inf.
int residual_norms(chol_num* f, int k, const double* B, int64_t ldb, const double* X,
                   int64_t ldx, double* rel, double* rmax) {
  chol_ctx* c = f->ctx;
  const chol_sym* sym = f->sym;
  const int64_t n = sym->S.n;
  CK(cudaMemsetAsync(f->d_norm, 0, 2 * 32 * 8, c->stream));
  prof_begin(c, kProfRefine);
  chol::launch_residual(sym->dev.csr_ptr, sym->dev.csr_col, sym->dev.csr_src, f->d_vals, n, k, X,
                        ldx, B, ldb, f->d_rr, n, c->stream);
  chol::launch_absmax(f->d_rr, n, n, k, f->d_norm, c->stream);
  chol::launch_absmax(X, ldx, n, k, f->d_norm + 32, c->stream);
  prof_end(c, kProfRefine, 2.0 * (double)sym->S.csr_ptr[n] * k,
           (12.0 * (double)sym->S.csr_ptr[n] + 24.0 * n) * k);
  unsigned long long h[64];
  CK(cudaMemcpyAsync(h, f->d_norm, 64 * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double worst = 0.0, rm = 0.0;
  for (int j = 0; j < k; j++) {
    double r, x;
    memcpy(&r, &h[j], 8);
    memcpy(&x, &h[32 + j], 8);
    const double v = (f->anorm > 0 && x > 0) ? r / (f->anorm * x) : r;
    worst = std::max(worst, v);
    rm = std::max(rm, r);
  }
  *rel = worst;
  *rmax = rm;
  return CHOL_OK;
}

// Refinement of k <= 32 device columns with factor g (f holds A's values and workspace).
// Returns CHOL_OK when the residual meets tol, CHOL_E_STALL when it stalls.
int refine_pass(chol_num* f, chol_num* g, int k, const double* B, int64_t ldb, double* X,
                int64_t ldx, double tol, int maxit, chol_refine_info* info) {
  chol_ctx* c = f->ctx;
  const int64_t n = f->sym->S.n;
  int rc;
  if ((rc = ensure_solve_ws(g, k))) return rc;
  if ((rc = enqueue_solve(g, k, B, ldb, X, ldx))) return rc;
  double prev = INFINITY, rel = 0, rmax = 0;
  int stall = 0;
  for (int it = 0;; it++) {
    if ((rc = residual_norms(f, k, B, ldb, X, ldx, &rel, &rmax))) return rc;
    info->residual = rel;
    if (rel <= tol) return CHOL_OK;
    if (it >= maxit) return CHOL_E_STALL;
    stall = rmax > 0.5 * prev ? stall + 1 : 0;
    if (stall >= 2) return CHOL_E_STALL;
    prev = rmax;
    if ((rc = enqueue_solve(g, k, f->d_rr, n, f->d_rd, n))) return rc;
    prof_begin(c, kProfRefine);
    chol::launch_axpy(X, ldx, f->d_rd, n, n, k, c->stream);
    prof_end(c, kProfRefine, (double)n * k, 24.0 * n * k);
    info->iterations++;
  }
}

// Refinement of a group's requests together (the serving loop): the same steps as
// refine_pass for every member (first solve, then residual, test, correction, update), but
// per iteration the members' residual norms land in one device array read back with one
// synchronization for the whole group, and every member's launches are enqueued before it.
// Members whose residual stalls, or that need more than one pass of right-hand sides, are
// finished by chol_refine afterwards (with its FP64 fallback for a mixed factor).  A member's
// arithmetic is the same as alone, so its result does not depend on the group.
int refine_group(chol_ctx* c, std::vector<GroupItem>& g) {
  const size_t G = g.size();
  constexpr int kSlots = 2 * 32 + 1;  // max |r| per column, max |x| per column, ||A||_inf
  std::vector<uint8_t> state(G, 0);  // 0 out, 1 active, 2 done, 3 to chol_refine
  for (size_t i = 0; i < G; i++) {
    GroupItem& it = g[i];
    memset(&it.info, 0, sizeof(it.info));
    it.status = chol_factor_status(c, it.f, nullptr);
    if (it.status) continue;
    if (it.k <= 0 || it.f->sym->S.n == 0) continue;
    if (it.k > 32 || it.f->fb) {
      state[i] = 3;
      continue;
    }
    if ((it.status = ensure_refine_ws(it.f, it.k)) || (it.status = ensure_solve_ws(it.f, it.k)))
      continue;
    state[i] = 1;
  }
  unsigned long long* d_g = nullptr;
  int rc = dev_alloc(c, (void**)&d_g, G * kSlots * 8);
  if (rc) return rc;
  struct Release {  // the norms' array goes back to the pool on every return path
    chol_ctx* c;
    void* p;
    ~Release() { dev_free(c, p); }
  } release{c, d_g};
  std::vector<unsigned long long> h(G * kSlots);
  cudaStream_t st = c->stream;
  // ||A||_inf of the members that have not computed it yet, then every first solve
  CK(cudaMemsetAsync(d_g, 0, G * kSlots * 8, st));
  bool any_anorm = false;
  for (size_t i = 0; i < G; i++) {
    if (state[i] != 1 || g[i].f->anorm >= 0.0) continue;
    const chol_num* f = g[i].f;
    chol::launch_anorm(f->sym->dev.csr_ptr, f->sym->dev.csr_src, f->d_vals, f->sym->S.n,
                       d_g + i * kSlots + 64, st);
    any_anorm = true;
  }
  if (any_anorm) {
    CK(cudaMemcpyAsync(h.data(), d_g, G * kSlots * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < G; i++)
      if (state[i] == 1 && g[i].f->anorm < 0.0) memcpy(&g[i].f->anorm, &h[i * kSlots + 64], 8);
  }
  for (size_t i = 0; i < G; i++) {
    if (state[i] != 1) continue;
    chol_num* f = g[i].f;
    const int64_t n = f->sym->S.n;
    CK(cudaMemcpy2DAsync(f->d_rb, n * 8, g[i].B, g[i].ldb * 8, n * 8, g[i].k,
                         cudaMemcpyHostToDevice, st));
    if ((g[i].status = enqueue_solve(f, g[i].k, f->d_rb, n, f->d_bx, n))) state[i] = 0;
  }
  std::vector<double> prev(G, INFINITY);
  std::vector<int> stall(G, 0);
  for (int iter = 0;; iter++) {
    bool any = false;
    CK(cudaMemsetAsync(d_g, 0, G * kSlots * 8, st));
    for (size_t i = 0; i < G; i++) {
      if (state[i] != 1) continue;
      any = true;
      chol_num* f = g[i].f;
      const chol_sym* sym = f->sym;
      const int64_t n = sym->S.n;
      prof_begin(c, kProfRefine);
      chol::launch_residual(sym->dev.csr_ptr, sym->dev.csr_col, sym->dev.csr_src, f->d_vals, n,
                            g[i].k, f->d_bx, n, f->d_rb, n, f->d_rr, n, st);
      chol::launch_absmax(f->d_rr, n, n, g[i].k, d_g + i * kSlots, st);
      chol::launch_absmax(f->d_bx, n, n, g[i].k, d_g + i * kSlots + 32, st);
      prof_end(c, kProfRefine, 2.0 * (double)sym->S.csr_ptr[n] * g[i].k,
               (12.0 * (double)sym->S.csr_ptr[n] + 24.0 * n) * g[i].k);
    }
    if (!any) break;
    CK(cudaMemcpyAsync(h.data(), d_g, G * kSlots * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < G; i++) {
      if (state[i] != 1) continue;
      GroupItem& it = g[i];
      chol_num* f = it.f;
      double worst = 0.0, rm = 0.0;
      for (int j = 0; j < it.k; j++) {
        double r, x;
        memcpy(&r, &h[i * kSlots + j], 8);
        memcpy(&x, &h[i * kSlots + 32 + j], 8);
        worst = std::max(worst, (f->anorm > 0 && x > 0) ? r / (f->anorm * x) : r);
        rm = std::max(rm, r);
      }
      it.info.residual = worst;
      if (worst <= it.tol) {
        state[i] = 2;
        continue;
      }
      stall[i] = rm > 0.5 * prev[i] ? stall[i] + 1 : 0;
      if (iter >= it.maxit || stall[i] >= 2) {
        state[i] = 3;  // refinement with this factor stalls: chol_refine decides
        continue;
      }
      prev[i] = rm;
      const int64_t n = f->sym->S.n;
      if ((it.status = enqueue_solve(f, it.k, f->d_rr, n, f->d_rd, n))) {
        state[i] = 0;
        continue;
      }
      prof_begin(c, kProfRefine);
      chol::launch_axpy(f->d_bx, n, f->d_rd, n, n, it.k, st);
      prof_end(c, kProfRefine, (double)n * it.k, 24.0 * n * it.k);
      it.info.iterations++;
    }
  }
  for (size_t i = 0; i < G; i++) {
    GroupItem& it = g[i];
    if (state[i] == 2) {
      const int64_t n = it.f->sym->S.n;
      CK(cudaMemcpy2DAsync(it.X, it.ldx * 8, it.f->d_bx, n * 8, n * 8, it.k,
                           cudaMemcpyDeviceToHost, st));
    } else if (state[i] == 3) {
      const int64_t before = it.info.iterations;
      it.status = chol_refine(c, it.f, it.k, it.B, it.ldb, it.X, it.ldx, CHOL_HOST, it.tol,
                              it.maxit, &it.info);
      it.info.iterations += before;
    }
  }
  CK(cudaStreamSynchronize(st));
  return CHOL_OK;
}

}  // namespace rt
}  // namespace chol

namespace chol {

// Workspace, in doubles, of a device-pointer solve of k <= 32 right-hand sides: the
// work-queue counters (3 per level), y and w (n k each), the backward partials (max tasks
// of a level x W x k) and, for owner assembly, the forward staging (max tasks of a level x
// kSolveRows x k).
size_t solve_scratch_doubles(const chol_num* f, int64_t k) {
  const Sym& S = f->sym->S;
  size_t d = (rt::solve_counters(S) * sizeof(int) + 255) / 256 * 256 / sizeof(double);
  d += 2 * (size_t)S.n * k + (size_t)f->sym->max_bwd_per_level * S.width_cap * k;
  if (f->assembly == CHOL_ASSEMBLY_OWNER) d += (size_t)S.max_fwd_per_level * kSolveRows * k;
  return d;
}

// The launch sequence of enqueue_solve on caller-provided workspace ws (at least
// solve_scratch_doubles(f, k) doubles).  Creates no events and allocates nothing.
int enqueue_solve_ws(chol_ctx* c, const chol_num* f, int k, const double* B, int64_t ldb,
                     double* X, int64_t ldx, double* ws) {
  const chol_sym* sym = f->sym;
  const Sym& S = sym->S;
  const size_t qd = (rt::solve_counters(S) * sizeof(int) + 255) / 256 * 256 / sizeof(double);
  rt::SolveBufs bf;
  bf.sq = reinterpret_cast<int*>(ws);  // work-queue counters, then the vectors
  bf.y = ws + qd;
  bf.w = bf.y + (size_t)S.n * k;
  bf.part = bf.w + (size_t)S.n * k;
  bf.fstage = f->assembly == CHOL_ASSEMBLY_OWNER
                  ? bf.part + (size_t)sym->max_bwd_per_level * S.width_cap * k
                  : nullptr;
  return rt::enqueue_solve_seq(c, f, k, B, ldb, X, ldx, bf, false);
}

// Checks the arguments of a device-pointer solve; on success *n_out holds the order.
int check_solve_args(chol_ctx* c, const chol_num* f, int64_t nrhs, const double* B,
                     int64_t ldb, const double* X, int64_t ldx, int64_t* n_out) {
  if (!c || !f || f->ctx != c || nrhs < 0 || !B || !X) return CHOL_E_INVALID;
  const int64_t n = f->sym->S.n;
  if (ldb < n || ldx < n || (B == X && ldb != ldx)) return CHOL_E_INVALID;
  *n_out = n;
  return CHOL_OK;
}

cudaStream_t ctx_stream(const chol_ctx* c) { return c->stream; }
int ctx_device(const chol_ctx* c) { return c->opts.device; }

}  // namespace chol

extern "C" {

int chol_version(void) { return 100; }

const char* chol_strerror(int s) {
  switch (s) {
    case CHOL_OK: return "ok";
    case CHOL_PENDING: return "pending";
    case CHOL_E_INVALID: return "invalid argument or malformed matrix";
    case CHOL_E_NOT_SPD: return "matrix is not positive definite";
    case CHOL_E_OOM: return "out of device memory or over the HBM budget";
    case CHOL_E_CUDA: return "CUDA runtime error";
    case CHOL_E_TIMEOUT: return "device-side wait timed out";
    case CHOL_E_NODEVICE: return "no usable CUDA device";
    case CHOL_E_STALL: return "iterative refinement did not converge";
    case CHOL_E_SCRATCH: return "request exceeds the fixed no-allocation scratch area";
    default: return "unknown status";
  }
}

void chol_default_opts(chol_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->width_cap = 64;
  o->assembly = CHOL_ASSEMBLY_ATOMIC;
  o->pivot_tau = 1e-5;
  o->relax = 0.05;
}

int chol_create(const chol_opts* opts, chol_ctx** out) {
  if (!out) return CHOL_E_INVALID;
  *out = nullptr;
  chol_ctx* c = new (std::nothrow) chol_ctx();
  if (!c) return CHOL_E_OOM;
  if (opts) c->opts = *opts; else chol_default_opts(&c->opts);
  if (c->opts.width_cap <= 0) c->opts.width_cap = 64;
  if (c->opts.width_cap > chol::kMaxWidth ||
      (c->opts.assembly != CHOL_ASSEMBLY_ATOMIC && c->opts.assembly != CHOL_ASSEMBLY_OWNER) ||
      (c->opts.fp64_schur != CHOL_SCHUR_OZAKI && c->opts.fp64_schur != CHOL_SCHUR_DMMA)) {
    delete c;
    return CHOL_E_INVALID;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->opts.device < 0 || c->opts.device >= ndev) {
    cudaGetLastError();
    delete c;
    return CHOL_E_NODEVICE;
  }
  if (cudaSetDevice(c->opts.device) != cudaSuccess) { delete c; return CHOL_E_NODEVICE; }
  if (c->opts.stream) {
    c->stream = (cudaStream_t)c->opts.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return CHOL_E_CUDA;
    }
    c->own_stream = true;
  }
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = c->opts.device;
  if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return CHOL_E_CUDA;
  }
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  prof_reset(c);
  *out = c;
  return CHOL_OK;
}

void chol_destroy(chol_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->opts.device);
  cudaStreamSynchronize(c->stream);
  prof_fold(c);
  for (cudaEvent_t e : c->spare_events) cudaEventDestroy(e);
  if (c->open_event) cudaEventDestroy(c->open_event);
  // detach handles that still hold device memory of this context (their later free_* or
  // any other call sees no context and does nothing / returns CHOL_E_INVALID)
  detach_batches(c);
  while (!c->nums.empty()) free_num_buffers(*c->nums.begin());
  while (!c->syms.empty()) free_devsym(*c->syms.begin());
  cudaStreamSynchronize(c->stream);
  cudaMemPoolDestroy(c->pool);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

int chol_analyze(const chol_opts* opts, int64_t n, const int64_t* colptr,
                 const int32_t* rowind, const int32_t* perm, chol_sym** out) {
  if (!out) return CHOL_E_INVALID;
  *out = nullptr;
  chol_sym* s = new (std::nothrow) chol_sym();
  if (!s) return CHOL_E_OOM;
  int rc;
  try {
    const double relax = !opts || opts->relax == 0.0 ? 0.05 : opts->relax;
    rc = chol::analyze(n, colptr, rowind, perm, opts ? opts->width_cap : 64, relax, &s->S);
  } catch (const std::bad_alloc&) {
    rc = CHOL_E_OOM;
  } catch (...) {
    rc = CHOL_E_INVALID;
  }
  if (rc) { delete s; return rc; }
  *out = s;
  return CHOL_OK;
}

int chol_sym_info(const chol_sym* s, chol_sym_stats* st) {
  if (!s || !st) return CHOL_E_INVALID;
  const Sym& S = s->S;
  st->n = S.n;
  st->nnz_a = S.nnz_a;
  st->nnz_l = S.nnz_l;
  st->l_storage = S.l_storage;
  st->nsuper = S.ns;
  st->nlevels = S.nlev;
  st->flops = S.flops;
  st->max_width = S.max_width;
  st->max_rows = S.max_rows;
  st->flops_panel = S.flops_panel;
  st->nfundamental = S.n_fundamental;
  st->ntrsm_tc = 0;
  for (int32_t c : S.lvl_trsmoz) st->ntrsm_tc += c;
  return CHOL_OK;
}

int chol_sym_export(const chol_sym* s, int32_t* parent, int64_t* colcount, int32_t* sn_start,
                    int32_t* sn_level) {
  if (!s) return CHOL_E_INVALID;
  const Sym& S = s->S;
  if (parent) std::copy(S.parent.begin(), S.parent.end(), parent);
  if (colcount) std::copy(S.colcount.begin(), S.colcount.end(), colcount);
  if (sn_start) std::copy(S.sn_start.begin(), S.sn_start.end(), sn_start);
  if (sn_level) std::copy(S.sn_level.begin(), S.sn_level.end(), sn_level);
  return CHOL_OK;
}

int chol_sym_rows(const chol_sym* s, int64_t* rowptr, int32_t* rows) {
  if (!s) return CHOL_E_INVALID;
  const Sym& S = s->S;
  if (rowptr) std::copy(S.sn_rowptr.begin(), S.sn_rowptr.end(), rowptr);
  if (rows) std::copy(S.rows.begin(), S.rows.end(), rows);
  return CHOL_OK;
}

void chol_free_sym(chol_sym* s) {
  if (!s) return;
  if (s->ctx) {
    cudaSetDevice(s->ctx->opts.device);
    free_devsym(s);
  }
  delete s;
}

int chol_factorize(chol_ctx* c, const chol_sym* sym_c, const double* vals, int where,
                   int precision, chol_num** out) {
  if (!c || !sym_c || !out || (!vals && sym_c->S.nnz_a > 0)) return CHOL_E_INVALID;
  if (where != CHOL_HOST && where != CHOL_DEVICE) return CHOL_E_INVALID;
  if (precision != CHOL_FP64 && precision != CHOL_MIXED) return CHOL_E_INVALID;
  *out = nullptr;
  chol_sym* sym = const_cast<chol_sym*>(sym_c);
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  int rc = ensure_uploaded(c, sym);
  if (rc) return rc;
  if ((rc = ensure_attrs(c))) return rc;
  return make_factor(c, sym, vals, where, precision, c->opts.assembly, out, true);
}

int chol_refactorize(chol_ctx* c, chol_num* f, const double* vals, int where) {
  if (!c || !f || f->ctx != c) return CHOL_E_INVALID;
  if (where != CHOL_HOST && where != CHOL_DEVICE) return CHOL_E_INVALID;
  const Sym& S = f->sym->S;
  if (!vals && S.nnz_a > 0) return CHOL_E_INVALID;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  if (S.nnz_a > 0)
    CK(cudaMemcpyAsync(f->d_vals, vals, (size_t)S.nnz_a * 8,
                       where == CHOL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       c->stream));
  if (f->fb) {  // values changed: a fallback factor of the old values is stale
    chol_free_num(f->fb);
    f->fb = nullptr;
  }
  return enqueue_factor(f);
}

int chol_factor_status(chol_ctx* c, const chol_num* f, int64_t* bad_col) {
  if (!c || !f || f->ctx != c) return CHOL_E_INVALID;
  unsigned long long ee[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(ee, f->d_err, sizeof(ee), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  if (ee[3]) return CHOL_E_TIMEOUT;  // a bounded tensor-core wait gave up
  if (ee[1]) return CHOL_E_INVALID;  // internal relative-map inconsistency
  const unsigned long long e = ee[0];
  if (e != ~0ull) {
    if (bad_col) *bad_col = (int64_t)(e - 1);
    return CHOL_E_NOT_SPD;
  }
  if (bad_col) *bad_col = -1;
  return CHOL_OK;
}

int chol_factor_export(chol_ctx* c, const chol_num* f, int64_t* Lp, int32_t* Li, double* Lx) {
  if (!c || !f || f->ctx != c) return CHOL_E_INVALID;
  const Sym& S = f->sym->S;
  const bool f32 = f->precision == CHOL_MIXED;
  std::vector<double> panels;
  std::vector<float> panels32;
  if (Lx) {
    try {
      if (f32) panels32.resize((size_t)S.l_storage);
      else panels.resize((size_t)S.l_storage);
    } catch (...) {
      return CHOL_E_OOM;
    }
    void* dst = f32 ? (void*)panels32.data() : (void*)panels.data();
    CK(cudaMemcpyAsync(dst, f->L, (size_t)S.l_storage * (f32 ? 4 : 8), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  // The exact pattern of L, by row subtrees of B = P^T A P: row i of L holds the columns met
  // walking up the elimination tree from every k < i with B_ik != 0 until i.  Panels of
  // relaxed supernodes also hold explicit zeros outside this pattern; they are skipped.
  const int64_t n = S.n;
  std::vector<int64_t> next;
  std::vector<int32_t> cursor, mark;
  try {
    next.resize(n);
    cursor.resize(n);
    mark.assign(n, -1);
  } catch (...) {
    return CHOL_E_OOM;
  }
  int64_t acc = 0;
  for (int64_t j = 0; j < n; j++) {
    next[j] = acc;
    if (Lp) Lp[j] = acc;
    acc += S.colcount[j];
    cursor[j] = j - S.sn_start[S.col2sn[j]];  // the diagonal's row in its panel
  }
  if (Lp) Lp[n] = acc;
  auto emit = [&](int32_t i, int32_t j) -> bool {
    const int64_t q = next[j]++;
    if (Li) Li[q] = i;
    if (Lx) {
      const int32_t s = S.col2sn[j], m = S.sn_m[s];
      const int32_t* rows = S.rows.data() + S.sn_rowptr[s];
      int32_t r = cursor[j];
      while (r < m && rows[r] != i) r++;
      if (r == m) return false;
      cursor[j] = r;
      const int64_t v = S.sn_valptr[s] + (int64_t)(j - S.sn_start[s]) * m + r;
      Lx[q] = f32 ? (double)panels32[v] : panels[v];
    }
    return true;
  };
  for (int32_t i = 0; i < (int32_t)n; i++) {
    mark[i] = i;
    if (!emit(i, i)) return CHOL_E_INVALID;
    const int32_t ai = S.perm[i];
    for (int64_t p = S.csr_ptr[ai]; p < S.csr_ptr[ai + 1]; p++) {
      const int32_t k = S.iperm[S.csr_col[p]];
      if (k >= i) continue;
      for (int32_t j = k; mark[j] != i; j = S.parent[j]) {
        mark[j] = i;
        if (!emit(i, j)) return CHOL_E_INVALID;  // panel rows miss an entry of L
      }
    }
  }
  return CHOL_OK;
}

}  // extern "C"

namespace {

// out[i] = in[i] as a double (FP32 panels of a mixed factor, widened for export).
__global__ void k_widen(const float* __restrict__ in, double* __restrict__ out, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

}  // namespace

extern "C" {

int chol_factor_panels(chol_ctx* c, const chol_num* f, int64_t first, int64_t count,
                       double* out, int where) {
  if (!c || !f || f->ctx != c || (where != CHOL_HOST && where != CHOL_DEVICE)) return CHOL_E_INVALID;
  const Sym& S = f->sym->S;
  if (first < 0 || count < 0 || first > S.ns || count > S.ns - first) return CHOL_E_INVALID;
  const int64_t v0 = S.sn_valptr[first], v1 = S.sn_valptr[first + count];
  if (v1 == v0) return CHOL_OK;
  if (!out) return CHOL_E_INVALID;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  const size_t nv = (size_t)(v1 - v0);
  if (f->precision != CHOL_MIXED) {
    CK(cudaMemcpyAsync(out, static_cast<const double*>(f->L) + v0, nv * sizeof(double),
                       where == CHOL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       c->stream));
  } else if (where == CHOL_DEVICE) {
    const int blocks = (int)std::min<int64_t>(((int64_t)nv + 255) / 256, 152 * 16);
    k_widen<<<blocks, 256, 0, c->stream>>>(static_cast<const float*>(f->L) + v0, out, (int64_t)nv);
    CK(cudaGetLastError());
  } else {
    std::vector<float> tmp;
    try {
      tmp.resize(nv);
    } catch (...) {
      return CHOL_E_OOM;
    }
    CK(cudaMemcpyAsync(tmp.data(), static_cast<const float*>(f->L) + v0, nv * sizeof(float),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < nv; i++) out[i] = (double)tmp[i];
  }
  if (where == CHOL_HOST) CK(cudaStreamSynchronize(c->stream));
  return CHOL_OK;
}

void chol_free_num(chol_num* f) {
  if (!f) return;
  if (f->fb) chol_free_num(f->fb);
  if (f->ctx) {
    cudaSetDevice(f->ctx->opts.device);
    free_num_buffers(f);
  }
  delete f;
}

int chol_solve(chol_ctx* c, const chol_num* fc, int64_t nrhs, const double* B, int64_t ldb,
               double* X, int64_t ldx, int where) {
  chol_num* f = const_cast<chol_num*>(fc);
  if (!c || !f || f->ctx != c || nrhs < 0 || !B || !X) return CHOL_E_INVALID;
  const int64_t n = f->sym->S.n;
  if (ldb < n || ldx < n || (where != CHOL_HOST && where != CHOL_DEVICE)) return CHOL_E_INVALID;
  if (B == X && ldb != ldx) return CHOL_E_INVALID;
  if (nrhs == 0 || n == 0) return CHOL_OK;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  const int64_t chunk = std::min<int64_t>(nrhs, 32);
  int rc = ensure_solve_ws(f, chunk);
  if (rc) return rc;
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int k = (int)std::min<int64_t>(chunk, nrhs - c0);
    if (where == CHOL_HOST) {
      CK(cudaMemcpy2DAsync(f->d_bx, n * 8, B + c0 * ldb, ldb * 8, n * 8, k,
                           cudaMemcpyHostToDevice, c->stream));
      if ((rc = enqueue_solve(f, k, f->d_bx, n, f->d_bx, n))) return rc;
      CK(cudaMemcpy2DAsync(X + c0 * ldx, ldx * 8, f->d_bx, n * 8, n * 8, k,
                           cudaMemcpyDeviceToHost, c->stream));
    } else {
      if ((rc = enqueue_solve(f, k, B + c0 * ldb, ldb, X + c0 * ldx, ldx))) return rc;
    }
  }
  if (where == CHOL_HOST) CK(cudaStreamSynchronize(c->stream));
  return CHOL_OK;
}

int chol_refine(chol_ctx* c, chol_num* f, int64_t nrhs, const double* B, int64_t ldb,
                double* X, int64_t ldx, int where, double tol, int maxit,
                chol_refine_info* info) {
  chol_refine_info local;
  if (!info) info = &local;
  memset(info, 0, sizeof(*info));
  if (!c || !f || f->ctx != c || nrhs < 0 || !B || !X || B == X || tol < 0 || maxit < 0)
    return CHOL_E_INVALID;
  const int64_t n = f->sym->S.n;
  if (ldb < n || ldx < n || (where != CHOL_HOST && where != CHOL_DEVICE)) return CHOL_E_INVALID;
  if (nrhs == 0 || n == 0) return CHOL_OK;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  int rc = chol_factor_status(c, f, nullptr);
  if (rc) return rc;
  unsigned long long redo = 0;
  CK(cudaMemcpy(&redo, f->d_err + 2, 8, cudaMemcpyDeviceToHost));
  info->pivot_redos = (int64_t)redo;
  const int64_t chunk = std::min<int64_t>(nrhs, 32);
  if ((rc = ensure_refine_ws(f, chunk)) || (rc = ensure_solve_ws(f, chunk)) ||
      (rc = compute_anorm(f)))
    return rc;
  double worst = 0.0;
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int k = (int)std::min<int64_t>(chunk, nrhs - c0);
    const double* Bd = B + c0 * ldb;
    double* Xd = X + c0 * ldx;
    int64_t lb = ldb, lx = ldx;
    if (where == CHOL_HOST) {
      CK(cudaMemcpy2DAsync(f->d_rb, n * 8, Bd, ldb * 8, n * 8, k, cudaMemcpyHostToDevice,
                           c->stream));
      Bd = f->d_rb;
      Xd = f->d_bx;
      lb = lx = n;
    }
    chol_refine_info part;
    memset(&part, 0, sizeof(part));
    rc = f->fb ? CHOL_E_STALL : refine_pass(f, f, k, Bd, lb, Xd, lx, tol, maxit, &part);
    if (rc == CHOL_E_STALL && f->precision == CHOL_MIXED) {
      // the mixed factor cannot deliver tol: factor A in FP64 once and refine with it
      if (!f->fb) {
        if ((rc = make_factor(c, const_cast<chol_sym*>(f->sym), f->d_vals, CHOL_DEVICE,
                              CHOL_FP64, f->assembly, &f->fb, true)))
          return rc;
        if ((rc = chol_factor_status(c, f->fb, nullptr))) return rc;
      }
      info->fell_back = 1;
      rc = refine_pass(f, f->fb, k, Bd, lb, Xd, lx, tol, maxit, &part);
    }
    info->iterations += part.iterations;
    worst = std::max(worst, part.residual);
    if (where == CHOL_HOST)
      CK(cudaMemcpy2DAsync(X + c0 * ldx, ldx * 8, f->d_bx, n * 8, n * 8, k,
                           cudaMemcpyDeviceToHost, c->stream));
    if (rc && rc != CHOL_E_STALL) return rc;
    if (rc == CHOL_E_STALL) {
      info->residual = worst;
      CK(cudaStreamSynchronize(c->stream));
      return CHOL_E_STALL;
    }
  }
  info->residual = worst;
  CK(cudaStreamSynchronize(c->stream));
  return CHOL_OK;
}

int chol_profile_enable(chol_ctx* c, int on) {
  if (!c) return CHOL_E_INVALID;
  c->prof_on = on != 0;
  return CHOL_OK;
}

int chol_set_device_wait(chol_ctx* c, long long cycles) {
  if (!c || cycles < 0) return CHOL_E_INVALID;
  c->acc_wait = cycles;
  return CHOL_OK;
}

int chol_profile_only(chol_ctx* c, const char* name) {
  if (!c) return CHOL_E_INVALID;
  if (!name || !name[0]) {
    c->prof_only = -1;
    return CHOL_OK;
  }
  for (int k = 0; k < kNumProf; k++)
    if (strcmp(name, kProfNames[k]) == 0) {
      c->prof_only = k;
      return CHOL_OK;
    }
  return CHOL_E_INVALID;
}

int chol_profile_read(chol_ctx* c, chol_prof_entry* out, int max, int* count) {
  if (!c || (!out && max > 0)) return CHOL_E_INVALID;
  cudaSetDevice(c->opts.device);
  CK(cudaStreamSynchronize(c->stream));
  prof_fold(c);
  for (int k = 0; k < kNumProf && k < max; k++) out[k] = c->prof[k];
  if (count) *count = kNumProf;
  return CHOL_OK;
}

int chol_profile_reset(chol_ctx* c) {
  if (!c) return CHOL_E_INVALID;
  cudaSetDevice(c->opts.device);
  CK(cudaStreamSynchronize(c->stream));
  prof_fold(c);
  prof_reset(c);
  return CHOL_OK;
}

}  // extern "C"
