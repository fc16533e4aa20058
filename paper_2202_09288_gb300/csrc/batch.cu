// batch.cu -- batched factorization of many matrices and the tile-policy autotuner.
//
// The paper runs independent supernodes of one elimination tree at the same time (Sec. 3,
// Fig. 1).  A batch extends that to the supernodes of many matrices: level l of the batch
// holds level l (counted from the leaves) of every member, so one launch per level and
// kernel kind factors all members together, and the whole sequence is captured once into
// a CUDA graph and replayed for new values.  Members keep their own panels, values and
// error words; they may have different patterns, but share a context, a precision and an
// assembly mode.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.h"
#include "chol_internal.h"
#include "kernels.h"
#include "runtime.h"

using namespace chol::rt;

struct chol_batch {
  chol_ctx* ctx = nullptr;
  std::vector<chol_num*> members;
  bool f32 = false, owner = false;
  // merged task lists (host copies, and their device images)
  std::vector<int32_t> tasks[chol::kNumTaskKinds];
  std::vector<int64_t> off[chol::kNumTaskKinds];
  std::vector<double> flops[chol::kNumTaskKinds];
  std::vector<int32_t> asm_src;
  int4* d_tasks[chol::kNumTaskKinds] = {};
  int4* d_asm_src = nullptr;
  SnDev* d_sn = nullptr;
  MatDev* d_mat = nullptr;
  int* d_ctr = nullptr;  // work-queue counters of the batch's launches
  void* d_oz = nullptr;  // FP64 tensor-core Schur tiles: slice scratch of all members
  int64_t oz_rows = 0;
  void* d_oy = nullptr;  // FP64 tensor-core TRSM: slices of the members' inverses
  int64_t oy_rows = 0;
  std::vector<int32_t> trsmoz;  // per level: the members' tensor-core TRSM supernodes
  int32_t nlev = 0;
  int max_width = 0;
  // captured factorization
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches[kNumProf] = {};
};

namespace {

void batch_release(chol_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (!b->ctx) return;
  for (int k = 0; k < chol::kNumTaskKinds; k++) dev_free(b->ctx, b->d_tasks[k]);
  dev_free(b->ctx, b->d_asm_src);
  dev_free(b->ctx, b->d_sn);
  dev_free(b->ctx, b->d_mat);
  dev_free(b->ctx, b->d_ctr);
  dev_free(b->ctx, b->d_oz);
  dev_free(b->ctx, b->d_oy);
  b->d_ctr = nullptr;
  b->d_oz = nullptr;
  b->d_oy = nullptr;
  for (int k = 0; k < chol::kNumTaskKinds; k++) b->d_tasks[k] = nullptr;
  b->d_asm_src = nullptr;
  b->d_sn = nullptr;
  b->d_mat = nullptr;
  b->ctx->batches.erase(b);
  b->ctx = nullptr;
}

chol::rt::TaskView batch_view(const chol_batch* b) {
  chol::rt::TaskView v;
  for (int k = 0; k < chol::kNumTaskKinds; k++) {
    v.d[k] = b->d_tasks[k];
    v.off[k] = b->off[k].data();
    v.flops[k] = b->flops[k].data();
  }
  v.asm_src = b->d_asm_src;
  v.trsmoz = b->trsmoz.data();
  v.nlev = b->nlev;
  v.max_width = b->max_width;
  return v;
}

int enqueue_batch(chol_batch* b) {
  for (chol_num* f : b->members) {
    int rc = enqueue_assembly(f);
    if (rc) return rc;
  }
  return enqueue_levels(b->ctx, batch_view(b), b->d_sn, b->d_mat, b->f32, b->owner, b->d_ctr,
                        b->d_oz, b->oz_rows, b->d_oy, b->oy_rows);
}

const int kFactorKinds[] = {chol::kTaskPotrf,    chol::kTaskTrsm,     chol::kTaskSchur64,
                            chol::kTaskSchur32,  chol::kTaskSchur16, chol::kTaskSchur128,
                            chol::kTaskOzSlice, chol::kTaskTrsmRest, chol::kTaskAsm};

}  // namespace

namespace chol {
namespace rt {

void detach_batches(chol_ctx* c) {
  while (!c->batches.empty()) batch_release(*c->batches.begin());
}

}  // namespace rt
}  // namespace chol

extern "C" {

int chol_batch_create(chol_ctx* c, int count, chol_num* const* nums, chol_batch** out) {
  if (!c || !out || count <= 0 || !nums) return CHOL_E_INVALID;
  *out = nullptr;
  for (int i = 0; i < count; i++) {
    if (!nums[i] || nums[i]->ctx != c) return CHOL_E_INVALID;
    if (nums[i]->precision != nums[0]->precision || nums[i]->assembly != nums[0]->assembly)
      return CHOL_E_INVALID;
    for (int j = 0; j < i; j++)
      if (nums[j] == nums[i]) return CHOL_E_INVALID;
  }
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  chol_batch* b = new (std::nothrow) chol_batch();
  if (!b) return CHOL_E_OOM;
  b->ctx = c;
  c->batches.insert(b);
  b->members.assign(nums, nums + count);
  b->f32 = nums[0]->precision == CHOL_MIXED;
  b->owner = nums[0]->assembly == CHOL_ASSEMBLY_OWNER;
  // descriptor arrays and task offsets of every member
  std::vector<SnDev> sn;
  std::vector<MatDev> mats(count);
  std::vector<int32_t> base(count), src_base(count);
  int32_t src_total = 0;
  for (int i = 0; i < count; i++) {
    const Sym& S = nums[i]->sym->S;
    base[i] = (int32_t)sn.size();
    src_base[i] = src_total;
    src_total += (int32_t)(S.asm_src.size() / 4);
    fill_descriptors(nums[i], i, base[i], &sn, &mats[i]);
    b->nlev = std::max(b->nlev, S.nlev);
    b->max_width = std::max<int>(b->max_width, (int)S.max_width);
  }
  for (int k : kFactorKinds) {
    b->off[k].assign(b->nlev + 1, 0);
    b->flops[k].assign(b->nlev, 0.0);
  }
  // FP64 tensor-core Schur tiles: each member's slice rows of a level follow the previous
  // members' in one batch scratch
  const bool oz = b->f32 || use_oz(c, nums[0]->sym);  // tensor-core 128-tiles need the scratch
  // FP64: the inverses' slices of the tensor-core TRSM follow the same pattern (every member
  // keeps its inverses when W <= kDinvMaxWidth, which the tensor-core tiles imply)
  bool oy = !b->f32 && oz;
  for (int i = 0; i < count; i++) oy = oy && nums[i]->d_dinv != nullptr;
  std::vector<int64_t> ozbase(count), oybase(count);
  b->trsmoz.assign(b->nlev, 0);
  for (int32_t l = 0; l < b->nlev; l++) {
    int64_t total = 0, ytotal = 0;
    for (int i = 0; i < count; i++) {
      const Sym& S = nums[i]->sym->S;
      ozbase[i] = total;
      oybase[i] = ytotal;
      if (l < S.nlev) {
        total += S.lvl_ozrows[l];
        ytotal += S.lvl_oyrows[l];
        b->trsmoz[l] += S.lvl_trsmoz[l];
      }
    }
    if (oz && total > 0) b->oz_rows = std::max(b->oz_rows, total + 128);
    if (oy) b->oy_rows = std::max(b->oy_rows, ytotal);
    for (int k : kFactorKinds) {
      for (int i = 0; i < count; i++) {
        const Sym& S = nums[i]->sym->S;
        if (l >= S.nlev) continue;
        for (int64_t q = S.task_off[k][l]; q < S.task_off[k][l + 1]; q++) {
          const int32_t* t = &S.tasks[k][4 * q];
          const int32_t zb = (int32_t)ozbase[i], yb = (int32_t)oybase[i];
          if (k == chol::kTaskAsm) {  // {t, cb, first, end}: target and source range move
            b->tasks[k].insert(b->tasks[k].end(),
                               {t[0] + base[i], t[1], t[2] + src_base[i], t[3] + src_base[i]});
          } else if (k == chol::kTaskSchur128) {  // {s, i0, k0, oz}
            b->tasks[k].insert(b->tasks[k].end(), {t[0] + base[i], t[1], t[2], t[3] + zb});
          } else if (k == chol::kTaskOzSlice) {   // {s, r0, oz, y}
            b->tasks[k].insert(b->tasks[k].end(),
                               {t[0] + base[i], t[1], t[2] + zb, t[3] >= 0 ? t[3] + yb : -1});
          } else if (k == chol::kTaskPotrf) {     // {s, first_bwd, nbwd, y or -1}
            b->tasks[k].insert(b->tasks[k].end(),
                               {t[0] + base[i], t[1], t[2], t[3] >= 0 ? t[3] + yb : -1});
          } else {
            b->tasks[k].insert(b->tasks[k].end(), {t[0] + base[i], t[1], t[2], t[3]});
          }
        }
        b->flops[k][l] += S.lvl_flops[k][l];
      }
      b->off[k][l + 1] = (int64_t)b->tasks[k].size() / 4;
    }
  }
  for (int i = 0; i < count; i++) {
    const Sym& S = nums[i]->sym->S;
    for (size_t q = 0; q < S.asm_src.size(); q += 4)
      b->asm_src.insert(b->asm_src.end(),
                        {S.asm_src[q] + base[i], S.asm_src[q + 1], S.asm_src[q + 2], 0});
  }
  int rc = CHOL_OK;
  for (int k : kFactorKinds) {
    const size_t bytes = b->tasks[k].size() * sizeof(int32_t);
    if ((rc = dev_alloc(c, (void**)&b->d_tasks[k], bytes))) break;
    if (bytes && cudaMemcpyAsync(b->d_tasks[k], b->tasks[k].data(), bytes,
                                 cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      rc = CHOL_E_CUDA;
      break;
    }
  }
  if (!rc) {
    const size_t ab = b->asm_src.size() * sizeof(int32_t);
    if (!(rc = dev_alloc(c, (void**)&b->d_asm_src, ab)) &&
        !(rc = dev_alloc(c, (void**)&b->d_sn, sn.size() * sizeof(SnDev))) &&
        !(rc = dev_alloc(c, (void**)&b->d_mat, mats.size() * sizeof(MatDev))) &&
        !(rc = dev_alloc(c, (void**)&b->d_ctr, factor_counters(b->nlev) * sizeof(int))) &&
        !(b->oz_rows > 0 &&
          (rc = dev_alloc(c, &b->d_oz, chol::oz_scratch_bytes(b->oz_rows)))) &&
        !(b->oy_rows > 0 &&
          (rc = dev_alloc(c, &b->d_oy, chol::oy_scratch_bytes(b->oy_rows))))) {
      if ((b->d_oz && cudaMemsetAsync(b->d_oz, 0, chol::oz_scratch_bytes(b->oz_rows),
                                      c->stream) != cudaSuccess) ||
          (b->d_oy && cudaMemsetAsync(b->d_oy, 0, chol::oy_scratch_bytes(b->oy_rows),
                                      c->stream) != cudaSuccess))
        rc = CHOL_E_CUDA;
      if ((ab && cudaMemcpyAsync(b->d_asm_src, b->asm_src.data(), ab, cudaMemcpyHostToDevice,
                                 c->stream) != cudaSuccess) ||
          cudaMemcpyAsync(b->d_sn, sn.data(), sn.size() * sizeof(SnDev), cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess ||
          cudaMemcpyAsync(b->d_mat, mats.data(), mats.size() * sizeof(MatDev),
                          cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        rc = CHOL_E_CUDA;
    }
  }
  if (rc) {
    cudaGetLastError();
    batch_release(b);
    delete b;
    return rc;
  }
  *out = b;
  return CHOL_OK;
}

int chol_batch_factorize(chol_ctx* c, chol_batch* b, const double* const* vals, int where,
                         int use_graph) {
  if (!c || !b || b->ctx != c || (where != CHOL_HOST && where != CHOL_DEVICE))
    return CHOL_E_INVALID;
  for (chol_num* f : b->members)
    if (f->ctx != c) return CHOL_E_INVALID;  // a member was freed or detached
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  for (size_t i = 0; i < b->members.size(); i++) {
    chol_num* f = b->members[i];
    const int64_t nnz = f->sym->S.nnz_a;
    if (vals && vals[i] && nnz > 0 &&
        cudaMemcpyAsync(f->d_vals, vals[i], (size_t)nnz * 8,
                        where == CHOL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess) {
      cudaGetLastError();
      return CHOL_E_CUDA;
    }
    if (f->fb) {  // values may have changed: a fallback factor of old values is stale
      chol_free_num(f->fb);
      f->fb = nullptr;
    }
    f->anorm = -1.0;
  }
  if (!use_graph) return enqueue_batch(b);
  if (!b->exec) {
    const bool prof = c->prof_on;
    int64_t before[kNumProf];
    for (int k = 0; k < kNumProf; k++) before[k] = c->prof[k].launches;
    c->prof_on = false;  // no event records inside the graph
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c->prof_on = prof;
      return CHOL_E_CUDA;
    }
    int rc = enqueue_batch(b);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
    c->prof_on = prof;
    for (int k = 0; k < kNumProf; k++) {
      b->graph_launches[k] = c->prof[k].launches - before[k];
      c->prof[k].launches = before[k];
    }
    if (rc || ec != cudaSuccess || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return rc ? rc : CHOL_E_CUDA;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      b->exec = nullptr;
      return CHOL_E_CUDA;
    }
    b->graph = g;
  }
  prof_begin(c, kProfGraph);
  if (cudaGraphLaunch(b->exec, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return CHOL_E_CUDA;
  }
  double fl = 0.0;
  for (int k : kFactorKinds)
    for (double x : b->flops[k]) fl += x;
  prof_end(c, kProfGraph, fl, 0.0);
  for (int k = 0; k < kNumProf; k++) c->prof[k].launches += b->graph_launches[k];
  return CHOL_OK;
}

void chol_batch_free(chol_batch* b) {
  if (!b) return;
  if (b->ctx) cudaSetDevice(b->ctx->opts.device);
  batch_release(b);
  delete b;
}

int chol_sym_get_tile_policy(const chol_sym* s, chol_tile_policy* p) {
  if (!s || !p) return CHOL_E_INVALID;
  p->min_rows_tile64 = s->S.policy.min_rows_tile64;
  p->min_rows_tile32 = s->S.policy.min_rows_tile32;
  p->min_level_tiles64 = s->S.policy.min_level_tiles64;
  p->min_rows_tile128 = s->S.policy.min_rows_tile128;
  p->min_level_tiles128 = s->S.policy.min_level_tiles128;
  p->granularity = s->S.policy.granularity;
  p->min_rows_trsm_tc = s->S.policy.min_rows_trsm_tc;
  return CHOL_OK;
}

int chol_opt_d(int64_t n, int32_t nsuper, const int32_t* counts, int32_t* D) {
  if (n < 0 || nsuper < 0 || !D || (nsuper > 0 && !counts)) return CHOL_E_INVALID;
  for (int32_t i = 0; i < nsuper; i++)
    if (counts[i] < 0) return CHOL_E_INVALID;
  *D = chol::opt_d_threshold(n, nsuper, counts);
  return CHOL_OK;
}

int chol_partition_tree(int32_t nv, const int32_t* parent, const double* work, int nparts,
                        double tol, int32_t* owner, double* imbalance) {
  if (nv < 0 || nparts < 1 || tol < 0 || (nv > 0 && (!parent || !work || !owner)))
    return CHOL_E_INVALID;
  for (int32_t v = 0; v < nv; v++)
    if (parent[v] < -1 || parent[v] >= nv || parent[v] == v || !(work[v] >= 0.0))
      return CHOL_E_INVALID;
  // every vertex must reach a root (no cycles)
  {
    std::vector<int8_t> state(nv, 0);  // 0 unknown, 1 on the current path, 2 reaches a root
    for (int32_t v = 0; v < nv; v++) {
      std::vector<int32_t> path;
      int32_t u = v;
      while (u >= 0 && state[u] == 0) {
        state[u] = 1;
        path.push_back(u);
        u = parent[u];
      }
      if (u >= 0 && state[u] == 1) return CHOL_E_INVALID;
      for (int32_t w : path) state[w] = 2;
    }
  }
  double imb = 1.0;
  try {
    imb = nv > 0 ? chol::partition_tree(nv, parent, work, nparts, tol, owner) : 1.0;
  } catch (...) {
    return CHOL_E_OOM;
  }
  if (imbalance) *imbalance = imb;
  return CHOL_OK;
}

int chol_sym_partition(const chol_sym* sym, int nparts, double tol, int32_t* owner,
                       double* imbalance, double* top_flops) {
  if (!sym || nparts < 1 || tol < 0 || !owner) return CHOL_E_INVALID;
  const chol::Sym& S = sym->S;
  std::vector<double> work(S.ns, 0.0);
  for (int32_t s = 0; s < S.ns; s++)
    for (int32_t j = S.sn_start[s]; j < S.sn_start[s + 1]; j++)
      work[s] += (double)S.colcount[j] * (double)S.colcount[j];
  double imb = 1.0;
  try {
    imb = S.ns > 0 ? chol::partition_tree(S.ns, S.sn_parent.data(), work.data(), nparts, tol,
                                          owner)
                   : 1.0;
  } catch (...) {
    return CHOL_E_OOM;
  }
  if (imbalance) *imbalance = imb;
  if (top_flops) {
    double t = 0.0;
    for (int32_t s = 0; s < S.ns; s++)
      if (owner[s] < 0) t += work[s];
    *top_flops = t;
  }
  return CHOL_OK;
}

int chol_sym_schur_tiles(const chol_sym* sym, int32_t* s, int32_t* i0, int32_t* k0,
                         int32_t* tile, int64_t* count) {
  if (!sym || !count) return CHOL_E_INVALID;
  const chol::Sym& S = sym->S;
  int64_t total = 0;
  for (int cls = 0; cls < chol::kNumTileClasses; cls++)
    total += (int64_t)S.tasks[chol::schur_kind(cls)].size() / 4;
  if (!s) {
    *count = total;
    return CHOL_OK;
  }
  if (*count < total || !i0 || !k0 || !tile) return CHOL_E_INVALID;
  int64_t q = 0;
  for (int cls = 0; cls < chol::kNumTileClasses; cls++) {
    const std::vector<int32_t>& t = S.tasks[chol::schur_kind(cls)];
    for (size_t e = 0; e < t.size(); e += 4, q++) {
      s[q] = t[e];
      i0[q] = t[e + 1];
      k0[q] = t[e + 2];
      tile[q] = chol::tile_of_class(cls);
    }
  }
  *count = total;
  return CHOL_OK;
}

int chol_sym_granularity(const chol_sym* s, int* rule, int32_t* D, int32_t* nsplit) {
  if (!s) return CHOL_E_INVALID;
  if (rule) *rule = s->S.gran_rule;
  if (D) *D = s->S.gran_D;
  if (nsplit) *nsplit = s->S.gran_split;
  return CHOL_OK;
}

int chol_sym_set_tile_policy(chol_sym* s, const chol_tile_policy* p) {
  if (!s || !p || p->min_rows_tile64 < 1 || p->min_rows_tile32 < 1 || p->min_level_tiles64 < 0 ||
      p->min_rows_tile128 < 1 || p->min_level_tiles128 < 0 || p->granularity < CHOL_GRAN_TILES ||
      p->granularity > CHOL_GRAN_HYBRID || p->min_rows_trsm_tc < 1)
    return CHOL_E_INVALID;
  chol::TilePolicy tp;
  tp.min_rows_tile64 = p->min_rows_tile64;
  tp.min_rows_tile32 = p->min_rows_tile32;
  tp.min_level_tiles64 = p->min_level_tiles64;
  tp.min_rows_tile128 = p->min_rows_tile128;
  tp.min_level_tiles128 = p->min_level_tiles128;
  tp.granularity = p->granularity;
  tp.min_rows_trsm_tc = p->min_rows_trsm_tc;
  chol::build_schur_tasks(&s->S, tp);
  if (!s->ctx) return CHOL_OK;
  chol_ctx* c = s->ctx;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  // the lists the tile classes decide: the Schur kinds, the slices, the TRSM without the
  // 128-tile supernodes, and POTRF (whose tasks record the inverses' slice rows)
  const int kinds[] = {chol::schur_kind(0), chol::schur_kind(1), chol::schur_kind(2),
                       chol::schur_kind(3), chol::kTaskOzSlice, chol::kTaskTrsmRest,
                       chol::kTaskPotrf};
  static_assert(chol::kNumTileClasses == 4, "one Schur kind per tile class");
  for (int k : kinds) {
    dev_free(c, s->dev.tasks[k]);
    s->dev.tasks[k] = nullptr;
    const size_t bytes = s->S.tasks[k].size() * sizeof(int32_t);
    int rc = dev_alloc(c, (void**)&s->dev.tasks[k], bytes);
    if (rc) return rc;
    if (bytes && cudaMemcpyAsync(s->dev.tasks[k], s->S.tasks[k].data(), bytes,
                                 cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      cudaGetLastError();
      return CHOL_E_CUDA;
    }
  }
  return CHOL_OK;
}

// Times reps refactorizations of num under policy p (the first one untimed).
static int time_policy(chol_ctx* c, chol_num* num, const chol_tile_policy& p, int reps,
                       double* ms) {
  int rc = chol_sym_set_tile_policy(const_cast<chol_sym*>(num->sym), &p);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CHOL_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CHOL_E_CUDA;
  }
  rc = enqueue_factor(num);
  if (!rc) {
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && !rc; r++) rc = enqueue_factor(num);
    cudaEventRecord(e1, c->stream);
  }
  float t = 0.f;
  if (!rc && (cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
    rc = CHOL_E_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  *ms = t / reps;
  return rc;
}

int chol_autotune(chol_ctx* c, chol_num* num, int reps, chol_tile_policy* best, double* best_ms) {
  if (!c || !num || num->ctx != c || !best) return CHOL_E_INVALID;
  if (reps < 1) reps = 1;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  const bool prof = c->prof_on;
  c->prof_on = false;
  chol_tile_policy cur;
  chol_sym_get_tile_policy(num->sym, &cur);
  double cur_ms = 0.0;
  int rc = time_policy(c, num, cur, reps, &cur_ms);
  // coordinate descent over the six thresholds (1 << 30 rows: no 128-wide tiles, or no
  // tensor-core TRSM)
  static const int kCand[6][5] = {{0, 152, 304, 608, 1216},
                                  {32, 48, 64, 96, 128},
                                  {1, 9, 17, 25, 33},
                                  {128, 192, 256, 512, 1 << 30},
                                  {0, 152, 304, 608, 1216},
                                  {4096, 8192, 16384, 32768, 1 << 30}};
  for (int pass = 0; pass < 6 && !rc; pass++) {
    const int* vals = kCand[pass];
    for (int q = 0; q < 5 && !rc; q++) {
      chol_tile_policy p = cur;
      int* fields[6] = {&p.min_level_tiles64, &p.min_rows_tile64, &p.min_rows_tile32,
                        &p.min_rows_tile128, &p.min_level_tiles128, &p.min_rows_trsm_tc};
      int* field = fields[pass];
      if (*field == vals[q]) continue;
      *field = vals[q];
      double ms = 0.0;
      rc = time_policy(c, num, p, reps, &ms);
      if (!rc && ms < cur_ms) {
        cur = p;
        cur_ms = ms;
      }
    }
  }
  if (!rc) rc = chol_sym_set_tile_policy(const_cast<chol_sym*>(num->sym), &cur);
  if (!rc) rc = enqueue_factor(num);  // leave num factored under the chosen policy
  c->prof_on = prof;
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return rc;
}

}  // extern "C"
