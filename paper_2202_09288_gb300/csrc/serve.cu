// serve.cu -- a request server: continuous batching of SPD systems on one GPU.
//
// Requests (a matrix pattern, its values, an ordering and right-hand sides) are queued by
// chol_submit.  Worker slots -- each a thread with its own context and stream -- take the
// oldest requests that fit the server's HBM budget (up to max_batch at a time), factor them
// together as one batch (level l of every member in one launch per kernel kind), refine
// every request's solution to its residual target, and complete it.  Requests that arrive
// while a group is on the GPU are admitted by the next free slot as soon as memory allows,
// so groups overlap on the device.  Host analyses run on analyzer threads ahead of the
// slots and are shared through a cache keyed by the pattern; each slot keeps the device
// copies of the analyses it used, so repeated patterns skip both analysis and upload.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "chol_internal.h"
#include "runtime.h"

using namespace chol::rt;

namespace {

// A host analysis shared by every slot (made once by an analyzer thread).
struct Proto {
  uint64_t key = 0;
  bool ready = false;
  int rc = CHOL_OK;
  chol_sym* sym = nullptr;  // host only: slots clone it before uploading
  ~Proto() {
    if (sym) chol_free_sym(sym);
  }
};

struct Request {
  uint64_t ticket = 0;
  std::shared_ptr<Proto> proto;
  uint64_t key = 0;  // pattern hash
  int64_t n = 0, nrhs = 0;
  std::vector<int64_t> colptr;
  std::vector<int32_t> rowind, perm;
  std::vector<double> vals, B;  // B: n x nrhs, ld n
  double* X = nullptr;
  int64_t ldx = 0;
  int precision = CHOL_FP64;
  double tol = 1e-12;
  double t_submit = 0;
};

struct SymEntry {
  uint64_t key;
  chol_sym* sym;
  size_t bytes;   // bytes of its device copy
  bool uploaded;  // device copy made (its bytes are held until eviction)
  int in_use;     // requests of the current group that use it
};

struct Slot {
  chol_ctx* ctx = nullptr;
  size_t cache_bytes = 0;   // device bytes of the uploaded analyses in the cache
  std::list<SymEntry> lru;  // front = most recent
  std::unordered_map<uint64_t, std::list<SymEntry>::iterator> index;
  std::thread th;
};

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < bytes; i++) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

struct chol_server {
  chol_server_opts opts;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;  // queue, results, budget
  std::condition_variable cv_work, cv_done, cv_mem;
  std::deque<Request*> incoming;  // submitted, not yet analyzed
  std::deque<Request*> queue;     // analyzed, waiting for a slot
  std::condition_variable cv_analyze, cv_proto;
  std::unordered_map<uint64_t, std::shared_ptr<Proto>> protos;
  std::deque<uint64_t> proto_order;  // insertion order, for eviction
  std::vector<std::thread> analyzers;
  std::unordered_map<uint64_t, chol_result> done;
  std::unordered_map<uint64_t, bool> pending;
  uint64_t next_ticket = 1;
  size_t held = 0;  // device bytes reserved by the groups in flight (all slots)
  // Budget split: every slot may keep analyses worth cache_cap bytes resident; groups in
  // flight share the rest (group_budget).  0 = no limit.
  size_t cache_cap = 0, group_budget = 0;
  bool stop = false;
  std::vector<Slot*> slots;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Slot s's copy of the analysis of r's pattern (cloned from the shared one if missing).
SymEntry* get_sym(chol_server* srv, Slot* s, const Request& r, int* rc) {
  auto it = s->index.find(r.key);
  if (it != s->index.end()) {
    s->lru.splice(s->lru.begin(), s->lru, it->second);
    return &*s->lru.begin();
  }
  if (r.proto->rc) {
    *rc = r.proto->rc;
    return nullptr;
  }
  chol_sym* sym = clone_sym(r.proto->sym);
  if (!sym) {
    *rc = CHOL_E_OOM;
    return nullptr;
  }
  s->lru.push_front({r.key, sym, sym_upload_bytes(sym), false, 0});
  s->index[r.key] = s->lru.begin();
  return &*s->lru.begin();
}

// Frees cached analyses of slot s that no request uses, oldest first, while the cache is
// over its entry count or byte cap (slot thread only).
void evict(chol_server* srv, Slot* s) {
  for (auto it = s->lru.end(); it != s->lru.begin();) {
    --it;
    const bool over = (int)s->lru.size() > srv->opts.sym_cache ||
                      (srv->cache_cap && s->cache_bytes > srv->cache_cap);
    if (!over) break;
    if (it->in_use) continue;
    if (it->uploaded) s->cache_bytes -= std::min(s->cache_bytes, it->bytes);
    chol_free_sym(it->sym);
    s->index.erase(it->key);
    it = s->lru.erase(it);
  }
}

size_t request_bytes(const chol_sym* sym, const Request& r, int assembly) {
  const int64_t k = r.nrhs < 32 ? r.nrhs : 32;
  size_t b = factor_bytes(sym, r.precision, assembly) + solve_ws_bytes(sym, k, assembly);
  if (r.precision == CHOL_MIXED)  // room for the FP64 factor a stalled refinement makes
    b += factor_bytes(sym, CHOL_FP64, assembly) + solve_ws_bytes(sym, k, assembly);
  return b;
}

void finish(chol_server* srv, Request* r, const chol_result& res) {
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->done[r->ticket] = res;
    srv->pending.erase(r->ticket);
  }
  srv->cv_done.notify_all();
  delete r;
}

// Analyzer thread: takes submitted requests, finds or makes the shared analysis of their
// pattern, and passes them on to the slots.
void analyzer_loop(chol_server* srv) {
  for (;;) {
    Request* r = nullptr;
    std::shared_ptr<Proto> pr;
    bool mine = false;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv_analyze.wait(lock, [&] { return srv->stop || !srv->incoming.empty(); });
      if (srv->stop) return;
      r = srv->incoming.front();
      srv->incoming.pop_front();
      auto it = srv->protos.find(r->key);
      if (it == srv->protos.end()) {
        pr = std::make_shared<Proto>();
        pr->key = r->key;
        srv->protos[r->key] = pr;
        srv->proto_order.push_back(r->key);
        mine = true;
        // bound the cache: drop the oldest finished analyses (requests keep theirs alive)
        while (srv->proto_order.size() > 4 * (size_t)srv->opts.sym_cache) {
          const uint64_t k = srv->proto_order.front();
          auto jt = srv->protos.find(k);
          if (jt != srv->protos.end() && !jt->second->ready) break;
          srv->proto_order.pop_front();
          if (jt != srv->protos.end()) srv->protos.erase(jt);
        }
      } else {
        pr = it->second;
      }
    }
    if (mine) {
      chol_opts o;
      chol_default_opts(&o);
      o.width_cap = srv->opts.width_cap;
      chol_sym* sym = nullptr;
      const int rc = chol_analyze(&o, r->n, r->colptr.data(), r->rowind.data(), r->perm.data(),
                                  &sym);
      {
        std::lock_guard<std::mutex> lock(srv->mu);
        pr->sym = sym;
        pr->rc = rc;
        pr->ready = true;
      }
      srv->cv_proto.notify_all();
    } else {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv_proto.wait(lock, [&] { return srv->stop || pr->ready; });
      if (srv->stop) {
        delete r;
        return;
      }
    }
    r->proto = pr;
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->queue.push_back(r);
    }
    srv->cv_work.notify_one();
  }
}

void slot_loop(chol_server* srv, Slot* s) {
  cudaSetDevice(srv->opts.device);
  for (;;) {
    std::vector<Request*> group;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      srv->cv_work.wait(lock, [&] { return srv->stop || !srv->queue.empty(); });
      if (srv->stop) return;
      while (!srv->queue.empty() && (int)group.size() < srv->opts.max_batch) {
        group.push_back(srv->queue.front());
        srv->queue.pop_front();
      }
    }
    // analyses (host work, outside the lock)
    std::vector<SymEntry*> syms(group.size(), nullptr);
    std::vector<int> status(group.size(), CHOL_OK);
    for (size_t i = 0; i < group.size(); i++) {
      syms[i] = get_sym(srv, s, *group[i], &status[i]);
      if (syms[i]) syms[i]->in_use++;
    }
    // admission: reserve memory for the longest prefix that fits; return the rest
    std::vector<size_t> need(group.size(), 0);
    size_t admitted = 0;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      const size_t budget = srv->group_budget;
      for (;;) {
        size_t total = 0;
        admitted = 0;
        for (size_t i = 0; i < group.size(); i++) {
          need[i] = 0;
          if (syms[i]) {
            bool first_use = !syms[i]->uploaded;
            for (size_t j = 0; j < i && first_use; j++)
              if (syms[j] == syms[i]) first_use = false;  // counted with request j
            need[i] = request_bytes(syms[i]->sym, *group[i], srv->opts.assembly) +
                      (first_use ? syms[i]->bytes : 0);
          }
          if (budget && srv->held + total + need[i] > budget) break;
          total += need[i];
          admitted = i + 1;
        }
        if (admitted > 0) break;
        if (srv->held == 0) {  // the first request alone exceeds the budget
          status[0] = CHOL_E_OOM;
          need[0] = 0;
          admitted = 1;
          break;
        }
        srv->cv_mem.wait(lock);  // a group in flight will release memory
      }
      for (size_t i = 0; i < admitted; i++) srv->held += need[i];
      for (size_t i = group.size(); i > admitted; i--) srv->queue.push_front(group[i - 1]);
    }
    if (admitted < group.size()) srv->cv_work.notify_one();
    for (size_t i = admitted; i < group.size(); i++)
      if (syms[i]) syms[i]->in_use--;
    group.resize(admitted);
    syms.resize(admitted);
    const double t_start = srv->now();
    // factor the group as one batch
    std::vector<chol_num*> nums(group.size(), nullptr);
    std::vector<chol_num*> live;
    for (size_t i = 0; i < group.size(); i++) {
      if (status[i]) continue;
      chol_sym* sym = syms[i]->sym;
      int rc = ensure_uploaded(s->ctx, sym);
      if (!rc && !syms[i]->uploaded) {
        syms[i]->uploaded = true;
        s->cache_bytes += syms[i]->bytes;
      }
      if (!rc) rc = ensure_attrs(s->ctx);
      if (!rc) rc = make_factor(s->ctx, sym, group[i]->vals.data(), CHOL_HOST,
                                group[i]->precision, srv->opts.assembly, &nums[i], false);
      status[i] = rc;
      if (!rc) live.push_back(nums[i]);
    }
    // one batch per precision (a batch runs one kernel family)
    for (int prec : {CHOL_FP64, CHOL_MIXED}) {
      std::vector<chol_num*> part;
      for (chol_num* f : live)
        if (f->precision == prec) part.push_back(f);
      if (part.empty()) continue;
      chol_batch* b = nullptr;
      int rc = chol_batch_create(s->ctx, (int)part.size(), part.data(), &b);
      if (!rc) rc = chol_batch_factorize(s->ctx, b, nullptr, CHOL_DEVICE, 0);
      if (b) chol_batch_free(b);
      if (rc)
        for (size_t i = 0; i < group.size(); i++)
          if (nums[i] && nums[i]->precision == prec) status[i] = rc;
    }
    // refine the group's requests together (one synchronization per iteration for the whole
    // group) and complete them
    std::vector<GroupItem> items;
    std::vector<size_t> slot_of(group.size(), SIZE_MAX);
    for (size_t i = 0; i < group.size(); i++) {
      if (status[i]) continue;
      GroupItem it;
      it.f = nums[i];
      it.k = (int)group[i]->nrhs;
      it.B = group[i]->B.data();
      it.ldb = group[i]->n;
      it.X = group[i]->X;
      it.ldx = group[i]->ldx;
      it.tol = group[i]->tol;
      it.maxit = 10;
      slot_of[i] = items.size();
      items.push_back(it);
    }
    if (!items.empty()) {
      const int rc = refine_group(s->ctx, items);
      if (rc)
        for (GroupItem& it : items) it.status = rc;
    }
    for (size_t i = 0; i < group.size(); i++) {
      Request* r = group[i];
      chol_result res;
      memset(&res, 0, sizeof(res));
      res.t_submit = r->t_submit;
      res.t_start = t_start;
      res.batch_size = (int)live.size();
      if (!status[i]) {
        const GroupItem& it = items[slot_of[i]];
        status[i] = it.status;
        res.iterations = it.info.iterations;
        res.fell_back = it.info.fell_back;
        res.residual = it.info.residual;
      }
      if (nums[i]) chol_free_num(nums[i]);
      res.status = status[i];
      res.t_done = srv->now();
      finish(srv, r, res);
    }
    cudaStreamSynchronize(s->ctx->stream);
    for (size_t i = 0; i < group.size(); i++)
      if (syms[i]) syms[i]->in_use--;
    evict(srv, s);  // keep the analysis cache within its share
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      for (size_t i = 0; i < group.size(); i++) srv->held -= std::min(srv->held, need[i]);
    }
    srv->cv_mem.notify_all();
  }
}

}  // namespace

extern "C" {

void chol_default_server_opts(chol_server_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->slots = 2;
  o->max_batch = 16;
  o->width_cap = 64;
  o->assembly = CHOL_ASSEMBLY_ATOMIC;
  o->sym_cache = 64;
  o->analyzers = 4;
}

int chol_server_create(const chol_server_opts* opts, chol_server** out) {
  if (!out) return CHOL_E_INVALID;
  *out = nullptr;
  chol_server* srv = new (std::nothrow) chol_server();
  if (!srv) return CHOL_E_OOM;
  if (opts) srv->opts = *opts; else chol_default_server_opts(&srv->opts);
  if (srv->opts.slots <= 0) srv->opts.slots = 2;
  if (srv->opts.max_batch <= 0) srv->opts.max_batch = 16;
  if (srv->opts.width_cap <= 0) srv->opts.width_cap = 64;
  if (srv->opts.sym_cache <= 0) srv->opts.sym_cache = 64;
  srv->t0 = std::chrono::steady_clock::now();
  if (srv->opts.hbm_budget) {
    srv->cache_cap = srv->opts.hbm_budget / (4 * (size_t)srv->opts.slots);
    srv->group_budget = srv->opts.hbm_budget - srv->cache_cap * srv->opts.slots;
  }
  for (int i = 0; i < srv->opts.slots; i++) {
    Slot* s = new (std::nothrow) Slot();
    chol_opts o;
    chol_default_opts(&o);
    o.device = srv->opts.device;
    o.width_cap = srv->opts.width_cap;
    o.assembly = srv->opts.assembly;
    int rc = s ? chol_create(&o, &s->ctx) : CHOL_E_OOM;
    if (rc) {
      delete s;
      chol_server_destroy(srv);
      return rc;
    }
    srv->slots.push_back(s);
  }
  for (Slot* s : srv->slots) s->th = std::thread(slot_loop, srv, s);
  const int na = srv->opts.analyzers > 0 ? srv->opts.analyzers : 4;
  for (int i = 0; i < na; i++) srv->analyzers.emplace_back(analyzer_loop, srv);
  *out = srv;
  return CHOL_OK;
}

int chol_submit(chol_server* srv, const chol_request* q, uint64_t* ticket) {
  if (!srv || !q || !ticket || q->n < 0 || q->nrhs < 1 || !q->colptr || !q->X ||
      (q->n > 0 && (!q->rowind || !q->vals || !q->perm || !q->B)) || q->ldb < q->n ||
      q->ldx < q->n || (q->precision != CHOL_FP64 && q->precision != CHOL_MIXED))
    return CHOL_E_INVALID;
  Request* r = new (std::nothrow) Request();
  if (!r) return CHOL_E_OOM;
  try {
    const int64_t nnz = q->colptr[q->n];
    r->n = q->n;
    r->nrhs = q->nrhs;
    r->colptr.assign(q->colptr, q->colptr + q->n + 1);
    r->rowind.assign(q->rowind, q->rowind + nnz);
    r->perm.assign(q->perm, q->perm + q->n);
    r->vals.assign(q->vals, q->vals + nnz);
    r->B.resize((size_t)q->n * q->nrhs);
    for (int64_t c = 0; c < q->nrhs; c++)
      memcpy(r->B.data() + c * q->n, q->B + c * q->ldb, (size_t)q->n * 8);
  } catch (...) {
    delete r;
    return CHOL_E_OOM;
  }
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, &r->n, sizeof(r->n));
  h = fnv1a(h, r->colptr.data(), r->colptr.size() * 8);
  h = fnv1a(h, r->rowind.data(), r->rowind.size() * 4);
  h = fnv1a(h, r->perm.data(), r->perm.size() * 4);
  r->key = h;
  r->X = q->X;
  r->ldx = q->ldx;
  r->precision = q->precision;
  r->tol = q->tol > 0 ? q->tol : 1e-12;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    r->ticket = srv->next_ticket++;
    r->t_submit = srv->now();
    srv->pending[r->ticket] = true;
    srv->incoming.push_back(r);
    *ticket = r->ticket;
  }
  srv->cv_analyze.notify_one();
  return CHOL_OK;
}

int chol_poll(chol_server* srv, uint64_t ticket, chol_result* res) {
  if (!srv || !res) return CHOL_E_INVALID;
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->done.find(ticket);
  if (it == srv->done.end()) return srv->pending.count(ticket) ? CHOL_PENDING : CHOL_E_INVALID;
  *res = it->second;
  srv->done.erase(it);
  return CHOL_OK;
}

int chol_wait(chol_server* srv, uint64_t ticket, chol_result* res) {
  if (!srv || !res) return CHOL_E_INVALID;
  std::unique_lock<std::mutex> lock(srv->mu);
  srv->cv_done.wait(lock, [&] { return srv->done.count(ticket) || !srv->pending.count(ticket); });
  auto it = srv->done.find(ticket);
  if (it == srv->done.end()) return CHOL_E_INVALID;
  *res = it->second;
  srv->done.erase(it);
  return CHOL_OK;
}

double chol_server_clock(chol_server* srv) { return srv ? srv->now() : 0.0; }

void chol_server_destroy(chol_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  srv->cv_mem.notify_all();
  srv->cv_analyze.notify_all();
  srv->cv_proto.notify_all();
  for (std::thread& t : srv->analyzers)
    if (t.joinable()) t.join();
  for (Slot* s : srv->slots)
    if (s->th.joinable()) s->th.join();
  for (Slot* s : srv->slots) {
    for (auto& e : s->lru) chol_free_sym(e.sym);
    if (s->ctx) chol_destroy(s->ctx);
    delete s;
  }
  for (Request* r : srv->queue) delete r;
  for (Request* r : srv->incoming) delete r;
  srv->protos.clear();
  delete srv;
}

}  // extern "C"
