// analyze.cpp -- host symbolic analysis for the supernodal factorization.
//
// Sec. 2 of the paper: the analysis phase reorders the matrix (here the ordering is an
// input), builds the elimination tree and merges adjacent columns into supernodes; Sec. 3
// and Fig. 1: supernodes whose subtrees are finished can be factored at the same time,
// which gives the level sets that the device schedule runs one after another.
//
// Algorithms (all standard, none shared with the test oracle):
//   elimination tree  Liu's algorithm with path compression over the rows of B
//   column counts     row-subtree traversal: row i of L is the union of the etree paths
//                     from every k with B_ik != 0 up to i; each visited column gets +1
//   supernodes        column j joins j-1 iff parent(j-1) = j, c_j = c_{j-1} - 1 and j has
//                     one child; then cut into pieces of at most W columns
//   row structure     rows(F) = own columns U rows of B below F U rows of F's children
//                     below F, merged with a marker array
//   levels            0 for supernodes without children, else 1 + max over children
#include <algorithm>
#include <cstring>
#include <numeric>

#include "chol_internal.h"

namespace chol {

namespace {

// Tile class of a supernode's Schur update (u off-diagonal rows), given how many 64- and
// 128-tiles its level holds.
int choose_tile_class(const TilePolicy& p, int64_t u, int64_t level_tiles64,
                      int64_t level_tiles128) {
  if (u >= p.min_rows_tile128 && level_tiles128 >= p.min_level_tiles128) return kTile128;
  if (u >= p.min_rows_tile64 && level_tiles64 >= p.min_level_tiles64) return kTile64;
  if (u >= p.min_rows_tile32) return kTile32;
  return kTile16;
}

// The coarsest tile class that covers an update of u rows in one task (128 wide above 64).
int whole_tile_class(int64_t u) {
  if (u <= 16) return kTile16;
  if (u <= 32) return kTile32;
  if (u <= 64) return kTile64;
  return kTile128;
}

void push4(std::vector<int32_t>& v, int32_t a, int32_t b, int32_t c, int32_t d) {
  v.push_back(a); v.push_back(b); v.push_back(c); v.push_back(d);
}

}  // namespace

int analyze(int64_t n, const int64_t* colptr, const int32_t* rowind, const int32_t* perm,
            int width_cap, double relax, Sym* S) {
  if (n < 0 || n >= (int64_t(1) << 31) || !colptr || (n > 0 && (!rowind || !perm)))
    return CHOL_E_INVALID;
  if (width_cap <= 0) width_cap = 64;
  if (width_cap > kMaxWidth) return CHOL_E_INVALID;
  S->n = n;
  S->width_cap = width_cap;
  if (colptr[0] != 0) return CHOL_E_INVALID;
  for (int64_t j = 0; j < n; j++)
    if (colptr[j + 1] < colptr[j]) return CHOL_E_INVALID;
  const int64_t nnz = colptr[n];
  S->nnz_a = nnz;

  // ---- permutation -------------------------------------------------------------------
  S->perm.assign(perm, perm + n);
  S->iperm.assign(n, -1);
  for (int64_t i = 0; i < n; i++) {
    if (perm[i] < 0 || perm[i] >= n || S->iperm[perm[i]] != -1) return CHOL_E_INVALID;
    S->iperm[perm[i]] = (int32_t)i;
  }
  const int32_t* ip = S->iperm.data();

  // ---- validate A and build the rows of B's strict lower part (CSR) --------------------
  std::vector<int64_t> rp(n + 1, 0);
  for (int64_t j = 0; j < n; j++) {
    for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
      int64_t i = rowind[p];
      if (i < j || i >= n) return CHOL_E_INVALID;
      if (p > colptr[j] && rowind[p - 1] >= i) return CHOL_E_INVALID;
      int32_t a = ip[i], b = ip[j];
      if (a != b) rp[std::max(a, b) + 1]++;
    }
  }
  for (int64_t i = 0; i < n; i++) rp[i + 1] += rp[i];
  std::vector<int32_t> rc(rp[n]);
  {
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    for (int64_t j = 0; j < n; j++)
      for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
        int32_t a = ip[rowind[p]], b = ip[j];
        if (a != b) rc[fill[std::max(a, b)]++] = std::min(a, b);
      }
  }

  // ---- A as given, and its full symmetric CSR for the residual --------------------------
  S->a_colptr.assign(colptr, colptr + n + 1);
  S->a_rowind.assign(rowind, rowind + nnz);
  {
    S->csr_ptr.assign(n + 1, 0);
    for (int64_t j = 0; j < n; j++)
      for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
        S->csr_ptr[rowind[p] + 1]++;
        if (rowind[p] != j) S->csr_ptr[j + 1]++;
      }
    for (int64_t i = 0; i < n; i++) S->csr_ptr[i + 1] += S->csr_ptr[i];
    if (S->csr_ptr[n] >= (int64_t(1) << 31) || nnz >= (int64_t(1) << 31)) return CHOL_E_INVALID;
    S->csr_col.assign(S->csr_ptr[n], 0);
    S->csr_src.assign(S->csr_ptr[n], 0);
    std::vector<int64_t> fill(S->csr_ptr.begin(), S->csr_ptr.end() - 1);
    // visiting columns in order keeps every CSR row sorted by column
    for (int64_t j = 0; j < n; j++)
      for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
        const int32_t i = rowind[p];
        if (i != j) {
          S->csr_col[fill[j]] = i;  // upper triangle: row j, column i > j (placed later)
          S->csr_src[fill[j]] = (int32_t)p;
          fill[j]++;
        }
        S->csr_col[fill[i]] = (int32_t)j;
        S->csr_src[fill[i]] = (int32_t)p;
        fill[i]++;
      }
  }

  // ---- elimination tree (Liu, path compression) ---------------------------------------
  S->parent.assign(n, -1);
  {
    std::vector<int32_t> anc(n, -1);
    for (int64_t i = 0; i < n; i++) {
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
        int32_t r = rc[p];
        while (anc[r] != -1 && anc[r] != i) {
          int32_t t = anc[r];
          anc[r] = (int32_t)i;
          r = t;
        }
        if (anc[r] == -1) {
          anc[r] = (int32_t)i;
          S->parent[r] = (int32_t)i;
        }
      }
    }
  }

  // ---- column counts by row subtrees ---------------------------------------------------
  S->colcount.assign(n, 1);
  {
    std::vector<int32_t> mark(n, -1);
    for (int64_t i = 0; i < n; i++) {
      mark[i] = (int32_t)i;
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
        for (int32_t j = rc[p]; mark[j] != i; j = S->parent[j]) {
          S->colcount[j]++;
          mark[j] = (int32_t)i;
        }
      }
    }
  }
  S->nnz_l = 0;
  S->flops = 0.0;
  for (int64_t j = 0; j < n; j++) {
    S->nnz_l += S->colcount[j];
    S->flops += (double)S->colcount[j] * (double)S->colcount[j];
  }

  // ---- fundamental supernodes ----------------------------------------------------------
  std::vector<int32_t> nchild(n, 0);
  for (int64_t j = 0; j < n; j++)
    if (S->parent[j] >= 0) nchild[S->parent[j]]++;
  std::vector<int32_t> fstart;  // fundamental supernode starts
  for (int64_t j = 0; j < n; j++) {
    bool joins = j > 0 && S->parent[j - 1] == j && S->colcount[j] == S->colcount[j - 1] - 1 &&
                 nchild[j] == 1;
    if (!joins) fstart.push_back((int32_t)j);
  }
  const int64_t nf = (int64_t)fstart.size();
  fstart.push_back((int32_t)n);
  S->n_fundamental = nf;

  // ---- relaxed amalgamation (Sec. 2: padding that buys wider dense blocks) ---------------
  // A supernode absorbs the next fundamental supernode f when f holds the parent of its last
  // column (the columns stay contiguous, the ordering is unchanged) and the merged panel
  // keeps few explicit zeros: at most 1/2 of its lower trapezoid for merged widths up to 16
  // columns, 1/5 up to 64, else `relax`.  The merged panel's rows are its own columns
  // followed by the rows below f; every absorbed column's rows lie among them, so it gains
  // (n + m_f - m) zero rows, n and m being the width and rows before the merge.
  std::vector<int32_t> rstart;  // relaxed supernode starts
  std::vector<int64_t> rm;      // relaxed supernode rows
  double zopen = 0.0;            // explicit zeros of the supernode being grown
  for (int64_t f = 0; f < nf; f++) {
    const int64_t wf = fstart[f + 1] - fstart[f], mf = S->colcount[fstart[f]];
    bool merge = false;
    if (f > 0 && relax > 0 && S->parent[fstart[f] - 1] == fstart[f]) {
      const int64_t cn = fstart[f] - rstart.back(), cm = rm.back();
      const double nn = (double)(cn + wf), mm = (double)(cn + mf);
      const double z = zopen + (double)cn * (double)(cn + mf - cm);
      const double zf = z / (nn * mm - nn * (nn - 1.0) / 2.0);
      merge = (nn <= 16 && zf <= 0.5) || (nn <= 64 && zf <= 0.2) || zf <= relax;
      if (merge) {
        zopen = z;
        rm.back() = cn + mf;
      }
    }
    if (!merge) {
      rstart.push_back(fstart[f]);
      rm.push_back(mf);
      zopen = 0.0;
    }
  }
  const int64_t nr = (int64_t)rstart.size();
  rstart.push_back((int32_t)n);
  std::vector<int32_t> r_of(n);
  for (int64_t r = 0; r < nr; r++)
    for (int32_t j = rstart[r]; j < rstart[r + 1]; j++) r_of[j] = (int32_t)r;

  // ---- row structures of the relaxed supernodes ----------------------------------------
  // rows(R) = columns of R, then the rows below R's last column of B's columns in R and of
  // the row lists of R's children (Sec. 2, elimination tree)
  // B's lower entries by column: column c holds rows r > c with B_rc != 0 (transpose of rc)
  std::vector<int64_t> cp(n + 1, 0);
  for (int64_t p = 0; p < rp[n]; p++) cp[rc[p] + 1]++;
  for (int64_t j = 0; j < n; j++) cp[j + 1] += cp[j];
  std::vector<int32_t> cr(rp[n]);
  {
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    for (int64_t i = 0; i < n; i++)
      for (int64_t p = rp[i]; p < rp[i + 1]; p++) cr[fill[rc[p]]++] = (int32_t)i;
  }
  std::vector<int64_t> frp(nr + 1, 0);
  std::vector<int32_t> frows;
  frows.reserve((size_t)std::min<int64_t>(S->nnz_l, (int64_t)64 << 20));
  std::vector<int32_t> fhead(nr, -1), fnext(nr, -1);
  {
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> tmp;
    for (int64_t f = 0; f < nr; f++) {
      const int32_t a = rstart[f], l = rstart[f + 1] - 1;
      tmp.clear();
      for (int32_t j = a; j <= l; j++) tmp.push_back(j);
      for (int32_t j = a; j <= l; j++)
        for (int64_t p = cp[j]; p < cp[j + 1]; p++) {
          int32_t i = cr[p];
          if (i > l && mark[i] != f) { mark[i] = (int32_t)f; tmp.push_back(i); }
        }
      for (int32_t c = fhead[f]; c != -1; c = fnext[c])
        for (int64_t p = frp[c]; p < frp[c + 1]; p++) {
          int32_t i = frows[p];
          if (i > l && mark[i] != f) { mark[i] = (int32_t)f; tmp.push_back(i); }
        }
      std::sort(tmp.begin() + (l - a + 1), tmp.end());
      if ((int64_t)tmp.size() != rm[f]) return CHOL_E_INVALID;  // inconsistent
      frows.insert(frows.end(), tmp.begin(), tmp.end());
      frp[f + 1] = (int64_t)frows.size();
      int32_t par = S->parent[l];
      if (par >= 0) {
        int32_t pf = r_of[par];
        fnext[f] = fhead[pf];
        fhead[pf] = (int32_t)f;
      }
    }
  }

  // ---- width cap: cut relaxed supernodes into chunks ----------------------------------
  S->sn_start.clear();
  std::vector<int32_t> chunk_f;
  for (int64_t f = 0; f < nr; f++)
    for (int32_t j = rstart[f]; j < rstart[f + 1]; j += width_cap) {
      S->sn_start.push_back(j);
      chunk_f.push_back((int32_t)f);
    }
  S->ns = (int32_t)S->sn_start.size();
  S->sn_start.push_back((int32_t)n);
  const int32_t ns = S->ns;
  S->col2sn.assign(n, 0);
  S->sn_m.assign(ns, 0);
  S->sn_rowptr.assign(ns + 1, 0);
  S->sn_valptr.assign(ns + 1, 0);
  S->sn_dinvptr.assign(ns + 1, 0);
  S->rows.clear();
  S->max_width = S->max_rows = 0;
  S->flops_panel = 0.0;
  for (int32_t s = 0; s < ns; s++) {
    const int32_t a = S->sn_start[s], b = S->sn_start[s + 1];
    const int32_t f = chunk_f[s];
    const int64_t off = a - rstart[f];
    for (int32_t j = a; j < b; j++) S->col2sn[j] = s;
    const int64_t m = (frp[f + 1] - frp[f]) - off;
    S->sn_m[s] = (int32_t)m;
    S->rows.insert(S->rows.end(), frows.begin() + frp[f] + off, frows.begin() + frp[f + 1]);
    S->sn_rowptr[s + 1] = (int64_t)S->rows.size();
    S->sn_valptr[s + 1] = S->sn_valptr[s] + m * (int64_t)(b - a);
    S->sn_dinvptr[s + 1] = S->sn_dinvptr[s] + (int64_t)(b - a) * (b - a);
    S->max_width = std::max<int64_t>(S->max_width, b - a);
    S->max_rows = std::max<int64_t>(S->max_rows, m);
    // the operations the panels really take: sum of c^2 over the padded columns
    for (int64_t k = 0; k < b - a; k++) S->flops_panel += (double)(m - k) * (double)(m - k);
  }
  S->l_storage = S->sn_valptr[ns];
  S->l_dinv = S->sn_dinvptr[ns];
  // runs of each supernode's off-diagonal rows by target supernode (the relative map's
  // index; the map itself is built on the device)
  S->sn_run0.assign(ns + 1, 0);
  S->run_a.clear();
  S->run_t.clear();
  S->run_base.clear();
  S->relmap_size = 0;
  for (int32_t s = 0; s < ns; s++) {
    const int32_t w = S->sn_start[s + 1] - S->sn_start[s], u = S->sn_m[s] - w;
    const int32_t* r = S->rows.data() + S->sn_rowptr[s] + w;
    for (int32_t i = 0; i < u; i++) {
      const int32_t t = S->col2sn[r[i]];
      if (i == 0 || t != S->run_t.back() || (int32_t)S->run_t.size() == S->sn_run0[s]) {
        S->run_a.push_back(i);
        S->run_t.push_back(t);
        S->run_base.push_back(S->relmap_size - i);
        S->relmap_size += u - i;
      }
    }
    S->sn_run0[s + 1] = (int32_t)S->run_a.size();
  }
  S->sn_parent.assign(ns, -1);
  S->sn_level.assign(ns, 0);
  for (int32_t s = 0; s < ns; s++) {
    int32_t last = S->sn_start[s + 1] - 1;
    if (S->parent[last] >= 0) S->sn_parent[s] = S->col2sn[S->parent[last]];
  }
  for (int32_t s = 0; s < ns; s++)
    if (S->sn_parent[s] >= 0)
      S->sn_level[S->sn_parent[s]] = std::max(S->sn_level[S->sn_parent[s]], S->sn_level[s] + 1);

  // ---- where every entry of A lands in the panels -------------------------------------
  S->amap.assign(nnz, 0);
  for (int64_t j = 0; j < n; j++)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
      int32_t a = ip[rowind[p]], b = ip[j];
      int32_t r = std::max(a, b), c = std::min(a, b);
      int32_t t = S->col2sn[c];
      const int32_t* rt = S->rows.data() + S->sn_rowptr[t];
      const int32_t* e = std::lower_bound(rt, rt + S->sn_m[t], r);
      if (e == rt + S->sn_m[t] || *e != r) return CHOL_E_INVALID;  // not in the structure
      S->amap[p] = S->sn_valptr[t] + (int64_t)(c - S->sn_start[t]) * S->sn_m[t] + (e - rt);
    }

  // ---- level sets ---------------------------------------------------------------------
  S->nlev = 0;
  for (int32_t s = 0; s < ns; s++) S->nlev = std::max(S->nlev, S->sn_level[s] + 1);
  S->lvl_ptr.assign(S->nlev + 1, 0);
  for (int32_t s = 0; s < ns; s++) S->lvl_ptr[S->sn_level[s] + 1]++;
  for (int32_t l = 0; l < S->nlev; l++) S->lvl_ptr[l + 1] += S->lvl_ptr[l];
  S->lvl_sn.assign(ns, 0);
  {
    std::vector<int32_t> fill(S->lvl_ptr.begin(), S->lvl_ptr.end() - 1);
    for (int32_t s = 0; s < ns; s++) S->lvl_sn[fill[S->sn_level[s]]++] = s;
  }

  // ---- per-level task lists -----------------------------------------------------------
  for (int k = 0; k < kNumTaskKinds; k++) {
    S->tasks[k].clear();
    S->task_off[k].assign(S->nlev + 1, 0);
    S->lvl_flops[k].assign(S->nlev, 0.0);
  }
  S->lvl_panel_bytes.assign(S->nlev, 0.0);
  S->sn_ustage.assign(ns, -1);
  S->asm_src.clear();
  S->fg_lvl.assign(1, 0);
  S->fg_ptr.assign(1, 0);
  S->fg_row.clear();
  S->fg_ent.clear();
  S->max_fwd_per_level = 0;
  S->stage_elems = 0;
  S->lvl_maxw.assign(S->nlev, 0);
  for (int32_t l = 0; l < S->nlev; l++) {
    int64_t stage = 0;
    for (int32_t q = S->lvl_ptr[l]; q < S->lvl_ptr[l + 1]; q++) {
      const int32_t s = S->lvl_sn[q];
      const int32_t w = S->sn_start[s + 1] - S->sn_start[s];
      S->lvl_maxw[l] = std::max(S->lvl_maxw[l], w);
      const int32_t u = S->sn_m[s] - w;
      const int32_t first_bwd = (int32_t)(S->tasks[kTaskBwd].size() / 4);
      const int32_t nbwd = (std::max(u, 1) + kSolveRows - 1) / kSolveRows;
      push4(S->tasks[kTaskPotrf], s, first_bwd, nbwd, -1);
      const double dn = w, du = u;
      S->lvl_flops[kTaskPotrf][l] += dn * (dn + 1) * (2 * dn + 1) / 6.0;
      S->lvl_flops[kTaskTrsm][l] += du * dn * dn;
      S->lvl_panel_bytes[l] += 8.0 * (dn + du) * dn;
      for (int32_t r0 = 0; r0 < u; r0 += kTrsmRows) push4(S->tasks[kTaskTrsm], s, r0, 0, 0);
      for (int32_t r0 = 0; r0 < std::max(u, 1); r0 += kSolveRows) {
        push4(S->tasks[kTaskFwd], s, r0, 0, 0);
        push4(S->tasks[kTaskBwd], s, r0, 0, 0);
      }
      if (u > 0) {
        S->sn_ustage[s] = stage;
        stage += (int64_t)u * u;
      }
    }
    S->stage_elems = std::max(S->stage_elems, stage);
    for (int k = 0; k < kNumTaskKinds; k++)
      S->task_off[k][l + 1] = (int64_t)S->tasks[k].size() / 4;
    S->max_fwd_per_level = std::max(S->max_fwd_per_level, S->task_off[kTaskFwd][l + 1] -
                                                              S->task_off[kTaskFwd][l]);
  }
  build_schur_tasks(S, TilePolicy());
  return CHOL_OK;
}

void build_owner_lists(Sym* S) {
  if (S->owner_lists) return;
  S->tasks[kTaskAsm].clear();
  S->task_off[kTaskAsm].assign(S->nlev + 1, 0);
  S->asm_src.clear();
  S->fg_lvl.assign(1, 0);
  S->fg_ptr.assign(1, 0);
  S->fg_row.clear();
  S->fg_ent.clear();
  for (int32_t l = 0; l < S->nlev; l++) {
    // owner assembly groups: for every target supernode t hit by this level, per block
    // of 32 target columns, the sources s of this level in ascending order
    {
      struct Src { int32_t t, cb, s, kb, ke; };
      std::vector<Src> srcs;
      for (int32_t q = S->lvl_ptr[l]; q < S->lvl_ptr[l + 1]; q++) {
        const int32_t s = S->lvl_sn[q];
        const int32_t w = S->sn_start[s + 1] - S->sn_start[s];
        const int32_t m = S->sn_m[s];
        const int32_t* rs = S->rows.data() + S->sn_rowptr[s];
        int32_t k = w;
        while (k < m) {
          const int32_t t = S->col2sn[rs[k]];
          const int32_t t0 = S->sn_start[t];
          const int32_t cb = (rs[k] - t0) / 32;
          int32_t ke = k;
          while (ke < m && S->col2sn[rs[ke]] == t && (rs[ke] - t0) / 32 == cb) ke++;
          srcs.push_back({t, cb, s, k - w, ke - w});
          k = ke;
        }
      }
      std::stable_sort(srcs.begin(), srcs.end(), [](const Src& x, const Src& y) {
        if (x.t != y.t) return x.t < y.t;
        if (x.cb != y.cb) return x.cb < y.cb;
        return x.s < y.s;
      });
      // kTaskAsm entries are groups {t, cb, first, end}: target supernode t, block cb of
      // 32 of its columns, and the range [first, end) of asm_src entries {s, kb, ke, -}
      // that update it, s ascending (the fixed summation order)
      size_t g = 0;
      while (g < srcs.size()) {
        size_t h = g;
        while (h < srcs.size() && srcs[h].t == srcs[g].t && srcs[h].cb == srcs[g].cb) h++;
        const int32_t first = (int32_t)(S->asm_src.size() / 4);
        for (size_t q = g; q < h; q++) push4(S->asm_src, srcs[q].s, srcs[q].kb, srcs[q].ke, 0);
        push4(S->tasks[kTaskAsm], srcs[g].t, srcs[g].cb, first, first + (int32_t)(h - g));
        g = h;
      }
    }
    S->task_off[kTaskAsm][l + 1] = (int64_t)S->tasks[kTaskAsm].size() / 4;
    // owner-ordered forward-solve gather lists of this level
    {
      const int64_t f0 = S->task_off[kTaskFwd][l], f1 = S->task_off[kTaskFwd][l + 1];
      std::vector<std::pair<int32_t, int32_t>> ent;  // (target row, slot)
      for (int64_t q = f0; q < f1; q++) {
        const int32_t s = S->tasks[kTaskFwd][4 * q], r0 = S->tasks[kTaskFwd][4 * q + 1];
        const int32_t w = S->sn_start[s + 1] - S->sn_start[s];
        const int32_t u = S->sn_m[s] - w;
        const int32_t* rs = S->rows.data() + S->sn_rowptr[s] + w;
        for (int32_t ii = 0; ii < kSolveRows && r0 + ii < u; ii++)
          ent.push_back({rs[r0 + ii], (int32_t)((q - f0) * kSolveRows + ii)});
      }
      // slots grow with the task index, and tasks are ordered by source supernode
      std::stable_sort(ent.begin(), ent.end(),
                       [](const std::pair<int32_t, int32_t>& x,
                          const std::pair<int32_t, int32_t>& y) { return x.first < y.first; });
      size_t e = 0;
      while (e < ent.size()) {
        size_t g = e;
        S->fg_row.push_back(ent[e].first);
        while (g < ent.size() && ent[g].first == ent[e].first) S->fg_ent.push_back(ent[g++].second);
        S->fg_ptr.push_back((int64_t)S->fg_ent.size());
        e = g;
      }
      S->fg_lvl.push_back((int64_t)S->fg_row.size());
    }
  }
  S->owner_lists = true;
}

int32_t opt_d_threshold(int64_t n, int32_t nsuper, const int32_t* counts) {
  // The threshold of Sec. 4.1 as a search: a threshold d splits the outer tasks with at least
  // d inner tasks, so with split(d) those outer tasks and tasks(d) = nsuper + their inner
  // tasks, D is the largest d in 1 .. max count at which
  //   tasks(d) >= max(1.1 nsuper, n / 14),  d <= 0.3 max count,  split(d) >= nsuper / 1000,
  // and 0 when no d meets all three.  split and tasks only grow as d falls and the middle
  // condition holds below a bound, so the qualifying d form a range from 1 up to D, and one
  // pass down a histogram of the counts with running suffix sums finds its top.
  int32_t top = 0;
  for (int32_t i = 0; i < nsuper; i++) top = std::max(top, counts[i]);
  std::vector<int64_t> hist(static_cast<size_t>(top) + 1, 0);
  for (int32_t i = 0; i < nsuper; i++) hist[counts[i]]++;
  const double goal = std::max(1.1 * nsuper, static_cast<double>(n) / 14.0);
  int64_t split = 0;
  double tasks = nsuper;
  for (int64_t d = top; d >= 1; d--) {
    split += hist[d];
    tasks += static_cast<double>(d) * static_cast<double>(hist[d]);
    if (tasks >= goal && static_cast<double>(d) <= 0.3 * top &&
        static_cast<double>(split) >= nsuper / 1000.0)
      return static_cast<int32_t>(d);
  }
  return 0;
}

double partition_tree(int32_t nv, const int32_t* parent, const double* work, int nparts,
                      double tol, int32_t* owner) {
  // Subtree work W[v] = work[v] + the work of its descendants, children lists, roots.
  std::vector<double> W(work, work + nv);
  std::vector<std::vector<int32_t>> kids(nv);
  std::vector<int32_t> roots;
  std::vector<int32_t> order;  // vertices with every child before its parent
  {
    std::vector<int32_t> nkid(nv, 0), stack;
    for (int32_t v = 0; v < nv; v++) {
      if (parent[v] >= 0) {
        kids[parent[v]].push_back(v);
        nkid[parent[v]]++;
      } else {
        roots.push_back(v);
      }
    }
    for (int32_t v = 0; v < nv; v++)
      if (nkid[v] == 0) stack.push_back(v);
    while (!stack.empty()) {
      const int32_t v = stack.back();
      stack.pop_back();
      order.push_back(v);
      if (parent[v] >= 0 && --nkid[parent[v]] == 0) stack.push_back(parent[v]);
    }
  }
  for (int32_t v : order)
    if (parent[v] >= 0) W[parent[v]] += W[v];
  // The layer: subtrees handed out whole.  Starting from the roots, the heaviest subtree
  // that can be split is replaced by its children (its own vertex joins the top part, done
  // after the exchange) until the layer's subtrees, dealt largest first to the least loaded
  // part, are within (1 + tol) of an even share -- or nothing is left to split.
  std::vector<int32_t> layer = roots;
  std::vector<int32_t> top;
  std::vector<int32_t> bin_of;
  double imbalance = 1.0;
  auto by_weight = [&](int32_t a, int32_t b) { return W[a] > W[b] || (W[a] == W[b] && a < b); };
  for (;;) {
    std::sort(layer.begin(), layer.end(), by_weight);
    std::vector<double> load(nparts, 0.0);
    bin_of.assign(layer.size(), 0);
    double total = 0.0;
    for (size_t i = 0; i < layer.size(); i++) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      load[b] += W[layer[i]];
      bin_of[i] = b;
      total += W[layer[i]];
    }
    const double mean = total / nparts, mx = *std::max_element(load.begin(), load.end());
    imbalance = mean > 0.0 ? mx / mean : 1.0;
    if ((int)layer.size() >= nparts && mx <= (1.0 + tol) * mean) break;
    size_t h = layer.size();  // the heaviest subtree with children
    for (size_t i = 0; i < layer.size(); i++)
      if (!kids[layer[i]].empty()) {
        h = i;
        break;
      }
    if (h == layer.size()) break;  // only single vertices left: the best this tree allows
    const int32_t v = layer[h];
    top.push_back(v);
    layer.erase(layer.begin() + (std::ptrdiff_t)h);
    layer.insert(layer.end(), kids[v].begin(), kids[v].end());
  }
  // owners: the top part -1, every layer subtree its part
  std::fill(owner, owner + nv, -1);
  std::vector<int32_t> stack;
  for (size_t i = 0; i < layer.size(); i++) {
    stack.push_back(layer[i]);
    while (!stack.empty()) {
      const int32_t v = stack.back();
      stack.pop_back();
      owner[v] = bin_of[i];
      for (int32_t c : kids[v]) stack.push_back(c);
    }
  }
  return imbalance;
}

void build_schur_tasks(Sym* S, const TilePolicy& policy) {
  S->policy = policy;
  const int kinds[] = {kTaskSchur64, kTaskSchur32, kTaskSchur16, kTaskSchur128, kTaskOzSlice,
                       kTaskTrsmRest};
  for (int k : kinds) {
    S->tasks[k].clear();
    S->task_off[k].assign(S->nlev + 1, 0);
    S->lvl_flops[k].assign(S->nlev, 0.0);
  }
  S->lvl_ozrows.assign(S->nlev, 0);
  S->oz_rows = 0;
  S->lvl_oyrows.assign(S->nlev, 0);
  S->lvl_trsmoz.assign(S->nlev, 0);
  S->oy_rows = 0;
  for (size_t q = 3; q < S->tasks[kTaskPotrf].size(); q += 4) S->tasks[kTaskPotrf][q] = -1;
  // pass 1: every supernode's tile class under the size thresholds
  std::vector<int8_t> cls0(S->ns, kTile16);
  for (int32_t l = 0; l < S->nlev; l++) {
    int64_t tiles64 = 0, tiles128 = 0;
    for (int32_t q = S->lvl_ptr[l]; q < S->lvl_ptr[l + 1]; q++) {
      const int32_t s = S->lvl_sn[q];
      const int64_t u = S->sn_m[s] - (S->sn_start[s + 1] - S->sn_start[s]);
      const int64_t nt = (u + 63) / 64, nt2 = (u + 127) / 128;
      tiles64 += nt * (nt + 1) / 2;
      tiles128 += nt2 * (nt2 + 1) / 2;
    }
    for (int32_t q = S->lvl_ptr[l]; q < S->lvl_ptr[l + 1]; q++) {
      const int32_t s = S->lvl_sn[q];
      const int64_t u = S->sn_m[s] - (S->sn_start[s + 1] - S->sn_start[s]);
      cls0[s] = static_cast<int8_t>(choose_tile_class(policy, u, tiles64, tiles128));
    }
  }
  // the granularity rule (Sec. 4): which outer tasks (Schur updates) are split into tiles
  int rule = policy.granularity;
  if (rule == kGranHybrid) {
    const double nnz_full = 2.0 * static_cast<double>(S->nnz_a) - static_cast<double>(S->n);
    const double avg = S->ns > 0 ? static_cast<double>(S->n) / S->ns : 0.0;
    const double density =
        S->n > 0 ? nnz_full / (static_cast<double>(S->n) * static_cast<double>(S->n)) : 0.0;
    rule = (avg > 50.0 || (avg > 20.0 && density < 1e-4)) ? kGranTiles : kGranOptDCost;
  }
  std::vector<uint8_t> whole(S->ns, 0);
  S->gran_rule = rule;
  S->gran_D = -1;
  S->gran_split = 0;
  if (rule != kGranTiles) {
    std::vector<int32_t> inner(S->ns, 0);
    for (int32_t s = 0; s < S->ns; s++) {
      const int32_t w = S->sn_start[s + 1] - S->sn_start[s];
      const int64_t u = S->sn_m[s] - w, T = tile_of_class(cls0[s]);
      const int64_t nt = (u + T - 1) / T;
      inner[s] = u > 0 ? static_cast<int32_t>(std::min<int64_t>(nt * (nt + 1) / 2, INT32_MAX)) : 0;
    }
    const int32_t D = opt_d_threshold(S->n, S->ns, inner.data());
    S->gran_D = D;
    for (int32_t s = 0; s < S->ns; s++) {
      const int32_t w = S->sn_start[s + 1] - S->sn_start[s];
      const int64_t T = tile_of_class(cls0[s]);
      // split when the update has at least D inner tasks (Sec. 4.1: "higher than or equal
      // to D"); an update with none is never split
      bool split = inner[s] > 0 && inner[s] >= D;
      // OPT-D-COST (Sec. 4.2): inner tasks of fewer than 50,000 flops are not worth a task
      if (split && rule == kGranOptDCost && 2.0 * T * T * w < 50000.0) split = false;
      if (inner[s] > 0) {
        if (split) S->gran_split++;
        else whole[s] = 1;
      }
    }
  }
  // pass 2: the task lists.  The 128-tile supernodes (FP64: slices on the tensor cores) of a
  // level whose 128-tile rows add up to policy.min_rows_trsm_tc also get their TRSM on the
  // tensor cores, with the slices of their diagonal blocks' inverses at 64 rows each of the
  // level's inverse slices (recorded in the POTRF tasks).  On a narrower level the inverse
  // and its slicing (~45 us of one SM per supernode on GB300, FP64 latency) cost more than
  // the FP64 TRSM they replace.  The other supernodes' TRSM tasks form kTaskTrsmRest.
  for (int32_t l = 0; l < S->nlev; l++) {
    int64_t ozrow = 0, oyrow = 0, rows128 = 0;
    for (int32_t q = S->lvl_ptr[l]; q < S->lvl_ptr[l + 1]; q++) {
      const int32_t s = S->lvl_sn[q];
      const int32_t u = S->sn_m[s] - (S->sn_start[s + 1] - S->sn_start[s]);
      if (u > 0 && (whole[s] ? whole_tile_class(u) : cls0[s]) == kTile128) rows128 += u;
    }
    const bool wide = rows128 >= policy.min_rows_trsm_tc;
    for (int32_t q = S->lvl_ptr[l]; q < S->lvl_ptr[l + 1]; q++) {
      const int32_t s = S->lvl_sn[q];
      const int32_t w = S->sn_start[s + 1] - S->sn_start[s];
      const int32_t u = S->sn_m[s] - w;
      if (u <= 0) continue;
      const int cls = whole[s] ? whole_tile_class(u) : cls0[s];
      const int T = tile_of_class(cls), k = schur_kind(cls);
      S->lvl_flops[k][l] += (double)u * (u + 1.0) * w;
      const bool tc = cls == kTile128 && wide;  // TRSM on the tensor cores
      if (cls == kTile128) {
        for (int32_t i0 = 0; i0 < u; i0 += T)
          for (int32_t k0 = 0; k0 <= i0; k0 += T) push4(S->tasks[k], s, i0, k0, (int32_t)ozrow);
        for (int32_t r0 = 0; r0 < u; r0 += 128)
          push4(S->tasks[kTaskOzSlice], s, r0, (int32_t)ozrow, tc ? (int32_t)oyrow : -1);
        ozrow += (u + 7) / 8 * 8;
      } else {
        for (int32_t i0 = 0; i0 < u; i0 += T)
          for (int32_t k0 = 0; k0 <= i0; k0 += T) push4(S->tasks[k], s, i0, k0, T);
      }
      if (tc) {
        S->tasks[kTaskPotrf][4 * (size_t)q + 3] = (int32_t)oyrow;
        oyrow += kOzInvRows;
        S->lvl_trsmoz[l]++;
      } else {
        for (int32_t r0 = 0; r0 < u; r0 += kTrsmRows) push4(S->tasks[kTaskTrsmRest], s, r0, 0, 0);
        S->lvl_flops[kTaskTrsmRest][l] += (double)u * w * w;  // kTaskTrsm's count
      }
    }
    S->lvl_ozrows[l] = ozrow;
    if (ozrow > 0) S->oz_rows = std::max(S->oz_rows, ozrow + 128);
    S->lvl_oyrows[l] = oyrow;
    S->oy_rows = std::max(S->oy_rows, oyrow);
    for (int k : kinds) S->task_off[k][l + 1] = (int64_t)S->tasks[k].size() / 4;
  }
}

}  // namespace chol
