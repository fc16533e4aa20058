// solve_kernels.cu -- supernodal forward and back substitution on the device.
//
// Sec. 1 and Sec. 2 of the paper: the solve phase solves L y = b and then L^T x = y.  With
// the supernodal factor both run over the level sets: the forward solve goes from the
// leaves up (a supernode's rows are final once all of its descendants are done), the back
// solve from the root down (a supernode needs the solution on its off-diagonal rows, which
// belong to ancestors).
//
// Vectors are n x nrhs column-major in the permuted numbering, ld = n, stored in FP64.  The
// arithmetic runs in the precision of the panels: FP64 for an FP64 factor; FP32 for the
// FP32 factor of the mixed path, whose solves only produce refinement corrections (the
// FP64 residual of the refinement loop restores FP64 accuracy).
//   forward  task {s, r0}: y_s <- L11^{-1} y_s (redundantly in every task of s; the task
//            with r0 = 0 stores it in w), then y[rows[n+i]] -= L21[i, :] y_s for its rows,
//            by atomics, or (owner order) staged and summed per row in a fixed order.
//   backward task {s, r0}: part_q[j, c] = sum_{i in block} L21[i, j] x[rows[n+i], c] into
//            a staging slot q; the supernode's last task to finish then forms
//            x_s = L11^{-T} (w_s - sum_q part_q), the partials summed in task order
//            (deterministic).
// Where the factor keeps the inverses Y = L11^{-1} of its diagonal blocks (formed once per
// factorization), L11^{-1} y_s and L11^{-T} r_s are products with Y and Y^T, parallel over
// the block's rows; otherwise they are substitutions, one step per column.
#include <cuda_runtime.h>

#include <algorithm>

#include "chol_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.h"

namespace chol {

// y[i, c] = B[perm[i], c] (* scale[perm[i]] when scale is given: the equilibrated system)
__global__ void k_gather_perm(const double* __restrict__ B, int64_t ldb,
                              const int32_t* __restrict__ perm, const double* __restrict__ scale,
                              int64_t n, int nrhs, double* __restrict__ y) {
  const int64_t total = n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / n, i = q - c * n;
    const int32_t o = perm[i];
    y[q] = scale ? B[c * ldb + o] * scale[o] : B[c * ldb + o];
  }
}

// X[perm[i], c] = w[i, c] (* scale[perm[i]])
__global__ void k_scatter_perm(const double* __restrict__ w, const int32_t* __restrict__ perm,
                               const double* __restrict__ scale, int64_t n, int nrhs,
                               double* __restrict__ X, int64_t ldx) {
  const int64_t total = n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / n, i = q - c * n;
    const int32_t o = perm[i];
    X[c * ldx + o] = scale ? w[q] * scale[o] : w[q];
  }
}

constexpr int kSolveThreads = kSolveRows;  // one off-diagonal row per thread

// Warp-level triangular solve of the n x n lower L11 (smem, column-major ld n) against
// xs (smem, n x nrhs, ld n).  Forward: xs <- L11^{-1} xs.  Backward: xs <- L11^{-T} xs.
// Lane l owns rows l, l+32, l+64, l+96 (n <= 128).
template <bool FORWARD, typename CT>
__device__ void warp_trisolve(const CT* L11, const CT* rdiag, CT* xs, int n, int nrhs) {
  const int lane = threadIdx.x & 31;
  // the CTA's warps share the right-hand sides: warp w solves columns w, w + nwarps, ...
  const int nwarps = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < nrhs; c += nwarps) {
    CT v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = lane + 32 * q;
      v[q] = r < n ? xs[c * n + r] : CT(0);
    }
    for (int jj = 0; jj < n; jj++) {
      const int j = FORWARD ? jj : n - 1 - jj;
      const int qj = j >> 5, lj = j & 31;
      CT own = v[0];
      if (qj == 1) own = v[1];
      if (qj == 2) own = v[2];
      if (qj == 3) own = v[3];
      const CT xj = __shfl_sync(0xffffffffu, own, lj) * rdiag[j];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int r = lane + 32 * q;
        if (r == j) v[q] = xj;
        else if (FORWARD ? (r > j && r < n) : (r < j)) {
          // forward: row r of column j of L11; backward: (L^T)_{r j} = L_{j r}
          const CT l = FORWARD ? L11[j * n + r] : L11[r * n + j];
          v[q] -= l * xj;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = lane + 32 * q;
      if (r < n) xs[c * n + r] = v[q];
    }
  }
}

// The lower triangle of L11 (the only part warp_trisolve reads) with every copy in flight
// at once, then the reciprocals of its diagonal.
template <typename P>
__device__ void load_l11(const SnDev& d, P* L11, P* rdiag) {
  stage_diag_block(L11, reinterpret_cast<const P*>(d.L), d.n, d.m);
  cp_async_wait_all();
  __syncthreads();
  const int n = d.n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) rdiag[j] = P(1) / L11[j * n + j];
  __syncthreads();
}

// Y (row-major, lower triangle) into shared memory with leading dimension n + 1 (odd: the
// threads of a warp reading one column of Y hit distinct banks), every copy in flight.
template <typename P>
__device__ void stage_dinv(P* Ys, const P* __restrict__ Y, int n) {
  const int ld = n + 1;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, k = idx - r * n;
    if (k <= r) cp_async_elem(Ys + r * ld + k, Y + idx);
  }
}

// xs = Y bin (FORWARD) or Y^T bin, n x nrhs (ld n), Y staged by stage_dinv.  Each output is a
// dot product over the triangle's part of a row (forward: k <= r) or column (backward:
// k >= r) of Y; with fewer outputs than threads the k range is cut into segments whose
// partial sums are added in segment order through red (blockDim.x entries); within a
// segment four interleaved partial sums.  Ends with a barrier.
template <bool FORWARD, typename P>
__device__ void dinv_apply(const P* Ys, const P* bin, P* xs, P* red, int n, int nrhs) {
  const int ld = n + 1, items = n * nrhs, nt = blockDim.x;
  const int nseg = items >= nt ? 1 : min(8, nt / items);
  const int seg = (n + nseg - 1) / nseg;
  for (int idx = threadIdx.x; idx < items * nseg; idx += nt) {
    const int sg = idx / items, it = idx - sg * items;
    const int c = it / n, r = it - c * n;
    int k0 = sg * seg, k1 = min(n, k0 + seg);
    if (FORWARD) k1 = min(k1, r + 1);
    else k0 = max(k0, r);
    const P* b = bin + c * n;
    // four independent chains: an FP64 FMA's result is available only tens of cycles later
    P a[4] = {P(0), P(0), P(0), P(0)};
    int k = k0;
    for (; k + 4 <= k1; k += 4)
#pragma unroll
      for (int q = 0; q < 4; q++)
        a[q] += (FORWARD ? Ys[r * ld + k + q] : Ys[(k + q) * ld + r]) * b[k + q];
    for (; k < k1; k++) a[0] += (FORWARD ? Ys[r * ld + k] : Ys[k * ld + r]) * b[k];
    const P v = (a[0] + a[1]) + (a[2] + a[3]);
    if (nseg == 1) xs[it] = v;
    else red[idx] = v;
  }
  __syncthreads();
  if (nseg > 1) {
    for (int it = threadIdx.x; it < items; it += nt) {
      P v = red[it];
      for (int sg = 1; sg < nseg; sg++) v += red[sg * items + it];
      xs[it] = v;
    }
    __syncthreads();
  }
}

// Panel block of a solve task in shared memory: X[j * kXld + i] = L21[r0 + i, j] for the
// task's rb rows (warps along the columns, lanes along the rows: coalesced reads; odd kXld:
// a warp reading one row across the columns hits distinct banks), every copy in flight.
constexpr int kXld = kSolveRows + 1;
template <typename P>
__device__ void stage_rows(P* X, const P* __restrict__ L21, int64_t m, int n, int rb) {
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int j = threadIdx.x >> 5; j < n; j += nwarp)
    for (int i = lane; i < rb; i += 32) cp_async_elem(X + j * kXld + i, L21 + (int64_t)j * m + i);
}

// Forms of the solve kernels (MODE), chosen per level on the host:
//  * kModeWide (factors that keep Y, levels whose tasks fit in one wave): kWideThreads
//    threads per task, the task's panel block and Y staged in shared memory with every copy
//    in flight at once.  On this part an FP64 FMA's result is available only tens of cycles
//    after issue, so a task alone on its SM is bound by the length of its dependent FMA
//    chains: the off-diagonal dot products are cut into kWideThreads / kSolveRows column
//    groups (forward) or up to 8 row groups (backward) whose partial sums are added in
//    group order.
//  * kModeStaged (backward only; factors that keep Y, the wide levels): kSolveThreads
//    threads, the panel block staged in shared memory (a thread per column reading down
//    the rows from global memory would fetch each cache line several times), Y staged by
//    the supernode's last task only.
//  * kModeGlobal: kSolveThreads threads, the panel read from global memory with eight loads
//    in flight per thread (the forward's rows are contiguous: coalesced), the small
//    footprint keeping many CTAs per SM; also every level of a factor without Y.
// Single-right-hand-side dot products keep four interleaved partial sums.
constexpr int kModeGlobal = 0, kModeStaged = 1, kModeWide = 2;
constexpr int kWideThreads = 4 * kSolveRows;

template <int MODE>
__host__ __device__ constexpr int solve_threads() { return MODE == kModeWide ? kWideThreads : kSolveThreads; }
// right-hand sides per pass when a product is split across thread groups (the size of the
// shared arrays of group partial sums)
template <int MODE, int NR>
__host__ __device__ constexpr int solve_chunk() { return MODE == kModeGlobal ? NR : (NR < 4 ? NR : 4); }
// interleaved partial sums per thread
template <int CH>
__host__ __device__ constexpr int solve_ilp() { return CH == 1 ? 4 : 1; }

// Shared memory of the solve kernels, in P elements (launch sizes in doubles cover both P).
// Forward with Y: Y n(n+1), [X n*kXld if wide], b n*nrhs, xs n*nrhs, red T,
// [red2 (G-1)*kSolveRows*CH if wide]; by substitution: L11 n*n, rdiag n, xs n*nrhs.
// Backward: [Y n(n+1) if wide], [X n*kXld if staged or wide], xg kSolveRows*nrhs, hred T*CH,
// then for the last task's diagonal step r, xo n*nrhs each and red T.  Global mode: the
// diagonal step reuses the space from 0, with Y as Y n(n+1), r, xo, red; by substitution as
// L11 n*n, rdiag n, r n*nrhs.  Staged mode: Y from 0 (over xg and hred when they are
// longer), then r, xo, red after whichever of the two is longer.
static inline size_t fwd_elems(int n, int nrhs, bool inv, int mode) {
  if (!inv) return (size_t)n * n + n + (size_t)n * nrhs;
  const size_t base = (size_t)n * (n + 1) + 2 * (size_t)n * nrhs;
  return mode == kModeWide ? base + (size_t)n * kXld + kWideThreads + 3 * (size_t)kSolveRows * 4
                           : base + kSolveThreads;
}
static inline size_t bwd_elems(int n, int nrhs, bool inv, int mode, int nr) {
  const size_t tail = 2 * (size_t)n * nrhs;  // r, xo
  if (mode == kModeWide)
    return (size_t)n * (n + 1) + (size_t)n * kXld + (size_t)kSolveRows * nrhs +
           (size_t)kWideThreads * 4 + tail + kWideThreads;
  if (mode == kModeStaged) {
    const size_t part = (size_t)n * kXld + (size_t)kSolveRows * nrhs + (size_t)kSolveThreads * 4;
    return std::max(part, (size_t)n * (n + 1)) + tail + kSolveThreads;
  }
  const size_t part = (size_t)kSolveRows * nrhs + (size_t)kSolveThreads * nr;
  return std::max(part, inv ? (size_t)n * (n + 1) + tail + kSolveThreads
                            : (size_t)n * n + n + (size_t)n * nrhs);
}

// Forward step of a level, one CTA per task {s, r0}: x_s = L11^{-1} y_s (in every task of
// s; the task with r0 = 0 stores it in w), then y[rows[n + r0 + i]] -= L21[r0 + i, :] x_s for
// the task's rows, by atomics or (OWNER) into the level's staging slots
// (q * kSolveRows + i) * nrhs + c.  With Y, x_s is a product with Y; by substitution (factors
// wider than kDinvMaxWidth, global mode only) a warp-level substitution.
template <typename P, bool OWNER, int NR, int MODE>
__global__ void __launch_bounds__(solve_threads<MODE>())
    k_fwd(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue, const SnDev* __restrict__ sns, int64_t ldv, int nrhs,
          double* __restrict__ y, double* __restrict__ w, double* __restrict__ fstage) {
  constexpr bool WIDE = MODE == kModeWide;
  constexpr int T = solve_threads<MODE>(), G = T / kSolveRows, CH = solve_chunk<MODE, NR>();
  constexpr int IL = solve_ilp<CH>();
  extern __shared__ __align__(16) double sm[];
  P* smp = reinterpret_cast<P*>(sm);
  __shared__ int s_next_task;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    const int rb = min(kSolveRows, u - tk.y);  // <= 0 for a supernode without rows below
    const P* Lp = reinterpret_cast<const P*>(d.L);
    P* xs;
    P* X = nullptr;
    if (WIDE || d.dinv) {
      P* Ys = smp;
      X = Ys + n * (n + 1);
      P* bin = X + (WIDE ? n * kXld : 0);
      xs = bin + n * nrhs;
      stage_dinv(Ys, reinterpret_cast<const P*>(d.dinv), n);
      if (WIDE && rb > 0) stage_rows(X, Lp + n + tk.y, m, n, rb);
      for (int idx = threadIdx.x; idx < n * nrhs; idx += T) {
        const int c = idx / n, j = idx - c * n;
        bin[idx] = (P)y[c * ldv + d.col0 + j];
      }
      cp_async_wait_all();
      __syncthreads();
      dinv_apply<true>(Ys, bin, xs, xs + n * nrhs, n, nrhs);
    } else {
      P* L11 = smp;
      P* rdiag = L11 + n * n;
      xs = rdiag + n;
      for (int idx = threadIdx.x; idx < n * nrhs; idx += T) {
        const int c = idx / n, j = idx - c * n;
        xs[idx] = (P)y[c * ldv + d.col0 + j];
      }
      load_l11<P>(d, L11, rdiag);
      warp_trisolve<true>(L11, rdiag, xs, n, nrhs);
      __syncthreads();
    }
    if (tk.y == 0)
      for (int idx = threadIdx.x; idx < n * nrhs; idx += T) {
        const int c = idx / n, j = idx - c * n;
        w[c * ldv + d.col0 + j] = xs[idx];
      }
    // off-diagonal rows: row i, column group g (columns j0 .. j1-1)
    const int i = threadIdx.x % kSolveRows, g = threadIdx.x / kSolveRows;
    const int cw = (n + G - 1) / G, j0 = min(n, g * cw), j1 = min(n, j0 + cw);
    P* red2 = xs + n * nrhs + T;  // (G-1) x CH x kSolveRows group partial sums (wide)
    const int64_t grow = i < rb ? d.rows[n + tk.y + i] : 0;
    for (int c0 = 0; c0 < nrhs; c0 += CH) {
      P acc[CH][IL];
#pragma unroll
      for (int c = 0; c < CH; c++)
#pragma unroll
        for (int q = 0; q < IL; q++) acc[c][q] = P(0);
      if (i < rb) {
        if (WIDE) {
          int j = j0;
          for (; j + IL <= j1; j += IL)
#pragma unroll
            for (int q = 0; q < IL; q++) {
              const P l = X[(j + q) * kXld + i];
#pragma unroll
              for (int c = 0; c < CH; c++)
                if (c0 + c < nrhs) acc[c][q] += l * xs[(c0 + c) * n + j + q];
            }
          for (; j < j1; j++) {
            const P l = X[j * kXld + i];
#pragma unroll
            for (int c = 0; c < CH; c++)
              if (c0 + c < nrhs) acc[c][0] += l * xs[(c0 + c) * n + j];
          }
        } else {
          // independent panel loads per step (16 of FP32 for one right-hand side, else 8):
          // the loads, not the FMAs, are the latency; more right-hand sides need the registers
          const P* L = Lp + n + tk.y + i;
          constexpr int QB = (sizeof(P) == 4 && NR == 1) ? 16 : 8;
          int j = 0;
          for (; j + QB <= n; j += QB) {
            P l[QB];
#pragma unroll
            for (int q = 0; q < QB; q++) l[q] = L[(int64_t)(j + q) * m];
#pragma unroll
            for (int q = 0; q < QB; q++)
#pragma unroll
              for (int c = 0; c < CH; c++)
                if (c0 + c < nrhs) acc[c][q % IL] += l[q] * xs[(c0 + c) * n + j + q];
          }
          for (; j < n; j++) {
            const P l = L[(int64_t)j * m];
#pragma unroll
            for (int c = 0; c < CH; c++)
              if (c0 + c < nrhs) acc[c][0] += l * xs[(c0 + c) * n + j];
          }
        }
      }
      P v[CH];
#pragma unroll
      for (int c = 0; c < CH; c++) {
        if constexpr (IL == 4) v[c] = (acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3]);
        else v[c] = acc[c][0];
      }
      if (G > 1) {
        if (g > 0 && i < rb)
#pragma unroll
          for (int c = 0; c < CH; c++) red2[((g - 1) * CH + c) * kSolveRows + i] = v[c];
        __syncthreads();
        if (g == 0 && i < rb)
          for (int gg = 1; gg < G; gg++)
#pragma unroll
            for (int c = 0; c < CH; c++) v[c] += red2[((gg - 1) * CH + c) * kSolveRows + i];
      }
      if (g == 0 && i < rb) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
          if (c0 + c >= nrhs) continue;
          if (OWNER)
            fstage[((int64_t)tq * kSolveRows + i) * nrhs + c0 + c] = (double)v[c];
          else
            red_add(&y[(int64_t)(c0 + c) * ldv + grow], -(double)v[c]);
        }
      }
      if (G > 1) __syncthreads();
    }
    __syncthreads();
    // a CTA's first task is its block index; only a grid smaller than the task list makes
    // CTAs take further tasks from this launch's work queue
    if (gridDim.x >= ntasks) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

// Owner-ordered forward update: row fg_row[i] of y subtracts its staged contributions in
// the fixed order of fg_ent (ascending source supernode).
__global__ void k_fwd_gather(const int32_t* __restrict__ fg_row, const int64_t* __restrict__ fg_ptr,
                             const int32_t* __restrict__ fg_ent, int64_t nrows, int64_t ldv,
                             int nrhs, const double* __restrict__ fstage, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = fg_row[i];
    for (int c = 0; c < nrhs; c++) {
      double s = 0.0;
      for (int64_t e = fg_ptr[i]; e < fg_ptr[i + 1]; e++) s += fstage[(int64_t)fg_ent[e] * nrhs + c];
      y[(int64_t)c * ldv + r] -= s;
    }
  }
}

// Backward step of a level, one CTA per task {s, r0} (a supernode's tasks are consecutive in
// the level's list, r0 = 0, kSolveRows, ...; every supernode has at least one).  Each task
// writes its partial part[q][c][j] = sum_{i in block} L21[r0 + i, j] x[rows[n + r0 + i], c]
// to the slot of its index q in the level; the last of the supernode's tasks to finish
// (counted on arrive[s] after a fence that publishes the partial) sums the slots in task
// order and finishes x_s = L11^{-T} (w_s - sum_q part_q): the same arithmetic whichever task
// comes last, and no CTA waits for another.  Thread (j, h): column j, row group h of
// min(8, T / n32) groups (n32: n rounded up to whole warps); the groups' sums are added in
// group order.
template <typename P, int NR, int MODE>
__global__ void __launch_bounds__(solve_threads<MODE>())
    k_bwd(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
          const SnDev* __restrict__ sns, int64_t ldv, int nrhs, int W, double* __restrict__ w,
          double* __restrict__ part, int* __restrict__ arrive) {
  constexpr bool WIDE = MODE == kModeWide, STG = MODE != kModeGlobal;
  constexpr int T = solve_threads<MODE>(), CH = solve_chunk<MODE, NR>(), IL = solve_ilp<CH>();
  extern __shared__ __align__(16) double sm[];
  P* smp = reinterpret_cast<P*>(sm);
  __shared__ int s_next_task, s_last;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    const int rb = max(0, min(kSolveRows, u - tk.y));
    const bool inv = d.dinv != nullptr;
    const P* Lp = reinterpret_cast<const P*>(d.L);
    P* Ys = smp;
    P* X = Ys + (WIDE ? n * (n + 1) : 0);
    P* xg = X + (STG ? n * kXld : 0);  // rb x nrhs
    P* hred = xg + kSolveRows * nrhs;   // group partial sums
    if (WIDE) stage_dinv(Ys, reinterpret_cast<const P*>(d.dinv), n);
    if (STG && rb > 0) stage_rows(X, Lp + n + tk.y, m, n, rb);
    for (int idx = threadIdx.x; idx < rb * nrhs; idx += T) {
      const int c = idx / rb, i = idx - c * rb;
      xg[idx] = (P)w[c * ldv + d.rows[n + tk.y + i]];
    }
    if (STG) cp_async_wait_all();
    __syncthreads();
    double* out = part + (int64_t)tq * W * nrhs;
    // column slots rounded up to whole warps, so that no warp straddles two row groups
    const int ns = (n + 31) & ~31, ng = max(1, min(8, T / ns));
    const int j = threadIdx.x % ns, h = threadIdx.x / ns;
    const int rw = (rb + ng - 1) / ng, ib = min(rb, h * rw), ie = min(rb, ib + rw);
    const bool act = h < ng && j < n;
    for (int c0 = 0; c0 < nrhs; c0 += CH) {
      P acc[CH][IL];
#pragma unroll
      for (int c = 0; c < CH; c++)
#pragma unroll
        for (int q = 0; q < IL; q++) acc[c][q] = P(0);
      if (act) {
        if (STG) {
          const P* col = X + j * kXld;
          int i = ib;
          for (; i + IL <= ie; i += IL)
#pragma unroll
            for (int q = 0; q < IL; q++) {
              const P l = col[i + q];
#pragma unroll
              for (int c = 0; c < CH; c++)
                if (c0 + c < nrhs) acc[c][q] += l * xg[(c0 + c) * rb + i + q];
            }
          for (; i < ie; i++) {
            const P l = col[i];
#pragma unroll
            for (int c = 0; c < CH; c++)
              if (c0 + c < nrhs) acc[c][0] += l * xg[(c0 + c) * rb + i];
          }
        } else {
          const P* col = Lp + (int64_t)j * m + n + tk.y;
          constexpr int QB = (sizeof(P) == 4 && NR == 1) ? 16 : 8;  // independent loads per step
          int i = ib;
          for (; i + QB <= ie; i += QB) {
            P l[QB];
#pragma unroll
            for (int q = 0; q < QB; q++) l[q] = col[i + q];
#pragma unroll
            for (int q = 0; q < QB; q++)
#pragma unroll
              for (int c = 0; c < CH; c++)
                if (c0 + c < nrhs) acc[c][q % IL] += l[q] * xg[(c0 + c) * rb + i + q];
          }
          for (; i < ie; i++) {
            const P l = col[i];
#pragma unroll
            for (int c = 0; c < CH; c++)
              if (c0 + c < nrhs) acc[c][0] += l * xg[(c0 + c) * rb + i];
          }
        }
      }
      P v[CH];
#pragma unroll
      for (int c = 0; c < CH; c++) {
        if constexpr (IL == 4) v[c] = (acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3]);
        else v[c] = acc[c][0];
      }
      if (ng > 1) {
        if (act && h > 0)
#pragma unroll
          for (int c = 0; c < CH; c++) hred[((h - 1) * CH + c) * n + j] = v[c];
        __syncthreads();
        if (act && h == 0)
          for (int hh = 1; hh < ng; hh++)
#pragma unroll
            for (int c = 0; c < CH; c++) v[c] += hred[((hh - 1) * CH + c) * n + j];
      }
      if (act && h == 0) {
#pragma unroll
        for (int c = 0; c < CH; c++)
          if (c0 + c < nrhs) out[(c0 + c) * W + j] = (double)v[c];
      }
      if (ng > 1) __syncthreads();
    }
    // publish the partial, then count this task in; the last one finishes the supernode
    __threadfence();
    __syncthreads();
    const int nq = (max(u, 1) + kSolveRows - 1) / kSolveRows;
    if (threadIdx.x == 0) s_last = atomicAdd(&arrive[tk.x], 1) == nq - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      const int first = tq - tk.y / kSolveRows;
      // w_s - sum of the partials: wide, after the partial-phase arrays; staged, after the
      // longer of Y and the partial-phase arrays; global mode reuses the space from 0, after
      // Y (with Y) or after L11 and rdiag (by substitution)
      P* r;
      if (WIDE) r = hred + T * 4;
      else if (STG) r = smp + max(n * (n + 1), n * kXld + kSolveRows * nrhs + T * 4);
      else r = inv ? smp + n * (n + 1) : smp + n * n + n;
      if (!WIDE && inv) stage_dinv(Ys, reinterpret_cast<const P*>(d.dinv), n);
      const double* pp0 = part + (int64_t)first * W * nrhs;
      const int64_t ps = (int64_t)W * nrhs;
      // w_s minus the partials of the supernode's tasks, summed in task order with eight
      // loads in flight (from L2: other CTAs wrote them)
      for (int idx = threadIdx.x; idx < n * nrhs; idx += T) {
        const int c = idx / n, jj = idx - c * n;
        const double* pp = pp0 + c * W + jj;
        double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int q = 0;
        for (; q + 8 <= nq; q += 8) {
#pragma unroll
          for (int t = 0; t < 8; t++) a[t] += __ldcg(pp + (q + t) * ps);
        }
        for (; q < nq; q++) a[0] += __ldcg(pp + q * ps);
        r[idx] = (P)(w[c * ldv + d.col0 + jj] -
                     (((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]))));
      }
      P* xo;
      if (inv) {
        if (!WIDE) cp_async_wait_all();
        __syncthreads();
        xo = r + n * nrhs;
        dinv_apply<false>(Ys, r, xo, xo + n * nrhs, n, nrhs);
      } else {
        load_l11<P>(d, smp, smp + n * n);
        warp_trisolve<false>(smp, smp + n * n, r, n, nrhs);
        __syncthreads();
        xo = r;
      }
      for (int idx = threadIdx.x; idx < n * nrhs; idx += T) {
        const int c = idx / n, jj = idx - c * n;
        w[c * ldv + d.col0 + jj] = xo[idx];
      }
    }
    __syncthreads();
    // a CTA's first task is its block index; only a grid smaller than the task list makes
    // CTAs take further tasks from this launch's work queue
    if (gridDim.x >= ntasks) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

// ---- launchers ---------------------------------------------------------------------------------
// Right-hand sides per pass of the panel products: the smallest of 1, 4, 8, 16, 32 >= nrhs.
static inline int rhs_pass(int nrhs) {
  return nrhs <= 1 ? 1 : nrhs <= 4 ? 4 : nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : 32;
}

// Launch sizes (bytes, elements of esz bytes: the panel precision) for supernodes of width
// <= W in the given mode; global mode covers both the layout with Y (widths <= kDinvMaxWidth)
// and the one by substitution.
static inline size_t fwd_smem(int W, int nrhs, int mode, size_t esz = sizeof(double)) {
  const int wy = std::min(W, kDinvMaxWidth);
  if (mode == kModeWide) return fwd_elems(wy, nrhs, true, mode) * esz;
  return std::max(fwd_elems(wy, nrhs, true, mode), fwd_elems(W, nrhs, false, mode)) * esz;
}
static inline size_t bwd_smem(int W, int nrhs, int mode, size_t esz = sizeof(double)) {
  const int wy = std::min(W, kDinvMaxWidth), nr = rhs_pass(nrhs);
  if (mode != kModeGlobal) return bwd_elems(wy, nrhs, true, mode, nr) * esz;
  return std::max(bwd_elems(wy, nrhs, true, mode, nr), bwd_elems(W, nrhs, false, mode, nr)) *
         esz;
}

// Mode of a level (factors that keep Y): wide when its tasks fit in one wave at one CTA per
// SM (the wide footprint is ~115 KB at width 64), where each task's latency is the level's
// critical path; otherwise throughput work: the forward in global mode (coalesced rows, many
// small CTAs per SM), the backward staged.  Measured on GB300.
constexpr int kWideMaxTasks = 152;
static inline int fwd_mode(bool inv, int ntasks) {
  return inv && ntasks <= kWideMaxTasks ? kModeWide : kModeGlobal;
}
static inline int bwd_mode(bool inv, int ntasks) {
  return !inv ? kModeGlobal : ntasks <= kWideMaxTasks ? kModeWide : kModeStaged;
}

static inline int grid_for(int64_t total) {
  return (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
}

void launch_gather_perm(const double* B, int64_t ldb, const int32_t* perm, const double* scale,
                        int64_t n, int nrhs, double* y, cudaStream_t st) {
  if (n <= 0) return;
  k_gather_perm<<<grid_for(n * nrhs), 256, 0, st>>>(B, ldb, perm, scale, n, nrhs, y);
}

void launch_scatter_perm(const double* w, const int32_t* perm, const double* scale, int64_t n,
                         int nrhs, double* X, int64_t ldx, cudaStream_t st) {
  if (n <= 0) return;
  k_scatter_perm<<<grid_for(n * nrhs), 256, 0, st>>>(w, perm, scale, n, nrhs, X, ldx);
}

template <typename P, int NR, int MODE>
static void fwd_nr(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                   int nrhs, int W, double* y, double* w, double* fstage, cudaStream_t st) {
  constexpr int T = solve_threads<MODE>();
  const size_t sm = fwd_smem(W, nrhs, MODE, sizeof(P));
  if (fstage)
    k_fwd<P, true, NR, MODE><<<task_grid(k_fwd<P, true, NR, MODE>, T, sm, ntasks), T, sm, st>>>(
        tasks, ntasks, queue, sns, ldv, nrhs, y, w, fstage);
  else
    k_fwd<P, false, NR, MODE><<<task_grid(k_fwd<P, false, NR, MODE>, T, sm, ntasks), T, sm, st>>>(
        tasks, ntasks, queue, sns, ldv, nrhs, y, w, nullptr);
}

template <typename P, int MODE>
static void fwd_t(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                  int nrhs, int W, double* y, double* w, double* fstage, cudaStream_t st) {
  switch (rhs_pass(nrhs)) {
    case 1: fwd_nr<P, 1, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    case 4: fwd_nr<P, 4, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    case 8: fwd_nr<P, 8, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    case 16: fwd_nr<P, 16, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    default: fwd_nr<P, 32, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
  }
}

template <typename P>
static void fwd_p(int mode, const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                  int64_t ldv, int nrhs, int W, double* y, double* w, double* fstage,
                  cudaStream_t st) {
  if (mode == kModeWide) fwd_t<P, kModeWide>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st);
  else fwd_t<P, kModeGlobal>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st);
}

void launch_fwd(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                int nrhs, int W, double* y, double* w, double* fstage, bool inv, bool f32,
                cudaStream_t st) {
  if (ntasks <= 0) return;
  const int mode = fwd_mode(inv, ntasks);
  if (f32) fwd_p<float>(mode, tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st);
  else fwd_p<double>(mode, tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st);
}

void launch_fwd_gather(const int32_t* fg_row, const int64_t* fg_ptr, const int32_t* fg_ent,
                       int64_t nrows, int64_t ldv, int nrhs, const double* fstage, double* y,
                       cudaStream_t st) {
  if (nrows <= 0) return;
  int blocks = (int)std::min<int64_t>((nrows + 127) / 128, 152 * 8);
  k_fwd_gather<<<blocks, 128, 0, st>>>(fg_row, fg_ptr, fg_ent, nrows, ldv, nrhs, fstage, y);
}

template <typename P, int NR, int MODE>
static void bwd_nr(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                   int nrhs, int W, int wl, double* w, double* part, int* arrive,
                   cudaStream_t st) {
  constexpr int T = solve_threads<MODE>();
  const size_t sm = bwd_smem(wl, nrhs, MODE, sizeof(P));
  k_bwd<P, NR, MODE><<<task_grid(k_bwd<P, NR, MODE>, T, sm, ntasks), T, sm, st>>>(
      tasks, ntasks, queue, sns, ldv, nrhs, W, w, part, arrive);
}

template <typename P, int MODE>
static void bwd_t(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                  int nrhs, int W, int wl, double* w, double* part, int* arrive, cudaStream_t st) {
  switch (rhs_pass(nrhs)) {
    case 1: bwd_nr<P, 1, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st); break;
    case 4: bwd_nr<P, 4, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st); break;
    case 8: bwd_nr<P, 8, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st); break;
    case 16: bwd_nr<P, 16, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st); break;
    default: bwd_nr<P, 32, MODE>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st); break;
  }
}

template <typename P>
static void bwd_p(int mode, const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                  int64_t ldv, int nrhs, int W, int wl, double* w, double* part, int* arrive,
                  cudaStream_t st) {
  if (mode == kModeWide)
    bwd_t<P, kModeWide>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st);
  else if (mode == kModeStaged)
    bwd_t<P, kModeStaged>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st);
  else
    bwd_t<P, kModeGlobal>(tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st);
}

void launch_bwd(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                int nrhs, int W, int wl, double* w, double* part, int* arrive, bool inv,
                bool f32, cudaStream_t st) {
  if (ntasks <= 0) return;
  const int mode = bwd_mode(inv, ntasks);
  if (f32) bwd_p<float>(mode, tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st);
  else bwd_p<double>(mode, tasks, ntasks, queue, sns, ldv, nrhs, W, wl, w, part, arrive, st);
}

template <typename K>
static bool set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
         cudaSuccess;
}

template <typename P, int NR>
static bool set_solve_nr(int W, int nrhs) {
  const size_t fg = fwd_smem(W, nrhs, kModeGlobal), fw = fwd_smem(W, nrhs, kModeWide);
  return set_smem(k_fwd<P, false, NR, kModeGlobal>, fg) &&
         set_smem(k_fwd<P, true, NR, kModeGlobal>, fg) &&
         set_smem(k_fwd<P, false, NR, kModeWide>, fw) &&
         set_smem(k_fwd<P, true, NR, kModeWide>, fw) &&
         set_smem(k_bwd<P, NR, kModeGlobal>, bwd_smem(W, nrhs, kModeGlobal)) &&
         set_smem(k_bwd<P, NR, kModeStaged>, bwd_smem(W, nrhs, kModeStaged)) &&
         set_smem(k_bwd<P, NR, kModeWide>, bwd_smem(W, nrhs, kModeWide));
}

template <typename P>
static bool set_solve_p(int W, int max_nrhs) {
  return set_solve_nr<P, 1>(W, max_nrhs) && set_solve_nr<P, 4>(W, max_nrhs) &&
         set_solve_nr<P, 8>(W, max_nrhs) && set_solve_nr<P, 16>(W, max_nrhs) &&
         set_solve_nr<P, 32>(W, max_nrhs);
}

int set_solve_kernel_attrs(int W, int max_nrhs) {
  return set_solve_p<double>(W, max_nrhs) && set_solve_p<float>(W, max_nrhs) ? CHOL_OK
                                                                             : CHOL_E_CUDA;
}

}  // namespace chol
