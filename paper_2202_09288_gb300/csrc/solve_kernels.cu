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
//            a staging slot q; then per supernode x_s = L11^{-T} (w_s - sum_q part_q), the
//            partials summed in task order (deterministic).
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
// partial sums are added in segment order through red (blockDim.x entries).  Ends with a
// barrier.
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
    P a0 = P(0), a1 = P(0);
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      a0 += (FORWARD ? Ys[r * ld + k] : Ys[k * ld + r]) * b[k];
      a1 += (FORWARD ? Ys[r * ld + k + 1] : Ys[(k + 1) * ld + r]) * b[k + 1];
    }
    if (k < k1) a0 += (FORWARD ? Ys[r * ld + k] : Ys[k * ld + r]) * b[k];
    if (nseg == 1) xs[it] = a0 + a1;
    else red[idx] = a0 + a1;
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

// smem: L11 n*n, rdiag n, xs n*nrhs (substitution), or Y n*(n+1), b n*nrhs, xs n*nrhs,
// red kSolveThreads (with Y).  STAGE: the off-diagonal products go to the level's
// staging slots (q * kSolveRows + ii) * nrhs + c instead of atomics into y.
template <typename P, bool STAGE, int NR>
__global__ void __launch_bounds__(kSolveThreads)
    k_fwd(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue, const SnDev* __restrict__ sns, int64_t ldv, int nrhs,
          double* __restrict__ y, double* __restrict__ w, double* __restrict__ fstage) {
  extern __shared__ __align__(16) double sm[];
  P* smp = reinterpret_cast<P*>(sm);
  __shared__ int s_next_task;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    P* xs;
    if (d.dinv) {
      P* Ys = smp;
      P* bin = Ys + n * (n + 1);
      xs = bin + n * nrhs;
      stage_dinv(Ys, reinterpret_cast<const P*>(d.dinv), n);
      for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
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
      for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
        const int c = idx / n, j = idx - c * n;
        xs[idx] = (P)y[c * ldv + d.col0 + j];
      }
      load_l11<P>(d, L11, rdiag);
      warp_trisolve<true>(L11, rdiag, xs, n, nrhs);
      __syncthreads();
    }
    if (tk.y == 0)
      for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
        const int c = idx / n, j = idx - c * n;
        w[c * ldv + d.col0 + j] = xs[idx];
      }
    const int i = tk.y + threadIdx.x;
    if (i < u) {
      const P* L = reinterpret_cast<const P*>(d.L) + n + i;
      const int64_t grow = d.rows[n + i];
      // NR (>= nrhs) right-hand sides per pass: each panel entry is read once
      for (int c0 = 0; c0 < nrhs; c0 += NR) {
        P acc[NR];
  #pragma unroll
        for (int c = 0; c < NR; c++) acc[c] = P(0);
        // independent panel loads per step (16 of FP32 for one right-hand side, else 8): the
        // loads, not the FMAs, are the latency; more right-hand sides need the registers
        constexpr int QB = (sizeof(P) == 4 && NR == 1) ? 16 : 8;
        int j = 0;
        for (; j + QB <= n; j += QB) {
          P l[QB];
  #pragma unroll
          for (int q = 0; q < QB; q++) l[q] = L[(int64_t)(j + q) * m];
  #pragma unroll
          for (int q = 0; q < QB; q++)
  #pragma unroll
            for (int c = 0; c < NR; c++)
              if (c0 + c < nrhs) acc[c] += l[q] * xs[(c0 + c) * n + j + q];
        }
        for (; j < n; j++) {
          const P l = L[(int64_t)j * m];
  #pragma unroll
          for (int c = 0; c < NR; c++)
            if (c0 + c < nrhs) acc[c] += l * xs[(c0 + c) * n + j];
        }
  #pragma unroll
        for (int c = 0; c < NR; c++) {
          if (c0 + c >= nrhs) continue;
          if (STAGE)
            fstage[((int64_t)tq * kSolveRows + threadIdx.x) * nrhs + c0 + c] = (double)acc[c];
          else
            atomicAdd(&y[(int64_t)(c0 + c) * ldv + grow], -(double)acc[c]);
        }
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

// Backward partials: the level's task q writes part[q * W * nrhs + c * W + j] =
// sum_{i in block} L21[i, j] x[rows[n + i], c].  Column j is read once for all NR (>= nrhs)
// right-hand sides: for n <= 64 two threads share a column (halves of the block's rows,
// combined through shared memory), otherwise one thread per column.
template <typename P, int NR>
__global__ void __launch_bounds__(kSolveThreads)
    k_bwd_partial(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue, const SnDev* __restrict__ sns,
                  int64_t ldv, int nrhs, int W, const double* __restrict__ w,
                  double* __restrict__ part) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_next_task;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    const int rb = min(kSolveRows, u - tk.y);
    P* xg = reinterpret_cast<P*>(sm);       // rb x nrhs
    P* red = xg + kSolveRows * NR;          // n x nrhs partial sums of the second half
    for (int idx = threadIdx.x; idx < rb * nrhs; idx += blockDim.x) {
      const int c = idx / rb, i = idx - c * rb;
      xg[idx] = (P)w[c * ldv + d.rows[n + tk.y + i]];
    }
    __syncthreads();
    double* out = part + (int64_t)tq * W * nrhs;
    const bool two = n <= kSolveThreads / 2;
    const int j = two ? (threadIdx.x % (kSolveThreads / 2)) : threadIdx.x;
    const int h = two ? threadIdx.x / (kSolveThreads / 2) : 0;
    const int half = two ? (rb + 1) / 2 : rb;
    const int ib = h * half, ie = min(rb, ib + half);
    P acc[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) acc[c] = P(0);
    if (j < n) {
      const P* col = reinterpret_cast<const P*>(d.L) + (int64_t)j * m + n + tk.y;
      constexpr int QB = (sizeof(P) == 4 && NR == 1) ? 16 : 8;  // independent loads per step
      int i = ib;
      for (; i + QB <= ie; i += QB) {
        P l[QB];
#pragma unroll
        for (int q = 0; q < QB; q++) l[q] = col[i + q];
#pragma unroll
        for (int q = 0; q < QB; q++)
#pragma unroll
          for (int c = 0; c < NR; c++)
            if (c < nrhs) acc[c] += l[q] * xg[c * rb + i + q];
      }
      for (; i < ie; i++) {
        const P l = col[i];
#pragma unroll
        for (int c = 0; c < NR; c++)
          if (c < nrhs) acc[c] += l * xg[c * rb + i];
      }
    }
    if (two && h == 1 && j < n) {
#pragma unroll
      for (int c = 0; c < NR; c++)
        if (c < nrhs) red[c * n + j] = acc[c];
    }
    __syncthreads();
    if (h == 0 && j < n) {
#pragma unroll
      for (int c = 0; c < NR; c++)
        if (c < nrhs) out[c * W + j] = (double)(two ? acc[c] + red[c * n + j] : acc[c]);
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

// Backward diagonal step, one CTA per supernode: task {s, first_bwd, nbwd}; first_bwd is
// a global index into the backward task list, base the first task of this level.
template <typename P>
__global__ void __launch_bounds__(kSolveThreads)
    k_bwd_diag(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue, int64_t base, const SnDev* __restrict__ sns,
               int64_t ldv, int nrhs, int W, const double* __restrict__ part,
               double* __restrict__ w) {
  extern __shared__ __align__(16) double sm[];
  P* smp = reinterpret_cast<P*>(sm);
  __shared__ int s_next_task;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n;
    const bool inv = d.dinv != nullptr;
    P* L11 = smp;
    P* rdiag = L11 + n * n;
    P* xs = inv ? smp + n * (n + 1) : rdiag + n;  // with Y: the right-hand side, then xs
    if (inv) stage_dinv(smp, reinterpret_cast<const P*>(d.dinv), n);
    const int u = d.m - n;
    // w_s minus the partials of the supernode's backward tasks, summed in a fixed order with
    // eight loads in flight
    const int nq = u > 0 ? tk.z : 0;
    for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
      const int c = idx / n, j = idx - c * n;
      const double* pp = part + (tk.y - base) * W * nrhs + c * W + j;
      const int64_t ps = (int64_t)W * nrhs;
      double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int q = 0;
      for (; q + 8 <= nq; q += 8) {
#pragma unroll
        for (int t = 0; t < 8; t++) a[t] += pp[(q + t) * ps];
      }
      for (; q < nq; q++) a[0] += pp[q * ps];
      xs[idx] = (P)(w[c * ldv + d.col0 + j] - (((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]))));
    }
    if (inv) {
      cp_async_wait_all();
      __syncthreads();
      P* xo = xs + n * nrhs;
      dinv_apply<false>(smp, xs, xo, xo + n * nrhs, n, nrhs);
      xs = xo;
    } else {
      load_l11<P>(d, L11, rdiag);
      warp_trisolve<false>(L11, rdiag, xs, n, nrhs);
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < n * nrhs; idx += blockDim.x) {
      const int c = idx / n, j = idx - c * n;
      w[c * ldv + d.col0 + j] = xs[idx];
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
static inline size_t solve_smem(int W, int nrhs) {
  const size_t sub = (size_t)W * W + W + (size_t)W * nrhs;
  const size_t inv = W <= kDinvMaxWidth ? (size_t)W * (W + 1) + 2 * (size_t)W * nrhs + kSolveThreads : 0;
  return std::max(sub, inv) * sizeof(double);
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

template <typename P, int NR>
static void fwd_nr(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                   int nrhs, int W, double* y, double* w, double* fstage, cudaStream_t st) {
  const size_t sm = solve_smem(W, nrhs);
  if (fstage)
    k_fwd<P, true, NR><<<task_grid(k_fwd<P, true, NR>, kSolveThreads, sm, ntasks),
                         kSolveThreads, sm, st>>>(tasks, ntasks, queue, sns, ldv, nrhs, y, w,
                                                  fstage);
  else
    k_fwd<P, false, NR><<<task_grid(k_fwd<P, false, NR>, kSolveThreads, sm, ntasks),
                          kSolveThreads, sm, st>>>(tasks, ntasks, queue, sns, ldv, nrhs, y, w,
                                                   nullptr);
}

// right-hand sides per pass of the panel products: the smallest of 1, 4, 16, 32 >= nrhs
static inline int rhs_pass(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 4 ? 4 : nrhs <= 16 ? 16 : 32; }

template <typename P>
static void fwd_t(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                  int nrhs, int W, double* y, double* w, double* fstage, cudaStream_t st) {
  switch (rhs_pass(nrhs)) {
    case 1: fwd_nr<P, 1>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    case 4: fwd_nr<P, 4>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    case 16: fwd_nr<P, 16>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
    default: fwd_nr<P, 32>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st); break;
  }
}

static inline size_t bwd_partial_smem(int W, int nr) {
  return ((size_t)kSolveRows * nr + (size_t)W * nr) * sizeof(double);
}

template <typename P, int NR>
static void bwd_partial_nr(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                           int64_t ldv, int nrhs, int W, const double* w, double* part,
                           cudaStream_t st) {
  const size_t sp = bwd_partial_smem(W, NR);
  k_bwd_partial<P, NR><<<task_grid(k_bwd_partial<P, NR>, kSolveThreads, sp, ntasks),
                         kSolveThreads, sp, st>>>(tasks, ntasks, queue, sns, ldv, nrhs, W, w,
                                                  part);
}

void launch_fwd(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int64_t ldv,
                int nrhs, int W, double* y, double* w, double* fstage, bool f32, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (f32) fwd_t<float>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st);
  else fwd_t<double>(tasks, ntasks, queue, sns, ldv, nrhs, W, y, w, fstage, st);
}

void launch_fwd_gather(const int32_t* fg_row, const int64_t* fg_ptr, const int32_t* fg_ent,
                       int64_t nrows, int64_t ldv, int nrhs, const double* fstage, double* y,
                       cudaStream_t st) {
  if (nrows <= 0) return;
  int blocks = (int)std::min<int64_t>((nrows + 127) / 128, 152 * 8);
  k_fwd_gather<<<blocks, 128, 0, st>>>(fg_row, fg_ptr, fg_ent, nrows, ldv, nrhs, fstage, y);
}

template <typename P>
static void bwd_t(const int4* bwd_tasks, int nbwd, int* queues, int64_t bwd_base,
                  const int4* diag_tasks, int ndiag, const SnDev* sns, int64_t ldv, int nrhs,
                  int W, double* w, double* part, cudaStream_t st) {
  if (nbwd > 0) {
    switch (rhs_pass(nrhs)) {
      case 1: bwd_partial_nr<P, 1>(bwd_tasks, nbwd, queues, sns, ldv, nrhs, W, w, part, st); break;
      case 4: bwd_partial_nr<P, 4>(bwd_tasks, nbwd, queues, sns, ldv, nrhs, W, w, part, st); break;
      case 16: bwd_partial_nr<P, 16>(bwd_tasks, nbwd, queues, sns, ldv, nrhs, W, w, part, st); break;
      default: bwd_partial_nr<P, 32>(bwd_tasks, nbwd, queues, sns, ldv, nrhs, W, w, part, st); break;
    }
  }
  if (ndiag > 0) {
    const size_t sm = solve_smem(W, nrhs);
    k_bwd_diag<P><<<task_grid(k_bwd_diag<P>, kSolveThreads, sm, ndiag), kSolveThreads, sm,
                    st>>>(diag_tasks, ndiag, queues + 1, bwd_base, sns, ldv, nrhs, W, part, w);
  }
}

void launch_bwd(const int4* bwd_tasks, int nbwd, int* queues, int64_t bwd_base,
                const int4* diag_tasks, int ndiag, const SnDev* sns, int64_t ldv, int nrhs,
                int W, double* w, double* part, bool f32, cudaStream_t st) {
  if (f32)
    bwd_t<float>(bwd_tasks, nbwd, queues, bwd_base, diag_tasks, ndiag, sns, ldv, nrhs, W, w,
                 part, st);
  else
    bwd_t<double>(bwd_tasks, nbwd, queues, bwd_base, diag_tasks, ndiag, sns, ldv, nrhs, W, w,
                  part, st);
}

template <typename K>
static bool set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
         cudaSuccess;
}

template <typename P, int NR>
static bool set_solve_nr(size_t sm, size_t sp) {
  return set_smem(k_fwd<P, false, NR>, sm) && set_smem(k_fwd<P, true, NR>, sm) &&
         set_smem(k_bwd_partial<P, NR>, sp);
}

int set_solve_kernel_attrs(int W, int max_nrhs) {
  const size_t sm = solve_smem(W, max_nrhs);
  bool ok = set_smem(k_bwd_diag<double>, sm) && set_smem(k_bwd_diag<float>, sm) &&
            set_solve_nr<double, 1>(sm, bwd_partial_smem(W, 1)) &&
            set_solve_nr<double, 4>(sm, bwd_partial_smem(W, 4)) &&
            set_solve_nr<double, 16>(sm, bwd_partial_smem(W, 16)) &&
            set_solve_nr<double, 32>(sm, bwd_partial_smem(W, 32)) &&
            set_solve_nr<float, 1>(sm, bwd_partial_smem(W, 1)) &&
            set_solve_nr<float, 4>(sm, bwd_partial_smem(W, 4)) &&
            set_solve_nr<float, 16>(sm, bwd_partial_smem(W, 16)) &&
            set_solve_nr<float, 32>(sm, bwd_partial_smem(W, 32));
  return ok ? CHOL_OK : CHOL_E_CUDA;
}

}  // namespace chol
