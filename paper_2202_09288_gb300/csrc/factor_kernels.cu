// factor_kernels.cu -- sm_103a kernels of the per-level supernodal factorization.
//
// The paper's factorization (Sec. 3, Listing 1) applies to every supernode the SYRK and
// GEMM updates of the supernodes that precede it, serializes their assembly with a lock,
// then runs POTRF on the diagonal block and TRSM on the rows below.  Here the same
// arithmetic is reorganized right-looking over the level sets of the supernodal
// elimination tree (Sec. 3, Fig. 1): all supernodes of a level are independent, so one
// launch factors every diagonal block of the level (POTRF), one solves all off-diagonal
// rows (TRSM), and one forms every Schur update U_s = L21 L21^T in tiles (the SYRK and
// GEMM of Listing 1) and subtracts it from the ancestor panels.  The lock becomes either
// device atomics or an owner-pulls assembly in a fixed order.
//
// FP64 throughput on GB300 is ~1 TFLOP/s for both DFMA and the FP64 `mma.sync` (DMMA)
// path, with DMMA a few percent ahead; the 32- and 64-wide Schur tiles here use m8n8k4
// DMMA, the 128-wide ones the bf16 tensor cores (oz_kernels.cu).
#include <cuda_runtime.h>

#include <algorithm>

#include "chol_internal.h"
#include "kernels.h"
#include "launch_util.h"
#include "device_common.cuh"
#include "oz_common.cuh"

namespace chol {

// ---- assembly of A into the zeroed panels ------------------------------------------------
template <typename T>
__global__ void k_assemble(const double* __restrict__ vals, const int64_t* __restrict__ amap,
                           int64_t nnz, T* __restrict__ L) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    L[amap[p]] = (T)vals[p];
}

// ---- diagonal-block Cholesky ---------------------------------------------------------------
// Cost model on this part: an FP64 warp instruction occupies its SM sub-partition's FP64 unit
// for ~64 cycles whether 1 or 32 lanes are active, a dependent DFMA chain advances one step
// per ~64 cycles, and the library's double sqrt and reciprocal take ~690 and ~440 cycles.
// The factorization is therefore organized so that (a) the serial per-column chain holds as
// few FP64 instructions as possible and (b) the bulk of the work runs with every lane busy.

// FMA in the block's precision.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// y = p^{-1/2} of a positive normal pivot: an FP32 seed y0 and one third-order correction.
// With r = 1 - p y0^2, p^{-1/2} = y0 (1 - r)^{-1/2} = y0 (1 + r/2 + 3r^2/8 + O(r^3)); the seed
// has |r| < 2^-20, so the dropped term is below 2^-58 relative, and the result is within an
// ulp or so.  p is first scaled by an even power of two into [1, 4) with integer exponent
// arithmetic (no FP32 overflow or underflow) and the result scaled back the same way: four
// FP64 instructions in all.  Subnormal, infinite and NaN p take the library path.
__device__ __forceinline__ double pivot_rsqrt(double p) {
  const int hi = __double2hiint(p), lo = __double2loint(p);
  const int ebits = (hi >> 20) & 0x7ff;
  if (ebits == 0 || ebits == 0x7ff) return 1.0 / sqrt(p);
  const int s = (ebits - 1023) & ~1;  // even, so that p 2^-s lies in [1, 4)
  const double ps = __hiloint2double(hi - s * (1 << 20), lo);
  const float y0f = rsqrtf((float)ps);
  const double y0 = (double)y0f, c1 = (double)(0.5f * y0f), c2 = (double)(0.375f * y0f);
  const double h = ps * y0;
  const double r = fma(-h, y0, 1.0);
  const double q = fma(r, c2, c1);  // y0/2 + 3 y0 r / 8
  const double y = fma(q, r, y0);
  return __hiloint2double(__double2hiint(y) - (s / 2) * (1 << 20), __double2loint(y));
}
// FP32: the hardware estimate and one Newton step.
__device__ __forceinline__ float pivot_rsqrt(float p) {
  const float y0 = rsqrtf(p);
  const float r = fmaf(-p * y0, y0, 1.f);
  return fmaf(0.5f * y0, r, y0);
}

// Threads of a POTRF CTA: warp 0 finishes the next column, the others update the trailing
// triangle (potrf_lookahead).
constexpr int kPotrfThreads = 256;

// Position table of the trailing update: the lower triangle of columns 2..n-1 taken column by
// column from the last (column n-1: 1 entry, column n-2: 2, ...), entry (C << 8) | R.  At step j
// the entries of columns j+2..n-1 are the first (n-j-2)(n-j-1)/2, so every step's work is a
// prefix, dealt evenly over the threads, and no index arithmetic is repeated per step.
__device__ __forceinline__ void build_update_table(uint16_t* tab, int n) {
  const int mm = n - 2, tot = mm > 0 ? mm * (mm + 1) / 2 : 0;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int cc = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if (cc * (cc + 1) / 2 > e) cc--;
    else if ((cc + 1) * (cc + 2) / 2 <= e) cc++;
    const int C = n - 1 - cc, R = C + (e - cc * (cc + 1) / 2);
    tab[e] = (uint16_t)((C << 8) | R);
  }
}
__host__ __device__ constexpr size_t update_table_bytes(int w) {
  return w > 2 ? (size_t)(w - 2) * (w - 1) / 2 * sizeof(uint16_t) : 0;
}
// FP64 POTRF's shared memory: the block (w^2 doubles), the update table, then (8-byte
// aligned) the w reciprocals of the diagonal that the in-place inverse uses
__host__ __device__ constexpr size_t potrf_rd_offset(int w) {
  return ((size_t)w * w * sizeof(double) + update_table_bytes(w) + 7) / 8 * 8;
}

// Right-looking Cholesky of the n x n block A (shared memory, column-major A[c * n + r]; only
// the lower triangle is read or written; n <= 128) with a one-column lookahead and one barrier
// per column.  Step j (column j final and scaled): warp 0 finishes column j+1 in registers --
// its update by column j, the pivot (a shuffle from the lane holding the diagonal), its
// reciprocal square root, the scaling (the diagonal becomes p y = sqrt(p)) -- while the other
// warps apply column j to columns j+2..n-1 through the position table (build_update_table),
// four elements per thread in flight.  Returns the first column whose pivot fails accept(p),
// else n.  A failed pivot does not stop the loop (every thread passes the same barriers); the
// caller discards the block.
template <typename T, typename Accept>
__device__ int potrf_lookahead(T* A, int n, const uint16_t* tab, Accept accept) {
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nupd = blockDim.x - 32;  // threads of the trailing update
  if (warp == 0) {
    T v[4];
#pragma unroll
    for (int g = 0; g < 4; g++) {
      if (32 * g >= n) break;
      const int r = 32 * g + lane;
      v[g] = r < n ? A[r] : T(0);
    }
    const T p = __shfl_sync(0xffffffffu, v[0], 0);
    const T y = pivot_rsqrt(p);
    if (lane == 0) s_bad = accept(p) ? n : 0;
#pragma unroll
    for (int g = 0; g < 4; g++) {
      if (32 * g >= n) break;
      const int r = 32 * g + lane;
      if (r < n) A[r] = v[g] * y;
    }
  }
  __syncthreads();
  for (int j = 0; j + 1 < n; j++) {
    const T* lj = A + j * n;
    if (warp == 0) {
      const int c = j + 1;
      T* ac = A + c * n;
      const T lc = lj[c];
      T v[4];
#pragma unroll
      for (int g = 0; g < 4; g++) {
        if (c + 32 * g >= n) break;
        const int r = c + 32 * g + lane;
        v[g] = r < n ? fma_t(-lj[r], lc, ac[r]) : T(0);
      }
      const T p = __shfl_sync(0xffffffffu, v[0], 0);  // lane 0 holds row c
      const T y = pivot_rsqrt(p);
      if (lane == 0 && s_bad == n && !accept(p)) s_bad = c;
#pragma unroll
      for (int g = 0; g < 4; g++) {
        if (c + 32 * g >= n) break;
        const int r = c + 32 * g + lane;
        if (r < n) ac[r] = v[g] * y;
      }
    } else {
      const int m = n - j - 2, tot = m * (m + 1) / 2;
      for (int e0 = tid - 32; e0 < tot; e0 += 4 * nupd) {
        int pos[4];
        T lr[4], lcv[4], av[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int e = e0 + q * nupd;
          pos[q] = -1;
          if (e < tot) {
            const int ent = tab[e], C = ent >> 8, R = ent & 255;
            pos[q] = C * n + R;
            lr[q] = lj[R];
            lcv[q] = lj[C];
            av[q] = A[pos[q]];
          }
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (pos[q] >= 0) A[pos[q]] = fma_t(-lr[q], lcv[q], av[q]);
      }
    }
    __syncthreads();
  }
  return s_bad;
}

template <typename T, typename S>
__device__ __forceinline__ void store_diag_block(T* __restrict__ L, const S* A, int n, int m) {
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < n; c += nwarp)
    for (int r = c + lane; r < n; r += 32) L[(int64_t)c * m + r] = (T)A[c * n + r];
}

// Y = L11^-1 in place in A (n x n, column-major, L11 in the lower triangle), by forward
// substitution on all columns of the identity at once: with l'_ij = L_ij / L_jj and Z = I, step
// j (one barrier) takes Z[i, c] -= l'_ij Z[j, c] for the rows i > j and columns c <= j (row j
// is final by then); Y[i, c] = Z[i, c] / L_ii.  l' lives in the strict lower triangle and the
// lower-triangular Z transposed in the upper triangle and the diagonal (Z[i, c] at
// A[i * n + c]), so that a warp's threads update consecutive words; on return A holds Y
// row-major (A[r * n + c] = Y[r, c], zeros above the diagonal).  rd: n doubles.
__device__ void invert_lower_inplace(double* A, double* rd, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) rd[j] = 1.0 / A[j * n + j];
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int c = idx / n, r = idx - c * n;
    if (r > c) A[idx] *= rd[c];          // l'_rc
    else A[idx] = r == c ? 1.0 : 0.0;    // Z[c, r] = I
  }
  __syncthreads();
  for (int j = 0; j + 1 < n; j++) {
    const int cols = j + 1, rows = n - 1 - j;
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int ii = idx / cols, c = idx - ii * cols, i = j + 1 + ii;
      A[i * n + c] -= A[j * n + i] * A[j * n + c];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    A[idx] = c <= r ? A[idx] * rd[r] : 0.0;
  }
  __syncthreads();
}

// The kOzInvRows slice rows of Y S (Y row-major in A, n x n; rows and columns past n are zero;
// S = diag(2^t_k), t_k the exponent of L11[k,k]) at slice rows y0 .. y0+63 of the scratch oy
// (planes oy_rows rows apart, then the rows' exponents, then the column shifts t_k): the
// right-hand operand of the supernode's tensor-core TRSM, A21 Y^T = (A21 S^-1)(Y S)^T.  The
// shift balances the operands: a column k of Y scales like 1/L_kk and the same column of A21
// like L_kk (rows and columns of A may span many decades), while Y S is the inverse of the
// unit-diagonal factor (exact: powers of two).  t: the n shifts; e: kOzInvRows ints.
__device__ void slice_inverse(const double* A, int n, const int* t, uint8_t* oy,
                              int64_t oy_rows, int64_t y0, int* e) {
  const size_t stride = (size_t)oy_rows * kOzRowBytes;
  int32_t* oexp = reinterpret_cast<int32_t*>(oy + kOzSlices * stride);
  for (int r = threadIdx.x; r < kOzInvRows; r += blockDim.x) {
    int f = 0;  // the largest exponent field of the row of Y S (fields shifted by t_k)
    if (r < n)
      for (int c = 0; c <= r; c++) {
        const int fc = oz_exp_field(A[r * n + c]);
        if (fc > 0) f = max(f, fc + t[c]);
      }
    e[r] = oz_row_exponent(f);
    oexp[y0 + r] = e[r];
    oexp[oy_rows + y0 + r] = r < n ? t[r] : 0;
  }
  __syncthreads();
  for (int item = threadIdx.x; item < kOzInvRows * 8; item += blockDim.x) {
    const int r = item >> 3, pc = item & 7;  // row, physical 16-byte chunk
    const int c = pc ^ (int)((y0 + r) & 7);  // logical chunk: columns 8c .. 8c+7
    long long R[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = 8 * c + j;
      R[j] = r < n && k < n ? oz_fixed(A[r * n + k], e[r] - t[k]) : 0;  // Y[r,k] 2^t_k
    }
    oz_write_chunk(R, oy + (size_t)(y0 + r) * kOzRowBytes + pc * 16, stride);
  }
}

// ---- POTRF of each diagonal block ---------------------------------------------------------
// One CTA (kPotrfThreads threads) per supernode; the n x n block is factored in shared memory by
// potrf_lookahead.  A non-positive pivot is an error (not SPD), recorded with its column.
// With oy, a task whose y field is set (a 128-tile supernode of the FP64 factor) also forms
// Y = L11^-1 (into d.dinv, row-major, for the solves) and Y's slices at rows y .. y+63 of oy,
// the operand of its tensor-core TRSM.
template <typename T>
__global__ void __launch_bounds__(kPotrfThreads) k_potrf(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
                                               const SnDev* __restrict__ sns,
                                               const MatDev* __restrict__ mats,
                                               uint8_t* __restrict__ oy, int64_t oy_rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_next_task;
  __shared__ int s_e[kOzInvRows], s_t[kOzInvRows];
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m;
    T* L = reinterpret_cast<T*>(d.L);
    uint16_t* tab = reinterpret_cast<uint16_t*>(smem_raw + (size_t)n * n * sizeof(double));
    stage_diag_block(A, L, n, m);
    build_update_table(tab, n);
    cp_async_wait_all();
    __syncthreads();
    const int bad = potrf_lookahead<T>(A, n, tab, [](T p) { return p > T(0); });
    if (bad < n && threadIdx.x == 0) record_error(mats[d.mat], d.col0 + bad);
    store_diag_block(L, A, n, m);
    __syncthreads();
    if constexpr (sizeof(T) == 8) {
      if (oy && tk.w >= 0 && d.dinv && n <= kOzInvRows) {
        double* Ad = reinterpret_cast<double*>(A);
        double* rd = reinterpret_cast<double*>(smem_raw + potrf_rd_offset(n));
        // column shifts t_k: the exponent of L11[k,k] (|L_kk| in [2^t, 2^(t+1)))
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
          const int f = oz_exp_field(Ad[k * n + k]);
          s_t[k] = f > 0 ? f - 1023 : 0;
        }
        invert_lower_inplace(Ad, rd, n);
        double* Y = reinterpret_cast<double*>(d.dinv);
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Y[idx] = Ad[idx];
        slice_inverse(Ad, n, s_t, oy, oy_rows, tk.w, s_e);
        __syncthreads();
      }
    }
    // a CTA's first task is its block index; only a grid smaller than the task list makes
    // CTAs take further tasks from this launch's work queue
    if (gridDim.x >= ntasks) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

// ---- TRSM of the off-diagonal rows --------------------------------------------------------
// Task {s, r0}: rows r0 .. r0+kTrsmRows-1 of L21 (panel rows n + r0 + lane), L21 = A21 L11^{-T},
// i.e. for each row x_j = (a_j - sum_{k<j} x_k L_jk) / L_jj.
//   k_trsm (any W <= 128): the substitution itself, one thread per row, partial rows in
//     shared memory.
// k_trsm_blk (W <= 64): a task's 32 rows (lane = row) are solved by all kTrsmWarps warps at
//   once, 16 columns at a time.  Block b (columns 16b .. 16b+15, diagonal block D_b of L11):
//   warp w takes the block's columns w, w + kTrsmWarps, ... and subtracts the products with
//   the solved columns of the earlier blocks, acc_k = a_k - sum_{j<16b} x_j L_kj; the partial
//   vectors are exchanged through shared memory and the block is finished as x_b = D_b^{-1}
//   acc_b with D_b^{-1} (lower triangular, formed per task by forward substitution on the
//   unit vectors).  Each warp thus issues 1/kTrsmWarps of a row's FMAs: on this part an FP64
//   warp instruction holds its warp for ~64 cycles, so the per-task latency (what the
//   single-supernode levels of the elimination tree's top wait for) falls with the warps.
constexpr int kTrsmWarps = 8;
constexpr int kTrsmCols = 16 / kTrsmWarps;  // columns of a block per warp

template <typename T>
constexpr size_t trsm_blk_smem() { return (64 * 64 + 64 * 32 + 16 * 32 + 4 * 16 * 16 + 64) * sizeof(T); }

template <typename T>
__global__ void __launch_bounds__(32 * kTrsmWarps) k_trsm_blk(const int4* __restrict__ tasks, int ntasks,
                                                              int* __restrict__ queue,
                                                              const SnDev* __restrict__ sns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);  // Ls[c * 64 + r] = L11[r][c]
  T* Xs = Ls + 64 * 64;                     // Xs[k * 32 + lane]: solved column k of the rows
  T* Acc = Xs + 64 * 32;                    // Acc[kk * 32 + lane]: block column kk before D_b^{-1}
  T* Dv = Acc + 16 * 32;                    // Dv[b * 256 + k * 16 + i] = (D_b^{-1})[k][i], k >= i
  T* rd = Dv + 4 * 16 * 16;                 // 1 / L11[k][k]
  __shared__ int s_next_task;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m;
    T* L = reinterpret_cast<T*>(d.L);
    stage_diag_block_ld(Ls, 64, L, n, m);
    // the warp's own columns k = 16 b + w + kTrsmWarps q of this task's row
    const int row = n + tk.y + lane;
    const bool live = row < m;
    T a[4 * kTrsmCols];
#pragma unroll
    for (int b = 0; b < 4; b++)
#pragma unroll
      for (int q = 0; q < kTrsmCols; q++) {
        const int k = 16 * b + w + kTrsmWarps * q;
        a[b * kTrsmCols + q] = (live && k < n) ? L[(int64_t)k * m + row] : T(0);
      }
    cp_async_wait_all();
    __syncthreads();
    if (threadIdx.x < n) rd[threadIdx.x] = T(1) / Ls[threadIdx.x * 65];
    __syncthreads();
    if (threadIdx.x < 64) {
      const int b = threadIdx.x >> 4, i = threadIdx.x & 15, c0 = 16 * b;
      if (c0 + i < n) {
        T* dv = Dv + b * 256;
        dv[i * 16 + i] = rd[c0 + i];
        for (int k = i + 1; k < 16 && c0 + k < n; k++) {
          T s = T(0);
          for (int j = i; j < k; j++) s = fma_t(Ls[(c0 + j) * 64 + c0 + k], dv[j * 16 + i], s);
          dv[k * 16 + i] = -s * rd[c0 + k];
        }
      }
    }
    __syncthreads();
    T out[4 * kTrsmCols] = {};
#pragma unroll
    for (int b = 0; b < 4; b++) {
      if (16 * b >= n) break;
      T acc[kTrsmCols];
#pragma unroll
      for (int q = 0; q < kTrsmCols; q++) acc[q] = a[b * kTrsmCols + q];
      const T* lrow = Ls + 16 * b + w;  // + j * 64 + kTrsmWarps q: L11[16b + w + kTrsmWarps q][j]
      for (int j = 0; j < 16 * b; j++) {
        const T xj = Xs[j * 32 + lane];
#pragma unroll
        for (int q = 0; q < kTrsmCols; q++) acc[q] = fma_t(-xj, lrow[j * 64 + kTrsmWarps * q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kTrsmCols; q++) Acc[(w + kTrsmWarps * q) * 32 + lane] = acc[q];
      __syncthreads();
      const T* dv = Dv + b * 256;
#pragma unroll
      for (int q = 0; q < kTrsmCols; q++) {
        const int kk = w + kTrsmWarps * q;
        T s = T(0);
        for (int i = 0; i <= kk; i++) s = fma_t(Acc[i * 32 + lane], dv[kk * 16 + i], s);
        out[b * kTrsmCols + q] = s;
        Xs[(16 * b + kk) * 32 + lane] = s;
      }
      __syncthreads();
    }
    if (live) {
#pragma unroll
      for (int b = 0; b < 4; b++)
#pragma unroll
        for (int q = 0; q < kTrsmCols; q++) {
          const int k = 16 * b + w + kTrsmWarps * q;
          if (k < n) L[(int64_t)k * m + row] = out[b * kTrsmCols + q];
        }
    }
    // a CTA's first task is its block index; only a grid smaller than the task list makes
    // CTAs take further tasks from this launch's work queue
    if (gridDim.x >= ntasks) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

template <typename T>
__global__ void __launch_bounds__(32) k_trsm(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
                                             const SnDev* __restrict__ sns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next_task;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m;
    T* L = reinterpret_cast<T*>(d.L);
    T* L11 = reinterpret_cast<T*>(smem_raw);  // n x n, column-major, ld n
    T* rdiag = L11 + n * n;                   // n
    T* X = rdiag + n;                         // n x 32: X[k * 32 + t]
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      int c = idx / n, r = idx - c * n;
      L11[idx] = r >= c ? L[(int64_t)c * m + r] : T(0);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) rdiag[j] = T(1) / L11[j * n + j];
    __syncthreads();
    const int t = threadIdx.x;
    for (int sub = 0; sub < kTrsmRows; sub += 32) {
      const int row = n + tk.y + sub + t;
      if (row < m) {
        for (int j = 0; j < n; j++) {
          T acc = L[(int64_t)j * m + row];
          for (int k = 0; k < j; k++) acc -= X[k * 32 + t] * L11[k * n + j];
          acc *= rdiag[j];
          X[j * 32 + t] = acc;
          L[(int64_t)j * m + row] = acc;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (gridDim.x >= ntasks) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

// ---- Schur update tiles ---------------------------------------------------------------------
// Task {s, i0, k0}: the T x T tile of U_s = L21 L21^T at rows i0.., columns k0.. (offsets
// into the off-diagonal rows of s), computed with FP64 m8n8k4 DMMA, then handed to
// schur_tile_epilogue.
template <int TILE>
struct SchurCfg {
  static constexpr int WARPS_M = TILE == 64 ? 2 : 1;
  static constexpr int WARPS_N = TILE == 64 ? 2 : 1;
  static constexpr int WT = TILE / WARPS_M;       // warp tile edge: 32 or 16
  static constexpr int MB = WT / 8;               // 8x8 blocks per warp edge
  static constexpr int THREADS = 32 * WARPS_M * WARPS_N;
  static constexpr int KC = 32;                   // K chunk staged in shared memory
  static constexpr int LDS = TILE + 8;            // padded stride (bank spread)
};

__device__ __forceinline__ void dmma_884(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

template <int TILE, bool OWNER>
__global__ void __launch_bounds__(SchurCfg<TILE>::THREADS)
    k_schur_f64(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue, const SnDev* __restrict__ sns,
                const MatDev* __restrict__ mats, int vsplit) {
  using Cfg = SchurCfg<TILE>;
  constexpr int KC = Cfg::KC, LDS = Cfg::LDS, MB = Cfg::MB;
  __shared__ __align__(16) double sh[2 * KC * LDS > TILE * (TILE + 1) ? 2 * KC * LDS
                                                                      : TILE * (TILE + 1)];
  double* As = sh;              // [KC][LDS]: As[kk][ii] = L21[i0 + ii][kc + kk]
  double* Bs = sh + KC * LDS;   // [KC][LDS]: Bs[kk][jj] = L21[k0 + jj][kc + kk]

  __shared__ int s_next_task;
  // with vsplit > 0 every task is 2^vsplit virtual tasks, one per sub-tile
  const int nv = ntasks << vsplit;
  for (int tq = blockIdx.x; tq < nv;) {
    const int4 tk = tasks[tq >> vsplit];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    // a task covers a (tk.w x tk.w) block of U_s (128 x 128 for the 128 class, whose .w
    // holds the slice offset instead); blocks larger than this kernel's tile are done as
    // TILE x TILE sub-tiles, skipping those wholly above the diagonal
    const int span = vsplit ? TILE << (vsplit >> 1) : (tk.w > TILE ? tk.w : TILE);
    const int sub_lo = vsplit ? (tq & ((1 << vsplit) - 1)) : 0;
    const int sub_hi = vsplit ? sub_lo + 1 : (span / TILE) * (span / TILE);
    for (int sub = sub_lo; sub < sub_hi; sub++) {
    const int i0 = tk.y + (sub / (span / TILE)) * TILE, k0 = tk.z + (sub % (span / TILE)) * TILE;
    if (i0 + TILE - 1 < k0 || i0 >= u || k0 >= u) continue;
    const double* L = reinterpret_cast<const double*>(d.L);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp / Cfg::WARPS_N, wn = warp % Cfg::WARPS_N;

    double acc[MB][MB][2];
  #pragma unroll
    for (int a = 0; a < MB; a++)
  #pragma unroll
      for (int b = 0; b < MB; b++) acc[a][b][0] = acc[a][b][1] = 0.0;

    for (int kc = 0; kc < n; kc += KC) {
      const int kw = min(KC, n - kc);
      for (int idx = tid; idx < KC * TILE; idx += Cfg::THREADS) {
        const int kk = idx / TILE, ii = idx - kk * TILE;
        double va = 0.0, vb = 0.0;
        if (kk < kw) {
          const int64_t col = (int64_t)(kc + kk) * m + n;
          if (i0 + ii < u) va = L[col + i0 + ii];
          if (k0 + ii < u) vb = L[col + k0 + ii];
        }
        As[kk * LDS + ii] = va;
        Bs[kk * LDS + ii] = vb;
      }
      __syncthreads();
      const int ksteps = (kw + 3) >> 2;
      for (int ks = 0; ks < ksteps; ks++) {
        const int kr = ks * 4 + (lane & 3);
        double af[MB], bf[MB];
  #pragma unroll
        for (int a = 0; a < MB; a++) af[a] = As[kr * LDS + wm * Cfg::WT + a * 8 + (lane >> 2)];
  #pragma unroll
        for (int b = 0; b < MB; b++) bf[b] = Bs[kr * LDS + wn * Cfg::WT + b * 8 + (lane >> 2)];
  #pragma unroll
        for (int a = 0; a < MB; a++)
  #pragma unroll
          for (int b = 0; b < MB; b++) dmma_884(acc[a][b], af[a], bf[b]);
      }
      __syncthreads();
    }
    // accumulators -> shared tile Cs[kk][ii] (ld TILE + 1)
    double* Cs = sh;
  #pragma unroll
    for (int a = 0; a < MB; a++)
  #pragma unroll
      for (int b = 0; b < MB; b++)
  #pragma unroll
        for (int e = 0; e < 2; e++) {
          const int ii = wm * Cfg::WT + a * 8 + (lane >> 2);
          const int kk = wn * Cfg::WT + b * 8 + (lane & 3) * 2 + e;
          Cs[kk * (TILE + 1) + ii] = acc[a][b][e];
        }
    __syncthreads();

    schur_tile_epilogue<double, TILE, Cfg::THREADS, OWNER>(
        Cs, d, i0, k0, sns, mats, static_cast<double*>(mats[d.mat].stage));
    __syncthreads();
    }
    __syncthreads();
    // a CTA's first task is its block index; only a grid smaller than the task list makes
    // CTAs take further tasks from this launch's work queue
    if (gridDim.x >= nv) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

// ---- FP32 Schur tiles (mixed precision) -------------------------------------------------------
// The same task and epilogue as k_schur_f64 on FP32 panels: each of the (T/4)^2 threads
// accumulates a 4 x 4 block of the tile in FP32 registers (rows ty + q T/4, columns
// tx + p T/4) from K chunks staged in shared memory.
template <int TILE>
struct SchurF32Cfg {
  static constexpr int S = TILE / 4;
  static constexpr int THREADS = S * S;
  static constexpr int KC = 32;
  static constexpr int LDS = TILE + 4;
};

template <int TILE, bool OWNER>
__global__ void __launch_bounds__(SchurF32Cfg<TILE>::THREADS)
    k_schur_f32(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue, const SnDev* __restrict__ sns,
                const MatDev* __restrict__ mats, int vsplit) {
  using Cfg = SchurF32Cfg<TILE>;
  constexpr int KC = Cfg::KC, LDS = Cfg::LDS, S = Cfg::S;
  __shared__ __align__(16) float sh[2 * KC * LDS > TILE * (TILE + 1) ? 2 * KC * LDS
                                                                     : TILE * (TILE + 1)];
  float* As = sh;
  float* Bs = sh + KC * LDS;
  __shared__ int s_next_task;
  // with vsplit > 0 every task is 2^vsplit virtual tasks, one per sub-tile
  const int nv = ntasks << vsplit;
  for (int tq = blockIdx.x; tq < nv;) {
    const int4 tk = tasks[tq >> vsplit];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    // a task covers a (tk.w x tk.w) block of U_s (128 x 128 for the 128 class, whose .w
    // holds the slice offset instead); blocks larger than this kernel's tile are done as
    // TILE x TILE sub-tiles, skipping those wholly above the diagonal
    const int span = vsplit ? TILE << (vsplit >> 1) : (tk.w > TILE ? tk.w : TILE);
    const int sub_lo = vsplit ? (tq & ((1 << vsplit) - 1)) : 0;
    const int sub_hi = vsplit ? sub_lo + 1 : (span / TILE) * (span / TILE);
    for (int sub = sub_lo; sub < sub_hi; sub++) {
    const int i0 = tk.y + (sub / (span / TILE)) * TILE, k0 = tk.z + (sub % (span / TILE)) * TILE;
    if (i0 + TILE - 1 < k0 || i0 >= u || k0 >= u) continue;
    const float* L = reinterpret_cast<const float*>(d.L);
    const int tid = threadIdx.x, tx = tid % S, ty = tid / S;
    float acc[4][4];
  #pragma unroll
    for (int q = 0; q < 4; q++)
  #pragma unroll
      for (int p = 0; p < 4; p++) acc[q][p] = 0.f;
    for (int kc = 0; kc < n; kc += KC) {
      const int kw = min(KC, n - kc);
      for (int idx = tid; idx < KC * TILE; idx += Cfg::THREADS) {
        const int kk = idx / TILE, ii = idx - kk * TILE;
        float va = 0.f, vb = 0.f;
        if (kk < kw) {
          const int64_t col = (int64_t)(kc + kk) * m + n;
          if (i0 + ii < u) va = L[col + i0 + ii];
          if (k0 + ii < u) vb = L[col + k0 + ii];
        }
        As[kk * LDS + ii] = va;
        Bs[kk * LDS + ii] = vb;
      }
      __syncthreads();
      for (int kk = 0; kk < kw; kk++) {
        float a[4], b[4];
  #pragma unroll
        for (int q = 0; q < 4; q++) a[q] = As[kk * LDS + ty + q * S];
  #pragma unroll
        for (int p = 0; p < 4; p++) b[p] = Bs[kk * LDS + tx + p * S];
  #pragma unroll
        for (int q = 0; q < 4; q++)
  #pragma unroll
          for (int p = 0; p < 4; p++) acc[q][p] = fmaf(a[q], b[p], acc[q][p]);
      }
      __syncthreads();
    }
    float* Cs = sh;
  #pragma unroll
    for (int q = 0; q < 4; q++)
  #pragma unroll
      for (int p = 0; p < 4; p++) Cs[(tx + p * S) * (TILE + 1) + ty + q * S] = acc[q][p];
    __syncthreads();
    schur_tile_epilogue<float, TILE, Cfg::THREADS, OWNER>(
        Cs, d, i0, k0, sns, mats, static_cast<float*>(mats[d.mat].stage));
    __syncthreads();
    }
    __syncthreads();
    // a CTA's first task is its block index; only a grid smaller than the task list makes
    // CTAs take further tasks from this launch's work queue
    if (gridDim.x >= nv) break;
    if (threadIdx.x == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
}

// ---- POTRF of the mixed-precision factor ---------------------------------------------------
// FP32 panels of the equilibrated matrix (unit diagonal before updates).  The block is
// factored in FP32; if any pivot falls below tau (tau times the original diagonal, which
// is 1 after equilibration), the block is factored again in FP64 from the panel's values,
// which are still unchanged in global memory, and the FP64 result is rounded into the panel.
// err[2] counts such redos.  The FP64 block overlays the FP32 one in shared memory.
__global__ void __launch_bounds__(kPotrfThreads) k_potrf_mixed(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
                                                     const SnDev* __restrict__ sns,
                                                     const MatDev* __restrict__ mats,
                                                     float tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next_task;
  float* A = reinterpret_cast<float*>(smem_raw);    // n x n FP32 work block
  double* D = reinterpret_cast<double*>(smem_raw);  // n x n FP64 block of a redo
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m;
    float* L = reinterpret_cast<float*>(d.L);
    uint16_t* tab = reinterpret_cast<uint16_t*>(smem_raw + (size_t)n * n * sizeof(double));
    stage_diag_block(A, L, n, m);
    build_update_table(tab, n);
    cp_async_wait_all();
    __syncthreads();
    const int stop = potrf_lookahead<float>(A, n, tab, [&](float p) { return p >= tau; });
    if (stop < n) {
      // a small FP32 pivot: the whole block again in FP64 (the barrier that ended the FP32
      // pass is behind every thread, so D may overwrite A)
      if (threadIdx.x == 0) atomicAdd(mats[d.mat].err + 2, 1ull);
      const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
      for (int c = threadIdx.x >> 5; c < n; c += nwarp)
        for (int r = c + lane; r < n; r += 32) D[c * n + r] = (double)L[(int64_t)c * m + r];
      __syncthreads();
      const int bad = potrf_lookahead<double>(D, n, tab, [](double p) { return p > 0.0; });
      if (bad < n && threadIdx.x == 0) record_error(mats[d.mat], d.col0 + bad);
      store_diag_block(L, D, n, m);
    } else {
      store_diag_block(L, A, n, m);
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

// ---- owner assembly -----------------------------------------------------------------------
// Group {t, cb, first, end}: every staged U_s entry of this level that falls into columns
// [32 cb, 32 cb + 32) of target t is subtracted, sources in ascending s, one source at a
// time: each panel entry sees its updates in a fixed order, so the result is bitwise
// reproducible.
constexpr int kAsmThreads = 256;
constexpr int kAsmRowChunk = 1024;

template <typename T>
__global__ void __launch_bounds__(kAsmThreads)
    k_assemble_owner(const int4* __restrict__ groups, int ntasks, int* __restrict__ queue, const int4* __restrict__ srcs,
                     const SnDev* __restrict__ sns, const MatDev* __restrict__ mats) {
  __shared__ int relpos[kAsmRowChunk];
  __shared__ int s_next_task;
  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 g = groups[tq];
    const SnDev td = sns[g.x];
    const MatDev md = mats[td.mat];
    T* Lt = reinterpret_cast<T*>(td.L);
    for (int q = g.z; q < g.w; q++) {
      const int4 sr = srcs[q];
      const SnDev sd = sns[sr.x];
      const int u = sd.m - sd.n;
      const int32_t* rows = sd.rows + sd.n;
      const T* U = static_cast<const T*>(md.stage) + sd.ustage;
      const long long rb = md.run_base[find_run(md, sd, sr.y)];
      for (int ib = sr.y; ib < u; ib += kAsmRowChunk) {
        const int ilen = min(kAsmRowChunk, u - ib);
        __syncthreads();
        for (int ii = threadIdx.x; ii < ilen; ii += blockDim.x) relpos[ii] = md.relmap[rb + ib + ii];
        __syncthreads();
        const int kw = sr.z - sr.y;
        for (int idx = threadIdx.x; idx < kw * ilen; idx += blockDim.x) {
          const int kk = idx / ilen, ii = idx - kk * ilen;
          const int k = sr.y + kk, i = ib + ii;
          if (i >= k && relpos[ii] >= 0) {
            const int c = rows[k] - td.col0;
            Lt[(int64_t)c * td.m + relpos[ii]] -= U[(int64_t)k * u + i];
          }
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

// ---- relative map -------------------------------------------------------------------------
// One CTA per supernode s: for every target run q of s (rows from run_a[q] on belong to the
// run's target t or to later targets, all of them rows of t by the elimination-tree
// property) the position of each row inside t's sorted row list; a row missing from t (an
// internal inconsistency) is stored as -1 and counted in *miss.
__global__ void k_build_relmap(const int32_t* __restrict__ sn_start, const int64_t* __restrict__ sn_rowptr,
                               const int32_t* __restrict__ rows, const int32_t* __restrict__ sn_run0,
                               const int32_t* __restrict__ run_a, const int32_t* __restrict__ run_t,
                               const int64_t* __restrict__ run_base, int32_t* __restrict__ relmap,
                               unsigned long long* __restrict__ miss) {
  const int s = blockIdx.x;
  const int n = sn_start[s + 1] - sn_start[s];
  const int64_t rp = sn_rowptr[s];
  const int u = (int)(sn_rowptr[s + 1] - rp) - n;
  const int32_t* r = rows + rp + n;
  for (int q = sn_run0[s]; q < sn_run0[s + 1]; q++) {
    const int t = run_t[q];
    const int tn = sn_start[t + 1] - sn_start[t], tcol0 = sn_start[t];
    const int64_t trp = sn_rowptr[t];
    const int tm = (int)(sn_rowptr[t + 1] - trp);
    const int32_t* tr = rows + trp;
    for (int i = run_a[q] + threadIdx.x; i < u; i += blockDim.x) {
      const int key = r[i];
      int p;
      if (key - tcol0 < tn) {
        p = key - tcol0;  // one of t's own columns
      } else {
        p = lower_bound_dev(tr, tm, key);
        if (p >= tm || tr[p] != key) {
          p = -1;
          atomicAdd(miss, 1ull);
        }
      }
      relmap[run_base[q] + i] = p;
    }
  }
}

void launch_build_relmap(int32_t ns, const int32_t* sn_start, const int64_t* sn_rowptr,
                         const int32_t* rows, const int32_t* sn_run0, const int32_t* run_a,
                         const int32_t* run_t, const int64_t* run_base, int32_t* relmap,
                         unsigned long long* miss, cudaStream_t st) {
  if (ns <= 0) return;
  k_build_relmap<<<ns, 256, 0, st>>>(sn_start, sn_rowptr, rows, sn_run0, run_a, run_t, run_base,
                                     relmap, miss);
}

// ---- launchers --------------------------------------------------------------------------------
void launch_assemble(const double* vals, const int64_t* amap, int64_t nnz, void* L, bool f32,
                     cudaStream_t st) {
  if (nnz <= 0) return;
  int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
  if (f32) k_assemble<float><<<blocks, 256, 0, st>>>(vals, amap, nnz, (float*)L);
  else k_assemble<double><<<blocks, 256, 0, st>>>(vals, amap, nnz, (double*)L);
}

static size_t potrf_smem(int w) { return potrf_rd_offset(w) + (size_t)w * sizeof(double); }

constexpr int kDinvThreads = 256;
template <typename P>
constexpr size_t dinv_smem() {
  return ((size_t)kDinvMaxWidth * kDinvMaxWidth + kDinvMaxWidth) * sizeof(P);
}

// Y = L11^-1 of the supernode of each task (POTRF tasks, one CTA per task) into d.dinv,
// row-major n x n (dinv[r * n + c] = Y[r, c], zeros above the diagonal), in the panel's
// precision; supernodes without dinv are skipped.  Forward substitution on all columns of
// the identity at once, right-looking: with l'_ij = L_ij / L_jj and Z = I, step j (one
// barrier) takes Z[i, c] -= l'_ij Z[j, c] for the rows i > j and columns c <= j (row j is
// final by then); Y[i, c] = Z[i, c] / L_ii at the end: n (n^2 - 1) / 6 multiply-adds, the n
// reciprocals once.  One n x n shared array holds both factors of each step: l' in the
// strict lower triangle (column-major, S[c * n + r]) and the lower-triangular Z transposed
// in the upper triangle and the diagonal (Z[i, c] at S[i * n + c]), so a warp's threads
// update consecutive words.  The solves apply Y instead of substituting serially (each FP64
// instruction holds its warp ~64 cycles, so a 64-step substitution chain costs ~10 us).
template <typename P>
__global__ void __launch_bounds__(kDinvThreads)
    k_diag_inverse(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
                   bool skip_sliced) {
  extern __shared__ __align__(16) double dsm[];
  const int4 tk = tasks[blockIdx.x];
  const SnDev d = sns[tk.x];
  if (!d.dinv || (skip_sliced && tk.w >= 0)) return;
  const int n = d.n;
  P* S = reinterpret_cast<P*>(dsm);
  P* rd = S + n * n;
  stage_diag_block(S, reinterpret_cast<const P*>(d.L), n, d.m);
  cp_async_wait_all();
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) rd[j] = P(1) / S[j * n + j];
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int c = idx / n, r = idx - c * n;
    if (r > c) S[idx] *= rd[c];          // l'_rc
    else S[idx] = r == c ? P(1) : P(0);  // Z[c, r] = I
  }
  __syncthreads();
  for (int j = 0; j + 1 < n; j++) {
    const int cols = j + 1, rows = n - 1 - j;
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int ii = idx / cols, c = idx - ii * cols, i = j + 1 + ii;
      S[i * n + c] -= S[j * n + i] * S[j * n + c];
    }
    __syncthreads();
  }
  P* Y = reinterpret_cast<P*>(d.dinv);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    Y[idx] = c <= r ? S[idx] * rd[r] : P(0);
  }
}

void launch_diag_inverse(const int4* tasks, int ntasks, const SnDev* sns, bool f32,
                         bool skip_sliced, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (f32)
    k_diag_inverse<float><<<ntasks, kDinvThreads, dinv_smem<float>(), st>>>(tasks, sns, false);
  else
    k_diag_inverse<double><<<ntasks, kDinvThreads, dinv_smem<double>(), st>>>(tasks, sns,
                                                                             skip_sliced);
}
static size_t potrf_mixed_smem(int w) {  // the FP64 block of a redo overlays the FP32 one
  return (size_t)w * w * sizeof(double) + update_table_bytes(w);
}
static size_t trsm_smem(int w) { return ((size_t)w * w + w + (size_t)w * 32) * sizeof(double); }

void launch_potrf(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                  const MatDev* mats, int max_width, bool f32, float tau, void* oy,
                  int64_t oy_rows, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (f32) {
    const size_t sm = potrf_mixed_smem(max_width);
    k_potrf_mixed<<<task_grid(k_potrf_mixed, kPotrfThreads, sm, ntasks), kPotrfThreads, sm, st>>>(
        tasks, ntasks, queue, sns, mats, tau);
  } else {
    const size_t sm = potrf_smem(max_width);
    k_potrf<double><<<task_grid(k_potrf<double>, kPotrfThreads, sm, ntasks), kPotrfThreads, sm, st>>>(
        tasks, ntasks, queue, sns, mats, static_cast<uint8_t*>(oy), oy_rows);
  }
}

template <typename T>
static void trsm_t(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int max_width,
                   cudaStream_t st) {
  if (max_width <= 64) {
    constexpr size_t sm = trsm_blk_smem<T>();
    k_trsm_blk<T><<<task_grid(k_trsm_blk<T>, 32 * kTrsmWarps, sm, ntasks), 32 * kTrsmWarps, sm, st>>>(
        tasks, ntasks, queue, sns);
    return;
  }
  const size_t sm = trsm_smem(max_width);
  k_trsm<T><<<task_grid(k_trsm<T>, 32, sm, ntasks), 32, sm, st>>>(tasks, ntasks, queue, sns);
}

void launch_trsm(const int4* tasks, int ntasks, int* queue, const SnDev* sns, int max_width,
                 bool f32, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (f32) trsm_t<float>(tasks, ntasks, queue, sns, max_width, st);
  else trsm_t<double>(tasks, ntasks, queue, sns, max_width, st);
}

template <int T, bool OWNER>
static void schur_f64_t(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                        const MatDev* mats, cudaStream_t st, int vsplit = 0) {
  constexpr int th = SchurCfg<T>::THREADS;
  k_schur_f64<T, OWNER><<<task_grid(k_schur_f64<T, OWNER>, th, 0, ntasks << vsplit), th, 0,
                         st>>>(tasks, ntasks, queue, sns, mats, vsplit);
}

template <int T, bool OWNER>
static void schur_f32_t(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                        const MatDev* mats, cudaStream_t st, int vsplit = 0) {
  constexpr int th = SchurF32Cfg<T>::THREADS;
  k_schur_f32<T, OWNER><<<task_grid(k_schur_f32<T, OWNER>, th, 0, ntasks << vsplit), th, 0,
                         st>>>(tasks, ntasks, queue, sns, mats, vsplit);
}

template <bool OWNER>
static void schur_cls(int cls, bool f32, const int4* tasks, int ntasks, int* queue,
                      const SnDev* sns, const MatDev* mats, cudaStream_t st) {
  if (f32) {
    // 128-wide tasks without the tensor-core scratch: four 64 x 64 virtual tasks
    if (cls == kTile128) schur_f32_t<64, OWNER>(tasks, ntasks, queue, sns, mats, st, 2);
    else if (cls == kTile64) schur_f32_t<64, OWNER>(tasks, ntasks, queue, sns, mats, st);
    else if (cls == kTile32) schur_f32_t<32, OWNER>(tasks, ntasks, queue, sns, mats, st);
    else schur_f32_t<16, OWNER>(tasks, ntasks, queue, sns, mats, st);
  } else {
    // FP64 128-wide tasks run as four 64 x 64 virtual tasks of the DMMA kernel
    if (cls == kTile128) schur_f64_t<64, OWNER>(tasks, ntasks, queue, sns, mats, st, 2);
    else if (cls == kTile64) schur_f64_t<64, OWNER>(tasks, ntasks, queue, sns, mats, st);
    else if (cls == kTile32) schur_f64_t<32, OWNER>(tasks, ntasks, queue, sns, mats, st);
    else schur_f64_t<16, OWNER>(tasks, ntasks, queue, sns, mats, st);
  }
}

void launch_schur(int cls, const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                  const MatDev* mats, bool owner, bool f32, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (owner) schur_cls<true>(cls, f32, tasks, ntasks, queue, sns, mats, st);
  else schur_cls<false>(cls, f32, tasks, ntasks, queue, sns, mats, st);
}

template <typename T>
static void asm_owner_t(const int4* groups, int ngroups, int* queue, const int4* srcs,
                        const SnDev* sns, const MatDev* mats, cudaStream_t st) {
  k_assemble_owner<T><<<task_grid(k_assemble_owner<T>, kAsmThreads, 0, ngroups),
                        kAsmThreads, 0, st>>>(groups, ngroups, queue, srcs, sns, mats);
}

void launch_assemble_owner(const int4* groups, int ngroups, int* queue, const int4* srcs,
                           const SnDev* sns, const MatDev* mats, bool f32, cudaStream_t st) {
  if (ngroups <= 0) return;
  if (f32) asm_owner_t<float>(groups, ngroups, queue, srcs, sns, mats, st);
  else asm_owner_t<double>(groups, ngroups, queue, srcs, sns, mats, st);
}

template <typename K>
static bool set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
         cudaSuccess;
}

int set_factor_kernel_attrs(int max_width) {
  bool ok = set_smem(k_diag_inverse<double>, dinv_smem<double>()) &&
            set_smem(k_diag_inverse<float>, dinv_smem<float>()) &&
            set_smem(k_potrf<double>, potrf_smem(max_width)) &&
            set_smem(k_potrf_mixed, potrf_mixed_smem(max_width)) &&
            set_smem(k_trsm_blk<double>, trsm_blk_smem<double>()) &&
            set_smem(k_trsm_blk<float>, trsm_blk_smem<float>()) &&
            set_smem(k_trsm<double>, trsm_smem(max_width)) &&
            set_smem(k_trsm<float>, trsm_smem(max_width));
  return ok ? CHOL_OK : CHOL_E_CUDA;
}

}  // namespace chol
