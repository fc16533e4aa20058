// device_common.cuh -- device helpers shared by the factorization kernels: the relative
// row lookup, error recording, and the epilogue that applies a finished Schur tile.
#pragma once

#include <cuda_runtime.h>

#include "chol_internal.h"

namespace chol {

__device__ __forceinline__ int lower_bound_dev(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Adds v to *p in global memory when the old value is not needed: a PTX reduction, which
// returns nothing, so the issuing warp never waits for the round trip to L2 (an atomicAdd
// can be compiled as an atomic that returns the old value into a register).
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v));
}
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v));
}

__device__ __forceinline__ void record_error(const MatDev& md, int col) {
  atomicMin(md.err, (unsigned long long)col + 1ull);
}

// Index of the target run of supernode d that holds its off-diagonal row position pos
// (runs start at increasing positions, the first at 0).
__device__ __forceinline__ int find_run(const MatDev& md, const SnDev& d, int pos) {
  int lo = d.run0, hi = d.run0 + d.nrun - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (md.run_a[mid] <= pos) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Applies a finished T x T tile of U_s (in shared memory, Cs[kk * (TILE + 1) + ii], rows
// i0 + ii and columns k0 + kk of the off-diagonal part of s): each entry U(i, k), i >= k,
// is subtracted from the target panel t owning column rows[k] -- column rows[k] - col0(t),
// row position of rows[i] inside t's row list (the relative map built once per pattern).
//   OWNER == false: added into the panel (red_add).
//   OWNER == true : the tile is written to the level staging buffer (U_s column-major,
//                   ld u) and k_assemble_owner applies it later in a fixed order.
template <typename T, int TILE, int THREADS, bool OWNER>
__device__ __forceinline__ void schur_tile_epilogue(const T* Cs, const SnDev& d, int i0, int k0,
                                                    const SnDev* __restrict__ sns,
                                                    const MatDev* __restrict__ mats,
                                                    T* __restrict__ stage) {
  constexpr int RB = THREADS >= TILE ? THREADS / TILE : 1;  // runs resolved at a time
  constexpr int LANES = THREADS < 32 ? THREADS : 32;
  __shared__ int tcol[TILE];                 // target supernode of every tile column
  __shared__ int run_start[TILE + 1];
  __shared__ int run_t[TILE];
  __shared__ long long run_rb[TILE];         // relative-map base of every run
  __shared__ int nruns;
  __shared__ int relpos[RB][TILE];
  const int tid = threadIdx.x;
  const int n = d.n, u = d.m - d.n;
  const int32_t* rows = d.rows + n;  // off-diagonal rows of s
  const int ilim = min(TILE, u - i0), klim = min(TILE, u - k0);
  if (OWNER) {
    T* U = stage + d.ustage;
    for (int idx = tid; idx < klim * TILE; idx += THREADS) {
      const int kk = idx / TILE, ii = idx - kk * TILE;
      if (ii < ilim && i0 + ii >= k0 + kk)
        U[(int64_t)(k0 + kk) * u + i0 + ii] = Cs[kk * (TILE + 1) + ii];
    }
    return;
  }
  const MatDev md = mats[d.mat];
  // targets of the tile columns, all at once
  for (int kk = tid; kk < klim; kk += THREADS) tcol[kk] = md.col2sn[rows[k0 + kk]];
  __syncthreads();
  // runs of columns with the same target, found with warp ballots by the first warp
  if (tid < LANES) {
    const unsigned mask = LANES == 32 ? 0xffffffffu : ((1u << LANES) - 1u);
    int nr = 0;
    for (int base = 0; base < klim; base += LANES) {
      const int kk = base + tid;
      const bool start = kk < klim && (kk == 0 || tcol[kk] != tcol[kk - 1]);
      const unsigned b = __ballot_sync(mask, start);
      if (start) {
        const int q = nr + __popc(b & ((1u << tid) - 1u));
        run_start[q] = kk;
        run_t[q] = tcol[kk];
        run_rb[q] = md.run_base[find_run(md, d, k0 + kk)];
      }
      nr += __popc(b);
    }
    if (tid == 0) {
      run_start[nr] = klim;
      nruns = nr;
    }
  }
  __syncthreads();
  for (int r0 = 0; r0 < nruns; r0 += RB) {
    // positions of the tile rows inside each target's rows, from the relative map (rows at
    // or below the run's first column row are all present in the target, by the
    // elimination-tree property)
    for (int idx = tid; idx < RB * TILE; idx += THREADS) {
      const int rr = idx / TILE, ii = idx - rr * TILE;
      const int r = r0 + rr;
      if (r < nruns && ii < ilim) {
        const int gi = i0 + ii;
        relpos[rr][ii] = gi >= k0 + run_start[r] ? md.relmap[run_rb[r] + gi] : -1;
      }
    }
    __syncthreads();
    for (int rr = 0; rr < RB && r0 + rr < nruns; rr++) {
      const int r = r0 + rr;
      const SnDev& td = sns[md.sn_base + run_t[r]];
      T* Lt = reinterpret_cast<T*>(td.L);
      const int kb = run_start[r], w = run_start[r + 1] - kb;
      for (int idx = tid; idx < w * TILE; idx += THREADS) {
        const int kk = kb + idx / TILE, ii = idx % TILE;
        const int p = relpos[rr][ii];
        if (ii < ilim && i0 + ii >= k0 + kk && p >= 0) {
          const int c = rows[k0 + kk] - td.col0;
          red_add(&Lt[(int64_t)c * td.m + p], -Cs[kk * (TILE + 1) + ii]);
        }
      }
    }
    __syncthreads();
  }
}

// Asynchronous 4- or 8-byte global -> shared copy (cp.async, L1-allocating).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The lower triangle of a supernode's n x n diagonal block (panel column c, rows c..n-1, leading
// dimension m) into A (column-major, leading dimension lda, or n): one warp per column, lanes
// along the rows, every copy in flight at once.  Followed by cp_async_wait_all and a barrier.
template <typename T>
__device__ __forceinline__ void stage_diag_block_ld(T* A, int lda, const T* __restrict__ L, int n, int m) {
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int c = threadIdx.x >> 5; c < n; c += nwarp)
    for (int r = c + lane; r < n; r += 32) cp_async_elem(A + c * lda + r, L + (int64_t)c * m + r);
}
template <typename T>
__device__ __forceinline__ void stage_diag_block(T* A, const T* __restrict__ L, int n, int m) {
  stage_diag_block_ld(A, n, L, n, m);
}

// Up to 128 off-diagonal rows of a supernode panel and its n columns into shared memory,
// X[k * ld + i] = L21[i, k] (L21 column-major with leading dimension m, rows from the block's
// first): rows below `valid` by cp.async, every copy in flight at once; rows from `valid` on
// are zero.  Followed by cp_async_wait_all and a barrier.
template <typename T>
__device__ __forceinline__ void stage_row_block(T* X, int ld, const T* __restrict__ L21,
                                                int64_t m, int n, int valid) {
  for (int idx = threadIdx.x; idx < n * 128; idx += blockDim.x) {
    const int k = idx >> 7, i = idx & 127;
    if (i < valid) cp_async_elem(X + k * ld + i, L21 + (int64_t)k * m + i);
    else X[k * ld + i] = T(0);
  }
}

}  // namespace chol
