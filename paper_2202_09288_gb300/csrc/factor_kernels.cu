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
// path, with DMMA a few percent ahead; the Schur tiles therefore use m8n8k4 DMMA.
#include <cuda_runtime.h>

#include <algorithm>

#include "chol_internal.h"
#include "kernels.h"

namespace chol {

__device__ __forceinline__ int lower_bound_dev(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void record_error(const MatDev& md, int col) {
  atomicMin(md.err, (unsigned long long)col + 1ull);
}

// Position of `key` in the sorted row list of a target supernode, or -1 (and a count in
// err[1]) if it is missing: the elimination-tree property guarantees it is present, so a
// miss is an internal inconsistency and the write is skipped rather than misdirected.
__device__ __forceinline__ int relative_row(const MatDev& md, const int32_t* rows, int m,
                                            int key) {
  const int p = lower_bound_dev(rows, m, key);
  if (p >= m || rows[p] != key) {
    atomicAdd(md.err + 1, 1ull);
    return -1;
  }
  return p;
}

// ---- assembly of A into the zeroed panels ------------------------------------------------
template <typename T>
__global__ void k_assemble(const double* __restrict__ vals, const int64_t* __restrict__ amap,
                           int64_t nnz, T* __restrict__ L) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    L[amap[p]] = (T)vals[p];
}

// ---- POTRF of each diagonal block ---------------------------------------------------------
// One CTA per supernode; the n x n lower block is factored in shared memory by the
// unblocked right-looking column algorithm: pivot sqrt, column scale, rank-1 update.
template <typename T>
__global__ void __launch_bounds__(128) k_potrf(const int4* __restrict__ tasks,
                                               const SnDev* __restrict__ sns,
                                               const MatDev* __restrict__ mats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  const int4 tk = tasks[blockIdx.x];
  const SnDev d = sns[tk.x];
  const int n = d.n, m = d.m;
  T* L = reinterpret_cast<T*>(d.L);
  __shared__ T piv_inv;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int c = idx / n, r = idx - c * n;
    A[idx] = r >= c ? L[(int64_t)c * m + r] : T(0);
  }
  __syncthreads();
  for (int j = 0; j < n; j++) {
    if (threadIdx.x == 0) {
      T p = A[j * n + j];
      if (!(p > T(0))) {
        record_error(mats[d.mat], d.col0 + j);
        p = T(1);
      }
      T s = sqrt(p);
      A[j * n + j] = s;
      piv_inv = T(1) / s;
    }
    __syncthreads();
    const T inv = piv_inv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[j * n + i] *= inv;
    __syncthreads();
    const int nt = n - j - 1;
    for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
      int c = idx / nt, r = idx - c * nt;
      if (r >= c) A[(j + 1 + c) * n + j + 1 + r] -= A[j * n + j + 1 + r] * A[j * n + j + 1 + c];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int c = idx / n, r = idx - c * n;
    if (r >= c) L[(int64_t)c * m + r] = A[idx];
  }
}

// ---- TRSM of the off-diagonal rows --------------------------------------------------------
// Task {s, r0}: rows r0 .. r0+31 of L21 (panel rows n + r0 + t), one row per thread:
// x_j = (a_j - sum_{k<j} x_k L_jk) / L_jj, i.e. L21 = A21 L11^{-T}.
template <typename T>
__global__ void __launch_bounds__(kTrsmRows) k_trsm(const int4* __restrict__ tasks,
                                                    const SnDev* __restrict__ sns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int4 tk = tasks[blockIdx.x];
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
  const int row = n + tk.y + t;
  if (row < m) {
    for (int j = 0; j < n; j++) {
      T acc = L[(int64_t)j * m + row];
      for (int k = 0; k < j; k++) acc -= X[k * kTrsmRows + t] * L11[k * n + j];
      acc *= rdiag[j];
      X[j * kTrsmRows + t] = acc;
      L[(int64_t)j * m + row] = acc;
    }
  }
}

// ---- Schur update tiles ---------------------------------------------------------------------
// Task {s, i0, k0}: the T x T tile of U_s = L21 L21^T at rows i0.., columns k0.. (offsets
// into the off-diagonal rows of s), computed with FP64 m8n8k4 DMMA.  Then each entry
// U(i, k), i >= k, is subtracted from the target panel t owning column rows[k]: column
// rows[k] - col0(t), row position of rows[i] inside t's row list (the relative map,
// found by binary search in t's sorted rows once per tile row and target).
//   OWNER == false: atomicAdd into the panel.
//   OWNER == true : the tile is written to the level staging buffer (U_s column-major,
//                   ld u) and k_assemble_owner applies it later in a fixed order.
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
    k_schur_f64(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
                const MatDev* __restrict__ mats, double* __restrict__ stage) {
  using Cfg = SchurCfg<TILE>;
  constexpr int KC = Cfg::KC, LDS = Cfg::LDS, MB = Cfg::MB;
  __shared__ __align__(16) double sh[2 * KC * LDS > TILE * (TILE + 1) ? 2 * KC * LDS
                                                                      : TILE * (TILE + 1)];
  __shared__ int run_start[TILE + 1];
  __shared__ int run_t[TILE];
  __shared__ int nruns;
  __shared__ int relpos[TILE];
  double* As = sh;              // [KC][LDS]: As[kk][ii] = L21[i0 + ii][kc + kk]
  double* Bs = sh + KC * LDS;   // [KC][LDS]: Bs[kk][jj] = L21[k0 + jj][kc + kk]

  const int4 tk = tasks[blockIdx.x];
  const SnDev d = sns[tk.x];
  const int n = d.n, m = d.m, u = m - n;
  const int i0 = tk.y, k0 = tk.z;
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

  const int32_t* rows = d.rows + n;  // off-diagonal rows of s
  const int ilim = min(TILE, u - i0), klim = min(TILE, u - k0);
  if (OWNER) {
    double* U = stage + d.ustage;
    for (int idx = tid; idx < klim * TILE; idx += Cfg::THREADS) {
      const int kk = idx / TILE, ii = idx - kk * TILE;
      if (ii < ilim && i0 + ii >= k0 + kk)
        U[(int64_t)(k0 + kk) * u + i0 + ii] = Cs[kk * (TILE + 1) + ii];
    }
    return;
  }
  const MatDev md = mats[d.mat];
  // runs of tile columns with the same target supernode
  if (tid == 0) {
    int nr = 0, prev = -1;
    for (int kk = 0; kk < klim; kk++) {
      const int t = md.col2sn[rows[k0 + kk]];
      if (t != prev) { run_start[nr] = kk; run_t[nr] = t; nr++; prev = t; }
    }
    run_start[nr] = klim;
    nruns = nr;
  }
  __syncthreads();
  for (int r = 0; r < nruns; r++) {
    const SnDev td = sns[md.sn_base + run_t[r]];
    const int kb = run_start[r], ke = run_start[r + 1];
    // relative map of the tile rows inside the target's rows (rows >= the run's first
    // column row are all present in the target, by the elimination-tree property)
    for (int ii = tid; ii < ilim; ii += Cfg::THREADS) {
      const int gi = i0 + ii;
      relpos[ii] = gi >= k0 + kb ? relative_row(md, td.rows, td.m, rows[gi]) : -1;
    }
    __syncthreads();
    double* Lt = reinterpret_cast<double*>(td.L);
    const int w = ke - kb;
    for (int idx = tid; idx < w * TILE; idx += Cfg::THREADS) {
      const int kk = kb + idx / TILE, ii = idx % TILE;
      if (ii < ilim && i0 + ii >= k0 + kk && relpos[ii] >= 0) {
        const int c = rows[k0 + kk] - td.col0;
        atomicAdd(&Lt[(int64_t)c * td.m + relpos[ii]], -Cs[kk * (TILE + 1) + ii]);
      }
    }
    __syncthreads();
  }
}

// ---- owner assembly -----------------------------------------------------------------------
// Group {t, cb, first, end}: every staged U_s entry of this level that falls into columns
// [32 cb, 32 cb + 32) of target t is subtracted, sources in ascending s, one source at a
// time: each panel entry sees its updates in a fixed order, so the result is bitwise
// reproducible.
constexpr int kAsmThreads = 256;
constexpr int kAsmRowChunk = 1024;

__global__ void __launch_bounds__(kAsmThreads)
    k_assemble_owner(const int4* __restrict__ groups, const int4* __restrict__ srcs,
                     const SnDev* __restrict__ sns, const MatDev* __restrict__ mats,
                     const double* __restrict__ stage) {
  __shared__ int relpos[kAsmRowChunk];
  const int4 g = groups[blockIdx.x];
  const SnDev td = sns[g.x];
  const MatDev md = mats[td.mat];
  double* Lt = reinterpret_cast<double*>(td.L);
  for (int q = g.z; q < g.w; q++) {
    const int4 sr = srcs[q];
    const SnDev sd = sns[sr.x];
    const int u = sd.m - sd.n;
    const int32_t* rows = sd.rows + sd.n;
    const double* U = stage + sd.ustage;
    for (int ib = sr.y; ib < u; ib += kAsmRowChunk) {
      const int ilen = min(kAsmRowChunk, u - ib);
      __syncthreads();
      for (int ii = threadIdx.x; ii < ilen; ii += blockDim.x)
        relpos[ii] = relative_row(md, td.rows, td.m, rows[ib + ii]);
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
}

// ---- launchers --------------------------------------------------------------------------------
void launch_assemble(const double* vals, const int64_t* amap, int64_t nnz, void* L, bool f32,
                     cudaStream_t st) {
  if (nnz <= 0) return;
  int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
  if (f32) k_assemble<float><<<blocks, 256, 0, st>>>(vals, amap, nnz, (float*)L);
  else k_assemble<double><<<blocks, 256, 0, st>>>(vals, amap, nnz, (double*)L);
}

void launch_potrf(const int4* tasks, int ntasks, const SnDev* sns, const MatDev* mats,
                  int max_width, cudaStream_t st) {
  if (ntasks <= 0) return;
  size_t sm = (size_t)max_width * max_width * sizeof(double);
  k_potrf<double><<<ntasks, 128, sm, st>>>(tasks, sns, mats);
}

void launch_trsm(const int4* tasks, int ntasks, const SnDev* sns, int max_width,
                 cudaStream_t st) {
  if (ntasks <= 0) return;
  size_t sm = ((size_t)max_width * max_width + max_width + (size_t)max_width * kTrsmRows) *
              sizeof(double);
  k_trsm<double><<<ntasks, kTrsmRows, sm, st>>>(tasks, sns);
}

void launch_schur(int cls, const int4* tasks, int ntasks, const SnDev* sns, const MatDev* mats,
                  double* stage, bool owner, cudaStream_t st) {
  if (ntasks <= 0) return;
#define CHOL_SCHUR(T)                                                                        \
  if (owner)                                                                                 \
    k_schur_f64<T, true><<<ntasks, SchurCfg<T>::THREADS, 0, st>>>(tasks, sns, mats, stage);  \
  else                                                                                       \
    k_schur_f64<T, false><<<ntasks, SchurCfg<T>::THREADS, 0, st>>>(tasks, sns, mats, stage);
  if (cls == kTile64) { CHOL_SCHUR(64) }
  else if (cls == kTile32) { CHOL_SCHUR(32) }
  else { CHOL_SCHUR(16) }
#undef CHOL_SCHUR
}

void launch_assemble_owner(const int4* groups, int ngroups, const int4* srcs, const SnDev* sns,
                           const MatDev* mats, const double* stage, cudaStream_t st) {
  if (ngroups <= 0) return;
  k_assemble_owner<<<ngroups, kAsmThreads, 0, st>>>(groups, srcs, sns, mats, stage);
}

int set_factor_kernel_attrs(int max_width) {
  size_t potrf = (size_t)max_width * max_width * sizeof(double);
  size_t trsm = ((size_t)max_width * max_width + max_width + (size_t)max_width * kTrsmRows) *
                sizeof(double);
  if (cudaFuncSetAttribute(k_potrf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)potrf) != cudaSuccess)
    return CHOL_E_CUDA;
  if (cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm) != cudaSuccess)
    return CHOL_E_CUDA;
  return CHOL_OK;
}

}  // namespace chol
