// refine_kernels.cu -- kernels of the mixed-precision factor and of FP64 iterative
// refinement.
//
// The paper factors in double precision (CHOLMOD).  On GB300 the FP64 units deliver about
// 1 TFLOP/s against ~72 TFLOP/s of FP32, so the library also offers a factor of the
// equilibrated matrix S A S (S = diag(a_jj)^{-1/2}) with FP32 panels, recovered to FP64
// accuracy by iterative refinement: r = b - A x in FP64 (CSR SpMV of the original A),
// d = solve(r) with the FP32 factor, x += d, until ||r||_inf / (||A||_inf ||x||_inf) meets
// the requested tolerance.
#include <cuda_runtime.h>

#include <algorithm>

#include "chol_internal.h"
#include "kernels.h"

namespace chol {

static inline int grid_for(int64_t total, int threads) {
  return (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 16);
}

// scale[j] = 1 / sqrt(a_jj) over the columns of A (lower CSC, diagonal first); a missing
// or non-positive diagonal is reported as a failing pivot at column iperm[j].
__global__ void k_diag_scale(const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowind,
                             const double* __restrict__ vals, const int32_t* __restrict__ iperm,
                             int64_t n, double* __restrict__ scale, unsigned long long* err) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = colptr[j];
    const bool ok = p < colptr[j + 1] && rowind[p] == j && vals[p] > 0.0;
    if (ok) {
      scale[j] = 1.0 / sqrt(vals[p]);
    } else {
      scale[j] = 1.0;
      atomicMin(err, (unsigned long long)iperm[j] + 1ull);
    }
  }
}

// L[amap[p]] = (float)(a_p * scale[row] * scale[col]) for every stored entry of A.
__global__ void k_assemble_scaled(const int64_t* __restrict__ colptr,
                                  const int32_t* __restrict__ rowind, const double* __restrict__ vals,
                                  const int64_t* __restrict__ amap, const double* __restrict__ scale,
                                  int64_t n, float* __restrict__ L) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double sj = scale[j];
    for (int64_t p = colptr[j]; p < colptr[j + 1]; p++)
      L[amap[p]] = (float)(vals[p] * scale[rowind[p]] * sj);
  }
}

// R[:, c] = B[:, c] - A X[:, c] with the full symmetric A in CSR form (csr_src indexes the
// stored lower values), FP64: one thread per row, all NR (>= nrhs) right-hand sides at once,
// so the row's entries are read once.
template <int NR>
__global__ void k_residual(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ src, const double* __restrict__ vals,
                           int64_t n, int nrhs, const double* __restrict__ X, int64_t ldx,
                           const double* __restrict__ B, int64_t ldb, double* __restrict__ R,
                           int64_t ldr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; e++) {
      const double v = vals[src[e]];
      const int64_t j = col[e];
#pragma unroll
      for (int c = 0; c < NR; c++)
        if (c < nrhs) s[c] += v * X[c * ldx + j];
    }
#pragma unroll
    for (int c = 0; c < NR; c++)
      if (c < nrhs) R[c * ldr + i] = B[c * ldb + i] - s[c];
  }
}

// Largest value of a block's threads (non-negative doubles order like their bit patterns), one
// atomic per block: v of every thread in, the result valid in thread 0.
__device__ __forceinline__ unsigned long long block_max(unsigned long long v) {
  __shared__ unsigned long long w[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) w[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? w[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  __syncthreads();
  return v;
}

// out[c] = max_i |V[i, c]|: column c = blockIdx.y, a grid-stride maximum per thread, then one
// atomic per block.
__global__ void k_absmax(const double* __restrict__ V, int64_t ld, int64_t n,
                         unsigned long long* __restrict__ out) {
  const int c = blockIdx.y;
  unsigned long long m = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(fabs(V[c * ld + i])));
  m = block_max(m);
  if (threadIdx.x == 0) atomicMax(out + c, m);
}

// ||A||_inf = max_i sum_e |a_ie| over the full CSR.
__global__ void k_anorm(const int64_t* __restrict__ ptr, const int32_t* __restrict__ src,
                        const double* __restrict__ vals, int64_t n,
                        unsigned long long* __restrict__ out) {
  unsigned long long m = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; e++) s += fabs(vals[src[e]]);
    m = max(m, (unsigned long long)__double_as_longlong(s));
  }
  m = block_max(m);
  if (threadIdx.x == 0) atomicMax(out, m);
}

// X[:, c] += D[:, c]
__global__ void k_axpy(double* __restrict__ X, int64_t ldx, const double* __restrict__ D,
                       int64_t ldd, int64_t n, int nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / n, i = q - c * n;
    X[c * ldx + i] += D[c * ldd + i];
  }
}

void launch_diag_scale(const int64_t* colptr, const int32_t* rowind, const double* vals,
                       const int32_t* iperm, int64_t n, double* scale, unsigned long long* err,
                       cudaStream_t st) {
  if (n <= 0) return;
  k_diag_scale<<<grid_for(n, 256), 256, 0, st>>>(colptr, rowind, vals, iperm, n, scale, err);
}

void launch_assemble_scaled(const int64_t* colptr, const int32_t* rowind, const double* vals,
                            const int64_t* amap, const double* scale, int64_t n, float* L,
                            cudaStream_t st) {
  if (n <= 0) return;
  k_assemble_scaled<<<grid_for(n, 256), 256, 0, st>>>(colptr, rowind, vals, amap, scale, n, L);
}

void launch_residual(const int64_t* ptr, const int32_t* col, const int32_t* src,
                     const double* vals, int64_t n, int nrhs, const double* X, int64_t ldx,
                     const double* B, int64_t ldb, double* R, int64_t ldr, cudaStream_t st) {
  if (n <= 0) return;
  // right-hand sides per pass: the smallest of 1, 4, 8, 16, 32 >= nrhs
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int k = std::min(32, nrhs - c0);
    const double* Xc = X + c0 * ldx;
    const double* Bc = B + c0 * ldb;
    double* Rc = R + c0 * ldr;
    const int g = grid_for(n, 256);
    if (k <= 1) k_residual<1><<<g, 256, 0, st>>>(ptr, col, src, vals, n, k, Xc, ldx, Bc, ldb, Rc, ldr);
    else if (k <= 4) k_residual<4><<<g, 256, 0, st>>>(ptr, col, src, vals, n, k, Xc, ldx, Bc, ldb, Rc, ldr);
    else if (k <= 8) k_residual<8><<<g, 256, 0, st>>>(ptr, col, src, vals, n, k, Xc, ldx, Bc, ldb, Rc, ldr);
    else if (k <= 16) k_residual<16><<<g, 256, 0, st>>>(ptr, col, src, vals, n, k, Xc, ldx, Bc, ldb, Rc, ldr);
    else k_residual<32><<<g, 256, 0, st>>>(ptr, col, src, vals, n, k, Xc, ldx, Bc, ldb, Rc, ldr);
  }
}

void launch_absmax(const double* V, int64_t ld, int64_t n, int nrhs, unsigned long long* out,
                   cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return;
  const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 152 * 2), (unsigned)nrhs);
  k_absmax<<<grid, 256, 0, st>>>(V, ld, n, out);
}

void launch_anorm(const int64_t* ptr, const int32_t* src, const double* vals, int64_t n,
                  unsigned long long* out, cudaStream_t st) {
  if (n <= 0) return;
  k_anorm<<<grid_for(n, 256), 256, 0, st>>>(ptr, src, vals, n, out);
}

void launch_axpy(double* X, int64_t ldx, const double* D, int64_t ldd, int64_t n, int nrhs,
                 cudaStream_t st) {
  if (n <= 0) return;
  k_axpy<<<grid_for(n * nrhs, 256), 256, 0, st>>>(X, ldx, D, ldd, n, nrhs);
}

}  // namespace chol
