// gmres.cu -- iterative refinement whose correction equations are solved by flexible GMRES
// preconditioned with the factor (chol_refine_gmres).
//
// Refinement with the factor alone (chol_refine) contracts the error by about
// kappa(A) * (the factor's relative accuracy) per step, so an FP32 factor stalls once kappa
// passes ~1e7.  Here every refinement step takes the FP64 residual r = b - A x and solves
// A d = r by GMRES with the factor as right preconditioner M^-1 (an FP32 factor of the
// equilibrated matrix, or an FP64 one), which converges for far larger kappa, then updates
// x += d in FP64.  The Krylov basis is orthonormalized in FP64 by classical Gram-Schmidt
// with one reorthogonalization.  The preconditioned vectors z_j = M^-1 v_j are kept and
// d = Z y (flexible GMRES): an FP32 solve rounds its input, so M^-1 (V y) is not the
// combination of the M^-1 v_j the Arnoldi relation was built from.
//
// Device kernels (FP64): the CSR SpMV y = A x, the dot products V^T w as fixed-order
// two-pass reductions (reproducible run to run), w -= V h, v = w / s and x += Z y.  The small
// Hessenberg least-squares problem (Givens rotations) is solved on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "chol_internal.h"
#include "kernels.h"
#include "runtime.h"

using namespace chol::rt;

namespace chol {
namespace {

constexpr int kGmThreads = 256;
constexpr int kGmDotChunks = 152;       // row chunks of a dot product (one block per SM)
constexpr int kGmMaxRestart = 64;       // Krylov vectors per GMRES cycle, at most
constexpr int kGmDefaultRestart = 30;
constexpr double kGmInnerTol = 1e-6;    // GMRES stops once the correction residual fell this much

int gm_grid(int64_t n) {
  return (int)std::min<int64_t>((n + kGmThreads - 1) / kGmThreads, 152 * 8);
}

// y = A x with the full symmetric A in CSR form (src indexes the stored lower values).
__global__ void k_gm_spmv(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ src, const double* __restrict__ vals,
                          int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; e++) s += vals[src[e]] * x[col[e]];
    y[i] = s;
  }
}

// part[c * G + g] = the dot product of V[:, c] and w over row chunk g (G = gridDim.x chunks,
// column c = blockIdx.y), summed in a fixed order.
__global__ void __launch_bounds__(kGmThreads)
    k_gm_dot_part(const double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                  int64_t n, double* __restrict__ part) {
  __shared__ double red[kGmThreads / 32];
  const int c = blockIdx.y, g = blockIdx.x, G = gridDim.x;
  const int64_t chunk = (n + G - 1) / G, r0 = (int64_t)g * chunk;
  const int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
  const double* v = V + (int64_t)c * ldv;
  double s = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s = fma(v[r], w[r], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kGmThreads / 32; k++) t += red[k];
    part[(int64_t)c * G + g] = t;
  }
}

// h[c] = sum over the chunks of part[c * G + g], in chunk order.
__global__ void k_gm_dot_final(const double* __restrict__ part, int G, int ncols,
                               double* __restrict__ h) {
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < G; g++) s += part[(int64_t)c * G + g];
    h[c] = s;
  }
}

// w[r] -= sum_c V[r, c] h[c]  (sub) or  x[r] += sum_c V[r, c] h[c]  (add)
template <bool ADD>
__global__ void __launch_bounds__(kGmThreads)
    k_gm_gemv(const double* __restrict__ V, int64_t ldv, int ncols, const double* __restrict__ h,
              double* __restrict__ w, int64_t n) {
  __shared__ double hs[kGmMaxRestart + 1];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < ncols; c++) s = fma(V[(int64_t)c * ldv + r], hs[c], s);
    w[r] = ADD ? w[r] + s : w[r] - s;
  }
}

// v = w * inv
__global__ void k_gm_scale(const double* __restrict__ w, double inv, int64_t n,
                           double* __restrict__ v) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    v[r] = w[r] * inv;
}

int ensure_gmres_ws(chol_num* f, int m) {
  if (f->gm_cap >= m) return CHOL_OK;
  chol_ctx* c = f->ctx;
  const int64_t n = f->sym->S.n;
  void* ptrs[] = {f->d_gv, f->d_gz, f->d_gw, f->d_gpart, f->d_gh};
  for (void* p : ptrs) dev_free(c, p);
  f->d_gv = f->d_gz = f->d_gw = f->d_gpart = f->d_gh = nullptr;
  f->gm_cap = 0;
  int rc;
  if ((rc = dev_alloc(c, (void**)&f->d_gv, (size_t)n * (m + 1) * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_gz, (size_t)n * m * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_gw, (size_t)n * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_gpart, (size_t)kGmDotChunks * (m + 1) * 8)) ||
      (rc = dev_alloc(c, (void**)&f->d_gh, (size_t)3 * (m + 1) * 8)))
    return rc;
  f->gm_cap = m;
  return CHOL_OK;
}

// Device work of one refinement context: f holds A's values and the workspace, g is the
// factor used as preconditioner (f itself, or its FP64 fallback).
struct Gm {
  chol_num* f;
  chol_num* g;
  chol_ctx* c;
  int64_t n;
  int m;

  // h[0 .. ncols) = V[:, 0 .. ncols)^T w (device)
  void dots(const double* V, int ncols, const double* w, double* h) {
    prof_begin(c, kProfRefine);
    k_gm_dot_part<<<dim3(kGmDotChunks, ncols), kGmThreads, 0, c->stream>>>(V, n, w, n,
                                                                            f->d_gpart);
    k_gm_dot_final<<<1, 64, 0, c->stream>>>(f->d_gpart, kGmDotChunks, ncols, h);
    prof_end(c, kProfRefine, 2.0 * n * ncols, 8.0 * n * (ncols + 1));
  }
  void gemv(bool add, const double* V, int ncols, const double* h, double* w) {
    prof_begin(c, kProfRefine);
    if (add)
      k_gm_gemv<true><<<gm_grid(n), kGmThreads, 0, c->stream>>>(V, n, ncols, h, w, n);
    else
      k_gm_gemv<false><<<gm_grid(n), kGmThreads, 0, c->stream>>>(V, n, ncols, h, w, n);
    prof_end(c, kProfRefine, 2.0 * n * ncols, 8.0 * n * (ncols + 2));
  }
  void spmv(const double* x, double* y) {
    const Sym& S = f->sym->S;
    prof_begin(c, kProfRefine);
    k_gm_spmv<<<gm_grid(n), kGmThreads, 0, c->stream>>>(f->sym->dev.csr_ptr, f->sym->dev.csr_col,
                                                         f->sym->dev.csr_src, f->d_vals, n, x, y);
    prof_end(c, kProfRefine, 2.0 * (double)S.csr_ptr[n], 12.0 * (double)S.csr_ptr[n] + 16.0 * n);
  }
  void scale(const double* w, double inv, double* v) {
    prof_begin(c, kProfRefine);
    k_gm_scale<<<gm_grid(n), kGmThreads, 0, c->stream>>>(w, inv, n, v);
    prof_end(c, kProfRefine, (double)n, 16.0 * n);
  }
};

// One right-hand side b (device, ld n) into x (device, ld n): x = M^-1 b, then refinement
// steps, each solving A d = b - A x by flexible GMRES(m) preconditioned with g, until the
// relative residual meets tol (CHOL_OK) or maxit GMRES iterations in all, or two steps in a
// row that do not halve the residual (CHOL_E_STALL).  *iters counts GMRES iterations.
int gmres_column(Gm& G, const double* b, double* x, double tol, int maxit, int* iters,
                 double* resid) {
  chol_num* f = G.f;
  chol_ctx* c = G.c;
  const int64_t n = G.n;
  const int m = G.m;
  int rc;
  if ((rc = enqueue_solve(G.g, 1, b, n, x, n))) return rc;
  std::vector<double> H((size_t)(m + 1) * m), gv(m + 1), cs(m), sn(m), y(m),
      hb((size_t)3 * (m + 1));
  double prev = INFINITY;
  int stall = 0;
  for (;;) {
    double rel = 0.0, rmax = 0.0;
    if ((rc = residual_norms(f, 1, b, n, x, n, &rel, &rmax))) return rc;  // r in f->d_rr
    *resid = rel;
    if (rel <= tol) return CHOL_OK;
    if (*iters >= maxit) return CHOL_E_STALL;
    stall = rmax > 0.5 * prev ? stall + 1 : 0;
    if (stall >= 2) return CHOL_E_STALL;
    prev = rmax;
    // v_0 = r / ||r||_2
    G.dots(f->d_rr, 1, f->d_rr, f->d_gh);
    double nr = 0.0;
    if (cudaMemcpyAsync(&nr, f->d_gh, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      return CHOL_E_CUDA;
    }
    const double beta = std::sqrt(nr);
    if (!(beta > 0.0)) return CHOL_OK;
    G.scale(f->d_rr, 1.0 / beta, f->d_gv);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;  // Krylov vectors used
    while (k < m) {
      double* vk = f->d_gv + (size_t)k * n;
      double* zk = f->d_gz + (size_t)k * n;
      if ((rc = enqueue_solve(G.g, 1, vk, n, zk, n))) return rc;  // z_k = M^-1 v_k
      G.spmv(zk, f->d_gw);                                         // w = A z_k
      // classical Gram-Schmidt, twice: h1 = V^T w, w -= V h1, h2 = V^T w, w -= V h2
      G.dots(f->d_gv, k + 1, f->d_gw, f->d_gh);
      G.gemv(false, f->d_gv, k + 1, f->d_gh, f->d_gw);
      G.dots(f->d_gv, k + 1, f->d_gw, f->d_gh + (m + 1));
      G.gemv(false, f->d_gv, k + 1, f->d_gh + (m + 1), f->d_gw);
      G.dots(f->d_gw, 1, f->d_gw, f->d_gh + 2 * (m + 1));
      if (cudaMemcpyAsync(hb.data(), f->d_gh, hb.size() * 8, cudaMemcpyDeviceToHost,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return CHOL_E_CUDA;
      }
      double* col = H.data() + (size_t)k * (m + 1);  // column k of the Hessenberg matrix
      for (int i = 0; i <= k; i++) col[i] = hb[i] + hb[(m + 1) + i];
      const double hn = std::sqrt(std::max(0.0, hb[2 * (m + 1)]));
      col[k + 1] = hn;
      // earlier rotations, then the one that zeroes col[k + 1]
      for (int i = 0; i < k; i++) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = std::hypot(col[k], col[k + 1]);
      cs[k] = den > 0.0 ? col[k] / den : 1.0;
      sn[k] = den > 0.0 ? col[k + 1] / den : 0.0;
      col[k] = den;
      col[k + 1] = 0.0;
      gv[k + 1] = -sn[k] * gv[k];
      gv[k] = cs[k] * gv[k];
      (*iters)++;
      k++;
      const bool done = std::fabs(gv[k]) <= kGmInnerTol * beta || !(hn > 0.0) ||
                        *iters >= maxit;
      if (hn > 0.0 && k < m && !done) G.scale(f->d_gw, 1.0 / hn, f->d_gv + (size_t)k * n);
      if (done) break;
    }
    // y = R^-1 g (upper triangular k x k), then x += Z y
    for (int i = k - 1; i >= 0; i--) {
      double s = gv[i];
      for (int j = i + 1; j < k; j++) s -= H[(size_t)j * (m + 1) + i] * y[j];
      const double d = H[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? s / d : 0.0;
    }
    if (cudaMemcpyAsync(f->d_gh, y.data(), (size_t)k * 8, cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess) {
      cudaGetLastError();
      return CHOL_E_CUDA;
    }
    G.gemv(true, f->d_gz, k, f->d_gh, x);
    // the host copy of y must stay alive until the copy ran: the next step synchronizes
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      return CHOL_E_CUDA;
    }
  }
}

}  // namespace
}  // namespace chol

extern "C" int chol_refine_gmres(chol_ctx* c, chol_num* f, int64_t nrhs, const double* B,
                                 int64_t ldb, double* X, int64_t ldx, int where, double tol,
                                 int restart, int maxit, chol_refine_info* info) {
  chol_refine_info local;
  if (!info) info = &local;
  memset(info, 0, sizeof(*info));
  if (!c || !f || f->ctx != c || nrhs < 0 || !B || !X || B == X || tol < 0 || maxit < 0 ||
      restart < 0 || restart > chol::kGmMaxRestart)
    return CHOL_E_INVALID;
  const int64_t n = f->sym->S.n;
  if (ldb < n || ldx < n || (where != CHOL_HOST && where != CHOL_DEVICE)) return CHOL_E_INVALID;
  if (nrhs == 0 || n == 0) return CHOL_OK;
  if (cudaSetDevice(c->opts.device) != cudaSuccess) return CHOL_E_NODEVICE;
  int rc = chol_factor_status(c, f, nullptr);
  if (rc) return rc;
  unsigned long long redo = 0;
  if (cudaMemcpy(&redo, f->d_err + 2, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return CHOL_E_CUDA;
  }
  info->pivot_redos = (int64_t)redo;
  const int m = restart > 0 ? restart : chol::kGmDefaultRestart;
  if (maxit == 0) maxit = 10 * m;
  if ((rc = ensure_refine_ws(f, 1)) || (rc = ensure_solve_ws(f, 1)) ||
      (rc = chol::ensure_gmres_ws(f, m)) || (rc = compute_anorm(f)) ||
      (f->fb && (rc = ensure_solve_ws(f->fb, 1))))
    return rc;
  double worst = 0.0;
  for (int64_t col = 0; col < nrhs; col++) {
    const double* Bd = B + col * ldb;
    double* Xd = X + col * ldx;
    if (where == CHOL_HOST) {
      if (cudaMemcpyAsync(f->d_rb, Bd, n * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return CHOL_E_CUDA;
      Bd = f->d_rb;
      Xd = f->d_bx;
    }
    int iters = 0;
    double resid = 0.0;
    chol::Gm G{f, f->fb ? f->fb : f, c, n, m};
    rc = chol::gmres_column(G, Bd, Xd, tol, maxit, &iters, &resid);
    if (rc == CHOL_E_STALL && f->precision == CHOL_MIXED && !f->fb) {
      // the FP32 factor cannot deliver tol even with GMRES: factor A in FP64 once, use it
      if ((rc = make_factor(c, const_cast<chol_sym*>(f->sym), f->d_vals, CHOL_DEVICE, CHOL_FP64,
                            f->assembly, &f->fb, true)))
        return rc;
      if ((rc = chol_factor_status(c, f->fb, nullptr))) return rc;
      if ((rc = ensure_solve_ws(f->fb, 1))) return rc;
      info->fell_back = 1;
      chol::Gm G2{f, f->fb, c, n, m};
      rc = chol::gmres_column(G2, Bd, Xd, tol, maxit + iters, &iters, &resid);
    }
    if (f->fb) info->fell_back = 1;
    info->iterations += iters;
    worst = std::max(worst, resid);
    if (where == CHOL_HOST &&
        cudaMemcpyAsync(X + col * ldx, f->d_bx, n * 8, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess)
      return CHOL_E_CUDA;
    if (rc && rc != CHOL_E_STALL) return rc;
    if (rc == CHOL_E_STALL) {
      info->residual = worst;
      cudaStreamSynchronize(c->stream);
      return CHOL_E_STALL;
    }
  }
  info->residual = worst;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return CHOL_E_CUDA;
  return CHOL_OK;
}
