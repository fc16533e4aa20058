// noalloc.cu -- a solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a solve: a host program
// that is capturing a stream in global capture mode (where cudaMalloc is an error), a
// runtime that owns the whole device memory pool and forbids allocations behind its
// back, or a latency-bound service loop that cannot afford the device-wide
// synchronization cudaMalloc may imply.  chol_solve() may grow its workspace on the
// first call with more right-hand sides; chol_solve_noalloc() never does: its workspace
// is one fixed array in the library's device image, sized kNoAllocScratchBytes.
//
// The array lives in every GPU that loads the library until the process exits.  Every
// call uses the same array and leaves its contents behind: the only part that must start
// at zero, the work-queue counters of the solve's launches at its head, is cleared by each
// call; every other workspace entry is written before it is read.  Two calls whose device
// work overlaps (different streams, or different contexts on one device) race on the
// array, so the caller must order them.
#include <cuda_runtime.h>

#include <mutex>

#include "api_internal.h"
#include "chol_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr size_t kNoAllocScratchDoubles = kNoAllocScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on `device` (the host-side symbol is only a stand-in).
// Looked up once per device with that device current.
int scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return CHOL_E_NODEVICE;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CHOL_E_CUDA;
    }
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return CHOL_OK;
}

// Runs the solve with `device` current and makes the caller's current device current again
// on every return path (the caller may drive another GPU from the same thread).
int solve_on_device(chol_ctx* ctx, const chol_num* num, int device, int64_t nrhs,
                    int64_t chunk, const double* B, int64_t ldb, double* X, int64_t ldx) {
  double* ws = nullptr;
  int rc = scratch_address(device, &ws);
  if (rc) return rc;
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int k = (int)(nrhs - c0 < chunk ? nrhs - c0 : chunk);
    rc = chol::enqueue_solve_ws(ctx, num, k, B + c0 * ldb, ldb, X + c0 * ldx, ldx, ws);
    if (rc) return rc;
  }
  return CHOL_OK;
}

}  // namespace

extern "C" size_t chol_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int chol_solve_noalloc(chol_ctx* ctx, const chol_num* num, int64_t nrhs,
                                  const double* B, int64_t ldb, double* X, int64_t ldx) {
  int64_t n = 0;
  int rc = chol::check_solve_args(ctx, num, nrhs, B, ldb, X, ldx, &n);
  if (rc) return rc;
  if (nrhs == 0 || n == 0) return CHOL_OK;
  const int64_t chunk = nrhs < 32 ? nrhs : 32;
  if (chol::solve_scratch_doubles(num, chunk) > kNoAllocScratchDoubles) return CHOL_E_SCRATCH;
  const int device = chol::ctx_device(ctx);
  int caller = -1;
  if (cudaGetDevice(&caller) != cudaSuccess) {
    cudaGetLastError();
    caller = -1;
  }
  if (caller != device && cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return CHOL_E_NODEVICE;
  }
  rc = solve_on_device(ctx, num, device, nrhs, chunk, B, ldb, X, ldx);
  if (caller >= 0 && caller != device && cudaSetDevice(caller) != cudaSuccess) {
    cudaGetLastError();
    if (!rc) rc = CHOL_E_CUDA;
  }
  return rc;
}
