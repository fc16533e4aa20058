// oz_kernels.cu -- FP64 Schur update tiles of the FP64 factor on the bf16 tcgen05 tensor
// cores by operand splitting (Ozaki's error-free splitting of a dot product).
//
// The update U_s = L21 L21^T (Sec. 3, Listing 1: SYRK + GEMM) of a 128-tile supernode is
// computed in two steps per level:
//   k_oz_slice  every row r of L21 gets an exponent e_r (max_k |L21[r,k]| < 2^e_r) and
//               kOzSlices integer slices s_p[r,k] of 7 bits with
//               L21[r,k] = 2^e_r sum_p s_p[r,k] 2^(-7(p+1)) + (error < 2^(e_r-57)),
//               stored as bf16 (exact) in rows of 128 bytes, 16-byte chunks pre-swizzled
//               for the tensor cores' 128-byte swizzle;
//   k_schur_oz  a 128 x 128 task is done as two 128 x 64 halves.  The 8 A slices (the
//               task's 128 rows) and 8 B slices (the half's 64 rows) are brought into
//               shared memory by bulk copies; one thread issues, for every slice pair
//               p + q < 8, the bf16 MMAs of D_{p+q} += S_p S_q^T into the tensor-memory
//               accumulator of the diagonal p + q (8 x 64 columns).  Every partial sum of
//               a diagonal is an integer below 2^23 (K <= 64), so FP32 accumulation is
//               exact.  The epilogue reads the accumulators (lane = tile row), forms
//               U[i,k] = 2^(e_i+e_k) sum_d 2^(-7(d+2)) D_d[i,k] in FP64 and scatters it
//               into the ancestors with FP64 atomics (or writes the owner staging buffer)
//               while the tensor cores already compute the next half.
// Every wait is bounded: after kOzSpinLimit polls the kernel records a timeout in err[3],
// waits (bounded) for its copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "chol_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.h"

namespace chol {

namespace {

constexpr int kOzThreads = 512;
constexpr int kOzM = 128;                                  // tile rows (UMMA M)
constexpr int kOzN = 64;                                   // columns per half (UMMA N)
constexpr uint32_t kOzASlice = kOzM * kOzRowBytes;         // 16 KB
constexpr uint32_t kOzBSlice = kOzN * kOzRowBytes;         // 8 KB
constexpr uint32_t kOzABytes = kOzSlices * kOzASlice;      // 128 KB
constexpr uint32_t kOzBBytes = kOzSlices * kOzBSlice;      // 64 KB
constexpr size_t kOzSmem = 1024 + kOzABytes + kOzBBytes;   // + alignment slack
constexpr uint32_t kOzTmemCols = kOzSlices * kOzN;         // 512: one accumulator per diagonal
constexpr long long kOzSpinLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row groups 1024 bytes
// apart (stride byte offset), descriptor version 1, leading byte offset unused (16).
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B (format 1), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzN >> 3) << 17) |
         ((uint32_t)(kOzM >> 4) << 24);
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kOzSpinLimit; it++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void oz_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void oz_bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                             uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void oz_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void oz_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(double lo, double hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn((float)lo), b = __float2bfloat16_rn((float)hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

}  // namespace

// Slices of L21 rows r0 .. r0+127 of supernode s (one row per thread), written at slice
// row oz + r; rows u .. roundup(u, 8) get zero slices.
__global__ void __launch_bounds__(128)
    k_oz_slice(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
               uint8_t* __restrict__ oz, int64_t oz_rows) {
  const int4 tk = tasks[blockIdx.x];
  const SnDev d = sns[tk.x];
  const int n = d.n, m = d.m, u = m - n;
  const int r = tk.y + threadIdx.x;
  if (r >= ((u + 7) & ~7)) return;
  const double* L = reinterpret_cast<const double*>(d.L) + n + r;  // L21[r, k] = L[k * m]
  const bool live = r < u;
  double amax = 0.0;
  if (live)
    for (int k = 0; k < n; k++) amax = fmax(amax, fabs(L[(int64_t)k * m]));
  int e = 0;
  if (amax > 0.0) frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
  const double sc = ldexp(1.0, -e);
  const int64_t row = tk.z + (int64_t)r;
  const size_t stride = (size_t)oz_rows * kOzRowBytes;
  uint8_t* base = oz + (size_t)row * kOzRowBytes;
  for (int c = 0; c < kOzRowBytes / 16; c++) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = 8 * c + j;
      x[j] = (live && k < n) ? L[(int64_t)k * m] * sc : 0.0;
    }
    const uint32_t chunk = (uint32_t)((c ^ (int)(row & 7)) << 4);
#pragma unroll
    for (int p = 0; p < kOzSlices; p++) {
      double s[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const double y = x[j] * 128.0;
        s[j] = rint(y);
        x[j] = y - s[j];  // exact: the fraction of y
      }
      uint4 w;
      w.x = pack_bf16(s[0], s[1]);
      w.y = pack_bf16(s[2], s[3]);
      w.z = pack_bf16(s[4], s[5]);
      w.w = pack_bf16(s[6], s[7]);
      *reinterpret_cast<uint4*>(base + p * stride + chunk) = w;
    }
  }
  reinterpret_cast<int32_t*>(oz + kOzSlices * stride)[row] = e;
}

// Eight accumulator columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void oz_tmem_load8(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// An FP32 value holding an integer of magnitude below 2^22, as that integer: adding
// 1.5 * 2^23 puts it in the low mantissa bits.
__device__ __forceinline__ int32_t oz_int(uint32_t f) {
  return __float_as_int(__uint_as_float(f) + 12582912.0f) - 0x4B400000;
}

// 2^e as a double (e in the normal range; others through ldexp).
__device__ __forceinline__ double oz_pow2(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52)
                                   : ldexp(1.0, e);
}

constexpr int kOzMaxRuns = 16;  // column targets per task whose relative rows are cached

template <bool OWNER>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_schur_oz(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
               const SnDev* __restrict__ sns, const MatDev* __restrict__ mats,
               const uint8_t* __restrict__ oz, int64_t oz_rows) {
  extern __shared__ __align__(1024) unsigned char oz_sm[];
  unsigned char* A =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz_sm) + 1023) & ~uintptr_t(1023));
  unsigned char* B = A + kOzABytes;
  __shared__ __align__(8) uint64_t bar_ld, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int s_eA[kOzM], s_eB[2 * kOzN];
  __shared__ int s_tcol[2 * kOzN], s_run[2 * kOzN], s_col[2 * kOzN];
  __shared__ int s_run_start[2 * kOzN + 1];
  __shared__ double* s_rL[kOzMaxRuns];
  __shared__ int s_rm[kOzMaxRuns];
  __shared__ int s_rp[kOzMaxRuns][kOzM];
  __shared__ int s_nruns, s_next, s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bld = smem_u32(&bar_ld), bmma = smem_u32(&bar_mma);
  const size_t stride = (size_t)oz_rows * kOzRowBytes;
  const int32_t* exps = reinterpret_cast<const int32_t*>(oz + kOzSlices * stride);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kOzTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bld));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bmma));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = oz_idesc();
  const uint64_t da0 = oz_desc(smem_u32(A)), db0 = oz_desc(smem_u32(B));
  uint32_t ld_phase = 0, mma_phase = 0;  // parity of the next phase of each barrier
  // thread 0: copies / MMAs issued but not yet observed complete, and their phase parity
  bool ld_inflight = false, mma_inflight = false;
  uint32_t ld_parity = 0, mma_parity = 0;

  // thread 0: bulk copies of a task's A slices and of one half's B slices
  auto issue_loads = [&](const int4& t, int h, bool with_a) {
    const uint32_t bytes = (with_a ? kOzABytes : 0u) + kOzBBytes;
    oz_expect(bld, bytes);
    if (with_a)
      for (int p = 0; p < kOzSlices; p++)
        oz_bulk_load(smem_u32(A + p * kOzASlice),
                     oz + p * stride + (size_t)(t.w + t.y) * kOzRowBytes, kOzASlice, bld);
    for (int p = 0; p < kOzSlices; p++)
      oz_bulk_load(smem_u32(B + p * kOzBSlice),
                   oz + p * stride + (size_t)(t.w + t.z + kOzN * h) * kOzRowBytes, kOzBSlice,
                   bld);
    ld_inflight = true;
    ld_parity = ld_phase;
  };
  // thread 0: D_{p+q} (+)= S_p S_q^T for every slice pair p + q < kOzSlices; a K step of
  // 16 bf16 advances both descriptors by 32 bytes (2 in the address field)
  auto issue_mmas = [&](int ksteps) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    for (int p = 0; p < kOzSlices; p++)
      for (int q = 0; p + q < kOzSlices; q++)
        for (int ks = 0; ks < ksteps; ks++)
          oz_mma(tmem + (uint32_t)((p + q) * kOzN),
                 da0 + (uint64_t)((p * kOzASlice) >> 4) + 2 * ks,
                 db0 + (uint64_t)((q * kOzBSlice) >> 4) + 2 * ks, idesc,
                 (p > 0 || ks > 0) ? 1u : 0u);
    oz_commit(bmma);
    mma_inflight = true;
    mma_parity = mma_phase;
  };

  int tq = blockIdx.x;
  if (tid == 0 && tq < ntasks) issue_loads(tasks[tq], 0, true);
  while (tq < ntasks) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, u = d.m - n;
    const int i0 = tk.y, k0 = tk.z;
    const int ksteps = (n + 15) >> 4;
    const int nh = (k0 + kOzN < u) ? 2 : 1;
    const int32_t* rows = d.rows + n;
    const MatDev md = mats[d.mat];
    // this task's exponents and column targets (the previous task's epilogue is done)
    for (int i = tid; i < kOzM; i += kOzThreads) s_eA[i] = (i0 + i < u) ? exps[tk.w + i0 + i] : 0;
    for (int kk = tid; kk < 2 * kOzN; kk += kOzThreads) {
      const int gk = k0 + kk;
      s_eB[kk] = gk < u ? exps[tk.w + gk] : 0;
      s_tcol[kk] = gk < u ? md.col2sn[rows[gk]] : -1;
    }
    if (tid == 0) s_next = gridDim.x >= ntasks ? ntasks : gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    // thread 0: the MMAs of the first half as soon as its operands are in
    if (tid == 0) {
      if (!oz_wait(bld, ld_phase)) s_fail = 1;
      else {
        ld_inflight = false;
        issue_mmas(ksteps);
      }
    }
    ld_phase ^= 1;
    if (!OWNER) {
      // runs of tile columns with one target (first warp, ballots), then the relative rows
      // of the tile rows inside the first kOzMaxRuns targets, while the tensor cores work
      if (warp == 0) {
        int nr = 0;
        for (int base = 0; base < 2 * kOzN; base += 32) {
          const int kk = base + lane;
          const bool live = k0 + kk < u;
          const bool start = live && (kk == 0 || s_tcol[kk] != s_tcol[kk - 1]);
          const unsigned b = __ballot_sync(0xffffffffu, start);
          if (start) s_run_start[nr + __popc(b & ((1u << lane) - 1u))] = kk;
          nr += __popc(b);
        }
        __syncwarp();
        if (lane == 0) s_nruns = nr;
        for (int r = lane; r < nr; r += 32) {
          const int kb = s_run_start[r];
          const int ke = r + 1 < nr ? s_run_start[r + 1] : min(2 * kOzN, u - k0);
          const SnDev& td = sns[md.sn_base + s_tcol[kb]];
          if (r < kOzMaxRuns) {
            s_rL[r] = reinterpret_cast<double*>(td.L);
            s_rm[r] = td.m;
          }
          for (int kk = kb; kk < ke; kk++) {
            s_run[kk] = r;
            s_col[kk] = rows[k0 + kk] - td.col0;
          }
        }
      }
      __syncthreads();
      const int nrc = min(s_nruns, kOzMaxRuns);
      for (int idx = tid; idx < nrc * kOzM; idx += kOzThreads) {
        const int r = idx / kOzM, i = idx - r * kOzM, gi = i0 + i;
        int p = -1;
        if (gi < u && gi >= k0 + s_run_start[r]) {
          const SnDev& td = sns[md.sn_base + s_tcol[s_run_start[r]]];
          const int key = rows[gi];
          p = (key - td.col0 < td.n) ? key - td.col0 : relative_row(md, td.rows, td.m, key);
        }
        s_rp[r][i] = p;
      }
    }
    const int next = s_next;
    const int i = 32 * (warp & 3) + lane;  // this thread's tile row
    const int gi = i0 + i;
    const int eA = s_eA[i];
    const int c0 = 16 * (warp >> 2);       // this thread's 16 columns of a half
    for (int h = 0; h < nh; h++) {
      if (!oz_wait(bmma, mma_phase)) s_fail = 1;
      else if (tid == 0) mma_inflight = false;
      mma_phase ^= 1;
      __syncthreads();
      if (s_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      // shared memory is free: start the next operands while this half is applied
      if (tid == 0) {
        if (h + 1 < nh) issue_loads(tk, h + 1, false);
        else if (next < ntasks) issue_loads(tasks[next], 0, true);
      }
      // accumulators -> integers -> W = V_hi 2^20 + round(V_lo / 2^8), where
      // V_hi = sum_{d<4} D_d 2^(7(3-d)), V_lo = sum_{d>=4} D_d 2^(7(7-d)) (|D_d| < 2^22,
      // |V_hi| < 2^42, |V_lo| < 2^44), so U = W 2^(e_i + e_k - 55)
      double val[16];
#pragma unroll
      for (int cc = 0; cc < 2; cc++) {
        long long vh[8], vl[8];
#pragma unroll
        for (int j = 0; j < 8; j++) vh[j] = vl[j] = 0;
        const uint32_t ta =
            tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 8 * cc);
#pragma unroll
        for (int dd = 0; dd < kOzSlices; dd++) {
          uint32_t v[8];
          oz_tmem_load8(ta + (uint32_t)(dd * kOzN), v);
#pragma unroll
          for (int j = 0; j < 8; j++) {
            if (dd < 4) vh[j] = vh[j] * 128 + oz_int(v[j]);
            else vl[j] = vl[j] * 128 + oz_int(v[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const long long w = vh[j] * (1ll << 20) + ((vl[j] + 128) >> 8);
          val[8 * cc + j] = (double)w * oz_pow2(eA + s_eB[h * kOzN + c0 + 8 * cc + j] - 55);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      // tensor memory is free: the second half's MMAs run during this half's scatter
      if (h + 1 < nh) {
        if (tid == 0) {
          if (!oz_wait(bld, ld_phase)) s_fail = 1;
          else {
            ld_inflight = false;
            issue_mmas(ksteps);
          }
        }
        ld_phase ^= 1;  // every thread counts the second half's load
      }
      // scatter this thread's row of the half
      if (gi < u) {
        const int kb = h * kOzN + c0;  // tile column of val[0]
        if (OWNER) {
          double* U = static_cast<double*>(md.stage) + d.ustage;
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int gk = k0 + kb + j;
            if (gk < u && gk <= gi) U[(int64_t)gk * u + gi] = val[j];
          }
        } else {
          const int key = rows[gi];
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int kk = kb + j, gk = k0 + kk;
            if (gk >= u || gk > gi) continue;
            const int r = s_run[kk];
            double* Lt;
            int mt, p;
            if (r < kOzMaxRuns) {
              Lt = s_rL[r];
              mt = s_rm[r];
              p = s_rp[r][i];
            } else {  // beyond the cached targets: look the row up here
              const SnDev& td = sns[md.sn_base + s_tcol[kk]];
              Lt = reinterpret_cast<double*>(td.L);
              mt = td.m;
              p = (key - td.col0 < td.n) ? key - td.col0 : relative_row(md, td.rows, td.m, key);
            }
            if (p >= 0) atomicAdd(&Lt[(int64_t)s_col[kk] * mt + p], -val[j]);
          }
        }
      }
    }
    __syncthreads();
    if (s_fail) {
      if (tid == 0) atomicAdd(md.err + 3, 1ull);
      break;
    }
    tq = next;
  }
  // bounded waits for anything still in flight before the memory is released
  if (tid == 0) {
    if (mma_inflight) oz_wait(bmma, mma_parity);
    if (ld_inflight) oz_wait(bld, ld_parity);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOzTmemCols));
}

void launch_oz_slice(const int4* tasks, int ntasks, const SnDev* sns, void* oz, int64_t oz_rows,
                     cudaStream_t st) {
  if (ntasks <= 0) return;
  k_oz_slice<<<ntasks, 128, 0, st>>>(tasks, sns, static_cast<uint8_t*>(oz), oz_rows);
}

void launch_schur_oz(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                     const MatDev* mats, bool owner, const void* oz, int64_t oz_rows,
                     cudaStream_t st) {
  if (ntasks <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntasks < sms ? ntasks : sms;  // one resident CTA per SM, tasks by queue
  const uint8_t* z = static_cast<const uint8_t*>(oz);
  if (owner)
    k_schur_oz<true><<<grid, kOzThreads, kOzSmem, st>>>(tasks, ntasks, queue, sns, mats, z, oz_rows);
  else
    k_schur_oz<false><<<grid, kOzThreads, kOzSmem, st>>>(tasks, ntasks, queue, sns, mats, z, oz_rows);
}

size_t oz_scratch_bytes(int64_t oz_rows) {
  return (size_t)oz_rows * (kOzSlices * kOzRowBytes + sizeof(int32_t));
}

int set_oz_kernel_attrs() {
  if (cudaFuncSetAttribute(k_schur_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kOzSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kOzSmem) != cudaSuccess)
    return CHOL_E_CUDA;
  return CHOL_OK;
}

}  // namespace chol
