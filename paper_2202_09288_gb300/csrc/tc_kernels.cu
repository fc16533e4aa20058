// tc_kernels.cu -- Schur update tiles of the mixed-precision factor on the fifth-generation
// tensor cores (tcgen05) of sm_103a.
//
// A task {s, i0, k0, 128} is the 128 x 128 tile U_s[i0.., k0..] = L21[i0.., :] L21[k0.., :]^T
// of a supernode's Schur update (the SYRK/GEMM of Sec. 3, Listing 1).  L21 is FP32 and the
// tile is accumulated in FP32 in tensor memory by tcgen05.mma kind::tf32 with the 3xTF32
// split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = tf32(a), a_lo = tf32(a - a_hi)),
// which keeps FP32-level accuracy.  Per K chunk of 32 columns, the CTA's threads stage the
// four operand tiles (A hi/lo, B hi/lo; 16 KB each) into shared memory in the 128-byte-
// swizzled K-major layout, one thread issues the MMAs and commits them to an mbarrier, and
// the CTA waits for it (bounded).  The finished tile is read from tensor memory with
// tcgen05.ld into shared memory and applied by the common Schur epilogue.
//
// Every wait is bounded: after kTcSpinLimit polls the kernel records a timeout in err[3],
// waits once more (bounded) for its MMAs in flight, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "chol_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.h"

namespace chol {

namespace {

constexpr int kTc = 128;             // tile edge: UMMA M = N = 128, cta_group::1
constexpr int kTcK = 32;             // K columns staged per chunk (128 bytes of FP32 per row)
constexpr int kTcThreads = 128;
constexpr uint32_t kTcOperandBytes = kTc * kTcK * 4;             // 16 KB
constexpr uint32_t kTcCsBytes = kTc * (kTc + 1) * 4;              // epilogue tile
constexpr uint32_t kTcBody = 4 * kTcOperandBytes > kTcCsBytes ? 4 * kTcOperandBytes : kTcCsBytes;
constexpr size_t kTcSmem = 1024 + kTcBody;                        // + alignment slack
constexpr long long kTcSpinLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row r, column k) of a 128 x 32 FP32 operand tile in the K-major
// layout with 128-byte swizzle: rows are 128 bytes, 8-row groups 1024 bytes apart, and the
// 16-byte chunk index within a row is XORed with the row index modulo 8.
__device__ __forceinline__ uint32_t swz(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) +
                    (k & 3) * 4);
}

// Shared-memory matrix descriptor: start address, leading byte offset (unused by swizzled
// K-major layouts), stride byte offset 1024 between 8-row groups, descriptor version 1,
// swizzle mode 128B.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTc >> 3) << 17) |
         ((uint32_t)(kTc >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kTcSpinLimit; it++) {
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

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_load32(uint32_t addr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

template <bool OWNER>
__global__ void __launch_bounds__(kTcThreads)
    k_schur_tc(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
               const SnDev* __restrict__ sns, const MatDev* __restrict__ mats) {
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_sm) + 1023) & ~uintptr_t(1023));
  unsigned char* Ahi = base;
  unsigned char* Alo = base + kTcOperandBytes;
  unsigned char* Bhi = base + 2 * kTcOperandBytes;
  unsigned char* Blo = base + 3 * kTcOperandBytes;
  float* Cs = reinterpret_cast<float*>(base);  // reused once the MMAs of a tile are done
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_next_task;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_tf32();
  uint32_t phase = 0;
  bool inflight = false;  // MMAs committed whose completion was not observed

  for (int tq = blockIdx.x; tq < ntasks;) {
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, m = d.m, u = m - n;
    const int i0 = tk.y, k0 = tk.z;
    const float* L = reinterpret_cast<const float*>(d.L);
    for (int kc = 0; kc < n; kc += kTcK) {
      const int kw = min(kTcK, n - kc);
      for (int idx = tid; idx < kTc * kTcK; idx += kTcThreads) {
        const int r = idx & (kTc - 1), k = idx >> 7;
        float a = 0.f, b = 0.f;
        if (k < kw) {
          const int64_t col = (int64_t)(kc + k) * m + n;
          if (i0 + r < u) a = L[col + i0 + r];
          if (k0 + r < u) b = L[col + k0 + r];
        }
        const float ah = to_tf32(a), bh = to_tf32(b);
        const uint32_t o = swz(r, k);
        *reinterpret_cast<float*>(Ahi + o) = ah;
        *reinterpret_cast<float*>(Alo + o) = to_tf32(a - ah);
        *reinterpret_cast<float*>(Bhi + o) = bh;
        *reinterpret_cast<float*>(Blo + o) = to_tf32(b - bh);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int ksteps = (kw + 7) >> 3;  // K = 8 per tf32 MMA
        for (int kk = 0; kk < ksteps; kk++) {
          const uint64_t ah = smem_desc(smem_u32(Ahi) + kk * 32);
          const uint64_t al = smem_desc(smem_u32(Alo) + kk * 32);
          const uint64_t bh = smem_desc(smem_u32(Bhi) + kk * 32);
          const uint64_t bl = smem_desc(smem_u32(Blo) + kk * 32);
          mma_tf32(tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar)
            : "memory");
      }
      inflight = true;
      if (!mbar_wait(bar, phase)) s_fail = 1;  // benign race: every writer stores 1
      else inflight = false;
      phase ^= 1;
      __syncthreads();
      if (s_fail) {
        if (tid == 0) atomicAdd(mats[d.mat].err + 3, 1ull);
        break;
      }
    }
    if (s_fail) break;
    // accumulator -> shared tile Cs[col * (kTc + 1) + row]
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int cc = 0; cc < kTc / 32; cc++) {
      uint32_t r[32];
      tmem_load32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), r);
#pragma unroll
      for (int j = 0; j < 32; j++) Cs[(cc * 32 + j) * (kTc + 1) + row] = __uint_as_float(r[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    schur_tile_epilogue<float, kTc, kTcThreads, OWNER>(Cs, d, i0, k0, sns, mats,
                                                       static_cast<float*>(mats[d.mat].stage));
    __syncthreads();
    if (gridDim.x >= ntasks) break;
    if (tid == 0) s_next_task = gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    tq = s_next_task;
  }
  if (s_fail && inflight) mbar_wait(bar, phase ^ 1);  // let the MMAs in flight finish (bounded)
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTc));
}

void launch_schur_tc(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                     const MatDev* mats, bool owner, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (owner)
    k_schur_tc<true><<<ntasks, kTcThreads, kTcSmem, st>>>(tasks, ntasks, queue, sns, mats);
  else
    k_schur_tc<false><<<ntasks, kTcThreads, kTcSmem, st>>>(tasks, ntasks, queue, sns, mats);
}

int set_tc_kernel_attrs() {
  if (cudaFuncSetAttribute(k_schur_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTcSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTcSmem) != cudaSuccess)
    return CHOL_E_CUDA;
  return CHOL_OK;
}

}  // namespace chol
