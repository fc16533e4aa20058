// tc_kernels.cu -- Schur update tiles of the mixed-precision factor on the fifth-generation
// tensor cores (tcgen05) of sm_103a: TF32 products accumulated in FP32.
//
// A task {s, i0, k0, oz} is the 128 x 128 tile U_s[i0.., k0..] = L21[i0.., :] L21[k0.., :]^T
// of a supernode's Schur update (the SYRK/GEMM of Sec. 3, Listing 1) on FP32 panels, with
// the 3xTF32 split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = tf32(a),
// a_lo = tf32(a - a_hi)), which keeps FP32-level accuracy.  Two kernels per level:
//   k_tf32_split  the hi and lo parts of every L21 row of the level's 128-tile supernodes,
//                 in planes (part, 32-column chunk) of 128-byte rows whose 16-byte pieces
//                 are pre-swizzled for the tensor cores' 128-byte swizzle;
//   k_schur_tf32  a persistent CTA per SM.  A load thread (its own warp) claims the tasks,
//                 hands each to the other roles through a ring and streams its operand
//                 chunks (A hi/lo, B hi/lo: 64 KB) into a 3-stage shared memory ring with
//                 bulk copies; an MMA thread (its own warp) issues, chunk by chunk in ring
//                 order, the MMAs (M = N = 128, three per K step of 8) into one of four
//                 128-column tensor-memory accumulators; four metadata warps build each
//                 task's column targets and relative rows ahead of use, into one of three
//                 buffers; 16 consumer warps read finished accumulators (tcgen05.ld, one row
//                 per thread) and add them into the ancestors with FP32 reductions (or write
//                 the owner staging buffer).  Loads, MMAs, metadata and the scatter of
//                 different tasks overlap through mbarriers: stage full/empty, accumulator
//                 full/empty, metadata full/empty, and the ring of the task sequence.
// Every wait is bounded in time (kTfWaitCycles SM clock cycles, about a second): then the
// thread records a timeout in err[3]
// and stops; its partners then time out as well, waits for copies and MMAs in flight are
// bounded too, and the tensor memory is freed before the kernel returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "chol_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "launch_util.h"

namespace chol {

namespace {

constexpr int kTfM = 128;                          // tile edge (UMMA M = N = 128)
constexpr int kTfChunk = 32;                       // K columns per chunk: 128 B of FP32
constexpr uint32_t kTfPlane = kTfM * kOzRowBytes;  // 16 KB: 128 rows of one (part, chunk)
constexpr int kTfStages = 3;
constexpr uint32_t kTfStageBytes = 4 * kTfPlane;   // A hi, A lo, B hi, B lo of one chunk
constexpr size_t kTfSmem = 1024 + kTfStages * kTfStageBytes;
constexpr int kTfSlots = 4;                        // accumulators of 128 TMEM columns
constexpr int kTfConsumers = 512;                  // 16 warps: drain + scatter
constexpr int kTfMetaThreads = 128;                // 4 warps: per-task column metadata
constexpr int kTfMmaWarp = kTfConsumers / 32;       // issues the MMAs (one thread)
constexpr int kTfLoadWarp = kTfMmaWarp + 1;         // claims tasks, issues the copies (one thread)
constexpr int kTfMetaBase = kTfConsumers + 64;      // first metadata thread
constexpr int kTfThreads = kTfMetaBase + kTfMetaThreads;
constexpr int kTfRing = 16;
constexpr int kTfMaxRuns = 8;   // column targets per task whose relative rows are cached
constexpr int kTfMetaBufs = 3;  // metadata buffers: the metadata warps run up to two tasks ahead
// Bound of every wait in SM clock cycles (~1 s at 2 GHz), counted with clock64(): a poll of
// mbarrier.try_wait may suspend the thread for a hardware-defined time.
constexpr long long kTfWaitCycles = 1ll << 31;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row groups 1024 bytes
// apart, descriptor version 1, leading byte offset unused (16).
__device__ __forceinline__ uint64_t tf_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B (format 2), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t tf_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTfM >> 3) << 17) |
         ((uint32_t)(kTfM >> 4) << 24);
}

__device__ __forceinline__ bool tf_wait(uint32_t bar, uint32_t parity,
                                        long long limit = kTfWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tf_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tf_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tf_bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                             uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tf_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tf_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 accumulator columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tf_tmem_load32(uint32_t addr, uint32_t (&r)[32]) {
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

// barrier among the metadata warps only
__device__ __forceinline__ void meta_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kTfMetaThreads) : "memory");
}

static_assert(kTfM == 128, "the run count sums four 32-column words");
struct TfMeta {
  float* cp[kTfM];  // each column's target panel column (its relative rows are added)
  int tcol[kTfM], run[kTfM];
  int run_start[kTfM + 1];
  int wcnt[kTfM / 32];  // run starts per 32 columns
  int fcnt[kTfMetaThreads / 32];  // the supernode's runs before the tile, per warp
  long long rb[kTfM];   // relative-map base of every run
  int rp[kTfMaxRuns][kTfM];
  int nruns;
  int u, i0, k0;                 // the task: update order, tile origin
  const int32_t* relmap;         // for runs beyond the cached ones
  float* ustage;                 // owner assembly: this supernode's staged U
};

}  // namespace

// hi and lo TF32 parts of the L21 rows r0 .. r0+127 of supernode s at slice rows oz + r:
// plane (part p, chunk c) at oz + (4 p + c) oz_rows 128 B, 16-byte piece q of a row (its
// columns 32 c + 4 q .. +3) stored at piece q ^ (row & 7).  Rows u .. roundup(u, 8) and
// columns n .. are zero.
__global__ void __launch_bounds__(256)
    k_tf32_split(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
                 uint8_t* __restrict__ oz, int64_t oz_rows) {
  extern __shared__ __align__(16) float xf[];  // [n][kTfM]
  const int4 tk = tasks[blockIdx.x];
  const SnDev d = sns[tk.x];
  const int n = d.n, m = d.m, u = m - n;
  const int r0 = tk.y;
  const int rows = min(kTfM, ((u + 7) & ~7) - r0);
  const int nch = (n + kTfChunk - 1) / kTfChunk;
  const float* L = reinterpret_cast<const float*>(d.L) + n + r0;
  stage_row_block(xf, kTfM, L, m, n, u - r0);
  cp_async_wait_all();
  __syncthreads();
  const int64_t row0 = tk.z + (int64_t)r0;
  const size_t stride = (size_t)oz_rows * kOzRowBytes;
  for (int item = threadIdx.x; item < kTfM * 8 * nch; item += blockDim.x) {
    const int c = item / (kTfM * 8), rest = item - c * (kTfM * 8);
    const int i = rest >> 3, pc = rest & 7;  // row, physical 16-byte piece
    if (i >= rows) continue;
    const int q = pc ^ (int)((row0 + i) & 7);
    float hi[4], lo[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int k = kTfChunk * c + 4 * q + j;
      const float x = k < n ? xf[k * kTfM + i] : 0.f;
      hi[j] = to_tf32(x);
      lo[j] = to_tf32(x - hi[j]);
    }
    uint8_t* dst = oz + (size_t)(row0 + i) * kOzRowBytes + pc * 16;
    *reinterpret_cast<float4*>(dst + (size_t)c * stride) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<float4*>(dst + (size_t)(4 + c) * stride) =
        make_float4(lo[0], lo[1], lo[2], lo[3]);
  }
}

template <bool OWNER>
__global__ void __launch_bounds__(kTfThreads, 1)
    k_schur_tf32(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
                 const SnDev* __restrict__ sns, const MatDev* __restrict__ mats,
                 const uint8_t* __restrict__ oz, int64_t oz_rows, long long acc_wait) {
  extern __shared__ __align__(1024) unsigned char tf_sm[];
  unsigned char* stage_base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tf_sm) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t st_full[kTfStages], st_empty[kTfStages];
  __shared__ __align__(8) uint64_t acc_full[kTfSlots], acc_empty[kTfSlots];
  __shared__ __align__(8) uint64_t ring_full[kTfRing];
  __shared__ int ring[kTfRing];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t meta_full[kTfMetaBufs], meta_empty[kTfMetaBufs];
  __shared__ TfMeta meta[kTfMetaBufs];
  __shared__ int s_mtq;  // the metadata warps' next task (or ntasks: stop)
  __shared__ int s_fail;
  __shared__ __align__(8) uint64_t never;  // test hook: a barrier nothing completes
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // a launch of an earlier level of this factorization already gave up on a wait: its
  // updates are missing and the factorization is reported failed, so skip the work (before
  // any barrier or tensor memory is set up); every thread reads the same word
  if (ntasks > 0 && *(volatile unsigned long long*)(mats[sns[tasks[0].x].mat].err + 3) != 0) return;
  const size_t stride = (size_t)oz_rows * kOzRowBytes;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTfSlots * kTfM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < kTfStages; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&st_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&st_empty[i])));
    }
    for (int i = 0; i < kTfSlots; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[i])),
                   "r"(kTfConsumers / 32));
    }
    for (int i = 0; i < kTfRing; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ring_full[i])));
    for (int i = 0; i < kTfMetaBufs; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&meta_full[i])),
                   "r"(kTfMetaThreads));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&meta_empty[i])),
                   "r"(kTfConsumers / 32));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&never)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == kTfLoadWarp) {
    // ---------------- loads: task claims, ring, bulk copies; one thread ----------------
    if (lane == 0) {
      long long item = 0;  // chunk loads issued (stage = item % kTfStages)
      int ord = 0;         // ring entries published
      bool ok = true;
      int tq = blockIdx.x;  // a CTA's first task is its block index
      for (;;) {
        ring[ord % kTfRing] = tq < ntasks ? tq : ntasks;  // the task order, at claim time
        tf_arrive(smem_u32(&ring_full[ord % kTfRing]));
        ord++;
        if (tq >= ntasks) break;
        const int4 t = tasks[tq];
        const int nch = (sns[t.x].n + kTfChunk - 1) / kTfChunk;
        const uint8_t* arow = oz + (size_t)(t.w + t.y) * kOzRowBytes;
        const uint8_t* brow = oz + (size_t)(t.w + t.z) * kOzRowBytes;
        for (int c = 0; c < nch && ok; c++, item++) {
          const int s = (int)(item % kTfStages);
          if (item >= kTfStages &&  // the stage's previous MMAs must have read it
              !tf_wait(smem_u32(&st_empty[s]), (uint32_t)(((item / kTfStages) - 1) & 1))) {
            ok = false;
            break;
          }
          unsigned char* sb = stage_base + (size_t)s * kTfStageBytes;
          const uint32_t bar = smem_u32(&st_full[s]);
          tf_expect(bar, kTfStageBytes);
          tf_bulk_load(smem_u32(sb), arow + (size_t)c * stride, kTfPlane, bar);
          tf_bulk_load(smem_u32(sb + kTfPlane), arow + (size_t)(4 + c) * stride, kTfPlane, bar);
          tf_bulk_load(smem_u32(sb + 2 * kTfPlane), brow + (size_t)c * stride, kTfPlane, bar);
          tf_bulk_load(smem_u32(sb + 3 * kTfPlane), brow + (size_t)(4 + c) * stride, kTfPlane,
                       bar);
        }
        if (!ok) break;
        tq = gridDim.x >= ntasks ? ntasks : (int)gridDim.x + atomicAdd(queue, 1);
      }
      if (!ok) {
        s_fail = 1;
        // the other roles stop at their next ring wait on an end marker
        ring[ord % kTfRing] = ntasks;
        tf_arrive(smem_u32(&ring_full[ord % kTfRing]));
      }
      // bounded waits for the copies still in flight: the last one of each stage
      for (long long q = item - kTfStages < 0 ? 0 : item - kTfStages; q < item; q++)
        tf_wait(smem_u32(&st_full[q % kTfStages]), (uint32_t)((q / kTfStages) & 1));
    }
  } else if (warp == kTfMmaWarp) {
    // ---------------- MMAs, one thread, in ring order ----------------
    if (lane == 0) {
      const uint32_t idesc = tf_idesc();
      long long done = 0;  // chunks whose MMAs are issued (stage = done % kTfStages)
      bool ok = true;
      for (int ord = 0; ok; ord++) {
        if (!tf_wait(smem_u32(&ring_full[ord % kTfRing]), (uint32_t)((ord / kTfRing) & 1))) {
          ok = false;
          break;
        }
        const int tq = ring[ord % kTfRing];
        if (tq >= ntasks) break;
        const int n = sns[tasks[tq].x].n;
        const int nch = (n + kTfChunk - 1) / kTfChunk;
        const int acc = ord % kTfSlots;
        for (int c = 0; c < nch; c++, done++) {
          const int s = (int)(done % kTfStages);
          if (!tf_wait(smem_u32(&st_full[s]), (uint32_t)((done / kTfStages) & 1)) ||
              (c == 0 && ord >= kTfSlots &&  // wait for the drain of the slot
               !tf_wait(smem_u32(&acc_empty[acc]), (uint32_t)(((ord / kTfSlots) - 1) & 1)))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int kw = min(kTfChunk, n - kTfChunk * c);
          const uint32_t sa = smem_u32(stage_base + (size_t)s * kTfStageBytes);
          const uint64_t ahi = tf_desc(sa), alo = tf_desc(sa + kTfPlane);
          const uint64_t bhi = tf_desc(sa + 2 * kTfPlane), blo = tf_desc(sa + 3 * kTfPlane);
          const uint32_t dt = tmem + (uint32_t)(acc * kTfM);
          for (int kk = 0; kk < (kw + 7) / 8; kk++) {  // K steps of 8 TF32 = 32 bytes
            tf_mma(dt, ahi + 2 * kk, bhi + 2 * kk, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            tf_mma(dt, ahi + 2 * kk, blo + 2 * kk, idesc, 1u);
            tf_mma(dt, alo + 2 * kk, bhi + 2 * kk, idesc, 1u);
          }
          tf_commit(smem_u32(&st_empty[s]));  // the stage is free once these MMAs are done
          if (c + 1 == nch) tf_commit(smem_u32(&acc_full[acc]));
        }
      }
      if (!ok) s_fail = 1;
      // bounded wait for the MMAs in flight (the last commit covers all earlier ones)
      if (done > 0)
        tf_wait(smem_u32(&st_empty[(done - 1) % kTfStages]), (uint32_t)(((done - 1) / kTfStages) & 1));
    }
  } else if (warp >= kTfMetaBase / 32) {
    // ---------------- metadata warps: one thread per tile column ----------------
    // For each task in ring order, into meta[ord % kTfMetaBufs] once the consumers have released it:
    // every column's target supernode, the runs of equal target (ballot per 32 columns), each
    // column's run and column inside its target, per run the relative-map base and target
    // panel, and the relative rows of the first kTfMaxRuns runs.  Thread 0 alone waits on
    // the ring and on the buffer, so that the group's decisions are uniform.
    const int mt = tid - kTfMetaBase, mwarp = mt >> 5;
    for (int ord = 0;; ord++) {
      const int buf = ord % kTfMetaBufs;
      if (mt == 0) {
        const int rs = ord % kTfRing;
        int tq = ntasks;
        if (!tf_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kTfRing) & 1)) ||
            (ring[rs] < ntasks && ord >= kTfMetaBufs &&
             !tf_wait(smem_u32(&meta_empty[buf]), (uint32_t)((ord / kTfMetaBufs - 1) & 1))))
          s_fail = 1;
        else
          tq = ring[rs];
        s_mtq = tq;
      }
      meta_sync();
      const int tq = s_mtq;
      meta_sync();  // s_mtq is rewritten only after every thread has read it
      if (tq >= ntasks) break;
      TfMeta& M = meta[buf];
      const int4 tk = tasks[tq];
      const SnDev d = sns[tk.x];
      const int n = d.n, u = d.m - n, i0 = tk.y, k0 = tk.z;
      const MatDev md = mats[d.mat];
      if (mt == 0) {
        M.u = u;
        M.i0 = i0;
        M.k0 = k0;
        M.relmap = md.relmap;
        M.ustage = OWNER ? static_cast<float*>(md.stage) + d.ustage : nullptr;
      }
      if (!OWNER) {
        const int32_t* rows = d.rows + n;
        const int gk = k0 + mt;
        const int grow = gk < u ? rows[gk] : 0;
        const int tc = gk < u ? md.col2sn[grow] : -1;
        M.tcol[mt] = tc;
        // the supernode's runs that start after position 0 and at or before k0: their count
        // is the index (from run0) of the run holding the tile's first column; the tile's
        // runs are that run and the ones after it, in order (runs split where the target
        // changes, and so do the tile's)
        int before = 0;
        for (int t = 1 + mt; t < d.nrun; t += kTfMetaThreads) before += md.run_a[d.run0 + t] <= k0 ? 1 : 0;
        before = __reduce_add_sync(0xffffffffu, before);
        if (lane == 0) M.fcnt[mwarp] = before;
        meta_sync();
        // a column starts a run when its target differs from its left neighbour's; its run
        // index is the number of starts up to it, less one
        const bool start = gk < u && (mt == 0 || M.tcol[mt - 1] != tc);
        const unsigned bl = __ballot_sync(0xffffffffu, start);
        if (lane == 0) M.wcnt[mwarp] = __popc(bl);
        meta_sync();
        int off = 0;
        for (int w2 = 0; w2 < mwarp; w2++) off += M.wcnt[w2];
        const int first = d.run0 + M.fcnt[0] + M.fcnt[1] + M.fcnt[2] + M.fcnt[3];
        if (gk < u) {
          const int r = off + __popc(bl & ((2u << lane) - 1u)) - 1;
          const SnDev& td = sns[md.sn_base + tc];
          M.run[mt] = r;
          M.cp[mt] = reinterpret_cast<float*>(td.L) + (int64_t)(grow - td.col0) * td.m;
          if (start) {  // the run's first column fetches its map base
            M.run_start[r] = mt;
            M.rb[r] = md.run_base[first + r];
          }
        }
        if (mt == 0) M.nruns = M.wcnt[0] + M.wcnt[1] + M.wcnt[2] + M.wcnt[3];
        meta_sync();
        // relative rows of the cached runs: this thread's tile row in each, all loads in flight
        static_assert(kTfMetaThreads == kTfM, "one metadata thread per tile row");
        const int nrc = min(M.nruns, kTfMaxRuns), gi = i0 + mt;
        int rpv[kTfMaxRuns];
#pragma unroll
        for (int r = 0; r < kTfMaxRuns; r++)
          rpv[r] = (r < nrc && gi < u && gi >= k0 + M.run_start[r]) ? md.relmap[M.rb[r] + gi] : -1;
#pragma unroll
        for (int r = 0; r < kTfMaxRuns; r++)
          if (r < nrc) M.rp[r][mt] = rpv[r];
      }
      tf_arrive(smem_u32(&meta_full[buf]));  // each thread after its own writes
    }
  } else {
    // ---------------- consumers: accumulator drain and scatter ----------------
    // Each wait's outcome is made uniform over the warp (tcgen05.ld is warp-collective).
    for (int ord = 0;; ord++) {
      const int rs = ord % kTfRing, buf = ord % kTfMetaBufs;
      if (!__all_sync(0xffffffffu, tf_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kTfRing) & 1)))) {
        s_fail = 1;
        break;
      }
      if (ring[rs] >= ntasks) break;
      const TfMeta& M = meta[buf];
      const int acc = ord % kTfSlots;
      if (!__all_sync(0xffffffffu, tf_wait(smem_u32(&meta_full[buf]), (uint32_t)((ord / kTfMetaBufs) & 1)) &&
                                       (acc_wait > 0  // test hook: a barrier never completed
                                            ? tf_wait(smem_u32(&never), 0u, acc_wait)
                                            : tf_wait(smem_u32(&acc_full[acc]),
                                                      (uint32_t)((ord / kTfSlots) & 1))))) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int u = M.u, i0 = M.i0, k0 = M.k0;
      const int i = 32 * (warp & 3) + lane;  // this thread's tile row
      const int c0 = 32 * (warp >> 2);       // and its 32 columns
      uint32_t v[32];
      tf_tmem_load32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(acc * kTfM + c0), v);
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) tf_arrive(smem_u32(&acc_empty[acc]));
      const int gi = i0 + i;
      if (gi < u) {
        if (OWNER) {
          float* U = M.ustage;
#pragma unroll
          for (int j = 0; j < 32; j++) {
            const int gk = k0 + c0 + j;
            if (gk < u && gk <= gi) U[(int64_t)gk * u + gi] = __uint_as_float(v[j]);
          }
        } else {
          // the relative row changes only with the run, which is the same for every lane
          int rprev = -1, p = -1;
#pragma unroll
          for (int j = 0; j < 32; j++) {
            const int kk = c0 + j, gk = k0 + kk;
            if (gk >= u || gk > gi) continue;
            const int r = M.run[kk];
            if (r != rprev) {
              rprev = r;
              p = r < kTfMaxRuns ? M.rp[r][i] : M.relmap[M.rb[r] + gi];
            }
            if (p >= 0) red_add(M.cp[kk] + p, -__uint_as_float(v[j]));
          }
        }
      }
      __syncwarp();
      if (lane == 0) tf_arrive(smem_u32(&meta_empty[buf]));
    }
  }
  __syncthreads();
  if (s_fail && tid == 0 && ntasks > 0) atomicAdd(mats[sns[tasks[0].x].mat].err + 3, 1ull);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTfSlots * kTfM));
}

void launch_tf32_split(const int4* tasks, int ntasks, const SnDev* sns, int max_width, void* oz,
                       int64_t oz_rows, cudaStream_t st) {
  if (ntasks <= 0) return;
  k_tf32_split<<<ntasks, 256, (size_t)max_width * kTfM * sizeof(float), st>>>(
      tasks, sns, static_cast<uint8_t*>(oz), oz_rows);
}

void launch_schur_tc(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                     const MatDev* mats, bool owner, const void* oz, int64_t oz_rows,
                     long long acc_wait, cudaStream_t st) {
  if (ntasks <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntasks < sms ? ntasks : sms;  // one resident CTA per SM, tasks by queue
  const uint8_t* z = static_cast<const uint8_t*>(oz);
  if (owner)
    k_schur_tf32<true><<<grid, kTfThreads, kTfSmem, st>>>(tasks, ntasks, queue, sns, mats, z,
                                                         oz_rows, acc_wait);
  else
    k_schur_tf32<false><<<grid, kTfThreads, kTfSmem, st>>>(tasks, ntasks, queue, sns, mats, z,
                                                          oz_rows, acc_wait);
}

int set_tc_kernel_attrs() {
  if (cudaFuncSetAttribute(k_schur_tf32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTfSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_tf32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTfSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tf32_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kMaxWidth * kTfM * sizeof(float))) != cudaSuccess)
    return CHOL_E_CUDA;
  return CHOL_OK;
}

}  // namespace chol
