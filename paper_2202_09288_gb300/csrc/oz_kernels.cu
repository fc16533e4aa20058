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
//   k_schur_oz  a 128 x 128 task is done as four 128 x 32 quarters.  The 8 A slices
//               (the task's 128 rows) and each quarter's 8 B slices (its 32 rows) are
//               brought into shared memory by bulk copies issued by a load thread, which
//               also claims the tasks; an MMA thread issues, for every slice pair p + q < 8,
//               the bf16 MMAs of D_{p+q} += S_p S_q^T into the quarter's set of tensor-memory
//               accumulators (one per diagonal p + q, 8 x 32 columns; two sets); tasks are
//               claimed in runs of up to four, so that the later tiles of a row strip reuse
//               the A slices.  Every partial sum of a diagonal is an integer below 2^22
//               (K <= 64), so FP32 accumulation is exact.  Consumer warps read a finished
//               set (lane = tile row), release it, form U[i,k] = 2^(e_i+e_k)
//               sum_d 2^(-7(d+2)) D_d[i,k] as an FP64 value (integer combination, one
//               int64 -> double conversion) and add it into the ancestors with FP64
//               reductions (or write the owner staging buffer) while the tensor cores compute
//               the next quarter; metadata warps prepare the coming tasks' targets ahead.
// Every wait is bounded in time (kOzWaitCycles SM clock cycles, about a second): then the
// kernel records a timeout in err[3],
// waits (bounded) for its copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "chol_internal.h"
#include "device_common.cuh"
#include "kernels.h"
#include "oz_common.cuh"
#include "launch_util.h"

namespace chol {

namespace {

constexpr int kOzConsumers = 512;                          // 16 warps: drain + scatter
constexpr int kOzMetaThreads = 128;                        // 4 warps: per-task metadata
constexpr int kOzMmaWarp = kOzConsumers / 32;              // issues the MMAs (one thread)
constexpr int kOzLoadWarp = kOzMmaWarp + 1;                // issues the bulk copies (one thread)
constexpr int kOzMetaBase = kOzConsumers + 64;             // first metadata thread
constexpr int kOzThreads = kOzMetaBase + kOzMetaThreads;
constexpr int kOzRing = 16;
constexpr int kOzM = 128;                                  // tile rows (UMMA M)
constexpr int kOzN = 64;                                   // columns per half (UMMA N)
constexpr uint32_t kOzASlice = kOzM * kOzRowBytes;         // 16 KB
constexpr int kOzQ = 32;                                   // columns per quarter
constexpr uint32_t kOzQSlice = kOzQ * kOzRowBytes;         // 4 KB: one slice of a quarter
constexpr uint32_t kOzQBytes = kOzSlices * kOzQSlice;      // 32 KB: a quarter's B operand
constexpr int kOzSetCols = kOzSlices * kOzQ;               // 256: TMEM columns of a set
constexpr uint32_t kOzABytes = kOzSlices * kOzASlice;      // 128 KB
constexpr size_t kOzSmem = 1024 + kOzABytes + 2 * kOzQBytes;  // + alignment slack
constexpr uint32_t kOzTmemCols = 2 * kOzSetCols;          // 512: two sets of 8 diagonals
// Bound of every wait in SM clock cycles (~1 s at 2 GHz; the waits of a working launch last
// microseconds).  Counted with clock64(), not in polls: a poll of mbarrier.try_wait may suspend
// the thread for a hardware-defined time.
constexpr long long kOzWaitCycles = 1ll << 31;

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
__device__ __forceinline__ uint32_t oz_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(kOzM >> 4) << 24);
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity,
                                        long long limit = kOzWaitCycles) {
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

}  // namespace

constexpr int kOzSliceThreads = 256;
constexpr int kOzSliceLd = kOzM + 1;  // padded column stride of the staged block

// Slices of the L21 rows r0 .. r0+127 of supernode s, at slice rows oz + r (rows u ..
// roundup(u, 8) get zero slices).  The block is staged column by column through shared
// memory (cp.async, all copies in flight); a row's exponent e_r is that of its largest entry; each
// entry becomes the 56-bit fixed-point integer x 2^(56-e_r), cut into 8 balanced digits
// of 7 bits (round to nearest: |s_0| <= 128, |s_p| <= 64, exact); thread t writes the
// 16-byte chunk t % 8 of row t / 8 of every slice (coalesced, pre-swizzled).
// With oy (the tensor-core TRSM's operand A21 S^-1, sliced before that TRSM), column k is
// scaled by 2^-t_k, the shift POTRF stored with the supernode's inverse slices in oy.
__global__ void __launch_bounds__(kOzSliceThreads)
    k_oz_slice(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
               uint8_t* __restrict__ oz, int64_t oz_rows, const uint8_t* __restrict__ oy,
               int64_t oy_rows) {
  extern __shared__ __align__(16) double xs[];  // [n][kOzSliceLd]
  __shared__ int s_e[kOzM], s_t[kOzInvRows];
  const int4 tk = tasks[blockIdx.x];
  if (oy && tk.w < 0) return;  // A21 slices only for the tensor-core TRSM's supernodes
  const SnDev d = sns[tk.x];
  const int n = d.n, m = d.m, u = m - n;
  const int r0 = tk.y;
  const int rows = min(kOzM, ((u + 7) & ~7) - r0);  // slice rows this block owns
  const double* L = reinterpret_cast<const double*>(d.L) + n + r0;  // L21[r0 + i, k] = L[k m + i]
  static_assert(kOzM == 128, "stage_row_block stages 128 rows");
  stage_row_block(xs, kOzSliceLd, L, m, n, u - r0);
  if (threadIdx.x < kOzInvRows) {
    // the shifts follow the inverse slices' row exponents in oy
    const int32_t* shift =
        oy ? reinterpret_cast<const int32_t*>(oy + kOzSlices * (size_t)oy_rows * kOzRowBytes) +
                 oy_rows + tk.w
           : nullptr;
    s_t[threadIdx.x] = shift && threadIdx.x < n ? shift[threadIdx.x] : 0;
  }
  cp_async_wait_all();
  __syncthreads();
  const int64_t row0 = tk.z + (int64_t)r0;
  const size_t stride = (size_t)oz_rows * kOzRowBytes;
  if (threadIdx.x < kOzM) {
    const int i = threadIdx.x;
    // the largest entry's exponent field by integer comparison (the FP64 unit is slow):
    // max |x| = f 2^e with f in [0.5, 1) has e = field - 1022 (0 for rows of zeros and
    // subnormals, whose slices are zero)
    int emax = 0;  // of the row scaled by 2^-t_k (exponent fields shifted by -t_k)
    for (int k = 0; k < n; k++) {
      const int f = oz_exp_field(xs[k * kOzSliceLd + i]);
      if (f > 0) emax = max(emax, f - s_t[k]);
    }
    const int e = oz_row_exponent(emax);
    s_e[i] = e;
    if (i < rows) reinterpret_cast<int32_t*>(oz + kOzSlices * stride)[row0 + i] = e;
  }
  __syncthreads();
  for (int item = threadIdx.x; item < kOzM * 8; item += kOzSliceThreads) {
    const int i = item >> 3, pc = item & 7;  // row, physical 16-byte chunk
    if (i >= rows) continue;
    const int c = pc ^ (int)((row0 + i) & 7);  // logical chunk: columns 8c .. 8c+7
    const int e = s_e[i];
    long long R[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int k = 8 * c + j;
      R[j] = k < n ? oz_fixed(xs[k * kOzSliceLd + i], e + s_t[k]) : 0;  // x 2^-t_k
    }
    oz_write_chunk(R, oz + (size_t)(row0 + i) * kOzRowBytes + pc * 16, stride);
  }
}

// Eight accumulator columns of this warp's 32 TMEM lanes (one row per thread); the caller
// waits (tcgen05.wait::ld) before using them.
__device__ __forceinline__ void oz_tmem_load8(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(addr));
}

__device__ __forceinline__ void oz_tmem_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The FP32 bits of x + 1.5 * 2^23 for an accumulator x holding an integer of magnitude below
// 2^22: 0x4B400000 + x, i.e. the integer plus a fixed offset in the low mantissa bits.
__device__ __forceinline__ uint32_t oz_fbits(uint32_t acc) {
  return __float_as_uint(__uint_as_float(acc) + 12582912.0f);
}

// W = V_hi 2^20 + round(V_lo / 2^8) from the offset bits f_d = 0x4B400000 + D_d of the eight
// diagonals (V_hi = sum_{d<4} D_d 2^(7(3-d)), V_lo = sum_{d>=4} D_d 2^(7(7-d)), |D_d| < 2^22, so
// |W| < 2^62).  The offsets are never subtracted one by one: kOzLoBias = 128 - 0x4B400000 S
// (S = 1 + 2^7 + 2^14 + 2^21) removes those of V_lo and adds the rounding constant before the
// shift; the high diagonals enter modulo 2^64 (f_3 2^20 and f_2 2^27 as 32 x 32 -> 64-bit
// multiply-adds, f_1 2^34 + f_0 2^41 in the high word alone), and kOzHiBias = -(0x4B400000
// 2^20 S) >> 32 removes their offsets (it has no low word).  Exact since |W| < 2^63.
constexpr unsigned long long kOzLoBias = 0xfff6850a14c00080ull;
constexpr uint32_t kOzHiBias = 0x50a14c00u;

__device__ __forceinline__ unsigned long long oz_low(uint32_t f4, uint32_t f5, uint32_t f6,
                                                     uint32_t f7) {
  unsigned long long v = (unsigned long long)f7 + kOzLoBias;
  v = (unsigned long long)f6 * 128ull + v;
  v = (unsigned long long)f5 * 16384ull + v;
  v = (unsigned long long)f4 * 2097152ull + v;
  return (unsigned long long)((long long)v >> 8);  // round(V_lo / 2^8), half up
}

__device__ __forceinline__ long long oz_high(unsigned long long lo, uint32_t f0, uint32_t f1,
                                             uint32_t f2, uint32_t f3) {
  unsigned long long w = (unsigned long long)f3 * 1048576ull + lo;
  w = (unsigned long long)f2 * 134217728ull + w;
  w += (unsigned long long)(f1 * 4u + f0 * 512u + kOzHiBias) << 32;
  return (long long)w;
}

// s W 2^E as a double (s = -1 when NEG), rounded to nearest (ties to even): the FP64 unit's
// int64 -> double conversion, then an add to the exponent field and, for NEG, to the sign bit
// (exact inside the normal range; a signed zero for W = 0, ldexp outside the range).  The FP64 unit is otherwise
// idle in this kernel, and one conversion there costs the consumer warps far fewer issue slots
// than normalizing and rounding the 64-bit integer with integer operations.
template <bool NEG>
__device__ __forceinline__ double oz_to_double(long long W, int E) {
  const double d = __ll2double_rn(W);
  const uint32_t hi = (uint32_t)__double2hiint(d);
  const int be = (int)((hi >> 20) & 0x7ffu) + E;
  if (hi == 0u) return NEG ? -0.0 : 0.0;  // W = 0: adds nothing (-0.0 leaves every sum as it is)
  if ((unsigned)(be - 1) < 2046u)
    return __hiloint2double((int)(hi + (uint32_t)E * 1048576u + (NEG ? 0x80000000u : 0u)),
                            __double2loint(d));
  const double r = ldexp(d, E);
  return NEG ? -r : r;
}

constexpr int kOzMaxRuns = 8;  // column targets per task whose relative rows are cached
constexpr int kOzMetaBufs = 3;  // metadata buffers: the metadata warps run up to two tasks ahead

// Per-task metadata, in kOzMetaBufs buffers: the metadata warps build the next tasks' copies
// while the consumers scatter with the current one.
static_assert(2 * kOzN == 128, "the run count sums four 32-column words");
struct OzMeta {
  double* cp[2 * kOzN];  // each column's target panel column (its relative rows are added)
  int eA[kOzM], eB[2 * kOzN];  // row exponents e_i; column exponents e_k - 55
  int tcol[2 * kOzN], run[2 * kOzN];
  int run_start[2 * kOzN + 1];
  int wcnt[2 * kOzN / 32];  // run starts per 32 columns
  int fcnt[kOzMetaThreads / 32];  // the supernode's runs before the tile, per warp
  long long rb[2 * kOzN];  // relative-map base of every run
  int rp[kOzMaxRuns][kOzM];
  int nruns;
  int u, i0, k0;           // the task: update order, tile origin
  const int32_t* relmap;   // for runs beyond the cached ones
  double* ustage;          // owner assembly: this supernode's staged U
};

// barrier among the metadata warps only
__device__ __forceinline__ void oz_meta_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kOzMetaThreads) : "memory");
}

__device__ __forceinline__ void oz_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// A task is done as 128 x 32 quarters.  A load thread (its own warp) claims the tasks, hands
// each one to the other roles through a ring as soon as it has claimed it, and bulk-copies
// the task's 8 A slices once and every quarter's B slices into one of two quarter buffers;
// an MMA thread (its own warp) issues each quarter's MMAs into one of two TMEM sets of 8
// diagonals x 32 columns, slice by slice; the 16 consumer warps drain a finished set (and
// release it) while the tensor cores compute the next quarter, then scatter; four metadata
// warps build each task's exponents, column targets and relative rows up to two tasks ahead.
// Barriers: a_full (a task's 8 A slices in; a task with the previous task's A rows reuses
// them), b_full[2] (quarter B buffers in), acc_full[2] (a set's MMAs done: also frees the B
// buffer they read, and after a task's last quarter the A slices), acc_empty[2] (a set
// drained), meta_full[] / meta_empty[] (a metadata buffer built / released), ring_full[]
// (the task order).
template <bool OWNER>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_schur_oz(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
               const SnDev* __restrict__ sns, const MatDev* __restrict__ mats,
               const uint8_t* __restrict__ oz, int64_t oz_rows, long long acc_wait) {
  extern __shared__ __align__(1024) unsigned char oz_sm[];
  unsigned char* A =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz_sm) + 1023) & ~uintptr_t(1023));
  unsigned char* Bq0 = A + kOzABytes;  // quarter buffers: Bq0, Bq0 + kOzQBytes
  __shared__ __align__(8) uint64_t a_full, b_full[2], acc_full[2], acc_empty[2];
  __shared__ __align__(8) uint64_t ring_full[kOzRing];
  __shared__ int2 ring[kOzRing];  // {task, quarters | K steps << 8} (task = ntasks: stop)
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t meta_full[kOzMetaBufs], meta_empty[kOzMetaBufs];
  __shared__ OzMeta meta[kOzMetaBufs];
  __shared__ __align__(8) uint64_t never;  // test hook: a barrier nothing completes
  __shared__ int s_mtq;  // the metadata warps' next task (or ntasks: stop)
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // a launch of an earlier level of this factorization already gave up on a wait: its
  // updates are missing and the factorization is reported failed, so skip the work (before
  // any barrier or tensor memory is set up); every thread reads the same word
  if (ntasks > 0 && *(volatile unsigned long long*)(mats[sns[tasks[0].x].mat].err + 3) != 0) return;
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&a_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&never)));
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&b_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[i])),
                   "r"(kOzConsumers / 64));  // the 8 warps of the set's consumer group
    }
    for (int i = 0; i < kOzRing; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ring_full[i])));
    for (int i = 0; i < kOzMetaBufs; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&meta_full[i])),
                   "r"(kOzMetaThreads));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&meta_empty[i])),
                   "r"(kOzConsumers / 32));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == kOzLoadWarp) {
    // ---------------- loads: task claims, ring, bulk copies; one thread ----------------
    if (lane == 0) {
      long long T = 0;                       // A slice loads issued
      long long qb = 0;                      // quarter B buffers issued (buffer = qb & 1)
      long long ord = 0;                     // ring entries published
      bool ok = true;
      // Tasks are claimed in runs (g0 per CTA at first, then from the queue): four while more
      // than 16 per CTA remain, then two while more than 4 do, then singles: the tasks of a
      // row strip are consecutive in the list, so the later tasks of a run usually have the
      // first one's A rows, which stay in shared memory.
      const int g0 = ntasks >= 8 * (int)gridDim.x ? 4 : (ntasks >= 4 * (int)gridDim.x ? 2 : 1);
      int tq = g0 * (int)blockIdx.x;         // a CTA's first run follows its block index
      int tend = min(tq + g0, ntasks);       // end of the claimed run
      // The ring runs one task ahead of the copies: a task is published (and the next one
      // claimed) before the current task's copies are issued, so that the metadata warps
      // can build its targets while the current task is still being copied and computed.
      int prow = -1;                         // slice row of the last published task's A rows
      struct Job {
        int4 t;
        int nq, ks;
        bool reuse;  // the A rows of the task before it (still in shared memory)
      };
      auto publish = [&](int ti) -> Job {
        Job jb{make_int4(0, 0, 0, 0), 0, 0, false};
        if (ti < ntasks) {
          jb.t = tasks[ti];
          const SnDev& dd = sns[jb.t.x];
          jb.nq = min(4, (dd.m - dd.n - jb.t.z + kOzQ - 1) / kOzQ);
          jb.ks = (dd.n + 15) >> 4;
          jb.reuse = jb.t.w + jb.t.y == prow;
          prow = jb.t.w + jb.t.y;
        }
        const int rs = (int)(ord % kOzRing);
        ring[rs] = make_int2(ti < ntasks ? ti : ntasks, jb.nq | (jb.ks << 8) | ((int)jb.reuse << 16));
        oz_arrive(smem_u32(&ring_full[rs]));
        ord++;
        return jb;
      };
      int cur = tq;
      Job job = publish(cur);
      while (cur < ntasks) {
        if (++tq >= tend) {  // the run is done: claim the next one
          const int g = tq < ntasks - 16 * (int)gridDim.x ? 4
                        : (tq < ntasks - 4 * (int)gridDim.x ? 2 : 1);
          tq = g0 * (int)gridDim.x >= ntasks ? ntasks
                                             : g0 * (int)gridDim.x + atomicAdd(queue, g);
          tend = min(tq + g, ntasks);
        }
        const Job next = publish(tq);  // the next task (or the stop entry)
        const int4 t = job.t;
        const int nq = job.nq;
        // quarter j's B slices, once the MMAs of the quarter two back (same buffer) are done
        auto load_b = [&](int j) -> bool {
          const int b = (int)(qb & 1);
          if (qb >= 2 && !oz_wait(smem_u32(&acc_full[b]), (uint32_t)(((qb >> 1) - 1) & 1)))
            return false;
          const uint32_t bar = smem_u32(&b_full[b]);
          unsigned char* dst = Bq0 + b * kOzQBytes;
          oz_expect(bar, kOzQBytes);
          for (int p = 0; p < kOzSlices; p++)
            oz_bulk_load(smem_u32(dst + p * kOzQSlice),
                         oz + p * stride + (size_t)(t.w + t.z + kOzQ * j) * kOzRowBytes,
                         kOzQSlice, bar);
          qb++;
          return true;
        };
        // the first quarter's B goes first: its buffer is free before the A slices are
        if (!load_b(0)) {
          ok = false;
          break;
        }
        // the A slices of this task (unless the previous task had the same rows), once the
        // previous task's last quarter (the latest quarter before this task's first, qb - 2)
        // is done: every K step reads every slice
        if (!job.reuse) {
          if (T >= 1 &&
              !oz_wait(smem_u32(&acc_full[(qb - 2) & 1]), (uint32_t)(((qb - 2) >> 1) & 1))) {
            ok = false;
            break;
          }
          oz_expect(smem_u32(&a_full), kOzABytes);
          for (int p = 0; p < kOzSlices; p++)
            oz_bulk_load(smem_u32(A + p * kOzASlice),
                         oz + p * stride + (size_t)(t.w + t.y) * kOzRowBytes, kOzASlice,
                         smem_u32(&a_full));
          T++;
        }
        for (int j = 1; j < nq && ok; j++) ok = load_b(j);
        if (!ok) break;
        job = next;
        cur = tq;
      }
      if (!ok) {
        s_fail = 1;
        const int rs = (int)(ord % kOzRing);
        ring[rs] = make_int2(ntasks, 0);
        oz_arrive(smem_u32(&ring_full[rs]));
      }
      // bounded waits for the copies still in flight: the last A load and the last B load of
      // each buffer
      if (T >= 1) oz_wait(smem_u32(&a_full), (uint32_t)((T - 1) & 1));
      for (long long qq = qb - 2 < 0 ? 0 : qb - 2; qq < qb; qq++)
        oz_wait(smem_u32(&b_full[qq & 1]), (uint32_t)((qq >> 1) & 1));
    }
  } else if (warp == kOzMmaWarp) {
    // ---------------- MMAs, one thread ----------------
    if (lane == 0) {
      // N = (8 - p) x 32: the MMA of slice p against slices 0 .. 7-p of a quarter
      uint32_t idesc[kOzSlices];
#pragma unroll
      for (int p = 0; p < kOzSlices; p++) idesc[p] = oz_idesc((kOzSlices - p) * kOzQ);
      const uint64_t da0 = oz_desc(smem_u32(A));
      const uint64_t db[2] = {oz_desc(smem_u32(Bq0)), oz_desc(smem_u32(Bq0 + kOzQBytes))};
      bool ok = true;
      long long q = 0;  // quarters issued (TMEM set and B buffer = q & 1)
      long long T = 0;  // A slice loads waited for
      for (long long ord = 0; ok; ord++) {
        const int rs = (int)(ord % kOzRing);
        if (!oz_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kOzRing) & 1))) {
          ok = false;
          break;
        }
        const int2 e = ring[rs];
        if (e.x >= ntasks) break;
        const int nq = e.y & 0xff, ks = (e.y >> 8) & 0xff;
        const bool reuse = (e.y >> 16) & 1;  // the previous task's A slices
        for (int j = 0; j < nq; j++, q++) {
          const int b = (int)(q & 1);
          if (!oz_wait(smem_u32(&b_full[b]), (uint32_t)((q >> 1) & 1)) ||
              (q >= 2 &&  // the set was drained (quarter q - 2)
               !oz_wait(smem_u32(&acc_empty[b]), (uint32_t)(((q >> 1) - 1) & 1)))) {
            ok = false;
            break;
          }
          if (j == 0 && !reuse && !oz_wait(smem_u32(&a_full), (uint32_t)(T & 1))) {  // the task's A
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          // K step outer, slice inner: consecutive MMAs start at different diagonals (measured
          // 2.3x faster than issuing one slice's K steps back to back into the same columns)
          for (int k = 0; k < ks; k++)
#pragma unroll
            for (int p = 0; p < kOzSlices; p++)
              oz_mma(tmem + (uint32_t)(b * kOzSetCols + p * kOzQ),
                     da0 + (uint64_t)((p * kOzASlice) >> 4) + 2 * k, db[b] + 2 * k, idesc[p],
                     (p > 0 || k > 0) ? 1u : 0u);
          oz_commit(smem_u32(&acc_full[b]));
        }
        if (!reuse) T++;
      }
      if (!ok) s_fail = 1;
      // bounded wait for the MMAs in flight (the last quarter's commit covers all earlier ones)
      if (q >= 1) oz_wait(smem_u32(&acc_full[(q - 1) & 1]), (uint32_t)(((q - 1) >> 1) & 1));
    }
  } else if (warp >= kOzMetaBase / 32) {
    // ---------------- metadata warps: one thread per tile row / column ----------------
    // For each task in ring order, into meta[ord % kOzMetaBufs] once the consumers have released it:
    // the rows' and columns' slice exponents, every column's target supernode, the runs of
    // equal target (ballot per 32 columns), each column's run and column inside its target,
    // per run the relative-map base and target panel, and the relative rows of the first
    // kOzMaxRuns runs.  Thread 0 alone waits on the ring and on the buffer, so that the
    // group's decisions are uniform.
    const int mt = tid - kOzMetaBase, mwarp = mt >> 5;
    for (int ord = 0;; ord++) {
      const int buf = ord % kOzMetaBufs;
      if (mt == 0) {
        const int rs = ord % kOzRing;
        int tq = ntasks;
        if (!oz_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kOzRing) & 1)) ||
            (ring[rs].x < ntasks && ord >= kOzMetaBufs &&
             !oz_wait(smem_u32(&meta_empty[buf]), (uint32_t)((ord / kOzMetaBufs - 1) & 1))))
          s_fail = 1;
        else
          tq = ring[rs].x;
        s_mtq = tq;
      }
      oz_meta_sync();
      const int tq = s_mtq;
      oz_meta_sync();  // s_mtq is rewritten only after every thread has read it
      if (tq >= ntasks) break;
      OzMeta& M = meta[buf];
      const int4 tk = tasks[tq];
      const SnDev d = sns[tk.x];
      const int n = d.n, u = d.m - n, i0 = tk.y, k0 = tk.z;
      const MatDev md = mats[d.mat];
      const int gk = k0 + mt;
      M.eA[mt] = (i0 + mt < u) ? exps[tk.w + i0 + mt] : 0;
      M.eB[mt] = (gk < u ? exps[tk.w + gk] : 0) - 55;  // U = W 2^(e_i + e_k - 55)
      if (mt == 0) {
        M.u = u;
        M.i0 = i0;
        M.k0 = k0;
        M.relmap = md.relmap;
        M.ustage = OWNER ? static_cast<double*>(md.stage) + d.ustage : nullptr;
      }
      if (!OWNER) {
        const int32_t* rows = d.rows + n;
        const int grow = gk < u ? rows[gk] : 0;
        const int tc = gk < u ? md.col2sn[grow] : -1;
        M.tcol[mt] = tc;
        // the supernode's runs that start after position 0 and at or before k0: their count
        // is the index (from run0) of the run holding the tile's first column; the tile's
        // runs are that run and the ones after it, in order (runs split where the target
        // changes, and so do the tile's)
        int before = 0;
        for (int t = 1 + mt; t < d.nrun; t += kOzMetaThreads) before += md.run_a[d.run0 + t] <= k0 ? 1 : 0;
        before = __reduce_add_sync(0xffffffffu, before);
        if (lane == 0) M.fcnt[mwarp] = before;
        oz_meta_sync();
        // a column starts a run when its target differs from its left neighbour's; its run
        // index is the number of starts up to it, less one
        const bool start = gk < u && (mt == 0 || M.tcol[mt - 1] != tc);
        const unsigned bl = __ballot_sync(0xffffffffu, start);
        if (lane == 0) M.wcnt[mwarp] = __popc(bl);
        oz_meta_sync();
        int off = 0;
        for (int w2 = 0; w2 < mwarp; w2++) off += M.wcnt[w2];
        const int first = d.run0 + M.fcnt[0] + M.fcnt[1] + M.fcnt[2] + M.fcnt[3];
        if (gk < u) {
          const int r = off + __popc(bl & ((2u << lane) - 1u)) - 1;
          const SnDev& td = sns[md.sn_base + tc];
          M.run[mt] = r;
          M.cp[mt] = reinterpret_cast<double*>(td.L) + (int64_t)(grow - td.col0) * td.m;
          if (start) {  // the run's first column fetches its map base
            M.run_start[r] = mt;
            M.rb[r] = md.run_base[first + r];
          }
        }
        if (mt == 0) M.nruns = M.wcnt[0] + M.wcnt[1] + M.wcnt[2] + M.wcnt[3];
        oz_meta_sync();
        // relative rows of the cached runs: this thread's tile row in each, all loads in flight
        static_assert(kOzMetaThreads == kOzM, "one metadata thread per tile row");
        const int nrc = min(M.nruns, kOzMaxRuns), g = i0 + mt;
        int rpv[kOzMaxRuns];
#pragma unroll
        for (int r = 0; r < kOzMaxRuns; r++)
          rpv[r] = (r < nrc && g < u && g >= k0 + M.run_start[r]) ? md.relmap[M.rb[r] + g] : -1;
#pragma unroll
        for (int r = 0; r < kOzMaxRuns; r++)
          if (r < nrc) M.rp[r][mt] = rpv[r];
      }
      oz_arrive(smem_u32(&meta_full[buf]));  // each thread after its own writes
    }
  } else {
    // ---------------- consumers: set drain and scatter ----------------
    // Two groups of 8 warps, one per TMEM set: group g takes the quarters on set g (global
    // quarter index q with q & 1 == g), a warp 32 rows x 16 columns of it as two chunks of 8
    // columns.  The groups work half a quarter apart, so one group's conversions (FP64 unit)
    // overlap the other's atomics (memory pipe) instead of all 16 warps running each phase
    // at once.  A set is released after the warp's second chunk is drained.  Each wait's
    // outcome is made uniform over the warp (tcgen05.ld is warp-collective).
    const int grp = warp >> 3;
    const int i = 32 * (warp & 3) + lane;     // this thread's tile row
    const int c16 = 16 * ((warp >> 2) & 1);   // this warp's 16 columns of a quarter
    long long q0 = 0;                         // global index of the task's first quarter
    for (int ord = 0;; ord++) {
      const int rs = ord % kOzRing, buf = ord % kOzMetaBufs;
      if (!__all_sync(0xffffffffu, oz_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kOzRing) & 1)))) {
        s_fail = 1;
        break;
      }
      if (ring[rs].x >= ntasks) break;
      const OzMeta& M = meta[buf];
      if (!__all_sync(0xffffffffu, oz_wait(smem_u32(&meta_full[buf]), (uint32_t)((ord / kOzMetaBufs) & 1)))) {
        s_fail = 1;
        break;
      }
      const int u = M.u, i0 = M.i0, k0 = M.k0;
      const int nq = min(4, (u - k0 + kOzQ - 1) / kOzQ);
      const int gi = i0 + i;
      const int eA = M.eA[i];
      bool stop = false;
      for (int j = 0; j < nq && !stop; j++) {
        const long long q = q0 + j;
        if ((int)(q & 1) != grp) continue;
        const int b = grp;
        // acc_wait > 0 (a test hook): wait that long on a barrier that never completes instead,
        // standing in for an accumulator that never finishes
        const bool got = acc_wait > 0 ? oz_wait(smem_u32(&never), 0u, acc_wait)
                                      : oz_wait(smem_u32(&acc_full[b]), (uint32_t)((q >> 1) & 1));
        if (!__all_sync(0xffffffffu, got)) {
          s_fail = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int c = 0; c < 2; c++) {
          const int c8 = c16 + 8 * c;  // this chunk's 8 columns of the quarter
          const int kb = kOzQ * j + c8, gk0 = k0 + kb;
          const int r0w = i0 + 32 * (warp & 3);  // the warp's first tile row
          // warp-uniform: no entry of the chunk in the lower triangle of the update (past
          // its order, or above the diagonal): nothing to read but the release
          const bool dead = r0w >= u || gk0 >= u || r0w + 31 < gk0;
          double val[8];
          if (!dead) {
            // the 8 diagonals of the chunk's columns -> W (exact integer) -> U = W 2^(e_i +
            // e_k - 55)
            const uint32_t ta =
                tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * kOzSetCols + c8);
            unsigned long long w[8];
            {
              uint32_t v[4][8];
#pragma unroll
              for (int dd = 0; dd < 4; dd++)
                oz_tmem_load8(ta + (uint32_t)((4 + dd) * kOzQ), v[dd]);
              oz_tmem_wait();
#pragma unroll
              for (int jj = 0; jj < 8; jj++)
                w[jj] = oz_low(oz_fbits(v[0][jj]), oz_fbits(v[1][jj]), oz_fbits(v[2][jj]),
                               oz_fbits(v[3][jj]));
            }
            {
              uint32_t v[4][8];
#pragma unroll
              for (int dd = 0; dd < 4; dd++) oz_tmem_load8(ta + (uint32_t)(dd * kOzQ), v[dd]);
              oz_tmem_wait();
#pragma unroll
              for (int jj = 0; jj < 8; jj++)
                w[jj] = (unsigned long long)oz_high(w[jj], oz_fbits(v[0][jj]),
                                                    oz_fbits(v[1][jj]), oz_fbits(v[2][jj]),
                                                    oz_fbits(v[3][jj]));
            }
            if (c == 1) {  // the warp's last reads of this set
              asm volatile("tcgen05.fence::before_thread_sync;");
              __syncwarp();
              if (lane == 0) oz_arrive(smem_u32(&acc_empty[b]));
            }
#pragma unroll
            for (int jj = 0; jj < 8; jj++)  // -U for the atomics, U for the staging buffer
              val[jj] = oz_to_double<!OWNER>((long long)w[jj], eA + M.eB[kb + jj]);
          } else if (c == 1) {
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) oz_arrive(smem_u32(&acc_empty[b]));
          }
          if (dead) continue;
          // scatter this thread's row of the chunk
          if (OWNER) {
            if (gi < u) {
              double* U = M.ustage;
#pragma unroll
              for (int jj = 0; jj < 8; jj++) {
                const int gk = gk0 + jj;
                if (gk < u && gk <= gi) U[(int64_t)gk * u + gi] = val[jj];
              }
            }
          } else if (r0w + 31 < u && gk0 + 7 < u && gk0 + 7 <= r0w &&
                     M.run[kb] == M.run[kb + 7]) {
            // warp-uniform fast path: every entry live, one target run for all 8 columns
            const int r = M.run[kb];
            const int p = r < kOzMaxRuns ? M.rp[r][i] : M.relmap[M.rb[r] + gi];
            if (p >= 0) {
#pragma unroll
              for (int jj = 0; jj < 8; jj++) red_add(M.cp[kb + jj] + p, val[jj]);
            }
          } else if (gi < u) {
            // the relative row changes only with the run, which is the same for every lane
            int rprev = -1, p = -1;
#pragma unroll
            for (int jj = 0; jj < 8; jj++) {
              const int kk = kb + jj, gk = k0 + kk;
              if (gk >= u || gk > gi) continue;
              const int r = M.run[kk];
              if (r != rprev) {
                rprev = r;
                p = r < kOzMaxRuns ? M.rp[r][i] : M.relmap[M.rb[r] + gi];
              }
              if (p >= 0) red_add(M.cp[kk] + p, val[jj]);
            }
          }
        }
      }
      if (stop) break;
      q0 += nq;
      __syncwarp();
      if (lane == 0) oz_arrive(smem_u32(&meta_empty[buf]));
    }
  }
  __syncthreads();
  if (s_fail && tid == 0 && ntasks > 0) atomicAdd(mats[sns[tasks[0].x].mat].err + 3, 1ull);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOzTmemCols));
}

// ---- TRSM of the 128-tile supernodes on the tensor cores ----------------------------------
// L21 = A21 L11^{-T} = A21 Y^T with Y = L11^{-1}, formed by POTRF, which also stored the
// slices of Y S (S = diag(2^t_k), t_k the exponent of L11[k,k]) and the shifts t_k in oy; the
// slices of A21 S^-1 come from the slicing kernel run on the panel just before.  L21 =
// (A21 S^-1)(Y S)^T is a product of row-sliced operands of exactly the Schur tiles' form,
// L21[i, j] = 2^(e_i + e_j) sum_{p+q<8} 2^(-7(p+q+2)) sum_k a_p[i,k] y_q[j,k], K = n <= 64, so
// every diagonal's partial sums are integers below 2^22 (exact in FP32) and the combination is
// the same integer one.  One CTA per task (128 rows of A21): one thread bulk-copies the task's
// 8 A slices (128 KB) and Y's 8 slices (64 rows each, 64 KB), then issues, per K step and A
// slice p, the MMAs of A_p against Y slices 0 .. 7-p in one go (N = (8-p) 64, at most 256 per
// MMA): diagonal p + q lands at TMEM columns (p + q) 64, the 8 diagonals fill the 512 columns.
// Eight warps then read the accumulators (warp w: TMEM lanes 32 (w & 3) .., columns
// 32 (w >> 2) ..), combine them exactly, round once to FP64 and store L21 into the panel.
// (Forming the slices inside this kernel as well was measured slower: one CTA per SM then
// serializes the slicing, the copies and the tensor work, which separate launches overlap.)
// Waits are bounded as in the Schur tiles; a timeout is recorded in err[3] and nothing stored.
constexpr int kToThreads = 256;
constexpr uint32_t kToBSlice = kOzInvRows * kOzRowBytes;  // 8 KB: one slice of Y's rows
constexpr uint32_t kToBBytes = kOzSlices * kToBSlice;      // 64 KB
constexpr size_t kToSmem = 1024 + kOzABytes + kToBBytes;   // + alignment slack
constexpr uint32_t kToTmemCols = kOzSlices * kOzInvRows;   // 512

__global__ void __launch_bounds__(kToThreads, 1)
    k_trsm_oz(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
              const MatDev* __restrict__ mats, const uint8_t* __restrict__ oz, int64_t oz_rows,
              const uint8_t* __restrict__ oy, int64_t oy_rows) {
  extern __shared__ __align__(1024) unsigned char to_sm[];
  unsigned char* A =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(to_sm) + 1023) & ~uintptr_t(1023));
  unsigned char* B = A + kOzABytes;
  __shared__ __align__(8) uint64_t full, done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 tk = tasks[blockIdx.x];
  if (tk.w < 0) return;  // the supernode keeps the FP64 TRSM
  const SnDev d = sns[tk.x];
  unsigned long long* err = mats[d.mat].err;
  // a launch of this factorization already gave up on a wait: skip (before any set-up)
  if (*(volatile unsigned long long*)(err + 3) != 0) return;
  const int n = d.n, m = d.m, u = m - n, r0 = tk.y;
  const int rb = min(kOzM, u - r0);
  const size_t sa = (size_t)oz_rows * kOzRowBytes, sb = (size_t)oy_rows * kOzRowBytes;
  const int32_t* ea = reinterpret_cast<const int32_t*>(oz + kOzSlices * sa);
  const int32_t* ey = reinterpret_cast<const int32_t*>(oy + kOzSlices * sb);
  const int64_t arow = (int64_t)tk.z + r0, yrow = tk.w;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kToTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t fb = smem_u32(&full);
    oz_expect(fb, kOzABytes + kToBBytes);
    for (int p = 0; p < kOzSlices; p++)
      oz_bulk_load(smem_u32(A + p * kOzASlice), oz + p * sa + (size_t)arow * kOzRowBytes,
                   kOzASlice, fb);
    for (int p = 0; p < kOzSlices; p++)
      oz_bulk_load(smem_u32(B + p * kToBSlice), oy + p * sb + (size_t)yrow * kOzRowBytes,
                   kToBSlice, fb);
    if (oz_wait(fb, 0)) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t da = oz_desc(smem_u32(A)), db = oz_desc(smem_u32(B));
      const int ks = (n + 15) >> 4;
      // K step outer, A slice inner (consecutive MMAs start at different diagonals); the
      // first K step of slice 0 writes every diagonal, everything after accumulates
      for (int k = 0; k < ks; k++)
        for (int p = 0; p < kOzSlices; p++)
          for (int q0 = 0; q0 < kOzSlices - p; q0 += 4) {
            const int nq = min(4, kOzSlices - p - q0);
            oz_mma(tmem + (uint32_t)((p + q0) * kOzInvRows),
                   da + (uint64_t)((p * kOzASlice) >> 4) + 2 * k,
                   db + (uint64_t)((q0 * kToBSlice) >> 4) + 2 * k, oz_idesc(nq * kOzInvRows),
                   (p > 0 || k > 0) ? 1u : 0u);
          }
      oz_commit(smem_u32(&done));
    } else {
      s_fail = 1;
      oz_arrive(smem_u32(&done));
      oz_wait(fb, 0);  // bounded: the copies in flight
    }
  }
  if (!oz_wait(smem_u32(&done), 0)) s_fail = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (!s_fail) {  // uniform: the warps' TMEM loads are collective
    const int lq = warp & 3, ch = warp >> 2;
    const int i = 32 * lq + lane;  // this thread's row of the task
    const int eA = i < rb ? ea[arow + i] - 55 : 0;
    double* out = reinterpret_cast<double*>(d.L) + n + r0 + i;
    for (int c8 = 0; c8 < 4; c8++) {
      const int col0 = 32 * ch + 8 * c8;
      uint32_t v[kOzSlices][8];
#pragma unroll
      for (int dd = 0; dd < kOzSlices; dd++)
        oz_tmem_load8(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(dd * kOzInvRows + col0), v[dd]);
      oz_tmem_wait();
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int col = col0 + j;
        if (i < rb && col < n) {
          const unsigned long long lo =
              oz_low(oz_fbits(v[4][j]), oz_fbits(v[5][j]), oz_fbits(v[6][j]), oz_fbits(v[7][j]));
          const long long W =
              oz_high(lo, oz_fbits(v[0][j]), oz_fbits(v[1][j]), oz_fbits(v[2][j]), oz_fbits(v[3][j]));
          out[(int64_t)col * m] = oz_to_double<false>(W, eA + ey[yrow + col]);
        }
      }
    }
  } else if (tid == 0) {
    atomicAdd(err + 3, 1ull);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kToTmemCols));
}

void launch_trsm_oz(const int4* tasks, int ntasks, const SnDev* sns, const MatDev* mats,
                    const void* oz, int64_t oz_rows, const void* oy, int64_t oy_rows,
                    cudaStream_t st) {
  if (ntasks <= 0) return;
  k_trsm_oz<<<ntasks, kToThreads, kToSmem, st>>>(tasks, sns, mats,
                                                 static_cast<const uint8_t*>(oz), oz_rows,
                                                 static_cast<const uint8_t*>(oy), oy_rows);
}

void launch_oz_slice(const int4* tasks, int ntasks, const SnDev* sns, void* oz, int64_t oz_rows,
                     const void* oy, int64_t oy_rows, cudaStream_t st) {
  if (ntasks <= 0) return;
  k_oz_slice<<<ntasks, kOzSliceThreads, (size_t)64 * kOzSliceLd * sizeof(double), st>>>(
      tasks, sns, static_cast<uint8_t*>(oz), oz_rows, static_cast<const uint8_t*>(oy), oy_rows);
}

size_t oy_scratch_bytes(int64_t oy_rows) {
  return oz_scratch_bytes(oy_rows) + (size_t)oy_rows * sizeof(int32_t);
}

void launch_schur_oz(const int4* tasks, int ntasks, int* queue, const SnDev* sns,
                     const MatDev* mats, bool owner, const void* oz, int64_t oz_rows,
                     long long acc_wait, cudaStream_t st) {
  if (ntasks <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntasks < sms ? ntasks : sms;  // one resident CTA per SM, tasks by queue
  const uint8_t* z = static_cast<const uint8_t*>(oz);
  if (owner)
    k_schur_oz<true><<<grid, kOzThreads, kOzSmem, st>>>(tasks, ntasks, queue, sns, mats, z, oz_rows,
                                                       acc_wait);
  else
    k_schur_oz<false><<<grid, kOzThreads, kOzSmem, st>>>(tasks, ntasks, queue, sns, mats, z,
                                                        oz_rows, acc_wait);
}

size_t oz_scratch_bytes(int64_t oz_rows) {
  return (size_t)oz_rows * (kOzSlices * kOzRowBytes + sizeof(int32_t));
}

int set_oz_kernel_attrs() {
  if (cudaFuncSetAttribute(k_oz_slice, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(64 * kOzSliceLd * sizeof(double))) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kOzSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kOzSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_trsm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kToSmem) != cudaSuccess)
    return CHOL_E_CUDA;
  return CHOL_OK;
}

}  // namespace chol
