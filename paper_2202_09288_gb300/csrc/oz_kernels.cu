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
//               brought into shared memory by bulk copies; one producer thread issues,
//               for every slice pair p + q < 8, the bf16 MMAs of D_{p+q} += S_p S_q^T into
//               the quarter's set of tensor-memory accumulators (one per diagonal p + q,
//               8 x 32 columns; two sets).  Every partial sum of a diagonal is an integer
//               below 2^22 (K <= 64), so FP32 accumulation is exact.  Consumer warps read a
//               finished set (lane = tile row), release it, form U[i,k] = 2^(e_i+e_k)
//               sum_d 2^(-7(d+2)) D_d[i,k] as an FP64 value (integer combination, one
//               int64 -> double conversion) and scatter it into the ancestors with FP64
//               atomics (or write the owner staging buffer) while the tensor cores compute
//               the next quarter; metadata warps prepare each task's targets one task ahead.
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

constexpr int kOzConsumers = 512;                          // 16 warps: drain + scatter
constexpr int kOzMetaThreads = 128;                        // 4 warps: per-task metadata
constexpr int kOzThreads = kOzConsumers + 32 + kOzMetaThreads;  // + the producer warp
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
__device__ __forceinline__ uint32_t oz_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
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

}  // namespace

// bf16 bits of an integer of magnitude at most 256 (exact).
__device__ __forceinline__ uint32_t oz_bf16_of_int(int v) {
  if (v == 0) return 0u;
  const uint32_t a = (uint32_t)(v < 0 ? -v : v);
  const int e = 31 - __clz(a);  // a in [2^e, 2^(e+1))
  return (v < 0 ? 0x8000u : 0u) | ((uint32_t)(127 + e) << 7) | ((a << (7 - e)) & 0x7Fu);
}

// x 2^(56 - e) as an integer (|x| < 2^e, so |result| < 2^56), truncated toward zero below
// 2^0 (an error below 2^(e-56)); subnormal x give 0.
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int exb = (int)((bits >> 52) & 0x7FF);
  if (exb == 0) return 0;
  const long long mant = (bits & ((1ll << 52) - 1)) | (1ll << 52);  // x = mant 2^(exb-1075)
  const int sh = exb - 1019 - e;
  const long long M = sh >= 0 ? mant << sh : (sh > -64 ? mant >> -sh : 0);
  return bits < 0 ? -M : M;
}

constexpr int kOzSliceThreads = 256;
constexpr int kOzSliceLd = kOzM + 1;  // padded column stride of the staged block

// Slices of the L21 rows r0 .. r0+127 of supernode s, at slice rows oz + r (rows u ..
// roundup(u, 8) get zero slices).  The block is staged column by column through shared
// memory (cp.async, all copies in flight); a row's exponent e_r is that of its largest entry; each
// entry becomes the 56-bit fixed-point integer x 2^(56-e_r), cut into 8 balanced digits
// of 7 bits (round to nearest: |s_0| <= 128, |s_p| <= 64, exact); thread t writes the
// 16-byte chunk t % 8 of row t / 8 of every slice (coalesced, pre-swizzled).
__global__ void __launch_bounds__(kOzSliceThreads)
    k_oz_slice(const int4* __restrict__ tasks, const SnDev* __restrict__ sns,
               uint8_t* __restrict__ oz, int64_t oz_rows) {
  extern __shared__ __align__(16) double xs[];  // [n][kOzSliceLd]
  __shared__ int s_e[kOzM];
  const int4 tk = tasks[blockIdx.x];
  const SnDev d = sns[tk.x];
  const int n = d.n, m = d.m, u = m - n;
  const int r0 = tk.y;
  const int rows = min(kOzM, ((u + 7) & ~7) - r0);  // slice rows this block owns
  const double* L = reinterpret_cast<const double*>(d.L) + n + r0;  // L21[r0 + i, k] = L[k m + i]
  static_assert(kOzM == 128, "stage_row_block stages 128 rows");
  stage_row_block(xs, kOzSliceLd, L, m, n, u - r0);
  cp_async_wait_all();
  __syncthreads();
  const int64_t row0 = tk.z + (int64_t)r0;
  const size_t stride = (size_t)oz_rows * kOzRowBytes;
  if (threadIdx.x < kOzM) {
    const int i = threadIdx.x;
    // the largest entry's exponent field by integer comparison (the FP64 unit is slow):
    // max |x| = f 2^e with f in [0.5, 1) has e = field - 1022 (0 for rows of zeros and
    // subnormals, whose slices are zero)
    int emax = 0;
    for (int k = 0; k < n; k++)
      emax = max(emax, (int)((__double_as_longlong(xs[k * kOzSliceLd + i]) >> 52) & 0x7FF));
    const int e = emax > 0 ? emax - 1022 : 0;
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
      R[j] = k < n ? oz_fixed(xs[k * kOzSliceLd + i], e) : 0;
    }
    uint8_t* dst = oz + (size_t)(row0 + i) * kOzRowBytes + pc * 16;
#pragma unroll
    for (int p = 0; p < kOzSlices; p++) {
      const int w = 49 - 7 * p;  // weight of digit p: 2^w
      uint32_t h[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        long long dgt;
        if (p + 1 < kOzSlices) {
          dgt = (R[j] + (1ll << (w - 1))) >> w;
          R[j] -= dgt << w;
        } else {
          dgt = R[j];  // the last digit takes the exact remainder (|R| <= 2^6)
        }
        h[j] = oz_bf16_of_int((int)dgt);
      }
      uint4 v;
      v.x = h[0] | (h[1] << 16);
      v.y = h[2] | (h[3] << 16);
      v.z = h[4] | (h[5] << 16);
      v.w = h[6] | (h[7] << 16);
      *reinterpret_cast<uint4*>(dst + p * stride) = v;
    }
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

// An FP32 value holding an integer of magnitude below 2^22, as that integer: adding
// 1.5 * 2^23 puts it in the low mantissa bits.
__device__ __forceinline__ int32_t oz_int(uint32_t f) {
  return __float_as_int(__uint_as_float(f) + 12582912.0f) - 0x4B400000;
}

// Four diagonals D_d .. D_d+3 of eight columns -> sum_j D_(d+j) 2^(7(3-j)) (< 2^44 in
// magnitude): two int32 Horner steps, one 64-bit combination.
__device__ __forceinline__ void oz_combine4(const uint32_t (&v)[4][8], long long (&out)[8]) {
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int hi = oz_int(v[0][j]) * 128 + oz_int(v[1][j]);  // |.| < 2^30
    const int lo = oz_int(v[2][j]) * 128 + oz_int(v[3][j]);
    out[j] = (long long)((unsigned long long)(long long)hi << 14) + lo;  // hi 2^14 + lo
  }
}


// W 2^E as a double, rounded to nearest (ties to even): the FP64 unit's int64 -> double
// conversion, then an add to the exponent field (exact inside the normal range; ldexp
// otherwise).  The FP64 unit is otherwise idle in this kernel, and one conversion there
// costs the consumer warps far fewer issue slots than normalizing and rounding the 64-bit
// integer with integer operations (measured: the Schur kernel 13 % faster).
__device__ __forceinline__ double oz_to_double(long long W, int E) {
  if (W == 0) return 0.0;
  const double d = __ll2double_rn(W);
  const long long bits = __double_as_longlong(d);
  const int be = (int)((bits >> 52) & 0x7ff) + E;
  if (be <= 0 || be >= 2047) return ldexp(d, E);
  return __longlong_as_double(bits + ((long long)E << 52));
}

constexpr int kOzMaxRuns = 16;  // column targets per task whose relative rows are cached

// Per-task metadata, double-buffered: the metadata warps build the next task's copy while
// the consumers scatter with the current one.
static_assert(2 * kOzN == 128, "the run count sums four 32-column words");
struct OzMeta {
  double* cp[2 * kOzN];  // each column's target panel column (its relative rows are added)
  int eA[kOzM], eB[2 * kOzN];
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

// A task is done as 128 x 32 quarters.  The producer thread (its own warp) loads the task's
// A slices once and the B slices of every quarter into one of two quarter buffers, and
// issues each quarter's MMAs into one of two TMEM sets of 8 diagonals x 32 columns; the 16
// consumer warps drain a finished set (and release it) while the tensor cores compute the
// next quarter, then scatter; four metadata warps build each task's exponents, column
// targets and relative rows ahead of use.  Barriers: a_full (A slices in), b_full[2]
// (quarter B buffers in), acc_full[2] (a set's MMAs done: also frees the B buffer they
// read), acc_empty[2] (a set drained), meta_full[2] / meta_empty[2] (a metadata buffer
// built / released), ring_full[] (the task order, for the consumers and metadata warps).
template <bool OWNER>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_schur_oz(const int4* __restrict__ tasks, int ntasks, int* __restrict__ queue,
               const SnDev* __restrict__ sns, const MatDev* __restrict__ mats,
               const uint8_t* __restrict__ oz, int64_t oz_rows) {
  extern __shared__ __align__(1024) unsigned char oz_sm[];
  unsigned char* A =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz_sm) + 1023) & ~uintptr_t(1023));
  unsigned char* Bq0 = A + kOzABytes;  // quarter buffers: Bq0, Bq0 + kOzQBytes
  __shared__ __align__(8) uint64_t a_full, b_full[2], acc_full[2], acc_empty[2];
  __shared__ __align__(8) uint64_t ring_full[kOzRing];
  __shared__ int ring[kOzRing];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t meta_full[2], meta_empty[2];
  __shared__ OzMeta meta[2];
  __shared__ int s_mtq;  // the metadata warps' next task (or ntasks: stop)
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&b_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[i])),
                   "r"(kOzConsumers / 32));
    }
    for (int i = 0; i < kOzRing; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ring_full[i])));
    for (int i = 0; i < 2; i++) {
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

  if (warp == kOzConsumers / 32) {
    // ---------------- producer: operand loads and MMAs, one thread ----------------
    if (lane == 0) {
      // N = (8 - p) x 32: the MMA of slice p against slices 0 .. 7-p of a quarter
      uint32_t idesc[kOzSlices];
#pragma unroll
      for (int p = 0; p < kOzSlices; p++) idesc[p] = oz_idesc((kOzSlices - p) * kOzQ);
      const uint64_t da0 = oz_desc(smem_u32(A));
      const uint64_t db[2] = {oz_desc(smem_u32(Bq0)), oz_desc(smem_u32(Bq0 + kOzQBytes))};
      long long a_issued = 0, b_issued[2] = {0, 0};  // loads issued per barrier
      auto load_a = [&](const int4& t) {
        const uint32_t bar = smem_u32(&a_full);
        oz_expect(bar, kOzABytes);
        for (int p = 0; p < kOzSlices; p++)
          oz_bulk_load(smem_u32(A + p * kOzASlice),
                       oz + p * stride + (size_t)(t.w + t.y) * kOzRowBytes, kOzASlice, bar);
        a_issued++;
      };
      auto load_b = [&](const int4& t, int j, int b) {
        const uint32_t bar = smem_u32(&b_full[b]);
        unsigned char* dst = Bq0 + b * kOzQBytes;
        oz_expect(bar, kOzQBytes);
        for (int p = 0; p < kOzSlices; p++)
          oz_bulk_load(smem_u32(dst + p * kOzQSlice),
                       oz + p * stride + (size_t)(t.w + t.z + kOzQ * j) * kOzRowBytes, kOzQSlice,
                       bar);
        b_issued[b]++;
      };
      auto quarters = [&](const int4& t) {
        const SnDev& dd = sns[t.x];
        return min(4, (dd.m - dd.n - t.z + kOzQ - 1) / kOzQ);
      };
      bool ok = true;
      long long q = 0;          // quarters issued (set and buffer = q & 1)
      long long a_use = 0;      // A loads completed-and-waited
      int ord = 0;
      int tq = blockIdx.x;
      ring[0] = tq < ntasks ? tq : ntasks;
      oz_arrive(smem_u32(&ring_full[0]));
      if (tq < ntasks) {
        load_a(tasks[tq]);
        load_b(tasks[tq], 0, 0);
      }
      while (ok && tq < ntasks) {
        const int4 t = tasks[tq];
        const int nq = quarters(t);
        const int ks = (sns[t.x].n + 15) >> 4;
        if (!oz_wait(smem_u32(&a_full), (uint32_t)(a_use & 1))) { ok = false; break; }
        a_use++;
        // the next task is fetched now so its first quarter can be prefetched
        const int next = gridDim.x >= ntasks ? ntasks : (int)gridDim.x + atomicAdd(queue, 1);
        for (int j = 0; j < nq && ok; j++, q++) {
          const int b = (int)(q & 1);
          if (!oz_wait(smem_u32(&b_full[b]), (uint32_t)((q >> 1) & 1)) ||
              (q >= 2 &&  // the set was drained (quarter q - 2)
               !oz_wait(smem_u32(&acc_empty[b]), (uint32_t)(((q >> 1) - 1) & 1)))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          for (int k = 0; k < ks; k++)
#pragma unroll
            for (int p = 0; p < kOzSlices; p++)
              oz_mma(tmem + (uint32_t)(b * kOzSetCols + p * kOzQ),
                     da0 + (uint64_t)((p * kOzASlice) >> 4) + 2 * k, db[b] + 2 * k, idesc[p],
                     (p > 0 || k > 0) ? 1u : 0u);
          oz_commit(smem_u32(&acc_full[b]));
          // prefetch the next quarter into the other buffer (its MMAs, quarter q - 1, must
          // be done); the next task's A waits for this quarter's MMAs
          const bool last = j + 1 == nq;
          if (!last || next < ntasks) {
            if (q >= 1 && !oz_wait(smem_u32(&acc_full[b ^ 1]), (uint32_t)(((q - 1) >> 1) & 1))) {
              ok = false;
              break;
            }
            if (last) {
              if (!oz_wait(smem_u32(&acc_full[b]), (uint32_t)((q >> 1) & 1))) { ok = false; break; }
              load_a(tasks[next]);
              load_b(tasks[next], 0, b ^ 1);
            } else {
              load_b(t, j + 1, b ^ 1);
            }
          }
        }
        if (!ok) break;
        ord++;
        tq = next;
        ring[ord % kOzRing] = tq < ntasks ? tq : ntasks;
        oz_arrive(smem_u32(&ring_full[ord % kOzRing]));
      }
      if (!ok) {
        s_fail = 1;
        ring[(ord + 1) % kOzRing] = ntasks;
        oz_arrive(smem_u32(&ring_full[(ord + 1) % kOzRing]));
      }
      // bounded waits for the MMAs and copies still in flight (a quarter's B buffer is
      // waited once per quarter issued: b_issued[b] - (quarters on b) loads remain)
      if (q >= 1) oz_wait(smem_u32(&acc_full[(q - 1) & 1]), (uint32_t)(((q - 1) >> 1) & 1));
      for (int b = 0; b < 2; b++) {
        const long long waited = (q + 1 - b) >> 1;  // quarters issued on buffer b
        if (b_issued[b] > waited) oz_wait(smem_u32(&b_full[b]), (uint32_t)(waited & 1));
      }
      if (a_issued > a_use) oz_wait(smem_u32(&a_full), (uint32_t)(a_use & 1));
    }
  } else if (warp > kOzConsumers / 32) {
    // ---------------- metadata warps: one thread per tile row / column ----------------
    // For each task in ring order, into meta[ord & 1] once the consumers have released it:
    // the rows' and columns' slice exponents, every column's target supernode, the runs of
    // equal target (ballot per 32 columns), each column's run and column inside its target,
    // per run the relative-map base and target panel, and the relative rows of the first
    // kOzMaxRuns runs.  Thread 0 alone waits on the ring and on the buffer, so that the
    // group's decisions are uniform.
    const int mt = tid - (kOzConsumers + 32), mwarp = mt >> 5;
    for (int ord = 0;; ord++) {
      const int buf = ord & 1;
      if (mt == 0) {
        const int rs = ord % kOzRing;
        int tq = ntasks;
        if (!oz_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kOzRing) & 1)) ||
            (ring[rs] < ntasks && ord >= 2 &&
             !oz_wait(smem_u32(&meta_empty[buf]), (uint32_t)(((ord >> 1) - 1) & 1))))
          s_fail = 1;
        else
          tq = ring[rs];
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
      M.eB[mt] = gk < u ? exps[tk.w + gk] : 0;
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
    // Each wait's outcome is made uniform over the warp (tcgen05.ld is warp-collective).
    long long q = 0;
    const int i = 32 * (warp & 3) + lane;  // this thread's tile row
    const int c8 = 8 * (warp >> 2);        // this thread's 8 columns of a quarter
    for (int ord = 0;; ord++) {
      const int rs = ord % kOzRing, buf = ord & 1;
      if (!__all_sync(0xffffffffu, oz_wait(smem_u32(&ring_full[rs]), (uint32_t)((ord / kOzRing) & 1)))) {
        s_fail = 1;
        break;
      }
      if (ring[rs] >= ntasks) break;
      const OzMeta& M = meta[buf];
      if (!__all_sync(0xffffffffu, oz_wait(smem_u32(&meta_full[buf]), (uint32_t)((ord >> 1) & 1)))) {
        s_fail = 1;
        break;
      }
      const int u = M.u, i0 = M.i0, k0 = M.k0;
      const int nq = min(4, (u - k0 + kOzQ - 1) / kOzQ);
      const int gi = i0 + i;
      const int eA = M.eA[i];
      bool stop = false;
      for (int j = 0; j < nq; j++, q++) {
        const int b = (int)(q & 1);
        if (!__all_sync(0xffffffffu, oz_wait(smem_u32(&acc_full[b]), (uint32_t)((q >> 1) & 1)))) {
          s_fail = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // the 8 diagonals of this thread's 8 columns -> integers -> W = V_hi 2^20 +
        // round(V_lo / 2^8) (V_hi = sum_{d<4} D_d 2^(7(3-d)), V_lo = sum_{d>=4} D_d
        // 2^(7(7-d)), |D_d| < 2^22): U = W 2^(e_i + e_k - 55)
        double val[8];
        {
          long long vh[8], vl[8];
          const uint32_t ta =
              tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * kOzSetCols + c8);
          {
            uint32_t v[4][8];
#pragma unroll
            for (int dd = 0; dd < 4; dd++) oz_tmem_load8(ta + (uint32_t)(dd * kOzQ), v[dd]);
            oz_tmem_wait();
            oz_combine4(v, vh);
          }
          {
            uint32_t v[4][8];
#pragma unroll
            for (int dd = 0; dd < 4; dd++) oz_tmem_load8(ta + (uint32_t)((4 + dd) * kOzQ), v[dd]);
            oz_tmem_wait();
            oz_combine4(v, vl);
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) oz_arrive(smem_u32(&acc_empty[b]));
#pragma unroll
          for (int jj = 0; jj < 8; jj++) {
            const long long w = (long long)((unsigned long long)vh[jj] << 20) + ((vl[jj] + 128) >> 8);
            const int e = eA + M.eB[kOzQ * j + c8 + jj] - 55;
            val[jj] = oz_to_double(OWNER ? w : -w, e);
          }
        }
        // scatter this thread's row of the quarter (val holds -U for the atomics)
        if (gi < u) {
          const int kb = kOzQ * j + c8;
          if (OWNER) {
            double* U = M.ustage;
#pragma unroll
            for (int jj = 0; jj < 8; jj++) {
              const int gk = k0 + kb + jj;
              if (gk < u && gk <= gi) U[(int64_t)gk * u + gi] = val[jj];
            }
          } else {
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
              if (p >= 0) atomicAdd(M.cp[kk] + p, val[jj]);
            }
          }
        }
      }
      if (stop) break;
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

void launch_oz_slice(const int4* tasks, int ntasks, const SnDev* sns, void* oz, int64_t oz_rows,
                     cudaStream_t st) {
  if (ntasks <= 0) return;
  k_oz_slice<<<ntasks, kOzSliceThreads, (size_t)64 * kOzSliceLd * sizeof(double), st>>>(
      tasks, sns, static_cast<uint8_t*>(oz), oz_rows);
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
  if (cudaFuncSetAttribute(k_oz_slice, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(64 * kOzSliceLd * sizeof(double))) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kOzSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_schur_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kOzSmem) != cudaSuccess)
    return CHOL_E_CUDA;
  return CHOL_OK;
}

}  // namespace chol
