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
// memory (coalesced loads); a row's exponent e_r is that of its largest entry; each
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
  for (int idx = threadIdx.x; idx < n * kOzM; idx += kOzSliceThreads) {
    const int k = idx / kOzM, i = idx - k * kOzM;
    xs[k * kOzSliceLd + i] = (r0 + i < u) ? L[(int64_t)k * m + i] : 0.0;
  }
  __syncthreads();
  const int64_t row0 = tk.z + (int64_t)r0;
  const size_t stride = (size_t)oz_rows * kOzRowBytes;
  if (threadIdx.x < kOzM) {
    const int i = threadIdx.x;
    double amax = 0.0;
    for (int k = 0; k < n; k++) amax = fmax(amax, fabs(xs[k * kOzSliceLd + i]));
    // amax = f 2^e with f in [0.5, 1): the exponent field minus 1022 (0 for zero rows)
    const int e = amax > 0.0 ? (int)((__double_as_longlong(amax) >> 52) & 0x7FF) - 1022 : 0;
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


// W 2^E as a double, rounded to nearest (ties to even), with integer operations only (the
// FP64 pipe is the scarce unit); results outside the normal range go through ldexp.
__device__ __forceinline__ double oz_to_double(long long W, int E) {
  if (W == 0) return 0.0;
  const unsigned long long sign = W < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = W < 0 ? (unsigned long long)(-W) : (unsigned long long)W;
  const int lz = __clzll((long long)a);
  a <<= lz;  // leading one at bit 63: W = a 2^(-lz)
  unsigned long long mant = a >> 11;
  const unsigned long long rem = a & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) mant++;
  int e2 = 63 - lz;  // |W| = mant 2^(e2 - 52)
  if (mant >> 53) {
    mant >>= 1;
    e2++;
  }
  const int be = e2 + E + 1023;
  if (be <= 0 || be >= 2047) return ldexp((double)W, E);
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1))));
}

constexpr int kOzMaxRuns = 16;  // column targets per task whose relative rows are cached

// Per-task metadata, double-buffered: a task's scatter reads one copy while the next
// task's is being built.
struct OzMeta {
  int eA[kOzM], eB[2 * kOzN];
  int tcol[2 * kOzN], run[2 * kOzN], col[2 * kOzN];
  int run_start[2 * kOzN + 1];
  double* rL[kOzMaxRuns];
  int rm[kOzMaxRuns];
  long long rb[2 * kOzN];  // relative-map base of every run
  int rp[kOzMaxRuns][kOzM];
  int nruns, next;
};

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
  __shared__ OzMeta meta[2];
  __shared__ int s_fail;
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
  // N = 64, 128, 192, 256: one MMA covers up to 4 consecutive B slices
  const uint32_t idesc[4] = {oz_idesc(kOzN), oz_idesc(2 * kOzN), oz_idesc(3 * kOzN),
                             oz_idesc(4 * kOzN)};
  const uint64_t da0 = oz_desc(smem_u32(A)), db0 = oz_desc(smem_u32(B));
  // thread 0 only: the load barrier's next phase, and what is in flight
  uint32_t ld_phase = 0;
  bool ld_inflight = false, mma_inflight = false;
  uint32_t ld_parity = 0, mma_parity = 0;
  uint32_t mma_phase = 0;  // every thread: parity of the next MMA commit

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
  // thread 0: wait for the operands, then D_{p+q} (+)= S_p S_q^T for every slice pair
  // p + q < kOzSlices.  The B slices lie one after another in shared memory, so one MMA of
  // S_p against slices q0 .. q0+3 (N up to 256) writes the accumulators of the diagonals
  // p+q0 .. p+q0+3 when its TMEM address starts at diagonal p + q0: 12 MMAs per K step
  // instead of 36 (the issue rate of a single thread, not the tensor cores, bounds small
  // MMAs).  A K step of 16 bf16 advances both descriptors by 32 bytes (2 in the address
  // field).  Returns false if the wait gave up.
  auto load_and_mma = [&](int ksteps) -> bool {
    if (!oz_wait(bld, ld_phase)) return false;
    ld_phase ^= 1;
    ld_inflight = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    for (int ks = 0; ks < ksteps; ks++)
      for (int p = 0; p < kOzSlices; p++)
        for (int q0 = 0; p + q0 < kOzSlices; q0 += 4) {
          const int nq = min(4, kOzSlices - p - q0);
          oz_mma(tmem + (uint32_t)((p + q0) * kOzN),
                 da0 + (uint64_t)((p * kOzASlice) >> 4) + 2 * ks,
                 db0 + (uint64_t)((q0 * kOzBSlice) >> 4) + 2 * ks, idesc[nq - 1],
                 (p > 0 || ks > 0) ? 1u : 0u);
        }
    oz_commit(bmma);
    mma_inflight = true;
    mma_parity = mma_phase;
    return true;
  };
  auto ksteps_of = [&](const int4& t) { return (sns[t.x].n + 15) >> 4; };

  int tq = blockIdx.x;
  if (tid == 0 && tq < ntasks) {
    issue_loads(tasks[tq], 0, true);
    if (!load_and_mma(ksteps_of(tasks[tq]))) s_fail = 1;
  }
  int buf = 0;
  while (tq < ntasks) {
    // the first half's MMAs of this task are running
    const int4 tk = tasks[tq];
    const SnDev d = sns[tk.x];
    const int n = d.n, u = d.m - n;
    const int i0 = tk.y, k0 = tk.z;
    const int ksteps = (n + 15) >> 4;
    const int nh = (k0 + kOzN < u) ? 2 : 1;
    const int32_t* rows = d.rows + n;
    const MatDev md = mats[d.mat];
    OzMeta& M = meta[buf];
    for (int i = tid; i < kOzM; i += kOzThreads) M.eA[i] = (i0 + i < u) ? exps[tk.w + i0 + i] : 0;
    for (int kk = tid; kk < 2 * kOzN; kk += kOzThreads) {
      const int gk = k0 + kk;
      M.eB[kk] = gk < u ? exps[tk.w + gk] : 0;
      M.tcol[kk] = gk < u ? md.col2sn[rows[gk]] : -1;
    }
    if (tid == 0) M.next = gridDim.x >= ntasks ? ntasks : gridDim.x + atomicAdd(queue, 1);
    __syncthreads();
    if (s_fail) break;
    if (!OWNER) {
      // runs of tile columns with one target (first warp, ballots), then the relative rows
      // of the tile rows inside the first kOzMaxRuns targets, while the tensor cores work
      if (warp == 0) {
        int nr = 0;
        for (int base = 0; base < 2 * kOzN; base += 32) {
          const int kk = base + lane;
          const bool live = k0 + kk < u;
          const bool start = live && (kk == 0 || M.tcol[kk] != M.tcol[kk - 1]);
          const unsigned b = __ballot_sync(0xffffffffu, start);
          if (start) M.run_start[nr + __popc(b & ((1u << lane) - 1u))] = kk;
          nr += __popc(b);
        }
        __syncwarp();
        if (lane == 0) M.nruns = nr;
        for (int r = lane; r < nr; r += 32) {
          const int kb = M.run_start[r];
          const int ke = r + 1 < nr ? M.run_start[r + 1] : min(2 * kOzN, u - k0);
          const SnDev& td = sns[md.sn_base + M.tcol[kb]];
          M.rb[r] = md.run_base[find_run(md, d, k0 + kb)];
          if (r < kOzMaxRuns) {
            M.rL[r] = reinterpret_cast<double*>(td.L);
            M.rm[r] = td.m;
          }
          for (int kk = kb; kk < ke; kk++) {
            M.run[kk] = r;
            M.col[kk] = rows[k0 + kk] - td.col0;
          }
        }
      }
      __syncthreads();
      const int nrc = min(M.nruns, kOzMaxRuns);
      for (int idx = tid; idx < nrc * kOzM; idx += kOzThreads) {
        const int r = idx / kOzM, i = idx - r * kOzM, gi = i0 + i;
        M.rp[r][i] = (gi < u && gi >= k0 + M.run_start[r]) ? md.relmap[M.rb[r] + gi] : -1;
      }
    }
    const int next = M.next;
    const int i = 32 * (warp & 3) + lane;  // this thread's tile row
    const int gi = i0 + i;
    const int eA = M.eA[i];
    const int c0 = 16 * (warp >> 2);       // this thread's 16 columns of a half
    bool stop = false;  // s_fail seen right after a barrier: the same in every thread
    for (int h = 0; h < nh; h++) {
      if (!oz_wait(bmma, mma_phase)) s_fail = 1;
      else if (tid == 0) mma_inflight = false;
      mma_phase ^= 1;
      __syncthreads();
      if (s_fail) {
        stop = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      // shared memory is free: start the next operands while the accumulators are read
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
        const uint32_t ta =
            tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + 8 * cc);
        {
          uint32_t v[4][8];
#pragma unroll
          for (int dd = 0; dd < 4; dd++) oz_tmem_load8(ta + (uint32_t)(dd * kOzN), v[dd]);
          oz_tmem_wait();
          oz_combine4(v, vh);
        }
        {
          uint32_t v[4][8];
#pragma unroll
          for (int dd = 0; dd < 4; dd++) oz_tmem_load8(ta + (uint32_t)((4 + dd) * kOzN), v[dd]);
          oz_tmem_wait();
          oz_combine4(v, vl);
        }
#pragma unroll
        for (int j = 0; j < 8; j++)
          val[8 * cc + j] = oz_to_double((long long)((unsigned long long)vh[j] << 20) +
                                             ((vl[j] + 128) >> 8),
                                         eA + M.eB[h * kOzN + c0 + 8 * cc + j] - 55);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      // tensor memory is free: the next MMAs (this task's second half, or the next task's
      // first) run during this half's scatter
      if (tid == 0) {
        if (h + 1 < nh) {
          if (!load_and_mma(ksteps)) s_fail = 1;
        } else if (next < ntasks) {
          if (!load_and_mma(ksteps_of(tasks[next]))) s_fail = 1;
        }
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
#pragma unroll
          for (int j = 0; j < 16; j++) {
            const int kk = kb + j, gk = k0 + kk;
            if (gk >= u || gk > gi) continue;
            const int r = M.run[kk];
            double* Lt;
            int mt, p;
            if (r < kOzMaxRuns) {
              Lt = M.rL[r];
              mt = M.rm[r];
              p = M.rp[r][i];
            } else {  // beyond the cached targets: read the relative map here
              const SnDev& td = sns[md.sn_base + M.tcol[kk]];
              Lt = reinterpret_cast<double*>(td.L);
              mt = td.m;
              p = md.relmap[M.rb[r] + gi];
            }
            if (p >= 0) atomicAdd(&Lt[(int64_t)M.col[kk] * mt + p], -val[j]);
          }
        }
      }
    }
    if (stop) break;
    buf ^= 1;
    tq = next;
  }
  __syncthreads();
  if (s_fail && tid == 0 && ntasks > 0) atomicAdd(mats[sns[tasks[min(tq, ntasks - 1)].x].mat].err + 3, 1ull);
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
