// oz_common.cuh -- the operand slicing shared by the FP64 tensor-core kernels (the Schur
// tiles' L21 rows, the TRSM's A21 rows and the rows of the diagonal-block inverses).
//
// A row r with exponent e_r (every |x| < 2^e_r) is the 56-bit fixed-point integer
// x 2^(56-e_r) per entry, cut into kOzSlices balanced digits of 7 bits (round to nearest:
// |s_0| <= 128, |s_p| <= 64, exact), x = 2^e_r sum_p s_p 2^(-7(p+1)) + (error < 2^(e_r-56)),
// each digit stored as bf16 (exact) in slice planes of 128-byte rows (64 entries, K <= 64)
// whose 16-byte chunks are pre-swizzled for the tensor cores' 128-byte swizzle: the chunk of
// columns 8c .. 8c+7 of slice row R sits at physical chunk c ^ (R & 7).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "chol_internal.h"

namespace chol {

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

// The exponent e of a row from the largest exponent field f among its entries (integer
// comparison, the FP64 unit is slow): max |x| = g 2^e with g in [0.5, 1) has e = f - 1022
// (0 for rows of zeros and subnormals, whose slices are zero).
__device__ __forceinline__ int oz_row_exponent(int max_field) {
  return max_field > 0 ? max_field - 1022 : 0;
}
__device__ __forceinline__ int oz_exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// The 16-byte chunk of logical columns 8c .. 8c+7 of one row in every slice plane: R[j] are
// the row's fixed-point integers of those columns (oz_fixed, 0 past the row's end); dst the
// chunk's address in plane 0, planes `stride` bytes apart.
__device__ __forceinline__ void oz_write_chunk(long long (&R)[8], uint8_t* dst, size_t stride) {
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

}  // namespace chol
