// oz_common.cuh -- the operand slicing shared by the FP64 tensor-core kernels (the Schur
// tiles' L21 rows, the TRSM's A21 rows and the rows of the diagonal-block inverses).
//
// A row r with exponent e_r (every |x| < 2^e_r) is the 56-bit fixed-point integer
// x 2^(56-e_r) per entry, cut into kOzSlices balanced digits of 7 bits (|s_0| <= 128,
// |s_p| <= 64, exact), x = 2^e_r sum_p s_p 2^(-7(p+1)) + (error < 2^(e_r-56)),
// each digit stored as bf16 (exact) in slice planes of 128-byte rows (64 entries, K <= 64)
// whose 16-byte chunks are pre-swizzled for the tensor cores' 128-byte swizzle: the chunk of
// columns 8c .. 8c+7 of slice row R sits at physical chunk c ^ (R & 7).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "chol_internal.h"

namespace chol {

// FP32 bits of an integer v with |v| < 2^22: 1.5 2^23 + v has the bits 0x4B400000 + v, and
// subtracting 1.5 2^23 leaves v exactly.  For |v| <= 256 the low 16 bits are zero, so the
// high half is v in bf16 (exact).
__device__ __forceinline__ uint32_t oz_f32_bits_of_int(int v) {
  return __float_as_uint(__uint_as_float(0x4B400000u + (uint32_t)v) - 12582912.0f);
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
// Digits, least significant first: d = ((R + 64) mod 128) - 64 in [-64, 63], then R = (R - d)
// / 2^7 (exact); digit 0 takes what is left, |s_0| <= 128 because |R| < 2^56 and the lower
// digits sum to less than 2^48 (128/127) in magnitude.  R = hi 2^28 + lo (0 <= lo < 2^28)
// keeps the work in 32-bit integers: lo gives digits 7 .. 4 and a carry (0 or 1) into hi,
// which gives digits 3 .. 0.
__device__ __forceinline__ void oz_write_chunk(long long (&R)[8], uint8_t* dst, size_t stride) {
  static_assert(kOzSlices == 8, "digits 7..4 from the low 28 bits, 3..0 from the rest");
  int lo[8], hi[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    lo[j] = (int)(R[j] & 0x0FFFFFFFll);
    hi[j] = (int)(R[j] >> 28);
  }
#pragma unroll
  for (int p = kOzSlices - 1; p >= 0; p--) {
    uint32_t h[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      int dg;
      if (p >= 4) {
        dg = ((lo[j] + 64) & 127) - 64;
        lo[j] = (lo[j] - dg) >> 7;
        if (p == 4) hi[j] += lo[j];  // the carry
      } else if (p >= 1) {
        dg = ((hi[j] + 64) & 127) - 64;
        hi[j] = (hi[j] - dg) >> 7;
      } else {
        dg = hi[j];
      }
      h[j] = oz_f32_bits_of_int(dg);
    }
    uint4 v;  // bf16 pairs: column 2t in the low half, 2t + 1 in the high half
    v.x = __byte_perm(h[0], h[1], 0x7632);
    v.y = __byte_perm(h[2], h[3], 0x7632);
    v.z = __byte_perm(h[4], h[5], 0x7632);
    v.w = __byte_perm(h[6], h[7], 0x7632);
    *reinterpret_cast<uint4*>(dst + p * stride) = v;
  }
}

}  // namespace chol
