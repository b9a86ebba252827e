// Digit slicing shared by the split-precision kernels (sc_split.cu: mma.sync
// TRSM/SYRK; sc_syrk_tc.cu: the tcgen05 SYRK): exact power-of-two scalings,
// the 64-bit fixed point of an FP64 value against a column exponent bound,
// its signed 8-bit digits as BF16 values, and the exact integer combination
// of the digit-group sums (see the header comment of sc_split.cu).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace sc {
namespace digits {

// 2^e exactly, for e in the normal range (built from the bit pattern)
__device__ __forceinline__ double pow2i(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

__device__ __forceinline__ int biased_exponent(double y) {
  return (int)((__double_as_longlong(y) >> 52) & 0x7FF);
}

// 64-bit fixed point of |y| * 2^-(emax - 1022) * 2^63 (truncated), emax the
// column's largest biased exponent.  Returns 0 for y == 0.
__device__ __forceinline__ uint64_t fixed_point(double y, int emax) {
  const uint64_t bits = (uint64_t)__double_as_longlong(y);
  int e = (int)((bits >> 52) & 0x7FF);
  uint64_t mant = bits & ((1ull << 52) - 1);
  if (e) mant |= (1ull << 52);
  else e = 1;                                   // subnormal: same scale as e = 1
  const int sh = e - emax + 10;                 // <= 10 because e <= emax
  if (sh >= 0) return mant << sh;
  if (sh > -64) return mant >> (-sh);
  return 0;
}

__device__ __forceinline__ __nv_bfloat16 digit_bf16(uint64_t X, int t, bool neg) {
  const int u = (int)((X >> (55 - 8 * t)) & 0xFF);
  return __float2bfloat16_rn(neg ? -(float)u : (float)u);   // |u| <= 255: exact
}

// ---------------------------------------------------------------------------
// Exact combination of the digit-group sums I_d into sum_d I_d 2^(-8(d+2)).
// The groups are folded by Horner's rule into two int64 words,
//   H = sum_{d<h} I_d 256^(h-1-d),   Lo = sum_{d>=h} I_d 256^(S-1-d),
// so the value is H 2^(8(S-h)) + Lo, times 2^(-8(S+1)).
template <int S>
struct Groups {
  static constexpr int h = (S + 1) / 2;
  long long H = 0, Lo = 0;
  __device__ __forceinline__ void add(int d, int I) {       // Horner step, d ascending
    if (d < h) H = H * 256 + I;
    else Lo = Lo * 256 + I;
  }
  __device__ __forceinline__ void accumulate(int d, int I) {   // add I_d in place
    if (d < h) H += (long long)I << (8 * (h - 1 - d));
    else Lo += (long long)I << (8 * (S - 1 - d));
  }
  // |I_d| < 2^24 (one 32-row block): the sum needs 73 bits at most; drop the
  // lowest cut = 11 bits of Lo (2^-53 of the column-bound product) and
  // convert once.
  static constexpr int kBits = 24 + 8 * (S - 1) + 1;
  static constexpr int kCut = kBits > 62 ? kBits - 62 : 0;
  // the block value is block_int() * 2^kBlockShift
  static constexpr int kBlockShift = kCut - 8 * (S + 1);
  __device__ __forceinline__ long long block_int() const { return (H << (8 * (S - h) - kCut)) + (Lo >> kCut); }
  // |I_d| < 2^31 (many blocks): two conversions and one FMA
  __device__ __forceinline__ double value_wide() const {
    return fma((double)H, pow2i(8 * (S - h) - 8 * (S + 1)), (double)Lo * pow2i(-8 * (S + 1)));
  }
};

}  // namespace digits
}  // namespace sc
