// Double-float arithmetic for the FP64 basis of the mixed-precision solve.
//
// GB300 issues FP64 at about 1/58 of its FP32 rate, which makes the FP64
// rotation and Gram products of the second phase ALU-bound.  There a value
// x is carried as an unevaluated sum h + l of two FP32 numbers (h: x
// truncated to 24 significant bits, l: the remainder rounded to FP32, so
// h + l is x within 2^-53 relative) and a product-sum is accumulated with
// error-free transformations in FP32 (Dekker's product through a fused
// multiply-add, Knuth's two-sum), about 2^-48 relative per term: the
// accuracy of an FP64 dot product of the lengths used here (at most a few
// dozen terms), at a fraction of the FP64 issue cost.  The split and the
// join touch the FP64 pipe only for the final addition: they build the bit
// patterns with integer operations (64-bit conversions issue on the narrow
// FP64 pipe too).  Every operation is an explicit round-to-nearest
// intrinsic, so the compiler cannot contract a rounded product into an FMA
// and break an error-free step.
#pragma once
#include <cstdint>

namespace lapeig {

// x = h + l (within 2^-53 |x|) for 2^-126 <= |x| < 2^115; smaller |x| gives
// 0 (an absolute error below 2^-126), larger or non-finite x goes through the
// conversion instructions.
__device__ __forceinline__ void split64(double x, float& h, float& l) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const int E = (int)((hi32 >> 20) & 0x7FFu);
  const unsigned sign = hi32 & 0x80000000u;
  if (E < 897) {
    h = 0.f;
    l = 0.f;
    return;
  }
  if (E > 1138) {
    h = __double2float_rz(x);
    l = __double2float_rn(x - (double)h);
    return;
  }
  // h: the FP32 exponent E - 896 and the top 23 bits of the 52-bit fraction
  h = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
  // l: the low 29 fraction bits times 2^(E - 1075), as 2^-64 * 2^(E - 1011)
  const float r = __uint2float_rn(lo32 & 0x1FFFFFFFu);
  const float s2 = __uint_as_float((unsigned)(E - 884) << 23);
  const float lv = __fmul_rn(__fmul_rn(r, 0x1p-64f), s2);
  l = sign ? -lv : lv;
}

// (double)f for a normal or zero f built from its bits (an FP32 denormal,
// below 2^-126, counts as 0); infinities and NaN through the conversion.
__device__ __forceinline__ double widen32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  if (e == 0xFFu) return (double)f;
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double join64(float h, float l) { return __dadd_rn(widen32(h), widen32(l)); }

// (H, L) += (ah + al)(bh + bl): Dekker's exact product of the high parts,
// the cross terms in FP32 (al bl, below 2^-48 of the product, dropped) and
// Knuth's two-sum of the high part into H.
__device__ __forceinline__ void mac64(float& H, float& L, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float s = __fadd_rn(H, p);
  const float bb = __fsub_rn(s, H);
  const float err = __fadd_rn(__fsub_rn(H, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  H = s;
  L = __fadd_rn(L, __fadd_rn(err, e));
}

}  // namespace lapeig
