// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two float32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// Built on the error-free transformations of Knuth (TwoSum, TAOCP vol. 2,
// 4.2.2) and Dekker (FastTwoSum and the split product, "A floating-point
// technique for extending the available precision", Numer. Math. 1971), the
// product's error taken with a fused multiply-add.  On GB300 a float64
// operation costs a warp 64 cycles (a float32 one about 1.3), so where the
// pose M-step needs more than float32 it uses these on the float32 pipes.
#pragma once

#include <math.h>

#ifndef VD_HD
#define VD_HD __host__ __device__
#endif

struct vd_df {
  float hi, lo;
};

#ifdef __CUDA_ARCH__
#define VD_FADD(a, b) __fadd_rn((a), (b))
#define VD_FSUB(a, b) __fsub_rn((a), (b))
#define VD_FMUL(a, b) __fmul_rn((a), (b))
#else
#define VD_FADD(a, b) ((float)((a) + (b)))
#define VD_FSUB(a, b) ((float)((a) - (b)))
#define VD_FMUL(a, b) ((float)((a) * (b)))
#endif

VD_HD __forceinline__ vd_df vd_df_make(float hi, float lo = 0.0f) { return vd_df{hi, lo}; }

// a + b = s + e exactly (TwoSum, any magnitudes).
VD_HD __forceinline__ vd_df vd_two_sum(float a, float b) {
  const float s = VD_FADD(a, b);
  const float bb = VD_FSUB(s, a);
  const float e = VD_FADD(VD_FSUB(a, VD_FSUB(s, bb)), VD_FSUB(b, bb));
  return vd_df{s, e};
}

// a + b = s + e exactly when |a| >= |b| or a == 0 (FastTwoSum).
VD_HD __forceinline__ vd_df vd_fast_two_sum(float a, float b) {
  const float s = VD_FADD(a, b);
  return vd_df{s, VD_FSUB(b, VD_FSUB(s, a))};
}

// a * b = p + e exactly (the error by a fused multiply-add).
VD_HD __forceinline__ vd_df vd_two_prod(float a, float b) {
  const float p = VD_FMUL(a, b);
  return vd_df{p, fmaf(a, b, -p)};
}

VD_HD __forceinline__ vd_df vd_df_add(vd_df x, vd_df y) {
  vd_df s = vd_two_sum(x.hi, y.hi);
  const vd_df t = vd_two_sum(x.lo, y.lo);
  s.lo = VD_FADD(s.lo, t.hi);
  s = vd_fast_two_sum(s.hi, s.lo);
  s.lo = VD_FADD(s.lo, t.lo);
  return vd_fast_two_sum(s.hi, s.lo);
}

VD_HD __forceinline__ vd_df vd_df_neg(vd_df x) { return vd_df{-x.hi, -x.lo}; }

VD_HD __forceinline__ vd_df vd_df_sub(vd_df x, vd_df y) { return vd_df_add(x, vd_df_neg(y)); }

VD_HD __forceinline__ vd_df vd_df_mul(vd_df x, vd_df y) {
  vd_df p = vd_two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return vd_fast_two_sum(p.hi, p.lo);
}

VD_HD __forceinline__ vd_df vd_df_mulf(vd_df x, float y) {
  vd_df p = vd_two_prod(x.hi, y);
  p.lo = fmaf(x.lo, y, p.lo);
  return vd_fast_two_sum(p.hi, p.lo);
}

// x * y + z
VD_HD __forceinline__ vd_df vd_df_fma(vd_df x, vd_df y, vd_df z) {
  return vd_df_add(vd_df_mul(x, y), z);
}

// 1 / x: float reciprocal, then one Newton step in df (r + r (1 - x r)).
VD_HD __forceinline__ vd_df vd_df_rcp(vd_df x) {
  const float r0 = 1.0f / x.hi;
  const vd_df e = vd_df_sub(vd_df_make(1.0f), vd_df_mulf(x, r0));   // 1 - x r0
  return vd_df_add(vd_df_make(r0), vd_df_mulf(e, r0));
}

VD_HD __forceinline__ vd_df vd_df_div(vd_df a, vd_df b) { return vd_df_mul(a, vd_df_rcp(b)); }

// 1 / sqrt(x), x > 0: float estimate, one Newton step in df
// (r + r (1 - x r^2) / 2).
VD_HD __forceinline__ vd_df vd_df_rsqrt(vd_df x) {
  const float r0 = 1.0f / sqrtf(x.hi);
  const vd_df xr2 = vd_df_mulf(vd_df_mulf(x, r0), r0);
  const vd_df e = vd_df_sub(vd_df_make(1.0f), xr2);
  return vd_df_add(vd_df_make(r0), vd_df_mulf(e, 0.5f * r0));
}

// df from a float64 value (exact to 48 bits) and back.
VD_HD __forceinline__ vd_df vd_df_from(double d) {
  const float hi = (float)d;
  return vd_df{hi, (float)(d - (double)hi)};
}
VD_HD __forceinline__ double vd_df_to(vd_df x) { return (double)x.hi + (double)x.lo; }

VD_HD __forceinline__ bool vd_df_gt0(vd_df x) { return x.hi > 0.0f || (x.hi == 0.0f && x.lo > 0.0f); }
VD_HD __forceinline__ bool vd_df_lt0(vd_df x) { return x.hi < 0.0f || (x.hi == 0.0f && x.lo < 0.0f); }
