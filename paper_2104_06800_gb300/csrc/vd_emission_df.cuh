// Projected positions of the rigidness emissions in double-float (hi, lo
// pairs of float32, vd_df64.cuh): the ray of a pixel, its homogeneous image
// point K (R r + rho tau) in frame t, the camera-plane test, the
// dehomogenised position, the image-border test and the bilinear tap of a
// position.  Host and device code, so that the CPU test-suite checks them
// against the float64 definitions.
//
// Why: the posterior of a rigidness chain (Sec. III-A, the E-step's
// forward-backward) reacts to an emission's rounding wherever the flow is
// steep (a depth edge moves the bilinear sample by tens of px per px of
// position) or a position lies on an image border or the camera plane;
// float32 positions (~1e-3 px off at 1216 px) put such entries outside 1e-4
// of the exact chain.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "vd_df64.cuh"

// 1 / x rounded to nearest (the correctly rounded reciprocal on both sides)
VD_HD __forceinline__ float vd_em_rcp(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}

// A short dot product accumulated in about twice the working precision: each
// product's rounding error recovered with a fused multiply-add, each sum's
// with TwoSum, all low parts and cross terms gathered in one float (the
// compensated dot product "Dot2" of Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005).
struct VdEmDot2 {
  float s, e;
  VD_HD __forceinline__ explicit VdEmDot2(float2 z) : s(z.x), e(z.y) {}
  VD_HD __forceinline__ void add(float2 a, vd_df b) {   // a * b, both double-float
    const vd_df p = vd_two_prod(a.x, b.hi);
    const vd_df t = vd_two_sum(s, p.hi);
    s = t.hi;
    e = fmaf(a.x, b.lo, fmaf(a.y, b.hi, e + (t.lo + p.lo)));
  }
  VD_HD __forceinline__ void add(float2 a, float b) {   // a * b, b a float
    const vd_df p = vd_two_prod(a.x, b);
    const vd_df t = vd_two_sum(s, p.hi);
    s = t.hi;
    e = fmaf(a.y, b, e + (t.lo + p.lo));
  }
  VD_HD __forceinline__ vd_df get() const { return vd_two_sum(s, e); }
};

// n / d for double-float n, d (d != 0; r = 1 / d.hi rounded): a float
// quotient, then one correction from the remainder n - q d.
VD_HD __forceinline__ vd_df vd_em_div(vd_df n, vd_df d, float r) {
  const float q = VD_FMUL(n.hi, r);
  const float rem = fmaf(-q, d.lo, fmaf(-q, d.hi, n.hi) + n.lo);
  return vd_fast_two_sum(q, rem * r);
}

// The float nearest to a - b (double-float a, b).
VD_HD __forceinline__ float vd_em_diff(vd_df a, vd_df b) {
  const vd_df s = vd_two_sum(a.hi, -b.hi);
  return VD_FADD(s.hi, s.lo + (a.lo - b.lo));
}

// a > b for normalised double-float values (|lo| <= ulp(hi) / 2).
VD_HD __forceinline__ bool vd_em_gt(vd_df a, float bhi, float blo) {
  return a.hi > bhi || (a.hi == bhi && a.lo > blo);
}

// 0 <= x <= W - 1 and 0 <= y <= H - 1, exactly
VD_HD __forceinline__ bool vd_em_inside(vd_df x, vd_df y, int W, int H) {
  const float xm = (float)(W - 1), ym = (float)(H - 1);
  return (x.hi > 0.0f || (x.hi == 0.0f && x.lo >= 0.0f)) &&
         (x.hi < xm || (x.hi == xm && x.lo <= 0.0f)) &&
         (y.hi > 0.0f || (y.hi == 0.0f && y.lo >= 0.0f)) &&
         (y.hi < ym || (y.hi == ym && y.lo <= 0.0f));
}

// The bilinear tap of an inside coordinate x in [0, n - 1] (n >= 2):
// x0 = min(floor(x), n - 2) and the weight x - x0 as a float (the last
// column or row is reached with weight 1).
VD_HD __forceinline__ int vd_em_tap(vd_df x, int n, float* w) {
  float f = floorf(x.hi);
  if (f == x.hi && x.lo < 0.0f) f -= 1.0f;
  float a = (x.hi - f) + x.lo;
  int x0 = (int)f;
  if (x0 > n - 2) {   // x = n - 1 exactly
    a += (float)(x0 - (n - 2));
    x0 = n - 2;
  }
  *w = a;
  return x0;
}

// The camera plane z = 1e-6 as a double-float pair.
#define VD_EM_ZHI ((float)1e-6)
#define VD_EM_ZLO ((float)(1e-6 - (double)VD_EM_ZHI))

// The calibrated ray ((u - cx) / fx, (v - cy) / fy) from the double-float
// intrinsics kdf (fx, fy, cx, cy, 1/fx, 1/fy as (hi, lo) pairs).
VD_HD __forceinline__ void vd_em_ray(const float* kdf, int u, int v, vd_df* rx, vd_df* ry) {
  const vd_df cx = vd_df_make(kdf[4], kdf[5]), cy = vd_df_make(kdf[6], kdf[7]);
  const vd_df ifx = vd_df_make(kdf[8], kdf[9]), ify = vd_df_make(kdf[10], kdf[11]);
  *rx = vd_df_mul(vd_df_sub(vd_df_make((float)u), cx), ifx);
  *ry = vd_df_mul(vd_df_sub(vd_df_make((float)v), cy), ify);
}

// Frame t's image point of the ray (rx, ry, 1) at inverse depth c through
// the double-float rows M = K [R | tau] (entries 0..8 the 3 x 3 part by
// rows, 9..11 the last column): in front of the camera (z > 1e-6) it sets
// (x, y) and returns true; behind it leaves them.
VD_HD __forceinline__ bool vd_em_project(const float2* M, vd_df rx, vd_df ry, float c, vd_df* x,
                                         vd_df* y) {
  VdEmDot2 hx(M[2]), hy(M[5]), hz(M[8]);
  hx.add(M[0], rx), hy.add(M[3], rx), hz.add(M[6], rx);
  hx.add(M[1], ry), hy.add(M[4], ry), hz.add(M[7], ry);
  hx.add(M[9], c), hy.add(M[10], c), hz.add(M[11], c);
  const vd_df Z = hz.get();
  if (!vd_em_gt(Z, VD_EM_ZHI, VD_EM_ZLO)) return false;
  const float r = vd_em_rcp(Z.hi);
  *x = vd_em_div(hx.get(), Z, r);
  *y = vd_em_div(hy.get(), Z, r);
  return true;
}
