// Minimal three-point pose (P3P) of the pose M-step (Eq. 7 of VOLDOR+) in
// double-float arithmetic (vd_df64.cuh): Grunert's distance formulation as
// reviewed by Haralick et al. (IJCV 1994), the same polynomial as the
// float64 solver of vd_geom64.cuh.
//
// With unit bearings f_i, squared side lengths a2 = |X1 X2|^2,
// b2 = |X0 X2|^2, c2 = |X0 X1|^2 and the cosines ca = f1.f2, cb = f0.f2,
// cg = f0.f1, the distances s2 = u s1, s3 = v s1 satisfy two conics in
// (u, v); their resultant in u is a quartic in v.  Every real root v > 0
// with u > 0 gives the camera-frame triangle s_i f_i, and the rigid motion
// maps the world triangle onto it.
//
// Roots: the quartic shifted to its roots' centroid (double-float), float32
// split points (roots of the shifted quartic's second and first
// derivatives), its signs at the split points in double-float, a float32
// bracketed Newton search per sign change, then bracketed double-float
// Newton steps on the factored resultant (quadratic convergence from the
// float32 estimate).
#pragma once

#include "vd_df64.cuh"

// The solver's steps are inlined on the device: out-of-line calls (arrays
// passed through local memory) measured 1.4x slower per P3P launch.
#ifdef __CUDA_ARCH__
#define VD_DF_CALL __forceinline__
#else
#define VD_DF_CALL inline
#endif

struct VdP3Pdf {
  vd_df f[9];                      // unit bearings
  vd_df a2, b2, c2, ca, cb, cg;
  vd_df omcb;                      // 1 - cb = |f0 - f2|^2 / 2, without cancellation
  vd_df A[3], B[2], C[4];          // the resultant is A(v)^2 - B(v) C(v)
};

VD_HD __forceinline__ vd_df vd_df_dot3(const vd_df* a, const vd_df* b) {
  return vd_df_add(vd_df_add(vd_df_mul(a[0], b[0]), vd_df_mul(a[1], b[1])), vd_df_mul(a[2], b[2]));
}

VD_HD __forceinline__ void vd_df_normalize3(vd_df* v) {
  const vd_df r = vd_df_rsqrt(vd_df_dot3(v, v));
  v[0] = vd_df_mul(v[0], r);
  v[1] = vd_df_mul(v[1], r);
  v[2] = vd_df_mul(v[2], r);
}

VD_HD __forceinline__ void vd_df_cross3(const vd_df* a, const vd_df* b, vd_df* o) {
  o[0] = vd_df_sub(vd_df_mul(a[1], b[2]), vd_df_mul(a[2], b[1]));
  o[1] = vd_df_sub(vd_df_mul(a[2], b[0]), vd_df_mul(a[0], b[2]));
  o[2] = vd_df_sub(vd_df_mul(a[0], b[1]), vd_df_mul(a[1], b[0]));
}

VD_HD __forceinline__ vd_df vd_df_dist2(const vd_df* X, int i, int k) {
  const vd_df a = vd_df_sub(X[3 * i], X[3 * k]);
  const vd_df b = vd_df_sub(X[3 * i + 1], X[3 * k + 1]);
  const vd_df c = vd_df_sub(X[3 * i + 2], X[3 * k + 2]);
  return vd_df_add(vd_df_add(vd_df_mul(a, a), vd_df_mul(b, b)), vd_df_mul(c, c));
}

// The instance and its quartic res[0..4] (low order first); false for a
// degenerate triangle (a side of length 0).
VD_HD VD_DF_CALL bool vd_p3p_df_quartic(const vd_df* fin, const vd_df* X, VdP3Pdf* g,
                                            vd_df* res) {
  for (int i = 0; i < 9; ++i) g->f[i] = fin[i];
  vd_df_normalize3(g->f);
  vd_df_normalize3(g->f + 3);
  vd_df_normalize3(g->f + 6);
  const vd_df* f = g->f;
  const vd_df a2 = vd_df_dist2(X, 1, 2), b2 = vd_df_dist2(X, 0, 2), c2 = vd_df_dist2(X, 0, 1);
  g->a2 = a2;
  g->b2 = b2;
  g->c2 = c2;
  if (!(vd_df_gt0(a2) && vd_df_gt0(b2) && vd_df_gt0(c2))) return false;
  const vd_df ca = vd_df_dot3(f + 3, f + 6), cb = vd_df_dot3(f, f + 6), cg = vd_df_dot3(f, f + 3);
  g->ca = ca;
  g->cb = cb;
  g->cg = cg;
  {
    vd_df e[3];
    for (int i = 0; i < 3; ++i) e[i] = vd_df_sub(f[i], f[6 + i]);
    g->omcb = vd_df_mulf(vd_df_dot3(e, e), 0.5f);
  }
  // conics p2 u^2 + p1 u + p0 and q2 u^2 + q1 u + q0, coefficients in v:
  //   p2 = -b2, p1 = 2 b2 cg, p0 = c2 (1 + v^2 - 2 v cb) - b2
  //   q2 = b2, q1 = -2 b2 ca v, q0 = b2 v^2 - a2 (1 + v^2 - 2 v cb)
  // resultant (p2 q0 - p0 q2)^2 - (p2 q1 - p1 q2)(p1 q0 - p0 q1) = A^2 - B C
  const vd_df two_b2 = vd_df_mulf(b2, 2.0f);
  const vd_df b2cg2 = vd_df_mul(two_b2, cg);                 // 2 b2 cg = p1
  const vd_df b2ca2 = vd_df_mul(two_b2, ca);                 // 2 b2 ca
  const vd_df c2cb2 = vd_df_mulf(vd_df_mul(c2, cb), 2.0f);   // 2 c2 cb
  const vd_df a2cb2 = vd_df_mulf(vd_df_mul(a2, cb), 2.0f);   // 2 a2 cb
  const vd_df p0[3] = {vd_df_sub(c2, b2), vd_df_neg(c2cb2), c2};
  const vd_df q0[3] = {vd_df_neg(a2), a2cb2, vd_df_sub(b2, a2)};
  // A = p2 q0 - p0 q2 = -b2 (q0 + p0)
  vd_df A[3];
  for (int i = 0; i < 3; ++i) A[i] = vd_df_neg(vd_df_mul(b2, vd_df_add(q0[i], p0[i])));
  // B = p2 q1 - p1 q2 = (-2 b2^2 cg, 2 b2^2 ca)
  const vd_df B0 = vd_df_neg(vd_df_mul(b2cg2, b2));
  const vd_df B1 = vd_df_mul(b2ca2, b2);
  // C = p1 q0 - p0 q1, q1 = (0, -2 b2 ca)
  vd_df C[4];
  C[0] = vd_df_mul(b2cg2, q0[0]);
  C[1] = vd_df_add(vd_df_mul(b2cg2, q0[1]), vd_df_mul(b2ca2, p0[0]));
  C[2] = vd_df_add(vd_df_mul(b2cg2, q0[2]), vd_df_mul(b2ca2, p0[1]));
  C[3] = vd_df_mul(b2ca2, p0[2]);
  for (int i = 0; i < 3; ++i) g->A[i] = A[i];
  g->B[0] = B0;
  g->B[1] = B1;
  for (int i = 0; i < 4; ++i) g->C[i] = C[i];
  res[0] = vd_df_sub(vd_df_mul(A[0], A[0]), vd_df_mul(B0, C[0]));
  res[1] = vd_df_sub(vd_df_mulf(vd_df_mul(A[0], A[1]), 2.0f),
                     vd_df_add(vd_df_mul(B0, C[1]), vd_df_mul(B1, C[0])));
  res[2] = vd_df_sub(vd_df_add(vd_df_mul(A[1], A[1]), vd_df_mulf(vd_df_mul(A[0], A[2]), 2.0f)),
                     vd_df_add(vd_df_mul(B0, C[2]), vd_df_mul(B1, C[1])));
  res[3] = vd_df_sub(vd_df_mulf(vd_df_mul(A[1], A[2]), 2.0f),
                     vd_df_add(vd_df_mul(B0, C[3]), vd_df_mul(B1, C[2])));
  res[4] = vd_df_sub(vd_df_mul(A[2], A[2]), vd_df_mul(B1, C[3]));
  return true;
}

VD_HD __forceinline__ vd_df vd_df_poly(const vd_df* c, int deg, vd_df x) {
  vd_df r = c[deg];
  for (int i = deg - 1; i >= 0; --i) r = vd_df_add(vd_df_mul(r, x), c[i]);
  return r;
}

VD_HD __forceinline__ float vd_polyf(const float* c, int deg, float x) {
  float r = c[deg];
  for (int i = deg - 1; i >= 0; --i) r = fmaf(r, x, c[i]);
  return r;
}

// A bracketed root of a float32 polynomial that changes sign on [lo, hi]
// (neg_lo: its sign at lo): Newton steps, a bisection step where Newton
// leaves the bracket; at most 40 steps, stops at a 1e-6 relative step.
VD_HD VD_DF_CALL float vd_bracketed_rootf(const float* c, int deg, float lo, float hi,
                                               bool neg_lo) {
  float d[4];
  for (int i = 1; i <= deg; ++i) d[i - 1] = c[i] * (float)i;
  float x = 0.5f * (lo + hi);
  for (int it = 0; it < 40; ++it) {
    const float f = vd_polyf(c, deg, x);
    if (f == 0.0f) break;
    if ((f < 0.0f) == neg_lo) lo = x;
    else hi = x;
    const float g = vd_polyf(d, deg - 1, x);
    const float stp = g != 0.0f ? f / g : 0.0f;
    if (g != 0.0f && fabsf(stp) <= 1e-6f * fmaxf(1.0f, fabsf(x))) {
      x -= stp;
      break;
    }
    float xn = g != 0.0f ? x - stp : 0.5f * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    x = xn;
    if (hi - lo <= 1e-6f * fmaxf(1.0f, fabsf(lo))) break;
  }
  return x;
}

// Bound on the magnitude of every root of a float32 polynomial (Fujiwara).
VD_HD VD_DF_CALL float vd_root_boundf(const float* c, int deg) {
  float b = 0.0f;
  for (int i = 0; i < deg; ++i) {
    float r = fabsf(c[i] / c[deg]);
    if (i == 0) r *= 0.5f;
    const int k = deg - i;
    const float rt = k == 1 ? r : (k == 2 ? sqrtf(r) : (k == 3 ? cbrtf(r) : sqrtf(sqrtf(r))));
    b = fmaxf(b, rt);
  }
  return 2.0f * b * 1.001f + 1e-30f;
}

// Float32 roots of a polynomial of degree `deg` on the intervals cut by the
// sorted split points (one per sign change), ascending; at most ncrit + 1.
VD_HD VD_DF_CALL int vd_split_rootsf(const float* c, int deg, const float* crit, int ncrit,
                                          float* out) {
  const float bound = vd_root_boundf(c, deg);
  float lo = -bound, flo = vd_polyf(c, deg, lo);
  int n = 0;
  for (int i = 0; i <= ncrit; ++i) {
    const float hi = i < ncrit ? fminf(fmaxf(crit[i], -bound), bound) : bound;
    if (!(hi > lo)) continue;
    const float fhi = vd_polyf(c, deg, hi);
    if (flo == 0.0f) out[n++] = lo;
    else if ((flo < 0.0f) != (fhi < 0.0f) && fhi != 0.0f)
      out[n++] = vd_bracketed_rootf(c, deg, lo, hi, flo < 0.0f);
    lo = hi;
    flo = fhi;
  }
  return n;
}

// The resultant and its derivative at v in the factored form
// A(v)^2 - B(v) C(v): near a root A^2 and B C cancel, and the expanded
// quartic's coefficients cancel far more (to many digits on an
// ill-conditioned instance), so the polish evaluates the factors.
VD_HD VD_DF_CALL void vd_p3p_df_resultant(const VdP3Pdf& g, vd_df v, vd_df* r, vd_df* dr) {
  const vd_df a = vd_df_add(vd_df_mul(vd_df_add(vd_df_mul(g.A[2], v), g.A[1]), v), g.A[0]);
  const vd_df da = vd_df_add(vd_df_mulf(vd_df_mul(g.A[2], v), 2.0f), g.A[1]);
  const vd_df b = vd_df_add(vd_df_mul(g.B[1], v), g.B[0]);
  const vd_df c = vd_df_poly(g.C, 3, v);
  const vd_df dc = vd_df_add(vd_df_mul(vd_df_add(vd_df_mulf(vd_df_mul(g.C[3], v), 3.0f),
                                                 vd_df_mulf(g.C[2], 2.0f)), v), g.C[1]);
  *r = vd_df_sub(vd_df_mul(a, a), vd_df_mul(b, c));
  *dr = vd_df_sub(vd_df_mulf(vd_df_mul(a, da), 2.0f),
                  vd_df_add(vd_df_mul(g.B[1], c), vd_df_mul(b, dc)));
}

// The root of the resultant in [lo + m, hi + m] (lo, hi: a sign change of
// the shifted quartic, found in float32; m the shift) to double-float
// precision, from the float32 estimate x0 + m: Newton steps on the factored
// resultant inside a double-float bracket, a bisection step where Newton
// leaves it or gains less than a halving (clustered roots converge
// linearly); stops at a 2^-44 relative step or bracket, or once the Newton
// steps, below 2^-34 relative, stop halving (the resultant's double-float
// rounding noise: on an ill-conditioned instance the steps never reach
// 2^-44 and the bracket would otherwise be bisected down), at most 80 steps.
VD_HD VD_DF_CALL vd_df vd_p3p_df_polish(const VdP3Pdf& g, vd_df m, float x0, float lo_f,
                                             float hi_f) {
  vd_df lo = vd_df_add(vd_df_make(lo_f), m), hi = vd_df_add(vd_df_make(hi_f), m);
  vd_df r, dr;
  vd_p3p_df_resultant(g, lo, &r, &dr);
  const bool neg_lo = vd_df_lt0(r);
  vd_df x = vd_df_add(vd_df_make(fminf(fmaxf(x0, lo_f), hi_f)), m);
  float last = hi_f - lo_f;
  for (int it = 0; it < 80; ++it) {
    vd_p3p_df_resultant(g, x, &r, &dr);
    if (r.hi == 0.0f && r.lo == 0.0f) return x;
    if (vd_df_lt0(r) == neg_lo) lo = x;
    else hi = x;
    const float tol = 5.7e-14f * fmaxf(1.0f, fabsf(x.hi));
    vd_df xn, stp = vd_df_make(0.0f);
    bool newton = dr.hi != 0.0f;
    if (newton) {
      stp = vd_df_div(r, dr);
      if (fabsf(stp.hi) <= tol ||
          (fabsf(stp.hi) <= 1024.0f * tol && fabsf(stp.hi) >= 0.5f * last))
        return vd_df_sub(x, stp);
      xn = vd_df_sub(x, stp);
      newton = vd_df_gt0(vd_df_sub(xn, lo)) && vd_df_gt0(vd_df_sub(hi, xn)) &&
               fabsf(stp.hi) < 0.5f * last;
    }
    const vd_df w = vd_df_sub(hi, lo);
    if (!newton) {
      stp = vd_df_mulf(w, 0.5f);
      xn = vd_df_add(lo, stp);
    }
    last = fabsf(stp.hi);
    x = xn;
    if (fabsf(w.hi) <= tol) return x;
  }
  return x;
}

// The quartic shifted to its roots' centroid: d(w) = res(w + m) with
// m = -res3 / (4 res4) (the depressed quartic), by repeated synthetic
// division in double-float.  Roots that cluster (an ill-conditioned
// instance, the coefficients of res cancelling to many digits) become small
// roots of d, whose coefficients keep their own magnitudes, so a float32
// search on d's leading digits still separates them.
VD_HD VD_DF_CALL vd_df vd_df_taylor_shift(const vd_df* res, vd_df* d) {
  const vd_df m = vd_df_neg(vd_df_div(res[3], vd_df_mulf(res[4], 4.0f)));
  for (int i = 0; i <= 4; ++i) d[i] = res[i];
  for (int i = 0; i < 4; ++i)
    for (int j = 3; j >= i; --j) d[j] = vd_df_add(d[j], vd_df_mul(m, d[j + 1]));
  return m;
}

// The real roots of the quartic (res, double-float; leading coefficient not
// negligible), ascending; sequential form of the warp search of the pose
// kernel (same intervals, same searches), on the shifted quartic.
VD_HD __forceinline__ int vd_p3p_df_roots(const VdP3Pdf& g, const vd_df* res, vd_df* out) {
  float mx = 0.0f;
  for (int i = 0; i <= 4; ++i) mx = fmaxf(mx, fabsf(res[i].hi));
  if (!(mx > 0.0f) || !(fabsf(res[4].hi) > 1e-7f * mx)) return 0;
  vd_df d[5];
  const vd_df m = vd_df_taylor_shift(res, d);
  float cf[5];
  float dm = 0.0f;
  for (int i = 0; i <= 4; ++i) dm = fmaxf(dm, fabsf(d[i].hi));
  const float s = 1.0f / dm;          // float32 coefficients scaled to unit size
  for (int i = 0; i <= 4; ++i) cf[i] = d[i].hi * s;
  const float q[3] = {cf[2] * 2.0f, cf[3] * 6.0f, cf[4] * 12.0f};
  const float split = -q[1] / (2.0f * q[2]);
  float r2[2], r3[3];
  const int n2 = vd_split_rootsf(q, 2, &split, 1, r2);
  const float cc[4] = {cf[1], cf[2] * 2.0f, cf[3] * 3.0f, cf[4] * 4.0f};
  const int n3 = vd_split_rootsf(cc, 3, r2, n2, r3);
  // the shifted quartic's signs at the split points in double-float
  const float bound = vd_root_boundf(cf, 4);
  float lo = -bound;
  bool nlo = vd_df_lt0(vd_df_poly(d, 4, vd_df_make(lo)));
  bool zlo = false;
  int n = 0;
  for (int i = 0; i <= n3; ++i) {
    const float hi = i < n3 ? fminf(fmaxf(r3[i], -bound), bound) : bound;
    if (!(hi > lo)) continue;
    const vd_df fh = vd_df_poly(d, 4, vd_df_make(hi));
    const bool nhi = vd_df_lt0(fh), zhi = fh.hi == 0.0f && fh.lo == 0.0f;
    if (zlo) {
      out[n++] = vd_df_add(vd_df_make(lo), m);
    } else if (nlo != nhi && !zhi) {
      const float x0 = vd_bracketed_rootf(cf, 4, lo, hi, nlo);
      out[n++] = vd_p3p_df_polish(g, m, x0, lo, hi);
    }
    lo = hi;
    nlo = nhi;
    zlo = zhi;
  }
  return n;
}

// Triad of a triangle: columns e1 (p1 -> p2), e2 = e3 x e1, e3 (normal).
VD_HD VD_DF_CALL void vd_df_triad(const vd_df* p, vd_df* F) {
  vd_df e1[3], d[3], e3[3], e2[3];
  for (int i = 0; i < 3; ++i) {
    e1[i] = vd_df_sub(p[3 + i], p[i]);
    d[i] = vd_df_sub(p[6 + i], p[i]);
  }
  vd_df_cross3(e1, d, e3);
  vd_df_normalize3(e1);
  vd_df_normalize3(e3);
  vd_df_cross3(e3, e1, e2);
  for (int i = 0; i < 3; ++i) {
    F[3 * i + 0] = e1[i];
    F[3 * i + 1] = e2[i];
    F[3 * i + 2] = e3[i];
  }
}

// Pose (world -> camera, 3x4 row-major) of the root v; false if v gives no
// valid triangle (v <= 0, u <= 0 or a vanishing distance).  Fp: the triad
// of the world points X (vd_df_triad), the same for every root.
VD_HD VD_DF_CALL bool vd_p3p_df_pose(const VdP3Pdf& g, const vd_df* X, const vd_df* Fp, vd_df v,
                                      vd_df* T) {
  if (!vd_df_gt0(v)) return false;
  const vd_df one = vd_df_make(1.0f);
  const vd_df v2 = vd_df_mul(v, v);
  // 1 + v^2 - 2 v cb = (1 - v)^2 + 2 v (1 - cb): no cancellation for nearly
  // parallel bearings (cb -> 1) and v -> 1
  const vd_df omv = vd_df_sub(one, v);
  const vd_df dd = vd_df_add(vd_df_mul(omv, omv), vd_df_mulf(vd_df_mul(v, g.omcb), 2.0f));
  const vd_df pp0 = vd_df_sub(vd_df_mul(g.c2, dd), g.b2);
  const vd_df qq1 = vd_df_neg(vd_df_mulf(vd_df_mul(vd_df_mul(g.b2, g.ca), v), 2.0f));
  const vd_df qq0 = vd_df_sub(vd_df_mul(g.b2, v2), vd_df_mul(g.a2, dd));
  const vd_df den = vd_df_add(vd_df_mul(g.b2, vd_df_mulf(vd_df_mul(g.b2, g.cg), 2.0f)),
                              vd_df_mul(g.b2, qq1));
  if (!(fabsf(den.hi) > 1e-30f)) return false;
  const vd_df u = vd_df_div(vd_df_neg(vd_df_mul(g.b2, vd_df_add(qq0, pp0))), den);
  if (!vd_df_gt0(u) || !vd_df_gt0(dd)) return false;
  const vd_df s1 = vd_df_mul(g.b2, vd_df_rsqrt(vd_df_mul(g.b2, dd)));     // sqrt(b2 / dd)
  const vd_df s2 = vd_df_mul(u, s1), s3 = vd_df_mul(v, s1);
  vd_df Q[9];
  for (int i = 0; i < 3; ++i) {
    Q[i] = vd_df_mul(s1, g.f[i]);
    Q[3 + i] = vd_df_mul(s2, g.f[3 + i]);
    Q[6 + i] = vd_df_mul(s3, g.f[6 + i]);
  }
  vd_df Fq[9];
  vd_df_triad(Q, Fq);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k)
      T[4 * i + k] = vd_df_add(vd_df_add(vd_df_mul(Fq[3 * i], Fp[3 * k]),
                                         vd_df_mul(Fq[3 * i + 1], Fp[3 * k + 1])),
                               vd_df_mul(Fq[3 * i + 2], Fp[3 * k + 2]));
  for (int i = 0; i < 3; ++i)
    T[4 * i + 3] = vd_df_sub(Q[i], vd_df_add(vd_df_add(vd_df_mul(T[4 * i], X[0]),
                                                       vd_df_mul(T[4 * i + 1], X[1])),
                                             vd_df_mul(T[4 * i + 2], X[2])));
  return true;
}

// All solutions of one instance (sequential; the pose kernel spreads the
// same steps over a warp).  bearings and points as float64, poses out as
// float64 3x4.  Returns the number of poses (<= 4).
VD_HD __forceinline__ int vd_p3p_df_solve(const double* fin, const double* Xin, double* poses) {
  vd_df f[9], X[9], res[5], v[4], T[12];
  for (int i = 0; i < 9; ++i) {
    f[i] = vd_df_from(fin[i]);
    X[i] = vd_df_from(Xin[i]);
  }
  VdP3Pdf g;
  if (!vd_p3p_df_quartic(f, X, &g, res)) return 0;
  const int nr = vd_p3p_df_roots(g, res, v);
  vd_df Fp[9];
  vd_df_triad(X, Fp);
  int ns = 0;
  for (int r = 0; r < nr; ++r)
    if (vd_p3p_df_pose(g, X, Fp, v[r], T)) {
      for (int i = 0; i < 12; ++i) poses[12 * ns + i] = vd_df_to(T[i]);
      ++ns;
    }
  return ns;
}
