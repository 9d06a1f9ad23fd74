// Float64 device geometry used by the pose M-step (Eq. 7 of VOLDOR+) and the
// monocular bootstrap: SE(3) exponential and logarithm, the minimal 3-point
// pose solver, a polynomial real-root finder and a Jacobi eigen-solver.
// Poses are 3x4 row-major [R | tau] (12 doubles).
#pragma once

#include <math.h>

#ifndef VD_HD
#define VD_HD __host__ __device__
#endif

// ---------------------------------------------------------------- fast float64 division
// On the device a float64 divide or square root is a long instruction
// sequence on a narrow pipe.  For Newton steps and normalisations a float
// seed refined by float64 Newton iterations is enough: the relative error
// squares per step (2^-24 -> ~2^-48 -> below rounding).
VD_HD __forceinline__ double vd_rcp64(double x) {
#ifdef __CUDA_ARCH__
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = r * (2.0 - x * r);
  r = r * (2.0 - x * r);
  return r;
#else
  return 1.0 / x;
#endif
}

VD_HD __forceinline__ double vd_rsqrt64(double x) {
#ifdef __CUDA_ARCH__
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double r = (double)rsqrtf((float)x);
  r = r * (1.5 - 0.5 * x * r * r);
  r = r * (1.5 - 0.5 * x * r * r);
  return r;
#else
  return 1.0 / sqrt(x);
#endif
}

// ---------------------------------------------------------------- small algebra
VD_HD __forceinline__ void vd_compose(const double* A, const double* B, double* O) {
  // O = A o B (apply B first)
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      O[4 * r + c] = A[4 * r] * B[c] + A[4 * r + 1] * B[4 + c] + A[4 * r + 2] * B[8 + c];
    O[4 * r + 3] = A[4 * r] * B[3] + A[4 * r + 1] * B[7] + A[4 * r + 2] * B[11] + A[4 * r + 3];
  }
}

VD_HD __forceinline__ void vd_inverse(const double* T, double* O) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) O[4 * r + c] = T[4 * c + r];
  for (int r = 0; r < 3; ++r)
    O[4 * r + 3] = -(O[4 * r] * T[3] + O[4 * r + 1] * T[7] + O[4 * r + 2] * T[11]);
}

// Rodrigues: R = I + a [w]x + b [w]x^2 with a = sin(th)/th, b = (1-cos th)/th^2.
VD_HD __forceinline__ void vd_so3_coeffs(double th2, double* a, double* b, double* cc) {
  // cc = (th - sin th) / th^3 (for the left Jacobian V)
  if (th2 < 1e-12) {
    *a = 1.0 - th2 / 6.0;
    *b = 0.5 - th2 / 24.0;
    *cc = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double th = sqrt(th2);
    const double s = sin(th), c = cos(th);
    *a = s / th;
    *b = (1.0 - c) / th2;
    *cc = (th - s) / (th2 * th);
  }
}

VD_HD __forceinline__ void vd_se3_exp(const double* xi, double* T) {
  const double wx = xi[0], wy = xi[1], wz = xi[2];
  const double th2 = wx * wx + wy * wy + wz * wz;
  double a, b, cc;
  vd_so3_coeffs(th2, &a, &b, &cc);
  const double K[9] = {0, -wz, wy, wz, 0, -wx, -wy, wx, 0};
  double K2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
  double V[9];
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    T[4 * (i / 3) + (i % 3)] = I + a * K[i] + b * K2[i];
    V[i] = I + b * K[i] + cc * K2[i];
  }
  for (int r = 0; r < 3; ++r)
    T[4 * r + 3] = V[3 * r] * xi[3] + V[3 * r + 1] * xi[4] + V[3 * r + 2] * xi[5];
}

// so(3) logarithm (rotation vector) of a rotation given as the 3x3 part of T.
VD_HD __forceinline__ void vd_so3_log(const double* T, double* w) {
  const double tr = T[0] + T[5] + T[10];
  const double c = 0.5 * (tr - 1.0);
  const double vx = 0.5 * (T[9] - T[6]), vy = 0.5 * (T[2] - T[8]), vz = 0.5 * (T[4] - T[1]);
  const double s = sqrt(vx * vx + vy * vy + vz * vz);
  const double th = atan2(s, c);
  if (s < 1e-8) {
    if (c > 0.0) {
      const double f = 1.0 + th * th / 6.0;
      w[0] = vx * f;
      w[1] = vy * f;
      w[2] = vz * f;
      return;
    }
    // angle near pi: axis from the largest diagonal entry of (R + I) / 2
    double B[3] = {0.5 * (T[0] + 1.0), 0.5 * (T[5] + 1.0), 0.5 * (T[10] + 1.0)};
    int k = (B[1] > B[0]) ? 1 : 0;
    if (B[2] > B[k]) k = 2;
    const double d = sqrt(fmax(B[k], 1e-300));
    double ax[3];
    for (int i = 0; i < 3; ++i) {
      const double Rik = T[4 * i + k] + (i == k ? 1.0 : 0.0);
      ax[i] = 0.5 * Rik / d;
    }
    w[0] = ax[0] * M_PI;
    w[1] = ax[1] * M_PI;
    w[2] = ax[2] * M_PI;
    return;
  }
  const double f = th / s;
  w[0] = vx * f;
  w[1] = vy * f;
  w[2] = vz * f;
}

// se(3) logarithm: w = log R, v = V(w)^-1 tau with the closed-form inverse
// V^-1 = I - [w]x / 2 + (1/th^2) (1 - a / (2 b)) [w]x^2.
VD_HD __forceinline__ void vd_se3_log(const double* T, double* xi) {
  vd_so3_log(T, xi);
  const double wx = xi[0], wy = xi[1], wz = xi[2];
  const double th2 = wx * wx + wy * wy + wz * wz;
  double e;
  if (th2 < 1e-10) {
    e = 1.0 / 12.0 + th2 / 720.0;
  } else {
    const double th = sqrt(th2);
    const double a = sin(th) / th, b = (1.0 - cos(th)) / th2;
    e = (1.0 - a / (2.0 * b)) / th2;
  }
  const double K[9] = {0, -wz, wy, wz, 0, -wx, -wy, wx, 0};
  const double t0 = T[3], t1 = T[7], t2 = T[11];
  const double Kt[3] = {K[0] * t0 + K[1] * t1 + K[2] * t2, K[3] * t0 + K[4] * t1 + K[5] * t2,
                        K[6] * t0 + K[7] * t1 + K[8] * t2};
  const double K2t[3] = {K[0] * Kt[0] + K[1] * Kt[1] + K[2] * Kt[2],
                         K[3] * Kt[0] + K[4] * Kt[1] + K[5] * Kt[2],
                         K[6] * Kt[0] + K[7] * Kt[1] + K[8] * Kt[2]};
  xi[3] = t0 - 0.5 * Kt[0] + e * K2t[0];
  xi[4] = t1 - 0.5 * Kt[1] + e * K2t[1];
  xi[5] = t2 - 0.5 * Kt[2] + e * K2t[2];
}

// ---------------------------------------------------------------- polynomials
// Value of sum_i c[i] x^i.
VD_HD __forceinline__ double vd_poly_eval(const double* c, int deg, double x) {
  double r = c[deg];
  for (int i = deg - 1; i >= 0; --i) r = r * x + c[i];
  return r;
}

// Root of a polynomial known to change sign on [lo, hi]: safeguarded Newton
// (a Newton step that leaves the bracket becomes a bisection step).  The
// search first runs in float32 to about 1e-6 and then continues in float64
// from there inside the float64 bracket, so the float64 phase needs only a
// few steps; the bracket keeps the result a root of the float64 polynomial.
// fp64_steps caps the float64 phase: 0 returns the float32 estimate (enough
// for a split point between roots), a few steps polish a simple root to
// float64 precision (Newton doubles the correct digits per step).
static VD_HD double vd_poly_bracketed_root(const double* c, int deg, double lo, double hi,
                                           int fp64_steps = 40) {
  double d[4];
  for (int i = 1; i <= deg; ++i) d[i - 1] = c[i] * i;
  double flo = vd_poly_eval(c, deg, lo);
  double x = 0.5 * (lo + hi);
  {
    float cf[5], df[4];
    for (int i = 0; i <= deg; ++i) cf[i] = (float)c[i];
    for (int i = 0; i < deg; ++i) df[i] = (float)d[i];
    float l = (float)lo, h = (float)hi, xf = (float)x;
    const bool neg_lo = flo < 0.0;
    for (int it = 0; it < 60; ++it) {
      float f = cf[deg];
      for (int i = deg - 1; i >= 0; --i) f = f * xf + cf[i];
      if (f == 0.0f) break;
      if ((f < 0.0f) == neg_lo) l = xf;
      else h = xf;
      float g = df[deg - 1];
      for (int i = deg - 2; i >= 0; --i) g = g * xf + df[i];
      const float stp = g != 0.0f ? f / g : 0.0f;
      if (g != 0.0f && fabsf(stp) <= 1e-6f * fmaxf(1.0f, fabsf(xf))) {   // converged
        xf -= stp;
        break;
      }
      float xn = (g != 0.0f) ? xf - stp : 0.5f * (l + h);
      if (!(xn > l && xn < h)) xn = 0.5f * (l + h);
      xf = xn;
      if (h - l <= 1e-6f * fmaxf(1.0f, fabsf(l))) break;
    }
    if ((double)xf > lo && (double)xf < hi) x = (double)xf;
  }
  // float64 phase: Newton converges quadratically from the float32 estimate
  // for a simple root (two or three steps); clustered roots converge
  // linearly, hence the cap.  Stops at a 4-ulp step.
  for (int it = 0; it < fp64_steps; ++it) {
    const double f = vd_poly_eval(c, deg, x);
    if (f == 0.0) return x;
    if ((f < 0.0) == (flo < 0.0)) {
      lo = x;
      flo = f;
    } else {
      hi = x;
    }
    const double df = vd_poly_eval(d, deg - 1, x);
    const double stp = df != 0.0 ? f * vd_rcp64(df) : 0.0;
    // a step below rounding means convergence (testing it after the bracket
    // safeguard would turn the null step into a bisection jump)
    if (df != 0.0 && fabs(stp) <= 8.9e-16 * fmax(1.0, fabs(x))) return x - stp;
    double xn = (df != 0.0) ? x - stp : 0.5 * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (hi - lo <= 8.9e-16 * fmax(1.0, fabs(lo))) return 0.5 * (lo + hi);
    x = xn;
  }
  return x;
}

// An upper bound on the magnitude of every root (Fujiwara:
// 2 max(|c_{n-1}/c_n|, |c_{n-2}/c_n|^(1/2), ..., |c_0/(2 c_n)|^(1/n))),
// evaluated in float32 with a safety margin (a bound needs no precision).
VD_HD __forceinline__ double vd_root_bound(const double* c, int deg) {
  float bf = 0.0f;
  for (int i = 0; i < deg; ++i) {
    float r = fabsf((float)(c[i] / c[deg]));
    if (i == 0) r *= 0.5f;
    const int k = deg - i;
    const float root = k == 1 ? r : (k == 2 ? sqrtf(r) : (k == 3 ? cbrtf(r) : sqrtf(sqrtf(r))));
    bf = fmaxf(bf, root);
  }
  if (!(bf < 1e30f)) {   // out of float range: the float64 Cauchy bound
    double b = 0.0;
    for (int i = 0; i < deg; ++i) b = fmax(b, fabs(c[i] / c[deg]));
    return b + 1.0;
  }
  return 2.0 * (double)bf * 1.001 + 1e-30;
}

// Real roots of a polynomial of exact degree `deg` (leading coefficient
// non-zero) on the intervals cut by the sorted split points `crit` (the real
// roots of its derivative): one root per interval with a sign change.
// Writes at most ncrit + 1 roots.
VD_HD __forceinline__ int vd_roots_between(const double* c, int deg, const double* crit,
                                                int ncrit, double* out, int fp64_steps = 40) {
  const double bound = vd_root_bound(c, deg);
  double lo = -bound;
  double flo = vd_poly_eval(c, deg, lo);
  int n = 0;
  for (int i = 0; i <= ncrit; ++i) {
    double hi = i < ncrit ? fmin(fmax(crit[i], -bound), bound) : bound;
    if (!(hi > lo)) continue;
    const double fhi = vd_poly_eval(c, deg, hi);
    if (flo == 0.0) {
      out[n++] = lo;
    } else if ((flo < 0.0) != (fhi < 0.0) && fhi != 0.0) {
      out[n++] = vd_poly_bracketed_root(c, deg, lo, hi, fp64_steps);
    }
    lo = hi;
    flo = fhi;
  }
  return n;
}

// Cap of the float64 Newton steps that polish a quartic's root found by the
// float32 phase (two or three for a simple root; the loop stops at a 4-ulp
// step).  The split-point stages need no float64 digits.
#define VD_P3P_POLISH_STEPS 40

// Real roots of a quartic with a non-negligible leading coefficient, as
// vd_poly_real_roots isolates them (second derivative, first derivative,
// quartic), with float32 split points and the float64 phase on the roots
// of the quartic itself only.
static VD_HD int vd_quartic_real_roots_fast(const double* c, double* out) {
  const double q[3] = {c[2] * 2.0, c[3] * 6.0, c[4] * 12.0};
  const double split = -q[1] / (2.0 * q[2]);
  double r2[2];
  const int n2 = vd_roots_between(q, 2, &split, 1, r2, 0);
  const double cc[4] = {c[1], c[2] * 2.0, c[3] * 3.0, c[4] * 4.0};
  double r3[3];
  const int n3 = vd_roots_between(cc, 3, r2, n2, r3, 0);
  return vd_roots_between(c, 4, r3, n3, out, VD_P3P_POLISH_STEPS);
}

// All real roots of sum_{i<=deg} c[i] x^i for deg <= 4, ascending.  Real
// roots are isolated between consecutive real roots of the derivative; the
// degrees are handled one by one without recursion (no dynamic stack).
static VD_HD int vd_poly_real_roots(const double* cin, int deg, double* out) {
  double c[5];
  double mx = 0.0;
  for (int i = 0; i <= deg; ++i) {
    c[i] = cin[i];
    mx = fmax(mx, fabs(c[i]));
  }
  if (mx == 0.0) return 0;
  while (deg > 0 && fabs(c[deg]) <= 1e-14 * mx) --deg;
  if (deg == 0) return 0;
  if (deg == 1) {
    out[0] = -c[0] / c[1];
    return 1;
  }
  // quadratic: split at the vertex
  double r2[2];
  int n2;
  {
    const int dq = deg - 2;      // the (deg-2)-th derivative is a quadratic
    double q[3];
    // coefficients of the (deg-2)-th derivative of c
    for (int i = 0; i <= 2; ++i) {
      double f = 1.0;
      for (int k = 1; k <= dq; ++k) f *= (double)(i + k);
      q[i] = c[i + dq] * f;
    }
    if (deg == 2) {
      const double split = -q[1] / (2.0 * q[2]);
      return vd_roots_between(q, 2, &split, 1, out);
    }
    const double split = -q[1] / (2.0 * q[2]);
    n2 = vd_roots_between(q, 2, &split, 1, r2);
  }
  // cubic (the derivative of c when deg == 4, else c itself)
  double r3[3];
  int n3;
  {
    const int dc = deg - 3;
    double cc[4];
    for (int i = 0; i <= 3; ++i) cc[i] = dc ? c[i + 1] * (double)(i + 1) : c[i];
    if (deg == 3) return vd_roots_between(cc, 3, r2, n2, out);
    n3 = vd_roots_between(cc, 3, r2, n2, r3);
  }
  return vd_roots_between(c, 4, r3, n3, out);
}

// ---------------------------------------------------------------- P3P
// Grunert's distance formulation (Haralick et al. 1994): with s2 = u s1 and
// s3 = v s1 the law of cosines gives two conics in (u, v):
//   p(u) = -b2 u^2 + 2 b2 cg u + c2 (1 + v^2 - 2 v cb) - b2
//   q(u) =  b2 u^2 - 2 b2 ca v u + b2 v^2 - a2 (1 + v^2 - 2 v cb)
// Their resultant in u, (p2 q0 - p0 q2)^2 - (p2 q1 - p1 q2)(p1 q0 - p0 q1), is a
// quartic in v; each real positive root gives the camera-frame triangle, and
// the rigid motion follows from the two point triads.
VD_HD __forceinline__ void vd_pmul(const double* a, int da, const double* b, int db, double* o) {
  for (int i = 0; i <= da + db; ++i) o[i] = 0.0;
  for (int i = 0; i <= da; ++i)
    for (int k = 0; k <= db; ++k) o[i + k] += a[i] * b[k];
}

VD_HD __forceinline__ void vd_normalize3(double* v) {
  const double r = vd_rsqrt64(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] *= r;
  v[1] *= r;
  v[2] *= r;
}

VD_HD __forceinline__ void vd_cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Orthonormal frame of a triangle: e1 along p1->p2, e3 its normal, e2 = e3 x e1.
VD_HD __forceinline__ void vd_triad(const double* p1, const double* p2, const double* p3,
                                    double* F) {
  double e1[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
  double d[3] = {p3[0] - p1[0], p3[1] - p1[1], p3[2] - p1[2]};
  double e3[3];
  vd_cross3(e1, d, e3);
  vd_normalize3(e1);
  vd_normalize3(e3);
  double e2[3];
  vd_cross3(e3, e1, e2);
  for (int i = 0; i < 3; ++i) {  // columns e1, e2, e3
    F[3 * i + 0] = e1[i];
    F[3 * i + 1] = e2[i];
    F[3 * i + 2] = e3[i];
  }
}

// Rigid motion mapping the triangle X onto the congruent triangle Q
// (Q_i = R X_i + tau): R = F_Q F_X^T from the two triangles' frames.
VD_HD __forceinline__ void vd_triangle_motion(const double* X, const double* Q, double* T) {
  double Fp[9], Fq[9];
  vd_triad(X, X + 3, X + 6, Fp);
  vd_triad(Q, Q + 3, Q + 6, Fq);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k)
      T[4 * i + k] = Fq[3 * i] * Fp[3 * k] + Fq[3 * i + 1] * Fp[3 * k + 1] + Fq[3 * i + 2] * Fp[3 * k + 2];
  for (int i = 0; i < 3; ++i)
    T[4 * i + 3] = Q[i] - (T[4 * i] * X[0] + T[4 * i + 1] * X[1] + T[4 * i + 2] * X[2]);
}

// One P3P instance: unit bearings, squared side lengths (a: X1X2, b: X0X2,
// c: X0X1) and the cosines of the angles between the bearings.
struct VdP3P {
  double f[9];
  double a2, b2, c2, ca, cb, cg;
};

// Quartic of the instance (coefficients res[0..4], low order first); -1 for a
// degenerate triangle, else 0.  bearings f[3][3] (any length), points X[3][3].
static VD_HD int vd_p3p_quartic(const double* fin, const double* X, VdP3P* g, double* res);

// The quartic's real roots (<= 4, ascending); -1 for a degenerate triangle.
static VD_HD int vd_p3p_roots(const double* fin, const double* X, VdP3P* g, double* v) {
  double res[5];
  if (vd_p3p_quartic(fin, X, g, res) < 0) return -1;
  return vd_poly_real_roots(res, 4, v);
}

static VD_HD int vd_p3p_quartic(const double* fin, const double* X, VdP3P* g, double* res) {
  for (int i = 0; i < 9; ++i) g->f[i] = fin[i];
  vd_normalize3(g->f);
  vd_normalize3(g->f + 3);
  vd_normalize3(g->f + 6);
  const double* f = g->f;
  auto d2 = [&](int i, int k) {
    const double a = X[3 * i] - X[3 * k], b = X[3 * i + 1] - X[3 * k + 1], c = X[3 * i + 2] - X[3 * k + 2];
    return a * a + b * b + c * c;
  };
  const double a2 = d2(1, 2), b2 = d2(0, 2), c2 = d2(0, 1);
  g->a2 = a2;
  g->b2 = b2;
  g->c2 = c2;
  if (!(a2 > 0.0 && b2 > 0.0 && c2 > 0.0)) return -1;
  const double ca = f[3] * f[6] + f[4] * f[7] + f[5] * f[8];
  const double cb = f[0] * f[6] + f[1] * f[7] + f[2] * f[8];
  const double cg = f[0] * f[3] + f[1] * f[4] + f[2] * f[5];
  g->ca = ca;
  g->cb = cb;
  g->cg = cg;
  // coefficients as polynomials in v (low order first)
  const double p2[1] = {-b2}, p1[1] = {2.0 * b2 * cg};
  const double p0[3] = {c2 - b2, -2.0 * c2 * cb, c2};
  const double q2[1] = {b2}, q1[2] = {0.0, -2.0 * b2 * ca};
  const double q0[3] = {-a2, 2.0 * a2 * cb, b2 - a2};
  double A[3], B[2], C[4], tmp[4], tmp2[4];
  vd_pmul(p2, 0, q0, 2, A);
  vd_pmul(p0, 2, q2, 0, tmp);
  for (int i = 0; i < 3; ++i) A[i] -= tmp[i];
  vd_pmul(p2, 0, q1, 1, B);
  vd_pmul(p1, 0, q2, 0, tmp);
  B[0] -= tmp[0];
  vd_pmul(p1, 0, q0, 2, tmp);
  vd_pmul(p0, 2, q1, 1, tmp2);
  for (int i = 0; i < 4; ++i) C[i] = (i < 3 ? tmp[i] : 0.0) - tmp2[i];
  double bc[5];
  vd_pmul(A, 2, A, 2, res);
  vd_pmul(B, 1, C, 3, bc);
  for (int i = 0; i < 5; ++i) res[i] -= bc[i];
  return 0;
}

// Camera pose of one root v: u from the common root of the two conics,
// s1 = b / sqrt(1 + v^2 - 2 v cb), camera points s_i f_i, then the rigid
// motion of the triangle.  false if the root gives no valid triangle.
static VD_HD bool vd_p3p_pose(const VdP3P& g, const double* X, double v, double* T) {
  if (!(v > 0.0)) return false;
  const double a2 = g.a2, b2 = g.b2, c2 = g.c2, ca = g.ca, cb = g.cb, cg = g.cg;
  const double pp0 = c2 * (1.0 + v * v - 2.0 * v * cb) - b2;
  const double qq1 = -2.0 * b2 * ca * v;
  const double qq0 = b2 * v * v - a2 * (1.0 + v * v - 2.0 * v * cb);
  const double den = b2 * (2.0 * b2 * cg) + b2 * qq1;
  if (fabs(den) < 1e-300) return false;
  const double u = (-b2 * qq0 - b2 * pp0) * vd_rcp64(den);
  if (!(u > 0.0)) return false;
  const double dd = 1.0 + v * v - 2.0 * v * cb;
  if (!(dd > 0.0)) return false;
  const double s1 = b2 * vd_rsqrt64(b2 * dd);      // sqrt(b2 / dd)
  const double* f = g.f;
  const double Q[9] = {s1 * f[0], s1 * f[1], s1 * f[2],
                       u * s1 * f[3], u * s1 * f[4], u * s1 * f[5],
                       v * s1 * f[6], v * s1 * f[7], v * s1 * f[8]};
  vd_triangle_motion(X, Q, T);
  return true;
}

// All P3P solutions (<= 4 poses, world -> camera) of one instance.
static VD_HD int vd_p3p(const double* fin, const double* X, double* poses) {
  VdP3P g;
  double v[4];
  const int nr = vd_p3p_roots(fin, X, &g, v);
  int ns = 0;
  for (int r = 0; r < nr; ++r)
    if (vd_p3p_pose(g, X, v[r], poses + 12 * ns)) ++ns;
  return ns;
}

// ---------------------------------------------------------------- symmetric eigen
// Cyclic Jacobi on a symmetric n x n matrix A (row-major, destroyed); writes
// eigenvalues to w and eigenvectors to the columns of V.
template <int NN>
static VD_HD void vd_jacobi_eig(double* A, double* w, double* V) {
  for (int i = 0; i < NN * NN; ++i) V[i] = (i % (NN + 1) == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < NN; ++p)
      for (int q = 0; q < NN; ++q) {
        tot += A[NN * p + q] * A[NN * p + q];
        if (p != q) off += A[NN * p + q] * A[NN * p + q];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < NN - 1; ++p)
      for (int q = p + 1; q < NN; ++q) {
        const double apq = A[NN * p + q];
        if (apq == 0.0) continue;
        const double theta = (A[NN * q + q] - A[NN * p + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < NN; ++k) {
          const double akp = A[NN * k + p], akq = A[NN * k + q];
          A[NN * k + p] = c * akp - s * akq;
          A[NN * k + q] = s * akp + c * akq;
        }
        for (int k = 0; k < NN; ++k) {
          const double apk = A[NN * p + k], aqk = A[NN * q + k];
          A[NN * p + k] = c * apk - s * aqk;
          A[NN * q + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < NN; ++k) {
          const double vkp = V[NN * k + p], vkq = V[NN * k + q];
          V[NN * k + p] = c * vkp - s * vkq;
          V[NN * k + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < NN; ++i) w[i] = A[NN * i + i];
}
