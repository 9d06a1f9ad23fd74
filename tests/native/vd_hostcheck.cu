// Host build of the library's float64 geometry (vd_geom64.cuh) so that the
// CPU test-suite can check the P3P solver, the polynomial root finder, the
// SE(3) maps and the Jacobi eigen-solver without a GPU, and of the
// double-float positions of the rigidness emissions (vd_emission_df.cuh).
#include "vd_emission_df.cuh"
#include "vd_geom64.cuh"
#include "vd_p3p_df.cuh"

extern "C" int hc_p3p(const double* f, const double* X, double* poses) { return vd_p3p(f, X, poses); }
extern "C" int hc_real_roots(const double* c, int deg, double* out) {
  return vd_poly_real_roots(c, deg, out);
}
extern "C" int hc_p3p_df(const double* f, const double* X, double* poses) {
  return vd_p3p_df_solve(f, X, poses);
}
extern "C" int hc_quartic_fast(const double* c, double* out) {
  return vd_quartic_real_roots_fast(c, out);
}
extern "C" void hc_se3_exp(const double* xi, double* T) { vd_se3_exp(xi, T); }
extern "C" void hc_se3_log(const double* T, double* xi) { vd_se3_log(T, xi); }
extern "C" void hc_jacobi9(double* A, double* w, double* V) { vd_jacobi_eig<9>(A, w, V); }
extern "C" void hc_jacobi3(double* A, double* w, double* V) { vd_jacobi_eig<3>(A, w, V); }

// Frame image point of pixel (u, v) at inverse depth c through the rows
// M24 = K [R | tau] as (hi, lo) pairs; out = x, y as hi + lo.  Returns 1 in
// front of the camera, 0 behind (out untouched).
extern "C" int hc_em_project(const float* M24, const float* kdf, int u, int v, float c,
                             double* out) {
  float2 M[12];
  for (int i = 0; i < 12; ++i) M[i] = make_float2(M24[2 * i], M24[2 * i + 1]);
  vd_df rx, ry, x, y;
  vd_em_ray(kdf, u, v, &rx, &ry);
  if (!vd_em_project(M, rx, ry, c, &x, &y)) return 0;
  out[0] = (double)x.hi + (double)x.lo;
  out[1] = (double)y.hi + (double)y.lo;
  return 1;
}
extern "C" int hc_em_inside(float xh, float xl, float yh, float yl, int W, int H) {
  return vd_em_inside(vd_df_make(xh, xl), vd_df_make(yh, yl), W, H) ? 1 : 0;
}
extern "C" int hc_em_tap(float hi, float lo, int n, float* w) {
  return vd_em_tap(vd_df_make(hi, lo), n, w);
}
