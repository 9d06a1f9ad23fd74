// Host build of the library's float64 geometry (vd_geom64.cuh) so that the
// CPU test-suite can check the P3P solver, the polynomial root finder, the
// SE(3) maps and the Jacobi eigen-solver without a GPU.
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
