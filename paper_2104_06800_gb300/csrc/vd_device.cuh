// Device-side building blocks of the dense-indirect EM: the Philox counter
// RNG, the Fisk residual energy, bilinear flow sampling and the per-pixel
// energy E_j(rho) of the depth M-step (Eq. 5 of VOLDOR+, Sec. III-A).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vd_internal.h"

#define VD_LN2 0.69314718055994530942f

// ---------------------------------------------------------------------------
// Checked build (-DVD_CHECKED; the stand-in for a memory checker): every
// index a kernel forms from data is checked against its buffer; the first
// index out of range is recorded (site, index, bound) with a count of all,
// and the index is clamped into range so that the access stays inside its
// buffer (the results are then wrong and the call reports it).  Each
// translation unit has its own record; vd_check_report gathers them.
// Without the flag VD_CHK is the index itself.
// ---------------------------------------------------------------------------
#ifdef VD_CHECKED
static __device__ unsigned long long g_vd_check[4];
__device__ __forceinline__ long long vd_checked(int site, long long i, long long n) {
  if (i >= 0 && i < n) return i;
  if (atomicCAS(&g_vd_check[0], 0ull, (unsigned long long)site) == 0ull) {
    g_vd_check[1] = (unsigned long long)i;
    g_vd_check[2] = (unsigned long long)n;
  }
  atomicAdd(&g_vd_check[3], 1ull);
  return i < 0 ? 0 : (n > 0 ? n - 1 : 0);
}
#define VD_CHK(site, i, n) vd_checked((site), (long long)(i), (long long)(n))
// host accessor of this unit's record: copies it to out[4] and clears it
#define VD_CHECK_ACCESSOR(name)                                                  \
  cudaError_t vd_check_take_##name(unsigned long long* out) {                    \
    cudaError_t e = cudaMemcpyFromSymbol(out, g_vd_check, 4 * sizeof(unsigned long long)); \
    const unsigned long long z[4] = {0, 0, 0, 0};                                \
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_vd_check, z, sizeof z);       \
    return e;                                                                    \
  }
#else
#define VD_CHK(site, i, n) (i)
#define VD_CHECK_ACCESSOR(name)                                                  \
  cudaError_t vd_check_take_##name(unsigned long long* out) {                    \
    for (int i = 0; i < 4; ++i) out[i] = 0;                                      \
    return cudaSuccess;                                                          \
  }
#endif
// sites of the checked build
enum { VD_SITE_BILINEAR = 1, VD_SITE_P3P_TAPS = 2, VD_SITE_SCATTER = 3, VD_SITE_PICK = 4,
       VD_SITE_VC_CELL = 5, VD_SITE_CHAIN = 6 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 bit
// multiplies, mixing with the key, key advanced by the Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 vd_philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;   // one wide multiply per product
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint32_t vd_word(const uint4& w, int i) {
  return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// (x >> 8) * 2^-24 as float (exact).
__device__ __forceinline__ float vd_u24(uint32_t x) {
  return __fmul_rn(__uint2float_rn(x >> 8), 5.9604644775390625e-8f);
}

// Hypothesis values, each operation rounded once (no contraction), so the
// float32 values are reproducible bit for bit.
__device__ __forceinline__ float vd_cand_uniform(uint32_t x, float rmin, float range) {
  return __fadd_rn(rmin, __fmul_rn(vd_u24(x), range));
}
__device__ __forceinline__ float vd_cand_perturb(uint32_t x, float rho, float s) {
  const float a = __fsub_rn(__fmul_rn(2.0f, vd_u24(x)), 1.0f);
  return __fmul_rn(rho, __fadd_rn(1.0f, __fmul_rn(s, a)));
}
__device__ __forceinline__ float vd_clamp(float c, float lo, float hi) {
  return fminf(fmaxf(c, lo), hi);
}

// ---------------------------------------------------------------------------
// Residual energy l = log(1 + P0 / p1(r)), p1 = density of a 2-D residual
// vector whose length is Fisk(alpha, beta) distributed and whose direction is
// uniform.  Returned in log2 units (multiply by ln 2).  Also returns
// y = P0 / p1 (the outlier-to-rigid likelihood ratio) for the E-step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vd_ratio_general(const DevParams& P, float r2, float alpha) {
  float r = sqrtf(r2);
  if (P.beta != 2.0f) r = fmaxf(r, VD_R_FLOOR);
  const float s = r / alpha;
  const float ls = __log2f(s);
  const float sb = exp2f(P.beta * ls);
  const float s2b = exp2f((2.0f - P.beta) * ls);
  const float one = 1.0f + sb;
  return P.cgen * alpha * alpha * s2b * one * one;
}

__device__ __forceinline__ float vd_ratio_y(const DevParams& P, float r2, float fmag2) {
  if (P.fast_beta2) {
    // beta = 2: P0 / p1 = P0 pi alpha^2 (1 + r^2 / alpha^2)^2
    const float s = fmaf(r2, P.inv_a2, 1.0f);
    return P.c0 * s * s;
  }
  return vd_ratio_general(P, r2, fmaf(P.alpha1, sqrtf(fmag2), P.alpha0));
}

// log2(1 + y).  Near the optimum y = P0 pi alpha^2 (1 + s^2)^2 is ~1e-3 and
// the MUFU log2 of 1 + y (absolute error ~2^-22) would lose most digits of
// the residual-dependent part, so small y uses the series
// ln(1 + y) = y - y^2/2 + y^3/3 - y^4/4 + y^5/5 (truncation < y^6/6).
__device__ __forceinline__ float vd_ell2(float y) {
  const float big = __log2f(1.0f + y);
  const float ser =
      y * fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.2f, -0.25f), 0.33333334f), -0.5f), 1.0f) *
      1.44269504f;
  return y < 0.03125f ? ser : big;
}

// log2(1 + P0 / p1) of a residual with r2 = r^2 and Fisk scale alpha.  Where
// the ratio y = P0 / p1 would overflow float32 (a residual of ~1e10 px and
// beyond), log2(1 + y) equals log2 y to float32 precision and is taken in the
// log domain; below that the value is vd_ell2(y).
__device__ __forceinline__ float vd_l2_general(const DevParams& P, float r2, float alpha) {
  float r = sqrtf(r2);
  if (P.beta != 2.0f) r = fmaxf(r, VD_R_FLOOR);
  const float s = r / alpha;
  const float ls = __log2f(s);
  const float sb = exp2f(P.beta * ls);
  const float s2b = exp2f((2.0f - P.beta) * ls);
  const float one = 1.0f + sb;
  const float y = P.cgen * alpha * alpha * s2b * one * one;
  if (y < 1e30f) return vd_ell2(y);
  const float l1 = sb < 1e30f ? __log2f(one) : P.beta * ls;   // log2(1 + s^beta)
  return __log2f(P.cgen * alpha * alpha) + (2.0f - P.beta) * ls + 2.0f * l1;
}

__device__ __forceinline__ float vd_l2_beta2(const DevParams& P, float r2) {
  // beta = 2: P0 / p1 = P0 pi alpha^2 (1 + r^2 / alpha^2)^2
  const float s = fmaf(r2, P.inv_a2, 1.0f);
  const float y = P.c0 * s * s;
  if (y < 1e30f) return vd_ell2(y);
  return fmaf(2.0f, __log2f(s), P.log2c0);
}

// The flow term's log2(1 + P0 / p1): alpha = alpha0 + alpha1 |X_t(x)|.
__device__ __forceinline__ float vd_l2_flow(const DevParams& P, float r2, float fmag2) {
  if (P.fast_beta2) return vd_l2_beta2(P, r2);
  return vd_l2_general(P, r2, fmaf(P.alpha1, sqrtf(fmag2), P.alpha0));
}

// ---------------------------------------------------------------------------
// Entry i of a frame's rows K [R | tau] from its float64 value: float32 for
// the depth and pose kernels, and as a double-float pair (hi, lo; hi + lo is
// the float64 value to 48 bits) for the rigidness emissions.  Every writer
// of the pose rows stores both.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void vd_store_pose_entry(float* __restrict__ pf, float2* __restrict__ pd,
                                                    int i, double v) {
  const float hi = (float)v;
  pf[i] = hi;
  pd[i] = make_float2(hi, (float)(v - (double)hi));
}

// ---------------------------------------------------------------------------
// Bilinear sample of one flow field at (x, y), which must be inside the image.
// Taps (x0, y0)..(x0+1, y0+1) with x0 = min(floor(x), W-2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 vd_bilinear(const float2* __restrict__ F, int W, int H, float x,
                                              float y) {
  const int x0 = min(__float2int_rd(x), W - 2);
  const int y0 = min(__float2int_rd(y), H - 2);
  const float ax = x - (float)x0;
  const float ay = y - (float)y0;
  const float2* p = F + VD_CHK(VD_SITE_BILINEAR, (long long)y0 * W + x0, (long long)W * H - W - 1);
  const float2 f00 = __ldg(p), f01 = __ldg(p + 1);
  const float2 f10 = __ldg(p + W), f11 = __ldg(p + W + 1);
  const float tx = fmaf(ax, f01.x - f00.x, f00.x), ty = fmaf(ax, f01.y - f00.y, f00.y);
  const float bx = fmaf(ax, f11.x - f10.x, f10.x), by = fmaf(ax, f11.y - f10.y, f10.y);
  return make_float2(fmaf(ay, bx - tx, tx), fmaf(ay, by - ty, ty));
}

__device__ __forceinline__ bool vd_inside(float x, float y, int W, int H) {
  return x >= 0.0f && x <= (float)(W - 1) && y >= 0.0f && y <= (float)(H - 1);
}

// ---------------------------------------------------------------------------
// Per-pixel constant part of the energy.  A_t = K R_t r_j (homogeneous image
// point of the ray), B_t = K tau_t is shared by all pixels (shared memory).
// ---------------------------------------------------------------------------
template <int NF>
struct VdPixel {
  float ax[NF], ay[NF], az[NF];
  float wl[NF];           // q_t * ln 2
  float f1x, f1y;         // X_1 at the pixel (x_0 = j exactly)
  float u, v;
  float pv;               // prior value (disparity or rho_hat)
  float pw;               // prior weight q_hat * conf (0 at holes / no prior)
};

// posef layout per frame t (0..N): 9 floats K R_t (row-major), 3 floats K tau_t.
template <int NF>
__device__ __forceinline__ void vd_pixel_setup(VdPixel<NF>& px, const DevParams& P,
                                               const float* __restrict__ sPose, int u, int v,
                                               const float* __restrict__ q, size_t npix, size_t j,
                                               const float2* __restrict__ flow,
                                               const float* __restrict__ prior_val,
                                               const float* __restrict__ qhat,
                                               const float* __restrict__ pconf) {
  const float rx = ((float)u - P.cx) / P.fx;
  const float ry = ((float)v - P.cy) / P.fy;
#pragma unroll
  for (int t = 0; t < NF; ++t) {
    const float* M = sPose + 12 * (t + 1);
    px.ax[t] = fmaf(M[0], rx, fmaf(M[1], ry, M[2]));
    px.ay[t] = fmaf(M[3], rx, fmaf(M[4], ry, M[5]));
    px.az[t] = fmaf(M[6], rx, fmaf(M[7], ry, M[8]));
    px.wl[t] = __ldg(q + (size_t)t * npix + j) * VD_LN2;
  }
  const float2 f1 = __ldg(flow + j);
  px.f1x = f1.x;
  px.f1y = f1.y;
  px.u = (float)u;
  px.v = (float)v;
  px.pw = 0.0f;
  px.pv = 0.0f;
  if (P.prior_kind != VD_PRIOR_NONE) {
    const float pvv = __ldg(prior_val + j);
    if (isfinite(pvv)) {
      px.pv = pvv;
      px.pw = __ldg(qhat + j) * __ldg(pconf + j);
    }
  }
}

// Prior term w_hat l_hat(c) of E_j (0 where the pixel has no prior).
template <int NF>
__device__ __forceinline__ float vd_prior_energy(const VdPixel<NF>& px, const DevParams& P,
                                                 float c) {
  if (!(px.pw > 0.0f)) return 0.0f;
  if (P.prior_kind == VD_PRIOR_STEREO) {
    const float d = px.pv - P.fxb * c;
    const float l2 = P.beta == 2.0f ? vd_l2_beta2(P, d * d) : vd_l2_general(P, d * d, P.alpha0);
    return px.pw * VD_LN2 * l2;
  }
  const float res = px.pv - c;
  const float sig = P.c_sigma * px.pv;
  const float z = fmaf(res * res, 0.5f / (sig * sig), P.logk);
  return px.pw * (z > 20.0f ? z : VD_LN2 * vd_ell2(__expf(z)));
}

// One flow term in log2 units.  (hx, hy, hz): homogeneous image point of the
// candidate in frame t; (xp, yp): its image point in frame t-1, where the
// flow (Fx, Fy) was read; obs: the point is in front of camera t-1 and
// inside image t-1.  Writes the image point in frame t and whether it is in
// front of camera t.
__device__ __forceinline__ float vd_flow_term(const DevParams& P, float hx, float hy, float hz,
                                              bool obs, float Fx, float Fy, float xp, float yp,
                                              float* x_out, float* y_out, bool* front_out) {
  const bool front = hz > VD_Z_EPS;
  const float iz = __fdividef(1.0f, hz);
  const float x = hx * iz, y = hy * iz;
  float l2;
  if (obs && front) {
    const float dx = Fx - (x - xp);
    const float dy = Fy - (y - yp);
    const float r2 = fmaf(dx, dx, dy * dy);
    l2 = vd_l2_flow(P, r2, fmaf(Fx, Fx, Fy * Fy));
  } else {
    l2 = obs ? (VD_L_BEHIND / VD_LN2) : 0.0f;
  }
  *x_out = x;
  *y_out = y;
  *front_out = front;
  return l2;
}

// E_j(c) in full, for latency-bound callers (the chain propagation): every
// frame's projection first, then every gathered flow's taps (all loads in
// flight together), then the terms in the order and arithmetic of
// vd_energy, so the value is vd_energy's without a bound.  A caller that
// compares the result with a bound gets vd_energy's decision (an early
// exit there returns a partial sum already at or above it).
template <int NF>
__device__ __forceinline__ float vd_energy_full(const VdPixel<NF>& px, const DevParams& P,
                                                const float* __restrict__ sPose,
                                                const float2* __restrict__ flow, size_t npix,
                                                float c) {
  float xs[NF], ys[NF];
  bool fr[NF];
#pragma unroll
  for (int t = 0; t < NF; ++t) {   // projection into frame t + 1 (as vd_flow_term forms it)
    const float* M = sPose + 12 * (t + 1);
    const float hx = fmaf(c, M[9], px.ax[t]);
    const float hy = fmaf(c, M[10], px.ay[t]);
    const float hz = fmaf(c, M[11], px.az[t]);
    fr[t] = hz > VD_Z_EPS;
    const float iz = __fdividef(1.0f, hz);
    xs[t] = hx * iz;
    ys[t] = hy * iz;
  }
  float2 F[NF];
  bool ob[NF];
  F[0] = make_float2(px.f1x, px.f1y);
  ob[0] = true;
#pragma unroll
  for (int t = 1; t < NF; ++t) {   // flow t read at the pixel's position in frame t
    ob[t] = fr[t - 1] && vd_inside(xs[t - 1], ys[t - 1], P.W, P.H);
    F[t] = make_float2(0.0f, 0.0f);
    if (ob[t]) F[t] = vd_bilinear(flow + (size_t)t * npix, P.W, P.H, xs[t - 1], ys[t - 1]);
  }
  float E = vd_prior_energy<NF>(px, P, c);
#pragma unroll
  for (int t = 0; t < NF; ++t) {
    const float xp = t == 0 ? px.u : xs[t - 1], yp = t == 0 ? px.v : ys[t - 1];
    float l2;
    if (ob[t] && fr[t]) {
      const float dx = F[t].x - (xs[t] - xp);
      const float dy = F[t].y - (ys[t] - yp);
      const float r2 = fmaf(dx, dx, dy * dy);
      l2 = vd_l2_flow(P, r2, fmaf(F[t].x, F[t].x, F[t].y * F[t].y));
    } else {
      l2 = ob[t] ? (VD_L_BEHIND / VD_LN2) : 0.0f;
    }
    E = fmaf(px.wl[t], l2, E);
  }
  return E;
}

// E_j(c): sum_t q_t l_t(c) + w_hat l_hat(c) in natural-log units.
// Every term is non-negative, so once the partial sum reaches `bound` the
// candidate cannot beat an energy of `bound`: the sum stops there and the
// partial value (>= bound) is returned.  The cheap terms come first: the
// prior, then X_1 (read at the pixel itself), then the gathered flows.
template <int NF>
__device__ __forceinline__ float vd_energy(const VdPixel<NF>& px, const DevParams& P,
                                           const float* __restrict__ sPose,
                                           const float2* __restrict__ flow, size_t npix,
                                           float c, float bound = INFINITY) {
  float E = vd_prior_energy<NF>(px, P, c);
  float xp = px.u, yp = px.v;
  bool front_prev = true;
#pragma unroll
  for (int t = 0; t < NF; ++t) {
    if (E >= bound) return E;
    const float* M = sPose + 12 * (t + 1);
    const float hx = fmaf(c, M[9], px.ax[t]);
    const float hy = fmaf(c, M[10], px.ay[t]);
    const float hz = fmaf(c, M[11], px.az[t]);
    bool obs;
    float Fx, Fy;
    if (t == 0) {
      obs = true;
      Fx = px.f1x;
      Fy = px.f1y;
    } else {
      obs = front_prev && vd_inside(xp, yp, P.W, P.H);
      float2 F = make_float2(0.0f, 0.0f);
      if (obs) F = vd_bilinear(flow + (size_t)t * npix, P.W, P.H, xp, yp);
      Fx = F.x;
      Fy = F.y;
    }
    float x, y;
    bool front;
    const float l2 = vd_flow_term(P, hx, hy, hz, obs, Fx, Fy, xp, yp, &x, &y, &front);
    E = fmaf(px.wl[t], l2, E);
    xp = x;
    yp = y;
    front_prev = front;
  }
  return E;
}
