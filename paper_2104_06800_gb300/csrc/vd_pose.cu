// Pose M-step of VOLDOR+ (Sec. III-A, Eq. 7): the posterior of each camera
// pose is approximated by S P3P samples drawn from the rigid pixels; every
// root is scored against all rigid pixels, each sample keeps its best root,
// and the pose is the mean-shift mode of the samples in se(3).
#include <algorithm>
#include <mutex>

#include "vd_device.cuh"
#include "vd_geom64.cuh"
#include "vd_p3p_df.cuh"

#define SCAN_BLOCK 256
#define SCORE_THREADS 256
#define SCORE_PPT 8

// ---------------------------------------------------------------------------
// Float64 track position x_{t-1} of pixel j at inverse depth rho (t >= 2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool vd_track64(const DevParams& P, const double* g, int u, int v,
                                           double rho, double* x, double* y) {
  const double rx = ((double)u - P.cx_d) / P.fx_d, ry = ((double)v - P.cy_d) / P.fy_d;
  const double X = g[0] * rx + g[1] * ry + g[2] + rho * g[3];
  const double Y = g[4] * rx + g[5] * ry + g[6] + rho * g[7];
  const double Z = g[8] * rx + g[9] * ry + g[10] + rho * g[11];
  const double hx = P.fx_d * X + P.cx_d * Z, hy = P.fy_d * Y + P.cy_d * Z;
  if (!(Z > (double)VD_Z_EPS)) return false;
  *x = hx / Z;
  *y = hy / Z;
  return true;
}

__device__ __forceinline__ bool vd_front64(const DevParams& P, const double* g, int u, int v,
                                           double rho) {
  const double rx = ((double)u - P.cx_d) / P.fx_d, ry = ((double)v - P.cy_d) / P.fy_d;
  return g[8] * rx + g[9] * ry + g[10] + rho * g[11] > (double)VD_Z_EPS;
}

__device__ __forceinline__ void vd_bilinear64(const float2* __restrict__ F, int W, int H, double x,
                                              double y, double* fx, double* fy) {
  const int x0 = min((int)floor(x), W - 2), y0 = min((int)floor(y), H - 2);
  const double ax = x - x0, ay = y - y0;
  const float2* p = F + (size_t)y0 * W + x0;
  const float2 a = p[0], b = p[1], c = p[W], d = p[W + 1];
  *fx = (1 - ay) * ((1 - ax) * a.x + ax * b.x) + ay * ((1 - ax) * c.x + ax * d.x);
  *fy = (1 - ay) * ((1 - ax) * a.y + ax * b.y) + ay * ((1 - ax) * c.y + ax * d.y);
}

// Membership of the rigid set (decisions in float64; a float32 test decides
// directly when it is far from every threshold, the float64 one otherwise).
__device__ bool vd_is_rigid(const DevParams& P, const double* __restrict__ G,
                            const float* __restrict__ posef, const float* __restrict__ rho,
                            const float* __restrict__ q, int t, int u, int v, size_t j) {
  const size_t npix = (size_t)P.W * P.H;
  if (!(q[(size_t)(t - 1) * npix + j] > 0.5f)) return false;
  const float c = rho[j];
  const float rx = ((float)u - P.cx) / P.fx, ry = ((float)v - P.cy) / P.fy;
  if (t >= 2) {
    const float* M = posef + 12 * (t - 1);
    const float hx = fmaf(c, M[9], fmaf(M[0], rx, fmaf(M[1], ry, M[2])));
    const float hy = fmaf(c, M[10], fmaf(M[3], rx, fmaf(M[4], ry, M[5])));
    const float hz = fmaf(c, M[11], fmaf(M[6], rx, fmaf(M[7], ry, M[8])));
    const float x = hx / hz, y = hy / hz;
    const float mg = 1e-2f;
    const bool clear = fabsf(hz - VD_Z_EPS) > 1e-3f && fabsf(x) > mg && fabsf(x - (P.W - 1)) > mg &&
                       fabsf(y) > mg && fabsf(y - (P.H - 1)) > mg && isfinite(x) && isfinite(y);
    bool ok;
    if (clear) {
      ok = hz > VD_Z_EPS && vd_inside(x, y, P.W, P.H);
    } else {
      double xd, yd;
      ok = vd_track64(P, G + 12 * (t - 1), u, v, (double)c, &xd, &yd) && xd >= 0.0 &&
           xd <= (double)(P.W - 1) && yd >= 0.0 && yd <= (double)(P.H - 1);
    }
    if (!ok) return false;
  }
  const float* M = posef + 12 * t;
  const float hz = fmaf(c, M[11], fmaf(M[6], rx, fmaf(M[7], ry, M[8])));
  if (fabsf(hz - VD_Z_EPS) > 1e-3f) return hz > VD_Z_EPS;
  return vd_front64(P, G + 12 * t, u, v, (double)c);
}

__global__ void __launch_bounds__(SCAN_BLOCK)
k_rigid_flags(DevParams P, const double* __restrict__ G, const float* __restrict__ posef,
              const float* __restrict__ rho, const float* __restrict__ q, int t,
              unsigned char* __restrict__ flags, int* __restrict__ blk_counts) {
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int f = 0;
  if (j < npix) {
    const int v = (int)(j / P.W), u = (int)(j - (size_t)v * P.W);
    f = vd_is_rigid(P, G, posef, rho, q, t, u, v, j) ? 1 : 0;
    flags[j] = (unsigned char)f;
  }
  const int cnt = __syncthreads_count(f);
  if (threadIdx.x == 0) blk_counts[blockIdx.x] = cnt;
}

// Scatter the rigid pixels in row-major order with their float32 scoring data:
// X = r_j / rho_j (reference frame), x_obs = x_{t-1} + X_t(x_{t-1}), w = q_t.
// Each block adds up the counts of the blocks before it (a few thousand
// integers from L2, instead of a separate scan launch); the last block
// writes the total.
__global__ void __launch_bounds__(SCAN_BLOCK)
k_rigid_scatter(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
                const float* __restrict__ rho, const float* __restrict__ q, int t,
                const unsigned char* __restrict__ flags, const int* __restrict__ counts,
                int* __restrict__ n_out, int* __restrict__ idx, float4* __restrict__ rpts,
                float4* __restrict__ robs) {
  __shared__ int warp_tot[SCAN_BLOCK / 32];
  __shared__ int warp_pre[SCAN_BLOCK / 32];
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  const int f = (j < npix) ? flags[j] : 0;
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // counts of the blocks before this one, a fixed-order integer sum
  int pre = 0;
  for (unsigned k = threadIdx.x; k < blockIdx.x; k += SCAN_BLOCK) pre += counts[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) {
    warp_tot[wid] = __popc(bal);
    warp_pre[wid] = pre;
  }
  __syncthreads();
  int offset = 0, before = 0, total = 0;
  for (unsigned w = 0; w < SCAN_BLOCK / 32; ++w) {
    offset += warp_pre[w];
    total += warp_tot[w];
    if (w < wid) before += warp_tot[w];
  }
  before += __popc(bal & ((1u << lane) - 1u));
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *n_out = offset + total;
  if (!f) return;
  const int pos = (int)VD_CHK(VD_SITE_SCATTER, offset + before, npix);
  const int v = (int)(j / P.W), u = (int)(j - (size_t)v * P.W);
  const float c = rho[j];
  const float rx = ((float)u - P.cx) / P.fx, ry = ((float)v - P.cy) / P.fy;
  const float th = 1.0f / c;
  float xp = (float)u, yp = (float)v;
  float2 F;
  if (t == 1) {
    F = flow[j];
  } else {
    const float* M = posef + 12 * (t - 1);
    const float hx = fmaf(c, M[9], fmaf(M[0], rx, fmaf(M[1], ry, M[2])));
    const float hy = fmaf(c, M[10], fmaf(M[3], rx, fmaf(M[4], ry, M[5])));
    const float hz = fmaf(c, M[11], fmaf(M[6], rx, fmaf(M[7], ry, M[8])));
    xp = hx / hz;
    yp = hy / hz;
    // the float64 membership test may accept a point the float32 position
    // puts a hair outside: clamp the sampling position
    xp = fminf(fmaxf(xp, 0.0f), (float)(P.W - 1));
    yp = fminf(fmaxf(yp, 0.0f), (float)(P.H - 1));
    F = vd_bilinear(flow + (size_t)(t - 1) * npix, P.W, P.H, xp, yp);
  }
  const float alpha = fmaf(P.alpha1, sqrtf(fmaf(F.x, F.x, F.y * F.y)), P.alpha0);
  idx[pos] = (int)j;
  rpts[pos] = make_float4(rx * th, ry * th, th, q[(size_t)(t - 1) * npix + j]);
  robs[pos] = make_float4(xp + F.x, yp + F.y, alpha, 0.0f);
}

// ---------------------------------------------------------------------------
// P3P sampling in double-float (vd_p3p_df.cuh): on this GPU a float64
// instruction costs a warp 64 cycles, a float32 one about 1.3.
// ---------------------------------------------------------------------------
// Correspondence of rigid pixel j in double-float: the point X = r_j / rho_j
// of the reference frame and the bearing K^-1 x_obs of its observation in
// frame t, x_obs = x_{t-1} + X_t(x_{t-1}) (x_0 = j; for t >= 2, x_{t-1} is
// the projection by G_{t-1}, given as 12 double-float values in g).
__device__ __forceinline__ void vd_correspondence_df(const DevParams& P, const vd_df* g,
                                     const float2* __restrict__ flow, const float* __restrict__ rho,
                                     int t, int j, vd_df* X, vd_df* bearing) {
  const int v = j / P.W, u = j - v * P.W;
  const vd_df fx = vd_df_make(P.kdf[0], P.kdf[1]), fy = vd_df_make(P.kdf[2], P.kdf[3]);
  const vd_df cx = vd_df_make(P.kdf[4], P.kdf[5]), cy = vd_df_make(P.kdf[6], P.kdf[7]);
  const vd_df ifx = vd_df_make(P.kdf[8], P.kdf[9]), ify = vd_df_make(P.kdf[10], P.kdf[11]);
  const float c = rho[j];
  const vd_df rx = vd_df_mul(vd_df_sub(vd_df_make((float)u), cx), ifx);
  const vd_df ry = vd_df_mul(vd_df_sub(vd_df_make((float)v), cy), ify);
  const vd_df th = vd_df_rcp(vd_df_make(c));
  X[0] = vd_df_mul(rx, th);
  X[1] = vd_df_mul(ry, th);
  X[2] = th;
  const size_t npix = (size_t)P.W * P.H;
  vd_df xp = vd_df_make((float)u), yp = vd_df_make((float)v);
  float2 F0 = flow[j];
  vd_df Fx = vd_df_make(F0.x), Fy = vd_df_make(F0.y);
  if (t >= 2) {
    const vd_df cc = vd_df_make(c);
    const vd_df Xc = vd_df_add(vd_df_add(vd_df_mul(g[0], rx), vd_df_mul(g[1], ry)),
                               vd_df_add(g[2], vd_df_mul(cc, g[3])));
    const vd_df Yc = vd_df_add(vd_df_add(vd_df_mul(g[4], rx), vd_df_mul(g[5], ry)),
                               vd_df_add(g[6], vd_df_mul(cc, g[7])));
    const vd_df Zc = vd_df_add(vd_df_add(vd_df_mul(g[8], rx), vd_df_mul(g[9], ry)),
                               vd_df_add(g[10], vd_df_mul(cc, g[11])));
    if (Zc.hi > VD_Z_EPS) {
      const vd_df iz = vd_df_rcp(Zc);
      xp = vd_df_mul(vd_df_add(vd_df_mul(fx, Xc), vd_df_mul(cx, Zc)), iz);
      yp = vd_df_mul(vd_df_add(vd_df_mul(fy, Yc), vd_df_mul(cy, Zc)), iz);
    }
    // members of the rigid set are inside the image; the clamp only guards
    // the gather against a position at or beyond the border
    const float wmax = (float)(P.W - 1), hmax = (float)(P.H - 1);
    if (!(xp.hi >= 0.0f)) xp = vd_df_make(0.0f);
    if (!(xp.hi <= wmax)) xp = vd_df_make(wmax);
    if (!(yp.hi >= 0.0f)) yp = vd_df_make(0.0f);
    if (!(yp.hi <= hmax)) yp = vd_df_make(hmax);
    // bilinear taps (x0, y0) .. (x0 + 1, y0 + 1), x0 = min(floor(x), W - 2)
    float x0 = floorf(xp.hi), y0 = floorf(yp.hi);
    if (xp.hi == x0 && xp.lo < 0.0f) x0 -= 1.0f;
    if (yp.hi == y0 && yp.lo < 0.0f) y0 -= 1.0f;
    x0 = fminf(fmaxf(x0, 0.0f), (float)(P.W - 2));
    y0 = fminf(fmaxf(y0, 0.0f), (float)(P.H - 2));
    const vd_df ax = vd_df_sub(xp, vd_df_make(x0)), ay = vd_df_sub(yp, vd_df_make(y0));
    const float2* q = flow + (size_t)(t - 1) * npix +
                      VD_CHK(VD_SITE_P3P_TAPS, (long long)y0 * P.W + (long long)x0,
                             (long long)npix - P.W - 1);
    const float2 f00 = q[0], f01 = q[1], f10 = q[P.W], f11 = q[P.W + 1];
    // F = t + ay (b - t), t = f00 + ax (f01 - f00), b = f10 + ax (f11 - f10)
    const vd_df tx = vd_df_add(vd_df_make(f00.x), vd_df_mul(ax, vd_two_sum(f01.x, -f00.x)));
    const vd_df ty = vd_df_add(vd_df_make(f00.y), vd_df_mul(ax, vd_two_sum(f01.y, -f00.y)));
    const vd_df bx = vd_df_add(vd_df_make(f10.x), vd_df_mul(ax, vd_two_sum(f11.x, -f10.x)));
    const vd_df by = vd_df_add(vd_df_make(f10.y), vd_df_mul(ax, vd_two_sum(f11.y, -f10.y)));
    Fx = vd_df_add(tx, vd_df_mul(ay, vd_df_sub(bx, tx)));
    Fy = vd_df_add(ty, vd_df_mul(ay, vd_df_sub(by, ty)));
  }
  bearing[0] = vd_df_mul(vd_df_sub(vd_df_add(xp, Fx), cx), ifx);
  bearing[1] = vd_df_mul(vd_df_sub(vd_df_add(yp, Fy), cy), ify);
  bearing[2] = vd_df_make(1.0f);
}

__device__ __forceinline__ vd_df vd_shfl_df(vd_df x, int src) {
  return vd_df{__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src)};
}

// vd_split_rootsf with the interval searches in parallel lanes (the same
// intervals and searches; every lane receives all roots).
__device__ int vd_split_rootsf_warp(const float* c, int deg, const float* crit, int ncrit,
                                    float* out, int lane) {
  const float bound = vd_root_boundf(c, deg);
  float lo = -bound, flo = vd_polyf(c, deg, lo);
  float mlo = 0.0f, mhi = 0.0f;
  bool mneg = false;
  int mkind = 0, kinds = 0, ni = 0;
  for (int i = 0; i <= ncrit; ++i) {
    const float hi = i < ncrit ? fminf(fmaxf(crit[i], -bound), bound) : bound;
    if (!(hi > lo)) continue;
    const float fhi = vd_polyf(c, deg, hi);
    const int kind = flo == 0.0f ? 1 : (((flo < 0.0f) != (fhi < 0.0f) && fhi != 0.0f) ? 2 : 0);
    kinds |= kind << (2 * ni);
    if (ni == lane) {
      mlo = lo;
      mhi = hi;
      mkind = kind;
      mneg = flo < 0.0f;
    }
    ++ni;
    lo = hi;
    flo = fhi;
  }
  const float mine = mkind == 2 ? vd_bracketed_rootf(c, deg, mlo, mhi, mneg) : mlo;
  int n = 0;
  for (int k = 0; k < 4; ++k) {
    const float r = __shfl_sync(0xffffffffu, mine, k);
    if (k < ni && ((kinds >> (2 * k)) & 3)) out[n++] = r;
  }
  return n;
}

// vd_p3p_df_roots with the shifted quartic's interval searches and
// double-float polish in parallel lanes; every lane receives all roots
// (ascending).  A
// quartic whose leading coefficient is negligible takes the float64 search
// of vd_geom64.cuh (lower degree), as the float64 solver does.
__device__ int vd_p3p_df_roots_warp(const VdP3Pdf& g, const vd_df* res, vd_df* out, int lane) {
  float mx = 0.0f;
  for (int i = 0; i <= 4; ++i) mx = fmaxf(mx, fabsf(res[i].hi));
  if (!(mx > 0.0f)) return 0;
  if (!(fabsf(res[4].hi) > 1e-7f * mx)) {
    double rd[5], vd[4];
    for (int i = 0; i <= 4; ++i) rd[i] = vd_df_to(res[i]);
    const int n = vd_poly_real_roots(rd, 4, vd);
    for (int i = 0; i < n; ++i) out[i] = vd_df_from(vd[i]);
    return n;
  }
  vd_df d[5];
  const vd_df m = vd_df_taylor_shift(res, d);
  float cf[5];
  float dm = 0.0f;
  for (int i = 0; i <= 4; ++i) dm = fmaxf(dm, fabsf(d[i].hi));
  const float s = 1.0f / dm;
  for (int i = 0; i <= 4; ++i) cf[i] = d[i].hi * s;
  const float q[3] = {cf[2] * 2.0f, cf[3] * 6.0f, cf[4] * 12.0f};
  const float split = -q[1] / (2.0f * q[2]);
  float r2[2], r3[3];
  const int n2 = vd_split_rootsf_warp(q, 2, &split, 1, r2, lane);
  const float cc[4] = {cf[1], cf[2] * 2.0f, cf[3] * 3.0f, cf[4] * 4.0f};
  const int n3 = vd_split_rootsf_warp(cc, 3, r2, n2, r3, lane);
  // the quartic's sign at the ends of the intervals, in double-float: lane
  // k < n3 + 2 evaluates end k (-bound, the split points, +bound)
  const float bound = vd_root_boundf(cf, 4);
  float e = -bound;
  if (lane >= 1 && lane <= n3) e = fminf(fmaxf(r3[lane - 1], -bound), bound);
  else if (lane == n3 + 1) e = bound;
  const vd_df fe = vd_df_poly(d, 4, vd_df_make(e));
  const int sgn = (fe.hi == 0.0f && fe.lo == 0.0f) ? 0 : (vd_df_lt0(fe) ? -1 : 1);
  // interval k = [end k, end k + 1] on lane k
  float mlo = 0.0f, mhi = 0.0f;
  int kind = 0;
  bool mneg = false;
  {
    const float ehi = __shfl_sync(0xffffffffu, e, lane < 31 ? lane + 1 : 0);
    const int shi = __shfl_sync(0xffffffffu, sgn, lane < 31 ? lane + 1 : 0);
    if (lane <= n3 && ehi > e) {
      mlo = e;
      mhi = ehi;
      mneg = sgn < 0;
      kind = sgn == 0 ? 1 : ((sgn != shi && shi != 0) ? 2 : 0);
    }
  }
  vd_df mine = vd_df_make(mlo);
  mine = vd_df_add(mine, m);        // back from the shifted variable
  if (kind == 2) {    // no warp-wide operation inside: lanes may diverge here
    const float x0 = vd_bracketed_rootf(cf, 4, mlo, mhi, mneg);
    mine = vd_p3p_df_polish(g, m, x0, mlo, mhi);
  }
  int n = 0;
  for (int k = 0; k < 4; ++k) {
    const int kk = __shfl_sync(0xffffffffu, kind, k);
    const vd_df r = vd_shfl_df(mine, k);
    if (k <= n3 && kk) out[n++] = r;
  }
  return n;
}

// One warp per sample (samples spread over the SMs).  Lanes 0-2 build the
// three correspondences, every lane forms the quartic, the root searches
// run in parallel lanes, lanes 0-3 turn one root each into a pose and its
// ordering key; each lane then finds its rank.  Writes the roots (float64,
// ordered by rotation vector, then translation), their count and their
// float K R | K tau for the dense scoring.
// Samples per block (one warp each): warps of one SM share the fetched
// instructions of the long straight-line double-float code.
#ifndef VD_P3P_WARPS
#define VD_P3P_WARPS 4
#endif

__global__ void __launch_bounds__(32 * VD_P3P_WARPS)
k_p3p_samples(DevParams P, const double* __restrict__ G, const float2* __restrict__ flow,
              const float* __restrict__ rho, const int* __restrict__ idx,
              const int* __restrict__ n_rigid, int t, uint32_t itcode, double* __restrict__ roots,
              int* __restrict__ root_count, float* __restrict__ rootsf,
              float* __restrict__ rootsr) {
  const int g = blockIdx.x * VD_P3P_WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= P.S) return;                       // whole warps leave together
  const int n = *n_rigid;
  int pick[3] = {0, 0, 0};
  bool ok = false;
  if (n >= 3) {
    for (uint32_t b = 0; b < VD_MAX_ATTEMPTS && !ok; ++b) {
      const uint4 w = vd_philox(
          make_uint4((uint32_t)g + 65536u * (uint32_t)t, itcode, VD_TAG_POSE, b), P.key0, P.key1);
      pick[0] = (int)(((unsigned long long)w.x * (unsigned long long)n) >> 32);
      pick[1] = (int)(((unsigned long long)w.y * (unsigned long long)n) >> 32);
      pick[2] = (int)(((unsigned long long)w.z * (unsigned long long)n) >> 32);
      ok = pick[0] != pick[1] && pick[0] != pick[2] && pick[1] != pick[2];
    }
  }
  if (!ok) {
    if (lane == 0) root_count[g] = 0;
    if (lane < 4)
      for (int i = 0; i < 12; ++i) rootsf[48 * g + 12 * lane + i] = 0.0f;
    return;
  }
  // G_{t-1} as double-float, one value per lane
  vd_df gl = vd_df_make(0.0f);
  if (t >= 2 && lane < 12) gl = vd_df_from(G[12 * (t - 1) + lane]);
  vd_df gt[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) gt[i] = vd_shfl_df(gl, i);
  vd_df Xl[3] = {vd_df_make(0.0f), vd_df_make(0.0f), vd_df_make(0.0f)};
  vd_df fl[3] = {vd_df_make(0.0f), vd_df_make(0.0f), vd_df_make(1.0f)};
  if (lane < 3)
    vd_correspondence_df(P, gt, flow, rho, t,
                         (int)VD_CHK(VD_SITE_PICK, idx[VD_CHK(VD_SITE_PICK, pick[lane], n)],
                                     (long long)P.W * P.H), Xl, fl);
  vd_df X[9], f[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X[3 * k + c] = vd_shfl_df(Xl[c], k);
      f[3 * k + c] = vd_shfl_df(fl[c], k);
    }
  VdP3Pdf geo;
  vd_df res[5], v[4];
  // the world points' triad (independent of the roots: its latency overlaps
  // the quartic's)
  vd_df Fp[9];
  vd_df_triad(X, Fp);
  const int nr = vd_p3p_df_quartic(f, X, &geo, res) ? vd_p3p_df_roots_warp(geo, res, v, lane) : 0;
  vd_df T[12];
  bool valid = false;
  if (lane < 4 && lane < nr) valid = vd_p3p_df_pose(geo, X, Fp, v[lane], T);
  float key[6] = {0, 0, 0, 0, 0, 0};
  if (valid) {
    // ordering key: rotation vector (float32 is plenty to order distinct
    // roots), then the translation
    const float cf = 0.5f * (T[0].hi + T[5].hi + T[10].hi - 1.0f);
    const float vx = 0.5f * (T[9].hi - T[6].hi), vy = 0.5f * (T[2].hi - T[8].hi);
    const float vz = 0.5f * (T[4].hi - T[1].hi);
    const float sn = sqrtf(vx * vx + vy * vy + vz * vz);
    const float th = atan2f(sn, cf);
    const float fk = sn < 1e-6f ? 1.0f + th * th * (1.0f / 6.0f) : th / sn;
    key[0] = vx * fk;
    key[1] = vy * fk;
    key[2] = vz * fk;
    key[3] = T[3].hi;
    key[4] = T[7].hi;
    key[5] = T[11].hi;
  }
  // rank among the valid roots by (rotation vector, translation), ties by lane
  int rank = 0, count = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool vk = __shfl_sync(0xffffffffu, valid, k);
    float kk[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) kk[i] = __shfl_sync(0xffffffffu, key[i], k);
    if (!vk) continue;
    ++count;
    if (!valid || k == lane) continue;
    int cmp = 0;
    for (int i = 0; i < 6 && cmp == 0; ++i) cmp = kk[i] < key[i] ? -1 : (kk[i] > key[i] ? 1 : 0);
    if (cmp < 0 || (cmp == 0 && k < lane)) ++rank;
  }
  if (valid) {
    double* out = roots + (size_t)g * 48 + 12 * rank;
    for (int i = 0; i < 12; ++i) out[i] = vd_df_to(T[i]);
    float* orr = rootsr + 48 * g + 12 * rank;      // float R | tau (the mean-shift's)
    for (int i = 0; i < 12; ++i) orr[i] = T[i].hi;
    // float K R | K tau of the root, for the dense scoring
    const float fxf = P.kdf[0], fyf = P.kdf[2], cxf = P.kdf[4], cyf = P.kdf[6];
    float* o = rootsf + 48 * g + 12 * rank;
    for (int i = 0; i < 4; ++i) {
      const float r0 = T[i].hi, r1 = T[4 + i].hi, r2 = T[8 + i].hi;
      o[i < 3 ? i : 9] = fmaf(fxf, r0, cxf * r2);
      o[i < 3 ? 3 + i : 10] = fmaf(fyf, r1, cyf * r2);
      o[i < 3 ? 6 + i : 11] = r2;
    }
  }
  if (lane < 4 && lane >= count)      // slots without a root
    for (int i = 0; i < 12; ++i) rootsf[48 * g + 12 * lane + i] = 0.0f;
  if (lane == 0) root_count[g] = count;
}

// ---------------------------------------------------------------------------
// Dense scoring: every root against every rigid pixel.  Each warp takes
// passes of 32 x SCORE_PPT consecutive rigid pixels of its block's range
// (pixels in registers) and, 32 roots at a time, accumulates one sum per
// root in every lane; a butterfly reduce-scatter (31 shuffles) then leaves
// lane L holding the warp's sum of root 32 g + L.  Warp sums are added in
// fixed order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
#ifndef VD_SCORE_PPT
#define VD_SCORE_PPT 4
#endif
#undef SCORE_PPT
#define SCORE_PPT VD_SCORE_PPT

// One pixel's term under one root in log2 units (the caller scales by ln 2),
// without branches.  FAST: beta = 2 and alpha1 = 0 (closed form; obs.z
// unused) with one MUFU log2: log2(1 + y) below y = 2^24, log2 y = log2 c0 +
// 2 log2 s above (equal to float32 precision there, and no overflow), the
// series of ln(1 + y) below y = 1/32.  A point behind the camera gives the
// constant term (its projection uses a denominator of 1 and is discarded).
template <bool FAST>
__device__ __forceinline__ float vd_score_term2(const DevParams& P, const float* Mr, float4 pt,
                                                float4 ob) {
  const float hx = fmaf(Mr[0], pt.x, fmaf(Mr[1], pt.y, fmaf(Mr[2], pt.z, Mr[9])));
  const float hy = fmaf(Mr[3], pt.x, fmaf(Mr[4], pt.y, fmaf(Mr[5], pt.z, Mr[10])));
  const float hz = fmaf(Mr[6], pt.x, fmaf(Mr[7], pt.y, fmaf(Mr[8], pt.z, Mr[11])));
  const bool front = hz > VD_Z_EPS;
  const float iz = __fdividef(1.0f, front ? hz : 1.0f);
  const float dx = fmaf(-hx, iz, ob.x), dy = fmaf(-hy, iz, ob.y);
  const float r2 = fmaf(dx, dx, dy * dy);
  float l2;
  if (FAST) {
    const float sq = fmaf(r2, P.inv_a2, 1.0f);
    const float y = P.c0 * sq * sq;
    const bool mid = y < 16777216.0f;
    const float L = __log2f(mid ? 1.0f + y : sq);
    const float big = mid ? L : fmaf(2.0f, L, P.log2c0);
    // log2(1 + y) = y (1 - y/2 + y^2/3 - y^3/4 + y^4/5) / ln 2 (below 1/32)
    const float ser = y * fmaf(y, fmaf(y, fmaf(y, fmaf(y, 0.28853901f, -0.36067376f),
                                                0.48089835f), -0.72134752f), 1.44269504f);
    l2 = y < 0.03125f ? ser : big;
  } else {
    l2 = vd_l2_general(P, r2, ob.z);
  }
  return front ? l2 : VD_L_BEHIND / VD_LN2;
}

// Dynamic shared memory of k_pose_score<THREADS> for M roots.
static inline size_t vd_score_smem(int M, int threads) {
  return sizeof(float) * (size_t)32 * (12 + threads / 32) + sizeof(int) * (size_t)(M + 1);
}

// acc[0..7] of every lane -> lanes with L % 8 == k return the warp's sum of
// acc[k] (recursive halving over lane bits 2, 1, 0, then the four copies
// summed over lane bits 3 and 4).
__device__ __forceinline__ float vd_reduce_scatter8(float* acc, int lane) {
#pragma unroll
  for (int s = 4; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = upper ? acc[i] : acc[i + s];
      const float keep = upper ? acc[i + s] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  float v = acc[0];
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// acc[0..31] of every lane -> lane L returns the warp's sum of acc[L]
// (recursive halving over lane bits 4..0: 31 shuffles).
__device__ __forceinline__ float vd_reduce_scatter32(float* acc, int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = upper ? acc[i] : acc[i + s];
      const float keep = upper ? acc[i + s] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return acc[0];
}

// Grid (pixel blocks, root groups of 32): block (b, g) scores the group's
// roots against pixel block b's contiguous range of rigid pixels; warps
// take passes of 32 x SCORE_PPT pixels in turn (pixels in registers), and
// per pass the roots eight at a time: every lane accumulates one sum per
// root over its pixels, then a reduce-scatter gives lane k < 8 the warp's
// sum of root k.  Warp sums are added in fixed order, so the result does
// not depend on scheduling.
template <int THREADS, bool FAST = false>
__global__ void __launch_bounds__(THREADS)
k_pose_score(DevParams P, const float4* __restrict__ rpts, const float4* __restrict__ robs,
             const int* __restrict__ n_ptr, int n_host, const float* __restrict__ rootsf,
             const int* __restrict__ root_count, int M, float* __restrict__ partial) {
  extern __shared__ float smem[];
  constexpr int nwarp = THREADS / 32;
  constexpr int PASS = 32 * SCORE_PPT;
  float* sRoot = smem;                       // 32 * 12: this group's roots
  float* sAcc = smem + 32 * 12;              // nwarp * 32
  int* sList = (int*)(sAcc + nwarp * 32);    // the real roots, in index order
  int* sNum = sList + M;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = n_ptr ? *n_ptr : n_host;     // issued early: its latency overlaps the prologue
  if (wid == 0) {
    // compact the roots that exist (slot r & 3 below its sample's root
    // count), in index order: every sample's count loaded at once, then a
    // warp prefix sum per 32 samples
    if (!root_count) {
      for (int r = lane; r < M; r += 32) sList[r] = r;
      if (lane == 0) *sNum = M;
    } else {
      const int S = M >> 2;
      int c[VD_MAX_SAMPLES / 32];
#pragma unroll
      for (int k = 0; k < VD_MAX_SAMPLES / 32; ++k) {
        const int g = 32 * k + lane;
        c[k] = g < S ? root_count[g] : 0;
      }
      int base = 0;
#pragma unroll
      for (int k = 0; k < VD_MAX_SAMPLES / 32; ++k) {
        if (32 * k >= S) break;                 // warp-uniform
        int pre = c[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int up = __shfl_up_sync(0xffffffffu, pre, o);
          if (lane >= o) pre += up;
        }
        const int g = 32 * k + lane;
        for (int i = 0; i < c[k]; ++i) sList[base + pre - c[k] + i] = 4 * g + i;
        base += __shfl_sync(0xffffffffu, pre, 31);
      }
      if (lane == 0) *sNum = base;
    }
  }
  for (int i = threadIdx.x; i < nwarp * 32; i += THREADS) sAcc[i] = 0.0f;
  __syncthreads();
  const int nroot = *sNum;
  const int g0 = 32 * blockIdx.y;
  if (g0 >= nroot) return;                   // whole block: no root in this group
  const int ng = min(32, nroot - g0);
  for (int i = threadIdx.x; i < 12 * ng; i += THREADS)
    sRoot[i] = rootsf[12 * sList[g0 + i / 12] + i % 12];
  __syncthreads();
  // contiguous pixel-block ranges of whole passes; passes go to the warps in turn
  const int per = ((n + gridDim.x - 1) / gridDim.x + PASS - 1) / PASS * PASS;
  const int beg = min(n, blockIdx.x * per);
  const int end = min(n, beg + per);
  float* wAcc = sAcc + wid * 32;             // this warp's sum per root of the group
  for (int base = beg + wid * PASS; base < end; base += nwarp * PASS) {
    float4 pt[SCORE_PPT], ob[SCORE_PPT];
#pragma unroll
    for (int k = 0; k < SCORE_PPT; ++k) {
      const int i = base + 32 * k + lane;
      if (i < end) {
        pt[k] = rpts[i];
        ob[k] = robs[i];
      } else {
        pt[k] = make_float4(0.f, 0.f, 1.f, 0.f);   // weight 0
        ob[k] = make_float4(0.f, 0.f, 1.f, 0.f);
      }
    }
#pragma unroll 1
    for (int r0 = 0; r0 < ng; r0 += 8) {
      float acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        acc[k] = 0.0f;
        if (r0 + k < ng) {                    // warp-uniform
          const float* Mr = sRoot + 12 * (r0 + k);
#pragma unroll
          for (int q = 0; q < SCORE_PPT; ++q)
            acc[k] = fmaf(pt[q].w, vd_score_term2<FAST>(P, Mr, pt[q], ob[q]), acc[k]);
        }
      }
      const float v = vd_reduce_scatter8(acc, lane);
      if (lane < 8 && r0 + lane < ng) wAcc[r0 + lane] += v;
    }
  }
  // the block's sum per root, warps in fixed order
  __syncthreads();
  if (threadIdx.x < ng) {
    float s = 0.0f;
    for (int w = 0; w < nwarp; ++w) s += sAcc[w * 32 + threadIdx.x];
    partial[(size_t)sList[g0 + threadIdx.x] * gridDim.x + blockIdx.x] = VD_LN2 * s;
  }
}

// float64 sum of the block partials of every root that exists (infinity for
// the others): one warp per root, each lane sums a strided subset, then a
// fixed-order butterfly over the lanes.
// With work non-null, each block adds (rigid pixels x its real roots) to
// *work (the scoring's evaluation count, read by the profiling).
__global__ void k_root_energy(const float* __restrict__ partial, int nblk, int M,
                              const int* __restrict__ root_count, double* __restrict__ energy,
                              const int* __restrict__ n_ptr, unsigned long long* __restrict__ work) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool real = r < M && !(root_count && (r & 3) >= root_count[r >> 2]);
  if (work) {
    const int nreal = __syncthreads_count(real && lane == 0);
    if (threadIdx.x == 0 && nreal) atomicAdd(work, (unsigned long long)*n_ptr * nreal);
  }
  if (r >= M) return;                 // whole warps leave together
  if (!real) {
    if (lane == 0) energy[r] = INFINITY;
    return;
  }
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += (double)partial[(size_t)r * nblk + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) energy[r] = s;
}

static inline cudaError_t launch_root_energy(const float* partial, int nblk, int M,
                                             const int* root_count, double* energy,
                                             cudaStream_t s, const int* n_ptr = nullptr,
                                             unsigned long long* work = nullptr) {
  k_root_energy<<<(M + 3) / 4, 128, 0, s>>>(partial, nblk, M, root_count, energy, n_ptr, work);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// float32 se(3) maps for the mean-shift iterations, whose arguments are
// poses relative to the current mode (small unless the sample is far away,
// in which case its Gaussian weight is zero anyway).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool vd_se3_log_f(const float* T, float* xi) {
  const float c = 0.5f * (T[0] + T[5] + T[10] - 1.0f);
  const float vx = 0.5f * (T[9] - T[6]), vy = 0.5f * (T[2] - T[8]), vz = 0.5f * (T[4] - T[1]);
  const float s = sqrtf(vx * vx + vy * vy + vz * vz);
  if (c < 0.0f && s < 1e-3f) return false;   // rotation by ~pi: weight 0
  const float th = atan2f(s, c);
  const float f = s < 1e-6f ? 1.0f + th * th * (1.0f / 6.0f) : th / s;
  const float wx = vx * f, wy = vy * f, wz = vz * f;
  const float th2 = wx * wx + wy * wy + wz * wz;
  // e = (1 - (th/2) cot(th/2)) / th^2 = 1/12 + th^2/720 + th^4/30240 + ...
  float e;
  if (th2 < 1e-2f) {
    e = (1.0f / 12.0f) + th2 * ((1.0f / 720.0f) + th2 * (1.0f / 30240.0f));
  } else {
    const float t = sqrtf(th2);
    float sn, cs;
    sincosf(t, &sn, &cs);
    e = (1.0f - (t * sn) / (2.0f * (1.0f - cs))) / th2;
  }
  const float t0 = T[3], t1 = T[7], t2 = T[11];
  // [w]x t and [w]x^2 t
  const float k0 = wy * t2 - wz * t1, k1 = wz * t0 - wx * t2, k2 = wx * t1 - wy * t0;
  const float q0 = wy * k2 - wz * k1, q1 = wz * k0 - wx * k2, q2 = wx * k1 - wy * k0;
  xi[0] = wx;
  xi[1] = wy;
  xi[2] = wz;
  xi[3] = t0 - 0.5f * k0 + e * q0;
  xi[4] = t1 - 0.5f * k1 + e * q1;
  xi[5] = t2 - 0.5f * k2 + e * q2;
  return true;
}

// vd_se3_log_f for the mean-shift's samples when the rotation kernel is
// narrow: a sample whose rotation part alone has Mahalanobis distance
// s^2 ivr >= 210 (s = sin of its angle) has weight exp(-m / 2) <= e^-105,
// which is 0 in float32: it returns false with no logarithm.  Near samples
// (angle below 14.5 sigma, cos > 0) take the angle asin(s) and the
// coefficient e of the translation part from their series (truncation below
// 1e-10 relative at that angle), without atan2f or sincosf.
__device__ __forceinline__ bool vd_se3_log_near_f(const float* T, float* xi, float ivr) {
  const float c = 0.5f * (T[0] + T[5] + T[10] - 1.0f);
  const float vx = 0.5f * (T[9] - T[6]), vy = 0.5f * (T[2] - T[8]), vz = 0.5f * (T[4] - T[1]);
  const float s2 = vx * vx + vy * vy + vz * vz;
  if (!(c > 0.0f) || s2 * ivr >= 210.0f) return false;
  // th / s = asin(s) / s = 1 + s^2/6 + 3 s^4/40 + 5 s^6/112 + 35 s^8/1152
  const float f = fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 35.0f / 1152.0f, 5.0f / 112.0f),
                                         3.0f / 40.0f), 1.0f / 6.0f), 1.0f);
  const float wx = vx * f, wy = vy * f, wz = vz * f;
  const float th2 = wx * wx + wy * wy + wz * wz;
  // e = (1 - (th/2) cot(th/2)) / th^2 = 1/12 + th^2/720 + th^4/30240 + th^6/1209600
  const float e = fmaf(th2, fmaf(th2, fmaf(th2, 1.0f / 1209600.0f, 1.0f / 30240.0f),
                                 1.0f / 720.0f), 1.0f / 12.0f);
  const float t0 = T[3], t1 = T[7], t2 = T[11];
  const float k0 = wy * t2 - wz * t1, k1 = wz * t0 - wx * t2, k2 = wx * t1 - wy * t0;
  const float q0 = wy * k2 - wz * k1, q1 = wz * k0 - wx * k2, q2 = wx * k1 - wy * k0;
  xi[0] = wx;
  xi[1] = wy;
  xi[2] = wz;
  xi[3] = t0 - 0.5f * k0 + e * q0;
  xi[4] = t1 - 0.5f * k1 + e * q1;
  xi[5] = t2 - 0.5f * k2 + e * q2;
  return true;
}

__device__ __forceinline__ void vd_se3_exp_f(const float* xi, float* T) {
  const float wx = xi[0], wy = xi[1], wz = xi[2];
  const float th2 = wx * wx + wy * wy + wz * wz;
  float a, b, cc;
  if (th2 < 1e-2f) {
    a = 1.0f - th2 * ((1.0f / 6.0f) - th2 * (1.0f / 120.0f));
    b = 0.5f - th2 * ((1.0f / 24.0f) - th2 * (1.0f / 720.0f));
    cc = (1.0f / 6.0f) - th2 * ((1.0f / 120.0f) - th2 * (1.0f / 5040.0f));
  } else {
    const float th = sqrtf(th2);
    float s, c;
    sincosf(th, &s, &c);
    a = s / th;
    b = (1.0f - c) / th2;
    cc = (th - s) / (th2 * th);
  }
  const float K[9] = {0, -wz, wy, wz, 0, -wx, -wy, wx, 0};
  float K2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
  float V[9];
  for (int i = 0; i < 9; ++i) {
    const float I = (i % 4 == 0) ? 1.0f : 0.0f;
    T[4 * (i / 3) + (i % 3)] = I + a * K[i] + b * K2[i];
    V[i] = I + b * K[i] + cc * K2[i];
  }
  for (int r = 0; r < 3; ++r)
    T[4 * r + 3] = V[3 * r] * xi[3] + V[3 * r + 1] * xi[4] + V[3 * r + 2] * xi[5];
}

// ---------------------------------------------------------------------------
// Per sample: the lowest-energy root; then the mode of the sample mixture
// (Sec. III-A, after Eq. 7) from the best sample: the fixed point of the
// mean-shift map x <- x exp(sum w_g d_g / sum w_g), d_g = log(x^-1 T_g),
// w_g = exp(-d^T Sigma^-1 d / 2), reached by safeguarded Newton steps on
// that map (below), at most VD_MS_MAX_ITERS steps.  The float64 definition
// iterates the map itself until |step| < 1e-12.  One warp: the sums are a
// warp reduce-scatter, every lane updates the same mode, no block barrier.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32)
k_select_meanshift(DevParams P, const double* __restrict__ roots, const int* __restrict__ root_count,
                   const float* __restrict__ roots_r, const double* __restrict__ root_energy,
                   int t, double* __restrict__ G, float* __restrict__ posef,
                   float2* __restrict__ posed,
                   double* __restrict__ sample_pose, double* __restrict__ sample_energy,
                   int* __restrict__ degenerate) {
  // one warp; lane l owns samples l, l + 32, ...
  __shared__ float sT[VD_MAX_SAMPLES][12];
  __shared__ unsigned char sValid[VD_MAX_SAMPLES];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  // Energies are sums of non-negative terms (or +inf for a missing root): as
  // bit patterns they order like the numbers, so the comparisons run on the
  // integer pipe instead of the float64 one.
  const long long INF_BITS = __double_as_longlong(INFINITY);
  long long bestE = INF_BITS;
  int bestS = 0x7fffffff;
  // two samples per lane at a time (g and g + 32), their loads in flight
  // together: the counts and all four energy slots (a slot without a root
  // holds +inf), then the kept roots
  for (int g0 = lane; g0 < P.S; g0 += 64) {
    int nr[2];
    long long e[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = g0 + 32 * h;
      nr[h] = g < P.S ? root_count[g] : 0;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        e[h][r] = g < P.S ? __double_as_longlong(root_energy[4 * g + r]) : INF_BITS;
    }
    int best[2];
    long long Eg[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // the sample's lowest-energy root (ties: lower index in the sorted order)
      best[h] = -1;
      Eg[h] = INF_BITS;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < nr[h] && (best[h] < 0 || e[h][r] < Eg[h])) {
          Eg[h] = e[h][r];
          best[h] = r;
        }
      if (best[h] < 0) Eg[h] = INF_BITS;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = g0 + 32 * h;
      if (g >= P.S) continue;
      const double* src = roots + (size_t)48 * g + 12 * (best[h] < 0 ? 0 : best[h]);
      const float* srf = roots_r + (size_t)48 * g + 12 * (best[h] < 0 ? 0 : best[h]);
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        sample_pose[12 * g + i] = best[h] >= 0 ? src[i] : 0.0;
        sT[g][i] = best[h] >= 0 ? srf[i] : 0.0f;
      }
      sample_energy[g] = __longlong_as_double(Eg[h]);
      sValid[g] = Eg[h] < INF_BITS;
      if (Eg[h] < bestE) {      // g ascends per lane: ties keep the lower index
        bestE = Eg[h];
        bestS = g;
      }
    }
  }
  // argmin over samples (lowest energy, then lowest index): a total order, so
  // every lane ends with the same pair
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long oE = __shfl_xor_sync(FULL, bestE, o);
    const int oS = __shfl_xor_sync(FULL, bestS, o);
    if (oE < bestE || (oE == bestE && oS < bestS)) {
      bestE = oE;
      bestS = oS;
    }
  }
  __syncwarp();
  if (!(bestE < INF_BITS)) {
    if (lane == 0) atomicAdd(degenerate, 1);
    return;
  }
  float x[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) x[i] = sT[bestS][i];
  const float tn = sqrtf(x[3] * x[3] + x[7] * x[7] + x[11] * x[11]);
  // kernel widths in float32 (a float64 division costs this part's weak
  // float64 pipe a long dependent sequence)
  const float sr = (float)P.ms_sig_rot, st_ = fmaf((float)P.ms_sig_rel, tn, (float)P.ms_sig_abs);
  const float ivr = 1.0f / (sr * sr), ivt = 1.0f / (st_ * st_);
  // convergence (below): a Newton step under tol, or under 10 tol and no
  // longer halving (the float32 floor of the relative poses, amplified by
  // the mode's conditioning); the float64 definition stops at 1e-12
  const float tol = (float)(VD_MS_TOL_F32 * (1.0 + (double)tn));
  // the narrow-kernel path of the logarithm applies while 14.5 sigma of
  // rotation stays below 0.2 rad (the default sigma is 0.01 rad)
  const bool near_log = 210.0f / ivr < 0.04f;
  // Whitened tangent coordinates z = Sigma^-1/2 d.  The plain step is the
  // weighted mean s of the z_g; it vanishes at the mode.  Moving the mode by
  // delta changes it, to first order, by -(I - C) delta, C the weighted
  // covariance of the z_g about s, so the Newton step is
  // delta = (I - C)^-1 s.  At a mode I - C is positive definite and the
  // plain iteration converges at the rate of C's largest eigenvalue, close
  // to 1 where only a few samples fall in the kernel's reach (as after a
  // rough bootstrap depth): hundreds of steps where Newton takes a few.  The
  // Newton step is taken when the Cholesky pivots of I - C exceed 1e-3 and
  // it stays within one kernel width, else the plain step; either way the
  // fixed point is the plain iteration's.
  const float sq[6] = {sqrtf(ivr), sqrtf(ivr), sqrtf(ivr), sqrtf(ivt), sqrtf(ivt), sqrtf(ivt)};
  float last = INFINITY;
  for (int it = 0; it < VD_MS_MAX_ITERS; ++it) {
    // per lane: w, w z (6), w z_i z_j (21, i <= j), then padding
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
    for (int g = lane; g < P.S; g += 32) {
      if (!sValid[g]) continue;
      const float* Tg = sT[g];
      // relative pose x^-1 T_g (translation error ~|tau| 2^-24, below the stop tolerance)
      float rel[12], d[6];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c)   // (R_x^T R_g)_{rc}
          rel[4 * r + c] = x[r] * Tg[c] + x[4 + r] * Tg[4 + c] + x[8 + r] * Tg[8 + c];
        // R_x^T (tau_g - tau_x)
        rel[4 * r + 3] = x[r] * (Tg[3] - x[3]) + x[4 + r] * (Tg[7] - x[7]) +
                         x[8 + r] * (Tg[11] - x[11]);
      }
      if (near_log ? vd_se3_log_near_f(rel, d, ivr) : vd_se3_log_f(rel, d)) {
        float z[6], m = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          z[i] = d[i] * sq[i];
          m = fmaf(z[i], z[i], m);
        }
        const float w = __expf(-0.5f * m);
        acc[0] += w;
        int k = 7;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const float wz = w * z[i];
          acc[1 + i] += wz;
#pragma unroll
          for (int j = i; j < 6; ++j, ++k) acc[k] = fmaf(wz, z[j], acc[k]);
        }
      }
    }
    // lane L ends with the warp's sum of acc[L] (each sum formed once, in a
    // fixed order), then every lane reads all 28
    const float mine = vd_reduce_scatter32(acc, lane);
    float v[28];
#pragma unroll
    for (int k = 0; k < 28; ++k) v[k] = __shfl_sync(FULL, mine, k);
    if (!(v[0] > 0.0f)) break;
    const float iw = 1.0f / v[0];
    float sz[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) sz[i] = v[1 + i] * iw;
    // A = I - C (packed lower triangle, row by row), then its Cholesky factor
    float A[21];
    {
      int k = 7;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j, ++k)
          A[j * (j + 1) / 2 + i] = (i == j ? 1.0f : 0.0f) - (v[k] * iw - sz[i] * sz[j]);
    }
    bool newton = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float dj = A[j * (j + 1) / 2 + j];
#pragma unroll
      for (int k = 0; k < j; ++k) dj -= A[j * (j + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
      newton = newton && dj > 1e-3f;
      const float lj = sqrtf(fmaxf(dj, 1e-3f));
      A[j * (j + 1) / 2 + j] = lj;
      const float il = 1.0f / lj;
#pragma unroll
      for (int i = j + 1; i < 6; ++i) {
        float a = A[i * (i + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) a -= A[i * (i + 1) / 2 + k] * A[j * (j + 1) / 2 + k];
        A[i * (i + 1) / 2 + j] = a * il;
      }
    }
    // (L L^T) y = s_z
    float y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float a = sz[i];
#pragma unroll
      for (int k = 0; k < i; ++k) a -= A[i * (i + 1) / 2 + k] * y[k];
      y[i] = a / A[i * (i + 1) / 2 + i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
      float a = y[i];
#pragma unroll
      for (int k = i + 1; k < 6; ++k) a -= A[k * (k + 1) / 2 + i] * y[k];
      y[i] = a / A[i * (i + 1) / 2 + i];
    }
    float mh = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) mh = fmaf(y[i], y[i], mh);
    newton = newton && mh <= 1.0f;
    float step[6], nrm = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      step[i] = (newton ? y[i] : sz[i]) / sq[i];
      nrm = fmaf(step[i], step[i], nrm);
    }
    nrm = sqrtf(nrm);
    const bool converged = newton ? (nrm < tol || (nrm < 10.0f * tol && nrm > 0.5f * last))
                                  : nrm < tol;
    if (newton) last = nrm;
    float E[12], xn[12];
    vd_se3_exp_f(step, E);
#pragma unroll
    for (int r = 0; r < 3; ++r) {   // x <- x o exp(step)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        xn[4 * r + c] = x[4 * r] * E[c] + x[4 * r + 1] * E[4 + c] + x[4 * r + 2] * E[8 + c];
      xn[4 * r + 3] = x[4 * r] * E[3] + x[4 * r + 1] * E[7] + x[4 * r + 2] * E[11] + x[4 * r + 3];
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) x[i] = xn[i];
    if (converged) break;
  }
  // re-orthonormalise the rotation (Gram-Schmidt on the rows, third row as
  // the cross product) in double-float on the FP32 pipe, every lane alike;
  // lane i < 12 stores entry i of the pose and of its float K R | K tau
  vd_df R[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) R[3 * r + c] = vd_df_make(x[4 * r + c]);
  {
    const vd_df s0 = vd_df_add(vd_df_add(vd_df_mul(R[0], R[0]), vd_df_mul(R[1], R[1])),
                               vd_df_mul(R[2], R[2]));
    const vd_df i0 = vd_df_rsqrt(s0);
#pragma unroll
    for (int c = 0; c < 3; ++c) R[c] = vd_df_mul(R[c], i0);
    const vd_df d01 = vd_df_add(vd_df_add(vd_df_mul(R[0], R[3]), vd_df_mul(R[1], R[4])),
                                vd_df_mul(R[2], R[5]));
#pragma unroll
    for (int c = 0; c < 3; ++c) R[3 + c] = vd_df_sub(R[3 + c], vd_df_mul(d01, R[c]));
    const vd_df s1 = vd_df_add(vd_df_add(vd_df_mul(R[3], R[3]), vd_df_mul(R[4], R[4])),
                               vd_df_mul(R[5], R[5]));
    const vd_df i1 = vd_df_rsqrt(s1);
#pragma unroll
    for (int c = 0; c < 3; ++c) R[3 + c] = vd_df_mul(R[3 + c], i1);
    R[6] = vd_df_sub(vd_df_mul(R[1], R[5]), vd_df_mul(R[2], R[4]));
    R[7] = vd_df_sub(vd_df_mul(R[2], R[3]), vd_df_mul(R[0], R[5]));
    R[8] = vd_df_sub(vd_df_mul(R[0], R[4]), vd_df_mul(R[1], R[3]));
  }
  double o[12];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) o[4 * r + c] = vd_df_to(R[3 * r + c]);
    o[4 * r + 3] = (double)x[4 * r + 3];
  }
  if (lane < 12) {
    G[12 * t + lane] = o[lane];
    // K R | K tau of the updated pose: row lane / 4, column lane % 4
    const int i = lane & 3, row = lane >> 2;
    float* pf = posef + 12 * t;
    float2* pd = posed + 12 * t;
    if (row == 0) vd_store_pose_entry(pf, pd, i < 3 ? i : 9, P.fx_d * o[i] + P.cx_d * o[8 + i]);
    else if (row == 1)
      vd_store_pose_entry(pf, pd, i < 3 ? 3 + i : 10, P.fy_d * o[4 + i] + P.cy_d * o[8 + i]);
    else vd_store_pose_entry(pf, pd, i < 3 ? 6 + i : 11, o[8 + i]);
  }
}

// Largest dynamic shared memory of the scoring kernel (VD_MAX_SAMPLES
// samples of 4 roots), granted once per device so that no launch, and no
// stream capture, has to change a function attribute.
cudaError_t vd_pose_prepare(void) {
  const int M = 4 * VD_MAX_SAMPLES;
  const int s256 = (int)vd_score_smem(M, 256), s512 = (int)vd_score_smem(M, 512);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_pose_score<256, false>, a, s256);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pose_score<256, true>, a, s256);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pose_score<512, false>, a, s512);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pose_score<512, true>, a, s512);
  return e;
}

// Dense scoring of the current roots against the current rigid set, then the
// float64 sum of the block partials: score_bps blocks per SM.
cudaError_t launch_pose_score_only(vd_ctx* c) {
  const DevParams& P = c->dp;
  const int M = 4 * P.S;
  // pixel blocks: half an SM's worth per unit of score_bps; the grid's
  // second dimension covers the root groups of 32 (those without a root exit)
  const int nblk = std::max(1, c->score_bps * c->num_sms / 2);
  const dim3 grid(nblk, (M + 31) / 32);
#define VD_SCORE_LAUNCH(TH, FAST)                                                     \
  k_pose_score<TH, FAST><<<grid, TH, vd_score_smem(M, TH), c->stream>>>(                   \
      P, c->rpts, c->robs, c->n_rigid, 0, c->rootsf, c->root_count, M, c->partial)
  if (c->score_threads == 512) {
    if (P.fast_beta2) VD_SCORE_LAUNCH(512, true);
    else VD_SCORE_LAUNCH(512, false);
  } else {
    if (P.fast_beta2) VD_SCORE_LAUNCH(256, true);
    else VD_SCORE_LAUNCH(256, false);
  }
#undef VD_SCORE_LAUNCH
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_root_energy(c->partial, nblk, M, c->root_count, c->root_energy, c->stream,
                            c->n_rigid, c->score_work);
}

cudaError_t launch_pose_frame(vd_ctx* c, uint32_t itcode, int t) {
  const DevParams& P = c->dp;
  c->last_pose_t = t;
  c->samples_set |= 1u << (t - 1);
  const size_t f = (size_t)(t - 1) * VD_MAX_SAMPLES;   // this frame's sample slots
  vd_prof_begin(c, VD_ST_RIGID);
  k_rigid_flags<<<c->nblk_scan, SCAN_BLOCK, 0, c->stream>>>(P, c->G, c->posef, c->rho, c->q, t,
                                                            c->flags, c->blk_counts);
  k_rigid_scatter<<<c->nblk_scan, SCAN_BLOCK, 0, c->stream>>>(P, c->posef, c->flow, c->rho, c->q, t,
                                                              c->flags, c->blk_counts,
                                                              c->n_rigid, c->rigid_idx, c->rpts,
                                                              c->robs);
  vd_prof_end(c, VD_ST_RIGID, 2);
  vd_prof_begin(c, VD_ST_P3P);
  k_p3p_samples<<<(P.S + VD_P3P_WARPS - 1) / VD_P3P_WARPS, 32 * VD_P3P_WARPS, 0, c->stream>>>(
      P, c->G, c->flow, c->rho, c->rigid_idx,
                                            c->n_rigid, t, itcode, c->roots, c->root_count,
                                            c->rootsf, c->rootsr);
  vd_prof_end(c, VD_ST_P3P, 1);
  vd_prof_begin(c, VD_ST_SCORE);
  launch_pose_score_only(c);
  vd_prof_end(c, VD_ST_SCORE, 2);
  vd_prof_begin(c, VD_ST_SELECT);
  k_select_meanshift<<<1, 32, 0, c->stream>>>(P, c->roots, c->root_count, c->rootsr,
                                               c->root_energy, t, c->G,
                                               c->posef, c->posed, c->sample_pose + 12 * f,
                                               c->sample_energy + f, c->degenerate);
  vd_prof_end(c, VD_ST_SELECT, 1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Standalone dense scoring on caller buffers (allocates its partial sums).
// ---------------------------------------------------------------------------
__global__ void k_poses_float(DevParams P, const double* __restrict__ poses, int m,
                              float* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double* g = poses + 12 * r;
  float* o = out + 12 * r;
  for (int i = 0; i < 4; ++i) {
    o[i < 3 ? i : 9] = (float)(P.fx_d * g[i] + P.cx_d * g[8 + i]);
    o[i < 3 ? 3 + i : 10] = (float)(P.fy_d * g[4 + i] + P.cy_d * g[8 + i]);
    o[i < 3 ? 6 + i : 11] = (float)g[8 + i];
  }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the standalone scoring: its scratch (float
// K R | K tau of every pose, then the per-block partial sums) lives in this
// fixed device array instead of memory allocated per call.
// ---------------------------------------------------------------------------
#define VD_NOALLOC_MAX_BLOCKS 512
#define VD_NOALLOC_FLOATS (VD_NOALLOC_MAX_POSES * (12 + VD_NOALLOC_MAX_BLOCKS))
static __device__ __align__(256) float g_noalloc_scratch[VD_NOALLOC_FLOATS];

#define VD_NOALLOC_MAX_DEVICES 64
static float* g_noalloc_ptr[VD_NOALLOC_MAX_DEVICES];
static int g_noalloc_blocks[VD_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device and the block
// count of its scoring launch (two per SM, at most VD_NOALLOC_MAX_BLOCKS),
// looked up once per device with that device current (host code must not
// use the symbol itself, which is only a host-side stand-in).
static cudaError_t noalloc_scratch(float** out, int* nblk) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= VD_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_blocks[dev] = std::max(1, std::min(2 * sms, VD_NOALLOC_MAX_BLOCKS));
    g_noalloc_ptr[dev] = (float*)p;
  }
  *out = g_noalloc_ptr[dev];
  *nblk = g_noalloc_blocks[dev];
  return cudaSuccess;
}

extern "C" vd_status vd_score_poses_noalloc(const float* points, const float* obs, int n,
                                            const double* poses, int m, const double* intrinsics,
                                            float beta, float p0, double* energies,
                                            void* cuda_stream) {
  if ((n > 0 && (!points || !obs)) || !poses || !intrinsics || !energies || n < 0 ||
      !(beta > 0.0f) || !(p0 > 0.0f))
    return VD_ERR_ARG;
  if (m < 1 || m > VD_NOALLOC_MAX_POSES) {
    vd_set_error("vd_score_poses_noalloc: m must be between 1 and VD_NOALLOC_MAX_POSES (256)");
    return VD_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  float* scratch = nullptr;
  int nblk = 0;
  cudaError_t e = noalloc_scratch(&scratch, &nblk);
  double K[4];
  if (e == cudaSuccess) e = cudaMemcpy(K, intrinsics, sizeof K, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  DevParams P{};
  P.fx_d = K[0]; P.fy_d = K[1]; P.cx_d = K[2]; P.cy_d = K[3];
  P.beta = beta;
  P.p0 = p0;
  P.fast_beta2 = 0;           // the per-point scale rides in obs.z
  P.cgen = p0 * 2.0f * 3.14159265358979f / beta;
  float* rootsf = scratch;                                  // m x 12
  float* partial = scratch + 12 * VD_NOALLOC_MAX_POSES;     // m x nblk
  k_poses_float<<<(m + 127) / 128, 128, 0, s>>>(P, poses, m, rootsf);
  const size_t smem = vd_score_smem(m, SCORE_THREADS);
  k_pose_score<SCORE_THREADS><<<dim3(nblk, (m + 31) / 32), SCORE_THREADS, smem, s>>>(
      P, (const float4*)points, (const float4*)obs, nullptr, n, rootsf, nullptr, m, partial);
  launch_root_energy(partial, nblk, m, nullptr, energies, s);
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  return VD_OK;
}

extern "C" vd_status vd_score_poses(const float* points, const float* obs, int n, const double* poses,
                                    int m, const double* intrinsics, float beta, float p0,
                                    double* energies, void* cuda_stream) {
  if ((n > 0 && (!points || !obs)) || !poses || !intrinsics || !energies || n < 0 || m < 1 ||
      m > 1024 || !(beta > 0.0f) || !(p0 > 0.0f))
    return VD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double K[4];
  if (cudaMemcpy(K, intrinsics, sizeof K, cudaMemcpyDefault) != cudaSuccess) {
    vd_set_error(cudaGetErrorString(cudaGetLastError()));
    return VD_ERR_CUDA;
  }
  DevParams P{};
  P.fx_d = K[0]; P.fy_d = K[1]; P.cx_d = K[2]; P.cy_d = K[3];
  P.beta = beta;
  P.p0 = p0;
  P.fast_beta2 = 0;           // the per-point scale rides in obs.z
  P.cgen = p0 * 2.0f * 3.14159265358979f / beta;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    vd_set_error(cudaGetErrorString(cudaGetLastError()));
    return VD_ERR_CUDA;
  }
  const int nblk = 2 * std::max(sms, 1);
  float* rootsf = nullptr;
  float* partial = nullptr;
  cudaError_t e = cudaMallocAsync(&rootsf, sizeof(float) * 12 * m, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&partial, sizeof(float) * (size_t)m * nblk, s);
  if (e != cudaSuccess) {
    if (rootsf) cudaFreeAsync(rootsf, s);
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_OOM;
  }
  k_poses_float<<<(m + 127) / 128, 128, 0, s>>>(P, poses, m, rootsf);
  const size_t smem = vd_score_smem(m, SCORE_THREADS);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_pose_score<SCORE_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  k_pose_score<SCORE_THREADS><<<dim3(nblk, (m + 31) / 32), SCORE_THREADS, smem, s>>>(
      P, (const float4*)points, (const float4*)obs, nullptr, n, rootsf, nullptr, m, partial);
  launch_root_energy(partial, nblk, m, nullptr, energies, s);
  e = cudaGetLastError();
  cudaFreeAsync(rootsf, s);
  cudaFreeAsync(partial, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  return VD_OK;
}

VD_CHECK_ACCESSOR(pose)
