// Pose M-step of VOLDOR+ (Sec. III-A, Eq. 7): the posterior of each camera
// pose is approximated by S P3P samples drawn from the rigid pixels; every
// root is scored against all rigid pixels, each sample keeps its best root,
// and the pose is the mean-shift mode of the samples in se(3).
#include <algorithm>
#include <mutex>

#include "vd_device.cuh"
#include "vd_geom64.cuh"

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

// Exclusive scan of the block counts by one block; total into n_out.
__global__ void k_scan_counts(const int* __restrict__ counts, int nblk, int* __restrict__ offsets,
                              int* __restrict__ n_out) {
  __shared__ int s[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += 1024) {
    const int i = base + threadIdx.x;
    const int x = i < nblk ? counts[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int y = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < nblk) offsets[i] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = carry;
}

// Scatter the rigid pixels in row-major order with their float32 scoring data:
// X = r_j / rho_j (reference frame), x_obs = x_{t-1} + X_t(x_{t-1}), w = q_t.
__global__ void __launch_bounds__(SCAN_BLOCK)
k_rigid_scatter(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
                const float* __restrict__ rho, const float* __restrict__ q, int t,
                const unsigned char* __restrict__ flags, const int* __restrict__ offsets,
                int* __restrict__ idx, float4* __restrict__ rpts, float4* __restrict__ robs) {
  __shared__ int warp_tot[SCAN_BLOCK / 32];
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  const int f = (j < npix) ? flags[j] : 0;
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) warp_tot[wid] = __popc(bal);
  __syncthreads();
  int before = 0;
  for (unsigned w = 0; w < wid; ++w) before += warp_tot[w];
  before += __popc(bal & ((1u << lane) - 1u));
  if (!f) return;
  const int pos = offsets[blockIdx.x] + before;
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
// One thread per sample: three distinct indices into the rigid set, float64
// correspondences, P3P, roots ordered by (rotation vector, translation).
// ---------------------------------------------------------------------------
__device__ void vd_correspondence64(const DevParams& P, const double* __restrict__ G,
                                    const float2* __restrict__ flow, const float* __restrict__ rho,
                                    int t, int j, double* X, double* bearing) {
  const int v = j / P.W, u = j - v * P.W;
  const double c = (double)rho[j];
  const double rx = ((double)u - P.cx_d) / P.fx_d, ry = ((double)v - P.cy_d) / P.fy_d;
  X[0] = rx / c;
  X[1] = ry / c;
  X[2] = 1.0 / c;
  const size_t npix = (size_t)P.W * P.H;
  double xp, yp, fx, fy;
  if (t == 1) {
    xp = u;
    yp = v;
    const float2 F = flow[j];
    fx = F.x;
    fy = F.y;
  } else {
    xp = 0.0;
    yp = 0.0;
    vd_track64(P, G + 12 * (t - 1), u, v, c, &xp, &yp);
    // members of the rigid set are inside the image; the clamp only guards
    // the gather against a non-finite position
    xp = fmin(fmax(xp, 0.0), (double)(P.W - 1));
    yp = fmin(fmax(yp, 0.0), (double)(P.H - 1));
    if (!(xp == xp)) xp = 0.0;
    if (!(yp == yp)) yp = 0.0;
    vd_bilinear64(flow + (size_t)(t - 1) * npix, P.W, P.H, xp, yp, &fx, &fy);
  }
  const double xo = xp + fx, yo = yp + fy;
  bearing[0] = (xo - P.cx_d) / P.fx_d;
  bearing[1] = (yo - P.cy_d) / P.fy_d;
  bearing[2] = 1.0;
}

// Real roots of a polynomial of exact degree `deg` split by the sorted points
// `crit`, with the interval searches spread over the lanes of a warp: the
// intervals and the bracketed search are those of vd_roots_between, so the
// roots are bitwise the same; every lane receives all roots.
__device__ int vd_roots_between_warp(const double* c, int deg, const double* crit, int ncrit,
                                     double* out, int lane) {
  const double bound = vd_root_bound(c, deg);
  double lo = -bound;
  double flo = vd_poly_eval(c, deg, lo);
  double mlo = 0.0, mhi = 0.0;      // this lane's interval
  int mkind = 0;                    // 0 none, 1 root at lo, 2 search
  int kinds = 0;                    // 2 bits per interval
  int ni = 0;
  for (int i = 0; i <= ncrit; ++i) {
    const double hi = i < ncrit ? fmin(fmax(crit[i], -bound), bound) : bound;
    if (!(hi > lo)) continue;
    const double fhi = vd_poly_eval(c, deg, hi);
    const int kind = flo == 0.0 ? 1 : (((flo < 0.0) != (fhi < 0.0) && fhi != 0.0) ? 2 : 0);
    kinds |= kind << (2 * ni);
    if (ni == lane) {
      mlo = lo;
      mhi = hi;
      mkind = kind;
    }
    ++ni;
    lo = hi;
    flo = fhi;
  }
  const double mine = mkind == 2 ? vd_poly_bracketed_root(c, deg, mlo, mhi) : mlo;
  int n = 0;
  for (int k = 0; k < 5; ++k) {
    const double r = __shfl_sync(0xffffffffu, mine, k);
    if (k < ni && ((kinds >> (2 * k)) & 3)) out[n++] = r;
  }
  return n;
}

// The real roots of the P3P quartic as vd_poly_real_roots finds them
// (second derivative, first derivative, quartic), each stage's interval
// searches in parallel lanes.
__device__ int vd_quartic_roots_warp(const double* cin, double* out, int lane) {
  double mx = 0.0;
  for (int i = 0; i <= 4; ++i) mx = fmax(mx, fabs(cin[i]));
  if (mx == 0.0) return 0;
  if (fabs(cin[4]) <= 1e-14 * mx) return vd_poly_real_roots(cin, 4, out);   // lower degree
  const double q[3] = {cin[2] * 2.0, cin[3] * 6.0, cin[4] * 12.0};
  const double split = -q[1] / (2.0 * q[2]);
  double r2[2];
  const int n2 = vd_roots_between_warp(q, 2, &split, 1, r2, lane);
  const double cc[4] = {cin[1], cin[2] * 2.0, cin[3] * 3.0, cin[4] * 4.0};
  double r3[3];
  const int n3 = vd_roots_between_warp(cc, 3, r2, n2, r3, lane);
  return vd_roots_between_warp(cin, 4, r3, n3, out, lane);
}

// One warp per sample (samples spread over the SMs: the float64 pipe is
// narrow, so the solve is latency-bound per warp).  Lanes 0-2 build the three
// correspondences, every lane forms the quartic, lanes 0-3 turn one root each
// into a pose and its ordering key; each lane then finds its rank.
__global__ void __launch_bounds__(32)
k_p3p_samples(DevParams P, const double* __restrict__ G, const float2* __restrict__ flow,
              const float* __restrict__ rho, const int* __restrict__ idx,
              const int* __restrict__ n_rigid, int t, uint32_t itcode, double* __restrict__ roots,
              int* __restrict__ root_count) {
  const int g = blockIdx.x;
  const int lane = threadIdx.x;
  if (g >= P.S) return;
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
    return;
  }
  double Xl[3] = {0, 0, 0}, fl[3] = {0, 0, 1};
  if (lane < 3)
    vd_correspondence64(P, G, flow, rho, t, idx[pick[lane < 3 ? lane : 0]], Xl, fl);
  double X[9], f[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X[3 * k + c] = __shfl_sync(0xffffffffu, Xl[c], k);
      f[3 * k + c] = __shfl_sync(0xffffffffu, fl[c], k);
    }
  VdP3P geo;
  double v[4], res[5];
  const int nr = vd_p3p_quartic(f, X, &geo, res) < 0 ? 0 : vd_quartic_roots_warp(res, v, lane);
  double T[12];
  bool valid = false;
  if (lane < 4 && lane < nr) valid = vd_p3p_pose(geo, X, v[lane], T);
  double key[6] = {0, 0, 0, 0, 0, 0};
  if (valid) {
    // ordering key: rotation vector (float32 is plenty to order distinct
    // roots; the float64 logarithm near a half turn), then the translation
    const float cf = 0.5f * ((float)T[0] + (float)T[5] + (float)T[10] - 1.0f);
    if (cf < -0.9f) {
      vd_so3_log(T, key);
    } else {
      const float vx = 0.5f * (float)(T[9] - T[6]), vy = 0.5f * (float)(T[2] - T[8]);
      const float vz = 0.5f * (float)(T[4] - T[1]);
      const float s = sqrtf(vx * vx + vy * vy + vz * vz);
      const float th = atan2f(s, cf);
      const float fk = s < 1e-6f ? 1.0f + th * th * (1.0f / 6.0f) : th / s;
      key[0] = vx * fk;
      key[1] = vy * fk;
      key[2] = vz * fk;
    }
    key[3] = T[3];
    key[4] = T[7];
    key[5] = T[11];
  }
  // rank among the valid roots by (rotation vector, translation), ties by lane
  int rank = 0, count = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool vk = __shfl_sync(0xffffffffu, valid, k);
    double kk[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) kk[i] = __shfl_sync(0xffffffffu, key[i], k);
    if (!vk) continue;
    ++count;
    if (!valid || k == lane) continue;
    int cmp = 0;
    for (int i = 0; i < 6 && cmp == 0; ++i) cmp = kk[i] < key[i] ? -1 : (kk[i] > key[i] ? 1 : 0);
    if (cmp < 0 || (cmp == 0 && k < lane)) ++rank;
  }
  double* out = roots + (size_t)g * 48;
  if (valid)
    for (int i = 0; i < 12; ++i) out[12 * rank + i] = T[i];
  if (lane == 0) root_count[g] = count;
}

// float K R | K tau of every root slot (invalid slots: zero).
__global__ void k_roots_float(DevParams P, const double* __restrict__ roots,
                              const int* __restrict__ root_count, float* __restrict__ rootsf) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 4 * P.S) return;
  float* o = rootsf + 12 * r;
  if ((r & 3) >= root_count[r >> 2]) {
    for (int i = 0; i < 12; ++i) o[i] = 0.0f;
    return;
  }
  const double* g = roots + 12 * r;
  for (int i = 0; i < 4; ++i) {
    o[i < 3 ? i : 9] = (float)(P.fx_d * g[i] + P.cx_d * g[8 + i]);
    o[i < 3 ? 3 + i : 10] = (float)(P.fy_d * g[4 + i] + P.cy_d * g[8 + i]);
    o[i < 3 ? 6 + i : 11] = (float)g[8 + i];
  }
}

// ---------------------------------------------------------------------------
// Dense scoring: every root against every rigid pixel.  Each block owns a
// contiguous range of rigid pixels, keeps SCORE_PPT of them per thread in
// registers and loops over the roots (broadcast from shared memory); warp
// sums go to per-warp shared slots, summed in fixed order at the end.
// ---------------------------------------------------------------------------
// One pixel's term under one root, without branches, so that the unrolled
// terms of a thread's pixels form one block the compiler can interleave.
// FAST: beta = 2 and alpha1 = 0 (closed form; obs.z unused).  A point behind
// the camera gives the constant term (its projection is computed from a
// denominator of 1 and discarded).
template <bool FAST>
__device__ __forceinline__ float vd_score_term(const DevParams& P, const float* Mr, float4 pt,
                                               float4 ob) {
  const float hx = fmaf(Mr[0], pt.x, fmaf(Mr[1], pt.y, fmaf(Mr[2], pt.z, Mr[9])));
  const float hy = fmaf(Mr[3], pt.x, fmaf(Mr[4], pt.y, fmaf(Mr[5], pt.z, Mr[10])));
  const float hz = fmaf(Mr[6], pt.x, fmaf(Mr[7], pt.y, fmaf(Mr[8], pt.z, Mr[11])));
  const bool front = hz > VD_Z_EPS;
  const float iz = __fdividef(1.0f, front ? hz : 1.0f);
  const float dx = ob.x - hx * iz, dy = ob.y - hy * iz;
  const float r2 = fmaf(dx, dx, dy * dy);
  const float l2 = FAST ? vd_l2_beta2(P, r2) : vd_l2_general(P, r2, ob.z);
  return front ? pt.w * VD_LN2 * l2 : pt.w * VD_L_BEHIND;
}

// Dynamic shared memory of k_pose_score<THREADS> for M roots.
static inline size_t vd_score_smem(int M, int threads) {
  return sizeof(float) * (size_t)M * (12 + threads / 32) + sizeof(int) * (size_t)(M + 1);
}

template <int THREADS, bool FAST = false>
__global__ void __launch_bounds__(THREADS)
k_pose_score(DevParams P, const float4* __restrict__ rpts, const float4* __restrict__ robs,
             const int* __restrict__ n_ptr, int n_host, const float* __restrict__ rootsf,
             const int* __restrict__ root_count, int M, float* __restrict__ partial) {
  extern __shared__ float smem[];
  constexpr int nwarp = THREADS / 32;
  float* sRoot = smem;                       // M * 12
  float* sAcc = smem + 12 * M;               // nwarp * M
  int* sList = (int*)(sAcc + nwarp * M);     // the real roots, in index order
  int* sNum = sList + M;
  for (int i = threadIdx.x; i < 12 * M; i += THREADS) sRoot[i] = rootsf[i];
  for (int i = threadIdx.x; i < nwarp * M; i += THREADS) sAcc[i] = 0.0f;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
    // compact the roots that exist (slot r & 3 below its sample's root count)
    int cnt = 0;
    for (int base = 0; base < M; base += 32) {
      const int r = base + lane;
      const bool ok = r < M && (!root_count || (r & 3) < root_count[r >> 2]);
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) sList[cnt + __popc(m & ((1u << lane) - 1u))] = r;
      cnt += __popc(m);
    }
    if (lane == 0) *sNum = cnt;
  }
  __syncthreads();
  const int nroot = *sNum;
  const int n = n_ptr ? *n_ptr : n_host;
  // contiguous ranges of whole warps, so that only the last warp is ragged
  const int per = (((n + gridDim.x - 1) / gridDim.x) + 31) & ~31;
  const int beg = min(n, blockIdx.x * per);
  const int end = min(n, beg + per);
  for (int base = beg; base < end; base += THREADS * SCORE_PPT) {
    // passes of this tile that hold at least one pixel (block-uniform)
    const int kact = min(SCORE_PPT, (end - base + THREADS - 1) / THREADS);
    float4 pt[SCORE_PPT], ob[SCORE_PPT];
#pragma unroll
    for (int k = 0; k < SCORE_PPT; ++k) {
      const int i = base + k * THREADS + threadIdx.x;
      if (i < end) {
        pt[k] = rpts[i];
        ob[k] = robs[i];
      } else {
        pt[k] = make_float4(0.f, 0.f, 1.f, 0.f);   // weight 0
        ob[k] = make_float4(0.f, 0.f, 1.f, 0.f);
      }
    }
    for (int m = 0; m < nroot; ++m) {
      const int r = sList[m];
      const float* Mr = sRoot + 12 * r;
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < SCORE_PPT; ++k)
        if (k < kact) acc += vd_score_term<FAST>(P, Mr, pt[k], ob[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sAcc[wid * M + r] += acc;
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nroot; m += THREADS) {
    const int r = sList[m];
    float s = 0.0f;
    for (int w = 0; w < nwarp; ++w) s += sAcc[w * M + r];
    partial[(size_t)r * gridDim.x + blockIdx.x] = s;
  }
}

// float64 sum of the block partials of every root that exists (infinity for
// the others): one warp per root, each lane sums a strided subset, then a
// fixed-order butterfly over the lanes.
__global__ void k_root_energy(const float* __restrict__ partial, int nblk, int M,
                              const int* __restrict__ root_count, double* __restrict__ energy) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= M) return;                 // whole warps leave together
  if (root_count && (r & 3) >= root_count[r >> 2]) {
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
                                             cudaStream_t s) {
  k_root_energy<<<(M + 3) / 4, 128, 0, s>>>(partial, nblk, M, root_count, energy);
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
// Per sample: the lowest-energy root; then mean-shift (Eq. 7) from the best
// sample: x <- x exp(sum w_g d_g / sum w_g), d_g = log(x^-1 T_g),
// w_g = exp(-d^T Sigma^-1 d / 2), at most 100 steps.  The float64 definition
// stops at |step| < 1e-12; these float32 iterations stop at the float32
// floor of the relative poses, 1e-6 (1 + |tau|).  One warp: the sums are
// warp butterflies, every lane updates the same mode, no block barrier.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32)
k_select_meanshift(DevParams P, const double* __restrict__ roots, const int* __restrict__ root_count,
                   const double* __restrict__ root_energy, int t, double* __restrict__ G,
                   float* __restrict__ posef, double* __restrict__ sample_pose,
                   double* __restrict__ sample_energy, int* __restrict__ degenerate) {
  // one warp; lane l owns samples l, l + 32, ...
  __shared__ float sT[VD_MAX_SAMPLES][12];
  __shared__ unsigned char sValid[VD_MAX_SAMPLES];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  double bestE = INFINITY;
  int bestS = 0x7fffffff;
  for (int g = lane; g < P.S; g += 32) {
    // the sample's lowest-energy root (ties: lower index in the sorted order)
    const int nr = root_count[g];
    int best = -1;
    double Eg = INFINITY;
    for (int r = 0; r < nr; ++r) {
      const double e = root_energy[4 * g + r];
      if (best < 0 || e < Eg) {
        Eg = e;
        best = r;
      }
    }
    const double* src = roots + (size_t)48 * g + 12 * (best < 0 ? 0 : best);
    for (int i = 0; i < 12; ++i) {
      const double v = best >= 0 ? src[i] : 0.0;
      sample_pose[12 * g + i] = v;
      sT[g][i] = (float)v;
    }
    if (best < 0) Eg = INFINITY;
    sample_energy[g] = Eg;
    sValid[g] = Eg < INFINITY;
    if (Eg < bestE) {           // g ascends per lane: ties keep the lower index
      bestE = Eg;
      bestS = g;
    }
  }
  // argmin over samples (lowest energy, then lowest index): a total order, so
  // every lane ends with the same pair
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double oE = __shfl_xor_sync(FULL, bestE, o);
    const int oS = __shfl_xor_sync(FULL, bestS, o);
    if (oE < bestE || (oE == bestE && oS < bestS)) {
      bestE = oE;
      bestS = oS;
    }
  }
  __syncwarp();
  if (!(bestE < INFINITY)) {
    if (lane == 0) atomicAdd(degenerate, 1);
    return;
  }
  float x[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) x[i] = sT[bestS][i];
  const float tn = sqrtf(x[3] * x[3] + x[7] * x[7] + x[11] * x[11]);
  const double st_ = P.ms_sig_rel * (double)tn + P.ms_sig_abs;
  const float ivr = (float)(1.0 / (P.ms_sig_rot * P.ms_sig_rot)), ivt = (float)(1.0 / (st_ * st_));
  // the float32 iterations stop at this step norm (the float32 floor of the
  // relative poses); the float64 definition stops at 1e-12
  const float tol = (float)(VD_MS_TOL_F32 * (1.0 + (double)tn));
  for (int it = 0; it < VD_MS_MAX_ITERS; ++it) {
    float acc[7] = {0, 0, 0, 0, 0, 0, 0};
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
      if (vd_se3_log_f(rel, d)) {
        const float m = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * ivr +
                        (d[3] * d[3] + d[4] * d[4] + d[5] * d[5]) * ivt;
        const float w = __expf(-0.5f * m);
        acc[0] += w;
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[1 + i] += w * d[i];
      }
    }
    // xor butterflies: float addition commutes, so partners hold equal sums
    // after every level and all lanes end with the same totals
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(FULL, acc[i], o);
    if (!(acc[0] > 0.0f)) break;
    float step[6], nrm = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      step[i] = acc[1 + i] / acc[0];
      nrm += step[i] * step[i];
    }
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
    if (sqrtf(nrm) < tol) break;
  }
  if (lane != 0) return;
  // re-orthonormalise the rotation in float64 (Gram-Schmidt on the rows,
  // third row as the cross product) and store the pose
  double R[9], o[12];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[3 * r + c] = (double)x[4 * r + c];
  double n0 = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  for (int c = 0; c < 3; ++c) R[c] /= n0;
  const double d01 = R[0] * R[3] + R[1] * R[4] + R[2] * R[5];
  for (int c = 0; c < 3; ++c) R[3 + c] -= d01 * R[c];
  const double n1 = sqrt(R[3] * R[3] + R[4] * R[4] + R[5] * R[5]);
  for (int c = 0; c < 3; ++c) R[3 + c] /= n1;
  R[6] = R[1] * R[5] - R[2] * R[4];
  R[7] = R[2] * R[3] - R[0] * R[5];
  R[8] = R[0] * R[4] - R[1] * R[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) o[4 * r + c] = R[3 * r + c];
    o[4 * r + 3] = (double)x[4 * r + 3];
  }
  for (int i = 0; i < 12; ++i) G[12 * t + i] = o[i];
  // float K R | K tau of the updated pose
  float* pf = posef + 12 * t;
  for (int i = 0; i < 4; ++i) {
    pf[i < 3 ? i : 9] = (float)(P.fx_d * o[i] + P.cx_d * o[8 + i]);
    pf[i < 3 ? 3 + i : 10] = (float)(P.fy_d * o[4 + i] + P.cy_d * o[8 + i]);
    pf[i < 3 ? 6 + i : 11] = (float)o[8 + i];
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
  const int nblk = c->score_bps * c->num_sms;
#define VD_SCORE_LAUNCH(TH, FAST)                                                     \
  k_pose_score<TH, FAST><<<nblk, TH, vd_score_smem(M, TH), c->stream>>>(                   \
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
  return launch_root_energy(c->partial, nblk, M, c->root_count, c->root_energy, c->stream);
}

cudaError_t launch_pose_frame(vd_ctx* c, uint32_t itcode, int t) {
  const DevParams& P = c->dp;
  c->last_pose_t = t;
  c->samples_set |= 1u << (t - 1);
  const size_t f = (size_t)(t - 1) * VD_MAX_SAMPLES;   // this frame's sample slots
  vd_prof_begin(c, VD_ST_RIGID);
  k_rigid_flags<<<c->nblk_scan, SCAN_BLOCK, 0, c->stream>>>(P, c->G, c->posef, c->rho, c->q, t,
                                                            c->flags, c->blk_counts);
  k_scan_counts<<<1, 1024, 0, c->stream>>>(c->blk_counts, c->nblk_scan, c->blk_offsets, c->n_rigid);
  k_rigid_scatter<<<c->nblk_scan, SCAN_BLOCK, 0, c->stream>>>(P, c->posef, c->flow, c->rho, c->q, t,
                                                              c->flags, c->blk_offsets,
                                                              c->rigid_idx, c->rpts, c->robs);
  vd_prof_end(c, VD_ST_RIGID, 3);
  vd_prof_begin(c, VD_ST_P3P);
  k_p3p_samples<<<P.S, 32, 0, c->stream>>>(P, c->G, c->flow, c->rho, c->rigid_idx,
                                                       c->n_rigid, t, itcode, c->roots,
                                                       c->root_count);
  const int M = 4 * P.S;
  k_roots_float<<<(M + 127) / 128, 128, 0, c->stream>>>(P, c->roots, c->root_count, c->rootsf);
  vd_prof_end(c, VD_ST_P3P, 2);
  vd_prof_begin(c, VD_ST_SCORE);
  launch_pose_score_only(c);
  vd_prof_end(c, VD_ST_SCORE, 2);
  vd_prof_begin(c, VD_ST_SELECT);
  k_select_meanshift<<<1, 32, 0, c->stream>>>(P, c->roots, c->root_count, c->root_energy, t, c->G,
                                               c->posef, c->sample_pose + 12 * f,
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
  k_pose_score<SCORE_THREADS><<<nblk, SCORE_THREADS, smem, s>>>(
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
  k_pose_score<SCORE_THREADS><<<nblk, SCORE_THREADS, smem, s>>>(P, (const float4*)points, (const float4*)obs,
                                                 nullptr, n, rootsf, nullptr, m, partial);
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
