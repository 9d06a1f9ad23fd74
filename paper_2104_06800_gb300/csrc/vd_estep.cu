// Rigidness E-step of VOLDOR+ (Sec. III-A): two-state hidden Markov chains
// along the rows or columns of every flow's rigidness map, smoothed by the
// forward-backward algorithm, and the depth confidence map of Eq. 6.
#include "vd_device.cuh"
#include "vd_emission_df.cuh"

#define VD_DISPATCH_NF(N, KERNEL_CALL)      \
  switch (N) {                              \
    case 1: { constexpr int NF = 1; KERNEL_CALL; } break; \
    case 2: { constexpr int NF = 2; KERNEL_CALL; } break; \
    case 3: { constexpr int NF = 3; KERNEL_CALL; } break; \
    case 4: { constexpr int NF = 4; KERNEL_CALL; } break; \
    case 5: { constexpr int NF = 5; KERNEL_CALL; } break; \
    case 6: { constexpr int NF = 6; KERNEL_CALL; } break; \
    case 7: { constexpr int NF = 7; KERNEL_CALL; } break; \
    case 8: { constexpr int NF = 8; KERNEL_CALL; } break; \
    default: return cudaErrorInvalidValue;  \
  }

// Bilinear sample at an inside double-float position, the taps of
// `vd_bilinear` (x0 = min(floor(x), W-2)).
__device__ __forceinline__ float2 em_bilinear_df(const float2* __restrict__ F, int W, int H,
                                                 vd_df x, vd_df y) {
  float ax, ay;
  const int x0 = vd_em_tap(x, W, &ax), y0 = vd_em_tap(y, H, &ay);
  const float2* p = F + VD_CHK(VD_SITE_BILINEAR, (long long)y0 * W + x0, (long long)W * H - W - 1);
  const float2 f00 = __ldg(p), f01 = __ldg(p + 1);
  const float2 f10 = __ldg(p + W), f11 = __ldg(p + W + 1);
  const float tx = fmaf(ax, f01.x - f00.x, f00.x), ty = fmaf(ax, f01.y - f00.y, f00.y);
  const float bx = fmaf(ax, f11.x - f10.x, f10.x), by = fmaf(ax, f11.y - f10.y, f10.y);
  return make_float2(fmaf(ay, bx - tx, tx), fmaf(ay, by - ty, ty));
}

// ---------------------------------------------------------------------------
// Emission ratio lam = e_rigid / e_outlier of every pixel and flow at the new
// depth: 1 / y for an observed term (y = P0 / p1), 0 when the point is behind
// camera t, 1 without observation.  Also the prior's isolated posterior q_hat.
// Positions, the camera-plane test and the image-border test in
// double-float (vd_emission_df.cuh); the flow sample and the Fisk ratio in
// float32.
// ---------------------------------------------------------------------------
template <int NF>
__global__ void __launch_bounds__(128)
k_emission(DevParams P, const float2* __restrict__ posed, const float2* __restrict__ flow,
           const float* __restrict__ rho, const float* __restrict__ prior_val,
           float* __restrict__ lam, float* __restrict__ qhat) {
  __shared__ float2 sPose[12 * (VD_MAX_FLOWS + 1)];
  for (int i = threadIdx.x + threadIdx.y * blockDim.x; i < 12 * (NF + 1); i += blockDim.x * blockDim.y)
    sPose[i] = posed[i];
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= P.W || v >= P.H) return;
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)v * P.W + u;
  const float c = rho[j];
  vd_df rx, ry;
  vd_em_ray(P.kdf, u, v, &rx, &ry);
  vd_df xp = vd_df_make((float)u), yp = vd_df_make((float)v);
  bool front_prev = true;
#pragma unroll
  for (int t = 0; t < NF; ++t) {
    vd_df x = xp, y = yp;
    const bool front = vd_em_project(sPose + 12 * (t + 1), rx, ry, c, &x, &y);
    bool obs;
    float2 F;
    if (t == 0) {
      obs = true;
      F = __ldg(flow + j);
    } else {
      obs = front_prev && vd_em_inside(xp, yp, P.W, P.H);
      F = make_float2(0.0f, 0.0f);
      if (obs) F = em_bilinear_df(flow + (size_t)t * npix, P.W, P.H, xp, yp);
    }
    float l;
    if (obs && front) {
      const float dx = F.x - vd_em_diff(x, xp);
      const float dy = F.y - vd_em_diff(y, yp);
      const float yv = vd_ratio_y(P, fmaf(dx, dx, dy * dy), fmaf(F.x, F.x, F.y * F.y));
      l = yv < 1e30f ? __frcp_rn(yv) : 0.0f;   // an overflowing (or 0 * inf) ratio: p1 / P0 = 0
    } else {
      l = obs ? 0.0f : 1.0f;
    }
    lam[(size_t)t * npix + j] = l;
    xp = x;
    yp = y;
    front_prev = front;
  }
  if (P.prior_kind != VD_PRIOR_NONE) {
    const float pv = prior_val[j];
    float qh = 0.0f;
    if (isfinite(pv)) {
      if (P.prior_kind == VD_PRIOR_STEREO) {
        const float d = pv - P.fxb * c;
        float yv;
        if (P.beta == 2.0f) {
          const float s = fmaf(d * d, P.inv_a2, 1.0f);
          yv = P.c0 * s * s;
        } else {
          yv = vd_ratio_general(P, d * d, P.alpha0);
        }
        qh = yv < 1e30f ? 1.0f / (1.0f + yv) : 0.0f;
      } else {
        const float res = pv - c;
        const float sig = P.c_sigma * pv;
        const float z = fmaf(res * res, 0.5f / (sig * sig), P.logk);
        qh = z > 80.0f ? 0.0f : 1.0f / (1.0f + __expf(z));
      }
    }
    qhat[j] = qh;
  }
}

// ---------------------------------------------------------------------------
// Forward-backward as an associative scan, one warp per chain.  With
// M_m = A diag(1, lam_m) (A[s'][s] = gamma if s = s' else 1 - gamma) the
// forward messages are alpha_m = (1, lam_0) M_1 ... M_m and the backward
// ones beta_m = M_{m+1} ... M_{L-1} (1, 1)^T.  Lane i owns the contiguous
// segment [a_i, b_i) of the chain: it forms the product S_i of its segment's
// matrices, a warp scan of the S_i (normalised 2x2 products) gives the
// message entering and leaving every segment, and each lane walks its
// segment forward (parking alpha in q) and backward (combining).
// ---------------------------------------------------------------------------
struct VdM2 {
  float a, b, c, d;   // [[a, b], [c, d]]
};

__device__ __forceinline__ VdM2 vd_m2_mul(const VdM2& x, const VdM2& y) {
  VdM2 r;
  r.a = fmaf(x.a, y.a, x.b * y.c);
  r.b = fmaf(x.a, y.b, x.b * y.d);
  r.c = fmaf(x.c, y.a, x.d * y.c);
  r.d = fmaf(x.c, y.b, x.d * y.d);
  const float s = 1.0f / (r.a + r.b + r.c + r.d);   // first column is positive: s finite
  r.a *= s;
  r.b *= s;
  r.c *= s;
  r.d *= s;
  return r;
}

__device__ __forceinline__ VdM2 vd_m2_shfl_up(const VdM2& x, int off) {
  VdM2 r;
  r.a = __shfl_up_sync(0xffffffffu, x.a, off);
  r.b = __shfl_up_sync(0xffffffffu, x.b, off);
  r.c = __shfl_up_sync(0xffffffffu, x.c, off);
  r.d = __shfl_up_sync(0xffffffffu, x.d, off);
  return r;
}

__device__ __forceinline__ VdM2 vd_m2_shfl_down(const VdM2& x, int off) {
  VdM2 r;
  r.a = __shfl_down_sync(0xffffffffu, x.a, off);
  r.b = __shfl_down_sync(0xffffffffu, x.b, off);
  r.c = __shfl_down_sync(0xffffffffu, x.c, off);
  r.d = __shfl_down_sync(0xffffffffu, x.d, off);
  return r;
}

__global__ void __launch_bounds__(128)
k_forward_backward_warp(DevParams P, const float* __restrict__ lam, float* __restrict__ q,
                        int direction) {
  const bool rows = (direction & 1) == 0;
  const int nchains = rows ? P.H : P.W;
  const int L = rows ? P.W : P.H;
  const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (wid >= nchains * P.N) return;               // whole warps leave together
  const int t = wid / nchains;
  const int ch = wid - t * nchains;
  const size_t npix = (size_t)P.W * P.H;
  const float* lt = lam + (size_t)t * npix;
  float* qt = q + (size_t)t * npix;
  const size_t base = rows ? (size_t)ch * P.W : (size_t)ch;
  const size_t step = rows ? 1 : (size_t)P.W;
  const float g = P.gamma, h = 1.0f - P.gamma;
  const int seg = (L + 31) >> 5;
  const int a0 = min(L, lane * seg), b0 = min(L, a0 + seg);
  const int first = max(a0, 1);                   // position 0 carries no matrix
  // segment product
  VdM2 S = {1.0f, 0.0f, 0.0f, 1.0f};
  for (int m = first; m < b0; ++m) {
    const float l = lt[base + step * m];
    const VdM2 M = {g, h * l, h, g * l};
    S = vd_m2_mul(S, M);
  }
  // inclusive prefix (left to right) and suffix (right to left) products
  VdM2 X = S, Z = S;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const VdM2 Y = vd_m2_shfl_up(X, off);
    if (lane >= off) X = vd_m2_mul(Y, X);
    const VdM2 Yd = vd_m2_shfl_down(Z, off);
    if (lane + off < 32) Z = vd_m2_mul(Z, Yd);
  }
  VdM2 Pin = vd_m2_shfl_up(X, 1);                 // product of the earlier segments
  VdM2 Qout = vd_m2_shfl_down(Z, 1);              // product of the later segments
  if (lane == 0) Pin = {1.0f, 0.0f, 0.0f, 1.0f};
  if (lane == 31) Qout = {1.0f, 0.0f, 0.0f, 1.0f};
  if (a0 >= b0) return;
  // forward walk: alpha entering the segment = (1, lam_0) Pin
  const float l0 = lt[base];
  float f0 = fmaf(1.0f, Pin.a, l0 * Pin.c), f1 = fmaf(1.0f, Pin.b, l0 * Pin.d);
  if (a0 == 0) {
    const float s = 1.0f / (f0 + f1);
    f0 *= s;
    f1 *= s;
    qt[base] = f1;
  }
  for (int m = first; m < b0; ++m) {
    const float l = lt[base + step * m];
    const float n0 = fmaf(f0, g, f1 * h);           // (alpha A)_0 * e0
    const float n1 = fmaf(f0, h, f1 * g) * l;       // (alpha A)_1 * e1
    const float s = 1.0f / (n0 + n1);
    f0 = n0 * s;
    f1 = n1 * s;
    qt[base + step * m] = f1;
  }
  // backward walk: beta leaving the segment = Qout (1, 1)^T
  float b0v = Qout.a + Qout.b, b1v = Qout.c + Qout.d;
  {
    const float s = 1.0f / (b0v + b1v);
    b0v *= s;
    b1v *= s;
  }
  for (int m = b0 - 1; m >= a0; --m) {
    if (m < b0 - 1) {
      const float l = lt[base + step * (m + 1)];
      const float y1 = b1v * l;
      const float n0 = fmaf(g, b0v, h * y1);
      const float n1 = fmaf(h, b0v, g * y1);
      const float s = 1.0f / (n0 + n1);
      b0v = n0 * s;
      b1v = n1 * s;
    }
    const float am = qt[base + step * m];
    const float num = am * b1v;
    qt[base + step * m] = num / (num + (1.0f - am) * b0v);
  }
}

// The same forward-backward with the chains staged in shared memory: a
// block takes blockDim.x / 32 adjacent chains of one flow (one warp each),
// loads their ratios with coalesced reads (consecutive threads read
// consecutive pixels of a row chain, or adjacent column chains at one row),
// runs the segment scan and both walks on shared memory, and writes the
// posteriors back the same way.  Lane k's segment sits at k * segp in its
// chain's slot array (segp = seg rounded up to odd: the 32 lanes' walks hit
// distinct banks; chains one float apart likewise).  The arithmetic is that
// of k_forward_backward_warp, in the same order.
__global__ void __launch_bounds__(256)
k_forward_backward_staged(DevParams P, const float* __restrict__ lam, float* __restrict__ q,
                          int direction) {
  extern __shared__ float fb_sm[];
  const bool rows = (direction & 1) == 0;
  const int nchains = rows ? P.H : P.W;
  const int L = rows ? P.W : P.H;
  const int CB = blockDim.x >> 5;
  const int t = blockIdx.y;
  const int ch0 = blockIdx.x * CB;
  const int seg = (L + 31) >> 5, segp = seg | 1;
  const int CS = 32 * segp + 1;                   // one chain's slots
  float* sl = fb_sm;                              // [CB][CS] ratios
  float* sq = fb_sm + CB * CS;                    // [CB][CS] posteriors
  const size_t npix = (size_t)P.W * P.H;
  const float* lt = lam + (size_t)t * npix;
  float* qt = q + (size_t)t * npix;
  const int total = CB * L;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = rows ? idx / L : idx % CB, m = rows ? idx - c * L : idx / CB;
    const int ch = ch0 + c;
    if (ch < nchains)
      sl[c * CS + (m / seg) * segp + m % seg] =
          lt[rows ? (size_t)ch * P.W + m : (size_t)m * P.W + ch];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (ch0 + w < nchains) {
    const float* l_ = sl + w * CS;
    float* q_ = sq + w * CS;
    const float g = P.gamma, h = 1.0f - P.gamma;
    const int a0 = min(L, lane * seg), b0 = min(L, a0 + seg);
    const int first = max(a0, 1);                 // position 0 carries no matrix
    const int o = lane * segp - a0;               // slot of position m: o + m
    VdM2 S = {1.0f, 0.0f, 0.0f, 1.0f};
    for (int m = first; m < b0; ++m) {
      const float l = l_[o + m];
      const VdM2 M = {g, h * l, h, g * l};
      S = vd_m2_mul(S, M);
    }
    VdM2 X = S, Z = S;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const VdM2 Y = vd_m2_shfl_up(X, off);
      if (lane >= off) X = vd_m2_mul(Y, X);
      const VdM2 Yd = vd_m2_shfl_down(Z, off);
      if (lane + off < 32) Z = vd_m2_mul(Z, Yd);
    }
    VdM2 Pin = vd_m2_shfl_up(X, 1);
    VdM2 Qout = vd_m2_shfl_down(Z, 1);
    if (lane == 0) Pin = {1.0f, 0.0f, 0.0f, 1.0f};
    if (lane == 31) Qout = {1.0f, 0.0f, 0.0f, 1.0f};
    if (a0 < b0) {
      const float l0 = l_[0];
      float f0 = fmaf(1.0f, Pin.a, l0 * Pin.c), f1 = fmaf(1.0f, Pin.b, l0 * Pin.d);
      if (a0 == 0) {
        const float s = 1.0f / (f0 + f1);
        f0 *= s;
        f1 *= s;
        q_[0] = f1;
      }
      for (int m = first; m < b0; ++m) {
        const float l = l_[o + m];
        const float n0 = fmaf(f0, g, f1 * h);
        const float n1 = fmaf(f0, h, f1 * g) * l;
        const float s = 1.0f / (n0 + n1);
        f0 = n0 * s;
        f1 = n1 * s;
        q_[o + m] = f1;
      }
      float b0v = Qout.a + Qout.b, b1v = Qout.c + Qout.d;
      {
        const float s = 1.0f / (b0v + b1v);
        b0v *= s;
        b1v *= s;
      }
      for (int m = b0 - 1; m >= a0; --m) {
        if (m < b0 - 1) {
          const float l = l_[o + m + 1];
          const float y1 = b1v * l;
          const float n0 = fmaf(g, b0v, h * y1);
          const float n1 = fmaf(h, b0v, g * y1);
          const float s = 1.0f / (n0 + n1);
          b0v = n0 * s;
          b1v = n1 * s;
        }
        const float am = q_[o + m];
        const float num = am * b1v;
        q_[o + m] = num / (num + (1.0f - am) * b0v);
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = rows ? idx / L : idx % CB, m = rows ? idx - c * L : idx / CB;
    const int ch = ch0 + c;
    if (ch < nchains)
      qt[rows ? (size_t)ch * P.W + m : (size_t)m * P.W + ch] =
          sq[c * CS + (m / seg) * segp + m % seg];
  }
}

// Eq. 6: C = (sum_t q_t + q_hat) / (N + 1) with a prior, sum_t q_t / N without.
__global__ void k_confidence(DevParams P, const float* __restrict__ q,
                             const float* __restrict__ qhat, float* __restrict__ conf) {
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npix) return;
  // float32 sum in flow order (at most 9 terms in [0, 1]: error below 1e-6;
  // a float64 sum costs this part's float64 pipe more than the rest)
  float s = 0.0f;
  for (int t = 0; t < P.N; ++t) s += q[(size_t)t * npix + j];
  if (P.prior_kind != VD_PRIOR_NONE) {
    s += qhat[j];
    conf[j] = s / (float)(P.N + 1);
  } else {
    conf[j] = s / (float)P.N;
  }
}

cudaError_t launch_estep(vd_ctx* c, int direction) {
  const dim3 blk(32, 4);
  const dim3 grd((c->W + 31) / 32, (c->H + 3) / 4);
  VD_DISPATCH_NF(c->N, (k_emission<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posed, c->flow, c->rho, c->prior_val, c->lam, c->qhat)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool rows = (direction & 1) == 0;
  const int nch = rows ? c->H : c->W, L = rows ? c->W : c->H;
  // chains per block of the staged kernel: 4 rows or 8 columns, fewer where
  // their slots would pass 48 KB; chains too long for one: the unstaged one
  const int seg = (L + 31) >> 5, segp = seg | 1;
  const size_t per_chain = 2 * sizeof(float) * (size_t)(32 * segp + 1);
  int cb = rows ? 4 : 8;
  while (cb > 1 && cb * per_chain > 48 * 1024) cb >>= 1;
  if (cb * per_chain <= 48 * 1024) {
    k_forward_backward_staged<<<dim3((nch + cb - 1) / cb, c->N), 32 * cb, cb * per_chain,
                                c->stream>>>(c->dp, c->lam, c->q, direction);
  } else {
    const int nwarps = nch * c->N;
    k_forward_backward_warp<<<(nwarps + 3) / 4, 128, 0, c->stream>>>(c->dp, c->lam, c->q,
                                                                      direction);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_confidence<<<(unsigned)((c->npix + 255) / 256), 256, 0, c->stream>>>(c->dp, c->q, c->qhat,
                                                                         c->conf);
  return cudaGetLastError();
}

VD_CHECK_ACCESSOR(estep)
