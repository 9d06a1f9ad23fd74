// Rigidness E-step of VOLDOR+ (Sec. III-A): two-state hidden Markov chains
// along the rows or columns of every flow's rigidness map, smoothed by the
// forward-backward algorithm, and the depth confidence map of Eq. 6.
#include "vd_device.cuh"

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

// ---------------------------------------------------------------------------
// Emission ratio lam = e_rigid / e_outlier of every pixel and flow at the new
// depth: 1 / y for an observed term (y = P0 / p1), 0 when the point is behind
// camera t, 1 without observation.  Also the prior's isolated posterior q_hat.
// ---------------------------------------------------------------------------
template <int NF>
__global__ void __launch_bounds__(128)
k_emission(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
           const float* __restrict__ rho, const float* __restrict__ prior_val,
           float* __restrict__ lam, float* __restrict__ qhat) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  for (int i = threadIdx.x + threadIdx.y * blockDim.x; i < 12 * (NF + 1); i += blockDim.x * blockDim.y)
    sPose[i] = posef[i];
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= P.W || v >= P.H) return;
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)v * P.W + u;
  const float c = rho[j];
  const float rx = ((float)u - P.cx) / P.fx;
  const float ry = ((float)v - P.cy) / P.fy;
  float xp = (float)u, yp = (float)v;
  bool front_prev = true;
#pragma unroll
  for (int t = 0; t < NF; ++t) {
    const float* M = sPose + 12 * (t + 1);
    const float hx = fmaf(c, M[9], fmaf(M[0], rx, fmaf(M[1], ry, M[2])));
    const float hy = fmaf(c, M[10], fmaf(M[3], rx, fmaf(M[4], ry, M[5])));
    const float hz = fmaf(c, M[11], fmaf(M[6], rx, fmaf(M[7], ry, M[8])));
    const bool front = hz > VD_Z_EPS;
    const float iz = __fdividef(1.0f, hz);
    const float x = hx * iz, y = hy * iz;
    bool obs;
    float2 F;
    if (t == 0) {
      obs = true;
      F = __ldg(flow + j);
    } else {
      obs = front_prev && vd_inside(xp, yp, P.W, P.H);
      F = make_float2(0.0f, 0.0f);
      if (obs) F = vd_bilinear(flow + (size_t)t * npix, P.W, P.H, xp, yp);
    }
    float l;
    if (obs && front) {
      const float dx = F.x - (x - xp);
      const float dy = F.y - (y - yp);
      l = __frcp_rn(vd_ratio_y(P, fmaf(dx, dx, dy * dy), fmaf(F.x, F.x, F.y * F.y)));
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
        qh = 1.0f / (1.0f + yv);
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
// Forward-backward on one chain per thread (flow t, row or column).  With
// a = P(rigid | left part), b = P(rigid | right part) normalised:
//   a_m ~ (a_{m-1} g + (1 - a_{m-1}) h) lam_m  vs  a_{m-1} h + (1 - a_{m-1}) g
//   b_m ~ g lam_{m+1} b_{m+1} + h (1 - b_{m+1})  vs  h lam_{m+1} b_{m+1} + g (1 - b_{m+1})
//   q_m = a_m b_m / (a_m b_m + (1 - a_m)(1 - b_m)),  g = gamma, h = 1 - gamma.
// The forward pass parks a_m in q; the backward pass combines.
// ---------------------------------------------------------------------------
__global__ void k_forward_backward(DevParams P, const float* __restrict__ lam,
                                   float* __restrict__ q, int direction) {
  const bool rows = (direction & 1) == 0;
  const int nchains = rows ? P.H : P.W;
  const int L = rows ? P.W : P.H;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nchains * P.N) return;
  const int t = gid / nchains;
  const int ch = gid - t * nchains;
  const size_t npix = (size_t)P.W * P.H;
  const float* lt = lam + (size_t)t * npix;
  float* qt = q + (size_t)t * npix;
  const size_t base = rows ? (size_t)ch * P.W : (size_t)ch;
  const size_t step = rows ? 1 : (size_t)P.W;
  const float g = P.gamma, h = 1.0f - P.gamma;
  float a = 0.5f;
  for (int m = 0; m < L; ++m) {
    const size_t j = base + step * m;
    const float l = lt[j];
    float x1, x0;
    if (m == 0) {
      x1 = l;
      x0 = 1.0f;
    } else {
      x1 = fmaf(a, g - h, h) * l;      // (a g + (1 - a) h) lam
      x0 = fmaf(a, h - g, g);          // a h + (1 - a) g
    }
    a = x1 / (x0 + x1);
    qt[j] = a;
  }
  float b = 0.5f;
  for (int m = L - 1; m >= 0; --m) {
    const size_t j = base + step * m;
    const float am = qt[j];
    if (m < L - 1) {
      const float ln = lt[j + step];
      const float y1 = fmaf(g * ln, b, h * (1.0f - b));
      const float y0 = fmaf(h * ln, b, g * (1.0f - b));
      b = y1 / (y0 + y1);
    }
    const float num = am * b;
    qt[j] = num / (num + (1.0f - am) * (1.0f - b));
  }
}

// Eq. 6: C = (sum_t q_t + q_hat) / (N + 1) with a prior, sum_t q_t / N without.
__global__ void k_confidence(DevParams P, const float* __restrict__ q,
                             const float* __restrict__ qhat, float* __restrict__ conf) {
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npix) return;
  double s = 0.0;
  for (int t = 0; t < P.N; ++t) s += (double)q[(size_t)t * npix + j];
  if (P.prior_kind != VD_PRIOR_NONE) {
    s += (double)qhat[j];
    conf[j] = (float)(s / (P.N + 1));
  } else {
    conf[j] = (float)(s / P.N);
  }
}

cudaError_t launch_estep(vd_ctx* c, int direction) {
  const dim3 blk(32, 4);
  const dim3 grd((c->W + 31) / 32, (c->H + 3) / 4);
  VD_DISPATCH_NF(c->N, (k_emission<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->rho, c->prior_val, c->lam, c->qhat)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool rows = (direction & 1) == 0;
  const int nthreads = (rows ? c->H : c->W) * c->N;
  k_forward_backward<<<(nthreads + 63) / 64, 64, 0, c->stream>>>(c->dp, c->lam, c->q, direction);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_confidence<<<(unsigned)((c->npix + 255) / 256), 256, 0, c->stream>>>(c->dp, c->q, c->qhat,
                                                                         c->conf);
  return cudaGetLastError();
}
