// Depth M-step of VOLDOR+ (Sec. III-A, Eq. 5): per-pixel hypothesis sampling
// and argmin (parallel phase) followed by propagation along alternately
// directed 1-D chains (sequential phase), plus the hierarchical option
// (coarse global pass + local full-resolution windows).
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
// float K R | K tau of every frame from the float64 absolute poses.
// ---------------------------------------------------------------------------
__global__ void k_posef(DevParams P, const double* __restrict__ G, float* __restrict__ posef) {
  const int t = threadIdx.x;
  if (t > P.N) return;
  const double* g = G + 12 * t;
  float* o = posef + 12 * t;
  for (int r = 0; r < 3; ++r) {
    const double k0 = r == 0 ? P.fx_d : (r == 1 ? 0.0 : 0.0);
    const double k1 = r == 1 ? P.fy_d : 0.0;
    const double k2 = r == 0 ? P.cx_d : (r == 1 ? P.cy_d : 1.0);
    // row r of K [R | tau] = k0 * row0 + k1 * row1 + k2 * row2
    for (int c = 0; c < 3; ++c)
      o[3 * r + c] = (float)(k0 * g[c] + k1 * g[4 + c] + k2 * g[8 + c]);
    o[9 + r] = (float)(k0 * g[3] + k1 * g[7] + k2 * g[11]);
  }
}

cudaError_t launch_posef(vd_ctx* c) {
  k_posef<<<1, 32, 0, c->stream>>>(c->dp, c->G, c->posef);
  return cudaGetLastError();
}

template <int NF>
__device__ __forceinline__ void vd_load_pose_smem(float* sPose, const float* __restrict__ posef) {
  const int nt = blockDim.x * blockDim.y;
  for (int i = threadIdx.x + threadIdx.y * blockDim.x; i < 12 * (NF + 1); i += nt) sPose[i] = posef[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// K1: K candidates per pixel, argmin of E (ties: lowest slot).
// Slot 0 = current value; slot 1 = prior where valid; slot k >= 1 otherwise
// draws Philox word k-1 of counter (j - u mod share, iter, TAG_DEPTH, (k-1)/4):
// slots 1..(K-1)/2 uniform in [rho_min, rho_max], the rest rho (1 + s (2u-1)).
// ---------------------------------------------------------------------------
// Launch shape of the sampling kernel (threads per block and the minimum
// number of resident blocks requested from the register allocator).
#ifndef VD_K1_BX
#define VD_K1_BX 32
#endif
#ifndef VD_K1_BY
#define VD_K1_BY 4
#endif
#ifndef VD_K1_MINB
#define VD_K1_MINB 6
#endif

template <int NF>
__global__ void __launch_bounds__(VD_K1_BX * VD_K1_BY, VD_K1_MINB)
k_depth_sample(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
               const float* __restrict__ rho, const float* __restrict__ q,
               const float* __restrict__ prior_val, const float* __restrict__ prior_rho,
               const float* __restrict__ qhat, const float* __restrict__ pconf, uint32_t itcode,
               float s_pert, float* __restrict__ rho_star, float* __restrict__ e_star) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  vd_load_pose_smem<NF>(sPose, posef);
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= P.W || v >= P.H) return;
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)v * P.W + u;
  VdPixel<NF> px;
  vd_pixel_setup<NF>(px, P, sPose, u, v, q, npix, j, flow, prior_val, qhat, pconf);

  const float rmin = P.rho_min, rmax = P.rho_max;
  const float range = __fsub_rn(rmax, rmin);
  const float cur = rho[j];
  float best = vd_clamp(cur, rmin, rmax);
  float bestE = vd_energy<NF>(px, P, sPose, flow, npix, best);
  const uint32_t ctr0 = (uint32_t)(j - (size_t)(u % P.share));
  const int n_unif = (P.K - 1) / 2;
  bool has_prior = false;
  float prior_c = 0.0f;
  if (P.prior_kind != VD_PRIOR_NONE) {
    const float pr = prior_rho[j];
    has_prior = isfinite(pr);
    prior_c = vd_clamp(pr, rmin, rmax);
  }
  uint4 w = make_uint4(0, 0, 0, 0);
  for (int k = 1; k < P.K; ++k) {
    const int wi = k - 1;
    if ((wi & 3) == 0)
      w = vd_philox(make_uint4(ctr0, itcode, VD_TAG_DEPTH, (uint32_t)(wi >> 2)), P.key0, P.key1);
    const uint32_t x = vd_word(w, wi & 3);
    float c = (k <= n_unif) ? vd_cand_uniform(x, rmin, range) : vd_cand_perturb(x, cur, s_pert);
    c = vd_clamp(c, rmin, rmax);
    if (k == 1 && has_prior) c = prior_c;
    const float E = vd_energy<NF>(px, P, sPose, flow, npix, c, bestE);
    if (E < bestE) {
      bestE = E;
      best = c;
    }
  }
  rho_star[j] = best;
  e_star[j] = bestE;
}

// ---------------------------------------------------------------------------
// K2: propagation along the chains.  Walking a chain in its direction,
// rho_new = rho* unless the predecessor's new value has strictly lower
// energy; `restart` > 0 starts afresh every `restart` pixels (local windows
// of the hierarchical scheme).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// K2, warp version: one warp per chain, lane i owns the contiguous segment
// [i*seg, (i+1)*seg) of the chain.  Phase A: every lane walks its segment as
// if its first pixel started the chain.  Correction rounds: a lane whose
// incoming value (the predecessor lane's end value) changed walks again from
// its segment start with that value and stops as soon as the carried value
// equals what it wrote at that pixel before (the rest of the walk depends on
// the carried value only, so it is unchanged).  The rounds end when no end
// value changes, so the result is exactly the sequential walk.
// ---------------------------------------------------------------------------
template <int NF>
__device__ __forceinline__ float vd_prop_step(const DevParams& P, const float* sPose,
                                              const float2* __restrict__ flow,
                                              const float* __restrict__ q,
                                              const float* __restrict__ prior_val,
                                              const float* __restrict__ qhat,
                                              const float* __restrict__ pconf, float cur, float own,
                                              float e_own, int u, int v, size_t j) {
  const size_t npix = (size_t)P.W * P.H;
  VdPixel<NF> px;
  vd_pixel_setup<NF>(px, P, sPose, u, v, q, npix, j, flow, prior_val, qhat, pconf);
  const float Ec = vd_energy<NF>(px, P, sPose, flow, npix, cur, e_own);
  return (Ec < e_own) ? cur : own;
}

template <int NF>
__global__ void __launch_bounds__(128)
k_propagate_warp(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
                 const float* __restrict__ q, const float* __restrict__ prior_val,
                 const float* __restrict__ qhat, const float* __restrict__ pconf,
                 const float* __restrict__ rho_star, const float* __restrict__ e_star,
                 float* __restrict__ rho_new, int direction, int restart) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  vd_load_pose_smem<NF>(sPose, posef);
  const bool rows = (direction & 1) == 0;
  const bool rev = direction >= 2;
  const int nchains = rows ? P.H : P.W;
  const int L = rows ? P.W : P.H;
  const int ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (ch >= nchains) return;          // whole warps leave together
  const int seg = (L + 31) >> 5;
  const int m0 = min(L, lane * seg), m1 = min(L, m0 + seg);
  auto pix = [&](int m, int* u, int* v) -> size_t {
    const int pos = rev ? L - 1 - m : m;
    *u = rows ? pos : ch;
    *v = rows ? ch : pos;
    return (size_t)(*v) * P.W + (*u);
  };
  // phase A
  float cur = 0.0f;
  for (int m = m0; m < m1; ++m) {
    int u, v;
    const size_t j = pix(m, &u, &v);
    const float own = rho_star[j];
    if (m == m0 || (restart > 0 && m % restart == 0)) {
      cur = own;
    } else {
      cur = vd_prop_step<NF>(P, sPose, flow, q, prior_val, qhat, pconf, cur, own, e_star[j], u, v, j);
    }
    rho_new[j] = cur;
  }
  float end = cur;                     // value carried out of the segment
  bool have_in = false;                // phase A assumed no incoming value
  float last_in = 0.0f;
  for (int round = 0; round < 32; ++round) {
    float in = __shfl_up_sync(0xffffffffu, end, 1);
    const bool has_pred = lane > 0 && m1 > m0 && m0 > 0;
    bool walk = has_pred && (!have_in || in != last_in);
    if (walk && restart > 0 && m0 % restart == 0) walk = false;   // forced fresh start
    bool changed = false;
    if (walk) {
      have_in = true;
      last_in = in;
      float c = in;
      bool merged = false;
      for (int m = m0; m < m1; ++m) {
        int u, v;
        const size_t j = pix(m, &u, &v);
        const float own = rho_star[j];
        float nc;
        if (restart > 0 && m % restart == 0)
          nc = own;
        else
          nc = vd_prop_step<NF>(P, sPose, flow, q, prior_val, qhat, pconf, c, own, e_star[j], u, v, j);
        if (nc == rho_new[j]) {
          merged = true;
          break;
        }
        rho_new[j] = nc;
        c = nc;
      }
      if (!merged && c != end) {
        end = c;
        changed = true;
      }
    }
    if (!__any_sync(0xffffffffu, changed)) break;
  }
}

// Hierarchical scheme, global pass: chains over the coarse grid of
// representative pixels (min(s uc, W-1), min(s vc, H-1)).
template <int NF>
__global__ void k_hier_coarse(DevParams P, const float* __restrict__ posef,
                              const float2* __restrict__ flow, const float* __restrict__ q,
                              const float* __restrict__ prior_val, const float* __restrict__ qhat,
                              const float* __restrict__ pconf, const float* __restrict__ rho_star,
                              const float* __restrict__ e_star, float* __restrict__ coarse,
                              int direction, int s) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  vd_load_pose_smem<NF>(sPose, posef);
  const int Wc = (P.W + s - 1) / s, Hc = (P.H + s - 1) / s;
  const bool rows = (direction & 1) == 0;
  const bool rev = direction >= 2;
  const int nchains = rows ? Hc : Wc;
  const int L = rows ? Wc : Hc;
  const int ch = blockIdx.x * blockDim.x + threadIdx.x;
  if (ch >= nchains) return;
  const size_t npix = (size_t)P.W * P.H;
  float cur = 0.0f;
  for (int m = 0; m < L; ++m) {
    const int pos = rev ? L - 1 - m : m;
    const int uc = rows ? pos : ch;
    const int vc = rows ? ch : pos;
    const int u = min(uc * s, P.W - 1), v = min(vc * s, P.H - 1);
    const size_t j = (size_t)v * P.W + u;
    const float own = rho_star[j];
    if (m == 0) {
      cur = own;
    } else {
      VdPixel<NF> px;
      vd_pixel_setup<NF>(px, P, sPose, u, v, q, npix, j, flow, prior_val, qhat, pconf);
      const float Ec = vd_energy<NF>(px, P, sPose, flow, npix, cur);
      if (!(Ec < e_star[j])) cur = own;
    }
    coarse[(size_t)vc * Wc + uc] = cur;
  }
}

// Hierarchical scheme: every pixel compares its own candidate with the value
// of its coarse cell.
template <int NF>
__global__ void __launch_bounds__(128)
k_hier_mix(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
           const float* __restrict__ q, const float* __restrict__ prior_val,
           const float* __restrict__ qhat, const float* __restrict__ pconf,
           const float* __restrict__ rho_star, const float* __restrict__ e_star,
           const float* __restrict__ coarse, int s, float* __restrict__ rho_mid,
           float* __restrict__ e_mid) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  vd_load_pose_smem<NF>(sPose, posef);
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= P.W || v >= P.H) return;
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)v * P.W + u;
  const int Wc = (P.W + s - 1) / s;
  const float up = coarse[(size_t)(v / s) * Wc + (u / s)];
  VdPixel<NF> px;
  vd_pixel_setup<NF>(px, P, sPose, u, v, q, npix, j, flow, prior_val, qhat, pconf);
  const float Eu = vd_energy<NF>(px, P, sPose, flow, npix, up);
  const float Es = e_star[j];
  const bool take = Eu < Es;
  rho_mid[j] = take ? up : rho_star[j];
  e_mid[j] = take ? Eu : Es;
}

template <int NF>
__global__ void __launch_bounds__(128)
k_eval_energy(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
              const float* __restrict__ q, const float* __restrict__ prior_val,
              const float* __restrict__ qhat, const float* __restrict__ pconf,
              const float* __restrict__ rho_in, float* __restrict__ e_out) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  vd_load_pose_smem<NF>(sPose, posef);
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= P.W || v >= P.H) return;
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)v * P.W + u;
  VdPixel<NF> px;
  vd_pixel_setup<NF>(px, P, sPose, u, v, q, npix, j, flow, prior_val, qhat, pconf);
  e_out[j] = vd_energy<NF>(px, P, sPose, flow, npix, rho_in[j]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline dim3 pix_grid(const vd_ctx* c, dim3 blk) {
  return dim3((c->W + blk.x - 1) / blk.x, (c->H + blk.y - 1) / blk.y);
}

cudaError_t launch_depth_sample(vd_ctx* c, uint32_t itcode, float s_pert, const float*) {
  const dim3 blk(VD_K1_BX, VD_K1_BY);
  const dim3 grd = pix_grid(c, blk);
  VD_DISPATCH_NF(c->N, (k_depth_sample<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->rho, c->q, c->prior_val, c->prior_rho,
                            c->qhat, c->prior_conf, itcode, s_pert, c->rho_star, c->e_star)));
  return cudaGetLastError();
}

cudaError_t launch_depth_propagate(vd_ctx* c, int direction) {
  const bool rows = (direction & 1) == 0;
  if (!c->prm.hierarchical) {
    const int nch = rows ? c->H : c->W;
    VD_DISPATCH_NF(c->N, (k_propagate_warp<NF><<<(nch + 3) / 4, 128, 0, c->stream>>>(
                              c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                              c->rho_star, c->e_star, c->rho, direction, 0)));
    return cudaGetLastError();
  }
  const int s = c->prm.hier_scale;
  const int Wc = (c->W + s - 1) / s, Hc = (c->H + s - 1) / s;
  const int nchc = rows ? Hc : Wc;
  VD_DISPATCH_NF(c->N, (k_hier_coarse<NF><<<(nchc + 63) / 64, 64, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            c->rho_star, c->e_star, c->coarse, direction, s)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 blk(32, 4);
  const dim3 grd = pix_grid(c, blk);
  VD_DISPATCH_NF(c->N, (k_hier_mix<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            c->rho_star, c->e_star, c->coarse, s, c->rho_mid, c->e_mid)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nch = rows ? c->H : c->W;
  VD_DISPATCH_NF(c->N, (k_propagate_warp<NF><<<(nch + 3) / 4, 128, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            c->rho_mid, c->e_mid, c->rho, direction, c->prm.hier_window)));
  return cudaGetLastError();
}

cudaError_t launch_eval_energy(vd_ctx* c, const float* rho_in, float* e_out) {
  const dim3 blk(32, 4);
  const dim3 grd = pix_grid(c, blk);
  VD_DISPATCH_NF(c->N, (k_eval_energy<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            rho_in, e_out)));
  return cudaGetLastError();
}
