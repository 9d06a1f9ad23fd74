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

// The same for kernels that need at least two flows.
#define VD_DISPATCH_NF2(N, KERNEL_CALL)     \
  switch (N) {                              \
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
__global__ void k_posef(DevParams P, const double* __restrict__ G, float* __restrict__ posef,
                        float2* __restrict__ posed) {
  const int t = threadIdx.x;
  if (t > P.N) return;
  const double* g = G + 12 * t;
  float* o = posef + 12 * t;
  float2* od = posed + 12 * t;
  for (int r = 0; r < 3; ++r) {
    const double k0 = r == 0 ? P.fx_d : (r == 1 ? 0.0 : 0.0);
    const double k1 = r == 1 ? P.fy_d : 0.0;
    const double k2 = r == 0 ? P.cx_d : (r == 1 ? P.cy_d : 1.0);
    // row r of K [R | tau] = k0 * row0 + k1 * row1 + k2 * row2
    for (int c = 0; c < 3; ++c)
      vd_store_pose_entry(o, od, 3 * r + c, k0 * g[c] + k1 * g[4 + c] + k2 * g[8 + c]);
    vd_store_pose_entry(o, od, 9 + r, k0 * g[3] + k1 * g[7] + k2 * g[11]);
  }
}

cudaError_t launch_posef(vd_ctx* c) {
  k_posef<<<1, 32, 0, c->stream>>>(c->dp, c->G, c->posef, c->posed);
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

// Candidate of slot k >= 1 (the value k_depth_sample draws for that slot).
__device__ __forceinline__ float vd_slot_candidate(const DevParams& P, uint32_t ctr0,
                                                   uint32_t itcode, int k, float cur, float s_pert,
                                                   bool has_prior, float prior_c) {
  if (k == 1 && has_prior) return prior_c;
  const int wi = k - 1;
  const uint4 w =
      vd_philox(make_uint4(ctr0, itcode, VD_TAG_DEPTH, (uint32_t)(wi >> 2)), P.key0, P.key1);
  const uint32_t x = vd_word(w, wi & 3);
  const float range = __fsub_rn(P.rho_max, P.rho_min);
  const float c = (k <= (P.K - 1) / 2) ? vd_cand_uniform(x, P.rho_min, range)
                                       : vd_cand_perturb(x, cur, s_pert);
  return vd_clamp(c, P.rho_min, P.rho_max);
}

// ---------------------------------------------------------------------------
// K1, staged schedule (N >= 2): the same candidates, energies and argmin as
// k_depth_sample, scheduled so that pruning frees lanes instead of leaving
// them idle.  A warp owns a row segment of 32 pixels.
//  * Pre-pass (lane = pixel): draw four slots per pixel, add the prior and
//    the X_1 term (neither needs a gather) and drop every candidate whose
//    partial key already exceeds the pixel's best key; the survivors go to
//    ring 1 in shared memory (most candidates end here).
//  * Stage 1: while ring 1 holds a full chunk, lane i takes its i-th entry,
//    of whichever pixel, adds flows 1..T1-1 and passes survivors to ring 2.
//  * Stage 2: full chunks of ring 2 add flows T1..N-1; a finished candidate
//    folds its key into the pixel's best key with atomicMin.
// Partial chunks wait for more entries until the last pre-pass.
// Key = energy bits << 32 | slot.  Energies are >= 0, so key order is
// (energy, slot) order and the minimum key is the argmin with ties to the
// lowest slot.  Dropping a candidate whose partial key exceeds a pixel's best
// key is exact: terms are non-negative, so its full key is at least the
// partial key, and the best key is that of a finished candidate.
// Ring bounds: the pre-pass runs only with fewer than 32 entries in ring 1
// and adds at most 128; a stage-1 chunk runs only with fewer than 32 entries
// in ring 2 and adds at most 32.
// ---------------------------------------------------------------------------
#define VD_KQ_R1 160
#define VD_KQ_R2 64
// resident blocks requested from the register allocator for 4 warps per
// block (scaled for other block sizes)
#ifndef VD_KQ_MINB
#define VD_KQ_MINB 5
#endif
#ifndef VD_KQ_T1
#define VD_KQ_T1 3
#endif
#ifndef VD_KQ_PRE_UNROLL
#define VD_KQ_PRE_UNROLL 1
#endif
#ifndef VD_KQ_STAGE_UNROLL
#define VD_KQ_STAGE_UNROLL 8
#endif
#define VD_STR(x) #x
#define VD_UNROLL(n) _Pragma(VD_STR(unroll n))

// Slot of ring position i >= 0 (unsigned: no sign correction of the
// remainder; a power-of-two ring is a mask)
template <unsigned R>
__device__ __forceinline__ unsigned vd_ring(int i) {
  return (unsigned)i % R;
}

// Flows [TA, TB) of one entry; false as soon as its partial energy exceeds
// `thr`, the entry's drop threshold (see vd_drop_threshold).
template <int TA, int TB>
__device__ __forceinline__ bool vd_stage_terms(const DevParams& P, const float4 (*sTw)[32],
                                               const float4* sTail,
                                               const float2* __restrict__ flow, size_t npix,
                                               int p, float thr, float c, float& E, float& xp,
                                               float& yp) {
  const float NaN = __int_as_float(0x7fc00000);
  VD_UNROLL(VD_KQ_STAGE_UNROLL)
  for (int t = TA; t < TB; ++t) {
    const float4 A = sTw[t - 1][p];
    const float4 M = sTail[t];
    const float hx = fmaf(c, M.x, A.x);
    const float hy = fmaf(c, M.y, A.y);
    const float hz = fmaf(c, M.z, A.z);
    const bool obs = vd_inside(xp, yp, P.W, P.H);   // false for NaN: behind camera t-1
    float2 F = make_float2(0.0f, 0.0f);
    if (obs) F = vd_bilinear(flow + (size_t)t * npix, P.W, P.H, xp, yp);
    float x, y;
    bool front;
    const float l2 = vd_flow_term(P, hx, hy, hz, obs, F.x, F.y, xp, yp, &x, &y, &front);
    E = fmaf(A.w, l2, E);
    xp = front ? x : NaN;
    yp = y;
    if (E > thr) return false;
  }
  return true;
}

// The key test "partial key > best key" as one float compare: for energies
// >= 0 the key order is the (energy, slot) order, so a candidate of a lower
// slot than the best is dropped when its energy exceeds the best energy, and
// one of a higher slot already when it equals it.
__device__ __forceinline__ float vd_drop_threshold(unsigned long long best, unsigned slot) {
  const float bE = __uint_as_float((unsigned)(best >> 32));
  if (slot < (unsigned)best) return bE;
  // the next float below bE (NaN stays NaN: a NaN best is beaten by any key)
  return bE <= 0.0f ? -1.0f : __int_as_float(__float_as_int(bE) - 1);
}

template <int NF, int WARPS>
__global__ void __launch_bounds__(32 * WARPS, (4 * VD_KQ_MINB) / WARPS)
k_depth_sample_q(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
                 const float* __restrict__ rho, const float* __restrict__ q,
                 const float* __restrict__ prior_val, const float* __restrict__ prior_rho,
                 const float* __restrict__ qhat, const float* __restrict__ pconf,
                 uint32_t itcode, float s_pert, float* __restrict__ rho_star,
                 float* __restrict__ e_star) {
  static_assert(NF >= 2, "the staged schedule needs a gathered flow term");
  constexpr int T1 = NF < VD_KQ_T1 ? NF : VD_KQ_T1;  // stage 1: flows [1, T1), stage 2: [T1, NF)
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  __shared__ float4 sTail[NF];                     // K tau of frame t+1 for flow t
  __shared__ float4 sT[WARPS][NF - 1][32];   // (a_x, a_y, a_z, q ln2) of flows 1..NF-1
  __shared__ float4 sR1[WARPS][VD_KQ_R1];    // (c, E, x, y) after flow T-1
  __shared__ float4 sR2[WARPS][VD_KQ_R2];
  __shared__ unsigned short sI1[WARPS][VD_KQ_R1];  // lane | slot << 5
  __shared__ unsigned short sI2[WARPS][VD_KQ_R2];
  __shared__ unsigned long long sBest[WARPS][32];
  const int tid = threadIdx.x;
  for (int i = tid; i < 12 * (NF + 1); i += blockDim.x) sPose[i] = posef[i];
  if (tid < NF)
    sTail[tid] = make_float4(posef[12 * (tid + 1) + 9], posef[12 * (tid + 1) + 10],
                             posef[12 * (tid + 1) + 11], 0.0f);
  __syncthreads();
  const int lane = tid & 31, wq = tid >> 5;
  const int u = blockIdx.x * 32 + lane;
  const int v = blockIdx.y * WARPS + wq;
  if (v >= P.H) return;                          // whole warps leave together
  const bool valid = u < P.W;
  const int uc = min(u, P.W - 1);
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)v * P.W + uc;
  const unsigned FULL = 0xffffffffu;
  const unsigned lt = (1u << lane) - 1u;
  const float NaN = __int_as_float(0x7fc00000);

  VdPixel<NF> px;
  vd_pixel_setup<NF>(px, P, sPose, uc, v, q, npix, j, flow, prior_val, qhat, pconf);
#pragma unroll
  for (int t = 1; t < NF; ++t)
    sT[wq][t - 1][lane] = make_float4(px.ax[t], px.ay[t], px.az[t], px.wl[t]);
  const float rmin = P.rho_min, rmax = P.rho_max;
  const float range = __fsub_rn(rmax, rmin);
  const float cur = rho[j];
  const float cur_c = vd_clamp(cur, rmin, rmax);
  {
    const float E0 = vd_energy<NF>(px, P, sPose, flow, npix, cur_c);
    sBest[wq][lane] = valid ? ((unsigned long long)__float_as_uint(E0) << 32) : 0ull;
  }
  const uint32_t ctr0 = (uint32_t)(j - (size_t)(uc % P.share));
  const int n_unif = (P.K - 1) / 2;
  bool has_prior = false;
  float prior_c = 0.0f;
  if (P.prior_kind != VD_PRIOR_NONE) {
    const float pr = prior_rho[j];
    has_prior = isfinite(pr);
    prior_c = vd_clamp(pr, rmin, rmax);
  }
  const float4 tail0 = sTail[0];
  const float4 (*sTw)[32] = sT[wq];
  unsigned long long* sBw = sBest[wq];
  __syncwarp();

  int h1 = 0, e1 = 0, h2 = 0, e2 = 0, k0 = 1;
  // one chunk of ring 2: flows T1..NF-1, then fold finished keys
  auto stage2 = [&]() {
    const int idx = h2 + lane;
    if (idx < e2) {
      const float4 e = sR2[wq][vd_ring<VD_KQ_R2>(idx)];
      const unsigned id = sI2[wq][vd_ring<VD_KQ_R2>(idx)];
      const int p = id & 31u;
      const unsigned slot = id >> 5;
      const float thr = vd_drop_threshold(*(volatile unsigned long long*)&sBw[p], slot);
      float E = e.y, xp = e.z, yp = e.w;
      if (vd_stage_terms<T1, NF>(P, sTw, sTail, flow, npix, p, thr, e.x, E, xp, yp))
        atomicMin(&sBw[p], ((unsigned long long)__float_as_uint(E) << 32) | slot);
    }
    h2 = min(h2 + 32, e2);
    __syncwarp();
  };
  while (true) {
    if (k0 < P.K) {
      // pre-pass over slots k0 .. k0+3 of every pixel of the warp
      const uint4 w = vd_philox(make_uint4(ctr0, itcode, VD_TAG_DEPTH, (uint32_t)((k0 - 1) >> 2)),
                                P.key0, P.key1);
      const unsigned long long bnd = *(volatile unsigned long long*)&sBw[lane];
VD_UNROLL(VD_KQ_PRE_UNROLL)
      for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        if (k >= P.K) break;
        const uint32_t x = vd_word(w, i);
        float cc = (k <= n_unif) ? vd_cand_uniform(x, rmin, range) : vd_cand_perturb(x, cur, s_pert);
        cc = vd_clamp(cc, rmin, rmax);
        if (k == 1 && has_prior) cc = prior_c;
        float Ek = vd_prior_energy<NF>(px, P, cc);
        const float hx = fmaf(cc, tail0.x, px.ax[0]);
        const float hy = fmaf(cc, tail0.y, px.ay[0]);
        const float hz = fmaf(cc, tail0.z, px.az[0]);
        float x1, y1;
        bool f1;
        const float l2 = vd_flow_term(P, hx, hy, hz, true, px.f1x, px.f1y, px.u, px.v, &x1, &y1, &f1);
        Ek = fmaf(px.wl[0], l2, Ek);
        const unsigned long long key = ((unsigned long long)__float_as_uint(Ek) << 32) | (unsigned)k;
        const bool keep = valid && key < bnd;
        const unsigned m = __ballot_sync(FULL, keep);
        if (keep) {
          const unsigned pos = vd_ring<VD_KQ_R1>(e1 + __popc(m & lt));
          sR1[wq][pos] = make_float4(cc, Ek, f1 ? x1 : NaN, y1);
          sI1[wq][pos] = (unsigned short)(lane | (k << 5));
        }
        e1 += __popc(m);
      }
      k0 += 4;
      __syncwarp();
    }
    const bool last = k0 >= P.K;
    while (e1 - h1 >= 32 || (last && e1 > h1)) {
      // one chunk of ring 1: flows 1..T1-1
      const int idx = h1 + lane;
      bool keep = false;
      float4 st = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      unsigned id = 0;
      if (idx < e1) {
        st = sR1[wq][vd_ring<VD_KQ_R1>(idx)];
        id = sI1[wq][vd_ring<VD_KQ_R1>(idx)];
        const int p = id & 31u;
        const unsigned slot = id >> 5;
        const float thr = vd_drop_threshold(*(volatile unsigned long long*)&sBw[p], slot);
        keep = vd_stage_terms<1, T1>(P, sTw, sTail, flow, npix, p, thr, st.x, st.y, st.z, st.w);
        if (T1 == NF && keep)
          atomicMin(&sBw[p], ((unsigned long long)__float_as_uint(st.y) << 32) | slot);
      }
      h1 = min(h1 + 32, e1);
      if (T1 < NF) {
        const unsigned m = __ballot_sync(FULL, keep);
        if (keep) {
          const unsigned pos = vd_ring<VD_KQ_R2>(e2 + __popc(m & lt));
          sR2[wq][pos] = st;
          sI2[wq][pos] = (unsigned short)id;
        }
        e2 += __popc(m);
        __syncwarp();
        while (e2 - h2 >= 32) stage2();
      } else {
        __syncwarp();
      }
    }
    if (last) {
      while (e2 > h2) stage2();
      break;
    }
  }
  __syncwarp();
  if (!valid) return;
  const unsigned long long kb = *(volatile unsigned long long*)&sBw[lane];
  const int kslot = (int)(kb & 0xffffffffull);
  rho_star[j] = kslot == 0 ? cur_c
                           : vd_slot_candidate(P, ctr0, itcode, kslot, cur, s_pert, has_prior, prior_c);
  e_star[j] = __uint_as_float((unsigned)(kb >> 32));
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
// The loads of one pixel's propagation step that do not depend on the
// carried value (its rigidness, X_1 at the pixel, the prior, rho* and E*),
// issued one pixel ahead of the step that uses them, so that their latency
// overlaps the current pixel's energy.
template <int NF>
struct VdPixLoads {
  float q[NF];
  float2 f1;
  float pv, qh, pc;
  float own, e;
};

template <int NF>
__device__ __forceinline__ void vd_pix_load(VdPixLoads<NF>& L, const DevParams& P,
                                            const float2* __restrict__ flow,
                                            const float* __restrict__ q,
                                            const float* __restrict__ prior_val,
                                            const float* __restrict__ qhat,
                                            const float* __restrict__ pconf,
                                            const float* __restrict__ rho_star,
                                            const float* __restrict__ e_star, size_t npix,
                                            size_t j) {
#pragma unroll
  for (int t = 0; t < NF; ++t) L.q[t] = __ldg(q + (size_t)t * npix + j);
  L.f1 = __ldg(flow + j);
  L.pv = 0.0f;
  L.qh = 0.0f;
  L.pc = 0.0f;
  if (P.prior_kind != VD_PRIOR_NONE) {
    L.pv = __ldg(prior_val + j);
    L.qh = __ldg(qhat + j);
    L.pc = __ldg(pconf + j);
  }
  L.own = rho_star[j];
  L.e = e_star[j];
}

// vd_pixel_setup from the preloaded values (the same arithmetic).
template <int NF>
__device__ __forceinline__ void vd_pixel_from_loads(VdPixel<NF>& px, const DevParams& P,
                                                    const float* __restrict__ sPose, int u, int v,
                                                    const VdPixLoads<NF>& L) {
  const float rx = ((float)u - P.cx) / P.fx;
  const float ry = ((float)v - P.cy) / P.fy;
#pragma unroll
  for (int t = 0; t < NF; ++t) {
    const float* M = sPose + 12 * (t + 1);
    px.ax[t] = fmaf(M[0], rx, fmaf(M[1], ry, M[2]));
    px.ay[t] = fmaf(M[3], rx, fmaf(M[4], ry, M[5]));
    px.az[t] = fmaf(M[6], rx, fmaf(M[7], ry, M[8]));
    px.wl[t] = L.q[t] * VD_LN2;
  }
  px.f1x = L.f1.x;
  px.f1y = L.f1.y;
  px.u = (float)u;
  px.v = (float)v;
  px.pw = 0.0f;
  px.pv = 0.0f;
  if (P.prior_kind != VD_PRIOR_NONE && isfinite(L.pv)) {
    px.pv = L.pv;
    px.pw = L.qh * L.pc;
  }
}

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
  const float Ec = vd_energy_full<NF>(px, P, sPose, flow, npix, cur);
  return (Ec < e_own) ? cur : own;
}

template <int NF>
__global__ void __launch_bounds__(128)
k_propagate_warp(DevParams P, const float* __restrict__ posef, const float2* __restrict__ flow,
                 const float* __restrict__ q, const float* __restrict__ prior_val,
                 const float* __restrict__ qhat, const float* __restrict__ pconf,
                 const float* __restrict__ rho_star, const float* __restrict__ e_star,
                 float* __restrict__ rho_new, int direction, int restart, int s) {
  __shared__ float sPose[12 * (VD_MAX_FLOWS + 1)];
  vd_load_pose_smem<NF>(sPose, posef);
  const bool rows = (direction & 1) == 0;
  const bool rev = direction >= 2;
  // s > 0: the chains of the coarse grid of representative pixels
  // (min(s uc, W - 1), min(s vc, H - 1)), written to the coarse map
  // rho_new[vc][uc] (the hierarchical scheme's global pass)
  const int Wc = s > 0 ? (P.W + s - 1) / s : P.W, Hc = s > 0 ? (P.H + s - 1) / s : P.H;
  const int nchains = rows ? Hc : Wc;
  const int L = rows ? Wc : Hc;
  const int ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (ch >= nchains) return;          // whole warps leave together
  const int seg = (L + 31) >> 5;
  const int m0 = min(L, lane * seg), m1 = min(L, m0 + seg);
  // position m of the chain: pixel (u, v) and index j of the inputs, and the
  // index of the output (j itself at full resolution)
  auto pix = [&](int m, int* u, int* v, size_t* o) -> size_t {
    const int pos = rev ? L - 1 - m : m;
    const int uc = rows ? pos : ch, vc = rows ? ch : pos;
    *u = s > 0 ? min(uc * s, P.W - 1) : uc;
    *v = s > 0 ? min(vc * s, P.H - 1) : vc;
    *o = (size_t)vc * Wc + uc;
    return (size_t)VD_CHK(VD_SITE_CHAIN, (long long)(*v) * P.W + (*u), (long long)P.W * P.H);
  };
  // phase A; the next pixel's loads are issued before this pixel's energy
  const size_t npix = (size_t)P.W * P.H;
  float cur = 0.0f;
  VdPixLoads<NF> Ln;
  int un = 0, vn = 0;
  size_t jn = 0, on = 0;
  if (m0 < m1) {
    jn = pix(m0, &un, &vn, &on);
    vd_pix_load<NF>(Ln, P, flow, q, prior_val, qhat, pconf, rho_star, e_star, npix, jn);
  }
  for (int m = m0; m < m1; ++m) {
    const VdPixLoads<NF> L = Ln;
    const int u = un, v = vn;
    const size_t o = on;
    if (m + 1 < m1) {
      jn = pix(m + 1, &un, &vn, &on);
      vd_pix_load<NF>(Ln, P, flow, q, prior_val, qhat, pconf, rho_star, e_star, npix, jn);
    }
    if (m == m0 || (restart > 0 && m % restart == 0)) {
      cur = L.own;
    } else {
      VdPixel<NF> px;
      vd_pixel_from_loads<NF>(px, P, sPose, u, v, L);
      // every gathered flow's taps in flight at once: the walk is a chain of
      // dependent energies, so their latency, not their work, sets its pace
      const float Ec = vd_energy_full<NF>(px, P, sPose, flow, npix, cur);
      cur = (Ec < L.e) ? cur : L.own;
    }
    rho_new[o] = cur;
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
        size_t o;
        const size_t j = pix(m, &u, &v, &o);
        const float own = rho_star[j];
        float nc;
        if (restart > 0 && m % restart == 0)
          nc = own;
        else
          nc = vd_prop_step<NF>(P, sPose, flow, q, prior_val, qhat, pconf, c, own, e_star[j], u, v, j);
        if (nc == rho_new[o]) {
          merged = true;
          break;
        }
        rho_new[o] = nc;
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

template <int WARPS>
static cudaError_t launch_depth_sample_q(vd_ctx* c, uint32_t itcode, float s_pert, int nf) {
  const dim3 blk(32 * WARPS);
  const dim3 grd((c->W + 31) / 32, (c->H + WARPS - 1) / WARPS);
  VD_DISPATCH_NF2(nf, (k_depth_sample_q<NF, WARPS><<<grd, blk, 0, c->stream>>>(
                          c->dp, c->posef, c->flow, c->rho, c->q, c->prior_val, c->prior_rho,
                          c->qhat, c->prior_conf, itcode, s_pert, c->rho_star, c->e_star)));
  return cudaGetLastError();
}

cudaError_t launch_depth_sample(vd_ctx* c, uint32_t itcode, float s_pert, int nf) {
#ifndef VD_K1_DIRECT
  if (nf >= 2) {
    switch (c->k1_warps) {
      case 1: return launch_depth_sample_q<1>(c, itcode, s_pert, nf);
      case 2: return launch_depth_sample_q<2>(c, itcode, s_pert, nf);
      case 4: return launch_depth_sample_q<4>(c, itcode, s_pert, nf);
      default: return cudaErrorInvalidValue;
    }
  }
#endif
  const dim3 blk(VD_K1_BX, VD_K1_BY);
  const dim3 grd = pix_grid(c, blk);
  VD_DISPATCH_NF(nf, (k_depth_sample<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->rho, c->q, c->prior_val, c->prior_rho,
                            c->qhat, c->prior_conf, itcode, s_pert, c->rho_star, c->e_star)));
  return cudaGetLastError();
}

cudaError_t launch_depth_propagate(vd_ctx* c, int direction, int nf) {
  const bool rows = (direction & 1) == 0;
  if (!c->prm.hierarchical) {
    const int nch = rows ? c->H : c->W;
    VD_DISPATCH_NF(nf, (k_propagate_warp<NF><<<(nch + 3) / 4, 128, 0, c->stream>>>(
                              c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                              c->rho_star, c->e_star, c->rho, direction, 0, 0)));
    return cudaGetLastError();
  }
  const int s = c->prm.hier_scale;
  const int Wc = (c->W + s - 1) / s, Hc = (c->H + s - 1) / s;
  const int nchc = rows ? Hc : Wc;
  // global pass on the coarse grid: the same segmented exact chain walk
  VD_DISPATCH_NF(nf, (k_propagate_warp<NF><<<(nchc + 3) / 4, 128, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            c->rho_star, c->e_star, c->coarse, direction, 0, s)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 blk(32, 4);
  const dim3 grd = pix_grid(c, blk);
  VD_DISPATCH_NF(nf, (k_hier_mix<NF><<<grd, blk, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            c->rho_star, c->e_star, c->coarse, s, c->rho_mid, c->e_mid)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nch = rows ? c->H : c->W;
  VD_DISPATCH_NF(nf, (k_propagate_warp<NF><<<(nch + 3) / 4, 128, 0, c->stream>>>(
                            c->dp, c->posef, c->flow, c->q, c->prior_val, c->qhat, c->prior_conf,
                            c->rho_mid, c->e_mid, c->rho, direction, c->prm.hier_window, 0)));
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

VD_CHECK_ACCESSOR(depth)
