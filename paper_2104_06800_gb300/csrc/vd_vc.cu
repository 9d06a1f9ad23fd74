// Visibility-coverage (VC) score of the reference depth in frames of known
// pose, and the VO stride / keyframe rules (Sec. III-B "VO Stride and
// Keyframe Selection", Eq. 8).
//
// One thread per reference pixel projects its depth into every scored frame.
// Warp ballots count the depth pixels and, per frame, the visible ones
// (64-bit integer atomics); a visible point stores 1 into the byte of its
// nearest pixel cell in the frame's coverage map (plain stores: every writer
// of a cell writes the same value), and a second kernel counts the covered
// cells (the popcount of words whose bytes are 0 or 1).  All decisions are
// taken in float32 with explicitly rounded operations (no contraction), in
// the order the header states, so the counts are exact integers and
// independent of the schedule.
#include "vd_device.cuh"

#define VC_BLOCK 256

static_assert(VD_VC_MAX_FRAMES >= VD_MAX_FLOWS, "one VC entry per flow");

__global__ void __launch_bounds__(VC_BLOCK)
k_vc_project(const float* __restrict__ rho, int W, int H, float fx, float fy, float cx, float cy,
             const double* __restrict__ poses, int nf, unsigned char* __restrict__ cover,
             size_t stride, unsigned long long* __restrict__ counts) {
  __shared__ float sT[(VD_MAX_FLOWS + 1) * 12];
  for (int i = threadIdx.x; i < 12 * nf; i += VC_BLOCK) sT[i] = (float)poses[i];
  __syncthreads();
  const unsigned FULL = 0xffffffffu;
  const size_t npix = (size_t)W * H;
  const size_t j = (size_t)blockIdx.x * VC_BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  float r = 0.0f;
  bool valid = false;
  int u = 0, v = 0;
  if (j < npix) {
    r = rho[j];
    valid = isfinite(r) && r > 0.0f;
    v = (int)(j / W);
    u = (int)(j - (size_t)v * W);
  }
  const unsigned bv = __ballot_sync(FULL, valid);
  if (lane == 0 && bv) atomicAdd(&counts[0], (unsigned long long)__popc(bv));
  const float rx = __fdiv_rn(__fsub_rn((float)u, cx), fx);
  const float ry = __fdiv_rn(__fsub_rn((float)v, cy), fy);
  const float xmax = (float)(W - 1), ymax = (float)(H - 1);
  for (int k = 0; k < nf; ++k) {
    const float* T = sT + 12 * k;   // row i: R_i0, R_i1, R_i2, tau_i
    bool in = false;
    size_t cell = 0;
    if (valid) {
      float h[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        h[i] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T[4 * i], rx), __fmul_rn(T[4 * i + 1], ry)),
                                   T[4 * i + 2]),
                         __fmul_rn(r, T[4 * i + 3]));
      if (h[2] > VD_Z_EPS) {
        const float x = __fadd_rn(__fmul_rn(fx, __fdiv_rn(h[0], h[2])), cx);
        const float y = __fadd_rn(__fmul_rn(fy, __fdiv_rn(h[1], h[2])), cy);
        if (x >= 0.0f && x <= xmax && y >= 0.0f && y <= ymax) {
          in = true;   // x + 1/2 <= W - 1/2, so the cell is inside the frame
          const int xi = (int)floorf(__fadd_rn(x, 0.5f));
          const int yi = (int)floorf(__fadd_rn(y, 0.5f));
          cell = (size_t)yi * W + xi;
        }
      }
    }
    const unsigned b = __ballot_sync(FULL, in);
    if (lane == 0 && b) atomicAdd(&counts[1 + k], (unsigned long long)__popc(b));
    if (in) cover[(size_t)k * stride + VD_CHK(VD_SITE_VC_CELL, (long long)cell, (long long)stride)] = 1;
  }
}

// Covered cells of each frame's map (frame = blockIdx.y) into
// counts[1 + nf + k]; `stride` bytes per map, a multiple of 16.
__global__ void __launch_bounds__(VC_BLOCK)
k_vc_popc(const unsigned char* __restrict__ cover, size_t stride, int nf,
          unsigned long long* __restrict__ counts) {
  const int k = blockIdx.y;
  const uint4* b = reinterpret_cast<const uint4*>(cover + (size_t)k * stride);
  const size_t n16 = stride / 16;
  unsigned long long n = 0;
  for (size_t w = (size_t)blockIdx.x * VC_BLOCK + threadIdx.x; w < n16;
       w += (size_t)gridDim.x * VC_BLOCK) {
    const uint4 q = b[w];
    n += (unsigned long long)(__popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&counts[1 + nf + k], n);
}

// Counts of the reference depth in nf frames with poses `poses_dev` (device,
// 12 doubles each), into `out` (host).
static vd_status vc_run(vd_ctx* c, const double* poses_dev, int nf, vd_vc* out) {
  const size_t stride = c->vc_stride;
  VD_CU(cudaMemsetAsync(c->vc_cover, 0, stride * nf, c->stream));
  VD_CU(cudaMemsetAsync(c->vc_counts, 0, sizeof(unsigned long long) * (1 + 2 * nf), c->stream));
  const int nblk = (int)((c->npix + VC_BLOCK - 1) / VC_BLOCK);
  k_vc_project<<<nblk, VC_BLOCK, 0, c->stream>>>(
      c->rho, c->W, c->H, (float)c->desc.fx, (float)c->desc.fy, (float)c->desc.cx,
      (float)c->desc.cy, poses_dev, nf, c->vc_cover, stride, c->vc_counts);
  VD_CU(cudaGetLastError());
  const int pblk =
      (int)std::min<size_t>((stride / 16 + VC_BLOCK - 1) / VC_BLOCK, (size_t)c->num_sms);
  k_vc_popc<<<dim3(pblk, nf), VC_BLOCK, 0, c->stream>>>(c->vc_cover, stride, nf, c->vc_counts);
  VD_CU(cudaGetLastError());
  unsigned long long h[1 + 2 * (VD_MAX_FLOWS + 1)];
  VD_CU(cudaMemcpyAsync(h, c->vc_counts, sizeof(unsigned long long) * (1 + 2 * nf),
                        cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof *out);
  out->n_frames = nf;
  out->n_pixels = (long long)c->npix;
  out->n_depth = (long long)h[0];
  for (int k = 0; k < nf; ++k) {
    out->n_visible[k] = (long long)h[1 + k];
    out->n_covered[k] = (long long)h[1 + nf + k];
    const double V = out->n_depth ? (double)out->n_visible[k] / (double)out->n_depth : 0.0;
    const double C = (double)out->n_covered[k] / (double)out->n_pixels;
    out->visibility[k] = V;
    out->coverage[k] = C;
    out->vc[k] = (V > 0.0 && C > 0.0) ? 2.0 * V * C / (V + C) : 0.0;
  }
  return VD_OK;
}

extern "C" vd_status vd_vc_scores(vd_ctx* c, vd_vc* out) {
  if (!c || !out) return VD_ERR_ARG;
  return vc_run(c, c->G + 12, c->N, out);
}

extern "C" vd_status vd_vc_pose(vd_ctx* c, const double* T, vd_vc* out) {
  if (!c || !T || !out) return VD_ERR_ARG;
  for (int i = 0; i < 12; ++i)
    if (!isfinite(T[i])) return VD_ERR_ARG;
  VD_CU(cudaMemcpyAsync(c->vc_pose, T, sizeof(double) * 12, cudaMemcpyHostToDevice, c->stream));
  return vc_run(c, c->vc_pose, 1, out);
}

extern "C" int vd_vc_stride(const double* vc, int n, double tau_stride) {
  if (!vc || n < 1) return 0;
  for (int t = 1; t <= n; ++t)
    if (vc[t - 1] < tau_stride) return t;
  return n;
}

extern "C" int vd_vc_is_keyframe(double vc, double tau_keyframe) {
  return vc < tau_keyframe ? 1 : 0;
}

VD_CHECK_ACCESSOR(vc)
