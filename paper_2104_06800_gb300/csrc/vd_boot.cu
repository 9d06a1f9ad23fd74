// Bootstrap of the EM (VOLDOR+ bootstraps from priors where it has them and
// from monocular flow otherwise, Sec. I and III-A) and small utility kernels.
// Monocular: the first relative pose from the epipolar constraint of X_1 by
// the linear 8-point method on calibrated rays (Longuet-Higgins 1981), made
// robust to the heavy-tailed Fisk noise by iterative re-weighting with the
// weight 1 / (1 + (d / alpha0)^2) of the Sampson distance d.
#include "vd_device.cuh"
#include "vd_df64.cuh"
#include "vd_geom64.cuh"

#define EP_THREADS 256

// ---------------------------------------------------------------------------
// Initial inverse depth: Philox word 0 of (j, ITER_BOOT, TAG_INIT, 0) mapped
// uniformly to [rho_min, rho_max]; the clamped prior where it is valid.
// ---------------------------------------------------------------------------
__global__ void k_initial_rho(DevParams P, const float* __restrict__ prior_rho,
                              float* __restrict__ rho) {
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npix) return;
  const uint4 w = vd_philox(make_uint4((uint32_t)j, VD_ITER_BOOT, VD_TAG_INIT, 0u), P.key0, P.key1);
  float r = vd_cand_uniform(w.x, P.rho_min, __fsub_rn(P.rho_max, P.rho_min));
  if (P.prior_kind != VD_PRIOR_NONE) {
    const float pr = prior_rho[j];
    if (isfinite(pr)) r = vd_clamp(pr, P.rho_min, P.rho_max);
  }
  rho[j] = r;
}

cudaError_t launch_initial_rho(vd_ctx* c) {
  k_initial_rho<<<(unsigned)((c->npix + 255) / 256), 256, 0, c->stream>>>(c->dp, c->prior_rho,
                                                                          c->rho);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weighted normal matrix M = sum_j w_j r_j r_j^T, r_j = b (x) a, upper
// triangle (45 entries) accumulated in double-float, per-block partial
// sums in float64.
// ---------------------------------------------------------------------------

// Accumulation in double-float (vd_df64.cuh): a product with its exact
// error, and a sum whose error term is carried along (the "sloppy" form:
// one TwoSum of the leading parts, the trailing parts added in float32),
// about 2^-44 per operation.
__device__ __forceinline__ vd_df ep_df_mul(vd_df a, vd_df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);          // exact error of the product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = p + e;
  return {s, e - (s - p)};
}
__device__ __forceinline__ vd_df ep_df_add(vd_df a, vd_df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float err = (a.hi - (s - bb)) + (b.hi - bb);   // TwoSum
  err += a.lo + b.lo;
  const float t = s + err;
  return {t, err - (t - s)};
}

// Calibrated rays of pixel (u, v) and of its flow end point, in
// double-float from the float32 inputs (no float64 instruction per pixel:
// on this GPU one costs a warp 64 cycles).
__device__ __forceinline__ void ep_rays(const DevParams& P, int u, int v, float2 F, vd_df* a0,
                                        vd_df* a1, vd_df* b0, vd_df* b1) {
  const vd_df cx = vd_df_make(P.kdf[4], P.kdf[5]), cy = vd_df_make(P.kdf[6], P.kdf[7]);
  const vd_df ifx = vd_df_make(P.kdf[8], P.kdf[9]), ify = vd_df_make(P.kdf[10], P.kdf[11]);
  const vd_df uu = vd_df_make((float)u), vv = vd_df_make((float)v);
  *a0 = vd_df_mul(vd_df_sub(uu, cx), ifx);
  *a1 = vd_df_mul(vd_df_sub(vv, cy), ify);
  *b0 = vd_df_mul(vd_df_sub(vd_two_sum((float)u, F.x), cx), ifx);
  *b1 = vd_df_mul(vd_df_sub(vd_two_sum((float)v, F.y), cy), ify);
}

__device__ __forceinline__ vd_df ep_shfl_xor(vd_df x, int o) {
  return {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

// two blocks per SM (128 registers, no spills): 0.95 -> 0.91 ms of bootstrap
// per kerb window against one block at 154 registers
#ifndef EP_MINB
#define EP_MINB 2
#endif
__global__ void __launch_bounds__(EP_THREADS, EP_MINB)
k_ep_normal(DevParams P, const float2* __restrict__ flow, const double* __restrict__ Eprev,
            int weighted, float2* __restrict__ partial) {
  __shared__ vd_df sW[EP_THREADS / 32][45];
  vd_df acc[45];
#pragma unroll
  for (int i = 0; i < 45; ++i) acc[i] = {0.0f, 0.0f};
  // the IRLS weight needs no extended precision: on noise-free flow every
  // row is orthogonal to E whatever the weights, on noisy flow a 1e-7
  // relative weight error moves E far below the pose tolerance
  float Ef[9];
  for (int i = 0; i < 9; ++i) Ef[i] = weighted ? (float)Eprev[i] : 0.0f;
  const float ff = sqrtf(P.fx * P.fy);
  const float ia = 1.0f / P.alpha0;
  const size_t npix = (size_t)P.W * P.H;
  for (size_t j = (size_t)blockIdx.x * EP_THREADS + threadIdx.x; j < npix;
       j += (size_t)gridDim.x * EP_THREADS) {
    const int v = (int)(j / P.W), u = (int)(j - (size_t)v * P.W);
    const float2 F = flow[j];
    vd_df A0, A1, B0, B1;
    ep_rays(P, u, v, F, &A0, &A1, &B0, &B1);
    float w = 1.0f;
    if (weighted) {
      const float af[3] = {A0.hi, A1.hi, 1.0f}, bf[3] = {B0.hi, B1.hi, 1.0f};
      float Ea[3], Etb[3];
      for (int i = 0; i < 3; ++i) {
        Ea[i] = Ef[3 * i] * af[0] + Ef[3 * i + 1] * af[1] + Ef[3 * i + 2] * af[2];
        Etb[i] = Ef[i] * bf[0] + Ef[3 + i] * bf[1] + Ef[6 + i] * bf[2];
      }
      const float num = bf[0] * Ea[0] + bf[1] * Ea[1] + bf[2] * Ea[2];
      const float den = Ea[0] * Ea[0] + Ea[1] * Ea[1] + Etb[0] * Etb[0] + Etb[1] * Etb[1];
      const float d = ff * fabsf(num) * rsqrtf(fmaxf(den, 1e-30f)) * ia;
      w = 1.0f / (1.0f + d * d);
    }
    // r = b (x) a with a2 = b2 = 1
    const vd_df one = {1.0f, 0.0f};
    vd_df r[9] = {ep_df_mul(B0, A0), ep_df_mul(B0, A1), B0,
                  ep_df_mul(B1, A0), ep_df_mul(B1, A1), B1,
                  A0,                A1,                one};
    int k = 0;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const vd_df wr = ep_df_mul(r[p], {w, 0.0f});
#pragma unroll
      for (int q = p; q < 9; ++q) acc[k] = ep_df_add(acc[k], ep_df_mul(wr, r[q])), ++k;
    }
  }
  // warp sums by a reduce-scatter over 64 slots (45 entries, zeros after):
  // at lane bit s the upper half-lanes keep the upper half of the slots and
  // receive their partner's copy of it, the lower ones the lower half, so
  // that lane L ends with the warp's sums of slots 2L and 2L + 1 (62
  // double-float additions instead of 45 x 5); then the block sum over
  // warps.  Fixed order throughout; one partial per block.
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  {
    vd_df r[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {   // s = 16: slots i and i + 32
      const bool upper = (lane & 16) != 0;
      const vd_df a = acc[i];
      const vd_df b = i + 32 < 45 ? acc[i + 32] : vd_df{0.0f, 0.0f};
      const vd_df send = upper ? a : b;
      r[i] = vd_df_add(upper ? b : a, ep_shfl_xor(send, 16));
    }
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
      const bool upper = (lane & s) != 0;
#pragma unroll
      for (int i = 0; i < 2 * s; ++i) {
        const vd_df send = upper ? r[i] : r[i + 2 * s];
        const vd_df keep = upper ? r[i + 2 * s] : r[i];
        r[i] = vd_df_add(keep, ep_shfl_xor(send, s));
      }
    }
    if (2 * lane < 45) sW[wid][2 * lane] = r[0];
    if (2 * lane + 1 < 45) sW[wid][2 * lane + 1] = r[1];
  }
  __syncthreads();
  if (threadIdx.x < 45) {
    vd_df s = sW[0][threadIdx.x];
    for (int w = 1; w < EP_THREADS / 32; ++w) s = vd_df_add(s, sW[w][threadIdx.x]);
    partial[(size_t)blockIdx.x * 45 + threadIdx.x] = make_float2(s.hi, s.lo);
  }
}

// Warp 0 of k_ep_solve (tid = lane): (M + d I)^-1 of the packed upper
// triangle sM, d = 1e-14 trace(M).  M + d I = L L^T column by column (every
// lane forms the pivot, lanes j+1..8 the entries of column j), then lanes
// 0..8 each solve for one column of the inverse.
__device__ __forceinline__ void ep_inverse(const double* sM, double* sA, double* sRd, double* sI,
                                           int tid) {
  if (tid < 9) {
    // lane q copies column q of the upper triangle into row q's lower part
    int k = 0;
    for (int p = 0; p < 9; ++p)
      for (int q = p; q < 9; ++q, ++k)
        if (q == tid) sA[9 * q + p] = sM[k];   // lower triangle, row q column p
  }
  __syncwarp();
  double tr = 0.0;
  for (int p = 0; p < 9; ++p) tr += sA[10 * p];
  const double shift = 1e-14 * tr + 1e-300;
  // Cholesky by columns: every lane forms the pivot of column j, lane i > j
  // its entry of the column (the same operations in the same order as the
  // row-by-row form, spread over lanes)
  for (int j = 0; j < 9; ++j) {
    double d = sA[10 * j] + shift;
    for (int m = 0; m < j; ++m) d -= sA[9 * j + m] * sA[9 * j + m];
    d = fmax(d, shift);
    const double r = vd_rsqrt64(d);
    if (tid == 0) sRd[j] = r;
    if (tid > j && tid < 9) {
      double s = sA[9 * tid + j];
      for (int m = 0; m < j; ++m) s -= sA[9 * tid + m] * sA[9 * j + m];
      sA[9 * tid + j] = s * r;
    }
    __syncwarp();
  }
  if (tid < 9) {   // column tid of the inverse: L L^T z = e_tid
    double y[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double s = (i == tid) ? 1.0 : 0.0;
#pragma unroll
      for (int m = 0; m < i; ++m) s -= sA[9 * i + m] * y[m];
      y[i] = s * sRd[i];
    }
#pragma unroll
    for (int i = 8; i >= 0; --i) {
      double s = y[i];
#pragma unroll
      for (int m = i + 1; m < 9; ++m) s -= sA[9 * m + i] * y[m];
      y[i] = s * sRd[i];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) sI[9 * tid + i] = y[i];
  }
  __syncwarp();
}

#ifndef EP_SQUARINGS
#define EP_SQUARINGS 4
#endif
// Sum the partials (fixed order) and take the eigenvector of the smallest
// eigenvalue as E (unit Frobenius norm), by inverse iteration on the
// symmetric positive semi-definite M shifted by 1e-14 trace(M): warp 0
// factors M + d I = L L^T, lanes 0..8 each solve one column of the inverse
// B; 81 threads square B / trace(B) EP_SQUARINGS times (every squaring
// does the work of as many steps as the last one did: 1, 2, 4, ...), the
// start vector goes through that power once, then every step
// x <- B x / |x| is a 9-lane matrix-vector product, until the iterate stops
// moving.  `warm` starts from the previous round's E, else from
// (1, ..., 1) / 3.
__global__ void __launch_bounds__(512)
k_ep_solve(const float2* __restrict__ partial, int nblk, double* __restrict__ Mout,
           double* __restrict__ Eio, int warm) {
  __shared__ double sM[45];
  __shared__ double sA[81];   // L (lower triangle)
  __shared__ double sRd[9];   // 1 / L_jj
  __shared__ double sI[81];   // (M + d I)^-1, column-major by solving lane
  __shared__ double sP[2][81];   // powers of B / trace(B)
  const int tid = threadIdx.x;
  {
    // entries wp, wp + 16, wp + 32 by warp wp (lanes: strided blocks), each
    // a double-float sum in fixed order, then one conversion to float64
    const int lane = tid & 31, wp = tid >> 5;
    vd_df s[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int b = lane; b < nblk; b += 32) {
      const float2* row = partial + (size_t)b * 45;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (wp + 16 * k < 45) {
          const float2 x = row[wp + 16 * k];
          s[k] = vd_df_add(s[k], vd_df_make(x.x, x.y));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      for (int o = 16; o > 0; o >>= 1) s[k] = vd_df_add(s[k], ep_shfl_xor(s[k], o));
      if (lane == 0 && wp + 16 * k < 45) {
        const double d = vd_df_to(s[k]);
        sM[wp + 16 * k] = d;
        Mout[wp + 16 * k] = d;
      }
    }
  }
  __syncthreads();
  if (tid < 32) ep_inverse(sM, sA, sRd, sI, tid);
  __syncthreads();
  // B / trace(B) (entries at most 1: B is positive definite), then its
  // squares; products of entries at most 1 neither overflow nor, over
  // EP_SQUARINGS <= 5 squarings of a unit-trace matrix, underflow the
  // dominant part
  if (tid < 81) {
    double tr = 0.0;
    for (int p = 0; p < 9; ++p) tr += sI[10 * p];
    sP[0][tid] = sI[tid] / tr;
  }
#pragma unroll 1
  for (int k = 0; k < EP_SQUARINGS; ++k) {
    __syncthreads();
    if (tid < 81) {
      const double* B = sP[k & 1];
      const int r = tid / 9, c = tid - 9 * r;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 9; ++m) acc = fma(B[9 * r + m], B[9 * m + c], acc);
      sP[(k + 1) & 1][tid] = acc;
    }
  }
  __syncthreads();
  if (tid >= 32) return;
  const double* Bq = sP[EP_SQUARINGS & 1];
  // lane i < 9 holds x_i
  double xi = 0.0;
  if (tid < 9) xi = warm ? Eio[tid] : 1.0 / 3.0;
  double n2 = xi * xi;
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  if (!(n2 > 0.0) || !isfinite(n2)) {
    xi = tid < 9 ? 1.0 / 3.0 : 0.0;
    n2 = 1.0;
  }
  xi *= vd_rsqrt64(n2);
  {
    // x <- B^(2^EP_SQUARINGS) x / |.|: its sign follows x (x^T B^k x >= 0)
    double yi = 0.0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const double xm = __shfl_sync(0xffffffffu, xi, m);
      if (tid < 9) yi = fma(Bq[9 * m + tid], xm, yi);
    }
    double n = yi * yi;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    // a start orthogonal to the dominant direction (or a power that
    // underflowed) keeps the start; the steps below then converge from it
    if (n > 0.0 && isfinite(n)) xi = yi * vd_rsqrt64(n);
  }
  double prev_diff = 1e300;
  for (int it = 0; it < 300; ++it) {
    double yi = 0.0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const double xm = __shfl_sync(0xffffffffu, xi, m);
      if (tid < 9) yi = fma(sI[9 * m + tid], xm, yi);   // inverse is symmetric
    }
    double n = yi * yi, dot = yi * xi;
    for (int o = 16; o > 0; o >>= 1) {
      n += __shfl_xor_sync(0xffffffffu, n, o);
      dot += __shfl_xor_sync(0xffffffffu, dot, o);
    }
    yi *= vd_rsqrt64(n);
    const double sg = dot < 0.0 ? -1.0 : 1.0;
    double diff = fabs(sg * yi - xi);
    for (int o = 16; o > 0; o >>= 1) diff = fmax(diff, __shfl_xor_sync(0xffffffffu, diff, o));
    xi = sg * yi;
    // converged: a change at rounding level, or a change that stopped
    // shrinking (rounding noise of an already converged iterate)
    if (diff < 4e-15 || (diff < 1e-12 && diff >= 0.5 * prev_diff)) break;
    prev_diff = diff;
  }
  if (tid < 9) Eio[tid] = xi;
}

// E = U diag(s) V^T with det U = det V = +1: the two rotations U W V^T and
// U W^T V^T with translation +-U[:, 2] give the four candidate motions.
__global__ void k_ep_decompose(const double* __restrict__ Ein, double* __restrict__ cand,
                               int* __restrict__ counts) {
  if (threadIdx.x != 0) return;
  double E[9];
  for (int i = 0; i < 9; ++i) E[i] = Ein[i];
  double A[9], w[3], V[9];
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q)
      A[3 * p + q] = E[p] * E[q] + E[3 + p] * E[3 + q] + E[6 + p] * E[6 + q];   // E^T E
  vd_jacobi_eig<3>(A, w, V);
  // order the eigenvalues descending
  int o[3] = {0, 1, 2};
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (w[o[b]] > w[o[a]]) {
        const int tmp = o[a];
        o[a] = o[b];
        o[b] = tmp;
      }
  double v[3][3];
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < 3; ++i) v[c][i] = V[3 * i + o[c]];
  double cr[3];
  vd_cross3(v[0], v[1], cr);
  if (cr[0] * v[2][0] + cr[1] * v[2][1] + cr[2] * v[2][2] < 0.0)
    for (int i = 0; i < 3; ++i) v[2][i] = -v[2][i];
  double U[3][3];
  for (int c = 0; c < 2; ++c) {
    for (int i = 0; i < 3; ++i) U[c][i] = E[3 * i] * v[c][0] + E[3 * i + 1] * v[c][1] + E[3 * i + 2] * v[c][2];
    vd_normalize3(U[c]);
  }
  vd_cross3(U[0], U[1], U[2]);
  // R = U W V^T with W = [[0,-1,0],[1,0,0],[0,0,1]]: R = u2 v1^T - u1 v2^T + u3 v3^T
  for (int s = 0; s < 2; ++s) {
    double R[9];
    const double sg = s == 0 ? 1.0 : -1.0;   // W or W^T
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k)
        R[3 * i + k] = sg * (U[1][i] * v[0][k] - U[0][i] * v[1][k]) + U[2][i] * v[2][k];
    for (int sgn = 0; sgn < 2; ++sgn) {
      double* T = cand + 12 * (2 * s + sgn);
      for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) T[4 * i + k] = R[3 * i + k];
        T[4 * i + 3] = (sgn == 0 ? 1.0 : -1.0) * U[2][i];
      }
    }
  }
  for (int i = 0; i < 4; ++i) counts[i] = 0;
}

// Pixels whose least-squares triangulation lam_b b = lam_a R a + t has both
// depths positive, for each of the four candidate motions.  A vote: taken
// in float32 (a pixel within rounding of a zero depth may count on either
// side; the winner is ahead by thousands of pixels), with the signs of the
// depths read from their numerators and the common determinant (no
// division).
__global__ void __launch_bounds__(EP_THREADS)
k_ep_cheirality(DevParams P, const float2* __restrict__ flow, const double* __restrict__ cand,
                int* __restrict__ counts) {
  __shared__ float sC[48];
  if (threadIdx.x < 48) sC[threadIdx.x] = (float)cand[threadIdx.x];
  __syncthreads();
  int cnt[4] = {0, 0, 0, 0};
  const size_t npix = (size_t)P.W * P.H;
  const float ifx = P.kdf[8], ify = P.kdf[10];
  for (size_t j = (size_t)blockIdx.x * EP_THREADS + threadIdx.x; j < npix;
       j += (size_t)gridDim.x * EP_THREADS) {
    const int v = (int)(j / P.W), u = (int)(j - (size_t)v * P.W);
    const float2 F = flow[j];
    const float a[3] = {((float)u - P.cx) * ifx, ((float)v - P.cy) * ify, 1.0f};
    const float b[3] = {((float)u + F.x - P.cx) * ifx, ((float)v + F.y - P.cy) * ify, 1.0f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float* T = sC + 12 * k;
      const float Ra[3] = {T[0] * a[0] + T[1] * a[1] + T[2] * a[2],
                           T[4] * a[0] + T[5] * a[1] + T[6] * a[2],
                           T[8] * a[0] + T[9] * a[1] + T[10] * a[2]};
      const float t[3] = {T[3], T[7], T[11]};
      const float m11 = Ra[0] * Ra[0] + Ra[1] * Ra[1] + Ra[2] * Ra[2];
      const float m12 = -(Ra[0] * b[0] + Ra[1] * b[1] + Ra[2] * b[2]);
      const float m22 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
      const float r1 = -(Ra[0] * t[0] + Ra[1] * t[1] + Ra[2] * t[2]);
      const float r2 = b[0] * t[0] + b[1] * t[1] + b[2] * t[2];
      const float det = m11 * m22 - m12 * m12;
      const float na = m22 * r1 - m12 * r2, nb = m11 * r2 - m12 * r1;
      const bool pos = det > 0.0f ? (na > 0.0f && nb > 0.0f)
                                  : (det < 0.0f && na < 0.0f && nb < 0.0f);
      cnt[k] += pos ? 1 : 0;
    }
  }
  for (int k = 0; k < 4; ++k) {
    int x = cnt[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(counts + k, x);
  }
}

// Keep the motion with most positive depths (first on ties), |tau_1| = 1,
// and constant-velocity guesses G_t = G_1 o G_{t-1}.
__global__ void k_ep_finalize(DevParams P, const double* __restrict__ cand,
                              const int* __restrict__ counts, double* __restrict__ G,
                              float* __restrict__ posef, float2* __restrict__ posed) {
  if (threadIdx.x != 0) return;
  int best = 0;
  for (int k = 1; k < 4; ++k)
    if (counts[k] > counts[best]) best = k;
  double G1[12];
  for (int i = 0; i < 12; ++i) G1[i] = cand[12 * best + i];
  const double n = sqrt(G1[3] * G1[3] + G1[7] * G1[7] + G1[11] * G1[11]);
  G1[3] /= n;
  G1[7] /= n;
  G1[11] /= n;
  double prev[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  for (int i = 0; i < 12; ++i) G[i] = prev[i];
  for (int t = 1; t <= P.N; ++t) {
    double cur[12];
    vd_compose(G1, prev, cur);
    for (int i = 0; i < 12; ++i) {
      G[12 * t + i] = cur[i];
      prev[i] = cur[i];
    }
  }
  for (int t = 0; t <= P.N; ++t) {
    const double* g = G + 12 * t;
    float* o = posef + 12 * t;
    float2* od = posed + 12 * t;
    for (int i = 0; i < 4; ++i) {
      vd_store_pose_entry(o, od, i < 3 ? i : 9, P.fx_d * g[i] + P.cx_d * g[8 + i]);
      vd_store_pose_entry(o, od, i < 3 ? 3 + i : 10, P.fy_d * g[4 + i] + P.cy_d * g[8 + i]);
      vd_store_pose_entry(o, od, i < 3 ? 6 + i : 11, g[8 + i]);
    }
  }
}

cudaError_t launch_eight_point(vd_ctx* c) {
  for (int r = 0; r < VD_IRLS_ITERS; ++r) {
    k_ep_normal<<<c->ep_blocks, EP_THREADS, 0, c->stream>>>(c->dp, c->flow, c->ep_E, r > 0 ? 1 : 0,
                                                            c->ep_partial);
    k_ep_solve<<<1, 512, 0, c->stream>>>(c->ep_partial, c->ep_blocks, c->ep_M, c->ep_E, r > 0);
  }
  k_ep_decompose<<<1, 32, 0, c->stream>>>(c->ep_E, c->ep_cand, c->ep_count);
  k_ep_cheirality<<<c->ep_blocks, EP_THREADS, 0, c->stream>>>(c->dp, c->flow, c->ep_cand,
                                                              c->ep_count);
  k_ep_finalize<<<1, 32, 0, c->stream>>>(c->dp, c->ep_cand, c->ep_count, c->G, c->posef,
                                      c->posed);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// utilities
// ---------------------------------------------------------------------------
__global__ void k_fill(float* __restrict__ p, float v, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

cudaError_t launch_fill(float* p, float v, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

__global__ void k_check_finite(const float* __restrict__ p, size_t n, int* __restrict__ flag) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(p[i])) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const float* p, size_t n, int* flag, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_check_finite<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, flag);
  return cudaGetLastError();
}

__global__ void k_copy_flow(const float* __restrict__ src, long pitch, int W, int H,
                            float2* __restrict__ dst) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (u >= W || v >= H) return;
  const float* s = src + (size_t)v * pitch + 2 * (size_t)u;
  dst[(size_t)v * W + u] = make_float2(s[0], s[1]);
}

cudaError_t launch_copy_flow(vd_ctx* c, int t, const float* src, long pitch) {
  k_copy_flow<<<dim3((c->W + 127) / 128, c->H), 128, 0, c->stream>>>(
      src, pitch, c->W, c->H, c->flow + (size_t)(t - 1) * c->npix);
  return cudaGetLastError();
}

// Prior maps: stereo disparity d -> value d, inverse depth d / (fx b);
// RGB-D depth z -> value and inverse depth 1 / z; holes -> NaN.
__global__ void k_prior_prepare(DevParams P, int kind, const float* __restrict__ raw,
                                const float* __restrict__ conf_in, float* __restrict__ val,
                                float* __restrict__ prho, float* __restrict__ conf) {
  const size_t npix = (size_t)P.W * P.H;
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npix) return;
  const float x = raw[j];
  const bool ok = isfinite(x) && x > 0.0f;
  float r = nanf("");
  float v = nanf("");
  if (ok) {
    if (kind == VD_PRIOR_STEREO) {
      r = __fdiv_rn(x, P.fxb);
      v = x;
    } else {
      r = __fdiv_rn(1.0f, x);
      v = r;
    }
  }
  val[j] = v;
  prho[j] = r;
  conf[j] = conf_in ? conf_in[j] : 1.0f;
}

cudaError_t launch_prior_prepare(vd_ctx* c, const float* raw, const float* conf) {
  k_prior_prepare<<<(unsigned)((c->npix + 255) / 256), 256, 0, c->stream>>>(
      c->dp, c->prior_kind, raw, conf, c->prior_val, c->prior_rho, c->prior_conf);
  return cudaGetLastError();
}

// Mean energy (of e_star after propagation is not kept; the energy of the new
// depth map is recomputed by the caller into e_mid) and mean rigidness.
__global__ void k_stats(const float* __restrict__ e, size_t npix, const float* __restrict__ q,
                        size_t nq, double* __restrict__ partial) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < nq; i += (size_t)gridDim.x * 256) {
    if (i < npix) a += (double)e[i];
    b += (double)q[i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0[0];
    partial[2 * blockIdx.x + 1] = s1[0];
  }
}

__global__ void k_stats_final(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  out[0] = a;
  out[1] = b;
}

cudaError_t launch_stats(vd_ctx* c, double* out2) {
  cudaError_t e = launch_eval_energy(c, c->rho, c->e_mid);
  if (e != cudaSuccess) return e;
  k_stats<<<c->stat_blocks, 256, 0, c->stream>>>(c->e_mid, c->npix, c->q, c->npix * c->N,
                                                 c->stat_partial);
  k_stats_final<<<1, 32, 0, c->stream>>>(c->stat_partial, c->stat_blocks, out2);
  return cudaGetLastError();
}

VD_CHECK_ACCESSOR(boot)
