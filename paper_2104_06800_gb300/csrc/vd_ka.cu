// Keyframe alignment (Sec. III-C "Keyframe Alignment", Eq. 9-12): the
// relative motion T and scale s of two keyframes' depth maps by
// point-to-plane registration in inverse-depth form, with a Cauchy kernel and
// confidence weights, solved by Levenberg-Marquardt; covariance (J^T J)^-1.
//
// The device evaluates, at a given (T, s), the energy and the normal
// equations of every associated pixel of keyframe 2: k_ka_normals computes
// depth map 1's normals once, k_ka_accum sums E, H (upper triangle of 7 x 7)
// and g per block over a fixed pixel range (float64 per pixel, warp
// butterflies and a fixed warp order within the block), k_ka_sum adds the
// blocks in index order.  The host runs the Levenberg-Marquardt schedule on
// the 37 sums of each evaluation.
#include <cmath>
#include <utility>

#include "vd_device.cuh"
#include "vd_geom64.cuh"

#define KA_BLOCK 256
#define KA_NS 37          // E, H (28), g (7), n
#define KA_KINK 0.2       // no normal where a second difference exceeds this of the span
#define KA_GATE 0.2       // a pair counts when the depths agree within this fraction
#define KA_LAMBDA0 1e-3
#define KA_STEP_TOL 1e-10

struct KaCam {
  double fx, fy, cx, cy;
  int W, H;
};

struct __align__(16) KaNormal {   // unit normal and a validity flag w
  double x, y, z, w;
};

__device__ __forceinline__ bool ka_valid(float t) { return isfinite(t) && t > 0.0f; }

__device__ __forceinline__ void ka_point(const KaCam& c, const float* th, int u, int v,
                                         double* P) {
  const double t = (double)th[(size_t)v * c.W + u];
  P[0] = t * (((double)u - c.cx) / c.fx);
  P[1] = t * (((double)v - c.cy) / c.fy);
  P[2] = t;
}

// Normals of depth map 1: central differences of its points, normalised,
// towards the camera; w = 1 where valid (inside the border, the five depths
// valid, a non-zero cross product, no depth edge or fold).
__global__ void __launch_bounds__(KA_BLOCK)
k_ka_normals(const float* __restrict__ theta1, KaCam c, KaNormal* __restrict__ n1) {
  const size_t npix = (size_t)c.W * c.H;
  const size_t j = (size_t)blockIdx.x * KA_BLOCK + threadIdx.x;
  if (j >= npix) return;
  const int v = (int)(j / c.W), u = (int)(j - (size_t)v * c.W);
  KaNormal out = {0.0, 0.0, 0.0, 0.0};
  if (u > 0 && v > 0 && u < c.W - 1 && v < c.H - 1 && ka_valid(theta1[j]) &&
      ka_valid(theta1[j - 1]) && ka_valid(theta1[j + 1]) && ka_valid(theta1[j - c.W]) &&
      ka_valid(theta1[j + c.W])) {
    double P[3], Pl[3], Pr[3], Pu[3], Pd[3];
    ka_point(c, theta1, u, v, P);
    ka_point(c, theta1, u - 1, v, Pl);
    ka_point(c, theta1, u + 1, v, Pr);
    ka_point(c, theta1, u, v - 1, Pu);
    ka_point(c, theta1, u, v + 1, Pd);
    double dx[3], dy[3], ddx[3], ddy[3];
    for (int i = 0; i < 3; ++i) {
      dx[i] = Pr[i] - Pl[i];
      dy[i] = Pd[i] - Pu[i];
      ddx[i] = Pr[i] - 2.0 * P[i] + Pl[i];
      ddy[i] = Pd[i] - 2.0 * P[i] + Pu[i];
    }
    const double n0 = dx[1] * dy[2] - dx[2] * dy[1];
    const double n1_ = dx[2] * dy[0] - dx[0] * dy[2];
    const double n2 = dx[0] * dy[1] - dx[1] * dy[0];
    const double nrm = sqrt(n0 * n0 + n1_ * n1_ + n2 * n2);
    const double lx = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
    const double ly = sqrt(dy[0] * dy[0] + dy[1] * dy[1] + dy[2] * dy[2]);
    const double kx = sqrt(ddx[0] * ddx[0] + ddx[1] * ddx[1] + ddx[2] * ddx[2]);
    const double ky = sqrt(ddy[0] * ddy[0] + ddy[1] * ddy[1] + ddy[2] * ddy[2]);
    if (nrm > 0.0 && kx <= KA_KINK * lx && ky <= KA_KINK * ly) {
      double a = n0 / nrm, b = n1_ / nrm, d = n2 / nrm;
      if (a * P[0] + b * P[1] + d * P[2] > 0.0) {
        a = -a;
        b = -b;
        d = -d;
      }
      out = KaNormal{a, b, d, 1.0};
    }
  }
  n1[j] = out;
}

// Block b sums pixels [b per, (b+1) per) of keyframe 2 into partial[b][37]:
// E, H_ik (i <= k, row by row), g_i, n.  Ts: T (12) at the evaluation.
__global__ void __launch_bounds__(KA_BLOCK)
k_ka_accum(const float* __restrict__ theta1, const KaNormal* __restrict__ n1,
           const float* __restrict__ theta2, const float* __restrict__ conf2, KaCam c,
           const double* __restrict__ Ts, double s, double cc, double* __restrict__ partial) {
  __shared__ double sT[12];
  __shared__ double sW[KA_BLOCK / 32][KA_NS];
  if (threadIdx.x < 12) sT[threadIdx.x] = Ts[threadIdx.x];
  __syncthreads();
  const size_t npix = (size_t)c.W * c.H;
  const size_t per = (npix + gridDim.x - 1) / gridDim.x;
  const size_t beg = min(npix, (size_t)blockIdx.x * per), end = min(npix, beg + per);
  double acc[KA_NS];
#pragma unroll
  for (int i = 0; i < KA_NS; ++i) acc[i] = 0.0;
  for (size_t j = beg + threadIdx.x; j < end; j += KA_BLOCK) {
    const float t2 = theta2[j];
    if (!ka_valid(t2)) continue;
    const int v = (int)(j / c.W), u = (int)(j - (size_t)v * c.W);
    const double X[3] = {(double)t2 * (((double)u - c.cx) / c.fx),
                         (double)t2 * (((double)v - c.cy) / c.fy), (double)t2};
    double P[3];
    for (int i = 0; i < 3; ++i)
      P[i] = X[0] * sT[4 * i] + X[1] * sT[4 * i + 1] + X[2] * sT[4 * i + 2] + sT[4 * i + 3];
    if (!(P[2] > (double)VD_Z_EPS)) continue;
    const double Z = P[2];
    const double x = c.fx * P[0] / Z + c.cx, y = c.fy * P[1] / Z + c.cy;
    if (!(x >= 0.0 && x <= (double)(c.W - 1) && y >= 0.0 && y <= (double)(c.H - 1))) continue;
    const int lu = (int)floor(x + 0.5), lv = (int)floor(y + 0.5);
    const size_t l = (size_t)lv * c.W + lu;
    const KaNormal n = n1[l];
    const float t1 = theta1[l];
    if (!(n.w > 0.0) || !ka_valid(t1)) continue;
    const double D = s * (double)t1;
    if (!(fabs(Z - D) <= KA_GATE * D)) continue;   // occlusion gate
    const double rl[3] = {((double)lu - c.cx) / c.fx, ((double)lv - c.cy) / c.fy, 1.0};
    const double A = n.x * rl[0] + n.y * rl[1] + n.z * rl[2];
    const double B = n.x * P[0] + n.y * P[1] + n.z * P[2];
    const double r = A / Z - B / (D * Z);
    const double C = conf2 ? (double)conf2[j] : 1.0;
    const double q = r / cc;
    const double w = C / (1.0 + q * q);
    acc[0] += C * (0.5 * cc * cc * log1p(q * q));
    // J = d r / d(omega, v, log s)
    double g3[3] = {-n.x / (D * Z), -n.y / (D * Z), -n.z / (D * Z)};
    g3[2] += (B - A * D) / (D * Z * Z);
    const double J[7] = {P[1] * g3[2] - P[2] * g3[1], P[2] * g3[0] - P[0] * g3[2],
                         P[0] * g3[1] - P[1] * g3[0], g3[0], g3[1], g3[2], B / (D * Z)};
    int q2 = 1;
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
      for (int k = i; k < 7; ++k) acc[q2++] += w * J[i] * J[k];
#pragma unroll
    for (int i = 0; i < 7; ++i) acc[29 + i] += w * J[i] * r;
    acc[36] += 1.0;
  }
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KA_NS; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sW[wq][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < KA_NS) {
    double v = 0.0;
    for (int k = 0; k < KA_BLOCK / 32; ++k) v += sW[k][threadIdx.x];
    partial[(size_t)blockIdx.x * KA_NS + threadIdx.x] = v;
  }
}

// Block i adds sum i over the partials: thread t takes blocks t, t + 256, ...
// in order, then a fixed tree over the threads.
__global__ void __launch_bounds__(KA_BLOCK)
k_ka_sum(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  __shared__ double sv[KA_BLOCK];
  const int i = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += KA_BLOCK) v += partial[(size_t)b * KA_NS + i];
  sv[threadIdx.x] = v;
  __syncthreads();
  for (int o = KA_BLOCK / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sv[threadIdx.x] += sv[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = sv[0];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

struct KaEval {
  double E, H[49], g[7];
  long long n;
};

struct KaRun {
  const float *th1, *th2, *conf2;
  KaCam cam;
  double cc;
  cudaStream_t st;
  KaNormal* n1;
  double* partial;
  double* sums;
  double* Tdev;
  int nblk;
};

cudaError_t ka_eval(const KaRun& k, const double* T, double s, KaEval* out) {
  cudaError_t e = cudaMemcpyAsync(k.Tdev, T, sizeof(double) * 12, cudaMemcpyHostToDevice, k.st);
  if (e != cudaSuccess) return e;
  k_ka_accum<<<k.nblk, KA_BLOCK, 0, k.st>>>(k.th1, k.n1, k.th2, k.conf2, k.cam, k.Tdev, s, k.cc,
                                            k.partial);
  k_ka_sum<<<KA_NS, KA_BLOCK, 0, k.st>>>(k.partial, k.nblk, k.sums);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double h[KA_NS];
  e = cudaMemcpyAsync(h, k.sums, sizeof h, cudaMemcpyDeviceToHost, k.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(k.st);
  if (e != cudaSuccess) return e;
  out->E = h[0];
  for (int i = 0, q = 1; i < 7; ++i)
    for (int j = i; j < 7; ++j, ++q) out->H[7 * i + j] = out->H[7 * j + i] = h[q];
  for (int i = 0; i < 7; ++i) out->g[i] = h[29 + i];
  out->n = (long long)h[36];
  return cudaSuccess;
}

// Solve A x = b (m x m, row-major) by Gaussian elimination with partial
// pivoting; false for a singular matrix.
bool ka_solve(int m, const double* Ain, const double* b, double* x) {
  double A[49], y[7];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[m * i + j] = Ain[m * i + j];
    y[i] = b[i];
  }
  for (int c = 0; c < m; ++c) {
    int p = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[m * r + c]) > fabs(A[m * p + c])) p = r;
    if (A[m * p + c] == 0.0) return false;
    if (p != c) {
      for (int j = 0; j < m; ++j) std::swap(A[m * c + j], A[m * p + j]);
      std::swap(y[c], y[p]);
    }
    for (int r = c + 1; r < m; ++r) {
      const double f = A[m * r + c] / A[m * c + c];
      for (int j = c; j < m; ++j) A[m * r + j] -= f * A[m * c + j];
      y[r] -= f * y[c];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    for (int j = i + 1; j < m; ++j) v -= A[m * i + j] * x[j];
    x[i] = v / A[m * i + i];
  }
  return true;
}

}  // namespace

extern "C" vd_status vd_ka_align(const float* depth1, const float* depth2, const float* conf2,
                                 int width, int height, const double* K, vd_ka* io,
                                 void* stream) {
  if (!depth1 || !depth2 || !K || !io || width < 3 || height < 3 || !(K[0] > 0) ||
      !(K[1] > 0) || !std::isfinite(K[2]) || !std::isfinite(K[3]) || !(io->cauchy_c > 0) ||
      io->max_iters < 0 || !(io->s > 0) || !std::isfinite(io->s))
    return VD_ERR_ARG;
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(io->pose[i])) return VD_ERR_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  VD_CU(cudaGetDevice(&dev));
  VD_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  KaRun k;
  k.th1 = depth1;
  k.th2 = depth2;
  k.conf2 = conf2;
  k.cam = KaCam{K[0], K[1], K[2], K[3], width, height};
  k.cc = io->cauchy_c;
  k.st = st;
  k.nblk = 4 * sms;
  const size_t npix = (size_t)width * height;
  void* mem = nullptr;
  const size_t bytes = sizeof(KaNormal) * npix + sizeof(double) * ((size_t)k.nblk * KA_NS + 64);
  VD_CU(cudaMallocAsync(&mem, bytes, st));
  k.n1 = (KaNormal*)mem;
  k.partial = (double*)(k.n1 + npix);
  k.sums = k.partial + (size_t)k.nblk * KA_NS;
  k.Tdev = k.sums + 48;
  vd_status status = VD_OK;
  auto fail = [&](cudaError_t e) {
    vd_set_error(cudaGetErrorString(e));
    status = e == cudaErrorMemoryAllocation ? VD_ERR_OOM : VD_ERR_CUDA;
  };
  const int m = io->fix_scale ? 6 : 7;
  double T[12], s = io->fix_scale ? 1.0 : io->s;
  for (int i = 0; i < 12; ++i) T[i] = io->pose[i];
  KaEval cur, cand;
  int it = 0;
  k_ka_normals<<<(int)((npix + KA_BLOCK - 1) / KA_BLOCK), KA_BLOCK, 0, st>>>(depth1, k.cam, k.n1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = ka_eval(k, T, s, &cur);
  double lam = KA_LAMBDA0;
  while (e == cudaSuccess && it < io->max_iters && lam <= 1e10 && cur.n > 0) {
    ++it;
    double A[49], b[7], delta[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) A[m * i + j] = cur.H[7 * i + j];
      A[m * i + i] += lam * cur.H[7 * i + i];
      b[i] = -cur.g[i];
    }
    if (!ka_solve(m, A, b, delta)) {
      lam *= 10.0;
      continue;
    }
    double E6[12], Tn[12];
    vd_se3_exp(delta, E6);
    vd_compose(E6, T, Tn);
    const double sn = io->fix_scale ? s : s * exp(delta[6]);
    if ((e = ka_eval(k, Tn, sn, &cand)) != cudaSuccess) break;
    if (cand.n > 0 && cand.E < cur.E) {
      for (int i = 0; i < 12; ++i) T[i] = Tn[i];
      s = sn;
      cur = cand;
      lam /= 10.0;
    } else {
      lam *= 10.0;
    }
    double dn = 0.0;
    for (int i = 0; i < m; ++i) dn += delta[i] * delta[i];
    if (sqrt(dn) < KA_STEP_TOL) break;
  }
  if (e != cudaSuccess) fail(e);
  cudaFreeAsync(mem, st);
  if (status != VD_OK) return status;
  // covariance: the pose block of H^-1 (columns of the inverse by solves)
  for (int i = 0; i < 36; ++i) io->cov[i] = NAN;
  if (cur.n > 0) {
    double Hm[49];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Hm[m * i + j] = cur.H[7 * i + j];
    for (int c = 0; c < 6; ++c) {
      double ec[7] = {0, 0, 0, 0, 0, 0, 0}, col[7];
      ec[c] = 1.0;
      if (!ka_solve(m, Hm, ec, col)) break;
      for (int r = 0; r < 6; ++r) io->cov[6 * r + c] = col[r];
    }
  }
  for (int i = 0; i < 12; ++i) io->pose[i] = T[i];
  io->s = s;
  io->energy = cur.E;
  io->iterations = it;
  io->n_valid = cur.n;
  return VD_OK;
}

VD_CHECK_ACCESSOR(ka)
