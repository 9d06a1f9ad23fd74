// Pose covariance from the P3P samples (Sec. III-A "Uncertainty-aware Pose
// Estimation"): an iterative Gaussian fit in se(3) with 3-sigma rejection and
// an eigenvalue floor, one warp per frame, float64.
//
// Lane l owns samples l, l + 32, ... (at most 8 with 256 samples), staged in
// shared memory.  Every sum
// over samples is a per-lane sum followed by an xor butterfly, so all lanes
// hold bit-identical totals and take the same decisions without a barrier;
// the small 6x6 algebra (the eigen-decomposition of the fit) is repeated by
// every lane on identical inputs.
#include "vd_device.cuh"
#include "vd_geom64.cuh"

#define PC_MAX_ROUNDS 50
#define PC_MEAN_ITERS 50
#define PC_MEAN_TOL 1e-12
#define PC_MIN_INLIERS 7
#define PC_PER_LANE (VD_MAX_SAMPLES / 32)

__device__ __forceinline__ double pc_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// d = log(mu^-1 T) for the 12 doubles of T
__device__ __forceinline__ void pc_coords(const double* mu_inv, const double* T, double* d) {
  double rel[12];
  vd_compose(mu_inv, T, rel);
  vd_se3_log(rel, d);
}

// Cholesky factor of a 6x6 symmetric matrix (A = L L^T, L lower, row-major);
// false when a pivot is not positive (A not positive definite).
__device__ bool pc_chol(const double* A, double* L) {
  for (int i = 0; i < 36; ++i) L[i] = 0.0;
  for (int j = 0; j < 6; ++j) {
    double d = A[7 * j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    L[7 * j] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double v = A[6 * i + j];
      for (int k = 0; k < j; ++k) v -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = v / ljj;
    }
  }
  return true;
}

// A^-1 = L^-T L^-1 from the Cholesky factor
__device__ void pc_chol_inv(const double* L, double* Ai) {
  double M[36];   // M = L^-1 (lower)
  for (int i = 0; i < 36; ++i) M[i] = 0.0;
  for (int c = 0; c < 6; ++c) {
    M[7 * c] = 1.0 / L[7 * c];
    for (int i = c + 1; i < 6; ++i) {
      double v = 0.0;
      for (int k = c; k < i; ++k) v -= L[6 * i + k] * M[6 * k + c];
      M[6 * i + c] = v / L[7 * i];
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) {
      double v = 0.0;
      for (int k = j; k < 6; ++k) v += M[6 * k + i] * M[6 * k + j];
      Ai[6 * i + j] = v;
      Ai[6 * j + i] = v;
    }
}

// S <- V diag(max(w, eps)) V^T and Sinv <- S^-1.  When S - eps I has a
// Cholesky factor every eigenvalue is already above eps and S stays as it
// is (the inverse from S's own factor); otherwise the eigen-decomposition
// raises the small eigenvalues.
__device__ void pc_floor(double* S, double* Sinv, double eps) {
  {
    double B[36], L[36];
    for (int i = 0; i < 36; ++i) B[i] = S[i];
    for (int i = 0; i < 6; ++i) B[7 * i] -= eps;
    if (pc_chol(B, L) && pc_chol(S, L)) {
      pc_chol_inv(L, Sinv);
      return;
    }
  }
  double A[36], w[6], V[36];
  for (int i = 0; i < 36; ++i) A[i] = S[i];
  vd_jacobi_eig<6>(A, w, V);
  for (int k = 0; k < 6; ++k) w[k] = fmax(w[k], eps);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0, si = 0.0;
      for (int k = 0; k < 6; ++k) {
        s += V[6 * i + k] * w[k] * V[6 * j + k];
        si += V[6 * i + k] / w[k] * V[6 * j + k];
      }
      S[6 * i + j] = s;
      Sinv[6 * i + j] = si;
    }
}

// out[52 t']: mean (12), cov (36), n_samples, n_inliers, rounds, degenerate
__global__ void __launch_bounds__(32)
k_pose_cov(DevParams P, const double* __restrict__ G, const double* __restrict__ sample_pose,
           const double* __restrict__ sample_energy, double eps, double* __restrict__ out) {
  const int t = blockIdx.x + 1;
  const int lane = threadIdx.x;
  const double* Ts = sample_pose + (size_t)(t - 1) * VD_MAX_SAMPLES * 12;
  const double* Es = sample_energy + (size_t)(t - 1) * VD_MAX_SAMPLES;
  __shared__ double T[VD_MAX_SAMPLES][12];   // sample g = lane + 32 k at row g
  unsigned valid = 0;
  int nv = 0;
  for (int k = 0; k < PC_PER_LANE; ++k) {
    const int g = lane + 32 * k;
    const bool ok = g < P.S && Es[g] < INFINITY;
    for (int i = 0; i < 12; ++i) T[g][i] = ok ? Ts[12 * g + i] : 0.0;
    valid |= (unsigned)ok << k;
    nv += ok;
  }
  const int n_samples = (int)pc_warp_sum((double)nv);
  double mu[12], S[36], Sinv[36];
  for (int i = 0; i < 12; ++i) mu[i] = G[12 * t + i];
  for (int i = 0; i < 36; ++i) S[i] = 0.0;
  int rounds = 0, n_in = n_samples, degenerate = n_samples < PC_MIN_INLIERS;
  if (!degenerate) {
    // robust start: diag((1.4826 median_g |d_gi|)^2) at the mode, the
    // medians selected by rank among the valid samples (exact, no arithmetic)
    __shared__ double sA[VD_MAX_SAMPLES][6];   // |d| of every sample at the mode
    __shared__ unsigned char sV[VD_MAX_SAMPLES];
    double mi[12];
    vd_inverse(mu, mi);
    for (int k = 0; k < PC_PER_LANE; ++k) {
      const int g = lane + 32 * k;
      double d[6] = {0, 0, 0, 0, 0, 0};
      if (valid >> k & 1u) pc_coords(mi, T[g], d);
      for (int i = 0; i < 6; ++i) sA[g][i] = fabs(d[i]);
      sV[g] = (unsigned char)(valid >> k & 1u);
    }
    __syncwarp();   // every lane's |d| and flags before the ranks
    const int r1 = (n_samples - 1) / 2, r2 = n_samples / 2;   // middle ranks
    for (int i = 0; i < 6; ++i) {
      double m1 = -1.0, m2 = -1.0;
      for (int k = 0; k < PC_PER_LANE; ++k) {
        if (!(valid >> k & 1u)) continue;
        const int g = lane + 32 * k;
        const double a = sA[g][i];
        int rank = 0;   // valid samples before g in (value, index) order
        for (int h = 0; h < P.S; ++h) {
          if (!sV[h]) continue;
          const double b = sA[h][i];
          rank += (b < a) || (b == a && h < g);
        }
        if (rank == r1) m1 = a;
        if (rank == r2) m2 = a;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
      }
      const double s = 1.4826 * ((m1 + m2) / 2.0);
      S[7 * i] = s * s;
    }
  }
  pc_floor(S, Sinv, eps);
  unsigned prev = 0;
  if (!degenerate) {
    for (int r = 1; r <= PC_MAX_ROUNDS; ++r) {
      rounds = r;
      double mi[12];
      vd_inverse(mu, mi);
      unsigned inl = 0;
      int ni = 0;
      for (int k = 0; k < PC_PER_LANE; ++k) {
        if (!(valid >> k & 1u)) continue;
        double d[6];
        pc_coords(mi, T[lane + 32 * k], d);
        double m = 0.0;
        for (int i = 0; i < 6; ++i) {
          double row = 0.0;
          for (int j = 0; j < 6; ++j) row += Sinv[6 * i + j] * d[j];
          m += d[i] * row;
        }
        if (m <= 9.0) {
          inl |= 1u << k;
          ++ni;
        }
      }
      n_in = (int)pc_warp_sum((double)ni);
      if (r > 1 && !__any_sync(0xffffffffu, inl != prev)) break;   // the same inlier set
      if (n_in < PC_MIN_INLIERS) {
        degenerate = 1;
        break;
      }
      // Frechet mean of the inliers
      for (int it = 0; it < PC_MEAN_ITERS; ++it) {
        vd_inverse(mu, mi);
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k < PC_PER_LANE; ++k) {
          if (!(inl >> k & 1u)) continue;
          double d[6];
          pc_coords(mi, T[lane + 32 * k], d);
          for (int i = 0; i < 6; ++i) acc[i] += d[i];
        }
        double step[6], nrm = 0.0;
        for (int i = 0; i < 6; ++i) {
          step[i] = pc_warp_sum(acc[i]) / n_in;
          nrm += step[i] * step[i];
        }
        double E[12], mn[12];
        vd_se3_exp(step, E);
        vd_compose(mu, E, mn);
        for (int i = 0; i < 12; ++i) mu[i] = mn[i];
        if (sqrt(nrm) < PC_MEAN_TOL) break;
      }
      // maximum-likelihood covariance at the mean, eigenvalues floored
      vd_inverse(mu, mi);
      double acc[21];
      for (int i = 0; i < 21; ++i) acc[i] = 0.0;
      for (int k = 0; k < PC_PER_LANE; ++k) {
        if (!(inl >> k & 1u)) continue;
        double d[6];
        pc_coords(mi, T[lane + 32 * k], d);
        for (int i = 0, q = 0; i < 6; ++i)
          for (int j = i; j < 6; ++j, ++q) acc[q] += d[i] * d[j];
      }
      for (int i = 0, q = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++q) {
          const double v = pc_warp_sum(acc[q]) / n_in;
          S[6 * i + j] = v;
          S[6 * j + i] = v;
        }
      pc_floor(S, Sinv, eps);
      prev = inl;
    }
  }
  if (lane == 0) {
    double* o = out + 52 * (t - 1);
    for (int i = 0; i < 12; ++i) o[i] = mu[i];
    for (int i = 0; i < 36; ++i) o[12 + i] = S[i];
    o[48] = n_samples;
    o[49] = n_in;
    o[50] = rounds;
    o[51] = degenerate;
  }
}

extern "C" vd_status vd_pose_covariance(vd_ctx* c, double eps, vd_pose_cov* out) {
  if (!c || !out || !(eps > 0.0) || !isfinite(eps)) return VD_ERR_ARG;
  if (c->samples_set != (1u << c->N) - 1u) {
    vd_set_error("every frame needs a pose M-step first");
    return VD_ERR_STATE;
  }
  k_pose_cov<<<c->N, 32, 0, c->stream>>>(c->dp, c->G, c->sample_pose, c->sample_energy, eps,
                                         c->pc_out);
  VD_CU(cudaGetLastError());
  double h[52 * VD_MAX_FLOWS];
  VD_CU(cudaMemcpyAsync(h, c->pc_out, sizeof(double) * 52 * c->N, cudaMemcpyDeviceToHost,
                        c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  for (int t = 0; t < c->N; ++t) {
    const double* o = h + 52 * t;
    vd_pose_cov& r = out[t];
    for (int i = 0; i < 12; ++i) r.mean[i] = o[i];
    for (int i = 0; i < 36; ++i) r.cov[i] = o[12 + i];
    r.n_samples = (int)o[48];
    r.n_inliers = (int)o[49];
    r.rounds = (int)o[50];
    r.degenerate = (int)o[51];
  }
  return VD_OK;
}

extern "C" vd_status vd_get_frame_samples(vd_ctx* c, int t, double* poses, double* energies) {
  if (!c || t < 1 || t > c->N) return VD_ERR_ARG;
  if (!(c->samples_set >> (t - 1) & 1u)) {
    vd_set_error("frame has no pose M-step yet");
    return VD_ERR_STATE;
  }
  const int S = c->prm.n_pose_samples;
  const size_t f = (size_t)(t - 1) * VD_MAX_SAMPLES;
  if (poses)
    VD_CU(cudaMemcpyAsync(poses, c->sample_pose + 12 * f, sizeof(double) * 12 * S,
                          cudaMemcpyDeviceToHost, c->stream));
  if (energies)
    VD_CU(cudaMemcpyAsync(energies, c->sample_energy + f, sizeof(double) * S,
                          cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

VD_CHECK_ACCESSOR(posecov)
