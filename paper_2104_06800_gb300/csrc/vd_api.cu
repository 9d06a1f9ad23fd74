// Host runtime of the library: context lifecycle, input upload, the EM
// schedule of VOLDOR+ (Sec. III-A) and result download.  Every function is
// a C-ABI entry point declared in voldor_em.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "vd_internal.h"

static thread_local char g_err[512] = "";

void vd_set_error(const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg ? msg : "");
}

extern "C" const char* vd_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// stage profiling: one event pair per recorded stage execution
// ---------------------------------------------------------------------------
struct ProfRec {
  int stage;
  cudaEvent_t a, b;
};
struct ProfState {
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  long long calls[VD_N_STAGES] = {};
  int open_stage = -1;
  cudaEvent_t open_ev = nullptr;
};

static cudaEvent_t prof_event(ProfState* ps) {
  if (ps->used == ps->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ps->pool.push_back(e);
  }
  return ps->pool[ps->used++];
}

void vd_prof_begin(vd_ctx* c, int stage) {
  if (!c->prof_on) return;
  ProfState* ps = (ProfState*)c->prof;
  cudaEvent_t e = prof_event(ps);
  if (!e) return;
  cudaEventRecord(e, c->stream);
  ps->open_stage = stage;
  ps->open_ev = e;
}

void vd_prof_end(vd_ctx* c, int stage, int n_launch) {
  c->launches[stage] += n_launch;
  if (!c->prof_on) return;
  ProfState* ps = (ProfState*)c->prof;
  if (ps->open_stage != stage || !ps->open_ev) return;
  cudaEvent_t e = prof_event(ps);
  if (!e) return;
  cudaEventRecord(e, c->stream);
  ps->recs.push_back({stage, ps->open_ev, e});
  ps->calls[stage] += 1;
  ps->open_stage = -1;
  ps->open_ev = nullptr;
}

static void prof_free(vd_ctx* c) {
  ProfState* ps = (ProfState*)c->prof;
  if (!ps) return;
  for (cudaEvent_t e : ps->pool) cudaEventDestroy(e);
  delete ps;
  c->prof = nullptr;
}

extern "C" vd_status vd_profile_enable(vd_ctx* c, int enable) {
  if (!c) return VD_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return VD_ERR_CUDA;
  if (!c->prof) c->prof = new ProfState();
  ProfState* ps = (ProfState*)c->prof;
  ps->recs.clear();
  ps->used = 0;
  for (int i = 0; i < VD_N_STAGES; ++i) {
    ps->calls[i] = 0;
    c->launches[i] = 0;
  }
  ps->open_stage = -1;
  c->prof_on = enable ? 1 : 0;
  if (cudaMemsetAsync(c->score_work, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
    return VD_ERR_CUDA;
  return VD_OK;
}

extern "C" vd_status vd_get_profile(vd_ctx* c, vd_profile* out) {
  if (!c || !out) return VD_ERR_ARG;
  memset(out, 0, sizeof *out);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  ProfState* ps = (ProfState*)c->prof;
  if (ps) {
    for (const ProfRec& r : ps->recs) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) out->ms[r.stage] += ms;
    }
    for (int i = 0; i < VD_N_STAGES; ++i) out->calls[i] = ps->calls[i];
  }
  for (int i = 0; i < VD_N_STAGES; ++i) {
    out->launches[i] = c->launches[i];
    out->total_launches += c->launches[i];
  }
  unsigned long long w = 0;
  e = cudaMemcpy(&w, c->score_work, sizeof w, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  out->score_evals = (long long)w;
  return VD_OK;
}

extern "C" const char* vd_status_str(vd_status s) {
  switch (s) {
    case VD_OK: return "ok";
    case VD_WARN_DEGENERATE: return "degenerate pose step (pose kept)";
    case VD_ERR_ARG: return "invalid argument";
    case VD_ERR_CUDA: return "CUDA error";
    case VD_ERR_OOM: return "out of device memory";
    case VD_ERR_STATE: return "call out of order";
    case VD_ERR_TIMEOUT: return "device wait timed out";
    case VD_ERR_NUMERIC: return "non-finite value in state";
  }
  return "unknown status";
}

extern "C" vd_status vd_params_default(vd_params* p) {
  if (!p) return VD_ERR_ARG;
  memset(p, 0, sizeof *p);
  p->fisk_alpha0 = 0.5f;
  p->fisk_alpha1 = 0.0f;
  p->fisk_beta = 2.0f;
  p->outlier_density = 1e-3f;
  p->gamma_stay = 0.95f;
  p->rho_min = 0.01f;
  p->rho_max = 1.0f;
  p->n_hyp = 64;
  p->n_pose_samples = 64;
  p->pose_sigma_rot = 0.01;
  p->pose_sigma_trans_rel = 0.01;
  p->pose_sigma_trans_abs = 1e-3;
  p->sample_share = 1;
  p->hierarchical = 0;
  p->hier_scale = 4;
  p->hier_window = 32;
  p->prior_c_sigma = 0.01f;
  p->prior_w_uniform = 2.0f;
  p->seed = 0;
  return VD_OK;
}

static bool params_ok(const vd_params* p) {
  return p->fisk_alpha0 > 0.0f && p->fisk_alpha1 >= 0.0f && p->fisk_beta > 0.0f &&
         p->fisk_beta <= 8.0f && p->outlier_density > 0.0f && p->gamma_stay >= 0.5f &&
         p->gamma_stay < 1.0f && p->rho_min > 0.0f && p->rho_max > p->rho_min &&
         isfinite(p->rho_max) && p->n_hyp >= 1 && p->n_hyp <= 1024 && p->n_pose_samples >= 1 &&
         p->n_pose_samples <= VD_MAX_SAMPLES && p->pose_sigma_rot > 0.0 &&
         p->pose_sigma_trans_rel >= 0.0 && p->pose_sigma_trans_abs > 0.0 &&
         p->sample_share >= 1 && p->sample_share <= 4096 && p->hier_scale >= 1 &&
         p->hier_window >= 1 && p->prior_c_sigma > 0.0f && p->prior_w_uniform > 0.0f;
}

static void fill_devparams(vd_ctx* c) {
  ++c->cfg_version;
  DevParams& d = c->dp;
  const vd_params& p = c->prm;
  d.W = c->W;
  d.H = c->H;
  d.N = c->N;
  d.K = p.n_hyp;
  d.S = p.n_pose_samples;
  d.fx_d = c->desc.fx;
  d.fy_d = c->desc.fy;
  d.cx_d = c->desc.cx;
  d.cy_d = c->desc.cy;
  d.fx = (float)c->desc.fx;
  d.fy = (float)c->desc.fy;
  d.cx = (float)c->desc.cx;
  d.cy = (float)c->desc.cy;
  d.alpha0 = p.fisk_alpha0;
  d.alpha1 = p.fisk_alpha1;
  d.beta = p.fisk_beta;
  d.p0 = p.outlier_density;
  d.fast_beta2 = (p.fisk_beta == 2.0f && p.fisk_alpha1 == 0.0f) ? 1 : 0;
  d.c0 = (float)((double)p.outlier_density * M_PI * (double)p.fisk_alpha0 * p.fisk_alpha0);
  d.log2c0 = (float)log2((double)p.outlier_density * M_PI * (double)p.fisk_alpha0 * p.fisk_alpha0);
  d.inv_a2 = (float)(1.0 / ((double)p.fisk_alpha0 * p.fisk_alpha0));
  d.cgen = (float)((double)p.outlier_density * 2.0 * M_PI / p.fisk_beta);
  d.gamma = p.gamma_stay;
  d.rho_min = p.rho_min;
  d.rho_max = p.rho_max;
  d.share = p.sample_share;
  d.key0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
  d.key1 = (uint32_t)(p.seed >> 32);
  d.prior_kind = c->prior_kind;
  d.fxb = c->fxb;
  d.c_sigma = p.prior_c_sigma;
  d.w_unif = p.prior_w_uniform;
  d.logk = (float)log(sqrt(2.0 * M_PI) * p.prior_c_sigma / p.prior_w_uniform);
  d.ms_sig_rot = p.pose_sigma_rot;
  d.ms_sig_rel = p.pose_sigma_trans_rel;
  d.ms_sig_abs = p.pose_sigma_trans_abs;
  const double kv[6] = {c->desc.fx, c->desc.fy, c->desc.cx, c->desc.cy, 1.0 / c->desc.fx,
                        1.0 / c->desc.fy};
  for (int i = 0; i < 6; ++i) {
    d.kdf[2 * i] = (float)kv[i];
    d.kdf[2 * i + 1] = (float)(kv[i] - (double)d.kdf[2 * i]);
  }
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

extern "C" vd_status vd_destroy(vd_ctx* c) {
  if (!c) return VD_ERR_ARG;
  if (c->batch_owned) {
    vd_set_error("a batch window is destroyed with its batch");
    return VD_ERR_STATE;
  }
  void* ptrs[] = {c->flow, c->prior_val, c->prior_rho, c->prior_conf, c->rho, c->q, c->qhat,
                  c->conf, c->G, c->G_init, c->posef, c->posed, c->rho_star, c->e_star, c->rho_mid, c->e_mid,
                  c->coarse, c->lam, c->flags, c->blk_counts, c->n_rigid,
                  c->rigid_idx, c->rpts, c->robs, c->roots, c->root_count, c->rootsf, c->rootsr, c->partial,
                  c->root_energy, c->score_work, c->sample_pose, c->sample_energy, c->degenerate, c->ep_partial,
                  c->ep_M, c->ep_E, c->ep_cand, c->ep_count, c->stat_partial, c->stat_out,
                  c->vc_cover, c->vc_counts, c->vc_pose, c->pc_out};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  prof_free(c);
  delete c;
  return VD_OK;
}

extern "C" vd_status vd_create(const vd_window_desc* desc, const vd_params* params, void* stream,
                               vd_ctx** out) {
  if (!desc || !out) return VD_ERR_ARG;
  *out = nullptr;
  vd_params p;
  if (params) p = *params;
  else vd_params_default(&p);
  if (desc->width < 2 || desc->height < 2 || desc->width > 16384 || desc->height > 16384 ||
      desc->n_flows < 1 || desc->n_flows > VD_MAX_FLOWS || !(desc->fx > 0) || !(desc->fy > 0) ||
      !isfinite(desc->cx) || !isfinite(desc->cy) || !params_ok(&p))
    return VD_ERR_ARG;
  vd_ctx* c = new vd_ctx();
  memset((void*)c, 0, sizeof *c);
  c->desc = *desc;
  c->prm = p;
  c->stream = (cudaStream_t)stream;
  c->W = desc->width;
  c->H = desc->height;
  c->N = desc->n_flows;
  c->npix = (size_t)c->W * c->H;
  c->prior_kind = VD_PRIOR_NONE;
  fill_devparams(c);
  const size_t np = c->npix, N = c->N;
  const int S = VD_MAX_SAMPLES;
  c->nblk_scan = (int)((np + 255) / 256);
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0 || vd_pose_prepare() != cudaSuccess) {
      vd_set_error("cannot query the device");
      delete c;
      return VD_ERR_CUDA;
    }
    c->num_sms = sms;
  }
  c->k1_warps = 4;
  c->score_bps = 2;
  c->score_threads = 256;
  c->nblk_score = VD_SCORE_BPS_MAX * c->num_sms;   // capacity of the partial sums
  c->ep_blocks = 2 * c->num_sms;
  c->stat_blocks = c->num_sms;
  const int s = p.hier_scale;
  cudaError_t e = cudaSuccess;
#define A(ptr, n) if (e == cudaSuccess) e = dalloc(&c->ptr, (n))
  A(flow, N * np);
  A(prior_val, np);
  A(prior_rho, np);
  A(prior_conf, np);
  A(rho, np);
  A(q, N * np);
  A(qhat, np);
  A(conf, np);
  A(G, 12 * (N + 1));
  A(G_init, 12 * (N + 1));
  A(posef, 12 * (N + 1));
  A(posed, 12 * (N + 1));
  A(rho_star, np);
  A(e_star, np);
  A(rho_mid, np);
  A(e_mid, np);
  A(coarse, np + c->W + c->H + 1);
  A(lam, N * np);
  A(flags, np);
  A(blk_counts, c->nblk_scan);
  A(n_rigid, 1);
  A(rigid_idx, np);
  A(rpts, np);
  A(robs, np);
  A(roots, (size_t)S * 48);
  A(root_count, S);
  A(rootsf, (size_t)4 * S * 12);
  A(rootsr, (size_t)4 * S * 12);
  A(partial, (size_t)4 * S * c->nblk_score);
  A(root_energy, 4 * S);
  A(score_work, 1);
  A(sample_pose, 12 * S * N);
  A(sample_energy, S * N);
  A(pc_out, 52 * N);
  A(degenerate, 1);
  A(ep_partial, (size_t)45 * c->ep_blocks);
  A(ep_M, 45);
  A(ep_E, 9);
  A(ep_cand, 48);
  A(ep_count, 4);
  A(stat_partial, 2 * c->stat_blocks);
  A(stat_out, 2);
  c->vc_stride = (np + 15) / 16 * 16;
  A(vc_cover, (N + 1) * c->vc_stride);
  A(vc_counts, 1 + 2 * (N + 1));
  A(vc_pose, 12);
#undef A
  (void)s;
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    vd_destroy(c);
    return e == cudaErrorMemoryAllocation ? VD_ERR_OOM : VD_ERR_CUDA;
  }
  // identity poses, unit rigidness, no prior
  std::vector<double> G(12 * (N + 1), 0.0);
  for (size_t t = 0; t <= N; ++t) G[12 * t] = G[12 * t + 5] = G[12 * t + 10] = 1.0;
  e = cudaMemcpyAsync(c->G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->G_init, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess) e = launch_fill(c->q, 1.0f, N * np, c->stream);
  if (e == cudaSuccess) e = launch_fill(c->qhat, 1.0f, np, c->stream);
  if (e == cudaSuccess) e = launch_fill(c->prior_conf, 1.0f, np, c->stream);
  if (e == cudaSuccess) e = launch_fill(c->prior_val, nanf(""), np, c->stream);
  if (e == cudaSuccess) e = launch_fill(c->prior_rho, nanf(""), np, c->stream);
  if (e == cudaSuccess) e = launch_fill(c->conf, 0.0f, np, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->degenerate, 0, sizeof(int), c->stream);

  if (e == cudaSuccess) e = cudaMemsetAsync(c->score_work, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = launch_posef(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    vd_destroy(c);
    return VD_ERR_CUDA;
  }
  *out = c;
  return VD_OK;
}

extern "C" vd_status vd_set_stream(vd_ctx* c, void* stream) {
  if (!c) return VD_ERR_ARG;
  if (c->batch_owned) {
    vd_set_error("the stream of a batch window belongs to the batch");
    return VD_ERR_STATE;
  }
  c->stream = (cudaStream_t)stream;
  return VD_OK;
}

extern "C" vd_status vd_set_params(vd_ctx* c, const vd_params* p) {
  if (!c || !p || !params_ok(p)) return VD_ERR_ARG;
  c->prm = *p;
  fill_devparams(c);
  return VD_OK;
}

// Copy a caller buffer of n floats into device memory `dst` on the ctx stream.
static cudaError_t upload(vd_ctx* c, float* dst, const float* src, size_t n, vd_mem mem) {
  return cudaMemcpyAsync(dst, src, sizeof(float) * n,
                         mem == VD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                         c->stream);
}

static cudaError_t download(vd_ctx* c, float* dst, const float* src, size_t n, vd_mem mem) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(float) * n,
                                  mem == VD_MEM_HOST ? cudaMemcpyDeviceToHost
                                                     : cudaMemcpyDeviceToDevice,
                                  c->stream);
  if (e == cudaSuccess && mem == VD_MEM_HOST) e = cudaStreamSynchronize(c->stream);
  return e;
}

extern "C" vd_status vd_push_flow(vd_ctx* c, int t, const float* uv, long pitch, vd_mem mem) {
  if (!c || !uv || t < 1 || t > c->N || pitch < 2L * c->W) return VD_ERR_ARG;
  float2* dst = c->flow + (size_t)(t - 1) * c->npix;
  if (mem == VD_MEM_HOST) {
    VD_CU(cudaMemcpy2DAsync(dst, sizeof(float2) * c->W, uv, sizeof(float) * pitch,
                            sizeof(float2) * c->W, c->H, cudaMemcpyHostToDevice, c->stream));
  } else {
    VD_CU(launch_copy_flow(c, t, uv, pitch));
  }
  // reject non-finite flow (uses the degenerate counter slot as a scratch flag)
  int* flag = c->n_rigid;
  VD_CU(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  VD_CU(launch_check_finite((const float*)dst, 2 * c->npix, flag, c->stream));
  int h = 0;
  VD_CU(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  if (h) {
    c->flow_pushed &= ~(1u << (t - 1));
    vd_set_error("flow contains NaN or Inf");
    return VD_ERR_ARG;
  }
  c->flow_pushed |= 1u << (t - 1);
  c->bootstrapped = 0;
  c->iter = 0;
  return VD_OK;
}

static vd_status push_prior(vd_ctx* c, int kind, const float* raw, const float* conf, vd_mem mem) {
  // stage raw (and conf) in e_mid / rho_mid, then convert
  VD_CU(upload(c, c->e_mid, raw, c->npix, mem));
  if (conf) VD_CU(upload(c, c->rho_mid, conf, c->npix, mem));
  c->prior_kind = kind;
  fill_devparams(c);
  VD_CU(launch_prior_prepare(c, c->e_mid, conf ? c->rho_mid : nullptr));
  VD_CU(cudaStreamSynchronize(c->stream));
  c->bootstrapped = 0;
  c->iter = 0;
  return VD_OK;
}

extern "C" vd_status vd_push_stereo_prior(vd_ctx* c, const float* disp, double baseline, vd_mem mem) {
  if (!c || !disp || !(baseline > 0.0) || !isfinite(baseline)) return VD_ERR_ARG;
  c->fxb = (float)(c->desc.fx * baseline);
  return push_prior(c, VD_PRIOR_STEREO, disp, nullptr, mem);
}

extern "C" vd_status vd_push_depth_prior(vd_ctx* c, const float* depth, const float* conf,
                                         const double* T_hat, vd_mem mem) {
  if (!c || !depth) return VD_ERR_ARG;
  if (T_hat) {
    static const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    for (int i = 0; i < 12; ++i)
      if (T_hat[i] != I[i]) {
        vd_set_error("depth prior: only the identity T_hat (reference-frame grid) is supported");
        return VD_ERR_ARG;
      }
  }
  return push_prior(c, VD_PRIOR_RGBD, depth, conf, mem);
}

extern "C" vd_status vd_clear_prior(vd_ctx* c) {
  if (!c) return VD_ERR_ARG;
  c->prior_kind = VD_PRIOR_NONE;
  fill_devparams(c);
  VD_CU(launch_fill(c->prior_val, nanf(""), c->npix, c->stream));
  VD_CU(launch_fill(c->prior_rho, nanf(""), c->npix, c->stream));
  VD_CU(launch_fill(c->prior_conf, 1.0f, c->npix, c->stream));
  c->bootstrapped = 0;
  return VD_OK;
}

static void compose12(const double* A, const double* B, double* O) {
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k)
      O[4 * r + k] = A[4 * r] * B[k] + A[4 * r + 1] * B[4 + k] + A[4 * r + 2] * B[8 + k];
    O[4 * r + 3] = A[4 * r] * B[3] + A[4 * r + 1] * B[7] + A[4 * r + 2] * B[11] + A[4 * r + 3];
  }
}

static void inverse12(const double* T, double* O) {
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) O[4 * r + k] = T[4 * k + r];
  for (int r = 0; r < 3; ++r)
    O[4 * r + 3] = -(O[4 * r] * T[3] + O[4 * r + 1] * T[7] + O[4 * r + 2] * T[11]);
}

extern "C" vd_status vd_set_poses(vd_ctx* c, const double* poses, vd_pose_kind kind) {
  if (!c || !poses) return VD_ERR_ARG;
  const int N = c->N;
  std::vector<double> G(12 * (N + 1));
  if (kind == VD_POSE_ABSOLUTE) {
    for (int i = 0; i < 12 * (N + 1); ++i) {
      if (!isfinite(poses[i])) return VD_ERR_ARG;
      G[i] = poses[i];
    }
  } else if (kind == VD_POSE_RELATIVE) {
    static const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    memcpy(G.data(), I, sizeof I);
    for (int t = 1; t <= N; ++t) {
      for (int i = 0; i < 12; ++i)
        if (!isfinite(poses[12 * (t - 1) + i])) return VD_ERR_ARG;
      compose12(poses + 12 * (t - 1), G.data() + 12 * (t - 1), G.data() + 12 * t);
    }
  } else {
    return VD_ERR_ARG;
  }
  VD_CU(cudaMemcpyAsync(c->G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice,
                        c->stream));
  VD_CU(cudaMemcpyAsync(c->G_init, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice,
                        c->stream));
  VD_CU(launch_posef(c));
  VD_CU(cudaStreamSynchronize(c->stream));
  c->poses_set = 1;
  c->samples_set = 0;   // the pose samples no longer belong to the state
  ++c->cfg_version;
  return VD_OK;
}

extern "C" vd_status vd_get_poses(vd_ctx* c, double* out, vd_pose_kind kind) {
  if (!c || !out) return VD_ERR_ARG;
  const int N = c->N;
  std::vector<double> G(12 * (N + 1));
  VD_CU(cudaMemcpyAsync(G.data(), c->G, sizeof(double) * G.size(), cudaMemcpyDeviceToHost,
                        c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  if (kind == VD_POSE_ABSOLUTE) {
    memcpy(out, G.data(), sizeof(double) * G.size());
  } else if (kind == VD_POSE_RELATIVE) {
    for (int t = 1; t <= N; ++t) {
      double inv[12];
      inverse12(G.data() + 12 * (t - 1), inv);
      compose12(G.data() + 12 * t, inv, out + 12 * (t - 1));
    }
  } else {
    return VD_ERR_ARG;
  }
  return VD_OK;
}

extern "C" vd_status vd_set_state(vd_ctx* c, const float* rho, const float* q, const float* qhat,
                                  vd_mem mem) {
  if (!c || !rho) return VD_ERR_ARG;
  VD_CU(upload(c, c->rho, rho, c->npix, mem));
  if (q) VD_CU(upload(c, c->q, q, c->npix * c->N, mem));
  else VD_CU(launch_fill(c->q, 1.0f, c->npix * c->N, c->stream));
  if (qhat) VD_CU(upload(c, c->qhat, qhat, c->npix, mem));
  else VD_CU(launch_fill(c->qhat, 1.0f, c->npix, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  c->bootstrapped = 1;
  c->samples_set = 0;   // the pose samples no longer belong to the state
  return VD_OK;
}

static bool flows_ready(const vd_ctx* c) { return c->flow_pushed == ((1u << c->N) - 1u); }

static inline uint32_t itcode_of(int iter) { return iter < 0 ? VD_ITER_BOOT : (uint32_t)iter; }

static inline float perturb_scale(int iter) {
  const int i = iter < 0 ? 0 : iter;
  double s = 0.5 * ldexp(1.0, -i);
  if (s < 1.0 / 64.0) s = 1.0 / 64.0;
  return (float)s;
}

static cudaError_t posef_step(vd_ctx* c) {
  cudaError_t e = launch_posef(c);
  vd_prof_end(c, VD_ST_OTHER, 1);
  return e;
}

// The pose rows (posef, posed) mirror G at every step boundary: the device
// writers of G (the eight-point bootstrap, the mode search) store the rows
// of what they write, and every host write of G is followed by
// launch_posef.  So the steps below use them as they are.

// One depth M-step.  boot: the monocular bootstrap's depth from X_1 alone
// (one flow; timed with the rest of the bootstrap).
static cudaError_t depth_step(vd_ctx* c, int iter, int direction, bool boot = false) {
  cudaError_t e = cudaSuccess;
  const int nf = boot ? 1 : c->N;
  const int st_sample = boot ? VD_ST_OTHER : VD_ST_SAMPLE;
  const int st_prop = boot ? VD_ST_OTHER : VD_ST_PROPAGATE;
  vd_prof_begin(c, st_sample);
  e = launch_depth_sample(c, itcode_of(iter), perturb_scale(iter), nf);
  vd_prof_end(c, st_sample, 1);
  if (e != cudaSuccess) return e;
  vd_prof_begin(c, st_prop);
  e = launch_depth_propagate(c, direction, nf);
  vd_prof_end(c, st_prop, c->prm.hierarchical ? 3 : 1);
  return e;
}

static cudaError_t estep(vd_ctx* c, int direction) {
  vd_prof_begin(c, VD_ST_ESTEP);
  cudaError_t e = launch_estep(c, direction);
  vd_prof_end(c, VD_ST_ESTEP, 3);
  return e;
}

static cudaError_t pose_step(vd_ctx* c, int iter, int t) {
  cudaError_t e = cudaSuccess;
  if (t > 0) return launch_pose_frame(c, itcode_of(iter), t);
  for (int k = 1; k <= c->N && e == cudaSuccess; ++k) e = launch_pose_frame(c, itcode_of(iter), k);
  return e;
}

// The bootstrap is a function of the inputs alone: it starts from the initial
// poses (identity, or those of vd_set_poses), not from a previous run's.
static cudaError_t bootstrap(vd_ctx* c) {
  c->samples_set = 0;   // a bootstrap with given poses runs no pose step
  vd_prof_begin(c, VD_ST_OTHER);
  cudaError_t e = cudaMemcpyAsync(c->G, c->G_init, sizeof(double) * 12 * (c->N + 1),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = launch_posef(c);
  if (e == cudaSuccess) e = launch_initial_rho(c);
  if (e == cudaSuccess) e = launch_fill(c->q, 1.0f, c->npix * c->N, c->stream);
  if (e == cudaSuccess) e = launch_fill(c->qhat, 1.0f, c->npix, c->stream);
  int n = 4;
  if (e == cudaSuccess && c->prior_kind == VD_PRIOR_NONE) {
    if (!c->poses_set) {
      e = launch_eight_point(c);
      n += 2 * VD_IRLS_ITERS + 3;
    }
    if (e == cudaSuccess && c->N > 1) {
      e = launch_fill(c->q + c->npix, 0.0f, c->npix * (c->N - 1), c->stream);
      ++n;
    }
  }
  vd_prof_end(c, VD_ST_OTHER, n);
  if (e != cudaSuccess) return e;
  if (c->prior_kind == VD_PRIOR_NONE) {
    // depth from X_1 alone, then every flow rigid again
    e = depth_step(c, -1, 0, true);
    if (e == cudaSuccess) e = launch_fill(c->q, 1.0f, c->npix * c->N, c->stream);
    vd_prof_end(c, VD_ST_OTHER, 1);
    if (e == cudaSuccess && !c->poses_set) e = pose_step(c, -1, 0);
  } else if (!c->poses_set) {
    e = pose_step(c, -1, 0);
  }
  return e;
}

// Bootstrap with the learned initialiser: the monocular bootstrap above
// (8-point pose, depth from X_1 alone, pose step) with the network's
// inverse depth as the initial value of its depth step
// (slot 0 of every pixel's candidates, in place of the random draw).  The
// rest is the plain bootstrap (q = 1; with a prior, the prior's inverse
// depth and no depth step).  The network's rigidness is not used here: its
// geometry input comes from the 8-point pose, and where that pose is poor a
// rigidness that excludes pixels from the first pose step keeps the EM from
// recovering, while q = 1 lets it.
static cudaError_t bootstrap_learned(vd_ctx* c, vd_cnn* net) {
  if (c->prior_kind != VD_PRIOR_NONE) return bootstrap(c);
  vd_prof_begin(c, VD_ST_OTHER);
  cudaError_t e = cudaMemcpyAsync(c->G, c->G_init, sizeof(double) * 12 * (c->N + 1),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = launch_posef(c);
  if (e == cudaSuccess) e = launch_fill(c->qhat, 1.0f, c->npix, c->stream);
  int n = 2;
  if (e == cudaSuccess && !c->poses_set) {
    e = launch_eight_point(c);
    n += 2 * VD_IRLS_ITERS + 3;
  }
  if (e == cudaSuccess) e = launch_cnn_init(net, c, c->rho, nullptr);
  if (e == cudaSuccess) e = launch_fill(c->q, 1.0f, c->npix * c->N, c->stream);
  vd_prof_end(c, VD_ST_OTHER, n + 3 + 2 * VD_CNN_LAYERS);
  if (e != cudaSuccess) return e;
  // depth from X_1 alone, starting from the network's value
  e = depth_step(c, -1, 0, true);
  if (e == cudaSuccess && !c->poses_set) e = pose_step(c, -1, 0);
  return e;
}

static vd_status finish_sync(vd_ctx* c, int* degenerate_out) {
  int h = 0;
  VD_CU(cudaMemcpyAsync(&h, c->degenerate, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  if (degenerate_out) *degenerate_out = h;
  return h ? VD_WARN_DEGENERATE : VD_OK;
}

extern "C" vd_status vd_bootstrap(vd_ctx* c) {
  if (!c) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  VD_CU(cudaMemsetAsync(c->degenerate, 0, sizeof(int), c->stream));
  VD_CU(bootstrap(c));
  c->bootstrapped = 1;
  c->iter = 0;
  return finish_sync(c, nullptr);
}

// Bootstrap (when asked, or when the state is not bootstrapped) and n_iters
// EM iterations of one window, issued on its stream without any host
// synchronisation (so that the sequence can be captured into a graph).
static cudaError_t enqueue_em(vd_ctx* c, int n_iters, bool boot, int* booted) {
  cudaError_t e = cudaMemsetAsync(c->degenerate, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return e;
  if (booted) *booted = 0;
  if (boot || !c->bootstrapped) {
    e = bootstrap(c);
    if (e != cudaSuccess) return e;
    c->bootstrapped = 1;
    c->iter = 0;
    if (booted) *booted = 1;
  }
  for (int k = 0; k < n_iters; ++k) {
    const int i = c->iter;
    const int d = i & 3;
    if ((e = depth_step(c, i, d)) != cudaSuccess) return e;
    if ((e = estep(c, d)) != cudaSuccess) return e;
    if ((e = pose_step(c, i, 0)) != cudaSuccess) return e;
    c->iter = i + 1;
  }
  return cudaSuccess;
}

extern "C" vd_status vd_eight_point(vd_ctx* c, double* T1) {
  if (!c || !T1) return VD_ERR_ARG;
  if (!(c->flow_pushed & 1u)) return VD_ERR_STATE;
  std::vector<double> G(12 * (c->N + 1));
  VD_CU(cudaMemcpyAsync(G.data(), c->G, sizeof(double) * G.size(), cudaMemcpyDeviceToHost,
                        c->stream));
  VD_CU(launch_eight_point(c));
  VD_CU(cudaMemcpyAsync(T1, c->G + 12, sizeof(double) * 12, cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaMemcpyAsync(c->G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice,
                        c->stream));
  VD_CU(launch_posef(c));
  VD_CU(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

extern "C" vd_status vd_bootstrap_learned(vd_ctx* c, vd_cnn* net) {
  if (!c || !net) return VD_ERR_ARG;
  if (vd_cnn_flows(net) != c->N) {
    vd_set_error("the network was built for another number of flows");
    return VD_ERR_ARG;
  }
  if (!flows_ready(c)) return VD_ERR_STATE;
  VD_CU(cudaMemsetAsync(c->degenerate, 0, sizeof(int), c->stream));
  VD_CU(bootstrap_learned(c, net));
  c->bootstrapped = 1;
  c->iter = 0;
  int tc = 0;
  VD_CU(cudaMemcpyAsync(&tc, vd_cnn_err_flag(net), sizeof(int), cudaMemcpyDeviceToHost,
                        c->stream));
  const vd_status st = finish_sync(c, nullptr);
  if (tc) {
    vd_set_error("a tensor-core wait gave up");
    return VD_ERR_TIMEOUT;
  }
  return st;
}

extern "C" vd_status vd_run_em(vd_ctx* c, int n_iters, vd_stats* stats) {
  if (!c || n_iters < 0) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  int booted = 0;
  VD_CU(enqueue_em(c, n_iters, false, &booted));
  int deg = 0;
  vd_status st = finish_sync(c, &deg);
  if (st < 0) return st;
  if (stats) {
    double h[2] = {0, 0};
    VD_CU(launch_stats(c, c->stat_out));
    VD_CU(cudaMemcpyAsync(h, c->stat_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    VD_CU(cudaStreamSynchronize(c->stream));
    stats->iterations = n_iters;
    stats->bootstrapped = booted;
    stats->degenerate_frames = deg;
    stats->mean_energy = h[0] / (double)c->npix;
    stats->rigid_fraction = h[1] / (double)(c->npix * c->N);
  }
  return st;
}

// ---------------------------------------------------------------------------
// Launch tuning: time every launch shape of the two tunable kernels on this
// window and keep the fastest (median of a few launches each).
// ---------------------------------------------------------------------------
static const int kK1Warps[3] = {1, 2, 4};

static bool tune_ok(const vd_tune* t) {
  return t && (t->k1_warps == 1 || t->k1_warps == 2 || t->k1_warps == 4) &&
         (t->score_threads == 256 || t->score_threads == 512) &&
         t->score_blocks_per_sm >= 1 && t->score_blocks_per_sm <= VD_SCORE_BPS_MAX;
}

template <class F>
static cudaError_t time_median(vd_ctx* c, int reps, F launch, float* ms_out) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  std::vector<float> t;
  if (e == cudaSuccess) e = launch();   // warm-up
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    t.push_back(ms);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return cudaSuccess;
}

extern "C" vd_status vd_autotune(vd_ctx* c, vd_tune* out) {
  if (!c) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  const int prof = c->prof_on;
  c->prof_on = 0;
  vd_tune t;
  memset(&t, 0, sizeof t);
  // a representative state: the bootstrap and one EM iteration
  cudaError_t e = enqueue_em(c, 1, true, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  const int it = c->iter;
  float best = INFINITY;
  t.k1_warps = c->k1_warps;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    c->k1_warps = kK1Warps[i];
    e = time_median(c, 5, [&] { return launch_depth_sample(c, itcode_of(it), perturb_scale(it), c->N); },
                    &t.k1_ms[i]);
    if (e == cudaSuccess && t.k1_ms[i] < best) {
      best = t.k1_ms[i];
      t.k1_warps = kK1Warps[i];
    }
  }
  best = INFINITY;
  t.score_blocks_per_sm = c->score_bps;
  t.score_threads = c->score_threads;
  for (int ti = 0; ti < 2 && e == cudaSuccess; ++ti) {
    c->score_threads = ti ? 512 : 256;
    for (int b = 1; b <= VD_SCORE_BPS_MAX && e == cudaSuccess; ++b) {
      c->score_bps = b;
      float* ms = &t.score_ms[ti][b - 1];
      e = time_median(c, 5, [&] { return launch_pose_score_only(c); }, ms);
      if (e == cudaSuccess && *ms < best) {
        best = *ms;
        t.score_blocks_per_sm = b;
        t.score_threads = c->score_threads;
      }
    }
  }
  c->prof_on = prof;
  c->k1_warps = t.k1_warps;
  c->score_bps = t.score_blocks_per_sm;
  c->score_threads = t.score_threads;
  c->tune_meas = t;
  ++c->cfg_version;
  VD_CU(e);
  if (out) *out = t;
  return VD_OK;
}

extern "C" vd_status vd_set_tune(vd_ctx* c, const vd_tune* t) {
  if (!c || !tune_ok(t)) return VD_ERR_ARG;
  c->k1_warps = t->k1_warps;
  c->score_bps = t->score_blocks_per_sm;
  c->score_threads = t->score_threads;
  ++c->cfg_version;
  return VD_OK;
}

extern "C" vd_status vd_get_tune(vd_ctx* c, vd_tune* out) {
  if (!c || !out) return VD_ERR_ARG;
  *out = c->tune_meas;
  out->k1_warps = c->k1_warps;
  out->score_blocks_per_sm = c->score_bps;
  out->score_threads = c->score_threads;
  return VD_OK;
}

// ---------------------------------------------------------------------------
// Batched EM: one CUDA graph runs the bootstrap and the iterations of every
// window, one graph branch per window.
// ---------------------------------------------------------------------------
struct vd_batch {
  std::vector<vd_ctx*> win;
  std::vector<cudaStream_t> branch;    // capture streams, one per window
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t stream = nullptr;       // the batch stream (the caller's; may be the legacy stream)
  cudaStream_t origin = nullptr;       // capture origin (a capture cannot start on the legacy stream)
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> key;          // launch signature of the captured graph
  int* d_deg = nullptr;                // [n] degenerate counters, gathered by the graph
  int* h_deg = nullptr;                // pinned host copy
  vd_batch_stats st;
};

static void batch_free(vd_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (vd_ctx* c : b->win) {
    c->batch_owned = 0;
    vd_destroy(c);
  }
  for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->d_deg) cudaFree(b->d_deg);
  if (b->h_deg) cudaFreeHost(b->h_deg);
  delete b;
}

extern "C" vd_status vd_batch_create(int n, const vd_window_desc* descs, const vd_params* params,
                                     int params_stride, void* stream, vd_batch** out) {
  if (!out) return VD_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !descs || (params_stride != 0 && params_stride != 1)) return VD_ERR_ARG;
  vd_batch* b = new vd_batch();
  memset(&b->st, 0, sizeof b->st);
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    vd_ctx* c = nullptr;
    const vd_status s = vd_create(&descs[i], params ? params + (params_stride ? i : 0) : nullptr,
                                  stream, &c);
    if (s != VD_OK) {
      batch_free(b);
      return s;
    }
    c->batch_owned = 1;
    b->win.push_back(c);
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branch.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_deg, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_deg, sizeof(int) * n);
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    batch_free(b);
    return e == cudaErrorMemoryAllocation ? VD_ERR_OOM : VD_ERR_CUDA;
  }
  b->st.windows = n;
  *out = b;
  return VD_OK;
}

extern "C" vd_status vd_batch_destroy(vd_batch* b) {
  if (!b) return VD_ERR_ARG;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return VD_OK;
}

extern "C" vd_status vd_batch_window(vd_batch* b, int i, vd_ctx** out) {
  if (!b || !out || i < 0 || i >= (int)b->win.size()) return VD_ERR_ARG;
  *out = b->win[i];
  return VD_OK;
}

extern "C" vd_status vd_batch_get_stats(vd_batch* b, vd_batch_stats* out) {
  if (!b || !out) return VD_ERR_ARG;
  *out = b->st;
  return VD_OK;
}

// Tune one window of every distinct launch configuration and hand its
// choice to the windows that share it.
static vd_status batch_capture(vd_batch* b, int n_iters, bool boot);

// Scoring shapes whose time alone is within this factor of the best shape of
// every window group take part in the whole-batch trial.
static const float kBatchTrialMargin = 1.25f;

// Time of one run of the captured batch graph (the second of two launches,
// so that the graph's upload is not counted).
static cudaError_t batch_time_run(vd_batch* b, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

static void batch_set_score_shape(vd_batch* b, int threads, int bps) {
  for (vd_ctx* o : b->win) {
    if (o->score_threads == threads && o->score_bps == bps) continue;
    o->score_threads = threads;
    o->score_bps = bps;
    ++o->cfg_version;
  }
}

// Tuning of a batch.  (1) One window of every distinct (size, N, K, S,
// prior) is tuned alone (vd_autotune) and its choice given to the others.
// (2) The windows' kernels share the SMs, so the scoring shape that is
// fastest alone is not always the fastest among the other windows' launches
// (one 512-thread block of ~90 registers per SM leaves little room beside
// it).  Every shape within kBatchTrialMargin of the best time alone of every
// group is therefore timed on whole-batch runs (the bootstrap and up to two
// iterations) and the fastest one is given to every window.  A trial leaves
// no state behind: the run that follows bootstraps again.
static vd_status batch_autotune(vd_batch* b, int n_iters) {
  const int n = (int)b->win.size();
  std::vector<int> done(n, 0);
  std::vector<vd_ctx*> leaders;
  for (int i = 0; i < n; ++i) {
    if (done[i]) continue;
    vd_ctx* c = b->win[i];
    const vd_status s = vd_autotune(c, nullptr);
    if (s < 0) return s;
    leaders.push_back(c);
    for (int k = i; k < n; ++k) {
      vd_ctx* o = b->win[k];
      if (o->W == c->W && o->H == c->H && o->N == c->N && o->dp.K == c->dp.K &&
          o->dp.S == c->dp.S && o->prior_kind == c->prior_kind) {
        done[k] = 1;
        if (o != c && (o->k1_warps != c->k1_warps || o->score_bps != c->score_bps ||
                       o->score_threads != c->score_threads)) {
          o->k1_warps = c->k1_warps;
          o->score_bps = c->score_bps;
          o->score_threads = c->score_threads;
          ++o->cfg_version;
        }
      }
    }
  }
  if (n < 2 || n_iters < 1) return VD_OK;
  std::vector<std::pair<int, int>> cand;   // (threads, blocks per SM)
  for (int ti = 0; ti < 2; ++ti)
    for (int bps = 1; bps <= VD_SCORE_BPS_MAX; ++bps) {
      bool ok = true;
      for (vd_ctx* c : leaders) {
        float best = INFINITY;
        for (int a = 0; a < 2; ++a)
          for (int q = 0; q < VD_SCORE_BPS_MAX; ++q) best = fminf(best, c->tune_meas.score_ms[a][q]);
        ok = ok && c->tune_meas.score_ms[ti][bps - 1] <= kBatchTrialMargin * best;
      }
      if (ok) cand.push_back({ti ? 512 : 256, bps});
    }
  if (cand.size() < 2) return VD_OK;
  const int trial_iters = n_iters < 2 ? n_iters : 2;
  float best = INFINITY;
  std::pair<int, int> pick = cand[0];
  for (const auto& cs : cand) {
    batch_set_score_shape(b, cs.first, cs.second);
    vd_status s = batch_capture(b, trial_iters, true);
    if (s < 0) return s;
    float ms = 0.0f;
    const cudaError_t e = batch_time_run(b, &ms);
    if (e != cudaSuccess) {
      b->key.clear();
      vd_set_error(cudaGetErrorString(e));
      return VD_ERR_CUDA;
    }
    if (ms < best) {
      best = ms;
      pick = cs;
    }
  }
  b->key.clear();                     // the run that follows captures its own graph
  batch_set_score_shape(b, pick.first, pick.second);
  return VD_OK;
}

static vd_status batch_capture(vd_batch* b, int n_iters, bool boot) {
  const int n = (int)b->win.size();
  std::vector<int> boot0(n), iter0(n);
  long long launches0 = 0, launches1 = 0;
  for (int i = 0; i < n; ++i) {
    boot0[i] = b->win[i]->bootstrapped;
    iter0[i] = b->win[i]->iter;
    for (int k = 0; k < VD_N_STAGES; ++k) launches0 += b->win[i]->launches[k];
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  e = cudaEventRecord(b->fork, b->origin);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    vd_ctx* c = b->win[i];
    const int prof = c->prof_on;
    c->prof_on = 0;
    c->stream = b->branch[i];
    e = cudaStreamWaitEvent(c->stream, b->fork, 0);
    if (e == cudaSuccess) e = enqueue_em(c, n_iters, boot, nullptr);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_deg + i, c->degenerate, sizeof(int), cudaMemcpyDeviceToDevice,
                          c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->join[i], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    c->stream = b->stream;
    c->prof_on = prof;
  }
  const cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
  }
  size_t nodes = 0;
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nodes);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    for (int i = 0; i < n; ++i) {   // nothing of the capture ran
      b->win[i]->bootstrapped = boot0[i];
      b->win[i]->iter = iter0[i];
    }
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    b->key.clear();
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < VD_N_STAGES; ++k) launches1 += b->win[i]->launches[k];
  b->st.captures += 1;
  b->st.graph_nodes = (long long)nodes;
  b->st.kernels_per_run = launches1 - launches0;
  return VD_OK;
}

extern "C" vd_status vd_batch_run(vd_batch* b, int n_iters, int flags, int* degenerate) {
  if (!b || n_iters < 0 || (flags & ~(VD_BATCH_BOOTSTRAP | VD_BATCH_AUTOTUNE)) ||
      ((flags & VD_BATCH_AUTOTUNE) && !(flags & VD_BATCH_BOOTSTRAP)))
    return VD_ERR_ARG;
  const int n = (int)b->win.size();
  for (vd_ctx* c : b->win)
    if (!flows_ready(c)) return VD_ERR_STATE;
  const bool boot = (flags & VD_BATCH_BOOTSTRAP) != 0;
  if (flags & VD_BATCH_AUTOTUNE) {
    const vd_status s = batch_autotune(b, n_iters);
    if (s < 0) return s;
  }
  // signature of the launches this run issues
  std::vector<long long> key = {n_iters, boot ? 1 : 0};
  for (vd_ctx* c : b->win) {
    key.push_back(c->cfg_version);
    key.push_back(boot ? -1 : ((long long)c->bootstrapped << 32) + c->iter);
  }
  if (!b->exec || key != b->key) {
    const vd_status s = batch_capture(b, n_iters, boot);
    if (s < 0) return s;
    b->key = key;
  } else {
    for (vd_ctx* c : b->win) {   // the host state the captured sequence leaves
      if (boot || !c->bootstrapped) {
        c->bootstrapped = 1;
        c->iter = 0;
      }
      c->iter += n_iters;
    }
    b->st.replays += 1;
  }
  VD_CU(cudaGraphLaunch(b->exec, b->stream));
  VD_CU(cudaMemcpyAsync(b->h_deg, b->d_deg, sizeof(int) * n, cudaMemcpyDeviceToHost, b->stream));
  VD_CU(cudaStreamSynchronize(b->stream));
  int any = 0;
  for (int i = 0; i < n; ++i) {
    if (degenerate) degenerate[i] = b->h_deg[i];
    any |= b->h_deg[i] != 0;
  }
  return any ? VD_WARN_DEGENERATE : VD_OK;
}

extern "C" vd_status vd_depth_mstep(vd_ctx* c, int iter, int direction) {
  if (!c || direction < 0 || direction > 3 || iter < -1) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  // iter -1 without a prior is the monocular bootstrap's own depth step (X_1 alone)
  VD_CU(depth_step(c, iter, direction, iter < 0 && c->prior_kind == VD_PRIOR_NONE));
  VD_CU(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

extern "C" vd_status vd_rigidness_estep(vd_ctx* c, int direction) {
  if (!c || direction < 0 || direction > 3) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  VD_CU(posef_step(c));
  VD_CU(estep(c, direction));
  VD_CU(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

extern "C" vd_status vd_pose_mstep(vd_ctx* c, int iter, int t) {
  if (!c || t < 0 || t > c->N || iter < -1) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  VD_CU(cudaMemsetAsync(c->degenerate, 0, sizeof(int), c->stream));
  VD_CU(pose_step(c, iter, t));
  return finish_sync(c, nullptr);
}

extern "C" vd_status vd_get_inv_depth(vd_ctx* c, float* out, vd_mem mem) {
  if (!c || !out) return VD_ERR_ARG;
  VD_CU(download(c, out, c->rho, c->npix, mem));
  return VD_OK;
}

extern "C" vd_status vd_get_rigidness(vd_ctx* c, float* out, vd_mem mem) {
  if (!c || !out) return VD_ERR_ARG;
  VD_CU(download(c, out, c->q, c->npix * c->N, mem));
  return VD_OK;
}

extern "C" vd_status vd_get_prior_rigidness(vd_ctx* c, float* out, vd_mem mem) {
  if (!c || !out) return VD_ERR_ARG;
  VD_CU(download(c, out, c->qhat, c->npix, mem));
  return VD_OK;
}

extern "C" vd_status vd_get_confidence(vd_ctx* c, float* out, vd_mem mem) {
  if (!c || !out) return VD_ERR_ARG;
  VD_CU(download(c, out, c->conf, c->npix, mem));
  return VD_OK;
}

extern "C" vd_status vd_get_depth_candidates(vd_ctx* c, float* rs, float* es, vd_mem mem) {
  if (!c || !rs || !es) return VD_ERR_ARG;
  VD_CU(download(c, rs, c->rho_star, c->npix, mem));
  VD_CU(download(c, es, c->e_star, c->npix, mem));
  return VD_OK;
}

extern "C" vd_status vd_eval_energy(vd_ctx* c, const float* rho, float* out, vd_mem mem) {
  if (!c || !rho || !out) return VD_ERR_ARG;
  if (!flows_ready(c)) return VD_ERR_STATE;
  VD_CU(upload(c, c->rho_mid, rho, c->npix, mem));
  VD_CU(launch_posef(c));
  VD_CU(launch_eval_energy(c, c->rho_mid, c->e_mid));
  VD_CU(download(c, out, c->e_mid, c->npix, mem));
  VD_CU(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

extern "C" vd_status vd_get_pose_samples(vd_ctx* c, double* poses, double* energies, int* n_rigid) {
  if (!c) return VD_ERR_ARG;
  const int S = c->prm.n_pose_samples;
  const size_t f = c->last_pose_t > 0 ? (size_t)(c->last_pose_t - 1) * VD_MAX_SAMPLES : 0;
  if (poses)
    VD_CU(cudaMemcpyAsync(poses, c->sample_pose + 12 * f, sizeof(double) * 12 * S,
                          cudaMemcpyDeviceToHost, c->stream));
  if (energies)
    VD_CU(cudaMemcpyAsync(energies, c->sample_energy + f, sizeof(double) * S,
                          cudaMemcpyDeviceToHost, c->stream));
  if (n_rigid)
    VD_CU(cudaMemcpyAsync(n_rigid, c->n_rigid, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

// ---------------------------------------------------------------------------
// checkpoint blob: header, then rho, q, q_hat, C (float32) and G (float64)
// ---------------------------------------------------------------------------
struct BlobHeader {
  char magic[8];
  int version, W, H, N, iter, bootstrapped, poses_set, pad;
};

extern "C" vd_status vd_export_state(vd_ctx* c, void* blob, size_t* bytes) {
  if (!c || !bytes) return VD_ERR_ARG;
  const size_t nf = c->npix * (3 + c->N);
  const size_t need = sizeof(BlobHeader) + sizeof(float) * nf + sizeof(double) * 12 * (c->N + 1);
  if (!blob) {
    *bytes = need;
    return VD_OK;
  }
  if (*bytes < need) return VD_ERR_ARG;
  BlobHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, "VDEMST01", 8);
  h.version = 1;
  h.W = c->W;
  h.H = c->H;
  h.N = c->N;
  h.iter = c->iter;
  h.bootstrapped = c->bootstrapped;
  h.poses_set = c->poses_set;
  char* p = (char*)blob;
  memcpy(p, &h, sizeof h);
  float* f = (float*)(p + sizeof h);
  const size_t np = c->npix;
  VD_CU(cudaMemcpyAsync(f, c->rho, sizeof(float) * np, cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaMemcpyAsync(f + np, c->q, sizeof(float) * np * c->N, cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaMemcpyAsync(f + np * (1 + c->N), c->qhat, sizeof(float) * np, cudaMemcpyDeviceToHost,
                        c->stream));
  VD_CU(cudaMemcpyAsync(f + np * (2 + c->N), c->conf, sizeof(float) * np, cudaMemcpyDeviceToHost,
                        c->stream));
  VD_CU(cudaMemcpyAsync((double*)(f + nf), c->G, sizeof(double) * 12 * (c->N + 1),
                        cudaMemcpyDeviceToHost, c->stream));
  VD_CU(cudaStreamSynchronize(c->stream));
  *bytes = need;
  return VD_OK;
}

extern "C" vd_status vd_import_state(vd_ctx* c, const void* blob, size_t bytes) {
  if (!c || !blob || bytes < sizeof(BlobHeader)) return VD_ERR_ARG;
  BlobHeader h;
  memcpy(&h, blob, sizeof h);
  if (memcmp(h.magic, "VDEMST01", 8) != 0 || h.version != 1 || h.W != c->W || h.H != c->H ||
      h.N != c->N)
    return VD_ERR_ARG;
  const size_t nf = c->npix * (3 + c->N);
  const size_t need = sizeof(BlobHeader) + sizeof(float) * nf + sizeof(double) * 12 * (c->N + 1);
  if (bytes < need) return VD_ERR_ARG;
  const float* f = (const float*)((const char*)blob + sizeof h);
  const size_t np = c->npix;
  VD_CU(cudaMemcpyAsync(c->rho, f, sizeof(float) * np, cudaMemcpyHostToDevice, c->stream));
  VD_CU(cudaMemcpyAsync(c->q, f + np, sizeof(float) * np * c->N, cudaMemcpyHostToDevice, c->stream));
  VD_CU(cudaMemcpyAsync(c->qhat, f + np * (1 + c->N), sizeof(float) * np, cudaMemcpyHostToDevice,
                        c->stream));
  VD_CU(cudaMemcpyAsync(c->conf, f + np * (2 + c->N), sizeof(float) * np, cudaMemcpyHostToDevice,
                        c->stream));
  VD_CU(cudaMemcpyAsync(c->G, (const double*)(f + nf), sizeof(double) * 12 * (c->N + 1),
                        cudaMemcpyHostToDevice, c->stream));
  // a later bootstrap starts from the imported poses if they were set by the
  // caller (the blob keeps no other copy of them), else from the identity
  std::vector<double> I(12 * (c->N + 1), 0.0);
  for (int t = 0; t <= c->N; ++t) I[12 * t] = I[12 * t + 5] = I[12 * t + 10] = 1.0;
  VD_CU(cudaMemcpyAsync(c->G_init, h.poses_set ? (const void*)(f + nf) : (const void*)I.data(),
                        sizeof(double) * 12 * (c->N + 1), cudaMemcpyHostToDevice, c->stream));
  VD_CU(launch_posef(c));
  VD_CU(cudaStreamSynchronize(c->stream));
  c->iter = h.iter;
  c->bootstrapped = h.bootstrapped;
  c->samples_set = 0;   // the blob holds no pose samples
  c->poses_set = h.poses_set;
  ++c->cfg_version;
  return VD_OK;
}

// ---------------------------------------------------------------------------
// Checked build: the index-check records of every translation unit.
// ---------------------------------------------------------------------------
cudaError_t vd_check_take_pose(unsigned long long*);
cudaError_t vd_check_take_depth(unsigned long long*);
cudaError_t vd_check_take_estep(unsigned long long*);
cudaError_t vd_check_take_boot(unsigned long long*);
cudaError_t vd_check_take_ka(unsigned long long*);
cudaError_t vd_check_take_posecov(unsigned long long*);
cudaError_t vd_check_take_cnn(unsigned long long*);
cudaError_t vd_check_take_vc(unsigned long long*);

extern "C" vd_status vd_check_report(long long* out) {
  if (!out) return VD_ERR_ARG;
  cudaError_t (*take[])(unsigned long long*) = {
      vd_check_take_pose, vd_check_take_depth, vd_check_take_estep, vd_check_take_boot,
      vd_check_take_ka, vd_check_take_posecov, vd_check_take_cnn, vd_check_take_vc};
  for (int i = 0; i < 4; ++i) out[i] = 0;
#ifdef VD_CHECKED
  out[4] = 1;
#else
  out[4] = 0;
#endif
  for (auto f : take) {
    unsigned long long r[4];
    VD_CU(f(r));
    if (r[3] && !out[0]) {
      out[0] = (long long)r[0];
      out[1] = (long long)r[1];
      out[2] = (long long)r[2];
    }
    out[3] += (long long)r[3];
  }
  return VD_OK;
}
