// Internal definitions shared by the library's translation units: the device
// parameter block, the context and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "voldor_em.h"

#define VD_MAX_FLOWS 8
#define VD_MAX_SAMPLES 256
#define VD_SCORE_BPS_MAX 4          // pose-scoring blocks per SM, upper bound of vd_tune
#define VD_MAX_ROOTS (4 * VD_MAX_SAMPLES)

// Constants of the model that both hosts and kernels use.
#define VD_Z_EPS 1e-6f
#define VD_L_BEHIND 64.0f           // energy of an observation the rigid model cannot explain
#define VD_R_FLOOR 1e-6f
#define VD_ITER_BOOT 0xFFFFFFFFu
#define VD_TAG_DEPTH 0u
#define VD_TAG_POSE 1u
#define VD_TAG_INIT 2u
#define VD_MS_MAX_ITERS 100
#define VD_MS_TOL 1e-12
#define VD_MS_TOL_F32 1e-6          // float32 mean-shift stop, relative to 1 + |tau|
#define VD_MAX_ATTEMPTS 8
#define VD_IRLS_ITERS 8

enum { VD_PRIOR_NONE = 0, VD_PRIOR_STEREO = 1, VD_PRIOR_RGBD = 2 };

// Everything a kernel needs to know about the window and the parameters,
// passed by value.
struct DevParams {
  int W, H, N, K, S;
  float fx, fy, cx, cy;
  float alpha0, alpha1, beta, p0;
  int fast_beta2;          // beta == 2 and alpha1 == 0: closed-form energy
  float c0;                // P0 * pi * alpha0^2
  float log2c0;            // log2 c0
  float inv_a2;            // 1 / alpha0^2
  float cgen;              // P0 * 2 pi / beta (general path factor, times alpha^2)
  float gamma;
  float rho_min, rho_max;
  int share;
  uint32_t key0, key1;
  int prior_kind;
  float fxb;               // fx * baseline (stereo)
  float c_sigma, w_unif, logk;   // RGB-D prior: logk = log(sqrt(2 pi) c_sigma / w)
  double fx_d, fy_d, cx_d, cy_d;
  double ms_sig_rot, ms_sig_rel, ms_sig_abs;
  // fx, fy, cx, cy, 1/fx, 1/fy as double-float (hi, lo) pairs
  float kdf[12];
};

struct vd_ctx {
  vd_window_desc desc;
  vd_params prm;
  DevParams dp;
  cudaStream_t stream;
  int W, H, N;
  size_t npix;

  // inputs
  float2* flow;            // [N][H][W]
  unsigned flow_pushed;    // bit t-1 set once X_t was pushed
  int prior_kind;
  float fxb;               // fx * stereo baseline
  float* prior_val;        // stereo: disparity; rgbd: inverse depth (NaN = hole)
  float* prior_rho;        // inverse depth of the prior (NaN = hole)
  float* prior_conf;       // confidence (1 if none given)

  // EM state
  float* rho;              // [H][W]
  float* q;                // [N][H][W]
  float* qhat;             // [H][W]
  float* conf;             // [H][W] Eq. 6
  double* G;               // [N+1][12] absolute poses
  double* G_init;          // [N+1][12] poses every bootstrap starts from (identity or vd_set_poses)
  float* posef;            // [N+1][12] float K R | K tau
  float2* posed;           // [N+1][12] the same rows as double-float (hi, lo)
  int bootstrapped;
  int poses_set;
  int iter;                // next EM iteration index

  // depth step scratch
  float* rho_star;
  float* e_star;
  float* rho_mid;
  float* e_mid;
  float* coarse;           // hierarchical coarse map
  float* lam;              // [N][H][W] rigid / outlier likelihood ratio

  // pose step scratch
  unsigned char* flags;    // [H*W]
  int* blk_counts;         // [nblk_scan]
  int* n_rigid;            // [1]
  int* rigid_idx;          // [H*W]
  float4* rpts;            // [H*W] (X, Y, Z, w)
  float4* robs;            // [H*W] (x_obs, y_obs, alpha, 0)
  double* roots;           // [S][4][12]
  int* root_count;         // [S]
  float* rootsf;           // [S*4][12] float K R | K tau of every root slot
  float* rootsr;           // [S*4][12] float R | tau of every root slot
  float* partial;          // [S*4][score blocks]
  double* root_energy;     // [S*4]
  unsigned long long* score_work;  // [1] rigid pixels x roots scored since vd_profile_enable
  double* sample_pose;     // [N][S][12] kept root of every sample, per frame
  double* sample_energy;   // [N][S] (+inf: no root)
  int last_pose_t;         // frame of the last pose M-step (0: none)
  unsigned samples_set;    // bit t-1: frame t's samples are from a pose M-step
  double* pc_out;          // [N][52] pose covariance results (mean, cov, info)
  int* degenerate;         // [1] counter of kept poses
  int nblk_scan;
  int nblk_score;

  // bootstrap scratch
  float2* ep_partial;      // [blocks][45] double-float partial sums of the normal matrix
  double* ep_M;            // [45]
  double* ep_E;            // [9] current essential matrix (row-major)
  double* ep_cand;         // [4][12]
  int* ep_count;           // [4]
  int ep_blocks;

  // launch shapes (vd_tune) and the device they were sized for
  int num_sms;
  int k1_warps;            // warps per block of the depth-sampling kernel
  int score_bps;           // pose-scoring blocks per SM
  int score_threads;       // pose-scoring threads per block (256 or 512)
  int batch_owned;         // window of a vd_batch (stream owned by the batch)
  vd_tune tune_meas;       // last vd_autotune measurement
  long long cfg_version;   // bumped by every change that alters a captured launch

  // profiling: event pairs per recorded stage execution, launch counters
  int prof_on;
  void* prof;              // ProfState (vd_api.cu)
  long long launches[VD_N_STAGES];

  // reductions for stats
  // visibility-coverage scratch: N + 1 coverage maps of one byte per pixel
  // cell (frames 1..N and a caller's pose), their counters, the caller's pose
  unsigned char* vc_cover;        // [N + 1][vc_stride]
  unsigned long long* vc_counts;  // [1 + 2 (N + 1)]
  double* vc_pose;                // [12]
  size_t vc_stride;               // npix rounded up to 16
  double* stat_partial;    // [blocks][2]
  double* stat_out;        // [2]
  int stat_blocks;
};

// ---- launchers (one per translation unit family) --------------------------
cudaError_t launch_posef(vd_ctx* c);
// nf: flows that enter the energy (c->N, or 1 for the depth-from-X_1 step of
// the monocular bootstrap, where q_t = 0 for t > 1 makes the other terms 0).
cudaError_t launch_depth_sample(vd_ctx* c, uint32_t itcode, float s_pert, int nf);
cudaError_t launch_depth_propagate(vd_ctx* c, int direction, int nf);
cudaError_t launch_eval_energy(vd_ctx* c, const float* rho_in, float* e_out);
cudaError_t launch_estep(vd_ctx* c, int direction);
cudaError_t launch_pose_frame(vd_ctx* c, uint32_t itcode, int t);
// one dense scoring pass of the current roots (frame t's rigid set), for tuning
cudaError_t launch_pose_score_only(vd_ctx* c);
// function attributes set once per device before any launch or capture
cudaError_t vd_pose_prepare(void);
cudaError_t launch_initial_rho(vd_ctx* c);
cudaError_t launch_eight_point(vd_ctx* c);
cudaError_t launch_fill(float* p, float v, size_t n, cudaStream_t s);
cudaError_t launch_stats(vd_ctx* c, double* out2);
cudaError_t launch_prior_prepare(vd_ctx* c, const float* raw, const float* conf);
cudaError_t launch_check_finite(const float* p, size_t n, int* flag, cudaStream_t s);
cudaError_t launch_copy_flow(vd_ctx* c, int t, const float* src, long pitch);
// learned initialiser (vd_cnn.cu): rho and q of the context from the network
int vd_cnn_flows(const vd_cnn* n);
// forward pass on the context's flows (geometry from its T_1); rho (context
// range) into rho_dst and the rigidness of every flow into q_dst (nullable)
cudaError_t launch_cnn_init(vd_cnn* n, vd_ctx* c, float* rho_dst, float* q_dst);
int* vd_cnn_err_flag(vd_cnn* n);

void vd_set_error(const char* msg);

// Return from a vd_status function on a CUDA error (recording its message).
#define VD_CU(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) {                          \
      vd_set_error(cudaGetErrorString(e_));           \
      return e_ == cudaErrorMemoryAllocation ? VD_ERR_OOM : VD_ERR_CUDA; \
    }                                                 \
  } while (0)
// stage profiling hooks (no-ops unless enabled); `n_launch` kernels are counted
void vd_prof_begin(vd_ctx* c, int stage);
void vd_prof_end(vd_ctx* c, int stage, int n_launch);

enum { VD_ST_SAMPLE = 0, VD_ST_PROPAGATE = 1, VD_ST_ESTEP = 2, VD_ST_RIGID = 3, VD_ST_P3P = 4,
       VD_ST_SCORE = 5, VD_ST_SELECT = 6, VD_ST_OTHER = 7 };
