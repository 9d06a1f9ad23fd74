/*
 * voldor_em.h -- C ABI of the GB300 (sm_103a) dense-indirect EM library.
 *
 * The library estimates, for one window of N dense optical-flow fields, the
 * inverse-depth map of the reference frame, per-flow rigidness maps and the
 * camera poses, by the generalised EM of VOLDOR+ (Min & Dunn, "VOLDOR+SLAM:
 * For the times when feature-based or direct methods are not good enough",
 * 2021, Sec. III-A, Eq. 1-7):
 *   depth M-step      -- sample inverse-depth hypotheses per pixel, keep the
 *                        argmin of flow energy + prior energy (Eq. 5, Eq. 4),
 *                        propagate along alternately directed 1-D chains;
 *   rigidness E-step  -- forward-backward smoothing of two-state chains;
 *   pose M-step       -- Monte-Carlo P3P samples scored against every rigid
 *                        pixel, mean-shift mode in se(3) (Eq. 7).
 *
 * Conventions used by every call
 *   - Pixel (u, v): u = column in [0, W), v = row in [0, H); maps are row-major
 *     [H][W] float32 (rigidness [N][H][W]).
 *   - Flow X_t (t = 1..N) lives on frame t-1's pixel grid and holds (dx, dy) in
 *     pixels, interleaved: uv[2 * (v * row_pitch + u) + {0, 1}].
 *   - Poses are float64 3x4 row-major [R | tau].  ABSOLUTE pose G_t maps
 *     reference-frame (frame 0) coordinates to frame t: X_t = R X_0 + tau.
 *     RELATIVE pose T_t = G_t G_{t-1}^-1 maps frame t-1 to frame t.
 *   - Host pointers (VD_MEM_HOST) may be pageable or pinned; device pointers
 *     (VD_MEM_DEVICE) must be device memory of the context's GPU.  The library
 *     copies inputs when they are pushed and never keeps a caller pointer.
 *     All buffers belong to the caller; the context owns its internal state.
 *   - Work is issued on the context's CUDA stream.  Calls that return data to
 *     host memory, and vd_run_em, synchronise that stream before returning.
 *   - No call aborts or throws.  Every call returns a vd_status; on
 *     VD_ERR_CUDA the CUDA error string is available from vd_last_error().
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef VOLDOR_EM_H
#define VOLDOR_EM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vd_ctx vd_ctx;

typedef enum {
  VD_OK = 0,
  VD_WARN_DEGENERATE = 1,  /* a pose M-step had < 3 rigid pixels or no valid
                              P3P sample; that pose was kept unchanged        */
  VD_ERR_ARG = -1,         /* invalid argument (null, size, range, NaN flow) */
  VD_ERR_CUDA = -2,        /* a CUDA call failed, see vd_last_error()         */
  VD_ERR_OOM = -3,         /* device allocation failed                        */
  VD_ERR_STATE = -4,       /* call out of order (e.g. EM before every flow)   */
  VD_ERR_TIMEOUT = -5,     /* a bounded device wait gave up (tensor-core
                              kernels, vd_check_bounded_wait)                 */
  VD_ERR_NUMERIC = -6      /* non-finite value detected in the state          */
} vd_status;

typedef enum { VD_MEM_HOST = 0, VD_MEM_DEVICE = 1 } vd_mem;
typedef enum { VD_POSE_ABSOLUTE = 0, VD_POSE_RELATIVE = 1 } vd_pose_kind;

/* Window geometry: image size, number of flow fields N (1..8), pinhole K. */
typedef struct {
  int width, height, n_flows;
  double fx, fy, cx, cy;
} vd_window_desc;

/* Hyper-parameters of the hot path.  The paper names several of them without
 * values (Sigma of Eq. 7, the chain schedule, the hierarchical scale and
 * window of Sec. III-A); vd_params_default() fills the library's choices. */
typedef struct {
  float fisk_alpha0;        /* Fisk scale of the end-point error, px            */
  float fisk_alpha1;        /* scale growth per px of observed flow magnitude   */
  float fisk_beta;          /* Fisk shape (2 selects the fast closed form)      */
  float outlier_density;    /* P0, density of an outlier residual, 1/px^2       */
  float gamma_stay;         /* rigidness chain: probability to keep the state   */
  float rho_min, rho_max;   /* inverse-depth search range (same units as tau)   */
  int n_hyp;                /* K hypotheses per pixel per iteration (1..1024)   */
  int n_pose_samples;       /* S P3P samples per frame (1..256)                 */
  double pose_sigma_rot;        /* mean-shift kernel, rad                      */
  double pose_sigma_trans_rel;  /* mean-shift kernel, fraction of |tau|        */
  double pose_sigma_trans_abs;  /* mean-shift kernel, absolute translation     */
  int sample_share;         /* pixels of an aligned row segment sharing draws   */
  int hierarchical;         /* 1: hierarchical propagation (Sec. III-A)        */
  int hier_scale;           /* coarse grid step of the global pass, px          */
  int hier_window;          /* length of the local full-resolution windows, px  */
  float prior_c_sigma;      /* RGB-D prior: sigma = c_sigma * rho_hat (Eq. 3)   */
  float prior_w_uniform;    /* RGB-D prior: uniform density 1/(w rho_hat)       */
  unsigned long long seed;  /* key of every Philox4x32-10 draw                  */
} vd_params;

/* Statistics of the last vd_run_em. */
typedef struct {
  int iterations;           /* EM iterations run by the call                     */
  int bootstrapped;         /* 1 if the call ran the bootstrap                   */
  int degenerate_frames;    /* pose M-steps that kept their pose                 */
  double mean_energy;       /* mean per-pixel energy after the last depth step   */
  double rigid_fraction;    /* mean rigidness over all flows after the E-step    */
} vd_stats;

/* Fill *out with the default hyper-parameters.  Never fails for non-null out. */
vd_status vd_params_default(vd_params* out);

/* Create a context for windows of the given geometry; allocates all device
 * state (about 4 + 2N float32 maps plus pose scratch).  cuda_stream may be
 * NULL (the legacy default stream).  Errors: VD_ERR_ARG for sizes outside
 * 2..16384 px, N outside 1..8, non-positive focal lengths or parameters out of
 * range; VD_ERR_OOM / VD_ERR_CUDA. */
vd_status vd_create(const vd_window_desc* desc, const vd_params* params, void* cuda_stream,
                    vd_ctx** out);
vd_status vd_destroy(vd_ctx* ctx);
vd_status vd_set_stream(vd_ctx* ctx, void* cuda_stream);
vd_status vd_set_params(vd_ctx* ctx, const vd_params* params);

/* Push flow field t (1..N).  row_pitch_floats >= 2W is the distance between
 * rows in floats (2W for a dense array).  Non-finite values are rejected with
 * VD_ERR_ARG (the check synchronises the stream).  Pushing a flow invalidates
 * the EM state: the next vd_run_em bootstraps again. */
vd_status vd_push_flow(vd_ctx* ctx, int t, const float* uv, long row_pitch_floats, vd_mem mem);

/* Stereo prior of the reference frame (Sec. III-A "Geometric Priors", last
 * paragraph; Sec. IV): disparity in px of a rectified pair with the given
 * baseline, so rho_hat = d / (fx b).  NaN or d <= 0 marks a hole. */
vd_status vd_push_stereo_prior(vd_ctx* ctx, const float* disparity, double baseline_m, vd_mem mem);

/* RGB-D prior (Eq. 3): depth in the units of tau (0 or NaN = hole), optional
 * per-pixel confidence in [0, 1] (NULL = 1) that multiplies the prior's
 * rigidness weight (Eq. 6 paragraph).  T_hat (12 doubles) must be NULL or the
 * identity: the prior is given on the reference frame's grid. */
vd_status vd_push_depth_prior(vd_ctx* ctx, const float* depth, const float* confidence,
                              const double* T_hat, vd_mem mem);
vd_status vd_clear_prior(vd_ctx* ctx);

/* Poses G (N+1 x 12, kind ABSOLUTE, G_0 must be the identity) or T (N x 12,
 * kind RELATIVE).  Setting poses skips the pose part of the bootstrap. */
vd_status vd_set_poses(vd_ctx* ctx, const double* poses, vd_pose_kind kind);
vd_status vd_get_poses(vd_ctx* ctx, double* poses_out, vd_pose_kind kind);

/* Set the EM state: inverse depth rho (H*W, > 0), rigidness q (N*H*W, NULL =
 * all 1) and prior rigidness q_hat (H*W, NULL = all 1).  Marks the context as
 * bootstrapped. */
vd_status vd_set_state(vd_ctx* ctx, const float* rho, const float* q, const float* q_hat,
                       vd_mem mem);

/* Bootstrap (Sec. I, III-A): with a prior, rho from the prior and one pose
 * M-step; monocular, 8-point G_1 (|tau_1| = 1), random rho, a depth M-step on
 * X_1 and one pose M-step.  Poses set with vd_set_poses are kept. */
vd_status vd_bootstrap(vd_ctx* ctx);

/* Run n_iters EM iterations (bootstrapping first if needed).  Iteration i of
 * the context (counted across calls) sweeps chain direction i mod 4
 * (0 L->R, 1 T->B, 2 R->L, 3 B->T).  Synchronises; returns VD_WARN_DEGENERATE
 * if any pose step kept its pose.  stats may be NULL. */
vd_status vd_run_em(vd_ctx* ctx, int n_iters, vd_stats* stats);

/* Single steps (for staged use and testing).  `iter` selects the random
 * streams (-1 = the bootstrap streams) and `direction` the chains.  On a
 * context without a prior, vd_depth_mstep with iter = -1 is the monocular
 * bootstrap's depth step: it weighs X_1 alone (the other flows' rigidness is
 * not read), exactly as vd_bootstrap does. */
vd_status vd_depth_mstep(vd_ctx* ctx, int iter, int direction);
vd_status vd_rigidness_estep(vd_ctx* ctx, int direction);
/* Pose M-step of frame t (1..N), or of every frame in order for t = 0. */
vd_status vd_pose_mstep(vd_ctx* ctx, int iter, int t);

/* Results.  Host outputs are written after a stream synchronisation. */
vd_status vd_get_inv_depth(vd_ctx* ctx, float* out, vd_mem mem);
vd_status vd_get_rigidness(vd_ctx* ctx, float* out, vd_mem mem);          /* N*H*W */
vd_status vd_get_prior_rigidness(vd_ctx* ctx, float* out, vd_mem mem);    /* H*W   */
vd_status vd_get_confidence(vd_ctx* ctx, float* out, vd_mem mem);         /* Eq. 6 */
/* rho* and E* of the last depth M-step before propagation (H*W each). */
vd_status vd_get_depth_candidates(vd_ctx* ctx, float* rho_star, float* e_star, vd_mem mem);
/* Energy E_j(rho_j) of every pixel for the given inverse-depth map under the
 * current state (Eq. 5 criterion; H*W in, H*W out). */
vd_status vd_eval_energy(vd_ctx* ctx, const float* rho, float* energy_out, vd_mem mem);

/* Per-sample results of the last pose M-step of a frame: the kept root of
 * every sample (S x 12, absolute), its energy (S; +inf for a void sample) and
 * the rigid-set size.  Host memory. */
vd_status vd_get_pose_samples(vd_ctx* ctx, double* poses, double* energies, int* n_rigid);

/* Dense pose scoring (Eq. 7 scoring step) as a standalone call on device
 * buffers: for every pose m (poses: m x 12 float64, absolute) computes
 *   E_m = sum_i w_i l(| obs_i - pi(K (R_m X_i + tau_m)) |)
 * with points[i] = (X, Y, Z, w) and obs[i] = (x, y, alpha, unused) as float4,
 * l the Fisk maximum-inlier energy with shape beta and outlier density p0,
 * and a large constant for points behind the camera.  energies: m float64.
 * Allocates its own scratch for the block partial sums; runs on cuda_stream
 * and synchronises it.  n >= 0 (points and obs may be NULL when n = 0, which
 * gives zero energies), 1 <= m <= 1024. */
vd_status vd_score_poses(const float* points, const float* obs, int n, const double* poses, int m,
                         const double* intrinsics, float beta, float p0, double* energies,
                         void* cuda_stream);

/* Stage profiling (tracing): CUDA events recorded on the context stream
 * around every stage, and kernel launch counters.  Stages: 0 depth sampling
 * (hypotheses + argmin), 1 depth propagation, 2 rigidness E-step, 3 rigid-set
 * compaction, 4 P3P sampling, 5 dense pose scoring, 6 sample selection and
 * mean-shift, 7 bootstrap and other work.  Enabling resets the counters;
 * vd_get_profile synchronises the stream. */
#define VD_N_STAGES 8
typedef struct {
  double ms[VD_N_STAGES];           /* summed event time per stage           */
  long long calls[VD_N_STAGES];     /* stage executions                      */
  long long launches[VD_N_STAGES];  /* kernel launches per stage             */
  long long total_launches;
  long long score_evals;            /* (rigid pixel, root) pairs scored by the
                                       pose M-steps since profiling was enabled
                                       (counted by the device, profiling on or off) */
} vd_profile;
vd_status vd_profile_enable(vd_ctx* ctx, int enable);
vd_status vd_get_profile(vd_ctx* ctx, vd_profile* out);

/* Dense pose scoring without any device allocation.  The paper has no
 * counterpart; this is a library convenience for callers that may not
 * allocate device memory at run time -- for example a host whose device memory
 * is entirely reserved by another allocator, or a real-time loop where a
 * cudaMalloc (which can synchronise the device and can fail under memory
 * pressure) is not allowed.  Same arguments and result as vd_score_poses, but
 * the block partial sums live in a fixed array of the library's device code
 * (VD_NOALLOC_MAX_POSES x (12 + 512) floats, about 0.5 MB, held by every GPU
 * that loads the library until the process exits).
 *   - m must be in 1..VD_NOALLOC_MAX_POSES, else VD_ERR_ARG (see vd_last_error);
 *     n = 0 gives zero energies.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address and the device's SM count with host-side CUDA
 *     queries.  The address is kept for the life of the process: after a
 *     cudaDeviceReset of that device it is stale, and the call must not be
 *     used again in that process.
 *   - All calls share the one array: calls that may overlap on the GPU (other
 *     streams, other host threads) race and must be serialised by the caller.
 *     Every scratch value a call reads is written earlier in the same call.
 *   - Runs on cuda_stream and synchronises it. */
#define VD_NOALLOC_MAX_POSES 256
vd_status vd_score_poses_noalloc(const float* points, const float* obs, int n,
                                 const double* poses, int m, const double* intrinsics,
                                 float beta, float p0, double* energies, void* cuda_stream);

/* ---- Launch tuning (the paper has none: GPU launch shapes) ---------------
 * Three launch shapes are tunable per context: the warps per block of the
 * depth-sampling kernel (1, 2 or 4; default 4), and the threads per block
 * (256 or 512; default 256) and the blocks setting b (1..4; default 2) of
 * the dense pose scoring, which launches b x SMs / 2 blocks of rigid pixels
 * for every group of 32 roots.  None changes any result bit except the
 * float32 summation
 * grouping of the pose scores (a rounding-level change).  vd_autotune times
 * every variant on this window and keeps the fastest: it needs all flows
 * pushed, and it OVERWRITES the EM state (it runs the bootstrap and one
 * iteration to reach a representative state), so call it before
 * vd_bootstrap.  Synchronises the stream. */
typedef struct {
  int k1_warps;                 /* 1, 2 or 4                                  */
  int score_threads;            /* 256 or 512                                 */
  int score_blocks_per_sm;      /* 1..4 (pixel blocks: this x SMs / 2)        */
  float k1_ms[3];               /* measured, for 1, 2, 4 warps (0 if unset)   */
  float score_ms[2][4];         /* measured, [256, 512 threads][1..4 per SM]  */
} vd_tune;
vd_status vd_autotune(vd_ctx* ctx, vd_tune* out /* nullable */);
vd_status vd_set_tune(vd_ctx* ctx, const vd_tune* tune);
vd_status vd_get_tune(vd_ctx* ctx, vd_tune* out);

/* ---- Batched EM over many windows (the paper has no counterpart: it runs
 * one window at a time; a server or an offline job runs many) ------------
 * A batch owns n independent windows (each its own vd_ctx, of its own size,
 * N and parameters).  vd_batch_run runs the bootstrap (if asked) and
 * n_iters EM iterations of every window as ONE CUDA graph: each window's
 * kernel sequence is one branch, forked from and joined to the batch stream,
 * so the latency-bound pose kernels of one window overlap the others' work.
 * Each window's results are bit-identical to vd_bootstrap + vd_run_em on
 * that window alone (same kernels, same order, same inputs).
 *   - descs/params: n entries each; params may be NULL (defaults) or point
 *     at one vd_params shared by all windows (params_stride = 0) or at n of
 *     them (params_stride = 1).
 *   - vd_batch_window gives window i's context for the per-window calls
 *     (push flows and priors, set poses, read results).  Those calls run on
 *     the batch stream; vd_set_stream on a window context is refused.
 *   - The graph is captured on the first run and replayed while every
 *     window starts from the same state as at capture (iteration counter,
 *     bootstrap flag, prior kind, poses set, parameters, tuning); otherwise it
 *     is captured again (vd_batch_stats counts captures).
 *   - flags: VD_BATCH_BOOTSTRAP re-bootstraps every window first (a new
 *     batch of flows); VD_BATCH_AUTOTUNE (with BOOTSTRAP) first tunes one
 *     window of every distinct (size, N, K, S, prior) and gives its choice to
 *     the others, then times whole-batch runs (bootstrap and up to two
 *     iterations) of every pose-scoring shape that was within 25 % of the
 *     best alone for every group and gives the fastest to every window
 *     (the windows' kernels share the SMs; the trials' results are replaced
 *     by the run itself).
 *   - degenerate: optional int[n] receiving each window's count of frames
 *     whose pose step kept the previous pose; the status is
 *     VD_WARN_DEGENERATE if any is non-zero.
 *   - Synchronises the batch stream. */
typedef struct vd_batch vd_batch;
#define VD_BATCH_BOOTSTRAP 1
#define VD_BATCH_AUTOTUNE 2
typedef struct {
  int windows;
  long long captures;           /* graph captures so far                     */
  long long replays;            /* runs that reused the captured graph       */
  long long graph_nodes;        /* nodes of the current graph                */
  long long kernels_per_run;    /* kernel launches one run performs          */
} vd_batch_stats;
vd_status vd_batch_create(int n, const vd_window_desc* descs, const vd_params* params,
                          int params_stride, void* cuda_stream, vd_batch** out);
vd_status vd_batch_destroy(vd_batch* b);
vd_status vd_batch_window(vd_batch* b, int i, vd_ctx** out);
vd_status vd_batch_run(vd_batch* b, int n_iters, int flags, int* degenerate);
vd_status vd_batch_get_stats(vd_batch* b, vd_batch_stats* out);

/* ---- Learned initialiser (the paper has none: every window starts from its
 * bootstrap there) -------------------------------------------------------
 * A convolutional network maps a window's flows to an initial inverse depth
 * and rigidness, to start the EM closer to its fixed point.  Six 3x3
 * convolutions, zero padding 1: C0 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 + N,
 * ReLU between layers; C0 = 16 if 2N + 4 <= 16, else 32.  Input planes, all
 * divided by 32 px: 2t + c is component c of flow t+1; then four geometry
 * planes from the pose T_1 of flow 1 (unit translation, the monocular
 * gauge): the flow the rotation of T_1 alone gives the pixel (2 planes), and
 * the extra flow of a point at inverse depth 0.1 under the whole T_1 (2
 * planes); the rest zero (the geometry planes too when no pose is given).
 * Heads: rho = clip(rho_c exp(z_0), rho_min, rho_max) with rho_c =
 * sqrt(rho_min rho_max), and the rigidness of flow t, q_t = sigmoid(z_t).
 * Weights and activations are bfloat16 with float32 accumulation on the
 * tensor cores; the master parameters are float32.
 * Parameter vector (vd_cnn_layout gives the offsets): for each layer l the
 * weights W_l[c_out][ky][kx][c_in] then the biases b_l[c_out].
 * Training (vd_cnn_train_step): loss over pixels with mask m,
 *   L = sum m (z_0 + log rho_c - log rho*)^2 / sum m
 *     + w_q sum_t sum m BCE(q_t, q*_t) / (N sum m),
 * gradients with dL/dz of every layer stored in bfloat16, then one Adam
 * step (b1 0.9, b2 0.999, eps 1e-8) when `update` is set.
 * All image buffers are device memory: flow [N][H][W][2] float32 (the layout
 * of vd_push_flow), inverse depth and mask [H][W], rigidness [N][H][W].
 * Calls run on `stream` and synchronise it;
 * a tensor-core wait that gives up returns VD_ERR_TIMEOUT. */
typedef struct vd_cnn vd_cnn;
#define VD_CNN_LAYERS 6
/* Self-test of the failure path of the tensor-core kernels' waits: one
 * thread waits on an mbarrier that nothing completes, with the bounded wait
 * the convolution's roles use (`polls` polls, 1..2^20), gives up, sets the
 * error flag and returns; the host reads the flag.  Returns VD_ERR_TIMEOUT,
 * the status of a convolution whose wait ran out (VD_ERR_ARG for polls out
 * of range); the device stays usable.  Synchronises `cuda_stream`. */
vd_status vd_check_bounded_wait(int polls, void* cuda_stream);

/* ---- Pipe throughput probes (measurement; the paper has none) ------------
 * Launch `blocks` blocks of 256 threads that run only independent chains of
 * FP32 fused multiply-adds (VD_PROBE_FP32) or of MUFU log2 operations
 * (VD_PROBE_MUFU), `iters` x 128 per thread, on cuda_stream, without
 * synchronising; *ops_out receives the number of thread-level operations
 * launched.  Timed with CUDA events around the call, ops / time is the
 * pipe's measured throughput, the denominator of the roofline fractions of
 * the depth sampling and pose scoring kernels.  blocks and iters in
 * 1..2^20, else VD_ERR_ARG. */
#define VD_PROBE_FP32 0
#define VD_PROBE_MUFU 1
vd_status vd_probe_pipe(int kind, int blocks, int iters, double* ops_out, void* cuda_stream);

/* ---- Checked build (the library's stand-in for a memory checker; the
 * paper has none) ----------------------------------------------------------
 * Built with -DVD_CHECKED, the library checks every index its kernels form
 * from data (bilinear taps of the flow, the P3P picks and their taps, the
 * rigid-set scatter, chain pixels, coverage cells) against its buffer,
 * records the first out-of-range one and clamps it into range (the access
 * stays inside the buffer; the results are then wrong).  out[5]: out[0]
 * the site of the first such index (0: none; 1 bilinear taps, 2 P3P taps,
 * 3 scatter, 4 P3P picks, 5 coverage cells, 6 chain pixels), out[1] the
 * index, out[2] its bound, out[3] how many were seen since the last report,
 * out[4] 1 in the checked build, 0 otherwise.  Clears the records; reads
 * device memory (synchronous). */
vd_status vd_check_report(long long* out);
typedef struct {
  double fx, fy, cx, cy;    /* intrinsics of the window                     */
  double T1[12];            /* pose of flow 1, [R | tau] row-major           */
} vd_cnn_geometry;
vd_status vd_cnn_create(int n_flows, unsigned long long seed, vd_cnn** out);
vd_status vd_cnn_destroy(vd_cnn* net);
vd_status vd_cnn_layout(vd_cnn* net, int* n_params, int* c_in /*[6]*/, int* c_out /*[6]*/,
                        long* w_offset /*[6]*/, long* b_offset /*[6]*/);
vd_status vd_cnn_get_params(vd_cnn* net, float* params /*host [n_params]*/);
vd_status vd_cnn_set_params(vd_cnn* net, const float* params /*host*/);   /* resets Adam */
vd_status vd_cnn_get_grads(vd_cnn* net, float* grads /*host [n_params]*/);
vd_status vd_cnn_forward(vd_cnn* net, const float* flow, int width, int height,
                         const vd_cnn_geometry* geom /*nullable*/, float rho_min, float rho_max,
                         float* rho_out /*nullable*/, float* q_out /*nullable*/,
                         void* cuda_stream);
/* Activations of the last forward pass, as float32 on the host: layer l in
 * 0..5 is the input a_l of layer l, [H][W][C_in(l)]; layer 6 is z of the
 * last layer, [H][W][16] (the first 1 + N channels used). */
vd_status vd_cnn_get_activation(vd_cnn* net, int layer, float* out, int width, int height);
vd_status vd_cnn_train_step(vd_cnn* net, const float* flow, int width, int height,
                            const vd_cnn_geometry* geom /*nullable*/, const float* rho_target,
                            const float* q_target, const unsigned char* mask, float rho_min,
                            float rho_max, float w_q, float lr, int update,
                            double* loss_out /*host, nullable*/, void* cuda_stream);
/* The monocular bootstrap's pose of flow 1 (IRLS 8-point on X_1, unit
 * translation), computed without changing the context's state: the geometry
 * a network is trained with.  Needs X_1 pushed.  Synchronises the stream. */
vd_status vd_eight_point(vd_ctx* ctx, double* T1_out /*host, 12*/);
/* Bootstrap a context with the network: vd_bootstrap with the network's
 * inverse depth (geometry planes from the 8-point pose, or from the poses
 * set on the context; within [rho_min, rho_max]) as the initial value of the
 * monocular depth step, in place of the random draw; the rest as in
 * vd_bootstrap (q = 1; with a prior, exactly vd_bootstrap).  The network's
 * rigidness is not used here (vd_cnn_forward gives it).  The network must
 * have the context's N. */
vd_status vd_bootstrap_learned(vd_ctx* ctx, vd_cnn* net);

/* ---- Pose covariance ----------------------------------------------------
 * Sec. III-A "Uncertainty-aware Pose Estimation": the uncertainty of each
 * camera pose from the samples of the last pose M-step (the kept root of
 * every sample with one).  Starting from the mean-shift mode and the robust
 * diagonal covariance diag((1.4826 median_g |d_gi|)^2) of the samples there,
 * rounds of: the samples within 3 sigma (d^T Sigma^-1 d <= 9 with
 * d = log(mean^-1 T) in se(3), rotation vector first), their Frechet mean,
 * and the maximum-likelihood covariance of their d at that mean with every
 * eigenvalue raised to eps; until the inlier set repeats (at most 50
 * rounds).  Fewer than 7 samples or inliers leave the frame degenerate with
 * its last fit (the mode and eps I without samples).  float64. */
typedef struct {
  double mean[12];   /* fitted mean pose (absolute, reference -> frame), 3x4 row-major */
  double cov[36];    /* 6x6 row-major, tangent space at the mean                         */
  int n_samples;     /* samples with a root                                             */
  int n_inliers;     /* inliers of the last round                                       */
  int rounds;
  int degenerate;
} vd_pose_cov;
/* out: N entries, frame t at out[t-1].  Needs a pose M-step of every frame
 * since the last vd_bootstrap, vd_set_poses, vd_set_state or
 * vd_import_state (VD_ERR_STATE otherwise).  Synchronises the context
 * stream. */
vd_status vd_pose_covariance(vd_ctx* ctx, double eps, vd_pose_cov* out);
/* The samples of frame t's last pose M-step (S x 12 absolute poses, S
 * energies, +inf for a sample without a root).  Host memory. */
vd_status vd_get_frame_samples(vd_ctx* ctx, int t, double* poses, double* energies);

/* ---- Keyframe alignment --------------------------------------------------
 * Sec. III-C "Keyframe Alignment", Eq. 9-12: the motion T and scale s of
 * two keyframes' depth maps theta_1, theta_2 (depth, not inverse depth;
 * same size and intrinsics) minimising
 *   E = sum_j C^j psi(<n_l, s theta_1^l r_l - P_j> / (s theta_1^l P_jz)),
 * P_j = R theta_2^j r_j + t (keyframe 2's pixel j in keyframe-1
 * coordinates), l the nearest pixel of its projection into keyframe 1
 * (a pair counts when |P_jz - s theta_1^l| <= 0.2 s theta_1^l: occlusions),
 * r = ((u - cx)/fx, (v - cy)/fy, 1), n_l the normal of depth map 1 (central
 * differences of its points, towards the camera; none at the border, next
 * to an invalid depth, or where a second difference of the points exceeds
 * 0.2 of the central span: a depth edge or fold), psi(r) = (c^2/2)
 * log(1 + r^2/c^2),
 * C^j keyframe 2's confidence (1 without a map).  Valid depth: finite, > 0.
 * Levenberg-Marquardt on a left increment of T in se(3) and log s (s fixed
 * at 1 with fix_scale): the step solves (H + lambda diag H) delta = -g with
 * H = sum w J J^T, g = sum w J r, w = C / (1 + r^2/c^2); taken when it
 * lowers E (lambda /= 10), refused otherwise (lambda *= 10); lambda starts at
 * 1e-3; stop after max_iters steps, a step below 1e-10, or lambda > 1e10.
 * cov = the pose block of H^-1 (rotation first), NaN without a pixel.
 * Device buffers; float64 arithmetic.  Synchronises the stream. */
typedef struct {
  double pose[12];   /* T; in: start, 3x4 keyframe-2 -> keyframe-1; out: estimate */
  double s;          /* in: start (> 0); out: estimate                          */
  double cauchy_c;   /* Cauchy kernel scale c (inverse-depth units, > 0)        */
  int fix_scale;     /* 1: s = 1 (depth of absolute scale)                      */
  int max_iters;     /* Levenberg-Marquardt steps at most (>= 0)                */
  double cov[36];    /* out: 6x6 row-major                                      */
  double energy;     /* out: E at the estimate                                  */
  int iterations;    /* out                                                     */
  long long n_valid; /* out: associated pixels at the estimate                  */
} vd_ka;
vd_status vd_ka_align(const float* depth1, const float* depth2, const float* conf2 /*nullable*/,
                      int width, int height, const double* intrinsics /*fx fy cx cy*/, vd_ka* io,
                      void* cuda_stream);

/* ---- Visibility-coverage score, VO stride and keyframe test ------------
 * Sec. III-B "VO Stride and Keyframe Selection", Eq. 8.  The reference
 * frame's depth pixels (finite rho > 0 of the context's current inverse
 * depth) are projected into a frame of known pose T = [R | tau] (reference
 * -> frame, 3x4 row-major): with r = ((u - cx)/fx, (v - cy)/fy, 1) and
 * h = R r + rho tau, the point is in front when h_z > 1e-6 and lands at
 * x = fx h_x/h_z + cx, y = fy h_y/h_z + cy; it is visible when in front and
 * 0 <= x <= W-1, 0 <= y <= H-1, and covers the pixel cell
 * (floor(x + 1/2), floor(y + 1/2)).  The projections are taken in float32,
 * one rounding per operation in the order written (R, tau and the
 * intrinsics rounded to float32 once), so the counts are exact integers.
 * visibility = n_visible / n_depth (0 without depth pixels), coverage =
 * n_covered / n_pixels, vc = 2 V C / (V + C) (0 when either is 0). */
#define VD_VC_MAX_FRAMES 8
typedef struct {
  int n_frames;                              /* entries filled                 */
  long long n_pixels;                        /* W * H                          */
  long long n_depth;                         /* depth pixels                   */
  long long n_visible[VD_VC_MAX_FRAMES];     /* depth pixels inside frame k    */
  long long n_covered[VD_VC_MAX_FRAMES];     /* pixel cells of frame k covered */
  double visibility[VD_VC_MAX_FRAMES];
  double coverage[VD_VC_MAX_FRAMES];
  double vc[VD_VC_MAX_FRAMES];
} vd_vc;
/* The reference depth in every frame t = 1..N of the window (entry t-1, the
 * context's current poses).  Synchronises the context stream. */
vd_status vd_vc_scores(vd_ctx* ctx, vd_vc* out);
/* The reference depth in one frame of pose T (host, 12 doubles, reference ->
 * frame): the keyframe test, with T the latest keyframe's pose relative to
 * the reference frame.  Entry 0.  Synchronises the context stream. */
vd_status vd_vc_pose(vd_ctx* ctx, const double* T, vd_vc* out);
/* Host rules.  The next batch's reference: the first t (1-based) with
 * vc[t-1] < tau_stride, n when there is none (0 for n < 1 or no vc).  The
 * reference frame becomes a keyframe when its VC with the latest keyframe
 * is below tau_keyframe (1) or not (0). */
int vd_vc_stride(const double* vc, int n, double tau_stride);
int vd_vc_is_keyframe(double vc, double tau_keyframe);

/* State export/import for checkpoint and resume: a self-describing blob with
 * rho, q, q_hat, C, the poses, the iteration counter and the bootstrap flag.
 * Call export with blob = NULL to learn the size. */
vd_status vd_export_state(vd_ctx* ctx, void* blob, size_t* bytes);
vd_status vd_import_state(vd_ctx* ctx, const void* blob, size_t bytes);

const char* vd_status_str(vd_status s);
const char* vd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VOLDOR_EM_H */
