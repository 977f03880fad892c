/*
 * epo.h -- C ABI of the GB300 (sm_103a) edge-alignment library.
 *
 * The library evaluates EPO's multi-view edge-alignment objective (Section 3,
 * "Edge Reprojection Loss", Eqs. 6-8) and its 6-DoF gradient with respect to
 * every camera pose, and runs the pose-only optimisation loop of Algorithm 2
 * (with the clamp anneal and batched residuals of Algorithm 3) entirely on
 * one GPU.  Everything here is plain C: pointers, sizes and status codes; no
 * exception crosses this boundary and the library never exits or traps.
 *
 * Conventions used by every entry point
 *   - Pose T_i = [R_i | t_i] maps world -> camera i (the extrinsic P_i of
 *     Section 3, Eq. 1), row-major 3x4, 12 doubles per view.
 *   - Pixel centres at integer coordinates; depth is z-depth; K_i given as
 *     (fx, fy, cx, cy).
 *   - Edge record of view i: (u, v, z) = pixel of an edge in E_i and its
 *     predicted depth Z_i(u, v).  EPO_F32 records are 16 bytes
 *     {float u, float v, float z, float 0}; EPO_F16 records are 8 bytes
 *     {uint16 u, uint16 v, half z, uint16 0}.
 *   - Map of view j: its distance transform field DTF_j (Section 3), H rows
 *     of W values, row-major, dense; EPO_F32 (float) or EPO_BF16.
 *   - Pairs: directed (i -> j) index pairs into the view array; the loss is
 *     L = (2/P) sum_p l_p with l_p the per-direction mean of Eq. 7, which is
 *     Eq. 6 when every undirected pair is listed in both directions.
 *   - Gradients are with respect to a left perturbation T <- Exp(xi) T,
 *     xi = (upsilon, omega) (translation first), 6 doubles per view.
 *   - A projected sample is valid iff its camera-j depth exceeds eps_z and
 *     it lands in [0, W-1] x [0, H-1]; invalid samples do not count in the
 *     per-direction mean (Algorithm 3, sum(rho) / sum(valid)).
 *
 * Streams and ownership
 *   - Every call is ordered on the CUDA stream given at creation (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Calls with host outputs synchronise that stream before returning;
 *     calls suffixed _dev take device pointers and do not synchronise.
 *   - A scene handle is not thread-safe: one host thread at a time.
 *   - epo_create_* copy every input into library-owned device memory; the
 *     caller may free its buffers as soon as the call returns.  A scene without
 *     focal or depth refinement also keeps every record lifted to its camera
 *     frame (16 bytes per record, computed once in double precision), since its
 *     intrinsics and depths do not change; device_bytes counts it.
 */
#ifndef EPO_H
#define EPO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPO_ABI_VERSION 4

typedef enum {
  EPO_OK = 0,
  EPO_ERR_INVALID_ARG = 1, /* bad sizes, indices, pointers, dtypes or non-finite maps */
  EPO_ERR_CUDA = 2,        /* a CUDA runtime call failed; see epo_last_error */
  EPO_ERR_OOM = 3,         /* device allocation failed */
  EPO_ERR_NUMERIC = 4,     /* non-finite loss or gradient; the pose update was refused */
  EPO_ERR_TIMEOUT = 5,     /* a bounded wait ran out */
  EPO_ERR_INTERNAL = 6,    /* a device-side consistency check failed: in builds with
                              EPO_DEBUG_BOUNDS, a gather cell outside its map (the sample is
                              skipped, the poses are not updated; the message names the
                              first offending pair and cell) */
  EPO_ERR_TOO_LARGE = 7    /* the problem exceeds a fixed capacity (epo_loss_and_grad_noalloc) */
} epo_status;

enum { EPO_F32 = 0, EPO_F16 = 1, EPO_BF16 = 2 };
/* Pose parameterisation: direct SE(3) parameters or the paper's pose MLP (Eq. 3). */
enum { EPO_POSE_SE3 = 0, EPO_POSE_MLP = 1 };
/* Parameters of one scene's pose MLP (12 -> 128 x 5 -> 12), in the order W1 (128x12, row-major
 * [out][in]), b1, W2..W5 (128x128), b2..b5, W6 (12x128), b6. */
#define EPO_POSE_MLP_PARAMS 69260
/* Per-direction normaliser: sum(valid) (Algorithm 3) or |E_i| (Eq. 7). */
enum { EPO_NORM_VALID = 0, EPO_NORM_ALL = 1 };
/* How the kernels read the 2x2 map footprint: plain loads, texture gather, or (pose-only
 * scenes, two or more records per thread) the two side by side: of the two samples a thread
 * has in flight, one through each path. */
enum { EPO_GATHER_AUTO = 0, EPO_GATHER_LDG = 1, EPO_GATHER_TEX = 2, EPO_GATHER_MIX = 3 };

typedef struct epo_scene* epo_scene_t;

/* One view: intrinsics K_i, its edge records (E_i with depth Z_i) and its
 * distance transform field DTF_i (Eq. 1 augmented as in Section 3). */
typedef struct {
  int32_t W, H;              /* map size; both >= 2 */
  double fx, fy, cx, cy;     /* pinhole intrinsics, fx, fy > 0 */
  const void* records;       /* n_records records of the scene's record dtype */
  int64_t n_records;         /* >= 0 */
  const void* map;           /* W*H values of the scene's map dtype, finite, >= 0 */
} epo_view_desc;

/* One scene: the views, the directed viewgraph E (Section 3, "Viewgraph
 * Estimation"; here supplied by the caller) and the gauge mask. */
typedef struct {
  int32_t n_views;           /* >= 1 */
  const epo_view_desc* views;
  int32_t n_pairs;           /* >= 1 */
  const int32_t* pairs;      /* 2*n_pairs ints: (i, j) per directed pair, i == j allowed;
                                at most 512 pairs share one source view */
  const uint8_t* fixed;      /* n_views bytes, 1 = pose frozen by epo_step; NULL = none */
  int32_t record_dtype;      /* EPO_F32 | EPO_F16 */
  int32_t map_dtype;         /* EPO_F32 | EPO_BF16 */
  int32_t pointers_on_device;/* 0: records/map are host pointers, 1: device pointers */
} epo_scene_desc;

/* Hyper-parameters (Section 3 "Implementation Details", Algorithm 3). */
typedef struct {
  double huber_delta;        /* Huber threshold (paper silent; default 1 px) */
  double lambda0, lambda1;   /* clamp anneal lambda0 -> lambda1 (Algorithm 3: 10 -> 6) */
  int32_t lambda_steps;      /* over this many steps, linear, then held (default 1000) */
  double eps_z;              /* minimum camera-j depth of a valid sample (default 1e-6) */
  int32_t norm_mode;         /* EPO_NORM_VALID | EPO_NORM_ALL */
  double lr_rot, lr_trans;   /* Adam step sizes for omega and upsilon */
  double beta1, beta2, adam_eps; /* Adam moments (Section 3: 0.9, 0.999) */
  int32_t autotune;          /* 1: pick the kernel schedule by timing on first use;
                                2: the same, each timed launch starting from a cold L2 */
  int32_t gather;            /* EPO_GATHER_* (AUTO = LDG unless autotuned) */
  int32_t block_threads;     /* 0 = default (256); else 64..512, multiple of 32 */
  int32_t records_per_thread;/* 0 = default (2); 1, 2, 4 or 8 (two in flight at a time;
                                refine scenes: 2) */
  int32_t grid_blocks;       /* 0 = default (persistent: SMs x resident blocks) */
  int32_t timing;            /* 1: bracket the edge kernel with CUDA events (epo_kernel_time) */
  int32_t tail_pairs;        /* work items of the last wave (as many as the grid has blocks):
                                0 = each covers all of its view's pairs, like the others;
                                n > 0 = split into items of at most n pairs, so that the
                                blocks finish together; -1 = default (autotuned when
                                autotune is on, else 0); n <= -2 = every work item, not
                                only the last wave's, covers at most -n pairs */
  int32_t refine;            /* 1: the scene also carries the focal and depth refinement of
                                Section 3 (Eq. 4: f_i = f_i^0 (1 + gamma_i) for both focal
                                lengths of view i; Eq. 5: every edge pixel's depth is
                                Z^0 alpha + beta), set by epo_set_refinement and used by every
                                evaluation and step; two records per thread */
  int32_t pair_budget;       /* M of Algorithm 3 (Appendix A.3): when a scene has more
                                pairs, every evaluation and step uses a fresh uniform random
                                subset of M of them, drawn on the device from the step
                                counter; 0 = every pair */
  uint64_t subsample_seed;   /* seed of the subset draws (SplitMix64 keys of (seed, step, pair)) */
  double sched_eps1, sched_eps2; /* Optimization Schedule (Section 3): thresholds in degrees */
  int32_t schedule;          /* 1: after every step, theta_95 = max of the 95th percentiles over
                                the scene's poses of the rotation and translation-direction
                                changes; phase 1 ends after sched_w1 consecutive steps with
                                theta_95 < sched_eps1, phase 2 (the run) after sched_w2 steps
                                below sched_eps2, and a converged scene's poses stop changing */
  int32_t sched_w1, sched_w2; /* window sizes (defaults: the paper's 25 / 50 and 0.5 / 0.1) */
  double lr_focal;           /* refine scenes: Adam step size of gamma (Eq. 4), applied by every
                                epo_step with the pose update; 0 (default) keeps gamma */
  double lr_depth;           /* refine scenes: Adam step size of alpha and beta (Eq. 5); > 0 adds
                                the depth kernel to every step (dL/dz per edge pixel from the
                                fused pass's per-sample derivatives, then Adam).  The depth
                                module steps only in phase 2 of the schedule (Algorithm 2) when
                                options.schedule is on, else from the first step; its Adam bias
                                correction counts its own steps.  0 (default) keeps alpha, beta */
  int32_t pose_param;        /* EPO_POSE_SE3 (default): each pose is its own parameter, Adam in
                                the tangent space; EPO_POSE_MLP: the paper's parameterisation
                                (Section 3, Pose Refinement, Eq. 3), P_i = phi(P_i^0 + MLP(P_i^0))
                                + [0 | delta_i] with one MLP per scene (set by epo_set_pose_mlp)
                                and AdamW; every view moves (fixed is not used) */
  double mlp_lr;             /* peak learning rate of the MLP and delta (default 3e-3) */
  int32_t mlp_warmup;        /* linear warm-up steps (default 25): step s < warmup uses
                                (s + 1) / warmup of mlp_lr */
  int32_t mlp_steps;         /* then cosine decay, reaching 0 at step mlp_steps - 1 (default 2000) */
  double mlp_wd, mlp_wd_delta; /* AdamW weight decay of the MLP and of delta (0.01, 0.1) */
  double mlp_eps;            /* AdamW epsilon (default 1e-8) */
} epo_options;

/* Per-scene facts, filled by epo_scene_info. */
typedef struct {
  int32_t n_scenes, n_views, n_pairs;
  int64_t n_records;         /* records kept on the device (all scenes) */
  int64_t n_dropped;         /* records dropped at creation (z <= 0 or non-finite) */
  int64_t evals_per_step;    /* sum over pairs of |E_i| : edge-pixel x pair evaluations (with a
                                pair budget: the expected number, min(1, M / P_s) of each pair's) */
  int64_t device_bytes;      /* library-owned device memory */
  int64_t record_bytes, map_bytes;
  int32_t n_tiles;           /* work items of the persistent kernels */
  int32_t gather, block_threads, records_per_thread, grid_blocks; /* schedule in use */
  int32_t kernels_per_step;  /* kernel launches in one epo_step */
  int32_t tail_pairs;        /* pairs per work item of the last wave (0 = not split; a
                                negative n: every work item covers at most -n pairs) */
} epo_scene_info;

/* Defaults: delta 1, lambda 10 -> 6 over 1000 steps, eps_z 1e-6, NORM_VALID,
 * lr_rot 2e-3, lr_trans 2e-2, beta (0.9, 0.999), adam_eps 1e-12, no autotune. */
void epo_default_options(epo_options* opts);

int32_t epo_abi_version(void);

/* Build one scene (Algorithm 1's products: E_i, DTF_i, the viewgraph).
 * Copies everything to the device.  Records with z <= 0 or non-finite are
 * dropped and counted; maps with a non-finite or negative value, W or H < 2,
 * pair indices out of range or unknown dtypes give EPO_ERR_INVALID_ARG.
 * Poses start at identity; set them with epo_set_poses. */
epo_status epo_create_scene(const epo_scene_desc* desc, const epo_options* opts, void* cuda_stream,
                            epo_scene_t* out);

/* Several independent scenes of uneven sizes in one handle: one persistent
 * launch evaluates all of them (the batching of Algorithm 3 extended across
 * scenes).  Views and poses of scene s follow those of scene s-1; the loss
 * is reported per scene. */
epo_status epo_create_batch(int32_t n_scenes, const epo_scene_desc* descs, const epo_options* opts,
                            void* cuda_stream, epo_scene_t* out);

void epo_destroy_scene(epo_scene_t scene);

/* Detail of the last failure on this handle (or of the last failed create
 * when scene is NULL).  Valid until the next call on the handle. */
const char* epo_last_error(epo_scene_t scene);

epo_status epo_scene_info_get(epo_scene_t scene, epo_scene_info* info);

/* Poses, n_views x 12 doubles (host).  set: synchronous copy; get: syncs. */
epo_status epo_set_poses(epo_scene_t scene, const double* T);
epo_status epo_get_poses(epo_scene_t scene, double* T);
/* Same with device pointers, stream-ordered. */
epo_status epo_set_poses_dev(epo_scene_t scene, const double* T_dev);
epo_status epo_get_poses_dev(epo_scene_t scene, double* T_dev);

/* Optimiser state for checkpoint / resume: the step counter (drives the
 * clamp anneal and Adam's bias correction) and Adam's moments (n_views x 6
 * each, host).  Resuming = set poses + set state. */
epo_status epo_get_state(epo_scene_t scene, int64_t* step, double* m, double* v);
epo_status epo_set_state(epo_scene_t scene, int64_t step, const double* m, const double* v);

/* Loss (Eq. 6, one value per scene) and gradient (n_views x 6) at the
 * current poses, with lambda from the anneal at the current step.  grad may
 * be NULL.  Host outputs; synchronises. */
epo_status epo_loss_and_grad(epo_scene_t scene, double* loss, double* grad);
/* Device outputs: loss_dev n_scenes doubles, grad_dev n_views x 6 (may be NULL). */
epo_status epo_loss_and_grad_dev(epo_scene_t scene, double* loss_dev, double* grad_dev);

/* Per-pair accumulators of the last evaluation, n_pairs x 8 doubles (host):
 * sum rho, n_valid, sum dRho/dY (3, camera-j frame), sum Y x dRho/dY (3).
 * The last six hold the gradient pass's sums; after a forward-only pass
 * they are zero. */
epo_status epo_pair_stats(epo_scene_t scene, double* stats);

/* Forward / adjoint pair behind an autograd function of the twists xi
 * (n_views x 6, device): poses T_i(xi) = Exp(xi_i) T_i.  forward writes the
 * per-scene loss; backward takes dL_out/dloss per scene (device, n_scenes)
 * and writes d(out)/d(xi) = J_l(xi)^T g (J_l the SE(3) left Jacobian, g the
 * left-perturbation gradient at T(xi)), recomputing every projection instead
 * of storing per-sample Jacobians (the analytical backward of Algorithm 2's
 * fused kernels).  xi_dev may be NULL (= zero).  backward must follow a
 * forward at the same xi (it reuses the forward's n_valid per pair). */
epo_status epo_forward_dev(epo_scene_t scene, const double* xi_dev, double* loss_dev);
epo_status epo_backward_dev(epo_scene_t scene, const double* xi_dev, const double* dloss_dev,
                            double* grad_xi_dev);

/* n_steps optimisation steps (Algorithm 2, pose-only reading): clamp anneal,
 * loss + gradient, tangent-space Adam, T_i <- Exp(-Delta_i) T_i for every
 * view not fixed.  Each step is one replay of a CUDA graph; lambda, the step
 * counter and Adam's state live on the device.  epo_step synchronises at the
 * end and returns EPO_ERR_NUMERIC if a step saw a non-finite loss or
 * gradient (that step and the later ones left the poses unchanged);
 * epo_step_async does not synchronise (check with epo_check). */
epo_status epo_step(epo_scene_t scene, int32_t n_steps);
epo_status epo_step_async(epo_scene_t scene, int32_t n_steps);

/* One optimisation step driven from the host, with a single synchronisation: the poses
 * T_in (n_views x 12 doubles, host; NULL keeps the current ones; not allowed under
 * EPO_POSE_MLP, whose poses come from its parameters) are copied in, the step runs, and the
 * poses after it (T_out, n_views x 12) and the loss it evaluated (loss, n_scenes) are copied
 * out; either output may be NULL.  The caller's buffers may be any host memory: the scene
 * keeps a pinned, device-mapped staging buffer, which the step's graph reads the poses from
 * (its first kernel) and writes poses, loss and status back into (its last kernel), so no
 * copy-engine transfer sits between the host and the step.  EPO_ERR_INVALID_ARG on a
 * non-finite input pose, EPO_ERR_NUMERIC as epo_step. */
epo_status epo_step_host(epo_scene_t scene, const double* T_in, double* T_out, double* loss);
/* The per-step form without the graph: the same kernels launched one by
 * one from the host every step (the plain form the graph is compared to). */
epo_status epo_step_plain(epo_scene_t scene, int32_t n_steps);
/* Synchronise and report a pending numeric flag (and clear it). */
epo_status epo_check(epo_scene_t scene);

/* Bounded host waits (failure detection; no counterpart in the paper).  With
 * seconds > 0, the calls that wait for the GPU on behalf of host outputs
 * (epo_step, epo_step_host, epo_check, epo_loss_and_grad, epo_last_loss,
 * epo_get_poses) poll the completion of the work they queued for at most
 * that long, then return EPO_ERR_TIMEOUT instead of blocking.  The queued
 * work is not cancelled: it runs to completion, the handle stays usable, and
 * the next call that needs it (any of the calls above) waits for it first,
 * within the same limit.  A call that ran out has not written its host
 * outputs; the device state it advanced (poses and optimiser state of the
 * steps it queued) is read back by epo_get_poses / epo_get_state once the
 * work has finished.  Host outputs go through pinned staging owned by the
 * scene, so nothing is written into caller memory after a call returns.
 * seconds = 0 (the default) waits without a limit.  Other synchronising calls
 * wait without a limit.  EPO_ERR_INVALID_ARG for a negative or non-finite
 * limit. */
epo_status epo_set_wait_limit(epo_scene_t scene, double seconds);

/* Loss per scene (host, n_scenes doubles) computed by the most recent
 * evaluation or step (a step evaluates before it updates).  Synchronises. */
epo_status epo_last_loss(epo_scene_t scene, double* loss);

/* Samples of the most recent evaluation whose FP32 position lay within its
 * rounding-error bound of a discontinuity (bilinear cell line, image border,
 * depth threshold, clamp) and were re-evaluated with FP64 decisions
 * (queued), and those that found their block's buffer full and kept their
 * FP32 decisions (overflow, normally 0).  Synchronises. */
epo_status epo_fixup_stats(epo_scene_t scene, int64_t* queued, int64_t* overflow);

/* Device time in milliseconds of the edge kernel (lift, projection, sampling,
 * robust penalty, adjoint and per-pair reduction) in the most recent
 * evaluation or step; needs options.timing = 1.  Synchronises. */
epo_status epo_kernel_time(epo_scene_t scene, float* ms);

/* Device times in milliseconds of the three stages of the most recent
 * evaluation or step: pair setup, edge kernel (with its exact re-evaluation of
 * ambiguous samples), pose kernel (loss, gradient gather, update).  ms: 3
 * floats.  Needs options.timing = 1.  Synchronises. */
epo_status epo_stage_times(epo_scene_t scene, float* ms);

/* Focal scales and per-pixel depth parameters of a scene created with
 * options.refine = 1 (Section 3, Camera Refinement and Depth Refinement,
 * Eqs. 4-5).  gamma: n_views doubles (> -1), the focal lengths of view v are
 * f^0 (1 + gamma_v); alpha, beta: one float each per kept record (the records
 * of epo_scene_info.n_records, in input order without the dropped ones), the
 * record's depth is z^0 alpha + beta.  Host arrays, copied; NULL = the
 * identity (0, 1, 0).  Also clears the Adam moments of gamma, alpha and beta
 * (options.lr_focal, lr_depth).  Synchronises.  EPO_ERR_INVALID_ARG on a scene
 * without refinement or non-finite values. */
epo_status epo_set_refinement(epo_scene_t scene, const double* gamma, const float* alpha, const float* beta);

/* Parameters of the pose MLP (options.pose_param = EPO_POSE_MLP; Section 3, Pose Refinement):
 * params holds n_scenes x EPO_POSE_MLP_PARAMS floats (host; the initialisation is the caller's,
 * e.g. Kaiming-normal layers with the last layer zero).  Clears the AdamW moments and the
 * offsets delta, keeps the initial poses P^0 (those of the last epo_set_poses) and sets the
 * current poses to P^s of the new parameters.  Synchronises.  EPO_ERR_INVALID_ARG on a scene
 * in SE(3) mode or non-finite values.  In MLP mode epo_set_poses sets P^0, clears delta and
 * recomputes the poses from the current parameters (all zero until this call: P^s = P^0). */
epo_status epo_set_pose_mlp(epo_scene_t scene, const float* params);

/* The current MLP parameters (n_scenes x EPO_POSE_MLP_PARAMS floats) and offsets (n_views x 3
 * floats); either may be NULL.  Host outputs.  Synchronises. */
epo_status epo_get_pose_mlp(epo_scene_t scene, float* params, float* delta);

/* The AdamW moments of the pose MLP: m and v of the parameters (n_scenes x
 * EPO_POSE_MLP_PARAMS floats each) and of the offsets (n_views x 3 each); any may be NULL.
 * Host outputs.  Synchronises. */
epo_status epo_get_pose_mlp_moments(epo_scene_t scene, float* m, float* v, float* dm, float* dv);

/* The current refinement (after the steps that updated it): gamma (n_views
 * doubles), alpha and beta (n_records floats each).  Host outputs, any may be
 * NULL.  Synchronises.  EPO_ERR_INVALID_ARG on a scene without refinement. */
epo_status epo_get_refinement(epo_scene_t scene, double* gamma, float* alpha, float* beta);

/* The objective at the current poses and refinement and its gradient with
 * respect to all of them: loss (n_scenes), grad (n_views x 6, left
 * perturbation), grad_gamma (n_views), grad_alpha and grad_beta (n_records,
 * dL/dalpha = dL/dz z^0, dL/dbeta = dL/dz).  One fused pass stores every
 * sample's d(rho)/dz (4 bytes per evaluation of library memory); a second
 * kernel weights them by the pairs' w / n once the pass has counted the valid
 * samples.  Host outputs; any gradient may be NULL.  Synchronises. */
epo_status epo_refine_loss_and_grad(epo_scene_t scene, double* loss, double* grad, double* grad_gamma,
                                    float* grad_alpha, float* grad_beta);

/* State of the optimisation schedule per scene (options.schedule): theta95
 * (n_scenes doubles, of the most recent step), phase (n_scenes: 1, 2, 3 =
 * converged), switch_step and stop_step (n_scenes each: the step at which
 * phase 2 began / the run converged, -1 if not yet).  Host outputs, any may be
 * NULL.  Synchronises. */
epo_status epo_get_schedule(epo_scene_t scene, double* theta95, int32_t* phase, int64_t* switch_step,
                            int64_t* stop_step);

/* The pairs the most recent evaluation or step used (1) or skipped (0):
 * n_pairs bytes (host).  Synchronises. */
epo_status epo_get_pair_active(epo_scene_t scene, uint8_t* active);

/* Evaluate only a subset of the pairs from now on (the stochastic viewgraph
 * sub-sampling of Algorithm 3 / Appendix A.3; the draw is the caller's).
 * pair_ids: n distinct indices (host); n = 0 restores all pairs.  The loss
 * then averages over the active pairs of each scene. */
epo_status epo_set_pair_subset(epo_scene_t scene, int32_t n, const int32_t* pair_ids);

/* Time the kernel schedules on the current poses and keep the fastest
 * (block size, records per thread, gather path).  With options.autotune == 2
 * each timed launch starts from a cold L2; a temporary scratch buffer of
 * twice the L2 size is allocated for that during the call. */
epo_status epo_autotune(epo_scene_t scene);

/* Distance transform field (Algorithm 1, ComputeDistanceFields): exact
 * Euclidean distance from every pixel to the nearest nonzero pixel of the
 * edge mask, W + H everywhere when the mask is empty.  edges_dev: W*H bytes,
 * map_dev: W*H floats (both device, row-major); map_dev also serves as the
 * intermediate.  Stream-ordered. */
epo_status epo_distance_field(const uint8_t* edges_dev, int32_t W, int32_t H, float* map_dev,
                              void* cuda_stream);
/* Round n floats to bfloat16 (round to nearest even), device buffers. */
epo_status epo_round_bf16(const float* src_dev, uint16_t* dst_dev, int64_t n, void* cuda_stream);

/* Viewgraph estimation (Section 3, Viewgraph Estimation, Eq. 2; Algorithm 1
 * BuildViewgraph), run once before the optimisation.  For every ordered pair
 * (i, j) of the n_views views: over the grid pixels (a stride, b stride) of
 * view i with a positive finite depth, the fraction whose round trip i -> j
 * -> i (projected with Z_i, lifted in j with Z_j at the nearest pixel,
 * projected back) stays in front of both cameras and inside view j and
 * returns within tau pixels.  W, H: n_views each; K: n_views x 4 (fx, fy, cx,
 * cy); T: n_views x 12 world -> camera [R|t] (host, FP64); depth_dev: the
 * views' W x H float depth maps concatenated (device, row-major).  Outputs
 * (host): frac n_views x n_views (may be NULL; diagonal 0), pairs 2 x
 * n_views (n_views - 1) int32 capacity (may be NULL): the directed pairs of
 * the undirected pairs whose fraction is >= min_frac both ways, row-major;
 * *n_pairs their count.  FP64 on the device; synchronises.  Invalid sizes or
 * intrinsics: EPO_ERR_INVALID_ARG; allocation failure: EPO_ERR_OOM. */
epo_status epo_build_viewgraph(int32_t n_views, const int32_t* W, const int32_t* H, const double* K, const double* T,
                               const float* depth_dev, int32_t stride, double tau, double min_frac, double* frac,
                               int32_t* pairs, int32_t* n_pairs, void* cuda_stream);

/* Gather-throughput probe for the roofline of the sampling step (Eq. 8's
 * bilinear sample; the paper names projection and sampling as the dominant
 * cost, Section 5 / Appendix A): 2x2 footprints per second that this GPU
 * serves from n_maps maps of W x H (map_dtype EPO_F32 or EPO_BF16, rows
 * padded to 128 bytes as in a scene), fetched with the edge kernel's form
 * (gather = EPO_GATHER_LDG: four read-only loads; EPO_GATHER_TEX: one
 * texture gather).  pattern 0: independent uniform positions per thread;
 * 1: the 32 lanes of a warp along a 32-pixel segment at a random place (the
 * locality of consecutive edge pixels; needs W >= 48, H >= 16).  About
 * `samples` footprints per launch; the median of `repeats` timed launches
 * (after two that fill L2) is written to *samples_per_s.  The buffers are
 * allocated and freed inside the call; synchronises the stream.  Invalid
 * sizes or modes: EPO_ERR_INVALID_ARG; a failed CUDA call: EPO_ERR_CUDA
 * (everything allocated is freed). */
epo_status epo_gather_probe(int32_t n_maps, int32_t W, int32_t H, int32_t map_dtype, int32_t gather,
                            int32_t pattern, int64_t samples, int32_t repeats, double* samples_per_s,
                            void* cuda_stream);

/* ------------------------------------------------------------------------
 * Loss and gradient without any device allocation.
 *
 * This entry point has no counterpart in the paper.  It exists for callers
 * that cannot call cudaMalloc: a host application that owns every byte of
 * device memory (a plugin running inside another engine, a fixed memory
 * budget handed out up front), a real-time loop in which an allocation may
 * block or fail, or code that runs while the device allocator is off limits.
 * Such a caller keeps its inputs and outputs in its own device buffers and
 * passes them in; no scene handle is created.
 *
 * It computes what epo_loss_and_grad_dev computes (Eqs. 6-8 and the
 * left-perturbation pose gradient, EPO_F32 records and FP32 maps) for one
 * scene, with every projection and branch decision taken in FP64.  The
 * intermediate per-pair sums live in one file-scope device array of the
 * library of fixed size: EPO_NOALLOC_MAX_PAIRS x 21 doubles = 688,128
 * bytes (672 KiB), which every GPU that loads the library reserves until
 * the process exits.  Hence the limits below: larger problems are rejected
 * with EPO_ERR_TOO_LARGE before any work.
 *
 *   - Records whose depth is not positive and finite are not part of the
 *     problem, as at scene creation: they are never valid samples, and
 *     under EPO_NORM_ALL the denominator |E_i| counts only the other
 *     records of view i.
 *
 *   - The first call on a device looks up that array's device address (with
 *     the device current) and keeps it; make that first call before any
 *     stream capture.
 *   - Every call reuses the same array and clears what must start at zero;
 *     calls that overlap on the GPU (another stream, another host thread)
 *     race on it and give wrong results.  Order them on one stream.
 *   - The call allocates nothing: no cudaMalloc, cudaFree or allocating
 *     library routine, on the device or the host.
 *   - Stream-ordered on cuda_stream; it does not synchronise.  Status codes:
 *     EPO_ERR_INVALID_ARG for a NULL pointer, a pointer not aligned to its
 *     element (records to 16 bytes), no view or pair, or an invalid lambda /
 *     huber_delta / eps_z / norm_mode; EPO_ERR_TOO_LARGE beyond the limits
 *     (views, pairs, or more than 2^31 - 1 tiles of 256 records in one
 *     view); EPO_ERR_CUDA if a launch fails.  Indices and sizes inside the
 *     device buffers are not checked: they must be consistent.
 * ------------------------------------------------------------------------ */
#define EPO_NOALLOC_MAX_VIEWS 1024
#define EPO_NOALLOC_MAX_PAIRS 4096

typedef struct {
  int32_t n_views, n_pairs;      /* 1..EPO_NOALLOC_MAX_VIEWS, 1..EPO_NOALLOC_MAX_PAIRS */
  const float* records;          /* device, 16-byte aligned: {u, v, z, 0} per record */
  const int64_t* rec_off;        /* device: n_views + 1 record offsets, view-major */
  int64_t max_records_per_view;  /* host value: the largest rec_off[i+1] - rec_off[i] */
  const float* maps;             /* device: every view's map, H rows of W floats, dense */
  const int64_t* map_off;        /* device: n_views offsets (in floats) into maps */
  const int32_t* W;              /* device: n_views map widths (>= 2) */
  const int32_t* H;              /* device: n_views map heights (>= 2) */
  const double* K;               /* device: n_views x 4 intrinsics (fx, fy, cx, cy) */
  const int32_t* pairs;          /* device: 2 x n_pairs directed pairs (i, j) */
  const double* T;               /* device: n_views x 12 poses [R|t], world -> camera */
  double lambda;                 /* clamp of the distance (Eq. 7) */
  double huber_delta;
  double eps_z;
  int32_t norm_mode;             /* EPO_NORM_VALID | EPO_NORM_ALL */
} epo_noalloc_problem;

/* loss_dev: 1 double (device); grad_dev: n_views x 6 doubles (device). */
epo_status epo_loss_and_grad_noalloc(const epo_noalloc_problem* problem, double* loss_dev,
                                     double* grad_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EPO_H */
