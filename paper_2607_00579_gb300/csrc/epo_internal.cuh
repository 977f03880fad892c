// Internal device-side layout and kernel launchers of the edge-alignment library.
//
// Data layout in HBM (all library-owned, built once by epo_create_*):
//   records  : one array for all views of all scenes, view-major, raster order inside a
//              view; 16 B {f32 u, f32 v, f32 z, 0} or 8 B {u16 u, u16 v, f16 z, 0}.
//   map atlas: every view's distance transform field, rows padded to a 128-byte pitch,
//              each view starting on a 512-byte boundary; f32 or bf16.  The texture path
//              reads per-view gather-capable CUDA arrays holding the same values.
//   views    : ViewDev table (intrinsics in f32 for the pixel math, sizes, offsets) and
//              the f64 intrinsics (K64) for the exact re-evaluation path.
//   tiles    : the persistent kernel's work list: (view, first record, count), view-major
//              so that blocks running at the same time share source and target maps.
//   pairs    : per source view a list of its outgoing pair ids (the pairs that reuse the
//              tile's lifted records), per pair the target view; per pose a list of
//              (pair, role) used by the deterministic FP64 gradient gather.
//   exact path: samples whose FP32 evaluation lies within its own rounding-error bound of
//              a discontinuity (bilinear cell line, image border, depth threshold, clamp)
//              are buffered per block in shared memory and re-evaluated with FP64
//              decisions by the same kernel.
//   poses    : f64 [R|t] per view, Adam moments, beta powers, step counter, lambda -- all
//              on device so that a whole optimisation step is a replayable CUDA graph.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

namespace epo {

// An NVTX range around one public call, named after it (shown by Nsight tools; a few
// nanoseconds when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define EPO_RANGE(name) ::epo::NvtxRange epo_nvtx_range_(name)

// unit roundoff of binary32
constexpr float kU32 = 5.9604645e-08f;

__device__ __forceinline__ float bf16_bits_to_float(unsigned int b) { return __uint_as_float(b << 16); }

// One edge record: EPO_F32 {f32 u, f32 v, f32 z, 0} (REC 0) or EPO_F16 {u16 u, u16 v, f16 z, 0}.
template <int REC>
__device__ __forceinline__ void load_record(const void* base, int64_t idx, float& u, float& v, float& z) {
  if (REC == 0) {
    float4 r = __ldg(reinterpret_cast<const float4*>(base) + idx);
    u = r.x;
    v = r.y;
    z = r.z;
  } else {
    uint2 r = __ldg(reinterpret_cast<const uint2*>(base) + idx);
    u = (float)(r.x & 0xffffu);
    v = (float)(r.x >> 16);
    z = __half2float(__ushort_as_half((unsigned short)(r.y & 0xffffu)));
  }
}

// Programmatic dependent launch: a kernel launched with launch_pdl() may start while its
// predecessor in the stream still runs; griddep_wait() returns once that predecessor has
// completed and its writes are visible (at once for a kernel launched without it), and
// griddep_launch_dependents() lets the successor start early.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// FP64 words per pair written by the pair setup: the relative pose R_ji (9), t_ji (3), and its
// projective form B = K_j R_ji K_i^-1 (9), c = K_j t_ji (3), with which a record (u, v, z)
// of view i lands at (Y3 u', Y3 v', Y3) = z B (u, v, 1) + c in view j
constexpr int kPP64 = 24;

constexpr int kAcc = 8;         // per-pair accumulator slots: sum rho, n_valid, sum gY (3), sum Y x gY (3)

// Bits of the device status word: a non-finite loss, gradient or pose (EPO_ERR_NUMERIC), and, in
// builds with EPO_DEBUG_BOUNDS, a gather cell outside its map (EPO_ERR_INTERNAL).  A step that
// starts with either bit set does not update the poses.
constexpr int kFlagNumeric = 1;
constexpr int kFlagBounds = 2;
constexpr int kFlagRefuse = kFlagNumeric | kFlagBounds;
constexpr int kLossChunk = 32;  // pairs per loss block of the pose kernel (one per lane)

enum Mode { MODE_FWD = 0, MODE_BWD = 1, MODE_FUSED = 2 };
// GATHER_MIX (pose-only scenes): of the two samples a thread has in flight, one is fetched by a
// texture gather and the other by plain loads, so that the texture unit and the load/store
// path serve the footprints side by side.
enum Gather { GATHER_LDG = 1, GATHER_TEX = 2, GATHER_MIX = 3 };

struct ViewDev {
  float fx, fy, cx, cy;   // intrinsics rounded to f32 for the pixel math
  int32_t W, H;           // map size
  int32_t pitch;          // map row pitch, elements
  int32_t scene;          // owning scene
  int64_t map_off;        // element offset of the map in the atlas
  int64_t rec_begin;      // first record of the view
  int32_t n_rec;          // records kept
  int32_t pad_;
};

struct TileDev {
  int32_t view;
  int32_t n;        // records in this tile
  int64_t begin;    // first record
  int32_t q0, q1;   // pairs [q0, q1) of the view's outgoing pair list (indices into it)
};

// Everything the edge kernel needs for one pair i -> j, built by the pair setup (a1):
// the relative pose T_ji = T_j T_i^-1 rounded to f32, the target's intrinsics and map,
// the pair constants of the FP32 rounding-error bound, and the pair's index and flag.  160
// bytes, read with uniform 16-byte loads per pair.  Stored in the order of the views'
// outgoing pair lists (entry q of src_pair_ids), so that a work item reads its pairs' entries
// directly, with no pair-list or flag load in front of them.
struct alignas(16) PairParam {
  float r[9];
  float t[3];
  float fx, fy, cx, cy;   // target intrinsics (f32)
  float hw, hh;           // (W-1)/2, (H-1)/2: the valid range is |u' - hw| <= hw
  int32_t p;              // the pair's index (p and active are read as one 8-byte word)
  int32_t active;         // the pair is evaluated in this step (copied from pair_active)
  float Et;               // rounding bound of Y from the rounded translation
  float cu, cv;           // rounding of u', v' themselves
  int32_t W, H, pitch;    // target map
  int64_t map_off;
  unsigned long long tex; // texture object of the target map
  int64_t dbase;          // refine scenes: dzr[dbase + r] holds d(rho)/dz of record r for this pair
  // the pose-only kernel's single rounding bound (scene creation): for a sample whose FP32
  // position lies within one pixel of the target image, |u' - u'(exact)| and |v' - v'(exact)|
  // are at most t = E |1/Y3| Kb + cb, with E the bound on the error of each component of Y
  float Kb, cb;
  float pad0_;
  float Wm2, Hm2;         // W - 2, H - 2: the cell x0 = floor(u') is valid iff 0 <= x0 <= W - 2
  float Wf, Hf;           // W, H: floor(u') + 1 in [0, W] iff u' lies within one pixel of the image
  float pad_;
};
static_assert(sizeof(PairParam) == 160, "PairParam layout");
static_assert(offsetof(PairParam, p) % 8 == 0 && offsetof(PairParam, active) == offsetof(PairParam, p) + 4,
              "p and active form one aligned 8-byte word");
static_assert(offsetof(PairParam, map_off) % 8 == 0 && offsetof(PairParam, dbase) % 8 == 0 &&
                  offsetof(PairParam, Kb) == 128,
              "PairParam alignment");

struct EdgeArgs {
  const void* rec;
  const void* map;
  const ViewDev* views;
  const double* K64;             // n_views x 6 (fx, fy, cx, cy, 1/fx, 1/fy) in f64
  const TileDev* tiles;
  int32_t n_tiles;
  const int32_t* src_pair_off;   // n_views + 1
  const int32_t* src_pair_ids;   // pairs grouped by source view
  const int32_t* pair_src;       // n_pairs
  const int32_t* pair_dst;       // n_pairs
  const PairParam* pp;           // n_pairs, in source-view pair-list order (index q)
  const double* pp64;            // n_pairs x kPP64 (f64): R_ji (9), t_ji (3), B (9), c (3)
  const uint8_t* pair_active;    // n_pairs
  const unsigned long long* tex; // n_views texture objects (GATHER_TEX)
  double* pair_acc;              // n_pairs x kAcc
  const double* lambda;          // device scalar
  unsigned int* q_count;         // samples re-evaluated on the exact path this evaluation
  unsigned int* q_overflow;      // samples that found the block buffer full (FP32 decisions)
  int* tile_counter;             // dynamic work distribution, reset by the pair setup
  int32_t max_pairs;             // most outgoing pairs of any view (shared accumulators)
  float delta;
  float eps_z;
  // focal and depth refinement (scenes created with refine = 1; Eqs. 4-5)
  const double* gamma;           // n_views: f = f0 (1 + gamma)
  const float* alpha;            // n_records: z = z0 alpha + beta
  const float* beta;
  double* pair_facc;             // n_pairs x 2: sums of the source- and target-focal terms
  float* dzr;                    // per (pair, source record): d(rho)/dz of the sample, 0 if it is
                                 // invalid (fused pass of refine scenes; at PairParam::dbase + r)
  const double* pair_lw;         // n_pairs: the pair's weight in its scene's loss
  int32_t norm_all;
  int32_t* flag;                 // the status word (kFlag* bits)
  int32_t* dbg;                  // EPO_DEBUG_BOUNDS builds: the first out-of-map gather (pair, x0, y0)
  const float4* lift;            // pose-only scenes: every record lifted once at creation, (X0, X1,
                                 // z, the bound on its share of Y's rounding error)
};

#ifdef EPO_DEBUG_BOUNDS
#ifndef EPO_DEBUG_BOUNDS_MARGIN
#define EPO_DEBUG_BOUNDS_MARGIN 0
#endif
// Debug builds: a gather's cell (x0, y0) must lie in [0, W - 2] x [0, H - 2].  A cell outside is
// recorded (status bit kFlagBounds, the first offender's pair and cell) and its fetch is skipped,
// so that the step reports EPO_ERR_INTERNAL instead of reading outside the map.  A test build may
// narrow the accepted range by EPO_DEBUG_BOUNDS_MARGIN columns, so that the report path runs on
// valid inputs without any access outside a map.
__device__ __forceinline__ bool debug_cell_ok(const EdgeArgs& a, int p, int W, int H, int x0, int y0) {
  if (x0 >= 0 && y0 >= 0 && x0 <= W - 2 - EPO_DEBUG_BOUNDS_MARGIN && y0 <= H - 2) return true;
  if (atomicCAS(a.dbg, -1, p) == -1) {
    a.dbg[1] = x0;
    a.dbg[2] = y0;
  }
  atomicOr(a.flag, kFlagBounds);
  return false;
}
#endif

// One (pair, role) entry of a pose's gradient gather, laid out at a fixed stride per pose so
// that the pose kernel reads it without an offset table; p < 0 marks padding.  The pair's
// weight in its scene's loss is pair_lw[p] (0 while the pair is not evaluated).
struct PoseEntry {
  int32_t p;
  int32_t scene_role;  // scene << 1 | role (0 = target view j, 1 = source view i)
};

struct StepArgs {
  int32_t n_views, n_pairs, n_scenes;
  // focal refinement (refine scenes): gamma per view, the FP64 base intrinsics and their
  // refined copy written by the pair setup, the per-pair focal sums and the focal gradient
  int32_t refine;
  double* gamma;                     // updated by the pose kernel's focal Adam (lr_focal)
  const double* K64;                 // n_views x 6: fx, fy, cx, cy, 1/fx, 1/fy (base)
  double* K64r;                      // the same at f0 (1 + gamma)
  double* pair_facc;                 // n_pairs x 2
  double* grad_gamma;                // n_views
  const unsigned long long* tex;     // n_views texture objects (copied into PairParam)
  const int32_t* pair_src;
  const int32_t* pair_dst;
  const int2* pair_ij;               // (i, j) of every pair
  const int32_t* pair_scene;
  const uint8_t* pair_active;
  const int32_t* scene_pair_off;     // n_scenes + 1 (pairs of a scene are contiguous)
  const int32_t* scene_active_pairs; // n_scenes
  const int32_t* pose_pair_off;      // n_views + 1
  const int32_t* pose_pair_ref;      // 2*n_pairs entries: pair*2 + role (0 = target j, 1 = source i)
  const ViewDev* views;
  const uint8_t* fixed;
  const double* T;                   // poses used by the evaluation (n_views x 12)
  double* T_store;                   // poses updated by the retraction
  // host-driven step (epo_step_host): mapped host memory (NULL if unused) that receives the
  // poses after the step, the loss and the status word from the pose kernel
  double* host_out;
  PairParam* pp;                     // n_pairs, in source-view pair-list order
  const int32_t* pair_q;             // n_pairs: the PairParam index q of pair p
  double* pp64;
  double* pair_acc;
  double* grad;                      // n_views x 6
  double* loss;                      // n_scenes
  double* m;                         // Adam moments
  double* v;
  double* bpow;                      // beta1^(s+1), beta2^(s+1) for the next step s
  int64_t* step;
  double* lambda;
  int32_t* flag;                     // bit 0: non-finite loss/gradient
  unsigned long long* done;          // completion counter of the pose kernel (blocks | flagged << 32)
  int32_t n_loss_chunks;             // pose-kernel blocks that sum the per-pair losses
  const int32_t* loss_chunk_off;     // n_scenes + 1: the scene's chunks (kLossChunk pairs each)
  const int32_t* loss_chunk_scene;   // n_loss_chunks
  double* loss_part;                 // n_loss_chunks partial sums of l_p
  const int2* loss_chunk_pairs;      // n_loss_chunks: [first, end) pairs of the chunk
  double* pair_lw;                   // n_pairs: the pair's weight in its scene's loss: 2 / (pairs the
                                     // scene evaluates), times 1 / |E_i| under Eq. 7; 0 if not evaluated
  uint8_t* pair_active_w;            // n_pairs: the same flags as pair_active, for the sub-sampling
  int32_t pair_budget;               // M of Algorithm 3 (0 = every pair)
  uint64_t subsample_seed;
  // optimisation schedule (Section 3): per-view changes of the step, per-scene state
  int32_t schedule;
  const int32_t* scene_view_off;     // n_scenes + 1
  double* pose_dR;                   // n_views: rotation change of the step, degrees
  double* pose_dt;                   // n_views: translation-direction change, degrees
  int32_t* sched_state;              // n_scenes x 2: phase (1, 2, 3 = converged), consecutive steps
  double* theta95;                   // n_scenes
  int64_t* sched_steps;              // n_scenes x 2: step of the switch to phase 2, of convergence
  double sched_eps1, sched_eps2;
  int32_t sched_w1, sched_w2;
  const PoseEntry* pose_entries;     // n_views x pose_stride
  int32_t pose_stride;
  unsigned int* scene_done;          // n_scenes completion counters of the loss chunks
  unsigned int* q_count;             // exact-path sample counter, reset by the pair setup
  int* tile_counter;                 // edge-kernel work counter, reset by the pair setup
  const double* gscale;              // per-scene scale of the gradient (NULL = 1)
  double lambda0, lambda1;
  int32_t lambda_steps;
  double inv_lambda_steps;
  int32_t norm_all;
  double lr_rot, lr_trans, beta1, beta2, adam_eps;
  // refinement optimiser (Algorithm 2 with the camera and depth modules)
  double lr_focal, lr_depth;
  float log_beta1, log_beta2;        // ln beta1, ln beta2 (the depth module's bias factors)
  double* mg;                        // n_views Adam moments of gamma (f64)
  double* vg;
  float* alpha;                      // n_records: z = z0 alpha + beta
  float* beta;
  float* ma;                         // n_records Adam moments of alpha and beta (f32)
  float* va;
  float* mb;
  float* vb;
  const float* dzr;                  // per (pair, record) d(rho)/dz of the fused pass
  float* pair_wz;                    // n_pairs (refine scenes): w_p / n_p in f32, written by the
                                     // pose kernel's loss blocks, read by the depth kernel
  const int32_t* src_pair_off;       // n_views + 1: the view's outgoing pairs in src_pair_ids
  const int32_t* src_pair_ids;
  float* grad_alpha;                 // n_records (gradient mode of the depth kernel)
  float* grad_beta;
  const void* rec;                   // records (z0)
  int32_t rec_dtype;
  int32_t max_view_records;          // most records of one view (grid of the depth update)
  // pose parameterisation (Section 3, Pose Refinement, Eq. 3): P^s = phi(P^0 + MLP(P^0)) +
  // [0 | delta]; the pose kernel then only forms the gradient (and gamma's step)
  int32_t pose_mlp;
  float* mlp_theta;                  // n_scenes x kMlpParams (layout of kMlpDims)
  float* mlp_m;                      // AdamW moments of theta
  float* mlp_v;
  const double* mlp_P0;              // n_views x 12: the initial poses (the MLP's input)
  const double* mlp_scale;           // n_scenes: RMS spread of the P^0 camera centres (the MLP acts
                                     // on the scene at unit scale: translations / s in, x s out)
  double* mlp_Pp;                    // n_views x 12: P^0 + MLP(P^0) of the current poses
  float* mlp_delta;                  // n_views x 3 translation offsets, their moments and gradient
  float* mlp_dm;
  float* mlp_dv;
  float* mlp_gdelta;
  float* mlp_x;                      // n_views x 12: the input as the MLP saw it (f32)
  float* mlp_z;                      // n_views x 5 x 128: pre-activations of the hidden layers
  float* mlp_dz;                     // n_views x (5 x 128 + 12): dL/dz of every layer
  unsigned int* mlp_done;            // completion counter of the update kernel
  float mlp_lr;                      // peak learning rate
  int32_t mlp_warmup, mlp_steps;     // linear warm-up steps; the cosine reaches 0 at mlp_steps - 1
  float mlp_wd, mlp_wd_delta, mlp_eps;
};

// Pose MLP: 12 -> 128 -> 128 -> 128 -> 128 -> 128 -> 12; parameters per scene in the order
// W1 (128x12, row-major [out][in]), b1, W2..W5 (128x128), b2..b5, W6 (12x128), b6.
constexpr int kMlpHid = 128;
constexpr int kMlpParams = kMlpHid * 12 + kMlpHid + 4 * (kMlpHid * kMlpHid + kMlpHid) + 12 * kMlpHid + 12;
constexpr int kMlpDz = 5 * kMlpHid + 12;  // per view: dL/dz of the five hidden layers and the output

// ---- launchers (epo_kernels.cu) ----
cudaError_t launch_pair_setup(const StepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_refine_intrinsics(const StepArgs& a, cudaStream_t s);
cudaError_t launch_subsample(const StepArgs& a, cudaStream_t s);
cudaError_t launch_schedule(const StepArgs& a, cudaStream_t s);
// pose MLP (epo_pose_mlp.cu): forward (new poses; change = 1 also records the pose changes of
// the step), backward through phi and the MLP, AdamW update of theta and delta
cudaError_t launch_mlp_forward(const StepArgs& a, int change, cudaStream_t s);
cudaError_t launch_mlp_backward(const StepArgs& a, cudaStream_t s);
cudaError_t launch_mlp_update(const StepArgs& a, cudaStream_t s);
// depth kernel: update 0 = dL/dalpha, dL/dbeta into grad_alpha, grad_beta; 1 = Adam step
cudaError_t launch_depth(const StepArgs& a, int update, cudaStream_t s);
cudaError_t launch_l2_read(const void* p, int64_t bytes, unsigned* sink, int sms, cudaStream_t s);
cudaError_t launch_edge(const EdgeArgs& a, int mode, int refine, int rec_dtype, int map_dtype, int gather,
                        int rpt, int block, int grid, cudaStream_t s);
// pose kernel: with_grad 0 = loss only, 1 = loss + gradient, 2 = + Adam/Exp update
cudaError_t launch_poses(const StepArgs& a, int with_grad, cudaStream_t s);
// A launch that allows programmatic dependent launch on stream s (see griddep_wait).
template <typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_io_copy(const double* src, double* dst, int64_t n, cudaStream_t s);
cudaError_t launch_twist_poses(const double* T, const double* xi, double* T_out, int n,
                               cudaStream_t s);
cudaError_t launch_apply_left_jacobian(const double* xi, const double* g, double* out, int n,
                                       cudaStream_t s);
cudaError_t launch_map_check(const void* map, int dtype, int64_t n, int32_t* bad, cudaStream_t s);
cudaError_t launch_edt(const uint8_t* edges, int W, int H, float* map, cudaStream_t s);
cudaError_t launch_round_bf16(const float* src, uint16_t* dst, int64_t n, cudaStream_t s);
// a2 for scenes whose intrinsics and depths stay fixed: each kept record's camera-frame point
// X = z ((u - cx) / fx, (v - cy) / fy, 1) in FP64, rounded to FP32, with its rounding bound
cudaError_t launch_lift_records(const void* rec, int rec_dtype, const ViewDev* views, const double* K64,
                                int n_views, float eps_z, float4* out, cudaStream_t s);
int edt_max_height();
const void* edge_kernel_ptr(int mode, int refine, int rec_dtype, int map_dtype, int gather, int rpt);
size_t edge_smem_bytes(int rpt, int block, int max_pairs, int refine);

}  // namespace epo
