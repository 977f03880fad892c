// Internal device-side layout and kernel launchers of the edge-alignment library.
//
// Data layout in HBM (all library-owned, built once by epo_create_*):
//   records  : one array for all views of all scenes, view-major, raster order inside a
//              view; 16 B {f32 u, f32 v, f32 z, 0} or 8 B {u16 u, u16 v, f16 z, 0}.
//   map atlas: every view's distance transform field, rows padded to a 128-byte pitch,
//              each view starting on a 512-byte boundary (so a pitched 2-D texture can
//              alias it); f32 or bf16.
//   views    : ViewDev table (intrinsics in f32 for the pixel math, sizes, offsets).
//   tiles    : the persistent kernels' work list: (view, first record, count), view-major
//              so that blocks running at the same time share source and target maps.
//   pairs    : per source view a list of its outgoing pair ids (the pairs that reuse the
//              tile's lifted records), per pair the target view; per pose a list of
//              (pair, role) used by the deterministic FP64 gradient gather.
//   poses    : f64 [R|t] per view, Adam moments, step counter, lambda -- all on device
//              so that a whole optimisation step is a replayable CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace epo {

constexpr int kAcc = 8;  // per-pair accumulator slots: sum rho, n_valid, sum gY (3), sum Y x gY (3)

enum Mode { MODE_FWD = 0, MODE_BWD = 1, MODE_FUSED = 2 };
enum Gather { GATHER_LDG = 1, GATHER_TEX = 2 };

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
};

// Relative pose T_ji = T_j T_i^-1 rounded to f32 for the pixel math (a1), one per pair.
struct PairParam {
  float r[9];
  float t[3];
};

struct EdgeArgs {
  const void* rec;
  const void* map;
  const ViewDev* views;
  const TileDev* tiles;
  int32_t n_tiles;
  const int32_t* src_pair_off;   // n_views + 1
  const int32_t* src_pair_ids;   // pairs grouped by source view
  const int32_t* pair_dst;       // n_pairs
  const PairParam* pp;           // n_pairs
  const uint8_t* pair_active;    // n_pairs
  const unsigned long long* tex; // n_views texture objects (GATHER_TEX)
  double* pair_acc;              // n_pairs x kAcc
  const double* lambda;          // device scalar
  float delta;
  float eps_z;
};

struct StepArgs {
  int32_t n_views, n_pairs, n_scenes;
  const int32_t* pair_src;
  const int32_t* pair_dst;
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
  PairParam* pp;
  double* pair_acc;
  double* pair_loss;                 // n_pairs
  double* contrib;                   // n_pairs x 12 (target part, source part)
  double* grad;                      // n_views x 6
  double* loss;                      // n_scenes
  double* m;                         // Adam moments
  double* v;
  int64_t* step;
  double* lambda;
  int32_t* flag;                     // bit 0: non-finite loss/gradient
  unsigned int* done;                // retraction completion counter
  const double* gscale;              // per-scene scale of the gradient (NULL = 1)
  double lambda0, lambda1;
  int32_t lambda_steps;
  int32_t norm_all;
  double lr_rot, lr_trans, beta1, beta2, adam_eps;
};

// ---- launchers (epo_kernels.cu) ----
cudaError_t launch_pair_setup(const StepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_edge(const EdgeArgs& a, int mode, int rec_dtype, int map_dtype, int gather,
                        int rpt, int block, int grid, cudaStream_t s);
cudaError_t launch_finalize(const StepArgs& a, int with_grad, cudaStream_t s);
cudaError_t launch_retract(const StepArgs& a, cudaStream_t s);
cudaError_t launch_twist_poses(const double* T, const double* xi, double* T_out, int n,
                               cudaStream_t s);
cudaError_t launch_apply_left_jacobian(const double* xi, const double* g, double* out, int n,
                                       cudaStream_t s);
cudaError_t launch_map_check(const void* map, int dtype, int64_t n, int32_t* bad, cudaStream_t s);
cudaError_t launch_edt(const uint8_t* edges, int W, int H, float* map, cudaStream_t s);
cudaError_t launch_round_bf16(const float* src, uint16_t* dst, int64_t n, cudaStream_t s);
int edt_max_height();

}  // namespace epo
