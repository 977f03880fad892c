// C ABI of the edge-alignment library: scene construction (device layout), evaluation,
// the graph-captured optimisation step, the autograd forward/adjoint pair, the autotuner.
// Declarations and argument conventions: include/epo.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <string>
#include <thread>
#include <vector>

#include "../../include/epo.h"
#include "epo_internal.cuh"

using namespace epo;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// IEEE binary16 -> float on the host (used to validate FP16-depth records).
float half_bits_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h >> 15) << 31;
  const uint32_t exp = (h >> 10) & 0x1f;
  const uint32_t man = h & 0x3ff;
  float f;
  if (exp == 0) {
    f = ldexpf((float)man, -24);
  } else if (exp == 31) {
    f = man ? NAN : INFINITY;
  } else {
    f = ldexpf((float)(man | 0x400), (int)exp - 25);
  }
  uint32_t bits;
  memcpy(&bits, &f, 4);
  bits |= sign;
  memcpy(&f, &bits, 4);
  return f;
}

}  // namespace

struct epo_scene {
  // configuration
  epo_options opt;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int rec_dtype = 0;  // 0 f32, 1 f16
  int map_dtype = 0;  // 0 f32, 1 bf16
  int n_scenes = 0, n_views = 0, n_pairs = 0;
  int64_t n_records = 0, n_dropped = 0, evals = 0;
  int sm_count = 0;
  // schedule
  int gather = GATHER_LDG, block = 256, rpt = 4, grid = 0;
  bool tuned = false;
  // host tables
  std::vector<ViewDev> views;
  std::vector<int32_t> pair_src, pair_dst, pair_scene, scene_pair_off, scene_active;
  std::vector<int32_t> src_pair_off, src_pair_ids;
  std::vector<int32_t> scene_view_begin;  // n_scenes + 1: the views of each scene (contiguous)
  std::vector<uint8_t> active;
  // device buffers
  std::vector<DevBuf> bufs;
  void* d_rec = nullptr;
  float4* d_lift = nullptr;  // pose-only scenes: the records lifted once (EdgeArgs::lift)
  void* d_map = nullptr;
  int64_t map_elems = 0;
  ViewDev* d_views = nullptr;
  TileDev* d_tiles = nullptr;
  int32_t n_tiles = 0;
  int tiles_for = -1;   // tile size the current table was built for
  int tiles_tail = -1;  // and its tail split
  int tiles_grid = -1;  // over the last wave of this many blocks
  int tail = 0;         // pairs per work item of the last wave (0 = not split)
  struct TileTable {
    int tile, tail, grid;
    TileDev* p;
    int32_t n;
  };
  std::vector<TileTable> tile_tables;  // every table built so far, kept for cheap switches
  int32_t *d_src_pair_off = nullptr, *d_src_pair_ids = nullptr, *d_pair_src = nullptr,
          *d_pair_dst = nullptr, *d_pair_scene = nullptr, *d_scene_pair_off = nullptr,
          *d_scene_active = nullptr, *d_pose_pair_off = nullptr, *d_pose_pair_ref = nullptr;
  uint8_t *d_active = nullptr, *d_fixed = nullptr;
  unsigned long long* d_tex = nullptr;
  std::vector<cudaTextureObject_t> tex;
  std::vector<cudaArray_t> arrays;
  PairParam* d_pp = nullptr;
  int32_t* d_pair_q = nullptr;  // the PairParam index of every pair (source-view order)
  double *d_pp64 = nullptr, *d_K64 = nullptr, *d_pair_acc = nullptr, *d_grad = nullptr,
         *d_loss = nullptr, *d_m = nullptr, *d_v = nullptr, *d_bpow = nullptr, *d_lambda = nullptr,
         *d_T = nullptr, *d_T_eval = nullptr;
  unsigned int *d_qcount = nullptr, *d_qoverflow = nullptr;
  int* d_tile_counter = nullptr;
  int max_pairs = 1;
  int64_t* d_step = nullptr;
  int32_t* d_flag = nullptr;
  int32_t* d_dbg = nullptr;   // the first out-of-map gather of a debug build (pair, x0, y0; pair -1 = none)
  unsigned long long* d_done = nullptr;
  // loss chunks: 32 consecutive pairs of one scene per pose-kernel block
  int32_t n_loss_chunks = 0;
  int32_t *d_loss_chunk_off = nullptr, *d_loss_chunk_scene = nullptr;
  double* d_loss_part = nullptr;
  unsigned int* d_scene_done = nullptr;
  int2* d_loss_chunk_pairs = nullptr;
  int2* d_pair_ij = nullptr;
  double* d_pair_lw = nullptr;
  PoseEntry* d_pose_entries = nullptr;
  // stochastic viewgraph sub-sampling (options.pair_budget)
  int subsample = 0;  // 1 when some scene has more pairs than the budget
  // optimisation schedule (options.schedule)
  int32_t* d_scene_view_off = nullptr;
  double *d_pose_dR = nullptr, *d_pose_dt = nullptr, *d_theta95 = nullptr;
  int32_t* d_sched_state = nullptr;
  int64_t* d_sched_steps = nullptr;
  // focal and depth refinement (options.refine)
  int refine = 0;
  double *d_gamma = nullptr, *d_K64r = nullptr, *d_pair_facc = nullptr, *d_grad_gamma = nullptr;
  float *d_alpha = nullptr, *d_beta = nullptr, *d_grad_alpha = nullptr, *d_grad_beta = nullptr;
  float* d_dzr = nullptr;  // per (pair, source record) d(rho)/dz of the fused pass
  float* d_pair_wz = nullptr;  // per pair w / n of the last evaluation (refine scenes)
  int64_t n_dzr = 0;       // sum over pairs of the source view's records
  // refinement optimiser: Adam moments of gamma (f64) and of alpha, beta (f32)
  double *d_mg = nullptr, *d_vg = nullptr;
  float *d_ma = nullptr, *d_va = nullptr, *d_mb = nullptr, *d_vb = nullptr;
  int depth_opt = 0;           // refine && lr_depth > 0: the depth module's kernel in every step
  // pose MLP (options.pose_param = EPO_POSE_MLP)
  int pose_mlp = 0;
  float *d_mlp_theta = nullptr, *d_mlp_m = nullptr, *d_mlp_v = nullptr, *d_mlp_delta = nullptr,
        *d_mlp_dm = nullptr, *d_mlp_dv = nullptr, *d_mlp_gdelta = nullptr, *d_mlp_x = nullptr,
        *d_mlp_z = nullptr, *d_mlp_dz = nullptr;
  double *d_mlp_P0 = nullptr, *d_mlp_Pp = nullptr, *d_mlp_scale = nullptr;
  unsigned int* d_mlp_done = nullptr;
  int32_t max_view_records = 0;
  int32_t pose_stride = 1;
  std::vector<int32_t> pose_off, pose_ref;  // (pair, role) entries of every pose, pose-major
  int32_t* h_flag = nullptr;  // pinned
  // host outputs go through pinned staging, so that a wait for them can be bounded:
  // h_out = [loss (n_scenes) | gradient (6 n_views) | poses (12 n_views)]
  double* h_out = nullptr;
  // bounded host waits (epo_set_wait_limit): 0 = wait without limit; ev_wait marks the work a
  // wait that ran out left queued (wait_pending), which the next call that reuses the staging
  // waits for first
  double wait_limit_s = 0.0;
  cudaEvent_t ev_wait = nullptr;
  bool wait_pending = false;
  double* d_io = nullptr;     // [poses (12 n_views) | loss (n_scenes) | flag (one word)]
  // epo_step_host's staging, pinned and mapped: h_in the input poses (12 n_views), h_io the
  // layout of d_io; dh_in, dh_io are their device addresses, read and written by the step's graph
  double* h_in = nullptr;
  double* h_io = nullptr;
  const double* dh_in = nullptr;
  double* dh_io = nullptr;
  int64_t device_bytes = 0;
  // stage timing events (options.timing): before setup, after setup, after the edge
  // kernel, after the pose kernel
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ev_recorded = false;
  // graph of one optimisation step, and the host-driven steps of epo_step_host without and
  // with input poses
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_host[2] = {nullptr, nullptr};
  bool graph_dirty = true;
  std::string err;
};

namespace {

epo_status fail(epo_scene* s, epo_status code, const std::string& msg) {
  if (s)
    s->err = msg;
  else
    g_create_error = msg;
  return code;
}

epo_status cuda_fail(epo_scene* s, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(s, e == cudaErrorMemoryAllocation ? EPO_ERR_OOM : EPO_ERR_CUDA, m);
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(S, e_, #call); \
  } while (0)

epo_status host_wait(epo_scene* S);

// The status a step's status word `flag` stands for, clearing the device word when it is set:
// EPO_ERR_INTERNAL for a gather cell outside its map (debug builds; the first one is named),
// EPO_ERR_NUMERIC for a non-finite loss, gradient or pose.
epo_status flag_status(epo_scene* S, int32_t flag, const char* numeric_msg) {
  if (!(flag & kFlagRefuse)) return EPO_OK;
  int32_t dbg[3] = {-1, 0, 0};
  if (flag & kFlagBounds) {
    cudaError_t e = cudaMemcpyAsync(dbg, S->d_dbg, 12, cudaMemcpyDeviceToHost, S->stream);
    if (e != cudaSuccess) return cuda_fail(S, e, "cudaMemcpyAsync");
    e = cudaMemsetAsync(S->d_dbg, 0xff, 16, S->stream);
    if (e != cudaSuccess) return cuda_fail(S, e, "cudaMemsetAsync");
  }
  cudaError_t e = cudaMemsetAsync(S->d_flag, 0, 4, S->stream);
  if (e != cudaSuccess) return cuda_fail(S, e, "cudaMemsetAsync");
  epo_status st = host_wait(S);
  if (st != EPO_OK) return st;
  if (flag & kFlagBounds)
    return fail(S, EPO_ERR_INTERNAL,
                "a gather cell outside its map (pair " + std::to_string(dbg[0]) + ", cell " + std::to_string(dbg[1]) +
                    ", " + std::to_string(dbg[2]) + "); its sample was skipped and the poses were not updated");
  return fail(S, EPO_ERR_NUMERIC, numeric_msg);
}

// Waits until the work queued before ev_wait has finished: without a limit by blocking on
// the event, with one by polling it until the limit runs out (EPO_ERR_TIMEOUT; the work stays
// queued, the handle stays usable, and the next call that needs it waits for it first).
epo_status poll_pending(epo_scene* S) {
  if (S->wait_limit_s <= 0.0) {
    cudaError_t e = cudaEventSynchronize(S->ev_wait);
    if (e != cudaSuccess) return cuda_fail(S, e, "cudaEventSynchronize");
    S->wait_pending = false;
    return EPO_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(S->ev_wait);
    if (e == cudaSuccess) {
      S->wait_pending = false;
      return EPO_OK;
    }
    if (e != cudaErrorNotReady) return cuda_fail(S, e, "cudaEventQuery");
    const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (waited >= S->wait_limit_s)
      return fail(S, EPO_ERR_TIMEOUT,
                  "the wait limit of " + std::to_string(S->wait_limit_s) +
                      " s ran out; the queued work continues and the next call waits for it");
    std::this_thread::yield();
  }
}

// Waits for everything queued on the scene's stream so far (see poll_pending).
epo_status host_wait(epo_scene* S) {
  cudaError_t e = cudaEventRecord(S->ev_wait, S->stream);
  if (e != cudaSuccess) return cuda_fail(S, e, "cudaEventRecord");
  S->wait_pending = true;
  return poll_pending(S);
}

// Before a call reuses host staging that work left queued by a timed-out wait may still read
// or write: wait for that work (within the limit).
epo_status drain(epo_scene* S) { return S->wait_pending ? poll_pending(S) : EPO_OK; }

template <typename T>
epo_status dalloc(epo_scene* S, T** p, size_t count) {
  void* q = nullptr;
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return cuda_fail(S, e, "cudaMalloc");
  S->bufs.push_back({q, bytes});
  S->device_bytes += (int64_t)bytes;
  *p = reinterpret_cast<T*>(q);
  return EPO_OK;
}

#define ALLOC(ptr, count)                       \
  do {                                          \
    epo_status st_ = dalloc(S, &(ptr), (count)); \
    if (st_ != EPO_OK) return st_;              \
  } while (0)

// Pair weights in their scene's loss and the per-pose gather entries, from the active pair
// set (rebuilt whenever it changes).
epo_status upload_weights(epo_scene* S, cudaStream_t st) {
  const bool norm_all = S->opt.norm_mode == EPO_NORM_ALL;
  std::vector<double> lw(S->n_pairs, 0.0);
  for (int p = 0; p < S->n_pairs; ++p) {
    const int sc = S->pair_scene[p];
    const int na = S->scene_active[sc];
    if (!S->active[p] || na <= 0) continue;
    double w = 2.0 / na;
    if (norm_all) {
      const int64_t n = S->views[S->pair_src[p]].n_rec;
      w = n > 0 ? w / (double)n : 0.0;
    }
    lw[p] = w;
  }
  std::vector<PoseEntry> ent((size_t)S->n_views * S->pose_stride, PoseEntry{-1, 0});
  for (int v = 0; v < S->n_views; ++v)
    for (int k = S->pose_off[v]; k < S->pose_off[v + 1]; ++k) {
      const int ref = S->pose_ref[k], p = ref >> 1;
      PoseEntry& e = ent[(size_t)v * S->pose_stride + (k - S->pose_off[v])];
      e.p = p;
      e.scene_role = (S->pair_scene[p] << 1) | (ref & 1);
    }
  CK(cudaMemcpyAsync(S->d_pair_lw, lw.data(), lw.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(S->d_pose_entries, ent.data(), ent.size() * sizeof(PoseEntry), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  return EPO_OK;
}

StepArgs step_args(epo_scene* S, const double* T_eval, const double* gscale) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.n_views = S->n_views;
  a.n_pairs = S->n_pairs;
  a.n_scenes = S->n_scenes;
  a.tex = S->d_tex;
  a.pair_src = S->d_pair_src;
  a.pair_dst = S->d_pair_dst;
  a.pair_scene = S->d_pair_scene;
  a.pair_active = S->d_active;
  a.scene_pair_off = S->d_scene_pair_off;
  a.scene_active_pairs = S->d_scene_active;
  a.pose_pair_off = S->d_pose_pair_off;
  a.pose_pair_ref = S->d_pose_pair_ref;
  a.views = S->d_views;
  a.fixed = S->d_fixed;
  a.T = T_eval;
  a.T_store = S->d_T;
  a.pp = S->d_pp;
  a.pair_q = S->d_pair_q;
  a.pp64 = S->d_pp64;
  a.pair_acc = S->d_pair_acc;
  a.grad = S->d_grad;
  a.bpow = S->d_bpow;
  a.q_count = S->d_qcount;
  a.tile_counter = S->d_tile_counter;
  a.loss = S->d_loss;
  a.m = S->d_m;
  a.v = S->d_v;
  a.step = S->d_step;
  a.lambda = S->d_lambda;
  a.flag = S->d_flag;
  a.done = S->d_done;
  a.n_loss_chunks = S->n_loss_chunks;
  a.loss_chunk_off = S->d_loss_chunk_off;
  a.loss_chunk_scene = S->d_loss_chunk_scene;
  a.loss_part = S->d_loss_part;
  a.scene_done = S->d_scene_done;
  a.loss_chunk_pairs = S->d_loss_chunk_pairs;
  a.pair_ij = S->d_pair_ij;
  a.pair_lw = S->d_pair_lw;
  a.pose_entries = S->d_pose_entries;
  a.pose_stride = S->pose_stride;
  a.pair_active_w = S->d_active;
  a.pair_budget = S->opt.pair_budget;
  a.subsample_seed = S->opt.subsample_seed;
  a.schedule = S->opt.schedule;
  a.scene_view_off = S->d_scene_view_off;
  a.pose_dR = S->d_pose_dR;
  a.pose_dt = S->d_pose_dt;
  a.sched_state = S->d_sched_state;
  a.theta95 = S->d_theta95;
  a.sched_steps = S->d_sched_steps;
  a.sched_eps1 = S->opt.sched_eps1;
  a.sched_eps2 = S->opt.sched_eps2;
  a.sched_w1 = S->opt.sched_w1;
  a.sched_w2 = S->opt.sched_w2;
  a.refine = S->refine;
  a.gamma = S->d_gamma;
  a.K64 = S->d_K64;
  a.K64r = S->d_K64r;
  a.pair_facc = S->d_pair_facc;
  a.grad_gamma = S->d_grad_gamma;
  a.gscale = gscale;
  a.lambda0 = S->opt.lambda0;
  a.lambda1 = S->opt.lambda1;
  a.lambda_steps = S->opt.lambda_steps;
  a.inv_lambda_steps = S->opt.lambda_steps > 0 ? 1.0 / S->opt.lambda_steps : 0.0;
  a.norm_all = S->opt.norm_mode == EPO_NORM_ALL;
  a.lr_rot = S->opt.lr_rot;
  a.lr_trans = S->opt.lr_trans;
  a.beta1 = S->opt.beta1;
  a.beta2 = S->opt.beta2;
  a.adam_eps = S->opt.adam_eps;
  a.lr_focal = S->opt.lr_focal;
  a.lr_depth = S->opt.lr_depth;
  a.log_beta1 = (float)log(S->opt.beta1);
  a.log_beta2 = (float)log(S->opt.beta2);
  a.mg = S->d_mg;
  a.vg = S->d_vg;
  a.alpha = S->d_alpha;
  a.beta = S->d_beta;
  a.ma = S->d_ma;
  a.va = S->d_va;
  a.mb = S->d_mb;
  a.vb = S->d_vb;
  a.dzr = S->d_dzr;
  a.pair_wz = S->d_pair_wz;
  a.src_pair_off = S->d_src_pair_off;
  a.src_pair_ids = S->d_src_pair_ids;
  a.grad_alpha = S->d_grad_alpha;
  a.grad_beta = S->d_grad_beta;
  a.rec = S->d_rec;
  a.rec_dtype = S->rec_dtype;
  a.max_view_records = S->max_view_records;
  a.pose_mlp = S->pose_mlp;
  a.mlp_theta = S->d_mlp_theta;
  a.mlp_m = S->d_mlp_m;
  a.mlp_v = S->d_mlp_v;
  a.mlp_P0 = S->d_mlp_P0;
  a.mlp_scale = S->d_mlp_scale;
  a.mlp_Pp = S->d_mlp_Pp;
  a.mlp_delta = S->d_mlp_delta;
  a.mlp_dm = S->d_mlp_dm;
  a.mlp_dv = S->d_mlp_dv;
  a.mlp_gdelta = S->d_mlp_gdelta;
  a.mlp_x = S->d_mlp_x;
  a.mlp_z = S->d_mlp_z;
  a.mlp_dz = S->d_mlp_dz;
  a.mlp_done = S->d_mlp_done;
  a.mlp_lr = (float)S->opt.mlp_lr;
  a.mlp_warmup = S->opt.mlp_warmup;
  a.mlp_steps = S->opt.mlp_steps;
  a.mlp_wd = (float)S->opt.mlp_wd;
  a.mlp_wd_delta = (float)S->opt.mlp_wd_delta;
  a.mlp_eps = (float)S->opt.mlp_eps;
  return a;
}

int resident_blocks(epo_scene* S, int gather, int rpt, int block);

// Work items of the edge kernel, in the order the blocks claim them: (view, records
// [begin, begin + n), pairs [q0, q1) of the view's outgoing pair list).  Each item covers
// `tile` records and all of the view's pairs, except the last `grid` items (the final wave
// of a grid of that many blocks), which are split into items of at most `tail` pairs so
// that the blocks run out of work at nearly the same time.
epo_status build_tiles(epo_scene* S, int tile, int tail, int grid) {
  if (tail == 0) grid = 0;
  if (S->tiles_for == tile && S->tiles_tail == tail && S->tiles_grid == grid) return EPO_OK;
  S->graph_dirty = true;
  for (const auto& tt : S->tile_tables)
    if (tt.tile == tile && tt.tail == tail && tt.grid == grid) {
      S->d_tiles = tt.p;
      S->n_tiles = tt.n;
      S->tiles_for = tile;
      S->tiles_tail = tail;
      S->tiles_grid = grid;
      return EPO_OK;
    }
  std::vector<TileDev> t;
  for (int v = 0; v < S->n_views; ++v) {
    const ViewDev& vd = S->views[v];
    const int32_t q0 = S->src_pair_off[v], q1 = S->src_pair_off[v + 1];
    if (vd.n_rec == 0 || q1 == q0) continue;
    for (int64_t b = 0; b < vd.n_rec; b += tile) {
      TileDev td;
      td.view = v;
      td.begin = vd.rec_begin + b;
      td.n = (int32_t)std::min<int64_t>(tile, vd.n_rec - b);
      td.q0 = q0;
      td.q1 = q1;
      t.push_back(td);
    }
  }
  if (tail > 0 && !t.empty()) {
    const size_t keep = t.size() > (size_t)grid ? t.size() - (size_t)grid : 0;
    std::vector<TileDev> u(t.begin(), t.begin() + keep);
    for (size_t k = keep; k < t.size(); ++k)
      for (int32_t q = t[k].q0; q < t[k].q1; q += tail) {
        TileDev td = t[k];
        td.q0 = q;
        td.q1 = std::min(q + tail, t[k].q1);
        u.push_back(td);
      }
    t.swap(u);
  }
  TileDev* d = nullptr;
  ALLOC(d, t.size());
  if (!t.empty()) CK(cudaMemcpy(d, t.data(), t.size() * sizeof(TileDev), cudaMemcpyHostToDevice));
  S->tile_tables.push_back({tile, tail, grid, d, (int32_t)t.size()});
  S->d_tiles = d;
  S->n_tiles = (int32_t)t.size();
  S->tiles_for = tile;
  S->tiles_tail = tail;
  S->tiles_grid = grid;
  return EPO_OK;
}

// Work items of a schedule: block * rpt records each; with tail > 0 the last wave is one item
// per resident block (items of at most `tail` pairs), with tail < 0 every item covers at most
// -tail pairs (more, smaller items).
epo_status build_tiles(epo_scene* S, int gather, int rpt, int block, int tail) {
  if (tail < 0) return build_tiles(S, block * rpt, -tail, INT_MAX);
  return build_tiles(S, block * rpt, tail, tail ? resident_blocks(S, gather, rpt, block) : 0);
}

// The work items of the current schedule.
epo_status build_tiles(epo_scene* S) { return build_tiles(S, S->gather, S->rpt, S->block, S->tail); }

EdgeArgs edge_args(epo_scene* S) {
  EdgeArgs a;
  memset(&a, 0, sizeof(a));
  a.rec = S->d_rec;
  a.map = S->d_map;
  a.views = S->d_views;
  a.K64 = S->d_K64;
  a.tiles = S->d_tiles;
  a.n_tiles = S->n_tiles;
  a.src_pair_off = S->d_src_pair_off;
  a.src_pair_ids = S->d_src_pair_ids;
  a.pair_src = S->d_pair_src;
  a.pair_dst = S->d_pair_dst;
  a.pp = S->d_pp;
  a.pp64 = S->d_pp64;
  a.q_count = S->d_qcount;
  a.q_overflow = S->d_qoverflow;
  a.tile_counter = S->d_tile_counter;
  a.max_pairs = S->max_pairs;
  a.pair_active = S->d_active;
  a.tex = S->d_tex;
  a.pair_acc = S->d_pair_acc;
  a.lambda = S->d_lambda;
  a.delta = (float)S->opt.huber_delta;
  a.eps_z = (float)S->opt.eps_z;
  if (S->refine) {
    a.K64 = S->d_K64r;  // the lift and the exact path use the refined intrinsics
    a.gamma = S->d_gamma;
    a.alpha = S->d_alpha;
    a.beta = S->d_beta;
    a.pair_facc = S->d_pair_facc;
    a.dzr = S->d_dzr;
  }
  a.pair_lw = S->d_pair_lw;
  a.norm_all = S->opt.norm_mode == EPO_NORM_ALL;
  a.flag = S->d_flag;
  a.dbg = S->d_dbg;
  a.lift = S->d_lift;
  return a;
}

// Blocks of the persistent edge kernel: every SM holds as many as its registers, threads
// and shared memory allow (or the caller's fixed grid size).
int resident_blocks(epo_scene* S, int gather, int rpt, int block) {
  if (S->opt.grid_blocks > 0) return S->opt.grid_blocks;
  int per_sm = 0;
  const void* k = edge_kernel_ptr(MODE_FUSED, S->refine, S->rec_dtype, S->map_dtype, gather, rpt);
  const size_t smem = edge_smem_bytes(rpt, block, S->max_pairs, S->refine);
  if (smem > 48 * 1024 && k) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem) != cudaSuccess || per_sm < 1)
    per_sm = std::max(1, 1024 / block);
  return std::max(1, S->sm_count * per_sm);
}

// Launch size of the edge kernel for the current tile table.
int grid_for(epo_scene* S, int gather, int rpt, int block) {
  return std::max(1, std::min(resident_blocks(S, gather, rpt, block), std::max(S->n_tiles, 1)));
}

constexpr size_t kMaxSmem = 227 * 1024;

bool schedule_fits(epo_scene* S, int rpt, int block) {
  return (!S->refine || rpt == 2) && edge_smem_bytes(rpt, block, S->max_pairs, S->refine) <= kMaxSmem;
}

// Record stage event k on stream s (inside a capture it becomes an event-record node).
epo_status mark(epo_scene* S, int k, cudaStream_t s) {
  if (!S->ev[k]) return EPO_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(s, &cap));
  const unsigned int f = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  CK(cudaEventRecordWithFlags(S->ev[k], s, f));
  if (k == 3) S->ev_recorded = true;
  return EPO_OK;
}

#define MARK(k, s)                         \
  do {                                     \
    epo_status m_ = mark(S, (k), (s));     \
    if (m_ != EPO_OK) return m_;           \
  } while (0)

epo_status run_edge(epo_scene* S, int mode, int gather, int rpt, int block, int tail, cudaStream_t s) {
  if (!schedule_fits(S, rpt, block))
    return fail(S, EPO_ERR_INVALID_ARG, "schedule needs more shared memory than a block has");
  if (gather == GATHER_MIX && (S->refine || rpt == 1))
    return fail(S, EPO_ERR_INVALID_ARG, "the mixed gather needs a pose-only scene and two or more records per thread");
  epo_status st = build_tiles(S, gather, rpt, block, tail);
  if (st != EPO_OK) return st;
  EdgeArgs ea = edge_args(S);
  int grid = grid_for(S, gather, rpt, block);
  CK(launch_edge(ea, mode, S->refine, S->rec_dtype, S->map_dtype, gather, rpt, block, grid, s));
  MARK(2, s);
  return EPO_OK;
}

// One evaluation with gradient (a1 .. a8) on stream s.
epo_status enqueue_loss_grad(epo_scene* S, cudaStream_t s, const double* T_eval) {
  StepArgs a = step_args(S, T_eval, nullptr);
  MARK(0, s);
  if (S->subsample) CK(launch_subsample(a, s));
  if (S->refine) CK(launch_refine_intrinsics(a, s));
  CK(launch_pair_setup(a, MODE_FUSED, s));
  MARK(1, s);
  epo_status st = run_edge(S, MODE_FUSED, S->gather, S->rpt, S->block, S->tail, s);
  if (st != EPO_OK) return st;
  CK(launch_poses(a, 1, s));
  MARK(3, s);
  return EPO_OK;
}

// One optimisation step (a1 .. a9): pair setup, edge kernel, pose kernel; no host
// synchronisation.
// Refine scenes: the fused pass also stores every sample's d(rho)/dz; the pose kernel updates
// the poses and gamma, and with the depth module (lr_depth > 0) the depth kernel weights those
// derivatives by the pairs' w / n and updates alpha and beta.
// host_out: the mapped output block of the host-driven step, written by the pose kernel
// (NULL: none)
epo_status enqueue_step(epo_scene* S, cudaStream_t s, double* host_out = nullptr) {
  StepArgs a = step_args(S, S->d_T, nullptr);
  a.host_out = host_out;
  MARK(0, s);
  if (S->subsample) CK(launch_subsample(a, s));
  if (S->refine) CK(launch_refine_intrinsics(a, s));
  CK(launch_pair_setup(a, MODE_FUSED, s));
  MARK(1, s);
  epo_status st = run_edge(S, MODE_FUSED, S->gather, S->rpt, S->block, S->tail, s);
  if (st != EPO_OK) return st;
  CK(launch_poses(a, 2, s));
  if (S->pose_mlp) {  // the poses' gradient through phi and the MLP; AdamW (advances the step)
    CK(launch_mlp_backward(a, s));
    CK(launch_mlp_update(a, s));
  }
  if (S->depth_opt) CK(launch_depth(a, 1, s));
  if (S->pose_mlp) CK(launch_mlp_forward(a, 1, s));  // the next poses and their change
  if (S->opt.schedule) CK(launch_schedule(a, s));
  MARK(3, s);
  return EPO_OK;
}

// The host-driven step (epo_step_host) in one graph: a copy kernel brings the input poses from
// the mapped staging (with_in; timed against the pair setup reading them itself, which was
// slower: its uncached host reads cost more than the launch), and the pose kernel writes
// poses, loss and status word into the mapped output block when it is the step's last
// kernel; otherwise a copy kernel does.
epo_status enqueue_host_step(epo_scene* S, cudaStream_t s, bool with_in) {
  const bool fold_out = !S->pose_mlp && !S->depth_opt && !S->opt.schedule;
  if (with_in) CK(launch_io_copy(S->dh_in, S->d_T, 12 * (int64_t)S->n_views, s));
  epo_status st = enqueue_step(S, s, fold_out ? S->dh_io : nullptr);
  if (st != EPO_OK) return st;
  if (!fold_out) CK(launch_io_copy(S->d_io, S->dh_io, 12 * (int64_t)S->n_views + S->n_scenes + 1, s));
  return EPO_OK;
}

// host: 0 the plain step, 1 the host-driven step keeping the device's poses, 2 with input poses
epo_status capture(epo_scene* S, int host, cudaGraphExec_t* out) {
  CK(cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal));
  epo_status st = host ? enqueue_host_step(S, S->cap_stream, host == 2) : enqueue_step(S, S->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(S->cap_stream, &g);
  if (st != EPO_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(S, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(S, e, "cudaGraphInstantiate");
  return EPO_OK;
}

// (Re)captures the step graph when the schedule or the tile table changed; the host-step
// graphs are dropped with it and captured again on their next use.  host: as in capture().
epo_status ensure_graph(epo_scene* S, int host = 0) {
  // build the tile table outside capture (it allocates)
  epo_status st = build_tiles(S);
  if (st != EPO_OK) return st;
  if (S->graph_dirty || !S->graph) {
    if (S->graph) cudaGraphExecDestroy(S->graph);
    for (auto& g : S->graph_host)
      if (g) cudaGraphExecDestroy(g);
    S->graph = S->graph_host[0] = S->graph_host[1] = nullptr;
    st = capture(S, 0, &S->graph);
    if (st != EPO_OK) return st;
    S->graph_dirty = false;
  }
  if (host && !S->graph_host[host - 1]) return capture(S, host, &S->graph_host[host - 1]);
  return EPO_OK;
}

epo_status maybe_autotune(epo_scene* S) {
  if (S->opt.autotune && !S->tuned) return epo_autotune(S);
  return EPO_OK;
}

epo_status create_impl(int32_t n_scenes, const epo_scene_desc* descs, const epo_options* opts,
                       void* cuda_stream, epo_scene_t* out, epo_scene* S) {
  if (!descs || !out || n_scenes < 1) return fail(nullptr, EPO_ERR_INVALID_ARG, "null descriptor or n_scenes < 1");
  epo_default_options(&S->opt);
  if (opts) S->opt = *opts;
  const epo_options& o = S->opt;
  if (!(o.huber_delta > 0) || !(o.eps_z >= 0) || o.lambda_steps < 0 || !(o.lambda0 > 0) || !(o.lambda1 > 0) ||
      (o.norm_mode != EPO_NORM_VALID && o.norm_mode != EPO_NORM_ALL) || !(o.beta1 >= 0 && o.beta1 < 1) ||
      !(o.beta2 >= 0 && o.beta2 < 1) || !(o.adam_eps >= 0))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "invalid options");
  if (o.block_threads != 0 && (o.block_threads < 64 || o.block_threads > 512 || o.block_threads % 32))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "block_threads must be 64..512, a multiple of 32");
  if (o.records_per_thread != 0 && o.records_per_thread != 1 && o.records_per_thread != 2 &&
      o.records_per_thread != 4 && o.records_per_thread != 8)
    return fail(nullptr, EPO_ERR_INVALID_ARG, "records_per_thread must be 1, 2, 4 or 8");
  if (o.gather < EPO_GATHER_AUTO || o.gather > EPO_GATHER_MIX)
    return fail(nullptr, EPO_ERR_INVALID_ARG, "unknown gather mode");
  if (o.gather == EPO_GATHER_MIX && (o.refine || o.records_per_thread == 1))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "EPO_GATHER_MIX needs a pose-only scene and two or more records per thread");
  if (o.tail_pairs == INT_MIN) return fail(nullptr, EPO_ERR_INVALID_ARG, "tail_pairs out of range");
  if (o.refine != 0 && o.refine != 1) return fail(nullptr, EPO_ERR_INVALID_ARG, "refine must be 0 or 1");
  if (o.pair_budget < 0) return fail(nullptr, EPO_ERR_INVALID_ARG, "pair_budget must be >= 0");
  if (o.schedule != 0 && o.schedule != 1) return fail(nullptr, EPO_ERR_INVALID_ARG, "schedule must be 0 or 1");
  if (o.schedule && (o.sched_w1 < 1 || o.sched_w2 < 1 || !(o.sched_eps1 >= 0) || !(o.sched_eps2 >= 0)))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "schedule windows must be >= 1 and thresholds >= 0");
  if (o.refine && o.records_per_thread != 0 && o.records_per_thread != 2)
    return fail(nullptr, EPO_ERR_INVALID_ARG, "refine scenes run two records per thread");
  if (!(o.lr_focal >= 0) || !(o.lr_depth >= 0) || !isfinite(o.lr_focal) || !isfinite(o.lr_depth))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "lr_focal and lr_depth must be finite and >= 0");
  if (!o.refine && (o.lr_focal != 0 || o.lr_depth != 0))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "lr_focal and lr_depth need options.refine = 1");
  if (o.pose_param != EPO_POSE_SE3 && o.pose_param != EPO_POSE_MLP)
    return fail(nullptr, EPO_ERR_INVALID_ARG, "unknown pose_param");
  if (o.pose_param == EPO_POSE_MLP &&
      (!(o.mlp_lr >= 0) || !isfinite(o.mlp_lr) || o.mlp_warmup < 0 || o.mlp_steps < 1 || !(o.mlp_wd >= 0) ||
       !(o.mlp_wd_delta >= 0) || !(o.mlp_eps > 0)))
    return fail(nullptr, EPO_ERR_INVALID_ARG, "pose MLP: lr, decays >= 0, warmup >= 0, steps >= 1, eps > 0");
  S->refine = o.refine;
  S->depth_opt = o.refine && o.lr_depth > 0;
  S->pose_mlp = o.pose_param == EPO_POSE_MLP;
  S->stream = (cudaStream_t)cuda_stream;
  const int rec_dtype = descs[0].record_dtype, map_dtype = descs[0].map_dtype;
  if (rec_dtype != EPO_F32 && rec_dtype != EPO_F16) return fail(nullptr, EPO_ERR_INVALID_ARG, "unknown record dtype");
  if (map_dtype != EPO_F32 && map_dtype != EPO_BF16) return fail(nullptr, EPO_ERR_INVALID_ARG, "unknown map dtype");
  S->rec_dtype = rec_dtype == EPO_F16 ? 1 : 0;
  S->map_dtype = map_dtype == EPO_BF16 ? 1 : 0;
  const size_t rec_size = S->rec_dtype ? 8 : 16;
  const size_t map_size = S->map_dtype ? 2 : 4;
  // ---- validate descriptors, count ----
  int64_t nv = 0, np = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const epo_scene_desc& d = descs[s];
    if (d.record_dtype != rec_dtype || d.map_dtype != map_dtype)
      return fail(nullptr, EPO_ERR_INVALID_ARG, "all scenes of a batch must share the dtypes");
    if (d.n_views < 1 || !d.views) return fail(nullptr, EPO_ERR_INVALID_ARG, "scene without views");
    if (d.n_pairs < 1 || !d.pairs) return fail(nullptr, EPO_ERR_INVALID_ARG, "scene without pairs");
    for (int v = 0; v < d.n_views; ++v) {
      const epo_view_desc& vd = d.views[v];
      if (vd.W < 2 || vd.H < 2) return fail(nullptr, EPO_ERR_INVALID_ARG, "view with W or H < 2");
      if (vd.W > 65535 || vd.H > 65535) return fail(nullptr, EPO_ERR_INVALID_ARG, "view larger than 65535");
      if (!(vd.fx > 0) || !(vd.fy > 0) || !isfinite(vd.cx) || !isfinite(vd.cy) || !isfinite(vd.fx) || !isfinite(vd.fy))
        return fail(nullptr, EPO_ERR_INVALID_ARG, "invalid intrinsics");
      if (vd.n_records < 0 || (vd.n_records > 0 && !vd.records))
        return fail(nullptr, EPO_ERR_INVALID_ARG, "invalid records");
      if (!vd.map) return fail(nullptr, EPO_ERR_INVALID_ARG, "view without a map");
    }
    for (int p = 0; p < d.n_pairs; ++p) {
      int i = d.pairs[2 * p], j = d.pairs[2 * p + 1];
      if (i < 0 || i >= d.n_views || j < 0 || j >= d.n_views)
        return fail(nullptr, EPO_ERR_INVALID_ARG, "pair index out of range");
    }
    nv += d.n_views;
    np += d.n_pairs;
  }
  if (nv > (1 << 28) || np > (1 << 28)) return fail(nullptr, EPO_ERR_INVALID_ARG, "too many views or pairs");
  S->n_scenes = n_scenes;
  S->n_views = (int)nv;
  S->n_pairs = (int)np;
  // ---- device properties ----
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
  // ---- records (host-side filtering) and host tables ----
  std::vector<uint8_t> rec_host;
  std::vector<uint8_t> tmp;
  S->views.resize(nv);
  std::vector<int32_t> pose_pair_cnt(nv, 0);
  std::vector<uint8_t> fixed(nv, 0);
  int64_t vbase = 0, map_off = 0, rec_off = 0;
  const int64_t pitch_mult = 128 / (int64_t)map_size;           // 128-byte rows
  const int64_t base_mult = 512 / (int64_t)map_size;            // 512-byte view starts
  S->scene_pair_off.push_back(0);
  for (int s = 0; s < n_scenes; ++s) {
    const epo_scene_desc& d = descs[s];
    for (int v = 0; v < d.n_views; ++v) {
      const epo_view_desc& vd = d.views[v];
      ViewDev& w = S->views[vbase + v];
      w.fx = (float)vd.fx; w.fy = (float)vd.fy; w.cx = (float)vd.cx; w.cy = (float)vd.cy;
      w.W = vd.W; w.H = vd.H;
      w.pitch = (int32_t)round_up(vd.W, pitch_mult);
      w.scene = s;
      map_off = round_up(map_off, base_mult);
      w.map_off = map_off;
      map_off += (int64_t)w.pitch * vd.H;
      w.rec_begin = rec_off;
      w.pad_ = 0;
      const uint8_t* src = (const uint8_t*)vd.records;
      if (vd.n_records > 0 && d.pointers_on_device) {
        tmp.resize((size_t)vd.n_records * rec_size);
        e = cudaMemcpy(tmp.data(), vd.records, tmp.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMemcpy records D2H");
        src = tmp.data();
      }
      int64_t kept = 0;
      for (int64_t r = 0; r < vd.n_records; ++r) {
        const uint8_t* q = src + (size_t)r * rec_size;
        float z, u, vv;
        if (S->rec_dtype == 0) {
          float f4[4];
          memcpy(f4, q, 16);
          u = f4[0]; vv = f4[1]; z = f4[2];
          if (!isfinite(u) || !isfinite(vv)) { ++S->n_dropped; continue; }
        } else {
          uint16_t h[4];
          memcpy(h, q, 8);
          z = half_bits_to_float(h[2]);
          (void)u; (void)vv;
        }
        if (!(z > 0.f) || !isfinite(z)) { ++S->n_dropped; continue; }
        rec_host.insert(rec_host.end(), q, q + rec_size);
        ++kept;
      }
      if (kept > INT32_MAX) return fail(nullptr, EPO_ERR_INVALID_ARG, "too many records in one view");
      w.n_rec = (int32_t)kept;
      rec_off += kept;
      if (d.fixed) fixed[vbase + v] = d.fixed[v] ? 1 : 0;
    }
    for (int p = 0; p < d.n_pairs; ++p) {
      const int i = (int)vbase + d.pairs[2 * p], j = (int)vbase + d.pairs[2 * p + 1];
      S->pair_src.push_back(i);
      S->pair_dst.push_back(j);
      S->pair_scene.push_back(s);
      pose_pair_cnt[i]++;
      pose_pair_cnt[j]++;
    }
    S->scene_pair_off.push_back((int32_t)S->pair_src.size());
    S->scene_active.push_back(d.n_pairs);
    vbase += d.n_views;
  }
  S->n_records = rec_off;
  S->map_elems = std::max<int64_t>(map_off, 1);
  S->active.assign(np, 1);
  // pairs grouped by source view
  S->src_pair_off.assign(nv + 1, 0);
  for (int p = 0; p < np; ++p) S->src_pair_off[S->pair_src[p] + 1]++;
  for (int v = 0; v < nv; ++v) {
    S->max_pairs = std::max(S->max_pairs, S->src_pair_off[v + 1]);
    S->src_pair_off[v + 1] += S->src_pair_off[v];
  }
  if (S->max_pairs > 512) return fail(nullptr, EPO_ERR_INVALID_ARG, "a view with more than 512 outgoing pairs");
  S->src_pair_ids.assign(np, 0);
  {
    std::vector<int32_t> fill(S->src_pair_off.begin(), S->src_pair_off.end() - 1);
    for (int p = 0; p < np; ++p) S->src_pair_ids[fill[S->pair_src[p]]++] = p;
  }
  // per pose: (pair, role) in pair order -> deterministic gather
  std::vector<int32_t>& pose_off = S->pose_off;
  std::vector<int32_t>& pose_ref = S->pose_ref;
  pose_off.assign(nv + 1, 0);
  pose_ref.assign(2 * np, 0);
  for (int v = 0; v < nv; ++v) pose_off[v + 1] = pose_off[v] + pose_pair_cnt[v];
  {
    std::vector<int32_t> fill(pose_off.begin(), pose_off.end() - 1);
    for (int p = 0; p < np; ++p) {
      pose_ref[fill[S->pair_dst[p]]++] = 2 * p + 0;
      pose_ref[fill[S->pair_src[p]]++] = 2 * p + 1;
    }
  }
  S->evals = 0;
  for (int p = 0; p < np; ++p) S->evals += S->views[S->pair_src[p]].n_rec;
  S->n_dzr = S->refine ? S->evals : 0;  // one d(rho)/dz per evaluation of a refine scene
  for (int sc = 0; sc < n_scenes; ++sc)
    if (o.pair_budget > 0 && S->scene_pair_off[sc + 1] - S->scene_pair_off[sc] > o.pair_budget) S->subsample = 1;
  // ---- device allocations (CK / ALLOC report into the handle under construction) ----
  {
    e = cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(S, e, "cudaStreamCreate");
    ALLOC(*(uint8_t**)&S->d_rec, std::max<size_t>(rec_host.size(), 16));
    if (!S->refine) ALLOC(S->d_lift, std::max<int64_t>(S->n_records, 1));
    {
      uint8_t* raw = nullptr;
      ALLOC(raw, (size_t)S->map_elems * map_size + 512);
      S->d_map = (void*)(((uintptr_t)raw + 511) & ~(uintptr_t)511);
    }
    ALLOC(S->d_views, nv);
    ALLOC(S->d_src_pair_off, nv + 1);
    ALLOC(S->d_src_pair_ids, np);
    ALLOC(S->d_pair_src, np);
    ALLOC(S->d_pair_dst, np);
    ALLOC(S->d_pair_scene, np);
    ALLOC(S->d_scene_pair_off, n_scenes + 1);
    ALLOC(S->d_scene_active, n_scenes);
    ALLOC(S->d_pose_pair_off, nv + 1);
    ALLOC(S->d_pose_pair_ref, 2 * np);
    ALLOC(S->d_active, np);
    ALLOC(S->d_fixed, nv);
    ALLOC(S->d_tex, nv);
    ALLOC(S->d_pp, np);
    ALLOC(S->d_pair_q, np);
    ALLOC(S->d_pp64, (size_t)kPP64 * np);
    ALLOC(S->d_K64, (size_t)6 * nv);
    ALLOC(S->d_pair_acc, (size_t)kAcc * np);
    ALLOC(S->d_grad, (size_t)6 * nv);
    // the poses, the per-scene loss and the status flag in one block, so that a host-driven
    // step (epo_step_host) reads them back with a single copy
    ALLOC(S->d_io, (size_t)12 * nv + n_scenes + 1);
    S->d_T = S->d_io;
    S->d_loss = S->d_io + 12 * (size_t)nv;
    S->d_flag = reinterpret_cast<int32_t*>(S->d_io + 12 * (size_t)nv + n_scenes);
    ALLOC(S->d_m, (size_t)6 * nv);
    ALLOC(S->d_v, (size_t)6 * nv);
    ALLOC(S->d_bpow, 2);
    {
      ALLOC(S->d_qcount, 1);
      ALLOC(S->d_qoverflow, 1);
      ALLOC(S->d_tile_counter, 1);
    }
    ALLOC(S->d_lambda, 1);
    ALLOC(S->d_T_eval, (size_t)12 * nv);
    ALLOC(S->d_step, 1);
    ALLOC(S->d_done, 1);
    std::vector<int32_t> chunk_off(1, 0), chunk_scene;
    for (int sc = 0; sc < n_scenes; ++sc) {
      const int32_t np_s = S->scene_pair_off[sc + 1] - S->scene_pair_off[sc];
      const int32_t nc = (np_s + kLossChunk - 1) / kLossChunk;
      for (int32_t c = 0; c < nc; ++c) chunk_scene.push_back(sc);
      chunk_off.push_back(chunk_off.back() + nc);
    }
    S->n_loss_chunks = chunk_off.back();
    std::vector<int2> chunk_pairs(chunk_scene.size());
    for (size_t c = 0; c < chunk_scene.size(); ++c) {
      const int sc = chunk_scene[c];
      const int first = S->scene_pair_off[sc] + (int)(c - chunk_off[sc]) * kLossChunk;
      chunk_pairs[c] = make_int2(first, std::min(first + kLossChunk, S->scene_pair_off[sc + 1]));
    }
    ALLOC(S->d_loss_chunk_off, n_scenes + 1);
    ALLOC(S->d_loss_chunk_scene, chunk_scene.size());
    ALLOC(S->d_loss_chunk_pairs, chunk_scene.size());
    ALLOC(S->d_loss_part, chunk_scene.size());
    ALLOC(S->d_scene_done, n_scenes);
    std::vector<int2> pair_ij(np);
    for (int p = 0; p < np; ++p) pair_ij[p] = make_int2(S->pair_src[p], S->pair_dst[p]);
    S->pose_stride = 1;
    for (int v = 0; v < nv; ++v) S->pose_stride = std::max(S->pose_stride, pose_off[v + 1] - pose_off[v]);
    ALLOC(S->d_pair_ij, np);
    ALLOC(S->d_pair_lw, np);
    ALLOC(S->d_pose_entries, (size_t)nv * S->pose_stride);
    S->scene_view_begin.assign(1, 0);
    for (int sc = 0; sc < n_scenes; ++sc) S->scene_view_begin.push_back(S->scene_view_begin.back() + descs[sc].n_views);
    if (o.schedule || o.pose_param == EPO_POSE_MLP) {  // views of each scene (contiguous)
      ALLOC(S->d_scene_view_off, n_scenes + 1);
      CK(cudaMemcpy(S->d_scene_view_off, S->scene_view_begin.data(), (n_scenes + 1) * 4, cudaMemcpyHostToDevice));
    }
    if (o.schedule) {
      ALLOC(S->d_pose_dR, nv);
      ALLOC(S->d_pose_dt, nv);
      ALLOC(S->d_sched_state, 2 * (size_t)n_scenes);
      ALLOC(S->d_theta95, n_scenes);
      ALLOC(S->d_sched_steps, 2 * (size_t)n_scenes);
      std::vector<int32_t> ss(2 * (size_t)n_scenes);
      for (int sc = 0; sc < n_scenes; ++sc) {
        ss[2 * sc] = 1;
        ss[2 * sc + 1] = 0;
      }
      std::vector<int64_t> steps(2 * (size_t)n_scenes, -1);
      std::vector<double> th(n_scenes, 0.0);
      CK(cudaMemcpy(S->d_sched_state, ss.data(), ss.size() * 4, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(S->d_sched_steps, steps.data(), steps.size() * 8, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(S->d_theta95, th.data(), th.size() * 8, cudaMemcpyHostToDevice));
      CK(cudaMemset(S->d_pose_dR, 0, (size_t)nv * 8));
      CK(cudaMemset(S->d_pose_dt, 0, (size_t)nv * 8));
    }
    if (S->pose_mlp) {
      const size_t np_ = (size_t)n_scenes * kMlpParams;
      ALLOC(S->d_mlp_theta, np_);
      ALLOC(S->d_mlp_m, np_);
      ALLOC(S->d_mlp_v, np_);
      ALLOC(S->d_mlp_P0, 12 * (size_t)nv);
      ALLOC(S->d_mlp_Pp, 12 * (size_t)nv);
      ALLOC(S->d_mlp_delta, 3 * (size_t)nv);
      ALLOC(S->d_mlp_dm, 3 * (size_t)nv);
      ALLOC(S->d_mlp_dv, 3 * (size_t)nv);
      ALLOC(S->d_mlp_gdelta, 3 * (size_t)nv);
      ALLOC(S->d_mlp_x, 12 * (size_t)nv);
      ALLOC(S->d_mlp_z, 5 * (size_t)kMlpHid * nv);
      ALLOC(S->d_mlp_dz, (size_t)kMlpDz * nv);
      ALLOC(S->d_mlp_done, 1);
      ALLOC(S->d_mlp_scale, n_scenes);
      {
        std::vector<double> one(n_scenes, 1.0);  // identity poses: the centres coincide
        CK(cudaMemcpy(S->d_mlp_scale, one.data(), one.size() * 8, cudaMemcpyHostToDevice));
      }
      for (float* q : {S->d_mlp_theta, S->d_mlp_m, S->d_mlp_v}) CK(cudaMemset(q, 0, np_ * 4));
      for (float* q : {S->d_mlp_delta, S->d_mlp_dm, S->d_mlp_dv, S->d_mlp_gdelta}) CK(cudaMemset(q, 0, 12 * (size_t)nv));
      CK(cudaMemset(S->d_mlp_done, 0, 4));
    }
    if (S->refine) {
      ALLOC(S->d_gamma, nv);
      ALLOC(S->d_K64r, (size_t)6 * nv);
      ALLOC(S->d_pair_facc, (size_t)2 * np);
      ALLOC(S->d_grad_gamma, nv);
      const size_t nr = (size_t)std::max<int64_t>(S->n_records, 1);
      ALLOC(S->d_alpha, nr);
      ALLOC(S->d_beta, nr);
      ALLOC(S->d_dzr, (size_t)std::max<int64_t>(S->n_dzr, 1));
      ALLOC(S->d_pair_wz, np);
      ALLOC(S->d_grad_alpha, nr);
      ALLOC(S->d_grad_beta, nr);
      ALLOC(S->d_mg, nv);
      ALLOC(S->d_vg, nv);
      ALLOC(S->d_ma, nr);
      ALLOC(S->d_va, nr);
      ALLOC(S->d_mb, nr);
      ALLOC(S->d_vb, nr);
      for (const ViewDev& w : S->views) S->max_view_records = std::max(S->max_view_records, w.n_rec);
    }
    CK(cudaMallocHost(&S->h_flag, sizeof(int32_t)));
    CK(cudaMallocHost(&S->h_out, ((size_t)n_scenes + 18 * nv) * 8));
    CK(cudaEventCreateWithFlags(&S->ev_wait, cudaEventDisableTiming));
    CK(cudaHostAlloc(&S->h_io, ((size_t)12 * nv + n_scenes + 1) * 8, cudaHostAllocMapped));
    CK(cudaHostAlloc(&S->h_in, (size_t)12 * nv * 8, cudaHostAllocMapped));
    memset(S->h_io, 0, ((size_t)12 * nv + n_scenes + 1) * 8);
    memset(S->h_in, 0, (size_t)12 * nv * 8);
    {
      void* d = nullptr;
      CK(cudaHostGetDevicePointer(&d, S->h_io, 0));
      S->dh_io = reinterpret_cast<double*>(d);
      CK(cudaHostGetDevicePointer(&d, S->h_in, 0));
      S->dh_in = reinterpret_cast<const double*>(d);
    }
    cudaStream_t st = S->stream;
    if (!rec_host.empty()) CK(cudaMemcpyAsync(S->d_rec, rec_host.data(), rec_host.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(S->d_map, 0, (size_t)S->map_elems * map_size, st));
    vbase = 0;
    for (int s = 0; s < n_scenes; ++s) {
      const epo_scene_desc& d = descs[s];
      for (int v = 0; v < d.n_views; ++v) {
        const ViewDev& w = S->views[vbase + v];
        CK(cudaMemcpy2DAsync((uint8_t*)S->d_map + w.map_off * map_size, (size_t)w.pitch * map_size,
                             d.views[v].map, (size_t)w.W * map_size, (size_t)w.W * map_size, w.H,
                             d.pointers_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      }
      vbase += d.n_views;
    }
    CK(cudaMemcpyAsync(S->d_views, S->views.data(), nv * sizeof(ViewDev), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_src_pair_off, S->src_pair_off.data(), (nv + 1) * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_src_pair_ids, S->src_pair_ids.data(), np * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_pair_src, S->pair_src.data(), np * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_pair_dst, S->pair_dst.data(), np * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_pair_scene, S->pair_scene.data(), np * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_scene_pair_off, S->scene_pair_off.data(), (n_scenes + 1) * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_scene_active, S->scene_active.data(), n_scenes * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_pose_pair_off, pose_off.data(), (nv + 1) * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_pose_pair_ref, pose_ref.data(), 2 * np * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_active, S->active.data(), np, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_fixed, fixed.data(), nv, cudaMemcpyHostToDevice, st));
    // identity poses, zero optimiser state
    std::vector<double> I(12 * (size_t)nv, 0.0);
    for (int v = 0; v < nv; ++v) I[12 * v] = I[12 * v + 5] = I[12 * v + 10] = 1.0;
    CK(cudaMemcpyAsync(S->d_T, I.data(), I.size() * 8, cudaMemcpyHostToDevice, st));
    if (S->pose_mlp) CK(cudaMemcpyAsync(S->d_mlp_P0, I.data(), I.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(S->d_m, 0, 6 * (size_t)nv * 8, st));
    CK(cudaMemsetAsync(S->d_v, 0, 6 * (size_t)nv * 8, st));
    {
      const double bp[2] = {o.beta1, o.beta2};
      CK(cudaMemcpy(S->d_bpow, bp, sizeof(bp), cudaMemcpyHostToDevice));
      std::vector<double> K64(6 * (size_t)nv);
      int64_t vb = 0;
      for (int s2 = 0; s2 < n_scenes; ++s2) {
        for (int v = 0; v < descs[s2].n_views; ++v) {
          const epo_view_desc& vd = descs[s2].views[v];
          K64[6 * (vb + v) + 0] = vd.fx;
          K64[6 * (vb + v) + 1] = vd.fy;
          K64[6 * (vb + v) + 2] = vd.cx;
          K64[6 * (vb + v) + 3] = vd.cy;
          K64[6 * (vb + v) + 4] = 1.0 / vd.fx;
          K64[6 * (vb + v) + 5] = 1.0 / vd.fy;
        }
        vb += descs[s2].n_views;
      }
      CK(cudaMemcpy(S->d_K64, K64.data(), K64.size() * 8, cudaMemcpyHostToDevice));
    }
    // the intrinsics and depths of a pose-only scene stay fixed: its records are lifted once
    if (S->d_lift)
      CK(launch_lift_records(S->d_rec, S->rec_dtype, S->d_views, S->d_K64, (int)nv, (float)o.eps_z, S->d_lift, st));
    CK(cudaMemsetAsync(S->d_qcount, 0, 4, st));
    CK(cudaMemsetAsync(S->d_qoverflow, 0, 4, st));
    CK(cudaMemsetAsync(S->d_step, 0, 8, st));
    CK(cudaMemsetAsync(S->d_flag, 0, 4, st));
    ALLOC(S->d_dbg, 4);
    CK(cudaMemsetAsync(S->d_dbg, 0xff, 16, st));
    CK(cudaMemsetAsync(S->d_done, 0, 8, st));
    CK(cudaMemsetAsync(S->d_scene_done, 0, 4 * (size_t)n_scenes, st));
    CK(cudaMemcpyAsync(S->d_loss_chunk_off, chunk_off.data(), chunk_off.size() * 4, cudaMemcpyHostToDevice, st));
    if (!chunk_pairs.empty())
      CK(cudaMemcpyAsync(S->d_loss_chunk_pairs, chunk_pairs.data(), chunk_pairs.size() * sizeof(int2),
                         cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_pair_ij, pair_ij.data(), (size_t)np * sizeof(int2), cudaMemcpyHostToDevice, st));
    if (!chunk_scene.empty())
      CK(cudaMemcpyAsync(S->d_loss_chunk_scene, chunk_scene.data(), chunk_scene.size() * 4, cudaMemcpyHostToDevice,
                         st));
    CK(cudaMemsetAsync(S->d_pair_acc, 0, (size_t)kAcc * np * 8, st));
    if (S->refine) {
      epo_status rs = epo_set_refinement(S, nullptr, nullptr, nullptr);  // identity: gamma 0, alpha 1, beta 0
      if (rs != EPO_OK) return rs;
      CK(cudaMemsetAsync(S->d_pair_facc, 0, (size_t)2 * np * 8, st));
    }
    if (S->pose_mlp) CK(launch_mlp_forward(step_args(S, S->d_T, nullptr), 0, st));  // zero MLP: P^s = P^0
    // validate maps on the device
    CK(launch_map_check(S->d_map, S->map_dtype, S->map_elems, S->d_flag, st));
    CK(cudaMemcpyAsync(S->h_flag, S->d_flag, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*S->h_flag != 0)
      return fail(nullptr, EPO_ERR_INVALID_ARG, "map with a non-finite or negative value");
    CK(cudaMemsetAsync(S->d_flag, 0, 4, st));
    // texture path: one gather-capable 2-D CUDA array per view (texture gather is defined
    // for arrays created with cudaArrayTextureGather), filled from the atlas
    S->tex.assign(nv, 0);
    S->arrays.assign(nv, nullptr);
    const cudaChannelFormatDesc cfd = S->map_dtype ? cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned)
                                                   : cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat);
    for (int v = 0; v < nv; ++v) {
      const ViewDev& w = S->views[v];
      CK(cudaMallocArray(&S->arrays[v], &cfd, w.W, w.H, cudaArrayTextureGather));
      S->device_bytes += (int64_t)w.W * w.H * (int64_t)map_size;
      CK(cudaMemcpy2DToArrayAsync(S->arrays[v], 0, 0, (uint8_t*)S->d_map + w.map_off * map_size,
                                  (size_t)w.pitch * map_size, (size_t)w.W * map_size, w.H,
                                  cudaMemcpyDeviceToDevice, st));
      cudaResourceDesc rd;
      memset(&rd, 0, sizeof(rd));
      rd.resType = cudaResourceTypeArray;
      rd.res.array.array = S->arrays[v];
      cudaTextureDesc td;
      memset(&td, 0, sizeof(td));
      td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
      td.filterMode = cudaFilterModePoint;
      td.readMode = cudaReadModeElementType;
      td.normalizedCoords = 0;
      CK(cudaCreateTextureObject(&S->tex[v], &rd, &td, nullptr));
    }
    std::vector<unsigned long long> th(S->tex.begin(), S->tex.end());
    CK(cudaMemcpyAsync(S->d_tex, th.data(), nv * 8, cudaMemcpyHostToDevice, st));
    // the fields of every PairParam that do not change with the poses: the target's
    // intrinsics, map and the constants of the rounding-error bound (the pair setup writes
    // the relative pose and its bound each step)
    {
      std::vector<PairParam> pp(np);
      std::vector<int32_t> pair_q(np);
      for (int k = 0; k < np; ++k) pair_q[S->src_pair_ids[k]] = k;
      for (int p = 0; p < np; ++p) {
        PairParam& q = pp[pair_q[p]];
        memset(&q, 0, sizeof(q));
        const ViewDev& vj = S->views[S->pair_dst[p]];
        q.fx = vj.fx; q.fy = vj.fy; q.cx = vj.cx; q.cy = vj.cy;
        q.p = p;
        q.active = 1;  // the pair setup copies the step's flag
        q.hw = 0.5f * (float)(vj.W - 1);
        q.hh = 0.5f * (float)(vj.H - 1);
        q.cu = 4.f * kU32 * (float)(vj.W + 1);
        q.cv = 4.f * kU32 * (float)(vj.H + 1);
        q.W = vj.W; q.H = vj.H; q.pitch = vj.pitch;
        q.map_off = vj.map_off;
        q.tex = th[S->pair_dst[p]];
        // the pose-only kernel's bound t = E |1/Y3| Kb + cb on the error of u' and v' (the
        // kernel's header derives it): for a sample within one pixel of the image
        // |u'* - cx| <= max(cx + 1, W - cx) + 1/4 once t <= 1/4; 1e-5 relative margin
        const double mu = std::max((double)vj.cx + 1.0, (double)vj.W - (double)vj.cx);
        const double mv = std::max((double)vj.cy + 1.0, (double)vj.H - (double)vj.cy);
        const double ku = (double)vj.fx + mu + 0.25, kv = (double)vj.fy + mv + 0.25;
        const double cu = (double)vj.W + 4.0 * mu + std::fabs((double)vj.cx);
        const double cv = (double)vj.H + 4.0 * mv + std::fabs((double)vj.cy);
        q.Kb = (float)(std::max(ku, kv) * (1.0 + 1e-5));
        q.cb = (float)((double)kU32 * std::max(cu, cv) * (1.0 + 1e-5));
        q.Wm2 = (float)(vj.W - 2);
        q.Hm2 = (float)(vj.H - 2);
        q.Wf = (float)vj.W;
        q.Hf = (float)vj.H;
      }
      if (S->refine) {  // each pair's block of d(rho)/dz values, one per source record
        int64_t run = 0;
        for (int v = 0; v < nv; ++v)
          for (int k = S->src_pair_off[v]; k < S->src_pair_off[v + 1]; ++k) {
            pp[k].dbase = run - S->views[v].rec_begin;
            run += S->views[v].n_rec;
          }
      }
      CK(cudaMemcpyAsync(S->d_pp, pp.data(), (size_t)np * sizeof(PairParam), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(S->d_pair_q, pair_q.data(), (size_t)np * 4, cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    }
    {
      epo_status ws = upload_weights(S, st);
      if (ws != EPO_OK) return ws;
    }
    if (o.timing)
      for (auto& e2 : S->ev) CK(cudaEventCreate(&e2));
    // schedule
    S->block = o.block_threads ? o.block_threads : 256;
    S->rpt = o.records_per_thread ? o.records_per_thread : 2;
    S->gather = o.gather == EPO_GATHER_TEX ? GATHER_TEX : (o.gather == EPO_GATHER_MIX ? GATHER_MIX : GATHER_LDG);
    if (!schedule_fits(S, S->rpt, S->block)) S->block = 128;
    S->tail = o.tail_pairs == -1 ? 0 : o.tail_pairs;
    epo_status bs = build_tiles(S);
    if (bs != EPO_OK) return bs;
    CK(cudaStreamSynchronize(st));
  }
  *out = S;
  return EPO_OK;
}

void destroy_impl(epo_scene* S) {
  if (!S) return;
  if (S->graph) cudaGraphExecDestroy(S->graph);
  for (auto g : S->graph_host)
    if (g) cudaGraphExecDestroy(g);
  for (auto e2 : S->ev)
    if (e2) cudaEventDestroy(e2);
  for (auto t : S->tex)
    if (t) cudaDestroyTextureObject(t);
  for (auto a : S->arrays)
    if (a) cudaFreeArray(a);
  for (auto& b : S->bufs)
    if (b.p) cudaFree(b.p);
  if (S->h_flag) cudaFreeHost(S->h_flag);
  if (S->h_out) cudaFreeHost(S->h_out);
  if (S->ev_wait) cudaEventDestroy(S->ev_wait);
  if (S->h_io) cudaFreeHost(S->h_io);
  if (S->h_in) cudaFreeHost(S->h_in);
  if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
  delete S;
}

}  // namespace

extern "C" {

void epo_default_options(epo_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->huber_delta = 1.0;
  o->lambda0 = 10.0;
  o->lambda1 = 6.0;
  o->lambda_steps = 1000;
  o->eps_z = 1e-6;
  o->norm_mode = EPO_NORM_VALID;
  o->lr_rot = 2e-3;
  o->lr_trans = 2e-2;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->adam_eps = 1e-12;
  o->autotune = 0;
  o->gather = EPO_GATHER_AUTO;
  o->tail_pairs = -1;
  o->sched_eps1 = 0.5;  // degrees; the paper's windows and tolerances
  o->sched_eps2 = 0.1;
  o->sched_w1 = 25;
  o->sched_w2 = 50;
  o->pose_param = EPO_POSE_SE3;
  o->mlp_lr = 3e-3;  // Section 3, Implementation Details
  o->mlp_warmup = 25;
  o->mlp_steps = 2000;
  o->mlp_wd = 0.01;
  o->mlp_wd_delta = 0.1;
  o->mlp_eps = 1e-8;
}

int32_t epo_abi_version(void) { return EPO_ABI_VERSION; }

epo_status epo_create_scene(const epo_scene_desc* desc, const epo_options* opts, void* cuda_stream,
                            epo_scene_t* out) {
  EPO_RANGE("epo_create_scene");
  return epo_create_batch(1, desc, opts, cuda_stream, out);
}

epo_status epo_create_batch(int32_t n_scenes, const epo_scene_desc* descs, const epo_options* opts,
                            void* cuda_stream, epo_scene_t* out) {
  EPO_RANGE("epo_create_batch");
  if (out) *out = nullptr;
  epo_scene* S = new (std::nothrow) epo_scene();
  if (!S) return fail(nullptr, EPO_ERR_OOM, "host allocation failed");
  epo_status st = create_impl(n_scenes, descs, opts, cuda_stream, out, S);
  if (st != EPO_OK) {
    if (!S->err.empty()) g_create_error = S->err;
    destroy_impl(S);
    if (out) *out = nullptr;
  }
  return st;
}

void epo_destroy_scene(epo_scene_t S) {
  EPO_RANGE("epo_destroy_scene");
  if (S) cudaStreamSynchronize(S->stream);
  destroy_impl(S);
}

const char* epo_last_error(epo_scene_t S) { return S ? S->err.c_str() : g_create_error.c_str(); }

epo_status epo_scene_info_get(epo_scene_t S, epo_scene_info* info) {
  EPO_RANGE("epo_scene_info_get");
  if (!S || !info) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  info->n_scenes = S->n_scenes;
  info->n_views = S->n_views;
  info->n_pairs = S->n_pairs;
  info->n_records = S->n_records;
  info->n_dropped = S->n_dropped;
  int64_t ev = 0;
  if (S->subsample) {
    // a random subset each step: the expected count, min(1, M / P_s) of every pair's records
    double e = 0.0;
    for (int sc = 0; sc < S->n_scenes; ++sc) {
      const int P = S->scene_pair_off[sc + 1] - S->scene_pair_off[sc];
      const double f = P > S->opt.pair_budget ? (double)S->opt.pair_budget / P : 1.0;
      for (int p = S->scene_pair_off[sc]; p < S->scene_pair_off[sc + 1]; ++p)
        e += f * (double)S->views[S->pair_src[p]].n_rec;
    }
    ev = (int64_t)llround(e);
  } else {
    for (int p = 0; p < S->n_pairs; ++p)
      if (S->active[p]) ev += S->views[S->pair_src[p]].n_rec;
  }
  info->evals_per_step = ev;
  info->device_bytes = S->device_bytes;
  info->record_bytes = S->n_records * (S->rec_dtype ? 8 : 16);
  info->map_bytes = S->map_elems * (S->map_dtype ? 2 : 4);
  info->n_tiles = S->n_tiles;
  info->gather = S->gather;
  info->block_threads = S->block;
  info->records_per_thread = S->rpt;
  info->grid_blocks = grid_for(S, S->gather, S->rpt, S->block);
  info->kernels_per_step = 3 + S->refine + S->subsample + S->opt.schedule + S->depth_opt + 3 * S->pose_mlp;
  info->tail_pairs = S->tail;
  return EPO_OK;
}

// Per scene the RMS distance of the camera centres c = -R^T t of the poses T from their
// centroid (1 if they coincide): the pose MLP acts on the scene at this unit scale.
static epo_status set_mlp_scale(epo_scene* S, const double* T) {
  std::vector<double> sc(S->n_scenes, 1.0);
  for (int s = 0; s < S->n_scenes; ++s) {
    const int v0 = S->scene_view_begin[s], v1 = S->scene_view_begin[s + 1];
    double mean[3] = {0, 0, 0}, acc = 0.0;
    std::vector<double> C(3 * (size_t)(v1 - v0));
    for (int v = v0; v < v1; ++v) {
      const double* P = T + 12 * (size_t)v;
      for (int k = 0; k < 3; ++k) {
        C[3 * (v - v0) + k] = -(P[k] * P[3] + P[4 + k] * P[7] + P[8 + k] * P[11]);
        mean[k] += C[3 * (v - v0) + k] / (v1 - v0);
      }
    }
    for (int v = 0; v < v1 - v0; ++v)
      for (int k = 0; k < 3; ++k) acc += (C[3 * v + k] - mean[k]) * (C[3 * v + k] - mean[k]);
    const double r = v1 > v0 ? sqrt(acc / (v1 - v0)) : 0.0;
    sc[s] = r > 0.0 ? r : 1.0;
  }
  CK(cudaMemcpyAsync(S->d_mlp_scale, sc.data(), sc.size() * 8, cudaMemcpyHostToDevice, S->stream));
  return EPO_OK;
}

epo_status epo_set_poses(epo_scene_t S, const double* T) {
  EPO_RANGE("epo_set_poses");
  if (!S || !T) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  for (int64_t k = 0; k < 12 * (int64_t)S->n_views; ++k)
    if (!isfinite(T[k])) return fail(S, EPO_ERR_INVALID_ARG, "non-finite pose");
  CK(cudaMemcpyAsync(S->d_T, T, 12 * (size_t)S->n_views * 8, cudaMemcpyHostToDevice, S->stream));
  if (S->pose_mlp) {  // the MLP's input P^0; the offsets restart at 0; the poses follow
    const size_t nv = (size_t)S->n_views;
    epo_status st = set_mlp_scale(S, T);
    if (st != EPO_OK) return st;
    CK(cudaMemcpyAsync(S->d_mlp_P0, T, 12 * nv * 8, cudaMemcpyHostToDevice, S->stream));
    for (float* q : {S->d_mlp_delta, S->d_mlp_dm, S->d_mlp_dv}) CK(cudaMemsetAsync(q, 0, 12 * nv, S->stream));
    CK(launch_mlp_forward(step_args(S, S->d_T, nullptr), 0, S->stream));
  }
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_set_pose_mlp(epo_scene_t S, const float* params) {
  EPO_RANGE("epo_set_pose_mlp");
  if (!S || !params) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  if (!S->pose_mlp) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.pose_param = EPO_POSE_MLP");
  const size_t n = (size_t)S->n_scenes * kMlpParams, nv = (size_t)S->n_views;
  for (size_t k = 0; k < n; ++k)
    if (!isfinite(params[k])) return fail(S, EPO_ERR_INVALID_ARG, "non-finite MLP parameter");
  CK(cudaMemcpyAsync(S->d_mlp_theta, params, n * 4, cudaMemcpyHostToDevice, S->stream));
  CK(cudaMemsetAsync(S->d_mlp_m, 0, n * 4, S->stream));
  CK(cudaMemsetAsync(S->d_mlp_v, 0, n * 4, S->stream));
  for (float* q : {S->d_mlp_delta, S->d_mlp_dm, S->d_mlp_dv}) CK(cudaMemsetAsync(q, 0, 12 * nv, S->stream));
  CK(launch_mlp_forward(step_args(S, S->d_T, nullptr), 0, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_get_pose_mlp_moments(epo_scene_t S, float* m, float* v, float* dm, float* dv) {
  EPO_RANGE("epo_get_pose_mlp_moments");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  if (!S->pose_mlp) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.pose_param = EPO_POSE_MLP");
  const size_t n = (size_t)S->n_scenes * kMlpParams * 4, nd = 12 * (size_t)S->n_views;
  if (m) CK(cudaMemcpyAsync(m, S->d_mlp_m, n, cudaMemcpyDeviceToHost, S->stream));
  if (v) CK(cudaMemcpyAsync(v, S->d_mlp_v, n, cudaMemcpyDeviceToHost, S->stream));
  if (dm) CK(cudaMemcpyAsync(dm, S->d_mlp_dm, nd, cudaMemcpyDeviceToHost, S->stream));
  if (dv) CK(cudaMemcpyAsync(dv, S->d_mlp_dv, nd, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_get_pose_mlp(epo_scene_t S, float* params, float* delta) {
  EPO_RANGE("epo_get_pose_mlp");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  if (!S->pose_mlp) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.pose_param = EPO_POSE_MLP");
  if (params)
    CK(cudaMemcpyAsync(params, S->d_mlp_theta, (size_t)S->n_scenes * kMlpParams * 4, cudaMemcpyDeviceToHost, S->stream));
  if (delta) CK(cudaMemcpyAsync(delta, S->d_mlp_delta, 12 * (size_t)S->n_views, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_get_poses(epo_scene_t S, double* T) {
  EPO_RANGE("epo_get_poses");
  if (!S || !T) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  epo_status st = drain(S);
  if (st != EPO_OK) return st;
  const size_t nv = (size_t)S->n_views;
  double* hp = S->h_out + S->n_scenes + 6 * nv;
  CK(cudaMemcpyAsync(hp, S->d_T, 12 * nv * 8, cudaMemcpyDeviceToHost, S->stream));
  st = host_wait(S);
  if (st != EPO_OK) return st;
  memcpy(T, hp, 12 * nv * 8);
  return EPO_OK;
}

epo_status epo_set_poses_dev(epo_scene_t S, const double* T) {
  EPO_RANGE("epo_set_poses_dev");
  if (!S || !T) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(S->d_T, T, 12 * (size_t)S->n_views * 8, cudaMemcpyDeviceToDevice, S->stream));
  if (S->pose_mlp) {  // as epo_set_poses: P^0, offsets cleared, poses recomputed
    const size_t nv = (size_t)S->n_views;
    std::vector<double> Th(12 * nv);
    CK(cudaMemcpyAsync(Th.data(), T, 12 * nv * 8, cudaMemcpyDeviceToHost, S->stream));
    CK(cudaStreamSynchronize(S->stream));
    epo_status st = set_mlp_scale(S, Th.data());
    if (st != EPO_OK) return st;
    CK(cudaMemcpyAsync(S->d_mlp_P0, T, 12 * nv * 8, cudaMemcpyDeviceToDevice, S->stream));
    for (float* q : {S->d_mlp_delta, S->d_mlp_dm, S->d_mlp_dv}) CK(cudaMemsetAsync(q, 0, 12 * nv, S->stream));
    CK(launch_mlp_forward(step_args(S, S->d_T, nullptr), 0, S->stream));
  }
  return EPO_OK;
}

epo_status epo_get_poses_dev(epo_scene_t S, double* T) {
  EPO_RANGE("epo_get_poses_dev");
  if (!S || !T) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(T, S->d_T, 12 * (size_t)S->n_views * 8, cudaMemcpyDeviceToDevice, S->stream));
  return EPO_OK;
}

epo_status epo_get_state(epo_scene_t S, int64_t* step, double* m, double* v) {
  EPO_RANGE("epo_get_state");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  if (step) CK(cudaMemcpyAsync(step, S->d_step, 8, cudaMemcpyDeviceToHost, S->stream));
  if (m) CK(cudaMemcpyAsync(m, S->d_m, 6 * (size_t)S->n_views * 8, cudaMemcpyDeviceToHost, S->stream));
  if (v) CK(cudaMemcpyAsync(v, S->d_v, 6 * (size_t)S->n_views * 8, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_set_state(epo_scene_t S, int64_t step, const double* m, const double* v) {
  EPO_RANGE("epo_set_state");
  if (!S || step < 0) return fail(S, EPO_ERR_INVALID_ARG, "null scene or negative step");
  CK(cudaMemcpyAsync(S->d_step, &step, 8, cudaMemcpyHostToDevice, S->stream));
  if (m) CK(cudaMemcpyAsync(S->d_m, m, 6 * (size_t)S->n_views * 8, cudaMemcpyHostToDevice, S->stream));
  else CK(cudaMemsetAsync(S->d_m, 0, 6 * (size_t)S->n_views * 8, S->stream));
  if (v) CK(cudaMemcpyAsync(S->d_v, v, 6 * (size_t)S->n_views * 8, cudaMemcpyHostToDevice, S->stream));
  else CK(cudaMemsetAsync(S->d_v, 0, 6 * (size_t)S->n_views * 8, S->stream));
  const double bp[2] = {pow(S->opt.beta1, (double)(step + 1)), pow(S->opt.beta2, (double)(step + 1))};
  CK(cudaMemcpyAsync(S->d_bpow, bp, sizeof(bp), cudaMemcpyHostToDevice, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_loss_and_grad_dev(epo_scene_t S, double* loss_dev, double* grad_dev) {
  EPO_RANGE("epo_loss_and_grad_dev");
  if (!S || !loss_dev) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  epo_status st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  st = enqueue_loss_grad(S, S->stream, S->d_T);
  if (st != EPO_OK) return st;
  CK(cudaMemcpyAsync(loss_dev, S->d_loss, (size_t)S->n_scenes * 8, cudaMemcpyDeviceToDevice, S->stream));
  if (grad_dev)
    CK(cudaMemcpyAsync(grad_dev, S->d_grad, 6 * (size_t)S->n_views * 8, cudaMemcpyDeviceToDevice, S->stream));
  return EPO_OK;
}

epo_status epo_loss_and_grad(epo_scene_t S, double* loss, double* grad) {
  EPO_RANGE("epo_loss_and_grad");
  if (!S || !loss) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  epo_status st = drain(S);
  if (st != EPO_OK) return st;
  st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  st = enqueue_loss_grad(S, S->stream, S->d_T);
  if (st != EPO_OK) return st;
  const size_t ns = (size_t)S->n_scenes, nv = (size_t)S->n_views;
  CK(cudaMemcpyAsync(S->h_out, S->d_loss, ns * 8, cudaMemcpyDeviceToHost, S->stream));
  if (grad) CK(cudaMemcpyAsync(S->h_out + ns, S->d_grad, 6 * nv * 8, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaMemcpyAsync(S->h_flag, S->d_flag, 4, cudaMemcpyDeviceToHost, S->stream));
  st = host_wait(S);
  if (st != EPO_OK) return st;
  memcpy(loss, S->h_out, ns * 8);
  if (grad) memcpy(grad, S->h_out + ns, 6 * nv * 8);
  return flag_status(S, *S->h_flag, "non-finite loss or gradient");
}

epo_status epo_pair_stats(epo_scene_t S, double* stats) {
  EPO_RANGE("epo_pair_stats");
  if (!S || !stats) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(stats, S->d_pair_acc, (size_t)kAcc * S->n_pairs * 8, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_forward_dev(epo_scene_t S, const double* xi_dev, double* loss_dev) {
  EPO_RANGE("epo_forward_dev");
  if (!S || !loss_dev) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  epo_status st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  CK(launch_twist_poses(S->d_T, xi_dev, S->d_T_eval, S->n_views, S->stream));
  StepArgs a = step_args(S, S->d_T_eval, nullptr);
  MARK(0, S->stream);
  if (S->subsample) CK(launch_subsample(a, S->stream));
  if (S->refine) CK(launch_refine_intrinsics(a, S->stream));
  CK(launch_pair_setup(a, MODE_FWD, S->stream));
  MARK(1, S->stream);
  st = run_edge(S, MODE_FWD, S->gather, S->rpt, S->block, S->tail, S->stream);
  if (st != EPO_OK) return st;
  CK(launch_poses(a, 0, S->stream));
  MARK(3, S->stream);
  CK(cudaMemcpyAsync(loss_dev, S->d_loss, (size_t)S->n_scenes * 8, cudaMemcpyDeviceToDevice, S->stream));
  return EPO_OK;
}

epo_status epo_backward_dev(epo_scene_t S, const double* xi_dev, const double* dloss_dev,
                            double* grad_xi_dev) {
  EPO_RANGE("epo_backward_dev");
  if (!S || !dloss_dev || !grad_xi_dev) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  CK(launch_twist_poses(S->d_T, xi_dev, S->d_T_eval, S->n_views, S->stream));
  StepArgs a = step_args(S, S->d_T_eval, dloss_dev);
  MARK(0, S->stream);
  if (S->subsample) CK(launch_subsample(a, S->stream));
  if (S->refine) CK(launch_refine_intrinsics(a, S->stream));
  CK(launch_pair_setup(a, MODE_BWD, S->stream));
  MARK(1, S->stream);
  epo_status st = run_edge(S, MODE_BWD, S->gather, S->rpt, S->block, S->tail, S->stream);
  if (st != EPO_OK) return st;
  CK(launch_poses(a, 1, S->stream));
  MARK(3, S->stream);
  CK(launch_apply_left_jacobian(xi_dev, S->d_grad, grad_xi_dev, S->n_views, S->stream));
  return EPO_OK;
}

epo_status epo_step_async(epo_scene_t S, int32_t n_steps) {
  EPO_RANGE("epo_step_async");
  if (!S || n_steps < 0) return fail(S, EPO_ERR_INVALID_ARG, "null scene or negative step count");
  epo_status st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  st = ensure_graph(S);
  if (st != EPO_OK) return st;
  for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(S->graph, S->stream));
  return EPO_OK;
}

// Copies n doubles from src to dst and returns whether all of them are finite (an exponent
// field of all ones is an infinity or a NaN): one branch-free pass that the compiler vectorises.
static bool copy_finite(double* __restrict dst, const double* __restrict src, size_t n) {
  constexpr uint64_t kExp = 0x7ff0000000000000ull;
  uint64_t bad = 0;
  for (size_t k = 0; k < n; ++k) {
    uint64_t b;
    memcpy(&b, src + k, 8);
    memcpy(dst + k, &b, 8);
    bad |= (uint64_t)((b & kExp) == kExp);
  }
  return bad == 0;
}

epo_status epo_step_host(epo_scene_t S, const double* T_in, double* T_out, double* loss) {
  EPO_RANGE("epo_step_host");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  const size_t nv = (size_t)S->n_views;
  if (T_in && S->pose_mlp) return fail(S, EPO_ERR_INVALID_ARG, "under the pose MLP the poses come from its parameters");
  // the staging is pinned and mapped: the step's first kernel reads the poses from it, and its
  // pose kernel (or a copy kernel after the step's last kernel) writes poses, loss and status
  // word back into it.  A step left queued by a wait that ran out still uses it: wait for it
  epo_status st = drain(S);
  if (st != EPO_OK) return st;
  // the poses go into the staging and are checked in the same pass (nothing runs for
  // non-finite ones; the staging is rewritten by the next call)
  if (T_in && !copy_finite(S->h_in, T_in, 12 * nv)) return fail(S, EPO_ERR_INVALID_ARG, "non-finite pose");
  st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  const int which = T_in ? 2 : 1;
  st = ensure_graph(S, which);
  if (st != EPO_OK) return st;
  CK(cudaGraphLaunch(S->graph_host[which - 1], S->stream));
  st = host_wait(S);
  if (st != EPO_OK) return st;
  if (T_out) memcpy(T_out, S->h_io, 12 * nv * 8);
  if (loss) memcpy(loss, S->h_io + 12 * nv, (size_t)S->n_scenes * 8);
  int32_t flag;
  memcpy(&flag, S->h_io + 12 * nv + S->n_scenes, 4);
  return flag_status(S, flag, "non-finite loss or gradient: pose update refused");
}

epo_status epo_check(epo_scene_t S) {
  EPO_RANGE("epo_check");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  CK(cudaMemcpyAsync(S->h_flag, S->d_flag, 4, cudaMemcpyDeviceToHost, S->stream));
  epo_status st = host_wait(S);
  if (st != EPO_OK) return st;
  return flag_status(S, *S->h_flag, "non-finite loss or gradient: pose update refused");
}

epo_status epo_last_loss(epo_scene_t S, double* loss) {
  EPO_RANGE("epo_last_loss");
  if (!S || !loss) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  epo_status st = drain(S);
  if (st != EPO_OK) return st;
  CK(cudaMemcpyAsync(S->h_out, S->d_loss, (size_t)S->n_scenes * 8, cudaMemcpyDeviceToHost, S->stream));
  st = host_wait(S);
  if (st != EPO_OK) return st;
  memcpy(loss, S->h_out, (size_t)S->n_scenes * 8);
  return EPO_OK;
}

epo_status epo_set_wait_limit(epo_scene_t S, double seconds) {
  EPO_RANGE("epo_set_wait_limit");
  if (!S || !(seconds >= 0.0) || !isfinite(seconds))
    return fail(S, EPO_ERR_INVALID_ARG, "null scene or a wait limit that is not a finite number >= 0");
  S->wait_limit_s = seconds;
  return EPO_OK;
}

epo_status epo_fixup_stats(epo_scene_t S, int64_t* queued, int64_t* overflow) {
  EPO_RANGE("epo_fixup_stats");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  unsigned int h[2] = {0u, 0u};
  CK(cudaMemcpyAsync(&h[0], S->d_qcount, 4, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaMemcpyAsync(&h[1], S->d_qoverflow, 4, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  if (queued) *queued = h[0];
  if (overflow) *overflow = h[1];
  return EPO_OK;
}

epo_status epo_kernel_time(epo_scene_t S, float* ms) {
  EPO_RANGE("epo_kernel_time");
  if (!S || !ms) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  if (!S->ev[0] || !S->ev_recorded) return fail(S, EPO_ERR_INVALID_ARG, "timing not enabled or nothing ran yet");
  CK(cudaEventSynchronize(S->ev[3]));
  CK(cudaEventElapsedTime(ms, S->ev[1], S->ev[2]));
  return EPO_OK;
}

epo_status epo_stage_times(epo_scene_t S, float* ms) {
  EPO_RANGE("epo_stage_times");
  if (!S || !ms) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  if (!S->ev[0] || !S->ev_recorded) return fail(S, EPO_ERR_INVALID_ARG, "timing not enabled or nothing ran yet");
  CK(cudaEventSynchronize(S->ev[3]));
  for (int k = 0; k < 3; ++k) CK(cudaEventElapsedTime(ms + k, S->ev[k], S->ev[k + 1]));
  return EPO_OK;
}

epo_status epo_step(epo_scene_t S, int32_t n_steps) {
  EPO_RANGE("epo_step");
  epo_status st = epo_step_async(S, n_steps);
  if (st != EPO_OK) return st;
  return epo_check(S);
}

epo_status epo_step_plain(epo_scene_t S, int32_t n_steps) {
  EPO_RANGE("epo_step_plain");
  if (!S || n_steps < 0) return fail(S, EPO_ERR_INVALID_ARG, "null scene or negative step count");
  epo_status st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  for (int k = 0; k < n_steps; ++k) {
    st = enqueue_step(S, S->stream);
    if (st != EPO_OK) return st;
  }
  return EPO_OK;
}

epo_status epo_set_refinement(epo_scene_t S, const double* gamma, const float* alpha, const float* beta) {
  EPO_RANGE("epo_set_refinement");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  if (!S->refine) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.refine = 1");
  const size_t nv = (size_t)S->n_views, nr = (size_t)S->n_records;
  std::vector<double> g(gamma ? gamma : nullptr, gamma ? gamma + nv : nullptr);
  if (!gamma) g.assign(nv, 0.0);
  for (double x : g)
    if (!(x > -1.0) || !isfinite(x)) return fail(S, EPO_ERR_INVALID_ARG, "gamma must be finite and > -1");
  std::vector<float> al(alpha ? alpha : nullptr, alpha ? alpha + nr : nullptr), be(beta ? beta : nullptr, beta ? beta + nr : nullptr);
  if (!alpha) al.assign(nr, 1.f);
  if (!beta) be.assign(nr, 0.f);
  for (size_t r = 0; r < nr; ++r)
    if (!isfinite(al[r]) || !isfinite(be[r])) return fail(S, EPO_ERR_INVALID_ARG, "non-finite alpha or beta");
  CK(cudaMemcpyAsync(S->d_gamma, g.data(), nv * 8, cudaMemcpyHostToDevice, S->stream));
  CK(cudaMemsetAsync(S->d_mg, 0, nv * 8, S->stream));
  CK(cudaMemsetAsync(S->d_vg, 0, nv * 8, S->stream));
  if (nr) {
    CK(cudaMemcpyAsync(S->d_alpha, al.data(), nr * 4, cudaMemcpyHostToDevice, S->stream));
    CK(cudaMemcpyAsync(S->d_beta, be.data(), nr * 4, cudaMemcpyHostToDevice, S->stream));
    for (float* q : {S->d_ma, S->d_va, S->d_mb, S->d_vb}) CK(cudaMemsetAsync(q, 0, nr * 4, S->stream));
  }
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_get_refinement(epo_scene_t S, double* gamma, float* alpha, float* beta) {
  EPO_RANGE("epo_get_refinement");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  if (!S->refine) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.refine = 1");
  const size_t nv = (size_t)S->n_views, nr = (size_t)S->n_records;
  if (gamma) CK(cudaMemcpyAsync(gamma, S->d_gamma, nv * 8, cudaMemcpyDeviceToHost, S->stream));
  if (alpha && nr) CK(cudaMemcpyAsync(alpha, S->d_alpha, nr * 4, cudaMemcpyDeviceToHost, S->stream));
  if (beta && nr) CK(cudaMemcpyAsync(beta, S->d_beta, nr * 4, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_refine_loss_and_grad(epo_scene_t S, double* loss, double* grad, double* grad_gamma, float* grad_alpha,
                                    float* grad_beta) {
  EPO_RANGE("epo_refine_loss_and_grad");
  if (!S || !loss) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  if (!S->refine) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.refine = 1");
  epo_status st = maybe_autotune(S);
  if (st != EPO_OK) return st;
  cudaStream_t s = S->stream;
  StepArgs a = step_args(S, S->d_T, nullptr);
  // one fused pass: the loss, the pose and focal sums per pair, every sample's d(rho)/dz; then
  // the per-record depth gradients weighted by the pairs' w / n
  if (S->subsample) CK(launch_subsample(a, s));
  CK(launch_refine_intrinsics(a, s));
  CK(launch_pair_setup(a, MODE_FUSED, s));
  st = run_edge(S, MODE_FUSED, S->gather, S->rpt, S->block, S->tail, s);
  if (st != EPO_OK) return st;
  CK(launch_poses(a, 1, s));
  CK(launch_depth(a, 0, s));
  CK(cudaMemcpyAsync(loss, S->d_loss, (size_t)S->n_scenes * 8, cudaMemcpyDeviceToHost, s));
  if (grad) CK(cudaMemcpyAsync(grad, S->d_grad, (size_t)S->n_views * 48, cudaMemcpyDeviceToHost, s));
  if (grad_gamma) CK(cudaMemcpyAsync(grad_gamma, S->d_grad_gamma, (size_t)S->n_views * 8, cudaMemcpyDeviceToHost, s));
  if (grad_alpha && S->n_records)
    CK(cudaMemcpyAsync(grad_alpha, S->d_grad_alpha, (size_t)S->n_records * 4, cudaMemcpyDeviceToHost, s));
  if (grad_beta && S->n_records)
    CK(cudaMemcpyAsync(grad_beta, S->d_grad_beta, (size_t)S->n_records * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return EPO_OK;
}

epo_status epo_get_schedule(epo_scene_t S, double* theta95, int32_t* phase, int64_t* switch_step,
                            int64_t* stop_step) {
  EPO_RANGE("epo_get_schedule");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  if (!S->opt.schedule) return fail(S, EPO_ERR_INVALID_ARG, "scene was not created with options.schedule = 1");
  const int ns = S->n_scenes;
  std::vector<int32_t> st(2 * (size_t)ns);
  std::vector<int64_t> steps(2 * (size_t)ns);
  CK(cudaMemcpyAsync(st.data(), S->d_sched_state, st.size() * 4, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaMemcpyAsync(steps.data(), S->d_sched_steps, steps.size() * 8, cudaMemcpyDeviceToHost, S->stream));
  if (theta95) CK(cudaMemcpyAsync(theta95, S->d_theta95, (size_t)ns * 8, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  for (int sc = 0; sc < ns; ++sc) {
    if (phase) phase[sc] = st[2 * sc];
    if (switch_step) switch_step[sc] = steps[2 * sc];
    if (stop_step) stop_step[sc] = steps[2 * sc + 1];
  }
  return EPO_OK;
}

epo_status epo_get_pair_active(epo_scene_t S, uint8_t* active) {
  EPO_RANGE("epo_get_pair_active");
  if (!S || !active) return fail(S, EPO_ERR_INVALID_ARG, "null argument");
  CK(cudaMemcpyAsync(active, S->d_active, (size_t)S->n_pairs, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return EPO_OK;
}

epo_status epo_set_pair_subset(epo_scene_t S, int32_t n, const int32_t* ids) {
  EPO_RANGE("epo_set_pair_subset");
  if (!S || n < 0 || (n > 0 && !ids)) return fail(S, EPO_ERR_INVALID_ARG, "invalid subset");
  if (S->opt.pair_budget > 0) return fail(S, EPO_ERR_INVALID_ARG, "the pairs are drawn on the device (pair_budget)");
  std::vector<uint8_t> act(S->n_pairs, n == 0 ? 1 : 0);
  for (int k = 0; k < n; ++k) {
    if (ids[k] < 0 || ids[k] >= S->n_pairs) return fail(S, EPO_ERR_INVALID_ARG, "pair id out of range");
    if (act[ids[k]]) return fail(S, EPO_ERR_INVALID_ARG, "duplicate pair id");
    act[ids[k]] = 1;
  }
  S->active = act;
  for (int s = 0; s < S->n_scenes; ++s) {
    int c = 0;
    for (int p = S->scene_pair_off[s]; p < S->scene_pair_off[s + 1]; ++p) c += act[p];
    S->scene_active[s] = c;
  }
  CK(cudaMemcpyAsync(S->d_active, S->active.data(), S->n_pairs, cudaMemcpyHostToDevice, S->stream));
  CK(cudaMemcpyAsync(S->d_scene_active, S->scene_active.data(), S->n_scenes * 4, cudaMemcpyHostToDevice, S->stream));
  return upload_weights(S, S->stream);
}

// Times every schedule of the edge kernel on this scene and keeps the fastest. Launches of
// different candidates are interleaved (one launch of each per pass), so that clock or
// thermal drift during tuning affects all of them alike, and each candidate is judged by
// the median of its launches. A first pass over all candidates (3 timed launches each)
// keeps the 4 best; with tail_pairs = -1 each of those is also tried with its last wave
// split into items of 2 pairs and of 1 pair, and 12 further passes decide.  (Every item split
// by pairs, tail_pairs <= -2, was never faster on the benchmark workloads: not a candidate.)
epo_status epo_autotune(epo_scene_t S) {
  EPO_RANGE("epo_autotune");
  if (!S) return fail(S, EPO_ERR_INVALID_ARG, "null scene");
  S->tuned = true;  // also guards against recursion through maybe_autotune
  struct Cand {
    int g, r, b, t;
    std::vector<float> ms;
    float med;
  };
  const int tail0 = S->opt.tail_pairs == -1 ? 0 : S->opt.tail_pairs;
  std::vector<Cand> cands;
  for (int g : {GATHER_LDG, GATHER_TEX, GATHER_MIX})
    for (int r : {1, 2, 4, 8})
      for (int b : {128, 256, 512}) {
        if (S->opt.gather == EPO_GATHER_LDG && g != GATHER_LDG) continue;
        if (S->opt.gather == EPO_GATHER_TEX && g != GATHER_TEX) continue;
        if (S->opt.gather == EPO_GATHER_MIX && g != GATHER_MIX) continue;
        if (g == GATHER_MIX && (S->refine || r == 1)) continue;
        if (!schedule_fits(S, r, b)) continue;
        cands.push_back({g, r, b, tail0, {}, 0.f});
      }
  if (cands.empty()) return fail(S, EPO_ERR_INVALID_ARG, "no edge-kernel schedule fits this scene");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  StepArgs a = step_args(S, S->d_T, nullptr);
  // autotune == 2: every timed launch starts from a cold L2 (a scratch buffer twice the
  // L2 size is written, then half of it read back, before each launch)
  void* flush = nullptr;
  size_t flush_bytes = 0;
  if (S->opt.autotune == 2) {
    int dev = 0, l2 = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    flush_bytes = std::max<size_t>((size_t)2 * (size_t)l2, (size_t)64 << 20);
    CK(cudaMalloc(&flush, flush_bytes + 16));
  }
  int fill = 0;
  // one launch of candidate c; its time is appended when `timed`
  auto launch = [&](Cand& c, bool timed) -> epo_status {
    epo_status st = build_tiles(S, c.g, c.r, c.b, c.t);  // outside the timed interval
    if (st != EPO_OK) return st;
    if (flush) {
      CK(cudaMemsetAsync(flush, ++fill & 0xff, flush_bytes, S->stream));
      CK(launch_l2_read(flush, (int64_t)flush_bytes / 2, (unsigned*)((char*)flush + flush_bytes), S->sm_count,
                        S->stream));
    }
    if (S->subsample) CK(launch_subsample(a, S->stream));
    if (S->refine) CK(launch_refine_intrinsics(a, S->stream));
    CK(launch_pair_setup(a, MODE_FUSED, S->stream));
    CK(cudaEventRecord(e0, S->stream));
    st = run_edge(S, MODE_FUSED, c.g, c.r, c.b, c.t, S->stream);
    if (st != EPO_OK) return st;
    CK(cudaEventRecord(e1, S->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (timed) c.ms.push_back(ms);
    return EPO_OK;
  };
  auto median = [](std::vector<float> v) {
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    return n % 2 ? v[n / 2] : 0.5f * (v[n / 2 - 1] + v[n / 2]);
  };
  epo_status st = EPO_OK;
  for (auto& c : cands)
    if ((st = launch(c, false)) != EPO_OK) break;  // warm-up: module load, first touch
  for (int pass = 0; pass < 3 && st == EPO_OK; ++pass)
    for (auto& c : cands)
      if ((st = launch(c, true)) != EPO_OK) break;
  if (st == EPO_OK) {
    for (auto& c : cands) c.med = median(c.ms);
    std::stable_sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.med < y.med; });
    if (cands.size() > 4) cands.resize(4);
    if (S->opt.tail_pairs == -1) {
      const size_t n4 = cands.size();
      for (size_t k = 0; k < n4; ++k)
        for (int t : {2, 1}) {
          Cand c = cands[k];
          c.t = t;
          c.ms.clear();
          cands.push_back(c);
        }
      for (size_t k = n4; k < cands.size() && st == EPO_OK; ++k) st = launch(cands[k], false);  // warm-up
    }
    for (int pass = 0; pass < 12 && st == EPO_OK; ++pass)
      for (auto& c : cands)
        if ((st = launch(c, true)) != EPO_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (flush) {
    cudaStreamSynchronize(S->stream);
    cudaFree(flush);
  }
  if (st != EPO_OK) return st;
  const Cand* best = &cands[0];
  for (auto& c : cands) {
    c.med = median(c.ms);
    if (c.med < best->med) best = &c;
  }
  S->gather = best->g;
  S->rpt = best->r;
  S->block = best->b;
  S->tail = best->t;
  S->graph_dirty = true;
  return build_tiles(S);
}

epo_status epo_distance_field(const uint8_t* edges_dev, int32_t W, int32_t H, float* map_dev,
                              void* cuda_stream) {
  EPO_RANGE("epo_distance_field");
  epo_scene* S = nullptr;
  if (!edges_dev || !map_dev || W < 1 || H < 1)
    return fail(nullptr, EPO_ERR_INVALID_ARG, "invalid distance-field arguments");
  if (H > edt_max_height()) return fail(nullptr, EPO_ERR_INVALID_ARG, "distance field: H above the supported maximum");
  CK(launch_edt(edges_dev, W, H, map_dev, (cudaStream_t)cuda_stream));
  return EPO_OK;
}

epo_status epo_round_bf16(const float* src, uint16_t* dst, int64_t n, void* cuda_stream) {
  EPO_RANGE("epo_round_bf16");
  epo_scene* S = nullptr;
  if (!src || !dst || n < 0) return fail(nullptr, EPO_ERR_INVALID_ARG, "invalid bf16 rounding arguments");
  if (n == 0) return EPO_OK;
  CK(launch_round_bf16(src, dst, n, (cudaStream_t)cuda_stream));
  return EPO_OK;
}

}  // extern "C"
