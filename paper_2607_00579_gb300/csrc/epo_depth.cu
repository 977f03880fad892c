// The per-record depth kernel of the refinement (Section 3, Depth Refinement, Eq. 5:
// z_r = Z0_r alpha_r + beta_r for every edge pixel r).
//
// The fused pass of a refine scene stores, for every (pair p, source record r), the sample's
// d(rho)/dz unweighted: the pair means' denominators (the valid counts n_p) are only known
// once the pass is over.  This kernel then forms
//     dL/dz_r = sum over the record's active outgoing pairs p of (w_p / n_p) d(rho_p,r)/dz
// (w_p = the pair's weight in its scene's loss; w_p alone under Eq. 7's normaliser), in the
// fixed order of the view's pair list, and either writes dL/dalpha_r = dL/dz_r Z0_r and
// dL/dbeta_r = dL/dz_r (gradient mode) or takes the depth module's Adam step on alpha_r and
// beta_r (Algorithm 2; update mode, inside the step graph).
//
// Storing one float per evaluation (4 B, written once and read once) replaces a second pass
// over the samples, which would cost a full re-projection and gather of every sample.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "epo_internal.cuh"

namespace epo {

// Blocks are (view, chunk of the view's records).  The block's first threads form the weights
// of the view's pairs in shared memory (0 for an inactive pair, whose values were not written
// this pass).  Update mode runs after the pose kernel, which advanced the step counter unless
// the step was refused; with the schedule a scene's depth module steps only in phase 2 and
// counts its own steps from the switch (the phase-2 steps s > s_switch are its steps 1, 2, ...),
// without it from the first step; the bias factors are formed once per block in FP64.
constexpr int kDepthThreads = 256;
constexpr int kDepthPerThread = 4;
constexpr int kDepthMaxPairs = 512;  // outgoing pairs of one view (the creation limit)

template <int REC, int UPDATE>
__global__ void __launch_bounds__(kDepthThreads) k_depth(StepArgs a, int chunks_per_view) {
  __shared__ float s_w[kDepthMaxPairs];
  __shared__ int64_t s_base[kDepthMaxPairs];
  __shared__ float s_c[2];
  __shared__ int s_go;
  const int v = blockIdx.x / chunks_per_view, ch = blockIdx.x % chunks_per_view;
  const ViewDev vd = a.views[v];
  if (threadIdx.x == 0) {
    int go = 1;
    if (UPDATE) {
      go = !(*a.flag & 1);  // a refused step moves nothing
      const int sc = vd.scene;
      const int64_t s_cur = *a.step - 1;  // the step just taken
      int64_t dt = s_cur + 1;
      if (a.schedule) {
        if (a.sched_state[2 * sc] != 2) go = 0;  // phase 1, or converged
        dt = s_cur - a.sched_steps[2 * sc];
      }
      if (dt < 1) go = 0;
      if (go) {
        s_c[0] = (float)(1.0 - pow(a.beta1, (double)dt));
        s_c[1] = (float)(1.0 - pow(a.beta2, (double)dt));
      }
    }
    s_go = go;
  }
  const int q0 = a.src_pair_off[v], nq = a.src_pair_off[v + 1] - q0;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const int p = a.src_pair_ids[q0 + k];
    float w = 0.f;
    int64_t base = -1;
    if (a.pair_active[p]) {
      const double n = a.pair_acc[(size_t)kAcc * p + 1];
      w = a.norm_all ? (float)a.pair_lw[p] : (n > 0.0 ? (float)(a.pair_lw[p] / n) : 0.f);
      base = a.pp[p].dbase;
    }
    s_w[k] = w;
    s_base[k] = base;
  }
  __syncthreads();
  if (!s_go) return;  // uniform over the block
  const int64_t r0 = vd.rec_begin, n = vd.n_rec;
  for (int64_t k = (int64_t)ch * kDepthThreads + threadIdx.x; k < n; k += (int64_t)chunks_per_view * kDepthThreads) {
    const int64_t r = r0 + k;
    float gz = 0.f;
    for (int q = 0; q < nq; ++q)
      if (s_base[q] >= 0) gz = fmaf(s_w[q], a.dzr[s_base[q] + r], gz);
    float u, w, z0;
    load_record<REC>(a.rec, r, u, w, z0);
    const float ga = gz * z0;
    if (!UPDATE) {
      a.grad_alpha[r] = ga;
      a.grad_beta[r] = gz;
      continue;
    }
    const float c1 = s_c[0], c2 = s_c[1];
    const float b1 = (float)a.beta1, b2 = (float)a.beta2, lr = (float)a.lr_depth, eps = (float)a.adam_eps;
    const float ma = b1 * a.ma[r] + (1.f - b1) * ga, va = b2 * a.va[r] + (1.f - b2) * ga * ga;
    const float mb = b1 * a.mb[r] + (1.f - b1) * gz, vb = b2 * a.vb[r] + (1.f - b2) * gz * gz;
    a.ma[r] = ma;
    a.va[r] = va;
    a.mb[r] = mb;
    a.vb[r] = vb;
    a.alpha[r] -= lr * (ma / c1) / (sqrtf(va / c2) + eps);
    a.beta[r] -= lr * (mb / c1) / (sqrtf(vb / c2) + eps);
  }
}

template <int REC>
static void launch_depth_rec(const StepArgs& a, int update, unsigned nb, int cpv, cudaStream_t s) {
  if (update) k_depth<REC, 1><<<nb, kDepthThreads, 0, s>>>(a, cpv);
  else k_depth<REC, 0><<<nb, kDepthThreads, 0, s>>>(a, cpv);
}

cudaError_t launch_depth(const StepArgs& a, int update, cudaStream_t s) {
  if (a.max_view_records <= 0 || a.n_views <= 0) return cudaSuccess;
  const int64_t per_block = (int64_t)kDepthThreads * kDepthPerThread;
  const int cpv = (int)std::max<int64_t>(1, ((int64_t)a.max_view_records + per_block - 1) / per_block);
  const unsigned nb = (unsigned)((int64_t)cpv * a.n_views);
  if (a.rec_dtype) launch_depth_rec<1>(a, update, nb, cpv, s);
  else launch_depth_rec<0>(a, update, nb, cpv, s);
  return cudaGetLastError();
}

}  // namespace epo
