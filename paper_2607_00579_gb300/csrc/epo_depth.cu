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

// Blocks are (view, chunk of the view's records).  The block's first warp lists the view's
// active pairs in shared memory with their weights (an inactive pair's values were not written
// this pass).  Update mode runs after the pose kernel, which advanced the step counter unless
// the step was refused; with the schedule a scene's depth module steps only in phase 2 and
// counts its own steps from the switch (the phase-2 steps s > s_switch are its steps 1, 2, ...),
// without it from the first step.  The bias factors 1 - beta^dt = -expm1(dt ln beta) are formed
// once per block in FP32 (accurate to a few ulp, where 1 - beta^dt itself would cancel; an FP64
// pow on one thread per block took most of the kernel's time on this GPU's FP64 pipe).
constexpr int kDepthThreads = 128;  // nine blocks per SM at 55 registers
constexpr int kDepthPerThread = 4;   // records per thread, independent (their loads overlap)
constexpr int kDepthMaxPairs = 512;  // outgoing pairs of one view (the creation limit)

template <int REC, int UPDATE>
__global__ void __launch_bounds__(kDepthThreads) k_depth(StepArgs a, int chunks_per_view) {
  __shared__ float s_w[kDepthMaxPairs];       // the view's active pairs, in list order:
  __shared__ int64_t s_base[kDepthMaxPairs];  // weight w_p / n_p and the pair's block of dzr
  __shared__ float s_c[2];
  __shared__ int s_go, s_n;
  const int v = blockIdx.x / chunks_per_view, ch = blockIdx.x % chunks_per_view;
  const int lane = threadIdx.x & 31;
  const ViewDev vd = a.views[v];
  const int64_t r0 = vd.rec_begin, n = vd.n_rec;
  const int64_t k0 = (int64_t)ch * kDepthThreads * kDepthPerThread + threadIdx.x;
  if (threadIdx.x < 32) {
    // warp 0: compact the view's active pairs (a fixed order: the view's pair list)
    const int q0 = a.src_pair_off[v], nq = a.src_pair_off[v + 1] - q0;
    int cnt = 0;
    for (int k0 = 0; k0 < nq; k0 += 32) {
      const int k = k0 + lane;
      const int p = k < nq ? a.src_pair_ids[q0 + k] : 0;
      const bool act = k < nq && a.pair_active[p];
      const unsigned bal = __ballot_sync(0xffffffffu, act);
      if (act) {  // the weight w_p / n_p from the pose kernel's loss blocks
        const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
        s_w[pos] = a.pair_wz[p];
        s_base[pos] = a.pp[q0 + k].dbase;
      }
      cnt += __popc(bal);
    }
    if (lane == 0) {
      s_n = cnt;
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
          const float fdt = (float)dt;
          s_c[0] = -expm1f(fdt * a.log_beta1);
          s_c[1] = -expm1f(fdt * a.log_beta2);
        }
      }
      s_go = go;
    }
  }
  __syncthreads();
  if (!s_go) return;  // uniform over the block
  const int np = s_n;
  // dL/dz of the thread's records: eight pairs' loads for all of them in flight together,
  // summed in the list order
  float gz[kDepthPerThread];
#pragma unroll
  for (int j = 0; j < kDepthPerThread; ++j) gz[j] = 0.f;
  constexpr int QB = 8;
  for (int qb = 0; qb < np; qb += QB) {
    float dv[QB][kDepthPerThread];
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      const bool qok = qb + u < np;
      const float* d = a.dzr + (qok ? s_base[qb + u] : 0) + r0;
#pragma unroll
      for (int j = 0; j < kDepthPerThread; ++j) {
        const int64_t k = k0 + j * kDepthThreads;
        dv[u][j] = (qok && k < n) ? __ldg(d + k) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      const float w = qb + u < np ? s_w[qb + u] : 0.f;
#pragma unroll
      for (int j = 0; j < kDepthPerThread; ++j) gz[j] = fmaf(w, dv[u][j], gz[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kDepthPerThread; ++j) {
    const int64_t k = k0 + j * kDepthThreads;
    if (k >= n) continue;
    const int64_t r = r0 + k;
    float u, w, z0;
    load_record<REC>(a.rec, r, u, w, z0);
    const float gb = gz[j], ga = gb * z0;
    if (!UPDATE) {
      a.grad_alpha[r] = ga;
      a.grad_beta[r] = gb;
      continue;
    }
    const float c1 = s_c[0], c2 = s_c[1];
    const float b1 = (float)a.beta1, b2 = (float)a.beta2, lr = (float)a.lr_depth, eps = (float)a.adam_eps;
    const float ma = b1 * a.ma[r] + (1.f - b1) * ga, va = b2 * a.va[r] + (1.f - b2) * ga * ga;
    const float mb = b1 * a.mb[r] + (1.f - b1) * gb, vb = b2 * a.vb[r] + (1.f - b2) * gb * gb;
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
