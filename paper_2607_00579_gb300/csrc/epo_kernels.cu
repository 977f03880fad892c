// Kernels of the edge-alignment library (sm_103a) around the edge kernel (epo_edge.cu).
//
// One optimisation step (Algorithm 2 with the pose-only reading) is three launches:
//   k_pair_setup   a1: T_ji = T_j T_i^-1 in FP64 (kept for the exact path) and rounded to
//                  FP32 for the pixel math; lambda from the step; counters reset.
//   k_edge         a2-a7 (epo_edge.cu).
//   k_poses        a8 + a9: per-scene loss (Eq. 6, Algorithm 3's sum(rho)/sum(valid)),
//                  deterministic FP64 per-pose gather of the pair sums (the source side
//                  through -Ad(T_ji)^T), tangent-space Adam and T <- Exp(-Delta) T.
// Both small kernels are FP64 latency chains on a few warps: they run 32-thread blocks, so
// that their FP64 work spreads over many SMs (an FP64 warp instruction occupies its
// sub-partition's FP64 pipe for many cycles on this GPU).
// Construction helpers: k_edt (exact distance transform field), k_round_bf16, k_map_check.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "epo_internal.cuh"

namespace epo {



// ------------------------------------------------------------------------------------
// a1: pair setup
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double lambda_at(const StepArgs& a, int64_t s) {
  double f = a.lambda_steps > 0 ? (double)s * a.inv_lambda_steps : 1.0;
  f = f > 1.0 ? 1.0 : f;
  return a.lambda0 + (a.lambda1 - a.lambda0) * f;
}

// 16 lanes per pair (two pairs per warp): lanes 0..8 form one entry of R_ji each, lanes
// 9..11 one entry of t_ji, lane 15 the rounding bound of the FP32 translation; every lane's
// FP64 chain is a few operations long.  The rest of the PairParam (the target's intrinsics
// and map) does not change with the poses and is written when the scene is created.
constexpr int kSetupLanes = 16;
constexpr int kSetupThreads = 32;  // two pairs per block: the FP64 chains spread over SMs

__global__ void __launch_bounds__(kSetupThreads) k_pair_setup(StepArgs a, int mode) {
  griddep_launch_dependents();  // the edge kernel may start its first records meanwhile
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt == 0) {
    *a.lambda = lambda_at(a, *a.step);
    *a.q_count = 0u;
    *a.tile_counter = 0;
  }
  const int lane = threadIdx.x & 31;
  const int base = lane & 16;
  const int e = lane & 15;
  const int p = gt / kSetupLanes;
  const bool pv = p < a.n_pairs;
  const int2 ij = pv ? a.pair_ij[p] : make_int2(0, 0);
  const int q = pv ? a.pair_q[p] : 0;
  const int act = pv && e == 13 ? (int)a.pair_active[p] : 0;
  const int i = ij.x, j = ij.y;
  const double* Ti = a.T + 12 * (size_t)i;
  const double* Tj = a.T + 12 * (size_t)j;
  double val = 0.0;
  if (pv && e < 9) {  // R_ji[r][c] = sum_k R_j[r][k] R_i[c][k]
    const int r = e / 3, c = e % 3;
    val = Tj[4 * r] * Ti[4 * c] + Tj[4 * r + 1] * Ti[4 * c + 1] + Tj[4 * r + 2] * Ti[4 * c + 2];
  }
  // t_ji[r] = t_j[r] - sum_c R_ji[r][c] t_i[c]: lane 9 + r reads row r of R_ji from lanes 3r..3r+2
  const int rr = e >= 9 && e < 12 ? e - 9 : 0;
  const double R0 = __shfl_sync(0xffffffffu, val, base + 3 * rr);
  const double R1 = __shfl_sync(0xffffffffu, val, base + 3 * rr + 1);
  const double R2 = __shfl_sync(0xffffffffu, val, base + 3 * rr + 2);
  if (pv && e >= 9 && e < 12) val = Tj[4 * rr + 3] - (R0 * Ti[3] + R1 * Ti[7] + R2 * Ti[11]);
  const float vf = (float)val;
  // |t| for the rounding bound of the FP32 translation
  const float t0 = __shfl_sync(0xffffffffu, vf, base + 9);
  const float t1 = __shfl_sync(0xffffffffu, vf, base + 10);
  const float t2 = __shfl_sync(0xffffffffu, vf, base + 11);
  // the exact path's projective form (FP64): with M = R_ji K_i^-1, lane (r, c) < 9 forms
  // B[r][c] = (K_j M)[r][c] and lane 9 + r forms c[r] = (K_j t_ji)[r]; K: fx, fy, cx, cy,
  // 1/fx, 1/fy (refine scenes: at f0 (1 + gamma))
  const double* K = a.refine ? a.K64r : a.K64;
  const double* Ki = K + 6 * (size_t)i;
  const double* Kj = K + 6 * (size_t)j;
  const int rb = e < 9 ? e / 3 : 0, cb = e < 9 ? e % 3 : 0;
  const double Rr0 = __shfl_sync(0xffffffffu, val, base + 3 * rb);      // R[r][0]
  const double Rr1 = __shfl_sync(0xffffffffu, val, base + 3 * rb + 1);  // R[r][1]
  // every lane runs the same FP64 instructions (selected operands, no divergent branches): on
  // this GPU each FP64 warp instruction holds the sub-partition's FP64 pipe for many cycles
  const double kx = pv ? Ki[2] * Ki[4] : 0.0, ky = pv ? Ki[3] * Ki[5] : 0.0;  // cx/fx, cy/fy of view i
  // M[r][c] = R[r][c] s_c + o, s = (1/fx_i, 1/fy_i, 1), o = -(R[r][0] cx_i/fx_i + R[r][1] cy_i/fy_i) for c = 2
  const double sc = cb == 0 ? (pv ? Ki[4] : 0.0) : (cb == 1 ? (pv ? Ki[5] : 0.0) : 1.0);
  const double oc = -fma(Rr0, kx, Rr1 * ky);
  const double Mv = fma(val, sc, cb == 2 ? oc : 0.0);
  const double M2c = __shfl_sync(0xffffffffu, Mv, base + 6 + cb);  // M[2][c]
  const double t2d = __shfl_sync(0xffffffffu, val, base + 11);     // t_ji[2]
  // B[r][c] = a_r M[r][c] + b_r M[2][c] and c[r] = a_r t[r] + b_r t[2], (a, b) = (fx_j, cx_j),
  // (fy_j, cy_j), (1, 0) for r = 0, 1, 2
  const bool tcol = e >= 9;
  const int rrow = tcol ? (e < 12 ? e - 9 : 2) : rb;
  const double fa = rrow == 0 ? (pv ? Kj[0] : 0.0) : (rrow == 1 ? (pv ? Kj[1] : 0.0) : 1.0);
  const double fb = rrow == 0 ? (pv ? Kj[2] : 0.0) : (rrow == 1 ? (pv ? Kj[3] : 0.0) : 0.0);
  const double Bv = fma(fa, tcol ? val : Mv, fb * (tcol ? t2d : M2c));
  const bool bad = pv && e < 12 && !isfinite(val);
  if (__ballot_sync(0xffffffffu, bad)) {
    if (bad) atomicOr(a.flag, 1);  // a non-finite pose: the step must not update
  }
  if (!pv) return;
  PairParam* out = a.pp + q;
  float* of = reinterpret_cast<float*>(out);
  if (e < 12) {
    a.pp64[kPP64 * (size_t)p + e] = val;  // R (9) then t (3), as in PairParam
    a.pp64[kPP64 * (size_t)p + 12 + e] = Bv;  // B (9) then c (3)
    of[e] = vf;
  } else if (e == 15) {
    out->Et = 4.f * (kU32 * 1.00001f) * (fabsf(t0) + fabsf(t1) + fabsf(t2));
  } else if (e == 13) {
    out->active = act;
  } else if (a.refine && e == 12) {
    // refine scenes: the target's intrinsics at f0 (1 + gamma_j) (Eq. 4), rounded to FP32;
    // the projection bound grows by one rounding of the focal length
    const double sc = 1.0 + a.gamma[j];
    const float fx = (float)(a.K64[6 * (size_t)j] * sc), fy = (float)(a.K64[6 * (size_t)j + 1] * sc);
    out->fx = fx;
    out->fy = fy;
    out->cu = 5.f * kU32 * (float)(out->W + 1);
    out->cv = 5.f * kU32 * (float)(out->H + 1);
  }
  if (e < kAcc) {
    const bool zero = (e < 2) ? (mode != MODE_BWD) : (mode != MODE_FWD);
    if (zero) a.pair_acc[(size_t)kAcc * p + e] = 0.0;
  }
  if (a.refine && mode != MODE_FWD && (e == 8 || e == 9)) a.pair_facc[2 * (size_t)p + e - 8] = 0.0;
}

// Refine scenes: the FP64 intrinsics at f0 (1 + gamma) of every view (fx, fy, cx, cy, 1/fx,
// 1/fy), read by the edge kernel's lift and exact path.
__global__ void k_refine_intrinsics(StepArgs a) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n_views; v += gridDim.x * blockDim.x) {
    const double sc = 1.0 + a.gamma[v];
    const double fx = a.K64[6 * (size_t)v] * sc, fy = a.K64[6 * (size_t)v + 1] * sc;
    double* K = a.K64r + 6 * (size_t)v;
    K[0] = fx;
    K[1] = fy;
    K[2] = a.K64[6 * (size_t)v + 2];
    K[3] = a.K64[6 * (size_t)v + 3];
    K[4] = 1.0 / fx;
    K[5] = 1.0 / fy;
  }
}

// ------------------------------------------------------------------------------------
// a8 + a9: per-scene loss, per-pose FP64 gather, tangent-space Adam, Exp retraction
// ------------------------------------------------------------------------------------
// One pose per 16 lanes (two per warp).  The pose's (pair, role) entries are spread over
// the 16 lanes (one FP64 division and one 6-vector per entry), reduced with a fixed
// shuffle tree; lanes 0..5 then own the twist components and lanes 0..11 the entries of
// the updated [R|t].  This keeps each warp's FP64 instruction chain short: on this GPU
// an FP64 warp instruction occupies its sub-partition's FP64 pipe for many cycles.
constexpr int kPoseThreads = 32;  // two poses per block: the FP64 chains spread over SMs
constexpr int kPosesPerBlock = kPoseThreads / 16;

// Taylor coefficients (in theta^2) of A = sin(t)/t, B = (1 - cos t)/t^2, C = (t - sin t)/t^3
__device__ constexpr double kExpA[5] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0};
__device__ constexpr double kExpB[5] = {0.5, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0};
__device__ constexpr double kExpC[5] = {1.0 / 6.0, -1.0 / 120.0, 1.0 / 5040.0, -1.0 / 362880.0, 1.0 / 39916800.0};

// R = I, t = 0: the relative pose a target entry of the pose gather reads
__device__ __align__(16) const double kIdentityPose[12] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0};

// 1/n for a sample count n >= 1: the FP32 approximate reciprocal (relative error below
// 2^-22 after rounding n to FP32) refined by one FP64 Newton step, relative error below 2^-43:
// two FP64 operations instead of a correctly rounded FP64 reciprocal
__device__ __forceinline__ double rcp_count(double n) {
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)n));
  const double r = (double)rf;
  return fma(r, fma(-n, r, 1.0), r);
}

// Entry (r, c) of [w]x = [[0, -w2, w1], [w2, 0, -w0], [-w1, w0, 0]] with runtime r, c.
__device__ __forceinline__ double cross_entry(int r, int c, double w0, double w1, double w2) {
  if (r == c) return 0.0;
  const int k = 3 - r - c;
  const double wk = k == 0 ? w0 : (k == 1 ? w1 : w2);
  return ((c - r + 3) % 3) == 1 ? -wk : wk;
}

__global__ void __launch_bounds__(kPoseThreads) k_poses(StepArgs a, int with_grad, int n_pose_blocks) {
  static_assert(kPoseThreads == 32 && kLossChunk == 32, "one warp per block, one pair per lane");
  const int64_t step = *a.step;
  int flag0 = *a.flag;
  bool bad_here = false;  // this thread set the non-finite flag in this step
  if ((int)blockIdx.x < n_pose_blocks) {
    const int lane = threadIdx.x & 31;
    const int base = lane & 16;
    const int e = lane & 15;
    const int v = blockIdx.x * kPosesPerBlock + (threadIdx.x >> 4);
    const bool vv = v < a.n_views && with_grad > 0;
    // the optimiser state and the old pose do not depend on the gradient: their loads are
    // issued first, so that they overlap the gather below
    double m_old = 0.0, v_old = 0.0, Tc0 = 0.0, Tc1 = 0.0, Tc2 = 0.0, bp0 = 0.0, bp1 = 0.0;
    if (with_grad == 2 && vv) {
      if (e < 6) {
        m_old = a.m[6 * (size_t)v + e];
        v_old = a.v[6 * (size_t)v + e];
      }
      if (e < 12) {
        const double* T = a.T_store + 12 * (size_t)v;
        Tc0 = T[e & 3];
        Tc1 = T[4 + (e & 3)];
        Tc2 = T[8 + (e & 3)];
      }
      bp0 = a.bpow[0];
      bp1 = a.bpow[1];
    }
    double mg_old = 0.0, vg_old = 0.0;
    if (with_grad == 2 && vv && a.refine && e == 0) {
      mg_old = a.mg[v];
      vg_old = a.vg[v];
    }
    // a scene whose schedule has converged keeps its poses
    const bool conv = with_grad == 2 && vv && a.schedule && a.sched_state[2 * a.views[v].scene] == 3;
    // the pose's entry list is fixed at scene creation: the lane's first entry is read before
    // the wait, so that only the pair sums' loads follow it
    const PoseEntry* ent = a.pose_entries + (size_t)(vv ? v : 0) * a.pose_stride;
    const PoseEntry en0 = (vv && e < a.pose_stride) ? ent[e] : PoseEntry{-1, 0};
    // the state loads above do not depend on the edge kernel; the pair sums below do
    griddep_wait();
    flag0 |= *reinterpret_cast<volatile const int*>(a.flag) & kFlagBounds;  // set by the edge kernel
    // the lane's partial sums: dL/dxi_v (six components), then (refine scenes) dL/dgamma_v
    // before its 1 / (1 + gamma_v) factor, then a zero pad
    double g[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (vv) {
      for (int k = e; k < a.pose_stride; k += 16) {
        const PoseEntry en = k == e ? en0 : ent[k];
        if (en.p < 0) continue;
        const int p = en.p;
        const bool src = (en.scene_role & 1) != 0;
        // the pair's sums (frame j), weight and relative pose are loaded together; a target
        // entry reads T_ji = I, so that both roles run the same instructions
        const double2* acc = reinterpret_cast<const double2*>(a.pair_acc + (size_t)kAcc * p);
        const double2* Rt = reinterpret_cast<const double2*>(src ? a.pp64 + kPP64 * (size_t)p : kIdentityPose);
        const double2 s01 = acc[0], s23 = acc[1], s45 = acc[2], s67 = acc[3];
        const double2 R01 = Rt[0], R23 = Rt[1], R45 = Rt[2], R67 = Rt[3], R8t0 = Rt[4], t12 = Rt[5];
        double c = a.pair_lw[p];  // the pair's weight in its scene's loss (0: not evaluated)
        if (c == 0.0) continue;
        if (!a.norm_all) {
          const double n = s01.y;  // Algorithm 3: the pair's mean runs over its valid samples
          if (!(n > 0.0)) continue;
          c *= rcp_count(n);
        }
        if (a.gscale) c *= a.gscale[en.scene_role >> 1];
        if (a.refine) g[6] += c * a.pair_facc[2 * (size_t)p + (src ? 0 : 1)];
        // the entry adds s (R^T ga, R^T (gb - t x ga)), (ga, gb) = c (sum g_Y, sum Y x g_Y):
        // the target's 6-vector as is (s = 1, R = I, t = 0) and the source's
        // -Ad(T_ji)^T (ga, gb) = (-R^T ga, R^T (t x ga) - R^T gb) (s = -1)
        if (src) c = -c;
        const double R[9] = {R01.x, R01.y, R23.x, R23.y, R45.x, R45.y, R67.x, R67.y, R8t0.x};
        const double t0 = R8t0.y, t1 = t12.x, t2 = t12.y;
        const double ga0 = c * s23.x, ga1 = c * s23.y, ga2 = c * s45.x;
        const double gb0 = c * s45.y, gb1 = c * s67.x, gb2 = c * s67.y;
        const double x0 = fma(t2, ga1, fma(-t1, ga2, gb0));
        const double x1 = fma(t0, ga2, fma(-t2, ga0, gb1));
        const double x2 = fma(t1, ga0, fma(-t0, ga1, gb2));
#pragma unroll
        for (int k3 = 0; k3 < 3; ++k3) {
          g[k3] = fma(R[6 + k3], ga2, fma(R[3 + k3], ga1, fma(R[k3], ga0, g[k3])));
          g[3 + k3] = fma(R[6 + k3], x2, fma(R[3 + k3], x1, fma(R[k3], x0, g[3 + k3])));
        }
      }
    }
    // fixed-order reduce-scatter over the pose's 16 lanes (8 FP64 additions instead of 4 per
    // value): lane e = 8 b3 + 4 b2 + 2 b1 + b0 ends with the sum of value 4 b3 + 2 b2 + b1, so
    // value k sits in lanes 2k and 2k + 1
    double sred;
    {
      const bool b3 = e & 8, b2 = e & 4, b1 = e & 2;
      double k4[4], k2[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double keep = b3 ? g[4 + i] : g[i], send = b3 ? g[i] : g[4 + i];
        k4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const double keep = b2 ? k4[2 + i] : k4[i], send = b2 ? k4[i] : k4[2 + i];
        k2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      const double keep = b1 ? k2[1] : k2[0], send = b1 ? k2[0] : k2[1];
      sred = keep + __shfl_xor_sync(0xffffffffu, send, 2);
      sred += __shfl_xor_sync(0xffffffffu, sred, 1);
    }
    // lane e < 6 takes component e of the gradient
    const double G = __shfl_sync(0xffffffffu, sred, base + 2 * (e < 6 ? e : 0));
    const double gg = __shfl_sync(0xffffffffu, sred, base + 12);
    if (a.refine && vv && e == 0) {
      const double g0 = a.gamma[v];
      const double Gg = gg / (1.0 + g0);  // dL/dgamma_v
      if (a.grad_gamma) a.grad_gamma[v] = Gg;
      if (with_grad == 2) {
        // Adam on the focal scale (Eq. 4), every step, in FP64 (one lane per view); the bias
        // factors are the pose optimiser's (the same step count)
        if (!isfinite(Gg)) {
          atomicOr(a.flag, 1);
          bad_here = true;
        } else if (!(flag0 & kFlagRefuse) && !conv) {
          const double m = a.beta1 * mg_old + (1.0 - a.beta1) * Gg;
          const double vm = a.beta2 * vg_old + (1.0 - a.beta2) * Gg * Gg;
          a.mg[v] = m;
          a.vg[v] = vm;
          a.gamma[v] = g0 - a.lr_focal * (m / (1.0 - bp0)) / (sqrt(vm / (1.0 - bp1)) + a.adam_eps);
        }
      }
    }
    if (vv && e < 6) {
      a.grad[6 * (size_t)v + e] = G;
      if (!isfinite(G)) {
        atomicOr(a.flag, 1);
        bad_here = true;
      }
    }
    if (with_grad == 2) {
      const bool bad = vv && e < 6 && !isfinite(G);
      const unsigned badmask = __ballot_sync(0xffffffffu, bad);
      // under the pose MLP the poses come from its forward kernel: only the gradient is formed
      const bool skip = !vv || (flag0 & kFlagRefuse) || a.fixed[v] || conv || a.pose_mlp || ((badmask >> base) & 0xffffu);
      double xi = 0.0;
      if (!skip && e < 6) {
        const size_t o = 6 * (size_t)v + e;
        const double m = a.beta1 * m_old + (1.0 - a.beta1) * G;
        const double vm = a.beta2 * v_old + (1.0 - a.beta2) * G * G;
        a.m[o] = m;
        a.v[o] = vm;
        // the step ratio m^ / (sqrt(v^) + eps) needs only single precision; the bias factors
        // 1 - beta^(s+1) are formed in FP64 (in FP32, 1 - beta2 cancels to ~1e-5 relative)
        const float mh = (float)m / (float)(1.0 - bp0);
        const float vh = (float)vm / (float)(1.0 - bp1);
        const float lr = (float)(e < 3 ? a.lr_trans : a.lr_rot);
        xi = -(double)(lr * mh / (sqrtf(vh) + (float)a.adam_eps));  // the update is Exp(-Delta)
      }
      double x[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) x[k] = __shfl_sync(0xffffffffu, xi, base + k);
      // lane e = 4r + c of the group forms entry (r, c) of Exp(xi) = [E_R | E_t]; the rows
      // are then exchanged by shuffles for the composition T <- Exp(xi) T
      const int r = (e >> 2) < 3 ? (e >> 2) : 2, c = e & 3;
      const double w0 = x[3], w1 = x[4], w2 = x[5];
      const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
      // theta < 0.05: Taylor polynomials in theta^2, truncation below 1e-20; lanes 0, 1, 2 of
      // the pose evaluate A, B, C (one polynomial per lane) and share them
      double tay;
      {
        const int q = e % 3;
        double co[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) co[i] = q == 0 ? kExpA[i] : (q == 1 ? kExpB[i] : kExpC[i]);
        tay = fma(th2, fma(th2, fma(th2, fma(th2, co[4], co[3]), co[2]), co[1]), co[0]);
      }
      double A = __shfl_sync(0xffffffffu, tay, base);
      double B = __shfl_sync(0xffffffffu, tay, base + 1);
      double C = __shfl_sync(0xffffffffu, tay, base + 2);
      if (!(th2 < 2.5e-3)) {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        A = sn / th;
        B = (1.0 - cs) / th2;
        C = (th - sn) / (th2 * th);
      }
      const double wr = r == 0 ? w0 : (r == 1 ? w1 : w2);
      double Erc;
      if (c < 3) {
        const double wc = c == 0 ? w0 : (c == 1 ? w1 : w2);
        const double I = r == c ? 1.0 : 0.0;
        Erc = I + A * cross_entry(r, c, w0, w1, w2) + B * (wr * wc - I * th2);
      } else {
        // translation: (I + B W + C W^2) upsilon = upsilon + B (w x upsilon) + C (w x (w x upsilon)),
        // row r
        const double p0 = fma(w1, x[2], -w2 * x[1]);
        const double p1 = fma(w2, x[0], -w0 * x[2]);
        const double p2 = fma(w0, x[1], -w1 * x[0]);
        const double pr = r == 0 ? p0 : (r == 1 ? p1 : p2);
        const double wa = r == 0 ? w1 : (r == 1 ? w2 : w0), wb = r == 0 ? w2 : (r == 1 ? w0 : w1);
        const double pa = r == 0 ? p1 : (r == 1 ? p2 : p0), pb = r == 0 ? p2 : (r == 1 ? p0 : p1);
        const double qr = fma(wa, pb, -wb * pa);  // (w x p)_r
        const double ur = r == 0 ? x[0] : (r == 1 ? x[1] : x[2]);
        Erc = fma(C, qr, fma(B, pr, ur));
      }
      const int rb = base + (e & 12);
      const double E0 = __shfl_sync(0xffffffffu, Erc, rb);
      const double E1 = __shfl_sync(0xffffffffu, Erc, rb + 1);
      const double E2 = __shfl_sync(0xffffffffu, Erc, rb + 2);
      const double E3 = __shfl_sync(0xffffffffu, Erc, rb + 3);
      double Tnew = 0.0;
      if (!skip && e < 12) Tnew = fma(E0, Tc0, fma(E1, Tc1, fma(E2, Tc2, c == 3 ? E3 : 0.0)));
      __syncwarp();  // every lane has read the old pose before any lane writes it
      if (!skip && e < 12) a.T_store[12 * (size_t)v + e] = Tnew;
      if (a.host_out && vv && e < 12)  // host-driven step: every pose, updated or kept
        a.host_out[12 * (size_t)v + e] = skip ? (r == 0 ? Tc0 : (r == 1 ? Tc1 : Tc2)) : Tnew;
      if (a.schedule && !a.pose_mlp) {
        // the step's pose change (Section 3, Optimization Schedule): lane (r, c) holds entry
        // (r, c) of the old and the new pose; tr(R_new R_old^T) and the translations' dot
        // product and norms are reduced over the pose's 16 lanes in a fixed order
        const double Told = r == 0 ? Tc0 : (r == 1 ? Tc1 : Tc2);
        const double Tn = skip ? Told : Tnew;
        double tr = (e < 12 && c < 3) ? Tn * Told : 0.0;
        double dot = (e < 12 && c == 3) ? Tn * Told : 0.0;
        double nn = (e < 12 && c == 3) ? Tn * Tn : 0.0;
        double no = (e < 12 && c == 3) ? Told * Told : 0.0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          tr += __shfl_xor_sync(0xffffffffu, tr, o);
          dot += __shfl_xor_sync(0xffffffffu, dot, o);
          nn += __shfl_xor_sync(0xffffffffu, nn, o);
          no += __shfl_xor_sync(0xffffffffu, no, o);
        }
        if (vv && e == 0) {
          const double deg = 180.0 / 3.14159265358979323846;
          const double cr = fmin(1.0, fmax(-1.0, (tr - 1.0) * 0.5));
          a.pose_dR[v] = deg * acos(cr);
          const double nm = sqrt(nn) * sqrt(no);
          a.pose_dt[v] = nm > 0.0 ? deg * acos(fmin(1.0, fmax(-1.0, dot / nm))) : 0.0;
        }
      }
    }
  } else {
    // per-scene loss (Eq. 6): this block sums l_p over kLossChunk consecutive pairs of one
    // scene (one pair per lane, fixed shuffle tree); the scene's last chunk to finish adds
    // the scene's partial sums in a fixed order, so the loss does not depend on timing
    griddep_wait();  // the pair sums come from the edge kernel
    flag0 |= *reinterpret_cast<volatile const int*>(a.flag) & kFlagBounds;
    const int c = blockIdx.x - n_pose_blocks;
    const int s = a.loss_chunk_scene[c];
    const int2 range = a.loss_chunk_pairs[c];
    const int p = range.x + (int)threadIdx.x;
    double acc = 0.0;
    if (p < range.y) {
      const double w = a.pair_lw[p];  // 0 for an inactive pair
      double wn = 0.0;                // the weight of the pair's samples: w / n_p (w under Eq. 7)
      if (w != 0.0) {
        const double* pa = a.pair_acc + (size_t)kAcc * p;
        if (a.norm_all) {
          wn = w;
        } else if (pa[1] > 0.0) {
          wn = w * __drcp_rn(pa[1]);
        }
        acc = wn * pa[0];
      }
      if (a.pair_wz) a.pair_wz[p] = (float)wn;  // refine scenes: read by the depth kernel
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    unsigned prev = 0u;
    if (threadIdx.x == 0) {
      a.loss_part[c] = acc;
      __threadfence();
      prev = atomicAdd(a.scene_done + s, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    const int c0 = a.loss_chunk_off[s], nc = a.loss_chunk_off[s + 1] - c0;
    if (prev == (unsigned)nc - 1u) {
      __threadfence();
      double t = 0.0;
      for (int k = threadIdx.x; k < nc; k += kLossChunk) t += __ldcg(a.loss_part + c0 + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) {
        const double L = t;  // the weights carry the 2 / (active pairs) factor
        a.loss[s] = L;
        if (a.host_out) a.host_out[12 * (size_t)a.n_views + s] = L;
        if (!isfinite(L)) {
          atomicOr(a.flag, 1);
          bad_here = true;
        }
        a.scene_done[s] = 0u;
      }
    }
  }
  if (with_grad == 2 && !a.pose_mlp) {
    // the last block to finish advances the step counter and the beta powers (under the pose
    // MLP its update kernel does), unless the step began flagged or a block flagged it.  The
    // blocks report completion and their flag in one atomic: low word a count, high word the
    // flagged blocks, so that no fence is needed (the last block reads nothing else that the
    // others wrote in this kernel)
    const bool bad_block = __any_sync(0xffffffffu, bad_here);
    if (threadIdx.x == 0) {
      const unsigned long long add = 1ull + (bad_block ? (1ull << 32) : 0ull);
      const unsigned long long prev = atomicAdd(a.done, add);
      if ((unsigned int)prev == gridDim.x - 1) {
        if (!(flag0 & kFlagRefuse) && ((prev + add) >> 32) == 0ull) {
          *a.step = step + 1;
          a.bpow[0] *= a.beta1;
          a.bpow[1] *= a.beta2;
        }
        if (a.host_out)  // the step's status word: the flag it began with or set
          *reinterpret_cast<int32_t*>(a.host_out + 12 * (size_t)a.n_views + a.n_scenes) =
              flag0 | (((prev + add) >> 32) ? 1 : 0);
        *a.done = 0ull;
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// SE(3) in FP64 for the autograd path (textbook closed forms; xi = (upsilon, omega))
// ------------------------------------------------------------------------------------
__device__ void se3_exp_dev(const double xi[6], double E[12]) {
  const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  const double th = sqrt(th2);
  double A, B, C;
  if (th < 1e-4) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    double s, c;
    sincos(th, &s, &c);
    A = s / th;
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
  }
  // W = [w]x, W^2 = w w^T - th2 I
  const double W[9] = {0, -w2, w1, w2, 0, -w0, -w1, w0, 0};
  const double w[3] = {w0, w1, w2};
  for (int r = 0; r < 3; ++r) {
    double tr = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double I = r == c ? 1.0 : 0.0;
      const double W2 = w[r] * w[c] - (r == c ? th2 : 0.0);
      E[4 * r + c] = I + A * W[3 * r + c] + B * W2;
      tr += (I + B * W[3 * r + c] + C * W2) * xi[c];
    }
    E[4 * r + 3] = tr;
  }
}

// out = E T (rigid 3x4 composition)
__device__ void compose_dev(const double E[12], const double* T, double* out) {
  double o[12];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c)
      o[4 * r + c] = E[4 * r] * T[c] + E[4 * r + 1] * T[4 + c] + E[4 * r + 2] * T[8 + c] +
                     (c == 3 ? E[4 * r + 3] : 0.0);
  for (int k = 0; k < 12; ++k) out[k] = o[k];
}

__global__ void k_twist_poses(const double* T, const double* xi, double* T_out, int n) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double x[6];
  for (int k = 0; k < 6; ++k) x[k] = xi ? xi[6 * (size_t)v + k] : 0.0;
  double E[12];
  se3_exp_dev(x, E);
  compose_dev(E, T + 12 * (size_t)v, T_out + 12 * (size_t)v);
}

// out = J_l(xi)^T g, J_l = [[Jw, Q], [0, Jw]] the SE(3) left Jacobian (Barfoot, Sec. 7.1.5).
__global__ void k_apply_left_jacobian(const double* xi, const double* g, double* out, int n) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double x[6], gg[6];
  for (int k = 0; k < 6; ++k) {
    x[k] = xi ? xi[6 * (size_t)v + k] : 0.0;
    gg[k] = g[6 * (size_t)v + k];
  }
  const double* p = x;      // upsilon
  const double* w = x + 3;  // omega
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double th = sqrt(th2);
  double B, C, c1, c2, c3;
  if (th < 0.05) {
    const double t4 = th2 * th2;
    B = 0.5 - th2 / 24.0 + t4 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + t4 / 5040.0;
    c1 = C;
    c2 = 1.0 / 24.0 - th2 / 720.0 + t4 / 40320.0;
    c3 = 1.0 / 120.0 - th2 / 2520.0 + t4 / 120960.0;
  } else {
    double s, c;
    sincos(th, &s, &c);
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
    c1 = C;
    c2 = (0.5 * th2 + c - 1.0) / (th2 * th2);
    c3 = (2.0 * th - 3.0 * s + th * c) / (2.0 * th2 * th2 * th);
  }
  auto hat = [](const double* a, double* M) {
    M[0] = 0; M[1] = -a[2]; M[2] = a[1]; M[3] = a[2]; M[4] = 0; M[5] = -a[0];
    M[6] = -a[1]; M[7] = a[0]; M[8] = 0;
  };
  auto mul = [](const double* A, const double* B2, double* Cm) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Cm[3 * r + c] = A[3 * r] * B2[c] + A[3 * r + 1] * B2[3 + c] + A[3 * r + 2] * B2[6 + c];
  };
  double Wm[9], Pm[9], W2[9], WP[9], PW[9], WPW[9], WWP[9], PWW[9], WPWW[9], WWPW[9];
  hat(w, Wm);
  hat(p, Pm);
  mul(Wm, Wm, W2);
  mul(Wm, Pm, WP);
  mul(Pm, Wm, PW);
  mul(WP, Wm, WPW);
  mul(Wm, WP, WWP);
  mul(PW, Wm, PWW);
  mul(WPW, Wm, WPWW);
  mul(Wm, WPW, WWPW);
  double Jw[9], Q[9];
  for (int k = 0; k < 9; ++k) {
    Jw[k] = ((k % 4) == 0 ? 1.0 : 0.0) + B * Wm[k] + C * W2[k];
    Q[k] = 0.5 * Pm[k] + c1 * (WP[k] + PW[k] + WPW[k]) + c2 * (WWP[k] + PWW[k] - 3.0 * WPW[k]) +
           c3 * (WPWW[k] + WWPW[k]);
  }
  // J^T g: top = Jw^T g_u ; bottom = Q^T g_u + Jw^T g_w
  for (int c = 0; c < 3; ++c) {
    double top = 0.0, bot = 0.0;
    for (int r = 0; r < 3; ++r) {
      top += Jw[3 * r + c] * gg[r];
      bot += Q[3 * r + c] * gg[r] + Jw[3 * r + c] * gg[3 + r];
    }
    out[6 * (size_t)v + c] = top;
    out[6 * (size_t)v + 3 + c] = bot;
  }
}

// ------------------------------------------------------------------------------------
// construction helpers
// ------------------------------------------------------------------------------------
__global__ void k_map_check(const void* map, int dtype, int64_t n, int32_t* bad) {
  int cnt = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    float x = dtype == 0 ? reinterpret_cast<const float*>(map)[k]
                         : bf16_bits_to_float(reinterpret_cast<const unsigned short*>(map)[k]);
    cnt += !(isfinite(x) && x >= 0.f);
  }
  if (cnt) atomicAdd(bad, cnt);
}

// Exact Euclidean distance transform, one block per strip of CB columns.  Pass 1 puts, for
// every pixel of the strip, the squared distance to the nearest edge of its own row into
// shared memory (outward scan of the mask row).  Pass 2 takes, per pixel, the minimum over
// rows y' of f(x, y') + (y - y')^2, scanning outward from y and stopping once (y - y')^2
// alone exceeds the best value.  Every value is an integer below 2^24, exact in f32; the
// final sqrtf is correctly rounded.
constexpr int kEdtCols = 32;
constexpr int kEdtMaxH = 1536;  // kEdtCols * kEdtMaxH * 4 B = 192 KB of shared memory

__global__ void k_edt(const uint8_t* edges, int W, int H, float* out) {
  extern __shared__ float f[];  // [H][kEdtCols]
  const float INF = 3.0e38f;
  const int xb = blockIdx.x * kEdtCols;
  const int nc = min(kEdtCols, W - xb);
  for (int e = threadIdx.x; e < nc * H; e += blockDim.x) {
    const int c = e % nc, y = e / nc;
    const int x = xb + c;
    const uint8_t* row = edges + (size_t)y * W;
    float best = INF;
    for (int d = 0; d < W; ++d) {
      const bool l = x - d >= 0 && row[x - d];
      const bool r = x + d < W && row[x + d];
      if (l || r) { best = (float)d * (float)d; break; }
      if (x - d < 0 && x + d >= W) break;
    }
    f[y * kEdtCols + c] = best;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * H; e += blockDim.x) {
    const int c = e % nc, y = e / nc;
    float best = f[y * kEdtCols + c];
    for (int d = 1; (float)d * (float)d < best && (y - d >= 0 || y + d < H); ++d) {
      const float dd = (float)d * (float)d;
      if (y - d >= 0) best = fminf(best, f[(y - d) * kEdtCols + c] + dd);
      if (y + d < H) best = fminf(best, f[(y + d) * kEdtCols + c] + dd);
    }
    out[(size_t)y * W + xb + c] = best >= INF ? (float)(W + H) : sqrtf(best);
  }
}

__global__ void k_round_bf16(const float* src, uint16_t* dst, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = __bfloat16_as_ushort(__float2bfloat16_rn(src[k]));
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------
// Stochastic viewgraph sub-sampling (Algorithm 3, Appendix A.3): each evaluation uses a
// fresh uniform random subset of min(P_s, M) of a scene's P_s pairs.  Pair p (index within
// its scene) at step s gets the key SplitMix64(seed ^ (s << 32 | p)) (the output function of
// Steele, Lea and Flood's generator, OOPSLA 2014, on state + its golden-ratio increment);
// the M smallest keys are taken, ties by index.  One block per scene finds the M-th
// smallest key by a radix select over its 8 bytes (a 256-bin histogram per byte, high byte
// first), then writes every pair's flag and loss weight.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t subsample_key(uint64_t seed, int64_t step, int p) {
  return splitmix64_out(seed ^ (((uint64_t)step << 32) | (uint32_t)p));
}

constexpr int kSubsampleThreads = 1024;

__global__ void __launch_bounds__(kSubsampleThreads) k_subsample(StepArgs a) {
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_k, s_eq;
  const int sc = blockIdx.x;
  const int off = a.scene_pair_off[sc], P = a.scene_pair_off[sc + 1] - off;
  const int M = a.pair_budget;
  const int64_t step = *a.step;
  const uint64_t seed = a.subsample_seed;
  const bool all = M <= 0 || P <= M;
  const int na = all ? P : M;
  uint64_t thr = ~0ull;
  int k_eq = 0;
  if (!all) {
    if (threadIdx.x == 0) {
      s_prefix = 0ull;
      s_k = M;  // rank (1-based) of the cut within the keys that share the prefix
    }
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
      __syncthreads();
      const uint64_t prefix = s_prefix;
      const uint64_t hm = shift == 56 ? 0ull : (~0ull << (shift + 8));
      for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const uint64_t key = subsample_key(seed, step, p);
        if ((key & hm) == (prefix & hm)) atomicAdd(&hist[(key >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned k = (unsigned)s_k;
        unsigned cum = 0u;
        int d = 0;
        for (; d < 255; ++d) {
          if (cum + hist[d] >= k) break;
          cum += hist[d];
        }
        s_k = (int)(k - cum);
        s_prefix = prefix | ((uint64_t)d << shift);
      }
      __syncthreads();
    }
    thr = s_prefix;  // the M-th smallest key
    k_eq = s_k;      // how many of the keys equal to it are taken
    if (threadIdx.x == 0) s_eq = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x)
      if (subsample_key(seed, step, p) == thr) atomicAdd(&s_eq, 1);
    __syncthreads();
  }
  const bool ties = !all && s_eq != k_eq;  // equal 64-bit keys across the cut: index order decides
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    bool act = true;
    if (!all) {
      const uint64_t key = subsample_key(seed, step, p);
      act = key < thr || (key == thr && !ties);
    }
    const int q = off + p;
    double w = 0.0;
    if (act) {
      w = 2.0 / na;
      if (a.norm_all) {
        const int32_t n = a.views[a.pair_src[q]].n_rec;
        w = n > 0 ? w / (double)n : 0.0;
      }
    }
    a.pair_active_w[q] = act ? 1 : 0;
    a.pair_lw[q] = w;
  }
  __syncthreads();  // every flag is written before the tied ones are set in index order
  if (ties && threadIdx.x == 0) {
    int taken = 0;
    for (int p = 0; p < P; ++p)
      if (subsample_key(seed, step, p) == thr) {
        const int q = off + p;
        const bool act = taken++ < k_eq;
        double w = 0.0;
        if (act) {
          w = 2.0 / na;
          if (a.norm_all) {
            const int32_t n = a.views[a.pair_src[q]].n_rec;
            w = n > 0 ? w / (double)n : 0.0;
          }
        }
        a.pair_active_w[q] = act ? 1 : 0;
        a.pair_lw[q] = w;
      }
  }
}

// ------------------------------------------------------------------------------------
// Optimization schedule (Section 3): after every step, theta_95 = max(95th percentile of
// the rotation changes, 95th percentile of the translation-direction changes) over the
// scene's poses, then the dual-phase rule.  One block per scene; the percentile takes the
// two order statistics around 0.95 (n - 1) by radix select over the bit patterns of the
// (non-negative) doubles and interpolates between them linearly.
// ------------------------------------------------------------------------------------
constexpr int kScheduleThreads = 256;

// k-th smallest (0-based) of n non-negative doubles; every thread of the block calls it.
__device__ double block_kth(const double* x, int n, int k, unsigned* hist, unsigned long long* s_prefix, int* s_k) {
  if (threadIdx.x == 0) {
    *s_prefix = 0ull;
    *s_k = k + 1;
  }
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    const unsigned long long prefix = *s_prefix;
    const unsigned long long hm = shift == 56 ? 0ull : (~0ull << (shift + 8));
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long key = (unsigned long long)__double_as_longlong(x[i]);
      if ((key & hm) == (prefix & hm)) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned kk = (unsigned)*s_k;
      unsigned cum = 0u;
      int d = 0;
      for (; d < 255; ++d) {
        if (cum + hist[d] >= kk) break;
        cum += hist[d];
      }
      *s_k = (int)(kk - cum);
      *s_prefix = prefix | ((unsigned long long)d << shift);
    }
    __syncthreads();
  }
  return __longlong_as_double((long long)*s_prefix);
}

__device__ double block_percentile95(const double* x, int n, unsigned* hist, unsigned long long* s_prefix, int* s_k) {
  if (n <= 0) return 0.0;
  const double pos = 0.95 * (double)(n - 1);
  const int lo = (int)floor(pos);
  const double a = block_kth(x, n, lo, hist, s_prefix, s_k);
  if (lo >= n - 1) return a;
  const double b = block_kth(x, n, lo + 1, hist, s_prefix, s_k);
  return a + (b - a) * (pos - (double)lo);
}

__global__ void __launch_bounds__(kScheduleThreads) k_schedule(StepArgs a) {
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_k;
  const int sc = blockIdx.x;
  const int v0 = a.scene_view_off[sc], n = a.scene_view_off[sc + 1] - v0;
  int32_t* st = a.sched_state + 2 * sc;
  if (st[0] == 3) return;  // uniform over the block: converged earlier
  const double pR = block_percentile95(a.pose_dR + v0, n, hist, &s_prefix, &s_k);
  const double pT = block_percentile95(a.pose_dt + v0, n, hist, &s_prefix, &s_k);
  if (threadIdx.x == 0) {
    const double theta = fmax(pR, pT);
    a.theta95[sc] = theta;
    const int64_t step = *a.step - 1;  // the step just taken (the pose kernel advanced the counter)
    if (st[0] == 1) {
      st[1] = theta < a.sched_eps1 ? st[1] + 1 : 0;
      if (st[1] >= a.sched_w1) {
        st[0] = 2;
        st[1] = 0;
        a.sched_steps[2 * sc] = step;
      }
    } else if (st[0] == 2) {
      st[1] = theta < a.sched_eps2 ? st[1] + 1 : 0;
      if (st[1] >= a.sched_w2) {
        st[0] = 3;
        a.sched_steps[2 * sc + 1] = step;
      }
    }
  }
}

cudaError_t launch_schedule(const StepArgs& a, cudaStream_t s) {
  k_schedule<<<a.n_scenes, kScheduleThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_subsample(const StepArgs& a, cudaStream_t s) {
  k_subsample<<<a.n_scenes, kSubsampleThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_refine_intrinsics(const StepArgs& a, cudaStream_t s) {
  k_refine_intrinsics<<<std::max((a.n_views + 127) / 128, 1), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pair_setup(const StepArgs& a, int mode, cudaStream_t s) {
  const int nb = std::max((a.n_pairs * kSetupLanes + kSetupThreads - 1) / kSetupThreads, 1);
  k_pair_setup<<<nb, kSetupThreads, 0, s>>>(a, mode);
  return cudaGetLastError();
}

// Read a buffer through L2 (values folded into one word, written only on an impossible
// match so the loads stay); with a preceding write of the same buffer this leaves L2 full
// of clean lines unrelated to the next kernel's inputs (a cold start for timing).
__global__ void __launch_bounds__(256) k_l2_read(const uint4* p, int64_t n, unsigned* sink) {
  unsigned acc = 0u;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    acc ^= __ldcg(p + k).x;
  if (acc == 0x9e3779b9u) *sink = acc;
}

cudaError_t launch_l2_read(const void* p, int64_t bytes, unsigned* sink, int sms, cudaStream_t s) {
  k_l2_read<<<4 * sms, 256, 0, s>>>((const uint4*)p, bytes / 16, sink);
  return cudaGetLastError();
}

cudaError_t launch_poses(const StepArgs& a, int with_grad, cudaStream_t s) {
  const int nbp = (a.n_views + kPosesPerBlock - 1) / kPosesPerBlock;
  return launch_pdl(k_poses, dim3(nbp + a.n_loss_chunks), dim3(kPoseThreads), 0, s, a, with_grad, nbp);
}

// Copy of n doubles between device memory and mapped pinned host memory, inside a step's
// graph (the host-driven step): the GPU reads and writes the host buffer directly, so no copy
// engine round trip sits on the step's critical path.  Reads use ld.global.cv, so that a line
// of host memory cached by an earlier step is fetched again.
// Copies between device memory and the mapped host staging: 16-byte accesses where both
// sides allow them, one element per thread (a host access waits on the link, so all of them
// are issued at once rather than in a loop per thread).
__global__ void __launch_bounds__(256) k_io_copy(const double* src, double* dst, int64_t n) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) dst[k] = __ldcv(src + k);
}
__global__ void __launch_bounds__(256) k_io_copy2(const double2* src, double2* dst, int64_t n2) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n2) dst[k] = __ldcv(src + k);
}

cudaError_t launch_io_copy(const double* src, double* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (((uintptr_t)src | (uintptr_t)dst) % 16 == 0 && n % 2 == 0) {
    k_io_copy2<<<(unsigned)((n / 2 + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(src),
                                                              reinterpret_cast<double2*>(dst), n / 2);
  } else {
    k_io_copy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
  }
  return cudaGetLastError();
}

// One block per view.  The stored X is within u |X| of the exact point (one rounding of an FP64
// value); with the rotation's rounded entries and the edge kernel's FMA chain (z taken last),
// every component of Y = R X + t is then within u (5 |X0| + 4 |X1| + 2 z) + 4u |t|_1 of the exact
// one, and the depth test's subtraction against the double-precision threshold adds 2u eps_z;
// the record's share, with a 1e-5 relative margin, is the stored fourth component.
template <int REC>
__global__ void __launch_bounds__(256) k_lift_records(const void* rec, const ViewDev* views, const double* K64,
                                                      float eps_z, float4* out) {
  const ViewDev vw = views[blockIdx.x];
  const double* K = K64 + 6 * (size_t)blockIdx.x;
  const double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
  for (int k = threadIdx.x; k < vw.n_rec; k += blockDim.x) {
    const int64_t r = vw.rec_begin + k;
    float u, v, z;
    load_record<REC>(rec, r, u, v, z);
    const float X0 = (float)(((double)u - cx) / fx * (double)z);
    const float X1 = (float)(((double)v - cy) / fy * (double)z);
    const float w = (kU32 * 1.00001f) * fmaf(5.f, fabsf(X0), fmaf(4.f, fabsf(X1), fmaf(2.f, z, 2.f * eps_z)));
    out[r] = make_float4(X0, X1, z, w);
  }
}

cudaError_t launch_lift_records(const void* rec, int rec_dtype, const ViewDev* views, const double* K64,
                                int n_views, float eps_z, float4* out, cudaStream_t s) {
  if (n_views <= 0) return cudaSuccess;
  if (rec_dtype == 0) k_lift_records<0><<<n_views, 256, 0, s>>>(rec, views, K64, eps_z, out);
  else k_lift_records<1><<<n_views, 256, 0, s>>>(rec, views, K64, eps_z, out);
  return cudaGetLastError();
}

cudaError_t launch_twist_poses(const double* T, const double* xi, double* T_out, int n,
                               cudaStream_t s) {
  k_twist_poses<<<(n + 127) / 128, 128, 0, s>>>(T, xi, T_out, n);
  return cudaGetLastError();
}

cudaError_t launch_apply_left_jacobian(const double* xi, const double* g, double* out, int n,
                                       cudaStream_t s) {
  k_apply_left_jacobian<<<(n + 127) / 128, 128, 0, s>>>(xi, g, out, n);
  return cudaGetLastError();
}

cudaError_t launch_map_check(const void* map, int dtype, int64_t n, int32_t* bad, cudaStream_t s) {
  int64_t nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  if (nb < 1) nb = 1;
  k_map_check<<<(int)nb, 256, 0, s>>>(map, dtype, n, bad);
  return cudaGetLastError();
}

int edt_max_height() { return kEdtMaxH; }

cudaError_t launch_edt(const uint8_t* edges, int W, int H, float* map, cudaStream_t s) {
  const size_t smem = sizeof(float) * kEdtCols * (size_t)H;
  cudaError_t e = cudaFuncSetAttribute(k_edt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * kEdtCols * kEdtMaxH));
  if (e != cudaSuccess) return e;
  k_edt<<<(W + kEdtCols - 1) / kEdtCols, 256, smem, s>>>(edges, W, H, map);
  return cudaGetLastError();
}

cudaError_t launch_round_bf16(const float* src, uint16_t* dst, int64_t n, cudaStream_t s) {
  int64_t nb = (n + 255) / 256;
  if (nb > 8192) nb = 8192;
  if (nb < 1) nb = 1;
  k_round_bf16<<<(int)nb, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace epo
