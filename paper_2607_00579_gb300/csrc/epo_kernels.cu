// Kernels of the edge-alignment library (sm_103a).
//
// Hot path (one optimisation step, Algorithm 2 with the pose-only reading):
//   k_pair_setup   a1: T_ji = T_j T_i^-1 in FP64, rounded to FP32; lambda from the step.
//   k_edge         a2-a7: persistent, work = (source view, tile of edge records).  Each
//                  thread lifts its records once (the split projection of Algorithm 2:
//                  lift once per image, project into every paired view), then for every
//                  outgoing pair i -> j: transform, project (Eq. 8), gather the 2x2
//                  footprint of DTF_j, bilinear value and slope, clamp + Huber (Eq. 7),
//                  the adjoint 6-vector, and a warp-shuffle + block reduction ending in
//                  one FP64 atomic per block per pair slot (the in-kernel per-pair
//                  reduction of the fused ProjectSampleHuber kernel, Appendix A.2).
//   k_fin_pairs    a8: per-pair mean (Algorithm 3: sum rho / sum valid), the pair's
//                  gradient contributions to its target and, through -Ad(T_ji)^T, to its
//                  source, in FP64.
//   k_fin_poses    a8: deterministic per-pose gather and per-scene loss (Eq. 6).
//   k_retract      a9: tangent-space Adam and T <- Exp(-Delta) T in FP64.
// Construction helpers: k_edt (exact distance transform field), k_round_bf16, k_map_check.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "epo_internal.cuh"

namespace epo {

// ------------------------------------------------------------------------------------
// a1: pair setup
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double lambda_at(const StepArgs& a, int64_t s) {
  double f = a.lambda_steps > 0 ? (double)s / (double)a.lambda_steps : 1.0;
  f = f > 1.0 ? 1.0 : f;
  return a.lambda0 + (a.lambda1 - a.lambda0) * f;
}

__global__ void k_pair_setup(StepArgs a, int mode) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) *a.lambda = lambda_at(a, *a.step);
  if (p >= a.n_pairs) return;
  const double* Ti = a.T + 12 * a.pair_src[p];
  const double* Tj = a.T + 12 * a.pair_dst[p];
  double R[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = Tj[4 * r] * Ti[4 * c] + Tj[4 * r + 1] * Ti[4 * c + 1] + Tj[4 * r + 2] * Ti[4 * c + 2];
  PairParam out;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double t = Tj[4 * r + 3] - (R[3 * r] * Ti[3] + R[3 * r + 1] * Ti[7] + R[3 * r + 2] * Ti[11]);
    out.t[r] = (float)t;
#pragma unroll
    for (int c = 0; c < 3; ++c) out.r[3 * r + c] = (float)R[3 * r + c];
  }
  a.pp[p] = out;
  double* acc = a.pair_acc + (size_t)kAcc * p;
  if (mode != MODE_BWD) { acc[0] = 0.0; acc[1] = 0.0; }
  if (mode != MODE_FWD) {
#pragma unroll
    for (int k = 2; k < kAcc; ++k) acc[k] = 0.0;
  }
}

// ------------------------------------------------------------------------------------
// a2-a7: the edge kernel
// ------------------------------------------------------------------------------------
template <int REC>
__device__ __forceinline__ void load_record(const void* base, int64_t idx, float& u, float& v,
                                            float& z) {
  if (REC == 0) {  // EPO_F32: {u, v, z, 0}
    float4 r = __ldg(reinterpret_cast<const float4*>(base) + idx);
    u = r.x; v = r.y; z = r.z;
  } else {         // EPO_F16: {u16 u, u16 v, f16 z, u16 0}
    uint2 r = __ldg(reinterpret_cast<const uint2*>(base) + idx);
    u = (float)(r.x & 0xffffu);
    v = (float)(r.x >> 16);
    z = __half2float(__ushort_as_half((unsigned short)(r.y & 0xffffu)));
  }
}

__device__ __forceinline__ float bf16_bits_to_float(unsigned int b) { return __uint_as_float(b << 16); }

// 2x2 footprint (x0, y0) .. (x0+1, y0+1) of a map.
template <int MAP, int GATHER>
__device__ __forceinline__ void taps(const void* map, int64_t off, int pitch, unsigned long long tex,
                                     int x0, int y0, float& m00, float& m01, float& m10, float& m11) {
  if (GATHER == GATHER_TEX) {
    // tex2Dgather at the centre of the 2x2 block returns it as (x: (x0, y0+1), y: (x0+1, y0+1),
    // z: (x0+1, y0), w: (x0, y0)); unnormalised coordinates, point fetch, no filtering.
    float fx = (float)x0 + 1.0f, fy = (float)y0 + 1.0f;
    if (MAP == 0) {
      float4 g = tex2Dgather<float4>((cudaTextureObject_t)tex, fx, fy, 0);
      m00 = g.w; m01 = g.z; m10 = g.x; m11 = g.y;
    } else {
      ushort4 g = tex2Dgather<ushort4>((cudaTextureObject_t)tex, fx, fy, 0);
      m00 = bf16_bits_to_float(g.w); m01 = bf16_bits_to_float(g.z);
      m10 = bf16_bits_to_float(g.x); m11 = bf16_bits_to_float(g.y);
    }
  } else {
    if (MAP == 0) {
      const float* m = reinterpret_cast<const float*>(map) + off + (int64_t)y0 * pitch + x0;
      m00 = __ldg(m); m01 = __ldg(m + 1); m10 = __ldg(m + pitch); m11 = __ldg(m + pitch + 1);
    } else {
      const unsigned short* m = reinterpret_cast<const unsigned short*>(map) + off + (int64_t)y0 * pitch + x0;
      m00 = bf16_bits_to_float(__ldg(m)); m01 = bf16_bits_to_float(__ldg(m + 1));
      m10 = bf16_bits_to_float(__ldg(m + pitch)); m11 = bf16_bits_to_float(__ldg(m + pitch + 1));
    }
  }
}

template <int MODE, int REC, int MAP, int GATHER, int RPT>
__global__ void __launch_bounds__(512) k_edge(EdgeArgs a) {
  constexpr int NACC = MODE == MODE_FWD ? 2 : (MODE == MODE_BWD ? 6 : 8);
  constexpr int SLOT0 = MODE == MODE_BWD ? 2 : 0;
  __shared__ float s_red[2][32][NACC];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const float lam = (float)(*a.lambda);
  const float delta = a.delta;
  const float eps_z = a.eps_z;
  int buf = 0;
  for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    const TileDev td = a.tiles[t];
    const ViewDev vi = a.views[td.view];
    // a2: lift once per record (camera-i frame), reused for every pair of this view
    float X0[RPT], X1[RPT], X2[RPT];
    bool have[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int idx = threadIdx.x + r * blockDim.x;
      have[r] = idx < td.n;
      float u = 0.f, v = 0.f, z = 0.f;
      if (have[r]) load_record<REC>(a.rec, td.begin + idx, u, v, z);
      X0[r] = (u - vi.cx) / vi.fx * z;
      X1[r] = (v - vi.cy) / vi.fy * z;
      X2[r] = z;
    }
    const int pb = a.src_pair_off[td.view];
    const int pe = a.src_pair_off[td.view + 1];
    for (int q = pb; q < pe; ++q) {
      const int p = a.src_pair_ids[q];
      if (!a.pair_active[p]) continue;  // uniform over the block
      const PairParam P = a.pp[p];
      const int j = a.pair_dst[p];
      const ViewDev vj = a.views[j];
      const unsigned long long tex = GATHER == GATHER_TEX ? a.tex[j] : 0ull;
      const float Wm1 = (float)(vj.W - 1), Hm1 = (float)(vj.H - 1);
      float acc[NACC];
#pragma unroll
      for (int k = 0; k < NACC; ++k) acc[k] = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        // a3: transform + project into view j
        const float Y0 = fmaf(P.r[0], X0[r], fmaf(P.r[1], X1[r], fmaf(P.r[2], X2[r], P.t[0])));
        const float Y1 = fmaf(P.r[3], X0[r], fmaf(P.r[4], X1[r], fmaf(P.r[5], X2[r], P.t[1])));
        const float Y2 = fmaf(P.r[6], X0[r], fmaf(P.r[7], X1[r], fmaf(P.r[8], X2[r], P.t[2])));
        bool ok = have[r] && (Y2 > eps_z);
        const float iz = ok ? __frcp_rn(Y2) : 0.f;
        const float up = fmaf(vj.fx, Y0 * iz, vj.cx);
        const float vp = fmaf(vj.fy, Y1 * iz, vj.cy);
        ok = ok && (up >= 0.f) && (up <= Wm1) && (vp >= 0.f) && (vp <= Hm1);
        if (ok) {
          // a4: bilinear sample of DTF_j and its slope
          const int x0 = min((int)floorf(up), vj.W - 2);
          const int y0 = min((int)floorf(vp), vj.H - 2);
          const float ca = up - (float)x0;
          const float cb = vp - (float)y0;
          float m00, m01, m10, m11;
          taps<MAP, GATHER>(a.map, vj.map_off, vj.pitch, tex, x0, y0, m00, m01, m10, m11);
          const float top = fmaf(ca, m01 - m00, m00);
          const float bot = fmaf(ca, m11 - m10, m10);
          const float d = fmaf(cb, bot - top, top);
          // a5: clamp + Huber
          const float dh = fminf(d, lam);
          const float adh = fabsf(dh);
          const float rho = adh <= delta ? 0.5f * dh * dh : delta * (adh - 0.5f * delta);
          if constexpr (MODE != MODE_BWD) {
            acc[0] += rho;
            acc[1] += 1.f;
          }
          if constexpr (MODE != MODE_FWD) {
            constexpr int G0 = MODE == MODE_BWD ? 0 : 2;  // first gradient slot in acc
            // a6: adjoint in camera-j coordinates
            const float drho = d <= lam ? (fabsf(d) <= delta ? d : copysignf(delta, d)) : 0.f;
            const float ddu = fmaf(cb, (m11 - m10) - (m01 - m00), m01 - m00);
            const float ddv = bot - top;
            const float gx = drho * ddu * vj.fx * iz;
            const float gy = drho * ddv * vj.fy * iz;
            const float gz = -(gx * Y0 + gy * Y1) * iz;
            acc[G0 + 0] += gx;
            acc[G0 + 1] += gy;
            acc[G0 + 2] += gz;
            acc[G0 + 3] += Y1 * gz - Y2 * gy;
            acc[G0 + 4] += Y2 * gx - Y0 * gz;
            acc[G0 + 5] += Y0 * gy - Y1 * gx;
          }
        }
      }
      // a7: warp shuffle -> block -> one FP64 atomic per slot
#pragma unroll
      for (int k = 0; k < NACC; ++k) {
        float s = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) s_red[buf][warp][k] = s;
      }
      __syncthreads();
      if (threadIdx.x < NACC) {
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += (double)s_red[buf][w][threadIdx.x];
        if (s != 0.0) atomicAdd(a.pair_acc + (size_t)kAcc * p + SLOT0 + threadIdx.x, s);
      }
      buf ^= 1;  // the other buffer is free: its readers finished before this barrier
    }
  }
}

// ------------------------------------------------------------------------------------
// a8: finalize (FP64)
// ------------------------------------------------------------------------------------
__global__ void k_fin_pairs(StepArgs a, int with_grad) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n_pairs) return;
  double* c12 = a.contrib + 12 * (size_t)p;
  if (!a.pair_active[p]) {
    a.pair_loss[p] = 0.0;
    if (with_grad)
      for (int k = 0; k < 12; ++k) c12[k] = 0.0;
    return;
  }
  const int i = a.pair_src[p];
  const int j = a.pair_dst[p];
  const double* acc = a.pair_acc + (size_t)kAcc * p;
  const double denom = a.norm_all ? (double)a.views[i].n_rec : acc[1];
  a.pair_loss[p] = denom > 0.0 ? acc[0] / denom : 0.0;
  if (!with_grad) return;
  const int s = a.pair_scene[p];
  const double gs = a.gscale ? a.gscale[s] : 1.0;
  const int na = a.scene_active_pairs[s];
  const double c = (denom > 0.0 && na > 0) ? (2.0 / na) * gs / denom : 0.0;
  double ga[3], gb[3];
  for (int k = 0; k < 3; ++k) {
    ga[k] = c * acc[2 + k];
    gb[k] = c * acc[5 + k];
    c12[k] = ga[k];
    c12[3 + k] = gb[k];
  }
  // source view: -Ad(T_ji)^T (ga, gb) = (-R^T ga, R^T (t x ga) - R^T gb)
  const double* Ti = a.T + 12 * i;
  const double* Tj = a.T + 12 * j;
  double R[9], t[3];
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc)
      R[3 * r + cc] = Tj[4 * r] * Ti[4 * cc] + Tj[4 * r + 1] * Ti[4 * cc + 1] + Tj[4 * r + 2] * Ti[4 * cc + 2];
  for (int r = 0; r < 3; ++r)
    t[r] = Tj[4 * r + 3] - (R[3 * r] * Ti[3] + R[3 * r + 1] * Ti[7] + R[3 * r + 2] * Ti[11]);
  const double tx[3] = {t[1] * ga[2] - t[2] * ga[1], t[2] * ga[0] - t[0] * ga[2], t[0] * ga[1] - t[1] * ga[0]};
  for (int cc = 0; cc < 3; ++cc) {
    double rta = R[cc] * ga[0] + R[3 + cc] * ga[1] + R[6 + cc] * ga[2];
    double rtx = R[cc] * tx[0] + R[3 + cc] * tx[1] + R[6 + cc] * tx[2];
    double rtb = R[cc] * gb[0] + R[3 + cc] * gb[1] + R[6 + cc] * gb[2];
    c12[6 + cc] = -rta;
    c12[9 + cc] = rtx - rtb;
  }
}

__global__ void k_fin_poses(StepArgs a, int with_grad, int n_pose_blocks) {
  __shared__ double s_sum[256];
  if ((int)blockIdx.x < n_pose_blocks) {
    if (!with_grad) return;
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.n_views) return;
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int e = a.pose_pair_off[v]; e < a.pose_pair_off[v + 1]; ++e) {
      int ref = a.pose_pair_ref[e];
      const double* c = a.contrib + 12 * (size_t)(ref >> 1) + 6 * (ref & 1);
      for (int k = 0; k < 6; ++k) g[k] += c[k];
    }
    bool fin = true;
    for (int k = 0; k < 6; ++k) {
      a.grad[6 * (size_t)v + k] = g[k];
      fin = fin && isfinite(g[k]);
    }
    if (!fin) atomicOr(a.flag, 1);
    return;
  }
  // per-scene loss, fixed-order reduction
  const int s = blockIdx.x - n_pose_blocks;
  const int pb = a.scene_pair_off[s], pe = a.scene_pair_off[s + 1];
  double acc = 0.0;
  for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) acc += a.pair_loss[p];
  s_sum[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int na = a.scene_active_pairs[s];
    const double L = na > 0 ? (2.0 / na) * s_sum[0] : 0.0;
    a.loss[s] = L;
    if (!isfinite(L)) atomicOr(a.flag, 1);
  }
}

// ------------------------------------------------------------------------------------
// a9: SE(3) in FP64 (textbook closed forms; xi = (upsilon, omega))
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

__global__ void k_retract(StepArgs a) {
  const int64_t s = *a.step;
  const int flag = *a.flag;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < a.n_views && !(flag & 1) && !a.fixed[v]) {
    const double bc1 = 1.0 - pow(a.beta1, (double)(s + 1));
    const double bc2 = 1.0 - pow(a.beta2, (double)(s + 1));
    double xi[6];
    for (int k = 0; k < 6; ++k) {
      const size_t o = 6 * (size_t)v + k;
      const double g = a.grad[o];
      const double m = a.beta1 * a.m[o] + (1.0 - a.beta1) * g;
      const double vv = a.beta2 * a.v[o] + (1.0 - a.beta2) * g * g;
      a.m[o] = m;
      a.v[o] = vv;
      const double lr = k < 3 ? a.lr_trans : a.lr_rot;
      xi[k] = -lr * (m / bc1) / (sqrt(vv / bc2) + a.adam_eps);
    }
    double E[12];
    se3_exp_dev(xi, E);
    compose_dev(E, a.T_store + 12 * (size_t)v, a.T_store + 12 * (size_t)v);
  }
  // the last block to finish advances the step counter (every block has read it)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(a.done, 1u);
    if (prev == gridDim.x - 1) {
      if (!(flag & 1)) *a.step = s + 1;
      *a.done = 0u;
      __threadfence();
    }
  }
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
cudaError_t launch_pair_setup(const StepArgs& a, int mode, cudaStream_t s) {
  const int nb = (a.n_pairs + 127) / 128;
  k_pair_setup<<<nb > 0 ? nb : 1, 128, 0, s>>>(a, mode);
  return cudaGetLastError();
}

template <int MODE, int REC, int MAP, int GATHER>
static cudaError_t launch_edge_rpt(const EdgeArgs& a, int rpt, int block, int grid, cudaStream_t s) {
  switch (rpt) {
    case 2: k_edge<MODE, REC, MAP, GATHER, 2><<<grid, block, 0, s>>>(a); break;
    case 4: k_edge<MODE, REC, MAP, GATHER, 4><<<grid, block, 0, s>>>(a); break;
    case 8: k_edge<MODE, REC, MAP, GATHER, 8><<<grid, block, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int MODE, int REC, int MAP>
static cudaError_t launch_edge_g(const EdgeArgs& a, int gather, int rpt, int block, int grid,
                                 cudaStream_t s) {
  if (gather == GATHER_TEX) return launch_edge_rpt<MODE, REC, MAP, GATHER_TEX>(a, rpt, block, grid, s);
  return launch_edge_rpt<MODE, REC, MAP, GATHER_LDG>(a, rpt, block, grid, s);
}

template <int MODE>
static cudaError_t launch_edge_m(const EdgeArgs& a, int rec, int map, int gather, int rpt, int block,
                                 int grid, cudaStream_t s) {
  if (rec == 0 && map == 0) return launch_edge_g<MODE, 0, 0>(a, gather, rpt, block, grid, s);
  if (rec == 0 && map == 1) return launch_edge_g<MODE, 0, 1>(a, gather, rpt, block, grid, s);
  if (rec == 1 && map == 0) return launch_edge_g<MODE, 1, 0>(a, gather, rpt, block, grid, s);
  return launch_edge_g<MODE, 1, 1>(a, gather, rpt, block, grid, s);
}

// rec_dtype: 0 = f32 records, 1 = f16-depth records; map_dtype: 0 = f32, 1 = bf16.
cudaError_t launch_edge(const EdgeArgs& a, int mode, int rec_dtype, int map_dtype, int gather,
                        int rpt, int block, int grid, cudaStream_t s) {
  if (a.n_tiles == 0) return cudaSuccess;
  switch (mode) {
    case MODE_FWD: return launch_edge_m<MODE_FWD>(a, rec_dtype, map_dtype, gather, rpt, block, grid, s);
    case MODE_BWD: return launch_edge_m<MODE_BWD>(a, rec_dtype, map_dtype, gather, rpt, block, grid, s);
    default: return launch_edge_m<MODE_FUSED>(a, rec_dtype, map_dtype, gather, rpt, block, grid, s);
  }
}

cudaError_t launch_finalize(const StepArgs& a, int with_grad, cudaStream_t s) {
  const int nbp = (a.n_pairs + 127) / 128;
  k_fin_pairs<<<nbp > 0 ? nbp : 1, 128, 0, s>>>(a, with_grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nbv = (a.n_views + 255) / 256;
  k_fin_poses<<<nbv + a.n_scenes, 256, 0, s>>>(a, with_grad, nbv);
  return cudaGetLastError();
}

cudaError_t launch_retract(const StepArgs& a, cudaStream_t s) {
  const int nb = (a.n_views + 127) / 128;
  k_retract<<<nb, 128, 0, s>>>(a);
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
