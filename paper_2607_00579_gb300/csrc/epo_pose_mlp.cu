// The paper's pose parameterisation (Section 3, Pose Refinement, Eq. 3) on the device:
//
//     P_i^s = phi(P_i^0 + MLP(P_i^0)) + [0 | delta_i]
//
// with a six-layer MLP of hidden width 128 (ReLU after the first five layers, the first
// layer's output added to the third's), phi = Gram-Schmidt on the 6D representation (the first
// two columns of the 3x3 block), one MLP per scene and one translation offset delta_i per view,
// trained by AdamW with a linear warm-up and cosine decay of the learning rate (Implementation
// Details).  The parameterisation acts on the scene at unit scale: with s the RMS spread of the
// P^0 camera centres, the MLP sees the translations divided by s, and its translation output and
// delta are multiplied by s (the paper's inputs are normalised foundation-model outputs).  A step in this mode is: the fused pass and the pose kernel's gradient G_i (the
// left-perturbation gradient of the objective at P^s), then
//   k_mlp_backward  one block per view: G_i -> derivatives of the pose entries (FP64), through
//                   phi (FP64, one thread) and the MLP's layers (FP32, 128 threads);
//   k_mlp_update    one thread per parameter: the gradient summed over the scene's views in a
//                   fixed order, AdamW; the last block advances the step counter;
//   k_mlp_forward   one block per view: the next poses P^{s+1} (MLP in FP32, phi and the pose
//                   in FP64) and the activations the next backward needs.
// The MLP is tiny (69 k parameters, one 128-wide mat-vec per layer and view): these are latency
// kernels, not contractions worth the tensor cores.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "epo_internal.cuh"

namespace epo {

namespace {

constexpr int H = kMlpHid;
// offsets of W_l and b_l (l = 0..5) in a scene's parameter vector
__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? 12 : H; }
__host__ __device__ constexpr int mlp_out(int l) { return l == 5 ? 12 : H; }
__host__ __device__ constexpr int mlp_w(int l) {
  int o = 0;
  for (int k = 0; k < l; ++k) o += mlp_out(k) * mlp_in(k) + mlp_out(k);
  return o;
}
__host__ __device__ constexpr int mlp_b(int l) { return mlp_w(l) + mlp_out(l) * mlp_in(l); }
static_assert(mlp_w(6) == kMlpParams, "pose MLP layout");

// Every block starts the scene's weights (280 KB) towards L2 at once: the layers then wait on
// L2 rather than on one DRAM round trip after another (each step starts with them cold).
__device__ __forceinline__ void prefetch_weights(const float* th) {
  constexpr int kLines = (kMlpParams * 4 + 127) / 128;
  for (int q = threadIdx.x; q < kLines; q += blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(th) + (size_t)q * 128));
}

__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

}  // namespace

// ------------------------------------------------------------------------------------------
// forward: P^s from the current parameters
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kMlpHid) k_mlp_forward(StepArgs a, int change) {
  const int v = blockIdx.x, j = threadIdx.x;
  const int sc = a.views[v].scene;
  const float* th = a.mlp_theta + (size_t)sc * kMlpParams;
  prefetch_weights(th);
  __shared__ float s_x[12], s_a[H], s_a1[H], s_y[12];
  const double sc_s = a.mlp_scale[sc];
  if (j < 12) {
    const float xv = (float)(a.mlp_P0[12 * (size_t)v + j] / ((j & 3) == 3 ? sc_s : 1.0));
    s_x[j] = xv;
    a.mlp_x[12 * (size_t)v + j] = xv;
  }
  __syncthreads();
  float* zs = a.mlp_z + (size_t)v * 5 * H;
  float z = th[mlp_b(0) + j];
#pragma unroll
  for (int k = 0; k < 12; ++k) z = fmaf(th[mlp_w(0) + j * 12 + k], s_x[k], z);
  zs[j] = z;
  float h = fmaxf(z, 0.f);
  s_a1[j] = h;
  s_a[j] = h;
  __syncthreads();
  // hidden layers: each warp forms four outputs at a time, its lanes reading the four weight
  // rows coalesced (lane l takes columns l, l + 32, l + 64, l + 96) and summing by shuffles
  __shared__ float s_z[H];
  const int lane = j & 31, warp = j >> 5;
  for (int l = 1; l <= 4; ++l) {
    const float* W = th + mlp_w(l);
    const float a0 = s_a[lane], a1 = s_a[lane + 32], a2 = s_a[lane + 64], a3 = s_a[lane + 96];
    for (int o0 = warp * 4; o0 < H; o0 += 16) {
      float acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* Wr = W + (size_t)(o0 + u) * H;
        acc[u] = fmaf(Wr[lane], a0, fmaf(Wr[lane + 32], a1, fmaf(Wr[lane + 64], a2, Wr[lane + 96] * a3)));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], off);
      if (lane < 4) s_z[o0 + lane] = th[mlp_b(l) + o0 + lane] + (lane == 0 ? acc[0] : lane == 1 ? acc[1] : lane == 2 ? acc[2] : acc[3]);
    }
    __syncthreads();  // every output is formed; every thread has read the layer's input
    z = s_z[j];
    zs[l * H + j] = z;
    h = fmaxf(z, 0.f);
    if (l == 2) h += s_a1[j];  // the skip connection after the third layer
    s_a[j] = h;
    __syncthreads();
  }
  {  // output layer: warp w forms outputs w, w + 4, w + 8
    const float* W = th + mlp_w(5);
    const float a0 = s_a[lane], a1 = s_a[lane + 32], a2 = s_a[lane + 64], a3 = s_a[lane + 96];
    for (int o = warp; o < 12; o += 4) {
      const float* Wr = W + (size_t)o * H;
      float acc = fmaf(Wr[lane], a0, fmaf(Wr[lane + 32], a1, fmaf(Wr[lane + 64], a2, Wr[lane + 96] * a3)));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) s_y[o] = th[mlp_b(5) + o] + acc;
    }
  }
  __syncthreads();
  if (j != 0) return;
  // P' = P^0 + MLP(P^0); phi: Gram-Schmidt on its first two columns; the offset delta (FP64)
  double Pp[12];
  for (int k = 0; k < 12; ++k) {
    Pp[k] = a.mlp_P0[12 * (size_t)v + k] + ((k & 3) == 3 ? sc_s : 1.0) * (double)s_y[k];
    a.mlp_Pp[12 * (size_t)v + k] = Pp[k];
  }
  const double a1[3] = {Pp[0], Pp[4], Pp[8]}, a2[3] = {Pp[1], Pp[5], Pp[9]};
  const double n1 = sqrt(dot3(a1, a1));
  const double b1[3] = {a1[0] / n1, a1[1] / n1, a1[2] / n1};
  const double c = dot3(b1, a2);
  const double u2[3] = {a2[0] - c * b1[0], a2[1] - c * b1[1], a2[2] - c * b1[2]};
  const double n2 = sqrt(dot3(u2, u2));
  const double b2[3] = {u2[0] / n2, u2[1] / n2, u2[2] / n2};
  double b3[3];
  cross3(b1, b2, b3);
  double T[12];
  bool finite = true;
  for (int r = 0; r < 3; ++r) {
    T[4 * r] = b1[r];
    T[4 * r + 1] = b2[r];
    T[4 * r + 2] = b3[r];
    T[4 * r + 3] = Pp[4 * r + 3] + sc_s * (double)a.mlp_delta[3 * (size_t)v + r];
  }
  for (int k = 0; k < 12; ++k) finite = finite && isfinite(T[k]);
  if (!finite) {
    atomicOr(a.flag, 1);  // the poses stay; the host reports the step as refused
    return;
  }
  double* Ts = a.T_store + 12 * (size_t)v;
  if (change && a.schedule) {
    // the step's pose change (Section 3, Optimization Schedule), as the pose kernel forms it
    double tr = 0.0, dot = 0.0, nn = 0.0, no = 0.0;
    for (int r = 0; r < 3; ++r) {
      for (int cc = 0; cc < 3; ++cc) tr += T[4 * r + cc] * Ts[4 * r + cc];
      dot += T[4 * r + 3] * Ts[4 * r + 3];
      nn += T[4 * r + 3] * T[4 * r + 3];
      no += Ts[4 * r + 3] * Ts[4 * r + 3];
    }
    const double deg = 180.0 / 3.14159265358979323846;
    a.pose_dR[v] = deg * acos(fmin(1.0, fmax(-1.0, (tr - 1.0) * 0.5)));
    const double nm = sqrt(nn) * sqrt(no);
    a.pose_dt[v] = nm > 0.0 ? deg * acos(fmin(1.0, fmax(-1.0, dot / nm))) : 0.0;
  }
  for (int k = 0; k < 12; ++k) Ts[k] = T[k];
}

// ------------------------------------------------------------------------------------------
// backward: dL/dz of every layer and dL/ddelta of every view
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kMlpHid) k_mlp_backward(StepArgs a) {
  const int v = blockIdx.x, j = threadIdx.x;
  const int sc = a.views[v].scene;
  const float* th = a.mlp_theta + (size_t)sc * kMlpParams;
  prefetch_weights(th);
  __shared__ float s_dy[12], s_dz[H];
  if (j == 0) {
    // G = (g_v, g_w) at T = P^s: dL/dt = g_v, and (for the tangent dR = [w]x R that phi
    // produces) dL/dR = 1/2 [g_w + g_v x t]x R; then back through Gram-Schmidt (FP64)
    const double* G = a.grad + 6 * (size_t)v;
    const double* T = a.T_store + 12 * (size_t)v;
    const double* Pp = a.mlp_Pp + 12 * (size_t)v;
    const double gv[3] = {G[0], G[1], G[2]}, t[3] = {T[3], T[7], T[11]};
    double w[3];
    cross3(gv, t, w);
    w[0] += G[3];
    w[1] += G[4];
    w[2] += G[5];
    // E = 1/2 [w]x R, column c: 1/2 w x R[:, c]
    double E[3][3];
    for (int cc = 0; cc < 3; ++cc) {
      const double col[3] = {T[cc], T[4 + cc], T[8 + cc]};
      double e[3];
      cross3(w, col, e);
      for (int r = 0; r < 3; ++r) E[r][cc] = 0.5 * e[r];
    }
    const double a1[3] = {Pp[0], Pp[4], Pp[8]}, a2[3] = {Pp[1], Pp[5], Pp[9]};
    const double n1 = sqrt(dot3(a1, a1));
    const double b1[3] = {a1[0] / n1, a1[1] / n1, a1[2] / n1};
    const double c = dot3(b1, a2);
    const double u2[3] = {a2[0] - c * b1[0], a2[1] - c * b1[1], a2[2] - c * b1[2]};
    const double n2 = sqrt(dot3(u2, u2));
    const double b2[3] = {u2[0] / n2, u2[1] / n2, u2[2] / n2};
    double g1[3] = {E[0][0], E[1][0], E[2][0]}, g2[3] = {E[0][1], E[1][1], E[2][1]};
    const double g3[3] = {E[0][2], E[1][2], E[2][2]};
    double x[3];
    cross3(b2, g3, x);  // b3 = b1 x b2
    for (int r = 0; r < 3; ++r) g1[r] += x[r];
    cross3(g3, b1, x);
    for (int r = 0; r < 3; ++r) g2[r] += x[r];
    const double p2 = dot3(g2, b2);  // b2 = u2 / n2
    double gu2[3];
    for (int r = 0; r < 3; ++r) gu2[r] = (g2[r] - p2 * b2[r]) / n2;
    const double q = dot3(gu2, b1);  // u2 = a2 - (b1 . a2) b1
    double ga2[3];
    for (int r = 0; r < 3; ++r) {
      ga2[r] = gu2[r] - q * b1[r];
      g1[r] -= q * a2[r] + c * gu2[r];
    }
    const double p1 = dot3(g1, b1);  // b1 = a1 / n1
    for (int r = 0; r < 3; ++r) {
      s_dy[4 * r] = (float)((g1[r] - p1 * b1[r]) / n1);
      s_dy[4 * r + 1] = (float)ga2[r];
      s_dy[4 * r + 2] = 0.f;  // the third column does not reach phi
      s_dy[4 * r + 3] = (float)(a.mlp_scale[sc] * gv[r]);  // the translation output is scaled by s
      a.mlp_gdelta[3 * (size_t)v + r] = (float)(a.mlp_scale[sc] * gv[r]);
    }
  }
  __syncthreads();
  float* dz = a.mlp_dz + (size_t)v * kMlpDz;
  const float* zs = a.mlp_z + (size_t)v * 5 * H;
  if (j < 12) dz[5 * H + j] = s_dy[j];
  // dL/da_5 = W6^T dy, then through the ReLU of layer 5
  float da = 0.f;
  {
    const float* W = th + mlp_w(5);
#pragma unroll
    for (int o = 0; o < 12; ++o) da = fmaf(W[o * H + j], s_dy[o], da);
  }
  float d = zs[4 * H + j] > 0.f ? da : 0.f;
  dz[4 * H + j] = d;
  s_dz[j] = d;
  __syncthreads();
  float dskip = 0.f;
  for (int l = 4; l >= 1; --l) {
    const float* W = th + mlp_w(l);
    da = 0.f;
#pragma unroll 16
    for (int i = 0; i < H; ++i) da = fmaf(W[(size_t)i * H + j], s_dz[i], da);  // (W_l^T dz_l)_j
    if (l == 3) dskip = da;  // a_3 = relu(z_2) + a_1
    if (l == 1) da += dskip;
    d = zs[(l - 1) * H + j] > 0.f ? da : 0.f;
    dz[(l - 1) * H + j] = d;
    __syncthreads();  // every thread has read dz_l
    s_dz[j] = d;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// AdamW on theta and delta (a scene whose schedule has converged keeps them); the last block
// advances the step counter
// ------------------------------------------------------------------------------------------
constexpr int kMlpUpdThreads = 256;

__device__ __forceinline__ float adamw_delta(float p, float g, float& m, float& v, float b1, float b2, float c1, float c2,
                                             float lr, float wd, float eps) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  return p * (1.f - lr * wd) - lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void __launch_bounds__(kMlpUpdThreads) k_mlp_update(StepArgs a) {
  const int64_t step = *a.step;
  const bool refused = (*a.flag & 1) != 0;
  const int64_t g = (int64_t)blockIdx.x * kMlpUpdThreads + threadIdx.x;
  const int64_t n_theta = (int64_t)a.n_scenes * kMlpParams;
  // learning rate of the step: linear warm-up to mlp_lr, then cosine decay to 0
  float lr;
  if (step < a.mlp_warmup) {
    lr = a.mlp_lr * (float)(step + 1) / (float)a.mlp_warmup;
  } else {
    const int64_t span = max(a.mlp_steps - a.mlp_warmup, 1);
    const float t = (float)min(step - a.mlp_warmup + 1, span) / (float)span;
    lr = a.mlp_lr * 0.5f * (1.f + cospif(t));
  }
  const float fs = (float)(step + 1);
  const float c1 = -expm1f(fs * a.log_beta1), c2 = -expm1f(fs * a.log_beta2);
  const float b1 = (float)a.beta1, b2 = (float)a.beta2;
  const auto converged = [&](int sc) { return a.schedule && a.sched_state[2 * sc] == 3; };
  if (!refused && g < n_theta && !converged((int)(g / kMlpParams))) {
    const int sc = (int)(g / kMlpParams), k = (int)(g % kMlpParams);
    int l = 0;
    while (l < 5 && k >= mlp_w(l + 1)) ++l;
    const bool bias = k >= mlp_b(l);
    const int o = bias ? k - mlp_b(l) : (k - mlp_w(l)) / mlp_in(l);
    const int i = bias ? 0 : (k - mlp_w(l)) % mlp_in(l);
    const int dz_off = l == 5 ? 5 * H + o : l * H + o;
    float grad = 0.f;
#pragma unroll 8
    for (int v = a.scene_view_off[sc]; v < a.scene_view_off[sc + 1]; ++v) {
      const float d = a.mlp_dz[(size_t)v * kMlpDz + dz_off];
      float in = 1.f;
      if (!bias) {
        const float* zs = a.mlp_z + (size_t)v * 5 * H;
        if (l == 0) in = a.mlp_x[12 * (size_t)v + i];
        else if (l == 3) in = fmaxf(zs[2 * H + i], 0.f) + fmaxf(zs[i], 0.f);  // the skip
        else in = fmaxf(zs[(l - 1) * H + i], 0.f);
      }
      grad = fmaf(d, in, grad);
    }
    float* p = a.mlp_theta + g;
    *p = adamw_delta(*p, grad, a.mlp_m[g], a.mlp_v[g], b1, b2, c1, c2, lr, a.mlp_wd, a.mlp_eps);
  } else if (!refused && g >= n_theta && g < n_theta + 3 * (int64_t)a.n_views &&
             !converged(a.views[(g - n_theta) / 3].scene)) {
    const int64_t k = g - n_theta;
    a.mlp_delta[k] = adamw_delta(a.mlp_delta[k], a.mlp_gdelta[k], a.mlp_dm[k], a.mlp_dv[k], b1, b2, c1, c2, lr,
                                 a.mlp_wd_delta, a.mlp_eps);
  }
  // the last block to finish advances the step counter and the beta powers (read by the
  // focal Adam of refine scenes).  The decision rests on the flag every block read at its
  // start, and every block has used its step count before it reports, so the count needs no
  // fence
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(a.mlp_done, 1u);
    if (prev == gridDim.x - 1) {
      if (!refused) {
        *a.step = step + 1;
        a.bpow[0] *= a.beta1;
        a.bpow[1] *= a.beta2;
      }
      *a.mlp_done = 0u;
    }
  }
}

cudaError_t launch_mlp_forward(const StepArgs& a, int change, cudaStream_t s) {
  if (a.n_views <= 0) return cudaSuccess;
  k_mlp_forward<<<a.n_views, kMlpHid, 0, s>>>(a, change);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const StepArgs& a, cudaStream_t s) {
  if (a.n_views <= 0) return cudaSuccess;
  k_mlp_backward<<<a.n_views, kMlpHid, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mlp_update(const StepArgs& a, cudaStream_t s) {
  const int64_t n = (int64_t)a.n_scenes * kMlpParams + 3 * (int64_t)a.n_views;
  k_mlp_update<<<(unsigned)((n + kMlpUpdThreads - 1) / kMlpUpdThreads), kMlpUpdThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace epo
