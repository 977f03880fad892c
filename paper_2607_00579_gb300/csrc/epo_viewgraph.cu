// Viewgraph estimation (Section 3, Viewgraph Estimation, Eq. 2; Algorithm 1 BuildViewgraph),
// run once before the optimisation.  For every ordered pair (i, j) of a scene, every source
// pixel of a regular grid of view i with a valid depth is projected into view j with Z_i
// (Eq. 2's pi), lifted there with Z_j at the nearest pixel and projected back into view i;
// the pair's fraction is the share of those pixels whose round trip stays in front of both
// cameras, inside view j, and returns within tau pixels.  A pair is kept when the fraction
// is at least min_frac in both directions (the paper's 12.5 % at tau = 3 px).
//
// One block per ordered pair, FP64 throughout (the construction is run once; ~100 FP64
// operations per grid pixel), with every product and sum rounded on its own in a fixed
// order, so the counts do not depend on how the compiler would fuse them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/epo.h"
#include "epo_internal.cuh"

namespace {

struct VgView {
  int32_t W, H;
  int64_t off;   // first depth element of the view
  double K[4];   // fx, fy, cx, cy
  double T[12];  // world -> camera [R|t], row-major
};

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// camera v pixel (x, y) at depth z -> camera w pixel; false when not in front of w.
__device__ bool reproject(const VgView& v, const VgView& w, double x, double y, double z, double& xo, double& yo) {
  const double Xc0 = mul(__ddiv_rn(sub(x, v.K[2]), v.K[0]), z);
  const double Xc1 = mul(__ddiv_rn(sub(y, v.K[3]), v.K[1]), z);
  const double q0 = sub(Xc0, v.T[3]), q1 = sub(Xc1, v.T[7]), q2 = sub(z, v.T[11]);
  double Xw[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) Xw[c] = add(add(mul(v.T[c], q0), mul(v.T[4 + c], q1)), mul(v.T[8 + c], q2));
  double Y[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    Y[r] = add(add(add(mul(w.T[4 * r], Xw[0]), mul(w.T[4 * r + 1], Xw[1])), mul(w.T[4 * r + 2], Xw[2])), w.T[4 * r + 3]);
  if (!(Y[2] > 0.0)) return false;
  xo = add(__ddiv_rn(mul(w.K[0], Y[0]), Y[2]), w.K[2]);
  yo = add(__ddiv_rn(mul(w.K[1], Y[1]), Y[2]), w.K[3]);
  return true;
}

constexpr int kVgThreads = 256;

__global__ void __launch_bounds__(kVgThreads) k_viewgraph(const VgView* views, const float* depth, int n, int stride,
                                                          double tau, double* frac) {
  const int i = blockIdx.x / n, j = blockIdx.x % n;
  if (i == j) {
    if (threadIdx.x == 0) frac[blockIdx.x] = 0.0;
    return;  // uniform over the block
  }
  const VgView vi = views[i], vj = views[j];
  const int gw = (vi.W + stride - 1) / stride, gh = (vi.H + stride - 1) / stride;
  unsigned valid = 0u, good = 0u;
  for (int g = threadIdx.x; g < gw * gh; g += blockDim.x) {
    const int x = (g % gw) * stride, y = (g / gw) * stride;
    const double z = (double)depth[vi.off + (int64_t)y * vi.W + x];
    if (!(z > 0.0) || !isfinite(z)) continue;
    ++valid;
    double xj, yj;
    if (!reproject(vi, vj, (double)x, (double)y, z, xj, yj)) continue;
    if (!(xj >= 0.0 && xj <= (double)(vj.W - 1) && yj >= 0.0 && yj <= (double)(vj.H - 1))) continue;
    const int xn = (int)floor(add(xj, 0.5)), yn = (int)floor(add(yj, 0.5));  // nearest pixel
    if (xn < 0 || xn >= vj.W || yn < 0 || yn >= vj.H) continue;
    const double zj = (double)depth[vj.off + (int64_t)yn * vj.W + xn];
    if (!(zj > 0.0) || !isfinite(zj)) continue;
    double xb, yb;
    if (!reproject(vj, vi, xj, yj, zj, xb, yb)) continue;
    const double dx = sub(xb, (double)x), dy = sub(yb, (double)y);
    if (__dsqrt_rn(add(mul(dx, dx), mul(dy, dy))) < tau) ++good;
  }
  // block sums in a fixed order
  __shared__ unsigned s_v[kVgThreads], s_g[kVgThreads];
  s_v[threadIdx.x] = valid;
  s_g[threadIdx.x] = good;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s_v[threadIdx.x] += s_v[threadIdx.x + w];
      s_g[threadIdx.x] += s_g[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) frac[blockIdx.x] = s_v[0] > 0 ? (double)s_g[0] / (double)s_v[0] : 0.0;
}

}  // namespace

extern "C" epo_status epo_build_viewgraph(int32_t n_views, const int32_t* W, const int32_t* H, const double* K,
                                          const double* T, const float* depth_dev, int32_t stride, double tau,
                                          double min_frac, double* frac, int32_t* pairs, int32_t* n_pairs,
                                          void* cuda_stream) {
  EPO_RANGE("epo_build_viewgraph");
  if (n_views < 1 || n_views > 46340 || !W || !H || !K || !T || !depth_dev || stride < 1 || !(tau > 0) ||
      !(min_frac >= 0) || !n_pairs)
    return EPO_ERR_INVALID_ARG;
  const int n = n_views;
  std::vector<VgView> hv(n);
  int64_t off = 0;
  for (int v = 0; v < n; ++v) {
    if (W[v] < 1 || H[v] < 1) return EPO_ERR_INVALID_ARG;
    hv[v].W = W[v];
    hv[v].H = H[v];
    hv[v].off = off;
    off += (int64_t)W[v] * H[v];
    for (int k = 0; k < 4; ++k) hv[v].K[k] = K[4 * v + k];
    for (int k = 0; k < 12; ++k) hv[v].T[k] = T[12 * v + k];
    if (!(hv[v].K[0] > 0) || !(hv[v].K[1] > 0)) return EPO_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  VgView* d_views = nullptr;
  double* d_frac = nullptr;
  std::vector<double> f((size_t)n * n);
  epo_status rc = EPO_OK;
  if (cudaMalloc(&d_views, sizeof(VgView) * n) != cudaSuccess ||
      cudaMalloc(&d_frac, sizeof(double) * (size_t)n * n) != cudaSuccess) {
    rc = EPO_ERR_OOM;
  } else if (cudaMemcpyAsync(d_views, hv.data(), sizeof(VgView) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    rc = EPO_ERR_CUDA;
  } else {
    k_viewgraph<<<n * n, kVgThreads, 0, st>>>(d_views, depth_dev, n, stride, tau, d_frac);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(f.data(), d_frac, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = EPO_ERR_CUDA;
  }
  if (d_views) cudaFree(d_views);
  if (d_frac) cudaFree(d_frac);
  if (rc != EPO_OK) return rc;
  // pairs kept in both directions, row-major
  int32_t m = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (i == j || std::min(f[(size_t)i * n + j], f[(size_t)j * n + i]) < min_frac) continue;
      if (pairs) {
        pairs[2 * m] = i;
        pairs[2 * m + 1] = j;
      }
      ++m;
    }
  *n_pairs = m;
  if (frac) std::copy(f.begin(), f.end(), frac);
  return EPO_OK;
}
