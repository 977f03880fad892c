// Loss and gradient without any device allocation.
//
// For callers that cannot call cudaMalloc: a host that owns every byte of device memory
// (a plugin inside someone else's engine, a fixed memory budget handed out up front), a
// real-time loop where an allocation may block or fail, or code that runs while the
// device allocator is off limits.  Such a caller passes its own device buffers for the
// inputs and the outputs; the intermediate sums live in one fixed-size array of this file,
// reserved on every GPU that loads the library for as long as the process runs.
//
// The computation is the one of epo_loss_and_grad_dev: per directed pair i -> j, every
// record of view i is lifted, moved by T_ji = T_j T_i^-1, projected into view j, the map
// is sampled bilinearly, clamped and Huber-penalised; per-pair means, the loss average and
// the left-perturbation gradient follow.  Here every projection and every branch decision
// is taken in FP64 (the value and slope terms in FP32), one block per (pair, tile of
// records), and the per-pose gradient is gathered by scanning all pairs: simple and exact,
// meant for problems up to the stated maximum size rather than for speed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/epo.h"

namespace {

constexpr int kNaMaxViews = EPO_NOALLOC_MAX_VIEWS;
constexpr int kNaMaxPairs = EPO_NOALLOC_MAX_PAIRS;
constexpr int kNaThreads = 256;

struct NaPair {
  double R[9];  // R_ji
  double t[3];  // t_ji
};

// Per pair: sum rho, n_valid, sum dRho/dY (3), sum Y x dRho/dY (3), and the number of usable
// records of the source view (the |E_i| of Eq. 7 under EPO_NORM_ALL)
constexpr int kNaAcc = 9;

struct NaScratch {
  double acc[kNaMaxPairs][kNaAcc];
  NaPair pair[kNaMaxPairs];
};
// 4096 pairs x (9 + 12) doubles = 688,128 bytes (672 KiB), the size the header states
static_assert(sizeof(NaScratch) == (size_t)kNaMaxPairs * (kNaAcc + 12) * sizeof(double), "scratch size");
static_assert(sizeof(NaScratch) == 688128, "scratch size stated in epo.h");

// The scratch: one file-scope device array shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

// Device address of g_noalloc_scratch per device, resolved once per device.
constexpr int kNaMaxDevices = 64;
NaScratch* g_scratch_ptr[kNaMaxDevices] = {};
std::mutex g_scratch_mutex;

__global__ void k_na_setup(epo_noalloc_problem pb, NaScratch* S) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pb.n_pairs) return;
  const int i = pb.pairs[2 * p], j = pb.pairs[2 * p + 1];
  const double* Ti = pb.T + 12 * (size_t)i;
  const double* Tj = pb.T + 12 * (size_t)j;
  NaPair& q = S->pair[p];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      q.R[3 * r + c] = Tj[4 * r] * Ti[4 * c] + Tj[4 * r + 1] * Ti[4 * c + 1] + Tj[4 * r + 2] * Ti[4 * c + 2];
  for (int r = 0; r < 3; ++r)
    q.t[r] = Tj[4 * r + 3] - (q.R[3 * r] * Ti[3] + q.R[3 * r + 1] * Ti[7] + q.R[3 * r + 2] * Ti[11]);
  for (int k = 0; k < kNaAcc; ++k) S->acc[p][k] = 0.0;  // the array keeps the previous call's sums
}

// blockIdx.y = pair, blockIdx.x = tile of kNaThreads records of the source view
__global__ void __launch_bounds__(kNaThreads) k_na_edge(epo_noalloc_problem pb, NaScratch* S) {
  __shared__ float s_red[kNaThreads / 32][kNaAcc];
  const int p = blockIdx.y;
  const int i = pb.pairs[2 * p], j = pb.pairs[2 * p + 1];
  const int64_t r0 = pb.rec_off[i], n = pb.rec_off[i + 1] - r0;
  const int64_t idx = (int64_t)blockIdx.x * kNaThreads + threadIdx.x;
  float acc[kNaAcc] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if ((int64_t)blockIdx.x * kNaThreads < n) {
    if (idx < n) {
      const float4 rec = reinterpret_cast<const float4*>(pb.records)[r0 + idx];
      const double* Ki = pb.K + 4 * (size_t)i;
      const double* Kj = pb.K + 4 * (size_t)j;
      const NaPair& q = S->pair[p];
      const double X[3] = {((double)rec.x - Ki[2]) / Ki[0] * (double)rec.z,
                           ((double)rec.y - Ki[3]) / Ki[1] * (double)rec.z, (double)rec.z};
      double Y[3];
      for (int r = 0; r < 3; ++r) Y[r] = q.R[3 * r] * X[0] + q.R[3 * r + 1] * X[1] + q.R[3 * r + 2] * X[2] + q.t[r];
      const int W = pb.W[j], H = pb.H[j];
      // records without a usable depth are not part of the problem (as at scene creation)
      const bool usable = rec.z > 0.f && isfinite(rec.x) && isfinite(rec.y) && isfinite(rec.z);
      acc[8] = usable ? 1.f : 0.f;
      if (usable && Y[2] > pb.eps_z) {
        const double up = Kj[0] * Y[0] / Y[2] + Kj[2];
        const double vp = Kj[1] * Y[1] / Y[2] + Kj[3];
        if (up >= 0.0 && up <= (double)(W - 1) && vp >= 0.0 && vp <= (double)(H - 1)) {
          const int x0 = min((int)floor(up), W - 2);
          const int y0 = min((int)floor(vp), H - 2);
          const double a = up - x0, b = vp - y0;
          const float* m = pb.maps + pb.map_off[j] + (int64_t)y0 * W + x0;
          const float m00 = m[0], m01 = m[1], m10 = m[W], m11 = m[W + 1];
          const double d = (1.0 - a) * (1.0 - b) * m00 + a * (1.0 - b) * m01 + (1.0 - a) * b * m10 + a * b * m11;
          const bool pass = d <= pb.lambda;
          const float lam = (float)pb.lambda, delta = (float)pb.huber_delta;
          const float df = (float)d, af = (float)a, bf = (float)b;
          const float dh = pass ? df : lam;
          const float adh = fabsf(dh);
          acc[0] = adh <= delta ? 0.5f * dh * dh : delta * (adh - 0.5f * delta);
          acc[1] = 1.f;
          const float drho = pass ? (fabsf(df) <= delta ? df : copysignf(delta, df)) : 0.f;
          const float ddu = (1.f - bf) * (m01 - m00) + bf * (m11 - m10);
          const float ddv = (1.f - af) * (m10 - m00) + af * (m11 - m01);
          const float y0f = (float)Y[0], y1f = (float)Y[1], y2f = (float)Y[2];
          const float iz = 1.f / y2f;
          const float gx = drho * ddu * (float)Kj[0] * iz;
          const float gy = drho * ddv * (float)Kj[1] * iz;
          const float gz = -(gx * y0f + gy * y1f) * iz;
          acc[2] = gx;
          acc[3] = gy;
          acc[4] = gz;
          acc[5] = y1f * gz - y2f * gy;
          acc[6] = y2f * gx - y0f * gz;
          acc[7] = y0f * gy - y1f * gx;
        }
      }
    }
  }
  // block reduction: warp shuffles, then a fixed-order sum over warps, one FP64 atomic per slot
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < kNaAcc; ++k) {
    float v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNaAcc) {
    float v = 0.f;
    for (int w = 0; w < kNaThreads / 32; ++w) v += s_red[w][threadIdx.x];
    if (v != 0.f) atomicAdd(&S->acc[p][threadIdx.x], (double)v);
  }
}

// One block: the loss (Eq. 6) and the per-pose gradient by a scan over all pairs.
__global__ void __launch_bounds__(kNaThreads) k_na_finish(epo_noalloc_problem pb, const NaScratch* S,
                                                          double* loss, double* grad) {
  __shared__ double s_sum[kNaThreads];
  const int P = pb.n_pairs;
  double part = 0.0;
  for (int p = threadIdx.x; p < P; p += kNaThreads) {
    const double denom = pb.norm_mode == EPO_NORM_ALL ? S->acc[p][8] : S->acc[p][1];
    if (denom > 0.0) part += S->acc[p][0] / denom;
  }
  s_sum[threadIdx.x] = part;
  __syncthreads();
  for (int w = kNaThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = P > 0 ? (2.0 / P) * s_sum[0] : 0.0;
  for (int e = threadIdx.x; e < 6 * pb.n_views; e += kNaThreads) {
    const int v = e / 6, k = e % 6;
    double g = 0.0;
    for (int p = 0; p < P; ++p) {
      const int i = pb.pairs[2 * p], j = pb.pairs[2 * p + 1];
      if (i != v && j != v) continue;
      const double* a = S->acc[p];
      const double denom = pb.norm_mode == EPO_NORM_ALL ? a[8] : a[1];
      if (!(denom > 0.0)) continue;
      const double c = 2.0 / P / denom;
      if (j == v) g += c * a[k < 3 ? 2 + k : 5 + (k - 3)];
      if (i == v) {
        // source view: -Ad(T_ji)^T (ga, gb) = (-R^T ga, R^T (t x ga) - R^T gb)
        const NaPair& q = S->pair[p];
        const double ga[3] = {c * a[2], c * a[3], c * a[4]};
        if (k < 3) {
          g -= q.R[k] * ga[0] + q.R[3 + k] * ga[1] + q.R[6 + k] * ga[2];
        } else {
          const int kk = k - 3;
          const double x[3] = {q.t[1] * ga[2] - q.t[2] * ga[1] - c * a[5], q.t[2] * ga[0] - q.t[0] * ga[2] - c * a[6],
                               q.t[0] * ga[1] - q.t[1] * ga[0] - c * a[7]};
          g += q.R[kk] * x[0] + q.R[3 + kk] * x[1] + q.R[6 + kk] * x[2];
        }
      }
    }
    grad[e] = g;
  }
}

}  // namespace

extern "C" epo_status epo_loss_and_grad_noalloc(const epo_noalloc_problem* pb, double* loss_dev,
                                                double* grad_dev, void* cuda_stream) {
  if (!pb || !loss_dev || !grad_dev) return EPO_ERR_INVALID_ARG;
  if (!pb->records || !pb->rec_off || !pb->maps || !pb->map_off || !pb->W || !pb->H || !pb->K || !pb->pairs ||
      !pb->T)
    return EPO_ERR_INVALID_ARG;
  if (pb->n_views < 1 || pb->n_pairs < 1 || pb->max_records_per_view < 0)
    return EPO_ERR_INVALID_ARG;
  // the kernels read records as 16-byte vectors and the other arrays at their natural width:
  // a misaligned pointer would fault on the device, so it is refused here
  if ((uintptr_t)pb->records % 16 != 0 || (uintptr_t)pb->rec_off % 8 != 0 || (uintptr_t)pb->maps % 4 != 0 ||
      (uintptr_t)pb->map_off % 8 != 0 || (uintptr_t)pb->W % 4 != 0 || (uintptr_t)pb->H % 4 != 0 ||
      (uintptr_t)pb->K % 8 != 0 || (uintptr_t)pb->pairs % 4 != 0 || (uintptr_t)pb->T % 8 != 0 ||
      (uintptr_t)loss_dev % 8 != 0 || (uintptr_t)grad_dev % 8 != 0)
    return EPO_ERR_INVALID_ARG;
  // one block per tile of kNaThreads records of a view: the tile count is the grid's x extent
  if ((pb->max_records_per_view + kNaThreads - 1) / kNaThreads > (int64_t)INT32_MAX) return EPO_ERR_TOO_LARGE;
  if (pb->n_views > kNaMaxViews || pb->n_pairs > kNaMaxPairs)
    return EPO_ERR_TOO_LARGE;
  if (!(pb->lambda > 0) || !(pb->huber_delta > 0) || !(pb->eps_z >= 0) ||
      (pb->norm_mode != EPO_NORM_VALID && pb->norm_mode != EPO_NORM_ALL))
    return EPO_ERR_INVALID_ARG;
  // the scratch array's device address, resolved once per device with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return EPO_ERR_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return EPO_ERR_INVALID_ARG;
  NaScratch* S = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return EPO_ERR_CUDA;
      g_scratch_ptr[dev] = reinterpret_cast<NaScratch*>(ptr);
    }
    S = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const epo_noalloc_problem prob = *pb;
  k_na_setup<<<(prob.n_pairs + 127) / 128, 128, 0, st>>>(prob, S);
  const int tiles = (int)((prob.max_records_per_view + kNaThreads - 1) / kNaThreads);
  if (tiles > 0) k_na_edge<<<dim3(tiles, prob.n_pairs), kNaThreads, 0, st>>>(prob, S);
  k_na_finish<<<1, kNaThreads, 0, st>>>(prob, S, loss_dev, grad_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return EPO_ERR_CUDA;
  return EPO_OK;
}
