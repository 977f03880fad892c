// Kernels of the edge-alignment library (sm_103a).
//
// Hot path (one optimisation step, Algorithm 2 with the pose-only reading):
//   k_pair_setup   a1: T_ji = T_j T_i^-1 in FP64 (kept for the exact path) and rounded to
//                  FP32 for the pixel math; lambda from the step; counters reset.
//   k_edge         a2-a7: persistent, work = (source view, tile of edge records).  Each
//                  thread lifts its records once (the split projection of Algorithm 2:
//                  lift once per image, project into every paired view), then for every
//                  outgoing pair i -> j: transform, project (Eq. 8), gather the 2x2
//                  footprint of DTF_j, bilinear value and slope, clamp + Huber (Eq. 7),
//                  the adjoint 6-vector, and a warp-shuffle + block reduction ending in
//                  one FP64 atomic per block per pair slot (the in-kernel per-pair
//                  reduction of the fused ProjectSampleHuber kernel, Appendix A.2).
//                  A sample whose FP32 position lies within its own rounding-error bound
//                  of a discontinuity of the objective (a bilinear cell line, the image
//                  border, the depth threshold, the clamp) is not accumulated but kept in
//                  a shared-memory buffer; the block re-evaluates those samples with every
//                  decision (validity, cell, clamp) taken in FP64, so the GPU objective
//                  takes exactly the branch an FP64 evaluation takes.
//   k_poses        a8 + a9: per-scene loss (Eq. 6, Algorithm 3's sum(rho)/sum(valid)),
//                  deterministic FP64 per-pose gather of the pair sums (the source side
//                  through -Ad(T_ji)^T), tangent-space Adam and T <- Exp(-Delta) T.
// Construction helpers: k_edt (exact distance transform field), k_round_bf16, k_map_check.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "epo_internal.cuh"

namespace epo {

// unit roundoff of binary32
constexpr float kU32 = 5.9604645e-08f;


// ------------------------------------------------------------------------------------
// a1: pair setup
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double lambda_at(const StepArgs& a, int64_t s) {
  double f = a.lambda_steps > 0 ? (double)s * a.inv_lambda_steps : 1.0;
  f = f > 1.0 ? 1.0 : f;
  return a.lambda0 + (a.lambda1 - a.lambda0) * f;
}

// 16 lanes per pair (two pairs per warp): lanes 0..8 form one entry of R_ji each, lanes
// 9..11 one entry of t_ji, lanes 12..15 the target's intrinsics and map; every lane's
// FP64 chain is a few operations long.
constexpr int kSetupLanes = 16;

__global__ void __launch_bounds__(128) k_pair_setup(StepArgs a, int mode) {
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
  const int i = pv ? a.pair_src[p] : 0;
  const int j = pv ? a.pair_dst[p] : 0;
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
  const bool bad = pv && e < 12 && !isfinite(val);
  if (__ballot_sync(0xffffffffu, bad)) {
    if (bad) atomicOr(a.flag, 1);  // a non-finite pose: the step must not update
  }
  if (!pv) return;
  PairParam* out = a.pp + p;
  float* of = reinterpret_cast<float*>(out);
  if (e < 12) {
    a.pp64[12 * (size_t)p + e] = val;  // R (9) then t (3), as in PairParam
    of[e] = vf;
  } else if (e == 12) {
    const ViewDev vj = a.views[j];
    out->fx = vj.fx; out->fy = vj.fy; out->cx = vj.cx; out->cy = vj.cy;
    out->fx2 = 2.f * vj.fx;
    out->fy2 = 2.f * vj.fy;
  } else if (e == 13) {
    const ViewDev vj = a.views[j];
    out->hw = 0.5f * (float)(vj.W - 1);
    out->hh = 0.5f * (float)(vj.H - 1);
    out->cu = 4.f * kU32 * (float)(vj.W + 1);
    out->cv = 4.f * kU32 * (float)(vj.H + 1);
  } else if (e == 14) {
    const ViewDev vj = a.views[j];
    out->W = vj.W; out->H = vj.H; out->pitch = vj.pitch;
    out->map_off = vj.map_off;
    out->tex = a.tex ? a.tex[j] : 0ull;
  } else {
    out->Et = 4.f * kU32 * (fabsf(t0) + fabsf(t1) + fabsf(t2));
  }
  if (e < kAcc) {
    const bool zero = (e < 2) ? (mode != MODE_BWD) : (mode != MODE_FWD);
    if (zero) a.pair_acc[(size_t)kAcc * p + e] = 0.0;
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

// rcp.approx: |rel. error| <= 2^-23 (PTX ISA), folded into the position error bound
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Butterfly reduce-scatter of 8 per-lane values over a warp: afterwards lane L holds the
// warp sum of value index slot(L) = (L&1)*4 + ((L>>1)&1)*2 + ((L>>2)&1).
__device__ __forceinline__ float warp_reduce_scatter8(float v[8], int lane) {
  const bool b0 = lane & 1, b1 = lane & 2, b2 = lane & 4;
  float k4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b0 ? v[4 + i] : v[i];
    const float send = b0 ? v[i] : v[4 + i];
    k4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
  float k2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b1 ? k4[2 + i] : k4[i];
    const float send = b1 ? k4[i] : k4[2 + i];
    k2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  const float keep = b2 ? k2[1] : k2[0];
  const float send = b2 ? k2[0] : k2[1];
  float s = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 8);
  s += __shfl_xor_sync(0xffffffffu, s, 16);
  return s;
}

__device__ __forceinline__ int scatter_slot(int lane) {
  return (lane & 1) * 4 + ((lane >> 1) & 1) * 2 + ((lane >> 2) & 1);
}

// A sample whose FP32 decisions its rounding-error bound cannot settle: its raw record and
// pair, kept in shared memory until the block re-evaluates it with FP64 decisions.
struct AmbEntry {
  float u, v, z;
  int p;
};
constexpr int kAmbCap = 512;  // entries per block; re-evaluated once more than half full

// The exact path: lift, transform and project in FP64, take the validity, cell and clamp
// decisions in FP64 (so the branch is the one an FP64 evaluation takes); the value and the
// slope terms are smooth given those decisions and are formed in FP32.  Adds straight to
// the pair's FP64 accumulators.
template <int MODE, int MAP>
__device__ void exact_eval(const EdgeArgs& a, const AmbEntry& en, double lam, float lamf) {
  const int p = en.p;
  const int i = a.pair_src[p];
  const PairParam& P = a.pp[p];
  const double* Ki = a.K64 + 6 * (size_t)i;
  const double* Kj = a.K64 + 6 * (size_t)a.pair_dst[p];
  // K64 holds fx, fy, cx, cy followed by 1/fx, 1/fy
  const double X[3] = {((double)en.u - Ki[2]) * Ki[4] * (double)en.z, ((double)en.v - Ki[3]) * Ki[5] * (double)en.z,
                       (double)en.z};
  const double* R = a.pp64 + 12 * (size_t)p;
  double Y[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) Y[r] = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + R[9 + r];
  if (!(Y[2] > (double)a.eps_z)) return;
  const double iz = __drcp_rn(Y[2]);
  const double up = Kj[0] * Y[0] * iz + Kj[2];
  const double vp = Kj[1] * Y[1] * iz + Kj[3];
  if (!(up >= 0.0 && up <= (double)(P.W - 1) && vp >= 0.0 && vp <= (double)(P.H - 1))) return;
  const int x0 = min((int)floor(up), P.W - 2);
  const int y0 = min((int)floor(vp), P.H - 2);
  const double ca = up - (double)x0, cb = vp - (double)y0;
  float f00, f01, f10, f11;
  taps<MAP, GATHER_LDG>(a.map, P.map_off, P.pitch, 0ull, x0, y0, f00, f01, f10, f11);
  const double d = (1.0 - ca) * (1.0 - cb) * f00 + ca * (1.0 - cb) * f01 + (1.0 - ca) * cb * f10 + ca * cb * f11;
  const bool pass = d <= lam;  // clamp decision in FP64
  const float delta = a.delta;
  const float df = (float)d, caf = (float)ca, cbf = (float)cb;
  const float dh = pass ? df : lamf;
  const float adh = fabsf(dh);
  const float rho = adh <= delta ? 0.5f * dh * dh : delta * (adh - 0.5f * delta);
  double* acc = a.pair_acc + (size_t)kAcc * p;
  if constexpr (MODE != MODE_BWD) {
    atomicAdd(acc + 0, (double)rho);
    atomicAdd(acc + 1, 1.0);
  }
  if constexpr (MODE != MODE_FWD) {
    const float drho = pass ? (fabsf(df) <= delta ? df : copysignf(delta, df)) : 0.f;
    if (drho != 0.f) {
      const float ddu = (1.f - cbf) * (f01 - f00) + cbf * (f11 - f10);
      const float ddv = (1.f - caf) * (f10 - f00) + caf * (f11 - f01);
      const float y0f = (float)Y[0], y1f = (float)Y[1], y2f = (float)Y[2];
      const float izf = (float)iz;
      const float gx = drho * ddu * P.fx * izf;
      const float gy = drho * ddv * P.fy * izf;
      const float gz = -(gx * y0f + gy * y1f) * izf;
      atomicAdd(acc + 2, (double)gx);
      atomicAdd(acc + 3, (double)gy);
      atomicAdd(acc + 4, (double)gz);
      atomicAdd(acc + 5, (double)(y1f * gz - y2f * gy));
      atomicAdd(acc + 6, (double)(y2f * gx - y0f * gz));
      atomicAdd(acc + 7, (double)(y0f * gy - y1f * gx));
    }
  }
}

template <int MODE, int REC, int MAP, int GATHER, int RPT>
__global__ void __launch_bounds__(512) k_edge(EdgeArgs a) {
  // dynamic shared memory: lifted records of the tile, their raw (u, v), then every warp's
  // partial sums per pair of the tile (summed in a fixed warp order at the flush, so the
  // result does not depend on warp timing)
  extern __shared__ float4 s_dyn[];
  float4* s_X = s_dyn;                                                    // [blockDim * RPT]
  float2* s_UV = reinterpret_cast<float2*>(s_dyn + blockDim.x * RPT);    // [blockDim * RPT]
  float* s_part = reinterpret_cast<float*>(s_UV + blockDim.x * RPT);     // [warps][max_pairs][8]
  __shared__ int s_tile, s_next;
  __shared__ int s_amb_n;
  __shared__ AmbEntry s_amb[kAmbCap];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  const float lam = (float)(*a.lambda);
  const float delta = a.delta;
  const float eps_z = a.eps_z;
  const double lam64 = *a.lambda;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(a.tile_counter, 1);
    s_amb_n = 0;
  }
  __syncthreads();
  while (s_tile < a.n_tiles) {
    const int t = s_tile;
    // claim the next tile now: the atomic's round trip overlaps this tile's work
    if (threadIdx.x == 0) s_next = atomicAdd(a.tile_counter, 1);
    const TileDev td = a.tiles[t];
    const ViewDev vi = a.views[td.view];
    // a2: stream the tile's records (coalesced 128-bit loads), lift once per record into
    // shared memory; each thread reads back only its own records
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int idx = threadIdx.x + r * blockDim.x;
      float u = 0.f, v = 0.f, z = 0.f;
      if (idx < td.n) load_record<REC>(a.rec, td.begin + idx, u, v, z);
      const float X0 = (u - vi.cx) / vi.fx * z, X1 = (v - vi.cy) / vi.fy * z;
      // rounding-error bound of Y = R X + t: 6u|X|_1 (rotation, lift and FMA roundings);
      // a record past the tile end gets w < 0 and is skipped
      const float XA = idx < td.n ? 6.f * kU32 * (fabsf(X0) + fabsf(X1) + fabsf(z)) : -1.f;
      s_X[idx] = make_float4(X0, X1, z, XA);
      s_UV[idx] = make_float2(u, v);
    }
    const int pb = a.src_pair_off[td.view];
    const int pe = a.src_pair_off[td.view + 1];
    for (int q = pb; q < pe; ++q) {
      const int p = a.src_pair_ids[q];
      if (!a.pair_active[p]) continue;  // uniform over the block
      const PairParam P = a.pp[p];
      const float Wm1 = (float)(P.W - 1), Hm1 = (float)(P.H - 1);
      float acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = 0.f;
      // the thread's RPT records, ILP of them in flight at a time: one reduction per pair
      // for all RPT samples, registers for only ILP
      constexpr int ILP = RPT < 2 ? RPT : 2;
#pragma unroll
      for (int g = 0; g < RPT; g += ILP) {
        // phase A: project every sample and take the decisions the FP32 bound allows
        float Y0[ILP], Y1[ILP], Y2[ILP], iz[ILP], up[ILP], vp[ILP], tu[ILP], tv[ILP];
        bool ok[ILP], amb[ILP];
        int x0[ILP], y0[ILP];
  #pragma unroll
        for (int r = 0; r < ILP; ++r) {
          const float4 X = s_X[threadIdx.x + (g + r) * blockDim.x];
          Y0[r] = fmaf(P.r[0], X.x, fmaf(P.r[1], X.y, fmaf(P.r[2], X.z, P.t[0])));
          Y1[r] = fmaf(P.r[3], X.x, fmaf(P.r[4], X.y, fmaf(P.r[5], X.z, P.t[1])));
          Y2[r] = fmaf(P.r[6], X.x, fmaf(P.r[7], X.y, fmaf(P.r[8], X.z, P.t[2])));
          const float E = X.w + P.Et;  // |Y_k - Y_k(exact)| <= E
          const bool front = (X.w >= 0.f) && (Y2[r] > eps_z - E);
          iz[r] = front ? rcp_approx(Y2[r]) : 0.f;
          const float xn = Y0[r] * iz[r], yn = Y1[r] * iz[r];
          up[r] = fmaf(P.fx, xn, P.cx);
          vp[r] = fmaf(P.fy, yn, P.cy);
          const float Eiz = E * iz[r];
          tu[r] = fmaf(P.fx2, fmaf(Eiz, fabsf(xn), Eiz), P.cu);  // bound on |u' - u'(exact)|
          tv[r] = fmaf(P.fy2, fmaf(Eiz, fabsf(yn), Eiz), P.cv);
          const bool cand = front && (fabsf(up[r] - P.hw) <= P.hw + tu[r]) && (fabsf(vp[r] - P.hh) <= P.hh + tv[r]);
          // within the bound of an integer coordinate (cell lines and the border are integers)
          // or of the depth threshold: the branch taken must come from the exact evaluation
          amb[r] = cand && (fabsf(up[r] - rintf(up[r])) <= tu[r] || fabsf(vp[r] - rintf(vp[r])) <= tv[r] ||
                            fabsf(Y2[r] - eps_z) <= E);
          ok[r] = cand && !amb[r];
          // cell of a valid sample: ok implies tu < u' < W-1-tu, so floor(u') is in [0, W-2];
          // the unsigned range check keeps every gather inside the map regardless
          x0[r] = __float2int_rd(up[r]);
          y0[r] = __float2int_rd(vp[r]);
          if (ok[r] && !((unsigned)x0[r] <= (unsigned)(P.W - 2) && (unsigned)y0[r] <= (unsigned)(P.H - 2))) {
            ok[r] = false;
            amb[r] = true;
          }
        }
        // phase B: all gathers in flight together
        float m00[ILP], m01[ILP], m10[ILP], m11[ILP];
  #pragma unroll
        for (int r = 0; r < ILP; ++r) {
          if (ok[r]) {
            taps<MAP, GATHER>(a.map, P.map_off, P.pitch, P.tex, x0[r], y0[r], m00[r], m01[r], m10[r], m11[r]);
          } else {
            m00[r] = m01[r] = m10[r] = m11[r] = 0.f;
          }
        }
        // phase C: bilinear value and slope, clamp, robust penalty, adjoint
  #pragma unroll
        for (int r = 0; r < ILP; ++r) {
          const float ca = up[r] - (float)x0[r];
          const float cb = vp[r] - (float)y0[r];
          const float top = fmaf(ca, m01[r] - m00[r], m00[r]);
          const float bot = fmaf(ca, m11[r] - m10[r], m10[r]);
          float d = fmaf(cb, bot - top, top);
          float ddu = fmaf(cb, (m11[r] - m10[r]) - (m01[r] - m00[r]), m01[r] - m00[r]);
          float ddv = bot - top;
          if (ok[r]) {
            // the clamp is a discontinuity of the slope term: same treatment
            const float td = fmaf(tu[r], fabsf(ddu), fmaf(tv[r], fabsf(ddv), 8.f * kU32 * (fabsf(d) + 1.f)));
            if (fabsf(d - lam) <= td) {
              ok[r] = false;
              amb[r] = true;
            }
          }
          // keep the ambiguous samples for the exact path (warp-aggregated append)
          const unsigned bal = __ballot_sync(0xffffffffu, amb[r]);
          if (bal) {
            const int leader = __ffs(bal) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&s_amb_n, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (amb[r]) {
              const int pos = base + __popc(bal & lanemask_lt);
              if (pos < kAmbCap) {
                const int li = threadIdx.x + (g + r) * blockDim.x;
                const float2 uv = s_UV[li];
                s_amb[pos] = AmbEntry{uv.x, uv.y, s_X[li].z, p};
              } else {
                // buffer full: evaluate this sample with FP32 decisions instead
                atomicAdd(a.q_overflow, 1u);
                ok[r] = (Y2[r] > eps_z) && (up[r] >= 0.f) && (up[r] <= Wm1) && (vp[r] >= 0.f) && (vp[r] <= Hm1);
                if (ok[r]) {
                  const int fx0 = min(max(x0[r], 0), P.W - 2), fy0 = min(max(y0[r], 0), P.H - 2);
                  const float fa = up[r] - (float)fx0, fb = vp[r] - (float)fy0;
                  float n00, n01, n10, n11;
                  taps<MAP, GATHER>(a.map, P.map_off, P.pitch, P.tex, fx0, fy0, n00, n01, n10, n11);
                  const float t2 = fmaf(fa, n01 - n00, n00);
                  const float b2 = fmaf(fa, n11 - n10, n10);
                  d = fmaf(fb, b2 - t2, t2);
                  ddu = fmaf(fb, (n11 - n10) - (n01 - n00), n01 - n00);
                  ddv = b2 - t2;
                }
              }
            }
          }
          if (ok[r]) {
            // a5: clamp + Huber
            const float dh = fminf(d, lam);
            const float adh = fabsf(dh);
            const float rho = adh <= delta ? 0.5f * dh * dh : delta * (adh - 0.5f * delta);
            if constexpr (MODE != MODE_BWD) {
              acc[0] += rho;
              acc[1] += 1.f;
            }
            if constexpr (MODE != MODE_FWD) {
              // a6: adjoint in camera-j coordinates
              const float drho = d <= lam ? (fabsf(d) <= delta ? d : copysignf(delta, d)) : 0.f;
              const float gx = drho * ddu * P.fx * iz[r];
              const float gy = drho * ddv * P.fy * iz[r];
              const float gz = -(gx * Y0[r] + gy * Y1[r]) * iz[r];
              acc[2] += gx;
              acc[3] += gy;
              acc[4] += gz;
              acc[5] += Y1[r] * gz - Y2[r] * gy;
              acc[6] += Y2[r] * gx - Y0[r] * gz;
              acc[7] += Y0[r] * gy - Y1[r] * gx;
            }
          }
        }
      }
      // a7: warp reduce-scatter; lanes 0..7 store the warp's 8 sums (no block barrier)
      const float sred = warp_reduce_scatter8(acc, lane);
      if (lane < 8) s_part[((size_t)warp * a.max_pairs + (q - pb)) * kAcc + scatter_slot(lane)] = sred;
    }
    __syncthreads();  // every warp has stored its partial sums for this tile
    // flush: warps summed in a fixed order, one FP64 atomic per used pair slot
    constexpr int S0 = MODE == MODE_BWD ? 2 : 0;
    constexpr int NS = MODE == MODE_FWD ? 2 : (MODE == MODE_BWD ? 6 : 8);
    const int nq = (pe - pb) * NS;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
      const int qq = k / NS, slot = S0 + k % NS;
      const int p = a.src_pair_ids[pb + qq];
      if (!a.pair_active[p]) continue;
      float s = 0.f;
      for (int w = 0; w < nwarp; ++w) s += s_part[((size_t)w * a.max_pairs + qq) * kAcc + slot];
      if (s != 0.f) atomicAdd(a.pair_acc + (size_t)kAcc * p + slot, (double)s);
    }
    if (threadIdx.x == 0) s_tile = s_next;
    __syncthreads();
    // exact path: when the buffer is more than half full, and once more before exiting
    const int n_amb = min(s_amb_n, kAmbCap);
    if (n_amb > (s_tile < a.n_tiles ? kAmbCap / 2 : 0)) {
      for (int k = threadIdx.x; k < n_amb; k += blockDim.x) exact_eval<MODE, MAP>(a, s_amb[k], lam64, lam);
      __syncthreads();
      if (threadIdx.x == 0) {
        atomicAdd(a.q_count, (unsigned)n_amb);
        s_amb_n = 0;
      }
      __syncthreads();
    }
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
constexpr int kPoseThreads = 128;
constexpr int kPosesPerBlock = kPoseThreads / 16;

// Taylor coefficients (in theta^2) of A = sin(t)/t, B = (1 - cos t)/t^2, C = (t - sin t)/t^3
__device__ constexpr double kExpA[5] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0};
__device__ constexpr double kExpB[5] = {0.5, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0};
__device__ constexpr double kExpC[5] = {1.0 / 6.0, -1.0 / 120.0, 1.0 / 5040.0, -1.0 / 362880.0, 1.0 / 39916800.0};

// Entry (r, c) of [w]x = [[0, -w2, w1], [w2, 0, -w0], [-w1, w0, 0]] with runtime r, c.
__device__ __forceinline__ double cross_entry(int r, int c, double w0, double w1, double w2) {
  if (r == c) return 0.0;
  const int k = 3 - r - c;
  const double wk = k == 0 ? w0 : (k == 1 ? w1 : w2);
  return ((c - r + 3) % 3) == 1 ? -wk : wk;
}

__global__ void __launch_bounds__(kPoseThreads) k_poses(StepArgs a, int with_grad, int n_pose_blocks) {
  __shared__ double s_sum[kPoseThreads];
  const int64_t step = *a.step;
  const int flag0 = *a.flag;
  if ((int)blockIdx.x < n_pose_blocks) {
    const int lane = threadIdx.x & 31;
    const int base = lane & 16;
    const int e = lane & 15;
    const int v = blockIdx.x * kPosesPerBlock + (threadIdx.x >> 4);
    const bool vv = v < a.n_views && with_grad > 0;
    double g[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (vv) {
      for (int k = a.pose_pair_off[v] + e; k < a.pose_pair_off[v + 1]; k += 16) {
        const int ref = a.pose_pair_ref[k];
        const int p = ref >> 1;
        if (!a.pair_active[p]) continue;
        const double* acc = a.pair_acc + (size_t)kAcc * p;
        const int i = a.pair_src[p];
        const double denom = a.norm_all ? (double)a.views[i].n_rec : acc[1];
        const int s = a.pair_scene[p];
        const int na = a.scene_active_pairs[s];
        if (!(denom > 0.0) || na <= 0) continue;
        const double c = (a.gscale ? a.gscale[s] : 1.0) * __drcp_rn((double)na * 0.5 * denom);
        const double ga0 = c * acc[2], ga1 = c * acc[3], ga2 = c * acc[4];
        const double gb0 = c * acc[5], gb1 = c * acc[6], gb2 = c * acc[7];
        if ((ref & 1) == 0) {  // target view j: the 6-vector as is
          g[0] += ga0; g[1] += ga1; g[2] += ga2;
          g[3] += gb0; g[4] += gb1; g[5] += gb2;
        } else {
          // source view i: -Ad(T_ji)^T (ga, gb) = (-R^T ga, R^T (t x ga) - R^T gb)
          const double* R = a.pp64 + 12 * (size_t)p;
          const double x0 = R[10] * ga2 - R[11] * ga1 - gb0;
          const double x1 = R[11] * ga0 - R[9] * ga2 - gb1;
          const double x2 = R[9] * ga1 - R[10] * ga0 - gb2;
#pragma unroll
          for (int k3 = 0; k3 < 3; ++k3) {
            g[k3] -= R[k3] * ga0 + R[3 + k3] * ga1 + R[6 + k3] * ga2;
            g[3 + k3] += R[k3] * x0 + R[3 + k3] * x1 + R[6 + k3] * x2;
          }
        }
      }
    }
    // fixed-order reduction over the 16 lanes of the pose
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 6; ++k) g[k] += __shfl_xor_sync(0xffffffffu, g[k], o);
    double G = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (e == k) G = g[k];
    if (vv && e < 6) {
      a.grad[6 * (size_t)v + e] = G;
      if (!isfinite(G)) atomicOr(a.flag, 1);
    }
    if (with_grad == 2) {
      const bool bad = vv && e < 6 && !isfinite(G);
      const unsigned badmask = __ballot_sync(0xffffffffu, bad);
      const bool skip = !vv || (flag0 & 1) || a.fixed[v] || ((badmask >> base) & 0xffffu);
      double xi = 0.0;
      if (!skip && e < 6) {
        const size_t o = 6 * (size_t)v + e;
        const double m = a.beta1 * a.m[o] + (1.0 - a.beta1) * G;
        const double vm = a.beta2 * a.v[o] + (1.0 - a.beta2) * G * G;
        a.m[o] = m;
        a.v[o] = vm;
        // the step ratio m^ / (sqrt(v^) + eps) needs only single precision
        const float mh = (float)m / (1.f - (float)a.bpow[0]);
        const float vh = (float)vm / (1.f - (float)a.bpow[1]);
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
      double A, B, C;
      if (th2 < 2.5e-3) {
        // theta < 0.05: Taylor polynomials in theta^2, truncation below 1e-20
        A = fma(th2, fma(th2, fma(th2, fma(th2, kExpA[4], kExpA[3]), kExpA[2]), kExpA[1]), kExpA[0]);
        B = fma(th2, fma(th2, fma(th2, fma(th2, kExpB[4], kExpB[3]), kExpB[2]), kExpB[1]), kExpB[0]);
        C = fma(th2, fma(th2, fma(th2, fma(th2, kExpC[4], kExpC[3]), kExpC[2]), kExpC[1]), kExpC[0]);
      } else {
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
        // translation: (I + B W + C W^2) upsilon, row r
        Erc = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double wk = k == 0 ? w0 : (k == 1 ? w1 : w2);
          const double I = r == k ? 1.0 : 0.0;
          Erc = fma(I + B * cross_entry(r, k, w0, w1, w2) + C * (wr * wk - I * th2), x[k], Erc);
        }
      }
      const int rb = base + (e & 12);
      const double E0 = __shfl_sync(0xffffffffu, Erc, rb);
      const double E1 = __shfl_sync(0xffffffffu, Erc, rb + 1);
      const double E2 = __shfl_sync(0xffffffffu, Erc, rb + 2);
      const double E3 = __shfl_sync(0xffffffffu, Erc, rb + 3);
      double Tnew = 0.0;
      if (!skip && e < 12) {
        const double* T = a.T_store + 12 * (size_t)v;
        Tnew = fma(E0, T[c], fma(E1, T[4 + c], fma(E2, T[8 + c], c == 3 ? E3 : 0.0)));
      }
      __syncwarp();  // every lane has read the old pose before any lane writes it
      if (!skip && e < 12) a.T_store[12 * (size_t)v + e] = Tnew;
    }
  } else {
    // per-scene loss (Eq. 6), fixed-order reduction
    const int s = blockIdx.x - n_pose_blocks;
    const int pb = a.scene_pair_off[s], pe = a.scene_pair_off[s + 1];
    double acc = 0.0;
    for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) {
      if (!a.pair_active[p]) continue;
      const double* pa = a.pair_acc + (size_t)kAcc * p;
      const double denom = a.norm_all ? (double)a.views[a.pair_src[p]].n_rec : pa[1];
      if (denom > 0.0) acc += pa[0] * __drcp_rn(denom);
    }
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
  if (with_grad == 2) {
    // the last block to finish advances the step counter and the beta powers
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned int prev = atomicAdd(a.done, 1u);
      if (prev == gridDim.x - 1) {
        __threadfence();
        const int flag_now = atomicOr(a.flag, 0);
        if (!(flag_now & 1)) {
          *a.step = step + 1;
          a.bpow[0] *= a.beta1;
          a.bpow[1] *= a.beta2;
        }
        *a.done = 0u;
        __threadfence();
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
cudaError_t launch_pair_setup(const StepArgs& a, int mode, cudaStream_t s) {
  const int nb = std::max((a.n_pairs * kSetupLanes + 127) / 128, 1);
  k_pair_setup<<<nb, 128, 0, s>>>(a, mode);
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

size_t edge_smem_bytes(int rpt, int block, int max_pairs) {
  // dynamic part: lifted records, raw (u, v), per-warp per-pair partial sums
  return sizeof(float4) * (size_t)rpt * block + sizeof(float2) * (size_t)rpt * block +
         sizeof(float) * kAcc * (size_t)max_pairs * (block / 32);
}

template <int MODE, int REC, int MAP, int GATHER, int R>
static cudaError_t launch_edge_one(const EdgeArgs& a, int block, int grid, cudaStream_t s) {
  const size_t smem = edge_smem_bytes(R, block, a.max_pairs);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_edge<MODE, REC, MAP, GATHER, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_edge<MODE, REC, MAP, GATHER, R><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, int REC, int MAP, int GATHER>
static cudaError_t launch_edge_rpt(const EdgeArgs& a, int rpt, int block, int grid, cudaStream_t s) {
  switch (rpt) {
    case 1: return launch_edge_one<MODE, REC, MAP, GATHER, 1>(a, block, grid, s);
    case 2: return launch_edge_one<MODE, REC, MAP, GATHER, 2>(a, block, grid, s);
    case 4: return launch_edge_one<MODE, REC, MAP, GATHER, 4>(a, block, grid, s);
    default: return cudaErrorInvalidValue;
  }
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

cudaError_t launch_poses(const StepArgs& a, int with_grad, cudaStream_t s) {
  const int nbp = (a.n_views + kPosesPerBlock - 1) / kPosesPerBlock;
  k_poses<<<nbp + a.n_scenes, kPoseThreads, 0, s>>>(a, with_grad, nbp);
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

template <int MODE, int REC, int MAP, int GATHER>
static const void* edge_ptr_rpt(int rpt) {
  switch (rpt) {
    case 1: return (const void*)k_edge<MODE, REC, MAP, GATHER, 1>;
    case 2: return (const void*)k_edge<MODE, REC, MAP, GATHER, 2>;
    case 4: return (const void*)k_edge<MODE, REC, MAP, GATHER, 4>;
    default: return nullptr;
  }
}

template <int MODE>
static const void* edge_ptr_m(int rec, int map, int gather, int rpt) {
  if (gather == GATHER_TEX) {
    if (rec == 0 && map == 0) return edge_ptr_rpt<MODE, 0, 0, GATHER_TEX>(rpt);
    if (rec == 0 && map == 1) return edge_ptr_rpt<MODE, 0, 1, GATHER_TEX>(rpt);
    if (rec == 1 && map == 0) return edge_ptr_rpt<MODE, 1, 0, GATHER_TEX>(rpt);
    return edge_ptr_rpt<MODE, 1, 1, GATHER_TEX>(rpt);
  }
  if (rec == 0 && map == 0) return edge_ptr_rpt<MODE, 0, 0, GATHER_LDG>(rpt);
  if (rec == 0 && map == 1) return edge_ptr_rpt<MODE, 0, 1, GATHER_LDG>(rpt);
  if (rec == 1 && map == 0) return edge_ptr_rpt<MODE, 1, 0, GATHER_LDG>(rpt);
  return edge_ptr_rpt<MODE, 1, 1, GATHER_LDG>(rpt);
}

const void* edge_kernel_ptr(int mode, int rec_dtype, int map_dtype, int gather, int rpt) {
  switch (mode) {
    case MODE_FWD: return edge_ptr_m<MODE_FWD>(rec_dtype, map_dtype, gather, rpt);
    case MODE_BWD: return edge_ptr_m<MODE_BWD>(rec_dtype, map_dtype, gather, rpt);
    default: return edge_ptr_m<MODE_FUSED>(rec_dtype, map_dtype, gather, rpt);
  }
}

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
