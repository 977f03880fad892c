// The edge kernel (sm_103a), steps a2-a7 of one optimisation step.
//
//   k_edge   persistent, work = (source view, tile of edge records).  Each thread lifts its
//            records once (the split projection of Algorithm 2: lift once per image,
//            project into every paired view), then for every outgoing pair i -> j:
//            transform, project (Eq. 8), gather the 2x2 footprint of DTF_j, bilinear value
//            and slope, clamp + Huber (Eq. 7), the adjoint 6-vector, and a warp-shuffle +
//            block reduction ending in one FP64 atomic per block per pair slot (the
//            in-kernel per-pair reduction of the fused ProjectSampleHuber kernel,
//            Appendix A.2).  A sample whose FP32 position lies within its own rounding-error
//            bound of a discontinuity of the objective (a bilinear cell line, the image
//            border, the depth threshold, the clamp) is not accumulated but kept in a
//            shared-memory buffer; the block re-evaluates those samples with every decision
//            (validity, cell, clamp) taken in FP64, so the GPU objective takes exactly the
//            branch an FP64 evaluation takes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "epo_internal.cuh"

namespace epo {

// ------------------------------------------------------------------------------------
// a2-a7: the edge kernel
// ------------------------------------------------------------------------------------

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

// Texture gather of the 2x2 block centred on (x, y) (unnormalised coordinates, FP32 texels) for
// the lanes where p holds: tld4 of component 0, as tex2Dgather returns it, (x: (x0, y0+1), y: (x0+1,
// y0+1), z: (x0+1, y0), w: (x0, y0)).  Where p does not hold nothing is fetched and the outputs
// are unspecified (the caller does not use them), so no register is cleared in advance.
__device__ __forceinline__ void tex_gather_if(bool p, unsigned long long tex, float x, float y, float& m00, float& m01,
                                              float& m10, float& m11) {
  float gx, gy, gz, gw;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
      "@q tld4.r.2d.v4.f32.f32 {%0, %1, %2, %3}, [%5, {%6, %7}];\n\t}"
      : "=f"(gx), "=f"(gy), "=f"(gz), "=f"(gw)
      : "r"((int)p), "l"(tex), "f"(x), "f"(y));
  m00 = gw;
  m01 = gz;
  m10 = gx;
  m11 = gy;
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
  int p;  // the pair
  int q;  // its PairParam
};
constexpr int kAmbCap = 512;  // entries per block
// re-evaluated once more than kAmbRun are buffered: earlier than half full, so that less of the
// work is left for the end of the kernel (measured: 1.3 % faster on the 200-view walk than at
// 256, neutral on the 32-view ring; after every tile it is 8 % slower)
constexpr int kAmbRun = 64;

// The exact path.  The lift and the transform run in FP64; every decision (in front, in
// bounds, bilinear cell, clamp) is then the one the FP64 evaluation of the definition takes,
// with as little FP64 arithmetic as that needs (on this GPU FP64 runs at 1/64 of FP32):
//   * with s_u = fx Y1 + cx Y3 = Y3 u' (Y3 > 0), u' >= k  <=>  s_u - k Y3 >= 0, so the border
//     and the cell are signs of single FMAs: no FP64 division;
//   * the cell index starts from an FP32 estimate of u' (relative error < 3e-7, so within
//     one cell) and is corrected by those signs;
//   * the bilinear value and slopes are formed in FP32 from the cell fractions; the clamp
//     decision d <= lambda takes the FP32 value unless it lies within its error bound of
//     lambda, in which case the fractions and d are formed again in FP64.
// Adds straight to the pair's FP64 accumulators.
// rec: the sample's record (refine scenes reload its pixel and prior depth for an FP64 z).
template <int MODE, int REC, int MAP, int REF>
__device__ void exact_eval(const EdgeArgs& a, const AmbEntry& en, int64_t rec, double lam, float lamf) {
  const int p = en.p;
  const PairParam& P = a.pp[en.q];
  // the pair's projective form from the pair setup: (Y3 u', Y3 v', Y3) = z B (u, v, 1) + c
  const double* Q = a.pp64 + kPP64 * (size_t)p + 12;
  double z = (double)en.z, u = (double)en.u, v = (double)en.v;
  if constexpr (REF) {  // the record's pixel, and Z0 alpha + beta in FP64 as the definition has it
    float u0, v0, z0;
    load_record<REC>(a.rec, rec, u0, v0, z0);
    u = (double)u0;
    v = (double)v0;
    z = fma((double)z0, (double)a.alpha[rec], (double)a.beta[rec]);
  }
  const double Y3 = fma(z, fma(Q[6], u, fma(Q[7], v, Q[8])), Q[11]);
  if (!(Y3 > (double)a.eps_z)) return;
  const double su = fma(z, fma(Q[0], u, fma(Q[1], v, Q[2])), Q[9]);  // Y3 u'
  const double sv = fma(z, fma(Q[3], u, fma(Q[4], v, Q[5])), Q[10]);  // Y3 v'
  if (!(su >= 0.0 && fma(-(double)(P.W - 1), Y3, su) <= 0.0 && sv >= 0.0 && fma(-(double)(P.H - 1), Y3, sv) <= 0.0))
    return;
  const float rz = rcp_approx((float)Y3);
  int x0 = __float2int_rd((float)su * rz), y0 = __float2int_rd((float)sv * rz);
  if (fma(-(double)x0, Y3, su) < 0.0) --x0;
  else if (fma(-(double)(x0 + 1), Y3, su) >= 0.0) ++x0;
  if (fma(-(double)y0, Y3, sv) < 0.0) --y0;
  else if (fma(-(double)(y0 + 1), Y3, sv) >= 0.0) ++y0;
  x0 = min(x0, P.W - 2);  // the last cell is clamped (u' = W - 1 is in bounds)
  y0 = min(y0, P.H - 2);
  const double sa = fma(-(double)x0, Y3, su), sb = fma(-(double)y0, Y3, sv);  // Y3 (u' - x0), Y3 (v' - y0)
  float f00, f01, f10, f11;
#ifdef EPO_DEBUG_BOUNDS
  if (!debug_cell_ok(a, p, P.W, P.H, x0, y0)) return;
#endif
  taps<MAP, GATHER_LDG>(a.map, P.map_off, P.pitch, 0ull, x0, y0, f00, f01, f10, f11);
  const float caf = (float)sa * rz, cbf = (float)sb * rz;  // relative error < 3e-7
  const float top = fmaf(caf, f01 - f00, f00), bot = fmaf(caf, f11 - f10, f10);
  float df = fmaf(cbf, bot - top, top);
  const float ddu = fmaf(cbf, (f11 - f10) - (f01 - f00), f01 - f00);
  const float ddv = bot - top;
  bool pass;
  const float tcl = 2.f * (6e-7f * (fabsf(ddu) + fabsf(ddv)) + 8.f * kU32 * (fabsf(df) + 1.f));
  if (fabsf(df - lamf) > tcl) {
    pass = df <= lamf;
  } else {  // near the clamp: decide on the FP64 value
    const double iz = 1.0 / Y3;
    const double ca = sa * iz, cb = sb * iz;
    const double d = (1.0 - ca) * (1.0 - cb) * f00 + ca * (1.0 - cb) * f01 + (1.0 - ca) * cb * f10 + ca * cb * f11;
    pass = d <= lam;
    df = (float)d;
  }
  const float delta = a.delta;
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
      // the adjoint in the fast path's form, from the normalised coordinates (xn, yn) of u', v'
      const float xn = ((float)su * rz - P.cx) / P.fx, yn = ((float)sv * rz - P.cy) / P.fy;
      const float ga = drho * (P.fx * ddu), gb = drho * (P.fy * ddv), gc = -fmaf(ga, xn, gb * yn);
      const float gx = ga * rz, gy = gb * rz, gz = gc * rz;
      atomicAdd(acc + 2, (double)gx);
      atomicAdd(acc + 3, (double)gy);
      atomicAdd(acc + 4, (double)gz);
      atomicAdd(acc + 5, (double)fmaf(yn, gc, -gb));
      atomicAdd(acc + 6, (double)fmaf(-xn, gc, ga));
      atomicAdd(acc + 7, (double)fmaf(xn, gb, -(yn * ga)));
      if constexpr (REF) {
        // R (x~, y~, 1) = dY/dz; dRho/dz = g . dY/dz; the focal terms as in the fast path (the
        // entry holds the record's unit-depth ray (x~, y~))
        const float xtf = en.u, ytf = en.v, zf = (float)z;
        const float* r = P.r;
        const float dz = gx * fmaf(r[0], xtf, fmaf(r[1], ytf, r[2])) + gy * fmaf(r[3], xtf, fmaf(r[4], ytf, r[5])) +
                         gz * fmaf(r[6], xtf, fmaf(r[7], ytf, r[8]));
        const float gr2 = gx * r[2] + gy * r[5] + gz * r[8];
        atomicAdd(a.pair_facc + 2 * (size_t)p, (double)(zf * (gr2 - dz)));
        atomicAdd(a.pair_facc + 2 * (size_t)p + 1, (double)(-gc));  // gx Y0 + gy Y1
        if constexpr (MODE == MODE_FUSED) a.dzr[P.dbase + rec] = dz;  // the fast path wrote 0
      }
    }
  }
}

// Per-pair sums a warp reduces: the 8 of the pose gradient, plus the two focal sums of a
// refine scene.
template <int REF>
__host__ __device__ constexpr int edge_slots() { return REF ? kAcc + 2 : kAcc; }

template <int MODE, int REC, int MAP, int GATHER, int RPT, int REF>
__global__ void __launch_bounds__(512) k_edge(EdgeArgs a) {
  // dynamic shared memory: lifted records of the tile, their raw (u, v) (refine scenes:
  // the unit-depth rays (x~, y~) instead), then every warp's partial sums per pair of the
  // tile (summed in a fixed warp order at the flush, so the result does not depend on warp
  // timing)
  constexpr int NSLOT = edge_slots<REF>();
  extern __shared__ float4 s_dyn[];
  float4* s_X = s_dyn;                                                    // [blockDim * RPT]
  float2* s_UV = reinterpret_cast<float2*>(s_dyn + blockDim.x * RPT);    // [blockDim * RPT]
  float* s_part = reinterpret_cast<float*>(s_UV + blockDim.x * RPT);     // [warps][max_pairs][NSLOT]
  __shared__ int s_tile, s_next;
  __shared__ int s_amb_n;
  __shared__ AmbEntry s_amb[kAmbCap];
  __shared__ int64_t s_amb_rec[REF ? kAmbCap : 1];  // refine scenes: the entries' records
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  float lam = 0.f;     // the step's clamp, read once the pair setup has run
  double lam64 = 0.0;
  bool waited = false;
  const float delta = a.delta;
  const float eps_z = a.eps_z;
  if (threadIdx.x == 0) {
    s_tile = blockIdx.x;  // the first work item is the block's own; later ones are claimed
    s_amb_n = 0;
  }
  __syncthreads();
  while (s_tile < a.n_tiles) {
    const int t = s_tile;
    const TileDev td = a.tiles[t];
    const ViewDev vi = a.views[td.view];
    float vfx = vi.fx, vfy = vi.fy;
    if constexpr (REF) {  // f = f0 (1 + gamma) (Eq. 4): the refined FP64 intrinsics, rounded
      vfx = (float)a.K64[6 * (size_t)td.view];
      vfy = (float)a.K64[6 * (size_t)td.view + 1];
    }
    // a2: stream the tile's records (coalesced 128-bit loads), lift once per record into
    // shared memory; each thread reads back only its own records
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int idx = threadIdx.x + r * blockDim.x;
      float u = 0.f, v = 0.f, z = 0.f;
      if (idx < td.n) load_record<REC>(a.rec, td.begin + idx, u, v, z);
      if constexpr (REF) {  // z = Z0 alpha + beta (Eq. 5)
        if (idx < td.n) z = fmaf(z, a.alpha[td.begin + idx], a.beta[td.begin + idx]);
        const float xt = (u - vi.cx) / vfx, yt = (v - vi.cy) / vfy;
        const float X0 = xt * z, X1 = yt * z;
        // rounding-error bound of Y = R X + t: 8u|X|_1 (rotation, lift, the rounded refined
        // focal length and depth, FMA roundings)
        const float XA = idx < td.n ? 8.f * kU32 * (fabsf(X0) + fabsf(X1) + fabsf(z)) : -INFINITY;
        s_X[idx] = make_float4(X0, X1, z, XA);
        s_UV[idx] = make_float2(xt, yt);
      } else {
        const float X0 = (u - vi.cx) / vfx * z, X1 = (v - vi.cy) / vfy * z;
        // rounding-error bound of Y = R X + t: 6u|X|_1 (rotation, lift and FMA roundings);
        // a record past the tile end gets w = -inf: never in front, never ambiguous
        const float XA = idx < td.n ? 6.f * kU32 * (fabsf(X0) + fabsf(X1) + fabsf(z)) : -INFINITY;
        s_X[idx] = make_float4(X0, X1, z, XA);
        s_UV[idx] = make_float2(u, v);
      }
    }
    if (!waited) {
      // everything from here on reads what the step's pair setup writes (PairParams, the clamp,
      // the work counter, the zeroed pair sums): wait for it after the first item's records are
      // lifted, so that this block's start overlaps the setup, then let the pose kernel start
      griddep_wait();
      griddep_launch_dependents();
      lam64 = *a.lambda;
      lam = (float)lam64;
      waited = true;
    }
    // claim the next tile now: the atomic's round trip overlaps this tile's work
    if (threadIdx.x == 0) s_next = (int)gridDim.x + atomicAdd(a.tile_counter, 1);
    // the item's pair range, loaded where it is needed (holding the whole item in
    // registers across the pair loop costs a block per SM)
    const int pb = __ldg(&a.tiles[t].q0);
    const int pe = __ldg(&a.tiles[t].q1);
    for (int q = pb; q < pe; ++q) {
      // the pair's index and flag first (one 8-byte load), the rest once it is evaluated:
      // holding every field from before the branch costs registers
      const int2 pact = *reinterpret_cast<const int2*>(&a.pp[q].p);
      if (!pact.y) continue;  // uniform over the block
      const int p = pact.x;
      const PairParam P = a.pp[q];
      const float Wm1 = (float)(P.W - 1), Hm1 = (float)(P.H - 1);
      float acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = 0.f;
      float facc0 = 0.f, facc1 = 0.f;  // refine: source- and target-focal sums
      // the thread's RPT records, ILP of them in flight at a time: one reduction per pair
      // for all RPT samples, registers for only ILP
      constexpr int ILP = RPT < 2 ? RPT : 2;
#pragma unroll
      for (int g = 0; g < RPT; g += ILP) {
        // phase A: project every sample and take the decisions the FP32 bound allows
        // Y = R X + t enters below only through Y3 and the normalised coordinates
        // (xn, yn) = (Y1, Y2) / Y3
        float Y2[ILP], iz[ILP], xn[ILP], yn[ILP], up[ILP], vp[ILP], tu[ILP], tv[ILP];
        bool ok[ILP], amb[ILP];
        int x0[ILP], y0[ILP];
  #pragma unroll
        for (int r = 0; r < ILP; ++r) {
          const float4 X = s_X[threadIdx.x + (g + r) * blockDim.x];
          // the pose kernel's order (z last), so that both kernels compute the same Y
          const float Y0 = fmaf(P.r[2], X.z, fmaf(P.r[1], X.y, fmaf(P.r[0], X.x, P.t[0])));
          const float Y1 = fmaf(P.r[5], X.z, fmaf(P.r[4], X.y, fmaf(P.r[3], X.x, P.t[1])));
          Y2[r] = fmaf(P.r[8], X.z, fmaf(P.r[7], X.y, fmaf(P.r[6], X.x, P.t[2])));
          // |Y_k - Y_k(exact)| <= E; a record past the tile end has X.w = -inf, so that
          // it is never in front and never ambiguous
          const float E = X.w + P.Et;
          const bool front = Y2[r] > eps_z - E;
          iz[r] = front ? rcp_approx(Y2[r]) : 0.f;
          xn[r] = Y0 * iz[r];
          yn[r] = Y1 * iz[r];
          up[r] = fmaf(P.fx, xn[r], P.cx);
          vp[r] = fmaf(P.fy, yn[r], P.cy);
          const float Eiz = 2.f * E * iz[r];  // with the bound's 2x safety factor
          tu[r] = fmaf(P.fx, fmaf(Eiz, fabsf(xn[r]), Eiz), P.cu);  // bound on |u' - u'(exact)|
          tv[r] = fmaf(P.fy, fmaf(Eiz, fabsf(yn[r]), Eiz), P.cv);
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
#ifdef EPO_DEBUG_BOUNDS
  #pragma unroll
        for (int r = 0; r < ILP; ++r)
          if (ok[r] && !debug_cell_ok(a, p, P.W, P.H, x0[r], y0[r])) ok[r] = false;
#endif
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
                const float2 uv = s_UV[li];  // refine scenes: reloaded from the record
                s_amb[pos] = AmbEntry{uv.x, uv.y, s_X[li].z, p, q};
                if constexpr (REF) s_amb_rec[pos] = td.begin + li;
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
          float dzs = 0.f;  // refine, fused pass: the sample's d(rho)/dz (0 unless valid)
          if (ok[r]) {
            // a5: clamp + Huber.  With ch = min(|min(d, lambda)|, delta),
            // H(min(d, lambda)) = ch (|min(d, lambda)| - ch / 2), both branches of Eq. 7 in one
            // form; H'(d) = d clamped to [-delta, delta], passed where d <= lambda
            const float dh = fminf(d, lam);
            const float ch = fminf(fabsf(dh), delta);
            const float rho = ch * fmaf(-0.5f, ch, fabsf(dh));
            if constexpr (MODE != MODE_BWD) {
              acc[0] += rho;
              acc[1] += 1.f;
            }
            if constexpr (MODE != MODE_FWD) {
              // a6: adjoint in camera-j coordinates.  With (ga, gb) = H' (fx dd/du', fy dd/dv')
              // and gc = -(ga xn + gb yn), the gradient at Y is g = (ga, gb, gc) / Y3 and, as
              // Y = Y3 (xn, yn, 1), Y x g = (xn, yn, 1) x (ga, gb, gc): no 1/Y3 factor there
              const float drho = d <= lam ? fmaxf(fminf(d, delta), -delta) : 0.f;
              const float ga = drho * (P.fx * ddu);
              const float gb = drho * (P.fy * ddv);
              const float gc = -fmaf(ga, xn[r], gb * yn[r]);
              acc[2] = fmaf(ga, iz[r], acc[2]);
              acc[3] = fmaf(gb, iz[r], acc[3]);
              acc[4] = fmaf(gc, iz[r], acc[4]);
              acc[5] += fmaf(yn[r], gc, -gb);
              acc[6] += fmaf(-xn[r], gc, ga);
              acc[7] += fmaf(xn[r], gb, -(yn[r] * ga));
              if constexpr (REF) {
                const float gx = ga * iz[r], gy = gb * iz[r], gz = gc * iz[r];
                // dY/dz = R (x~, y~, 1): dRho/dz = g . dY/dz; the source focal term
                // -g . R (X0, X1, 0) = z (g . r_2 - dRho/dz) (times 1 + gamma_i) and the
                // target focal term gx Y0 + gy Y1 (times 1 + gamma_j)
                const int li = threadIdx.x + (g + r) * blockDim.x;
                const float2 xy = s_UV[li];
                const float zr = s_X[li].z;
                const float dz = gx * fmaf(P.r[0], xy.x, fmaf(P.r[1], xy.y, P.r[2])) +
                                 gy * fmaf(P.r[3], xy.x, fmaf(P.r[4], xy.y, P.r[5])) +
                                 gz * fmaf(P.r[6], xy.x, fmaf(P.r[7], xy.y, P.r[8]));
                const float gr2 = gx * P.r[2] + gy * P.r[5] + gz * P.r[8];
                facc0 += zr * (gr2 - dz);
                facc1 -= gc;  // gx Y0 + gy Y1 = ga xn + gb yn
                dzs = dz;
              }
            }
          }
          if constexpr (REF && MODE == MODE_FUSED) {
            // every record of the tile gets its value for this pair (an ambiguous sample's is
            // written again by the exact path after the block barrier); the depth kernel
            // weights them by the pairs' w / n once the pass has counted the valid samples
            const int li = threadIdx.x + (g + r) * blockDim.x;
            if (li < td.n) a.dzr[P.dbase + td.begin + li] = dzs;
          }
        }
      }
      // a7: warp reduce-scatter; lanes 0..7 store the warp's 8 sums (no block barrier)
      const float sred = warp_reduce_scatter8(acc, lane);
      if (lane < 8) s_part[((size_t)warp * a.max_pairs + (q - pb)) * NSLOT + scatter_slot(lane)] = sred;
      if constexpr (REF && MODE != MODE_FWD) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          facc0 += __shfl_xor_sync(0xffffffffu, facc0, o);
          facc1 += __shfl_xor_sync(0xffffffffu, facc1, o);
        }
        if (lane == 8 || lane == 9)
          s_part[((size_t)warp * a.max_pairs + (q - pb)) * NSLOT + lane] = lane == 8 ? facc0 : facc1;
      }
    }
    __syncthreads();  // every warp has stored its partial sums for this tile
    // the exact-path count is read between the two barriers: every append of this tile is done,
    // and no warp appends for the next tile before the second one
    const int n_amb = min(s_amb_n, kAmbCap);
    // flush: warps summed in a fixed order, one FP64 atomic per used pair slot
    constexpr int S0 = MODE == MODE_BWD ? 2 : 0;
    constexpr int NS = MODE == MODE_FWD ? 2 : NSLOT - S0;
    const int nq = (pe - pb) * NS;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
      const int qq = k / NS, slot = S0 + k % NS;
      const int2 pact = *reinterpret_cast<const int2*>(&a.pp[pb + qq].p);
      if (!pact.y) continue;
      const int p = pact.x;
      float s = 0.f;
      for (int w = 0; w < nwarp; ++w) s += s_part[((size_t)w * a.max_pairs + qq) * NSLOT + slot];
      if (s != 0.f) {
        if (slot < kAcc) atomicAdd(a.pair_acc + (size_t)kAcc * p + slot, (double)s);
        else atomicAdd(a.pair_facc + 2 * (size_t)p + (slot - kAcc), (double)s);
      }
    }
    if (threadIdx.x == 0) s_tile = s_next;
    __syncthreads();
    // exact path: when the buffer holds more than kAmbRun entries, and once more before exiting
    if (n_amb > (s_tile < a.n_tiles ? kAmbRun : 0)) {
      for (int k = threadIdx.x; k < n_amb; k += blockDim.x) exact_eval<MODE, REC, MAP, REF>(a, s_amb[k], REF ? s_amb_rec[k] : (int64_t)0, lam64, lam);
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
// a2-a7 for pose-only scenes: the same work items, lift, per-pair reduction, flush and exact
// path as k_edge, with a leaner per-sample screen.
//
// Decisions are taken in FP32 wherever a rigorous bound on the sample's rounding error shows
// them to be those of the exact evaluation.  With u = 2^-24:
//
// Error of Y.  Every component of the FP32 Y = R X + t is within
//   E = X.w + Et,  X.w = u (5 |X0| + 4 |X1| + 2 z + 2 eps_z),  Et = 4u |t|_1
// of the exact one (each with a 1e-5 relative margin for the second-order terms).  The records
// are lifted once at scene creation in FP64 and rounded (u |X|); the rotation's entries are
// rounded (u); the FMA chain, which takes z (the largest component) last, rounds z once, X1
// twice, X0 and t three times; the translation itself is rounded once.  The 2u eps_z covers the
// depth test's subtraction against the threshold given in double precision.
//
// Error of u' (and v').  With iz = rcp.approx(Y3) (relative error 2u), xn = Y1 iz and
// u' = fma(fx, xn, cx) in the FP32 intrinsics of view j,
//   |u' - u'*| <= E |1/Y3| (fx + |u'* - cx|) + u (|u'| + 4 |u' - cx| + |cx|):
// the first term is fx |Y1/Y3 - Y1*/Y3*|, at most fx E (1 + |xn*|) / |Y3| for components
// within E, the second the roundings of the product, the reciprocal, the FMA and the
// intrinsics.  For a sample whose FP32 position lies within one pixel of the image and whose
// bound is at most 1/4, |u'* - cx| <= max(cx + 1, W - cx) + 1/4, so one bound
//   t = E |1/Y3| Kb + cb,  Kb = max over the axes of f + max(c + 1, W - c) + 1/4,
//                          cb = u max over the axes of W + 4 max(c + 1, W - c) + |c|
// (1e-5 margin, which also covers the FP32 evaluation of t) holds for both coordinates.
//
// With x0 = floor(u'), a = u' - x0 (exact in FP32), the sample lies within t of a cell line
// or the border iff min(a (1 - a), b (1 - b)) <= t (1 - t) (t < 1/2 here), one test for both
// axes and every integer.  Validity in FP32 is then exact: a sample that is in front by more
// than E, in a cell 0 <= x0 <= W - 2, 0 <= y0 <= H - 2 (unsigned compares of the non-negative
// float bits) and farther than t from every integer has the cell, the border decision and the
// depth decision of the exact evaluation.  Samples within t of an integer that land within
// one pixel of the image, within E of the depth threshold, or whose t exceeds 1/4 go to the
// exact path; samples within the clamp's bound of lambda too, as in k_edge.  The 1/4 cap makes
// the samples left out safe: with t <= 1/4, E |1/Y3| Kb <= 1/4, and a sample that FP32 puts a
// distance s >= 1 outside the image (it is dropped) has an error of at most (1 + s) / 4 plus
// the roundings, less than s however large its |xn|, so it is outside in the exact evaluation
// too.
// Records past the tile's end carry NaN coordinates, so that every comparison on them is false.
// ------------------------------------------------------------------------------------
// Registers per thread: 56 keeps nine 128-thread blocks per SM (measured on the 16-scene batch:
// 48 and 64 were no faster at four records per thread).  A variant build may set another cap.
#ifdef EPO_POSE_MAXNREG
#define EPO_POSE_BOUNDS __maxnreg__(EPO_POSE_MAXNREG)
#else
#define EPO_POSE_BOUNDS __maxnreg__(56)
#endif
// The exact path for one buffered sample of a pose-only scene, reloading its record (a call,
// not inlined, so that its FP64 registers do not count against the kernel's).
template <int MODE, int REC, int MAP>
__device__ __noinline__ void exact_eval_rec(const EdgeArgs& a, int64_t rec, int p, int q, double lam, float lamf) {
  float u, v, z;
  load_record<REC>(a.rec, rec, u, v, z);
  exact_eval<MODE, REC, MAP, 0>(a, AmbEntry{u, v, z, p, q}, (int64_t)0, lam, lamf);
}

// An ambiguous sample of the pose kernel: its record and PairParam; the exact path reloads the
// record (rare), so that the kernel keeps no copy of the raw pixels in shared memory.
struct AmbRef {
  int64_t rec;
  int32_t q;
  int32_t pad_;
};
// A small buffer, re-evaluated once more than a third full: the shared memory a block leaves
// unused goes to the L1 cache that serves the map gathers.
#ifndef EPO_POSE_AMBCAP
#define EPO_POSE_AMBCAP 256
#endif
constexpr int kAmbCapPose = EPO_POSE_AMBCAP;
constexpr int kAmbRunPose = kAmbCapPose * 3 / 8;

template <int MODE, int REC, int MAP, int GATHER, int RPT>
__global__ void EPO_POSE_BOUNDS k_edge_pose(EdgeArgs a) {
  extern __shared__ float4 s_dyn[];
  float4* s_X = s_dyn;                                                    // [blockDim * RPT]
  float* s_part = reinterpret_cast<float*>(s_X + blockDim.x * RPT);      // [warps][max_pairs][kAcc]
  __shared__ int s_tile, s_next;
  __shared__ int s_amb_n;
  __shared__ AmbRef s_amb[kAmbCapPose];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  float lam = 0.f;
  double lam64 = 0.0;
  bool waited = false;
  const float delta = a.delta;
  const float eps_z = a.eps_z;
  if (threadIdx.x == 0) {
    s_tile = blockIdx.x;
    s_amb_n = 0;
  }
  __syncthreads();
  while (s_tile < a.n_tiles) {
    const int t = s_tile;
    const TileDev td = a.tiles[t];
    // a2: the tile's records, lifted at scene creation with their share of the rounding bound,
    // staged in shared memory (coalesced 128-bit loads)
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int idx = threadIdx.x + r * blockDim.x;
      if (idx < td.n) {
        s_X[idx] = __ldg(a.lift + td.begin + idx);
      } else {
        s_X[idx] = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000), 0.f);
      }
    }
    if (!waited) {
      griddep_wait();
      griddep_launch_dependents();
      lam64 = *a.lambda;
      lam = (float)lam64;
      waited = true;
    }
    if (threadIdx.x == 0) s_next = (int)gridDim.x + atomicAdd(a.tile_counter, 1);
    const int pb = __ldg(&a.tiles[t].q0);
    const int pe = __ldg(&a.tiles[t].q1);
    // the clamp's own rounding: 8u (|d| + 1), with |d| <= lambda + 1 wherever it matters
    const float c_lam = 8.f * kU32 * (fabsf(lam) + 2.f);
    for (int q = pb; q < pe; ++q) {
      const int2 pact = *reinterpret_cast<const int2*>(&a.pp[q].p);
      if (!pact.y) continue;  // uniform over the block
      const PairParam& P = a.pp[q];
      const float r0 = P.r[0], r1 = P.r[1], r2 = P.r[2], r3 = P.r[3], r4 = P.r[4], r5 = P.r[5], r6 = P.r[6],
                  r7 = P.r[7], r8 = P.r[8], t0 = P.t[0], t1 = P.t[1], t2 = P.t[2];
      const float fx = P.fx, fy = P.fy, cx = P.cx, cy = P.cy, Et = P.Et, Kb = P.Kb, cb = P.cb;
      const unsigned Wm2 = __float_as_uint(P.Wm2), Hm2 = __float_as_uint(P.Hm2);
      float acc[kAcc];
#pragma unroll
      for (int k = 0; k < kAcc; ++k) acc[k] = 0.f;
      constexpr int ILP = RPT < 2 ? RPT : 2;  // two samples in flight (four spill)
#pragma unroll
      for (int g = 0; g < RPT; g += ILP) {
        float fu1[ILP], fv1[ILP], ca[ILP], cbf[ILP], xn[ILP], yn[ILP], iz[ILP], tb[ILP], dze[ILP];
        bool ok[ILP], fetch[ILP], amb[ILP];
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
          const float4 X = s_X[threadIdx.x + (g + r) * blockDim.x];
          // z, the largest component of X, enters last (rounded once), X0 and t first
          const float Y0 = fmaf(r2, X.z, fmaf(r1, X.y, fmaf(r0, X.x, t0)));
          const float Y1 = fmaf(r5, X.z, fmaf(r4, X.y, fmaf(r3, X.x, t1)));
          const float Y2 = fmaf(r8, X.z, fmaf(r7, X.y, fmaf(r6, X.x, t2)));
          iz[r] = rcp_approx(Y2);
          xn[r] = Y0 * iz[r];
          yn[r] = Y1 * iz[r];
          const float up = fmaf(fx, xn[r], cx), vp = fmaf(fy, yn[r], cy);
          const float fu = floorf(up), fv = floorf(vp);
          ca[r] = up - fu;
          cbf[r] = vp - fv;
          fu1[r] = fu + 1.f;
          fv1[r] = fv + 1.f;
          const float E = X.w + Et;
          const float dz = Y2 - eps_z;
          tb[r] = fmaf(E * iz[r], Kb, cb);
          const float T = fmaf(-tb[r], tb[r], tb[r]);
          const float nm = fminf(fmaf(-ca[r], ca[r], ca[r]), fmaf(-cbf[r], cbf[r], cbf[r]));
          const bool near = nm <= T;
          const bool in_cell = __float_as_uint(fu) <= Wm2 && __float_as_uint(fv) <= Hm2;
          // beyond t = 1/4 (or NaN) the bound is not relied on: the exact path decides
          const bool guard = !(tb[r] <= 0.25f);
          // the footprint is fetched wherever FP32 says the sample is valid; it is accumulated
          // where no decision is in doubt (and, should the exact path's buffer be full, where
          // FP32 says valid)
          fetch[r] = dz > 0.f && in_cell;
          ok[r] = fetch[r] && dz > E && !near && !guard;
          // candidates for the exact path; whether they are near the image is checked on the
          // rare path (they are about 0.5 % of the samples)
          dze[r] = fabsf(dz) - E;  // <= 0: within E of the depth threshold
          amb[r] = guard || near || dze[r] <= 0.f;
        }
        // all gathers in flight together.  A sample that is not fetched gets unspecified tap
        // values, which it never accumulates
#ifdef EPO_DEBUG_BOUNDS
#pragma unroll
        for (int r = 0; r < ILP; ++r)
          if (fetch[r] && !debug_cell_ok(a, P.p, P.W, P.H, (int)fu1[r] - 1, (int)fv1[r] - 1)) fetch[r] = ok[r] = false;
#endif
        float m00[ILP], m01[ILP], m10[ILP], m11[ILP];
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
          if (MAP == 0 && (GATHER == GATHER_TEX || (GATHER == GATHER_MIX && r == 0))) {
            tex_gather_if(fetch[r], P.tex, fu1[r], fv1[r], m00[r], m01[r], m10[r], m11[r]);
          } else {
            m00[r] = m01[r] = m10[r] = m11[r] = 0.f;
            if (fetch[r]) {
              if (GATHER == GATHER_TEX || (GATHER == GATHER_MIX && r == 0)) {
                const ushort4 gq = tex2Dgather<ushort4>((cudaTextureObject_t)P.tex, fu1[r], fv1[r], 0);
                m00[r] = bf16_bits_to_float(gq.w); m01[r] = bf16_bits_to_float(gq.z);
                m10[r] = bf16_bits_to_float(gq.x); m11[r] = bf16_bits_to_float(gq.y);
              } else {
                taps<MAP, GATHER_LDG>(a.map, P.map_off, P.pitch, 0ull, (int)fu1[r] - 1, (int)fv1[r] - 1, m00[r],
                                      m01[r], m10[r], m11[r]);
              }
            }
          }
        }
        float dv_[ILP], du_[ILP], dd_[ILP];
        bool qa[ILP], use[ILP];
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
          const float d01 = m01[r] - m00[r], d11 = m11[r] - m10[r];
          const float top = fmaf(ca[r], d01, m00[r]);
          const float bot = fmaf(ca[r], d11, m10[r]);
          dv_[r] = bot - top;
          dd_[r] = fmaf(cbf[r], dv_[r], top);
          du_[r] = fmaf(cbf[r], d11 - d01, d01);
          // the clamp is a discontinuity of the slope term: within its bound of lambda the
          // sample goes to the exact path as well
          const bool at_clamp = fabsf(dd_[r] - lam) <=
                                fmaf(tb[r], fabsf(du_[r]) + fabsf(dv_[r]), fmaf(8.f * kU32, fabsf(dd_[r]), c_lam));
          qa[r] = amb[r] || (ok[r] && at_clamp);
          use[r] = ok[r] && !at_clamp;
        }
        bool any_qa = false;
#pragma unroll
        for (int r = 0; r < ILP; ++r) any_qa = any_qa || qa[r];
        if (__any_sync(0xffffffffu, any_qa)) {
          // rare: of the candidates, keep those in front within E of the threshold or beyond,
          // and within one pixel of the image (floor(u') + 1 in [0, W]) or beyond the bound, for
          // the exact path (warp-aggregated append)
#pragma unroll
          for (int r = 0; r < ILP; ++r) {
            if (qa[r] && !ok[r]) {
              const bool front = dze[r] <= 0.f || (dze[r] > 0.f && iz[r] > 0.f);  // dz > -E
              const bool in_ext = __float_as_uint(fu1[r]) <= __float_as_uint(P.Wf) &&
                                  __float_as_uint(fv1[r]) <= __float_as_uint(P.Hf);
              qa[r] = front && (!(tb[r] <= 0.25f) || in_ext);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, qa[r]);
            const int leader = bal ? __ffs(bal) - 1 : 0;
            int base = 0;
            if (bal && lane == leader) base = atomicAdd(&s_amb_n, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (qa[r]) {
              const int pos = base + __popc(bal & lanemask_lt);
              const int li = threadIdx.x + (g + r) * blockDim.x;
              if (pos < kAmbCapPose) {
                s_amb[pos] = AmbRef{td.begin + li, q, 0};
              } else {
                // buffer full (a tile with hundreds of samples on cell lines): the sample keeps
                // its FP32 decisions, counted in q_overflow
                atomicAdd(a.q_overflow, 1u);
                use[r] = fetch[r];
              }
            }
          }
        }
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
          if (use[r]) {
            const float d = dd_[r], ddu = du_[r], ddv = dv_[r];
            // a5: clamp + Huber, both branches of Eq. 7 in one form: with ch = min(|min(d,
            // lambda)|, delta), H(min(d, lambda)) = ch (|min(d, lambda)| - ch / 2); H'(d) = d
            // clamped to [-delta, delta] where d <= lambda
            const float dh = fminf(d, lam);
            const float ch = fminf(fabsf(dh), delta);
            if (MODE != MODE_BWD) {
              acc[0] = fmaf(ch, fmaf(-0.5f, ch, fabsf(dh)), acc[0]);
              acc[1] += 1.f;
            }
            if (MODE != MODE_FWD) {
              // a6: adjoint in camera-j coordinates; with (ga, gb) = H' (fx dd/du', fy dd/dv')
              // and gc = -(ga xn + gb yn), dRho/dY = (ga, gb, gc) / Y3 and Y x dRho/dY =
              // (xn, yn, 1) x (ga, gb, gc)
              const float drho = d <= lam ? copysignf(ch, d) : 0.f;
              const float ga = drho * (fx * ddu);
              const float gb = drho * (fy * ddv);
              const float gc = -fmaf(ga, xn[r], gb * yn[r]);
              acc[2] = fmaf(ga, iz[r], acc[2]);
              acc[3] = fmaf(gb, iz[r], acc[3]);
              acc[4] = fmaf(gc, iz[r], acc[4]);
              acc[5] = fmaf(yn[r], gc, acc[5]) - gb;
              acc[6] = fmaf(-xn[r], gc, acc[6]) + ga;
              acc[7] = fmaf(-yn[r], ga, fmaf(xn[r], gb, acc[7]));
            }
          }
        }
      }
      // a7: warp reduce-scatter; lanes 0..7 store the warp's 8 sums (no block barrier)
      const float sred = warp_reduce_scatter8(acc, lane);
      if (lane < 8) s_part[((size_t)warp * a.max_pairs + (q - pb)) * kAcc + scatter_slot(lane)] = sred;
    }
    __syncthreads();  // every warp has stored its partial sums and appended its exact-path samples
    // the exact-path counts are read between the two barriers: every append of this tile is
    // done, and no warp appends for the next tile before the second one
    const int n_amb = min(s_amb_n, kAmbCapPose);
    constexpr int S0 = MODE == MODE_BWD ? 2 : 0;
    constexpr int NS = MODE == MODE_FWD ? 2 : kAcc - S0;
    const int nq = (pe - pb) * NS;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
      const int qq = k / NS, slot = S0 + k % NS;
      const int2 pact = *reinterpret_cast<const int2*>(&a.pp[pb + qq].p);
      if (!pact.y) continue;
      float sum = 0.f;
      for (int w = 0; w < nwarp; ++w) sum += s_part[((size_t)w * a.max_pairs + qq) * kAcc + slot];
      if (sum != 0.f) atomicAdd(a.pair_acc + (size_t)kAcc * pact.x + slot, (double)sum);
    }
    if (threadIdx.x == 0) s_tile = s_next;
    __syncthreads();
    if (n_amb > (s_tile < a.n_tiles ? kAmbRunPose : 0)) {
      for (int k = threadIdx.x; k < n_amb; k += blockDim.x) {
        const AmbRef ar = s_amb[k];
        exact_eval_rec<MODE, REC, MAP>(a, ar.rec, a.pp[ar.q].p, ar.q, lam64, lam);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        atomicAdd(a.q_count, (unsigned)n_amb);
        s_amb_n = 0;
      }
      __syncthreads();
    }
  }
}

size_t edge_smem_bytes(int rpt, int block, int max_pairs, int refine) {
  // dynamic part: lifted records, (refine scenes) their rays, per-warp per-pair partial sums
  return sizeof(float4) * (size_t)rpt * block +
         (refine ? sizeof(float2) * (size_t)rpt * block : 0) +
         sizeof(float) * (refine ? edge_slots<1>() : edge_slots<0>()) * (size_t)max_pairs * (block / 32);
}

// The kernel of a schedule: pose-only scenes run k_edge_pose, refine scenes k_edge.
template <int MODE, int REC, int MAP, int GATHER, int R, int REF>
static auto edge_kernel_of() {
  if constexpr (REF) return k_edge<MODE, REC, MAP, GATHER, R, 1>;
  else return k_edge_pose<MODE, REC, MAP, GATHER, R>;
}

template <int MODE, int REC, int MAP, int GATHER, int R, int REF>
static cudaError_t launch_edge_one(const EdgeArgs& a, int block, int grid, cudaStream_t s) {
  const size_t smem = edge_smem_bytes(R, block, a.max_pairs, REF);
  const auto k = edge_kernel_of<MODE, REC, MAP, GATHER, R, REF>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(k, dim3(grid), dim3(block), smem, s, a);
}

// Refine scenes run two records per thread only (one set of instantiations).
template <int MODE, int REC, int MAP, int GATHER, int REF>
static cudaError_t launch_edge_rpt(const EdgeArgs& a, int rpt, int block, int grid, cudaStream_t s) {
  if constexpr (REF) {
    if (rpt != 2) return cudaErrorInvalidValue;
    return launch_edge_one<MODE, REC, MAP, GATHER, 2, 1>(a, block, grid, s);
  } else {
    switch (rpt) {
      case 1: return launch_edge_one<MODE, REC, MAP, GATHER, 1, 0>(a, block, grid, s);
      case 2: return launch_edge_one<MODE, REC, MAP, GATHER, 2, 0>(a, block, grid, s);
      case 4: return launch_edge_one<MODE, REC, MAP, GATHER, 4, 0>(a, block, grid, s);
      case 8: return launch_edge_one<MODE, REC, MAP, GATHER, 8, 0>(a, block, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

template <int MODE, int REC, int MAP, int REF>
static cudaError_t launch_edge_g(const EdgeArgs& a, int gather, int rpt, int block, int grid,
                                 cudaStream_t s) {
  if (gather == GATHER_TEX) return launch_edge_rpt<MODE, REC, MAP, GATHER_TEX, REF>(a, rpt, block, grid, s);
  if constexpr (!REF) {
    if (gather == GATHER_MIX) return launch_edge_rpt<MODE, REC, MAP, GATHER_MIX, REF>(a, rpt, block, grid, s);
  }
  if (gather != GATHER_LDG) return cudaErrorInvalidValue;
  return launch_edge_rpt<MODE, REC, MAP, GATHER_LDG, REF>(a, rpt, block, grid, s);
}

template <int MODE, int REF>
static cudaError_t launch_edge_m(const EdgeArgs& a, int rec, int map, int gather, int rpt, int block,
                                 int grid, cudaStream_t s) {
  if (rec == 0 && map == 0) return launch_edge_g<MODE, 0, 0, REF>(a, gather, rpt, block, grid, s);
  if (rec == 0 && map == 1) return launch_edge_g<MODE, 0, 1, REF>(a, gather, rpt, block, grid, s);
  if (rec == 1 && map == 0) return launch_edge_g<MODE, 1, 0, REF>(a, gather, rpt, block, grid, s);
  return launch_edge_g<MODE, 1, 1, REF>(a, gather, rpt, block, grid, s);
}

template <int MODE>
static cudaError_t launch_edge_r(const EdgeArgs& a, int refine, int rec, int map, int gather, int rpt, int block,
                                 int grid, cudaStream_t s) {
  if (refine) return launch_edge_m<MODE, 1>(a, rec, map, gather, rpt, block, grid, s);
  return launch_edge_m<MODE, 0>(a, rec, map, gather, rpt, block, grid, s);
}

// rec_dtype: 0 = f32 records, 1 = f16-depth records; map_dtype: 0 = f32, 1 = bf16.
cudaError_t launch_edge(const EdgeArgs& a, int mode, int refine, int rec_dtype, int map_dtype, int gather,
                        int rpt, int block, int grid, cudaStream_t s) {
  if (a.n_tiles == 0) return cudaSuccess;
  switch (mode) {
    case MODE_FWD: return launch_edge_r<MODE_FWD>(a, refine, rec_dtype, map_dtype, gather, rpt, block, grid, s);
    case MODE_BWD: return launch_edge_r<MODE_BWD>(a, refine, rec_dtype, map_dtype, gather, rpt, block, grid, s);
    default: return launch_edge_r<MODE_FUSED>(a, refine, rec_dtype, map_dtype, gather, rpt, block, grid, s);
  }
}

template <int MODE, int REC, int MAP, int GATHER, int REF>
static const void* edge_ptr_rpt(int rpt) {
  if constexpr (REF) {
    return rpt == 2 ? (const void*)k_edge<MODE, REC, MAP, GATHER, 2, 1> : nullptr;
  } else {
    switch (rpt) {
      case 1: return (const void*)edge_kernel_of<MODE, REC, MAP, GATHER, 1, 0>();
      case 2: return (const void*)edge_kernel_of<MODE, REC, MAP, GATHER, 2, 0>();
      case 4: return (const void*)edge_kernel_of<MODE, REC, MAP, GATHER, 4, 0>();
      case 8: return (const void*)edge_kernel_of<MODE, REC, MAP, GATHER, 8, 0>();
      default: return nullptr;
    }
  }
}

template <int MODE, int REF>
static const void* edge_ptr_m(int rec, int map, int gather, int rpt) {
  if constexpr (!REF) {
    if (gather == GATHER_MIX) {
      if (rec == 0 && map == 0) return edge_ptr_rpt<MODE, 0, 0, GATHER_MIX, REF>(rpt);
      if (rec == 0 && map == 1) return edge_ptr_rpt<MODE, 0, 1, GATHER_MIX, REF>(rpt);
      if (rec == 1 && map == 0) return edge_ptr_rpt<MODE, 1, 0, GATHER_MIX, REF>(rpt);
      return edge_ptr_rpt<MODE, 1, 1, GATHER_MIX, REF>(rpt);
    }
  }
  if (gather == GATHER_MIX) return nullptr;
  if (gather == GATHER_TEX) {
    if (rec == 0 && map == 0) return edge_ptr_rpt<MODE, 0, 0, GATHER_TEX, REF>(rpt);
    if (rec == 0 && map == 1) return edge_ptr_rpt<MODE, 0, 1, GATHER_TEX, REF>(rpt);
    if (rec == 1 && map == 0) return edge_ptr_rpt<MODE, 1, 0, GATHER_TEX, REF>(rpt);
    return edge_ptr_rpt<MODE, 1, 1, GATHER_TEX, REF>(rpt);
  }
  if (rec == 0 && map == 0) return edge_ptr_rpt<MODE, 0, 0, GATHER_LDG, REF>(rpt);
  if (rec == 0 && map == 1) return edge_ptr_rpt<MODE, 0, 1, GATHER_LDG, REF>(rpt);
  if (rec == 1 && map == 0) return edge_ptr_rpt<MODE, 1, 0, GATHER_LDG, REF>(rpt);
  return edge_ptr_rpt<MODE, 1, 1, GATHER_LDG, REF>(rpt);
}

const void* edge_kernel_ptr(int mode, int refine, int rec_dtype, int map_dtype, int gather, int rpt) {
  if (refine) {
    switch (mode) {
      case MODE_FWD: return edge_ptr_m<MODE_FWD, 1>(rec_dtype, map_dtype, gather, rpt);
      case MODE_BWD: return edge_ptr_m<MODE_BWD, 1>(rec_dtype, map_dtype, gather, rpt);
      default: return edge_ptr_m<MODE_FUSED, 1>(rec_dtype, map_dtype, gather, rpt);
    }
  }
  switch (mode) {
    case MODE_FWD: return edge_ptr_m<MODE_FWD, 0>(rec_dtype, map_dtype, gather, rpt);
    case MODE_BWD: return edge_ptr_m<MODE_BWD, 0>(rec_dtype, map_dtype, gather, rpt);
    default: return edge_ptr_m<MODE_FUSED, 0>(rec_dtype, map_dtype, gather, rpt);
  }
}

}  // namespace epo
