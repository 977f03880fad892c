/*
 * Seeded synthetic scene rasteriser (input generation only).
 *
 * Renders, for one pinhole camera, the z-depth of a world made of textured
 * rectangles ("planes") and thin 3D line segments, and marks the edge pixels
 * the way an edge detector on such a rendering would find them: the visible
 * pixels of every segment plus the foreground side of every depth
 * discontinuity.  This stands in for the foundation-model depth Z_i and the
 * Canny edge map E_i of Section 3 (Eq. 1); it holds none of the alignment
 * objective's arithmetic (no distance transform, no robust penalty, no
 * relative-pose projection of edge records).
 *
 * Conventions (shared with the callers through plain arrays only):
 *   camera pose T = [R | t] maps world -> camera, row-major 3x4 (12 doubles);
 *   camera frame x right, y down, z forward; pixel (x, y) has its centre at
 *   integer coordinates; K = (fx, fy, cx, cy).
 *   plane record (15 doubles): centre c[3], unit axis e1[3], unit axis e2[3],
 *   unit normal n[3], half sizes h1, h2, and one unused slot.
 *   segment record (6 doubles): endpoints A[3], B[3].
 *
 * Output per view: depth (float, 0 where no surface is hit) and an edge mask
 * (uint8, 1 = edge pixel).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PLANE_STRIDE 15
#define SEG_STRIDE 6

static void cam_ray(const double* T, const double* K, double x, double y,
                    double C[3], double d[3]) {
  /* camera centre C = -R^T t; ray direction d = R^T K^-1 [x, y, 1] (z-component 1 in camera) */
  const double* R0 = T;      /* row 0: R00 R01 R02 t0 */
  const double* R1 = T + 4;
  const double* R2 = T + 8;
  double t0 = R0[3], t1 = R1[3], t2 = R2[3];
  for (int k = 0; k < 3; ++k) C[k] = -(R0[k] * t0 + R1[k] * t1 + R2[k] * t2);
  double qx = (x - K[2]) / K[0];
  double qy = (y - K[3]) / K[1];
  for (int k = 0; k < 3; ++k) d[k] = R0[k] * qx + R1[k] * qy + R2[k];
}

static void world_to_cam(const double* T, const double P[3], double Y[3]) {
  for (int r = 0; r < 3; ++r)
    Y[r] = T[4 * r] * P[0] + T[4 * r + 1] * P[1] + T[4 * r + 2] * P[2] + T[4 * r + 3];
}

/* Nearest rectangle hit along the ray (depth = ray parameter, since the
 * camera-frame direction has unit z).  Returns 0 when nothing is hit. */
static double cast_planes(const double* planes, int n_planes, const double C[3],
                          const double d[3]) {
  double best = 0.0;
  for (int p = 0; p < n_planes; ++p) {
    const double* q = planes + (size_t)p * PLANE_STRIDE;
    const double* c = q;
    const double* e1 = q + 3;
    const double* e2 = q + 6;
    const double* n = q + 9;
    double nd = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
    if (fabs(nd) < 1e-12) continue;
    double s = (n[0] * (c[0] - C[0]) + n[1] * (c[1] - C[1]) + n[2] * (c[2] - C[2])) / nd;
    if (s <= 1e-3) continue;
    if (best > 0.0 && s >= best) continue;
    double w[3] = {C[0] + s * d[0] - c[0], C[1] + s * d[1] - c[1], C[2] + s * d[2] - c[2]};
    double a1 = w[0] * e1[0] + w[1] * e1[1] + w[2] * e1[2];
    double a2 = w[0] * e2[0] + w[1] * e2[1] + w[2] * e2[2];
    if (fabs(a1) <= q[12] && fabs(a2) <= q[13]) best = s;
  }
  return best;
}

/*
 * Render one view.  depth: H*W floats; edge: H*W bytes; both overwritten.
 * jump_rel: relative depth jump (e.g. 0.05) that marks a discontinuity.
 * Returns the number of edge pixels.
 */
int64_t synth_render_view(const double* planes, int n_planes, const double* segs, int n_segs,
                          int W, int H, const double* K, const double* T, double jump_rel,
                          float* depth, uint8_t* edge) {
  double C[3], d[3];
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      cam_ray(T, K, (double)x, (double)y, C, d);
      depth[(size_t)y * W + x] = (float)cast_planes(planes, n_planes, C, d);
    }
  }
  memset(edge, 0, (size_t)W * H);
  /* discontinuities first (they are judged on the surface depth alone) */
  uint8_t* disc = (uint8_t*)calloc((size_t)W * H, 1);
  if (!disc) return -1;
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      float z = depth[(size_t)y * W + x];
      if (!(z > 0.f)) continue;
      const int nx[4] = {x - 1, x + 1, x, x};
      const int ny[4] = {y, y, y - 1, y + 1};
      for (int k = 0; k < 4; ++k) {
        if (nx[k] < 0 || nx[k] >= W || ny[k] < 0 || ny[k] >= H) continue;
        float zq = depth[(size_t)ny[k] * W + nx[k]];
        if (!(zq > 0.f) || (double)(zq - z) > jump_rel * (double)z) {
          disc[(size_t)y * W + x] = 1;
          break;
        }
      }
    }
  }
  /* segments: sampled densely in 3D, z-buffered against the surfaces */
  for (int s = 0; s < n_segs; ++s) {
    const double* A = segs + (size_t)s * SEG_STRIDE;
    const double* B = A + 3;
    double YA[3], YB[3];
    world_to_cam(T, A, YA);
    world_to_cam(T, B, YB);
    /* pixel length bound from the projected endpoints after near clipping */
    const double znear = 0.1;
    if (YA[2] < znear && YB[2] < znear) continue;
    double ta = 0.0, tb = 1.0;
    if (YA[2] < znear) ta = (znear - YA[2]) / (YB[2] - YA[2]);
    if (YB[2] < znear) tb = (znear - YA[2]) / (YB[2] - YA[2]);
    double P0[3], P1[3];
    for (int k = 0; k < 3; ++k) {
      P0[k] = YA[k] + ta * (YB[k] - YA[k]);
      P1[k] = YA[k] + tb * (YB[k] - YA[k]);
    }
    double u0 = K[0] * P0[0] / P0[2] + K[2], v0 = K[1] * P0[1] / P0[2] + K[3];
    double u1 = K[0] * P1[0] / P1[2] + K[2], v1 = K[1] * P1[1] / P1[2] + K[3];
    double len = fabs(u1 - u0) + fabs(v1 - v0);
    if (len > 8.0 * (W + H)) len = 8.0 * (W + H);
    int n = (int)(3.0 * len) + 2;
    for (int k = 0; k <= n; ++k) {
      double a = (double)k / n;
      double Y[3];
      for (int q = 0; q < 3; ++q) Y[q] = P0[q] + a * (P1[q] - P0[q]);
      if (Y[2] <= znear) continue;
      double u = K[0] * Y[0] / Y[2] + K[2];
      double v = K[1] * Y[1] / Y[2] + K[3];
      int xi = (int)floor(u + 0.5), yi = (int)floor(v + 0.5);
      if (xi < 0 || xi >= W || yi < 0 || yi >= H) continue;
      size_t o = (size_t)yi * W + xi;
      float zs = (float)Y[2];
      float zc = depth[o];
      if (zc > 0.f && !(zs < zc * (1.0f - 1e-3f))) continue;
      depth[o] = zs;
      edge[o] = 1;
    }
  }
  int64_t count = 0;
  for (size_t o = 0; o < (size_t)W * H; ++o) {
    if (disc[o] && depth[o] > 0.f) edge[o] = 1;
    count += edge[o];
  }
  free(disc);
  return count;
}

/* Render many views in parallel.  Offsets index the flat depth/edge buffers. */
int64_t synth_render_views(const double* planes, int n_planes, const double* segs, int n_segs,
                           int n_views, const int* W, const int* H, const double* K,
                           const double* T, double jump_rel, const int64_t* px_off,
                           float* depth, uint8_t* edge, int64_t* edge_count) {
  int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (int v = 0; v < n_views; ++v) {
    int64_t c = synth_render_view(planes, n_planes, segs, n_segs, W[v], H[v], K + 4 * v,
                                  T + 12 * v, jump_rel, depth + px_off[v], edge + px_off[v]);
    edge_count[v] = c;
    if (c < 0) bad += 1;
  }
  return bad ? -1 : 0;
}
