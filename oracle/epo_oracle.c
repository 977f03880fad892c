/*
 * EPO FP64 CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct double-precision restatement of the EPO
 * edge-alignment objective (Section 3, Eqs. 6-8) and its analytic pose
 * gradient, the distance transform field it samples (Section 3, Algorithm 1,
 * "ComputeDistanceFields"), and the pose update used by the optimisation
 * loop (Algorithm 2, with the tangent-space Adam reading stated below).
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source with the CUDA library.
 *
 * Readings of points the paper leaves open (each is repeated at its use):
 *   - Pose T = [R|t] maps world -> camera (the extrinsic P of Section 3).
 *   - Depth is z-depth; pixel centres sit at integer coordinates.
 *   - A projected sample is valid iff Y3 > eps_z and 0 <= u' <= W-1 and
 *     0 <= v' <= H-1 (no occlusion test; the paper has none).
 *   - Bilinear cell: x0 = min(floor(u'), W-2), y0 = min(floor(v'), H-2).
 *   - Huber H_delta(x) = x^2/2 for |x| <= delta, delta(|x| - delta/2) else;
 *     the clamp d^ = min(d, lambda) passes the gradient when d <= lambda.
 *   - Per-direction mean: sum(rho) / sum(valid) (Algorithm 3) by default,
 *     or sum(rho) / |E_i| (Eq. 7) when norm_mode == 1.
 *   - Directed pair list of length P: L = (2/P) * sum_p l_p, which equals
 *     Eq. 6 for a symmetric list (every undirected pair counted both ways).
 *   - Pose gradient is taken w.r.t. a left perturbation T <- Exp(xi) T with
 *     xi = (upsilon, omega), translation first.
 *
 * Precision: every value is double; inputs that the GPU stores in reduced
 * precision are passed here already rounded and widened.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 3

/* ------------------------------------------------------------------ */
/* Distance transform field (Section 3; exact L2 EDT of Felzenszwalb   */
/* and Huttenlocher, "Distance transforms of sampled functions").      */
/* ------------------------------------------------------------------ */

/* 1-D squared distance transform of f over n samples: d(q) = min_p (q - p)^2 + f(p),
 * computed as the lower envelope of parabolas (Felzenszwalb-Huttenlocher).
 * Samples with f >= INF add no parabola.  v, z are work arrays of n and n+1 entries. */
static void edt_1d(const double* f, int n, double* d, int* v, double* z) {
  const double INF = 1e300;
  int q0 = 0;
  while (q0 < n && f[q0] >= INF) ++q0;
  if (q0 == n) {
    for (int q = 0; q < n; ++q) d[q] = INF;
    return;
  }
  int k = 0;
  v[0] = q0;
  z[0] = -INF;
  z[1] = INF;
  for (int q = q0 + 1; q < n; ++q) {
    if (f[q] >= INF) continue;
    double s = ((f[q] + (double)q * q) - (f[v[k]] + (double)v[k] * v[k])) / (2.0 * q - 2.0 * v[k]);
    while (s <= z[k]) {
      --k;
      s = ((f[q] + (double)q * q) - (f[v[k]] + (double)v[k] * v[k])) / (2.0 * q - 2.0 * v[k]);
    }
    ++k;
    v[k] = q;
    z[k] = s;
    z[k + 1] = INF;
  }
  k = 0;
  for (int q = 0; q < n; ++q) {
    while (z[k + 1] < q) ++k;
    double dq = (double)q - v[k];
    d[q] = dq * dq + f[v[k]];
  }
}

/* Number of OpenMP threads the loss and gradient use (n > 0 sets it); returns the count in
 * effect.  Timing aid for the CPU baseline: one thread against all cores. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* dist[y*W + x] = Euclidean distance from pixel (x, y) to the nearest edge
 * pixel; a view without edges gets W + H everywhere. */
int oracle_edt(const uint8_t* edge, int W, int H, double* dist) {
  if (W < 1 || H < 1) return ORACLE_EINVAL;
  int any = 0;
  for (int64_t o = 0; o < (int64_t)W * H; ++o) any |= edge[o];
  if (!any) {
    for (int64_t o = 0; o < (int64_t)W * H; ++o) dist[o] = (double)(W + H);
    return ORACLE_OK;
  }
  int n = W > H ? W : H;
  double* f = (double*)malloc(sizeof(double) * n);
  double* d = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * (n + 1));
  int* v = (int*)malloc(sizeof(int) * n);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)W * H);
  if (!f || !d || !z || !v || !tmp) {
    free(f); free(d); free(z); free(v); free(tmp);
    return ORACLE_ENOMEM;
  }
  const double INF = 1e300;
  /* rows */
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) f[x] = edge[(size_t)y * W + x] ? 0.0 : INF;
    edt_1d(f, W, d, v, z);
    for (int x = 0; x < W; ++x) tmp[(size_t)y * W + x] = d[x];
  }
  /* columns */
  for (int x = 0; x < W; ++x) {
    for (int y = 0; y < H; ++y) f[y] = tmp[(size_t)y * W + x];
    edt_1d(f, H, d, v, z);
    for (int y = 0; y < H; ++y) dist[(size_t)y * W + x] = sqrt(d[y]);
  }
  free(f); free(d); free(z); free(v); free(tmp);
  return ORACLE_OK;
}

/* Brute-force EDT: min over all edge pixels, for tiny images. */
int oracle_edt_brute(const uint8_t* edge, int W, int H, double* dist) {
  int any = 0;
  for (int64_t o = 0; o < (int64_t)W * H; ++o) any |= edge[o];
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      if (!any) { dist[(size_t)y * W + x] = (double)(W + H); continue; }
      double best = 1e300;
      for (int yy = 0; yy < H; ++yy)
        for (int xx = 0; xx < W; ++xx)
          if (edge[(size_t)yy * W + xx]) {
            double dd = (double)(x - xx) * (x - xx) + (double)(y - yy) * (y - yy);
            if (dd < best) best = dd;
          }
      dist[(size_t)y * W + x] = sqrt(best);
    }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Robust penalty (Eq. 7): Huber of the clamped distance.               */
/* ------------------------------------------------------------------ */
static double huber(double x, double delta) {
  double ax = fabs(x);
  return ax <= delta ? 0.5 * x * x : delta * (ax - 0.5 * delta);
}
static double huber_prime(double x, double delta) {
  if (fabs(x) <= delta) return x;
  return x > 0 ? delta : -delta;
}
/* rho = H(min(d, lambda)); drho = dH/dd with the clamp passing the gradient
 * for d <= lambda and blocking it above. */
void oracle_robust(double d, double lambda, double delta, double* rho, double* drho) {
  double dh = d < lambda ? d : lambda;
  *rho = huber(dh, delta);
  *drho = d <= lambda ? huber_prime(d, delta) : 0.0;
}

/* ------------------------------------------------------------------ */
/* Scene description (flat arrays, all double)                          */
/* ------------------------------------------------------------------ */
typedef struct {
  int n_views;
  const int* W;
  const int* H;
  const double* K;        /* n_views x 4: fx fy cx cy */
  const int64_t* rec_off; /* n_views + 1 */
  const double* rec;      /* n_rec x 3: u v z */
  const int64_t* map_off; /* n_views: offset of view's W*H map */
  const double* map;
  int n_pairs;
  const int* pairs;       /* 2 x n_pairs interleaved: (i, j) */
} oracle_scene;

typedef struct {
  double lambda, delta, eps_z;
  int norm_mode;          /* 0: sum(valid) (Algorithm 3), 1: |E_i| (Eq. 7) */
  double near_margin;     /* pixel distance from a validity boundary counted as "near" */
} oracle_params;

static void mat3_vec(const double* T, const double X[3], double Y[3]) {
  /* Y = R X + t for T = [R|t] row-major 3x4 */
  for (int r = 0; r < 3; ++r)
    Y[r] = T[4 * r] * X[0] + T[4 * r + 1] * X[1] + T[4 * r + 2] * X[2] + T[4 * r + 3];
}

/* UnprojectEdgesTo3D (Algorithm 2): X_world = P^-1 K^-1 [u, v, 1]^T z.
 * With P = [R|t], P^-1 X_c = R^T (X_c - t). */
static void unproject(const double* K, const double* T, const double* rec, double Xc[3],
                      double Xw[3]) {
  double u = rec[0], v = rec[1], z = rec[2];
  Xc[0] = (u - K[2]) / K[0] * z;
  Xc[1] = (v - K[3]) / K[1] * z;
  Xc[2] = z;
  double q[3] = {Xc[0] - T[3], Xc[1] - T[7], Xc[2] - T[11]};
  for (int c = 0; c < 3; ++c) Xw[c] = T[c] * q[0] + T[4 + c] * q[1] + T[8 + c] * q[2];
}

/*
 * Per-pair accumulation for one directed pair (i -> j) (Eq. 8 and the
 * summand of Eq. 7).  stats[0] = sum rho, stats[1] = n_valid,
 * stats[2..4] = sum dRho/dY (frame j), stats[5..7] = sum Y x dRho/dY,
 * gi[6], gj[6] = un-normalised pose-gradient sums for views i and j,
 * *near = samples whose validity lies within near_margin of flipping.
 */
static void pair_terms(const oracle_scene* S, const double* T, const double* Xw_all,
                       const oracle_params* prm, int p, double stats[8], double gi[6],
                       double gj[6], int64_t* near, double absum[6], double* maxterm) {
  int i = S->pairs[2 * p], j = S->pairs[2 * p + 1];
  const double* Ti = T + 12 * i;
  const double* Tj = T + 12 * j;
  const double* Ki = S->K + 4 * i;
  const double* Kj = S->K + 4 * j;
  int Wj = S->W[j], Hj = S->H[j];
  const double* map = S->map + S->map_off[j];
  double fx = Kj[0], fy = Kj[1], cx = Kj[2], cy = Kj[3];
  for (int k = 0; k < 8; ++k) stats[k] = 0.0;
  for (int k = 0; k < 6; ++k) gi[k] = gj[k] = absum[k] = 0.0;
  *near = 0;
  *maxterm = 0.0;
  for (int64_t r = S->rec_off[i]; r < S->rec_off[i + 1]; ++r) {
    const double* Xw = Xw_all + 3 * r;
    double Y[3];
    mat3_vec(Tj, Xw, Y); /* second half of pi: world -> camera j */
    double up = 0, vp = 0;
    int in_front = Y[2] > prm->eps_z;
    if (fabs(Y[2] - prm->eps_z) <= 1e-9 * (1.0 + fabs(Y[2]))) ++*near;
    if (!in_front) continue;
    up = fx * Y[0] / Y[2] + cx;
    vp = fy * Y[1] / Y[2] + cy;
    double m = prm->near_margin;
    if (fabs(up) <= m || fabs(up - (Wj - 1)) <= m || fabs(vp) <= m || fabs(vp - (Hj - 1)) <= m)
      ++*near;
    if (!(up >= 0.0 && up <= Wj - 1 && vp >= 0.0 && vp <= Hj - 1)) continue;
    /* bilinear sample of DTF_j */
    int x0 = (int)floor(up);
    if (x0 > Wj - 2) x0 = Wj - 2;
    int y0 = (int)floor(vp);
    if (y0 > Hj - 2) y0 = Hj - 2;
    double a = up - x0, b = vp - y0;
    double m00 = map[(int64_t)y0 * Wj + x0];
    double m01 = map[(int64_t)y0 * Wj + x0 + 1];
    double m10 = map[(int64_t)(y0 + 1) * Wj + x0];
    double m11 = map[(int64_t)(y0 + 1) * Wj + x0 + 1];
    double d = (1 - a) * (1 - b) * m00 + a * (1 - b) * m01 + (1 - a) * b * m10 + a * b * m11;
    double dd_du = (1 - b) * (m01 - m00) + b * (m11 - m10);
    double dd_dv = (1 - a) * (m10 - m00) + a * (m11 - m01);
    double rho, drho;
    oracle_robust(d, prm->lambda, prm->delta, &rho, &drho);
    stats[0] += rho;
    stats[1] += 1.0;
    /* chain rule to Y (camera-j coordinates) */
    double z = Y[2];
    double gY[3];
    gY[0] = drho * dd_du * fx / z;
    gY[1] = drho * dd_dv * fy / z;
    gY[2] = -drho * (dd_du * fx * Y[0] + dd_dv * fy * Y[1]) / (z * z);
    double c[3] = {Y[1] * gY[2] - Y[2] * gY[1], Y[2] * gY[0] - Y[0] * gY[2],
                   Y[0] * gY[1] - Y[1] * gY[0]};
    double tn = sqrt(gY[0] * gY[0] + gY[1] * gY[1] + gY[2] * gY[2] + c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (tn > *maxterm) *maxterm = tn;
    for (int k = 0; k < 3; ++k) {
      stats[2 + k] += gY[k];
      stats[5 + k] += c[k];
      absum[k] += fabs(gY[k]);
      absum[3 + k] += fabs(c[k]);
      gj[k] += gY[k];
      gj[3 + k] += c[k];
    }
    /* view i: Y = R_j R_i^T (X_c - t_i) + t_j, X_c the camera-i lift.
     * A left perturbation of T_i moves X_c by -(upsilon + omega x X_c) in
     * camera i, so dRho/dxi_i = (-h, -X_c x h), h = R_i R_j^T gY. */
    double Xc[3];
    {
      const double* rec = S->rec + 3 * r;
      Xc[0] = (rec[0] - Ki[2]) / Ki[0] * rec[2];
      Xc[1] = (rec[1] - Ki[3]) / Ki[1] * rec[2];
      Xc[2] = rec[2];
    }
    double w[3]; /* R_j^T gY */
    for (int c2 = 0; c2 < 3; ++c2) w[c2] = Tj[c2] * gY[0] + Tj[4 + c2] * gY[1] + Tj[8 + c2] * gY[2];
    double h[3]; /* R_i w */
    for (int r2 = 0; r2 < 3; ++r2) h[r2] = Ti[4 * r2] * w[0] + Ti[4 * r2 + 1] * w[1] + Ti[4 * r2 + 2] * w[2];
    double xh[3] = {Xc[1] * h[2] - Xc[2] * h[1], Xc[2] * h[0] - Xc[0] * h[2],
                    Xc[0] * h[1] - Xc[1] * h[0]};
    for (int k = 0; k < 3; ++k) {
      gi[k] -= h[k];
      gi[3 + k] -= xh[k];
    }
  }
}

/*
 * Objective and gradient (Eqs. 6-8).  T: n_views x 12.  Outputs:
 *   loss (scalar), grad (n_views x 6, may be NULL), pair_stats (P x 8, may be
 *   NULL), pair_near (P, may be NULL), pair_loss (P, may be NULL), pair_abs (P x 6,
 *   may be NULL: sum over valid samples of |dRho/dY_k| and |(Y x dRho/dY)_k|, the scale
 *   of the cancellation inside stats[2..7]), pair_maxterm (P, may be NULL: largest
 *   norm of one valid sample's (dRho/dY, Y x dRho/dY)).
 */
int oracle_loss_grad(const oracle_scene* S, const double* T, const oracle_params* prm,
                     double* loss, double* grad, double* pair_stats, int64_t* pair_near,
                     double* pair_loss, double* pair_abs, double* pair_maxterm) {
  if (!S || !T || !prm || !loss) return ORACLE_EINVAL;
  int n = S->n_views, P = S->n_pairs;
  for (int p = 0; p < P; ++p) {
    int i = S->pairs[2 * p], j = S->pairs[2 * p + 1];
    if (i < 0 || i >= n || j < 0 || j >= n) return ORACLE_EINVAL;
  }
  int64_t n_rec = S->rec_off[n];
  double* Xw = (double*)malloc(sizeof(double) * 3 * (n_rec > 0 ? n_rec : 1));
  double* st = (double*)malloc(sizeof(double) * 8 * (P > 0 ? P : 1));
  double* gi = (double*)malloc(sizeof(double) * 6 * (P > 0 ? P : 1));
  double* gj = (double*)malloc(sizeof(double) * 6 * (P > 0 ? P : 1));
  int64_t* nr = (int64_t*)malloc(sizeof(int64_t) * (P > 0 ? P : 1));
  double* ab = (double*)malloc(sizeof(double) * 6 * (P > 0 ? P : 1));
  double* mt = (double*)malloc(sizeof(double) * (P > 0 ? P : 1));
  if (!Xw || !st || !gi || !gj || !nr || !ab || !mt) {
    free(Xw); free(st); free(gi); free(gj); free(nr); free(ab); free(mt);
    return ORACLE_ENOMEM;
  }
  /* UnprojectEdgesTo3D: once per view (Algorithm 2) */
  for (int v = 0; v < n; ++v)
    for (int64_t r = S->rec_off[v]; r < S->rec_off[v + 1]; ++r) {
      double Xc[3];
      unproject(S->K + 4 * v, T + 12 * v, S->rec + 3 * r, Xc, Xw + 3 * r);
    }
  /* ProjectSampleHuber for every directed pair */
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = 0; p < P; ++p)
    pair_terms(S, T, Xw, prm, p, st + 8 * p, gi + 6 * p, gj + 6 * p, nr + p, ab + 6 * p, mt + p);
  /* per-direction means and the pair average, in fixed order */
  double L = 0.0;
  if (grad)
    for (int k = 0; k < 6 * n; ++k) grad[k] = 0.0;
  for (int p = 0; p < P; ++p) {
    int i = S->pairs[2 * p], j = S->pairs[2 * p + 1];
    double denom = prm->norm_mode == 1 ? (double)(S->rec_off[i + 1] - S->rec_off[i]) : st[8 * p + 1];
    double lp = denom > 0 ? st[8 * p] / denom : 0.0;
    double c = denom > 0 ? (2.0 / P) / denom : 0.0;
    L += lp;
    if (pair_loss) pair_loss[p] = lp;
    if (grad)
      for (int k = 0; k < 6; ++k) {
        grad[6 * i + k] += c * gi[6 * p + k];
        grad[6 * j + k] += c * gj[6 * p + k];
      }
    if (pair_stats)
      for (int k = 0; k < 8; ++k) pair_stats[8 * p + k] = st[8 * p + k];
    if (pair_near) pair_near[p] = nr[p];
    if (pair_abs)
      for (int k = 0; k < 6; ++k) pair_abs[6 * p + k] = ab[6 * p + k];
    if (pair_maxterm) pair_maxterm[p] = mt[p];
  }
  *loss = P > 0 ? (2.0 / P) * L : 0.0;
  free(Xw); free(st); free(gi); free(gj); free(nr); free(ab); free(mt);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Stochastic viewgraph sub-sampling (Appendix A.3, Algorithm 3): a fresh */
/* uniform random subset of min(|E|, M) pairs every step.               */
/* ------------------------------------------------------------------ */
/* SplitMix64's output function (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) applied to state + the golden-ratio increment. */
uint64_t oracle_splitmix64(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* The random key of pair p (index within its scene) at step s: one counter per (s, p). */
uint64_t oracle_pair_key(uint64_t seed, int64_t step, int32_t p) {
  return oracle_splitmix64(seed ^ (((uint64_t)step << 32) | (uint32_t)p));
}

/* The pairs of one scene evaluated at step s: the M with the smallest keys (ties by index),
 * all of them when the scene has at most M.  active: n_pairs bytes (1 = evaluated). */
int oracle_subsample(uint64_t seed, int64_t step, int32_t n_pairs, int32_t M, uint8_t* active) {
  if (n_pairs < 0 || M < 0 || (n_pairs > 0 && !active)) return ORACLE_EINVAL;
  for (int32_t p = 0; p < n_pairs; ++p) active[p] = 0;
  if (n_pairs <= M) {
    for (int32_t p = 0; p < n_pairs; ++p) active[p] = 1;
    return ORACLE_OK;
  }
  /* selection by repeated minimum: plain and slow, for the small scenes of the tests */
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_pairs);
  if (!key) return ORACLE_ENOMEM;
  for (int32_t p = 0; p < n_pairs; ++p) key[p] = oracle_pair_key(seed, step, p);
  for (int32_t m = 0; m < M; ++m) {
    int32_t best = -1;
    for (int32_t p = 0; p < n_pairs; ++p)
      if (!active[p] && (best < 0 || key[p] < key[best])) best = p;
    active[best] = 1;
  }
  free(key);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Viewgraph estimation (Section 3, Eq. 2; Algorithm 1 BuildViewgraph):   */
/* the fraction of grid pixels of view i that survive the round trip     */
/* i -> j -> i within tau pixels.                                        */
/* ------------------------------------------------------------------ */
/* Depth of view v at the pixel nearest to (x, y); 0 when outside the image. */
static double depth_nearest(const float* Z, int W, int H, double x, double y) {
  int xi = (int)floor(x + 0.5), yi = (int)floor(y + 0.5);
  if (xi < 0 || xi >= W || yi < 0 || yi >= H) return 0.0;
  return (double)Z[(int64_t)yi * W + xi];
}

/* camera v pixel (x, y) at depth z -> camera w pixel; returns 0 when not in front. */
static int reproject(const double* Kv, const double* Tv, const double* Kw, const double* Tw, double x, double y,
                     double z, double* xo, double* yo) {
  double Xc[3] = {(x - Kv[2]) / Kv[0] * z, (y - Kv[3]) / Kv[1] * z, z};
  double q[3] = {Xc[0] - Tv[3], Xc[1] - Tv[7], Xc[2] - Tv[11]};
  double Xw[3];
  for (int c = 0; c < 3; ++c) Xw[c] = Tv[c] * q[0] + Tv[4 + c] * q[1] + Tv[8 + c] * q[2];
  double Y[3];
  for (int r = 0; r < 3; ++r) Y[r] = Tw[4 * r] * Xw[0] + Tw[4 * r + 1] * Xw[1] + Tw[4 * r + 2] * Xw[2] + Tw[4 * r + 3];
  if (!(Y[2] > 0.0)) return 0;
  *xo = Kw[0] * Y[0] / Y[2] + Kw[2];
  *yo = Kw[1] * Y[1] / Y[2] + Kw[3];
  return 1;
}

/*
 * For every ordered pair (i, j), i != j: over the source pixels (x, y) = (a g, b g) of view i
 * whose depth is positive and finite, the fraction whose round trip
 *   p -> p_{i->j} (with Z_i at p) -> p_{i->j->i} (with Z_j at the pixel nearest p_{i->j})
 * stays in front of both cameras, inside view j, and returns within tau pixels of p.
 * depth: the views' W x H maps concatenated (row-major, float).  frac: n x n (diagonal 0).
 */
int oracle_viewgraph(int n, const int* W, const int* H, const double* K, const double* T, const float* depth,
                     int stride, double tau, double* frac) {
  if (n < 1 || stride < 1 || !W || !H || !K || !T || !depth || !frac) return ORACLE_EINVAL;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  if (!off) return ORACLE_ENOMEM;
  off[0] = 0;
  for (int v = 0; v < n; ++v) off[v + 1] = off[v] + (int64_t)W[v] * H[v];
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) {
    const float* Zi = depth + off[i];
    for (int j = 0; j < n; ++j) {
      if (i == j) {
        frac[(int64_t)i * n + j] = 0.0;
        continue;
      }
      const float* Zj = depth + off[j];
      int64_t valid = 0, good = 0;
      for (int y = 0; y < H[i]; y += stride)
        for (int x = 0; x < W[i]; x += stride) {
          double z = (double)Zi[(int64_t)y * W[i] + x];
          if (!(z > 0.0) || !isfinite(z)) continue;
          ++valid;
          double xj, yj;
          if (!reproject(K + 4 * i, T + 12 * i, K + 4 * j, T + 12 * j, x, y, z, &xj, &yj)) continue;
          if (!(xj >= 0.0 && xj <= W[j] - 1 && yj >= 0.0 && yj <= H[j] - 1)) continue;
          double zj = depth_nearest(Zj, W[j], H[j], xj, yj);
          if (!(zj > 0.0) || !isfinite(zj)) continue;
          double xb, yb;
          if (!reproject(K + 4 * j, T + 12 * j, K + 4 * i, T + 12 * i, xj, yj, zj, &xb, &yb)) continue;
          double dx = xb - x, dy = yb - y;
          if (sqrt(dx * dx + dy * dy) < tau) ++good;
        }
      frac[(int64_t)i * n + j] = valid > 0 ? (double)good / (double)valid : 0.0;
    }
  }
  free(off);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Optimization schedule (Section 3): per-view pose change in degrees,  */
/* its 95th percentile over the poses, and the dual-phase convergence.  */
/* ------------------------------------------------------------------ */
/* Rotation change: the angle of R_new R_prev^T, 180/pi arccos((tr - 1) / 2); translation
 * change: the angle between t_new and t_prev, 180/pi arccos(t_new . t_prev / (|t_new| |t_prev|))
 * (0 when either is the zero vector).  The arccos arguments are clipped to [-1, 1]. */
void oracle_pose_change(const double* T_prev, const double* T_new, int n, double* dR, double* dt) {
  const double deg = 180.0 / 3.14159265358979323846;
  for (int v = 0; v < n; ++v) {
    const double* A = T_new + 12 * v;
    const double* B = T_prev + 12 * v;
    double tr = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) tr += A[4 * r + c] * B[4 * r + c];
    double cr = (tr - 1.0) / 2.0;
    if (cr > 1.0) cr = 1.0;
    if (cr < -1.0) cr = -1.0;
    dR[v] = deg * acos(cr);
    double na = sqrt(A[3] * A[3] + A[7] * A[7] + A[11] * A[11]);
    double nb = sqrt(B[3] * B[3] + B[7] * B[7] + B[11] * B[11]);
    if (na == 0.0 || nb == 0.0) {
      dt[v] = 0.0;
      continue;
    }
    double ct = (A[3] * B[3] + A[7] * B[7] + A[11] * B[11]) / (na * nb);
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    dt[v] = deg * acos(ct);
  }
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* q-th percentile (0..100) with linear interpolation between the closest order statistics
 * (the default of the common numerical libraries). */
double oracle_percentile(const double* x, int n, double q) {
  if (n <= 0) return 0.0;
  double* s = (double*)malloc(sizeof(double) * n);
  if (!s) return NAN;
  memcpy(s, x, sizeof(double) * n);
  qsort(s, n, sizeof(double), cmp_double);
  double pos = q / 100.0 * (n - 1);
  int lo = (int)floor(pos);
  if (lo >= n - 1) {
    double r = s[n - 1];
    free(s);
    return r;
  }
  double r = s[lo] + (s[lo + 1] - s[lo]) * (pos - lo);
  free(s);
  return r;
}

/* theta_95 = max(95th percentile of dR, 95th percentile of dt) over the n poses. */
double oracle_theta95(const double* T_prev, const double* T_new, int n) {
  double* dR = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* dt = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  if (!dR || !dt) { free(dR); free(dt); return NAN; }
  oracle_pose_change(T_prev, T_new, n, dR, dt);
  double a = oracle_percentile(dR, n, 95.0), b = oracle_percentile(dt, n, 95.0);
  free(dR); free(dt);
  return a > b ? a : b;
}

/* One step of the dual-phase schedule.  state[0]: phase (1, 2; 3 = converged),
 * state[1]: consecutive steps below the current phase's threshold.  Phase 1 ends (depth
 * optimisation starts) after w1 consecutive steps with theta < eps1; phase 2 ends (the run
 * stops) after w2 consecutive steps with theta < eps2.  Returns the new phase. */
int oracle_converge_update(int32_t* state, double theta, double eps1, int w1, double eps2, int w2) {
  if (state[0] == 1) {
    state[1] = theta < eps1 ? state[1] + 1 : 0;
    if (state[1] >= w1) {
      state[0] = 2;
      state[1] = 0;
    }
  } else if (state[0] == 2) {
    state[1] = theta < eps2 ? state[1] + 1 : 0;
    if (state[1] >= w2) state[0] = 3;
  }
  return state[0];
}

/* ------------------------------------------------------------------ */
/* Camera and depth refinement (Section 3, Camera Refinement and Depth  */
/* Refinement, Eqs. 4-5): f_i = f_i^0 (1 + gamma_i) scales both focal    */
/* lengths of view i; each edge pixel's depth is Z^0 alpha + beta.       */
/* ------------------------------------------------------------------ */
/*
 * Objective (Eqs. 6-8) at poses T, focal scales gamma (n_views) and per-record depth
 * parameters alpha, beta (n_rec), and its gradient with respect to all of them:
 *   grad (n_views x 6, left perturbation as in oracle_loss_grad), grad_gamma (n_views),
 *   grad_alpha, grad_beta (n_rec).  Any gradient pointer may be NULL.
 * Two plain passes: the first sums rho and counts the valid samples of every pair (the
 * pair means' denominators), the second differentiates every sample with its pair's
 * weight (2/P) / denom and adds it to the parameters it depends on, pair by pair in order.
 * For a sample of record r (view i) in pair i -> j, with X_c its camera-i lift, Y its
 * camera-j position and gY = dRho/dY:
 *   h = R_i R_j^T gY = dRho/dX_c;
 *   dRho/dz_r = h . X_c / z_r (X_c is linear in z), so dRho/dalpha_r = dRho/dz_r Z^0_r and
 *   dRho/dbeta_r = dRho/dz_r;
 *   dRho/dgamma_i = -(h_0 X_c0 + h_1 X_c1) / (1 + gamma_i) (X_c0, X_c1 scale as 1 / f_i);
 *   dRho/dgamma_j = drho (dd/du' (u' - c_x) + dd/dv' (v' - c_y)) / (1 + gamma_j)
 *   (u' - c_x = f_j Y_0 / Y_2 scales as f_j).
 */
int oracle_loss_grad_full(const oracle_scene* S0, const double* T, const double* gamma,
                          const double* alpha, const double* beta, const oracle_params* prm,
                          double* loss, double* grad, double* grad_gamma, double* grad_alpha,
                          double* grad_beta) {
  if (!S0 || !T || !gamma || !alpha || !beta || !prm || !loss) return ORACLE_EINVAL;
  int n = S0->n_views, P = S0->n_pairs;
  int64_t n_rec = S0->rec_off[n];
  /* the refined intrinsics and depths, then the objective of oracle_loss_grad on them */
  double* K = (double*)malloc(sizeof(double) * 4 * (n > 0 ? n : 1));
  double* rec = (double*)malloc(sizeof(double) * 3 * (n_rec > 0 ? n_rec : 1));
  double* gz = (double*)calloc((size_t)(n_rec > 0 ? n_rec : 1), sizeof(double));
  double* st = (double*)malloc(sizeof(double) * 8 * (P > 0 ? P : 1));
  if (!K || !rec || !gz || !st) {
    free(K); free(rec); free(gz); free(st);
    return ORACLE_ENOMEM;
  }
  for (int v = 0; v < n; ++v) {
    K[4 * v + 0] = S0->K[4 * v + 0] * (1.0 + gamma[v]);
    K[4 * v + 1] = S0->K[4 * v + 1] * (1.0 + gamma[v]);
    K[4 * v + 2] = S0->K[4 * v + 2];
    K[4 * v + 3] = S0->K[4 * v + 3];
  }
  for (int64_t r = 0; r < n_rec; ++r) {
    rec[3 * r + 0] = S0->rec[3 * r + 0];
    rec[3 * r + 1] = S0->rec[3 * r + 1];
    rec[3 * r + 2] = S0->rec[3 * r + 2] * alpha[r] + beta[r];
  }
  oracle_scene S = *S0;
  S.K = K;
  S.rec = rec;
  int rc = oracle_loss_grad(&S, T, prm, loss, grad, st, NULL, NULL, NULL, NULL);
  if (rc != ORACLE_OK) {
    free(K); free(rec); free(gz); free(st);
    return rc;
  }
  if (grad_gamma)
    for (int v = 0; v < n; ++v) grad_gamma[v] = 0.0;
  /* second pass: the gradients with respect to gamma and the depths */
  for (int p = 0; p < P; ++p) {
    int i = S.pairs[2 * p], j = S.pairs[2 * p + 1];
    double denom = prm->norm_mode == 1 ? (double)(S.rec_off[i + 1] - S.rec_off[i]) : st[8 * p + 1];
    if (!(denom > 0)) continue;
    double c = (2.0 / P) / denom;
    const double* Ti = T + 12 * i;
    const double* Tj = T + 12 * j;
    const double* Ki = K + 4 * i;
    const double* Kj = K + 4 * j;
    int Wj = S.W[j], Hj = S.H[j];
    const double* map = S.map + S.map_off[j];
    double fx = Kj[0], fy = Kj[1], cx = Kj[2], cy = Kj[3];
    for (int64_t r = S.rec_off[i]; r < S.rec_off[i + 1]; ++r) {
      double Xc[3], Xw[3], Y[3];
      unproject(Ki, Ti, rec + 3 * r, Xc, Xw);
      mat3_vec(Tj, Xw, Y);
      if (!(Y[2] > prm->eps_z)) continue;
      double up = fx * Y[0] / Y[2] + cx;
      double vp = fy * Y[1] / Y[2] + cy;
      if (!(up >= 0.0 && up <= Wj - 1 && vp >= 0.0 && vp <= Hj - 1)) continue;
      int x0 = (int)floor(up);
      if (x0 > Wj - 2) x0 = Wj - 2;
      int y0 = (int)floor(vp);
      if (y0 > Hj - 2) y0 = Hj - 2;
      double a = up - x0, b = vp - y0;
      double m00 = map[(int64_t)y0 * Wj + x0];
      double m01 = map[(int64_t)y0 * Wj + x0 + 1];
      double m10 = map[(int64_t)(y0 + 1) * Wj + x0];
      double m11 = map[(int64_t)(y0 + 1) * Wj + x0 + 1];
      double d = (1 - a) * (1 - b) * m00 + a * (1 - b) * m01 + (1 - a) * b * m10 + a * b * m11;
      double dd_du = (1 - b) * (m01 - m00) + b * (m11 - m10);
      double dd_dv = (1 - a) * (m10 - m00) + a * (m11 - m01);
      double rho, drho;
      oracle_robust(d, prm->lambda, prm->delta, &rho, &drho);
      double z = Y[2];
      double gY[3];
      gY[0] = drho * dd_du * fx / z;
      gY[1] = drho * dd_dv * fy / z;
      gY[2] = -drho * (dd_du * fx * Y[0] + dd_dv * fy * Y[1]) / (z * z);
      double w[3], h[3];
      for (int c2 = 0; c2 < 3; ++c2) w[c2] = Tj[c2] * gY[0] + Tj[4 + c2] * gY[1] + Tj[8 + c2] * gY[2];
      for (int r2 = 0; r2 < 3; ++r2) h[r2] = Ti[4 * r2] * w[0] + Ti[4 * r2 + 1] * w[1] + Ti[4 * r2 + 2] * w[2];
      /* X_c = z (x~, y~, 1) with x~ = (u - c_x) / f_x: dX_c/dz = (x~, y~, 1) */
      const double xt = (rec[3 * r + 0] - Ki[2]) / Ki[0], yt = (rec[3 * r + 1] - Ki[3]) / Ki[1];
      gz[r] += c * (h[0] * xt + h[1] * yt + h[2]);
      if (grad_gamma) {
        grad_gamma[i] += c * -(h[0] * Xc[0] + h[1] * Xc[1]) / (1.0 + gamma[i]);
        grad_gamma[j] += c * drho * (dd_du * (up - cx) + dd_dv * (vp - cy)) / (1.0 + gamma[j]);
      }
    }
  }
  for (int64_t r = 0; r < n_rec; ++r) {
    if (grad_alpha) grad_alpha[r] = gz[r] * S0->rec[3 * r + 2];
    if (grad_beta) grad_beta[r] = gz[r];
  }
  free(K); free(rec); free(gz); free(st);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* SE(3): exponential, logarithm, left Jacobian (textbook Lie algebra;  */
/* xi = (upsilon, omega), translation first).                           */
/* ------------------------------------------------------------------ */
static void hat(const double w[3], double M[9]) {
  M[0] = 0; M[1] = -w[2]; M[2] = w[1];
  M[3] = w[2]; M[4] = 0; M[5] = -w[0];
  M[6] = -w[1]; M[7] = w[0]; M[8] = 0;
}
static void mm3(const double* A, const double* B, double* C) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
      C[3 * r + c] = s;
    }
}

/* Exp(xi) as a row-major 3x4 [R|t]:
 * R = I + A W + B W^2, t = (I + B W + C W^2) upsilon, with
 * A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3, W = omega^. */
void oracle_se3_exp(const double xi[6], double T[12]) {
  const double* ups = xi;
  const double* w = xi + 3;
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double A, B, C;
  if (th < 1e-4) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
    C = (th - sin(th)) / (th2 * th);
  }
  double Wm[9], W2[9];
  hat(w, Wm);
  mm3(Wm, Wm, W2);
  for (int r = 0; r < 3; ++r) {
    double tr = 0;
    for (int c = 0; c < 3; ++c) {
      double I = r == c ? 1.0 : 0.0;
      T[4 * r + c] = I + A * Wm[3 * r + c] + B * W2[3 * r + c];
      tr += (I + B * Wm[3 * r + c] + C * W2[3 * r + c]) * ups[c];
    }
    T[4 * r + 3] = tr;
  }
}

/* Log of a rigid transform (inverse of oracle_se3_exp for rotation angles < pi). */
void oracle_se3_log(const double T[12], double xi[6]) {
  double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
  double c = (R[0] + R[4] + R[8] - 1.0) / 2.0;
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  double th = acos(c);
  double w[3];
  double vee[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
  if (th < 1e-4) {
    double f = 0.5 * (1.0 + th * th / 6.0);
    for (int k = 0; k < 3; ++k) w[k] = f * vee[k];
  } else if (th > 3.14159265358979 - 1e-6) {
    /* near pi: omega from the symmetric part (R + I)/2 = n n^T */
    int k = 0;
    if (R[4] > R[3 * k + k]) k = 1;
    if (R[8] > R[3 * k + k]) k = 2;
    double n[3];
    double s = sqrt((R[3 * k + k] + 1.0) / 2.0);
    for (int q = 0; q < 3; ++q) n[q] = (q == k) ? s : (R[3 * k + q] + R[3 * q + k]) / (4.0 * s);
    double sgn = (n[0] * vee[0] + n[1] * vee[1] + n[2] * vee[2]) < 0 ? -1.0 : 1.0;
    for (int q = 0; q < 3; ++q) w[q] = sgn * th * n[q];
  } else {
    double f = th / (2.0 * sin(th));
    for (int k2 = 0; k2 < 3; ++k2) w[k2] = f * vee[k2];
  }
  /* upsilon = V^-1 t,  V^-1 = I - W/2 + (1/th^2)(1 - A/(2B)) W^2 */
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double thh = sqrt(th2);
  double D;
  if (thh < 1e-4) {
    D = 1.0 / 12.0 + th2 / 720.0;
  } else {
    double A = sin(thh) / thh, B = (1.0 - cos(thh)) / th2;
    D = (1.0 - A / (2.0 * B)) / th2;
  }
  double Wm[9], W2[9];
  hat(w, Wm);
  mm3(Wm, Wm, W2);
  double t[3] = {T[3], T[7], T[11]};
  for (int r = 0; r < 3; ++r) {
    double s = 0;
    for (int c2 = 0; c2 < 3; ++c2) {
      double I = r == c2 ? 1.0 : 0.0;
      s += (I - 0.5 * Wm[3 * r + c2] + D * W2[3 * r + c2]) * t[c2];
    }
    xi[r] = s;
  }
  for (int k = 0; k < 3; ++k) xi[3 + k] = w[k];
}

/* Left Jacobian of SE(3), J (6x6 row-major) with Exp(xi + e) ~ Exp(J e) Exp(xi):
 * J = [[Jw, Q], [0, Jw]], Jw = I + B W + C W^2 (SO(3) left Jacobian) and
 * Q(upsilon, omega) the translation-rotation coupling block (Barfoot,
 * "State Estimation for Robotics", Sec. 7.1.5). */
void oracle_se3_left_jacobian(const double xi[6], double J[36]) {
  const double* ups = xi;
  const double* w = xi + 3;
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double B, C, c1, c2, c3;
  if (th < 0.05) {
    double t4 = th2 * th2;
    B = 0.5 - th2 / 24.0 + t4 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + t4 / 5040.0;
    c1 = 1.0 / 6.0 - th2 / 120.0 + t4 / 5040.0;
    c2 = 1.0 / 24.0 - th2 / 720.0 + t4 / 40320.0;
    c3 = 1.0 / 120.0 - th2 / 2520.0 + t4 / 120960.0;
  } else {
    double s = sin(th), c = cos(th);
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
    c1 = (th - s) / (th2 * th);
    c2 = (th2 / 2.0 + c - 1.0) / (th2 * th2);
    c3 = (2.0 * th - 3.0 * s + th * c) / (2.0 * th2 * th2 * th);
  }
  double Wm[9], W2[9], P[9];
  hat(w, Wm);
  mm3(Wm, Wm, W2);
  hat(ups, P);
  double WP[9], PW[9], WPW[9], WWP[9], PWW[9], WPWW[9], WWPW[9];
  mm3(Wm, P, WP);
  mm3(P, Wm, PW);
  mm3(WP, Wm, WPW);
  mm3(Wm, WP, WWP);
  mm3(PW, Wm, PWW);
  mm3(WPW, Wm, WPWW);
  mm3(Wm, WPW, WWPW);
  double Q[9], Jw[9];
  for (int k = 0; k < 9; ++k) {
    Q[k] = 0.5 * P[k] + c1 * (WP[k] + PW[k] + WPW[k]) + c2 * (WWP[k] + PWW[k] - 3.0 * WPW[k]) +
           c3 * (WPWW[k] + WWPW[k]);
    Jw[k] = ((k % 4) == 0 ? 1.0 : 0.0) + B * Wm[k] + C * W2[k];
  }
  for (int k = 0; k < 36; ++k) J[k] = 0.0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      J[6 * r + c] = Jw[3 * r + c];
      J[6 * r + 3 + c] = Q[3 * r + c];
      J[6 * (3 + r) + 3 + c] = Jw[3 * r + c];
    }
}

/* ------------------------------------------------------------------ */
/* Optimisation loop (Algorithm 2 with the pose-only reading):          */
/* lambda anneal (Algorithm 3), gradient, tangent-space Adam, Exp.      */
/* ------------------------------------------------------------------ */
typedef struct {
  double lambda0, lambda1;
  int lambda_steps;
  double delta, eps_z;
  int norm_mode;
  double lr_rot, lr_trans, beta1, beta2, eps;
  int pair_budget;        /* M of Algorithm 3 (0 = every pair every step) */
  uint64_t seed;          /* of the sub-sampling keys */
} oracle_opt;

/* lambda_s: linear from lambda0 to lambda1 over lambda_steps, then held. */
double oracle_lambda(const oracle_opt* o, int64_t s) {
  double f = o->lambda_steps > 0 ? (double)s / o->lambda_steps : 1.0;
  if (f > 1.0) f = 1.0;
  return o->lambda0 + (o->lambda1 - o->lambda0) * f;
}

/*
 * Run n_steps optimisation steps from step index `step0`.  T (n x 12) is
 * updated in place; m, v (n x 6) are the Adam moments (in/out); loss_hist
 * (n_steps, may be NULL) receives the loss evaluated before each update.
 */
/*
 * One step of the full refinement (Algorithm 2 with the camera and depth modules): the
 * objective at (T, gamma, alpha, beta) with lambda of step s and its gradient, then
 *   poses: tangent-space Adam and T <- Exp(-Delta) T as in oracle_optimize (fixed views kept);
 *   gamma: Adam, gamma <- gamma - lr_focal m^/(sqrt(v^) + eps), bias-corrected with s + 1;
 *   alpha, beta: the same with lr_depth and the depth step count depth_t (>= 1) when
 *   depth_t > 0 (the depth module steps only in the schedule's second phase).
 * m/v arrays: pose n x 6, gamma n, alpha and beta n_rec each, updated in place.
 */
int oracle_refine_step(const oracle_scene* S, double* T, double* gamma, double* alpha, double* beta,
                       const uint8_t* fixed, const oracle_opt* o, int64_t s, int64_t depth_t, double lr_focal,
                       double lr_depth, double* m, double* v, double* mg, double* vg, double* ma, double* va,
                       double* mb, double* vb, double* loss) {
  int n = S->n_views;
  int64_t n_rec = S->rec_off[n];
  double* G = (double*)malloc(sizeof(double) * 6 * n);
  double* Gg = (double*)malloc(sizeof(double) * n);
  double* Ga = (double*)malloc(sizeof(double) * (n_rec > 0 ? n_rec : 1));
  double* Gb = (double*)malloc(sizeof(double) * (n_rec > 0 ? n_rec : 1));
  if (!G || !Gg || !Ga || !Gb) {
    free(G); free(Gg); free(Ga); free(Gb);
    return ORACLE_ENOMEM;
  }
  oracle_params prm;
  prm.lambda = oracle_lambda(o, s);
  prm.delta = o->delta;
  prm.eps_z = o->eps_z;
  prm.norm_mode = o->norm_mode;
  prm.near_margin = 0.0;
  double L;
  int rc = oracle_loss_grad_full(S, T, gamma, alpha, beta, &prm, &L, G, Gg, Ga, Gb);
  if (rc) {
    free(G); free(Gg); free(Ga); free(Gb);
    return rc;
  }
  if (loss) *loss = L;
  double bc1 = 1.0 - pow(o->beta1, (double)(s + 1)), bc2 = 1.0 - pow(o->beta2, (double)(s + 1));
  for (int i = 0; i < n; ++i) {
    /* focal scale of every view */
    mg[i] = o->beta1 * mg[i] + (1.0 - o->beta1) * Gg[i];
    vg[i] = o->beta2 * vg[i] + (1.0 - o->beta2) * Gg[i] * Gg[i];
    gamma[i] -= lr_focal * (mg[i] / bc1) / (sqrt(vg[i] / bc2) + o->eps);
    if (fixed && fixed[i]) continue;
    double delta[6];
    for (int k = 0; k < 6; ++k) {
      double g = G[6 * i + k];
      m[6 * i + k] = o->beta1 * m[6 * i + k] + (1.0 - o->beta1) * g;
      v[6 * i + k] = o->beta2 * v[6 * i + k] + (1.0 - o->beta2) * g * g;
      double lr = k < 3 ? o->lr_trans : o->lr_rot;
      delta[k] = -lr * (m[6 * i + k] / bc1) / (sqrt(v[6 * i + k] / bc2) + o->eps);
    }
    double E[12], Tn[12];
    oracle_se3_exp(delta, E);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 4; ++c) {
        double acc = c == 3 ? E[4 * r + 3] : 0.0;
        for (int k = 0; k < 3; ++k) acc += E[4 * r + k] * T[12 * i + 4 * k + c];
        Tn[4 * r + c] = acc;
      }
    memcpy(T + 12 * i, Tn, sizeof(Tn));
  }
  if (depth_t > 0) {
    double dc1 = 1.0 - pow(o->beta1, (double)depth_t), dc2 = 1.0 - pow(o->beta2, (double)depth_t);
    for (int64_t r = 0; r < n_rec; ++r) {
      ma[r] = o->beta1 * ma[r] + (1.0 - o->beta1) * Ga[r];
      va[r] = o->beta2 * va[r] + (1.0 - o->beta2) * Ga[r] * Ga[r];
      mb[r] = o->beta1 * mb[r] + (1.0 - o->beta1) * Gb[r];
      vb[r] = o->beta2 * vb[r] + (1.0 - o->beta2) * Gb[r] * Gb[r];
      alpha[r] -= lr_depth * (ma[r] / dc1) / (sqrt(va[r] / dc2) + o->eps);
      beta[r] -= lr_depth * (mb[r] / dc1) / (sqrt(vb[r] / dc2) + o->eps);
    }
  }
  free(G); free(Gg); free(Ga); free(Gb);
  return ORACLE_OK;
}

int oracle_optimize(const oracle_scene* S, double* T, const uint8_t* fixed, const oracle_opt* o,
                    int64_t step0, int n_steps, double* m, double* v, double* loss_hist) {
  int n = S->n_views;
  double* G = (double*)malloc(sizeof(double) * 6 * n);
  int P = S->n_pairs;
  int* sub = (int*)malloc(sizeof(int) * 2 * (P > 0 ? P : 1));
  uint8_t* act = (uint8_t*)malloc(P > 0 ? (size_t)P : 1);
  if (!G || !sub || !act) {
    free(G); free(sub); free(act);
    return ORACLE_ENOMEM;
  }
  oracle_params prm;
  prm.delta = o->delta;
  prm.eps_z = o->eps_z;
  prm.norm_mode = o->norm_mode;
  prm.near_margin = 0.0;
  for (int it = 0; it < n_steps; ++it) {
    int64_t s = step0 + it;
    prm.lambda = oracle_lambda(o, s);
    /* Algorithm 3: the step's pairs, a fresh uniform subset when the budget is exceeded */
    oracle_scene Ss = *S;
    if (o->pair_budget > 0 && P > o->pair_budget) {
      int rc0 = oracle_subsample(o->seed, s, P, o->pair_budget, act);
      if (rc0) { free(G); free(sub); free(act); return rc0; }
      int k = 0;
      for (int p = 0; p < P; ++p)
        if (act[p]) {
          sub[2 * k] = S->pairs[2 * p];
          sub[2 * k + 1] = S->pairs[2 * p + 1];
          ++k;
        }
      Ss.pairs = sub;
      Ss.n_pairs = k;
    }
    double L;
    int rc = oracle_loss_grad(&Ss, T, &prm, &L, G, NULL, NULL, NULL, NULL, NULL);
    if (rc) { free(G); free(sub); free(act); return rc; }
    if (loss_hist) loss_hist[it] = L;
    double bc1 = 1.0 - pow(o->beta1, (double)(s + 1));
    double bc2 = 1.0 - pow(o->beta2, (double)(s + 1));
    for (int i = 0; i < n; ++i) {
      if (fixed && fixed[i]) continue;
      double delta[6];
      for (int k = 0; k < 6; ++k) {
        double g = G[6 * i + k];
        m[6 * i + k] = o->beta1 * m[6 * i + k] + (1.0 - o->beta1) * g;
        v[6 * i + k] = o->beta2 * v[6 * i + k] + (1.0 - o->beta2) * g * g;
        double mh = m[6 * i + k] / bc1, vh = v[6 * i + k] / bc2;
        double lr = k < 3 ? o->lr_trans : o->lr_rot;
        delta[k] = -lr * mh / (sqrt(vh) + o->eps);
      }
      double E[12], Tn[12];
      oracle_se3_exp(delta, E);
      /* T <- Exp(-Delta) T */
      for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
          double acc = c == 3 ? E[4 * r + 3] : 0.0;
          for (int k = 0; k < 3; ++k) acc += E[4 * r + k] * T[12 * i + 4 * k + c];
          Tn[4 * r + c] = acc;
        }
      }
      memcpy(T + 12 * i, Tn, sizeof(Tn));
    }
  }
  free(G); free(sub); free(act);
  return ORACLE_OK;
}
