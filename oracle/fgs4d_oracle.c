/*
 * fgs4d_oracle.c -- plain FP64 CPU oracle of the 4D Gaussian Splatting render
 * path (forward image and its exact reverse-mode derivative).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA path.  Inputs are the same FP32 parameter arrays the GPU receives,
 * upcast to FP64; every formula below is the paper's definition written out
 * directly, with no blocking, fusion or reordering.
 *
 * Paper: "4D Gaussian Splatting: Modeling Dynamic Scenes with Native 4D
 * Primitives" (arXiv 2412.20720).
 *   Sec. 3.1, Eq. 1          unnormalized Gaussian
 *   Sec. 3.1, Eqs. 3-4       EWA projection of mean and covariance
 *   Sec. 3.2, Eqs. 5-6       4D pixel blending, p(u,v,t) = p(t) p(u,v|t)
 *   Sec. 3.2                 Sigma = R S S^T R^T, R = L(q_l) R(q_r)
 *   Sec. 3.2                 conditional 3D Gaussian and marginal p(t)
 *   Sec. 3.2                 4D spherindrical harmonics Z_nl^m
 *   Sec. 8.1.1 (impl.)       temporal filter p(t) < 0.05
 * Readings where the paper is silent (compositing constants 1/255, 0.99, 1e-4,
 * 3-sigma extent, pixel centres, rect membership, colour offset) follow the
 * tile rasterizer the paper adapts (Sec. 3.2, last paragraph of
 * "Representation of 4D Gaussian") and are listed in the design notes.
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py and
 * tests/test_oracle_grad_fd.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MAX_L 3
#define ORC_MAX_N 8

/* ------------------------------------------------------------------ types */

/* Parameters in FP64 (the caller upcasts the FP32 arrays the GPU gets). */
typedef struct {
  const double *mean;          /* [n][4] (x, y, z, t) */
  const double *log_scale;     /* [n][4] log(s_x, s_y, s_z, s_t) */
  const double *q_l;           /* [n][4] (a, b, c, d), not necessarily unit */
  const double *q_r;           /* [n][4] (p, q, r, s) */
  const double *opacity_logit; /* [n] */
  const double *sh;            /* [n][K][3], K = (L+1)^2 (n_max+1) */
  int64_t n;
  const double *mask_logit;    /* [n] or NULL: Compact-4DGS significance mask m (Sec. 4.3) */
  double mask_threshold;       /* epsilon of the mask indicator */
} orc_params;

typedef struct {
  int32_t width, height, pad0, pad1;
  double fx, fy, cx, cy;
  double viewmat[12]; /* world -> camera, row-major 3x4 [W | T] */
  double campos[3];   /* camera centre in world coordinates */
  double t;           /* render timestamp */
} orc_view;

typedef struct {
  int32_t sh_degree, t_order, tile, pad;
  double period;     /* T of the temporal Fourier basis */
  double near_plane; /* cull when camera-space z <= near_plane */
  double dilation;   /* added to the diagonal of the 2D covariance */
  double p_t_min;    /* temporal filter threshold (0.05) */
  double bg[3];
} orc_settings;

typedef struct {
  int32_t *status; /* [n] 0 visible; 1 invalid; 2 temporal; 3 near; 4 det; 5 rect; 6 a < 1/255; 7 masked */
  int32_t *rect;   /* [n][4] tile rect x0, y0, x1, y1 (half-open) */
  double *p_t;     /* [n] marginal temporal weight */
  double *a_eff;   /* [n] sigmoid(logit) * p_t */
  double *mu3;     /* [n][3] conditional mean at t */
  double *cov3;    /* [n][9] conditional covariance at t */
  double *pc;      /* [n][3] camera-space centre */
  double *cov2d;   /* [n][3] 2D covariance (xx, xy, yy) incl. dilation */
  double *conic;   /* [n][3] inverse 2D covariance (A, B, C) */
  double *uv;      /* [n][2] projected centre in pixels */
  double *radius;  /* [n] 3-sigma radius in pixels (integer valued) */
  double *depth;   /* [n] camera-space z */
  double *rgb;     /* [n][3] 4DSH colour after offset and clamp */
  double *margin;  /* [n] relative distance of the closest discrete decision */
  float *depth_f32;/* [n] depth rounded to FP32 (the sort key) */
  /* Filled by orc_preprocess_relaxed only (may be NULL otherwise): */
  int32_t *uncertain; /* [n] bit 1: a cull decision lies within the relaxation of its threshold, so the
                         Gaussian may be present or absent; bit 2: the colour clamp max(0, .) is within
                         the relaxation (the value is continuous there, its derivative is not) */
  int32_t *rect_lo;   /* [n][4] tiles inside the rect for every admissible radius and edge rounding */
  int32_t *rect_hi;   /* [n][4] tiles inside the rect for some admissible radius and edge rounding */
} orc_proj;

typedef struct {
  double *mean;          /* [n][4] */
  double *log_scale;     /* [n][4] */
  double *q_l;           /* [n][4] */
  double *q_r;           /* [n][4] */
  double *opacity_logit; /* [n] */
  double *sh;            /* [n][K][3] */
  double *g_uv;          /* [n][2]  dL/d(u, v) */
  double *g_conic;       /* [n][3]  dL/d(A, B, C) */
  double *g_a;           /* [n]     dL/d(effective opacity) */
  double *g_rgb;         /* [n][3]  dL/d(colour) */
  double *g_z;           /* [n]     dL/d(camera depth of the sliced mean), depth channel only */
  double *mask_logit;    /* [n]     dL/dm of the significance mask (straight-through) */
} orc_grads;

/* Per-Gaussian intermediate values of the forward chain, kept for the
 * adjoint. */
typedef struct {
  double m[4], ls[4], ql[4], qr[4], logit;
  double s[4], sig, qln[4], qrn[4], nql, nqr;
  double Lm[16], Rm[16], R[16], S[16];
  double dt, c, pt, b[3];
  double mu3[3], cov3[9];
  double pc[3];
  double J[6], M[6];
  double cov2[4], det, conic[3], uv[2], lam, radius;
  int rect[4];
  double w[3], rw, dir[3];
  int L, NT, K;
  double Y[(ORC_MAX_L + 1) * (ORC_MAX_L + 1)];
  double cosn[ORC_MAX_N + 1], sinn[ORC_MAX_N + 1];
  double raw[3], rgb[3];
  double a;
  double mask; /* M = sigmoid(m), 1 without a mask */
  int status;
  double margin;
  double relax;    /* 0: plain decisions; > 0: see orc_preprocess_relaxed */
  int uncertain;   /* bits as orc_proj.uncertain */
  int rect_lo[4], rect_hi[4];
} orc_ctx;

/* ------------------------------------------------------------ helpers */

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

static void mat4_mul(const double *A, const double *B, double *C) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += A[4 * i + k] * B[4 * k + j];
      C[4 * i + j] = acc;
    }
}

/* Left isoclinic rotation matrix L(q_l), Sec. 3.2 (first printed matrix). */
static void left_matrix(const double *q, double *L) {
  const double a = q[0], b = q[1], c = q[2], d = q[3];
  const double v[16] = {a, -b, -c, -d,
                        b,  a, -d,  c,
                        c,  d,  a, -b,
                        d, -c,  b,  a};
  memcpy(L, v, sizeof v);
}

/* Right isoclinic rotation matrix R(q_r), Sec. 3.2 (second printed matrix). */
static void right_matrix(const double *q, double *R) {
  const double p = q[0], qq = q[1], r = q[2], s = q[3];
  const double v[16] = {p, -qq,  -r,  -s,
                        qq,  p,   s,  -r,
                        r,  -s,   p,  qq,
                        s,   r, -qq,   p};
  memcpy(R, v, sizeof v);
}

/* Associated Legendre functions P_l^m(x), m >= 0, with the Condon-Shortley
 * phase, by the standard three-term recurrence in l.  P[l][m]. */
static void legendre(int L, double x, double P[ORC_MAX_L + 2][ORC_MAX_L + 2]) {
  memset(P, 0, sizeof(double) * (ORC_MAX_L + 2) * (ORC_MAX_L + 2));
  const double sx = sqrt(dmax(0.0, 1.0 - x * x));
  double pmm = 1.0;
  for (int m = 0; m <= L; ++m) {
    if (m > 0) pmm *= -(2.0 * m - 1.0) * sx; /* P_m^m = (-1)^m (2m-1)!! (1-x^2)^(m/2) */
    P[m][m] = pmm;
    if (m + 1 <= L) P[m + 1][m] = x * (2.0 * m + 1.0) * pmm;
    for (int l = m + 2; l <= L; ++l)
      P[l][m] = ((2.0 * l - 1.0) * x * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
  }
}

static double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

/* Real spherical harmonics Y_lm(theta, phi), orthonormal on the sphere,
 * from the complex ones with the Condon-Shortley phase kept in P_l^m:
 *   m > 0: sqrt(2) K_l^m P_l^m(cos th) cos(m ph)
 *   m = 0: K_l^0 P_l^0(cos th)
 *   m < 0: sqrt(2) K_l^|m| P_l^|m|(cos th) sin(|m| ph)
 * with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  Index l*l + l + m.
 * Optionally returns dY/dtheta and dY/dphi. */
static void real_sh(int L, double theta, double phi, double *Y, double *dYdth, double *dYdph) {
  double P[ORC_MAX_L + 2][ORC_MAX_L + 2];
  const double x = cos(theta), st = sin(theta);
  legendre(L + 1, x, P);
  for (int l = 0; l <= L; ++l) {
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial(l - am) / factorial(l + am));
      if (m != 0) K *= sqrt(2.0);
      double trig, dtrig;
      if (m > 0) { trig = cos(m * phi); dtrig = -m * sin(m * phi); }
      else if (m < 0) { trig = sin(am * phi); dtrig = am * cos(am * phi); }
      else { trig = 1.0; dtrig = 0.0; }
      const int idx = l * l + l + m;
      Y[idx] = K * P[l][am] * trig;
      if (dYdth) {
        /* dP_l^m/dtheta = (l x P_l^m - (l+m) P_{l-1}^m) / sin(theta), from
         * (x^2-1) dP_l^m/dx = l x P_l^m - (l+m) P_{l-1}^m, x = cos(theta). */
        const double plm1 = (l - 1 >= am) ? P[l - 1][am] : 0.0;
        const double dPdth = (l * x * P[l][am] - (l + am) * plm1) / st;
        dYdth[idx] = K * dPdth * trig;
        dYdph[idx] = K * P[l][am] * dtrig;
      }
    }
  }
}

/* ------------------------------------------------------ forward chain */

static int is_finite4(const double *v) {
  return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]);
}

/* Relative closeness of a value to an integer boundary (for margins). */
static double frac_margin(double x, double scale) {
  const double d = fabs(x - nearbyint(x));
  return d / dmax(1.0, scale);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* One cull decision of the forward chain, `fails` taken in FP64, `m` its
 * relative distance from the threshold.  Returns 1 when the chain stops.
 * Plain mode (relax = 0): a failing test stops the chain with `code`.
 * Relaxed mode: a decision within relax of its threshold could go either way
 * in another precision; the Gaussian is marked uncertain (bit 1) and, if the
 * FP64 test failed, `status` keeps the FP64 decision while the chain goes on
 * so that the values it would have if it passed are available. */
static int cull(orc_ctx *g, int fails, double m, int code) {
  g->margin = dmin(g->margin, m);
  const int near = m < g->relax;
  if (near) g->uncertain |= 1;
  if (!fails) return 0;
  if (near) {
    if (!g->status) g->status = code;
    return 0;
  }
  g->status = code;
  return 1;
}

/* Forward chain for Gaussian i at one view: Sec. 3.2 (covariance, rotation,
 * conditional and marginal), Sec. 3.1 Eqs. 3-4 (EWA projection), Sec. 3.2
 * (4D spherindrical harmonic colour), Sec. 8.1.1 (temporal filter). */
static void gauss_forward(const orc_params *P, int64_t i, const orc_view *V,
                          const orc_settings *S, orc_ctx *g, double relax) {
  memset(g, 0, sizeof *g);
  g->margin = INFINITY;
  g->relax = relax;
  for (int k = 0; k < 4; ++k) {
    g->m[k] = P->mean[4 * i + k];
    g->ls[k] = P->log_scale[4 * i + k];
    g->ql[k] = P->q_l[4 * i + k];
    g->qr[k] = P->q_r[4 * i + k];
  }
  g->logit = P->opacity_logit[i];
  g->L = S->sh_degree;
  g->NT = S->t_order;
  g->K = (g->L + 1) * (g->L + 1) * (g->NT + 1);

  if (!is_finite4(g->m) || !is_finite4(g->ls) || !is_finite4(g->ql) ||
      !is_finite4(g->qr) || !isfinite(g->logit)) {
    g->status = 1;
    return;
  }
  /* Compact-4DGS mask (Sec. 4.3): M = sigmoid(m), M_hat = 1{M > eps} in
   * value (the stop-gradient term), S_hat = M_hat S, alpha_hat = M_hat alpha.
   * M_hat = 0 removes the Gaussian (zero scales and opacity); M_hat = 1
   * leaves S and alpha unchanged. */
  g->mask = 1.0;
  if (P->mask_logit) {
    const double mlog = P->mask_logit[i];
    if (!isfinite(mlog)) {
      g->status = 1;
      return;
    }
    g->mask = 1.0 / (1.0 + exp(-mlog));
    if (cull(g, !(g->mask > P->mask_threshold), fabs(g->mask - P->mask_threshold) / dmax(P->mask_threshold, 1e-12),
             7))
      return;
  }
  /* Activations: s = exp(log s), alpha = sigmoid(logit), unit quaternions. */
  for (int k = 0; k < 4; ++k) g->s[k] = exp(g->ls[k]);
  g->sig = 1.0 / (1.0 + exp(-g->logit));
  g->nql = sqrt(g->ql[0] * g->ql[0] + g->ql[1] * g->ql[1] + g->ql[2] * g->ql[2] + g->ql[3] * g->ql[3]);
  g->nqr = sqrt(g->qr[0] * g->qr[0] + g->qr[1] * g->qr[1] + g->qr[2] * g->qr[2] + g->qr[3] * g->qr[3]);
  if (!(g->nql > 0.0) || !(g->nqr > 0.0)) {
    g->status = 1;
    return;
  }
  for (int k = 0; k < 4; ++k) {
    g->qln[k] = g->ql[k] / g->nql;
    g->qrn[k] = g->qr[k] / g->nqr;
  }
  /* R = L(q_l) R(q_r); Sigma = R S S^T R^T with S = diag(s). */
  left_matrix(g->qln, g->Lm);
  right_matrix(g->qrn, g->Rm);
  mat4_mul(g->Lm, g->Rm, g->R);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += g->R[4 * a + k] * g->R[4 * b + k] * g->s[k] * g->s[k];
      g->S[4 * a + b] = acc;
    }
  /* Marginal p(t) = N(t; mu_4, Sigma_44), used unnormalized (Sec. 3.1). */
  g->dt = V->t - g->m[3];
  g->c = g->S[15];
  g->pt = exp(-0.5 * g->dt * g->dt / g->c);
  if (cull(g, !(g->pt >= S->p_t_min), fabs(g->pt - S->p_t_min) / S->p_t_min, 2)) return;
  /* Conditional 3D Gaussian at t (Sec. 3.2). */
  for (int a = 0; a < 3; ++a) g->b[a] = g->S[4 * a + 3];
  for (int a = 0; a < 3; ++a) g->mu3[a] = g->m[a] + g->b[a] * g->dt / g->c;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      g->cov3[3 * a + b] = g->S[4 * a + b] - g->b[a] * g->b[b] / g->c;
  /* Camera-space centre. */
  const double *W = V->viewmat;
  for (int a = 0; a < 3; ++a)
    g->pc[a] = W[4 * a + 0] * g->mu3[0] + W[4 * a + 1] * g->mu3[1] + W[4 * a + 2] * g->mu3[2] + W[4 * a + 3];
  const double x = g->pc[0], y = g->pc[1], z = g->pc[2];
  /* (a relaxed chain goes on only while z stays positive) */
  if (cull(g, !(z > S->near_plane), fabs(z - S->near_plane) / dmax(S->near_plane, 1e-3), 3)) return;
  if (!(z > 0.0)) {
    g->status = 3;
    g->uncertain = 0;
    return;
  }
  /* Eq. 4: Sigma_2d = (J W Sigma W^T J^T)_{1:2,1:2} + dilation I. */
  g->J[0] = V->fx / z; g->J[1] = 0.0;       g->J[2] = -V->fx * x / (z * z);
  g->J[3] = 0.0;       g->J[4] = V->fy / z; g->J[5] = -V->fy * y / (z * z);
  for (int r = 0; r < 2; ++r)
    for (int col = 0; col < 3; ++col) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += g->J[3 * r + k] * W[4 * k + col];
      g->M[3 * r + col] = acc;
    }
  for (int r = 0; r < 2; ++r)
    for (int col = 0; col < 2; ++col) {
      double acc = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += g->M[3 * r + a] * g->cov3[3 * a + b] * g->M[3 * col + b];
      g->cov2[2 * r + col] = acc + (r == col ? S->dilation : 0.0);
    }
  g->det = g->cov2[0] * g->cov2[3] - g->cov2[1] * g->cov2[2];
  /* A non-positive determinant has no conic: that cull is never relaxed. */
  if (!(g->det > 0.0)) {
    g->margin = 0.0;
    g->status = 4;
    g->uncertain = 0;
    return;
  }
  cull(g, 0, g->det / (fabs(g->cov2[0] * g->cov2[3]) + 1e-300), 4);
  g->conic[0] = g->cov2[3] / g->det;
  g->conic[1] = -g->cov2[1] / g->det;
  g->conic[2] = g->cov2[0] / g->det;
  /* Eq. 3: projected centre (pixel coordinates, pinhole K). */
  g->uv[0] = V->fx * x / z + V->cx;
  g->uv[1] = V->fy * y / z + V->cy;
  /* 3-sigma extent from the largest eigenvalue (floor 0.1 under the root). */
  const double mid = 0.5 * (g->cov2[0] + g->cov2[3]);
  const double disc = mid * mid - g->det;
  g->margin = dmin(g->margin, fabs(disc - 0.1) / dmax(mid * mid, 1.0));
  g->lam = mid + sqrt(dmax(0.1, disc));
  const double r3 = 3.0 * sqrt(g->lam);
  g->radius = ceil(r3);
  g->margin = dmin(g->margin, frac_margin(r3, r3));
  /* Tile rect: tiles whose pixel range meets [u - r, u + r] x [v - r, v + r]. */
  const double B = (double)S->tile;
  const int gw = (V->width + S->tile - 1) / S->tile, gh = (V->height + S->tile - 1) / S->tile;
  const double ex[4] = {(g->uv[0] - g->radius) / B, (g->uv[1] - g->radius) / B,
                        (g->uv[0] + g->radius) / B, (g->uv[1] + g->radius) / B};
  for (int k = 0; k < 4; ++k) g->margin = dmin(g->margin, frac_margin(ex[k], fabs(ex[k]) * B) * B);
  const double lim = 1e9;
  g->rect[0] = clampi((int)floor(dmax(-lim, dmin(lim, ex[0]))), 0, gw);
  g->rect[1] = clampi((int)floor(dmax(-lim, dmin(lim, ex[1]))), 0, gh);
  g->rect[2] = clampi((int)floor(dmax(-lim, dmin(lim, ex[2]))) + 1, 0, gw);
  g->rect[3] = clampi((int)floor(dmax(-lim, dmin(lim, ex[3]))) + 1, 0, gh);
  /* Relaxed: the radius may round to any integer in [ceil(r3 (1 - relax)),
   * ceil(r3 (1 + relax))], and each rect edge u -/+ r (resp. v) may move by
   * relax max(1, |u -/+ r|) pixels before it is divided by the tile edge and
   * rounded down; rect_lo holds the tiles inside every such rect, rect_hi
   * those inside some. */
  for (int k = 0; k < 4; ++k) g->rect_lo[k] = g->rect_hi[k] = g->rect[k];
  if (relax > 0.0) {
    const double rr[2] = {ceil(r3 * (1.0 - relax)), ceil(r3 * (1.0 + relax))};
    for (int axis = 0; axis < 2; ++axis) {
      const int lim_t = axis == 0 ? gw : gh;
      int lo_min = 1 << 30, lo_max = -(1 << 30), hi_min = 1 << 30, hi_max = -(1 << 30);
      for (int a = 0; a < 2; ++a)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          const double e0 = g->uv[axis] - rr[a], e1 = g->uv[axis] + rr[a];
          const double w0 = relax * dmax(1.0, fabs(e0)), w1 = relax * dmax(1.0, fabs(e1));
          const int t0 = clampi((int)floor(dmax(-lim, dmin(lim, (e0 + sgn * w0) / B))), 0, lim_t);
          const int t1 = clampi((int)floor(dmax(-lim, dmin(lim, (e1 + sgn * w1) / B))) + 1, 0, lim_t);
          lo_min = t0 < lo_min ? t0 : lo_min;
          lo_max = t0 > lo_max ? t0 : lo_max;
          hi_min = t1 < hi_min ? t1 : hi_min;
          hi_max = t1 > hi_max ? t1 : hi_max;
        }
      g->rect_hi[axis] = lo_min;
      g->rect_hi[axis + 2] = hi_max;
      g->rect_lo[axis] = lo_max;
      g->rect_lo[axis + 2] = hi_min;
    }
    if (g->rect_hi[0] < g->rect_hi[2] && g->rect_hi[1] < g->rect_hi[3] &&
        (g->rect_lo[0] != g->rect_hi[0] || g->rect_lo[1] != g->rect_hi[1] || g->rect_lo[2] != g->rect_hi[2] ||
         g->rect_lo[3] != g->rect_hi[3]))
      g->margin = dmin(g->margin, 0.0);
  }
  if (g->rect[0] >= g->rect[2] || g->rect[1] >= g->rect[3]) {
    /* empty in FP64: relaxed, the Gaussian stays (absent or present) while
     * some admissible rect holds a tile */
    if (!(relax > 0.0 && g->rect_hi[0] < g->rect_hi[2] && g->rect_hi[1] < g->rect_hi[3])) {
      g->status = 5;
      g->uncertain = 0;
      return;
    }
    if (!g->status) g->status = 5;
    g->uncertain |= 1;
  }
  /* A Gaussian whose effective opacity is below 1/255 is skipped at every
   * pixel (alpha <= a), so dropping it leaves the image unchanged. */
  g->a = g->sig * g->pt;
  if (cull(g, g->a * 255.0 < 1.0, fabs(g->a * 255.0 - 1.0), 6)) return;
  /* 4DSH colour (Sec. 3.2): Z_nl^m = cos(2 pi n dt / T) Y_l^m(d), with the
   * view direction d from the camera centre to the sliced mean and
   * dt = t - mu_t; colour = max(0, sum c Z + 0.5). */
  for (int a = 0; a < 3; ++a) g->w[a] = g->mu3[a] - V->campos[a];
  g->rw = sqrt(g->w[0] * g->w[0] + g->w[1] * g->w[1] + g->w[2] * g->w[2]);
  for (int a = 0; a < 3; ++a) g->dir[a] = g->w[a] / g->rw;
  const double theta = acos(dmax(-1.0, dmin(1.0, g->dir[2])));
  const double phi = atan2(g->dir[1], g->dir[0]);
  real_sh(g->L, theta, phi, g->Y, NULL, NULL);
  for (int nn = 0; nn <= g->NT; ++nn) {
    g->cosn[nn] = cos(2.0 * ORC_PI * nn * g->dt / S->period);
    g->sinn[nn] = sin(2.0 * ORC_PI * nn * g->dt / S->period);
  }
  const int nlm = (g->L + 1) * (g->L + 1);
  const double *sh = P->sh + (size_t)i * g->K * 3;
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0.0;
    for (int nn = 0; nn <= g->NT; ++nn)
      for (int lm = 0; lm < nlm; ++lm)
        acc += sh[(nn * nlm + lm) * 3 + ch] * g->cosn[nn] * g->Y[lm];
    g->raw[ch] = acc;
    g->rgb[ch] = dmax(0.0, acc + 0.5);
    if (!isfinite(g->rgb[ch])) {
      g->status = 1;
      g->uncertain = 0;
      return;
    }
    if (fabs(acc + 0.5) < relax) g->uncertain |= 2;
  }
}

/* Stores every value the chain reached (zeros past the cull point); the
 * rect of a culled Gaussian is empty. */
static void store_proj(const orc_ctx *g, int64_t i, orc_proj *o) {
  o->status[i] = g->status;
  o->margin[i] = g->margin;
  for (int k = 0; k < 4; ++k) o->rect[4 * i + k] = g->status == 0 ? g->rect[k] : 0;
  const int alive = g->status == 0 || (g->uncertain & 1);
  if (o->uncertain) o->uncertain[i] = alive ? g->uncertain : 0;
  if (o->rect_lo)
    for (int k = 0; k < 4; ++k) o->rect_lo[4 * i + k] = g->status == 0 && !(g->uncertain & 1) ? g->rect_lo[k] : 0;
  if (o->rect_hi)
    for (int k = 0; k < 4; ++k) o->rect_hi[4 * i + k] = alive ? g->rect_hi[k] : 0;
  o->p_t[i] = g->pt;
  o->a_eff[i] = g->a;
  for (int k = 0; k < 3; ++k) o->mu3[3 * i + k] = g->mu3[k];
  for (int k = 0; k < 9; ++k) o->cov3[9 * i + k] = g->cov3[k];
  for (int k = 0; k < 3; ++k) o->pc[3 * i + k] = g->pc[k];
  o->cov2d[3 * i + 0] = g->cov2[0];
  o->cov2d[3 * i + 1] = g->cov2[1];
  o->cov2d[3 * i + 2] = g->cov2[3];
  for (int k = 0; k < 3; ++k) o->conic[3 * i + k] = g->conic[k];
  o->uv[2 * i + 0] = g->uv[0];
  o->uv[2 * i + 1] = g->uv[1];
  o->radius[i] = g->radius;
  o->depth[i] = g->pc[2];
  o->depth_f32[i] = (float)g->pc[2];
  for (int k = 0; k < 3; ++k) o->rgb[3 * i + k] = g->rgb[k];
}

int orc_preprocess(const orc_params *P, const orc_view *V, const orc_settings *S, orc_proj *out) {
  if (S->sh_degree < 0 || S->sh_degree > ORC_MAX_L || S->t_order < 0 || S->t_order > ORC_MAX_N) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < P->n; ++i) {
    orc_ctx g;
    gauss_forward(P, i, V, S, &g, 0.0);
    store_proj(&g, i, out);
  }
  return 0;
}

/* The per-Gaussian chain with every discrete decision relaxed by `relax`
 * (relative): a decision that another precision could take the other way
 * (a cull threshold, the integer radius, a tile-rect edge, the colour clamp)
 * is marked in out->uncertain, rect_lo / rect_hi bound the tile rect over
 * the admissible roundings, and a Gaussian culled within the relaxation gets
 * the values it would have had (its status keeps the FP64 decision).  The
 * FP64 values, status and rect equal orc_preprocess's. */
int orc_preprocess_relaxed(const orc_params *P, const orc_view *V, const orc_settings *S, double relax,
                           orc_proj *out) {
  if (S->sh_degree < 0 || S->sh_degree > ORC_MAX_L || S->t_order < 0 || S->t_order > ORC_MAX_N) return -1;
  if (!(relax >= 0.0) || !out->uncertain || !out->rect_lo || !out->rect_hi) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < P->n; ++i) {
    orc_ctx g;
    gauss_forward(P, i, V, S, &g, relax);
    store_proj(&g, i, out);
  }
  return 0;
}

/* ------------------------------------------------------- compositing */

typedef struct {
  float depth;
  int64_t idx;
} orc_entry;

static int entry_cmp(const void *pa, const void *pb) {
  const orc_entry *a = pa, *b = pb;
  if (a->depth < b->depth) return -1;
  if (a->depth > b->depth) return 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* Front-to-back compositing of one pixel over its depth-sorted list
 * (Sec. 3.2, Eq. 6: p_i(t) p_i(u,v|t) alpha_i c_i prod_{j<i}(1 - ...)).
 * Per entry: power = -1/2 d^T conic d; skip if power > 0; alpha =
 * min(0.99, a_eff exp(power)); skip if alpha < 1/255; stop before adding an
 * entry that would take T below 1e-4.  Sample point is the pixel centre.
 * If rec != NULL, the contributing entries are recorded for the adjoint. */
typedef struct {
  int64_t idx;
  int32_t pos;
  double alpha, G, T, dx, dy;
  int clamped;
} orc_contrib;

static void composite_pixel(const orc_proj *P, const orc_settings *S, const orc_entry *list, int64_t len,
                            int px, int py, double out[3], double *T_out, int32_t *ncontrib,
                            double *margin, int32_t *signature, orc_contrib *rec, int64_t *nrec,
                            const double *aux, double aux_out[3]) {
  const double pxc = px + 0.5, pyc = py + 0.5;
  double T = 1.0, C[3] = {0.0, 0.0, 0.0}, X[3] = {0.0, 0.0, 0.0};
  double mg = INFINITY;
  int32_t last = 0, nclamp = 0;
  int64_t nr = 0;
  uint32_t prev_bits = 0;
  int have_prev = 0;
  for (int64_t j = 0; j < len; ++j) {
    const int64_t i = list[j].idx;
    const uint32_t bits = f32_bits(list[j].depth);
    /* Two entries within 2 ulp of depth may swap order in FP32. */
    if (have_prev && bits - prev_bits <= 2u) mg = 0.0;
    prev_bits = bits;
    have_prev = 1;
    const double A = P->conic[3 * i + 0], B = P->conic[3 * i + 1], Cc = P->conic[3 * i + 2];
    const double dx = P->uv[2 * i + 0] - pxc, dy = P->uv[2 * i + 1] - pyc;
    const double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
    if (fabs(power) < 1e-6) mg = 0.0;
    if (power > 0.0) continue;
    const double G = exp(power);
    const double aG = P->a_eff[i] * G;
    mg = dmin(mg, fabs(aG - 0.99) / 0.99);
    const double alpha = dmin(0.99, aG);
    mg = dmin(mg, fabs(alpha * 255.0 - 1.0));
    if (alpha < 1.0 / 255.0) continue;
    const double Tn = T * (1.0 - alpha);
    mg = dmin(mg, fabs(Tn - 1e-4) / 1e-4);
    if (Tn < 1e-4) break;
    for (int ch = 0; ch < 3; ++ch) C[ch] += P->rgb[3 * i + ch] * alpha * T;
    if (aux)
      for (int ch = 0; ch < 3; ++ch) X[ch] += aux[3 * i + ch] * alpha * T;
    if (rec) {
      rec[nr].idx = i;
      rec[nr].pos = (int32_t)j;
      rec[nr].alpha = alpha;
      rec[nr].G = G;
      rec[nr].T = T;
      rec[nr].dx = dx;
      rec[nr].dy = dy;
      rec[nr].clamped = aG > 0.99;
    }
    ++nr;
    nclamp += aG > 0.99;
    T = Tn;
    last = (int32_t)(j + 1);
  }
  for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * S->bg[ch];
  if (aux_out)
    for (int ch = 0; ch < 3; ++ch) aux_out[ch] = X[ch];
  if (T_out) *T_out = T;
  if (ncontrib) *ncontrib = last;
  if (margin) *margin = mg;
  /* Discrete outcome of this pixel: contributors and clamped alphas. */
  if (signature) *signature = (int32_t)nr + 65536 * nclamp;
  if (nrec) *nrec = nr;
}

/* Tile lists: for every tile, the visible Gaussians whose tile rect contains
 * it, sorted by (FP32 depth, index). */
typedef struct {
  int64_t *off;  /* [ntiles + 1] */
  orc_entry *ent;
} orc_tiles;

static int build_tiles(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P, orc_tiles *T) {
  const int gw = (V->width + S->tile - 1) / S->tile, gh = (V->height + S->tile - 1) / S->tile;
  const int64_t nt = (int64_t)gw * gh;
  T->off = calloc((size_t)nt + 1, sizeof(int64_t));
  if (!T->off) return -1;
  for (int64_t i = 0; i < n; ++i) {
    if (P->status[i] != 0) continue;
    const int32_t *r = P->rect + 4 * i;
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) T->off[(int64_t)ty * gw + tx + 1]++;
  }
  for (int64_t t = 0; t < nt; ++t) T->off[t + 1] += T->off[t];
  T->ent = malloc(sizeof(orc_entry) * (size_t)(T->off[nt] > 0 ? T->off[nt] : 1));
  int64_t *fill = calloc((size_t)nt, sizeof(int64_t));
  if (!T->ent || !fill) return -1;
  for (int64_t i = 0; i < n; ++i) {
    if (P->status[i] != 0) continue;
    const int32_t *r = P->rect + 4 * i;
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) {
        const int64_t t = (int64_t)ty * gw + tx;
        orc_entry e = {P->depth_f32[i], i};
        T->ent[T->off[t] + fill[t]++] = e;
      }
  }
  free(fill);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < nt; ++t)
    qsort(T->ent + T->off[t], (size_t)(T->off[t + 1] - T->off[t]), sizeof(orc_entry), entry_cmp);
  return 0;
}

static void free_tiles(orc_tiles *T) {
  free(T->off);
  free(T->ent);
}

int orc_render(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P,
               double *img, double *T_out, int32_t *ncontrib, double *margin, int32_t *signature) {
  orc_tiles tl;
  if (build_tiles(V, S, n, P, &tl)) return -1;
  const int W = V->width, H = V->height, gw = (W + S->tile - 1) / S->tile;
  const int64_t HW = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int py = 0; py < H; ++py) {
    for (int px = 0; px < W; ++px) {
      const int64_t t = (int64_t)(py / S->tile) * gw + px / S->tile;
      const int64_t p = (int64_t)py * W + px;
      double out[3];
      composite_pixel(P, S, tl.ent + tl.off[t], tl.off[t + 1] - tl.off[t], px, py, out,
                      T_out ? &T_out[p] : NULL, ncontrib ? &ncontrib[p] : NULL,
                      margin ? &margin[p] : NULL, signature ? &signature[p] : NULL, NULL, NULL, NULL, NULL);
      for (int ch = 0; ch < 3; ++ch) img[ch * HW + p] = out[ch];
    }
  }
  free_tiles(&tl);
  return 0;
}

/* Selected pixels only: each pixel's list is gathered by a scan over all
 * Gaussians (used to check full-size renders at sampled pixels). */
int orc_render_pixels(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P,
                      int64_t npix, const int64_t *pix, double *rgb, double *T_out,
                      int32_t *ncontrib, double *margin) {
  const int W = V->width;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < npix; ++q) {
    const int px = (int)(pix[q] % W), py = (int)(pix[q] / W);
    const int tx = px / S->tile, ty = py / S->tile;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *r = P->rect + 4 * i;
      if (P->status[i] == 0 && tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) ++cnt;
    }
    orc_entry *list = malloc(sizeof(orc_entry) * (size_t)(cnt > 0 ? cnt : 1));
    if (!list) {
      err = 1;
      continue;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *r = P->rect + 4 * i;
      if (P->status[i] == 0 && tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) {
        orc_entry e = {P->depth_f32[i], i};
        list[k++] = e;
      }
    }
    qsort(list, (size_t)cnt, sizeof(orc_entry), entry_cmp);
    composite_pixel(P, S, list, cnt, px, py, rgb + 3 * q, T_out ? &T_out[q] : NULL,
                    ncontrib ? &ncontrib[q] : NULL, margin ? &margin[q] : NULL, NULL, NULL, NULL, NULL, NULL);
    free(list);
  }
  return err ? -1 : 0;
}

/* ------------------------------------------- admissible pixel results */

/* The compositing of Eq. 6 takes discrete decisions per pixel: an entry is
 * skipped when alpha < 1/255 (or when the exponent is positive), and the
 * walk stops before an entry that would take T below 1e-4; the list order
 * comes from FP32 depths, and tile membership from the integer radius and
 * rect edges.  A renderer working in FP32 takes each decision from values
 * within a known error of the FP64 ones, so where an FP64 value lies within
 * that error of its threshold either outcome is correct.  This function
 * walks every combination of such outcomes (depth-first, state copied only
 * where the walk branches) and returns each distinct result.  With zero
 * tolerances and a plain (relax = 0) projection it takes exactly the
 * decisions of composite_pixel and returns its result, bit for bit; with
 * any tolerances that result is always one of those returned.
 *
 * Error model of one alpha (relative).  The exponent is taken as a sum of
 * two squares, -power = ((u11 dx)^2 + (u12 dx + u22 dy)^2) / 2 with the
 * conic Q = U U^T, U upper triangular (the form in which FP32 evaluation
 * does not cancel); with u11, u22 known to a relative eps_conic and u12 to
 * eps_conic (|u12| + sqrt(Q11)), the exponent is known to eps_conic ((u11
 * dx)^2 + |e| (|u12 dx| + sqrt(Q11) |dx| + u22 |dy|)), e = u12 dx + u22 dy.
 * Added to that: the exponent's change under a centre
 * error of eps_uv |u| + eps_uv_abs pixels (resp. v), plus eps_a (effective opacity)
 * and eps_alpha (the exponential and rounding).  The transmittance's
 * relative error bound accumulates alpha * e / (1 - alpha) per composited
 * entry, plus eps_alpha for the rounding of the update.  Depth keys may differ from the FP64 depth rounded to FP32 by
 * depth_ulps units in the last place, so two entries whose keys differ by at
 * most 2 depth_ulps may be composited in either order. */
typedef struct {
  double eps_conic, eps_uv, eps_uv_abs, eps_a, eps_alpha;
  int32_t depth_ulps;
  int32_t max_leaves; /* walk budget per pixel; past it the pixel is flagged (bit 4) */
} orc_tol;

enum { ORC_SKIP = 1, ORC_TAKE = 2 };

/* Alpha of Gaussian i at the sample point (pxc, pyc) (Eq. 6: min(0.99,
 * a exp(power))) and the relative error bound e of an FP32 renderer's alpha
 * there (the model above). */
static void adm_alpha(const orc_proj *P, const orc_tol *tol, int64_t i, double pxc, double pyc, double *power_out,
                      double *aG_out, double *alpha_out, double *err_out) {
  const double A = P->conic[3 * i + 0], Bc = P->conic[3 * i + 1], Cc = P->conic[3 * i + 2];
  const double u = P->uv[2 * i + 0], v = P->uv[2 * i + 1];
  const double dx = u - pxc, dy = v - pyc;
  const double power = -0.5 * (A * dx * dx + Cc * dy * dy) - Bc * dx * dy;
  const double aG = P->a_eff[i] * exp(power);
  /* the exponent as a sum of two squares, Q = U U^T with U upper
   * triangular: -power = ((u11 dx)^2 + (u12 dx + u22 dy)^2) / 2 */
  const double u22 = sqrt(Cc), u12 = Bc / u22, u11 = sqrt(dmax(0.0, A * Cc - Bc * Bc) / Cc);
  const double ex = u11 * dx, ey = u12 * dx + u22 * dy;
  const double pfac = ex * ex + fabs(ey) * (fabs(u12 * dx) + sqrt(A) * fabs(dx) + u22 * fabs(dy));
  const double gx = fabs(A * dx + Bc * dy), gy = fabs(Cc * dy + Bc * dx);
  *err_out = tol->eps_conic * pfac + gx * (tol->eps_uv * fabs(u) + tol->eps_uv_abs) +
             gy * (tol->eps_uv * fabs(v) + tol->eps_uv_abs) + tol->eps_a + tol->eps_alpha;
  *power_out = power;
  *aG_out = aG;
  *alpha_out = dmin(0.99, aG);
}

/* alpha and its error bound for npairs (Gaussian, pixel) pairs, the pixel
 * given by its linear id py * width + px (sample point at its centre). */
void orc_alpha_bounds(const orc_view *V, const orc_proj *P, const orc_tol *tol, int64_t npairs, const int64_t *idx,
                      const int64_t *pix, double *alpha, double *err) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < npairs; ++k) {
    double power, aG;
    adm_alpha(P, tol, idx[k], (double)(pix[k] % V->width) + 0.5, (double)(pix[k] / V->width) + 0.5, &power, &aG,
              &alpha[k], &err[k]);
  }
}

typedef struct {
  int64_t idx;
  uint32_t bits;
  int opts;     /* ORC_SKIP | ORC_TAKE: outcomes admissible at this pixel */
  double alpha; /* min(0.99, a G) */
  double err;   /* relative error bound of alpha */
  int gflag;    /* the derivative of a take is uncertain (near the 0.99 clamp, or colour clamp) */
} orc_adm_entry;

typedef struct {
  double T, errT;
  int32_t nr;
  int gflag;
  double C[3];
  double X[64];
} orc_adm_state;

typedef struct {
  const orc_proj *P;
  const orc_settings *S;
  const double *extra;
  int nextra;
  const orc_adm_entry *seq; /* entries with an outcome other than skip, in FP64 list order */
  const int64_t *gstart;    /* groups of entries that may swap: [gstart[g], gstart[g + 1]) */
  int64_t ngroups;
  int32_t depth_ulps;
  double eps_step;          /* rounding of one transmittance update (eps_alpha) */
  int32_t max_cands, max_leaves;
  double *cands;            /* [max_cands][5 + nextra]: r, g, b, T, contributors, extra... */
  int32_t ncands, leaves;
  int flags;
} orc_adm_ctx;

static void adm_leaf(orc_adm_ctx *c, const orc_adm_state *s) {
  const int nv = 5 + c->nextra;
  double v[5 + 64];
  for (int ch = 0; ch < 3; ++ch) v[ch] = s->C[ch] + s->T * c->S->bg[ch];
  v[3] = s->T;
  v[4] = s->nr;
  for (int k = 0; k < c->nextra; ++k) v[5 + k] = s->X[k];
  if (s->gflag) c->flags |= 2;
  for (int32_t j = 0; j < c->ncands; ++j)
    if (memcmp(c->cands + (int64_t)j * nv, v, sizeof(double) * (size_t)nv) == 0) return;
  if (c->ncands >= c->max_cands) {
    c->flags |= 4;
    return;
  }
  memcpy(c->cands + (int64_t)c->ncands * nv, v, sizeof(double) * (size_t)nv);
  ++c->ncands;
}

/* Outcomes of entry e at state s: up to three successor states (skip; take
 * and go on) or a stop.  Returns the number of successors; *stop is set when
 * stopping before e is admissible. */
static int adm_options(const orc_adm_ctx *c, const orc_adm_entry *e, const orc_adm_state *s, orc_adm_state out[2],
                       int *stop) {
  int k = 0;
  *stop = 0;
  if (e->opts & ORC_SKIP) out[k++] = *s;
  if (e->opts & ORC_TAKE) {
    const double alpha = e->alpha;
    const double Tn = s->T * (1.0 - alpha);
    const double errTn = s->errT + alpha * e->err / (1.0 - alpha) + c->eps_step;
    if (Tn * (1.0 - errTn) < 1e-4) *stop = 1;
    if (Tn * (1.0 + errTn) >= 1e-4) {
      orc_adm_state n = *s;
      const int64_t i = e->idx;
      for (int ch = 0; ch < 3; ++ch) n.C[ch] += c->P->rgb[3 * i + ch] * alpha * s->T;
      for (int q = 0; q < c->nextra; ++q) n.X[q] += c->extra[(int64_t)c->nextra * i + q] * alpha * s->T;
      n.T = Tn;
      n.errT = errTn;
      n.nr = s->nr + 1;
      n.gflag |= e->gflag;
      out[k++] = n;
    }
  }
  return k;
}

static void adm_walk(orc_adm_ctx *c, int64_t g, uint32_t rem, const orc_adm_state *s0);

/* Entry m of group g composited next (m's bit already cleared from rem). */
static void adm_member(orc_adm_ctx *c, int64_t g, uint32_t rem, int m, const orc_adm_state *s) {
  orc_adm_state nx[2];
  int stop;
  const int k = adm_options(c, &c->seq[c->gstart[g] + m], s, nx, &stop);
  if (k + stop > 1) c->flags |= 1;
  if (stop) {
    if (++c->leaves > c->max_leaves) {
      c->flags |= 4;
      return;
    }
    adm_leaf(c, s);
  }
  for (int j = 0; j < k; ++j) adm_walk(c, g, rem, &nx[j]);
}

/* Composites, from state s0, the members of group g still in rem and then
 * every later group.  The members of a group may be composited in any order
 * in which each pair that is out of FP64 order has keys within 2 depth_ulps. */
static void adm_walk(orc_adm_ctx *c, int64_t g, uint32_t rem, const orc_adm_state *s0) {
  if (c->leaves > c->max_leaves) return;
  orc_adm_state s = *s0;
  for (;;) {
    while (rem == 0) {
      if (++g >= c->ngroups) {
        if (++c->leaves > c->max_leaves) {
          c->flags |= 4;
          return;
        }
        adm_leaf(c, &s);
        return;
      }
      const int64_t len = c->gstart[g + 1] - c->gstart[g];
      rem = len >= 32 ? 0xffffffffu : ((1u << len) - 1u);
    }
    const orc_adm_entry *grp = c->seq + c->gstart[g];
    int first = -1;
    for (int m = 0; m < 32; ++m) {
      if (!(rem & (1u << m))) continue;
      /* m may come next if every remaining member before it is within range */
      int ok = 1;
      for (int j = 0; j < m && ok; ++j)
        if ((rem & (1u << j)) && grp[m].bits - grp[j].bits > 2u * (uint32_t)c->depth_ulps) ok = 0;
      if (!ok) continue;
      if (first < 0) {
        first = m;
        continue;
      }
      c->flags |= 1;
      adm_member(c, g, rem & ~(1u << m), m, &s);
      if (c->leaves > c->max_leaves) return;
    }
    /* the first admissible member (the FP64 order) continues in this frame
     * along its last outcome */
    rem &= ~(1u << first);
    orc_adm_state nx[2];
    int stop;
    const int k = adm_options(c, &grp[first], &s, nx, &stop);
    if (k + stop > 1) c->flags |= 1;
    if (stop) {
      if (++c->leaves > c->max_leaves) {
        c->flags |= 4;
        return;
      }
      adm_leaf(c, &s);
    }
    if (k == 0) return;
    for (int j = 0; j + 1 < k; ++j) {
      adm_walk(c, g, rem, &nx[j]);
      if (c->leaves > c->max_leaves) return;
    }
    s = nx[k - 1];
  }
}

/* Admissible results at selected pixels (linear ids py * W + px) of one view.
 * P: from orc_preprocess_relaxed (or orc_preprocess with uncertain, rect_lo
 * and rect_hi set by the caller).  A Gaussian enters a pixel's list when it
 * is visible or uncertain (bit 1) and its rect_hi holds the pixel's tile; its
 * membership is uncertain unless it is visible, certain and inside rect_lo.
 * extra: optional [n][nextra] per-Gaussian values composited like colour
 * (nextra <= 64).  Outputs per pixel q: ncands[q] distinct results in
 * cands[q][max_cands][5 + nextra] (r, g, b, T, contributors, extra...), and
 * flags[q]: bit 1 some decision had two admissible outcomes, bit 2 a
 * composited entry's derivative is uncertain (alpha within its error of the
 * 0.99 clamp, or its colour clamp uncertain), bit 4 the walk ran out of its
 * budget (results incomplete).  Returns 0, or -1 on bad arguments or memory. */
typedef struct {
  int64_t tile, q;
} orc_pixq;

static int pixq_cmp(const void *pa, const void *pb) {
  const orc_pixq *a = pa, *b = pb;
  if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
  return (a->q > b->q) - (a->q < b->q);
}

int orc_render_pixels_admissible(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P,
                                 const orc_tol *tol, const double *extra, int32_t nextra, int64_t npix,
                                 const int64_t *pix, int32_t max_cands, double *cands, int32_t *ncands,
                                 int32_t *flags) {
  if (!P->uncertain || !P->rect_lo || !P->rect_hi || nextra < 0 || nextra > 64 || max_cands < 1) return -1;
  const int W = V->width, B = S->tile;
  const int gw = (W + B - 1) / B;
  const int nv = 5 + nextra;
  /* pixels grouped by tile, so each tile's list is gathered once */
  orc_pixq *qs = malloc(sizeof(orc_pixq) * (size_t)(npix > 0 ? npix : 1));
  int64_t *runs = malloc(sizeof(int64_t) * (size_t)(npix + 1));
  if (!qs || !runs) {
    free(qs);
    free(runs);
    return -1;
  }
  for (int64_t q = 0; q < npix; ++q) {
    const int px = (int)(pix[q] % W), py = (int)(pix[q] / W);
    qs[q].tile = (int64_t)(py / B) * gw + px / B;
    qs[q].q = q;
  }
  qsort(qs, (size_t)npix, sizeof(orc_pixq), pixq_cmp);
  int64_t nruns = 0;
  for (int64_t a = 0; a < npix; ++a)
    if (a == 0 || qs[a].tile != qs[a - 1].tile) runs[nruns++] = a;
  runs[nruns] = npix;
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t rix = 0; rix < nruns; ++rix) {
    const int64_t t = qs[runs[rix]].tile;
    const int tx = (int)(t % gw), ty = (int)(t / gw);
    /* the tile's list: every Gaussian some admissible outcome puts here */
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *r = P->rect_hi + 4 * i;
      if ((P->status[i] == 0 || (P->uncertain[i] & 1)) && tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) ++cnt;
    }
    orc_entry *list = malloc(sizeof(orc_entry) * (size_t)(cnt > 0 ? cnt : 1));
    orc_adm_entry *seq = malloc(sizeof(orc_adm_entry) * (size_t)(cnt > 0 ? cnt : 1));
    int64_t *gstart = malloc(sizeof(int64_t) * (size_t)(cnt + 2));
    if (!list || !seq || !gstart) {
      err = 1;
      free(list);
      free(seq);
      free(gstart);
      continue;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int32_t *r = P->rect_hi + 4 * i;
      if ((P->status[i] == 0 || (P->uncertain[i] & 1)) && tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) {
        orc_entry e = {P->depth_f32[i], i};
        list[k++] = e;
      }
    }
    qsort(list, (size_t)cnt, sizeof(orc_entry), entry_cmp);
    for (int64_t qq = runs[rix]; qq < runs[rix + 1]; ++qq) {
      const int64_t q = qs[qq].q;
      const int px = (int)(pix[q] % W), py = (int)(pix[q] / W);
      const double pxc = px + 0.5, pyc = py + 0.5;
      /* outcomes of every entry at this pixel; entries that are skipped
       * under every admissible outcome are left out */
      int64_t ns = 0;
      for (int64_t j = 0; j < cnt; ++j) {
        const int64_t i = list[j].idx;
        double power, aG, alpha, e;
        adm_alpha(P, tol, i, pxc, pyc, &power, &aG, &alpha, &e);
        const double gpu_lo = alpha * (1.0 - e), gpu_hi = alpha * (1.0 + e);
        int opts = 0;
        if (power > 0.0 || gpu_lo < 1.0 / 255.0) opts |= ORC_SKIP;
        if (gpu_hi >= 1.0 / 255.0) opts |= ORC_TAKE;
        const int32_t *rl = P->rect_lo + 4 * i;
        const int certain = P->status[i] == 0 && !(P->uncertain[i] & 1) && tx >= rl[0] && tx < rl[2] &&
                            ty >= rl[1] && ty < rl[3];
        if (!certain) opts |= ORC_SKIP;
        if (!(opts & ORC_TAKE)) continue;
        seq[ns].idx = i;
        seq[ns].bits = f32_bits(list[j].depth);
        seq[ns].opts = opts;
        seq[ns].alpha = alpha;
        seq[ns].err = e;
        seq[ns].gflag = fabs(aG - 0.99) <= 0.99 * e || (P->uncertain[i] & 2) ? 1 : 0;
        ++ns;
      }
      /* groups of consecutive entries whose keys lie within 2 depth_ulps */
      int64_t ng = 0;
      for (int64_t j = 0; j < ns; ++j)
        if (j == 0 || tol->depth_ulps <= 0 || seq[j].bits - seq[j - 1].bits > 2u * (uint32_t)tol->depth_ulps ||
            j - gstart[ng - 1] >= 20)
          gstart[ng++] = j;
      gstart[ng] = ns;
      orc_adm_ctx c;
      memset(&c, 0, sizeof c);
      c.P = P;
      c.S = S;
      c.extra = extra;
      c.nextra = extra ? nextra : 0;
      c.seq = seq;
      c.gstart = gstart;
      c.ngroups = ng;
      c.depth_ulps = tol->depth_ulps;
      c.eps_step = tol->eps_alpha;
      c.max_cands = max_cands;
      c.max_leaves = tol->max_leaves > 0 ? tol->max_leaves : 4096;
      c.cands = cands + (int64_t)q * max_cands * nv;
      orc_adm_state s0;
      memset(&s0, 0, sizeof s0);
      s0.T = 1.0;
      adm_walk(&c, -1, 0u, &s0);
      /* a group cut at 20 members leaves pairs across the cut unordered */
      for (int64_t gi = 1; gi < ng; ++gi)
        if (tol->depth_ulps > 0 && seq[gstart[gi]].bits - seq[gstart[gi] - 1].bits <= 2u * (uint32_t)tol->depth_ulps)
          c.flags |= 4;
      ncands[q] = c.ncands;
      flags[q] = c.flags;
    }
    free(list);
    free(seq);
    free(gstart);
  }
  free(qs);
  free(runs);
  return err ? -1 : 0;
}

/* ----------------------------------------------- auxiliary channels */

/* Per visible Gaussian: camera-space depth z of the sliced mean and the
 * image-plane displacement of the sliced mean over a time step dt (Sec. 8.1.3,
 * "emerged dynamics": the trajectory of mu_xyz|t projected between two
 * consecutive frames).  mu_xyz|t is linear in t with velocity
 * Sigma_{1:3,4} / Sigma_44, so the displaced camera-space centre is
 * pc + W v dt; the flow is pi(pc + W v dt) - pi(pc) with pi the pinhole
 * projection of Eq. 3, and 0 when the displaced centre is not in front of the
 * near plane.  aux[n][3] = (z, flow_u, flow_v); zeros for culled Gaussians
 * (with relax > 0 and P from orc_preprocess_relaxed at that relax, also for
 * the Gaussians it marks as possibly present). */
int orc_aux(const orc_params *Pp, const orc_view *V, const orc_settings *S, double flow_dt, double relax,
            const orc_proj *P, double *aux) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < Pp->n; ++i) {
    aux[3 * i + 0] = aux[3 * i + 1] = aux[3 * i + 2] = 0.0;
    /* P from orc_preprocess_relaxed with the same relax: a Gaussian culled
     * within the relaxation gets the values it would have if kept */
    const int maybe = relax > 0.0 && P->uncertain && (P->uncertain[i] & 1);
    if (P->status[i] != 0 && !maybe) continue;
    orc_ctx g;
    gauss_forward(Pp, i, V, S, &g, maybe ? relax : 0.0);
    const double *W = V->viewmat;
    double vel[3], pc2[3];
    for (int a = 0; a < 3; ++a) vel[a] = g.b[a] / g.c;
    for (int a = 0; a < 3; ++a)
      pc2[a] = g.pc[a] + (W[4 * a + 0] * vel[0] + W[4 * a + 1] * vel[1] + W[4 * a + 2] * vel[2]) * flow_dt;
    aux[3 * i + 0] = g.pc[2];
    if (pc2[2] > S->near_plane) {
      aux[3 * i + 1] = V->fx * pc2[0] / pc2[2] + V->cx - g.uv[0];
      aux[3 * i + 2] = V->fy * pc2[1] / pc2[2] + V->cy - g.uv[1];
    }
  }
  return 0;
}

/* Image plus auxiliary channels blended with the colour weights of Eq. 6
 * (w_i = alpha_i T_i): out_aux[4][H][W] = (depth sum w z, opacity 1 - T,
 * flow_u sum w f_u, flow_v sum w f_v). */
int orc_render_aux(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P, const double *aux,
                   double *img, double *T_out, double *out_aux, double *margin) {
  orc_tiles tl;
  if (build_tiles(V, S, n, P, &tl)) return -1;
  const int W = V->width, H = V->height, gw = (W + S->tile - 1) / S->tile;
  const int64_t HW = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int py = 0; py < H; ++py) {
    for (int px = 0; px < W; ++px) {
      const int64_t t = (int64_t)(py / S->tile) * gw + px / S->tile;
      const int64_t p = (int64_t)py * W + px;
      double out[3], x[3], T;
      composite_pixel(P, S, tl.ent + tl.off[t], tl.off[t + 1] - tl.off[t], px, py, out, &T, NULL,
                      margin ? &margin[p] : NULL, NULL, NULL, NULL, aux, x);
      for (int ch = 0; ch < 3; ++ch) img[ch * HW + p] = out[ch];
      if (T_out) T_out[p] = T;
      out_aux[p] = x[0];
      out_aux[HW + p] = 1.0 - T;
      out_aux[2 * HW + p] = x[1];
      out_aux[3 * HW + p] = x[2];
    }
  }
  free_tiles(&tl);
  return 0;
}

/* ------------------------------------------------ feature rendering */

/* Scale-gated feature of Gaussian i (Sec. 7, "Scale-gated features"):
 * f^s = S(s) (.) f with the gate vector S(s) given, normalised; the map is
 * rendered like colour in Eq. 6 with a zero background.  Returns |g|. */
static double gated_unit_feature(const double *f, const double *gate, int D, double *fhat) {
  double nn = 0.0;
  for (int c = 0; c < D; ++c) {
    fhat[c] = (gate ? gate[c] : 1.0) * f[c];
    nn += fhat[c] * fhat[c];
  }
  const double norm = sqrt(nn);
  for (int c = 0; c < D; ++c) fhat[c] = norm > 0.0 ? fhat[c] / norm : 0.0;
  return norm;
}

/* The normalised scale-gated feature of every Gaussian (gate NULL = all
 * ones): fhat[n][D]. */
void orc_gated_features(const double *feat, int64_t n, int D, const double *gate, double *fhat) {
  for (int64_t i = 0; i < n; ++i) gated_unit_feature(feat + (int64_t)D * i, gate, D, fhat + (int64_t)D * i);
}

/* out[D][H][W] = sum_i w_i fhat_i per pixel, w_i = alpha_i T_i of the colour
 * compositing (same skip and stop decisions). */
int orc_render_features(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P, const double *feat,
                        int D, const double *gate, double *out, double *margin) {
  orc_tiles tl;
  if (build_tiles(V, S, n, P, &tl)) return -1;
  const int W = V->width, H = V->height, gw = (W + S->tile - 1) / S->tile;
  const int64_t HW = (int64_t)W * H;
  int64_t maxlen = 1;
  for (int64_t t = 0; t < (int64_t)gw * ((H + S->tile - 1) / S->tile); ++t)
    if (tl.off[t + 1] - tl.off[t] > maxlen) maxlen = tl.off[t + 1] - tl.off[t];
  int err = 0;
#pragma omp parallel
  {
    orc_contrib *rec = malloc(sizeof(orc_contrib) * (size_t)maxlen);
    double *fhat = malloc(sizeof(double) * (size_t)D);
    if (!rec || !fhat) err = 1;
#pragma omp for schedule(dynamic, 1)
    for (int py = 0; py < H; ++py) {
      if (!rec || !fhat) continue;
      for (int px = 0; px < W; ++px) {
        const int64_t t = (int64_t)(py / S->tile) * gw + px / S->tile;
        const int64_t p = (int64_t)py * W + px;
        double rgb[3], T;
        int64_t nr = 0;
        composite_pixel(P, S, tl.ent + tl.off[t], tl.off[t + 1] - tl.off[t], px, py, rgb, &T, NULL,
                        margin ? &margin[p] : NULL, NULL, rec, &nr, NULL, NULL);
        for (int c = 0; c < D; ++c) out[c * HW + p] = 0.0;
        for (int64_t k = 0; k < nr; ++k) {
          gated_unit_feature(feat + (size_t)rec[k].idx * D, gate, D, fhat);
          for (int c = 0; c < D; ++c) out[c * HW + p] += rec[k].alpha * rec[k].T * fhat[c];
        }
      }
    }
    free(rec);
    free(fhat);
  }
  free_tiles(&tl);
  return err ? -1 : 0;
}

/* Reverse mode of orc_render_features with the geometry held fixed (the
 * features are trained on a pre-trained 4DGS): dL/dfhat_i = sum_p w_i dF(p);
 * with g = gate (.) f and fhat = g / |g|, dL/dg = (dL/dfhat - fhat (fhat .
 * dL/dfhat)) / |g|; dL/df = gate (.) dL/dg and dL/dgate = sum_i f_i (.) dL/dg_i
 * (both ADDED). */
int orc_render_features_backward(const orc_view *V, const orc_settings *S, int64_t n, const orc_proj *P,
                                 const double *feat, int D, const double *gate, const double *dF,
                                 double *g_feat, double *g_gate) {
  orc_tiles tl;
  if (build_tiles(V, S, n, P, &tl)) return -1;
  const int W = V->width, H = V->height, gw = (W + S->tile - 1) / S->tile;
  const int64_t HW = (int64_t)W * H;
  int64_t maxlen = 1;
  for (int64_t t = 0; t < (int64_t)gw * ((H + S->tile - 1) / S->tile); ++t)
    if (tl.off[t + 1] - tl.off[t] > maxlen) maxlen = tl.off[t + 1] - tl.off[t];
  double *gfhat = calloc((size_t)n * D + 1, sizeof(double));
  orc_contrib *rec = malloc(sizeof(orc_contrib) * (size_t)maxlen);
  double *fhat = malloc(sizeof(double) * (size_t)D + 1);
  if (!gfhat || !rec || !fhat) return -1;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const int64_t t = (int64_t)(py / S->tile) * gw + px / S->tile;
      const int64_t p = (int64_t)py * W + px;
      double rgb[3], T;
      int64_t nr = 0;
      composite_pixel(P, S, tl.ent + tl.off[t], tl.off[t + 1] - tl.off[t], px, py, rgb, &T, NULL, NULL, NULL,
                      rec, &nr, NULL, NULL);
      for (int64_t k = 0; k < nr; ++k)
        for (int c = 0; c < D; ++c) gfhat[(size_t)rec[k].idx * D + c] += rec[k].alpha * rec[k].T * dF[c * HW + p];
    }
  for (int64_t i = 0; i < n; ++i) {
    if (P->status[i] != 0) continue;
    const double norm = gated_unit_feature(feat + (size_t)i * D, gate, D, fhat);
    if (!(norm > 0.0)) continue;
    double dot = 0.0;
    for (int c = 0; c < D; ++c) dot += fhat[c] * gfhat[(size_t)i * D + c];
    for (int c = 0; c < D; ++c) {
      const double dg = (gfhat[(size_t)i * D + c] - fhat[c] * dot) / norm;
      g_feat[(size_t)i * D + c] += (gate ? gate[c] : 1.0) * dg;
      if (g_gate) g_gate[c] += feat[(size_t)i * D + c] * dg;
    }
  }
  free(gfhat);
  free(rec);
  free(fhat);
  free_tiles(&tl);
  return 0;
}

/* ------------------------------------------------------------ adjoint */

/* Reverse-mode derivative of one pixel's colour C (RGB) with respect to the
 * per-Gaussian alpha inputs.  With T_i = prod_{j<i} (1 - alpha_j) and
 * C = sum_i c_i alpha_i T_i + T_final bg:
 *   dC/dc_i     = alpha_i T_i
 *   dC/dalpha_i = c_i T_i - (sum_{j>i} c_j alpha_j T_j + T_final bg) / (1 - alpha_i)
 * and alpha = min(0.99, a G), G = exp(power), power = -1/2 d^T Q d. */
/* With gX != NULL also the depth channel D = sum_i z_i alpha_i T_i and the
 * opacity O = 1 - T_final = sum_i alpha_i T_i (gX = dL/dD, dL/dO): the same
 * rule with x_i = z_i, resp. 1, and a zero background; dD/dz_i = alpha_i T_i. */
static void pixel_adjoint(const orc_proj *P, const orc_settings *S, const orc_contrib *rec,
                          int64_t nr, double T_final, const double gC[3], const double *gX, orc_grads *out) {
  double rest[3], restD = 0.0, restO = 0.0;
  for (int ch = 0; ch < 3; ++ch) rest[ch] = T_final * S->bg[ch];
  for (int64_t k = nr - 1; k >= 0; --k) {
    const orc_contrib *e = &rec[k];
    const int64_t i = e->idx;
    const double *c = P->rgb + 3 * i;
    double g_alpha = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      out->g_rgb[3 * i + ch] += gC[ch] * e->alpha * e->T;
      g_alpha += gC[ch] * (c[ch] * e->T - rest[ch] / (1.0 - e->alpha));
    }
    for (int ch = 0; ch < 3; ++ch) rest[ch] += c[ch] * e->alpha * e->T;
    if (gX) {
      const double z = P->depth[i];
      out->g_z[i] += gX[0] * e->alpha * e->T;
      g_alpha += gX[0] * (z * e->T - restD / (1.0 - e->alpha)) + gX[1] * (e->T - restO / (1.0 - e->alpha));
      restD += z * e->alpha * e->T;
      restO += e->alpha * e->T;
    }
    if (e->clamped) continue; /* min(0.99, .) is locally constant */
    const double a = P->a_eff[i];
    out->g_a[i] += g_alpha * e->G;
    const double g_pow = g_alpha * a * e->G;
    const double A = P->conic[3 * i + 0], B = P->conic[3 * i + 1], Cc = P->conic[3 * i + 2];
    out->g_conic[3 * i + 0] += g_pow * (-0.5 * e->dx * e->dx);
    out->g_conic[3 * i + 1] += g_pow * (-e->dx * e->dy);
    out->g_conic[3 * i + 2] += g_pow * (-0.5 * e->dy * e->dy);
    out->g_uv[2 * i + 0] += g_pow * (-(A * e->dx + B * e->dy));
    out->g_uv[2 * i + 1] += g_pow * (-(Cc * e->dy + B * e->dx));
  }
}

/* Adjoint of the per-Gaussian forward chain, from dL/d(u, v, A, B, C, a,
 * rgb) back to the raw parameters. */
static void gauss_adjoint(const orc_params *Pp, int64_t i, const orc_view *V, const orc_settings *S,
                          const orc_ctx *g, const double g_uv[2], const double g_conic[3],
                          double g_a, const double g_rgb[3], double g_z, orc_grads *out) {
  const int nlm = (g->L + 1) * (g->L + 1);
  const double *sh = Pp->sh + (size_t)i * g->K * 3;
  double g_mu3[3] = {0, 0, 0}, g_dt = 0.0, g_pc[3] = {0, 0, 0};

  /* Colour: rgb = max(0, raw + 0.5), raw = sum_n sum_lm c cos_n Y_lm. */
  double graw[3];
  for (int ch = 0; ch < 3; ++ch) graw[ch] = (g->raw[ch] + 0.5 > 0.0) ? g_rgb[ch] : 0.0;
  double gY[(ORC_MAX_L + 1) * (ORC_MAX_L + 1)] = {0};
  for (int nn = 0; nn <= g->NT; ++nn)
    for (int lm = 0; lm < nlm; ++lm)
      for (int ch = 0; ch < 3; ++ch) {
        const int k = (nn * nlm + lm) * 3 + ch;
        out->sh[(size_t)i * g->K * 3 + k] += graw[ch] * g->cosn[nn] * g->Y[lm];
        gY[lm] += graw[ch] * sh[k] * g->cosn[nn];
        g_dt += graw[ch] * sh[k] * g->Y[lm] * (-g->sinn[nn]) * (2.0 * ORC_PI * nn / S->period);
      }
  {
    /* dY/dw through theta = acos(w_z/|w|), phi = atan2(w_y, w_x). */
    double Y[16], dth[16], dph[16];
    const double theta = acos(dmax(-1.0, dmin(1.0, g->dir[2])));
    const double phi = atan2(g->dir[1], g->dir[0]);
    real_sh(g->L, theta, phi, Y, dth, dph);
    const double st = sin(theta), ct = cos(theta), sp = sin(phi), cp = cos(phi);
    const double gth[3] = {ct * cp / g->rw, ct * sp / g->rw, -st / g->rw};
    const double gph[3] = {-sp / (g->rw * st), cp / (g->rw * st), 0.0};
    for (int lm = 0; lm < nlm; ++lm)
      for (int a = 0; a < 3; ++a) g_mu3[a] += gY[lm] * (dth[lm] * gth[a] + dph[lm] * gph[a]);
  }
  /* Opacity: a = sigmoid(logit) p_t. */
  const double g_sig = g_a * g->pt;
  double g_pt = g_a * g->sig;
  out->opacity_logit[i] += g_sig * g->sig * (1.0 - g->sig);
  /* Straight-through mask gradient (Sec. 4.3): dL/dM_hat = sum_k dL/ds_hat_k s_k
   * + dL/dalpha_hat alpha at M_hat = 1, and dM_hat/dm = M (1 - M). */
  double g_mhat = g_sig * g->sig;

  /* Projected centre, Eq. 3. */
  const double x = g->pc[0], y = g->pc[1], z = g->pc[2];
  g_pc[0] += g_uv[0] * V->fx / z;
  g_pc[1] += g_uv[1] * V->fy / z;
  g_pc[2] += -g_uv[0] * V->fx * x / (z * z) - g_uv[1] * V->fy * y / (z * z);
  g_pc[2] += g_z; /* depth channel: z is the camera-space depth itself */

  /* Conic = inverse(cov2): dL/dcov2 = -Q GQ Q, with GQ the full-matrix
   * gradient of Q = [[A, B], [B, C]] (B enters twice). */
  const double Q[4] = {g->conic[0], g->conic[1], g->conic[1], g->conic[2]};
  const double GQ[4] = {g_conic[0], 0.5 * g_conic[1], 0.5 * g_conic[1], g_conic[2]};
  double tmp[4], G2[4];
  for (int r = 0; r < 2; ++r)
    for (int col = 0; col < 2; ++col) tmp[2 * r + col] = Q[2 * r + 0] * GQ[0 * 2 + col] + Q[2 * r + 1] * GQ[1 * 2 + col];
  for (int r = 0; r < 2; ++r)
    for (int col = 0; col < 2; ++col)
      G2[2 * r + col] = -(tmp[2 * r + 0] * Q[0 * 2 + col] + tmp[2 * r + 1] * Q[1 * 2 + col]);

  /* Eq. 4: cov2 = M cov3 M^T + dil I, M = J W. */
  double g_cov3[9], g_M[6], g_J[6];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int r = 0; r < 2; ++r)
        for (int col = 0; col < 2; ++col) acc += g->M[3 * r + a] * G2[2 * r + col] * g->M[3 * col + b];
      g_cov3[3 * a + b] = acc;
    }
  for (int r = 0; r < 2; ++r)
    for (int a = 0; a < 3; ++a) {
      double acc = 0.0;
      for (int col = 0; col < 2; ++col)
        for (int b = 0; b < 3; ++b) acc += G2[2 * r + col] * g->M[3 * col + b] * g->cov3[3 * b + a];
      g_M[3 * r + a] = 2.0 * acc;
    }
  const double *W = V->viewmat;
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int col = 0; col < 3; ++col) acc += g_M[3 * r + col] * W[4 * k + col];
      g_J[3 * r + k] = acc;
    }
  g_pc[0] += g_J[2] * (-V->fx / (z * z));
  g_pc[1] += g_J[5] * (-V->fy / (z * z));
  g_pc[2] += g_J[0] * (-V->fx / (z * z)) + g_J[2] * (2.0 * V->fx * x / (z * z * z)) +
             g_J[4] * (-V->fy / (z * z)) + g_J[5] * (2.0 * V->fy * y / (z * z * z));

  /* pc = W mu3 + T. */
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) g_mu3[a] += W[4 * k + a] * g_pc[k];

  /* Conditional Gaussian: mu3 = m + b dt / c, cov3 = Sxx - b b^T / c. */
  double g_b[3], g_c = 0.0, mub = 0.0, bgb = 0.0;
  for (int a = 0; a < 3; ++a) mub += g_mu3[a] * g->b[a];
  for (int a = 0; a < 3; ++a) {
    double acc = 0.0;
    for (int k = 0; k < 3; ++k) acc += (g_cov3[3 * a + k] + g_cov3[3 * k + a]) * g->b[k];
    g_b[a] = g_mu3[a] * g->dt / g->c - acc / g->c;
  }
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) bgb += g->b[a] * g_cov3[3 * a + k] * g->b[k];
  g_dt += mub / g->c;
  g_c += -mub * g->dt / (g->c * g->c) + bgb / (g->c * g->c);
  /* Marginal p_t = exp(-dt^2 / (2 c)). */
  g_dt += g_pt * g->pt * (-g->dt / g->c);
  g_c += g_pt * g->pt * (0.5 * g->dt * g->dt / (g->c * g->c));
  for (int a = 0; a < 3; ++a) out->mean[4 * i + a] += g_mu3[a];
  out->mean[4 * i + 3] += -g_dt;

  /* Symmetric gradient of Sigma: GS_ij = g_cov3_ij (i,j<3), GS_i3 = GS_3i =
   * g_b_i / 2, GS_33 = g_c.  Sigma = R D R^T gives dL/dR = 2 GS R D and
   * dL/d(s_k^2) = (R^T GS R)_kk. */
  double GS[16];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) GS[4 * a + b] = 0.5 * (g_cov3[3 * a + b] + g_cov3[3 * b + a]);
  for (int a = 0; a < 3; ++a) {
    GS[4 * a + 3] = 0.5 * g_b[a];
    GS[4 * 3 + a] = 0.5 * g_b[a];
  }
  GS[15] = g_c;
  double gR[16];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 4; ++k) {
      double acc = 0.0;
      for (int b = 0; b < 4; ++b) acc += GS[4 * a + b] * g->R[4 * b + k];
      gR[4 * a + k] = 2.0 * acc * g->s[k] * g->s[k];
    }
  for (int k = 0; k < 4; ++k) {
    double acc = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) acc += g->R[4 * a + k] * GS[4 * a + b] * g->R[4 * b + k];
    out->log_scale[4 * i + k] += acc * 2.0 * g->s[k] * g->s[k];
    g_mhat += acc * 2.0 * g->s[k] * g->s[k]; /* dL/ds_k s_k = dL/dlog s_k */
  }
  if (Pp->mask_logit && out->mask_logit) out->mask_logit[i] += g_mhat * g->mask * (1.0 - g->mask);
  /* R = Lm Rm: dL/dLm = gR Rm^T, dL/dRm = Lm^T gR. */
  double gL[16], gRr[16];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double acc1 = 0.0, acc2 = 0.0;
      for (int k = 0; k < 4; ++k) {
        acc1 += gR[4 * a + k] * g->Rm[4 * b + k];
        acc2 += g->Lm[4 * k + a] * gR[4 * k + b];
      }
      gL[4 * a + b] = acc1;
      gRr[4 * a + b] = acc2;
    }
  /* Entries of L(q) and R(q) are +-q components; collect by pattern. */
  double gqln[4], gqrn[4];
  gqln[0] = gL[0] + gL[5] + gL[10] + gL[15];
  gqln[1] = -gL[1] + gL[4] - gL[11] + gL[14];
  gqln[2] = -gL[2] + gL[7] + gL[8] - gL[13];
  gqln[3] = -gL[3] - gL[6] + gL[9] + gL[12];
  gqrn[0] = gRr[0] + gRr[5] + gRr[10] + gRr[15];
  gqrn[1] = -gRr[1] + gRr[4] + gRr[11] - gRr[14];
  gqrn[2] = -gRr[2] - gRr[7] + gRr[8] + gRr[13];
  gqrn[3] = -gRr[3] + gRr[6] - gRr[9] + gRr[12];
  /* q_hat = q / |q|: dL/dq = (g - q_hat (q_hat . g)) / |q|. */
  double dl = 0.0, dr = 0.0;
  for (int k = 0; k < 4; ++k) {
    dl += g->qln[k] * gqln[k];
    dr += g->qrn[k] * gqrn[k];
  }
  for (int k = 0; k < 4; ++k) {
    out->q_l[4 * i + k] += (gqln[k] - g->qln[k] * dl) / g->nql;
    out->q_r[4 * i + k] += (gqrn[k] - g->qrn[k] * dr) / g->nqr;
  }
}

/* dL/d(parameters) for a loss whose gradient with respect to the rendered
 * image is dimg ([3][H][W]).  Per-Gaussian 2D gradients are also returned. */
int orc_render_backward(const orc_params *Pp, const orc_view *V, const orc_settings *S,
                        const orc_proj *P, const double *dimg, orc_grads *out) {
  const int64_t n = Pp->n;
  orc_tiles tl;
  if (build_tiles(V, S, n, P, &tl)) return -1;
  const int W = V->width, H = V->height, gw = (W + S->tile - 1) / S->tile;
  const int64_t HW = (int64_t)W * H;
  int64_t maxlen = 1;
  for (int64_t t = 0; t < (int64_t)gw * ((H + S->tile - 1) / S->tile); ++t)
    if (tl.off[t + 1] - tl.off[t] > maxlen) maxlen = tl.off[t + 1] - tl.off[t];
  orc_contrib *rec = malloc(sizeof(orc_contrib) * (size_t)maxlen);
  if (!rec) return -1;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const int64_t t = (int64_t)(py / S->tile) * gw + px / S->tile;
      const int64_t p = (int64_t)py * W + px;
      const double gC[3] = {dimg[p], dimg[HW + p], dimg[2 * HW + p]};
      if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0) continue;
      double outc[3], T;
      int64_t nr = 0;
      composite_pixel(P, S, tl.ent + tl.off[t], tl.off[t + 1] - tl.off[t], px, py, outc, &T, NULL, NULL,
                      NULL, rec, &nr, NULL, NULL);
      pixel_adjoint(P, S, rec, nr, T, gC, NULL, out);
    }
  free(rec);
  free_tiles(&tl);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (P->status[i] != 0) continue;
    orc_ctx g;
    gauss_forward(Pp, i, V, S, &g, 0.0);
    gauss_adjoint(Pp, i, V, S, &g, out->g_uv + 2 * i, out->g_conic + 3 * i, out->g_a[i],
                  out->g_rgb + 3 * i, out->g_z[i], out);
  }
  return 0;
}

/* dL/d(parameters) for a loss on the image and the depth and opacity
 * channels of orc_render_aux: dimg [3][H][W], daux [4][H][W] (depth,
 * opacity, flow_u, flow_v; the flow planes are not differentiated and must
 * be zero). */
int orc_render_aux_backward(const orc_params *Pp, const orc_view *V, const orc_settings *S,
                            const orc_proj *P, const double *dimg, const double *daux, orc_grads *out) {
  const int64_t n = Pp->n;
  orc_tiles tl;
  if (build_tiles(V, S, n, P, &tl)) return -1;
  const int W = V->width, H = V->height, gw = (W + S->tile - 1) / S->tile;
  const int64_t HW = (int64_t)W * H;
  for (int64_t p = 0; p < HW; ++p)
    if (daux[2 * HW + p] != 0.0 || daux[3 * HW + p] != 0.0) {
      free_tiles(&tl);
      return -2;
    }
  int64_t maxlen = 1;
  for (int64_t t = 0; t < (int64_t)gw * ((H + S->tile - 1) / S->tile); ++t)
    if (tl.off[t + 1] - tl.off[t] > maxlen) maxlen = tl.off[t + 1] - tl.off[t];
  orc_contrib *rec = malloc(sizeof(orc_contrib) * (size_t)maxlen);
  if (!rec) return -1;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      const int64_t t = (int64_t)(py / S->tile) * gw + px / S->tile;
      const int64_t p = (int64_t)py * W + px;
      const double gC[3] = {dimg[p], dimg[HW + p], dimg[2 * HW + p]};
      const double gX[2] = {daux[p], daux[HW + p]};
      if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0 && gX[0] == 0.0 && gX[1] == 0.0) continue;
      double outc[3], T;
      int64_t nr = 0;
      composite_pixel(P, S, tl.ent + tl.off[t], tl.off[t + 1] - tl.off[t], px, py, outc, &T, NULL, NULL,
                      NULL, rec, &nr, NULL, NULL);
      pixel_adjoint(P, S, rec, nr, T, gC, gX, out);
    }
  free(rec);
  free_tiles(&tl);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (P->status[i] != 0) continue;
    orc_ctx g;
    gauss_forward(Pp, i, V, S, &g, 0.0);
    gauss_adjoint(Pp, i, V, S, &g, out->g_uv + 2 * i, out->g_conic + 3 * i, out->g_a[i],
                  out->g_rgb + 3 * i, out->g_z[i], out);
  }
  return 0;
}

/* Adjoint of the per-Gaussian chain alone, from given 2D gradients (used to
 * check the preprocess adjoint separately from compositing). */
int orc_preprocess_backward(const orc_params *Pp, const orc_view *V, const orc_settings *S,
                            const double *g_uv, const double *g_conic, const double *g_a,
                            const double *g_rgb, orc_grads *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < Pp->n; ++i) {
    orc_ctx g;
    gauss_forward(Pp, i, V, S, &g, 0.0);
    if (g.status != 0) continue;
    gauss_adjoint(Pp, i, V, S, &g, g_uv + 2 * i, g_conic + 3 * i, g_a[i], g_rgb + 3 * i, 0.0, out);
  }
  return 0;
}

/* ------------------------------------------------ densification */

/* Split sampling in spacetime (Sec. 3.3, "Densification in spacetime";
 * Sec. 8.1.3, "More ablations": the complete 4D Gaussian is the PDF of the
 * new positions).  A draw from N(mu, Sigma) with Sigma = R S S^T R^T is
 * mu + R S eps for a standard normal eps (R S (R S)^T = Sigma).  Child
 * j * K + c of Gaussian idx[j]: that draw for eps[j][c]; log-scales reduced
 * by log(shrink); rotation, opacity and colour coefficients copied.  Output
 * arrays have m K rows; the SH row length is K3 doubles. */
int orc_split_sample(const orc_params *Pp, const int64_t *idx, int64_t m, int K, const double *eps,
                     double shrink, int64_t K3, double *o_mean, double *o_log_scale, double *o_q_l,
                     double *o_q_r, double *o_logit, double *o_sh) {
  for (int64_t j = 0; j < m; ++j) {
    const int64_t i = idx[j];
    if (i < 0 || i >= Pp->n) return -1;
    double ql[4], qr[4], nl = 0.0, nr = 0.0, Lm[16], Rm[16], R[16], s[4];
    for (int k = 0; k < 4; ++k) {
      nl += Pp->q_l[4 * i + k] * Pp->q_l[4 * i + k];
      nr += Pp->q_r[4 * i + k] * Pp->q_r[4 * i + k];
      s[k] = exp(Pp->log_scale[4 * i + k]);
    }
    for (int k = 0; k < 4; ++k) {
      ql[k] = Pp->q_l[4 * i + k] / sqrt(nl);
      qr[k] = Pp->q_r[4 * i + k] / sqrt(nr);
    }
    left_matrix(ql, Lm);
    right_matrix(qr, Rm);
    mat4_mul(Lm, Rm, R);
    for (int c = 0; c < K; ++c) {
      const int64_t o = j * K + c;
      const double *e = eps + 4 * o;
      for (int a = 0; a < 4; ++a) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += R[4 * a + k] * s[k] * e[k];
        o_mean[4 * o + a] = Pp->mean[4 * i + a] + acc;
        o_log_scale[4 * o + a] = Pp->log_scale[4 * i + a] - log(shrink);
        o_q_l[4 * o + a] = Pp->q_l[4 * i + a];
        o_q_r[4 * o + a] = Pp->q_r[4 * i + a];
      }
      o_logit[o] = Pp->opacity_logit[i];
      for (int64_t k = 0; k < K3; ++k) o_sh[K3 * o + k] = Pp->sh[K3 * i + k];
    }
  }
  return 0;
}

/* ------------------------------------------------- pieces for the pins */

/* R = L(q_l) R(q_r) for unit-normalised q_l, q_r (row-major 4x4). */
void orc_rotation(const double *q_l, const double *q_r, double *R) {
  double ql[4], qr[4], Lm[16], Rm[16];
  double nl = 0.0, nr = 0.0;
  for (int k = 0; k < 4; ++k) {
    nl += q_l[k] * q_l[k];
    nr += q_r[k] * q_r[k];
  }
  nl = sqrt(nl);
  nr = sqrt(nr);
  for (int k = 0; k < 4; ++k) {
    ql[k] = q_l[k] / nl;
    qr[k] = q_r[k] / nr;
  }
  left_matrix(ql, Lm);
  right_matrix(qr, Rm);
  mat4_mul(Lm, Rm, R);
}

/* Real SH values Y_lm for a unit direction (x, y, z). */
void orc_real_sh(int L, const double *dir, double *Y) {
  const double theta = acos(dmax(-1.0, dmin(1.0, dir[2])));
  const double phi = atan2(dir[1], dir[0]);
  real_sh(L, theta, phi, Y, NULL, NULL);
}

/* Instance list of a tile-binned view, as the paper's tile rasterizer sorts
 * it: one (tile, Gaussian) pair per tile of each visible Gaussian's rect,
 * key = (tile << 32) | bits(depth_f32), sorted by (tile, depth, index).
 * ranges[t] = [start, end) of tile t. Returns the instance count, or -1 if
 * it exceeds cap. */
typedef struct {
  int64_t tile;
  float depth;
  int64_t idx;
} orc_inst;

static int inst_cmp(const void *pa, const void *pb) {
  const orc_inst *a = pa, *b = pb;
  if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
  if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

int64_t orc_sort_instances(int64_t n, const int32_t *rect, const float *depth, int32_t gw, int32_t gh, int64_t cap,
                           uint64_t *keys, int64_t *vals, int64_t *ranges) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *r = rect + 4 * i;
    if (r[2] > r[0] && r[3] > r[1]) m += (int64_t)(r[2] - r[0]) * (r[3] - r[1]);
  }
  if (m > cap) return -1;
  orc_inst *a = malloc(sizeof(orc_inst) * (size_t)(m > 0 ? m : 1));
  if (!a) return -1;
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *r = rect + 4 * i;
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) {
        a[k].tile = (int64_t)ty * gw + tx;
        a[k].depth = depth[i];
        a[k].idx = i;
        ++k;
      }
  }
  /* (tile, depth, index) is a total order, so qsort's lack of stability is
   * irrelevant. */
  qsort(a, (size_t)m, sizeof(orc_inst), inst_cmp);
  for (int64_t t = 0; t < (int64_t)gw * gh; ++t) {
    ranges[2 * t] = 0;
    ranges[2 * t + 1] = 0;
  }
  for (int64_t j = 0; j < m; ++j) {
    keys[j] = ((uint64_t)a[j].tile << 32) | f32_bits(a[j].depth);
    vals[j] = a[j].idx;
    if (j == 0 || a[j].tile != a[j - 1].tile) ranges[2 * a[j].tile] = j;
    ranges[2 * a[j].tile + 1] = j + 1;
  }
  free(a);
  return m;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel regions (timing on a given core count). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
