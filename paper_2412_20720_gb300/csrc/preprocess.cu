// Per-Gaussian stage of the 4D Gaussian render path and its adjoint.
//
// Forward (Sec. 3.2 of "4D Gaussian Splatting", arXiv 2412.20720; Sec. 3.1,
// Eqs. 3-4; Sec. 8.1.1 temporal filter): one thread per (view, Gaussian) of a
// logical block; persistent blocks take logical blocks by ticket, and the
// visible pairs are compacted in (view, Gaussian) order by a block scan plus
// a decoupled look-back over the tickets, so slot numbering is deterministic
// whatever the grid.
//
// Numerics: the conditional covariance is evaluated in factored form.  With
// A = R_{1:3,:} diag(s), v = diag(s) R_{4,:}^T, c = |v|^2 = Sigma_44 and
// u = v / sqrt(c), the Schur complement
//   Sigma_xyz|t = Sigma_xyz - Sigma_x4 Sigma_4x / Sigma_44 = G G^T,
//   G = A (I - u u^T),
// and the conditional mean is mu_xyz + (A u) (t - mu_t) / sqrt(c).  The 2D
// covariance is then H H^T + dilation I with H = J W G (2x4), whose
// determinant follows from Cauchy-Binet as a sum of squares.  This avoids the
// cancellation of the plain Schur formula in FP32 for Gaussians whose large
// temporal axis is rotated into space; it is the same quantity (the FP64
// oracle uses the plain formula).
#include <math.h>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {

struct PreArgs {
  const float4 *mean, *log_scale, *q_l, *q_r;
  const float *logit, *sh;
  const float *mask_logit;  // optional significance mask
  float mask_threshold;
  int32_t n, t_order, k3;
  float period_inv, near_plane, dilation, p_t_min;
  int32_t nviews, blocks_per_view;
  int64_t vis_cap;
  uint32_t *counters;
  uint64_t *lb;
  float4 *rec_geom, *rec_color;
  float *rec_blue, *rec_tau;
  int4 *rec_meta;
  uint32_t *depth_key;
};

struct BwdArgs {
  const float4 *mean, *log_scale, *q_l, *q_r;
  const float *logit, *sh;
  const float *mask_logit;  // optional significance mask
  float *g_mask;            // optional dL/dm
  int32_t n, nviews, t_order, k3;
  float period_inv, near_plane, dilation, p_t_min;
  int64_t vis_cap;
  const uint32_t *counters;
  const int4 *rec_meta;
  const float4 *slot_grad;
  float4 *g_mean, *g_log_scale, *g_q_l, *g_q_r;
  float *g_logit, *g_sh;
  float4 *densify_stats;  // optional
};

constexpr float kTwoPi = 6.283185307179586f;

// Real orthonormal spherical harmonics with the Condon-Shortley phase,
// Y_lm at a unit direction (x, y, z), index l*l + l + m.  The polynomials
// follow from Y_lm = sqrt(2) K_l^|m| P_l^|m|(z) {cos, sin}(|m| phi) with
// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), sin^m(theta) {cos, sin}(m phi) =
// {Re, Im}(x + i y)^m and the associated Legendre polynomials of degree <= 3.
template <int L>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
  Y[0] = 0.28209479177387814f;
  if (L >= 1) {
    Y[1] = -0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = -0.4886025119029199f * x;
  }
  if (L >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    if (L >= 3) {
      Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
      Y[10] = 2.890611442640554f * x * y * z;
      Y[11] = -0.4570457994644658f * y * (5.0f * zz - 1.0f);
      Y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
      Y[13] = -0.4570457994644658f * x * (5.0f * zz - 1.0f);
      Y[14] = 1.445305721320277f * z * (xx - yy);
      Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
    }
  }
}

// Adds sum_lm gY[lm] * grad(Y_lm)(x, y, z) (gradient of the polynomials above
// in R^3; the radial part is projected out by the caller).
template <int L>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float *gY, float *g) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (L >= 1) {
    const float c1 = 0.4886025119029199f;
    gy -= c1 * gY[1];
    gz += c1 * gY[2];
    gx -= c1 * gY[3];
  }
  if (L >= 2) {
    const float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    gx += c2a * y * gY[4];
    gy += c2a * x * gY[4];
    gy -= c2a * z * gY[5];
    gz -= c2a * y * gY[5];
    gz += 6.0f * c2b * z * gY[6];
    gx -= c2a * z * gY[7];
    gz -= c2a * x * gY[7];
    gx += 2.0f * c2c * x * gY[8];
    gy -= 2.0f * c2c * y * gY[8];
    if (L >= 3) {
      const float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f,
                  c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
      const float xx = x * x, yy = y * y, zz = z * z;
      gx -= 6.0f * c3a * x * y * gY[9];
      gy -= c3a * (3.0f * xx - 3.0f * yy) * gY[9];
      gx += c3b * y * z * gY[10];
      gy += c3b * x * z * gY[10];
      gz += c3b * x * y * gY[10];
      gy -= c3c * (5.0f * zz - 1.0f) * gY[11];
      gz -= 10.0f * c3c * y * z * gY[11];
      gz += c3d * (15.0f * zz - 3.0f) * gY[12];
      gx -= c3c * (5.0f * zz - 1.0f) * gY[13];
      gz -= 10.0f * c3c * x * z * gY[13];
      gx += 2.0f * c3e * x * z * gY[14];
      gy -= 2.0f * c3e * y * z * gY[14];
      gz += c3e * (xx - yy) * gY[14];
      gx -= c3a * (3.0f * xx - 3.0f * yy) * gY[15];
      gy += 6.0f * c3a * x * y * gY[15];
    }
  }
  g[0] += gx;
  g[1] += gy;
  g[2] += gz;
}

__device__ __forceinline__ bool finite4(float4 v) {
  return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

// Everything the forward chain computes for one (Gaussian, view), kept in
// registers so the adjoint can reuse it.
struct Chain {
  float m[4], s[4], sig;
  float ql[4], qr[4], nql, nqr;  // normalised quaternions and the raw norms
  float R[4][4];
  float v[4], c, sqc, u[4];
  float B[3][4], Bu[3], G[3][4];
  float dt, pt;
  float mu[3], pc[3], iz;
  float M[2][3], H[2][4];
  float Sa, Sb, Sd, det;  // 2D covariance [[Sa, Sb], [Sb, Sd]]
  float conA, conB, conC; // its inverse
  float uv[2];
  int32_t rect[4];
  float dir[3], rw;
  float cn[FGS4D_MAX_T_ORDER + 1], sn[FGS4D_MAX_T_ORDER + 1];
  float raw[3], rgb[3];
  float a;
};

template <int L>
__device__ __forceinline__ bool forward_chain(int32_t i, const float4 *__restrict__ mean,
                                              const float4 *__restrict__ log_scale, const float4 *__restrict__ q_l,
                                              const float4 *__restrict__ q_r, const float *__restrict__ logit,
                                              const float *__restrict__ sh, int32_t t_order, int32_t k3,
                                              float period_inv, float near_plane, float dilation, float p_t_min,
                                              const PreView &cam, Chain &h) {
  const float4 m = __ldg(&mean[i]);
  const float4 ls = __ldg(&log_scale[i]);
  const float4 a4 = __ldg(&q_l[i]);
  const float4 b4 = __ldg(&q_r[i]);
  const float lg = __ldg(&logit[i]);
  if (!finite4(m) || !finite4(ls) || !finite4(a4) || !finite4(b4) || !isfinite(lg)) return false;
  h.m[0] = m.x; h.m[1] = m.y; h.m[2] = m.z; h.m[3] = m.w;
  h.s[0] = expf(ls.x); h.s[1] = expf(ls.y); h.s[2] = expf(ls.z); h.s[3] = expf(ls.w);
  h.sig = 1.0f / (1.0f + expf(-lg));
  h.nql = sqrtf(a4.x * a4.x + a4.y * a4.y + a4.z * a4.z + a4.w * a4.w);
  h.nqr = sqrtf(b4.x * b4.x + b4.y * b4.y + b4.z * b4.z + b4.w * b4.w);
  if (!(h.nql > 0.0f) || !(h.nqr > 0.0f)) return false;
  const float il = 1.0f / h.nql, ir = 1.0f / h.nqr;
  const float a = a4.x * il, b = a4.y * il, c = a4.z * il, d = a4.w * il;
  const float p = b4.x * ir, q = b4.y * ir, r = b4.z * ir, s = b4.w * ir;
  h.ql[0] = a; h.ql[1] = b; h.ql[2] = c; h.ql[3] = d;
  h.qr[0] = p; h.qr[1] = q; h.qr[2] = r; h.qr[3] = s;
  // R = L(q_l) R(q_r) (Sec. 3.2).
  const float Lm[4][4] = {{a, -b, -c, -d}, {b, a, -d, c}, {c, d, a, -b}, {d, -c, b, a}};
  const float Rm[4][4] = {{p, -q, -r, -s}, {q, p, s, -r}, {r, -s, p, q}, {s, r, -q, p}};
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
      h.R[x][y] = Lm[x][0] * Rm[0][y] + Lm[x][1] * Rm[1][y] + Lm[x][2] * Rm[2][y] + Lm[x][3] * Rm[3][y];
  // Marginal p(t) with Sigma_44 = |diag(s) R_4^T|^2 and the temporal filter.
#pragma unroll
  for (int k = 0; k < 4; ++k) h.v[k] = h.R[3][k] * h.s[k];
  h.c = h.v[0] * h.v[0] + h.v[1] * h.v[1] + h.v[2] * h.v[2] + h.v[3] * h.v[3];
  h.dt = cam.t - h.m[3];
  h.pt = expf(-0.5f * h.dt * h.dt / h.c);
  if (!(h.pt >= p_t_min)) return false;
  // Conditional Gaussian at t in factored form.
  h.sqc = sqrtf(h.c);
  const float isq = 1.0f / h.sqc;
#pragma unroll
  for (int k = 0; k < 4; ++k) h.u[k] = h.v[k] * isq;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
#pragma unroll
    for (int k = 0; k < 4; ++k) h.B[x][k] = h.R[x][k] * h.s[k];
    h.Bu[x] = h.B[x][0] * h.u[0] + h.B[x][1] * h.u[1] + h.B[x][2] * h.u[2] + h.B[x][3] * h.u[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) h.G[x][k] = h.B[x][k] - h.Bu[x] * h.u[k];
    h.mu[x] = h.m[x] + h.Bu[x] * (h.dt * isq);
  }
  // Camera transform and near cull.
#pragma unroll
  for (int x = 0; x < 3; ++x)
    h.pc[x] = cam.W[3 * x + 0] * h.mu[0] + cam.W[3 * x + 1] * h.mu[1] + cam.W[3 * x + 2] * h.mu[2] + cam.T[x];
  if (!(h.pc[2] > near_plane)) return false;
  // EWA (Sec. 3.1, Eq. 4): M = J W, H = M G, Sigma_2d = H H^T + dilation I.
  h.iz = 1.0f / h.pc[2];
  const float j00 = cam.fx * h.iz, j02 = -cam.fx * h.pc[0] * h.iz * h.iz;
  const float j11 = cam.fy * h.iz, j12 = -cam.fy * h.pc[1] * h.iz * h.iz;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    h.M[0][x] = j00 * cam.W[x] + j02 * cam.W[6 + x];
    h.M[1][x] = j11 * cam.W[3 + x] + j12 * cam.W[6 + x];
  }
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int k = 0; k < 4; ++k) h.H[rr][k] = h.M[rr][0] * h.G[0][k] + h.M[rr][1] * h.G[1][k] + h.M[rr][2] * h.G[2][k];
  float n0 = 0.f, n1 = 0.f, n01 = 0.f, minors = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    n0 += h.H[0][k] * h.H[0][k];
    n1 += h.H[1][k] * h.H[1][k];
    n01 += h.H[0][k] * h.H[1][k];
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = x + 1; y < 4; ++y) {
      const float mnr = h.H[0][x] * h.H[1][y] - h.H[0][y] * h.H[1][x];
      minors += mnr * mnr;
    }
  h.Sa = n0 + dilation;
  h.Sd = n1 + dilation;
  h.Sb = n01;
  h.det = minors + dilation * (n0 + n1) + dilation * dilation;
  if (!(h.det > 0.0f)) return false;
  const float idet = 1.0f / h.det;
  h.conA = h.Sd * idet;
  h.conB = -h.Sb * idet;
  h.conC = h.Sa * idet;
  // Eq. 3: projected centre; 3-sigma radius; tile rect.
  h.uv[0] = cam.fx * h.pc[0] * h.iz + cam.cx;
  h.uv[1] = cam.fy * h.pc[1] * h.iz + cam.cy;
  const float mid = 0.5f * (h.Sa + h.Sd);
  const float hd = 0.5f * (h.Sa - h.Sd);
  const float disc = hd * hd + h.Sb * h.Sb;
  const float lam = mid + sqrtf(fmaxf(0.1f, disc));
  const float rad = ceilf(3.0f * sqrtf(lam));
  const float inv_tile = cam.inv_tile;
  h.rect[0] = min(max(__float2int_rd((h.uv[0] - rad) * inv_tile), 0), cam.gw);
  h.rect[1] = min(max(__float2int_rd((h.uv[1] - rad) * inv_tile), 0), cam.gh);
  h.rect[2] = min(max(__float2int_rd((h.uv[0] + rad) * inv_tile) + 1, 0), cam.gw);
  h.rect[3] = min(max(__float2int_rd((h.uv[1] + rad) * inv_tile) + 1, 0), cam.gh);
  if (h.rect[0] >= h.rect[2] || h.rect[1] >= h.rect[3]) return false;
  // alpha <= a everywhere: below 1/255 the Gaussian is skipped at every pixel.
  h.a = h.sig * h.pt;
  if (!(h.a * 255.0f >= 1.0f)) return false;
  // 4DSH colour (Sec. 3.2).
  const float wx = h.mu[0] - cam.campos[0], wy = h.mu[1] - cam.campos[1], wz = h.mu[2] - cam.campos[2];
  h.rw = sqrtf(wx * wx + wy * wy + wz * wz);
  const float irw = 1.0f / h.rw;
  h.dir[0] = wx * irw; h.dir[1] = wy * irw; h.dir[2] = wz * irw;
  constexpr int NLM = (L + 1) * (L + 1);
  float Y[NLM];
  sh_basis<L>(h.dir[0], h.dir[1], h.dir[2], Y);
  // cos / sin of 2 pi n dt / T by the angle-addition recurrence.
  const float ph = 2.0f * h.dt * period_inv;
  const float c1 = cospif(ph), s1 = sinpif(ph);
  h.cn[0] = 1.0f;
  h.sn[0] = 0.0f;
#pragma unroll
  for (int nn = 1; nn <= FGS4D_MAX_T_ORDER; ++nn) {
    h.cn[nn] = h.cn[nn - 1] * c1 - h.sn[nn - 1] * s1;
    h.sn[nn] = h.sn[nn - 1] * c1 + h.cn[nn - 1] * s1;
  }
  float acc[3] = {0.f, 0.f, 0.f};
  const float *shg = sh + (size_t)i * k3;
#pragma unroll
  for (int nn = 0; nn <= FGS4D_MAX_T_ORDER; ++nn) {
    if (nn > t_order) break;
    const float *cf = shg + nn * NLM * 3;
    float part[3] = {0.f, 0.f, 0.f};
    if ((NLM * 3) % 4 == 0) {
      const float4 *cf4 = reinterpret_cast<const float4 *>(cf);
#pragma unroll
      for (int k4 = 0; k4 < NLM * 3 / 4; ++k4) {
        const float4 w4 = __ldg(&cf4[k4]);
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * k4 + e;
          part[k % 3] += wv[e] * Y[k / 3];
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < NLM * 3; ++k) part[k % 3] += __ldg(&cf[k]) * Y[k / 3];
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) acc[ch] += h.cn[nn] * part[ch];
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    h.raw[ch] = acc[ch];
    h.rgb[ch] = fmaxf(0.0f, acc[ch] + 0.5f);
    if (!isfinite(h.rgb[ch])) return false;
  }
  return true;
}

template <int L, int MAXV>
__global__ void __launch_bounds__(kPreBlock) preprocess_kernel(PreArgs A, PreViews<MAXV> views) {
  grid_dependency_sync();
  __shared__ uint32_t s_ticket;
  __shared__ uint32_t s_scan[9];
  __shared__ uint64_t s_base;
  const int32_t nlogical = A.nviews * A.blocks_per_view;
  // Persistent: logical blocks of kPreBlock (view, Gaussian) pairs are taken
  // by ticket, so a logical block's look-back only waits on logical blocks
  // that running blocks hold.
  while (true) {
  if (threadIdx.x == 0) s_ticket = atomicAdd(&A.counters[kCtrTicketPre], 1u);
  __syncthreads();
  const int32_t w = (int32_t)s_ticket;
  if (w >= nlogical) break;
  const int32_t view = MAXV == 1 ? 0 : w / A.blocks_per_view;
  const int32_t gb = MAXV == 1 ? w : w % A.blocks_per_view;
  const int32_t i = gb * kPreBlock + (int32_t)threadIdx.x;
  const PreView &cam = views.v[view];

  Chain h;
  // Compact-4DGS mask (Sec. 4.3): M_hat = 1{sigmoid(m) > eps} in value, so a
  // Gaussian is either removed (zero scales and opacity) or unchanged.
  bool kept = i < A.n;
  if (kept && A.mask_logit) {
    const float mk = A.mask_logit[i];
    kept = isfinite(mk) && 1.0f / (1.0f + expf(-mk)) > A.mask_threshold;
  }
  const bool vis = kept && forward_chain<L>(i, A.mean, A.log_scale, A.q_l, A.q_r, A.logit, A.sh, A.t_order, A.k3,
                                            A.period_inv, A.near_plane, A.dilation, A.p_t_min, cam, h);
  uint32_t total;
  const uint32_t local = block_exclusive_scan(vis ? 1u : 0u, s_scan, &total);
  if (threadIdx.x < 32) {
    const uint64_t prefix = lookback_u64_warp(A.lb, w, total, &A.counters[kCtrStatus]);
    if (threadIdx.x == 0) s_base = prefix;
    if (threadIdx.x == 0 && w == nlogical - 1) {
      const uint64_t all = prefix + total;
      A.counters[kCtrNeedVisible] = (uint32_t)umin64(all, 0xffffffffull);
      A.counters[kCtrVisible] = (uint32_t)umin64(all, (uint64_t)A.vis_cap);
      if (all > (uint64_t)A.vis_cap) atomicOr(&A.counters[kCtrStatus], kStatusVisOverflow);
    }
  }
  __syncthreads();
  const uint64_t slot = s_base + local;
  if (vis && slot < (uint64_t)A.vis_cap) {
    // The exponent in base 2, q = (1/2) log2(e) d^T Sigma_2d^-1 d, as a sum of
    // two squares: Sigma_2d^-1 = U U^T with U upper triangular gives
    // q = (a1 dx)^2 + (b1 dx + b2 dy)^2, a1 = sqrt(k / Sa), b1 = -Sb sqrt(k /
    // (Sa det)), b2 = Sa sqrt(k / (Sa det)), k = log2(e) / 2.  Evaluated this
    // way q has no cancellation (the expanded conic form loses precision along
    // the long axis of an elongated footprint, in proportion to its condition
    // number); det is the Cauchy-Binet sum of squares.
    const float kq = 0.5f * kLog2e;
    const float a1 = sqrtf(kq / h.Sa);
    const float rs = sqrtf(kq / (h.Sa * h.det));
    A.rec_geom[slot] = make_float4(h.uv[0], h.uv[1], a1, -h.Sb * rs);
    A.rec_color[slot] = make_float4(h.Sa * rs, log2f(h.a), h.rgb[0], h.rgb[1]);
    A.rec_blue[slot] = h.rgb[2];
    // alpha = a 2^power2 >= 1/255 needs -power2 <= log2(255 a); the margin
    // keeps the per-tile test of the instance emission conservative under
    // rounding.
    A.rec_tau[slot] = log2f(255.0f * h.a) + kTauMargin;
    A.rec_meta[slot] = make_int4(i, view, h.rect[0] | (h.rect[1] << 16), h.rect[2] | (h.rect[3] << 16));
    A.depth_key[slot] = __float_as_uint(h.pc[2]);
  }
  __syncthreads();  // s_ticket and s_base are reused by the next logical block
  }
}

// ------------------------------------------------------------- adjoint

__device__ __forceinline__ void red_add4(float4 *p, float x, float y, float z, float w) {
  atomicAdd(p, make_float4(x, y, z, w));
}

// Auxiliary records per visible slot (depth, opacity and flow channels):
// camera depth of the sliced mean and the image-plane displacement of the
// sliced mean over flow_dt (Sec. 8.1.3: the trajectory of mu_xyz|t projected
// between consecutive frames).  mu_xyz|t moves with velocity
// Sigma_{1:3,4} / Sigma_44 = (B u) / sqrt(Sigma_44) in the factored form, so the
// displaced camera-space centre is pc + W v flow_dt; the flow is 0 when that
// point is not in front of the near plane.  The chain is re-run with the
// colour basis cut to degree 0 (the slot is known to be visible; only its
// geometry is used).
struct AuxArgs {
  const float4 *mean, *log_scale, *q_l, *q_r;
  const float *logit, *sh;
  int32_t t_order, k3;
  float period_inv, near_plane, dilation, p_t_min, flow_dt;
  int64_t vis_cap;
  const uint32_t *counters;
  const int4 *rec_meta;
  float4 *rec_aux;
};

template <int MAXV>
__global__ void __launch_bounds__(128) aux_records_kernel(AuxArgs A, PreViews<MAXV> views) {
  grid_dependency_sync();
  const int64_t nvis = min64((int64_t)A.counters[kCtrVisible], A.vis_cap);
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nvis) return;
  const int4 meta = A.rec_meta[slot];
  const PreView &cam = views.v[MAXV == 1 ? 0 : meta.y];
  Chain h;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (forward_chain<0>(meta.x, A.mean, A.log_scale, A.q_l, A.q_r, A.logit, A.sh, A.t_order, A.k3, A.period_inv,
                       A.near_plane, A.dilation, A.p_t_min, cam, h)) {
    const float k = A.flow_dt / h.sqc;  // velocity = B u / sqrt(Sigma_44)
    const float d0 = h.Bu[0] * k, d1 = h.Bu[1] * k, d2 = h.Bu[2] * k;
    float p2[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) p2[x] = h.pc[x] + cam.W[3 * x + 0] * d0 + cam.W[3 * x + 1] * d1 + cam.W[3 * x + 2] * d2;
    out.x = h.pc[2];
    if (p2[2] > A.near_plane) {
      out.y = cam.fx * p2[0] / p2[2] + cam.cx - h.uv[0];
      out.z = cam.fy * p2[1] / p2[2] + cam.cy - h.uv[1];
    }
  }
  A.rec_aux[slot] = out;
}

template <int L, int MAXV>
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(BwdArgs A, PreViews<MAXV> views) {
  grid_dependency_sync();
  const int64_t nvis = min64((int64_t)A.counters[kCtrVisible], A.vis_cap);
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nvis) return;
  const int4 meta = A.rec_meta[slot];
  const int32_t i = meta.x, view = meta.y;
  if (i < 0 || i >= A.n || view < 0 || view >= A.nviews) return;  // only after a recorded timeout
  const PreView &cam = views.v[view];
  Chain h;
  if (!forward_chain<L>(i, A.mean, A.log_scale, A.q_l, A.q_r, A.logit, A.sh, A.t_order, A.k3, A.period_inv,
                        A.near_plane, A.dilation, A.p_t_min, cam, h))
    return;  // cannot happen for a slot the forward produced with the same inputs
  const float4 g0 = A.slot_grad[3 * slot + 0];  // du, dv, dA, dB
  const float4 g1 = A.slot_grad[3 * slot + 1];  // dC, da, dr, dg
  const float4 g2 = A.slot_grad[3 * slot + 2];  // db, dz
  const float gu = g0.x, gv = g0.y, gA = g0.z, gB = g0.w, gC = g1.x, ga = g1.y;
  const float grgb[3] = {g1.z, g1.w, g2.x};

  float g_mu[3] = {0.f, 0.f, 0.f}, g_dt = 0.f;
  // ---- colour: rgb = max(0, raw + 0.5), raw = sum_n cos_n sum_lm c Y_lm.
  constexpr int NLM = (L + 1) * (L + 1);
  float graw[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) graw[ch] = (h.raw[ch] + 0.5f > 0.0f) ? grgb[ch] : 0.0f;
  float Y[NLM], gY[NLM];
  sh_basis<L>(h.dir[0], h.dir[1], h.dir[2], Y);
#pragma unroll
  for (int k = 0; k < NLM; ++k) gY[k] = 0.f;
  const float *shg = A.sh + (size_t)i * A.k3;
  float *gsh = A.g_sh + (size_t)i * A.k3;
  const bool any_col = graw[0] != 0.f || graw[1] != 0.f || graw[2] != 0.f;
  if (any_col) {
#pragma unroll
    for (int nn = 0; nn <= FGS4D_MAX_T_ORDER; ++nn) {
      if (nn > A.t_order) break;
      const float *cf = shg + nn * NLM * 3;
      float gcos = 0.f;
      if ((NLM * 3) % 4 == 0) {
        const float4 *cf4 = reinterpret_cast<const float4 *>(cf);
        float4 *g4 = reinterpret_cast<float4 *>(gsh + nn * NLM * 3);
#pragma unroll
        for (int k4 = 0; k4 < NLM * 3 / 4; ++k4) {
          const float4 w4 = __ldg(&cf4[k4]);
          const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
          float gv4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = 4 * k4 + e, lm = k / 3, ch = k % 3;
            gv4[e] = graw[ch] * h.cn[nn] * Y[lm];
            gY[lm] += graw[ch] * wv[e] * h.cn[nn];
            gcos += graw[ch] * wv[e] * Y[lm];
          }
          red_add4(&g4[k4], gv4[0], gv4[1], gv4[2], gv4[3]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NLM * 3; ++k) {
          const int lm = k / 3, ch = k % 3;
          const float wv = __ldg(&cf[k]);
          atomicAdd(&gsh[nn * NLM * 3 + k], graw[ch] * h.cn[nn] * Y[lm]);
          gY[lm] += graw[ch] * wv * h.cn[nn];
          gcos += graw[ch] * wv * Y[lm];
        }
      }
      // d cos(2 pi n dt / T) / d dt = -sin(.) 2 pi n / T
      g_dt += gcos * (-h.sn[nn]) * (kTwoPi * (float)nn * A.period_inv);
    }
    float gdir[3] = {0.f, 0.f, 0.f};
    sh_basis_grad<L>(h.dir[0], h.dir[1], h.dir[2], gY, gdir);
    const float dd = gdir[0] * h.dir[0] + gdir[1] * h.dir[1] + gdir[2] * h.dir[2];
    const float irw = 1.0f / h.rw;
#pragma unroll
    for (int x = 0; x < 3; ++x) g_mu[x] += (gdir[x] - h.dir[x] * dd) * irw;
  }
  // ---- opacity a = sigmoid(logit) p_t.
  const float g_sig = ga * h.pt;
  float g_pt = ga * h.sig;
  atomicAdd(&A.g_logit[i], g_sig * h.sig * (1.0f - h.sig));
  // ---- projected centre.
  const float iz = h.iz, x = h.pc[0], y = h.pc[1];
  float g_pc[3];
  g_pc[0] = gu * cam.fx * iz;
  g_pc[1] = gv * cam.fy * iz;
  g_pc[2] = -(gu * cam.fx * x + gv * cam.fy * y) * iz * iz;
  g_pc[2] += g2.y;  // depth channel (zero unless the loss uses it): z is pc_z itself
  // ---- conic = inverse(Sigma_2d): dL/dSigma_2d = -Q GQ Q (full symmetric).
  const float q00 = h.conA, q01 = h.conB, q11 = h.conC;
  const float G00 = gA, G01 = 0.5f * gB, G11 = gC;
  const float t00 = q00 * G00 + q01 * G01, t01 = q00 * G01 + q01 * G11;
  const float t10 = q01 * G00 + q11 * G01, t11 = q01 * G01 + q11 * G11;
  const float s00 = -(t00 * q00 + t01 * q01);
  const float s01 = -(t00 * q01 + t01 * q11);
  const float s11 = -(t10 * q01 + t11 * q11);
  // ---- Sigma_2d = H H^T + dil I: dL/dH = 2 S H.
  float gH[2][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    gH[0][k] = 2.0f * (s00 * h.H[0][k] + s01 * h.H[1][k]);
    gH[1][k] = 2.0f * (s01 * h.H[0][k] + s11 * h.H[1][k]);
  }
  // ---- H = M G.
  float gM[2][3], gG[3][4];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int xx = 0; xx < 3; ++xx)
      gM[rr][xx] = gH[rr][0] * h.G[xx][0] + gH[rr][1] * h.G[xx][1] + gH[rr][2] * h.G[xx][2] + gH[rr][3] * h.G[xx][3];
#pragma unroll
  for (int xx = 0; xx < 3; ++xx)
#pragma unroll
    for (int k = 0; k < 4; ++k) gG[xx][k] = h.M[0][xx] * gH[0][k] + h.M[1][xx] * gH[1][k];
  // ---- M = J W; J depends on the camera-space centre.
  float gJ[2][3];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      gJ[rr][k] = gM[rr][0] * cam.W[3 * k + 0] + gM[rr][1] * cam.W[3 * k + 1] + gM[rr][2] * cam.W[3 * k + 2];
  const float iz2 = iz * iz, iz3 = iz2 * iz;
  g_pc[0] += gJ[0][2] * (-cam.fx * iz2);
  g_pc[1] += gJ[1][2] * (-cam.fy * iz2);
  g_pc[2] += gJ[0][0] * (-cam.fx * iz2) + gJ[0][2] * (2.0f * cam.fx * x * iz3) + gJ[1][1] * (-cam.fy * iz2) +
             gJ[1][2] * (2.0f * cam.fy * y * iz3);
  // ---- pc = W mu + T.
#pragma unroll
  for (int xx = 0; xx < 3; ++xx)
    g_mu[xx] += cam.W[xx] * g_pc[0] + cam.W[3 + xx] * g_pc[1] + cam.W[6 + xx] * g_pc[2];
  // ---- mu = m + Bu dt / sqrt(c); G = B - Bu u^T; Bu = B u; u = v / sqrt(c).
  const float isq = 1.0f / h.sqc;
  float gBu[3], gu4[4] = {0.f, 0.f, 0.f, 0.f}, gB4[3][4], g_sqc = 0.f;
  float mub = 0.f;
#pragma unroll
  for (int xx = 0; xx < 3; ++xx) {
    gBu[xx] = g_mu[xx] * h.dt * isq;
    mub += g_mu[xx] * h.Bu[xx];
  }
  g_dt += mub * isq;
  g_sqc += -mub * h.dt * isq * isq;
#pragma unroll
  for (int xx = 0; xx < 3; ++xx) {
    float gGu = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      gB4[xx][k] = gG[xx][k];
      gGu += gG[xx][k] * h.u[k];
      gu4[k] -= gG[xx][k] * h.Bu[xx];
    }
    gBu[xx] -= gGu;
  }
#pragma unroll
  for (int xx = 0; xx < 3; ++xx)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      gB4[xx][k] += gBu[xx] * h.u[k];
      gu4[k] += h.B[xx][k] * gBu[xx];
    }
  float gv4[4], gc = 0.f, uv_dot = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) uv_dot += gu4[k] * h.v[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) gv4[k] = gu4[k] * isq;
  g_sqc += -uv_dot * isq * isq;
  // ---- p_t = exp(-dt^2 / (2c)).
  g_dt += g_pt * h.pt * (-h.dt / h.c);
  gc += g_pt * h.pt * (0.5f * h.dt * h.dt / (h.c * h.c));
  gc += g_sqc * 0.5f * isq;
#pragma unroll
  for (int k = 0; k < 4; ++k) gv4[k] += 2.0f * h.v[k] * gc;
  // ---- v_k = R_4k s_k; B_xk = R_xk s_k.
  float gR[4][4], gs[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    gR[3][k] = gv4[k] * h.s[k];
    gs[k] = gv4[k] * h.R[3][k];
#pragma unroll
    for (int xx = 0; xx < 3; ++xx) {
      gR[xx][k] = gB4[xx][k] * h.s[k];
      gs[k] += gB4[xx][k] * h.R[xx][k];
    }
  }
  red_add4(&A.g_mean[i], g_mu[0], g_mu[1], g_mu[2], -g_dt);
  // Densification indicators of this (view, Gaussian): |dL/dmu_2d| and
  // |dL/dmu_t| (Sec. 3.3, densification in spacetime), plus the view count.
  if (A.densify_stats) red_add4(&A.densify_stats[i], sqrtf(gu * gu + gv * gv), fabsf(g_dt), 1.0f, 0.0f);
  red_add4(&A.g_log_scale[i], gs[0] * h.s[0], gs[1] * h.s[1], gs[2] * h.s[2], gs[3] * h.s[3]);
  // Straight-through mask gradient (Sec. 4.3): at M_hat = 1, dL/dM_hat =
  // sum_k dL/dlog s_k + dL/dalpha alpha, and dM_hat/dm = M (1 - M).
  if (A.mask_logit && A.g_mask) {
    const float M = 1.0f / (1.0f + expf(-A.mask_logit[i]));
    const float g_mhat = g_sig * h.sig + gs[0] * h.s[0] + gs[1] * h.s[1] + gs[2] * h.s[2] + gs[3] * h.s[3];
    atomicAdd(&A.g_mask[i], g_mhat * M * (1.0f - M));
  }
  // ---- R = Lm Rm: dL/dLm = gR Rm^T, dL/dRm = Lm^T gR; collect by entry pattern.
  const float a = h.ql[0], b = h.ql[1], c = h.ql[2], d = h.ql[3];
  const float p = h.qr[0], q = h.qr[1], r = h.qr[2], s = h.qr[3];
  const float Lm[4][4] = {{a, -b, -c, -d}, {b, a, -d, c}, {c, d, a, -b}, {d, -c, b, a}};
  const float Rm[4][4] = {{p, -q, -r, -s}, {q, p, s, -r}, {r, -s, p, q}, {s, r, -q, p}};
  float gL[4][4], gRr[4][4];
#pragma unroll
  for (int xx = 0; xx < 4; ++xx)
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
      gL[xx][yy] = gR[xx][0] * Rm[yy][0] + gR[xx][1] * Rm[yy][1] + gR[xx][2] * Rm[yy][2] + gR[xx][3] * Rm[yy][3];
      gRr[xx][yy] = Lm[0][xx] * gR[0][yy] + Lm[1][xx] * gR[1][yy] + Lm[2][xx] * gR[2][yy] + Lm[3][xx] * gR[3][yy];
    }
  float gql[4], gqr[4];
  gql[0] = gL[0][0] + gL[1][1] + gL[2][2] + gL[3][3];
  gql[1] = -gL[0][1] + gL[1][0] - gL[2][3] + gL[3][2];
  gql[2] = -gL[0][2] + gL[1][3] + gL[2][0] - gL[3][1];
  gql[3] = -gL[0][3] - gL[1][2] + gL[2][1] + gL[3][0];
  gqr[0] = gRr[0][0] + gRr[1][1] + gRr[2][2] + gRr[3][3];
  gqr[1] = -gRr[0][1] + gRr[1][0] + gRr[2][3] - gRr[3][2];
  gqr[2] = -gRr[0][2] - gRr[1][3] + gRr[2][0] + gRr[3][1];
  gqr[3] = -gRr[0][3] + gRr[1][2] - gRr[2][1] + gRr[3][0];
  // ---- q_hat = q / |q|.
  const float dl = gql[0] * a + gql[1] * b + gql[2] * c + gql[3] * d;
  const float dr = gqr[0] * p + gqr[1] * q + gqr[2] * r + gqr[3] * s;
  const float il = 1.0f / h.nql, ir = 1.0f / h.nqr;
  red_add4(&A.g_q_l[i], (gql[0] - a * dl) * il, (gql[1] - b * dl) * il, (gql[2] - c * dl) * il,
           (gql[3] - d * dl) * il);
  red_add4(&A.g_q_r[i], (gqr[0] - p * dr) * ir, (gqr[1] - q * dr) * ir, (gqr[2] - r * dr) * ir,
           (gqr[3] - s * dr) * ir);
}

template <int MAXV>
bool fill_pre_views(const fgs4d_view *views, int32_t nviews, int32_t tile, PreViews<MAXV> *pv) {
  if (nviews > MAXV) return false;
  for (int v = 0; v < MAXV; ++v) {
    PreView &o = pv->v[v];
    if (v >= nviews) {
      o = PreView{};
      continue;
    }
    const fgs4d_view &c = views[v];
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) o.W[3 * r + k] = c.viewmat[4 * r + k];
      o.T[r] = c.viewmat[4 * r + 3];
      o.campos[r] = c.campos[r];
    }
    o.fx = c.fx;
    o.fy = c.fy;
    o.cx = c.cx;
    o.cy = c.cy;
    o.t = c.t;
    o.width = c.width;
    o.height = c.height;
    o.gw = (c.width + tile - 1) / tile;
    o.gh = (c.height + tile - 1) / tile;
    o.tile = tile;
    o.inv_tile = 1.0f / (float)tile;
  }
  return true;
}

template <int L, int MAXV>
cudaError_t launch_pre_typed(const PreLaunch &p, const fgs4d_view *views, int32_t nviews) {
  PreViews<MAXV> pv;
  fill_pre_views<MAXV>(views, nviews, p.L->tile, &pv);
  const Layout &Lo = *p.L;
  PreArgs A;
  A.mean = reinterpret_cast<const float4 *>(p.g->mean);
  A.log_scale = reinterpret_cast<const float4 *>(p.g->log_scale);
  A.q_l = reinterpret_cast<const float4 *>(p.g->q_l);
  A.q_r = reinterpret_cast<const float4 *>(p.g->q_r);
  A.logit = p.g->opacity_logit;
  A.mask_logit = p.g->mask_logit;
  A.mask_threshold = p.g->mask_threshold;
  A.sh = p.g->sh;
  A.n = (int32_t)p.g->n;
  A.t_order = p.s->t_order;
  A.k3 = (L + 1) * (L + 1) * (p.s->t_order + 1) * 3;
  A.period_inv = 1.0f / p.s->period;
  A.near_plane = p.s->near_plane;
  A.dilation = p.s->dilation;
  A.p_t_min = p.s->p_t_min;
  A.nviews = nviews;
  A.blocks_per_view = Lo.pre_blocks_per_view;
  A.vis_cap = Lo.vis_cap;
  A.counters = reinterpret_cast<uint32_t *>(p.ws + Lo.counters);
  A.lb = reinterpret_cast<uint64_t *>(p.ws + Lo.lb_pre);
  A.rec_geom = reinterpret_cast<float4 *>(p.ws + Lo.rec_geom);
  A.rec_color = reinterpret_cast<float4 *>(p.ws + Lo.rec_color);
  A.rec_blue = reinterpret_cast<float *>(p.ws + Lo.rec_blue);
  A.rec_tau = reinterpret_cast<float *>(p.ws + Lo.rec_tau);
  A.rec_meta = reinterpret_cast<int4 *>(p.ws + Lo.rec_meta);
  A.depth_key = reinterpret_cast<uint32_t *>(p.ws + Lo.depth_key);
  if (Lo.pre_blocks == 0) return cudaSuccess;
  return launch_pdl(preprocess_kernel<L, MAXV>, (unsigned)Lo.pre_grid, kPreBlock, p.stream, A, pv);
}

template <int L, int MAXV>
cudaError_t launch_bwd_typed(const PreLaunch &p, const fgs4d_view *views, int32_t nviews,
                             const fgs4d_gaussians_grad *gr) {
  PreViews<MAXV> pv;
  fill_pre_views<MAXV>(views, nviews, p.L->tile, &pv);
  const Layout &Lo = *p.L;
  BwdArgs A;
  A.mean = reinterpret_cast<const float4 *>(p.g->mean);
  A.log_scale = reinterpret_cast<const float4 *>(p.g->log_scale);
  A.q_l = reinterpret_cast<const float4 *>(p.g->q_l);
  A.q_r = reinterpret_cast<const float4 *>(p.g->q_r);
  A.logit = p.g->opacity_logit;
  A.sh = p.g->sh;
  A.n = (int32_t)p.g->n;
  A.nviews = nviews;
  A.t_order = p.s->t_order;
  A.k3 = (L + 1) * (L + 1) * (p.s->t_order + 1) * 3;
  A.period_inv = 1.0f / p.s->period;
  A.near_plane = p.s->near_plane;
  A.dilation = p.s->dilation;
  A.p_t_min = p.s->p_t_min;
  A.vis_cap = Lo.vis_cap;
  A.counters = reinterpret_cast<const uint32_t *>(p.ws + Lo.counters);
  A.rec_meta = reinterpret_cast<const int4 *>(p.ws + Lo.rec_meta);
  A.slot_grad = reinterpret_cast<const float4 *>(p.ws + Lo.slot_grad);
  A.g_mean = reinterpret_cast<float4 *>(gr->mean);
  A.g_log_scale = reinterpret_cast<float4 *>(gr->log_scale);
  A.g_q_l = reinterpret_cast<float4 *>(gr->q_l);
  A.g_q_r = reinterpret_cast<float4 *>(gr->q_r);
  A.g_logit = gr->opacity_logit;
  A.g_sh = gr->sh;
  A.mask_logit = p.g->mask_logit;
  A.g_mask = gr->mask_logit;
  A.densify_stats = reinterpret_cast<float4 *>(gr->densify_stats);
  const int64_t blocks = (Lo.vis_cap + 127) / 128;
  if (blocks == 0) return cudaSuccess;
  return launch_pdl(preprocess_bwd_kernel<L, MAXV>, (unsigned)blocks, 128u, p.stream, A, pv);
}

template <int MAXV>
cudaError_t launch_aux_typed(const PreLaunch &p, const fgs4d_view *views, int32_t nviews, float flow_dt) {
  PreViews<MAXV> pv;
  fill_pre_views<MAXV>(views, nviews, p.L->tile, &pv);
  const Layout &Lo = *p.L;
  AuxArgs A;
  A.mean = reinterpret_cast<const float4 *>(p.g->mean);
  A.log_scale = reinterpret_cast<const float4 *>(p.g->log_scale);
  A.q_l = reinterpret_cast<const float4 *>(p.g->q_l);
  A.q_r = reinterpret_cast<const float4 *>(p.g->q_r);
  A.logit = p.g->opacity_logit;
  A.sh = p.g->sh;
  A.t_order = p.s->t_order;
  A.k3 = (p.s->sh_degree + 1) * (p.s->sh_degree + 1) * (p.s->t_order + 1) * 3;
  A.period_inv = 1.0f / p.s->period;
  A.near_plane = p.s->near_plane;
  A.dilation = p.s->dilation;
  A.p_t_min = p.s->p_t_min;
  A.flow_dt = flow_dt;
  A.vis_cap = Lo.vis_cap;
  A.counters = reinterpret_cast<const uint32_t *>(p.ws + Lo.counters);
  A.rec_meta = reinterpret_cast<const int4 *>(p.ws + Lo.rec_meta);
  A.rec_aux = reinterpret_cast<float4 *>(p.ws + Lo.rec_aux);
  const int64_t blocks = (Lo.vis_cap + 127) / 128;
  if (blocks == 0) return cudaSuccess;
  return launch_pdl(aux_records_kernel<MAXV>, (unsigned)blocks, 128u, p.stream, A, pv);
}

}  // namespace

cudaError_t launch_preprocess(const PreLaunch &p, const fgs4d_view *views, int32_t nviews) {
  const bool one = nviews == 1;
  switch (p.s->sh_degree) {
    case 0: return one ? launch_pre_typed<0, 1>(p, views, nviews) : launch_pre_typed<0, FGS4D_MAX_VIEWS>(p, views, nviews);
    case 1: return one ? launch_pre_typed<1, 1>(p, views, nviews) : launch_pre_typed<1, FGS4D_MAX_VIEWS>(p, views, nviews);
    case 2: return one ? launch_pre_typed<2, 1>(p, views, nviews) : launch_pre_typed<2, FGS4D_MAX_VIEWS>(p, views, nviews);
    default: return one ? launch_pre_typed<3, 1>(p, views, nviews) : launch_pre_typed<3, FGS4D_MAX_VIEWS>(p, views, nviews);
  }
}

cudaError_t launch_preprocess_bwd(const PreLaunch &p, const fgs4d_view *views, int32_t nviews,
                                  const fgs4d_gaussians_grad *grads) {
  const bool one = nviews == 1;
  switch (p.s->sh_degree) {
    case 0: return one ? launch_bwd_typed<0, 1>(p, views, nviews, grads) : launch_bwd_typed<0, FGS4D_MAX_VIEWS>(p, views, nviews, grads);
    case 1: return one ? launch_bwd_typed<1, 1>(p, views, nviews, grads) : launch_bwd_typed<1, FGS4D_MAX_VIEWS>(p, views, nviews, grads);
    case 2: return one ? launch_bwd_typed<2, 1>(p, views, nviews, grads) : launch_bwd_typed<2, FGS4D_MAX_VIEWS>(p, views, nviews, grads);
    default: return one ? launch_bwd_typed<3, 1>(p, views, nviews, grads) : launch_bwd_typed<3, FGS4D_MAX_VIEWS>(p, views, nviews, grads);
  }
}

cudaError_t launch_aux_records(const PreLaunch &p, const fgs4d_view *views, int32_t nviews, float flow_dt) {
  if (nviews == 1) return launch_aux_typed<1>(p, views, nviews, flow_dt);
  return launch_aux_typed<FGS4D_MAX_VIEWS>(p, views, nviews, flow_dt);
}


namespace {

// Split sampling in spacetime: child = mu + R diag(s) eps with the 4D
// rotation of the parent (Sec. 3.2) -- a draw from the parent's full 4D
// Gaussian N(mu, Sigma), Sigma = R S S^T R^T (Sec. 3.3 / Sec. 8.1.3).
struct SplitArgs {
  const float4 *mean, *log_scale, *q_l, *q_r;
  const float *logit, *sh;
  int64_t n;
  const int32_t *idx;
  const float4 *eps;
  int64_t m;
  int32_t k_children, k3;
  float log_shrink;
  float4 *o_mean, *o_log_scale, *o_q_l, *o_q_r;
  float *o_logit, *o_sh;
};

// One thread per child for the draw; the children's SH rows (the bulk of
// the bytes) are then copied by whole warps, consecutive lanes on
// consecutive floats of a row.
__global__ void __launch_bounds__(128) split_kernel(SplitArgs A) {
  grid_dependency_sync();
  __shared__ int32_t s_src[128];  // parent of each child of the block, -1: none
  const int64_t total = A.m * A.k_children;
  const int64_t c0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t child = c0 + threadIdx.x;
  int32_t src = -1;
  if (child < total) {
    const int64_t j = child / A.k_children;
    const int32_t i = A.idx[j];
    if (i < 0 || (int64_t)i >= A.n) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      A.o_mean[child] = A.o_log_scale[child] = A.o_q_l[child] = A.o_q_r[child] = z;
      A.o_logit[child] = 0.f;
    } else {
      src = i;
      const float4 m = A.mean[i], ls = A.log_scale[i], a4 = A.q_l[i], b4 = A.q_r[i];
      const float il = rsqrtf(a4.x * a4.x + a4.y * a4.y + a4.z * a4.z + a4.w * a4.w);
      const float ir = rsqrtf(b4.x * b4.x + b4.y * b4.y + b4.z * b4.z + b4.w * b4.w);
      const float a = a4.x * il, b = a4.y * il, c = a4.z * il, d = a4.w * il;
      const float p = b4.x * ir, q = b4.y * ir, r = b4.z * ir, s = b4.w * ir;
      const float Lm[4][4] = {{a, -b, -c, -d}, {b, a, -d, c}, {c, d, a, -b}, {d, -c, b, a}};
      const float Rm[4][4] = {{p, -q, -r, -s}, {q, p, s, -r}, {r, -s, p, q}, {s, r, -q, p}};
      const float4 e = A.eps[child];
      const float se[4] = {expf(ls.x) * e.x, expf(ls.y) * e.y, expf(ls.z) * e.z, expf(ls.w) * e.w};
      float off[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float acc = 0.f;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const float Rxy = Lm[x][0] * Rm[0][y] + Lm[x][1] * Rm[1][y] + Lm[x][2] * Rm[2][y] + Lm[x][3] * Rm[3][y];
          acc += Rxy * se[y];
        }
        off[x] = acc;
      }
      A.o_mean[child] = make_float4(m.x + off[0], m.y + off[1], m.z + off[2], m.w + off[3]);
      A.o_log_scale[child] =
          make_float4(ls.x - A.log_shrink, ls.y - A.log_shrink, ls.z - A.log_shrink, ls.w - A.log_shrink);
      A.o_q_l[child] = a4;
      A.o_q_r[child] = b4;
      A.o_logit[child] = A.logit[i];
    }
  }
  s_src[threadIdx.x] = src;
  __syncthreads();
  const int nchild = (int)min64((int64_t)blockDim.x, total - c0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // float4 copies when rows of both arrays start on 16-byte boundaries
  const bool vec = (A.k3 & 3) == 0 && ((reinterpret_cast<uintptr_t>(A.sh) | reinterpret_cast<uintptr_t>(A.o_sh)) & 15) == 0;
  const int width = vec ? A.k3 >> 2 : A.k3;
  for (int c = warp; c < nchild; c += nwarps) {
    const int32_t i = s_src[c];
    const int64_t orow = (c0 + c) * A.k3, irow = (int64_t)(i >= 0 ? i : 0) * A.k3;
    for (int k = lane; k < width; k += 32) {
      if (vec)
        reinterpret_cast<float4 *>(A.o_sh + orow)[k] =
            i >= 0 ? reinterpret_cast<const float4 *>(A.sh + irow)[k] : make_float4(0.f, 0.f, 0.f, 0.f);
      else
        A.o_sh[orow + k] = i >= 0 ? A.sh[irow + k] : 0.f;
    }
  }
}

}  // namespace

cudaError_t launch_split(const fgs4d_gaussians *src, const int32_t *idx, int64_t m, int32_t k_children,
                         const float *eps, float shrink, int32_t k3, const fgs4d_gaussians_out *dst,
                         cudaStream_t stream) {
  SplitArgs A;
  A.mean = reinterpret_cast<const float4 *>(src->mean);
  A.log_scale = reinterpret_cast<const float4 *>(src->log_scale);
  A.q_l = reinterpret_cast<const float4 *>(src->q_l);
  A.q_r = reinterpret_cast<const float4 *>(src->q_r);
  A.logit = src->opacity_logit;
  A.sh = src->sh;
  A.n = src->n;
  A.idx = idx;
  A.eps = reinterpret_cast<const float4 *>(eps);
  A.m = m;
  A.k_children = k_children;
  A.k3 = k3;
  A.log_shrink = logf(shrink);
  A.o_mean = reinterpret_cast<float4 *>(dst->mean);
  A.o_log_scale = reinterpret_cast<float4 *>(dst->log_scale);
  A.o_q_l = reinterpret_cast<float4 *>(dst->q_l);
  A.o_q_r = reinterpret_cast<float4 *>(dst->q_r);
  A.o_logit = dst->opacity_logit;
  A.o_sh = dst->sh;
  const int64_t total = m * k_children;
  if (total == 0) return cudaSuccess;
  return launch_pdl(split_kernel, (unsigned)((total + 127) / 128), 128u, stream, A);
}

}  // namespace fgs4d
