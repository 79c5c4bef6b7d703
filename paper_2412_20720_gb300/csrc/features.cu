// Scale-gated feature rendering for 4D segmentation (Sec. 7 of arXiv
// 2412.20720, "Scale-gated features"): each Gaussian carries a feature
// f in R^D; at a scale s the gate vector S(s) in [0,1]^D gives
// f^s = S(s) (.) f, which is normalised and composited exactly like the
// colour of Eq. 6 (zero background).  The geometry is that of a pre-trained
// 4DGS, so the backward pass returns dL/df and dL/dS(s) only.
//
// Forward: one CTA per (view, 16x16 tile), a thread owns a vertical strip of
// kFeatPPT pixels; records are staged in batches with the normalised feature
// of each entry (and its norm) in shared memory.  Skip/stop decisions are
// pixel_alpha's, so the weights equal those of the colour compositor bit for
// bit.
//
// Backward: the same front-to-back traversal recomputes the weights w_i; per
// entry a warp sums w dL/dF over its pixels (one D-vector), reduces it with a
// transposed butterfly (lane c ends with component c), applies the
// normalisation Jacobian (linear, so partial sums may be projected
// separately): dL/dg = (v - fhat (fhat . v)) / |g|, and adds
// dL/df = S (.) dL/dg per lane; dL/dS(s) = f (.) dL/dg is summed per block.
#include <algorithm>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {

constexpr int kFeatPPT = 2;
// Threads per block and records per staged batch (one per thread) for a
// TILE x TILE tile: 128 at 16x16, 32 at 8x8.
template <int TILE>
__host__ __device__ constexpr int feat_threads() {
  return TILE * TILE / kFeatPPT;
}
// The adjoint reduces D sums per (warp, entry): with D <= 16 it takes 4-pixel
// strips at 16x16 (64 threads), half the warps per tile and so half the
// reductions.  Alpha does not depend on the strip shape (row groups), so it
// still equals the forward's bit for bit.
template <int TILE, int D>
__host__ __device__ constexpr int feat_bwd_ppt() {
  return (TILE == 16 && D <= 16) ? 4 : kFeatPPT;
}
template <int TILE, int D>
__host__ __device__ constexpr int feat_bwd_threads() {
  return TILE * TILE / feat_bwd_ppt<TILE, D>();
}

struct FeatArgs {
  const uint2 *ranges;
  const uint32_t *inst_val;
  const float4 *rec_geom, *rec_color;
  const int4 *rec_meta;
  uint32_t vis_cap;
  int64_t n;
  const float *feat;  // [n][D]
  const float *gate;  // [D] or null (ones)
  float *out;         // [views][D][H][W]
  const float *dL_dF; // backward: [views][D][H][W]
  float *g_feat;      // backward: [n][D]
  float *g_gate;      // backward: [D] or null
};

// Stages entry `k` of the batch: geometry, opacity, normalised gated feature
// and its norm (rows padded to D + 1 floats against bank conflicts).
template <int D>
__device__ __forceinline__ void stage_feature(const FeatArgs &A, const float *s_gate, uint32_t idx, int k,
                                              float4 *s_geom, float2 *s_ca, float *s_fhat, float *s_f,
                                              float *s_norm, int32_t *s_gi) {
  const uint32_t s = A.inst_val[idx];
  float4 geom = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 ca = make_float2(0.f, kLogAlphaNone);  // (b2, log2 a): every pixel skips the entry
  int32_t gi = -1;
  if (s < A.vis_cap) {
    geom = A.rec_geom[s];
    const float4 c = A.rec_color[s];
    ca = make_float2(c.x, c.y);
    gi = A.rec_meta[s].x;
    if (gi < 0 || (int64_t)gi >= A.n) {
      gi = -1;
      ca.y = kLogAlphaNone;
    }
  }
  s_geom[k] = geom;
  s_ca[k] = ca;
  s_gi[k] = gi;
  float g[D];
  float nn = 0.f;
  if (gi >= 0) {
    const float4 *row = reinterpret_cast<const float4 *>(A.feat + (int64_t)gi * D);
#pragma unroll
    for (int c4 = 0; c4 < D / 4; ++c4) {
      const float4 v = row[c4];
      g[4 * c4 + 0] = v.x;
      g[4 * c4 + 1] = v.y;
      g[4 * c4 + 2] = v.z;
      g[4 * c4 + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) g[c] = 0.f;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (s_f) s_f[k * (D + 1) + c] = g[c];
    g[c] *= s_gate[c];
    nn += g[c] * g[c];
  }
  const float norm = sqrtf(nn);
  const float inv = norm > 0.f ? 1.0f / norm : 0.f;
#pragma unroll
  for (int c = 0; c < D; ++c) s_fhat[k * (D + 1) + c] = g[c] * inv;
  if (s_norm) s_norm[k] = norm;
}

template <int MAXV, int TILE, int D>
__global__ void __launch_bounds__(feat_threads<TILE>()) render_features_kernel(FeatArgs A, RasterViews<MAXV> rv) {
  grid_dependency_sync();
  constexpr int kFeatBatch = feat_threads<TILE>();
  __shared__ float4 s_geom[kFeatBatch];
  __shared__ float2 s_ca[kFeatBatch];
  __shared__ int32_t s_gi[kFeatBatch];
  __shared__ float s_fhat[kFeatBatch * (D + 1)];
  __shared__ float s_gate[D];
  const int32_t gt = blockIdx.x;
  const RasterView &V = rv.v[find_view<MAXV>(rv, gt)];
  const int32_t lt = gt - V.tile_base;
  const int32_t tx = lt % V.gw, ty = lt / V.gw;
  const int32_t px = tx * TILE + (threadIdx.x & (TILE - 1));
  const int32_t py0 = ty * TILE + (threadIdx.x / TILE) * kFeatPPT;
  const uint2 range = tile_range(A.ranges, gt);
  const float pxc = (float)px + 0.5f;
  if (threadIdx.x < D) s_gate[threadIdx.x] = A.gate ? A.gate[threadIdx.x] : 1.0f;
  static_assert(kFeatPPT <= 4, "a strip inside one row group");
  const float gyc = row_group_centre(py0);
  float T[kFeatPPT], off[kFeatPPT], F[kFeatPPT][D];
  bool live = false;
#pragma unroll
  for (int k = 0; k < kFeatPPT; ++k) {
    const bool in = px < V.width && py0 + k < V.height;
    T[k] = in ? 1.0f : -1.0f;
    off[k] = in ? row_offset(py0 + k) : stopped_offset();
#pragma unroll
    for (int c = 0; c < D; ++c) F[k][c] = 0.f;
    live = live || in;
  }
  for (uint32_t base = range.x; base < range.y; base += kFeatBatch) {
    if (__syncthreads_count(live) == 0) break;
    if (base + threadIdx.x < range.y)
      stage_feature<D>(A, s_gate, base + threadIdx.x, threadIdx.x, s_geom, s_ca, s_fhat, nullptr, nullptr, s_gi);
    __syncthreads();
    const int nb = (int)min(range.y - base, (uint32_t)kFeatBatch);
    for (int j = 0; j < nb && live; ++j) {
      const float4 geom = s_geom[j];
      const float2 ca = s_ca[j];
      const ColumnTerms ct = column_terms(geom, pxc, ca.y);
      const float w4 = group_w(ct, geom.y, ca.x, gyc);
      const bool clamp = entry_clamps(ca.y);
#pragma unroll
      for (int k = 0; k < kFeatPPT; ++k) {
        const AlphaEval e = pixel_alpha(ct, w4, ca.x, off[k], clamp);
        if (e.alpha >= kAlphaMin) {  // false for stopped pixels (row offset +inf)
          const float w = __fmul_rn(e.alpha, T[k]);
          const float Tn = __fsub_rn(T[k], w);
          if (Tn < kTMin) {
            T[k] = -T[k];
            off[k] = stopped_offset();
          } else {
#pragma unroll
            for (int c = 0; c < D; ++c) F[k][c] = __fmaf_rn(s_fhat[j * (D + 1) + c], w, F[k][c]);
            T[k] = Tn;
          }
        }
      }
      live = false;
#pragma unroll
      for (int k = 0; k < kFeatPPT; ++k) live = live || T[k] > 0.0f;
    }
  }
  const int64_t HW = (int64_t)V.width * V.height;
  float *out = A.out + V.pix_base * D;
#pragma unroll
  for (int k = 0; k < kFeatPPT; ++k) {
    if (!(px < V.width && py0 + k < V.height)) continue;
    const int64_t p = (int64_t)(py0 + k) * V.width + px;
#pragma unroll
    for (int c = 0; c < D; ++c) out[c * HW + p] = F[k][c];
  }
}

// Sums D <= 32 per-lane values over the warp; on return a[0] of lane l holds
// the total of value l (lanes >= D hold totals of zero padding).
template <int D>
__device__ __forceinline__ float warp_transpose_sum(float (&a)[32], int lane) {
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? a[i] : a[i + half];
      const float keep = up ? a[i + half] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return a[0];
}

template <int MAXV, int TILE, int D>
__global__ void __launch_bounds__(feat_bwd_threads<TILE, D>())
    render_features_bwd_kernel(FeatArgs A, RasterViews<MAXV> rv) {
  grid_dependency_sync();
  constexpr int kPPT = feat_bwd_ppt<TILE, D>();
  constexpr int kFeatBatch = feat_bwd_threads<TILE, D>();
  __shared__ float4 s_geom[kFeatBatch];
  __shared__ float2 s_ca[kFeatBatch];
  __shared__ int32_t s_gi[kFeatBatch];
  __shared__ float s_fhat[kFeatBatch * (D + 1)];
  __shared__ float s_f[kFeatBatch * (D + 1)];
  __shared__ float s_norm[kFeatBatch];
  __shared__ float s_gate[D];
  __shared__ float s_ggate[D];
  const int32_t gt = blockIdx.x;
  const RasterView &V = rv.v[find_view<MAXV>(rv, gt)];
  const int32_t lt = gt - V.tile_base;
  const int32_t tx = lt % V.gw, ty = lt / V.gw;
  const int32_t px = tx * TILE + (threadIdx.x & (TILE - 1));
  const int32_t py0 = ty * TILE + (threadIdx.x / TILE) * kPPT;
  const uint2 range = tile_range(A.ranges, gt);
  const float pxc = (float)px + 0.5f;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < D) {
    s_gate[threadIdx.x] = A.gate ? A.gate[threadIdx.x] : 1.0f;
    s_ggate[threadIdx.x] = 0.f;
  }
  const int64_t HW = (int64_t)V.width * V.height;
  const float *dF = A.dL_dF + V.pix_base * D;
  const float gyc = row_group_centre(py0);
  float T[kPPT], off[kPPT], G[kPPT][D];
  bool live = false;
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    const bool in = px < V.width && py0 + k < V.height;
    T[k] = in ? 1.0f : -1.0f;
    off[k] = in ? row_offset(py0 + k) : stopped_offset();
    const int64_t p = (int64_t)(py0 + k) * V.width + px;
#pragma unroll
    for (int c = 0; c < D; ++c) G[k][c] = in ? dF[c * HW + p] : 0.f;
    live = live || in;
  }
  for (uint32_t base = range.x; base < range.y; base += kFeatBatch) {
    if (__syncthreads_count(live) == 0) break;
    if (base + threadIdx.x < range.y)
      stage_feature<D>(A, s_gate, base + threadIdx.x, threadIdx.x, s_geom, s_ca, s_fhat, s_f, s_norm, s_gi);
    __syncthreads();
    const int nb = (int)min(range.y - base, (uint32_t)kFeatBatch);
    for (int j = 0; j < nb; ++j) {
      if (!__any_sync(0xffffffffu, live)) break;  // the warp's pixels have all stopped
      const float4 geom = s_geom[j];
      const float2 ca = s_ca[j];
      const ColumnTerms ct = column_terms(geom, pxc, ca.y);
      const float w4 = group_w(ct, geom.y, ca.x, gyc);
      const bool clamp = entry_clamps(ca.y);
      float v[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = 0.f;
      bool contrib = false;
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        const AlphaEval e = pixel_alpha(ct, w4, ca.x, off[k], clamp);
        if (e.alpha >= kAlphaMin) {  // false for stopped pixels (row offset +inf)
          const float w = __fmul_rn(e.alpha, T[k]);
          const float Tn = __fsub_rn(T[k], w);
          if (Tn < kTMin) {
            T[k] = -T[k];
            off[k] = stopped_offset();
          } else {
            contrib = true;
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = __fmaf_rn(G[k][c], w, v[c]);
            T[k] = Tn;
          }
        }
      }
      live = false;
#pragma unroll
      for (int k = 0; k < kPPT; ++k) live = live || T[k] > 0.0f;
      if (!__any_sync(0xffffffffu, contrib)) continue;
      const int32_t gi = s_gi[j];
      const float vc = warp_transpose_sum<D>(v, lane);  // lane c: component c of the warp's sum
      const float fh = lane < D ? s_fhat[j * (D + 1) + lane] : 0.f;
      const float dot = warp_sum(fh * vc);
      const float norm = s_norm[j];
      if (gi >= 0 && norm > 0.f && lane < D) {
        const float dg = (vc - fh * dot) / norm;
        atomicAdd(&A.g_feat[(int64_t)gi * D + lane], s_gate[lane] * dg);
        if (A.g_gate) atomicAdd(&s_ggate[lane], s_f[j * (D + 1) + lane] * dg);
      }
    }
  }
  __syncthreads();
  if (A.g_gate && threadIdx.x < D && s_ggate[threadIdx.x] != 0.f) atomicAdd(&A.g_gate[threadIdx.x], s_ggate[threadIdx.x]);
}

template <int MAXV, int TILE, int D>
cudaError_t launch_feat_tile(const FeatArgs &A, const RasterViews<MAXV> &rv, unsigned grid, bool backward,
                             cudaStream_t st) {
  constexpr unsigned NT = feat_threads<TILE>();
  if (backward)
    return launch_pdl(render_features_bwd_kernel<MAXV, TILE, D>, grid, (unsigned)feat_bwd_threads<TILE, D>(), st, A,
                      rv);
  return launch_pdl(render_features_kernel<MAXV, TILE, D>, grid, NT, st, A, rv);
}

template <int MAXV, int D>
cudaError_t launch_feat_typed(const Layout &L, const FeatArgs &A, const fgs4d_view *views, int32_t nviews,
                              bool backward, cudaStream_t st) {
  RasterViews<MAXV> rv;
  if (!make_raster_views<MAXV>(L, views, nviews, &rv)) return cudaErrorInvalidValue;
  if (L.total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)L.total_tiles;
  if (L.tile == 8) return launch_feat_tile<MAXV, 8, D>(A, rv, grid, backward, st);
  return launch_feat_tile<MAXV, 16, D>(A, rv, grid, backward, st);
}

template <int D>
cudaError_t launch_feat_d(const Layout &L, const FeatArgs &A, const fgs4d_view *views, int32_t nviews,
                          bool backward, cudaStream_t st) {
  if (nviews == 1) return launch_feat_typed<1, D>(L, A, views, nviews, backward, st);
  return launch_feat_typed<FGS4D_MAX_VIEWS, D>(L, A, views, nviews, backward, st);
}

}  // namespace

bool feature_dim_supported(int32_t D) { return D == 8 || D == 16 || D == 32; }

cudaError_t launch_render_features(const Layout &L, const fgs4d_view *views, int32_t nviews, unsigned char *ws,
                                   int64_t n, const float *feat, int32_t D, const float *gate, float *out,
                                   const float *dL_dF, float *g_feat, float *g_gate, cudaStream_t st) {
  FeatArgs A;
  A.ranges = reinterpret_cast<const uint2 *>(ws + L.ranges);
  A.inst_val = reinterpret_cast<const uint32_t *>(ws + L.inst_val[L.tile_passes & 1]);
  A.rec_geom = reinterpret_cast<const float4 *>(ws + L.rec_geom);
  A.rec_color = reinterpret_cast<const float4 *>(ws + L.rec_color);
  A.rec_meta = reinterpret_cast<const int4 *>(ws + L.rec_meta);
  A.vis_cap = (uint32_t)L.vis_cap;
  A.n = n;
  A.feat = feat;
  A.gate = gate;
  A.out = out;
  A.dL_dF = dL_dF;
  A.g_feat = g_feat;
  A.g_gate = g_gate;
  const bool bwd = dL_dF != nullptr;
  switch (D) {
    case 8: return launch_feat_d<8>(L, A, views, nviews, bwd, st);
    case 16: return launch_feat_d<16>(L, A, views, nviews, bwd, st);
    default: return launch_feat_d<32>(L, A, views, nviews, bwd, st);
  }
}

}  // namespace fgs4d
