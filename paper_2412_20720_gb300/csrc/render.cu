// Per-tile front-to-back compositing (Sec. 3.2, Eq. 6 of arXiv 2412.20720)
// and its reverse-mode derivative, plus the photometric L1 loss (Sec. 3.3).
//
// Forward: one CTA per (view, 16x16 tile), one pixel per thread.  The tile's
// depth-sorted list is staged through shared memory in batches of 256
// records; a CTA stops loading once every pixel has hit the transmittance
// cutoff (__syncthreads_count).  alpha = min(0.99, a 2^power2), skip when
// power2 > 0 or alpha < 1/255, stop before the entry that would take T below
// 1e-4 -- evaluated by eval_alpha, shared with the backward pass so that both
// take bit-identical decisions.
//
// Backward: the same tiles traversed back to front from each pixel's last
// composited entry, recomputing T_i = T_{i+1} / (1 - alpha_i) from the final
// transmittance.  Per-Gaussian sums are reduced across the warp by shuffles
// before one vector atomic per warp.
#include <algorithm>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {

struct RenderArgs {
  const uint2 *ranges;
  const uint32_t *inst_val;
  const float4 *rec_geom, *rec_color;
  const float *rec_blue;
  uint32_t vis_cap;
  float *out_rgb, *out_T;
  float *pix_T;
  uint32_t *pix_last;
  float bg0, bg1, bg2;
};

struct RenderBwdArgs {
  const uint2 *ranges;
  const uint32_t *inst_val;
  const float4 *rec_geom, *rec_color;
  const float *rec_blue;
  uint32_t vis_cap;
  const float *pix_T;
  const uint32_t *pix_last;
  const float *dL_drgb;
  float4 *slot_grad;
  float bg0, bg1, bg2;
};

template <int MAXV>
__device__ __forceinline__ int find_view(const RasterViews<MAXV> &rv, int32_t gt) {
  if (MAXV == 1) return 0;
  int lo = 0, hi = rv.nviews - 1;
  while (lo < hi) {  // last view with tile_base <= gt
    const int mid = (lo + hi + 1) >> 1;
    if (rv.v[mid].tile_base <= gt) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// kStats: also counts the pixel-entry alpha evaluations and the composited
// entries (diagnostic variant used to state the algorithmic work).
template <int MAXV, bool kStats>
__global__ void __launch_bounds__(kTilePixels) render_fwd_kernel(RenderArgs A, RasterViews<MAXV> rv,
                                                                 unsigned long long *stats) {
  __shared__ float4 s_geom[kTilePixels];
  __shared__ float4 s_col[kTilePixels];
  __shared__ float s_blue[kTilePixels];
  const int32_t gt = blockIdx.x;
  const RasterView &V = rv.v[find_view<MAXV>(rv, gt)];
  const int32_t lt = gt - V.tile_base;
  const int32_t tx = lt % V.gw, ty = lt / V.gw;
  const int32_t px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int32_t py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < V.width && py < V.height;
  const uint2 range = A.ranges[gt];
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0u, n_eval = 0u, n_comp = 0u;
  bool done = !inside;
  for (uint32_t base = range.x; base < range.y; base += kTilePixels) {
    if (__syncthreads_count(done) == kTilePixels) break;
    const uint32_t idx = base + threadIdx.x;
    if (idx < range.y) {
      const uint32_t s = A.inst_val[idx];
      if (s < A.vis_cap) {
        s_geom[threadIdx.x] = A.rec_geom[s];
        s_col[threadIdx.x] = A.rec_color[s];
        s_blue[threadIdx.x] = A.rec_blue[s];
      } else {  // only after a recorded timeout: contributes nothing
        s_geom[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_col[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_blue[threadIdx.x] = 0.f;
      }
    }
    __syncthreads();
    const int nb = (int)min(range.y - base, (uint32_t)kTilePixels);
    if (!done) {
      for (int j = 0; j < nb; ++j) {
        const float4 col = s_col[j];
        const AlphaEval e = eval_alpha(s_geom[j], col.x, col.y, pxc, pyc);
        if (kStats) ++n_eval;
        if (e.power2 > 0.0f || e.alpha < kAlphaMin) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, e.alpha));
        if (Tn < kTMin) {
          done = true;
          break;
        }
        const float w = e.alpha * T;
        C0 += col.z * w;
        C1 += col.w * w;
        C2 += s_blue[j] * w;
        T = Tn;
        last = base + j - range.x + 1;
        if (kStats) ++n_comp;
      }
    }
  }
  if (kStats) {
    unsigned long long ev = n_eval, co = n_comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_xor_sync(0xffffffffu, ev, o);
      co += __shfl_xor_sync(0xffffffffu, co, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], ev);
      atomicAdd(&stats[1], co);
    }
  }
  if (!inside) return;
  const int64_t HW = (int64_t)V.width * V.height;
  const int64_t p = (int64_t)py * V.width + px;
  float *img = A.out_rgb + V.pix_base * 3;
  img[p] = C0 + T * A.bg0;
  img[HW + p] = C1 + T * A.bg1;
  img[2 * HW + p] = C2 + T * A.bg2;
  A.pix_T[V.pix_base + p] = T;
  A.pix_last[V.pix_base + p] = last;
  if (A.out_T) A.out_T[V.pix_base + p] = T;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int MAXV>
__global__ void __launch_bounds__(kTilePixels) render_bwd_kernel(RenderBwdArgs A, RasterViews<MAXV> rv) {
  __shared__ float4 s_geom[kTilePixels];
  __shared__ float4 s_col[kTilePixels];
  __shared__ float s_blue[kTilePixels];
  __shared__ uint32_t s_slot[kTilePixels];
  __shared__ uint32_t s_maxlast;
  const int32_t gt = blockIdx.x;
  const RasterView &V = rv.v[find_view<MAXV>(rv, gt)];
  const int32_t lt = gt - V.tile_base;
  const int32_t tx = lt % V.gw, ty = lt / V.gw;
  const int32_t px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int32_t py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < V.width && py < V.height;
  const uint2 range = A.ranges[gt];
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const int64_t HW = (int64_t)V.width * V.height;
  const int64_t p = (int64_t)py * V.width + px;
  float T = 1.0f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
  uint32_t last = 0u;
  if (inside) {
    T = A.pix_T[V.pix_base + p];
    last = A.pix_last[V.pix_base + p];
    const float *g = A.dL_drgb + V.pix_base * 3;
    dC0 = g[p];
    dC1 = g[HW + p];
    dC2 = g[2 * HW + p];
  }
  if (threadIdx.x == 0) s_maxlast = 0u;
  __syncthreads();
  if (last) atomicMax(&s_maxlast, last);
  __syncthreads();
  const uint32_t end = range.x + min(s_maxlast, range.y - range.x);
  float r0 = T * A.bg0, r1 = T * A.bg1, r2 = T * A.bg2;  // colour composited behind entry i
  const int lane = threadIdx.x & 31;
  const int nbatch = (int)((end - range.x + kTilePixels - 1) / kTilePixels);
  for (int bi = nbatch - 1; bi >= 0; --bi) {
    const uint32_t base = range.x + (uint32_t)bi * kTilePixels;
    __syncthreads();
    const uint32_t idx = base + threadIdx.x;
    if (idx < end) {
      const uint32_t s = A.inst_val[idx];
      s_slot[threadIdx.x] = s;
      if (s < A.vis_cap) {
        s_geom[threadIdx.x] = A.rec_geom[s];
        s_col[threadIdx.x] = A.rec_color[s];
        s_blue[threadIdx.x] = A.rec_blue[s];
      } else {  // only after a recorded timeout: contributes nothing
        s_geom[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_col[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_blue[threadIdx.x] = 0.f;
      }
    }
    __syncthreads();
    const int nb = (int)min(end - base, (uint32_t)kTilePixels);
    for (int j = nb - 1; j >= 0; --j) {
      const uint32_t pos = base + j - range.x;  // entry index in the tile list
      float gu = 0.f, gv = 0.f, gA = 0.f, gB = 0.f, gC = 0.f, ga = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
      bool contrib = false;
      if (pos < last) {
        const float4 geom = s_geom[j];
        const float4 col = s_col[j];
        const AlphaEval e = eval_alpha(geom, col.x, col.y, pxc, pyc);
        if (!(e.power2 > 0.0f || e.alpha < kAlphaMin)) {
          contrib = true;
          const float om = __fsub_rn(1.0f, e.alpha);
          T = __fdiv_rn(T, om);  // transmittance in front of this entry
          const float w = e.alpha * T;
          const float blue = s_blue[j];
          gr = dC0 * w;
          gg = dC1 * w;
          gb = dC2 * w;
          const float io = 1.0f / om;
          const float g_alpha = dC0 * (col.z * T - r0 * io) + dC1 * (col.w * T - r1 * io) + dC2 * (blue * T - r2 * io);
          r0 += col.z * w;
          r1 += col.w * w;
          r2 += blue * w;
          if (!(e.aG > 0.99f)) {  // min(0.99, .) is locally constant when clamped
            ga = g_alpha * e.G;
            const float gp = g_alpha * e.alpha;  // d alpha / d (natural-log power)
            const float An = 2.0f * kLn2 * geom.z, Bn = kLn2 * geom.w, Cn = 2.0f * kLn2 * col.x;
            gA = -0.5f * e.dx * e.dx * gp;
            gB = -e.dx * e.dy * gp;
            gC = -0.5f * e.dy * e.dy * gp;
            gu = -(An * e.dx + Bn * e.dy) * gp;
            gv = -(Cn * e.dy + Bn * e.dx) * gp;
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        gu = warp_sum(gu); gv = warp_sum(gv); gA = warp_sum(gA); gB = warp_sum(gB); gC = warp_sum(gC);
        ga = warp_sum(ga); gr = warp_sum(gr); gg = warp_sum(gg); gb = warp_sum(gb);
        if (lane == 0 && s_slot[j] < A.vis_cap) {
          float4 *dst = A.slot_grad + 3 * (size_t)s_slot[j];
          atomicAdd(dst + 0, make_float4(gu, gv, gA, gB));
          atomicAdd(dst + 1, make_float4(gC, ga, gr, gg));
          atomicAdd(reinterpret_cast<float *>(dst + 2), gb);
        }
      }
    }
  }
}

__global__ void l1_loss_kernel(const float *__restrict__ img, const float *__restrict__ target, int64_t count,
                               float inv_count, float *loss, float *grad) {
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - target[i];
    acc += fabsf(d);
    grad[i] = d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f);
  }
  acc = warp_sum(acc);
  __shared__ float s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.f;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(loss, v * inv_count);
  }
}

template <int MAXV>
cudaError_t render_fwd_typed(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                             unsigned char *ws, float *out_rgb, float *out_T, unsigned long long *stats,
                             cudaStream_t st) {
  RasterViews<MAXV> rv;
  if (!make_raster_views<MAXV>(L, views, nviews, &rv)) return cudaErrorInvalidValue;
  RenderArgs A;
  A.ranges = reinterpret_cast<const uint2 *>(ws + L.ranges);
  A.inst_val = reinterpret_cast<const uint32_t *>(ws + L.inst_val[L.tile_passes & 1]);
  A.rec_geom = reinterpret_cast<const float4 *>(ws + L.rec_geom);
  A.rec_color = reinterpret_cast<const float4 *>(ws + L.rec_color);
  A.rec_blue = reinterpret_cast<const float *>(ws + L.rec_blue);
  A.vis_cap = (uint32_t)L.vis_cap;
  A.out_rgb = out_rgb;
  A.out_T = out_T;
  A.pix_T = reinterpret_cast<float *>(ws + L.pix_T);
  A.pix_last = reinterpret_cast<uint32_t *>(ws + L.pix_last);
  A.bg0 = s->bg[0];
  A.bg1 = s->bg[1];
  A.bg2 = s->bg[2];
  if (L.total_tiles == 0) return cudaSuccess;
  if (stats)
    render_fwd_kernel<MAXV, true><<<(unsigned)L.total_tiles, kTilePixels, 0, st>>>(A, rv, stats);
  else
    render_fwd_kernel<MAXV, false><<<(unsigned)L.total_tiles, kTilePixels, 0, st>>>(A, rv, nullptr);
  return cudaGetLastError();
}

template <int MAXV>
cudaError_t render_bwd_typed(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                             unsigned char *ws, const float *dL_drgb, cudaStream_t st) {
  RasterViews<MAXV> rv;
  if (!make_raster_views<MAXV>(L, views, nviews, &rv)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(ws + L.slot_grad, 0, (size_t)L.vis_cap * kSlotGradFloats * sizeof(float), st);
  if (e != cudaSuccess) return e;
  RenderBwdArgs A;
  A.ranges = reinterpret_cast<const uint2 *>(ws + L.ranges);
  A.inst_val = reinterpret_cast<const uint32_t *>(ws + L.inst_val[L.tile_passes & 1]);
  A.rec_geom = reinterpret_cast<const float4 *>(ws + L.rec_geom);
  A.rec_color = reinterpret_cast<const float4 *>(ws + L.rec_color);
  A.rec_blue = reinterpret_cast<const float *>(ws + L.rec_blue);
  A.vis_cap = (uint32_t)L.vis_cap;
  A.pix_T = reinterpret_cast<const float *>(ws + L.pix_T);
  A.pix_last = reinterpret_cast<const uint32_t *>(ws + L.pix_last);
  A.dL_drgb = dL_drgb;
  A.slot_grad = reinterpret_cast<float4 *>(ws + L.slot_grad);
  A.bg0 = s->bg[0];
  A.bg1 = s->bg[1];
  A.bg2 = s->bg[2];
  if (L.total_tiles == 0) return cudaSuccess;
  render_bwd_kernel<MAXV><<<(unsigned)L.total_tiles, kTilePixels, 0, st>>>(A, rv);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_fwd(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                              unsigned char *ws, float *out_rgb, float *out_T, unsigned long long *stats,
                              cudaStream_t stream) {
  if (nviews == 1) return render_fwd_typed<1>(L, s, views, nviews, ws, out_rgb, out_T, stats, stream);
  return render_fwd_typed<FGS4D_MAX_VIEWS>(L, s, views, nviews, ws, out_rgb, out_T, stats, stream);
}

cudaError_t launch_render_bwd(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                              unsigned char *ws, const float *dL_drgb, cudaStream_t stream) {
  if (nviews == 1) return render_bwd_typed<1>(L, s, views, nviews, ws, dL_drgb, stream);
  return render_bwd_typed<FGS4D_MAX_VIEWS>(L, s, views, nviews, ws, dL_drgb, stream);
}

cudaError_t launch_l1_loss(const float *img, const float *target, int64_t count, float *loss, float *grad,
                           cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 8);
  l1_loss_kernel<<<blocks, 256, 0, stream>>>(img, target, count, 1.0f / (float)count, loss, grad);
  return cudaGetLastError();
}

}  // namespace fgs4d
