// C ABI entry points of the fgs4d library (declared in include/fgs4d.h):
// host-side argument checks, workspace layout, and kernel launches on the
// caller's stream.  No device memory is allocated here.
#include <math.h>
#include <cmath>
#include <string.h>

#include <algorithm>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kMaxCap = (1ll << 30) - 1;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool finite_f(float x) { return isfinite(x); }

int check_settings(const fgs4d_settings *s) {
  if (!s) return FGS4D_ERR_ARG;
  if (s->sh_degree < 0 || s->sh_degree > FGS4D_MAX_SH_DEGREE) return FGS4D_ERR_UNSUPPORTED;
  if (s->t_order < 0 || s->t_order > FGS4D_MAX_T_ORDER) return FGS4D_ERR_UNSUPPORTED;
  if (s->tile != 16 && s->tile != 8) return FGS4D_ERR_UNSUPPORTED;
  if (!finite_f(s->period) || !(s->period > 0.f)) return FGS4D_ERR_ARG;
  if (!finite_f(s->near_plane) || !(s->near_plane > 0.f)) return FGS4D_ERR_ARG;
  if (!finite_f(s->dilation) || s->dilation < 0.f) return FGS4D_ERR_ARG;
  if (!finite_f(s->p_t_min) || s->p_t_min < 0.f || s->p_t_min >= 1.f) return FGS4D_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (!finite_f(s->bg[k])) return FGS4D_ERR_ARG;
  if (s->inst_capacity <= 0 || s->inst_capacity > kMaxCap) return FGS4D_ERR_ARG;
  if (s->vis_capacity < 0 || s->vis_capacity > kMaxCap) return FGS4D_ERR_ARG;
  // Compositor strip heights per tile edge: 16 -> 2, 4, 8; 8 -> 1, 2 (0 = default).
  const int ppt = s->pixels_per_thread;
  if (ppt != 0 && !(s->tile == 16 ? (ppt == 2 || ppt == 4 || ppt == 8) : (ppt == 1 || ppt == 2)))
    return FGS4D_ERR_UNSUPPORTED;
  if (s->shared_batch != 0 && s->shared_batch != 128 && s->shared_batch != 256) return FGS4D_ERR_UNSUPPORTED;
  if (s->stage_blocks_per_sm < 0 || s->stage_blocks_per_sm > 8) return FGS4D_ERR_UNSUPPORTED;
  return FGS4D_OK;
}

int check_views(const fgs4d_view *views, int32_t nviews) {
  if (!views || nviews < 1 || nviews > FGS4D_MAX_VIEWS) return FGS4D_ERR_ARG;
  for (int v = 0; v < nviews; ++v) {
    const fgs4d_view &c = views[v];
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return FGS4D_ERR_ARG;
    if (!finite_f(c.fx) || !finite_f(c.fy) || !finite_f(c.cx) || !finite_f(c.cy) || !finite_f(c.t)) return FGS4D_ERR_ARG;
    for (int k = 0; k < 12; ++k)
      if (!finite_f(c.viewmat[k])) return FGS4D_ERR_ARG;
    for (int k = 0; k < 3; ++k)
      if (!finite_f(c.campos[k])) return FGS4D_ERR_ARG;
  }
  return FGS4D_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int check_gaussians(const fgs4d_gaussians *g) {
  if (!g || g->n < 0 || g->n > (int64_t)INT32_MAX - 1024) return FGS4D_ERR_ARG;
  if (g->n == 0) return FGS4D_OK;
  const void *ptrs[6] = {g->mean, g->log_scale, g->q_l, g->q_r, g->opacity_logit, g->sh};
  for (int k = 0; k < 6; ++k)
    if (!ptrs[k]) return FGS4D_ERR_ARG;
  // float4 loads of the [n][4] planes and of the SH rows.
  if (!aligned16(g->mean) || !aligned16(g->log_scale) || !aligned16(g->q_l) || !aligned16(g->q_r) ||
      !aligned16(g->sh))
    return FGS4D_ERR_ARG;
  if (g->mask_logit && !(finite_f(g->mask_threshold) && g->mask_threshold >= 0.f && g->mask_threshold < 1.f))
    return FGS4D_ERR_ARG;
  return FGS4D_OK;
}

int check_workspace(const Layout &L, const void *ws, size_t bytes) {
  if (!ws || ((uintptr_t)ws & (kAlign - 1)) != 0) return FGS4D_ERR_WORKSPACE;
  if (bytes < L.total) return FGS4D_ERR_WORKSPACE;
  return FGS4D_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FGS4D_OK : FGS4D_ERR_CUDA; }

}  // namespace

int compute_layout(const fgs4d_settings *s, int64_t n, const fgs4d_view *views, int32_t nviews, Layout *out) {
  int rc = check_settings(s);
  if (rc) return rc;
  rc = check_views(views, nviews);
  if (rc) return rc;
  if (n < 0 || n > (int64_t)INT32_MAX - 1024) return FGS4D_ERR_ARG;
  Layout L;
  memset(&L, 0, sizeof L);
  L.n = n;
  L.nviews = nviews;
  L.tile = s->tile;
  L.vis_cap = s->vis_capacity ? s->vis_capacity : n * (int64_t)nviews;
  if (L.vis_cap > kMaxCap) return FGS4D_ERR_ARG;  // set vis_capacity explicitly
  L.inst_cap = s->inst_capacity;
  for (int v = 0; v < nviews; ++v) {
    const int64_t gw = (views[v].width + s->tile - 1) / s->tile, gh = (views[v].height + s->tile - 1) / s->tile;
    L.total_tiles += gw * gh;
    L.total_pixels += (int64_t)views[v].width * views[v].height;
  }
  if (L.total_tiles > INT32_MAX) return FGS4D_ERR_ARG;
  int bits = 1;
  while ((1ll << bits) < L.total_tiles) ++bits;
  L.tile_bits = bits;
  L.tile_passes = (bits + kRadixBits - 1) / kRadixBits;
  if (L.tile_passes > kMaxPasses) return FGS4D_ERR_UNSUPPORTED;
  L.depth_passes = 4;  // 31 bits of a positive FP32 depth
  L.pre_blocks_per_view = (int32_t)((n + kPreBlock - 1) / kPreBlock);
  const int64_t pb = (int64_t)L.pre_blocks_per_view * nviews;
  if (pb > INT32_MAX) return FGS4D_ERR_ARG;
  L.pre_blocks = (int32_t)pb;
  L.emit_blocks = (int32_t)((L.vis_cap + kEmitBlock - 1) / kEmitBlock);
  L.pair_cap = std::min<int64_t>(8 * L.inst_cap, (int64_t)INT32_MAX);
  L.chunk_cap = (int32_t)((L.pair_cap + kEmitChunk - 1) / kEmitChunk);
  // Grids of the latency-bound stages (152 SMs): full-GPU by default, or at
  // most k blocks per SM for preprocess and the radix passes and 2k for the
  // emission when other work shares the GPU (stage_blocks_per_sm = k).
  const int k = s->stage_blocks_per_sm;
  L.pre_grid = k ? std::min(L.pre_blocks, 152 * k) : L.pre_blocks;
  L.sort_grid = 152 * (k ? k : 4);
  L.tile_sort_sub = s->inst_capacity >= kWideTileSortMinCap ? 3 : 1;
  L.tile_sort_grid = 152 * (k ? std::min(k, 3) : 3);
  L.emit_grid = std::max(1, std::min(L.chunk_cap, 152 * (k ? 2 * k : 8)));
  L.depth_blocks = (int32_t)((L.vis_cap + kDepthSortTile - 1) / kDepthSortTile);
  L.tile_blocks = (int32_t)((L.inst_cap + kInstSortTile - 1) / kInstSortTile);

  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L.counters = take(kCtrCount * sizeof(uint32_t));
  L.lb_pre = take((size_t)L.pre_blocks * sizeof(uint64_t));
  L.hist_depth = take(kMaxPasses * kRadixBins * sizeof(uint32_t));
  L.hist_tile = take(kMaxPasses * kRadixBins * sizeof(uint32_t));
  L.lb_emit = take((size_t)L.emit_blocks * sizeof(uint64_t));
  L.control_end = off;
  L.lb_chunk = take((size_t)L.chunk_cap * sizeof(uint64_t));
  L.pair_prefix = take(((size_t)L.vis_cap + 1) * sizeof(uint32_t));
  L.emit_rec = take((size_t)L.vis_cap * 48);
  L.rec_aux = take((size_t)L.vis_cap * sizeof(float4));
  L.chunk_first = take((size_t)L.chunk_cap * sizeof(uint32_t));
  const size_t vc = (size_t)L.vis_cap, ic = (size_t)L.inst_cap;
  L.rec_geom = take(vc * 16);
  L.rec_color = take(vc * 16);
  L.rec_blue = take(vc * 4);
  L.rec_tau = take(vc * 4);
  L.rec_meta = take(vc * 16);
  L.depth_key = take(vc * 4);
  for (int k = 0; k < 2; ++k) {
    L.dsort_key[k] = take(vc * 4);
    L.dsort_val[k] = take(vc * 4);
  }
  L.depth_state = take((size_t)L.depth_passes * L.depth_blocks * kRadixBins * sizeof(uint32_t));
  for (int k = 0; k < 2; ++k) {
    L.inst_key[k] = take(ic * 4);
    L.inst_val[k] = take(ic * 4);
  }
  L.tile_state = take((size_t)L.tile_passes * L.tile_blocks * kRadixBins * sizeof(uint32_t));
  L.ranges = take((size_t)L.total_tiles * 8);
  L.pix_T = take((size_t)L.total_pixels * 4);
  L.pix_last = take((size_t)L.total_pixels * 4);
  L.slot_grad = take(vc * kSlotGradFloats * sizeof(float));
  L.total = off;
  *out = L;
  return FGS4D_OK;
}

}  // namespace fgs4d

using namespace fgs4d;

extern "C" {

int fgs4d_workspace_size(const fgs4d_settings *settings, int64_t n, const fgs4d_view *views, int32_t nviews,
                         size_t *bytes_out) {
  if (!bytes_out) return FGS4D_ERR_ARG;
  Layout L;
  const int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  *bytes_out = L.total;
  return FGS4D_OK;
}

int fgs4d_workspace_layout(const fgs4d_settings *settings, int64_t n, const fgs4d_view *views, int32_t nviews,
                           fgs4d_layout *o) {
  if (!o) return FGS4D_ERR_ARG;
  Layout L;
  const int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  memset(o, 0, sizeof *o);
  o->bytes = L.total;
  o->counters = L.counters;
  o->rec_geom = L.rec_geom;
  o->rec_color = L.rec_color;
  o->rec_blue = L.rec_blue;
  o->rec_tau = L.rec_tau;
  o->rec_meta = L.rec_meta;
  o->depth_key = L.depth_key;
  o->sorted_slots = L.dsort_val[(L.depth_passes - 1) & 1];
  o->inst_tile = L.inst_key[L.tile_passes & 1];
  o->inst_slot = L.inst_val[L.tile_passes & 1];
  o->tile_ranges = L.ranges;
  o->pix_T = L.pix_T;
  o->pix_last = L.pix_last;
  o->slot_grad = L.slot_grad;
  o->vis_capacity = L.vis_cap;
  o->inst_capacity = L.inst_cap;
  o->total_tiles = L.total_tiles;
  o->total_pixels = L.total_pixels;
  return FGS4D_OK;
}

int fgs4d_preprocess(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                     const fgs4d_settings *settings, void *workspace, size_t workspace_bytes, void *stream) {
  int rc = check_gaussians(gaussians);
  if (rc) return rc;
  Layout L;
  rc = compute_layout(settings, gaussians->n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Counters, status word and the preprocess look-back states start at zero.
  cudaError_t e = cudaMemsetAsync(ws, 0, L.lb_pre + (size_t)L.pre_blocks * sizeof(uint64_t), st);
  if (e != cudaSuccess) return FGS4D_ERR_CUDA;
  PreLaunch p{gaussians, settings, &L, ws, st};
  return cuda_status(launch_preprocess(p, views, nviews));
}

int fgs4d_bin_sort(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                   void *workspace, size_t workspace_bytes, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  return cuda_status(launch_bin_sort(L, views, nviews, static_cast<unsigned char *>(workspace),
                                     static_cast<cudaStream_t>(stream)));
}

int fgs4d_bin_sort_kernels(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                           int32_t *count_out) {
  if (!count_out) return FGS4D_ERR_ARG;
  Layout L;
  const int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  *count_out = bin_sort_kernel_count(L, nviews);
  return FGS4D_OK;
}

int fgs4d_render_fwd(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                     void *workspace, size_t workspace_bytes, float *out_rgb, float *out_T, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  if (!out_rgb) return FGS4D_ERR_ARG;
  return cuda_status(launch_render_fwd(L, settings, views, nviews, static_cast<unsigned char *>(workspace), out_rgb,
                                       out_T, nullptr, nullptr, static_cast<cudaStream_t>(stream)));
}

int fgs4d_render_image(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                       void *workspace, size_t workspace_bytes, float *out_rgb, float *out_T, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  if (!out_rgb) return FGS4D_ERR_ARG;
  return cuda_status(launch_render_fwd(L, settings, views, nviews, static_cast<unsigned char *>(workspace), out_rgb,
                                       out_T, nullptr, nullptr, static_cast<cudaStream_t>(stream), true));
}

int fgs4d_render_aux(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                     const fgs4d_settings *settings, void *workspace, size_t workspace_bytes, float flow_dt,
                     float *out_rgb, float *out_T, float *out_aux, void *stream) {
  int rc = check_gaussians(gaussians);
  if (rc) return rc;
  Layout L;
  rc = compute_layout(settings, gaussians->n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  if (!out_rgb || !out_aux || !std::isfinite(flow_dt)) return FGS4D_ERR_ARG;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PreLaunch p{gaussians, settings, &L, ws, st};
  cudaError_t e = launch_aux_records(p, views, nviews, flow_dt);
  if (e != cudaSuccess) return FGS4D_ERR_CUDA;
  return cuda_status(launch_render_fwd(L, settings, views, nviews, ws, out_rgb, out_T, nullptr, out_aux, st));
}

int fgs4d_render_stats(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                       void *workspace, size_t workspace_bytes, float *out_rgb, uint64_t *stats_out, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  if (!out_rgb || !stats_out || ((uintptr_t)stats_out & 7u)) return FGS4D_ERR_ARG;
  return cuda_status(launch_render_fwd(L, settings, views, nviews, static_cast<unsigned char *>(workspace), out_rgb,
                                       nullptr, reinterpret_cast<unsigned long long *>(stats_out), nullptr,
                                       static_cast<cudaStream_t>(stream)));
}

namespace {

int check_grads(const fgs4d_gaussians *gaussians, const fgs4d_gaussians_grad *grads) {
  if (!grads) return FGS4D_ERR_ARG;
  if (gaussians->n > 0) {
    if (!grads->mean || !grads->log_scale || !grads->q_l || !grads->q_r || !grads->opacity_logit || !grads->sh)
      return FGS4D_ERR_ARG;
    if (!aligned16(grads->mean) || !aligned16(grads->log_scale) || !aligned16(grads->q_l) ||
        !aligned16(grads->q_r) || !aligned16(grads->sh) || !aligned16(grads->densify_stats))
      return FGS4D_ERR_ARG;
  }
  return FGS4D_OK;
}

int render_bwd_common(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                      const fgs4d_settings *settings, void *workspace, size_t workspace_bytes, const float *dL_drgb,
                      const float *dL_daux, const fgs4d_gaussians_grad *grads, void *stream) {
  int rc = check_gaussians(gaussians);
  if (rc) return rc;
  Layout L;
  rc = compute_layout(settings, gaussians->n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  if (!dL_drgb) return FGS4D_ERR_ARG;
  rc = check_grads(gaussians, grads);
  if (rc) return rc;
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_render_bwd(L, settings, views, nviews, ws, dL_drgb, dL_daux, st);
  if (e != cudaSuccess) return FGS4D_ERR_CUDA;
  PreLaunch p{gaussians, settings, &L, ws, st};
  return cuda_status(launch_preprocess_bwd(p, views, nviews, grads));
}

}  // namespace

int fgs4d_render_bwd(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                     const fgs4d_settings *settings, void *workspace, size_t workspace_bytes, const float *dL_drgb,
                     const fgs4d_gaussians_grad *grads, void *stream) {
  return render_bwd_common(gaussians, views, nviews, settings, workspace, workspace_bytes, dL_drgb, nullptr, grads,
                           stream);
}

int fgs4d_render_bwd_composite(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                               void *workspace, size_t workspace_bytes, const float *dL_drgb, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  if (!dL_drgb) return FGS4D_ERR_ARG;
  return cuda_status(launch_render_bwd(L, settings, views, nviews, static_cast<unsigned char *>(workspace), dL_drgb,
                                       nullptr, static_cast<cudaStream_t>(stream)));
}

int fgs4d_render_bwd_preprocess(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                                const fgs4d_settings *settings, void *workspace, size_t workspace_bytes,
                                const fgs4d_gaussians_grad *grads, void *stream) {
  int rc = check_gaussians(gaussians);
  if (rc) return rc;
  Layout L;
  rc = compute_layout(settings, gaussians->n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  rc = check_grads(gaussians, grads);
  if (rc) return rc;
  PreLaunch p{gaussians, settings, &L, static_cast<unsigned char *>(workspace), static_cast<cudaStream_t>(stream)};
  return cuda_status(launch_preprocess_bwd(p, views, nviews, grads));
}

int fgs4d_render_aux_bwd(const fgs4d_gaussians *gaussians, const fgs4d_view *views, int32_t nviews,
                         const fgs4d_settings *settings, void *workspace, size_t workspace_bytes,
                         const float *dL_drgb, const float *dL_daux, const fgs4d_gaussians_grad *grads,
                         void *stream) {
  if (!dL_daux) return FGS4D_ERR_ARG;
  return render_bwd_common(gaussians, views, nviews, settings, workspace, workspace_bytes, dL_drgb, dL_daux, grads,
                           stream);
}

int fgs4d_split_gaussians(const fgs4d_gaussians *src, const int32_t *idx, int64_t m, int32_t k_children,
                          const float *eps, float shrink, const fgs4d_settings *settings,
                          const fgs4d_gaussians_out *dst, void *stream) {
  int rc = check_gaussians(src);
  if (rc) return rc;
  rc = check_settings(settings);
  if (rc) return rc;
  if (m < 0 || k_children < 1 || k_children > 64 || !dst || !(shrink > 0.f) || !std::isfinite(shrink))
    return FGS4D_ERR_ARG;
  if (m == 0) return FGS4D_OK;
  if (src->n == 0 || !idx || !eps || !aligned16(eps)) return FGS4D_ERR_ARG;
  if (m > ((int64_t)INT32_MAX - 1024) / k_children || dst->n < m * k_children) return FGS4D_ERR_ARG;
  const void *ptrs[6] = {dst->mean, dst->log_scale, dst->q_l, dst->q_r, dst->opacity_logit, dst->sh};
  for (int k = 0; k < 6; ++k)
    if (!ptrs[k]) return FGS4D_ERR_ARG;
  if (!aligned16(dst->mean) || !aligned16(dst->log_scale) || !aligned16(dst->q_l) || !aligned16(dst->q_r))
    return FGS4D_ERR_ARG;
  const int32_t k3 = (settings->sh_degree + 1) * (settings->sh_degree + 1) * (settings->t_order + 1) * 3;
  return cuda_status(launch_split(src, idx, m, k_children, eps, shrink, k3, dst, static_cast<cudaStream_t>(stream)));
}

namespace {

int check_features(int64_t n, const float *features, int32_t D, const float *gate) {
  if (!feature_dim_supported(D)) return FGS4D_ERR_UNSUPPORTED;
  if (n > 0 && (!features || !aligned16(features))) return FGS4D_ERR_ARG;
  (void)gate;
  return FGS4D_OK;
}

}  // namespace

int fgs4d_render_features(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                          void *workspace, size_t workspace_bytes, const float *features, int32_t D,
                          const float *gate, float *out_features, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  rc = check_features(n, features, D, gate);
  if (rc) return rc;
  if (!out_features) return FGS4D_ERR_ARG;
  return cuda_status(launch_render_features(L, views, nviews, static_cast<unsigned char *>(workspace), n, features,
                                            D, gate, out_features, nullptr, nullptr, nullptr,
                                            static_cast<cudaStream_t>(stream)));
}

int fgs4d_render_features_bwd(int64_t n, const fgs4d_view *views, int32_t nviews, const fgs4d_settings *settings,
                              void *workspace, size_t workspace_bytes, const float *features, int32_t D,
                              const float *gate, const float *dL_dfeatures, float *grad_features,
                              float *grad_gate, void *stream) {
  Layout L;
  int rc = compute_layout(settings, n, views, nviews, &L);
  if (rc) return rc;
  rc = check_workspace(L, workspace, workspace_bytes);
  if (rc) return rc;
  rc = check_features(n, features, D, gate);
  if (rc) return rc;
  if (!dL_dfeatures || (n > 0 && !grad_features)) return FGS4D_ERR_ARG;
  return cuda_status(launch_render_features(L, views, nviews, static_cast<unsigned char *>(workspace), n, features,
                                            D, gate, nullptr, dL_dfeatures, grad_features, grad_gate,
                                            static_cast<cudaStream_t>(stream)));
}

int fgs4d_adam_tick(int32_t *step, void *stream) {
  if (!step) return FGS4D_ERR_ARG;
  return cuda_status(launch_adam_tick(step, static_cast<cudaStream_t>(stream)));
}

int fgs4d_adam_update(float *param, const float *grad, float *exp_avg, float *exp_avg_sq, int64_t count, float lr,
                      float beta1, float beta2, float eps, const int32_t *step, void *stream) {
  if (count < 0 || !step) return FGS4D_ERR_ARG;
  if (count == 0) return FGS4D_OK;
  if (!param || !grad || !exp_avg || !exp_avg_sq) return FGS4D_ERR_ARG;
  if (!aligned16(param) || !aligned16(grad) || !aligned16(exp_avg) || !aligned16(exp_avg_sq)) return FGS4D_ERR_ARG;
  if (!finite_f(lr) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return FGS4D_ERR_ARG;
  return cuda_status(launch_adam(param, grad, exp_avg, exp_avg_sq, count, lr, beta1, beta2, eps, step,
                                 static_cast<cudaStream_t>(stream)));
}

int fgs4d_adam_update_set(const fgs4d_adam_tensor *tensors, int32_t ntensors, float beta1, float beta2, float eps,
                          const int32_t *step, int32_t zero_grad, void *stream) {
  static_assert(FGS4D_ADAM_MAX_TENSORS == kAdamMaxTensors, "tensor table sizes");
  if (ntensors < 0 || ntensors > FGS4D_ADAM_MAX_TENSORS || !step || (ntensors > 0 && !tensors))
    return FGS4D_ERR_ARG;
  if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f)) return FGS4D_ERR_ARG;
  AdamTensorDev dev[kAdamMaxTensors];
  for (int32_t k = 0; k < ntensors; ++k) {
    const fgs4d_adam_tensor &t = tensors[k];
    if (t.count < 0 || !finite_f(t.lr)) return FGS4D_ERR_ARG;
    if (t.count > 0 && (!t.param || !t.grad || !t.exp_avg || !t.exp_avg_sq || !aligned16(t.param) ||
                        !aligned16(t.grad) || !aligned16(t.exp_avg) || !aligned16(t.exp_avg_sq)))
      return FGS4D_ERR_ARG;
    dev[k] = AdamTensorDev{t.param, t.grad, t.exp_avg, t.exp_avg_sq, t.count, t.lr};
  }
  return cuda_status(launch_adam_set(dev, ntensors, beta1, beta2, eps, step, zero_grad != 0,
                                     static_cast<cudaStream_t>(stream)));
}

int fgs4d_mask_loss(const float *mask_logit, int64_t n, float *loss_out, float *grad_out, void *stream) {
  if (n < 0 || (n > 0 && (!mask_logit || !loss_out || !grad_out))) return FGS4D_ERR_ARG;
  return cuda_status(launch_mask_loss(mask_logit, n, loss_out, grad_out, static_cast<cudaStream_t>(stream)));
}

int fgs4d_l1_loss(const float *img, const float *target, int64_t count, float *loss_out, float *dL_dimg,
                  void *stream) {
  if (count < 0 || (count > 0 && (!img || !target || !loss_out || !dL_dimg))) return FGS4D_ERR_ARG;
  return cuda_status(launch_l1_loss(img, target, count, count, loss_out, dL_dimg, static_cast<cudaStream_t>(stream)));
}

int fgs4d_l1_loss_part(const float *img, const float *target, int64_t count, int64_t mean_count, float *loss_out,
                       float *dL_dimg, void *stream) {
  if (count < 0 || mean_count < count || mean_count <= 0 ||
      (count > 0 && (!img || !target || !loss_out || !dL_dimg)))
    return FGS4D_ERR_ARG;
  return cuda_status(launch_l1_loss(img, target, count, mean_count, loss_out, dL_dimg,
                                    static_cast<cudaStream_t>(stream)));
}

int fgs4d_get_status(const void *workspace, size_t workspace_bytes, void *stream, int64_t *counts_out) {
  if (!workspace || workspace_bytes < kCtrCount * sizeof(uint32_t)) return FGS4D_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return FGS4D_ERR_CUDA;
  uint32_t c[8];
  if (cudaMemcpy(c, workspace, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return FGS4D_ERR_CUDA;
  if (counts_out) {
    counts_out[0] = c[kCtrVisible];
    counts_out[1] = c[kCtrInstances];
    counts_out[2] = c[kCtrNeedVisible];
    counts_out[3] = c[kCtrNeedInstances];
  }
  const uint32_t s = c[kCtrStatus];
  if (s & (kStatusVisOverflow | kStatusInstOverflow)) return FGS4D_ERR_CAPACITY;
  if (s & kStatusTimeout) return FGS4D_ERR_TIMEOUT;
  if (s & kStatusInternal) return FGS4D_ERR_INTERNAL;
  return FGS4D_OK;
}

const char *fgs4d_status_string(int status) {
  switch (status) {
    case FGS4D_OK: return "ok";
    case FGS4D_ERR_ARG: return "invalid argument";
    case FGS4D_ERR_CUDA: return "CUDA runtime error";
    case FGS4D_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FGS4D_ERR_CAPACITY: return "visible or instance capacity exceeded";
    case FGS4D_ERR_TIMEOUT: return "bounded inter-block wait ran out";
    case FGS4D_ERR_INTERNAL: return "internal consistency check failed";
    case FGS4D_ERR_UNSUPPORTED: return "setting outside the compiled range";
    default: return "unknown status";
  }
}

}  // extern "C"
