// Per-tile front-to-back compositing (Sec. 3.2, Eq. 6 of arXiv 2412.20720)
// and its reverse-mode derivative, plus the photometric L1 loss (Sec. 3.3).
//
// Forward: one CTA per (view, 16x16 tile).  A thread owns a vertical strip of
// kPPT pixels of one column, so the per-entry work that does not depend on the
// row (shared-memory loads, dx, (a1 dx)^2, b1 dx) is done once for kPPT pixels.
// The tile's depth-sorted list is staged through shared memory in batches of
// 256 records; the CTA stops loading once every pixel has reached the
// transmittance cutoff (__syncthreads_count).  alpha = min(0.99, a 2^-q),
// skip when alpha < 1/255, stop before the entry that would take T below 1e-4
// -- evaluated by pixel_alpha, shared with the backward pass so both take
// bit-identical decisions.  The power > 0 skip of the reference rasteriser is
// not taken: q is a positive definite form, so q < 0 only arises by rounding
// next to the Gaussian's centre, where skipping would drop the entry.
//
// Backward: the same tiles traversed back to front from each pixel's last
// composited entry, recomputing T_i = T_{i+1} / (1 - alpha_i) from the final
// transmittance.  A thread first sums its strip's contributions; the sums are
// then reduced across the warp by shuffles and added with two float4 and one
// float2 atomic per warp and entry.
#include <algorithm>
#include <type_traits>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {


struct RenderArgs {
  const uint2 *ranges;
  const uint32_t *inst_val;
  const float4 *rec_geom, *rec_color;  // rec_geom: (u, v, a1, b1); rec_color: (b2, log2 a, r, g)
  const float *rec_blue;
  const float4 *rec_aux;  // auxiliary mode only
  uint32_t vis_cap;
  float *out_rgb, *out_T;
  float *out_aux;  // [views][4][H][W]: depth, opacity, flow_u, flow_v (auxiliary mode only)
  float *pix_T;
  uint32_t *pix_last;
  float bg0, bg1, bg2;
};

struct RenderBwdArgs {
  const uint2 *ranges;
  const uint32_t *inst_val;
  const float4 *rec_geom, *rec_color;
  const float *rec_blue;
  const float4 *rec_aux;  // auxiliary mode only
  uint32_t vis_cap;
  const float *pix_T;
  const uint32_t *pix_last;
  const float *dL_drgb;
  const float *dL_daux;  // [views][4][H][W] (depth, opacity used), auxiliary mode only
  float4 *slot_grad;
  float bg0, bg1, bg2;
};

// Pixels per thread of the compositor kernels (the autotuned block shape):
// 16x16 tiles take 2, 4 (default) or 8, 8x8 tiles 1 or 2 (default).
inline int render_ppt(const fgs4d_settings *s) {
  if (s->tile == 8) return s->pixels_per_thread == 1 ? 1 : 2;
  return (s->pixels_per_thread == 2 || s->pixels_per_thread == 8) ? s->pixels_per_thread : 4;
}


// Stages records [base, min(base + kBatch, end)) of the tile list into shared
// memory; slots out of range (only possible after a recorded timeout) stage a
// record that every pixel skips.
template <int NT, int kBatch>
__device__ __forceinline__ void stage_batch(const uint32_t *inst_val, const float4 *rec_geom,
                                            const float4 *rec_color, const float *rec_blue, uint32_t vis_cap,
                                            uint32_t base, uint32_t end, float4 *s_geom, float4 *s_col,
                                            float *s_blue, uint32_t *s_slot, const float4 *rec_aux = nullptr,
                                            float4 *s_aux = nullptr) {
#pragma unroll
  for (int i = 0; i < kBatch / NT; ++i) {
    const int k = threadIdx.x + i * NT;
    const uint32_t idx = base + k;
    if (idx < end) {
      const uint32_t s = inst_val[idx];
      if (s_slot) s_slot[k] = s;
      if (s < vis_cap) {
        s_geom[k] = rec_geom[s];
        s_col[k] = rec_color[s];
        s_blue[k] = rec_blue[s];
        if (s_aux) s_aux[k] = rec_aux[s];
      } else {
        s_geom[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_col[k] = make_float4(0.f, kLogAlphaNone, 0.f, 0.f);
        s_blue[k] = 0.f;
        if (s_aux) s_aux[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

// kMode 0: image (and the per-pixel state of the backward pass); 3: image
// only -- no last-contributor index is tracked (the plane is written as 0);
// 1 (kStats): also counts the pixel-entry alpha evaluations, the composited
// entries and the evaluations up to each pixel's last composited entry (the
// ones the backward pass repeats) -- a diagnostic variant used to state the
// algorithmic work; 2 (kAux): also blends the per-slot depth and flow with
// the colour weights and writes depth, opacity 1 - T and flow planes.
// A pixel that has stopped is marked by a negative T (its final transmittance
// negated; a live pixel always has T >= 1e-4) and by the row offset +inf,
// which makes every later alpha fail the 1/255 test, so the inner loop tests
// no flag.  The update stays a branch: whole warps skip it for entries that
// miss all their pixels.
// Resident blocks per SM asked of the compiler for the image-only form of the
// 64-thread 4-pixel-strip blocks: 20 (at most 51 registers a thread, 48 used,
// no spills) instead of 18 at 56, for frames rendered concurrently.  The form
// that keeps the backward's state (mode 0) loses with the same bound.
template <int TILE, int PPT, int kMode>
constexpr int fwd_min_blocks() {
  return (TILE == 16 && PPT == 4 && kMode == 3) ? 20 : 1;
}

template <int MAXV, int TILE, int PPT, int kMode, int kBatch>
__global__ void __launch_bounds__(TILE *TILE / PPT, (fwd_min_blocks<TILE, PPT, kMode>()))
    render_fwd_kernel(RenderArgs A, RasterViews<MAXV> rv, unsigned long long *stats) {
  grid_dependency_sync();
  constexpr bool kStats = kMode == 1, kAux = kMode == 2, kTrack = kMode != 3;
  constexpr int NT = TILE * TILE / PPT;
  __shared__ float4 s_geom[kBatch];
  __shared__ float4 s_col[kBatch];
  __shared__ float s_blue[kBatch];
  __shared__ float4 s_aux[kAux ? kBatch : 1];
  const int32_t gt = blockIdx.x;
  const RasterView &V = rv.v[find_view<MAXV>(rv, gt)];
  const int32_t lt = gt - V.tile_base;
  const int32_t tx = lt % V.gw, ty = lt / V.gw;
  const int32_t px = tx * TILE + (threadIdx.x & (TILE - 1));
  const int32_t py0 = ty * TILE + (threadIdx.x / TILE) * PPT;
  const uint2 range = tile_range(A.ranges, gt);
  const float pxc = (float)px + 0.5f;
  // Row groups of the strip (one for strips of up to 4 rows, which never
  // straddle a group; PPT / 4 otherwise) and each pixel's row offset.
  constexpr int kGroups = (PPT + 3) / 4;
  float gyc[kGroups];
#pragma unroll
  for (int g = 0; g < kGroups; ++g) gyc[g] = row_group_centre(py0 + 4 * g);
  float T[PPT], C0[PPT], C1[PPT], C2[PPT], off[PPT];
  float X0[kAux ? PPT : 1], X1[kAux ? PPT : 1], X2[kAux ? PPT : 1];  // depth, flow_u, flow_v sums
  uint32_t last[PPT];
  uint32_t pend[kStats ? PPT : 1];  // evaluations since the pixel's last composited entry
  int nlive = 0;  // pixels of this thread still compositing
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const bool in = px < V.width && py0 + k < V.height;
    if (kStats) pend[k] = 0u;
    T[k] = in ? 1.0f : -1.0f;
    C0[k] = C1[k] = C2[k] = 0.f;
    if (kAux) X0[k] = X1[k] = X2[k] = 0.f;
    last[k] = 0u;
    off[k] = in ? row_offset(py0 + k) : stopped_offset();
    nlive += in;
  }
  uint32_t n_eval = 0u, n_comp = 0u, n_evb = 0u;
  for (uint32_t base = range.x; base < range.y; base += kBatch) {
    if (__syncthreads_count(nlive > 0) == 0) break;
    stage_batch<NT, kBatch>(A.inst_val, A.rec_geom, A.rec_color, A.rec_blue, A.vis_cap, base, range.y, s_geom, s_col,
                    s_blue, nullptr, kAux ? A.rec_aux : nullptr, kAux ? s_aux : nullptr);
    const int nb = (int)min(range.y - base, (uint32_t)kBatch);
    // Whether any staged entry can reach the 0.99 clamp (opacity > 0.98, rare):
    // each thread checks the entries it staged, and the barrier that
    // publishes the batch ORs the answers.
    bool my_clamp = false;
#pragma unroll
    for (int i = 0; i < kBatch / NT; ++i) {
      const int k = threadIdx.x + i * NT;
      if (k < nb) my_clamp = my_clamp || entry_clamps(s_col[k].y);
    }
    const bool clamp_any = __syncthreads_or(my_clamp) != 0;
    const uint32_t pos0 = base - range.x + 1u;
    // One entry of the list at every pixel of the thread; the clamp case is a
    // separate copy of the pixel loop.
    auto entry = [&](int j, auto clamp_tag) {
      const float4 geom = s_geom[j];
      const float4 col = s_col[j];
      const float blue = s_blue[j];
      const float4 xa = kAux ? s_aux[j] : make_float4(0.f, 0.f, 0.f, 0.f);  // depth and flow of the entry
      const ColumnTerms ct = column_terms(geom, pxc, col.y);
      float w4[kGroups];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) w4[g] = group_w(ct, geom.y, col.x, gyc[g]);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const AlphaEval e = pixel_alpha<decltype(clamp_tag)::value>(ct, w4[k >> 2], col.x, off[k]);
        if (kStats) {
          n_eval += T[k] > 0.0f;
          pend[k] += T[k] > 0.0f;
        }
        if (e.alpha >= kAlphaMin) {  // false for stopped pixels (row offset +inf)
          const float w = __fmul_rn(e.alpha, T[k]);
          const float Tn = __fsub_rn(T[k], w);
          if (Tn < kTMin) {
            T[k] = -T[k];
            off[k] = stopped_offset();
            --nlive;
          } else {
            C0[k] = __fmaf_rn(col.z, w, C0[k]);
            C1[k] = __fmaf_rn(col.w, w, C1[k]);
            C2[k] = __fmaf_rn(blue, w, C2[k]);
            if (kAux) {
              X0[k] = __fmaf_rn(xa.x, w, X0[k]);
              X1[k] = __fmaf_rn(xa.y, w, X1[k]);
              X2[k] = __fmaf_rn(xa.z, w, X2[k]);
            }
            T[k] = Tn;
            if (kTrack) last[k] = pos0 + (uint32_t)j;
            if (kStats) {
              ++n_comp;
              n_evb += pend[k];
              pend[k] = 0u;
            }
          }
        }
      }
    };
    if (clamp_any) {
      for (int j = 0; j < nb && nlive > 0; ++j) {
        if (entry_clamps(s_col[j].y)) entry(j, std::true_type());
        else entry(j, std::false_type());
      }
    } else {
      // No entry of the batch can clamp: two entries per iteration, the
      // liveness test once per pair (a pixel that stopped at the first
      // takes no alpha from the second: its row offset is +inf).
      int j = 0;
      for (; j + 1 < nb && nlive > 0; j += 2) {
        entry(j, std::false_type());
        entry(j + 1, std::false_type());
      }
      if (j < nb && nlive > 0) entry(j, std::false_type());
    }
  }
  if (kStats) {
    unsigned long long ev = n_eval, co = n_comp, eb = n_evb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_xor_sync(0xffffffffu, ev, o);
      co += __shfl_xor_sync(0xffffffffu, co, o);
      eb += __shfl_xor_sync(0xffffffffu, eb, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], ev);
      atomicAdd(&stats[1], co);
      atomicAdd(&stats[2], eb);
    }
  }
  const int64_t HW = (int64_t)V.width * V.height;
  float *img = A.out_rgb + V.pix_base * 3;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!(px < V.width && py0 + k < V.height)) continue;
    const int64_t p = (int64_t)(py0 + k) * V.width + px;
    const float Tend = fabsf(T[k]);
    img[p] = C0[k] + Tend * A.bg0;
    img[HW + p] = C1[k] + Tend * A.bg1;
    img[2 * HW + p] = C2[k] + Tend * A.bg2;
    A.pix_T[V.pix_base + p] = Tend;
    A.pix_last[V.pix_base + p] = kTrack ? last[k] : 0u;
    if (A.out_T) A.out_T[V.pix_base + p] = Tend;
    if (kAux) {
      float *aux = A.out_aux + V.pix_base * 4;
      aux[p] = X0[k];
      aux[HW + p] = 1.0f - Tend;
      aux[2 * HW + p] = X1[k];
      aux[3 * HW + p] = X2[k];
    }
  }
}

// Sums eight per-lane values over the warp with 9 shuffles instead of 40: at
// each halving step a lane keeps half of its values and trades the other half
// with its partner.  On return a[0] of lane l holds the warp total of value
// l >> 2.
__device__ __forceinline__ void warp_sum8_transposed(float (&a)[8], int lane) {
  const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0, u4 = (lane & 4) != 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = u16 ? a[i] : a[i + 4];
    const float keep = u16 ? a[i + 4] : a[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = u8 ? a[i] : a[i + 2];
    const float keep = u8 ? a[i + 2] : a[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const float send = u4 ? a[0] : a[1];
    const float keep = u4 ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 2);
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// 1/x to within an ulp or so (MUFU reciprocal); the backward pass only needs
// T recovered to the accuracy of its own accumulated rounding.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// kAux: the loss also has gradients dL/dD, dL/dO with respect to the depth
// and opacity channels (zero background, x_i = z_i resp. 1 in the colour
// rule); adds dL/dz_i = sum dL/dD alpha_i T_i per slot.
template <int MAXV, int TILE, int kPPT, bool kAux, int kBatch>
__global__ void __launch_bounds__(TILE *TILE / kPPT) render_bwd_kernel(RenderBwdArgs A, RasterViews<MAXV> rv) {
  grid_dependency_sync();
  constexpr int kRenderThreads = TILE * TILE / kPPT;
  __shared__ float4 s_geom[kBatch];
  __shared__ float4 s_col[kBatch];
  __shared__ float s_blue[kBatch];
  __shared__ float4 s_aux[kAux ? kBatch : 1];
  __shared__ uint32_t s_slot[kBatch];
  __shared__ uint32_t s_maxlast;
  const int32_t gt = blockIdx.x;
  const RasterView &V = rv.v[find_view<MAXV>(rv, gt)];
  const int32_t lt = gt - V.tile_base;
  const int32_t tx = lt % V.gw, ty = lt / V.gw;
  const int32_t px = tx * TILE + (threadIdx.x & (TILE - 1));
  const int32_t py0 = ty * TILE + (threadIdx.x / TILE) * kPPT;
  const uint2 range = tile_range(A.ranges, gt);
  const float pxc = (float)px + 0.5f;
  const int64_t HW = (int64_t)V.width * V.height;
  // Dr[k] = sum over channels of dL/dX * (X composited behind the current
  // entry), X = R, G, B (and depth, opacity): the "behind" terms of
  // dL/dalpha enter only through this sum, which grows by w * (dL/dX . x_i).
  constexpr int kGroups = (kPPT + 3) / 4;  // row groups of the strip (see group_w)
  float gyc[kGroups];
#pragma unroll
  for (int g = 0; g < kGroups; ++g) gyc[g] = row_group_centre(py0 + 4 * g);
  // Row offsets of the strip's pixels within their groups: -(k mod 4) when
  // the strip starts a group (4 and 8 rows), else -((py0 + k) mod 4).
  const float base_off = row_offset(py0);
  float T[kPPT], dC0[kPPT], dC1[kPPT], dC2[kPPT], Dr[kPPT], off[kPPT];
  float dD[kAux ? kPPT : 1], dO[kAux ? kPPT : 1];
  uint32_t last[kPPT];
  uint32_t my_max = 0u;
  const float *g = A.dL_drgb + V.pix_base * 3;
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    off[k] = row_offset(py0 + k);
    T[k] = 1.0f;
    dC0[k] = dC1[k] = dC2[k] = 0.f;
    last[k] = 0u;
    if (px < V.width && py0 + k < V.height) {
      const int64_t p = (int64_t)(py0 + k) * V.width + px;
      T[k] = A.pix_T[V.pix_base + p];
      last[k] = A.pix_last[V.pix_base + p];
      dC0[k] = g[p];
      dC1[k] = g[HW + p];
      dC2[k] = g[2 * HW + p];
    }
    if (kAux) {
      dD[k] = dO[k] = 0.f;
      if (px < V.width && py0 + k < V.height) {
        const int64_t p = (int64_t)(py0 + k) * V.width + px;
        const float *ga = A.dL_daux + V.pix_base * 4;
        dD[k] = ga[p];
        dO[k] = ga[HW + p];
      }
    }
    Dr[k] = T[k] * (dC0[k] * A.bg0 + dC1[k] * A.bg1 + dC2[k] * A.bg2);  // the background behind all
    my_max = max(my_max, last[k]);
  }
  if (threadIdx.x == 0) s_maxlast = 0u;
  __syncthreads();
  if (my_max) atomicMax(&s_maxlast, my_max);
  __syncthreads();
  const uint32_t end = range.x + min(s_maxlast, range.y - range.x);
  const int lane = threadIdx.x & 31;
  const int nbatch = (int)((end - range.x + kBatch - 1) / kBatch);
  for (int bi = nbatch - 1; bi >= 0; --bi) {
    const uint32_t base = range.x + (uint32_t)bi * kBatch;
    __syncthreads();
    stage_batch<kRenderThreads, kBatch>(A.inst_val, A.rec_geom, A.rec_color, A.rec_blue, A.vis_cap, base, end, s_geom,
                                s_col, s_blue, s_slot, kAux ? A.rec_aux : nullptr, kAux ? s_aux : nullptr);
    __syncthreads();
    const int nb = (int)min(end - base, (uint32_t)kBatch);
    // One list entry; kClamp is the entry's clamp case (entry_clamps), taken
    // per entry as in the forward so that pixels evaluate pixel_alpha<false>
    // without a per-pixel select for the vast majority of entries.
    auto entry = [&](int j, uint32_t pos, auto clamp_tag) {
      constexpr bool kClamp = decltype(clamp_tag)::value;
      const float4 geom = s_geom[j];
      const float4 col = s_col[j];
      const float blue = s_blue[j];
      const ColumnTerms ct = column_terms(geom, pxc, col.y);
      // group_w, keeping v - (group row centre) for the pixels' dy
      float dy4[kGroups], w4[kGroups];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        dy4[g] = __fsub_rn(geom.y, gyc[g]);
        w4[g] = __fmaf_rn(col.x, dy4[g], ct.bdx);
      }
      // The conic and centre gradients of the strip share dx: accumulate the
      // moments S0 = sum gp, S1 = sum gp dy, S2 = sum gp dy^2 of
      // gp = dL/d(natural-log power) and form the five sums once per entry.
      // A pixel that is not skipped has alpha = a 2^-q (below the clamp), so
      // gp = g_alpha a 2^-q is also the opacity term: dL/da = S0 / a.
      // Per row group: P0 = sum gp, P1 = sum o gp, P2 = sum o^2 gp with the
      // pixel's dy = dyb - o, o = k mod 4 (a constant of the unrolled loop),
      // so that S1 = dyb P0 - P1 and S2 = dyb^2 P0 - 2 dyb P1 + P2 follow
      // once per entry.
      float P0[kGroups], P1[kGroups], P2[kGroups];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) P0[g] = P1[g] = P2[g] = 0.f;
      float gr = 0.f, gg = 0.f, gb = 0.f, gz = 0.f;
      const float zj = kAux ? s_aux[j].x : 0.f;
      bool contrib = false;
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        if (pos >= last[k]) continue;
        const AlphaEval e = pixel_alpha<kClamp>(ct, w4[k >> 2], col.x, kPPT >= 4 ? -(float)(k & 3) : off[k]);
        if (!(e.alpha >= kAlphaMin)) continue;  // the forward's skip decision, NaN included
        contrib = true;
        const float io = rcp_approx(__fsub_rn(1.0f, e.alpha));
        T[k] = T[k] * io;  // transmittance in front of this entry
        const float w = e.alpha * T[k];
        gr += dC0[k] * w;
        gg += dC1[k] * w;
        gb += dC2[k] * w;
        float Dc = dC0[k] * col.z + dC1[k] * col.w + dC2[k] * blue;  // dL/dX . x_i
        if (kAux) {
          Dc += dD[k] * zj + dO[k];
          gz += dD[k] * w;
        }
        const float g_alpha = T[k] * Dc - io * Dr[k];
        Dr[k] += w * Dc;
        if (!(kClamp && e.aG > 0.99f)) {  // min(0.99, .) is locally constant when clamped
          const float gp = g_alpha * e.alpha;  // d alpha / d (natural-log power)
          const float o = (float)(k & 3);
          P0[k >> 2] += gp;
          if (k & 3) {
            P1[k >> 2] = __fmaf_rn(o, gp, P1[k >> 2]);
            P2[k >> 2] = __fmaf_rn(o * o, gp, P2[k >> 2]);
          }
        }
      }
      if (!__any_sync(0xffffffffu, contrib)) return;
      // the strip's moments S0 = sum gp, S1 = sum gp dy, S2 = sum gp dy^2
      float S0 = 0.f, S1 = 0.f, S2 = 0.f;
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        const float dyb = dy4[g] + base_off;  // dy of the group's first row in the strip
        S0 += P0[g];
        S1 += dyb * P0[g] - P1[g];
        S2 += dyb * (dyb * P0[g] - 2.0f * P1[g]) + P2[g];
      }
      const float dx = ct.dx;
      // the natural-log conic (A, B, C) of the record's factors: A' = a1^2 +
      // b1^2, B' = 2 b1 b2, C' = b2^2 in base 2
      const float An = 2.0f * kLn2 * __fmaf_rn(geom.z, geom.z, geom.w * geom.w);
      const float Bn = 2.0f * kLn2 * (geom.w * col.x), Cn = 2.0f * kLn2 * (col.x * col.x);
      // g = (du, dv, dA', dB', dC', da, dr, dg), plus db.
      float g[8] = {-(An * dx * S0 + Bn * S1), -(Cn * S1 + Bn * dx * S0), -0.5f * dx * dx * S0, -dx * S1,
                    -0.5f * S2, S0 * ex2_approx(-col.y), gr, gg};
      warp_sum8_transposed(g, lane);
      gb = warp_sum(gb);
      if (kAux) gz = warp_sum(gz);
      // Lane 4k holds sum k: lanes 0 and 16 gather sums 0-3 and 4-7 and add
      // them with one vector atomic each; lane 1 adds (db, dz).
      const float s1 = __shfl_down_sync(0xffffffffu, g[0], 4);
      const float s2 = __shfl_down_sync(0xffffffffu, g[0], 8);
      const float s3 = __shfl_down_sync(0xffffffffu, g[0], 12);
      const uint32_t slot = s_slot[j];
      if (slot < A.vis_cap) {
        float4 *dst = A.slot_grad + 3 * (size_t)slot;
        if ((lane & 15) == 0) atomicAdd(dst + (lane >> 4), make_float4(g[0], s1, s2, s3));
        else if (lane == 1) atomicAdd(reinterpret_cast<float2 *>(dst + 2), make_float2(gb, kAux ? gz : 0.0f));
      }
    };
    for (int j = nb - 1; j >= 0; --j) {
      const uint32_t pos = base + j - range.x;  // entry index in the tile list
      if (!__any_sync(0xffffffffu, pos < my_max)) continue;  // no pixel of this warp reached it
      if (entry_clamps(s_col[j].y)) entry(j, pos, std::true_type());
      else entry(j, pos, std::false_type());
    }
  }
}

__global__ void l1_loss_kernel(const float *__restrict__ img, const float *__restrict__ target, int64_t count,
                               float inv_count, float *loss, float *grad) {
  grid_dependency_sync();
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

// Adam (the optimiser of the training step): with t the device step count,
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps).
struct AdamArgs {
  float *p;
  const float *g;
  float *m, *v;
  int64_t count;
  float lr, b1, b2, eps;
  const int32_t *step;
};

__device__ __forceinline__ float adam_one(float &p, float g, float &m, float &v, float b1, float b2, float eps,
                                          float step_size, float inv_sqrt_bc2) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  p -= step_size * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
  return p;
}

__global__ void adam_kernel(AdamArgs A) {
  grid_dependency_sync();
  const float t = (float)*A.step;
  const float bc1 = 1.0f - powf(A.b1, t), bc2 = 1.0f - powf(A.b2, t);
  const float step_size = A.lr / bc1, inv_sqrt_bc2 = rsqrtf(bc2);
  const int64_t n4 = A.count / 4;
  float4 *p4 = reinterpret_cast<float4 *>(A.p);
  const float4 *g4 = reinterpret_cast<const float4 *>(A.g);
  float4 *m4 = reinterpret_cast<float4 *>(A.m);
  float4 *v4 = reinterpret_cast<float4 *>(A.v);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 p = p4[i], m = m4[i], v = v4[i];
    const float4 g = g4[i];
    adam_one(p.x, g.x, m.x, v.x, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
    adam_one(p.y, g.y, m.y, v.y, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
    adam_one(p.z, g.z, m.z, v.z, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
    adam_one(p.w, g.w, m.w, v.w, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
    p4[i] = p;
    m4[i] = m;
    v4[i] = v;
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.count; i += stride)
    adam_one(A.p[i], A.g[i], A.m[i], A.v[i], A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
}

// Adam over a set of tensors in one launch: unit u of the set is float4 u -
// first[k] of tensor k (the last unit of a tensor whose count is not a
// multiple of 4 takes its 1-3 trailing scalars).  Each element gets exactly
// adam_one, as in adam_kernel; with zero the gradient is cleared after it is
// read, so the next step accumulates into zeros without a separate fill.
struct AdamSetArgs {
  AdamTensorDev t[kAdamMaxTensors];
  int64_t first[kAdamMaxTensors + 1];  // prefix of the tensors' unit counts
  int32_t n;
  float b1, b2, eps;
  const int32_t *step;
  int32_t zero;
};

__global__ void adam_set_kernel(AdamSetArgs A) {
  grid_dependency_sync();
  const float t = (float)*A.step;
  const float bc1 = 1.0f - powf(A.b1, t), bc2 = 1.0f - powf(A.b2, t);
  const float inv_sqrt_bc2 = rsqrtf(bc2);
  const int64_t total = A.first[A.n];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int k = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += stride) {
    while (u >= A.first[k + 1]) ++k;  // units only grow along the loop
    const AdamTensorDev &T = A.t[k];
    const float step_size = T.lr / bc1;
    const int64_t i = u - A.first[k];
    if (4 * i + 4 <= T.count) {
      float4 *p4 = reinterpret_cast<float4 *>(T.p) + i;
      float4 *g4 = reinterpret_cast<float4 *>(T.g) + i;
      float4 *m4 = reinterpret_cast<float4 *>(T.m) + i;
      float4 *v4 = reinterpret_cast<float4 *>(T.v) + i;
      float4 p = *p4, m = *m4, v = *v4;
      const float4 g = *g4;
      adam_one(p.x, g.x, m.x, v.x, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
      adam_one(p.y, g.y, m.y, v.y, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
      adam_one(p.z, g.z, m.z, v.z, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
      adam_one(p.w, g.w, m.w, v.w, A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
      *p4 = p;
      *m4 = m;
      *v4 = v;
      if (A.zero) *g4 = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int64_t e = 4 * i; e < T.count; ++e) {
        adam_one(T.p[e], T.g[e], T.m[e], T.v[e], A.b1, A.b2, A.eps, step_size, inv_sqrt_bc2);
        if (A.zero) T.g[e] = 0.f;
      }
    }
  }
}

__global__ void adam_tick_kernel(int32_t *step) {
  grid_dependency_sync();
  if (threadIdx.x == 0) *step += 1;
}

// Mask compression loss (Sec. 4.3): L = mean sigmoid(m), dL/dm = M (1 - M) / n.
__global__ void mask_loss_kernel(const float *__restrict__ m, int64_t n, float inv_n, float *loss, float *grad) {
  grid_dependency_sync();
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float M = 1.0f / (1.0f + expf(-m[i]));
    acc += M;
    grad[i] += M * (1.0f - M) * inv_n;
  }
  acc = warp_sum(acc);
  __shared__ float s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.f;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(loss, v * inv_n);
  }
}

template <int MAXV, int TILE, int PPT, int B>
cudaError_t launch_fwd_batch(const RenderArgs &A, const RasterViews<MAXV> &rv, unsigned grid,
                             unsigned long long *stats, bool image_only, cudaStream_t st) {
  constexpr unsigned NT = TILE * TILE / PPT;
  if (image_only)
    return launch_pdl(render_fwd_kernel<MAXV, TILE, PPT, 3, B>, grid, NT, st, A, rv, (unsigned long long *)nullptr);
  if (stats) return launch_pdl(render_fwd_kernel<MAXV, TILE, PPT, 1, B>, grid, NT, st, A, rv, stats);
  if (A.out_aux)
    return launch_pdl(render_fwd_kernel<MAXV, TILE, PPT, 2, B>, grid, NT, st, A, rv, (unsigned long long *)nullptr);
  return launch_pdl(render_fwd_kernel<MAXV, TILE, PPT, 0, B>, grid, NT, st, A, rv, (unsigned long long *)nullptr);
}

template <int MAXV, int TILE, int PPT>
cudaError_t launch_fwd_ppt(const RenderArgs &A, const RasterViews<MAXV> &rv, unsigned grid,
                           unsigned long long *stats, int batch, bool image_only, cudaStream_t st) {
  if (batch == 128) return launch_fwd_batch<MAXV, TILE, PPT, 128>(A, rv, grid, stats, image_only, st);
  return launch_fwd_batch<MAXV, TILE, PPT, 256>(A, rv, grid, stats, image_only, st);
}

template <int MAXV>
cudaError_t render_fwd_typed(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                             unsigned char *ws, float *out_rgb, float *out_T, unsigned long long *stats,
                             float *out_aux, bool image_only, cudaStream_t st) {
  RasterViews<MAXV> rv;
  if (!make_raster_views<MAXV>(L, views, nviews, &rv)) return cudaErrorInvalidValue;
  RenderArgs A;
  A.ranges = reinterpret_cast<const uint2 *>(ws + L.ranges);
  A.inst_val = reinterpret_cast<const uint32_t *>(ws + L.inst_val[L.tile_passes & 1]);
  A.rec_geom = reinterpret_cast<const float4 *>(ws + L.rec_geom);
  A.rec_color = reinterpret_cast<const float4 *>(ws + L.rec_color);
  A.rec_blue = reinterpret_cast<const float *>(ws + L.rec_blue);
  A.rec_aux = reinterpret_cast<const float4 *>(ws + L.rec_aux);
  A.vis_cap = (uint32_t)L.vis_cap;
  A.out_rgb = out_rgb;
  A.out_T = out_T;
  A.out_aux = out_aux;
  A.pix_T = reinterpret_cast<float *>(ws + L.pix_T);
  A.pix_last = reinterpret_cast<uint32_t *>(ws + L.pix_last);
  A.bg0 = s->bg[0];
  A.bg1 = s->bg[1];
  A.bg2 = s->bg[2];
  if (L.total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)L.total_tiles;
  if (s->tile == 8) {
    if (render_ppt(s) == 1) return launch_fwd_ppt<MAXV, 8, 1>(A, rv, grid, stats, s->shared_batch, image_only, st);
    return launch_fwd_ppt<MAXV, 8, 2>(A, rv, grid, stats, s->shared_batch, image_only, st);
  }
  switch (render_ppt(s)) {
    case 2: return launch_fwd_ppt<MAXV, 16, 2>(A, rv, grid, stats, s->shared_batch, image_only, st);
    case 8: return launch_fwd_ppt<MAXV, 16, 8>(A, rv, grid, stats, s->shared_batch, image_only, st);
    default: return launch_fwd_ppt<MAXV, 16, 4>(A, rv, grid, stats, s->shared_batch, image_only, st);
  }
}

template <int MAXV, int TILE, int PPT, int B>
cudaError_t launch_bwd_batch(const RenderBwdArgs &A, const RasterViews<MAXV> &rv, unsigned grid, cudaStream_t st) {
  constexpr unsigned NT = TILE * TILE / PPT;
  if (A.dL_daux) return launch_pdl(render_bwd_kernel<MAXV, TILE, PPT, true, B>, grid, NT, st, A, rv);
  return launch_pdl(render_bwd_kernel<MAXV, TILE, PPT, false, B>, grid, NT, st, A, rv);
}

template <int MAXV, int TILE, int PPT>
cudaError_t launch_bwd_ppt(const RenderBwdArgs &A, const RasterViews<MAXV> &rv, unsigned grid, int batch,
                           cudaStream_t st) {
  if (batch == 128) return launch_bwd_batch<MAXV, TILE, PPT, 128>(A, rv, grid, st);
  return launch_bwd_batch<MAXV, TILE, PPT, 256>(A, rv, grid, st);
}

template <int MAXV>
cudaError_t render_bwd_typed(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                             unsigned char *ws, const float *dL_drgb, const float *dL_daux, cudaStream_t st) {
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
  A.dL_daux = dL_daux;
  A.rec_aux = reinterpret_cast<const float4 *>(ws + L.rec_aux);
  A.slot_grad = reinterpret_cast<float4 *>(ws + L.slot_grad);
  A.bg0 = s->bg[0];
  A.bg1 = s->bg[1];
  A.bg2 = s->bg[2];
  if (L.total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)L.total_tiles;
  if (s->tile == 8) {
    if (render_ppt(s) == 1) return launch_bwd_ppt<MAXV, 8, 1>(A, rv, grid, s->shared_batch, st);
    return launch_bwd_ppt<MAXV, 8, 2>(A, rv, grid, s->shared_batch, st);
  }
  switch (render_ppt(s)) {
    case 2: return launch_bwd_ppt<MAXV, 16, 2>(A, rv, grid, s->shared_batch, st);
    case 8: return launch_bwd_ppt<MAXV, 16, 8>(A, rv, grid, s->shared_batch, st);
    default: return launch_bwd_ppt<MAXV, 16, 4>(A, rv, grid, s->shared_batch, st);
  }
}

}  // namespace

cudaError_t launch_render_fwd(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                              unsigned char *ws, float *out_rgb, float *out_T, unsigned long long *stats,
                              float *out_aux, cudaStream_t stream, bool image_only) {
  if (nviews == 1)
    return render_fwd_typed<1>(L, s, views, nviews, ws, out_rgb, out_T, stats, out_aux, image_only, stream);
  return render_fwd_typed<FGS4D_MAX_VIEWS>(L, s, views, nviews, ws, out_rgb, out_T, stats, out_aux, image_only,
                                           stream);
}

cudaError_t launch_render_bwd(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                              unsigned char *ws, const float *dL_drgb, const float *dL_daux, cudaStream_t stream) {
  if (nviews == 1) return render_bwd_typed<1>(L, s, views, nviews, ws, dL_drgb, dL_daux, stream);
  return render_bwd_typed<FGS4D_MAX_VIEWS>(L, s, views, nviews, ws, dL_drgb, dL_daux, stream);
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t count, float lr, float b1, float b2,
                        float eps, const int32_t *step, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  AdamArgs A{p, g, m, v, count, lr, b1, b2, eps, step};
  const int blocks = (int)std::min<int64_t>((count / 4 + 255) / 256 + 1, 152 * 8);
  return launch_pdl(adam_kernel, (unsigned)blocks, 256u, stream, A);
}

cudaError_t launch_adam_set(const AdamTensorDev *tensors, int32_t n, float b1, float b2, float eps,
                            const int32_t *step, bool zero_grad, cudaStream_t stream) {
  AdamSetArgs A{};
  A.n = n;
  A.first[0] = 0;
  for (int32_t k = 0; k < n; ++k) {
    A.t[k] = tensors[k];
    A.first[k + 1] = A.first[k] + (tensors[k].count + 3) / 4;
  }
  A.b1 = b1;
  A.b2 = b2;
  A.eps = eps;
  A.step = step;
  A.zero = zero_grad ? 1 : 0;
  const int64_t total = A.first[n];
  if (total == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  return launch_pdl(adam_set_kernel, (unsigned)blocks, 256u, stream, A);
}

cudaError_t launch_adam_tick(int32_t *step, cudaStream_t stream) {
  return launch_pdl(adam_tick_kernel, 1u, 32u, stream, step);
}

cudaError_t launch_mask_loss(const float *mask_logit, int64_t n, float *loss, float *grad, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  return launch_pdl(mask_loss_kernel, (unsigned)blocks, 256u, stream, mask_logit, n, 1.0f / (float)n, loss, grad);
}

cudaError_t launch_l1_loss(const float *img, const float *target, int64_t count, int64_t mean_count, float *loss,
                           float *grad, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 8);
  return launch_pdl(l1_loss_kernel, (unsigned)blocks, 256u, stream, img, target, count, 1.0f / (float)mean_count,
                    loss, grad);
}

}  // namespace fgs4d
