// Internal declarations shared by the CUDA translation units of the fgs4d
// library.  Nothing here is part of the C ABI (include/fgs4d.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fgs4d.h"

namespace fgs4d {

constexpr int kTile = 16;           // default tile edge in pixels (8 is the other supported size)
constexpr int kTilePixels = kTile * kTile;
constexpr int kPreBlock = 256;      // threads per preprocess block
constexpr int kEmitBlock = 256;     // threads per pair-scan / emission block
constexpr int kEmitChunk = 2048;    // (slot, rect tile) pairs per emission chunk
constexpr int kSortThreads = 256;   // threads per radix block
constexpr int kSortItems = 8;       // keys per thread per radix block (instance sort)
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kDepthSortItems = 4;  // keys per thread per radix block of the depth sort
constexpr int kDepthSortTile = kSortThreads * kDepthSortItems;
constexpr int kInstSortItems = 8;   // keys per thread per radix block of the instance (tile-id) sort
constexpr int kInstSortTile = kSortThreads * kInstSortItems;
// Instance capacity from which the instance sort takes three sub-tiles per
// ticket (a third of the look-backs, fewer resident blocks).
constexpr int64_t kWideTileSortMinCap = int64_t(1) << 26;
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kMaxPasses = 4;
constexpr int kSlotGradFloats = 12;

// Status bits of the workspace status word.
constexpr unsigned kStatusVisOverflow = 1u;
constexpr unsigned kStatusInstOverflow = 2u;
constexpr unsigned kStatusTimeout = 4u;
constexpr unsigned kStatusInternal = 8u;

// Bounded inter-block waits: polls (each followed by a short sleep) before a
// wait gives up, records kStatusTimeout and proceeds with clamped indices.
constexpr uint32_t kSpinLimit = 1u << 21;

// uint32 counters at workspace offset 0.
enum Counter : int {
  kCtrVisible = 0,
  kCtrInstances = 1,
  kCtrStatus = 2,
  kCtrNeedVisible = 3,
  kCtrNeedInstances = 4,
  kCtrTicketPre = 5,
  // bytes [0, 32) are reset by preprocess only; the rest by bin_sort as well
  kCtrTicketEmit = 8,
  kCtrTicketChunk = 9,
  kCtrTicketDepth = 10,  // kMaxPasses entries
  kCtrTicketTile = 14,   // kMaxPasses entries
  kCtrPairs = 19,        // (slot, rect tile) pairs of all visible slots
  kCtrCount = 64
};
constexpr size_t kSortControlStart = 32;

// ------------------------------------------------------------ view tables

struct PreView {
  float W[9];
  float T[3];
  float fx, fy, cx, cy;
  float campos[3];
  float t;
  int32_t width, height, gw, gh;
  int32_t tile;     // tile edge in pixels
  float inv_tile;
};

template <int MAXV>
struct PreViews {
  PreView v[MAXV];
};

struct RasterView {
  int32_t tile_base, gw, gh, width, height, tile;  // tile: edge in pixels
  int64_t pix_base;
};

template <int MAXV>
struct RasterViews {
  RasterView v[MAXV];
  int32_t nviews;
  int32_t total_tiles;
};

// ------------------------------------------------------- workspace layout

struct Layout {
  size_t counters;
  size_t lb_pre;        // uint64 per preprocess block
  size_t hist_depth;    // uint32 [kMaxPasses][256]
  size_t hist_tile;     // uint32 [kMaxPasses][256]
  size_t lb_emit;       // uint64 per pair-scan block
  size_t lb_chunk;      // uint64 per emission chunk: look-back state (cleared by the pair scan)
  size_t pair_prefix;   // uint32 [vis_cap + 1]: exclusive prefix of rect areas in depth order
  size_t emit_rec;      // 3 x 16 B [vis_cap]: emission record per depth-sorted position
  size_t rec_aux;       // float4 [vis_cap]: (camera depth, flow_u, flow_v, 0) per slot (auxiliary render)
  size_t chunk_first;   // uint32 [chunk_cap]: depth-sorted position holding each chunk's first pair
  size_t control_end;
  size_t rec_geom, rec_color, rec_blue, rec_tau, rec_meta;
  size_t depth_key;                 // uint32 per slot (written by preprocess)
  size_t dsort_key[2], dsort_val[2];  // depth-sort ping-pong buffers
  size_t depth_state;   // uint32 [kMaxPasses][depth_blocks][256]
  size_t inst_key[2], inst_val[2];
  size_t tile_state;    // uint32 [kMaxPasses][tile_blocks][256]
  size_t ranges;
  size_t pix_T, pix_last;
  size_t slot_grad;
  size_t total;

  int64_t n;
  int32_t nviews;
  int32_t tile;           // tile edge in pixels (8 or 16)
  int64_t vis_cap, inst_cap;
  int64_t total_tiles, total_pixels;
  int32_t pre_blocks_per_view, pre_blocks;
  int32_t emit_blocks;    // pair-scan blocks (one visible slot per thread)
  int64_t pair_cap;       // max (slot, rect tile) pairs: 8 x inst_cap, at most 2^31 - 1
  int32_t chunk_cap;      // emission chunks of kEmitChunk pairs
  int32_t emit_grid;      // persistent emission blocks
  int32_t pre_grid;       // persistent preprocess blocks
  int32_t sort_grid;      // persistent radix-pass blocks (at most; one radix tile each at least)
  int32_t tile_sort_sub;  // sub-tiles of kInstSortTile keys per ticket of the instance sort (1 or 3)
  int32_t tile_sort_grid; // persistent instance-sort blocks with 3 sub-tiles per ticket
  int32_t depth_blocks, tile_blocks;
  int32_t depth_passes, tile_passes;
  int32_t tile_bits;
};

// Host: computes the layout; returns FGS4D_OK or an error code.
int compute_layout(const fgs4d_settings *s, int64_t n, const fgs4d_view *views, int32_t nviews, Layout *out);

// --------------------------------------------------------- device helpers

// Programmatic dependent launch.  Every kernel of the pipeline starts with
// grid_dependency_sync(): it waits until the grid before it on the stream has
// completed and its writes are visible, then lets the next grid be launched,
// so that grid's launch overlaps this one's work.  The wait comes first in
// every block, including blocks that exit at once, which makes the completion
// of each grid imply the completion of all earlier ones.  Without the launch
// attribute (launch_pdl) both instructions are no-ops.
__device__ __forceinline__ void grid_dependency_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                                   cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                              Args... args) {
  return launch_pdl_smem(kernel, grid, block, 0, st, args...);
}

// Lets `kernel` take `bytes` of dynamic shared memory (above the 48 KB
// default); set on the current device (a per-function attribute, not a
// stream operation, so it may run while a stream is being captured).
template <typename... KArgs>
inline cudaError_t allow_dynamic_smem(void (*kernel)(KArgs...), size_t bytes) {
  return cudaFuncSetAttribute(reinterpret_cast<const void *>(kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Relaxed (non-ordering) accesses for look-back words whose flag and value
// share one word: a reader needs only that word, and no block reads data
// that another block of the same launch published beside it, so no
// acquire / release ordering is needed.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Decoupled look-back over uint64 block states (flag in bits 62-63: 1 =
// aggregate only, 2 = inclusive prefix).  Called by one thread of logical
// block `bid` with the block's aggregate; returns the exclusive prefix.
// Predecessors hold smaller tickets, so they are resident or finished and the
// wait ends; the poll count is still bounded.
__device__ __forceinline__ uint64_t lookback_u64(uint64_t *state, int32_t bid, uint64_t agg, uint32_t *status) {
  constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62, kMask = (1ull << 62) - 1;
  if (bid == 0) {
    st_relaxed(&state[0], kInc | agg);
    return 0;
  }
  st_relaxed(&state[bid], kAgg | agg);
  uint64_t prefix = 0;
  int32_t j = bid - 1;
  uint32_t polls = 0;
  while (j >= 0) {
    const uint64_t s = ld_relaxed(&state[j]);
    const uint64_t f = s & ~kMask;
    if (f == 0) {
      if (++polls > kSpinLimit) {
        atomicOr(status, kStatusTimeout);
        break;
      }
      __nanosleep(32);
      continue;
    }
    prefix += s & kMask;
    if (f == kInc) break;
    --j;
  }
  st_relaxed(&state[bid], kInc | (prefix + agg));
  return prefix;
}

// The same look-back run by a whole warp, reading 32 predecessor states per
// step: lane i looks at block (window - i).  The walk stops at the nearest
// inclusive prefix; a lane that is not ready yet makes the warp poll again
// (bounded).  Every lane returns the exclusive prefix; lane 0 publishes.
__device__ __forceinline__ uint64_t lookback_u64_warp(uint64_t *state, int32_t bid, uint64_t agg,
                                                      uint32_t *status) {
  constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62, kMask = (1ull << 62) - 1;
  const int lane = threadIdx.x & 31;
  if (bid == 0) {
    if (lane == 0) st_relaxed(&state[0], kInc | agg);
    return 0;
  }
  if (lane == 0) st_relaxed(&state[bid], kAgg | agg);
  uint64_t prefix = 0;
  int32_t window = bid - 1;
  uint32_t polls = 0;
  while (true) {
    const int32_t j = window - lane;
    const uint64_t s = j >= 0 ? ld_relaxed(&state[j]) : kInc;  // before block 0: inclusive 0
    const uint64_t f = s & ~kMask;
    const uint32_t not_ready = __ballot_sync(0xffffffffu, f == 0);
    const uint32_t inc = __ballot_sync(0xffffffffu, f == kInc);
    const uint32_t stop = not_ready | inc;
    const int first = stop ? __ffs(stop) - 1 : 32;  // nearest lane that is pending or inclusive
    if (first < 32 && ((not_ready >> first) & 1u)) {
      if (++polls > kSpinLimit) {
        if (lane == 0) atomicOr(status, kStatusTimeout);
        break;
      }
      __nanosleep(32);
      continue;
    }
    uint64_t v = lane <= first ? (s & kMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (first < 32) break;  // reached an inclusive prefix
    window -= 32;
  }
  if (lane == 0) st_relaxed(&state[bid], kInc | (prefix + agg));
  return prefix;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x == 256).
// `smem` needs 8 + 1 words.  Returns the exclusive prefix; *total = sum.
template <int kWarps = 8>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *smem, uint32_t *total) {
  static_assert(kWarps >= 1 && kWarps <= 32, "one warp scans the warp totals");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? smem[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kWarps) smem[lane] = wi - w;
    if (lane == kWarps - 1) smem[kWarps] = wi;
  }
  __syncthreads();
  const uint32_t r = smem[warp] + inc - x;
  *total = smem[kWarps];
  __syncthreads();
  return r;
}

// Shared alpha evaluation of the compositor, used verbatim by the forward
// and backward kernels so both take identical skip/stop decisions.  The
// exponent in base 2 is power2 = -q with q = (a1 dx)^2 + (b1 dx + b2 dy)^2
// (the conic A' dx^2 + B' dx dy + C' dy^2 with A' = a1^2 + b1^2, B' = 2 b1 b2,
// C' = b2^2, as a sum of two squares), so that a thread covering a column of
// pixels computes the dx terms once per entry and no term cancels.  The
// record holds la = log2 a instead of the opacity a, and la is folded into
// the dx term: a 2^-q = 2^-(q - la), one exponential and no product per
// pixel.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The base-2 exponent of a record is q = (a1 dx)^2 + (b1 dx + b2 dy)^2 with
// geom = (u, v, a1, b1), color.x = b2 and (dx, dy) = (u, v) - pixel centre.
// A thread's pixels share dx, so the column terms are formed once per entry:
// adx2 = (a1 dx)^2 - log2 a and bdx = b1 dx.
struct ColumnTerms {
  float dx, adx2, bdx;
};

__device__ __forceinline__ ColumnTerms column_terms(float4 geom, float pxc, float la) {
  ColumnTerms c;
  c.dx = __fsub_rn(geom.x, pxc);
  const float ax = __fmul_rn(geom.z, c.dx);
  c.adx2 = __fmaf_rn(ax, ax, -la);
  c.bdx = __fmul_rn(geom.w, c.dx);
  return c;
}

// Pixel rows are taken in groups of four (rows 4m .. 4m + 3).  At row y the
// second factor w = b2 (v - (y + 0.5)) + b1 dx is evaluated as
// fma(b2, -(y mod 4), w4) from the group's w4 = fma(b2, v - (4m + 0.5), b1 dx):
// one FFMA per pixel once w4 is formed per entry, and the same rounding for
// a pixel whatever the block's strip shape, so every compositor (forward,
// backward, features) takes the same alpha bit for bit.
__device__ __forceinline__ float row_group_centre(int32_t y) { return (float)(y & ~3) + 0.5f; }
__device__ __forceinline__ float row_offset(int32_t y) { return -(float)(y & 3); }
__device__ __forceinline__ float group_w(const ColumnTerms &c, float v, float b2, float gyc) {
  return __fmaf_rn(b2, __fsub_rn(v, gyc), c.bdx);
}

struct AlphaEval {
  float aG, alpha;  // aG = a 2^-q before the 0.99 clamp
};

// min(x, y) that returns NaN when either operand is NaN (fminf returns the
// other operand), so a NaN alpha fails every "alpha >= 1/255" test.
__device__ __forceinline__ float min_nan(float x, float y) {
  float r;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
  return r;
}

// A pixel that has stopped (or lies outside the image) is given the row
// offset +inf: w = +inf (or NaN when b2 = 0) makes q = +inf (or NaN), so
// alpha is 0 (or NaN) and fails the 1/255 test without a separate per-pixel
// flag test.
__device__ __forceinline__ float stopped_offset() { return __int_as_float(0x7f800000); }

// alpha = min(0.99, a 2^-q).  The clamp can only act for a > 0.98: with
// q >= 0 (a positive definite form, up to rounding) a 2^-q stays below 0.99
// otherwise.  Every compositor decides per entry with entry_clamps() and
// evaluates pixel_alpha<false> for the entries that cannot clamp, so the
// forward, backward and feature passes take the same alpha bit for bit.
constexpr float kLog2NoClamp = -0.0291463f;  // log2(0.98)
__device__ __forceinline__ bool entry_clamps(float la) { return la > kLog2NoClamp; }

// w4: group_w of the pixel's row group; off: row_offset of its row (or
// stopped_offset); b2: color.x of the record.
template <bool kClamp>
__device__ __forceinline__ AlphaEval pixel_alpha(const ColumnTerms &c, float w4, float b2, float off) {
  AlphaEval e;
  const float w = __fmaf_rn(b2, off, w4);
  e.aG = ex2_approx(-__fmaf_rn(w, w, c.adx2));
  e.alpha = kClamp ? min_nan(0.99f, e.aG) : e.aG;
  return e;
}

__device__ __forceinline__ AlphaEval pixel_alpha(const ColumnTerms &c, float w4, float b2, float off, bool clamp) {
  return clamp ? pixel_alpha<true>(c, w4, b2, off) : pixel_alpha<false>(c, w4, b2, off);
}

constexpr float kAlphaMin = 1.0f / 255.0f;
// log2 a of a staged entry that no pixel may take: alpha <= 2^-100, and
// 2^100 (the 1/a of the backward) stays finite.
constexpr float kLogAlphaNone = -100.0f;
constexpr float kTauMargin = 4e-3f;  // log2 units (0.3% in alpha)
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Sum over the 32 lanes of a warp (every lane gets the total).
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// [start, end) of a tile's list; a tile without instances may hold any
// start >= end (the sort writes (0xffffffff, 0)) and reads as (0, 0).
__device__ __forceinline__ uint2 tile_range(const uint2 *ranges, int32_t gt) {
  const uint2 r = ranges[gt];
  return r.x < r.y ? r : make_uint2(0u, 0u);
}

// Global tile -> its view (binary search over the views' first tiles).
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

// ------------------------------------------------------ host-side launchers

struct PreLaunch {
  const fgs4d_gaussians *g;
  const fgs4d_settings *s;
  const Layout *L;
  unsigned char *ws;
  cudaStream_t stream;
};

cudaError_t launch_preprocess(const PreLaunch &p, const fgs4d_view *views, int32_t nviews);
cudaError_t launch_preprocess_bwd(const PreLaunch &p, const fgs4d_view *views, int32_t nviews,
                                  const fgs4d_gaussians_grad *grads);
cudaError_t launch_bin_sort(const Layout &L, const fgs4d_view *views, int32_t nviews, unsigned char *ws,
                            cudaStream_t stream);
// Kernel launches launch_bin_sort makes for this layout on the current device.
int bin_sort_kernel_count(const Layout &L, int32_t nviews);
// image_only: no last-contributor index is tracked (fgs4d_render_image).
cudaError_t launch_render_fwd(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                              unsigned char *ws, float *out_rgb, float *out_T, unsigned long long *stats,
                              float *out_aux, cudaStream_t stream, bool image_only = false);
bool feature_dim_supported(int32_t D);
cudaError_t launch_render_features(const Layout &L, const fgs4d_view *views, int32_t nviews, unsigned char *ws,
                                   int64_t n, const float *feat, int32_t D, const float *gate, float *out,
                                   const float *dL_dF, float *g_feat, float *g_gate, cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t count, float lr, float b1, float b2,
                        float eps, const int32_t *step, cudaStream_t stream);
cudaError_t launch_adam_tick(int32_t *step, cudaStream_t stream);
// One tensor of a multi-tensor Adam step (fgs4d_adam_update_set).
constexpr int kAdamMaxTensors = 16;
struct AdamTensorDev {
  float *p, *g, *m, *v;
  int64_t count;
  float lr;
};
cudaError_t launch_adam_set(const AdamTensorDev *tensors, int32_t n, float b1, float b2, float eps,
                            const int32_t *step, bool zero_grad, cudaStream_t stream);
cudaError_t launch_mask_loss(const float *mask_logit, int64_t n, float *loss, float *grad, cudaStream_t stream);
cudaError_t launch_aux_records(const PreLaunch &p, const fgs4d_view *views, int32_t nviews, float flow_dt);
cudaError_t launch_split(const fgs4d_gaussians *src, const int32_t *idx, int64_t m, int32_t k_children,
                         const float *eps, float shrink, int32_t k3, const fgs4d_gaussians_out *dst,
                         cudaStream_t stream);
cudaError_t launch_render_bwd(const Layout &L, const fgs4d_settings *s, const fgs4d_view *views, int32_t nviews,
                              unsigned char *ws, const float *dL_drgb, const float *dL_daux, cudaStream_t stream);
cudaError_t launch_l1_loss(const float *img, const float *target, int64_t count, int64_t mean_count, float *loss,
                           float *grad, cudaStream_t stream);

// Fills a raster view table; returns false if nviews exceeds MAXV.
template <int MAXV>
inline bool make_raster_views(const Layout &L, const fgs4d_view *views, int32_t nviews, RasterViews<MAXV> *out) {
  if (nviews > MAXV) return false;
  int64_t tb = 0, pb = 0;
  for (int v = 0; v < nviews; ++v) {
    RasterView &r = out->v[v];
    r.width = views[v].width;
    r.height = views[v].height;
    r.gw = (views[v].width + L.tile - 1) / L.tile;
    r.gh = (views[v].height + L.tile - 1) / L.tile;
    r.tile_base = (int32_t)tb;
    r.pix_base = pb;
    r.tile = L.tile;
    tb += (int64_t)r.gw * r.gh;
    pb += (int64_t)r.width * r.height;
  }
  for (int v = nviews; v < MAXV; ++v) out->v[v] = RasterView{};
  out->nviews = nviews;
  out->total_tiles = (int32_t)tb;
  return true;
}

}  // namespace fgs4d
