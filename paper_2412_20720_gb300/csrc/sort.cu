// Tile binning and sorting for the tile rasterizer the paper adapts
// (Sec. 3.2 of arXiv 2412.20720; depth-ordered blending of Eq. 6).
//
// The required order of a tile's list is (FP32 depth, slot) ascending, where
// slots number the visible pairs in (view, Gaussian index) order.  Instead of
// sorting every (tile, Gaussian) instance on a 64-bit (tile << 32 | depth)
// key, the visible pairs are first sorted by depth alone (31 key bits, one
// element per pair), the instances are then emitted in that order, and a
// stable sort on the tile id alone (13-19 bits) groups them per tile.  Both
// sorts are stable LSD radix sorts, so the result equals the sort on the
// 64-bit key with the slot as tie-break, while the instance array (8x larger
// than the visible set at the benchmark sizes) is only passed over
// ceil(tile_bits / 8) times.
//
// Each radix pass is one kernel: blocks take tickets in launch order, rank
// their keys stably with warp ballots, publish per-digit counts and find
// their per-digit global offsets by decoupled look-back over the earlier
// tickets (bounded waits), then scatter through shared memory.
#include <algorithm>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {


constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = kFlagAgg - 1u;

// Decoupled look-back of digit d for ticket b (one or more radix sub-tiles):
// publishes the ticket's count of the digit, sums the counts of the tickets
// before it back to the nearest inclusive prefix (reading a window of kWin
// predecessors per round trip: their words are independent loads), publishes
// the ticket's inclusive prefix and returns the exclusive one.  Flag and value share one word, so relaxed
// accesses suffice.  A predecessor that never posts makes the wait give up
// after kSpinLimit polls: the timeout bit is set and the partial prefix
// returned (the caller's bounds checks keep every store in range).
__device__ __forceinline__ uint32_t radix_lookback(uint32_t *state, int64_t b, int d, uint32_t cnt, uint32_t *status) {
  constexpr int kWin = 8;
  uint32_t prefix = 0u;
  if (b == 0) {
    st_relaxed(&state[d], kFlagInc | cnt);
    return 0u;
  }
  st_relaxed(&state[b * kRadixBins + d], kFlagAgg | cnt);
  int64_t j = b - 1;
  uint32_t polls = 0;
  while (j >= 0) {
    uint32_t w[kWin];
#pragma unroll
    for (int k = 0; k < kWin; ++k) w[k] = j - k >= 0 ? ld_relaxed(&state[(j - k) * kRadixBins + d]) : kFlagInc;
    int used = 0;
    bool done = false;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      if (done || used < k) continue;  // stop at the first tile not yet posted
      const uint32_t f = w[k] & ~kValMask;
      if (f == 0u) continue;
      prefix += w[k] & kValMask;
      ++used;
      done = f == kFlagInc;
    }
    if (done) break;
    j -= used;
    if (used == 0) {
      if (++polls > kSpinLimit) {
        atomicOr(status, kStatusTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
  st_relaxed(&state[b * kRadixBins + d], kFlagInc | ((prefix + cnt) & kValMask));
  return prefix;
}

// Digit histograms of keys [0, count) for `passes` 8-bit digits starting at
// bit 0, grid-stride over radix tiles (kSortThreads x kItems keys); also
// clears each tile's look-back rows and the tile ranges.
template <int kItems>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t *__restrict__ keys,
                                                                  const uint32_t *__restrict__ count_ptr, int64_t cap,
                                                                  int32_t passes, uint32_t *hist, uint32_t *state,
                                                                  int32_t state_blocks, uint2 *ranges,
                                                                  int64_t nranges) {
  grid_dependency_sync();
  __shared__ uint32_t s_hist[kMaxPasses][kRadixBins];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nranges; r += (int64_t)gridDim.x * blockDim.x)
    ranges[r] = make_uint2(0u, 0u);
  const int64_t count = min64((int64_t)*count_ptr, cap);
  constexpr int kTileKeys = kSortThreads * kItems;
  if ((int64_t)blockIdx.x * kTileKeys >= count) return;
  for (int p = 0; p < passes; ++p) s_hist[p][threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  for (int64_t ob = blockIdx.x; ob * kTileKeys < count && ob < state_blocks; ob += gridDim.x) {
    for (int p = 0; p < passes; ++p) state[((int64_t)p * state_blocks + ob) * kRadixBins + threadIdx.x] = 0u;
#pragma unroll 2
    for (int i = 0; i < kItems; ++i) {
      const int64_t idx = ob * kTileKeys + i * kSortThreads + threadIdx.x;
      const bool valid = idx < count;
      const uint32_t k = valid ? keys[idx] : 0u;
      for (int p = 0; p < passes; ++p) {
        // The high digits of depth and tile keys take few values: a warp whose
        // lanes all share the digit adds once instead of serialising 32 times.
        const int d = valid ? (int)((k >> (kRadixBits * p)) & (kRadixBins - 1)) : -1;
        const int d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, d == d0)) {
          if (lane == 0 && d0 >= 0) atomicAdd(&s_hist[p][d0], 32u);
        } else if (valid) {
          atomicAdd(&s_hist[p][d], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = s_hist[p][threadIdx.x];
    if (c) atomicAdd(&hist[p * kRadixBins + threadIdx.x], c);
  }
}

// 16-byte asynchronous copy global -> shared; bytes past src_bytes are
// zero-filled and not read.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Waits until at most n (0..2) of this thread's copy groups are pending.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  if (n <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  else asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

// Shared memory of one radix block: the ticket's keys and values (input,
// then the block-local order), per-warp digit counts (two sets, alternating
// between sub-tiles), per-sub-tile digit starts and the digits' global
// starts.
template <int kItems, int kSub>
struct RadixSmem {
  uint32_t keys[kSortThreads * kItems * kSub];
  uint32_t vals[kSortThreads * kItems * kSub];
  uint32_t wcount[kSub > 1 ? 2 : 1][kSortThreads / 32][kRadixBins];
  uint32_t bstart[kSub][kRadixBins];  // first block-local position of each digit in sub-tile s
  uint32_t sbase[kSub][kRadixBins];   // keys of each digit in the sub-tiles before s
  uint32_t gstart[kRadixBins];        // global position of the ticket's first key of each digit
  uint32_t scan[12];
  uint32_t ticket;
};
template <int kItems, int kSub>
constexpr size_t radix_smem_bytes() {
  return sizeof(RadixSmem<kItems, kSub>);
}

// One stable 8-bit LSD pass.  A block takes tickets in launch order; a
// ticket is kSub consecutive sub-tiles of kSortThreads x kItems keys.  Each
// warp copies the keys (and values) it ranks into shared memory with
// cp.async, one copy group per sub-tile, so later sub-tiles arrive while the
// first is ranked (16-byte copies: keys_in and vals_in start on 16-byte
// boundaries, as the workspace's arrays do).  Ranking is stable within a
// warp's segment (item-major, lane-minor): the lanes holding the same digit
// are found by nine ballots
// (eight digit bits and the padding bit), and the lowest of them adds the
// group's size to the warp's count of that digit.  Each sub-tile is then
// placed in block-local digit order in its own part of the buffer.  One
// decoupled look-back per ticket gives the ticket's global start of each
// digit, and the scatter writes each sub-tile's digit runs.  Small sorts
// (the depth sort) take short sub-tiles, so that more SMs share a pass;
// very large instance sorts take three sub-tiles per ticket, which divides
// the look-backs per key by three.
//
// With `ranges` (the last pass of the tile sort, keys = global tile ids
// below total_tiles) the pass also records each tile's [start, end) in the
// sorted list.  A sub-tile's staged keys are ordered by the full key (the
// pass input is ordered by the lower digits and the staging is stable), so
// the equal keys of a sub-tile form one run; its first and last output
// positions go to atomicMin on start and atomicMax on end, which the
// emission initialised to (0xffffffff, 0).  A tile with no instance keeps
// start > end, which every reader takes as empty.
template <bool kValsAreIndex, int kItems, int kSub>
__global__ void __launch_bounds__(kSortThreads) radix_pass_kernel(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const uint32_t *__restrict__ count_ptr, int64_t cap, int32_t shift,
    const uint32_t *__restrict__ hist, uint32_t *state, uint32_t *ticket, uint32_t *status, uint2 *ranges,
    int64_t total_tiles) {
  static_assert(kSub >= 1 && kSub <= 3, "copy groups are waited for by count (at most 2 pending)");
  static_assert(kItems % 4 == 0, "whole 16-byte copies per warp segment");
  grid_dependency_sync();
  constexpr int kSubKeys = kSortThreads * kItems;
  constexpr int kTileKeys = kSubKeys * kSub;
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kSegKeys = 32 * kItems;  // keys of one warp in a sub-tile
  extern __shared__ __align__(16) unsigned char radix_smem[];
  RadixSmem<kItems, kSub> &S = *reinterpret_cast<RadixSmem<kItems, kSub> *>(radix_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t count = min64((int64_t)*count_ptr, cap);
  for (int i = threadIdx.x; i < (int)(sizeof S.wcount / sizeof(uint32_t)); i += kSortThreads) (&S.wcount[0][0][0])[i] = 0u;
  uint32_t total;
  // Keys of the digits below each digit over the whole input: the same for
  // every ticket.
  const uint32_t gpre = block_exclusive_scan(hist[threadIdx.x], S.scan, &total);
  // Persistent: tickets are taken in order, so a ticket's look-back only
  // waits on tickets that running blocks already hold.
  while (true) {
    if (threadIdx.x == 0) S.ticket = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t b = S.ticket;
    const int64_t tile0 = b * kTileKeys;
    if (tile0 >= count) return;
#pragma unroll
    for (int s = 0; s < kSub; ++s) {
      const int seg = s * kSubKeys + warp * kSegKeys;
      for (int c = lane; c < kSegKeys / 4; c += 32) {
        const int64_t i0 = tile0 + seg + 4 * c;
        if (i0 < count) {
          const int bytes = (int)min64(16, (count - i0) * 4);
          cp_async16(&S.keys[seg + 4 * c], keys_in + i0, bytes);
          if (!kValsAreIndex) cp_async16(&S.vals[seg + 4 * c], vals_in + i0, bytes);
        }
      }
      cp_async_commit();
    }
    const int d = threadIdx.x;  // the digit this thread scans and looks back for
    uint32_t tot = 0u;          // keys of digit d in the sub-tiles so far
#pragma unroll
    for (int s = 0; s < kSub; ++s) {
      uint32_t(&wc)[kWarps][kRadixBins] = S.wcount[kSub > 1 ? (s & 1) : 0];
      cp_async_wait_pending(kSub - 1 - s);
      __syncwarp();  // the warp's copies of sub-tile s are visible to all its lanes
      const int seg = s * kSubKeys + warp * kSegKeys;
      uint32_t key[kItems], val[kItems], rank[kItems];
      int dig[kItems];
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        const int li = seg + k * 32 + lane;
        if (tile0 + li < count) {
          key[k] = S.keys[li];
          val[k] = kValsAreIndex ? (uint32_t)(tile0 + li) : S.vals[li];
          dig[k] = (key[k] >> shift) & (kRadixBins - 1);
        } else {
          key[k] = 0u;
          val[k] = 0u;
          dig[k] = kRadixBins;  // padding: ranked nowhere
        }
      }
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        const int dk = dig[k];
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < 9; ++bit) {
          const uint32_t set = (uint32_t)((dk >> bit) & 1);
          peers &= ~(__ballot_sync(0xffffffffu, set) ^ (0u - set));
        }
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0u;
        if (lane == leader && dk < kRadixBins) base = atomicAdd(&wc[warp][dk], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        __syncwarp();  // item k's counts land before item k + 1's
        rank[k] = base + __popc(peers & lt_mask);
      }
      __syncthreads();
      // Per digit: exclusive prefix over warps; sub-tile count and start.
      uint32_t cnt = 0u;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wc[w][d];
        wc[w][d] = cnt;
        cnt += c;
      }
      S.sbase[s][d] = tot;
      tot += cnt;
      S.bstart[s][d] = block_exclusive_scan(cnt, S.scan, &total);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        if (dig[k] < kRadixBins) {
          const uint32_t pos = s * kSubKeys + S.bstart[s][dig[k]] + wc[warp][dig[k]] + rank[k];
          S.keys[pos] = key[k];
          S.vals[pos] = val[k];
        }
      }
      __syncwarp();
      for (int i = lane; i < kRadixBins; i += 32) wc[warp][i] = 0u;  // the warp's row, for sub-tile s + 2
    }
    S.gstart[d] = gpre + radix_lookback(state, b, d, tot, status);
    __syncthreads();
    // Coalesced runs per digit and sub-tile.
    const int32_t nvalid = (int32_t)min64(kTileKeys, count - tile0);
    for (int p = threadIdx.x; p < nvalid; p += kSortThreads) {
      const int s = p / kSubKeys, q = p - s * kSubKeys;
      const uint32_t kk = S.keys[p];
      const int dd = (kk >> shift) & (kRadixBins - 1);
      const uint32_t gpos = S.gstart[dd] + S.sbase[s][dd] + ((uint32_t)q - S.bstart[s][dd]);
      if ((int64_t)gpos < count) {
        keys_out[gpos] = kk;
        vals_out[gpos] = S.vals[p];
        if (ranges) {
          if ((int64_t)kk < total_tiles) {
            const int qend = min(kSubKeys, nvalid - s * kSubKeys);
            uint32_t *r = reinterpret_cast<uint32_t *>(&ranges[kk]);
            if (q == 0 || S.keys[p - 1] != kk) atomicMin(&r[0], gpos);
            if (q == qend - 1 || S.keys[p + 1] != kk) atomicMax(&r[1], gpos + 1u);
          } else {
            atomicOr(status, kStatusInternal);
          }
        }
      } else {
        atomicOr(status, kStatusInternal);
      }
    }
    __syncthreads();  // shared memory is reused by the next ticket
  }
}

// Does the ellipse {d : q(d) <= tau} around (u, v) meet the box [x0, x1] x
// [y0, y1] of a tile's pixel centres?  q(d) = (a1 d_x)^2 + (b1 d_x + b2 d_y)^2
// is the record's exponent as a sum of two squares.  Exact minimum of q over
// the box: 0 if the centre is inside, else the least of the four edge minima.
// On an edge d_x = X, q is least at d_y = kx X (kx = -b1 / b2), where it is
// (a1 X)^2; on an edge d_y = Y at d_x = ky Y (ky = -b1 b2 / (a1^2 + b1^2)); a
// minimiser outside the edge is clamped to it.  q is evaluated at the
// (clamped) point as the sum of two squares, so nothing cancels.  Every
// operation is an explicitly rounded FP32 operation in a fixed order, so the
// decision is reproducible bit for bit.  Entries of tiles it rejects are
// skipped at every pixel of the tile (alpha < 1/255), so dropping them leaves
// the image unchanged.  kx and ky depend on the Gaussian only and are
// computed once per slot (edge_slopes).
__device__ __forceinline__ float2 edge_slopes(float a1, float b1, float b2) {
  return make_float2(__fdiv_rn(-b1, b2),
                     __fdiv_rn(__fmul_rn(-b1, b2), __fmaf_rn(a1, a1, __fmul_rn(b1, b1))));
}

__device__ __forceinline__ float sum_sq(float a1, float b1, float b2, float x, float y) {
  const float ax = __fmul_rn(a1, x);
  const float w = __fmaf_rn(b2, y, __fmul_rn(b1, x));
  return __fmaf_rn(w, w, __fmul_rn(ax, ax));
}

__device__ __forceinline__ bool ellipse_meets_box(float u, float v, float a1, float b1, float b2, float kx,
                                                  float ky, float tau, float x0, float x1, float y0, float y1) {
  const float lx = __fsub_rn(x0, u), hx = __fsub_rn(x1, u);
  const float ly = __fsub_rn(y0, v), hy = __fsub_rn(y1, v);
  if (lx <= 0.0f && hx >= 0.0f && ly <= 0.0f && hy >= 0.0f) return tau >= 0.0f;
  float m = INFINITY;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float X = k ? hx : lx;
    const float Yv = fminf(fmaxf(__fmul_rn(kx, X), ly), hy);
    m = fminf(m, sum_sq(a1, b1, b2, X, Yv));
    const float Y = k ? hy : ly;
    const float Xv = fminf(fmaxf(__fmul_rn(ky, Y), lx), hx);
    m = fminf(m, sum_sq(a1, b1, b2, Xv, Y));
  }
  return m <= tau;
}

struct EmitArgs {
  const uint32_t *sorted_slots;
  const int4 *meta;
  const float4 *geom, *color;
  const float *tau;
  uint32_t *counters;
  int64_t vis_cap, inst_cap, pair_cap;
  int32_t chunk_cap;
  uint32_t *pair_prefix;
  int4 *emit_rec;  // 3 per depth-sorted position
  uint32_t *chunk_first;
  uint32_t *inst_key, *inst_val;
  uint64_t *lb_scan;
  uint64_t *lb_chunk;  // look-back state per emission chunk (cleared by the pair scan)
  // Tile sort set-up done while emitting: digit histograms, cleared look-back
  // rows and tile ranges.
  int32_t tile_passes, tile_blocks;
  uint32_t *hist_tile, *tile_state;
  uint2 *ranges;
  int64_t total_tiles;
};

// Emission record of depth-sorted position j holding slot s: (u, v, a1, b1),
// (b2, kx, ky, tau), (slot, view, packed rect lo, packed rect hi); returns
// the number of (slot, tile) pairs to enumerate for it.  Only tiles whose
// pixel-centre box meets the 1/255 ellipse q <= tau are kept, so the pairs
// are enumerated over the rect cut to the ellipse's bounding box: with q =
// (a1 dx)^2 + (b1 dx + b2 dy)^2 the half-extents are sqrt(tau) / a1 and
// sqrt(tau (a1^2 + b1^2)) / (a1 b2), widened by 0.1% + 0.05 px against
// rounding (a box outside them is far outside the ellipse, which the exact
// test of the emission rejects as well).  With tile
// edge T, tile tx's centre box [T tx + 0.5, T tx + T - 0.5] can meet
// [u - rx, u + rx] only for ceil((u - rx - T + 0.5) / T) <= tx <= floor((u + rx - 0.5) / T).
template <int MAXV>
__device__ __forceinline__ uint32_t pair_record(const EmitArgs &A, const RasterViews<MAXV> &rv, uint32_t s, int64_t j,
                                                int64_t nvis) {
  uint32_t area = 0u;
  int4 mm = make_int4(0, 0, 0, 0);
  float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
  float cc = 0.f, tau = -1.0f;
  if ((int64_t)s < nvis) {
    mm = A.meta[s];
    g = A.geom[s];
    cc = A.color[s].x;
    tau = A.tau[s];
    int x0 = mm.z & 0xffff, y0 = (uint32_t)mm.z >> 16, x1 = mm.w & 0xffff, y1 = (uint32_t)mm.w >> 16;
    if (tau < 0.0f) {
      x1 = x0;
    } else if (g.z > 0.0f && cc > 0.0f) {
      const RasterView &V = rv.v[MAXV == 1 ? 0 : min(max(mm.y, 0), rv.nviews - 1)];
      const float T = (float)V.tile, iT = 1.0f / T;
      const float st = sqrtf(tau);
      const float rx = st / g.z * 1.001f + 0.05f;
      const float ry = st * sqrtf(g.z * g.z + g.w * g.w) / (g.z * cc) * 1.001f + 0.05f;
      const float lx = ceilf((g.x - rx - (T - 0.5f)) * iT), hx = floorf((g.x + rx - 0.5f) * iT);
      const float ly = ceilf((g.y - ry - (T - 0.5f)) * iT), hy = floorf((g.y + ry - 0.5f) * iT);
      if (lx > (float)x0) x0 = (int)fminf(lx, (float)x1);
      if (hx + 1.0f < (float)x1) x1 = (int)fmaxf(hx + 1.0f, (float)x0);
      if (ly > (float)y0) y0 = (int)fminf(ly, (float)y1);
      if (hy + 1.0f < (float)y1) y1 = (int)fmaxf(hy + 1.0f, (float)y0);
    }
    area = (uint32_t)(max(x1 - x0, 0) * max(y1 - y0, 0));
    mm.z = x0 | (y0 << 16);
    mm.w = x1 | (y1 << 16);
  } else {
    atomicOr(&A.counters[kCtrStatus], kStatusInternal);
  }
  const float2 k = edge_slopes(g.z, g.w, cc);
  A.emit_rec[3 * j + 0] = make_int4(__float_as_int(g.x), __float_as_int(g.y), __float_as_int(g.z),
                                    __float_as_int(g.w));
  A.emit_rec[3 * j + 1] = make_int4(__float_as_int(cc), __float_as_int(k.x), __float_as_int(k.y),
                                    __float_as_int(tau));
  A.emit_rec[3 * j + 2] = make_int4((int)s, MAXV == 1 ? 0 : min(max(mm.y, 0), rv.nviews - 1), mm.z, mm.w);
  return area;
}

// Pairs [p0, p1) of depth-sorted position j: every emission chunk whose first
// pair falls among them records j and has its look-back word cleared.
__device__ __forceinline__ void mark_chunks(const EmitArgs &A, int64_t j, uint64_t p0, uint64_t p1) {
  for (uint64_t c = (p0 + kEmitChunk - 1) / kEmitChunk; c * kEmitChunk < p1 && c < (uint64_t)A.chunk_cap; ++c) {
    A.chunk_first[c] = (uint32_t)j;
    A.lb_chunk[c] = 0ull;
  }
}

// Sets the pair total (clamped to the pair capacity) and, when pairs are lost
// to the clamp, the instance bound and the overflow flag.
__device__ __forceinline__ void set_pair_total(const EmitArgs &A, int64_t nvis, uint64_t all) {
  A.pair_prefix[nvis] = (uint32_t)umin64(all, (uint64_t)A.pair_cap);
  A.counters[kCtrPairs] = (uint32_t)umin64(all, (uint64_t)A.pair_cap);
  if (all > (uint64_t)A.pair_cap) {
    // Some pairs cannot be examined: report the pair total as the bound on
    // the instances needed.
    A.counters[kCtrNeedInstances] = (uint32_t)umin64(all, 0xffffffffull);
    atomicOr(&A.counters[kCtrStatus], kStatusInstOverflow);
  }
}

// No visible slot: no pairs, no instances.
__device__ __forceinline__ void set_empty_totals(const EmitArgs &A) {
  A.counters[kCtrPairs] = 0u;
  A.counters[kCtrInstances] = 0u;
  A.counters[kCtrNeedInstances] = 0u;
}

// Pair scan, one thread per depth-sorted visible slot: the exclusive prefix
// of the slots' rect areas in depth order (decoupled look-back), plus the
// emission record of every position and the chunk marks.
template <int MAXV>
__global__ void __launch_bounds__(kEmitBlock) pair_scan_kernel(EmitArgs A, RasterViews<MAXV> rv) {
  grid_dependency_sync();
  __shared__ uint32_t s_ticket;
  __shared__ uint32_t s_scan[9];
  const int64_t nvis = min64((int64_t)A.counters[kCtrVisible], A.vis_cap);
  if (threadIdx.x == 0) s_ticket = atomicAdd(&A.counters[kCtrTicketEmit], 1u);
  __syncthreads();
  const int64_t b = s_ticket;
  if (b == 0 && nvis == 0 && threadIdx.x == 0) set_empty_totals(A);
  if (b * kEmitBlock >= nvis) return;
  const int64_t j = b * kEmitBlock + threadIdx.x;
  const uint32_t area = j < nvis ? pair_record<MAXV>(A, rv, A.sorted_slots[j], j, nvis) : 0u;
  uint32_t total;
  const uint32_t excl = block_exclusive_scan(area, s_scan, &total);
  __shared__ uint64_t s_base;
  if (threadIdx.x < 32) {
    const uint64_t prefix = lookback_u64_warp(A.lb_scan, (int32_t)b, total, &A.counters[kCtrStatus]);
    if (threadIdx.x == 0) s_base = prefix;
    if (threadIdx.x == 0 && (b + 1) * kEmitBlock >= nvis) set_pair_total(A, nvis, prefix + total);
  }
  __syncthreads();
  if (j < nvis) {
    const uint64_t p0 = umin64(s_base + excl, (uint64_t)A.pair_cap);
    const uint64_t p1 = umin64(s_base + excl + area, (uint64_t)A.pair_cap);
    A.pair_prefix[j] = (uint32_t)p0;
    mark_chunks(A, j, p0, p1);
  }
}

// Instance emission in depth order.  The (slot, rect tile) pairs of all
// visible slots, in depth order and row-major within a rect, are cut into
// chunks of kEmitChunk pairs; a pair is kept when its slot's 1/255 ellipse
// meets the tile.  emit_kernel takes chunks by ticket, decides every pair of
// a chunk, gets the chunk's output offset by a decoupled look-back over the
// chunks' kept counts, and writes the kept pairs in pair order.  Every chunk
// is the same amount of work, so a screen-sized Gaussian is spread over many
// blocks.

constexpr int kEmitRecCache = 256;  // emission records cached per chunk

// Shared-memory view of one chunk: the pair prefix and (when they fit) the
// emission records of the depth-sorted positions its pairs belong to.
struct EmitChunkSmem {
  uint32_t j0, ns;
  uint32_t pref[kEmitChunk + 1];
  int4 rec[kEmitRecCache * 3];
};

__device__ __forceinline__ void load_emit_chunk(const EmitArgs &A, uint32_t c, uint32_t f1, uint32_t npairs,
                                                int64_t nvis, EmitChunkSmem &S) {
  if (threadIdx.x == 0) {  // positions holding pair f0 and, at most one past, pair f1 - 1
    const int64_t j0 = A.chunk_first[c];
    const int64_t j1 = f1 == npairs ? nvis - 1 : (int64_t)A.chunk_first[c + 1];
    S.j0 = (uint32_t)j0;
    S.ns = (uint32_t)min64(max64(j1 - j0 + 1, 1), kEmitChunk);
  }
  __syncthreads();
  const uint32_t j0 = S.j0, ns = S.ns;
  for (uint32_t k = threadIdx.x; k <= ns; k += kEmitBlock)
    S.pref[k] = (int64_t)(j0 + k) <= nvis ? A.pair_prefix[j0 + k] : npairs;
  if (ns <= (uint32_t)kEmitRecCache)
    for (uint32_t k = threadIdx.x; k < 3 * ns; k += kEmitBlock) S.rec[k] = A.emit_rec[3 * (size_t)j0 + k];
  __syncthreads();
}

// Walk over consecutive pairs of a chunk: the depth-sorted position the
// current pair belongs to, its rect and the current tile (row-major).
struct PairWalk {
  int lo;  // position within the chunk
  int x0, y0, x1, tx, ty;
  uint32_t slot, view;
  float u, v, a1, b1, b2, kx, ky, tau;
};

__device__ __forceinline__ void walk_load(const EmitArgs &A, const EmitChunkSmem &S, int lo, PairWalk &w) {
  const int4 *er = S.ns <= (uint32_t)kEmitRecCache ? S.rec + 3 * lo : A.emit_rec + 3 * (size_t)(S.j0 + lo);
  const int4 r0 = er[0], r1 = er[1], r2 = er[2];
  w.lo = lo;
  w.u = __int_as_float(r0.x);
  w.v = __int_as_float(r0.y);
  w.a1 = __int_as_float(r0.z);
  w.b1 = __int_as_float(r0.w);
  w.b2 = __int_as_float(r1.x);
  w.kx = __int_as_float(r1.y);
  w.ky = __int_as_float(r1.z);
  w.tau = __int_as_float(r1.w);
  w.slot = (uint32_t)r2.x;
  w.view = (uint32_t)r2.y;
  w.x0 = r2.z & 0xffff;
  w.y0 = (uint32_t)r2.z >> 16;
  w.x1 = r2.w & 0xffff;
}

// Positions the walk at pair f (one binary search over the chunk's prefix).
__device__ __forceinline__ PairWalk walk_begin(const EmitArgs &A, const EmitChunkSmem &S, uint32_t f) {
  int lo = 0, hi = (int)S.ns - 1;
  while (lo < hi) {  // last position whose pair prefix is <= f
    const int mid = (lo + hi + 1) >> 1;
    if (S.pref[mid] <= f) lo = mid;
    else hi = mid - 1;
  }
  PairWalk w;
  walk_load(A, S, lo, w);
  const uint32_t local = f - S.pref[lo];
  const uint32_t wd = (uint32_t)max(w.x1 - w.x0, 1);
  const uint32_t qy = local / wd;
  w.tx = w.x0 + (int)(local - qy * wd);
  w.ty = w.y0 + (int)qy;
  return w;
}

// Advances the walk to pair f, the pair after the current one.
__device__ __forceinline__ void walk_next(const EmitArgs &A, const EmitChunkSmem &S, PairWalk &w, uint32_t f) {
  if (++w.tx >= w.x1) {
    w.tx = w.x0;
    ++w.ty;
  }
  if (S.pref[w.lo + 1] <= f) {
    int lo = w.lo + 1;
    while (S.pref[lo + 1] <= f) ++lo;  // positions without pairs (capacity clamp)
    walk_load(A, S, lo, w);
    w.tx = w.x0;
    w.ty = w.y0;
  }
}

template <int MAXV>
__device__ __forceinline__ bool walk_keep(const RasterViews<MAXV> &rv, const PairWalk &w) {
  const RasterView &V = rv.v[MAXV == 1 ? 0 : w.view];
  const int T = V.tile;
  const float bx0 = (float)(w.tx * T) + 0.5f, by0 = (float)(w.ty * T) + 0.5f;
  const float bx1 = (float)min(w.tx * T + T - 1, V.width - 1) + 0.5f;
  const float by1 = (float)min(w.ty * T + T - 1, V.height - 1) + 0.5f;
  return ellipse_meets_box(w.u, w.v, w.a1, w.b1, w.b2, w.kx, w.ky, w.tau, bx0, bx1, by0, by1);
}

template <int MAXV>
__device__ __forceinline__ uint32_t walk_tile(const RasterViews<MAXV> &rv, const PairWalk &w) {
  const RasterView &V = rv.v[MAXV == 1 ? 0 : w.view];
  return (uint32_t)(V.tile_base + w.ty * V.gw + w.tx);
}

constexpr int kPairsPerThread = kEmitChunk / kEmitBlock;
// Radix tiles of the instance sort whose look-back rows chunk c clears: the
// instances never outnumber the pairs, so rows [0, nchunks x this) suffice.
constexpr int kRadixTilesPerChunk = kEmitChunk / kInstSortTile;
static_assert(kRadixTilesPerChunk * kInstSortTile == kEmitChunk, "chunk covers whole radix tiles");
static_assert(kPairsPerThread == 8, "one keep byte per thread");

// Sets the instance total (clamped to the capacity) and its overflow flag.
__device__ __forceinline__ void set_instance_total(const EmitArgs &A, uint64_t all) {
  A.counters[kCtrInstances] = (uint32_t)umin64(all, (uint64_t)A.inst_cap);
  // A pair overflow (flagged by the pair scan) already set the bound.
  if (!(A.counters[kCtrStatus] & kStatusInstOverflow) || all > (uint64_t)A.inst_cap)
    A.counters[kCtrNeedInstances] =
        (uint32_t)umin64(max((uint64_t)A.counters[kCtrNeedInstances], all), 0xffffffffull);
  if (all > (uint64_t)A.inst_cap) atomicOr(&A.counters[kCtrStatus], kStatusInstOverflow);
}

// Thread t of chunk c decides pairs c kEmitChunk + 8 t + [0, 8) and keeps
// the tile ids and slots of the kept ones in registers; a block scan and the
// look-back over the chunks give their output positions (the pairs are staged
// in shared memory meanwhile and written with coalesced stores).  Persistent: chunks
// are taken by ticket, so a chunk's look-back only waits on chunks that
// running blocks hold.  Also clears the tile sort's look-back rows of the
// radix tiles covering chunk c's pairs (there are no more instances than
// pairs) and the tile ranges, and takes the tile-id digit histograms.
template <int MAXV>
__global__ void __launch_bounds__(kEmitBlock) emit_kernel(EmitArgs A, RasterViews<MAXV> rv) {
  grid_dependency_sync();
  __shared__ EmitChunkSmem S;
  __shared__ uint32_t s_scan[kEmitBlock / 32 + 1];
  __shared__ uint32_t s_hist[kMaxPasses][kRadixBins];
  __shared__ uint32_t s_ticket;
  __shared__ uint64_t s_prefix;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < A.total_tiles;
       r += (int64_t)gridDim.x * blockDim.x)
    A.ranges[r] = make_uint2(0xffffffffu, 0u);  // empty until the last tile-sort pass records a run
  const int64_t nvis = min64((int64_t)A.counters[kCtrVisible], A.vis_cap);
  const uint32_t npairs = A.counters[kCtrPairs];
  const uint32_t nchunks = (uint32_t)min64((npairs + kEmitChunk - 1) / kEmitChunk, A.chunk_cap);
  if (nchunks == 0u) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && nvis > 0) set_instance_total(A, 0ull);
    return;
  }
  for (int p = 0; p < A.tile_passes; ++p) s_hist[p][threadIdx.x] = 0u;
  while (true) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(&A.counters[kCtrTicketChunk], 1u);
    __syncthreads();
    const uint32_t c = s_ticket;
    if (c >= nchunks) break;
    for (int r = 0; r < kRadixTilesPerChunk; ++r) {
      const int64_t rt = (int64_t)c * kRadixTilesPerChunk + r;
      if (rt < A.tile_blocks)
        for (int p = 0; p < A.tile_passes; ++p)
          A.tile_state[((size_t)p * A.tile_blocks + rt) * kRadixBins + threadIdx.x] = 0u;
    }
    const uint32_t f0 = c * kEmitChunk, f1 = min(f0 + (uint32_t)kEmitChunk, npairs);
    load_emit_chunk(A, c, f1, npairs, nvis, S);
    const uint32_t fa = f0 + kPairsPerThread * threadIdx.x;
    uint32_t m = 0u;
    uint32_t kt[kPairsPerThread], ks[kPairsPerThread];
    if (fa < f1) {
      PairWalk w = walk_begin(A, S, fa);
#pragma unroll
      for (int k = 0; k < kPairsPerThread; ++k) {
        if (k) {
          if (fa + k >= f1) break;
          walk_next(A, S, w, fa + k);
        }
        m |= walk_keep<MAXV>(rv, w) ? (1u << k) : 0u;
        kt[k] = walk_tile<MAXV>(rv, w);
        ks[k] = w.slot;
      }
    }
    uint32_t total;
    const uint32_t local = block_exclusive_scan(__popc(m), s_scan, &total);
    // The kept pairs go to shared memory in pair order, and the tile-id
    // histograms are taken, while warp 0 looks back (it stages its own
    // afterwards); the chunk is then written with coalesced stores.  The
    // walk is over (the scan's barriers), so the chunk's records and pair
    // prefix hold the staged tile ids and slots.
    static_assert(sizeof S.rec >= kEmitChunk * sizeof(uint32_t) && sizeof S.pref >= kEmitChunk * sizeof(uint32_t),
                  "staging fits");
    uint32_t *s_stage_key = reinterpret_cast<uint32_t *>(S.rec), *s_stage_val = S.pref;
    auto stage = [&]() {
      uint32_t q = local;
#pragma unroll
      for (int k = 0; k < kPairsPerThread; ++k) {
        if (m & (1u << k)) {
          s_stage_key[q] = kt[k];
          s_stage_val[q] = ks[k];
          ++q;
          for (int p = 0; p < A.tile_passes; ++p)
            atomicAdd(&s_hist[p][(kt[k] >> (kRadixBits * p)) & (kRadixBins - 1)], 1u);
        }
      }
    };
    if (threadIdx.x >= 32) stage();
    if (threadIdx.x < 32) {
      const uint64_t prefix = lookback_u64_warp(A.lb_chunk, (int32_t)c, total, &A.counters[kCtrStatus]);
      if (threadIdx.x == 0) {
        s_prefix = prefix;
        if (c == nchunks - 1u) set_instance_total(A, prefix + total);
      }
      stage();
    }
    __syncthreads();
    const uint64_t base = s_prefix;
    for (uint32_t t = threadIdx.x; t < total; t += kEmitBlock) {
      const uint64_t pos = base + t;
      if (pos < (uint64_t)A.inst_cap) {
        A.inst_key[pos] = s_stage_key[t];
        A.inst_val[pos] = s_stage_val[t];
      }
    }
    __syncthreads();  // S, the staged pairs, s_ticket and s_prefix are reused by the next chunk
  }
  for (int p = 0; p < A.tile_passes; ++p) {
    const uint32_t h = s_hist[p][threadIdx.x];
    if (h) atomicAdd(&A.hist_tile[p * kRadixBins + threadIdx.x], h);
  }
}

template <int MAXV>
cudaError_t bin_sort_typed(const Layout &L, const fgs4d_view *views, int32_t nviews, unsigned char *ws,
                           cudaStream_t st) {
  RasterViews<MAXV> rv;
  if (!make_raster_views<MAXV>(L, views, nviews, &rv)) return cudaErrorInvalidValue;
  uint32_t *ctr = reinterpret_cast<uint32_t *>(ws + L.counters);
  uint32_t *status = ctr + kCtrStatus;
  cudaError_t e = cudaMemsetAsync(ws + kSortControlStart, 0, L.control_end - kSortControlStart, st);
  if (e != cudaSuccess) return e;
  // 1. Depth sort of the visible slots (31 key bits: depth > near > 0); the
  // per-slot keys stay intact, the passes ping-pong between two buffers.
  const uint32_t *dkey = reinterpret_cast<const uint32_t *>(ws + L.depth_key);
  uint32_t *dk[2] = {reinterpret_cast<uint32_t *>(ws + L.dsort_key[0]), reinterpret_cast<uint32_t *>(ws + L.dsort_key[1])};
  uint32_t *dv[2] = {reinterpret_cast<uint32_t *>(ws + L.dsort_val[0]), reinterpret_cast<uint32_t *>(ws + L.dsort_val[1])};
  uint32_t *dstate = reinterpret_cast<uint32_t *>(ws + L.depth_state);
  uint32_t *hist_d = reinterpret_cast<uint32_t *>(ws + L.hist_depth);
  uint32_t *sorted = dv[(L.depth_passes - 1) & 1];
  uint32_t *tstate = reinterpret_cast<uint32_t *>(ws + L.tile_state);
  uint32_t *hist_t = reinterpret_cast<uint32_t *>(ws + L.hist_tile);
  uint2 *ranges = reinterpret_cast<uint2 *>(ws + L.ranges);
  uint32_t *ik[2] = {reinterpret_cast<uint32_t *>(ws + L.inst_key[0]), reinterpret_cast<uint32_t *>(ws + L.inst_key[1])};
  uint32_t *iv[2] = {reinterpret_cast<uint32_t *>(ws + L.inst_val[0]), reinterpret_cast<uint32_t *>(ws + L.inst_val[1])};
  EmitArgs ea;
  ea.sorted_slots = sorted;
  ea.meta = reinterpret_cast<const int4 *>(ws + L.rec_meta);
  ea.geom = reinterpret_cast<const float4 *>(ws + L.rec_geom);
  ea.color = reinterpret_cast<const float4 *>(ws + L.rec_color);
  ea.tau = reinterpret_cast<const float *>(ws + L.rec_tau);
  ea.counters = ctr;
  ea.vis_cap = L.vis_cap;
  ea.inst_cap = L.inst_cap;
  ea.pair_cap = L.pair_cap;
  ea.chunk_cap = L.chunk_cap;
  ea.pair_prefix = reinterpret_cast<uint32_t *>(ws + L.pair_prefix);
  ea.emit_rec = reinterpret_cast<int4 *>(ws + L.emit_rec);
  ea.chunk_first = reinterpret_cast<uint32_t *>(ws + L.chunk_first);
  ea.inst_key = ik[0];
  ea.inst_val = iv[0];
  ea.lb_scan = reinterpret_cast<uint64_t *>(ws + L.lb_emit);
  ea.lb_chunk = reinterpret_cast<uint64_t *>(ws + L.lb_chunk);
  ea.tile_passes = L.tile_passes;
  ea.tile_blocks = L.tile_blocks;
  ea.hist_tile = hist_t;
  ea.tile_state = tstate;
  ea.ranges = ranges;
  ea.total_tiles = L.total_tiles;
  if (L.emit_blocks == 0) {  // no visible slot possible: empty tile lists
    e = cudaMemsetAsync(ranges, 0, (size_t)L.total_tiles * sizeof(uint2), st);
    if (e != cudaSuccess) return e;
  } else {
    if (L.depth_blocks > 0) {
      const int hb = std::min(L.depth_blocks, L.sort_grid);
      const int pb = std::min(L.depth_blocks, L.sort_grid);
      constexpr size_t smem = radix_smem_bytes<kDepthSortItems, 1>();
      e = launch_pdl(radix_hist_kernel<kDepthSortItems>, (unsigned)hb, kSortThreads, st, dkey,
                     (const uint32_t *)(ctr + kCtrVisible), (int64_t)L.vis_cap, (int32_t)L.depth_passes, hist_d,
                     dstate, (int32_t)L.depth_blocks, (uint2 *)nullptr, (int64_t)0);
      if (e != cudaSuccess) return e;
      for (int p = 0; p < L.depth_passes; ++p) {
        const int out = p & 1, in = out ^ 1;
        uint32_t *state = dstate + (size_t)p * L.depth_blocks * kRadixBins;
        const uint32_t *kin = p == 0 ? dkey : dk[in];
        const uint32_t *vin = p == 0 ? nullptr : dv[in];
        e = launch_pdl_smem(p == 0 ? radix_pass_kernel<true, kDepthSortItems, 1>
                                   : radix_pass_kernel<false, kDepthSortItems, 1>,
                            (unsigned)pb, kSortThreads, smem, st, kin, vin, dk[out], dv[out],
                       (const uint32_t *)(ctr + kCtrVisible), (int64_t)L.vis_cap, (int32_t)(kRadixBits * p),
                       (const uint32_t *)(hist_d + p * kRadixBins), state, ctr + kCtrTicketDepth + p, status,
                       (uint2 *)nullptr, (int64_t)0);
        if (e != cudaSuccess) return e;
      }
    }
    // 2. Instances in depth order.
    e = launch_pdl(pair_scan_kernel<MAXV>, (unsigned)L.emit_blocks, kEmitBlock, st, ea, rv);
    if (e != cudaSuccess) return e;
    e = launch_pdl(emit_kernel<MAXV>, (unsigned)L.emit_grid, kEmitBlock, st, ea, rv);
    if (e != cudaSuccess) return e;
  }
  // 3. Stable sort of the instances by global tile id (digit histograms
  // taken by the emission); the last pass also records the tile ranges.
  // Very large instance lists take three sub-tiles per ticket (at most 3
  // blocks of 73 KB per SM), the others one.
  const bool wide = L.tile_sort_sub == 3;
  const int tickets = (L.tile_blocks + L.tile_sort_sub - 1) / L.tile_sort_sub;
  const int pbt = std::min(tickets, wide ? L.tile_sort_grid : L.sort_grid);
  constexpr size_t smem1 = radix_smem_bytes<kInstSortItems, 1>(), smem3 = radix_smem_bytes<kInstSortItems, 3>();
  if (wide) {
    e = allow_dynamic_smem(radix_pass_kernel<false, kInstSortItems, 3>, smem3);
    if (e != cudaSuccess) return e;
  }
  for (int p = 0; p < L.tile_passes; ++p) {
    const int in = p & 1, out = in ^ 1;
    const bool last = p == L.tile_passes - 1;
    uint32_t *state = tstate + (size_t)p * L.tile_blocks * kRadixBins;
    e = launch_pdl_smem(wide ? radix_pass_kernel<false, kInstSortItems, 3> : radix_pass_kernel<false, kInstSortItems, 1>,
                        (unsigned)pbt, kSortThreads, wide ? smem3 : smem1, st, (const uint32_t *)ik[in],
                        (const uint32_t *)iv[in], ik[out], iv[out], (const uint32_t *)(ctr + kCtrInstances),
                        (int64_t)L.inst_cap, (int32_t)(kRadixBits * p), (const uint32_t *)(hist_t + p * kRadixBins),
                        state, ctr + kCtrTicketTile + p, status, last ? ranges : (uint2 *)nullptr,
                        (int64_t)L.total_tiles);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

int bin_sort_kernel_count(const Layout &L, int32_t nviews) {
  (void)nviews;
  const int tail = L.tile_passes;  // tile-sort passes (the last records the ranges)
  if (L.emit_blocks == 0) return tail;
  // depth histogram and passes, pair scan, emission
  return (L.depth_blocks > 0 ? 1 + L.depth_passes : 0) + 2 + tail;
}

cudaError_t launch_bin_sort(const Layout &L, const fgs4d_view *views, int32_t nviews, unsigned char *ws,
                            cudaStream_t stream) {
  if (nviews == 1) return bin_sort_typed<1>(L, views, nviews, ws, stream);
  return bin_sort_typed<FGS4D_MAX_VIEWS>(L, views, nviews, ws, stream);
}

}  // namespace fgs4d

// ---------------------------------------------------------------------------
// Self-test of the failure detection: the two kinds of bounded inter-block
// wait run against a predecessor that never posts.  Warp 0 is block 1 of a
// warp-wide look-back chain (the compactions of preprocess, pair scan and
// emission); the other warps are radix tile 1 of a digit look-back (the sort
// passes).  Both give up after kSpinLimit polls, set the timeout bit and
// return.
namespace fgs4d {
namespace {

constexpr size_t kSelftestLb = 0, kSelftestDigits = 256, kSelftestStatus = 256 + 2 * kRadixBins * 4;
static_assert(kSelftestStatus + 4 <= FGS4D_WAIT_SELFTEST_BYTES, "self-test scratch layout");

__global__ void __launch_bounds__(kRadixBins) wait_selftest_kernel(unsigned char *scratch) {
  uint64_t *lb = reinterpret_cast<uint64_t *>(scratch + kSelftestLb);
  uint32_t *digits = reinterpret_cast<uint32_t *>(scratch + kSelftestDigits);
  uint32_t *status = reinterpret_cast<uint32_t *>(scratch + kSelftestStatus);
  if (threadIdx.x < 32) (void)lookback_u64_warp(lb, 1, 5ull, status);
  else (void)radix_lookback(digits, 1, (int)threadIdx.x, 1u, status);
}

}  // namespace
}  // namespace fgs4d

extern "C" int fgs4d_wait_selftest(void *scratch, size_t scratch_bytes, void *stream) {
  using namespace fgs4d;
  if (!scratch || scratch_bytes < FGS4D_WAIT_SELFTEST_BYTES || (reinterpret_cast<uintptr_t>(scratch) & 15u))
    return FGS4D_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(scratch);
  if (cudaMemsetAsync(ws, 0, FGS4D_WAIT_SELFTEST_BYTES, st) != cudaSuccess) return FGS4D_ERR_CUDA;
  wait_selftest_kernel<<<1, kRadixBins, 0, st>>>(ws);
  if (cudaGetLastError() != cudaSuccess) return FGS4D_ERR_CUDA;
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, ws + kSelftestStatus, sizeof status, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FGS4D_ERR_CUDA;
  return (status & kStatusTimeout) ? FGS4D_ERR_TIMEOUT : FGS4D_ERR_INTERNAL;
}

// ---------------------------------------------------------------------------
// Depth sort that allocates nothing: fgs4d_sort_depth_static.
//
// Some callers cannot hand the library a workspace: plug-ins whose host
// application owns every device allocation, and render loops that must not
// call cudaMalloc between frames because it can synchronise the device or
// fail under a fixed memory budget.  For them this entry point runs the same
// radix passes as the depth sort inside fgs4d_bin_sort, with its scratch
// (ping-pong buffers, histograms, look-back rows, tickets) in one file-scope
// device array of fixed size.  The array exists once per GPU that loads the
// library and lives until the process exits.
namespace fgs4d {

namespace {

constexpr int kStaticSortBlocks = FGS4D_STATIC_SORT_MAX / kSortTile;
constexpr int kMaxStaticDevices = 64;

struct StaticSortScratch {
  uint32_t keys[2][FGS4D_STATIC_SORT_MAX];
  uint32_t vals[2][FGS4D_STATIC_SORT_MAX];
  uint32_t state[kMaxPasses][kStaticSortBlocks][kRadixBins];
  uint32_t hist[kMaxPasses][kRadixBins];
  uint32_t ctl[64];  // [0] key count, [1] status bits, [8 + p] ticket of pass p
};

static __device__ __align__(256) StaticSortScratch g_static_sort;

// Device address of g_static_sort on each device, looked up once per device
// (with that device current) at the first call made on it.
StaticSortScratch *g_static_addr[kMaxStaticDevices] = {};

// Every call starts from zeroed histograms and tickets: the previous call's
// contents stay in the array.
__global__ void static_sort_init_kernel(StaticSortScratch *s, uint32_t n) {
  for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) (&s->hist[0][0])[i] = 0u;
  if (threadIdx.x < 64) s->ctl[threadIdx.x] = threadIdx.x == 0 ? n : 0u;
}

int static_scratch(StaticSortScratch **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FGS4D_ERR_CUDA;
  if (dev < 0 || dev >= kMaxStaticDevices) return FGS4D_ERR_UNSUPPORTED;
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_sort) != cudaSuccess || p == nullptr) return FGS4D_ERR_CUDA;
    g_static_addr[dev] = static_cast<StaticSortScratch *>(p);
  }
  *out = g_static_addr[dev];
  return FGS4D_OK;
}

}  // namespace

}  // namespace fgs4d

extern "C" int fgs4d_sort_depth_static(const uint32_t *depth_keys, int64_t n, uint32_t *sorted_slots,
                                       void *stream) {
  using namespace fgs4d;
  if (n < 0 || n > FGS4D_STATIC_SORT_MAX) return FGS4D_ERR_ARG;
  if (n == 0) return FGS4D_OK;
  if (!depth_keys || !sorted_slots) return FGS4D_ERR_ARG;
  StaticSortScratch *s = nullptr;
  const int rc = static_scratch(&s);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((n + kSortTile - 1) / kSortTile);
  constexpr size_t smem = radix_smem_bytes<kSortItems, 1>();
  static_sort_init_kernel<<<1, 256, 0, st>>>(s, (uint32_t)n);
  radix_hist_kernel<kSortItems><<<blocks, kSortThreads, 0, st>>>(depth_keys, &s->ctl[0], FGS4D_STATIC_SORT_MAX,
                                                          kMaxPasses, &s->hist[0][0], &s->state[0][0][0],
                                                          kStaticSortBlocks, nullptr, 0);
  // The passes stage keys with 16-byte copies: keys that do not start on a
  // 16-byte boundary are first copied into the buffer pass 0 does not write.
  const uint32_t *keys0 = depth_keys;
  if (reinterpret_cast<uintptr_t>(depth_keys) & 15u) {
    if (cudaMemcpyAsync(s->keys[1], depth_keys, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return FGS4D_ERR_CUDA;
    keys0 = s->keys[1];
  }
  for (int p = 0; p < kMaxPasses; ++p) {
    const int out = p & 1, in = out ^ 1;
    const uint32_t *kin = p == 0 ? keys0 : s->keys[in];
    uint32_t *vout = p == kMaxPasses - 1 ? sorted_slots : s->vals[out];
    if (p == 0)
      radix_pass_kernel<true, kSortItems, 1><<<blocks, kSortThreads, smem, st>>>(kin, nullptr, s->keys[out], vout, &s->ctl[0],
                                                               FGS4D_STATIC_SORT_MAX, kRadixBits * p, s->hist[p],
                                                               &s->state[p][0][0], &s->ctl[8 + p], &s->ctl[1], nullptr, 0);
    else
      radix_pass_kernel<false, kSortItems, 1><<<blocks, kSortThreads, smem, st>>>(kin, s->vals[in], s->keys[out], vout, &s->ctl[0],
                                                                FGS4D_STATIC_SORT_MAX, kRadixBits * p, s->hist[p],
                                                                &s->state[p][0][0], &s->ctl[8 + p], &s->ctl[1], nullptr, 0);
  }
  return cudaGetLastError() == cudaSuccess ? FGS4D_OK : FGS4D_ERR_CUDA;
}

extern "C" int fgs4d_sort_depth_static_status(void *stream) {
  using namespace fgs4d;
  StaticSortScratch *s = nullptr;
  const int rc = static_scratch(&s);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The status bits of the last call: the radix passes OR a timed-out
  // look-back or an out-of-range position into ctl[1]; the next call's init
  // kernel clears the word, so it is read here, after the stream drains.
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, &s->ctl[1], sizeof status, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FGS4D_ERR_CUDA;
  if (status & kStatusTimeout) return FGS4D_ERR_TIMEOUT;
  if (status & kStatusInternal) return FGS4D_ERR_INTERNAL;
  return FGS4D_OK;
}
