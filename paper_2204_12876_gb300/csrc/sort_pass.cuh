// sort_pass.cuh -- the device passes of the counting sort by tile (k_sort.cu):
// the count pass (transform + bin + per-tile counts, then the ray thresholds of
// the pre-update map), the single-block allocation of the tiles' record ranges
// and the fusion's work lists, and the scatter pass.  Each pass runs on the
// blocks of a Grid: its own kernel's, or the persistent kernel's (k_persist.cu).
#pragma once

#include "em_point.cuh"

namespace em {

constexpr int kPointThreads = 256;
constexpr int kCellThreads = 256;

// Block-contiguous partition of the point space into chunks of whole warps.
__device__ __forceinline__ void block_range(int64_t n, Grid gr, int64_t& beg, int64_t& end) {
  int64_t per = (n + gr.nb - 1) / gr.nb;
  per = (per + 31) & ~int64_t(31);
  beg = (int64_t)gr.bid * per;
  end = beg + per < n ? beg + per : n;
}
__device__ __forceinline__ void block_range(int64_t n, int64_t& beg, int64_t& end) {
  block_range(n, own_grid(), beg, end);
}

// Shared memory of the point passes: a staging row per warp, and the
// counter flush.
struct PointSmem {
  float4 stage[kPointThreads / 32][24];
  FlushSmem flush;
};

// Add a lane's or warp's drift-compensation sums to the map's slot of this update.
__device__ __forceinline__ void drift_add(const MapDev& m, long long h, unsigned long long l,
                                          unsigned long long n) {
  const int slot = m.t_now & 1;
  atomicAdd(reinterpret_cast<unsigned long long*>(&m.ctl->drift_h[slot]), (unsigned long long)h);
  atomicAdd(&m.ctl->drift_l[slot], l);
  atomicAdd(&m.ctl->drift_n[slot], n);
}

// Ray threshold of physical cell p for the march (Eq. 3): h - sqrt(var_eff); for
// an empty cell -inf (never penetrated), or its upper bound with that layer.
__device__ __forceinline__ float ray_threshold(const MapDev& m, int32_t p, float h, float var) {
  if (!isfinite(var)) return m.upper ? m.upper[p] : __int_as_float(0xff800000);
  return __fsub_rn(h, __fsqrt_rn(var_eff(m, var, m.t_last[p])));
}

template <bool kExt>
__device__ __forceinline__ void count_pass(const BatchDev& b, Grid gr, PointSmem& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per-update counters start at zero (the previous update is complete)
  if (gr.bid == 0 && threadIdx.x == 0) {
    b.ctl->rec_total = 0;
    b.ctl->n_split = 0;
    b.ctl->n_pieces = 0;
    b.ctl->n_heavy = 0;
    b.ctl->n_light = 0;
    b.ctl->fuse_next = 0;
    b.ctl->ray_next = 0;
    for (int mi = 0; mi < b.n_maps; ++mi) {
      const MapDev& m = b.maps[mi];
      atomicAdd(&m.ctl->stats[kStUpdates], 1ull);
      if (m.drift_flat > 0.f) {  // clear the next update's drift slot (this one's was cleared before)
        const int nxt = (m.t_now + 1) & 1;
        m.ctl->drift_h[nxt] = 0;
        m.ctl->drift_l[nxt] = 0;
        m.ctl->drift_n[nxt] = 0;
      }
    }
  }
  int64_t beg, end;
  block_range(b.n_points, gr, beg, end);
  MapCounters mc;
  const int idx[2] = {kStValid, kStInMap};
  int hint = -1;
  for (int64_t wbase = beg + warp * 32; wbase < end; wbase += kPointThreads) {
    float px, py, pz;
    const int ci = load_warp_points(b, wbase, end, S.stage[warp], px, py, pz, hint);
    const int64_t g = wbase + lane;
    const bool live = g < end;
    const CloudDev& c = b.clouds[ci];
    const MapDev& m = b.maps[c.map];
    const PointGeom pg = point_geom<kExt>(m, c, px, py, pz);
    const bool inm = live && pg.in_range && in_map(m, pg.ix, pg.iy);
    const int32_t key = inm ? phys_index(m, pg.ix, pg.iy) : -1;
    if (live) {
      unsigned long long inc[2] = {pg.in_range ? 1ull : 0ull, inm ? 1ull : 0ull};
      add_counter(b, mc, c.map, idx, 2, inc);
      if (b.tr_status) {
        b.tr_ix[g] = pg.finite ? pg.ix : INT32_MIN;
        b.tr_iy[g] = pg.finite ? pg.iy : INT32_MIN;
        b.tr_status[g] = !pg.finite ? kPtNonFinite : !pg.in_range ? kPtRange : !inm ? kPtOutside : kPtFused;
      }
    }
    // one count per tile and warp: the lanes whose points share a tile add
    // together; the tile's map for the fusion's work list (every writer agrees)
    const uint32_t tile = inm ? (uint32_t)((m.cell_begin + key) / kTile) : 0xffffffffu;
    const unsigned grp = __match_any_sync(kFull, tile);
    if (inm && lane == __ffs(grp) - 1) {
      atomicAdd(&b.tile_cnt[tile], __popc(grp));
      b.tile_map[tile] = c.map;
    }
  }
  flush_counters(b, mc, idx, 2, S.flush);
  // ray thresholds of the pre-update map over the cell space (Eq. 3)
  for_each_tile(b, gr, [&](const MapDev& m, int, int32_t p0, int32_t count) {
    if (m.ray_step <= 0.f || m.drift_flat > 0.f) return;  // with drift: k_drift, after the shift
    for (int32_t i = threadIdx.x; i < count; i += kPointThreads) {
      const int32_t p = p0 + i;
      // an empty cell is never penetrated (-inf); with the upper-bound layer it holds
      // the cell's bound instead, so a ray sample below the bound takes the march's
      // candidate path and lowers it (Section II-H)
      const float var = m.var[p];
      float t;
      if (kExt) {
        t = ray_threshold(m, p, isfinite(var) ? m.h[p] : 0.f, var);
      } else {  // no upper-bound layer in this batch: an empty cell is never penetrated
        t = __int_as_float(0xff800000);
        if (isfinite(var)) t = __fsub_rn(m.h[p], __fsqrt_rn(var_eff(m, var, m.t_last[p])));
      }
      int32_t lx, ly;
      logical_of(m, p, lx, ly);
      m.thr[ly * m.W + lx] = t;  // logical layout: the ray march indexes it without the ring wrap
    }
  });
  __syncthreads();  // the shared memory is free again
}

__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* warp_tot,
                                                                   unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
    unsigned long long wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - w;
    if (lane == 31) warp_tot[32] = wi;
  }
  __syncthreads();
  const unsigned long long res = warp_tot[warp] + incl - v;
  total = warp_tot[32];
  __syncthreads();
  return res;
}

// One block: the record ranges of all tiles, in tile order, by a running block
// scan of their counts (the counts and the claim cursors go back to zero for
// the next update), and the fusion's work lists:
//   pieces  tiles with more than heavy_thresh records get an accumulator slot
//           while slots last and are cut into ceil(count / heavy_thresh)
//           near-equal pieces;
//   heavy   the rest of those tiles, fused whole (before the light tiles);
//   light   every other non-empty tile, in tile order.
// The same scan counts the light tiles (count in the low word, one in the high
// word: a chunk's records stay below 2^31, so the words do not mix).
constexpr int kAllocThreads = 1024;

struct AllocSmem {
  unsigned long long warp_tot[33];
  int heavy, split;
  int32_t tile[kMaxSplit], cnt[kMaxSplit], r0[kMaxSplit], map[kMaxSplit];
};

// One block of NT threads (k_alloc, or one block of the persistent kernel).
template <int NT>
__device__ __forceinline__ void alloc_pass(const BatchDev& b, AllocSmem& S) {
  const int64_t n_tiles = b.n_cells / kTile;
  const int slots = min(b.split_slots, kMaxSplit);
  const int thresh = b.heavy_thresh;
  int base = 0, n_light = 0;
  if (threadIdx.x == 0) {
    S.heavy = 0;
    S.split = 0;
  }
  __syncthreads();
  for (int64_t t0 = 0; t0 < n_tiles; t0 += NT) {
    const int64_t t = t0 + threadIdx.x;
    const int c = t < n_tiles ? b.tile_cnt[t] : 0;
    const int mp = c > 0 ? b.tile_map[t] : 0;
    const bool light = c > 0 && c <= thresh;
    unsigned long long tot;
    const unsigned long long off =
        block_exclusive_scan((unsigned long long)(uint32_t)c | ((unsigned long long)light << 32), S.warp_tot, tot);
    if (t < n_tiles) {
      const int32_t r0 = base + (int32_t)(uint32_t)off;
      b.tile_base[t] = r0;
      b.tile_cnt[t] = 0;
      b.tile_cur[t] = 0;
      const FuseItem whole{(int32_t)t, mp, r0, r0 + c, r0, r0 + c, -1, 1};
      if (light) {
        b.light[n_light + (int)(off >> 32)] = whole;
      } else if (c > thresh) {
        const int sl = slots > 0 ? atomicAdd(&S.split, 1) : slots;
        if (sl < slots) {
          S.tile[sl] = (int32_t)t;
          S.cnt[sl] = c;
          S.r0[sl] = r0;
          S.map[sl] = mp;
        } else {
          b.heavy[atomicAdd(&S.heavy, 1)] = whole;
        }
      }
    }
    base += (int32_t)(uint32_t)tot;
    n_light += (int)(tot >> 32);
  }
  __syncthreads();
  // the piece list: split tile i has np = ceil(count / heavy_thresh) pieces of
  // ceil(count / np) records (the last ones may be shorter)
  const int n_split = min(S.split, slots);
  unsigned long long n_pieces = 0;
  bool fits = true;
  for (int i0 = 0; i0 < n_split; i0 += NT) {
    const int i = i0 + threadIdx.x;
    const int np = i < n_split ? (S.cnt[i] + thresh - 1) / thresh : 0;
    unsigned long long tot;
    const int first = (int)(n_pieces + block_exclusive_scan((unsigned long long)np, S.warp_tot, tot));
    n_pieces += tot;
    fits = n_pieces <= (unsigned long long)b.max_pieces;  // holds by the workspace's size
    if (fits && np > 0) {
      const int32_t c = S.cnt[i], r0 = S.r0[i];
      const int32_t len = (c + np - 1) / np;
      for (int k = 0; k < np; ++k) {
        const int32_t q0 = r0 + (int32_t)min((int64_t)c, (int64_t)k * len);
        const int32_t q1 = r0 + (int32_t)min((int64_t)c, (int64_t)(k + 1) * len);
        b.pieces[first + k] = FuseItem{S.tile[i], S.map[i], r0, r0 + c, q0, q1, i, np};
      }
    }
  }
  if (threadIdx.x == 0) {
    b.tile_base[n_tiles] = base;
    b.ctl->rec_total = base;
    b.ctl->n_split = fits ? n_split : 0;
    b.ctl->n_pieces = fits ? (int32_t)n_pieces : 0;
    b.ctl->n_heavy = S.heavy;
    b.ctl->n_light = n_light;
    if (!fits) atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
  }
  __syncthreads();  // the shared memory is free again
}

// Warps take the point space in waves (warp w: points (w + k W) 32 .. + 31, W
// the warps of the grid).  Each point claims a slot in its tile's range (one
// claim per tile and warp) and writes its record there; a tile's range fills
// in order, so its open sectors stay in L2 until they are full.
template <bool kExt>
__device__ __forceinline__ void scatter_pass(const BatchDev& b, Grid gr, PointSmem& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  const int64_t end = b.n_points;
  for (int64_t wbase = ((int64_t)gr.bid * (kPointThreads / 32) + warp) * 32; wbase < end;
       wbase += (int64_t)gr.nb * kPointThreads) {
    float px, py, pz;
    int hint = -1;  // consecutive waves lie far apart in the point space: no cloud to guess
    const int ci = load_warp_points(b, wbase, end, S.stage[warp], px, py, pz, hint);
    const int64_t g = wbase + lane;
    const bool live = g < end;
    const CloudDev& c = b.clouds[ci];
    const MapDev& m = b.maps[c.map];
    const PointGeom pg = point_geom<kExt>(m, c, px, py, pz);
    const bool inm = live && pg.in_range && in_map(m, pg.ix, pg.iy);
    const int64_t cell = inm ? m.cell_begin + phys_index(m, pg.ix, pg.iy) : -1;
    const uint32_t tile = inm ? (uint32_t)(cell / kTile) : 0xffffffffu;
    const unsigned grp = __match_any_sync(kFull, tile);
    const int leader = __ffs(grp) - 1;
    // the range is read before the claim so both loads are in flight together
    const int32_t lo = inm ? __ldg(b.tile_base + tile) : 0, hi = inm ? __ldg(b.tile_base + tile + 1) : 0;
    int old = 0;
    if (inm && lane == leader) old = atomicAdd(&b.tile_cur[tile], __popc(grp));
    old = __shfl_sync(kFull, old, leader);
    if (inm) {
      const int64_t pos = (int64_t)lo + old + __popc(grp & below);
      // the count pass found the same tile for this point, so pos lies in the
      // tile's range; anything else is recorded instead of written
      if (pos >= hi || pos >= b.n_points) {
        atomicCAS(&m.ctl->err, 0, kErrInternal);
      } else {
        b.rz[pos] = pg.z;
        b.rv[pos] = point_variance(m, pg.d);
        b.rc[pos] = (uint16_t)(cell % kTile);
        if (b.idx_sorted) b.idx_sorted[pos] = (int32_t)g;
      }
    }
  }
  __syncthreads();  // every warp is done with its staging row: the shared memory is free again
}

}  // namespace em
