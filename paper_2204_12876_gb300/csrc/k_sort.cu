// k_sort.cu -- grouping of points by tile of the cell space: a counting sort
// keyed by the tile of kTile = 1024 physical cells the point falls into.
//
//   k_count    per point: transform + bin, per-tile counts (one atomic per tile
//              and warp: the lanes whose points share a tile add together);
//              then per cell: the ray-march threshold h - sqrt(var_eff) of the
//              pre-update map, stored in logical order (one 4-byte gather per
//              ray sample later, with no ring-buffer wrap)
//   k_alloc    one block: every tile's range [base, base + count) of the record
//              arrays by a running scan in tile order; the fusion's work lists
//   k_scatter  per point: transform + bin again, claim a slot in the tile's
//              range, write the record (z, sigma_p^2, cell within the tile)
//
// The order of records inside a tile's range depends on atomic arrival order.
// The fusion kernel sums the records of a cell exactly in integer fixed point,
// so the order does not change a result.
#include "em_point.cuh"

namespace em {

constexpr int kPointThreads = 256;
constexpr int kCellThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// Block-contiguous partition of the point space into chunks of whole warps.
__device__ __forceinline__ void block_range(int64_t n, int64_t& beg, int64_t& end) {
  int64_t per = (n + gridDim.x - 1) / gridDim.x;
  per = (per + 31) & ~int64_t(31);
  beg = (int64_t)blockIdx.x * per;
  end = beg + per < n ? beg + per : n;
}

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
__global__ void __launch_bounds__(kPointThreads) k_count(const BatchDev* __restrict__ bp) {
  __shared__ float4 stage[kPointThreads / 32][24];
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per-update counters start at zero (the previous update is complete)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.ctl->rec_total = 0;
    b.ctl->n_split = 0;
    b.ctl->n_pieces = 0;
    b.ctl->n_heavy = 0;
    b.ctl->n_light = 0;
    b.ctl->fuse_next = 0;
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
  block_range(b.n_points, beg, end);
  MapCounters mc;
  const int idx[2] = {kStValid, kStInMap};
  for (int64_t wbase = beg + warp * 32; wbase < end; wbase += kPointThreads) {
    float px, py, pz;
    const int ci = load_warp_points(b, wbase, end, stage[warp], px, py, pz);
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
  flush_counters(b, mc, idx, 2);
  // ray thresholds of the pre-update map over the cell space (Eq. 3)
  for_each_tile(b, [&](const MapDev& m, int, int32_t p0, int32_t count) {
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
}

// Drift-compensation sums (Section II-D): per point of a map with drift
// compensation, its error against a flat cell holding an estimate (previous
// normal n_z >= drift_flatness; a NaN normal is not flat), summed exactly per map.
template <bool kExt>
__global__ void __launch_bounds__(kPointThreads) k_drift_sum(const BatchDev* __restrict__ bp) {
  __shared__ float4 stage[kPointThreads / 32][24];
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t beg, end;
  block_range(b.n_points, beg, end);
  int dmap = -1;
  long long dh = 0;
  unsigned long long dl = 0, dn = 0;
  for (int64_t wbase = beg + warp * 32; wbase < end; wbase += kPointThreads) {
    const int c0 = find_cloud(b.clouds, b.n_clouds, wbase);
    const CloudDev& cl0 = b.clouds[c0];
    if (wbase + 32 <= cl0.begin + cl0.n && b.maps[cl0.map].drift_flat <= 0.f) continue;  // a whole warp without drift
    float px, py, pz;
    const int ci = load_warp_points(b, wbase, end, stage[warp], px, py, pz);
    const int64_t g = wbase + lane;
    const CloudDev& c = b.clouds[ci];
    const MapDev& m = b.maps[c.map];
    const PointGeom pg = point_geom<kExt>(m, c, px, py, pz);
    if (g < end && m.drift_flat > 0.f && pg.in_range && in_map(m, pg.ix, pg.iy)) {
      const int32_t key = phys_index(m, pg.ix, pg.iy);
      // the three loads are independent: all in flight at once
      const float var = m.var[key], nz = m.nz[key], hc = m.h[key];
      if (isfinite(var) && nz >= m.drift_flat) {
        if (c.map != dmap) {
          if (dmap >= 0) drift_add(b.maps[dmap], dh, dl, dn);
          dmap = c.map;
          dh = 0;
          dl = dn = 0;
        }
        const Fix e = to_fix(__fsub_rn(pg.z, hc));
        dh += e.h;
        dl += e.l;
        ++dn;
      }
    }
  }
  // One atomic triple per block when the block's sums all belong to one map (the
  // usual case): every block adding to the same three words of that map would
  // otherwise queue at one L2 slice.  Else per warp or per lane.
  __shared__ int s_map;
  __shared__ long long s_h[kPointThreads / 32];
  __shared__ unsigned long long s_l[kPointThreads / 32], s_n[kPointThreads / 32];
  if (threadIdx.x == 0) s_map = -1;
  __syncthreads();
  if (dn) atomicMax(&s_map, dmap);
  __syncthreads();
  const int bm = s_map;
  if (__syncthreads_and(dn == 0 || dmap == bm)) {
    for (int o = 16; o > 0; o >>= 1) {
      dh += __shfl_xor_sync(kFull, dh, o);
      dl += __shfl_xor_sync(kFull, dl, o);
      dn += __shfl_xor_sync(kFull, dn, o);
    }
    if (lane == 0) {
      s_h[warp] = dh;
      s_l[warp] = dl;
      s_n[warp] = dn;
    }
    __syncthreads();
    if (threadIdx.x == 0 && bm >= 0) {
      long long th = 0;
      unsigned long long tl = 0, tn = 0;
      for (int w = 0; w < kPointThreads / 32; ++w) {
        th += s_h[w];
        tl += s_l[w];
        tn += s_n[w];
      }
      if (tn) drift_add(b.maps[bm], th, tl, tn);
    }
    return;
  }
  const int d0 = __shfl_sync(kFull, dmap, 0);
  if (__all_sync(kFull, dmap == d0 || dn == 0)) {
    for (int o = 16; o > 0; o >>= 1) {
      dh += __shfl_xor_sync(kFull, dh, o);
      dl += __shfl_xor_sync(kFull, dl, o);
      dn += __shfl_xor_sync(kFull, dn, o);
    }
    if (lane == 0 && d0 >= 0 && dn) drift_add(b.maps[d0], dh, dl, dn);
  } else if (dmap >= 0 && dn) {
    drift_add(b.maps[dmap], dh, dl, dn);
  }
}

// Height drift compensation (Section II-D): every estimate moves by the mean
// error of this update's points in flat cells (k_count summed them exactly, so
// every thread derives the same mean); then the ray thresholds of the moved map.
__global__ void __launch_bounds__(kPointThreads) k_drift(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  for_each_tile(b, [&](const MapDev& m, int, int32_t p0, int32_t count) {
    if (m.drift_flat <= 0.f) return;
    const int slot = m.t_now & 1;
    const unsigned long long n = m.ctl->drift_n[slot];
    const float mean =
        n ? __fdiv_rn(fixed_to_float(fix128(m.ctl->drift_h[slot], m.ctl->drift_l[slot])), (float)n) : 0.f;
    if (p0 == 0 && threadIdx.x == 0) {  // once per map: its first tile
      atomicAdd(&m.ctl->stats[kStDriftPoints], n);
      m.ctl->drift_last = mean;
    }
    for (int32_t i = threadIdx.x; i < count; i += kPointThreads) {
      const int32_t p = p0 + i;
      const float var = m.var[p];
      float h = m.h[p];
      if (isfinite(var) && n) {
        h = __fadd_rn(h, mean);
        m.h[p] = h;
      }
      if (m.ray_step > 0.f) {
        int32_t lx, ly;
        logical_of(m, p, lx, ly);
        m.thr[ly * m.W + lx] = ray_threshold(m, p, h, var);
      }
    }
  });
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
static_assert(kMaxSplit <= kAllocThreads, "one thread per split tile in the piece scan");

__global__ void __launch_bounds__(kAllocThreads) k_alloc(const BatchDev* __restrict__ bp) {
  __shared__ unsigned long long warp_tot[33];
  __shared__ int s_heavy, s_split;
  __shared__ int32_t s_tile[kMaxSplit], s_cnt[kMaxSplit], s_r0[kMaxSplit], s_map[kMaxSplit];
  const BatchDev& b = *bp;
  const int64_t n_tiles = b.n_cells / kTile;
  const int slots = min(b.split_slots, kMaxSplit);
  const int thresh = b.heavy_thresh;
  int base = 0, n_light = 0;
  if (threadIdx.x == 0) {
    s_heavy = 0;
    s_split = 0;
  }
  __syncthreads();
  for (int64_t t0 = 0; t0 < n_tiles; t0 += kAllocThreads) {
    const int64_t t = t0 + threadIdx.x;
    const int c = t < n_tiles ? b.tile_cnt[t] : 0;
    const int mp = c > 0 ? b.tile_map[t] : 0;
    const bool light = c > 0 && c <= thresh;
    unsigned long long tot;
    const unsigned long long off =
        block_exclusive_scan((unsigned long long)(uint32_t)c | ((unsigned long long)light << 32), warp_tot, tot);
    if (t < n_tiles) {
      const int32_t r0 = base + (int32_t)(uint32_t)off;
      b.tile_base[t] = r0;
      b.tile_cnt[t] = 0;
      b.tile_cur[t] = 0;
      const FuseItem whole{(int32_t)t, mp, r0, r0 + c, r0, r0 + c, -1, 1};
      if (light) {
        b.light[n_light + (int)(off >> 32)] = whole;
      } else if (c > thresh) {
        const int sl = slots > 0 ? atomicAdd(&s_split, 1) : slots;
        if (sl < slots) {
          s_tile[sl] = (int32_t)t;
          s_cnt[sl] = c;
          s_r0[sl] = r0;
          s_map[sl] = mp;
        } else {
          b.heavy[atomicAdd(&s_heavy, 1)] = whole;
        }
      }
    }
    base += (int32_t)(uint32_t)tot;
    n_light += (int)(tot >> 32);
  }
  __syncthreads();
  // the piece list: split tile i has np = ceil(count / heavy_thresh) pieces of
  // ceil(count / np) records (the last ones may be shorter)
  const int n_split = min(s_split, slots);
  const int i = threadIdx.x;
  const int np = i < n_split ? (s_cnt[i] + thresh - 1) / thresh : 0;
  unsigned long long n_pieces;
  const int first = (int)block_exclusive_scan((unsigned long long)np, warp_tot, n_pieces);
  const bool fits = n_pieces <= (unsigned long long)b.max_pieces;  // holds by the workspace's size
  if (fits && np > 0) {
    const int32_t c = s_cnt[i], r0 = s_r0[i];
    const int32_t len = (c + np - 1) / np;
    for (int k = 0; k < np; ++k) {
      const int32_t q0 = r0 + (int32_t)min((int64_t)c, (int64_t)k * len);
      const int32_t q1 = r0 + (int32_t)min((int64_t)c, (int64_t)(k + 1) * len);
      b.pieces[first + k] = FuseItem{s_tile[i], s_map[i], r0, r0 + c, q0, q1, i, np};
    }
  }
  if (threadIdx.x == 0) {
    b.tile_base[n_tiles] = base;
    b.ctl->rec_total = base;
    b.ctl->n_split = fits ? n_split : 0;
    b.ctl->n_pieces = fits ? (int32_t)n_pieces : 0;
    b.ctl->n_heavy = s_heavy;
    b.ctl->n_light = n_light;
    if (!fits) atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
  }
}

// Warps take the point space in waves (warp w: points (w + k W) 32 .. + 31, W
// the warps of the grid).  Each point claims a slot in its tile's range (one
// claim per tile and warp) and writes its record there; a tile's range fills
// in order, so its open sectors stay in L2 until they are full.
template <bool kExt>
__global__ void __launch_bounds__(kPointThreads, 6) k_scatter(const BatchDev* __restrict__ bp) {
  __shared__ float4 stage[kPointThreads / 32][24];
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  const int64_t end = b.n_points;
  for (int64_t wbase = ((int64_t)blockIdx.x * (kPointThreads / 32) + warp) * 32; wbase < end;
       wbase += (int64_t)gridDim.x * kPointThreads) {
    float px, py, pz;
    const int ci = load_warp_points(b, wbase, end, stage[warp], px, py, pz);
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
}

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = sms;
  }
  return cached[dev];
}

static int point_grid(int64_t n) {
  const int sms = sm_count();
  int64_t want = (n + kPointThreads - 1) / kPointThreads;  // one 32-point chunk per warp
  int64_t cap = (int64_t)sms * 16;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

static int tile_grid(int64_t n_cells) {
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * 8;
  const int64_t g = tiles < cap ? tiles : cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_bin(const BatchDev* b, int64_t n_points, int64_t n_cells, bool ext, cudaStream_t s) {
  const int64_t tiles = n_cells / kTile;
  int grid = point_grid(n_points);
  if (grid < tiles && tiles < (int64_t)sm_count() * 8) grid = (int)tiles;  // enough blocks for the cell pass
  if (ext) k_count<true><<<grid, kPointThreads, 0, s>>>(b);
  else k_count<false><<<grid, kPointThreads, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_drift(const BatchDev* b, int64_t n_points, int64_t n_cells, bool ext, cudaStream_t s) {
  if (n_points > 0 && ext) k_drift_sum<true><<<point_grid(n_points), kPointThreads, 0, s>>>(b);
  if (n_points > 0 && !ext) k_drift_sum<false><<<point_grid(n_points), kPointThreads, 0, s>>>(b);
  k_drift<<<tile_grid(n_cells), kPointThreads, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_alloc(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  (void)n_cells;
  k_alloc<<<1, kAllocThreads, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const BatchDev* b, int64_t n_points, bool ext, cudaStream_t s) {
  if (n_points <= 0) return cudaSuccess;
  if (ext) k_scatter<true><<<point_grid(n_points), kPointThreads, 0, s>>>(b);
  else k_scatter<false><<<point_grid(n_points), kPointThreads, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace em
