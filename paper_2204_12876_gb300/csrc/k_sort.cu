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
#include "sort_pass.cuh"

namespace em {

template <bool kExt>
__global__ void __launch_bounds__(kPointThreads) k_count(const BatchDev* __restrict__ bp) {
  __shared__ PointSmem S;
  count_pass<kExt>(*bp, own_grid(), S);
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
  int hint = -1;
  for (int64_t wbase = beg + warp * 32; wbase < end; wbase += kPointThreads) {
    const int c0 = find_cloud(b.clouds, b.n_clouds, wbase, hint);
    hint = c0;
    const CloudDev& cl0 = b.clouds[c0];
    if (wbase + 32 <= cl0.begin + cl0.n && b.maps[cl0.map].drift_flat <= 0.f) continue;  // a whole warp without drift
    float px, py, pz;
    const int ci = load_warp_points(b, wbase, end, stage[warp], px, py, pz, hint);
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

__global__ void __launch_bounds__(kAllocThreads) k_alloc(const BatchDev* __restrict__ bp) {
  __shared__ AllocSmem S;
  alloc_pass<kAllocThreads>(*bp, S);
}

template <bool kExt>
__global__ void __launch_bounds__(kPointThreads, 6) k_scatter(const BatchDev* __restrict__ bp) {
  __shared__ PointSmem S;
  scatter_pass<kExt>(*bp, own_grid(), S);
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

const void* alloc_kernel() { return reinterpret_cast<const void*>(&k_alloc); }

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
