// k_ray.cu -- visibility cleanup by ray casting (Section II-E of the paper).
//
// k_ray: a group of G lanes per valid point.  The ray from the sensor origin o
// (the pose translation) to the point is sampled at
// s_k = o + (k step / d) (R p_s) for k = 1, 2, ... while k step < d; lane j of
// the group takes k = k_lo + j, k_lo + j + G, ..., so the group keeps G
// independent gathers in flight.  A sample inside the map, outside the point's
// own cell, below the cell's threshold h - sqrt(sigma_m^2) of the pre-update
// map (Eq. 3; the threshold layer is -inf for empty cells) and -- when
// alpha_n > 0 -- with |rhat . n| > alpha_n for the cell's previous normal
// (Eq. 4; a NaN normal counts as (0, 0, 1)) marks the cell in a bitmask
// (atomicOr: idempotent, so the marks do not depend on thread order).  Only
// the k whose samples can lie inside the map's box are visited.  The kernel
// runs before the fusion, so it sees the pre-update map.
//
// k_clear: after the fusion, every marked cell that holds an estimate and was
// last written at least max(1, cleanup_min_age) updates ago is removed; the
// bitmask is reset for the next update.  Tiles start on multiples of kTile
// cells, so a tile owns whole mark words.
#include "em_point.cuh"

namespace em {

constexpr int kRayThreads = 256;

// Narrow [lo, hi] (metres along the ray) to where the track o + (s/d) v stays
// inside [a0, a1); false when it never does.
__device__ __forceinline__ bool slab(float o, float v, float d, float a0, float a1, float& lo, float& hi) {
  if (v == 0.f) return o >= a0 && o < a1;
  const float sa = (a0 - o) * d / v;
  const float sb = (a1 - o) * d / v;
  lo = fmaxf(lo, fminf(sa, sb));
  hi = fminf(hi, fmaxf(sa, sb));
  return true;
}

template <int G>
__global__ void __launch_bounds__(kRayThreads) k_ray(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  const int gl = (threadIdx.x & 31) % G;
  const int64_t group = ((int64_t)blockIdx.x * kRayThreads + threadIdx.x) / G;
  const int64_t n_groups = (int64_t)gridDim.x * kRayThreads / G;
  MapCounters mc;
  const int stat_idx[1] = {kStRaySamples};
  unsigned long long samples = 0;
  for (int64_t g = group; g < b.n_points; g += n_groups) {
    const int ci = find_cloud(b.clouds, b.n_clouds, g);
    const CloudDev& c = b.clouds[ci];
    const MapDev& m = b.maps[c.map];
    if (m.ray_step <= 0.f) continue;
    float px, py, pz;
    load_point(c, g - c.begin, px, py, pz);
    const PointGeom pg = point_geom(m, c, px, py, pz);
    if (!pg.in_range || !(pg.d > 0.f)) continue;
    if (c.map != mc.map) {  // fold this map's samples in, then switch maps
      if (mc.map >= 0) add_counter(b, mc, mc.map, stat_idx, 1, &samples);
      samples = 0;
      add_counter(b, mc, c.map, stat_idx, 1, &samples);
    }
    // clip the sample range to the map box (conservative by 1 mm + 1 step)
    float lo = 0.f, hi = pg.d;
    const float ext_x = __fmul_rn((float)m.W, m.res), ext_y = __fmul_rn((float)m.H, m.res);
    if (!slab(c.t[0], pg.vx, pg.d, m.x0, m.x0 + ext_x, lo, hi)) continue;
    if (!slab(c.t[1], pg.vy, pg.d, m.y0, m.y0 + ext_y, lo, hi)) continue;
    if (lo > hi + 1e-3f) continue;
    const float step = m.ray_step;
    const float kl = floorf((lo - 1e-3f) / step) - 1.f;
    const float kh = ceilf((hi + 1e-3f) / step) + 1.f;
    const int32_t k_lo = kl < 1.f ? 1 : (int32_t)kl;
    const int32_t k_hi = kh > 1.0e9f ? 1000000000 : (int32_t)kh;
    const float cstep = __fdiv_rn(step, pg.d);  // f_k = k * step / d
    const float inv_res = __frcp_rn(m.res);
    const bool guard = m.alpha_n > 0.f;
    for (int32_t k = k_lo + gl; k <= k_hi; k += G) {
      const float len = __fmul_rn((float)k, step);
      if (!(len < pg.d)) break;
      const float f = __fmul_rn((float)k, cstep);
      const float sx = __fmaf_rn(f, pg.vx, c.t[0]);
      const float sy = __fmaf_rn(f, pg.vy, c.t[1]);
      const int32_t cx = clamp_floor(__fmul_rn(__fsub_rn(sx, m.x0), inv_res));
      const int32_t cy = clamp_floor(__fmul_rn(__fsub_rn(sy, m.y0), inv_res));
      if (!in_map(m, cx, cy)) continue;
      ++samples;
      if (cx == pg.ix && cy == pg.iy) continue;
      const int32_t p = phys_index(m, cx, cy);
      const float sz = __fmaf_rn(f, pg.vz, c.t[2]);
      if (!(sz < __ldg(m.thr + p))) continue;
      if (guard) {
        float n0 = m.nx[p], n1 = m.ny[p], n2 = m.nz[p];
        if (!(isfinite(n0) && isfinite(n1) && isfinite(n2))) { n0 = 0.f; n1 = 0.f; n2 = 1.f; }
        const float rx = __fdiv_rn(pg.vx, pg.d), ry = __fdiv_rn(pg.vy, pg.d), rz = __fdiv_rn(pg.vz, pg.d);
        const float dot = fabsf(__fmaf_rn(rx, n0, __fmaf_rn(ry, n1, __fmul_rn(rz, n2))));
        if (!(dot > m.alpha_n)) continue;
      }
      // many rays graze the same surface cells: skip the atomic when the bit is
      // already set (marks are only ever set during this kernel)
      const uint32_t bit = 1u << (p & 31);
      if (!(*(volatile uint32_t*)(m.mark + (p >> 5)) & bit)) atomicOr(&m.mark[p >> 5], bit);
    }
  }
  if (mc.map >= 0) add_counter(b, mc, mc.map, stat_idx, 1, &samples);
  flush_counters(b, mc, stat_idx, 1);
}

constexpr int kClearThreads = 256;

__global__ void __launch_bounds__(kClearThreads) k_clear(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  MapCounters mc;
  const int idx[1] = {kStCleared};
  // a tile of kTile cells is kTile / 32 mark words; one word per thread
  for_each_tile(b, [&](const MapDev& m, int mi, int32_t p0, int32_t count) {
    const int32_t min_age = m.min_age > 1 ? m.min_age : 1;
    const int32_t nword = (count + 31) >> 5;
    unsigned long long cleared = 0;
    for (int32_t wi = threadIdx.x; wi < nword; wi += kClearThreads) {
      const int32_t w = (p0 >> 5) + wi;
      uint32_t bits = m.mark[w];
      if (!bits) continue;
      m.mark[w] = 0u;
      while (bits) {
        const int bit = __ffs(bits) - 1;
        bits &= bits - 1;
        const int32_t p = w * 32 + bit;
        if (p >= p0 + count) break;
        if (!isfinite(m.var[p])) continue;
        if (m.t_now - m.t_last[p] < min_age) continue;
        m.h[p] = __int_as_float(0x7fc00000);
        m.var[p] = __int_as_float(0x7f800000);
        ++cleared;
      }
    }
    add_counter(b, mc, mi, idx, 1, &cleared);
  });
  flush_counters(b, mc, idx, 1);
}

cudaError_t launch_ray(const BatchDev* b, int64_t n_points, int group, cudaStream_t s) {
  if (n_points <= 0) return cudaSuccess;
  const int g = (group == 1 || group == 2 || group == 4 || group == 8 || group == 16 || group == 32) ? group : 4;
  const int64_t want = (n_points * g + kRayThreads - 1) / kRayThreads;
  const int64_t cap = (int64_t)sm_count() * 16;
  const int grid = (int)(want < cap ? want : cap);
  switch (g) {
    case 1: k_ray<1><<<grid, kRayThreads, 0, s>>>(b); break;
    case 2: k_ray<2><<<grid, kRayThreads, 0, s>>>(b); break;
    case 4: k_ray<4><<<grid, kRayThreads, 0, s>>>(b); break;
    case 8: k_ray<8><<<grid, kRayThreads, 0, s>>>(b); break;
    case 32: k_ray<32><<<grid, kRayThreads, 0, s>>>(b); break;
    case 16: k_ray<16><<<grid, kRayThreads, 0, s>>>(b); break;
    default: k_ray<4><<<grid, kRayThreads, 0, s>>>(b); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_clear(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap);
  k_clear<<<grid, kClearThreads, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace em
