// k_ray.cu -- visibility cleanup by ray casting (Section II-E of the paper).
//
// k_ray: one ray per valid point, marched by a group of G lanes.  The ray from
// the sensor origin o (the pose translation) to the point is sampled at
// s_k = o + (k step / d) (R p_s) for k = 1, 2, ... while k step < d (computed
// as a + k b in cell units: one FMA per coordinate); lane j of the group takes
// k = k_lo + j, k_lo + j + G, ..., so the group keeps G independent gathers in
// flight, and each lane loads the thresholds of 4 samples before testing them.  A sample inside the map, outside the point's
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
// inside [a0, a1); false when it never does.  An estimate (the sample range
// gets 1 mm + 1 step of slack and every sample is tested exactly), so a fast
// division does: its 2-ulp error is micrometres at tens of metres.
__device__ __forceinline__ bool slab(float o, float v, float d, float a0, float a1, float& lo, float& hi) {
  if (v == 0.f) return o >= a0 && o < a1;
  const float dv = __fdividef(d, v);
  const float sa = (a0 - o) * dv;
  const float sb = (a1 - o) * dv;
  lo = fmaxf(lo, fminf(sa, sb));
  hi = fminf(hi, fmaxf(sa, sb));
  return true;
}

// Per-ray set-up shared by the lanes that march it.  Sample k lies at
// q = a + k b in cell units (x, y) and at z = az + k bz, i.e. the track
// o + (k step / d) (R p_s) measured from the map corner in cells.
// Samples per ray are capped at 2^24 - 1, so the float sample index is exact.
constexpr int32_t kMaxRayK = (1 << 24) - 1;

struct RaySetup {
  float ax, bx, ay, by, az, bz;
  float vx, vy, vz, d;  // for the Eq. 4 guard
  int32_t ix, iy, k_lo, n, map;
};

// Each warp takes 32 consecutive points: first every lane sets up one ray
// (transform, distance, own cell, the k range inside the map box and before
// the point), then the warp marches them G lanes per ray, 32 / G rays at a
// time, so the set-up cost is paid once per ray.
template <int G, bool kExt>
__global__ void __launch_bounds__(kRayThreads) k_ray(const BatchDev* __restrict__ bp) {
  __shared__ RaySetup s_ray[kRayThreads];
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RaySetup* wr = s_ray + warp * 32;
  const int64_t n_warps = (int64_t)gridDim.x * (kRayThreads / 32);
  int smap = -1;  // map of this lane's sample count
  unsigned long long samples = 0;
  for (int64_t wbase = ((int64_t)blockIdx.x * (kRayThreads / 32) + warp) * 32; wbase < b.n_points;
       wbase += n_warps * 32) {
    // ---- set-up: one ray per lane
    RaySetup r;
    r.n = 0;
    r.map = 0;
    const int64_t g = wbase + lane;
    if (g < b.n_points) {
      const int ci = find_cloud(b.clouds, b.n_clouds, g);
      const CloudDev& c = b.clouds[ci];
      const MapDev& m = b.maps[c.map];
      r.map = c.map;
      if (m.ray_step > 0.f) {
        float px, py, pz;
        load_point(c, g - c.begin, px, py, pz);
        const PointGeom pg = point_geom<kExt>(m, c, px, py, pz);
        // clip the sample range to the map box (conservative by 1 mm + 1 step)
        float lo = 0.f, hi = pg.d;
        const float ext_x = __fmul_rn((float)m.W, m.res), ext_y = __fmul_rn((float)m.H, m.res);
        if (pg.in_range && pg.d > 0.f && slab(c.t[0], pg.vx, pg.d, m.x0, m.x0 + ext_x, lo, hi) &&
            slab(c.t[1], pg.vy, pg.d, m.y0, m.y0 + ext_y, lo, hi) && lo <= hi + 1e-3f) {
          const float step = m.ray_step;
          const float kl = floorf(__fdividef(lo - 1e-3f, step)) - 1.f;
          const float kh = ceilf(__fdividef(hi + 1e-3f, step)) + 1.f;
          const int32_t k_lo = kl < 1.f ? 1 : kl > (float)kMaxRayK ? kMaxRayK : (int32_t)kl;
          int32_t k_hi = kh > (float)kMaxRayK ? kMaxRayK : (int32_t)kh;
          // last k with k * step < d, decided exactly as sample by sample
          // (the estimate is within a few units of the answer; past kMaxRayK the
          // range is capped anyway, so the searches stop there)
          float kf = fminf(floorf(__fdividef(pg.d, step)), (float)kMaxRayK);  // an estimate, made exact just below
          int32_t k_last = (int32_t)kf;
          for (int it = 0; it < 64 && k_last > 0 && !(__fmul_rn((float)k_last, step) < pg.d); ++it) --k_last;
          for (int it = 0; it < 64 && k_last < kMaxRayK && __fmul_rn((float)(k_last + 1), step) < pg.d; ++it) ++k_last;
          if (k_last < k_hi) k_hi = k_last;
          const float cstep = __fdiv_rn(step, pg.d);  // f_k = k * step / d
          r.ax = __fmul_rn(__fsub_rn(c.t[0], m.x0), m.inv_res);
          r.ay = __fmul_rn(__fsub_rn(c.t[1], m.y0), m.inv_res);
          r.bx = __fmul_rn(__fmul_rn(cstep, pg.vx), m.inv_res);
          r.by = __fmul_rn(__fmul_rn(cstep, pg.vy), m.inv_res);
          r.az = c.t[2];
          r.bz = __fmul_rn(cstep, pg.vz);
          r.vx = pg.vx; r.vy = pg.vy; r.vz = pg.vz;
          r.d = pg.d;
          r.ix = pg.ix;
          r.iy = pg.iy;
          r.k_lo = k_lo;
          r.n = k_hi >= k_lo ? k_hi - k_lo + 1 : 0;
        }
      }
    }
    wr[lane] = r;
    __syncwarp();
    // ---- march: G lanes per ray, 4 samples per lane and step (4 gathers in flight)
    const int gl = lane % G;
    for (int r0 = 0; r0 < 32; r0 += 32 / G) {
      const RaySetup& R = wr[r0 + lane / G];
      if (R.n <= 0) continue;
      if (R.map != smap) {  // count this lane's samples per map
        if (smap >= 0 && samples) atomicAdd(&b.maps[smap].ctl->stats[kStRaySamples], samples);
        samples = 0;
        smap = R.map;
      }
      if (gl == 0) samples += (unsigned long long)R.n;
      const MapDev& m = b.maps[R.map];
      const int32_t W = m.W, H = m.H, ox = m.ox, oy = m.oy;
      const float* __restrict__ thr = m.thr;
      const bool guard = m.alpha_n > 0.f;
      const int32_t k_end = R.k_lo + R.n, rix = R.ix, riy = R.iy;
      const float ax = R.ax, bx = R.bx, ay = R.ay, by = R.by, az = R.az, bz = R.bz;
      float kf = (float)(R.k_lo + gl);  // sample index as a float, stepped exactly (k < 2^24)
      for (int32_t k = R.k_lo + gl; k < k_end; k += 4 * G) {
        int32_t pl[4];
        float zz[4], th[4];
        bool any = false;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          // floor(t) of t = fma(k, b, a) by one add rounded down: t + 1.5 2^23 lands where the
          // float spacing is 1, so its bits hold floor(t) + 0x4B400000 (|t| < 2^22; anything
          // farther out gives an index outside [0, 2^22) and fails the box test below)
          const int32_t cx = __float_as_int(__fadd_rd(__fmaf_rn(kf, bx, ax), 12582912.0f)) - 0x4B400000;
          const int32_t cy = __float_as_int(__fadd_rd(__fmaf_rn(kf, by, ay), 12582912.0f)) - 0x4B400000;
          const bool ok = k + u * G < k_end && (uint32_t)cx < (uint32_t)W && (uint32_t)cy < (uint32_t)H &&
                          !(cx == rix && cy == riy);
          pl[u] = cy * W + cx;  // logical index
          zz[u] = __fmaf_rn(kf, bz, az);
          th[u] = ok ? __ldg(thr + pl[u]) : __int_as_float(0xff800000);
          kf = __fadd_rn(kf, (float)G);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) any |= zz[u] < th[u];
        if (!any) continue;  // the common case: no sample of these four is below its cell
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!(zz[u] < th[u])) continue;  // also skips the samples that are not taken (th = -inf)
          // physical cell of the sample (ring-buffer layout of the map layers)
          const int32_t cy = pl[u] / W, cx = pl[u] - cy * W;
          int32_t px = cx + ox;
          px -= (px >= W) ? W : 0;
          int32_t py = cy + oy;
          py -= (py >= H) ? H : 0;
          const int32_t p = py * W + px;
          if (kExt && !isfinite(m.var[p])) {
            // an empty cell (its threshold is the upper bound): the sample lowers
            // the bound (Section II-H); float minimum through the ordered bits
            const float z = zz[u];
            if (__float_as_int(z) >= 0) atomicMin(reinterpret_cast<int*>(m.upper + p), __float_as_int(z));
            else atomicMax(reinterpret_cast<unsigned int*>(m.upper + p), __float_as_uint(z));
            continue;
          }
          if (guard) {
            float n0 = m.nx[p], n1 = m.ny[p], n2 = m.nz[p];
            if (!(isfinite(n0) && isfinite(n1) && isfinite(n2))) { n0 = 0.f; n1 = 0.f; n2 = 1.f; }
            const float rx = __fdiv_rn(R.vx, R.d), ry = __fdiv_rn(R.vy, R.d), rz = __fdiv_rn(R.vz, R.d);
            const float dot = fabsf(__fmaf_rn(rx, n0, __fmaf_rn(ry, n1, __fmul_rn(rz, n2))));
            if (!(dot > m.alpha_n)) continue;
          }
          // many rays graze the same surface cells: skip the atomic when the bit is
          // already set (marks are only ever set during this kernel)
          const uint32_t bit = 1u << (p & 31);
          if (!(*(volatile uint32_t*)(m.mark + (p >> 5)) & bit)) atomicOr(&m.mark[p >> 5], bit);
        }
      }
    }
    __syncwarp();
  }
  // samples per map: a warp sum when the warp's lanes end on one map, else per
  // lane (no block barrier: warps of a block finish at different times)
  const int m0 = __shfl_sync(0xffffffffu, smap, 0);
  if (__all_sync(0xffffffffu, smap == m0 || samples == 0)) {
    unsigned long long t = samples;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0 && m0 >= 0 && t) atomicAdd(&b.maps[m0].ctl->stats[kStRaySamples], t);
  } else if (smap >= 0 && samples) {
    atomicAdd(&b.maps[smap].ctl->stats[kStRaySamples], samples);
  }
}

constexpr int kClearThreads = 256;

// One block per tile of kTile cells, four consecutive cells per thread, so the
// loads of all marked cells of a tile are in flight together (the marks of a
// LiDAR frame are dense along the rays: one thread walking a word's bits would
// chain its loads).
static_assert(kTile == 4 * kClearThreads, "k_clear: four cells per thread");
__global__ void __launch_bounds__(kClearThreads) k_clear(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  const int64_t n_tiles = b.n_cells / kTile;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t g0 = t * kTile;
    const int mi = find_map_cell(b.maps, b.n_maps, g0);
    const MapDev& m = b.maps[mi];
    const int64_t p0 = g0 - m.cell_begin;
    const int32_t ncell = m.W * m.H;
    if (p0 >= ncell) continue;  // padding at the end of a map (block-uniform)
    const int32_t c0 = (int32_t)p0 + 4 * threadIdx.x;  // this thread's cells c0 .. c0 + 3 (one word's quarter byte)
    const int32_t w = c0 >> 5;
    const uint32_t word = c0 < ncell ? m.mark[w] : 0u;
    const uint32_t bits = (word >> (c0 & 31)) & 15u;
    unsigned cleared = 0;
    if (bits) {
      const int32_t min_age = m.min_age > 1 ? m.min_age : 1;
      float var[4];
      int32_t tl[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // all loads first
        const bool mk = ((bits >> k) & 1u) && c0 + k < ncell;
        var[k] = mk ? m.var[c0 + k] : __int_as_float(0x7f800000);
        tl[k] = mk ? m.t_last[c0 + k] : 0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!isfinite(var[k]) || m.t_now - tl[k] < min_age) continue;
        m.h[c0 + k] = __int_as_float(0x7fc00000);
        m.var[c0 + k] = __int_as_float(0x7f800000);
        ++cleared;
      }
    }
    // the word is reset by the thread holding its first cells, after its 8 readers
    // (one warp) have read it
    __syncwarp();
    if ((c0 & 31) == 0 && word) m.mark[w] = 0u;
    const unsigned tot = __reduce_add_sync(0xffffffffu, cleared);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&m.ctl->stats[kStCleared], (unsigned long long)tot);
  }
}

template <bool kExt>
static void launch_ray_g(const BatchDev* b, int g, int grid, cudaStream_t s) {
  switch (g) {
    case 1: k_ray<1, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 2: k_ray<2, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 8: k_ray<8, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 16: k_ray<16, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 32: k_ray<32, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    default: k_ray<4, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
  }
}

cudaError_t launch_ray(const BatchDev* b, int64_t n_points, int group, bool ext, cudaStream_t s) {
  if (n_points <= 0) return cudaSuccess;
  const int g = (group == 1 || group == 2 || group == 4 || group == 8 || group == 16 || group == 32) ? group : 4;
  const int64_t want = (n_points + kRayThreads - 1) / kRayThreads;  // one 32-ray chunk per warp
  const int64_t cap = (int64_t)sm_count() * 16;
  const int grid = (int)(want < cap ? want : cap);
  if (ext) launch_ray_g<true>(b, g, grid, s);
  else launch_ray_g<false>(b, g, grid, s);
  return cudaGetLastError();
}

// Overlap clearance (Section II-F): after the update, an estimate whose cell
// centre lies within overlap_radius of the robot (the first cloud's sensor
// origin) and whose height is more than overlap_dz from the robot's belongs to
// another floor and is removed.
__global__ void __launch_bounds__(kClearThreads) k_overlap(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  for_each_tile(b, [&](const MapDev& m, int, int32_t p0, int32_t count) {
    if (m.ovl_dz <= 0.f) return;
    for (int32_t i = threadIdx.x; i < count; i += kClearThreads) {
      const int32_t p = p0 + i;
      if (!isfinite(m.var[p])) continue;
      int32_t lx, ly;
      logical_of(m, p, lx, ly);
      const float cx = __fsub_rn(__fmaf_rn(__fadd_rn((float)lx, 0.5f), m.res, m.x0), m.ref_x);
      const float cy = __fsub_rn(__fmaf_rn(__fadd_rn((float)ly, 0.5f), m.res, m.y0), m.ref_y);
      if (__fmaf_rn(cx, cx, __fmul_rn(cy, cy)) <= m.ovl_r2 && fabsf(__fsub_rn(m.h[p], m.z_ref)) > m.ovl_dz) {
        m.h[p] = __int_as_float(0x7fc00000);
        m.var[p] = __int_as_float(0x7f800000);
      }
    }
  });
}

cudaError_t launch_overlap(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * 8;
  k_overlap<<<(int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap), kClearThreads, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_clear(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  const int64_t tiles = n_cells / kTile;  // a block per tile
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap);
  k_clear<<<grid, kClearThreads, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace em
