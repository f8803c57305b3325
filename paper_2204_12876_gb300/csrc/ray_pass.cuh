// ray_pass.cuh -- the device passes of the visibility cleanup (k_ray.cu): the
// coarse threshold grid, the ray march with its exact chunk test, the removal
// of marked cells and the overlap clearance.  Each pass runs on the blocks of
// a Grid: its own kernel's, or the persistent kernel's (k_persist.cu).
#pragma once

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

// Per-ray set-up, made by one lane and read by the lanes that test and march
// the ray's chunks.  Sample k lies at q = a + k b in cell units (x, y) and at
// z = az + k bz, i.e. the track o + (k step / d) (R p_s) measured from the map
// corner in cells.  Samples per ray are capped at 2^24 - 1, so the float
// sample index is exact.
constexpr int32_t kMaxRayK = (1 << 24) - 1;

struct RaySetup {
  float ax, bx, ay, by, az, bz;
  float vx, vy, vz, d;  // for the Eq. 4 guard
  int32_t ix, iy, k_lo, n, map;
  int32_t cn;           // samples per chunk
};

// floor(t) of a cell coordinate by one add rounded down: t + 1.5 2^23 lands
// where the float spacing is 1, so its bits hold floor(t) + 0x4B400000 (|t| <
// 2^22; anything farther out gives an index outside [0, 2^22) and fails the
// map's box test)
__device__ __forceinline__ int32_t cell_floor(float t) {
  return __float_as_int(__fadd_rd(t, 12582912.0f)) - 0x4B400000;
}

// Largest ray threshold per coarse block of every map with the ray march.
constexpr int kCoarseThreads = 256;
__device__ __forceinline__ void coarse_pass(const BatchDev& b, Grid gr) {
  for (int64_t g = (int64_t)gr.bid * blockDim.x + threadIdx.x; g < b.n_coarse; g += (int64_t)gr.nb * blockDim.x) {
    int lo = 0, hi = b.n_maps - 1;  // the last map whose coarse range starts at or before g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.maps[mid].cbegin <= g) lo = mid; else hi = mid - 1;
    }
    const MapDev& m = b.maps[lo];
    const int32_t q = (int32_t)(g - m.cbegin);
    const int32_t by = q / m.CW, bx = q - by * m.CW;
    const int32_t x0 = bx << kCoarseShift, y0 = by << kCoarseShift;
    const int32_t nx = min(kCoarse, m.W - x0), ny = min(kCoarse, m.H - y0);
    float mx = __int_as_float(0xff800000);
    for (int32_t y = 0; y < ny; ++y) {
      const float* row = m.thr + (int64_t)(y0 + y) * m.W + x0;
      for (int32_t x = 0; x < nx; ++x) mx = fmaxf(mx, __ldg(row + x));  // a NaN never marks: skipped
    }
    m.cthr[q] = mx;
  }
}

// Shared memory of the march: the warps' rays, one array per field (lanes
// reading the fields of different rays hit different banks), and the chunk
// queues.
constexpr int kRayQ = 256;  // queued chunks per warp (a ring)
constexpr int kRayRun = 8;   // 32-point batches per take from the work counter, at most
struct RaySmem {
  float ax[kRayThreads], bx[kRayThreads], ay[kRayThreads], by[kRayThreads], az[kRayThreads], bz[kRayThreads];
  float vx[kRayThreads], vy[kRayThreads], vz[kRayThreads], d[kRayThreads];
  int32_t ix[kRayThreads], iy[kRayThreads], k_lo[kRayThreads], n[kRayThreads], map[kRayThreads],
      cn[kRayThreads];
  int2 q[kRayThreads / 32][kRayQ];  // {ray | samples << 8, first sample}
};

__device__ __forceinline__ void put_ray(RaySmem& S, int t, const RaySetup& r) {
  S.ax[t] = r.ax; S.bx[t] = r.bx; S.ay[t] = r.ay; S.by[t] = r.by; S.az[t] = r.az; S.bz[t] = r.bz;
  S.vx[t] = r.vx; S.vy[t] = r.vy; S.vz[t] = r.vz; S.d[t] = r.d;
  S.ix[t] = r.ix; S.iy[t] = r.iy; S.k_lo[t] = r.k_lo; S.n[t] = r.n; S.map[t] = r.map; S.cn[t] = r.cn;
}

// Each warp takes 32 consecutive points: every lane sets up one ray (transform,
// distance, own cell, the k range inside the map box and before the point, its
// chunk length) and tests its ray's chunks one after another; the warp queues
// the chunks that may mark a cell and marches them 4 x 32 / G at a time, G
// lanes per chunk and one sample per lane and round (4 gathers in flight).
template <int G, bool kExt>
__device__ __forceinline__ void ray_pass(const BatchDev& b, Grid gr, RaySmem& S) {
  constexpr int kWarps = kRayThreads / 32;
  constexpr int kU = G >= 4 ? 4 : G;         // samples per lane and march round, all of one chunk
  constexpr int kLPC = G / kU;               // lanes per chunk in the march
  constexpr int kFQ = 32 / kLPC;             // chunks per march round (at most 32)
  constexpr int kCU = 4;                     // chunks per lane and test round (their loads in flight together)
  constexpr int kQ = kRayQ;
  static_assert(kQ >= kFQ - 1 + 32 * kCU && kFQ <= 32, "queue capacity");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wb = warp * 32;  // the warp's rays in S
  int2* q = S.q[warp];
  // warps take runs of consecutive 32-point batches from the work counter
  // (rays of uneven maps differ in length: the counter balances them); a run
  // mostly lies in one cloud and map (one sample count per map change below).
  // Runs are as long as leaves every warp of the grid two of them, at most
  // kRayRun batches.
  const int64_t n_batches = (b.n_points + 31) / 32;
  const int64_t run_len = max((int64_t)1, min((int64_t)kRayRun, n_batches / (2 * (int64_t)gr.nb * kWarps)));
  int smap = -1;  // the map of the warp's running sample count (warp-uniform)
  int hint = -1;  // this lane's cloud in the previous batch
  unsigned long long samples = 0;
  int64_t wbase = 0, w_end = 0;
  for (;;) {
    if (wbase >= w_end) {  // the next run (warp-uniform)
      int run = 0;
      if (lane == 0) run = atomicAdd(&b.ctl->ray_next, 1);
      run = __shfl_sync(0xffffffffu, run, 0);
      const int64_t b0 = (int64_t)run * run_len;
      if (run < 0 || b0 >= n_batches) break;
      wbase = b0 * 32;
      w_end = min(b0 + run_len, n_batches) * 32;
    }
    // ---- set-up: one ray per lane
    RaySetup r;
    r.n = 0;
    r.map = 0;
    r.cn = 1;
    const int64_t g = wbase + lane;
    if (g < b.n_points) {
      const int ci = find_cloud(b.clouds, b.n_clouds, g, hint);
      hint = ci;
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
          // a chunk and the next chunk's first sample span about kCoarse cells per axis at
          // most, so they touch at most 2 x 2 blocks (a rounding case that touches more is
          // marched untested)
          const float span = fmaxf(fmaxf(fabsf(r.bx), fabsf(r.by)), 1e-6f);
          r.cn = (int32_t)fminf((float)G, fmaxf(1.f, floorf(__fdividef((float)kCoarse, span))));
        }
      }
    }
    {  // samples of the march, per map: a warp sum when the batch's rays share a map
      const int m0 = __shfl_sync(0xffffffffu, r.map, 0);
      unsigned long long t = (unsigned long long)r.n;
      if (__all_sync(0xffffffffu, r.map == m0 || r.n == 0)) {
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (m0 != smap) {
          if (lane == 0 && smap >= 0 && samples) atomicAdd(&b.maps[smap].ctl->stats[kStRaySamples], samples);
          samples = 0;
          smap = m0;
        }
        samples += t;
      } else if (r.n > 0) {  // a batch across a map boundary: per lane
        atomicAdd(&b.maps[r.map].ctl->stats[kStRaySamples], t);
      }
    }
    put_ray(S, wb + lane, r);
    __syncwarp();
    // ---- the chunks of the warp's rays against the coarse grid, kCU consecutive
    // chunks of one ray per lane and round.  A ray has nq such quads.  When
    // the rays' lengths differ (points in random order), lanes that each test
    // only their own ray would idle while the longest ray is tested: the quads
    // are then dealt out in order across the lanes (quad j of the warp goes to
    // lane j mod 32 in round j / 32), which the warp does when that saves at
    // least a quarter of the rounds.
    const int32_t nch = r.n > 0 ? (r.n + r.cn - 1) / r.cn : 0;
    const int32_t nq = (nch + kCU - 1) / kCU;
    int32_t qinc = nq;  // inclusive scan of the quads over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, qinc, o);
      if (lane >= o) qinc += t;
    }
    const int32_t qtot = __shfl_sync(0xffffffffu, qinc, 31);
    const int32_t qmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)nq);
    const bool flat = 4 * ((qtot + 31) >> 5) <= 3 * qmax;  // warp-uniform
    const int32_t rounds = flat ? (qtot + 31) >> 5 : qmax;
    int qh = 0, qn = 0;  // queue head and length (warp-uniform)
    for (int32_t it = 0; it < rounds; ++it) {
      // this lane's quad: ray `src`, chunks c0 .. c0 + kCU - 1
      int src = lane;
      int32_t c0 = it * kCU;
      bool act = it < nq;
      if (flat) {
        const int32_t j = it * 32 + lane;
        int o = 0;  // lanes whose quads all come before quad j: the owner of quad j
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
          const int32_t v = __shfl_sync(0xffffffffu, qinc, o + s - 1);
          if (v <= j) o += s;
        }
        act = j < qtot;
        src = o < 32 ? o : 31;
        c0 = (j - __shfl_sync(0xffffffffu, qinc - nq, src)) * kCU;
      }
      const int sr = wb + src;
      const int32_t k_lo = S.k_lo[sr], n = S.n[sr], cn = S.cn[sr];
      const float ax = S.ax[sr], bx = S.bx[sr], ay = S.ay[sr], by = S.by[sr], az = S.az[sr], bz = S.bz[sr];
      const MapDev& m = b.maps[S.map[sr]];
      const float* __restrict__ ct = m.cthr;
      const int32_t W = m.W, H = m.H, CW = m.CW;
      // The round's chunks c0 .. c0 + kCU - 1 and their end samples: chunk u is
      // tested over its own samples and the next chunk's first one (a superset,
      // so the test stays exact), so neighbouring chunks share an end and its
      // block.  All loads of the round come first (predicated, no branches
      // between them), then the tests.
      const int32_t klast = k_lo + n - 1;
      int32_t xc[kCU + 1], yc[kCU + 1], bxs[kCU + 1], bys[kCU + 1];
      float zc[kCU + 1], ve[kCU + 1];
#pragma unroll
      for (int u = 0; u <= kCU; ++u) {
        const float kf = (float)min(k_lo + (c0 + u) * cn, klast);
        xc[u] = cell_floor(__fmaf_rn(kf, bx, ax));
        yc[u] = cell_floor(__fmaf_rn(kf, by, ay));
        zc[u] = __fmaf_rn(kf, bz, az);
        bxs[u] = min(max(xc[u], 0), W - 1) >> kCoarseShift;
        bys[u] = min(max(yc[u], 0), H - 1) >> kCoarseShift;
        ve[u] = act ? __ldg(ct + bys[u] * CW + bxs[u]) : __int_as_float(0xff800000);
      }
      bool keep[kCU];
      int32_t k0[kCU], cnt[kCU];
#pragma unroll
      for (int u = 0; u < kCU; ++u) {
        const int32_t c = c0 + u;
        k0[u] = k_lo + c * cn;
        cnt[u] = min(cn, n - c * cn);
        const int32_t xl = min(xc[u], xc[u + 1]), xh = max(xc[u], xc[u + 1]);
        const int32_t yl = min(yc[u], yc[u + 1]), yh = max(yc[u], yc[u + 1]);
        // some sample of the chunk may be inside the map
        const bool inside = act && c * cn < n && xh >= 0 && xl < W && yh >= 0 && yl < H;
        // more than 2 x 2 blocks (not for the chunk lengths above): march it untested
        const bool wide = abs(bxs[u + 1] - bxs[u]) > 1 || abs(bys[u + 1] - bys[u]) > 1;
        // the two other corners of the 2 x 2 box, when the chunk crosses a block row and column
        const bool cross = inside && !wide && bxs[u] != bxs[u + 1] && bys[u] != bys[u + 1];
        const float o1 = cross ? __ldg(ct + bys[u] * CW + bxs[u + 1]) : __int_as_float(0xff800000);
        const float o2 = cross ? __ldg(ct + bys[u + 1] * CW + bxs[u]) : __int_as_float(0xff800000);
        const float mx = fmaxf(fmaxf(ve[u], ve[u + 1]), fmaxf(o1, o2));
        keep[u] = inside && (wide || fminf(zc[u], zc[u + 1]) < mx);
      }
      // ---- queue the chunks that may mark a cell
#pragma unroll
      for (int u = 0; u < kCU; ++u) {
        const unsigned km = __ballot_sync(0xffffffffu, keep[u]);
        if (keep[u])
          q[(qh + qn + __popc(km & ((1u << lane) - 1u))) & (kQ - 1)] = make_int2(src | (cnt[u] << 8), k0[u]);
        qn += __popc(km);
      }
      __syncwarp();
      // ---- march the queued chunks, kFQ at a time (all of them after the last test)
      const bool last = it + 1 >= rounds;
      while (qn >= kFQ || (last && qn > 0)) {
        // lane: chunk qi, samples sj, sj + kLPC, ...; every threshold first (kU gathers
        // in flight), then the marks
        const int qi = lane / kLPC, sj = lane % kLPC;
        const int2 e = q[(qh + qi) & (kQ - 1)];
        const int32_t ne = e.x >> 8;
        const int sr = wb + (e.x & 31);
        const int32_t rmap = S.map[sr];
        const bool live = qi < qn && (unsigned)rmap < (unsigned)b.n_maps;
        const MapDev& mm = b.maps[live ? rmap : 0];
        const int32_t Wm = mm.W, Hm = mm.H, ox = mm.ox, oy = mm.oy;
        const float* __restrict__ tm = mm.thr;
        uint32_t* __restrict__ mk = mm.mark;
        const float ax = S.ax[sr], bx = S.bx[sr], ay = S.ay[sr], by = S.by[sr], az = S.az[sr], bz = S.bz[sr];
        const int32_t rix = S.ix[sr], riy = S.iy[sr];
        float zz[kU], th[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int32_t j = sj + u * kLPC;
          const float kf = (float)(e.y + j);
          const int32_t cx = cell_floor(__fmaf_rn(kf, bx, ax));
          const int32_t cy = cell_floor(__fmaf_rn(kf, by, ay));
          const bool ok = live && j < ne && (uint32_t)cx < (uint32_t)Wm && (uint32_t)cy < (uint32_t)Hm &&
                          !(cx == rix && cy == riy);
          zz[u] = __fmaf_rn(kf, bz, az);
          th[u] = ok ? __ldg(tm + cy * Wm + cx) : __int_as_float(0xff800000);  // logical index; -inf: never below
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          if (!(zz[u] < th[u])) continue;  // the common case, and every sample not taken
          // the sample's cell again (the same rounded arithmetic as above: no
          // register holds it through the gathers), then its physical index in
          // the ring-buffer layout of the map layers
          const float kf = (float)(e.y + sj + u * kLPC);
          const int32_t cx = cell_floor(__fmaf_rn(kf, bx, ax));
          const int32_t cy = cell_floor(__fmaf_rn(kf, by, ay));
          int32_t px = cx + ox;
          px -= (px >= Wm) ? Wm : 0;
          int32_t py = cy + oy;
          py -= (py >= Hm) ? Hm : 0;
          const int32_t p = py * Wm + px;
          if (kExt && !isfinite(mm.var[p])) {
            // an empty cell (its threshold is the upper bound): the sample lowers
            // the bound (Section II-H); float minimum through the ordered bits
            if (__float_as_int(zz[u]) >= 0) atomicMin(reinterpret_cast<int*>(mm.upper + p), __float_as_int(zz[u]));
            else atomicMax(reinterpret_cast<unsigned int*>(mm.upper + p), __float_as_uint(zz[u]));
            continue;
          }
          if (mm.alpha_n > 0.f) {
            float n0 = mm.nx[p], n1 = mm.ny[p], n2 = mm.nz[p];
            if (!(isfinite(n0) && isfinite(n1) && isfinite(n2))) { n0 = 0.f; n1 = 0.f; n2 = 1.f; }
            const float rd = S.d[sr];
            const float rx = __fdiv_rn(S.vx[sr], rd), ry = __fdiv_rn(S.vy[sr], rd), rz = __fdiv_rn(S.vz[sr], rd);
            const float dot = fabsf(__fmaf_rn(rx, n0, __fmaf_rn(ry, n1, __fmul_rn(rz, n2))));
            if (!(dot > mm.alpha_n)) continue;
          }
          // many rays graze the same surface cells: skip the atomic when the bit is
          // already set.  Bits are only ever set during this kernel, so a stale read
          // can only cost a redundant atomic, never a lost mark.
          const uint32_t bit = 1u << (p & 31);
          if (!(mk[p >> 5] & bit)) atomicOr(&mk[p >> 5], bit);
        }
        const int took = min(qn, kFQ);
        qh = (qh + took) & (kQ - 1);
        qn -= took;
        __syncwarp();
      }
    }
    __syncwarp();
    wbase += 32;
  }
  if (lane == 0 && smap >= 0 && samples) atomicAdd(&b.maps[smap].ctl->stats[kStRaySamples], samples);
  __syncthreads();  // the shared memory is free again
}

constexpr int kClearThreads = 256;

// One block per tile of kTile cells, four consecutive cells per thread, so the
// loads of all marked cells of a tile are in flight together (the marks of a
// LiDAR frame are dense along the rays: one thread walking a word's bits would
// chain its loads).
static_assert(kTile == 4 * kClearThreads, "k_clear: four cells per thread");
__device__ __forceinline__ void clear_pass(const BatchDev& b, Grid gr) {
  const int64_t n_tiles = b.n_cells / kTile;
  for (int64_t t = gr.bid; t < n_tiles; t += gr.nb) {
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

// Overlap clearance (Section II-F): after the update, an estimate whose cell
// centre lies within overlap_radius of the robot (the first cloud's sensor
// origin) and whose height is more than overlap_dz from the robot's belongs to
// another floor and is removed.
__device__ __forceinline__ void overlap_pass(const BatchDev& b, Grid gr) {
  for_each_tile(b, gr, [&](const MapDev& m, int, int32_t p0, int32_t count) {
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

}  // namespace em
