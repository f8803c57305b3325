// k_fuse.cu -- per-cell fusion (Section II-C of the paper).
//
// Every cell that received points in this update is fused once from its
// records (z, sigma_p^2):
//   1. wall rule: in a valid cell with more than wall_num_thresh points, points
//      below the current height are dropped (before the outlier test);
//   2. Mahalanobis gate against the pre-update estimate: reject iff
//      |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k, tested as
//      (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2) (no division or square root);
//      every rejection adds outlier_variance to sigma_m^2;
//   3. Eq. 1 and Eq. 2 for all accepted points at once, in information form:
//        Lambda = 1 / (sigma_m^2 + n_rej v_out) + sum_i 1/sigma_p,i^2
//        h'     = h_ref + sum_i (z_i - h_ref) / sigma_p,i^2 / Lambda,   sigma_m^2' = 1 / Lambda
//      with h_ref = h for a valid cell (an empty cell has 1/sigma_m^2 = 0 and
//      h_ref = the map's reference height z_ref).  Applying Eq. 1/2 point
//      after point gives the same result in exact arithmetic.
//
// The two sums are accumulated exactly: every float32 term is converted to a
// fixed-point integer with 44 fractional bits (kept as h 2^27 + l) and the
// integers are added.  Integer addition is associative, so the result is the
// same for every order of the points and every split of the work, bit for bit
// (no float atomics).
//
// Work split: one block per tile of kTile cells (the records of a tile are one
// range, k_sort.cu).  The block stages the tile's pre-update state (h and the
// effective variance) in shared memory, streams the tile's records with every
// thread on one record (the next window's loads in flight), reduces each run
// of equal cells in consecutive lanes with a segmented scan, and adds the
// run's sums to the cell's accumulators in shared memory (64-bit integer
// atomics).  Then every touched cell of the tile is written once.  Blocks take
// tiles from a counter, the heavy tiles (many records) first.
#include "em_point.cuh"

namespace em {

constexpr unsigned kFull = 0xffffffffu;

// The cell's snapshot and the decisions that do not depend on single points.
struct CellCtx {
  float h, ve, href, k2;
  bool valid, wall_on, gate_on;
};

// The pre-update state of a cell, loaded ahead of its use.
struct Snap {
  float h, var;
  int32_t t_last;
};

__device__ __forceinline__ Snap load_snap(const MapDev& m, int32_t cell) {
  return Snap{m.h[cell], m.var[cell], m.t_last[cell]};
}

__device__ __forceinline__ CellCtx make_cell(const MapDev& m, const Snap& sn, bool wall_armed) {
  CellCtx c;
  c.h = sn.h;
  c.valid = isfinite(sn.var);
  c.ve = c.valid ? var_eff(m, sn.var, sn.t_last) : sn.var;
  c.href = c.valid ? c.h : m.z_ref;
  c.wall_on = wall_armed && c.valid;
  c.gate_on = c.valid && m.k > 0.f;
  c.k2 = __fmul_rn(m.k, m.k);
  return c;
}

__device__ __forceinline__ CellCtx load_cell(const MapDev& m, int32_t cell, bool wall_armed) {
  return make_cell(m, load_snap(m, cell), wall_armed);
}

// One record: wall rule, gate, and its two fixed-point terms when accepted
// (zero terms otherwise).
__device__ __forceinline__ uint8_t fuse_one(const CellCtx& c, float z, float vp, Fix& fw, Fix& ft) {
  fw = Fix{0, 0u};
  ft = Fix{0, 0u};
  if (c.wall_on && z < c.h) return kPtWall;
  if (c.gate_on) {
    // |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k  <=>  (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2)  (k > 0)
    const float dz = __fsub_rn(z, c.h);
    if (__fmul_rn(dz, dz) > __fmul_rn(c.k2, __fadd_rn(c.ve, vp))) return kPtRejected;
  }
  const float w = __frcp_rn(vp);
  fw = to_fix(w);
  ft = to_fix(__fmul_rn(w, __fsub_rn(z, c.href)));
  return kPtFused;
}

// New state of the cell from its complete sums (one thread); true when the
// cell took a point (accepted or rejected).
__device__ __forceinline__ bool write_cell(const MapDev& m, int32_t cell, const CellCtx& c, __int128 qw,
                                           __int128 qt, int acc, int rej) {
  if (acc + rej == 0) return false;
  float h_new, var_new;
  const float sw = fixed_to_float(qw);
  const float st = fixed_to_float(qt);
  if (c.valid) {
    const float vprior = __fadd_rn(c.ve, __fmul_rn((float)rej, m.v_out));
    if (acc == 0) {
      h_new = c.h;
      var_new = vprior;
    } else {
      const float lam = __fadd_rn(__frcp_rn(vprior), sw);
      h_new = __fadd_rn(c.h, __fdiv_rn(st, lam));
      var_new = __frcp_rn(lam);
    }
  } else {
    h_new = __fadd_rn(c.href, __fdiv_rn(st, sw));
    var_new = __frcp_rn(sw);
  }
  m.h[cell] = h_new;
  m.var[cell] = var_new;
  m.t_last[cell] = m.t_now;
  if (m.upper) m.upper[cell] = __int_as_float(0x7f800000);  // observed: no bound (Section II-H)
  return true;
}

// Per-cell accumulators of one tile in shared memory, and its staged state.
struct TileSmem {
  long long wh[kTile], th[kTile];            // fixed-point sums: high parts
  unsigned long long wl[kTile], tl[kTile];   // ... and low parts (value h 2^27 + l)
  unsigned long long n[kTile];               // accepted | rejected << 32
  float h[kTile], ve[kTile];                 // pre-update height, effective variance (+inf: empty)
  uint32_t cnt[kTile];                       // records per cell (the wall rule)
  int work;
  unsigned long long stat[4];                // accepted, rejected, wall, cells of the tile
};

template <int NT>
__global__ void __launch_bounds__(NT) k_fuse(const BatchDev* __restrict__ bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31;
  const int64_t n_tiles = b.n_cells / kTile;
  const int n_heavy = b.ctl->n_heavy;
  // every block takes work items from the counter until they run out; a block
  // takes at most all of them (a bound that holds whatever the counter reads)
  for (int64_t items = 0;; ++items) {
    if (threadIdx.x == 0) S.work = atomicAdd(&b.ctl->fuse_next, 1);
    __syncthreads();
    const int w = S.work;
    if (items > n_tiles + n_heavy || w < 0 || n_heavy < 0 || n_heavy > n_tiles) {
      if (threadIdx.x == 0) atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
      break;
    }
    int64_t t;
    if (w < n_heavy) {
      t = b.heavy[w];
    } else {
      t = w - n_heavy;
      if (t >= n_tiles) break;  // block-uniform
    }
    const int32_t r0 = b.tile_base[t], r1 = b.tile_base[t + 1];
    if (r1 == r0 || (w >= n_heavy && r1 - r0 > b.heavy_thresh)) {  // nothing to fuse, or a heavy tile done first
      __syncthreads();
      continue;
    }
    const int mi = find_map_cell(b.maps, b.n_maps, t * kTile);
    const MapDev& m = b.maps[mi];
    const int32_t p0 = (int32_t)(t * kTile - m.cell_begin);
    const int32_t ncell = min(kTile, m.W * m.H - p0);
    const bool wall_on = m.wall > 0;
    // ---- the tile's pre-update state; accumulators to zero
    for (int c = threadIdx.x; c < kTile; c += NT) {
      float h = 0.f, ve = __int_as_float(0x7f800000);
      if (c < ncell) {
        const float var = __ldg(m.var + p0 + c);
        h = __ldg(m.h + p0 + c);
        const int32_t tl = __ldg(m.t_last + p0 + c);
        if (isfinite(var)) ve = var_eff(m, var, tl);
      }
      S.h[c] = h;
      S.ve[c] = ve;
      S.wh[c] = 0;
      S.th[c] = 0;
      S.wl[c] = 0;
      S.tl[c] = 0;
      S.n[c] = 0;
      S.cnt[c] = 0;
    }
    if (threadIdx.x < 4) S.stat[threadIdx.x] = 0;
    __syncthreads();
    if (wall_on) {  // records per cell first: the wall rule looks at the cell's count
      for (int32_t r = r0 + threadIdx.x; r < r1; r += NT) atomicAdd(&S.cnt[__ldg(b.rc + r)], 1u);
      __syncthreads();
    }
    const float k2 = __fmul_rn(m.k, m.k);
    uint32_t acc = 0, rej = 0, wal = 0;
    // ---- records, NT at a time; the next window's loads in flight
    int32_t r = r0 + threadIdx.x;
    float z = 0.f, vp = 1.f;
    uint32_t c = 0;
    if (r < r1) { z = __ldg(b.rz + r); vp = __ldg(b.rv + r); c = __ldg(b.rc + r); }
    for (int32_t base = r0; base < r1; base += NT) {
      const bool live = r < r1;
      const int32_t rn = r + NT;
      float zn = 0.f, vpn = 1.f;
      uint32_t cn = 0;
      if (rn < r1) { zn = __ldg(b.rz + rn); vpn = __ldg(b.rv + rn); cn = __ldg(b.rc + rn); }
      Fix fw{0, 0u}, ft{0, 0u};
      uint8_t st = kPtFused;
      if (live) {
        const float h = S.h[c], ve = S.ve[c];
        const bool valid = isfinite(ve);
        if (wall_on && valid && (int32_t)S.cnt[c] > m.wall && z < h) {
          st = kPtWall;
        } else if (valid && m.k > 0.f && __fmul_rn(__fsub_rn(z, h), __fsub_rn(z, h)) > __fmul_rn(k2, __fadd_rn(ve, vp))) {
          // |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k  <=>  (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2)  (k > 0)
          st = kPtRejected;
        } else {
          const float wgt = __frcp_rn(vp);
          fw = to_fix(wgt);
          ft = to_fix(__fmul_rn(wgt, __fsub_rn(z, valid ? h : m.z_ref)));
        }
        acc += st == kPtFused;
        rej += st == kPtRejected;
        wal += st == kPtWall;
        if (b.tr_status) b.tr_status[b.idx_sorted[r]] = st;
      }
      unsigned long long nn = !live ? 0ull : st == kPtFused ? 1ull : st == kPtRejected ? (1ull << 32) : 0ull;
      // runs of equal cells in consecutive lanes: a segmented inclusive scan, as
      // many steps as the longest run needs; the run's last lane adds its sums
      const unsigned long long tag = live ? (unsigned long long)c : ~0ull;
      int head, len;
      key_runs(tag, head, len);
      // the run's last lane (every lane takes part in the shuffle)
      const unsigned long long next = __shfl_down_sync(kFull, tag, 1);
      const bool tail = lane == 31 || next != tag;
      const int maxrun = (int)__reduce_max_sync(kFull, live ? (unsigned)(lane - head + 1) : 1u);
      long long wh = fw.h, th = ft.h;
      unsigned long long wl = fw.l, tl = ft.l;
      for (int o = 1; o < maxrun; o <<= 1) {
        const long long awh = __shfl_up_sync(kFull, wh, o), ath = __shfl_up_sync(kFull, th, o);
        const unsigned long long awl = __shfl_up_sync(kFull, wl, o), atl = __shfl_up_sync(kFull, tl, o);
        const unsigned long long an = __shfl_up_sync(kFull, nn, o);
        if (lane - o >= head) {
          wh += awh;
          th += ath;
          wl += awl;
          tl += atl;
          nn += an;
        }
      }
      if (live && tail) {
        if (nn) atomicAdd(&S.n[c], nn);
        if (wh | (long long)wl) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&S.wh[c]), (unsigned long long)wh);
          atomicAdd(&S.wl[c], wl);
          atomicAdd(reinterpret_cast<unsigned long long*>(&S.th[c]), (unsigned long long)th);
          atomicAdd(&S.tl[c], tl);
        }
      }
      r = rn;
      z = zn;
      vp = vpn;
      c = cn;
    }
    __syncthreads();
    // ---- every touched cell of the tile, once
    uint32_t cells = 0;
    for (int cc = threadIdx.x; cc < ncell; cc += NT) {
      const unsigned long long nn = S.n[cc];
      if (!nn) continue;
      CellCtx cx;
      cx.h = S.h[cc];
      cx.ve = S.ve[cc];
      cx.valid = isfinite(cx.ve);
      cx.href = cx.valid ? cx.h : m.z_ref;
      cells += write_cell(m, p0 + cc, cx, fix128(S.wh[cc], S.wl[cc]), fix128(S.th[cc], S.tl[cc]),
                          (int)(uint32_t)nn, (int)(nn >> 32));
    }
    // ---- the tile's statistics: one atomic per counter
    const uint32_t v[4] = {acc, rej, wal, cells};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = __reduce_add_sync(kFull, v[k]);
      if (lane == 0 && x) atomicAdd(&S.stat[k], (unsigned long long)x);
    }
    __syncthreads();
    if (threadIdx.x < 4 && S.stat[threadIdx.x]) {
      const int idx[4] = {kStAccepted, kStRejected, kStWall, kStCellsUpdated};
      atomicAdd(&m.ctl->stats[idx[threadIdx.x]], S.stat[threadIdx.x]);
    }
    __syncthreads();
  }
}

template <int NT>
static cudaError_t launch_fuse_t(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {  // more than the 48 KB of static shared memory
    cudaError_t e = cudaFuncSetAttribute(k_fuse<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TileSmem));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fuse<NT>, NT, sizeof(TileSmem));
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);  // one resident wave
  const int grid = (int)(tiles < cap ? (tiles < 1 ? 1 : tiles) : cap);
  k_fuse<NT><<<grid, NT, sizeof(TileSmem), s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_fuse(const BatchDev* b, int64_t n_cells, int threads, cudaStream_t s) {
  return threads >= 512 ? launch_fuse_t<512>(b, n_cells, s) : launch_fuse_t<256>(b, n_cells, s);
}

}  // namespace em
