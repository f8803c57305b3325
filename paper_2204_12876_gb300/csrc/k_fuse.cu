// k_fuse.cu -- per-cell fusion (Section II-C of the paper).
//
// For every cell that received points in this update, its segment of records
// (z, sigma_p^2) is walked:
//   1. wall rule: in a valid cell with more than wall_num_thresh points, points
//      below the current height are dropped (before the outlier test);
//   2. Mahalanobis gate against the pre-update estimate: reject iff
//      |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k, tested as
//      (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2) (no division or square root);
//      every rejection adds outlier_variance to sigma_m^2;
//   3. Eq. 1 and Eq. 2 for all accepted points at once, in information form:
//        Lambda = 1 / (sigma_m^2 + n_rej v_out) + sum_i 1/sigma_p,i^2
//        h'     = h + sum_i (z_i - h) / sigma_p,i^2 / Lambda,   sigma_m^2' = 1 / Lambda
//      (an empty cell has 1/sigma_m^2 = 0 and uses the smallest z of its
//      segment as the reference height).  Applying Eq. 1/2 point after point
//      gives the same result in exact arithmetic.
//
// The two sums are accumulated exactly: every float32 term is converted to a
// signed 128-bit fixed-point integer with 44 fractional bits and the integers
// are added.  Integer addition is associative, so the result is the same for
// every order of the points, bit for bit (no float atomics, no dependence on
// the order records reached their segment or on how lanes split a segment).
//
// Three tiers by segment length, in one launch:
//   large  (> big_thresh records)   one whole block per cell, cells taken from
//                                   a counter (atomicAdd; no block waits);
//   medium (> small_thresh)         a group of G lanes per cell, grid-stride;
//   small  (1 .. small_thresh)      one thread per cell, walking the tiles of
//                                   the cell space (coalesced per-cell loads).
#include "em_point.cuh"

namespace em {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFuseThreads = 256;
constexpr int kFuseWarps = kFuseThreads / 32;

// trunc(a * 2^44) as a signed 128-bit integer, exact for |a| >= 2^-44 (bits
// below 2^-44 are dropped, the same way for every order of summation).  The
// 24-bit significand is placed with 64-bit shifts into the two halves.
__device__ __forceinline__ __int128 to_fixed(float a) {
  const uint32_t u = __float_as_uint(a);
  const int e = (int)((u >> 23) & 0xffu);
  const unsigned long long mant = (u & 0x7fffffu) | 0x800000u;
  int sh = e - 106;          // a = mant * 2^(e - 150); a * 2^44 = mant * 2^(e - 106)
  sh = sh > 100 ? 100 : sh;  // |a| >= 2^78: saturate (never reached by bounded inputs)
  unsigned long long lo, hi;
  if (e == 0 || sh <= -32) {
    lo = 0; hi = 0;
  } else if (sh < 0) {
    lo = mant >> (-sh); hi = 0;
  } else if (sh <= 40) {
    lo = mant << sh; hi = 0;
  } else if (sh < 64) {
    lo = mant << sh; hi = mant >> (64 - sh);
  } else {
    lo = 0; hi = mant << (sh - 64);
  }
  const __int128 r = (__int128)(((unsigned __int128)hi << 64) | lo);
  return (u >> 31) ? -r : r;
}

// s * 2^-44 rounded to the nearest float (ties to even), in integer arithmetic
// (this part's FP64 rate is a small fraction of its integer rate).  Every
// nonzero |s| < 2^127 gives a normal float: 2^-44 <= |s| 2^-44 < 2^83.
__device__ __forceinline__ float from_fixed(__int128 s) {
  if (s == 0) return 0.f;
  const uint32_t sign = s < 0 ? 0x80000000u : 0u;
  const unsigned __int128 a = s < 0 ? (unsigned __int128)(-s) : (unsigned __int128)s;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading one
  uint32_t mant;
  int e = msb;
  if (msb <= 23) {
    mant = (uint32_t)(lo << (23 - msb));  // exact
  } else {
    const int sh = msb - 23;
    mant = (uint32_t)(a >> sh);  // 24 bits, leading one at bit 23
    const unsigned __int128 rem = a & ((((unsigned __int128)1) << sh) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1u))) {
      if (++mant == (1u << 24)) {
        mant >>= 1;
        ++e;
      }
    }
  }
  // value = mant 2^(e - 23) 2^-44: biased exponent e - 44 + 127
  return __uint_as_float(sign | ((uint32_t)(e + 83) << 23) | (mant & 0x7fffffu));
}

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
  const unsigned long long lo = (unsigned long long)v;
  const unsigned long long hi = (unsigned long long)((unsigned __int128)v >> 64);
  const unsigned long long lo2 = __shfl_xor_sync(kFull, lo, o);
  const unsigned long long hi2 = __shfl_xor_sync(kFull, hi, o);
  return (__int128)(((unsigned __int128)hi2 << 64) | lo2);
}

// partial sums of one lane over a segment
struct Acc {
  __int128 qw, qt;
  int acc, rej, wal;
};

template <int G>
__device__ __forceinline__ void group_reduce(Acc& a) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    a.qw += shfl_xor_i128(a.qw, o);
    a.qt += shfl_xor_i128(a.qt, o);
    a.acc += __shfl_xor_sync(kFull, a.acc, o);
    a.rej += __shfl_xor_sync(kFull, a.rej, o);
    a.wal += __shfl_xor_sync(kFull, a.wal, o);
  }
}

template <int G>
__device__ __forceinline__ float group_min(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// The cell's snapshot and the decisions that do not depend on single points.
struct CellCtx {
  int32_t cell, base, len;
  float h, ve, k2;
  bool valid, wall_on, gate_on;
};

__device__ __forceinline__ CellCtx load_cell(const MapDev& m, int32_t cell, int32_t base, int32_t len) {
  CellCtx c;
  c.cell = cell;
  c.base = base;
  c.len = len;
  c.h = m.h[cell];
  const float var = m.var[cell];
  c.valid = isfinite(var);
  c.ve = c.valid ? var_eff(m, var, m.t_last[cell]) : var;
  c.wall_on = m.wall > 0 && c.valid && len > m.wall;
  c.gate_on = c.valid && m.k > 0.f;
  c.k2 = __fmul_rn(m.k, m.k);
  return c;
}

// Records i0, i0 + stride, ... of the cell's segment into this lane's partials.
__device__ __forceinline__ void fuse_records(const BatchDev& b, const MapDev& m, const CellCtx& c, float href,
                                             int i0, int stride, Acc& a) {
  const float2* __restrict__ rec = b.zw_sorted + c.base;
  for (int i = i0; i < c.len; i += stride) {
    const float2 r = rec[i];
    const float z = r.x, vp = r.y;
    uint8_t st = kPtFused;
    if (c.wall_on && z < c.h) {
      st = kPtWall;
    } else if (c.gate_on) {
      // |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k  <=>  (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2)  (k > 0)
      const float dz = __fsub_rn(z, c.h);
      if (__fmul_rn(dz, dz) > __fmul_rn(c.k2, __fadd_rn(c.ve, vp))) st = kPtRejected;
    }
    if (st == kPtFused) {
      const float w = __frcp_rn(vp);
      a.qw += to_fixed(w);
      a.qt += to_fixed(__fmul_rn(w, __fsub_rn(z, href)));
      ++a.acc;
    } else if (st == kPtRejected) {
      ++a.rej;
    } else {
      ++a.wal;
    }
    if (b.tr_status) b.tr_status[b.idx_sorted[c.base + i]] = st;
  }
}

// New state of the cell from the reduced sums (one thread).
__device__ __forceinline__ bool write_cell(const MapDev& m, const CellCtx& c, float href, const Acc& a) {
  if (a.acc + a.rej == 0) return false;
  float h_new, var_new;
  const float sw = from_fixed(a.qw);
  const float st = from_fixed(a.qt);
  if (c.valid) {
    const float vprior = __fadd_rn(c.ve, __fmul_rn((float)a.rej, m.v_out));
    if (a.acc == 0) {
      h_new = c.h;
      var_new = vprior;
    } else {
      const float lam = __fadd_rn(__frcp_rn(vprior), sw);
      h_new = __fadd_rn(c.h, __fdiv_rn(st, lam));
      var_new = __frcp_rn(lam);
    }
  } else {
    h_new = __fadd_rn(href, __fdiv_rn(st, sw));
    var_new = __frcp_rn(sw);
  }
  m.h[c.cell] = h_new;
  m.var[c.cell] = var_new;
  m.t_last[c.cell] = m.t_now;
  return true;
}

__device__ __forceinline__ void count_cell(const BatchDev& b, MapCounters& mc, int map, const Acc& a, bool upd) {
  const int idx[4] = {kStAccepted, kStRejected, kStWall, kStCellsUpdated};
  unsigned long long inc[4] = {(unsigned long long)a.acc, (unsigned long long)a.rej, (unsigned long long)a.wal,
                               upd ? 1ull : 0ull};
  add_counter(b, mc, map, idx, 4, inc);
}

template <int G>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse(const BatchDev* __restrict__ bp) {
  __shared__ int s_slot;
  __shared__ float s_min[kFuseWarps];
  __shared__ __int128 s_q[2][kFuseWarps];
  __shared__ int s_n[3][kFuseWarps];
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  MapCounters mc;

  // ---- large cells: one block each, taken from a counter
  const int n_big = min(b.ctl->n_big, b.big_cap);
  if (n_big > 0) {
    for (;;) {
      if (threadIdx.x == 0) s_slot = atomicAdd(&b.ctl->big_next, 1);
      __syncthreads();
      const int jb = s_slot;
      __syncthreads();
      if (jb >= n_big) break;
      const int2 e = b.big_list[jb];
      const MapDev& m = b.maps[e.x];
      const CellCtx c = load_cell(m, e.y, m.cell_base[e.y], m.cell_len[e.y]);
      float href = c.h;
      if (!c.valid) {
        float zmin = __int_as_float(0x7f800000);
        for (int i = threadIdx.x; i < c.len; i += kFuseThreads) zmin = fminf(zmin, b.zw_sorted[c.base + i].x);
        zmin = group_min<32>(zmin);
        if (lane == 0) s_min[warp] = zmin;
        __syncthreads();
        zmin = s_min[0];
        for (int w = 1; w < kFuseWarps; ++w) zmin = fminf(zmin, s_min[w]);
        href = zmin;
      }
      Acc a{0, 0, 0, 0, 0};
      fuse_records(b, m, c, href, threadIdx.x, kFuseThreads, a);
      group_reduce<32>(a);
      if (lane == 0) {
        s_q[0][warp] = a.qw;
        s_q[1][warp] = a.qt;
        s_n[0][warp] = a.acc;
        s_n[1][warp] = a.rej;
        s_n[2][warp] = a.wal;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        Acc t{0, 0, 0, 0, 0};
        for (int w = 0; w < kFuseWarps; ++w) {
          t.qw += s_q[0][w];
          t.qt += s_q[1][w];
          t.acc += s_n[0][w];
          t.rej += s_n[1][w];
          t.wal += s_n[2][w];
        }
        const bool upd = write_cell(m, c, href, t);
        count_cell(b, mc, e.x, t, upd);
      }
      __syncthreads();
    }
  }

  // ---- medium cells: groups of G lanes, grid-stride over the list
  constexpr int kGroupsPerWarp = 32 / G;
  const int n_med = min(b.ctl->n_med, b.med_cap);
  const int gl = lane % G, gw = lane / G;
  const int warp_global = blockIdx.x * kFuseWarps + warp;
  const int warp_stride = gridDim.x * kFuseWarps;
  for (int jb = warp_global * kGroupsPerWarp; jb < n_med; jb += warp_stride * kGroupsPerWarp) {
    const int j = jb + gw;
    const bool has = j < n_med;
    int2 e = make_int2(0, 0);
    CellCtx c;
    if (has) {
      e = b.med_list[j];
      const MapDev& m = b.maps[e.x];
      c = load_cell(m, e.y, m.cell_base[e.y], m.cell_len[e.y]);
    } else {
      c.len = 0;
      c.valid = true;
      c.h = 0.f;
    }
    const MapDev& m = b.maps[e.x];
    float zmin = __int_as_float(0x7f800000);
    if (!c.valid)
      for (int i = gl; i < c.len; i += G) zmin = fminf(zmin, b.zw_sorted[c.base + i].x);
    zmin = group_min<G>(zmin);
    const float href = c.valid ? c.h : zmin;
    Acc a{0, 0, 0, 0, 0};
    if (has) fuse_records(b, m, c, href, gl, G, a);
    group_reduce<G>(a);
    if (has && gl == 0) {
      const bool upd = write_cell(m, c, href, a);
      count_cell(b, mc, e.x, a, upd);
    }
  }

  // ---- small cells: one thread per cell over the tiles of the cell space
  for_each_tile(b, [&](const MapDev& m, int mi, int32_t p0, int32_t count) {
    for (int32_t i = threadIdx.x; i < count; i += kFuseThreads) {
      const int32_t p = p0 + i;
      const int32_t len = m.cell_len[p];
      if (len < 1 || len > b.small_thresh) continue;
      const CellCtx c = load_cell(m, p, m.cell_base[p], len);
      float href = c.h;
      if (!c.valid) {
        href = __int_as_float(0x7f800000);
        for (int k = 0; k < len; ++k) href = fminf(href, b.zw_sorted[c.base + k].x);
      }
      Acc a{0, 0, 0, 0, 0};
      fuse_records(b, m, c, href, 0, 1, a);
      const bool upd = write_cell(m, c, href, a);
      count_cell(b, mc, mi, a, upd);
    }
  });

  const int idx[4] = {kStAccepted, kStRejected, kStWall, kStCellsUpdated};
  if (mc.map >= 0) {  // fold nothing new; flush per block
    unsigned long long zero[4] = {0, 0, 0, 0};
    add_counter(b, mc, mc.map, idx, 4, zero);
  }
  flush_counters(b, mc, idx, 4);
}

cudaError_t launch_fuse(const BatchDev* b, int64_t n_cells, int64_t n_points, int group, cudaStream_t s) {
  const int g = (group == 4 || group == 8 || group == 16 || group == 32) ? group : 8;
  const int64_t tiles = n_cells / kTile;
  int64_t want = tiles > 1 ? tiles : 1;
  const int64_t med_blocks = (n_points / (kMinSmall + 1)) / (kFuseThreads / g) + 1;
  if (med_blocks > want) want = med_blocks;
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(want < cap ? want : cap);
  switch (g) {
    case 4: k_fuse<4><<<grid, kFuseThreads, 0, s>>>(b); break;
    case 16: k_fuse<16><<<grid, kFuseThreads, 0, s>>>(b); break;
    case 32: k_fuse<32><<<grid, kFuseThreads, 0, s>>>(b); break;
    default: k_fuse<8><<<grid, kFuseThreads, 0, s>>>(b); break;
  }
  return cudaGetLastError();
}

}  // namespace em
