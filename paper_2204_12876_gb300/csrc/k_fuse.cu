// k_fuse.cu -- per-cell fusion (Section II-C of the paper).
//
// For every cell that received points in this update, its segment of records
// (z, sigma_p^2) is walked by a group of lanes:
//   1. wall rule: in a valid cell with more than wall_num_thresh points, points
//      below the current height are dropped (before the outlier test);
//   2. Mahalanobis gate against the pre-update estimate: reject iff
//      |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k; every rejection adds
//      outlier_variance to sigma_m^2;
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
// Work split: cells with at most big_thresh records (front of the touched list)
// go to groups of G lanes; larger cells (back of the list) go to whole blocks,
// which take them one at a time from a counter (atomicAdd; no block ever waits
// for another).
#include "em_internal.cuh"

namespace em {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFuseThreads = 256;
constexpr int kFuseWarps = kFuseThreads / 32;

// trunc(a * 2^44) as a signed 128-bit integer, exact for |a| >= 2^-44 (bits
// below 2^-44 are dropped, the same way for every order of summation).
__device__ __forceinline__ __int128 to_fixed(float a) {
  const uint32_t u = __float_as_uint(a);
  const int e = (int)((u >> 23) & 0xffu);
  if (e == 0) return 0;
  const uint32_t mant = (u & 0x7fffffu) | 0x800000u;
  int sh = e - 106;  // a = mant * 2^(e - 150); a * 2^44 = mant * 2^(e - 106)
  unsigned __int128 v;
  if (sh >= 0) {
    if (sh > 100) sh = 100;  // |a| >= 2^78: saturate (never reached by bounded inputs)
    v = (unsigned __int128)mant << sh;
  } else if (sh > -32) {
    v = (unsigned __int128)(mant >> (-sh));
  } else {
    v = 0;
  }
  const __int128 r = (__int128)v;
  return (u >> 31) ? -r : r;
}

// s * 2^-44 rounded to float (through a double of the magnitude).
__device__ __forceinline__ float from_fixed(__int128 s) {
  const bool neg = s < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-s) : (unsigned __int128)s;
  const double hi = (double)(unsigned long long)(a >> 64);
  const double lo = (double)(unsigned long long)a;
  const double v = (hi * 18446744073709551616.0 + lo) * 5.684341886080801486968994140625e-14;  // 2^-44
  const float f = (float)v;
  return neg ? -f : f;
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
  float h, ve;
  bool valid, wall_on, gate_on;
};

__device__ __forceinline__ CellCtx load_cell(const MapDev& m, int slot) {
  CellCtx c;
  c.cell = m.touched[slot];
  c.base = m.seg_base[slot];
  c.len = m.seg_len[slot];
  c.h = m.h[c.cell];
  const float var = m.var[c.cell];
  c.valid = isfinite(var);
  c.ve = c.valid ? var_eff(m, var, m.t_last[c.cell]) : var;
  c.wall_on = m.wall > 0 && c.valid && c.len > m.wall;
  c.gate_on = c.valid && m.k > 0.f;
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
      const float sd = __fsqrt_rn(__fadd_rn(c.ve, vp));
      const float md = __fdiv_rn(fabsf(__fsub_rn(z, c.h)), sd);
      if (md > m.k) st = kPtRejected;
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

template <int G>
__global__ void __launch_bounds__(kFuseThreads) k_fuse(const BatchDev* __restrict__ bp) {
  __shared__ int s_slot;
  __shared__ float s_min[kFuseWarps];
  __shared__ __int128 s_q[2][kFuseWarps];
  __shared__ int s_n[3][kFuseWarps];
  __shared__ unsigned long long s_c[4];
  const BatchDev& b = *bp;
  if ((int)blockIdx.y >= b.n_maps) return;
  const MapDev& m = b.maps[blockIdx.y];
  const int32_t ncell = m.W * m.H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long n_acc = 0, n_rej = 0, n_wall = 0, n_upd = 0;

  // ---- large cells: one block each, taken from a counter
  const int n_big = m.ctl->n_big;
  for (;;) {
    if (threadIdx.x == 0) s_slot = atomicAdd(&m.ctl->big_next, 1);
    __syncthreads();
    const int jb = s_slot;
    __syncthreads();
    if (jb >= n_big) break;
    const CellCtx c = load_cell(m, ncell - 1 - jb);
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
      n_acc += t.acc;
      n_rej += t.rej;
      n_wall += t.wal;
      n_upd += write_cell(m, c, href, t);
    }
    __syncthreads();
  }

  // ---- small cells: groups of G lanes
  constexpr int kGroupsPerWarp = 32 / G;
  const int n_small = m.ctl->n_touched;
  const int gl = lane % G, gw = lane / G;
  const int warp_global = blockIdx.x * kFuseWarps + warp;
  const int warp_stride = gridDim.x * kFuseWarps;
  for (int jb = warp_global * kGroupsPerWarp; jb < n_small; jb += warp_stride * kGroupsPerWarp) {
    const int j = jb + gw;
    const bool has = j < n_small;
    CellCtx c;
    if (has) {
      c = load_cell(m, j);
    } else {
      c.len = 0;
      c.valid = true;
      c.h = 0.f;
    }
    float zmin = __int_as_float(0x7f800000);
    if (!c.valid)
      for (int i = gl; i < c.len; i += G) zmin = fminf(zmin, b.zw_sorted[c.base + i].x);
    zmin = group_min<G>(zmin);
    const float href = c.valid ? c.h : zmin;
    Acc a{0, 0, 0, 0, 0};
    if (has) fuse_records(b, m, c, href, gl, G, a);
    group_reduce<G>(a);
    if (has && gl == 0) {
      n_acc += a.acc;
      n_rej += a.rej;
      n_wall += a.wal;
      n_upd += write_cell(m, c, href, a);
    }
  }

  // ---- block-level counters (the block is map-uniform): one atomic per counter
  if (threadIdx.x < 4) s_c[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long v[4] = {n_acc, n_rej, n_wall, n_upd};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long x = v[k];
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0 && x) atomicAdd(&s_c[k], x);
  }
  __syncthreads();
  if (threadIdx.x < 4 && s_c[threadIdx.x]) {
    const int idx = threadIdx.x == 0 ? kStAccepted : threadIdx.x == 1 ? kStRejected
                  : threadIdx.x == 2 ? kStWall : kStCellsUpdated;
    atomicAdd(&m.ctl->stats[idx], s_c[threadIdx.x]);
  }
}

cudaError_t launch_fuse(const BatchDev* b, int32_t n_maps, int32_t max_cells, int group, cudaStream_t s) {
  const int g = (group == 4 || group == 8 || group == 16 || group == 32) ? group : 8;
  const int per_block = kFuseThreads / g;
  const int want = (max_cells + per_block - 1) / per_block;
  int cap = sm_count() * 8 / (n_maps > 0 ? n_maps : 1);
  if (cap < 4) cap = 4;
  const int gx = want < cap ? want : cap;
  dim3 grid(gx < 1 ? 1 : gx, n_maps);
  switch (g) {
    case 4: k_fuse<4><<<grid, kFuseThreads, 0, s>>>(b); break;
    case 16: k_fuse<16><<<grid, kFuseThreads, 0, s>>>(b); break;
    case 32: k_fuse<32><<<grid, kFuseThreads, 0, s>>>(b); break;
    default: k_fuse<8><<<grid, kFuseThreads, 0, s>>>(b); break;
  }
  return cudaGetLastError();
}

}  // namespace em
