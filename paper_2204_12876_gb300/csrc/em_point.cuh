// em_point.cuh -- per-point arithmetic shared by the binning and ray kernels.
//
// Both kernels must find the same cell for a point (the ray march skips the
// point's own cell), so the arithmetic is written with explicit rounding
// intrinsics: no contraction choice of the compiler can make the two differ.
#pragma once

#include "em_internal.cuh"

namespace em {

constexpr unsigned kFull = 0xffffffffu;  // all lanes of a warp

struct PointGeom {
  float vx, vy, vz;  // R * p_s: sensor-to-point vector in the map frame
  float x, y, z;     // p_m = R * p_s + t
  float d;           // |p_s|, distance from the sensor (Section II-C noise model)
  int32_t ix, iy;    // logical cell indices (unbounded, clamped to +-1e9)
  bool finite;
  bool in_range;
};

// Transform by the sensor pose (Section II-A), distance, cell indices
// ix = floor((x - x0) / r) of the robot-centric grid (as (x - x0) * (1/r)).
// kExt: kernels built for batches that use the exclusion area or the upper-bound
// layer; the others carry none of that code (every kernel of one update is
// launched with the same kExt, so they all agree on which points are valid).
template <bool kExt>
__device__ __forceinline__ PointGeom point_geom(const MapDev& m, const CloudDev& c, float px, float py,
                                                float pz) {
  PointGeom g;
  g.finite = isfinite(px) && isfinite(py) && isfinite(pz);
  float d2 = __fmaf_rn(px, px, __fmaf_rn(py, py, __fmul_rn(pz, pz)));
  g.d = __fsqrt_rn(d2);
  g.in_range = g.finite && g.d >= m.min_range && g.d <= m.max_range;
  g.vx = __fmaf_rn(c.R[0], px, __fmaf_rn(c.R[1], py, __fmul_rn(c.R[2], pz)));
  g.vy = __fmaf_rn(c.R[3], px, __fmaf_rn(c.R[4], py, __fmul_rn(c.R[5], pz)));
  g.vz = __fmaf_rn(c.R[6], px, __fmaf_rn(c.R[7], py, __fmul_rn(c.R[8], pz)));
  g.x = __fadd_rn(g.vx, c.t[0]);
  g.y = __fadd_rn(g.vy, c.t[1]);
  g.z = __fadd_rn(g.vz, c.t[2]);
  g.ix = clamp_floor(__fmul_rn(__fsub_rn(g.x, m.x0), m.inv_res));
  g.iy = clamp_floor(__fmul_rn(__fsub_rn(g.y, m.y0), m.inv_res));
  // exclusion area (Section II-C): a point above the ramp over its horizontal
  // distance r from the sensor is ignored (counted as out of range)
  if (kExt && g.in_range && m.excl_d > 0.f) {
    const float r = __fsqrt_rn(__fmaf_rn(g.vx, g.vx, __fmul_rn(g.vy, g.vy)));
    float lim = r <= m.excl_c ? m.excl_b : __fmaf_rn(__fsub_rn(r, m.excl_c), m.excl_tan, m.excl_b);
    lim = fminf(lim, m.excl_d);
    if (g.vz > lim) g.in_range = false;
  }
  return g;
}

// sigma_p^2 = max((a0 + a1 d + a2 d^2)^2, var_min)  (Section II-C noise model)
__device__ __forceinline__ float point_variance(const MapDev& m, float d) {
  float s = __fmaf_rn(__fmaf_rn(m.a2, d, m.a1), d, m.a0);
  return fmaxf(__fmul_rn(s, s), m.var_min);
}

__device__ __forceinline__ bool in_map(const MapDev& m, int32_t ix, int32_t iy) {
  return ix >= 0 && iy >= 0 && ix < m.W && iy < m.H;
}

// ---- exact fixed-point sums (fusion, drift compensation): order-independent

// trunc(|a| 2^44) with the sign of a -- the fixed-point value of a float32 term
// (44 fractional bits; bits below 2^-44 are dropped, the same way for every
// order of summation) -- split as h 2^27 + l with 0 <= l < 2^27.  Exact for
// |a| < 2^46: |a| 2^17 = F + r with F = trunc, r in [0, 1) exact (Sterbenz),
// and r 2^27 is exact; a negative value borrows one from h so l stays >= 0.
// Straight-line float and conversion instructions, no 128-bit shifts.
struct Fix {
  long long h;
  uint32_t l;
};
__device__ __forceinline__ Fix to_fix(float a) {
  const float A = __fmul_rn(fabsf(a), 131072.0f);  // |a| 2^17
  const float F = truncf(A);
  long long h = (long long)F;
  uint32_t l = (uint32_t)__fmul_rn(__fsub_rn(A, F), 134217728.0f);  // r 2^27
  if (a < 0.f) {
    h = l ? -h - 1 : -h;
    l = l ? (1u << 27) - l : 0u;
  }
  return Fix{h, l};
}

// h 2^27 + l as a 128-bit integer (l may be a sum of many 27-bit parts)
__device__ __forceinline__ __int128 fix128(long long h, unsigned long long l) {
  return (__int128)h * 134217728 + (__int128)l;
}

// t 2^-44 as a float, from its magnitude split into 32-bit pieces (all
// non-negative, so no cancellation): within 2 ulp of the exact value and a
// fixed function of t, so equal sums give equal floats.
__device__ __forceinline__ float fixed_to_float(__int128 t) {
  const bool neg = t < 0;
  const unsigned __int128 m = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
  const unsigned long long top = (unsigned long long)(m >> 64), mid = (unsigned long long)m;
  float v;
  if (top == 0) {  // |value| < 2^20
    v = __fmaf_rn((float)(uint32_t)(mid >> 32), 2.44140625e-4f,                  // 2^32 2^-44
                  __fmul_rn((float)(uint32_t)mid, 5.684341886080801486968994140625e-14f));  // 2^-44
  } else {
    v = __fmaf_rn((float)(uint32_t)(top >> 32), 4503599627370496.0f,             // 2^96 2^-44
                  __fmaf_rn((float)(uint32_t)top, 1048576.0f,                    // 2^64 2^-44
                            __fmul_rn((float)(uint32_t)(mid >> 32), 2.44140625e-4f)));
  }
  return neg ? -v : v;
}

// Per-thread statistics counters of one map.  They are flushed with one atomic
// per block and counter when the whole block saw a single map (the usual
// case), else per thread: many threads adding to one address serialise on a
// single L2 slice.
struct MapCounters {
  int map = -1;
  unsigned long long v[4] = {0, 0, 0, 0};
};

// shared memory of flush_counters (the caller's)
struct FlushSmem {
  int map;
  unsigned long long sum[4];
};

__device__ __forceinline__ void flush_counters(const BatchDev& b, MapCounters& mc, const int* idx, int n,
                                               FlushSmem& fs) {
  if (threadIdx.x == 0) fs.map = mc.map;
  if (threadIdx.x < 4) fs.sum[threadIdx.x] = 0;
  __syncthreads();
  const bool uniform = __syncthreads_and(mc.map == fs.map || mc.map < 0);
  if (uniform) {
    for (int k = 0; k < n; ++k) {
      unsigned long long v = mc.v[k];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(&fs.sum[k], v);
    }
    __syncthreads();
    if ((int)threadIdx.x < n && fs.map >= 0 && fs.sum[threadIdx.x])
      atomicAdd(&b.maps[fs.map].ctl->stats[idx[threadIdx.x]], fs.sum[threadIdx.x]);
    __syncthreads();  // the shared sums are free again
  } else if (mc.map >= 0) {
    for (int k = 0; k < n; ++k)
      if (mc.v[k]) atomicAdd(&b.maps[mc.map].ctl->stats[idx[k]], mc.v[k]);
  }
}

__device__ __forceinline__ void add_counter(const BatchDev& b, MapCounters& mc, int map, const int* idx, int n,
                                            const unsigned long long* inc) {
  if (map != mc.map) {
    if (mc.map >= 0)
      for (int k = 0; k < n; ++k)
        if (mc.v[k]) atomicAdd(&b.maps[mc.map].ctl->stats[idx[k]], mc.v[k]);
    mc.map = map;
    for (int k = 0; k < n; ++k) mc.v[k] = 0;
  }
  for (int k = 0; k < n; ++k) mc.v[k] += inc[k];
}

// Runs of equal keys in consecutive lanes (sensor order puts neighbouring
// points in the same cell): head = first lane of this lane's run, len = run
// length (meaningful on the head lane).  All 32 lanes must call it.
__device__ __forceinline__ void key_runs(unsigned long long tag, int& head, int& len) {
  const int lane = threadIdx.x & 31;
  const unsigned long long prev = __shfl_up_sync(0xffffffffu, tag, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != tag);
  const unsigned le = lane == 31 ? 0xffffffffu : ((1u << (lane + 1)) - 1u);
  head = 31 - __clz(heads & le);
  const unsigned above = heads & ~le;
  len = (above ? __ffs(above) - 1 : 32) - lane;
}

// Load point g of cloud c (stride 3 or 4) with scalar loads.
__device__ __forceinline__ void load_point(const CloudDev& c, int64_t i, float& px, float& py, float& pz) {
  const float* p = c.pts + i * c.stride;
  px = __ldg(p);
  py = __ldg(p + 1);
  pz = __ldg(p + 2);
}

// Load the warp's 32 points [wbase, wbase + 32).  When the whole chunk sits in
// one cloud with 16-byte aligned rows the warp reads it with float4 loads:
// stride 4 -> one float4 per lane; stride 3 -> 24 float4 staged in shared memory.
// `hint` is the cloud of the warp's previous chunk (-1: none); it becomes the
// cloud of this chunk's first point.
__device__ __forceinline__ int load_warp_points(const BatchDev& b, int64_t wbase, int64_t end, float4* stage,
                                                float& px, float& py, float& pz, int& hint) {
  const int lane = threadIdx.x & 31;
  const int64_t g = wbase + lane;
  const int c0 = find_cloud(b.clouds, b.n_clouds, wbase, hint);
  hint = c0;
  const CloudDev& cl0 = b.clouds[c0];
  const bool whole = (wbase + 32 <= end) && (wbase + 32 <= cl0.begin + cl0.n);
  int ci = c0;
  if (whole) {
    const int64_t i0 = wbase - cl0.begin;
    const float* base = cl0.pts + i0 * cl0.stride;
    if (cl0.stride == 4 && ((reinterpret_cast<uintptr_t>(base) & 15) == 0)) {
      float4 q = __ldg(reinterpret_cast<const float4*>(base) + lane);
      px = q.x; py = q.y; pz = q.z;
      return ci;
    }
    if (cl0.stride == 3 && ((reinterpret_cast<uintptr_t>(base) & 15) == 0)) {
      if (lane < 24) stage[lane] = __ldg(reinterpret_cast<const float4*>(base) + lane);
      __syncwarp();
      const float* sf = reinterpret_cast<const float*>(stage);
      px = sf[lane * 3];
      py = sf[lane * 3 + 1];
      pz = sf[lane * 3 + 2];
      __syncwarp();
      return ci;
    }
  } else if (g < end) {
    ci = find_cloud(b.clouds, b.n_clouds, g, c0);
  }
  if (g < end) {
    load_point(b.clouds[ci], g - b.clouds[ci].begin, px, py, pz);
  } else {
    px = py = pz = __int_as_float(0x7fc00000);
  }
  return ci;
}

}  // namespace em
