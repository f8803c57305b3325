// k_fuse.cu -- per-cell fusion (Section II-C of the paper).
//
// For every cell that received points in this update, a group of G lanes walks
// the cell's segment of records (z, sigma_p^2):
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
// the order records reached their segment).
#include "em_internal.cuh"

namespace em {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFuseThreads = 256;

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

template <int G>
__device__ __forceinline__ __int128 group_sum(__int128 v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const unsigned long long lo = (unsigned long long)v;
    const unsigned long long hi = (unsigned long long)((unsigned __int128)v >> 64);
    const unsigned long long lo2 = __shfl_xor_sync(kFull, lo, o);
    const unsigned long long hi2 = __shfl_xor_sync(kFull, hi, o);
    v += (__int128)(((unsigned __int128)hi2 << 64) | lo2);
  }
  return v;
}

template <int G>
__device__ __forceinline__ int group_sum(int v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_min(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

template <int G>
__global__ void __launch_bounds__(kFuseThreads) k_fuse(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  if ((int)blockIdx.y >= b.n_maps) return;
  const MapDev& m = b.maps[blockIdx.y];
  const int n_touched = m.ctl->n_touched;
  constexpr int kGroupsPerWarp = 32 / G;
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const int gw = lane / G;
  const int warp_global = blockIdx.x * (kFuseThreads / 32) + (threadIdx.x >> 5);
  const int warp_stride = gridDim.x * (kFuseThreads / 32);
  const float2* __restrict__ rec = b.zw_sorted;
  unsigned long long n_acc = 0, n_rej = 0, n_wall = 0, n_upd = 0;

  for (int jb = warp_global * kGroupsPerWarp; jb < n_touched; jb += warp_stride * kGroupsPerWarp) {
    const int j = jb + gw;
    const bool has = j < n_touched;
    int32_t cell = 0, base = 0, len = 0;
    float h = 0.f, var = __int_as_float(0x7f800000);
    int32_t tl = 0;
    if (has) {
      cell = m.touched[j];
      base = m.seg_base[j];
      len = m.seg_len[j];
      h = m.h[cell];
      var = m.var[cell];
      tl = m.t_last[cell];
    }
    const bool valid = isfinite(var);
    const float ve = valid ? var_eff(m, var, tl) : var;
    // empty cell: the smallest z of the segment is the reference height
    float zmin = __int_as_float(0x7f800000);
    if (!valid)
      for (int i = gl; i < len; i += G) zmin = fminf(zmin, rec[base + i].x);
    zmin = group_min<G>(zmin);
    const float href = valid ? h : zmin;
    const bool wall_on = m.wall > 0 && valid && len > m.wall;
    const bool gate_on = valid && m.k > 0.f;
    __int128 qw = 0, qt = 0;
    int acc = 0, rej = 0, wal = 0;
    for (int i = gl; i < len; i += G) {
      const float2 r = rec[base + i];
      const float z = r.x, vp = r.y;
      uint8_t st = kPtFused;
      if (wall_on && z < h) {
        st = kPtWall;
      } else if (gate_on) {
        const float sd = __fsqrt_rn(__fadd_rn(ve, vp));
        const float md = __fdiv_rn(fabsf(__fsub_rn(z, h)), sd);
        if (md > m.k) st = kPtRejected;
      }
      if (st == kPtFused) {
        const float w = __frcp_rn(vp);
        qw += to_fixed(w);
        qt += to_fixed(__fmul_rn(w, __fsub_rn(z, href)));
        ++acc;
      } else if (st == kPtRejected) {
        ++rej;
      } else {
        ++wal;
      }
      if (b.tr_status) b.tr_status[b.idx_sorted[base + i]] = st;
    }
    qw = group_sum<G>(qw);
    qt = group_sum<G>(qt);
    acc = group_sum<G>(acc);
    rej = group_sum<G>(rej);
    wal = group_sum<G>(wal);
    if (has && gl == 0) {
      n_acc += acc;
      n_rej += rej;
      n_wall += wal;
      if (acc + rej > 0) {
        float h_new, var_new;
        const float sw = from_fixed(qw);
        const float st = from_fixed(qt);
        if (valid) {
          const float vprior = __fadd_rn(ve, __fmul_rn((float)rej, m.v_out));
          if (acc == 0) {
            h_new = h;
            var_new = vprior;
          } else {
            const float lam = __fadd_rn(__frcp_rn(vprior), sw);
            h_new = __fadd_rn(h, __fdiv_rn(st, lam));
            var_new = __frcp_rn(lam);
          }
        } else {
          h_new = __fadd_rn(href, __fdiv_rn(st, sw));
          var_new = __frcp_rn(sw);
        }
        m.h[cell] = h_new;
        m.var[cell] = var_new;
        m.t_last[cell] = m.t_now;
        ++n_upd;
      }
    }
  }
  // block-level counters (the block is map-uniform): one atomic per counter
  __shared__ unsigned long long s_c[4];
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
  const int idx[4] = {kStAccepted, kStRejected, kStWall, kStCellsUpdated};
  if (threadIdx.x < 4 && s_c[threadIdx.x]) atomicAdd(&m.ctl->stats[idx[threadIdx.x]], s_c[threadIdx.x]);
}

cudaError_t launch_fuse(const BatchDev* b, int32_t n_maps, int32_t max_cells, int group, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_block = kFuseThreads / (group > 0 ? group : 8);
  int want = (max_cells + per_block - 1) / per_block;
  int cap = sms * 8 / (n_maps > 0 ? n_maps : 1);
  if (cap < 4) cap = 4;
  int gx = want < cap ? want : cap;
  dim3 grid(gx < 1 ? 1 : gx, n_maps);
  switch (group) {
    case 4: k_fuse<4><<<grid, kFuseThreads, 0, s>>>(b); break;
    case 16: k_fuse<16><<<grid, kFuseThreads, 0, s>>>(b); break;
    case 32: k_fuse<32><<<grid, kFuseThreads, 0, s>>>(b); break;
    default: k_fuse<8><<<grid, kFuseThreads, 0, s>>>(b); break;
  }
  return cudaGetLastError();
}

}  // namespace em
