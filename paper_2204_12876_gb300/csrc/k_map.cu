// k_map.cu -- per-cell passes over whole maps.
//
//   k_normals  least-squares plane over the valid cells of the 3x3
//              neighbourhood (Section II-A, "normal calculation")
//   k_smooth   5x5 box mean over valid cells (Section II-I smoothing filter)
//   k_inpaint  minimum in-painting of small enclosed holes (Section II-I)
//   k_shift    empties the cells a map shift brings into view
//   k_layers_* logical <-> physical (ring) copies for em_get/set_layers
//
// All stencils work on logical coordinates: a neighbour outside [0, W) x
// [0, H) does not exist (the ring never wraps a stencil).
#include <math.h>

#include <algorithm>

#include "em.h"
#include "em_point.cuh"

namespace em {

constexpr int kMapThreads = 256;

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }
__device__ __forceinline__ float pinf() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ bool valid_at(const MapDev& m, int32_t p) { return isfinite(m.var[p]); }

__global__ void __launch_bounds__(kMapThreads) k_normals(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  for_each_tile(b, [&](const MapDev& m, int, int32_t p0, int32_t count) {
  if (!m.nx || !(m.flags & EM_F_NORMALS)) return;  // a batch may mix maps with and without normals
  for (int32_t i = threadIdx.x; i < count; i += kMapThreads) {
    const int32_t p = p0 + i;
    int32_t lx, ly;
    logical_of(m, p, lx, ly);
    float rx = qnan(), ry = qnan(), rz = qnan();
    if (valid_at(m, p)) {
      const float hc = m.h[p];
      int n = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
      float sh = 0.f, sih = 0.f, sjh = 0.f;
      for (int dy = -1; dy <= 1; ++dy) {
        const int32_t jy = ly + dy;
        if (jy < 0 || jy >= m.H) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int32_t jx = lx + dx;
          if (jx < 0 || jx >= m.W) continue;
          const int32_t q = phys_index(m, jx, jy);
          if (!valid_at(m, q)) continue;
          const float dh = m.h[q] - hc;
          ++n; si += dx; sj += dy; sii += dx * dx; sjj += dy * dy; sij += dx * dy;
          sh += dh; sih += dx * dh; sjh += dy * dh;
        }
      }
      // centred normal equations scaled by n (exact integers on the left)
      const int cxx = n * sii - si * si, cyy = n * sjj - sj * sj, cxy = n * sij - si * sj;
      const int det = cxx * cyy - cxy * cxy;  // 0 iff the valid cells are collinear
      if (n >= 3 && det != 0) {
        const float cxh = n * sih - si * sh, cyh = n * sjh - sj * sh;
        const float a = ((float)cyy * cxh - (float)cxy * cyh) / ((float)det * m.res);
        const float bb = ((float)cxx * cyh - (float)cxy * cxh) / ((float)det * m.res);
        const float inv = rsqrtf(a * a + bb * bb + 1.f);
        rx = -a * inv;
        ry = -bb * inv;
        rz = inv;
      }
    }
    m.nx[p] = rx;
    m.ny[p] = ry;
    m.nz[p] = rz;
  }
  });
}

// 5x5 smoothing of valid cells over the valid cells of the window (Section
// II-I): the box mean (EM_F_SMOOTH), the lower median (EM_F_MEDIAN: the value of
// rank floor((n - 1) / 2) of the n valid heights, found by counting ranks in
// registers) or a Gaussian with sigma = 1 cell renormalised over the valid
// cells (EM_F_GAUSS).  Sums run in a fixed window order.
__global__ void __launch_bounds__(kMapThreads) k_smooth(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  for_each_tile(b, [&](const MapDev& m, int, int32_t p0, int32_t count) {
  if (!m.smooth) return;
  const int mode = (m.flags & EM_F_MEDIAN) ? 1 : (m.flags & EM_F_GAUSS) ? 2 : 0;
  for (int32_t i = threadIdx.x; i < count; i += kMapThreads) {
    const int32_t p = p0 + i;
    int32_t lx, ly;
    logical_of(m, p, lx, ly);
    float out = qnan();
    if (valid_at(m, p)) {
      float v[25];  // the window's heights, +inf where not valid
      int n = 0;
#pragma unroll
      for (int dy = -2; dy <= 2; ++dy) {
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
          const int32_t jx = lx + dx, jy = ly + dy;
          float h = pinf();
          if (jx >= 0 && jx < m.W && jy >= 0 && jy < m.H) {
            const int32_t q = phys_index(m, jx, jy);
            if (valid_at(m, q)) {
              h = m.h[q];
              ++n;
            }
          }
          v[(dy + 2) * 5 + dx + 2] = h;
        }
      }
      if (mode == 0) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 25; ++k)
          if (v[k] != pinf()) s += v[k];
        out = s / (float)n;
      } else if (mode == 1) {
        // rank of v[k] = #{j : v[j] < v[k]} + #{j < k : v[j] == v[k]}; the invalid
        // (+inf) entries rank last, so rank (n - 1) / 2 is the lower median
        const int want = (n - 1) / 2;
#pragma unroll
        for (int k = 0; k < 25; ++k) {
          int rank = 0;
#pragma unroll
          for (int j = 0; j < 25; ++j) rank += (v[j] < v[k]) || (j < k && v[j] == v[k]);
          if (rank == want) out = v[k];
        }
      } else {
        float s = 0.f, ws = 0.f;
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy) {
#pragma unroll
          for (int dx = -2; dx <= 2; ++dx) {
            const float h = v[(dy + 2) * 5 + dx + 2];
            if (h == pinf()) continue;
            const float w = expf(-0.5f * (float)(dx * dx + dy * dy));
            s = __fmaf_rn(w, h, s);
            ws += w;
          }
        }
        out = __fdiv_rn(s, ws);
      }
    }
    m.smooth[p] = out;
  }
  });
}

// Every empty cell explores its 4-connected component of empty cells until
// it has found 9 cells.  A component with at most 8 cells that does not touch the map border
// is a hole: all its cells take the minimum height of the valid cells
// 8-adjacent to the component (each cell of the component computes the same
// value independently, so no labels are needed).
__global__ void __launch_bounds__(kMapThreads) k_inpaint(const BatchDev* __restrict__ bp) {
  const BatchDev& b = *bp;
  for_each_tile(b, [&](const MapDev& m, int, int32_t p0, int32_t count) {
  if (!m.inpaint) return;
  for (int32_t i = threadIdx.x; i < count; i += kMapThreads) {
    const int32_t p = p0 + i;
    int32_t lx, ly;
    logical_of(m, p, lx, ly);
    if (valid_at(m, p)) {
      m.inpaint[p] = m.h[p];
      continue;
    }
    int32_t qx[8], qy[8];
    int n = 1, head = 0;
    qx[0] = lx;
    qy[0] = ly;
    bool hole = true;
    while (head < n && hole) {
      const int32_t x = qx[head], y = qy[head];
      ++head;
      if (x == 0 || y == 0 || x == m.W - 1 || y == m.H - 1) { hole = false; break; }
      const int ddx[4] = {1, -1, 0, 0}, ddy[4] = {0, 0, 1, -1};
      for (int k = 0; k < 4 && hole; ++k) {
        const int32_t jx = x + ddx[k], jy = y + ddy[k];
        if (valid_at(m, phys_index(m, jx, jy))) continue;
        bool seen = false;
        for (int t = 0; t < n; ++t) seen |= (qx[t] == jx && qy[t] == jy);
        if (seen) continue;
        if (n == 8) { hole = false; break; }  // a 9th cell: too large
        qx[n] = jx;
        qy[n] = jy;
        ++n;
      }
    }
    float out = qnan();
    if (hole) {
      float mn = pinf();
      for (int t = 0; t < n; ++t)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int32_t q = phys_index(m, qx[t] + dx, qy[t] + dy);  // in range: holes avoid the border
            if (valid_at(m, q)) mn = fminf(mn, m.h[q]);
          }
      out = mn;
    }
    m.inpaint[p] = out;
  }
  });
}

__device__ __forceinline__ void empty_cell(const MapDev& m, int32_t p) {
  m.h[p] = qnan();
  m.var[p] = pinf();
  m.t_last[p] = 0;
  if (m.nx) { m.nx[p] = qnan(); m.ny[p] = qnan(); m.nz[p] = qnan(); }
  if (m.smooth) m.smooth[p] = qnan();
  if (m.inpaint) m.inpaint[p] = qnan();
  if (m.upper) m.upper[p] = pinf();
}

// exposed logical columns [cx0, cx1) over all rows, and rows [ry0, ry1) over all columns
__global__ void __launch_bounds__(kMapThreads) k_shift(MapDev m, int32_t cx0, int32_t cx1, int32_t ry0, int32_t ry1) {
  const int32_t ncol = (cx1 - cx0) * m.H;
  const int32_t nrow = (ry1 - ry0) * m.W;
  for (int32_t i = blockIdx.x * kMapThreads + threadIdx.x; i < ncol + nrow; i += gridDim.x * kMapThreads) {
    int32_t lx, ly;
    if (i < ncol) { lx = cx0 + i % (cx1 - cx0); ly = i / (cx1 - cx0); }
    else { const int32_t k = i - ncol; lx = k % m.W; ly = ry0 + k / m.W; }
    empty_cell(m, phys_index(m, lx, ly));
  }
}

__global__ void __launch_bounds__(kMapThreads) k_fill(MapDev m) {
  const int32_t ncell = m.W * m.H;
  for (int32_t p = blockIdx.x * kMapThreads + threadIdx.x; p < ncell; p += gridDim.x * kMapThreads) {
    empty_cell(m, p);
    m.cnt[p] = 0;
    m.cell_seg[p] = make_int2(0, 0);
    if ((p & 31) == 0) m.mark[p >> 5] = 0u;
  }
}

// layer bits (see em.h)
enum : uint32_t {
  L_ELEV = 1u << 0, L_VAR = 1u << 1, L_TIME = 1u << 2, L_NX = 1u << 3, L_NY = 1u << 4, L_NZ = 1u << 5,
  L_SMOOTH = 1u << 6, L_INPAINT = 1u << 7, L_VALID = 1u << 8, L_VAR_NOW = 1u << 9, L_UPPER = 1u << 10
};

// The layers of one map in mask (ascending bit order, logical row-major), cells
// c = first, first + stride, ... of the map.
__device__ __forceinline__ void layers_out(const MapDev& m, uint32_t mask, float* __restrict__ dst, int32_t first,
                                           int32_t stride) {
  const int32_t ncell = m.W * m.H;
  for (int32_t c = first; c < ncell; c += stride) {
    const int32_t lx = c % m.W, ly = c / m.W;
    const int32_t p = phys_index(m, lx, ly);
    const bool v = isfinite(m.var[p]);
    int k = 0;
    for (uint32_t bit = 1; bit <= L_UPPER; bit <<= 1) {
      if (!(mask & bit)) continue;
      float x;
      switch (bit) {
        case L_ELEV: x = v ? m.h[p] : qnan(); break;
        case L_VAR: x = v ? m.var[p] : pinf(); break;
        case L_TIME: x = (float)m.t_last[p]; break;
        case L_NX: x = m.nx ? m.nx[p] : qnan(); break;
        case L_NY: x = m.ny ? m.ny[p] : qnan(); break;
        case L_NZ: x = m.nz ? m.nz[p] : qnan(); break;
        case L_SMOOTH: x = m.smooth ? m.smooth[p] : qnan(); break;
        case L_INPAINT: x = m.inpaint ? m.inpaint[p] : qnan(); break;
        case L_VALID: x = v ? 1.f : 0.f; break;
        case L_VAR_NOW: x = v ? var_eff(m, m.var[p], m.t_last[p]) : pinf(); break;
        default: x = m.upper ? m.upper[p] : pinf(); break;
      }
      dst[(size_t)k * ncell + c] = x;
      ++k;
    }
  }
}

__global__ void __launch_bounds__(kMapThreads) k_layers_out(MapDev m, uint32_t mask, float* __restrict__ dst) {
  layers_out(m, mask, dst, blockIdx.x * kMapThreads + threadIdx.x, gridDim.x * kMapThreads);
}

// Many maps at once: blockIdx.y picks the job (the jobs travel as the kernel's
// parameter block, so there is nothing to upload).
__global__ void __launch_bounds__(kMapThreads) k_layers_out_multi(ReadJobs jobs) {
  const ReadJob& j = jobs.job[blockIdx.y];
  layers_out(j.m, j.mask, j.dst, blockIdx.x * kMapThreads + threadIdx.x, gridDim.x * kMapThreads);
}

__global__ void __launch_bounds__(kMapThreads) k_layers_in(MapDev m, uint32_t mask, const float* __restrict__ src) {
  const int32_t ncell = m.W * m.H;
  for (int32_t c = blockIdx.x * kMapThreads + threadIdx.x; c < ncell; c += gridDim.x * kMapThreads) {
    const int32_t lx = c % m.W, ly = c / m.W;
    const int32_t p = phys_index(m, lx, ly);
    int k = 0;
    for (uint32_t bit = 1; bit <= L_UPPER; bit <<= 1) {
      if (!(mask & bit)) continue;
      const float x = src[(size_t)k * ncell + c];
      switch (bit) {
        case L_ELEV: m.h[p] = x; break;
        case L_VAR: m.var[p] = isfinite(x) ? x : pinf(); break;
        case L_TIME: m.t_last[p] = (int32_t)x; break;
        case L_NX: if (m.nx) m.nx[p] = x; break;
        case L_NY: if (m.ny) m.ny[p] = x; break;
        case L_NZ: if (m.nz) m.nz[p] = x; break;
        default: if (m.upper) m.upper[p] = x; break;  // L_UPPER (the only other bit allowed in)
      }
      ++k;
    }
    if (!isfinite(m.var[p])) m.h[p] = qnan();
  }
}

static int cell_grid(int64_t cells) {
  int64_t g = (cells + kMapThreads - 1) / kMapThreads;
  if (g > 2048) g = 2048;
  return g < 1 ? 1 : (int)g;
}

static int tile_grid(int64_t n_cells) {
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * 8;
  return (int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap);
}

cudaError_t launch_normals(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  k_normals<<<tile_grid(n_cells), kMapThreads, 0, s>>>(b);
  return cudaGetLastError();
}
cudaError_t launch_smooth(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  k_smooth<<<tile_grid(n_cells), kMapThreads, 0, s>>>(b);
  return cudaGetLastError();
}
cudaError_t launch_inpaint(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  k_inpaint<<<tile_grid(n_cells), kMapThreads, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_shift_clear(const MapDev& m, int32_t dx, int32_t dy, cudaStream_t s) {
  int32_t cx0 = 0, cx1 = 0, ry0 = 0, ry1 = 0;
  if (dx > 0) { cx0 = m.W - dx; cx1 = m.W; } else if (dx < 0) { cx0 = 0; cx1 = -dx; }
  if (dy > 0) { ry0 = m.H - dy; ry1 = m.H; } else if (dy < 0) { ry0 = 0; ry1 = -dy; }
  const int64_t n = (int64_t)(cx1 - cx0) * m.H + (int64_t)(ry1 - ry0) * m.W;
  if (n == 0) return cudaSuccess;
  k_shift<<<cell_grid(n), kMapThreads, 0, s>>>(m, cx0, cx1, ry0, ry1);
  return cudaGetLastError();
}

cudaError_t launch_fill_map(const MapDev& m, cudaStream_t s) {
  k_fill<<<cell_grid((int64_t)m.W * m.H), kMapThreads, 0, s>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_layers_out(const MapDev& m, uint32_t mask, float* dst, cudaStream_t s) {
  k_layers_out<<<cell_grid((int64_t)m.W * m.H), kMapThreads, 0, s>>>(m, mask, dst);
  return cudaGetLastError();
}

cudaError_t launch_layers_out_multi(const ReadJobs& jobs, cudaStream_t s) {
  if (jobs.n <= 0) return cudaSuccess;
  int64_t most = 1;
  for (int i = 0; i < jobs.n; ++i) most = std::max(most, (int64_t)jobs.job[i].m.W * jobs.job[i].m.H);
  const int gx = std::max(1, std::min(cell_grid(most), 2 * sm_count() * 8 / jobs.n));
  k_layers_out_multi<<<dim3(gx, jobs.n), kMapThreads, 0, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_layers_in(const MapDev& m, uint32_t mask, const float* src, cudaStream_t s) {
  k_layers_in<<<cell_grid((int64_t)m.W * m.H), kMapThreads, 0, s>>>(m, mask, src);
  return cudaGetLastError();
}

}  // namespace em
