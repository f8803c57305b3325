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

// Normals work on logical tiles of kNmT x kNmT cells with the heights of the
// tile and a 1-cell rim staged in shared memory (+inf where empty or outside).
constexpr int kNmT = 32, kNmSpan = kNmT + 2;
static_assert(kNmT * kNmT == 4 * kMapThreads, "k_normals: four cells per thread");

__global__ void __launch_bounds__(kMapThreads) k_normals(const BatchDev* __restrict__ bp) {
  __shared__ float s_h[kNmSpan][kNmSpan + 1];
  const BatchDev& b = *bp;
  for (int mi = 0; mi < b.n_maps; ++mi) {
    const MapDev& m = b.maps[mi];
    if (!m.nx || !(m.flags & EM_F_NORMALS)) continue;  // a batch may mix maps with and without normals
    const int32_t ntx = (m.W + kNmT - 1) / kNmT, nty = (m.H + kNmT - 1) / kNmT;
    for (int32_t tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
      const int32_t x0 = (tile % ntx) * kNmT - 1, y0 = (tile / ntx) * kNmT - 1;  // window origin
      for (int e = threadIdx.x; e < kNmSpan * kNmSpan; e += kMapThreads) {
        const int wi = e % kNmSpan, wj = e / kNmSpan;
        const int32_t x = x0 + wi, y = y0 + wj;
        float h = pinf();
        if (x >= 0 && x < m.W && y >= 0 && y < m.H) {
          const int32_t q = phys_index(m, x, y);
          if (valid_at(m, q)) h = m.h[q];
        }
        s_h[wj][wi] = h;
      }
      __syncthreads();
      for (int k = 0; k < 4; ++k) {
        const int ci = threadIdx.x % kNmT, cj = threadIdx.x / kNmT + k * (kMapThreads / kNmT);
        const int32_t lx = x0 + 1 + ci, ly = y0 + 1 + cj;
        if (lx >= m.W || ly >= m.H) continue;
        float rx = qnan(), ry = qnan(), rz = qnan();
        const float hc = s_h[cj + 1][ci + 1];
        if (hc != pinf()) {  // a valid centre
          int n = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
          float sh = 0.f, sih = 0.f, sjh = 0.f;
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              const float hq = s_h[cj + 1 + dy][ci + 1 + dx];
              if (hq == pinf()) continue;
              const float dh = hq - hc;
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
        const int32_t p = phys_index(m, lx, ly);
        m.nx[p] = rx;
        m.ny[p] = ry;
        m.nz[p] = rz;
      }
      __syncthreads();
    }
  }
}

// 5x5 smoothing of valid cells over the valid cells of the window (Section
// II-I): the box mean (EM_F_SMOOTH), the lower median (EM_F_MEDIAN: the value of
// rank floor((n - 1) / 2) of the n valid heights, found by counting ranks in
// registers) or a Gaussian with sigma = 1 cell renormalised over the valid
// cells (EM_F_GAUSS).  Sums run in a fixed window order.
// Smoothing works on logical tiles of kSmT x kSmT cells: the heights of the
// tile and a 2-cell rim (+inf where empty or outside the map) are staged in
// shared memory once, so the 25 reads of a cell's window hit shared memory.
constexpr int kSmT = 32, kSmRim = 2, kSmSpan = kSmT + 2 * kSmRim;
static_assert(kSmT * kSmT == 4 * kMapThreads, "k_smooth: four cells per thread");

__global__ void __launch_bounds__(kMapThreads) k_smooth(const BatchDev* __restrict__ bp) {
  __shared__ float s_h[kSmSpan][kSmSpan + 1];
  const BatchDev& b = *bp;
  for (int mi = 0; mi < b.n_maps; ++mi) {
    const MapDev& m = b.maps[mi];
    if (!m.smooth) continue;
    const int mode = (m.flags & EM_F_MEDIAN) ? 1 : (m.flags & EM_F_GAUSS) ? 2 : 0;
    const int32_t ntx = (m.W + kSmT - 1) / kSmT, nty = (m.H + kSmT - 1) / kSmT;
    for (int32_t tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
      const int32_t x0 = (tile % ntx) * kSmT - kSmRim, y0 = (tile / ntx) * kSmT - kSmRim;  // window origin
      for (int e = threadIdx.x; e < kSmSpan * kSmSpan; e += kMapThreads) {
        const int wi = e % kSmSpan, wj = e / kSmSpan;
        const int32_t x = x0 + wi, y = y0 + wj;
        float h = pinf();
        if (x >= 0 && x < m.W && y >= 0 && y < m.H) {
          const int32_t q = phys_index(m, x, y);
          if (valid_at(m, q)) h = m.h[q];
        }
        s_h[wj][wi] = h;
      }
      __syncthreads();
      for (int k = 0; k < 4; ++k) {
        const int ci = threadIdx.x % kSmT, cj = threadIdx.x / kSmT + k * (kMapThreads / kSmT);
        const int32_t lx = x0 + kSmRim + ci, ly = y0 + kSmRim + cj;
        if (lx >= m.W || ly >= m.H) continue;
        float out = qnan();
        if (s_h[cj + kSmRim][ci + kSmRim] != pinf()) {  // a valid centre
          float v[25];  // the window's heights, +inf where not valid
          int n = 0;
#pragma unroll
          for (int dy = 0; dy < 5; ++dy)
#pragma unroll
            for (int dx = 0; dx < 5; ++dx) {
              const float h = s_h[cj + dy][ci + dx];
              n += h != pinf();
              v[dy * 5 + dx] = h;
            }
          if (mode == 0) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < 25; ++q)
              if (v[q] != pinf()) s += v[q];
            out = s / (float)n;
          } else if (mode == 1) {
            // rank of v[q] = #{j : v[j] < v[q]} + #{j < q : v[j] == v[q]}; the invalid
            // (+inf) entries rank last, so rank (n - 1) / 2 is the lower median
            const int want = (n - 1) / 2;
#pragma unroll
            for (int q = 0; q < 25; ++q) {
              int rank = 0;
#pragma unroll
              for (int j = 0; j < 25; ++j) rank += (v[j] < v[q]) || (j < q && v[j] == v[q]);
              if (rank == want) out = v[q];
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
        m.smooth[phys_index(m, lx, ly)] = out;
      }
      __syncthreads();
    }
  }
}

// Every empty cell explores its 4-connected component of empty cells until
// it has found 9 cells.  A component with at most 8 cells that does not touch the map border
// is a hole: all its cells take the minimum height of the valid cells
// 8-adjacent to the component (each cell of the component computes the same
// value independently, so no labels are needed).
// In-painting works on logical tiles of kIpT x kIpT cells.  A hole has at most
// 8 cells, so every cell of it lies within 7 cells of any other: the empty
// cells of the tile and a rim of kIpRim cells, one bit each, are all a tile
// needs to find its holes (shared memory, one 64-bit word per row).
constexpr int kIpT = 32, kIpRim = 8, kIpSpan = kIpT + 2 * kIpRim;  // 48 bits of a row word
static_assert(kIpT * kIpT == 4 * kMapThreads, "k_inpaint: four cells per thread");

// Is cell (i, j) of the tile window empty and inside the map?  Bits outside the
// map are clear, so the search never leaves it; a hole may not touch the map
// edge, which is tested on the cells themselves.
__device__ __forceinline__ bool ip_empty(const uint64_t* rows, int i, int j) { return (rows[j] >> i) & 1ull; }

// Empty cells in a run of 9 or more along a row or a column are part of a
// component too large to be a hole (the window holds 8 cells on either side).
__device__ __forceinline__ int run_through(uint64_t word, int bit) {
  const int up = __ffsll((long long)~(word >> bit)) - 1;       // set bits from bit upwards
  const int down = __clzll((long long)~(word << (63 - bit)));  // set bits from bit downwards
  return up + down - 1;
}

// The component of window cell (i, j) (logical (lx, ly)): a hole gets the
// lowest estimate among its 8-neighbours, anything else NaN.  A breadth-first
// search of at most 8 cells, each stored as one byte (dx + 8) | (dy + 8) << 4
// of a 64-bit word.
__device__ float inpaint_cell(const MapDev& m, const uint64_t* rows, int i, int j, int32_t lx, int32_t ly) {
  uint64_t cells = 0x88ull;  // the start cell: dx = dy = 0
  int n = 1, head = 0;
  bool hole = true;
  while (head < n && hole) {
    const uint32_t c = (uint32_t)(cells >> (8 * head)) & 0xffu;
    ++head;
    const int dx = (int)(c & 15u) - 8, dy = (int)(c >> 4) - 8;
    const int32_t x = lx + dx, y = ly + dy;
    if (x == 0 || y == 0 || x == m.W - 1 || y == m.H - 1) { hole = false; break; }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ex = dx + (q == 0) - (q == 1), ey = dy + (q == 2) - (q == 3);
      if (!ip_empty(rows, i + ex, j + ey)) continue;
      // 8 cells from the start needs a path of 9: too large (and not codable)
      if (ex < -7 || ex > 7 || ey < -7 || ey > 7) { hole = false; break; }
      const uint64_t code = (uint64_t)((ex + 8) | ((ey + 8) << 4));
      const uint64_t v = cells ^ (code * 0x0101010101010101ull);  // a zero byte: already found
      if ((v - 0x0101010101010101ull) & ~v & 0x8080808080808080ull) continue;
      if (n == 8) { hole = false; break; }  // a 9th cell: too large
      cells |= code << (8 * n);
      ++n;
    }
  }
  if (!hole) return qnan();
  // lowest estimate among the 8-neighbours (all inside the map: holes avoid the
  // edge, so a cell there that is not empty holds an estimate)
  float mn = pinf();
  for (int t = 0; t < n; ++t) {
    const uint32_t c = (uint32_t)(cells >> (8 * t)) & 0xffu;
    const int32_t x = lx + (int)(c & 15u) - 8, y = ly + (int)(c >> 4) - 8;
    const int wi = i + (int)(c & 15u) - 8, wj = j + (int)(c >> 4) - 8;
#pragma unroll
    for (int ddy = -1; ddy <= 1; ++ddy)
#pragma unroll
      for (int ddx = -1; ddx <= 1; ++ddx)
        if (!ip_empty(rows, wi + ddx, wj + ddy)) mn = fminf(mn, m.h[phys_index(m, x + ddx, y + ddy)]);
  }
  return mn;
}

__global__ void __launch_bounds__(kMapThreads, 4) k_inpaint(const BatchDev* __restrict__ bp) {
  __shared__ uint64_t s_rows[kIpSpan];
  __shared__ uint64_t s_cols[kIpSpan];      // the same bits by column
  __shared__ uint16_t s_queue[kIpT * kIpT];  // tile cells that need the search
  __shared__ int s_queued;
  const BatchDev& b = *bp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int mi = 0; mi < b.n_maps; ++mi) {
    const MapDev& m = b.maps[mi];
    if (!m.inpaint) continue;
    const int32_t ntx = (m.W + kIpT - 1) / kIpT, nty = (m.H + kIpT - 1) / kIpT;
    for (int32_t tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
      const int32_t x0 = (tile % ntx) * kIpT - kIpRim, y0 = (tile / ntx) * kIpT - kIpRim;  // window origin
      if (threadIdx.x == 0) s_queued = 0;
      // empty bits of the window: each warp takes 6 rows of 32 + 16 columns, with
      // all 12 loads in flight before the votes
      constexpr int kRowsPerWarp = kIpSpan / (kMapThreads / 32);
      static_assert(kRowsPerWarp * (kMapThreads / 32) == kIpSpan, "k_inpaint: rows per warp");
      bool empty[kRowsPerWarp][2];
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int32_t y = y0 + warp * kRowsPerWarp + k, x = x0 + half * 32 + lane;
          const bool in = y >= 0 && y < m.H && x >= 0 && x < m.W && half * 32 + lane < kIpSpan;
          empty[k][half] = in && !isfinite(__ldg(m.var + (in ? phys_index(m, x, y) : 0)));
        }
#pragma unroll
      for (int k = 0; k < kRowsPerWarp; ++k) {
        const uint64_t word = (uint64_t)__ballot_sync(0xffffffffu, empty[k][0]) |
                              (uint64_t)__ballot_sync(0xffffffffu, empty[k][1]) << 32;
        if (lane == 0) s_rows[warp * kRowsPerWarp + k] = word;
      }
      __syncthreads();
      if (threadIdx.x < kIpSpan) {  // transpose
        uint64_t col = 0;
        for (int r = 0; r < kIpSpan; ++r) col |= ((s_rows[r] >> threadIdx.x) & 1ull) << r;
        s_cols[threadIdx.x] = col;
      }
      __syncthreads();
      // every cell: estimates copied, cells of long empty runs NaN, the rest queued
      for (int k = 0; k < 4; ++k) {
        const int ci = threadIdx.x % kIpT, cj = threadIdx.x / kIpT + k * (kMapThreads / kIpT);
        const int32_t lx = x0 + kIpRim + ci, ly = y0 + kIpRim + cj;
        const bool in = lx < m.W && ly < m.H;
        const int i = kIpRim + ci, j = kIpRim + cj;  // the cell in the window
        bool search = false;
        if (in) {
          const int32_t p = phys_index(m, lx, ly);
          if (!ip_empty(s_rows, i, j)) m.inpaint[p] = m.h[p];
          else if (run_through(s_rows[j], i) > 8 || run_through(s_cols[i], j) > 8) m.inpaint[p] = qnan();
          else search = true;
        }
        const unsigned want = __ballot_sync(0xffffffffu, search);
        int base = 0;
        if (lane == 0 && want) base = atomicAdd(&s_queued, __popc(want));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (search) s_queue[base + __popc(want & ((1u << lane) - 1u))] = (uint16_t)(cj * kIpT + ci);
      }
      __syncthreads();
      // the searches, one per thread (the queue keeps the lanes of a warp busy)
      for (int q = threadIdx.x; q < s_queued; q += kMapThreads) {
        const int ci = s_queue[q] % kIpT, cj = s_queue[q] / kIpT;
        const int32_t lx = x0 + kIpRim + ci, ly = y0 + kIpRim + cj;
        m.inpaint[phys_index(m, lx, ly)] = inpaint_cell(m, s_rows, kIpRim + ci, kIpRim + cj, lx, ly);
      }
      __syncthreads();
    }
  }
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
