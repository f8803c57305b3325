// em_internal.cuh -- device-side descriptors and kernel launchers of libem.so.
//
// One update is a "batch": one or more maps, each with one or more clouds.
// The plain em_update is a batch of one map and one cloud.  All sizes that
// change from update to update live in device memory (BatchDev / MapDev /
// CloudDev), so the same kernels serve the plain, multi-cloud and batched
// forms, and launches can be captured in a CUDA graph.
//
// Pipeline of one update (Section II-A of the paper: transform, height update
// and ray casting in the same iteration, then per-cell passes):
//   k_count    transform + noise variance + cell binning, per-cell counts;
//              per-cell ray thresholds of the pre-update map   (Section II-C)
//   k_ray      visibility ray march against the pre-update map (Section II-E)
//   k_alloc    one segment of the sorted record array per touched cell
//   k_scatter  records into their cell's segment (counting sort by cell)
//   k_fuse     per cell: wall rule, Mahalanobis gate, Eq. 1/2 in information
//              form with exact integer accumulation          (Section II-C)
//   k_clear    remove penetrated cells not written recently   (Section II-E)
//   k_normals / k_smooth / k_inpaint                          (Section II-A, II-I)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace em {

// per-map counters (device), in em_stats order
enum StatIdx {
  kStUpdates = 0, kStIn, kStValid, kStInMap, kStAccepted, kStRejected, kStWall, kStCellsUpdated,
  kStCleared, kStRaySamples, kStCount
};

// per-map device control block: counters that live across kernels of an update
struct MapCtl {
  unsigned long long stats[kStCount];
  int32_t n_touched;   // small touched cells this update, front of the touched list (reset by k_clear)
  int32_t seg_cursor;  // records allocated to segments this update (reset by k_clear)
  int32_t err;         // first device-side error code of this map (sticky until read)
  int32_t n_big;       // large touched cells, back of the touched list (reset by k_clear)
  int32_t big_next;    // work-stealing cursor over the large cells (reset by k_clear)
  int32_t pad[3];
};

// point status codes (trace)
enum PointStatus : uint8_t { kPtNonFinite = 0, kPtRange = 1, kPtOutside = 2, kPtFused = 3, kPtRejected = 4, kPtWall = 5 };

struct MapDev {
  // layers, physical ring layout [py][px], px = (ix + ox) mod W
  float* h;
  float* var;       // +inf = empty cell
  int32_t* t_last;
  float* nx;        // normals (may be null)
  float* ny;
  float* nz;
  float* smooth;    // may be null
  float* inpaint;   // may be null
  uint32_t* mark;   // visibility marks, one bit per physical cell, zero between updates
  float* thr;       // per physical cell: h - sqrt(var_eff) of the pre-update map, -inf if empty
  int32_t* cnt;     // per physical cell point count, zero between updates
  int32_t* cell_base;  // per physical cell: start of its segment (valid for touched cells)
  int32_t* touched;    // touched physical cells this update (capacity W*H): cells with at most
                       // big_thresh records from the front, larger ones from the back
  int32_t* seg_base;   // per touched entry: segment start (absolute record index)
  int32_t* seg_len;    // per touched entry: segment length
  MapCtl* ctl;
  int64_t pt_begin;    // this map's records occupy [pt_begin, pt_begin + pt_count)
  int64_t pt_count;
  int32_t W, H, ox, oy;
  float x0, y0, res;
  int32_t t_now;       // index of this update
  // method parameters
  float a0, a1, a2, var_min, min_range, max_range, k, v_out, sigma_t2, ray_step, alpha_n;
  int32_t wall, min_age;
  uint32_t flags;
  int32_t big_thresh;  // segments longer than this are fused by a whole block
};

struct CloudDev {
  const float* pts;
  int64_t n;
  int64_t begin;   // first index of this cloud in the batch point space
  int32_t stride;
  int32_t map;
  float R[9];
  float t[3];
};

struct BatchDev {
  int32_t n_maps, n_clouds;
  int64_t n_points;
  const MapDev* maps;
  const CloudDev* clouds;
  float2* zw_sorted;   // records (z, sigma_p^2) grouped by cell
  int32_t* idx_sorted; // original point index per sorted record (trace only, else null)
  int32_t* tr_ix;      // trace (null unless EM_F_TRACE)
  int32_t* tr_iy;
  uint8_t* tr_status;
};

// number of SMs of the current device (cached)
int sm_count();

// ---- launchers (each returns cudaGetLastError() of its launches)
cudaError_t launch_bin(const BatchDev* b, int64_t n_points, cudaStream_t s);
cudaError_t launch_ray(const BatchDev* b, int64_t n_points, int group, cudaStream_t s);
cudaError_t launch_alloc(const BatchDev* b, int32_t n_maps, int32_t max_cells, cudaStream_t s);
cudaError_t launch_scatter(const BatchDev* b, int64_t n_points, cudaStream_t s);
cudaError_t launch_fuse(const BatchDev* b, int32_t n_maps, int32_t max_cells, int group, cudaStream_t s);
cudaError_t launch_clear(const BatchDev* b, int32_t n_maps, int32_t max_cells, cudaStream_t s);
cudaError_t launch_normals(const BatchDev* b, int32_t n_maps, int32_t max_cells, cudaStream_t s);
cudaError_t launch_smooth(const BatchDev* b, int32_t n_maps, int32_t max_cells, cudaStream_t s);
cudaError_t launch_inpaint(const BatchDev* b, int32_t n_maps, int32_t max_cells, cudaStream_t s);
cudaError_t launch_shift_clear(const MapDev& m, int32_t dx, int32_t dy, cudaStream_t s);
cudaError_t launch_layers_out(const MapDev& m, uint32_t mask, float* dst, cudaStream_t s);
cudaError_t launch_layers_in(const MapDev& m, uint32_t mask, const float* src, cudaStream_t s);
cudaError_t launch_fill_map(const MapDev& m, cudaStream_t s);

// ---- small device helpers shared by the kernels

__device__ __forceinline__ int32_t clamp_floor(float q) {
  float f = floorf(q);
  f = fminf(fmaxf(f, -1.0e9f), 1.0e9f);
  return (int32_t)f;
}

// physical index of logical cell (ix, iy), both in range
__device__ __forceinline__ int32_t phys_index(const MapDev& m, int32_t ix, int32_t iy) {
  int32_t px = ix + m.ox;
  px -= (px >= m.W) ? m.W : 0;
  int32_t py = iy + m.oy;
  py -= (py >= m.H) ? m.H : 0;
  return py * m.W + px;
}

// effective variance of a cell at update t_now (lazy time variance)
__device__ __forceinline__ float var_eff(const MapDev& m, float var, int32_t t_last) {
  return __fmaf_rn(m.sigma_t2, (float)(m.t_now - t_last), var);
}

// index of the cloud that holds batch point g (clouds sorted by begin)
__device__ __forceinline__ int find_cloud(const CloudDev* cl, int n_clouds, int64_t g) {
  int lo = 0, hi = n_clouds - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cl[mid].begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace em
