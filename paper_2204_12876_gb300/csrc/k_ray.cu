// k_ray.cu -- visibility cleanup by ray casting (Section II-E of the paper).
//
// k_ray: one ray per valid point.  The ray from the sensor origin o (the pose
// translation) to the point is sampled at s_k = o + (k step / d) (R p_s) for
// k = 1, 2, ... while k step < d (computed as a + k b in cell units: one FMA
// per coordinate).  A sample inside the map, outside the point's own cell,
// below the cell's threshold h - sqrt(sigma_m^2) of the pre-update map (Eq. 3;
// the threshold layer is -inf for empty cells) and -- when alpha_n > 0 -- with
// |rhat . n| > alpha_n for the cell's previous normal (Eq. 4; a NaN normal
// counts as (0, 0, 1)) marks the cell in a bitmask (atomicOr: idempotent, so
// the marks do not depend on thread order).  Only the k whose samples can lie
// inside the map's box are visited.  The kernel sees the pre-update map.
//
// Most samples of a scan pass far above the surface.  k_coarse keeps, per
// block of kCoarse x kCoarse cells, the largest threshold of the block.  The
// march cuts each ray into chunks of at most G samples spanning at most
// kCoarse cells per axis; a chunk's samples lie in the cells between those of
// its first sample and the next chunk's first sample (both coordinates and z
// are monotone in k, and the same rounded arithmetic gives every sample), so
// when the lower of those two heights is not below the largest threshold of
// the (at most 2 x 2) blocks they span, none of its samples can mark a cell
// and it is skipped -- an exact test, not a heuristic.  Each lane tests its own ray's chunks; the warp
// queues the others and marches them G lanes per chunk, one sample per lane.
//
// k_clear: after the fusion, every marked cell that holds an estimate and was
// last written at least max(1, cleanup_min_age) updates ago is removed; the
// bitmask is reset for the next update.  Tiles start on multiples of kTile
// cells, so a tile owns whole mark words.
#include "ray_pass.cuh"

namespace em {

__global__ void __launch_bounds__(kCoarseThreads) k_coarse(const BatchDev* __restrict__ bp) {
  coarse_pass(*bp, own_grid());
}

template <int G, bool kExt>
__global__ void __launch_bounds__(kRayThreads, 4) k_ray(const BatchDev* __restrict__ bp) {
  __shared__ RaySmem S;
  ray_pass<G, kExt>(*bp, own_grid(), S);
}

__global__ void __launch_bounds__(kClearThreads) k_clear(const BatchDev* __restrict__ bp) {
  clear_pass(*bp, own_grid());
}

template <bool kExt>
static void launch_ray_g(const BatchDev* b, int g, int grid, cudaStream_t s) {
  switch (g) {
    case 1: k_ray<1, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 2: k_ray<2, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 4: k_ray<4, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 16: k_ray<16, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    case 32: k_ray<32, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
    default: k_ray<8, kExt><<<grid, kRayThreads, 0, s>>>(b); break;
  }
}

cudaError_t launch_ray(const BatchDev* b, int64_t n_points, int64_t n_cells, int group, bool ext, cudaStream_t s) {
  if (n_points <= 0) return cudaSuccess;
  // the coarse grids first (grid-stride: any batch up to the capacities)
  const int64_t blocks = n_cells / (kCoarse * kCoarse) + 1;
  const int64_t ccap = (int64_t)sm_count() * 8;
  const int64_t cgrid = (blocks + kCoarseThreads - 1) / kCoarseThreads;
  k_coarse<<<(int)(cgrid < ccap ? cgrid : ccap), kCoarseThreads, 0, s>>>(b);
  const int g = (group == 1 || group == 2 || group == 4 || group == 8 || group == 16 || group == 32) ? group : 8;
  const int64_t want = (n_points + kRayThreads - 1) / kRayThreads;  // one 32-ray chunk per warp
  const int64_t cap = (int64_t)sm_count() * 16;
  const int grid = (int)(want < cap ? want : cap);
  if (ext) launch_ray_g<true>(b, g, grid, s);
  else launch_ray_g<false>(b, g, grid, s);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kClearThreads) k_overlap(const BatchDev* __restrict__ bp) {
  overlap_pass(*bp, own_grid());
}

cudaError_t launch_overlap(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * 8;
  k_overlap<<<(int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap), kClearThreads, 0, s>>>(b);
  return cudaGetLastError();
}

const void* coarse_kernel() { return reinterpret_cast<const void*>(&k_coarse); }
const void* clear_kernel() { return reinterpret_cast<const void*>(&k_clear); }

cudaError_t launch_clear(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  const int64_t tiles = n_cells / kTile;  // a block per tile
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap);
  k_clear<<<grid, kClearThreads, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace em
