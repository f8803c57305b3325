// em_internal.cuh -- device-side descriptors and kernel launchers of libem.so.
//
// One update is a "batch": one or more maps, each with one or more clouds.
// The plain em_update is a batch of one map and one cloud.  All sizes that
// change from update to update live in device memory (BatchDev / MapDev /
// CloudDev), so the same kernels serve the plain, multi-cloud and batched
// forms, and launches can be captured in a CUDA graph.
//
// Work spaces of a batch:
//   points  the clouds of all maps concatenated (per-point kernels, 1D grid);
//   cells   the cells of all maps concatenated, each map's range padded to a
//           multiple of kTile cells, so every tile of kTile cells lies in one
//           map (per-cell kernels, 1D grid over tiles: uneven maps balance).
//
// Pipeline of one update (Section II-A of the paper: transform, height update
// and ray casting in the same iteration, then per-cell passes):
//   k_count    transform + noise variance + cell binning, per-tile record
//              counts; per cell: ray thresholds of the pre-update map
//                                                              (Section II-C)
//   k_ray      visibility ray march against the pre-update map (Section II-E)
//   k_alloc    one range of the record arrays per tile of 1024 cells; the
//              fusion's work lists (dense tiles cut into pieces)
//   k_scatter  records into their tile's range (counting sort by tile)
//   k_fuse     per work item, one block: the tile's state in shared memory;
//              per cell: wall rule, Mahalanobis gate, Eq. 1/2 in information
//              form with exact integer accumulation (Section II-C)
//   k_clear    remove penetrated cells not written recently   (Section II-E)
//   k_normals / k_smooth / k_inpaint                          (Section II-A, II-I)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace em {

constexpr int kTile = 1024;  // cells per tile of the cell space
// The ray march's coarse grid: per block of kCoarse x kCoarse logical cells the
// largest ray threshold of the block (a chunk of samples whose lowest z is not
// below it cannot mark any cell).
constexpr int kCoarseShift = 3;
constexpr int kCoarse = 1 << kCoarseShift;
inline int32_t coarse_dim(int32_t cells) { return (cells + kCoarse - 1) >> kCoarseShift; }


// per-map counters (device), in em_stats order
enum StatIdx {
  kStUpdates = 0, kStIn, kStValid, kStInMap, kStAccepted, kStRejected, kStWall, kStCellsUpdated,
  kStCleared, kStRaySamples, kStDriftPoints, kStCount
};

// per-map device control block
struct MapCtl {
  unsigned long long stats[kStCount];
  int32_t err;         // first device-side error code of this map (sticky until read)
  float drift_last;    // height error added by the last drift compensation
  int32_t pad[2];
  // drift-compensation sums, one slot per update parity: update t accumulates
  // into slot t & 1 (k_count) and reads it (k_drift); k_count of update t clears
  // slot (t + 1) & 1, last read by update t - 1, which has completed
  long long drift_h[2];           // sum of the errors' fixed-point high parts
  unsigned long long drift_l[2];  // ... and low parts (value h 2^27 + l, 2^-44 m units)
  unsigned long long drift_n[2];  // points in the sum
};

// per-batch device control block (reset by k_count and k_alloc)
struct BatchCtl {
  int32_t rec_total;         // records of this update (all maps)
  int32_t fuse_next;         // work counter of the fusion: pieces, heavy tiles, then light tiles
  int32_t n_split;           // tiles split into pieces (one accumulator slot each)
  int32_t n_pieces;          // entries of the three work lists of the fusion
  int32_t n_heavy;
  int32_t n_light;
  int32_t ray_next;          // work counter of the ray march: runs of kRayRun 32-point batches
  int32_t pad;
  // grid barrier of the persistent kernel (k_persist.cu): block tickets, blocks
  // done, and the abort flag of a barrier wait that ran out; zero between launches
  unsigned long long bar_ticket;
  int32_t bar_done;
  int32_t bar_abort;
};

// A tile with more than heavy_thresh records is split, while accumulator
// slots last, into pieces of at most heavy_thresh records, fused by different
// blocks: each adds its exact sums to the tile's slot (kSplitWords 64-bit words
// per cell) and the last piece to finish writes the cells.
constexpr int kMaxSplit = 512;       // accumulator slots at most
constexpr int kSplitWords = 5;       // per cell: weight sum (high, low), term sum (high, low), counts

// One work item of the fusion, written by k_alloc: a non-empty tile (whole) or
// a piece of a split tile.  The tile's records are [r0, r1); the item fuses
// [q0, q1) of them (the whole range unless it is a piece).
struct FuseItem {
  int32_t tile, map;                 // tile of the batch cell space, and the map it lies in
  int32_t r0, r1, q0, q1;
  int32_t slot, np;                  // accumulator slot and pieces of a split tile; -1 and 1 otherwise
};
static_assert(sizeof(FuseItem) == 32, "work items are read as two 16-byte words");

// Records: one per in-map point, grouped by tile of kTile cells of the batch
// cell space (a tile lies in one map: map cell ranges are padded to whole
// tiles).  Structure of arrays: z (map frame), sigma_p^2, and the cell's index
// within its tile.  Tile t's records fill [tile_base[t], tile_base[t + 1]).
constexpr int kMinHeavy = 32;        // tuning bounds of the heavy-tile threshold (x 16 records)
constexpr int kMaxHeavy = 1023;

// device-side error word value for a failed internal consistency check (EM_ERR_CUDA)
constexpr int32_t kErrInternal = -3;
// ... and for a bounded device-side wait that ran out (EM_ERR_TIMEOUT)
constexpr int32_t kErrTimeout = -4;

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
  float* upper;     // upper bound of the ground height (Section II-H), +inf where none; may be null
  uint32_t* mark;   // visibility marks, one bit per physical cell, zero between updates
  float* thr;       // per LOGICAL cell [iy][ix]: h - sqrt(var_eff) of the pre-update map, -inf if empty
  float* cthr;      // per coarse block [by][bx] (CW x CH of them): the largest thr of its cells
  MapCtl* ctl;
  int64_t cbegin;   // this map's first block in the batch's coarse space (maps with the ray march)
  int32_t CW, CH;   // coarse blocks per row and column; 0 x 0 without the ray march
  int64_t cell_begin;  // this map's first cell in the batch cell space (multiple of kTile)
  int32_t W, H, ox, oy;
  float x0, y0, res, inv_res;  // inv_res = 1 / res rounded to float
  float drift_flat;    // drift compensation: flat iff previous normal n_z >= this; 0 = off
  float excl_b, excl_c, excl_tan, excl_d;  // exclusion ramp (tan of its angle); excl_d <= 0 = off
  float ovl_r2, ovl_dz, ref_x, ref_y;      // overlap clearance: radius^2, height gap, robot position
  float z_ref;         // reference height of empty cells in the fusion sums: the z of the
                       // first cloud's sensor origin (any fixed value gives the same result
                       // up to rounding; one near the points keeps the terms small)
  int32_t t_now;       // index of this update
  // method parameters
  float a0, a1, a2, var_min, min_range, max_range, k, v_out, sigma_t2, ray_step, alpha_n;
  int32_t wall, min_age;
  uint32_t flags;
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
  int64_t n_cells;     // padded size of the cell space
  int64_t n_coarse;    // blocks of the coarse grids of all maps
  const MapDev* maps;
  const CloudDev* clouds;
  // records grouped by tile (layout above); capacity: the points of the batch
  float* rz;
  float* rv;
  uint16_t* rc;
  int32_t* idx_sorted; // original point index per record (trace only, else null)
  int32_t* tr_ix;      // trace (null unless EM_F_TRACE)
  int32_t* tr_iy;
  uint8_t* tr_status;
  BatchCtl* ctl;
  // per tile of the cell space (n_cells / kTile tiles): the records counted by
  // k_count (zero between updates), their first record (k_alloc; one more
  // entry holds the total), k_scatter's claims (zeroed by k_alloc), and the
  // map of every non-empty tile (k_count)
  int32_t* tile_cnt;
  int32_t* tile_base;
  int32_t* tile_cur;
  int32_t* tile_map;
  // the fusion's work lists (k_alloc): pieces of split tiles (max_pieces
  // entries), tiles with more than heavy_thresh records fused whole when the
  // slots ran out, and the other non-empty tiles (one entry per tile each)
  FuseItem* pieces;
  FuseItem* heavy;
  FuseItem* light;
  // split tiles: per slot kSplitWords x kTile accumulator words and a count of
  // finished pieces, both zero between updates
  unsigned long long* split_acc;
  int32_t* split_done;
  int32_t split_slots; // 0: no tile is split
  int32_t max_pieces;
  int32_t heavy_thresh;
  int32_t fuse_threads;  // threads per fusion block: 256 or 512
  uint32_t passes;       // kPass* bits: optional passes some map of the batch needs
};
enum : uint32_t { kPassRay = 1u, kPassOverlap = 2u };

inline int64_t pad_tile(int64_t cells) { return (cells + kTile - 1) / kTile * kTile; }
// The kernels read points and layers as 4-byte words: a buffer that does not
// start on a 4-byte boundary is refused on the host (it would fault on the device).
inline bool word_aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

// number of SMs of the current device (cached)
int sm_count();

// Launch ray(stream) beside rest() (which launches on s) and join both before
// the next launch on s: the ray work goes to the side stream between two
// events.  While s is being captured into a graph the two run in order on s
// (a capture never spans a second stream, and nothing edits a capture while
// it runs; em_batch.cu rearranges its own finished graphs instead).
template <class Ray, class Rest>
cudaError_t launch_beside(cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, Ray ray,
                          Rest rest) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone || !side) {
    e = ray(s);
    return e == cudaSuccess ? rest() : e;
  }
  e = cudaEventRecord(fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
  if (e != cudaSuccess) return e;
  e = ray(side);
  // the join is made whatever happened since the fork
  cudaError_t je = cudaEventRecord(join, side);
  if (e == cudaSuccess) e = rest();
  if (je == cudaSuccess) je = cudaStreamWaitEvent(s, join, 0);
  return e == cudaSuccess ? je : e;
}

// The kernels a captured sequence is rearranged by (em_batch.cu).
const void* coarse_kernel();
const void* alloc_kernel();
const void* clear_kernel();
bool is_fuse_kernel(const void* f);

// ---- launchers (each returns cudaGetLastError() of its launches)
// ext: some map of the batch uses the exclusion area or the upper-bound layer
cudaError_t launch_bin(const BatchDev* b, int64_t n_points, int64_t n_cells, bool ext, cudaStream_t s);
cudaError_t launch_drift(const BatchDev* b, int64_t n_points, int64_t n_cells, bool ext, cudaStream_t s);
// the coarse threshold grids, then the march (group: samples per chunk and lanes per marched chunk)
cudaError_t launch_ray(const BatchDev* b, int64_t n_points, int64_t n_cells, int group, bool ext, cudaStream_t s);
cudaError_t launch_alloc(const BatchDev* b, int64_t n_cells, cudaStream_t s);
cudaError_t launch_scatter(const BatchDev* b, int64_t n_points, bool ext, cudaStream_t s);
cudaError_t launch_fuse(const BatchDev* b, int64_t n_cells, int threads, cudaStream_t s);
cudaError_t launch_clear(const BatchDev* b, int64_t n_cells, cudaStream_t s);
// The whole update but the drift compensation and the stencils (count, coarse
// grids, tile ranges, scatter, ray march, fusion, removal, overlap clearance)
// in one cooperative launch with grid barriers; barrier waits are bounded by
// wait_ms.  cudaErrorNotSupported when the device cannot run it.
cudaError_t launch_persist(const BatchDev* b, int group, bool ext, int wait_ms, cudaStream_t s);
// The bounded wait of the persistent kernel on a word that nothing sets: one
// block, budget wait_us; *timed_out (device memory) becomes 1 when it runs out.
cudaError_t launch_wait_selftest(const unsigned long long* word, int* timed_out, int wait_us, cudaStream_t s);
cudaError_t launch_overlap(const BatchDev* b, int64_t n_cells, cudaStream_t s);
cudaError_t launch_normals(const BatchDev* b, int64_t n_cells, cudaStream_t s);
cudaError_t launch_smooth(const BatchDev* b, int64_t n_cells, cudaStream_t s);
cudaError_t launch_inpaint(const BatchDev* b, int64_t n_cells, cudaStream_t s);
cudaError_t launch_shift_clear(const MapDev& m, int32_t dx, int32_t dy, cudaStream_t s);
cudaError_t launch_layers_out(const MapDev& m, uint32_t mask, float* dst, cudaStream_t s);
// Layer reads of up to kMaxReadJobs maps in one launch (the jobs are the kernel parameters).
constexpr int kMaxReadJobs = 32;
struct ReadJob {
  MapDev m;
  uint32_t mask;
  float* dst;
};
struct ReadJobs {
  int n;
  ReadJob job[kMaxReadJobs];
};
cudaError_t launch_layers_out_multi(const ReadJobs& jobs, cudaStream_t s);
static_assert(sizeof(ReadJobs) <= 32000, "the read jobs must fit a kernel's parameter block");
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

// logical coordinates of physical cell p
__device__ __forceinline__ void logical_of(const MapDev& m, int32_t p, int32_t& lx, int32_t& ly) {
  const int32_t py = p / m.W, px = p - py * m.W;
  lx = px - m.ox;
  lx += (lx < 0) ? m.W : 0;
  ly = py - m.oy;
  ly += (ly < 0) ? m.H : 0;
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

// The same, tried first on cloud `hint` (the cloud of the caller's previous
// point: passes walk the point space in order, so it usually holds g); an
// empty cloud never holds g, so the answer is the search's.
__device__ __forceinline__ int find_cloud(const CloudDev* cl, int n_clouds, int64_t g, int hint) {
  if ((unsigned)hint < (unsigned)n_clouds && cl[hint].begin <= g && g < cl[hint].begin + cl[hint].n) return hint;
  return find_cloud(cl, n_clouds, g);
}

// index of the map whose cell range holds batch cell g (maps sorted by cell_begin)
__device__ __forceinline__ int find_map_cell(const MapDev* maps, int n_maps, int64_t g) {
  int lo = 0, hi = n_maps - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (maps[mid].cell_begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The blocks that share a pass: a kernel's own grid, or the blocks of the
// persistent kernel (k_persist.cu) that the pass runs on.
struct Grid {
  int bid, nb;
};
__device__ __forceinline__ Grid own_grid() { return Grid{(int)blockIdx.x, (int)gridDim.x}; }

// Iterate over the tiles of the cell space: for each tile the map it lies in
// (block-uniform) and the tile's first physical cell.  body(m, map, p0, count).
template <class F>
__device__ __forceinline__ void for_each_tile(const struct BatchDev& b, Grid gr, F body) {
  const int64_t n_tiles = b.n_cells / kTile;
  for (int64_t t = gr.bid; t < n_tiles; t += gr.nb) {
    const int64_t g0 = t * kTile;
    const int mi = find_map_cell(b.maps, b.n_maps, g0);
    const MapDev& m = b.maps[mi];
    const int64_t p0 = g0 - m.cell_begin;
    const int32_t ncell = m.W * m.H;
    if (p0 >= ncell) continue;  // padding at the end of a map
    const int32_t cnt = (int32_t)(ncell - p0 < kTile ? ncell - p0 : kTile);
    body(m, mi, (int32_t)p0, cnt);
  }
}
template <class F>
__device__ __forceinline__ void for_each_tile(const struct BatchDev& b, F body) {
  for_each_tile(b, own_grid(), body);
}

}  // namespace em
