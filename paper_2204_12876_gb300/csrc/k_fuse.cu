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
// atomics).  Then every touched cell of the tile is written once and its
// accumulators go back to zero.
//
// A tile with many records (a dense depth image puts tens of thousands in one
// tile) is cut into pieces that different blocks fuse at the same time: each
// piece adds its runs' sums to the tile's accumulator slot in global memory
// (64-bit integer atomics, exact like the rest) and counts itself done;
// the block that finishes the tile's last piece reads the slot, writes the
// cells and zeroes the slot for the next update.  No block waits for another.
// Blocks take work from a counter: pieces first, then tiles listed heavy
// (fused whole when the slots ran out), then every other tile.
#include "fuse_pass.cuh"

namespace em {

// MINB resident blocks per SM.  Updates with many tiles take three blocks of
// 512 threads (40 registers: the kernel waits on memory, and 75 % of the warp
// slots hide more of it than the 50 % that 60 registers allow); updates with
// fewer tiles than three blocks per SM could use take two (60 registers, the
// faster block); blocks of 256 threads: four (shared memory allows no more).
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_fuse(const BatchDev* __restrict__ bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fuse_pass<NT>(*bp, *reinterpret_cast<TileSmem*>(smem_raw));
}

template <int NT, int MINB>
static cudaError_t launch_fuse_t(const BatchDev* b, int64_t n_cells, cudaStream_t s) {
  // per device, once: the shared-memory limit above the static 48 KB, and the
  // resident blocks per SM (the host queries cost tens of microseconds)
  static int per_sm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int resident = 1;
  if (dev >= 0 && dev < 64) {
    if (!per_sm[dev]) {
      cudaError_t e = cudaFuncSetAttribute(k_fuse<NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(TileSmem));
      if (e != cudaSuccess) return e;
      int n = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse<NT, MINB>, NT, sizeof(TileSmem));
      per_sm[dev] = n > 0 ? n : 1;
    }
    resident = per_sm[dev];
  }
  const int64_t tiles = n_cells / kTile;
  const int64_t cap = (int64_t)sm_count() * resident;  // one resident wave
  const int grid = (int)(tiles < cap ? (tiles < 1 ? 1 : tiles) : cap);
  k_fuse<NT, MINB><<<grid, NT, sizeof(TileSmem), s>>>(b);
  return cudaGetLastError();
}

bool is_fuse_kernel(const void* f) {
  return f == reinterpret_cast<const void*>(&k_fuse<256, 4>) || f == reinterpret_cast<const void*>(&k_fuse<512, 2>) ||
         f == reinterpret_cast<const void*>(&k_fuse<512, 3>);
}

cudaError_t launch_fuse(const BatchDev* b, int64_t n_cells, int threads, cudaStream_t s) {
  if (threads < 512) return launch_fuse_t<256, 4>(b, n_cells, s);
  return n_cells / kTile >= 3 * (int64_t)sm_count() ? launch_fuse_t<512, 3>(b, n_cells, s)
                                                    : launch_fuse_t<512, 2>(b, n_cells, s);
}

}  // namespace em
