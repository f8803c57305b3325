// k_persist.cu -- the batched form in one persistent launch: the passes of an
// update over every map of a batch (transform, noise, binning, grouping by
// tile, wall rule, gate, Eq. 1/2 fusion, ray march and removal; Section II-A
// to II-E of the paper) in one cooperative kernel whose blocks are all
// resident, with a grid-wide barrier wherever a pass needs the one before:
//
//   count: transform + bin + per-tile counts, then the ray thresholds
//   | tile ranges and the fusion's work lists (one block, sort_pass.cuh) and
//   |   the coarse threshold grids (every other block)
//   | scatter of the records, then the ray march (independent of each other)
//   | fusion: blocks take tiles and pieces from the work queue
//   | removal of marked cells (| overlap clearance)
//
// The stencils (normals, smoothing, in-painting) follow as their own kernels.
// The passes share one shared-memory buffer; each one ends with a block
// barrier, so the next pass of the same block never writes into it early.
// A barrier hands out tickets from one counter: barrier j of a launch holds
// tickets [j nb, (j + 1) nb), and a block waits until the counter reaches the
// end of its barrier's range.  The last block to finish the launch sets the
// counter back to zero.  Every wait is bounded by a clock64 budget: a wait
// that runs out raises the abort flag, writes EM_ERR_TIMEOUT into the maps'
// error words, and every block leaves at its next barrier.
#include "sort_pass.cuh"
#include "ray_pass.cuh"
#include "fuse_pass.cuh"

namespace em {

constexpr int kPersistThreads = 256;
static_assert(kPersistThreads == kPointThreads && kPersistThreads == kRayThreads &&
                  kPersistThreads == kClearThreads,
              "the passes share one block size");

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
// the passes run one after another and share one shared-memory buffer
constexpr size_t kPersistSmem = cmax(cmax(sizeof(TileSmem), sizeof(RaySmem)), cmax(sizeof(PointSmem), sizeof(AllocSmem)));

// Wait until *word >= target, or until `abort` is raised, for at most budget
// SM clock cycles; true when the word got there.
__device__ __forceinline__ bool wait_at_least(const unsigned long long* word, unsigned long long target,
                                              const int* abort, long long budget) {
  const long long t0 = clock64();
  while (*(const volatile unsigned long long*)word < target) {
    if ((abort && *(const volatile int*)abort) || clock64() - t0 > budget) return false;
    __nanosleep(100);
  }
  return true;
}

// Barrier of all nb blocks of the launch; false when this block should leave.
__device__ __forceinline__ bool grid_barrier(const BatchDev& b, int nb, long long budget, int& s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    BatchCtl* c = b.ctl;
    __threadfence();  // this block's writes before its arrival
    const unsigned long long t = atomicAdd(&c->bar_ticket, 1ull);
    const unsigned long long target = (t / (unsigned long long)nb + 1ull) * (unsigned long long)nb;
    bool ok = wait_at_least(&c->bar_ticket, target, &c->bar_abort, budget);
    if (!ok && atomicExch(&c->bar_abort, 1) == 0) {  // the first block to give up records it
      for (int mi = 0; mi < b.n_maps; ++mi) atomicCAS(&b.maps[mi].ctl->err, 0, kErrTimeout);
    }
    __threadfence();  // the other blocks' writes before this block goes on
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int G, bool kExt>
__global__ void __launch_bounds__(kPersistThreads, 4) k_persist(const BatchDev* __restrict__ bp, long long budget) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_ok;
  const BatchDev& b = *bp;
  const int nb = gridDim.x, bid = blockIdx.x;
  const Grid all{bid, nb};
  const bool ray = (b.passes & kPassRay) != 0;
  count_pass<kExt>(b, all, *reinterpret_cast<PointSmem*>(sm));
  bool ok = grid_barrier(b, nb, budget, s_ok);
  if (ok) {
    if (bid == 0) alloc_pass<kPersistThreads>(b, *reinterpret_cast<AllocSmem*>(sm));
    else if (ray) coarse_pass(b, Grid{bid - 1, nb - 1});
    ok = grid_barrier(b, nb, budget, s_ok);
  }
  if (ok) {
    scatter_pass<kExt>(b, all, *reinterpret_cast<PointSmem*>(sm));
    if (ray) ray_pass<G, kExt>(b, all, *reinterpret_cast<RaySmem*>(sm));
    ok = grid_barrier(b, nb, budget, s_ok);
  }
  if (ok) {
    fuse_pass<kPersistThreads>(b, *reinterpret_cast<TileSmem*>(sm));
    ok = grid_barrier(b, nb, budget, s_ok);
  }
  if (ok) {
    clear_pass(b, all);
    if (b.passes & kPassOverlap) {
      ok = grid_barrier(b, nb, budget, s_ok);
      if (ok) overlap_pass(b, all);
    }
  }
  // the last block to leave makes the barrier state ready for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&b.ctl->bar_done, 1) == nb - 1) {
      b.ctl->bar_ticket = 0ull;
      b.ctl->bar_done = 0;
      b.ctl->bar_abort = 0;
      __threadfence();
    }
  }
}

__global__ void k_wait_selftest(const unsigned long long* word, int* timed_out, long long budget) {
  if (threadIdx.x == 0) *timed_out = wait_at_least(word, 1ull, nullptr, budget) ? 0 : 1;
}

namespace {

long long clock_budget(int ms_times_1000_us) {  // SM cycles of the given microseconds
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) khz = 2000000;
  return (long long)khz * ms_times_1000_us / 1000;
}

template <int G, bool kExt>
cudaError_t launch_persist_t(const BatchDev* b, long long budget, cudaStream_t s) {
  // per device, once: the shared-memory limit above the static 48 KB, and the
  // blocks that fit at once (the cooperative launch needs all of them resident)
  static int per_sm[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorNotSupported;
  int& n = per_sm[dev][kExt ? 1 : 0];
  if (n == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_persist<G, kExt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPersistSmem);
    if (e != cudaSuccess) return e;
    int v = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_persist<G, kExt>, kPersistThreads, kPersistSmem);
    if (e != cudaSuccess) return e;
    n = v > 0 ? v : -1;
  }
  if (n < 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * sm_count()));
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = kPersistSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persist<G, kExt>, b, budget);
}

template <bool kExt>
cudaError_t launch_persist_g(const BatchDev* b, int g, long long budget, cudaStream_t s) {
  switch (g) {
    case 1: return launch_persist_t<1, kExt>(b, budget, s);
    case 2: return launch_persist_t<2, kExt>(b, budget, s);
    case 4: return launch_persist_t<4, kExt>(b, budget, s);
    case 16: return launch_persist_t<16, kExt>(b, budget, s);
    case 32: return launch_persist_t<32, kExt>(b, budget, s);
    default: return launch_persist_t<8, kExt>(b, budget, s);
  }
}

}  // namespace

cudaError_t launch_persist(const BatchDev* b, int group, bool ext, int wait_ms, cudaStream_t s) {
  const long long budget = clock_budget(wait_ms * 1000);
  return ext ? launch_persist_g<true>(b, group, budget, s) : launch_persist_g<false>(b, group, budget, s);
}

cudaError_t launch_wait_selftest(const unsigned long long* word, int* timed_out, int wait_us, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(word, timed_out, clock_budget(wait_us));
  return cudaGetLastError();
}

}  // namespace em
