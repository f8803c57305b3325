// em_noalloc.cu -- em_update_noalloc: one map update that allocates no memory.
//
// Some callers cannot call cudaMalloc at update time: a real-time control loop
// that forbids allocation after start-up (an allocation can block on the
// driver for milliseconds), or a host framework whose own caching allocator
// has already claimed the device memory.  For them this entry point runs the
// same kernels as em_update (binning, counting sort by cell, gate + fusion, ray
// march, removal) on map layers the caller owns, and keeps every piece of
// scratch memory in one file-scope __device__ array of fixed size.  The call's
// descriptor goes to the device as a kernel parameter (no host buffer, no
// copy), and its only other preparation is a memset of the scratch.
//
// Limits: at most kMaxCells cells per map and kMaxPoints points per update
// (about 6.1 MiB of scratch, held by every GPU that loads the library until the
// process exits).  Every call shares the array and it keeps the last call's
// contents; the call clears what must start at zero.  Calls whose GPU work
// overlaps (e.g. on two streams) race on the array.
#include <cuda_runtime.h>
#include <string.h>

#include <cmath>
#include <cstddef>
#include <mutex>

#include "em.h"
#include "em_host.h"
#include "em_internal.cuh"

using namespace em;

namespace {

constexpr int32_t kMaxCells = EM_NOALLOC_MAX_CELLS;
constexpr int64_t kMaxPoints = EM_NOALLOC_MAX_POINTS;
constexpr int kMaxCloudsNA = EM_NOALLOC_MAX_CLOUDS;

constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Everything one call's kernels read from the descriptor, passed by value to
// k_put_desc (well below the 32 KB of a kernel's parameters).
struct Desc {
  BatchDev b;
  MapDev m;
  CloudDev c[kMaxCloudsNA];
};
static_assert(sizeof(Desc) <= 4096, "the descriptor travels as a kernel parameter");

// scratch layout; the part that must start at zero (ctl, marks, tile counts) is contiguous
constexpr size_t kMaxTiles = ((size_t)kMaxCells + kTile - 1) / kTile;
constexpr size_t kOffDesc = 0;
constexpr size_t kOffCtl = kOffDesc + up256(sizeof(Desc));
constexpr size_t kOffBCtl = kOffCtl + up256(sizeof(MapCtl));
constexpr size_t kOffMark = kOffBCtl + up256(sizeof(BatchCtl));
constexpr size_t kOffTCnt = kOffMark + up256(((size_t)kMaxCells + 31) / 32 * sizeof(uint32_t));
constexpr size_t kOffTBase = kOffTCnt + up256((kMaxTiles + 1) * sizeof(int32_t));
constexpr size_t kOffTCur = kOffTBase + up256((kMaxTiles + 1) * sizeof(int32_t));
constexpr size_t kOffTMap = kOffTCur + up256((kMaxTiles + 1) * sizeof(int32_t));
constexpr size_t kOffHeavy = kOffTMap + up256(kMaxTiles * sizeof(int32_t));
constexpr size_t kOffLight = kOffHeavy + up256(kMaxTiles * sizeof(FuseItem));
constexpr size_t kOffThr = kOffLight + up256(kMaxTiles * sizeof(FuseItem));
// coarse blocks of a map of at most kMaxCells cells: (W/8 + 1)(H/8 + 1) <= kMaxCells/64 + (W + H)/8 + 1
constexpr size_t kMaxCoarse = (size_t)kMaxCells / 64 + ((size_t)kMaxCells + 1) / 8 + 2;
constexpr size_t kOffCThr = kOffThr + up256((size_t)kMaxCells * sizeof(float));
constexpr size_t kOffRz = kOffCThr + up256(kMaxCoarse * sizeof(float));
constexpr size_t kOffRv = kOffRz + up256((size_t)kMaxPoints * sizeof(float));
constexpr size_t kOffRc = kOffRv + up256((size_t)kMaxPoints * sizeof(float));
constexpr size_t kScratchBytes = kOffRc + up256((size_t)kMaxPoints * sizeof(uint16_t));

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The descriptor, from the kernel's parameters into the front of the scratch
// (the kernels that follow on the stream read it there).
static_assert(kOffDesc == 0 && sizeof(Desc) % 4 == 0, "word copy of the descriptor");
__global__ void k_put_desc(const Desc d) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&d);
  uint32_t* dst = reinterpret_cast<uint32_t*>(g_noalloc_scratch + kOffDesc);
  for (int i = threadIdx.x; i < (int)(sizeof(Desc) / 4); i += blockDim.x) dst[i] = src[i];
}

namespace {

int na_status(cudaError_t e, const char* what) {
  return e == cudaSuccess ? EM_OK : map_record_error(what, e);
}

// Device address of the scratch on the current device, looked up once per
// device with that device current.
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return EM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return na_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return EM_OK;
}

bool na_params_ok(const em_params* p) {
  if (!p || p->width < 1 || p->height < 1 || p->width > (1 << 22) || p->height > (1 << 22)) return false;
  if (!(std::isfinite(p->resolution) && p->resolution > 0.f)) return false;
  const float f[] = {p->noise_a0, p->noise_a1, p->noise_a2, p->var_min, p->min_range, p->mahalanobis_k,
                     p->outlier_variance, p->time_variance, p->ray_step, p->cleanup_normal_thresh};
  for (float v : f)
    if (!std::isfinite(v)) return false;
  return p->var_min > 0.f && !std::isnan(p->max_range) && p->max_range >= p->min_range &&
         p->outlier_variance >= 0.f && p->time_variance >= 0.f && p->ray_step >= 0.f &&
         p->wall_num_thresh >= 0 && p->cleanup_min_age >= 0 && std::isfinite(p->drift_flatness) &&
         p->drift_flatness >= 0.f && p->drift_flatness <= 1.f &&
         !(p->flags & EM_F_UPPER);  // the upper-bound layer is not one of the caller's layers here
}

}  // namespace

extern "C" int em_update_noalloc(const em_params* params, int64_t shift_x, int64_t shift_y, int32_t t_now,
                                 float* h, float* var, int32_t* t_last, const float* nx, const float* ny,
                                 const float* nz, const em_cloud* clouds, int32_t n_clouds, em_stream_t stream) {
  if (!na_params_ok(params) || !h || !var || !t_last || !clouds || n_clouds < 1 || t_now < 1)
    return EM_ERR_INVALID_ARG;
  if (!word_aligned(h) || !word_aligned(var) || !word_aligned(t_last) || !word_aligned(nx) || !word_aligned(ny) ||
      !word_aligned(nz))
    return EM_ERR_INVALID_ARG;
  if ((params->cleanup_normal_thresh > 0.f || params->drift_flatness > 0.f) && (!nx || !ny || !nz))
    return EM_ERR_INVALID_ARG;
  if ((int64_t)params->width * params->height > kMaxCells || n_clouds > kMaxCloudsNA) return EM_ERR_CAPACITY;
  int64_t total = 0;
  for (int i = 0; i < n_clouds; ++i) {
    const em_cloud& c = clouds[i];
    if (c.n < 0 || (c.stride != 3 && c.stride != 4) || (c.n > 0 && !c.points) || !word_aligned(c.points))
      return EM_ERR_INVALID_ARG;
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(c.pose[k])) return EM_ERR_INVALID_ARG;
    total += c.n;
  }
  if (total > kMaxPoints) return EM_ERR_CAPACITY;

  int dev = 0;
  int rc = na_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  unsigned char* base = nullptr;
  rc = scratch_address(dev, &base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t W = params->width, H = params->height, ncell = W * H;

  // descriptor, built here and handed to k_put_desc by value
  Desc desc;
  memset(&desc, 0, sizeof(desc));
  BatchDev* b = &desc.b;
  MapDev* m = &desc.m;
  CloudDev* cd = desc.c;
  m->h = h;
  m->var = var;
  m->t_last = t_last;
  m->nx = const_cast<float*>(nx);
  m->ny = const_cast<float*>(ny);
  m->nz = const_cast<float*>(nz);
  m->mark = reinterpret_cast<uint32_t*>(base + kOffMark);
  m->thr = reinterpret_cast<float*>(base + kOffThr);
  if (params->ray_step > 0.f) {
    m->cthr = reinterpret_cast<float*>(base + kOffCThr);
    m->CW = coarse_dim(W);
    m->CH = coarse_dim(H);
  }
  m->ctl = reinterpret_cast<MapCtl*>(base + kOffCtl);
  m->cell_begin = 0;
  m->z_ref = clouds[0].pose[11];
  m->W = W;
  m->H = H;
  const double r = (double)params->resolution;
  m->x0 = (float)(r * ((double)shift_x - 0.5 * W));
  m->y0 = (float)(r * ((double)shift_y - 0.5 * H));
  m->res = params->resolution;
  m->inv_res = (float)(1.0 / (double)params->resolution);
  m->t_now = t_now;
  m->a0 = params->noise_a0; m->a1 = params->noise_a1; m->a2 = params->noise_a2; m->var_min = params->var_min;
  m->min_range = params->min_range; m->max_range = params->max_range; m->k = params->mahalanobis_k;
  m->v_out = params->outlier_variance; m->sigma_t2 = params->time_variance; m->ray_step = params->ray_step;
  m->alpha_n = params->cleanup_normal_thresh; m->wall = params->wall_num_thresh;
  m->min_age = params->cleanup_min_age;
  m->drift_flat = params->drift_flatness;
  m->excl_b = params->excl_b; m->excl_c = params->excl_c; m->excl_d = params->excl_d;
  m->excl_tan = (float)std::tan((double)params->excl_theta);
  m->ovl_r2 = params->overlap_radius * params->overlap_radius; m->ovl_dz = params->overlap_dz;
  m->ref_x = clouds[0].pose[3];
  m->ref_y = clouds[0].pose[7];
  int64_t begin = 0;
  for (int i = 0; i < n_clouds; ++i) {
    cd[i].pts = clouds[i].points;
    cd[i].n = clouds[i].n;
    cd[i].begin = begin;
    cd[i].stride = clouds[i].stride;
    cd[i].map = 0;
    for (int row = 0; row < 3; ++row) {
      for (int k = 0; k < 3; ++k) cd[i].R[row * 3 + k] = clouds[i].pose[row * 4 + k];
      cd[i].t[row] = clouds[i].pose[row * 4 + 3];
    }
    begin += clouds[i].n;
  }
  b->n_maps = 1;
  b->n_clouds = n_clouds;
  b->n_points = total;
  b->maps = reinterpret_cast<const MapDev*>(base + kOffDesc + offsetof(Desc, m));
  b->clouds = reinterpret_cast<const CloudDev*>(base + kOffDesc + offsetof(Desc, c));
  b->rz = reinterpret_cast<float*>(base + kOffRz);
  b->rv = reinterpret_cast<float*>(base + kOffRv);
  b->rc = reinterpret_cast<uint16_t*>(base + kOffRc);
  b->tile_cnt = reinterpret_cast<int32_t*>(base + kOffTCnt);
  b->tile_base = reinterpret_cast<int32_t*>(base + kOffTBase);
  b->tile_cur = reinterpret_cast<int32_t*>(base + kOffTCur);
  b->tile_map = reinterpret_cast<int32_t*>(base + kOffTMap);
  b->heavy = reinterpret_cast<FuseItem*>(base + kOffHeavy);
  b->light = reinterpret_cast<FuseItem*>(base + kOffLight);
  b->n_cells = pad_tile(ncell);
  b->n_coarse = (int64_t)m->CW * m->CH;
  b->ctl = reinterpret_cast<BatchCtl*>(base + kOffBCtl);
  b->heavy_thresh = 4096;
  b->split_slots = 0;  // no tile is split: heavy tiles are fused whole
  b->fuse_threads = 256;

  const BatchDev* bd = reinterpret_cast<const BatchDev*>(base + kOffDesc + offsetof(Desc, b));
  k_put_desc<<<1, 128, 0, s>>>(desc);
  rc = na_status(cudaGetLastError(), "k_put_desc");
  if (rc) return rc;
  // counters, marks and per-tile counts start at zero
  rc = na_status(cudaMemsetAsync(base + kOffCtl, 0, kOffTBase - kOffCtl, s), "cudaMemsetAsync");
  if (rc) return rc;
  const int64_t cells = pad_tile(ncell);
  const bool ext = params->excl_d > 0.f;  // no upper-bound layer here
  cudaError_t e = launch_bin(bd, total, cells, ext, s);
  if (e == cudaSuccess && params->drift_flatness > 0.f) e = launch_drift(bd, total, cells, ext, s);
  if (total > 0) {
    if (e == cudaSuccess && params->ray_step > 0.f) e = launch_ray(bd, total, cells, 8, ext, s);
    if (e == cudaSuccess) e = launch_alloc(bd, cells, s);
    if (e == cudaSuccess) e = launch_scatter(bd, total, ext, s);
    if (e == cudaSuccess) e = launch_fuse(bd, cells, 256, s);
  }
  if (e == cudaSuccess) e = launch_clear(bd, cells, s);
  if (e == cudaSuccess && params->overlap_dz > 0.f) e = launch_overlap(bd, cells, s);
  return na_status(e, "em_update_noalloc launch");
}
