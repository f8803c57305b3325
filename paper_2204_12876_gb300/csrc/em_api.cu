// em_api.cu -- host runtime and C ABI of libem.so (declared in include/em.h).
//
// A map owns its layers (physical ring layout), per-cell scratch, a per-update
// workspace that grows on demand, and a small ring of update descriptors
// (pinned host + device copies, each guarded by an event) so that em_update
// returns without waiting for the GPU.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "em.h"
#include "em_internal.cuh"

using namespace em;

namespace {

thread_local char g_cuda_msg[256] = "";

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return EM_OK;
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? EM_ERR_OOM : EM_ERR_CUDA;
}

#define EM_TRY(expr, what)                           \
  do {                                               \
    int _rc = cuda_status((expr), (what));           \
    if (_rc != EM_OK) return _rc;                    \
  } while (0)

constexpr int kSlots = 4;
constexpr int kMaxClouds = 64;
constexpr size_t kDescBytes = sizeof(BatchDev) + sizeof(MapDev) + kMaxClouds * sizeof(CloudDev) + 64;

template <class T>
cudaError_t dev_alloc(T** p, size_t count, int64_t* total) {
  size_t bytes = (count ? count : 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess && total) *total += (int64_t)bytes;
  return e;
}

int set_device(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) EM_TRY(cudaSetDevice(dev), "cudaSetDevice");
  return EM_OK;
}

}  // namespace

struct em_map {
  em_params p{};
  int device = 0;
  // layers (physical ring layout)
  float* h = nullptr;
  float* var = nullptr;
  int32_t* t_last = nullptr;
  float* nx = nullptr;
  float* ny = nullptr;
  float* nz = nullptr;
  float* smooth = nullptr;
  float* inpaint = nullptr;
  float* upper = nullptr;
  // per-cell scratch
  uint32_t* mark = nullptr;
  float* thr = nullptr;
  float* cthr = nullptr;  // coarse grid of the ray thresholds (maps with the ray march)
  int32_t* tile_cnt = nullptr;   // per tile of 1024 cells: record counts, ranges, claims
  int32_t* tile_base = nullptr;
  int32_t* tile_cur = nullptr;
  int32_t* tile_map = nullptr;
  FuseItem* heavy = nullptr;                // the fusion's work lists (one entry per tile)
  FuseItem* light = nullptr;
  unsigned long long* split_acc = nullptr;  // accumulator slots of split tiles (zero between updates)
  int32_t* split_done = nullptr;
  int32_t split_slots = 0;
  FuseItem* pieces = nullptr;               // piece list (with the record workspace)
  int32_t max_pieces = 0;
  MapCtl* ctl = nullptr;
  BatchCtl* bctl = nullptr;
  // geometry
  int32_t ox = 0, oy = 0;
  int64_t shift_x = 0, shift_y = 0;
  int32_t t_now = 0;
  // per-update workspace
  int64_t cap = 0;
  float* rz = nullptr;
  float* rv = nullptr;
  uint16_t* rc = nullptr;
  int32_t* idx_sorted = nullptr;
  int32_t* tr_ix = nullptr;
  int32_t* tr_iy = nullptr;
  uint8_t* tr_status = nullptr;
  int64_t last_n = 0;
  // descriptors
  unsigned char* desc_host = nullptr;
  unsigned char* desc_dev = nullptr;
  cudaEvent_t desc_ev[kSlots] = {};
  int slot = 0;
  // host staging for em_update_host
  float* host_stage = nullptr;
  float* dev_stage = nullptr;
  int64_t stage_cap = 0;  // floats
  cudaEvent_t stage_ev = nullptr;
  // layer staging
  float* layer_stage = nullptr;
  size_t layer_stage_cap = 0;
  cudaStream_t last_stream = nullptr;
  cudaStream_t side = nullptr;  // the ray march, beside the sort and fusion (maps with a ray step)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int64_t layer_bytes = 0;
  int64_t work_bytes = 0;
  int fuse_threads = 512;
  int ray_group = 8;
  int heavy_thresh = 256 * 16;
  int64_t points_in = 0;
  // per-kernel profiling
  bool prof = false;
  bool prof_pending = false;
  cudaEvent_t prof_ev[2 * EM_PROF_SLOTS] = {};
  bool prof_used[EM_PROF_SLOTS] = {};
  double prof_ms[EM_PROF_SLOTS] = {};
  int64_t prof_n[EM_PROF_SLOTS] = {};
};

namespace {

void host_origin(const em_map* m, double* x0, double* y0) {
  const double r = (double)m->p.resolution;
  *x0 = r * ((double)m->shift_x - 0.5 * m->p.width);
  *y0 = r * ((double)m->shift_y - 0.5 * m->p.height);
}

MapDev make_mapdev(const em_map* m) {
  MapDev d;
  memset(&d, 0, sizeof(d));
  d.h = m->h; d.var = m->var; d.t_last = m->t_last;
  d.nx = m->nx; d.ny = m->ny; d.nz = m->nz; d.smooth = m->smooth; d.inpaint = m->inpaint; d.upper = m->upper;
  d.mark = m->mark; d.thr = m->thr; d.cthr = m->cthr;
  if (m->cthr) {
    d.CW = coarse_dim(m->p.width);
    d.CH = coarse_dim(m->p.height);
  }
  d.ctl = m->ctl;
  d.cell_begin = 0;
  d.W = m->p.width; d.H = m->p.height; d.ox = m->ox; d.oy = m->oy;
  double x0, y0;
  host_origin(m, &x0, &y0);
  d.x0 = (float)x0; d.y0 = (float)y0; d.res = m->p.resolution;
  d.inv_res = (float)(1.0 / (double)m->p.resolution);
  d.t_now = m->t_now;
  d.a0 = m->p.noise_a0; d.a1 = m->p.noise_a1; d.a2 = m->p.noise_a2; d.var_min = m->p.var_min;
  d.min_range = m->p.min_range; d.max_range = m->p.max_range; d.k = m->p.mahalanobis_k;
  d.v_out = m->p.outlier_variance; d.sigma_t2 = m->p.time_variance; d.ray_step = m->p.ray_step;
  d.alpha_n = m->p.cleanup_normal_thresh; d.wall = m->p.wall_num_thresh; d.min_age = m->p.cleanup_min_age;
  d.drift_flat = m->p.drift_flatness;
  d.excl_b = m->p.excl_b; d.excl_c = m->p.excl_c; d.excl_d = m->p.excl_d;
  d.excl_tan = (float)std::tan((double)m->p.excl_theta);
  d.ovl_r2 = m->p.overlap_radius * m->p.overlap_radius; d.ovl_dz = m->p.overlap_dz;
  d.flags = m->p.flags;
  return d;
}

bool params_ok(const em_params* p) {
  if (!p) return false;
  if (p->width < 1 || p->height < 1 || p->width > (1 << 22) || p->height > (1 << 22)) return false;
  if ((int64_t)p->width * p->height > (int64_t(1) << 26)) return false;
  if (!(std::isfinite(p->resolution) && p->resolution > 0.f)) return false;
  const float f[] = {p->noise_a0, p->noise_a1, p->noise_a2, p->var_min, p->min_range, p->mahalanobis_k,
                     p->outlier_variance, p->time_variance, p->ray_step, p->cleanup_normal_thresh};
  for (float v : f)
    if (!std::isfinite(v)) return false;
  if (!(p->var_min > 0.f)) return false;
  if (!(p->max_range >= p->min_range) || std::isnan(p->max_range)) return false;
  if (p->outlier_variance < 0.f || p->time_variance < 0.f || p->ray_step < 0.f) return false;
  if (p->wall_num_thresh < 0 || p->cleanup_min_age < 0) return false;
  const uint32_t sm = p->flags & (EM_F_SMOOTH | EM_F_MEDIAN | EM_F_GAUSS);
  if (sm & (sm - 1)) return false;  // one smoothing filter at most
  // drift compensation reads the normal layer of the previous update
  if (!(std::isfinite(p->drift_flatness) && p->drift_flatness >= 0.f && p->drift_flatness <= 1.f)) return false;
  if (p->drift_flatness > 0.f && !((p->flags & EM_F_NORMALS) || p->cleanup_normal_thresh > 0.f)) return false;
  const float g[] = {p->excl_b, p->excl_c, p->excl_theta, p->excl_d, p->overlap_radius, p->overlap_dz};
  for (float v : g)
    if (!std::isfinite(v)) return false;
  if (p->excl_d > 0.f && !(p->excl_theta > -1.5707963f && p->excl_theta < 1.5707963f)) return false;
  return true;
}

void free_workspace(em_map* m) {
  cudaFree(m->rz); cudaFree(m->rv); cudaFree(m->rc); cudaFree(m->idx_sorted);
  cudaFree(m->tr_ix); cudaFree(m->tr_iy); cudaFree(m->tr_status); cudaFree(m->pieces);
  m->rz = m->rv = nullptr; m->rc = nullptr; m->idx_sorted = nullptr; m->tr_ix = m->tr_iy = nullptr;
  m->tr_status = nullptr;
  m->pieces = nullptr;
  m->max_pieces = 0;
  m->cap = 0;
  m->work_bytes = 0;
}

int grow_workspace(em_map* m, int64_t n) {
  if (n <= m->cap) return EM_OK;
  if (n > (int64_t(1) << 31) - 1) return EM_ERR_CAPACITY;
  int64_t want = n + n / 4;
  if (want < 4096) want = 4096;
  if (want > (int64_t(1) << 31) - 1) want = (int64_t(1) << 31) - 1;
  EM_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  free_workspace(m);
  const bool trace = (m->p.flags & EM_F_TRACE) != 0;
  int64_t tot = 0;
  EM_TRY(dev_alloc(&m->rz, (size_t)want, &tot), "alloc workspace");
  EM_TRY(dev_alloc(&m->rv, (size_t)want, &tot), "alloc workspace");
  EM_TRY(dev_alloc(&m->rc, (size_t)want, &tot), "alloc workspace");
  // pieces: a split tile has more than 16 kMinHeavy records per piece but its last
  const int64_t np = want / (kMinHeavy * 16) + kMaxSplit + 1;
  EM_TRY(dev_alloc(&m->pieces, (size_t)np, &tot), "alloc workspace");
  m->max_pieces = (int32_t)np;
  if (trace) {
    EM_TRY(dev_alloc(&m->idx_sorted, (size_t)want, &tot), "alloc trace");
    EM_TRY(dev_alloc(&m->tr_ix, (size_t)want, &tot), "alloc trace");
    EM_TRY(dev_alloc(&m->tr_iy, (size_t)want, &tot), "alloc trace");
    EM_TRY(dev_alloc(&m->tr_status, (size_t)want, &tot), "alloc trace");
  }
  m->cap = want;
  m->work_bytes = tot;
  return EM_OK;
}

void release(em_map* m) {
  if (!m) return;
  for (int i = 0; i < 2 * EM_PROF_SLOTS; ++i)
    if (m->prof_ev[i]) cudaEventDestroy(m->prof_ev[i]);
  cudaFree(m->h); cudaFree(m->var); cudaFree(m->t_last);
  cudaFree(m->nx); cudaFree(m->ny); cudaFree(m->nz); cudaFree(m->smooth); cudaFree(m->inpaint); cudaFree(m->upper);
  cudaFree(m->mark); cudaFree(m->thr); cudaFree(m->cthr);
  cudaFree(m->tile_cnt); cudaFree(m->tile_base); cudaFree(m->tile_cur); cudaFree(m->tile_map);
  cudaFree(m->heavy); cudaFree(m->light);
  cudaFree(m->split_acc); cudaFree(m->split_done);
  cudaFree(m->ctl); cudaFree(m->bctl);
  if (m->side) cudaStreamDestroy(m->side);
  if (m->fork_ev) cudaEventDestroy(m->fork_ev);
  if (m->join_ev) cudaEventDestroy(m->join_ev);
  free_workspace(m);
  cudaFree(m->desc_dev);
  cudaFreeHost(m->desc_host);
  for (int i = 0; i < kSlots; ++i)
    if (m->desc_ev[i]) cudaEventDestroy(m->desc_ev[i]);
  cudaFreeHost(m->host_stage);
  cudaFree(m->dev_stage);
  if (m->stage_ev) cudaEventDestroy(m->stage_ev);
  cudaFree(m->layer_stage);
  delete m;
}

bool pose_ok(const float* pose) {
  if (!pose) return false;
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(pose[i])) return false;
  return true;
}

// Build and upload the descriptor of a one-map update; returns the device
// address of its BatchDev.
int upload_desc(em_map* m, const em_cloud* clouds, int32_t n_clouds, int64_t total, cudaStream_t s,
                const BatchDev** out) {
  const int slot = m->slot;
  m->slot = (m->slot + 1) % kSlots;
  EM_TRY(cudaEventSynchronize(m->desc_ev[slot]), "cudaEventSynchronize");
  unsigned char* hb = m->desc_host + (size_t)slot * kDescBytes;
  unsigned char* db = m->desc_dev + (size_t)slot * kDescBytes;
  BatchDev* b = reinterpret_cast<BatchDev*>(hb);
  MapDev* md = reinterpret_cast<MapDev*>(hb + sizeof(BatchDev));
  CloudDev* cd = reinterpret_cast<CloudDev*>(hb + sizeof(BatchDev) + sizeof(MapDev));
  memset(b, 0, sizeof(BatchDev));
  *md = make_mapdev(m);
  md->z_ref = n_clouds > 0 ? clouds[0].pose[11] : 0.f;  // the first cloud's sensor origin
  md->ref_x = n_clouds > 0 ? clouds[0].pose[3] : 0.f;
  md->ref_y = n_clouds > 0 ? clouds[0].pose[7] : 0.f;
  int64_t begin = 0;
  for (int i = 0; i < n_clouds; ++i) {
    CloudDev& c = cd[i];
    memset(&c, 0, sizeof(c));
    c.pts = clouds[i].points;
    c.n = clouds[i].n;
    c.begin = begin;
    c.stride = clouds[i].stride;
    c.map = 0;
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) c.R[r * 3 + k] = clouds[i].pose[r * 4 + k];
      c.t[r] = clouds[i].pose[r * 4 + 3];
    }
    begin += clouds[i].n;
  }
  b->n_maps = 1;
  b->n_clouds = n_clouds;
  b->n_points = total;
  b->maps = reinterpret_cast<const MapDev*>(db + sizeof(BatchDev));
  b->clouds = reinterpret_cast<const CloudDev*>(db + sizeof(BatchDev) + sizeof(MapDev));
  b->rz = m->rz;
  b->rv = m->rv;
  b->rc = m->rc;
  b->idx_sorted = m->idx_sorted;
  b->tr_ix = m->tr_ix;
  b->tr_iy = m->tr_iy;
  b->tr_status = m->tr_status;
  b->n_cells = pad_tile((int64_t)m->p.width * m->p.height);
  b->n_coarse = (int64_t)md->CW * md->CH;
  b->ctl = m->bctl;
  b->tile_cnt = m->tile_cnt;
  b->tile_base = m->tile_base;
  b->tile_cur = m->tile_cur;
  b->tile_map = m->tile_map;
  b->heavy = m->heavy;
  b->light = m->light;
  b->pieces = m->pieces;
  b->max_pieces = m->max_pieces;
  b->split_acc = m->split_acc;
  b->split_done = m->split_done;
  b->split_slots = m->split_slots;
  b->heavy_thresh = m->heavy_thresh;
  b->fuse_threads = m->fuse_threads;
  const size_t bytes = sizeof(BatchDev) + sizeof(MapDev) + (size_t)n_clouds * sizeof(CloudDev);
  EM_TRY(cudaMemcpyAsync(db, hb, bytes, cudaMemcpyHostToDevice, s), "upload descriptor");
  *out = reinterpret_cast<const BatchDev*>(db);
  return slot;
}

// Fold the previous update's kernel timings into the accumulators.
int prof_collect(em_map* m) {
  if (!m->prof_pending) return EM_OK;
  m->prof_pending = false;
  for (int k = 0; k < EM_PROF_SLOTS; ++k) {
    if (!m->prof_used[k]) continue;
    m->prof_used[k] = false;
    EM_TRY(cudaEventSynchronize(m->prof_ev[2 * k + 1]), "cudaEventSynchronize");
    float ms = 0.f;
    EM_TRY(cudaEventElapsedTime(&ms, m->prof_ev[2 * k], m->prof_ev[2 * k + 1]), "cudaEventElapsedTime");
    m->prof_ms[k] += ms;
    m->prof_n[k] += 1;
  }
  return EM_OK;
}

// Launch through `fn` with profiling events around it when enabled.
template <class F>
cudaError_t timed(em_map* m, int slot, cudaStream_t s, F fn) {
  if (!m->prof) return fn();
  cudaEventRecord(m->prof_ev[2 * slot], s);
  cudaError_t e = fn();
  cudaEventRecord(m->prof_ev[2 * slot + 1], s);
  m->prof_used[slot] = true;
  m->prof_pending = true;
  return e;
}

}  // namespace

// ---- internal accessors for the batched and served forms (em_host.h)
namespace em {

int map_device(const em_map* m) { return m->device; }
uint32_t map_flags(const em_map* m) { return m->p.flags; }
int32_t map_cells(const em_map* m) { return m->p.width * m->p.height; }
const em_params& map_params(const em_map* m) { return m->p; }

MapDev map_begin_update(em_map* m, int64_t points) {
  m->t_now += 1;
  m->points_in += points;
  return make_mapdev(m);
}

void map_end_update(em_map* m, cudaStream_t s, int64_t points) {
  m->last_stream = s;
  m->last_n = points;
}

void map_undo_update(em_map* m, int64_t points) {
  m->t_now -= 1;
  m->points_in -= points;
}

int map_copy_state(em_map* dst, const em_map* src, cudaStream_t s) {
  if (dst->p.width != src->p.width || dst->p.height != src->p.height) return EM_ERR_INVALID_ARG;
  const size_t nc = (size_t)src->p.width * src->p.height;
  EM_TRY(cudaMemcpyAsync(dst->h, src->h, nc * 4, cudaMemcpyDeviceToDevice, s), "copy state");
  EM_TRY(cudaMemcpyAsync(dst->var, src->var, nc * 4, cudaMemcpyDeviceToDevice, s), "copy state");
  EM_TRY(cudaMemcpyAsync(dst->t_last, src->t_last, nc * 4, cudaMemcpyDeviceToDevice, s), "copy state");
  if (dst->nx && src->nx) {
    EM_TRY(cudaMemcpyAsync(dst->nx, src->nx, nc * 4, cudaMemcpyDeviceToDevice, s), "copy state");
    EM_TRY(cudaMemcpyAsync(dst->ny, src->ny, nc * 4, cudaMemcpyDeviceToDevice, s), "copy state");
    EM_TRY(cudaMemcpyAsync(dst->nz, src->nz, nc * 4, cudaMemcpyDeviceToDevice, s), "copy state");
  }
  dst->ox = src->ox;
  dst->oy = src->oy;
  dst->shift_x = src->shift_x;
  dst->shift_y = src->shift_y;
  dst->t_now = src->t_now;
  return EM_OK;
}

int map_record_error(const char* what, cudaError_t e) { return cuda_status(e, what); }

int map_read_layers(em_map* m, uint32_t mask, float* dst, cudaStream_t s) {
  EM_TRY(launch_layers_out(make_mapdev(m), mask, dst, s), "k_layers_out");
  m->last_stream = s;
  return EM_OK;
}

int maps_read_layers(em_map* const* maps, const uint32_t* masks, float* const* dst, int n, cudaStream_t s) {
  ReadJobs jobs;
  for (int i0 = 0; i0 < n; i0 += kMaxReadJobs) {
    jobs.n = std::min(kMaxReadJobs, n - i0);
    for (int i = 0; i < jobs.n; ++i) {
      jobs.job[i].m = make_mapdev(maps[i0 + i]);
      jobs.job[i].mask = masks[i0 + i];
      jobs.job[i].dst = dst[i0 + i];
      maps[i0 + i]->last_stream = s;
    }
    EM_TRY(launch_layers_out_multi(jobs, s), "k_layers_out_multi");
  }
  return EM_OK;
}

}  // namespace em

extern "C" {

const char* em_status_str(int status) {
  switch (status) {
    case EM_OK: return "ok";
    case EM_ERR_INVALID_ARG: return "invalid argument";
    case EM_ERR_OOM: return "out of memory";
    case EM_ERR_CUDA: return "CUDA error";
    case EM_ERR_TIMEOUT: return "timeout";
    case EM_ERR_REJECTED: return "rejected by admission";
    case EM_ERR_BUSY: return "busy";
    case EM_ERR_CAPACITY: return "capacity exceeded";
    default: return "unknown status";
  }
}

const char* em_last_cuda_error(void) { return g_cuda_msg; }

int em_create(const em_params* params, int device, em_map** out) {
  if (!out) return EM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params_ok(params)) return EM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EM_ERR_INVALID_ARG;
  int rc = set_device(device);
  if (rc) return rc;
  em_map* m = new (std::nothrow) em_map();
  if (!m) return EM_ERR_OOM;
  m->p = *params;
  m->device = device;
  const size_t nc = (size_t)params->width * params->height;
  int64_t tot = 0;
  const bool normals = (params->flags & EM_F_NORMALS) || params->cleanup_normal_thresh > 0.f;
  cudaError_t e = cudaSuccess;
#define EM_ALLOC(ptr, n)                                   \
  if (e == cudaSuccess) e = dev_alloc(&(ptr), (n), &tot);
  EM_ALLOC(m->h, nc) EM_ALLOC(m->var, nc) EM_ALLOC(m->t_last, nc)
  if (normals) { EM_ALLOC(m->nx, nc) EM_ALLOC(m->ny, nc) EM_ALLOC(m->nz, nc) }
  if (params->flags & (EM_F_SMOOTH | EM_F_MEDIAN | EM_F_GAUSS)) { EM_ALLOC(m->smooth, nc) }
  if (params->flags & EM_F_INPAINT) { EM_ALLOC(m->inpaint, nc) }
  if (params->flags & EM_F_UPPER) { EM_ALLOC(m->upper, nc) }
  const size_t ntile = (size_t)(pad_tile((int64_t)nc) / kTile);
  EM_ALLOC(m->mark, (nc + 31) / 32) EM_ALLOC(m->thr, nc)
  if (params->ray_step > 0.f) { EM_ALLOC(m->cthr, (size_t)coarse_dim(params->width) * coarse_dim(params->height)) }
  EM_ALLOC(m->tile_cnt, ntile + 1) EM_ALLOC(m->tile_base, ntile + 1) EM_ALLOC(m->tile_cur, ntile + 1)
  EM_ALLOC(m->tile_map, ntile) EM_ALLOC(m->heavy, ntile) EM_ALLOC(m->light, ntile)
  m->split_slots = (int32_t)(ntile < (size_t)kMaxSplit ? ntile : (size_t)kMaxSplit);
  EM_ALLOC(m->split_acc, (size_t)m->split_slots * kSplitWords * kTile) EM_ALLOC(m->split_done, m->split_slots)
  EM_ALLOC(m->ctl, 1) EM_ALLOC(m->bctl, 1)
  EM_ALLOC(m->desc_dev, kDescBytes * kSlots)
#undef EM_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost((void**)&m->desc_host, kDescBytes * kSlots);
  for (int i = 0; i < kSlots && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&m->desc_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->stage_ev, cudaEventDisableTiming);
  if (e == cudaSuccess && params->ray_step > 0.f) {
    e = cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->join_ev, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMemset(m->ctl, 0, sizeof(MapCtl));
  if (e == cudaSuccess) e = cudaMemset(m->tile_cnt, 0, (ntile + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(m->bctl, 0, sizeof(BatchCtl));
  if (e == cudaSuccess)
    e = cudaMemset(m->split_acc, 0, (size_t)m->split_slots * kSplitWords * kTile * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(m->split_done, 0, (size_t)m->split_slots * sizeof(int32_t));
  if (e == cudaSuccess) e = cuda_status(launch_fill_map(make_mapdev(m), nullptr), "fill") ? cudaErrorUnknown : cudaSuccess;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    int code = cuda_status(e, "em_create");
    release(m);
    return code;
  }
  m->layer_bytes = tot;
  // tuning knobs (defaults chosen by measurement; the environment overrides them)
  if (const char* g = getenv("EM_FUSE_THREADS")) {
    int v = atoi(g);
    if (v == 256 || v == 512) m->fuse_threads = v;
  }
  if (const char* g = getenv("EM_RAY_GROUP")) {
    int v = atoi(g);
    if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32) m->ray_group = v;
  }
  if (const char* g = getenv("EM_HEAVY_THRESH")) {
    int v = atoi(g);
    if (v >= kMinHeavy && v <= kMaxHeavy) m->heavy_thresh = v * 16;
  }
  *out = m;
  return EM_OK;
}

int em_destroy(em_map* m) {
  if (!m) return EM_OK;
  set_device(m->device);
  cudaDeviceSynchronize();
  release(m);
  return EM_OK;
}

int em_reserve(em_map* m, int64_t max_points) {
  if (!m || max_points < 0) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  return grow_workspace(m, max_points);
}

static int update_impl(em_map* m, const em_cloud* clouds, int32_t n_clouds, cudaStream_t s) {
  if (m->prof) {
    int prc = prof_collect(m);
    if (prc) return prc;
  }
  int64_t total = 0;
  for (int i = 0; i < n_clouds; ++i) total += clouds[i].n;
  int rc = grow_workspace(m, total);
  if (rc) return rc;
  m->t_now += 1;
  const BatchDev* bd = nullptr;
  int slot = upload_desc(m, clouds, n_clouds, total, s, &bd);
  if (slot < 0) {
    m->t_now -= 1;
    return slot;
  }
  const int64_t ncell = pad_tile((int64_t)m->p.width * m->p.height);
  const bool ext = m->p.excl_d > 0.f || (m->p.flags & EM_F_UPPER);  // kernels with the extended features
  EM_TRY(timed(m, EM_PROF_COUNT, s, [&] { return launch_bin(bd, total, ncell, ext, s); }), "k_count");
  if (m->p.drift_flatness > 0.f)
    EM_TRY(timed(m, EM_PROF_DRIFT, s, [&] { return launch_drift(bd, total, ncell, ext, s); }), "k_drift");
  if (total > 0) {
    // the ray march reads only the ray thresholds and the points and writes only
    // the marks (read by k_clear): it runs on the side stream beside the sort and
    // the fusion, unless the map has the upper-bound layer (both write it)
    auto ray = [&](cudaStream_t rs) {
      return timed(m, EM_PROF_RAY, rs, [&] { return launch_ray(bd, total, ncell, m->ray_group, ext, rs); });
    };
    auto rest = [&] {
      cudaError_t r = timed(m, EM_PROF_ALLOC, s, [&] { return launch_alloc(bd, ncell, s); });
      if (r == cudaSuccess) r = timed(m, EM_PROF_SCATTER, s, [&] { return launch_scatter(bd, total, ext, s); });
      if (r == cudaSuccess) r = timed(m, EM_PROF_FUSE, s, [&] { return launch_fuse(bd, ncell, m->fuse_threads, s); });
      return r;
    };
    if (m->p.ray_step > 0.f && !(m->p.flags & EM_F_UPPER)) {
      EM_TRY(launch_beside(s, m->side, m->fork_ev, m->join_ev, ray, rest), "k_ray / k_alloc / k_scatter / k_fuse");
    } else {
      if (m->p.ray_step > 0.f) EM_TRY(ray(s), "k_ray");
      EM_TRY(rest(), "k_alloc / k_scatter / k_fuse");
    }
  }
  EM_TRY(timed(m, EM_PROF_CLEAR, s, [&] { return launch_clear(bd, ncell, s); }), "k_clear");
  if (m->p.overlap_dz > 0.f && n_clouds > 0)
    EM_TRY(timed(m, EM_PROF_OVERLAP, s, [&] { return launch_overlap(bd, ncell, s); }), "k_overlap");
  if (m->p.flags & EM_F_NORMALS)
    EM_TRY(timed(m, EM_PROF_NORMALS, s, [&] { return launch_normals(bd, ncell, s); }), "k_normals");
  if (m->p.flags & (EM_F_SMOOTH | EM_F_MEDIAN | EM_F_GAUSS))
    EM_TRY(timed(m, EM_PROF_SMOOTH, s, [&] { return launch_smooth(bd, ncell, s); }), "k_smooth");
  if (m->p.flags & EM_F_INPAINT)
    EM_TRY(timed(m, EM_PROF_INPAINT, s, [&] { return launch_inpaint(bd, ncell, s); }), "k_inpaint");
  EM_TRY(cudaEventRecord(m->desc_ev[slot], s), "cudaEventRecord");
  m->last_stream = s;
  m->last_n = total;
  m->points_in += total;
  return EM_OK;
}

static int check_clouds(const em_cloud* clouds, int32_t n_clouds) {
  if (n_clouds < 1 || n_clouds > kMaxClouds || !clouds) return EM_ERR_INVALID_ARG;
  for (int i = 0; i < n_clouds; ++i) {
    const em_cloud& c = clouds[i];
    if (c.n < 0 || (c.stride != 3 && c.stride != 4) || (c.n > 0 && !c.points) || !word_aligned(c.points) ||
        !pose_ok(c.pose))
      return EM_ERR_INVALID_ARG;
  }
  return EM_OK;
}

int em_update_multi(em_map* m, const em_cloud* clouds, int32_t n_clouds, em_stream_t stream) {
  if (!m) return EM_ERR_INVALID_ARG;
  int rc = check_clouds(clouds, n_clouds);
  if (rc) return rc;
  rc = set_device(m->device);
  if (rc) return rc;
  return update_impl(m, clouds, n_clouds, (cudaStream_t)stream);
}

int em_update(em_map* m, const float* points, int64_t n, int32_t stride, const float pose[12], em_stream_t stream) {
  if (!m || !pose) return EM_ERR_INVALID_ARG;
  em_cloud c;
  c.points = points;
  c.n = n;
  c.stride = stride;
  memcpy(c.pose, pose, sizeof(c.pose));
  return em_update_multi(m, &c, 1, stream);
}

int em_update_host(em_map* m, const em_cloud* clouds, int32_t n_clouds, em_stream_t stream) {
  if (!m) return EM_ERR_INVALID_ARG;
  int rc = check_clouds(clouds, n_clouds);
  if (rc) return rc;
  rc = set_device(m->device);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t floats = 0;
  for (int i = 0; i < n_clouds; ++i) floats += clouds[i].n * clouds[i].stride;
  EM_TRY(cudaEventSynchronize(m->stage_ev), "cudaEventSynchronize");
  if (floats > m->stage_cap) {
    int64_t want = floats + floats / 4 + 1024;
    cudaFreeHost(m->host_stage);
    cudaFree(m->dev_stage);
    m->host_stage = nullptr;
    m->dev_stage = nullptr;
    m->stage_cap = 0;
    EM_TRY(cudaMallocHost((void**)&m->host_stage, (size_t)want * sizeof(float)), "cudaMallocHost");
    EM_TRY(cudaMalloc((void**)&m->dev_stage, (size_t)want * sizeof(float)), "cudaMalloc");
    m->stage_cap = want;
  }
  em_cloud local[kMaxClouds];
  int64_t off = 0;
  for (int i = 0; i < n_clouds; ++i) {
    const size_t nf = (size_t)(clouds[i].n * clouds[i].stride);
    if (nf) memcpy(m->host_stage + off, clouds[i].points, nf * sizeof(float));
    local[i] = clouds[i];
    local[i].points = m->dev_stage + off;
    off += (int64_t)nf;
    off = (off + 3) & ~int64_t(3);  // keep every cloud 16-byte aligned
  }
  if (off) EM_TRY(cudaMemcpyAsync(m->dev_stage, m->host_stage, (size_t)off * sizeof(float), cudaMemcpyHostToDevice, s),
                  "upload points");
  rc = update_impl(m, local, n_clouds, s);
  if (rc) return rc;
  EM_TRY(cudaEventRecord(m->stage_ev, s), "cudaEventRecord");
  return EM_OK;
}

int em_shift(em_map* m, int32_t dx, int32_t dy, em_stream_t stream) {
  if (!m) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t W = m->p.width, H = m->p.height;
  m->shift_x += dx;
  m->shift_y += dy;
  if ((int64_t)dx >= W || (int64_t)dx <= -W || (int64_t)dy >= H || (int64_t)dy <= -H) {
    m->ox = 0;
    m->oy = 0;
    EM_TRY(launch_fill_map(make_mapdev(m), s), "k_fill");
  } else {
    m->ox = (int32_t)((((int64_t)m->ox + dx) % W + W) % W);
    m->oy = (int32_t)((((int64_t)m->oy + dy) % H + H) % H);
    EM_TRY(launch_shift_clear(make_mapdev(m), dx, dy, s), "k_shift");
  }
  m->last_stream = s;
  return EM_OK;
}

static int ensure_layer_stage(em_map* m, size_t floats) {
  if (floats <= m->layer_stage_cap) return EM_OK;
  EM_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  cudaFree(m->layer_stage);
  m->layer_stage = nullptr;
  m->layer_stage_cap = 0;
  EM_TRY(cudaMalloc((void**)&m->layer_stage, floats * sizeof(float)), "cudaMalloc");
  m->layer_stage_cap = floats;
  return EM_OK;
}

int em_get_layers(em_map* m, uint32_t mask, float* dst, int dst_is_host, em_stream_t stream) {
  if (!m || !dst || !mask || (mask >> 11) || !word_aligned(dst)) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t floats = (size_t)__builtin_popcount(mask) * m->p.width * m->p.height;
  if (!dst_is_host) {
    EM_TRY(launch_layers_out(make_mapdev(m), mask, dst, s), "k_layers_out");
    m->last_stream = s;
    return EM_OK;
  }
  rc = ensure_layer_stage(m, floats);
  if (rc) return rc;
  EM_TRY(launch_layers_out(make_mapdev(m), mask, m->layer_stage, s), "k_layers_out");
  EM_TRY(cudaMemcpyAsync(dst, m->layer_stage, floats * sizeof(float), cudaMemcpyDeviceToHost, s), "download layers");
  EM_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return EM_OK;
}

int em_set_layers(em_map* m, uint32_t mask, const float* src, int src_is_host, em_stream_t stream) {
  const uint32_t allowed = EM_LAYER_ELEVATION | EM_LAYER_VARIANCE | EM_LAYER_TIME | EM_LAYER_NORMAL_X |
                           EM_LAYER_NORMAL_Y | EM_LAYER_NORMAL_Z | EM_LAYER_UPPER;
  if (!m || !src || !mask || (mask & ~allowed) || !word_aligned(src)) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t floats = (size_t)__builtin_popcount(mask) * m->p.width * m->p.height;
  const float* from = src;
  if (src_is_host) {
    rc = ensure_layer_stage(m, floats);
    if (rc) return rc;
    EM_TRY(cudaMemcpyAsync(m->layer_stage, src, floats * sizeof(float), cudaMemcpyHostToDevice, s), "upload layers");
    from = m->layer_stage;
  }
  EM_TRY(launch_layers_in(make_mapdev(m), mask, from, s), "k_layers_in");
  if (src_is_host) EM_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  m->last_stream = s;
  return EM_OK;
}

int em_set_time(em_map* m, int32_t t_now) {
  if (!m || t_now < 0) return EM_ERR_INVALID_ARG;
  m->t_now = t_now;
  return EM_OK;
}

int em_get_info(const em_map* m, em_info* out) {
  if (!m || !out) return EM_ERR_INVALID_ARG;
  out->width = m->p.width;
  out->height = m->p.height;
  out->resolution = m->p.resolution;
  out->t_now = m->t_now;
  out->shift_x = m->shift_x;
  out->shift_y = m->shift_y;
  host_origin(m, &out->x0, &out->y0);
  out->point_capacity = m->cap;
  out->device_bytes = m->layer_bytes + m->work_bytes + (int64_t)m->layer_stage_cap * 4 + m->stage_cap * 4;
  return EM_OK;
}

int em_sync(em_map* m) {
  if (!m) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  EM_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  int32_t err = 0;
  EM_TRY(cudaMemcpy(&err, &m->ctl->err, sizeof(err), cudaMemcpyDeviceToHost), "read error word");
  if (err) {
    int32_t zero = 0;
    cudaMemcpy(&m->ctl->err, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    return err;
  }
  return EM_OK;
}

int em_get_stats(em_map* m, em_stats* out) {
  if (!m || !out) return EM_ERR_INVALID_ARG;
  int rc = em_sync(m);
  MapCtl ctl;
  int rc2 = cuda_status(cudaMemcpy(&ctl, m->ctl, sizeof(ctl), cudaMemcpyDeviceToHost), "read stats");
  if (rc2) return rc2;
  out->updates = (int64_t)ctl.stats[kStUpdates];
  out->points_in = m->points_in;
  out->points_valid = (int64_t)ctl.stats[kStValid];
  out->points_in_map = (int64_t)ctl.stats[kStInMap];
  out->points_accepted = (int64_t)ctl.stats[kStAccepted];
  out->points_rejected = (int64_t)ctl.stats[kStRejected];
  out->points_wall = (int64_t)ctl.stats[kStWall];
  out->cells_updated = (int64_t)ctl.stats[kStCellsUpdated];
  out->cells_cleared = (int64_t)ctl.stats[kStCleared];
  out->ray_samples = (int64_t)ctl.stats[kStRaySamples];
  out->drift_points = (int64_t)ctl.stats[kStDriftPoints];
  out->drift_last = (double)ctl.drift_last;
  return rc;
}

int em_get_trace(em_map* m, int32_t* ix, int32_t* iy, uint8_t* status, int64_t n) {
  if (!m || !(m->p.flags & EM_F_TRACE) || n != m->last_n || (n > 0 && (!ix || !iy || !status)))
    return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  EM_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if (n == 0) return EM_OK;
  EM_TRY(cudaMemcpy(ix, m->tr_ix, (size_t)n * 4, cudaMemcpyDeviceToHost), "trace");
  EM_TRY(cudaMemcpy(iy, m->tr_iy, (size_t)n * 4, cudaMemcpyDeviceToHost), "trace");
  EM_TRY(cudaMemcpy(status, m->tr_status, (size_t)n, cudaMemcpyDeviceToHost), "trace");
  return EM_OK;
}

int em_profile(em_map* m, int enable) {
  if (!m) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  if (enable && !m->prof_ev[0]) {
    for (int i = 0; i < 2 * EM_PROF_SLOTS; ++i) EM_TRY(cudaEventCreate(&m->prof_ev[i]), "cudaEventCreate");
  }
  if (!enable) {
    rc = prof_collect(m);
    if (rc) return rc;
  }
  if (enable && !m->prof) {
    for (int k = 0; k < EM_PROF_SLOTS; ++k) { m->prof_ms[k] = 0.0; m->prof_n[k] = 0; }
  }
  m->prof = enable != 0;
  return EM_OK;
}

int em_profile_read(em_map* m, double* ms, int64_t* launches) {
  if (!m || !ms || !launches) return EM_ERR_INVALID_ARG;
  int rc = set_device(m->device);
  if (rc) return rc;
  rc = prof_collect(m);
  if (rc) return rc;
  for (int k = 0; k < EM_PROF_SLOTS; ++k) {
    ms[k] = m->prof_ms[k];
    launches[k] = m->prof_n[k];
  }
  return EM_OK;
}

}  // extern "C"
