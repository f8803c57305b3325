// em_batch.cu -- the batched form: many maps updated by one kernel sequence.
//
// Every kernel of the update already works on a list of maps and clouds (the
// device descriptor), so a batch is the same launch sequence as one em_update
// with more maps in the descriptor: per-point kernels span all clouds of all
// maps, per-cell kernels walk the tiles of all maps' cells.  With EM_BATCH_GRAPH the
// sequence is captured once per descriptor slot (grids sized from the batch
// capacities) and replayed by one cudaGraphLaunch.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "em.h"
#include "em_host.h"
#include "em_internal.cuh"

using namespace em;

namespace {

constexpr int kSlots = 3;

#define EB_TRY(expr, what)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return map_record_error((what), _e); \
  } while (0)

bool tuning_ok(const em_tuning& t) {
  const int r = t.ray_group, f = t.fuse_chunk;
  return (r == 1 || r == 2 || r == 4 || r == 8 || r == 16 || r == 32) && f >= 64 && f <= 1024 && (f & (f - 1)) == 0 &&
         t.big_thresh >= kMinHeavy && t.big_thresh <= kMaxHeavy;
}

// what a captured graph depends on besides the slot
struct GraphKey {
  em_tuning t;
  bool ray;
  bool drift;
  bool overlap;
  bool ext;    // some map uses the exclusion area or the upper-bound layer
  bool upper;  // some map has the upper-bound layer (the ray march then runs before the fusion)
  uint32_t stencils;
  bool operator==(const GraphKey& o) const {
    return t.ray_group == o.t.ray_group && t.fuse_chunk == o.t.fuse_chunk && t.big_thresh == o.t.big_thresh &&
           ray == o.ray && drift == o.drift && overlap == o.overlap && ext == o.ext && upper == o.upper &&
           stencils == o.stencils;
  }
};

}  // namespace

struct em_batch {
  int device = 0;
  int32_t max_maps = 0, max_clouds = 0, max_cells = 0;
  int64_t max_points = 0;
  uint32_t flags = 0;
  float* rz = nullptr;  // records (k_sort.cu layout), max_points of each
  float* rv = nullptr;
  uint16_t* rc = nullptr;
  BatchCtl* bctl = nullptr;
  int64_t max_tiles = 0;  // tiles of the padded cell space of a full batch
  int32_t* tile_cnt = nullptr;
  int32_t* tile_base = nullptr;
  int32_t* tile_cur = nullptr;
  int32_t* tile_map = nullptr;
  FuseItem* heavy = nullptr;  // the fusion's work lists (one entry per tile)
  FuseItem* light = nullptr;
  unsigned long long* split_acc = nullptr;  // accumulator slots of split tiles (zero between updates)
  int32_t* split_done = nullptr;
  int32_t split_slots = 0;
  FuseItem* pieces = nullptr;
  int32_t max_pieces = 0;
  size_t desc_bytes = 0;
  unsigned char* desc_host = nullptr;
  unsigned char* desc_dev = nullptr;
  cudaEvent_t ev[kSlots] = {};
  int slot = 0;
  em_tuning tune{8, 512, 256};
  cudaStream_t capture_stream = nullptr;
  cudaStream_t side = nullptr;  // the ray march, beside the sort and fusion
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t graph[kSlots] = {};
  GraphKey graph_key[kSlots] = {};
  // host scratch for grouping
  std::vector<int> first_of, order, map_of;
  std::vector<em_map*> uniq;
  // per-kernel profiling
  bool prof = false;
  bool prof_pending = false;
  cudaEvent_t pev[2 * EM_PROF_SLOTS] = {};
  bool pused[EM_PROF_SLOTS] = {};
  double pms[EM_PROF_SLOTS] = {};
  int64_t pn[EM_PROF_SLOTS] = {};
};

namespace {

// Events around one launch when the batch is profiling (prof may be null).
template <class F>
cudaError_t timed(em_batch* prof, int slot, cudaStream_t s, F fn) {
  if (!prof || !prof->prof) return fn();
  cudaEventRecord(prof->pev[2 * slot], s);
  cudaError_t e = fn();
  cudaEventRecord(prof->pev[2 * slot + 1], s);
  prof->pused[slot] = true;
  prof->prof_pending = true;
  return e;
}

int prof_collect(em_batch* b) {
  if (!b->prof_pending) return EM_OK;
  b->prof_pending = false;
  for (int k = 0; k < EM_PROF_SLOTS; ++k) {
    if (!b->pused[k]) continue;
    b->pused[k] = false;
    EB_TRY(cudaEventSynchronize(b->pev[2 * k + 1]), "cudaEventSynchronize");
    float ms = 0.f;
    EB_TRY(cudaEventElapsedTime(&ms, b->pev[2 * k], b->pev[2 * k + 1]), "cudaEventElapsedTime");
    b->pms[k] += ms;
    b->pn[k] += 1;
  }
  return EM_OK;
}

// The kernel sequence of one update over the descriptor at `bd`.  The ray
// march reads only the ray thresholds (k_count / k_drift) and the points, and
// writes only the visibility marks (read by k_clear), so it runs on the side
// stream beside the sort and the fusion -- unless a map has the upper-bound
// layer, which both the march and the fusion write.
cudaError_t launch_sequence(em_batch* b, const BatchDev* bd, int64_t grid_points, int64_t grid_cells,
                            const GraphKey& k, cudaStream_t s, em_batch* prof = nullptr) {
  cudaError_t e = cudaSuccess;
  // EM_BATCH_PERSISTENT: the update's passes in one launch (k_persist.cu), when
  // the device can run it and no map needs the drift compensation
  bool persisted = false;
  if ((b->flags & EM_BATCH_PERSISTENT) && !k.drift) {
    e = timed(prof, EM_PROF_PERSIST, s, [&] { return launch_persist(bd, k.t.ray_group, k.ext, EM_PERSIST_WAIT_MS, s); });
    persisted = e != cudaErrorNotSupported;
    if (!persisted) {
      cudaGetLastError();
      e = cudaSuccess;
    }
  }
  if (!persisted) {
    e = timed(prof, EM_PROF_COUNT, s, [&] { return launch_bin(bd, grid_points, grid_cells, k.ext, s); });
    if (e == cudaSuccess && k.drift)
      e = timed(prof, EM_PROF_DRIFT, s, [&] { return launch_drift(bd, grid_points, grid_cells, k.ext, s); });
    if (grid_points > 0) {
      auto ray = [&](cudaStream_t rs) {
        return timed(prof, EM_PROF_RAY, rs,
                     [&] { return launch_ray(bd, grid_points, grid_cells, k.t.ray_group, k.ext, rs); });
      };
      auto rest = [&] {
        cudaError_t r = timed(prof, EM_PROF_ALLOC, s, [&] { return launch_alloc(bd, grid_cells, s); });
        if (r == cudaSuccess)
          r = timed(prof, EM_PROF_SCATTER, s, [&] { return launch_scatter(bd, grid_points, k.ext, s); });
        if (r == cudaSuccess)
          r = timed(prof, EM_PROF_FUSE, s, [&] { return launch_fuse(bd, grid_cells, k.t.fuse_chunk, s); });
        return r;
      };
      if (e == cudaSuccess) {
        if (k.ray && !k.upper) {
          e = launch_beside(s, b->side, b->fork_ev, b->join_ev, ray, rest);
        } else {
          if (k.ray) e = ray(s);
          if (e == cudaSuccess) e = rest();
        }
      }
    }
    if (e == cudaSuccess) e = timed(prof, EM_PROF_CLEAR, s, [&] { return launch_clear(bd, grid_cells, s); });
    if (e == cudaSuccess && k.overlap)
      e = timed(prof, EM_PROF_OVERLAP, s, [&] { return launch_overlap(bd, grid_cells, s); });
  }
  if (e == cudaSuccess && (k.stencils & EM_F_NORMALS))
    e = timed(prof, EM_PROF_NORMALS, s, [&] { return launch_normals(bd, grid_cells, s); });
  if (e == cudaSuccess && (k.stencils & (EM_F_SMOOTH | EM_F_MEDIAN | EM_F_GAUSS)))
    e = timed(prof, EM_PROF_SMOOTH, s, [&] { return launch_smooth(bd, grid_cells, s); });
  if (e == cudaSuccess && (k.stencils & EM_F_INPAINT))
    e = timed(prof, EM_PROF_INPAINT, s, [&] { return launch_inpaint(bd, grid_cells, s); });
  return e;
}

struct Prepared {
  const BatchDev* bd = nullptr;
  int slot = -1;
  int64_t points = 0;
  int32_t n_maps = 0;
  int64_t cells = 0;  // padded size of the cell space
  GraphKey key{};
};

// Group the pairs by map, build the descriptor in slot `slot` and upload it.
int prepare(em_batch* b, em_map* const* maps, const em_cloud* clouds, int32_t count, const em_tuning& tune,
            cudaStream_t s, Prepared* out) {
  if (!maps || !clouds || count < 1) return EM_ERR_INVALID_ARG;
  if (count > b->max_clouds) return EM_ERR_CAPACITY;
  b->uniq.clear();
  b->map_of.assign(count, -1);
  for (int i = 0; i < count; ++i) {
    const em_cloud& c = clouds[i];
    if (!maps[i] || c.n < 0 || (c.stride != 3 && c.stride != 4) || (c.n > 0 && !c.points) || !word_aligned(c.points))
      return EM_ERR_INVALID_ARG;
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(c.pose[k])) return EM_ERR_INVALID_ARG;
    if (map_device(maps[i]) != b->device) return EM_ERR_INVALID_ARG;
    int u = -1;
    for (size_t j = 0; j < b->uniq.size(); ++j)
      if (b->uniq[j] == maps[i]) { u = (int)j; break; }
    if (u < 0) {
      if ((int)b->uniq.size() >= b->max_maps) return EM_ERR_CAPACITY;
      if (map_cells(maps[i]) > b->max_cells) return EM_ERR_CAPACITY;
      u = (int)b->uniq.size();
      b->uniq.push_back(maps[i]);
    }
    b->map_of[i] = u;
  }
  const int nm = (int)b->uniq.size();
  std::vector<int64_t> map_pts(nm, 0);
  int64_t total = 0;
  for (int i = 0; i < count; ++i) {
    map_pts[b->map_of[i]] += clouds[i].n;
    total += clouds[i].n;
  }
  if (total > b->max_points) return EM_ERR_CAPACITY;

  const int slot = b->slot;
  b->slot = (b->slot + 1) % kSlots;
  EB_TRY(cudaEventSynchronize(b->ev[slot]), "cudaEventSynchronize");
  unsigned char* hb = b->desc_host + (size_t)slot * b->desc_bytes;
  unsigned char* db = b->desc_dev + (size_t)slot * b->desc_bytes;
  BatchDev* bd = reinterpret_cast<BatchDev*>(hb);
  MapDev* md = reinterpret_cast<MapDev*>(hb + sizeof(BatchDev));
  CloudDev* cd = reinterpret_cast<CloudDev*>(hb + sizeof(BatchDev) + (size_t)b->max_maps * sizeof(MapDev));
  memset(bd, 0, sizeof(BatchDev));
  GraphKey key{tune, false, false, false, false, false, 0u};
  int64_t cells = 0, coarse = 0;
  for (int u = 0; u < nm; ++u) {
    md[u] = map_begin_update(b->uniq[u], map_pts[u]);
    md[u].cell_begin = cells;
    cells += pad_tile(map_cells(b->uniq[u]));
    md[u].cbegin = coarse;
    coarse += (int64_t)md[u].CW * md[u].CH;
    key.ray |= md[u].ray_step > 0.f;
    key.drift |= md[u].drift_flat > 0.f;
    key.overlap |= md[u].ovl_dz > 0.f;
    key.ext |= md[u].excl_d > 0.f || md[u].upper != nullptr;
    key.upper |= md[u].upper != nullptr;
    key.stencils |= map_flags(b->uniq[u]) & (EM_F_NORMALS | EM_F_SMOOTH | EM_F_MEDIAN | EM_F_GAUSS | EM_F_INPAINT);
  }
  // clouds ordered by map (stable), so each map's points are contiguous
  int ci = 0;
  int64_t begin = 0;
  for (int u = 0; u < nm; ++u)
    for (int i = 0, first = 1; i < count; ++i) {
      if (b->map_of[i] != u) continue;
      if (first) {  // the map's first cloud's sensor origin, as in em_update_multi
        md[u].z_ref = clouds[i].pose[11];
        md[u].ref_x = clouds[i].pose[3];
        md[u].ref_y = clouds[i].pose[7];
      }
      first = 0;
      CloudDev& c = cd[ci++];
      memset(&c, 0, sizeof(c));
      c.pts = clouds[i].points;
      c.n = clouds[i].n;
      c.begin = begin;
      c.stride = clouds[i].stride;
      c.map = u;
      for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) c.R[r * 3 + k] = clouds[i].pose[r * 4 + k];
        c.t[r] = clouds[i].pose[r * 4 + 3];
      }
      begin += clouds[i].n;
    }
  bd->n_maps = nm;
  bd->n_clouds = count;
  bd->n_points = total;
  bd->maps = reinterpret_cast<const MapDev*>(db + sizeof(BatchDev));
  bd->clouds = reinterpret_cast<const CloudDev*>(db + sizeof(BatchDev) + (size_t)b->max_maps * sizeof(MapDev));
  bd->rz = b->rz;
  bd->rv = b->rv;
  bd->rc = b->rc;
  bd->n_cells = cells;
  bd->n_coarse = coarse;
  bd->ctl = b->bctl;
  bd->tile_cnt = b->tile_cnt;
  bd->tile_base = b->tile_base;
  bd->tile_cur = b->tile_cur;
  bd->tile_map = b->tile_map;
  bd->heavy = b->heavy;
  bd->light = b->light;
  bd->pieces = b->pieces;
  bd->max_pieces = b->max_pieces;
  bd->split_acc = b->split_acc;
  bd->split_done = b->split_done;
  bd->split_slots = b->split_slots;
  bd->heavy_thresh = tune.big_thresh * 16;
  bd->passes = (key.ray ? kPassRay : 0u) | (key.overlap ? kPassOverlap : 0u);
  bd->fuse_threads = tune.fuse_chunk;
  // upload header + maps, and the clouds at their fixed offset
  cudaError_t e = cudaMemcpyAsync(db, hb, sizeof(BatchDev) + (size_t)nm * sizeof(MapDev), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(db + sizeof(BatchDev) + (size_t)b->max_maps * sizeof(MapDev), cd,
                        (size_t)count * sizeof(CloudDev), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    for (int u = 0; u < nm; ++u) map_undo_update(b->uniq[u], map_pts[u]);
    return map_record_error("upload batch descriptor", e);
  }
  out->bd = reinterpret_cast<const BatchDev*>(db);
  out->slot = slot;
  out->points = total;
  out->n_maps = nm;
  out->cells = cells;
  out->key = key;
  return EM_OK;
}

void finish(em_batch* b, const Prepared& p, cudaStream_t s) {
  for (size_t u = 0; u < b->uniq.size(); ++u) map_end_update(b->uniq[u], s, 0);
  cudaEventRecord(b->ev[p.slot], s);
}

// A captured sequence is one chain of kernel nodes.  Let the ray march
// (k_coarse -> k_ray) hang off the node before it and join again at k_clear, so
// it runs beside k_alloc -> k_scatter -> k_fuse (the ray march reads only the
// ray thresholds and the points and writes only the marks, which k_clear reads).
// Anything but the expected chain is left as it is.  False when an edit failed
// half way (the graph must not be used).
bool overlap_ray_march(cudaGraph_t g) {
  cudaGraphNode_t root = nullptr;
  size_t n = 0;
  if (cudaGraphGetRootNodes(g, nullptr, &n) != cudaSuccess || n != 1) return true;
  if (cudaGraphGetRootNodes(g, &root, &n) != cudaSuccess) return true;
  std::vector<cudaGraphNode_t> chain;
  for (cudaGraphNode_t cur = root; cur && chain.size() < 64;) {
    chain.push_back(cur);
    size_t nd = 0;
    if (cudaGraphNodeGetDependentNodes(cur, nullptr, nullptr, &nd) != cudaSuccess || nd > 1) return true;
    cudaGraphNode_t next = nullptr;
    if (nd == 1 && cudaGraphNodeGetDependentNodes(cur, &next, nullptr, &nd) != cudaSuccess) return true;
    cur = nd == 1 ? next : nullptr;
  }
  auto fn = [](cudaGraphNode_t node) -> const void* {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(node, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) return nullptr;
    cudaKernelNodeParams kp = {};
    if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess) return nullptr;
    return kp.func;
  };
  for (size_t i = 1; i + 5 < chain.size(); ++i) {
    if (fn(chain[i]) != coarse_kernel()) continue;
    // chain: prev -> coarse -> ray -> alloc -> scatter -> fuse -> clear
    if (fn(chain[i + 2]) != alloc_kernel() || !is_fuse_kernel(fn(chain[i + 4])) || fn(chain[i + 5]) != clear_kernel())
      return true;
    cudaGraphNode_t prev = chain[i - 1], ray = chain[i + 1], alloc = chain[i + 2], clear = chain[i + 5];
    if (cudaGraphRemoveDependencies(g, &ray, &alloc, nullptr, 1) != cudaSuccess) {
      cudaGetLastError();
      return true;  // nothing changed
    }
    const bool ok = cudaGraphAddDependencies(g, &prev, &alloc, nullptr, 1) == cudaSuccess &&
                    cudaGraphAddDependencies(g, &ray, &clear, nullptr, 1) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
  }
  return true;
}

int run_graph(em_batch* b, const Prepared& p, cudaStream_t s) {
  if (!b->graph[p.slot] || !(b->graph_key[p.slot] == p.key)) {
    if (b->graph[p.slot]) {
      cudaGraphExecDestroy(b->graph[p.slot]);
      b->graph[p.slot] = nullptr;
    }
    cudaGraph_t g = nullptr;
    EB_TRY(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t le = launch_sequence(b, p.bd, b->max_points, (int64_t)b->max_maps * pad_tile(b->max_cells), p.key,
                                     b->capture_stream);
    cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      // Another thread can break a capture (a device-wide synchronize while it
      // runs invalidates it).  The sequence then runs without a graph this
      // time, and the next update of this kind tries the capture again.
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      EB_TRY(launch_sequence(b, p.bd, p.points, p.cells, p.key, s), "launch (capture failed)");
      return EM_OK;
    }
    if (p.key.ray && !p.key.upper && !overlap_ray_march(g)) {  // a half-edited graph is not used
      cudaGraphDestroy(g);
      EB_TRY(launch_sequence(b, p.bd, p.points, p.cells, p.key, s), "launch (graph edit failed)");
      return EM_OK;
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    EB_TRY(ie, "cudaGraphInstantiate");
    b->graph[p.slot] = ex;
    b->graph_key[p.slot] = p.key;
  }
  EB_TRY(cudaGraphLaunch(b->graph[p.slot], s), "cudaGraphLaunch");
  return EM_OK;
}

int set_dev(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) EB_TRY(cudaSetDevice(dev), "cudaSetDevice");
  return EM_OK;
}

void release(em_batch* b) {
  for (int i = 0; i < 2 * EM_PROF_SLOTS; ++i)
    if (b->pev[i]) cudaEventDestroy(b->pev[i]);
  for (int i = 0; i < kSlots; ++i) {
    if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  }
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->join_ev) cudaEventDestroy(b->join_ev);
  cudaFree(b->rz);
  cudaFree(b->rv);
  cudaFree(b->rc);
  cudaFree(b->bctl);
  cudaFree(b->tile_cnt);
  cudaFree(b->tile_base);
  cudaFree(b->tile_cur);
  cudaFree(b->tile_map);
  cudaFree(b->heavy);
  cudaFree(b->light);
  cudaFree(b->split_acc);
  cudaFree(b->split_done);
  cudaFree(b->pieces);
  cudaFree(b->desc_dev);
  cudaFreeHost(b->desc_host);
  delete b;
}

}  // namespace

extern "C" {

int em_wait_selftest(int device, int32_t wait_us) {
  if (wait_us < 1 || wait_us > 10 * 1000 * 1000) return EM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EM_ERR_INVALID_ARG;
  int rc = set_dev(device);
  if (rc) return rc;
  unsigned long long* word = nullptr;  // nothing ever sets it
  int* flag = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaMalloc((void**)&word, sizeof(*word));
  if (e == cudaSuccess) e = cudaMalloc((void**)&flag, sizeof(*flag));
  if (e == cudaSuccess) e = cudaMemset(word, 0, sizeof(*word));
  if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(*flag));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = launch_wait_selftest(word, flag, wait_us, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int timed_out = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&timed_out, flag, sizeof(timed_out), cudaMemcpyDeviceToHost);
  if (s) cudaStreamDestroy(s);
  cudaFree(word);
  cudaFree(flag);
  if (e != cudaSuccess) return map_record_error("em_wait_selftest", e);
  return timed_out ? EM_ERR_TIMEOUT : EM_OK;
}

int em_batch_create(int device, int32_t max_maps, int32_t max_clouds, int64_t max_points, int32_t max_cells,
                    uint32_t flags, em_batch** out) {
  if (!out) return EM_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_maps < 1 || max_maps > 65535 || max_clouds < 1 || max_points < 0 || max_points > (int64_t(1) << 31) - 1 ||
      max_cells < 1 || max_cells > (1 << 26) || (flags & ~(uint32_t)(EM_BATCH_GRAPH | EM_BATCH_PERSISTENT)))
    return EM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EM_ERR_INVALID_ARG;
  int rc = set_dev(device);
  if (rc) return rc;
  em_batch* b = new (std::nothrow) em_batch();
  if (!b) return EM_ERR_OOM;
  b->device = device;
  b->max_maps = max_maps;
  b->max_clouds = max_clouds;
  b->max_points = max_points;
  b->max_cells = max_cells;
  b->flags = flags;
  b->desc_bytes = (sizeof(BatchDev) + (size_t)max_maps * sizeof(MapDev) + (size_t)max_clouds * sizeof(CloudDev) + 255) &
                  ~size_t(255);
  const size_t np = (size_t)(max_points > 0 ? max_points : 1);
  b->max_tiles = (int64_t)max_maps * (pad_tile(max_cells) / kTile);
  const size_t nt = (size_t)b->max_tiles + 1;
  cudaError_t e = cudaMalloc((void**)&b->rz, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->rv, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->rc, np * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->bctl, sizeof(BatchCtl));
  if (e == cudaSuccess) e = cudaMemset(b->bctl, 0, sizeof(BatchCtl));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->tile_cnt, nt * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(b->tile_cnt, 0, nt * sizeof(int32_t));  // k_alloc keeps it zero after
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->tile_base, nt * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->tile_cur, nt * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->tile_map, nt * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->heavy, nt * sizeof(FuseItem));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->light, nt * sizeof(FuseItem));
  // split tiles: at most kMaxSplit slots of kSplitWords x kTile words; pieces of
  // more than 16 kMinHeavy records but the last of each tile
  b->split_slots = (int32_t)(b->max_tiles < kMaxSplit ? b->max_tiles : kMaxSplit);
  b->max_pieces = (int32_t)(np / (kMinHeavy * 16) + kMaxSplit + 1);
  const size_t acc_bytes = (size_t)b->split_slots * kSplitWords * kTile * sizeof(unsigned long long);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->split_acc, acc_bytes);
  if (e == cudaSuccess) e = cudaMemset(b->split_acc, 0, acc_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->split_done, (size_t)b->split_slots * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(b->split_done, 0, (size_t)b->split_slots * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->pieces, (size_t)b->max_pieces * sizeof(FuseItem));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->desc_dev, b->desc_bytes * kSlots);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->desc_host, b->desc_bytes * kSlots);
  for (int i = 0; i < kSlots && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release(b);
    return map_record_error("em_batch_create", e);
  }
  *out = b;
  return EM_OK;
}

int em_batch_destroy(em_batch* b) {
  if (!b) return EM_OK;
  set_dev(b->device);
  cudaDeviceSynchronize();
  release(b);
  return EM_OK;
}

int em_update_batch(em_batch* b, em_map* const* maps, const em_cloud* clouds, int32_t count, em_stream_t stream) {
  if (!b) return EM_ERR_INVALID_ARG;
  int rc = set_dev(b->device);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (b->prof) {
    rc = prof_collect(b);
    if (rc) return rc;
  }
  Prepared p;
  rc = prepare(b, maps, clouds, count, b->tune, s, &p);
  if (rc) return rc;
  if ((b->flags & EM_BATCH_GRAPH) && !b->prof) {
    rc = run_graph(b, p, s);
  } else {
    cudaError_t e = launch_sequence(b, p.bd, p.points, p.cells, p.key, s, b);
    rc = e == cudaSuccess ? EM_OK : map_record_error("batch launches", e);
  }
  finish(b, p, s);
  return rc;
}

int em_batch_profile(em_batch* b, int enable) {
  if (!b) return EM_ERR_INVALID_ARG;
  int rc = set_dev(b->device);
  if (rc) return rc;
  if (enable && !b->pev[0])
    for (int i = 0; i < 2 * EM_PROF_SLOTS; ++i) EB_TRY(cudaEventCreate(&b->pev[i]), "cudaEventCreate");
  if (!enable) {
    rc = prof_collect(b);
    if (rc) return rc;
  }
  if (enable && !b->prof)
    for (int k = 0; k < EM_PROF_SLOTS; ++k) { b->pms[k] = 0.0; b->pn[k] = 0; }
  b->prof = enable != 0;
  return EM_OK;
}

int em_batch_profile_read(em_batch* b, double* ms, int64_t* launches) {
  if (!b || !ms || !launches) return EM_ERR_INVALID_ARG;
  int rc = set_dev(b->device);
  if (rc) return rc;
  rc = prof_collect(b);
  if (rc) return rc;
  for (int k = 0; k < EM_PROF_SLOTS; ++k) {
    ms[k] = b->pms[k];
    launches[k] = b->pn[k];
  }
  return EM_OK;
}

int em_batch_set_tuning(em_batch* b, const em_tuning* t) {
  if (!b || !t || !tuning_ok(*t)) return EM_ERR_INVALID_ARG;
  b->tune = *t;
  return EM_OK;
}

int em_batch_get_tuning(const em_batch* b, em_tuning* t) {
  if (!b || !t) return EM_ERR_INVALID_ARG;
  *t = b->tune;
  return EM_OK;
}

int em_batch_autotune(em_batch* b, em_map* const* maps, const em_cloud* clouds, int32_t count, em_stream_t stream,
                      int32_t reps, em_tuning* out) {
  if (!b || !maps || !clouds || count < 1) return EM_ERR_INVALID_ARG;
  int rc = set_dev(b->device);
  if (rc) return rc;
  if (reps < 1) reps = 3;
  cudaStream_t s = (cudaStream_t)stream;
  // scratch copies of the distinct maps
  std::vector<em_map*> uniq, clones;
  std::vector<em_map*> cmaps(count);
  for (int i = 0; i < count; ++i) {
    if (!maps[i]) return EM_ERR_INVALID_ARG;
    size_t j = 0;
    while (j < uniq.size() && uniq[j] != maps[i]) ++j;
    if (j == uniq.size()) {
      em_params p = map_params(maps[i]);
      p.flags &= ~(uint32_t)EM_F_TRACE;
      em_map* c = nullptr;
      rc = em_create(&p, b->device, &c);
      if (rc) {
        for (em_map* x : clones) em_destroy(x);
        return rc;
      }
      uniq.push_back(maps[i]);
      clones.push_back(c);
    }
    cmaps[i] = clones[j];
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_one = [&](const em_tuning& t, float* ms_out) -> int {
    std::vector<float> ms;
    for (int r = 0; r < reps + 1; ++r) {
      for (size_t j = 0; j < uniq.size(); ++j) {
        int c = map_copy_state(clones[j], uniq[j], s);
        if (c) return c;
      }
      Prepared p;
      int c = prepare(b, cmaps.data(), clouds, count, t, s, &p);
      if (c) return c;
      cudaEventRecord(e0, s);
      cudaError_t le = launch_sequence(b, p.bd, p.points, p.cells, p.key, s);
      cudaEventRecord(e1, s);
      finish(b, p, s);
      if (le != cudaSuccess) return map_record_error("autotune launches", le);
      if (cudaEventSynchronize(e1) != cudaSuccess) return EM_ERR_CUDA;
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      if (r > 0) ms.push_back(x);  // the first run warms up
    }
    std::sort(ms.begin(), ms.end());
    *ms_out = ms[ms.size() / 2];
    return EM_OK;
  };
  em_tuning best = b->tune;
  float best_ms = 0.f;
  rc = time_one(best, &best_ms);
  const int ray_c[] = {1, 2, 4, 8, 16};
  const int chunk_c[] = {256, 512, 256, 512, 256};  // fusion block sizes (repeats are skipped)
  const int big_c[] = {64, 128, 256, 512, 1023};
  const bool any_ray = [&] {
    for (em_map* m : uniq)
      if (map_params(m).ray_step > 0.f) return true;
    return false;
  }();
  // coordinate descent: ray group, then fusion block size, then the heavy-tile threshold
  for (int pass = 0; pass < 3 && rc == EM_OK; ++pass) {
    if (pass == 0 && !any_ray) continue;
    const int* cand = pass == 0 ? ray_c : pass == 1 ? chunk_c : big_c;
    for (int i = 0; i < 5 && rc == EM_OK; ++i) {
      em_tuning t = best;
      if (pass == 0) t.ray_group = cand[i];
      if (pass == 1) t.fuse_chunk = cand[i];
      if (pass == 2) t.big_thresh = cand[i];
      if (t.ray_group == best.ray_group && t.fuse_chunk == best.fuse_chunk && t.big_thresh == best.big_thresh)
        continue;
      float ms = 0.f;
      rc = time_one(t, &ms);
      if (rc == EM_OK && ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (em_map* x : clones) em_destroy(x);
  if (rc) return rc;
  b->tune = best;
  if (out) *out = best;
  return EM_OK;
}

}  // extern "C"
