/*
 * em.h -- C ABI of libem.so: GPU fusion of point clouds into a robot-centric
 * 2.5D elevation map, after Miki et al., "Elevation Mapping for Locomotion and
 * Navigation using GPU" (arXiv 2204.12876), Section II.
 *
 * Conventions shared by every entry point:
 *   - Return value: EM_OK (0) or a negative EM_ERR_* code.  No C++ exception
 *     crosses this boundary.  em_status_str() names a code.
 *   - Calls that take a stream enqueue their GPU work on it and return without
 *     waiting for it, unless stated.  A NULL stream is the legacy default
 *     stream.  The caller keeps every device buffer it passes alive until the
 *     stream has reached the call.
 *   - The library owns all device memory of a map.  Caller buffers are never
 *     freed or retained by the library.
 *   - Maps are not thread-safe; distinct maps may be used from distinct host
 *     threads.
 *   - Map layers are float32.  Layer arrays exchanged with the caller are in
 *     logical row-major order [iy][ix], cell (ix, iy) covering
 *     [x0 + ix r, x0 + (ix+1) r) x [y0 + iy r, y0 + (iy+1) r) of the map frame.
 *   - Errors found by a kernel (a capacity overflow, a bounded wait that ran
 *     out) are recorded on the device and reported by the next em_sync() or
 *     em_get_stats() of that map.
 */
#ifndef EM_H
#define EM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct em_map em_map;
typedef struct CUstream_st* em_stream_t; /* the same handle as cudaStream_t */

/* status codes */
enum {
  EM_OK = 0,
  EM_ERR_INVALID_ARG = -1, /* NULL pointer, bad size / stride, non-finite pose, bad parameter */
  EM_ERR_OOM = -2,         /* a device or pinned-host allocation failed */
  EM_ERR_CUDA = -3,        /* a CUDA call failed; the CUDA error is logged by em_last_cuda_error() */
  EM_ERR_TIMEOUT = -4,     /* a bounded wait ran out (host or device side) */
  EM_ERR_REJECTED = -5,    /* admission refused (memory budget or slot limit) */
  EM_ERR_BUSY = -6,        /* the object is in use by work that has not finished */
  EM_ERR_CAPACITY = -7     /* a request exceeds a fixed capacity chosen at creation */
};

/* em_params.flags */
enum {
  EM_F_NORMALS = 1u << 0, /* keep the per-cell normal layer (Section II-A, "normal calculation") */
  EM_F_SMOOTH = 1u << 1,  /* keep a 5x5 box-smoothed elevation layer (Section II-I) */
  EM_F_INPAINT = 1u << 2, /* keep a minimum-in-painted elevation layer (Section II-I) */
  EM_F_MEDIAN = 1u << 3,  /* the smoothed layer holds the 5x5 median instead (lower median of the
                             window's valid heights; Section II-I) */
  EM_F_GAUSS = 1u << 4,   /* the smoothed layer holds a 5x5 Gaussian instead (sigma = 1 cell, weights
                             renormalised over the window's valid cells; Section II-I).  At most one
                             of EM_F_SMOOTH, EM_F_MEDIAN, EM_F_GAUSS may be set. */
  EM_F_UPPER = 1u << 5,   /* keep an upper-bound layer (Section II-H): every ray sample in a cell
                             that holds no estimate lowers the cell's bound to the sample height
                             (a running minimum over updates); a cell that takes an estimate, or
                             comes into view by a shift, has no bound (+inf).  Needs ray_step > 0. */
  EM_F_TRACE = 1u << 8    /* record per-point cells and decisions of the last update (testing) */
};

/* layer bits for em_get_layers / em_set_layers (ascending bit order in the buffers) */
enum {
  EM_LAYER_ELEVATION = 1u << 0, /* h, NaN where the cell is empty */
  EM_LAYER_VARIANCE = 1u << 1,  /* sigma_m^2 as stored at the cell's last write (TIME); +inf if empty */
  EM_LAYER_TIME = 1u << 2,      /* index of the update that last wrote the cell (exact below 2^24) */
  EM_LAYER_NORMAL_X = 1u << 3,
  EM_LAYER_NORMAL_Y = 1u << 4,
  EM_LAYER_NORMAL_Z = 1u << 5,
  EM_LAYER_SMOOTH = 1u << 6,
  EM_LAYER_INPAINT = 1u << 7,
  EM_LAYER_VALID = 1u << 8,       /* 1.0 where the cell holds an estimate, else 0.0 (get only) */
  EM_LAYER_VARIANCE_NOW = 1u << 9, /* sigma_m^2 plus time variance up to the current update (get only) */
  EM_LAYER_UPPER = 1u << 10        /* upper bound of the ground height (EM_F_UPPER); +inf where none */
};

/* Map and method parameters.  The paper leaves most of them user-defined
 * (Section II-C noise model alpha_d, time variance sigma_t^2, Mahalanobis
 * distance, wall count; Section II-E ray step, update age, alpha_n). */
typedef struct em_params {
  int32_t width, height;        /* cells, 1 .. 2^22 each, width*height <= 2^26 */
  float resolution;             /* metres per cell, > 0 */
  float noise_a0, noise_a1, noise_a2; /* sigma_p = a0 + a1 d + a2 d^2; the paper's alpha_d d^2 is a1 = sqrt(alpha_d) */
  float var_min;                /* floor on sigma_p^2, > 0 */
  float min_range, max_range;   /* points with d outside [min_range, max_range] are dropped */
  float mahalanobis_k;          /* reject iff |p_z - h| / sqrt(sigma_m^2 + sigma_p^2) > k; <= 0 disables */
  float outlier_variance;       /* added to sigma_m^2 per rejected point; 0 disables */
  int32_t wall_num_thresh;      /* > 0: with more points than this in a valid cell, drop those below h */
  float time_variance;          /* sigma_t^2 added per update since the cell was last written; 0 disables */
  float ray_step;               /* visibility ray-march step in metres; 0 disables visibility cleanup */
  int32_t cleanup_min_age;      /* remove only cells last written >= max(1, this) updates ago */
  float cleanup_normal_thresh;  /* alpha_n of Eq. 4; <= 0 disables the normal guard */
  uint32_t flags;               /* EM_F_* */
  float drift_flatness;         /* height drift compensation (Section II-D), 0 disables: the mean error
                                   z - h of the points that fall into cells holding an estimate whose
                                   previous normal has n_z >= drift_flatness (flat cells; the paper's
                                   traversability threshold) is added to every estimate before the
                                   update; in (0, 1], needs the normal layer (EM_F_NORMALS or
                                   cleanup_normal_thresh > 0) */
  /* Exclusion area (Section II-C; its figure is not available, so this is a
   * reading): a point whose height above the sensor exceeds excl_b within a
   * horizontal distance excl_c of it, else excl_b + (r - excl_c) tan(excl_theta),
   * at most excl_d, is ignored (no fusion, no ray).  excl_d <= 0 disables. */
  float excl_b, excl_c, excl_theta, excl_d;
  /* Overlap clearance (Section II-F): after the update, estimates whose cell
   * centre lies within overlap_radius (horizontally) of the first cloud's sensor
   * origin and whose height differs from the origin's by more than overlap_dz
   * are cleared.  overlap_dz <= 0 disables. */
  float overlap_radius, overlap_dz;
} em_params;

/* One point cloud: n points of `stride` floats (3 = xyz, 4 = xyz + pad) in the
 * sensor frame, and the sensor-to-map pose as a row-major 3x4 [R | t].  Every
 * buffer the library reads or writes as floats (points, layers, read-backs)
 * must start on a 4-byte boundary; calls refuse others with EM_ERR_INVALID_ARG. */
typedef struct em_cloud {
  const float* points;
  int64_t n;
  int32_t stride;
  float pose[12];
} em_cloud;

typedef struct em_info {
  int32_t width, height;
  float resolution;
  int32_t t_now;           /* number of updates fused so far */
  int64_t shift_x, shift_y;/* cumulative em_shift in cells; the map centre is (shift_x r, shift_y r) */
  double x0, y0;           /* lower-left corner of the map in the map frame */
  int64_t point_capacity;  /* points per update the workspace holds without growing */
  int64_t device_bytes;    /* device memory held by the map */
} em_info;

typedef struct em_stats {
  /* cumulative since em_create */
  int64_t updates;
  int64_t points_in;        /* all points offered */
  int64_t points_valid;     /* finite and within [min_range, max_range] */
  int64_t points_in_map;    /* valid and inside the map */
  int64_t points_accepted;  /* fused */
  int64_t points_rejected;  /* Mahalanobis outliers */
  int64_t points_wall;      /* dropped by the wall rule */
  int64_t cells_updated;    /* (cell, update) pairs written by fusion */
  int64_t cells_cleared;    /* (cell, update) pairs removed by visibility cleanup */
  int64_t ray_samples;      /* ray-march sample positions in each ray's k range clipped to the map box */
  int64_t drift_points;     /* points that entered a drift-compensation mean */
  double drift_last;        /* height error added by the last update's drift compensation (metres) */
} em_stats;

/* Create a map of params->width x params->height empty cells centred on the
 * map-frame origin on CUDA device `device`.  Validates every parameter
 * (EM_ERR_INVALID_ARG), allocates the map's layers and a workspace for
 * `params`-independent default capacity (grown on demand).  *out receives the
 * handle.  Cites: 2.5D grid of Section I/II; initial sigma_m^2 "large"
 * (Section II-C) is represented as +inf (an empty cell). */
int em_create(const em_params* params, int device, em_map** out);

/* Release the map and all its device memory.  NULL-safe; waits for the map's
 * outstanding work first. */
int em_destroy(em_map* map);

/* Grow the workspace so that updates of up to max_points points (all clouds
 * of one update together) need no allocation.  Synchronous. */
int em_reserve(em_map* map, int64_t max_points);

/* Fuse one point cloud (device pointer, n points, stride 3 or 4 floats) seen
 * from a sensor with pose pose[12] (host memory, row-major 3x4, sensor -> map)
 * into the map: transform, noise variance, binning, wall rule, Mahalanobis
 * gate, Eq. 1/Eq. 2 fusion, visibility ray casting and removal (Eq. 3, Eq. 4),
 * then the filters selected by params->flags (Section II-A to II-I).  n = 0 is
 * a valid empty update (time advances).  Non-finite points are dropped and
 * counted.  Asynchronous on `stream`; grows the workspace (synchronously) if n
 * exceeds the current capacity. */
int em_update(em_map* map, const float* points, int64_t n, int32_t stride, const float pose[12],
              em_stream_t stream);

/* One update made of several clouds (e.g. several cameras of one robot): all
 * points are gated against the same pre-update map and fused together; each
 * cloud's rays start at its own sensor origin.  clouds[] is host memory,
 * clouds[i].points device memory. */
int em_update_multi(em_map* map, const em_cloud* clouds, int32_t n_clouds, em_stream_t stream);

/* Same as em_update_multi with clouds[i].points in HOST memory: the library
 * copies the points to the device on `stream` (through a pinned staging
 * buffer it owns) before fusing.  Returns once the points are staged. */
int em_update_host(em_map* map, const em_cloud* clouds, int32_t n_clouds, em_stream_t stream);

/* Move the map with the robot by (dx, dy) cells (robot-centric map, Section
 * I): afterwards cell (ix, iy) holds what cell (ix + dx, iy + dy) held; cells
 * that come into view are empty.  O(exposed cells) on the GPU. */
int em_shift(em_map* map, int32_t dx, int32_t dy, em_stream_t stream);

/* Copy the layers selected by layer_mask (EM_LAYER_*) in ascending bit order,
 * each width*height floats in logical row-major order, to dst (device memory,
 * or host memory if dst_is_host; then the call waits for the copy). */
int em_get_layers(em_map* map, uint32_t layer_mask, float* dst, int dst_is_host, em_stream_t stream);

/* Overwrite the selected layers from src (same layout).  Accepts ELEVATION,
 * VARIANCE, TIME and NORMAL_X/Y/Z; a non-finite variance makes a cell empty.
 * With em_set_time it restores a checkpoint taken with em_get_layers. */
int em_set_layers(em_map* map, uint32_t layer_mask, const float* src, int src_is_host, em_stream_t stream);

/* Set the update counter (the index the next update will use is t_now + 1). */
int em_set_time(em_map* map, int32_t t_now);

/* Geometry and bookkeeping; host only, does not synchronise. */
int em_get_info(const em_map* map, em_info* out);

/* Cumulative counters; waits for the map's outstanding work.  Returns a
 * recorded device error (e.g. EM_ERR_TIMEOUT) if one occurred. */
int em_get_stats(em_map* map, em_stats* out);

/* Wait for the map's outstanding work and report any recorded error. */
int em_sync(em_map* map);

/* With EM_F_TRACE: per point of the last update (clouds concatenated) its
 * logical cell (ix, iy) and its status (0 non-finite, 1 out of range, 2 outside
 * the map, 3 fused, 4 rejected, 5 wall rule).  Host buffers of n entries (n must
 * equal the last update's point count); waits for the map's work. */
int em_get_trace(em_map* map, int32_t* ix, int32_t* iy, uint8_t* status, int64_t n);

/* Per-kernel timing with CUDA events recorded on the update's stream around
 * each kernel the library launches.  While enabled, every update first waits
 * for the previous update's events (so timing adds a host wait per update).
 * Slots of em_profile_read, in this order: */
enum {
  EM_PROF_COUNT = 0,   /* k_count: transform + bin + per-tile counts; ray thresholds */
  EM_PROF_RAY,         /* k_ray: visibility ray march */
  EM_PROF_ALLOC,       /* k_alloc: record ranges of the tiles */
  EM_PROF_SCATTER,     /* k_scatter: records into their tile's range */
  EM_PROF_FUSE,        /* k_fuse: per-cell gate + fusion, one tile per block */
  EM_PROF_CLEAR,       /* k_clear: removal of penetrated cells */
  EM_PROF_NORMALS,
  EM_PROF_SMOOTH,
  EM_PROF_INPAINT,
  EM_PROF_DRIFT,       /* k_drift: drift compensation of the estimates (and the ray thresholds) */
  EM_PROF_OVERLAP,     /* k_overlap: overlap clearance near the robot */
  EM_PROF_PERSIST,     /* k_persist: the passes of a batched update in one launch (EM_BATCH_PERSISTENT) */
  EM_PROF_SLOTS
};
int em_profile(em_map* map, int enable);
/* Accumulated milliseconds and launch counts per slot since profiling was
 * enabled (both arrays EM_PROF_SLOTS long, host memory); waits for the map. */
int em_profile_read(em_map* map, double* ms, int64_t* launches);

/* ---- Batched form: many maps (each with one or more clouds) updated by one
 * sequence of kernels over all of them -- the per-point and per-cell work of
 * every map shares each launch, so small updates no longer pay a launch
 * sequence each.  The arithmetic per map is exactly em_update's.
 * A batch object owns the record workspace (max_points records), a ring of
 * device descriptors, and -- with EM_BATCH_GRAPH -- one captured CUDA graph
 * per descriptor slot, replayed with a single cudaGraphLaunch per batch (grids
 * are sized from the capacities; actual sizes are read from the descriptor). */
typedef struct em_batch em_batch;

/* EM_BATCH_PERSISTENT: one cooperative launch of all blocks that fit on the
 * device at once runs the passes of the update (transform, binning, grouping,
 * gate, fusion, ray march, removal) over every map, with grid-wide barriers
 * between them, instead of one kernel per pass (the normals, smoothing and
 * in-painting stencils stay kernels of their own).  Every barrier wait is
 * bounded (EM_PERSIST_WAIT_MS): a wait that runs out gives EM_ERR_TIMEOUT at
 * the maps' next em_sync.  Batches with a drift-compensated map, and devices
 * that cannot run the launch, use the kernel sequence.  Same results either
 * way, bit for bit. */
enum { EM_BATCH_GRAPH = 1u << 0, EM_BATCH_PERSISTENT = 1u << 1 };
enum { EM_PERSIST_WAIT_MS = 1000 };

/* The bounded device-side wait of the persistent launch, on a word that
 * nothing sets, for wait_us microseconds: EM_ERR_TIMEOUT when the wait ran
 * out as it must (and the device is still usable), EM_OK if it did not, or
 * another error.  A check of the wait itself; synchronous. */
int em_wait_selftest(int device, int32_t wait_us);

/* Launch shapes picked by the autotuner (or set by hand).  None of them
 * changes a result: every shape gives the same maps bit for bit. */
typedef struct em_tuning {
  int32_t ray_group;    /* ray march: samples per chunk tested against the coarse threshold grid,
                           and lanes per marched chunk: 1, 2, 4, 8, 16 or 32 */
  int32_t fuse_chunk;   /* threads per fusion block (one tile of 1024 cells per block): 64 .. 1024, a
                           power of two; 512 and more run 512-thread blocks (three resident per SM
                           when the cell space has at least three tiles per SM -- for a graph-
                           replayed batch the capacity's, else the update's -- otherwise two),
                           the rest 256-thread ones */
  int32_t big_thresh;   /* tiles with more than 16 x big_thresh records are fused first: 32 .. 1023 */
} em_tuning;

/* Capacities: at most max_maps distinct maps, max_clouds clouds and
 * max_points points per batch, maps of at most max_cells cells. */
int em_batch_create(int device, int32_t max_maps, int32_t max_clouds, int64_t max_points, int32_t max_cells,
                    uint32_t flags, em_batch** out);
int em_batch_destroy(em_batch* batch); /* NULL-safe; waits for the batch's work */

/* Fuse clouds[i] into maps[i] for i < count (host arrays; points on the device).
 * A map may appear several times: its clouds form one multi-cloud update
 * (em_update_multi).  Every listed map advances by one update.  Returns
 * EM_ERR_CAPACITY beyond the batch's capacities.  Asynchronous on `stream`. */
int em_update_batch(em_batch* batch, em_map* const* maps, const em_cloud* clouds, int32_t count,
                    em_stream_t stream);

int em_batch_set_tuning(em_batch* batch, const em_tuning* tuning);
int em_batch_get_tuning(const em_batch* batch, em_tuning* tuning);

/* Per-kernel CUDA-event timing of the batch's launches (EM_PROF_* slots, as
 * em_profile / em_profile_read).  While enabled the batch launches kernels
 * directly (no graph) and every update first waits for the previous one. */
int em_batch_profile(em_batch* batch, int enable);
int em_batch_profile_read(em_batch* batch, double* ms, int64_t* launches);

/* Autotuner: times candidate launch shapes on this workload (median of `reps`
 * runs each, coordinate by coordinate) on scratch copies of the maps -- the
 * maps themselves are not changed -- and keeps the fastest.  Synchronous.
 * *out (may be NULL) receives the choice. */
int em_batch_autotune(em_batch* batch, em_map* const* maps, const em_cloud* clouds, int32_t count,
                      em_stream_t stream, int32_t reps, em_tuning* out);

/* ---- Served form: a request loop for many robots / sensors.
 * The server keeps every map resident on its device and runs a worker thread.
 * Requests (one update of one map) are admitted while the admitted ones fit in
 * max_slots and their bytes fit in the memory budget (resident maps included);
 * the rest wait in arrival order.  In EM_SERVE_BATCHED mode the worker starts a
 * batch (em_update_batch) on any free stream whenever admitted requests wait,
 * so requests that arrive while earlier batches run join the next batch and
 * batches on different streams overlap on the device (continuous batching).  A
 * map takes at most one update per batch and a map with an update in flight
 * waits, so every request sees exactly the map it would see served alone.  In
 * EM_SERVE_PLAIN mode the worker issues one em_update_multi per request in
 * arrival order on one stream (the plain per-request path). */
typedef struct em_server em_server;

enum { EM_SERVE_BATCHED = 0, EM_SERVE_PLAIN = 1 };

/* Admission accounting: each admitted request holds this many bytes per point
 * (one grouped record per point), and each batch stream a workspace of
 * max_batch_points records. */
enum { EM_SERVE_RECORD_BYTES = 16 };

typedef struct em_server_cfg {
  int32_t device;
  int64_t budget_bytes;     /* device bytes for resident maps + batch workspaces + admitted requests */
  int32_t max_slots;        /* requests admitted at a time */
  int32_t n_streams;        /* batches in flight at a time (batched mode) */
  int32_t max_batch_maps;   /* maps per batch */
  int64_t max_batch_points; /* points per batch (also the largest request) */
  int32_t max_map_cells;    /* largest map the server accepts */
  uint32_t mode;            /* EM_SERVE_BATCHED or EM_SERVE_PLAIN */
  uint32_t batch_flags;     /* EM_BATCH_GRAPH */
  int32_t fail_alloc_at;    /* fault injection: the n-th em_server_add_map (1-based) fails with EM_ERR_OOM; 0 = off */
} em_server_cfg;

typedef struct em_result {
  int32_t status;           /* EM_OK, EM_ERR_REJECTED, EM_ERR_TIMEOUT (cancelled), or the launch's error */
  int32_t map_id;
  int64_t points;
  int32_t batch_size;       /* requests in the batch that carried this one */
  int64_t t_submit_ns;      /* steady-clock timestamps */
  int64_t t_start_ns;       /* launched */
  int64_t t_done_ns;        /* the worker saw the GPU finish */
} em_result;

typedef struct em_server_stats {
  int64_t submitted, completed, rejected, cancelled, batches, batched_requests;
  int64_t max_batch_size, bytes_in_use, peak_bytes, slots_in_use;
} em_server_stats;

int em_server_create(const em_server_cfg* cfg, em_server** out);
/* Create a resident map; EM_ERR_REJECTED when it does not fit the budget. */
int em_server_add_map(em_server* srv, const em_params* params, int32_t* map_id);
/* The resident map (to read layers after em_server_drain; do not update it directly). */
int em_server_map(em_server* srv, int32_t map_id, em_map** out);
/* Queue one update of map_id from n_clouds device clouds (host array of
 * descriptors; the points stay valid until the request completes).  Returns at
 * once with a ticket; EM_ERR_REJECTED when the request can never fit. */
int em_server_submit(em_server* srv, int32_t map_id, const em_cloud* clouds, int32_t n_clouds, uint64_t* ticket);
/* Same, but the request's GPU work first waits for `ready` (a cudaEvent_t
 * recorded by the caller after it wrote the points, e.g. a host-to-device
 * copy on its own stream).  The event must stay valid until the request
 * completes. */
int em_server_submit_after(em_server* srv, int32_t map_id, const em_cloud* clouds, int32_t n_clouds,
                           void* ready, uint64_t* ticket);
/* One request of em_server_submit_many. */
typedef struct em_request {
  int32_t map_id;
  int32_t n_clouds;          /* 1..8 */
  const em_cloud* clouds;    /* points valid until the ticket finishes (device memory unless clouds_on_host) */
  uint32_t read_mask;        /* EM_LAYER_* bits to read back right after the update; 0 = none */
  int32_t read_to_host;      /* read_dst is page-locked host memory (else device memory) */
  float* read_dst;           /* popcount(read_mask) * width * height floats, em_get_layers layout */
  int32_t clouds_on_host;    /* clouds[i].points are page-locked host memory: once the request is admitted
                                the server copies them by DMA (one cudaMemcpyAsync per cloud, on a copy
                                stream of its own, after `ready`) into its device input arena; the
                                request's batch waits for that copy, so it overlaps running batches */
} em_request;

/* Queue n requests under one lock, so that those that fit reach the same batch;
 * each first waits for `ready` (a cudaEvent_t recorded after the points were
 * written, or NULL).  A request with read_mask != 0 gets its map's layers
 * written to read_dst on the batch's stream right after its update (the map
 * state the update produced); its ticket finishes once they have landed.  A
 * host read_dst must be page-locked (cudaHostAlloc, cudaHostRegister): the GPU
 * writes it directly.  Host clouds (clouds_on_host) must be page-locked too; the
 * first such request makes the server allocate its input arena, (n_streams +
 * 2) x max_batch_points x 16 bytes, counted in its byte budget
 * (EM_ERR_REJECTED if it does not fit); a host request is admitted only when
 * its clouds fit the arena's free room.  All or nothing: EM_ERR_INVALID_ARG for a malformed
 * request (pageable or unknown read_dst memory included) and EM_ERR_REJECTED
 * for one that can never fit leave nothing queued; else tickets[i] is request
 * i's ticket. */
int em_server_submit_many(em_server* srv, const em_request* reqs, int32_t n, void* ready, uint64_t* tickets);
/* Wait for a ticket (timeout_us < 0: forever); EM_ERR_TIMEOUT when it has not
 * finished in time (the request stays queued).  Fills *out and forgets the
 * ticket once finished. */
int em_server_wait(em_server* srv, uint64_t ticket, int64_t timeout_us, em_result* out);
/* Wait for n distinct tickets (timeout_us < 0: forever, else for all of them
 * together).  On EM_OK every ticket is finished and forgotten and out[i] (if
 * out is not NULL) is ticket i's result; on EM_ERR_TIMEOUT none is forgotten.
 * EM_ERR_INVALID_ARG for an unknown or repeated ticket. */
int em_server_wait_many(em_server* srv, const uint64_t* tickets, int32_t n, int64_t timeout_us, em_result* out);
/* Withdraw a request that has not been launched; EM_ERR_BUSY if it already runs. */
int em_server_cancel(em_server* srv, uint64_t ticket);
/* Wait until every submitted request has finished. */
int em_server_drain(em_server* srv, int64_t timeout_us);
int em_server_get_stats(em_server* srv, em_server_stats* out);
/* Launch shapes of the server's batches (e.g. from em_batch_autotune); call while idle (after em_server_drain). */
int em_server_set_tuning(em_server* srv, const em_tuning* tuning);
int em_server_destroy(em_server* srv); /* NULL-safe: drains, stops the worker, frees the maps */

/* ---- Update without allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they update a map -- a real-time loop
 * that forbids allocation after start-up, or a framework whose own allocator
 * already holds the device memory.  It runs the update of em_update (binning, counting sort by cell,
 * wall rule, Mahalanobis gate, Eq. 1/2 fusion, ray march and removal; not the
 * per-cell filters) on layers the caller owns, in logical row-major order
 * without a ring offset:
 *   h, var      float32 [height][width], device memory, read and written;
 *               an empty cell has var = +inf (h is then NaN)
 *   t_last      int32 [height][width], device memory, read and written
 *   nx, ny, nz  float32 [height][width], device memory, read only; required
 *               when cleanup_normal_thresh > 0 or drift_flatness > 0, else may be
 *               NULL (EM_F_UPPER is not available here: EM_ERR_INVALID_ARG)
 *   shift_x/y   the map centre is (shift_x r, shift_y r) (see em_info)
 *   t_now       index of this update (>= 1): cells it writes get t_last = t_now
 *   clouds[]    host array; clouds[i].points device memory
 * All scratch lives in one static device array of the library (about 6.1 MiB,
 * held by every GPU that loads the library until the process exits).  The
 * first call on a device looks up that array's address with the device
 * current; make that first call before any stream capture.  Every call uses
 * the same array and it keeps the previous call's contents (the call clears
 * what must start at zero); calls whose GPU work overlaps race on it.  Calls
 * no cudaMalloc / cudaFree.  Returns EM_ERR_CAPACITY when width*height >
 * EM_NOALLOC_MAX_CELLS, the points of all clouds > EM_NOALLOC_MAX_POINTS or
 * n_clouds > EM_NOALLOC_MAX_CLOUDS; EM_ERR_INVALID_ARG for bad arguments
 * (the library cannot check the layers' sizes: each must hold width*height
 * elements).  The call's descriptor travels as a kernel parameter; it uses no
 * host buffer and copies nothing between host and device.  Asynchronous on
 * `stream`; a failed CUDA call returns EM_ERR_CUDA and is logged for
 * em_last_cuda_error(); device-side errors are not reported. */
#define EM_NOALLOC_MAX_CELLS 65536
#define EM_NOALLOC_MAX_POINTS 327680
#define EM_NOALLOC_MAX_CLOUDS 8
int em_update_noalloc(const em_params* params, int64_t shift_x, int64_t shift_y, int32_t t_now, float* h,
                      float* var, int32_t* t_last, const float* nx, const float* ny, const float* nz,
                      const em_cloud* clouds, int32_t n_clouds, em_stream_t stream);

/* Text for a status code (static storage). */
const char* em_status_str(int status);

/* Text of the last CUDA error seen by this thread in the library (static
 * thread-local storage). */
const char* em_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EM_H */
