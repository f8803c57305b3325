// k_fuse.cu -- per-cell fusion (Section II-C of the paper).
//
// Every cell that received points in this update is fused once from its
// segment of records (z, sigma_p^2):
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
// signed 128-bit fixed-point integer with 44 fractional bits and the integers
// are added.  Integer addition is associative, so the result is the same for
// every order of the points and every split of a segment between lanes, bit
// for bit (no float atomics).
//
// Work split, one launch:
//   chunks  the record array is cut into chunks of `chunk` records; a warp owns
//           the cells whose segment STARTS in its chunk and streams their
//           records 32 at a time (one record per lane, coalesced 16-byte
//           loads).  Lanes of the same cell form a run; a segmented inclusive
//           scan over the runs gives each run's sums at its last lane, which
//           writes the cell.  A run that reaches lane 31 carries its partial
//           sums into the next 32 records.  Load balance follows the records,
//           not the cells, so uneven cells and maps cost no divergence.
//   large   cells with more than big_thresh records (flagged in their records
//           and listed by k_alloc) are skipped by the chunks and fused by a
//           whole block each, taken from a counter (atomicAdd; no block waits).
#include "em_point.cuh"

namespace em {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFuseThreads = 256;
constexpr int kFuseWarps = kFuseThreads / 32;
#ifndef EM_FUSE_BLOCKS_PER_SM
// 4 resident blocks (64 registers, a few spilled) measured 5-6 % faster than 3
// (80 registers, no spills) on both the served round and the 64-map batch
#define EM_FUSE_BLOCKS_PER_SM 4
#endif
constexpr int kFuseBlocksPerSM = EM_FUSE_BLOCKS_PER_SM;  // resident blocks per SM (sets the register budget)

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
  const unsigned long long lo = (unsigned long long)v;
  const unsigned long long hi = (unsigned long long)((unsigned __int128)v >> 64);
  const unsigned long long lo2 = __shfl_xor_sync(kFull, lo, o);
  const unsigned long long hi2 = __shfl_xor_sync(kFull, hi, o);
  return (__int128)(((unsigned __int128)hi2 << 64) | lo2);
}

// Partial sums of a run of records: the two fixed-point sums as (h, l) pairs
// (value h 2^27 + l) and the counts packed as accepted | rejected << 10 |
// dropped-by-wall << 20 (a run holds at most kMaxBigThresh records).  Within
// 32 records the l parts stay below 2^32; across passes they are carried in
// 64 bits.
struct Part {
  long long wh, th;
  unsigned long long wl, tl;
  uint32_t n;
};
constexpr uint32_t kCntAcc = 1u, kCntRej = 1u << 10, kCntWall = 1u << 20;
__device__ __forceinline__ int cnt_acc(uint32_t n) { return (int)(n & 1023u); }
__device__ __forceinline__ int cnt_rej(uint32_t n) { return (int)((n >> 10) & 1023u); }
__device__ __forceinline__ int cnt_wall(uint32_t n) { return (int)(n >> 20); }

// The cell's snapshot and the decisions that do not depend on single points.
struct CellCtx {
  float h, ve, href, k2;
  bool valid, wall_on, gate_on;
};

// The pre-update state of a cell, loaded ahead of its use.
struct Snap {
  float h, var;
  int32_t t_last;
};

__device__ __forceinline__ Snap load_snap(const MapDev& m, int32_t cell) {
  return Snap{m.h[cell], m.var[cell], m.t_last[cell]};
}

__device__ __forceinline__ CellCtx make_cell(const MapDev& m, const Snap& sn, bool wall_armed) {
  CellCtx c;
  c.h = sn.h;
  c.valid = isfinite(sn.var);
  c.ve = c.valid ? var_eff(m, sn.var, sn.t_last) : sn.var;
  c.href = c.valid ? c.h : m.z_ref;
  c.wall_on = wall_armed && c.valid;
  c.gate_on = c.valid && m.k > 0.f;
  c.k2 = __fmul_rn(m.k, m.k);
  return c;
}

__device__ __forceinline__ CellCtx load_cell(const MapDev& m, int32_t cell, bool wall_armed) {
  return make_cell(m, load_snap(m, cell), wall_armed);
}

// One record: wall rule, gate, and its two fixed-point terms when accepted
// (zero terms otherwise).
__device__ __forceinline__ uint8_t fuse_one(const CellCtx& c, float z, float vp, Fix& fw, Fix& ft) {
  fw = Fix{0, 0u};
  ft = Fix{0, 0u};
  if (c.wall_on && z < c.h) return kPtWall;
  if (c.gate_on) {
    // |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k  <=>  (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2)  (k > 0)
    const float dz = __fsub_rn(z, c.h);
    if (__fmul_rn(dz, dz) > __fmul_rn(c.k2, __fadd_rn(c.ve, vp))) return kPtRejected;
  }
  const float w = __frcp_rn(vp);
  fw = to_fix(w);
  ft = to_fix(__fmul_rn(w, __fsub_rn(z, c.href)));
  return kPtFused;
}

// New state of the cell from its complete sums (one thread); true when the
// cell took a point (accepted or rejected).
__device__ __forceinline__ bool write_cell(const MapDev& m, int32_t cell, const CellCtx& c, __int128 qw,
                                           __int128 qt, int acc, int rej) {
  if (acc + rej == 0) return false;
  float h_new, var_new;
  const float sw = fixed_to_float(qw);
  const float st = fixed_to_float(qt);
  if (c.valid) {
    const float vprior = __fadd_rn(c.ve, __fmul_rn((float)rej, m.v_out));
    if (acc == 0) {
      h_new = c.h;
      var_new = vprior;
    } else {
      const float lam = __fadd_rn(__frcp_rn(vprior), sw);
      h_new = __fadd_rn(c.h, __fdiv_rn(st, lam));
      var_new = __frcp_rn(lam);
    }
  } else {
    h_new = __fadd_rn(c.href, __fdiv_rn(st, sw));
    var_new = __frcp_rn(sw);
  }
  m.h[cell] = h_new;
  m.var[cell] = var_new;
  m.t_last[cell] = m.t_now;
  if (m.upper) m.upper[cell] = __int_as_float(0x7f800000);  // observed: no bound (Section II-H)
  return true;
}

// Statistics of one warp for its current map, in lane registers: each lane
// counts its own records and the cells it wrote; a flush (warp sums, four
// atomics by lane 0) happens when the warp moves to another map and at the end.
struct WarpCount {
  int map = -1;
  uint32_t acc = 0, rej = 0, wal = 0, cells = 0;
};

__device__ __forceinline__ void add_stats(const BatchDev& b, int mi, uint32_t acc, uint32_t rej, uint32_t wal,
                                          uint32_t cells) {
  unsigned long long* st = b.maps[mi].ctl->stats;
  if (acc) atomicAdd(st + kStAccepted, (unsigned long long)acc);
  if (rej) atomicAdd(st + kStRejected, (unsigned long long)rej);
  if (wal) atomicAdd(st + kStWall, (unsigned long long)wal);
  if (cells) atomicAdd(st + kStCellsUpdated, (unsigned long long)cells);
}

// all 32 lanes
__device__ __forceinline__ void warp_flush(const BatchDev& b, WarpCount& wc) {
  const uint32_t a = __reduce_add_sync(kFull, wc.acc), r = __reduce_add_sync(kFull, wc.rej);
  const uint32_t w = __reduce_add_sync(kFull, wc.wal), c = __reduce_add_sync(kFull, wc.cells);
  if ((threadIdx.x & 31) == 0 && wc.map >= 0) add_stats(b, wc.map, a, r, w, c);
  wc.acc = wc.rej = wc.wal = wc.cells = 0;
}

__device__ __forceinline__ unsigned long long rec_tag(const float4& q) {
  return ((unsigned long long)__float_as_uint(q.w) << 32) | (unsigned long long)__float_as_uint(q.z);
}

// Write a carried run that ended at the previous pass (one lane).  Its records
// were counted in their passes; the cell is counted here.
__device__ __forceinline__ void finish_tag(const BatchDev& b, WarpCount& wc, unsigned long long tag, const Part& a) {
  const uint32_t w = (uint32_t)(tag >> 32);
  const int mi = (int)(w & kRecMapMask);
  const int32_t cell = (int32_t)(uint32_t)tag;
  const MapDev& m = b.maps[mi];
  const CellCtx c = load_cell(m, cell, (w & kRecWall) != 0);
  if (write_cell(m, cell, c, fix128(a.wh, a.wl), fix128(a.th, a.tl), cnt_acc(a.n), cnt_rej(a.n))) {
    if (mi == wc.map) ++wc.cells; else add_stats(b, mi, 0, 0, 0, 1);
  }
}

// Record r of the batch (zeros beyond n_rec).
__device__ __forceinline__ float4 load_rec(const BatchDev& b, int64_t r, int32_t n_rec) {
  return r < n_rec ? __ldg(b.rec + r) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// A record's map and cell words are in range (every record in [0, rec_total)
// was written by k_scatter this update; anything else is recorded and skipped).
__device__ __forceinline__ bool rec_sane(const BatchDev& b, const float4& q) {
  const int mi = (int)(__float_as_uint(q.w) & kRecMapMask);
  return mi < b.n_maps && (uint32_t)__float_as_int(q.z) < (uint32_t)(b.maps[mi].W * b.maps[mi].H);
}

// Cell state for a record, loaded one pass ahead (a cell is written only by the
// warp that owns it, when its run ends, so the prefetched value is current).
__device__ __forceinline__ Snap prefetch_snap(const BatchDev& b, const float4& q, bool inr) {
  if (!inr || !rec_sane(b, q)) return Snap{0.f, 0.f, 0};
  return load_snap(b.maps[__float_as_uint(q.w) & kRecMapMask], __float_as_int(q.z));
}

// The cells whose segment starts in [ch * chunk, (ch + 1) * chunk), one warp.
// Software pipeline: the records of pass i + 2 and the cell state of pass i + 1
// are in flight while pass i is fused.
__device__ __forceinline__ void fuse_chunk(const BatchDev& b, WarpCount& wc, int64_t ch, int32_t n_rec) {
  const int lane = threadIdx.x & 31;
  const unsigned upto = lane == 31 ? kFull : ((1u << (lane + 1)) - 1u);  // lanes <= this lane
  const int64_t win_end = (ch + 1) * (int64_t)b.chunk;
  int64_t pos = ch * (int64_t)b.chunk;
  // carried run: 0 none, 1 ours (partial sums in cp), 2 not ours (started before the chunk)
  int cmode = 0;
  unsigned long long ctag = 0;
  Part cp{0, 0, 0ull, 0ull, 0u};
  if (pos > 0) {
    ctag = rec_tag(__ldg(b.rec + pos - 1));
    cmode = 2;
  }
  float4 q = load_rec(b, pos + lane, n_rec);
  float4 qn = load_rec(b, pos + 32 + lane, n_rec);
  Snap sn = prefetch_snap(b, q, pos + lane < n_rec);
  for (;;) {
    const int64_t r = pos + lane;
    const bool inr = r < n_rec;
    const float4 qnn = load_rec(b, pos + 64 + lane, n_rec);
    const Snap snn = prefetch_snap(b, qn, pos + 32 + lane < n_rec);
    const unsigned long long tag = inr ? rec_tag(q) : ~0ull;
    unsigned long long prev = __shfl_up_sync(kFull, tag, 1);
    if (lane == 0) prev = cmode ? ctag : ~tag;  // nothing carried: lane 0 starts a run
    const bool head = inr && tag != prev;
    // the carried run of ours ends where this pass starts another run (or nothing)
    if (cmode == 1 && __shfl_sync(kFull, !inr || head, 0)) {
      if (lane == 0) finish_tag(b, wc, ctag, cp);
      cmode = 0;
    }
    const unsigned stops = __ballot_sync(kFull, !inr || (head && r >= win_end));
    const int first_stop = stops ? __ffs(stops) - 1 : 32;
    if (first_stop == 0) break;
    const bool live = lane < first_stop;
    const unsigned heads = __ballot_sync(kFull, head && live);
    const unsigned hm = heads & upto;
    const bool cont = live && hm == 0;  // continues the carried run
    const int hd = hm ? 31 - __clz(hm) : 0;
    const uint32_t w = __float_as_uint(q.w);
    const bool big = (w & kRecBig) != 0;
    const int mi = (int)(w & kRecMapMask);
    const int32_t cell = __float_as_int(q.z);
    const bool sane = live && rec_sane(b, q);
    if (live && !sane) atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
    const bool ours = sane && !big && !(cont && cmode == 2);
    // statistics: one map per pass (the usual case) goes to the lane registers
    const int pm = ours ? mi : -1;
    bool mixed = false;
    if (!__all_sync(kFull, pm < 0 || pm == wc.map)) {
      const unsigned om = __ballot_sync(kFull, pm >= 0);
      const int first = __shfl_sync(kFull, pm, __ffs(om) - 1);
      if (__all_sync(kFull, pm < 0 || pm == first)) {
        warp_flush(b, wc);
        wc.map = first;
      } else {
        mixed = true;  // a pass across a map boundary: count with atomics
      }
    }
    Fix fw{0, 0u}, ft{0, 0u};
    uint32_t n = 0u;
    CellCtx c;
    if (ours) {
      c = make_cell(b.maps[mi], sn, (w & kRecWall) != 0);
      const uint8_t st = fuse_one(c, q.x, q.y, fw, ft);
      n = st == kPtFused ? kCntAcc : st == kPtRejected ? kCntRej : kCntWall;
      if (!mixed) {
        wc.acc += st == kPtFused;
        wc.rej += st == kPtRejected;
        wc.wal += st == kPtWall;
      } else {
        add_stats(b, mi, st == kPtFused, st == kPtRejected, st == kPtWall, 0);
      }
      if (b.tr_status) b.tr_status[b.idx_sorted[r]] = st;
    }
    // segmented inclusive scan: lane l sums lanes hd(l) .. l of its run; only as
    // many steps as the longest run of this pass needs
    const int runlen = live ? lane - hd + 1 : 0;
    const int maxrun = (int)__reduce_max_sync(kFull, (unsigned)runlen);
    long long wh = fw.h, th = ft.h;
    uint32_t wl = fw.l, tl = ft.l;
    for (int o = 1; o < maxrun; o <<= 1) {
      const long long awh = __shfl_up_sync(kFull, wh, o), ath = __shfl_up_sync(kFull, th, o);
      const uint32_t awl = __shfl_up_sync(kFull, wl, o), atl = __shfl_up_sync(kFull, tl, o);
      const uint32_t an = __shfl_up_sync(kFull, n, o);
      if (lane - o >= hd) {
        wh += awh;
        th += ath;
        wl += awl;
        tl += atl;
        n += an;
      }
    }
    Part v{wh, th, (unsigned long long)wl, (unsigned long long)tl, n};
    if (cont && cmode == 1) {  // the carried partial sums belong to this run
      v.wh += cp.wh;
      v.th += cp.th;
      v.wl += cp.wl;
      v.tl += cp.tl;
      v.n += cp.n;
    }
    const bool next_head = lane < 31 && ((heads >> (lane + 1)) & 1u);
    const bool end = live && (next_head || (lane == first_stop - 1 && first_stop < 32));
    if (end && ours &&
        write_cell(b.maps[mi], cell, c, fix128(v.wh, v.wl), fix128(v.th, v.tl), cnt_acc(v.n), cnt_rej(v.n))) {
      if (!mixed) ++wc.cells; else add_stats(b, mi, 0, 0, 0, 1);
    }
    if (first_stop < 32) break;
    // lane 31's run goes on in the next 32 records
    const unsigned long long t31 = __shfl_sync(kFull, tag, 31);
    if (__shfl_sync(kFull, ours, 31)) {
      cp.wh = __shfl_sync(kFull, v.wh, 31);
      cp.th = __shfl_sync(kFull, v.th, 31);
      cp.wl = __shfl_sync(kFull, v.wl, 31);
      cp.tl = __shfl_sync(kFull, v.tl, 31);
      cp.n = __shfl_sync(kFull, v.n, 31);
      cmode = 1;
      ctag = t31;
    } else if (__shfl_sync(kFull, big && sane, 31)) {
      // skip the rest of a large cell: its segment end from the cell's (base, count)
      const uint32_t w31 = (uint32_t)(t31 >> 32);
      const int2 sg = b.maps[w31 & kRecMapMask].cell_seg[(int32_t)(uint32_t)t31];
      const int64_t next = (int64_t)sg.x + sg.y;
      if (next > pos + 32) {  // restart the pipeline there
        pos = next;
        cmode = 0;
        q = load_rec(b, pos + lane, n_rec);
        qn = load_rec(b, pos + 32 + lane, n_rec);
        sn = prefetch_snap(b, q, pos + lane < n_rec);
        continue;
      }
      cmode = 0;
    } else {
      cmode = 2;  // a run that started before the chunk
      ctag = t31;
    }
    pos += 32;
    q = qn;
    qn = qnn;
    sn = snn;
  }
}

// A large cell with a whole block: lane partial sums, warp and block reductions.
__device__ __forceinline__ void fuse_big(const BatchDev& b, int2 e, __int128* s_q, uint32_t* s_n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const MapDev& m = b.maps[e.x];
  const int2 sg = m.cell_seg[e.y];
  const CellCtx c = load_cell(m, e.y, m.wall > 0 && sg.y > m.wall);
  long long wh = 0, th = 0;
  unsigned long long wl = 0, tl = 0;
  uint32_t acc = 0, rej = 0, wal = 0;
  for (int i = threadIdx.x; i < sg.y; i += kFuseThreads) {
    const float4 q = __ldg(b.rec + sg.x + i);
    Fix fw, ft;
    const uint8_t st = fuse_one(c, q.x, q.y, fw, ft);
    wh += fw.h;
    wl += fw.l;
    th += ft.h;
    tl += ft.l;
    acc += st == kPtFused;
    rej += st == kPtRejected;
    wal += st == kPtWall;
    if (b.tr_status) b.tr_status[b.idx_sorted[sg.x + i]] = st;
  }
  __int128 qw = fix128(wh, wl), qt = fix128(th, tl);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    qw += shfl_xor_i128(qw, o);
    qt += shfl_xor_i128(qt, o);
  }
  acc = __reduce_add_sync(kFull, acc);
  rej = __reduce_add_sync(kFull, rej);
  wal = __reduce_add_sync(kFull, wal);
  if (lane == 0) {
    s_q[warp] = qw;
    s_q[kFuseWarps + warp] = qt;
    s_n[warp] = acc;
    s_n[kFuseWarps + warp] = rej;
    s_n[2 * kFuseWarps + warp] = wal;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __int128 tw = 0, tt = 0;
    uint32_t ta = 0, tr = 0, tl2 = 0;
    for (int k = 0; k < kFuseWarps; ++k) {
      tw += s_q[k];
      tt += s_q[kFuseWarps + k];
      ta += s_n[k];
      tr += s_n[kFuseWarps + k];
      tl2 += s_n[2 * kFuseWarps + k];
    }
    const bool upd = write_cell(m, e.y, c, tw, tt, (int)ta, (int)tr);
    add_stats(b, e.x, ta, tr, tl2, upd ? 1u : 0u);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFuseThreads, kFuseBlocksPerSM) k_fuse(const BatchDev* __restrict__ bp) {
  __shared__ int s_slot;
  __shared__ __int128 s_q[2 * kFuseWarps];
  __shared__ uint32_t s_n[3 * kFuseWarps];
  const BatchDev& b = *bp;

  // ---- large cells first (the longest jobs): one block each, taken from a counter
  const int n_big = min(b.ctl->n_big, b.big_cap);
  if (n_big > 0) {
    for (;;) {
      if (threadIdx.x == 0) s_slot = atomicAdd(&b.ctl->big_next, 1);
      __syncthreads();
      const int jb = s_slot;
      __syncthreads();
      if (jb >= n_big) break;
      fuse_big(b, b.big_list[jb], s_q, s_n);
    }
  }

  // ---- record chunks, one warp each (grid-stride)
  const int32_t n_rec = (int32_t)min((int64_t)b.ctl->rec_total, b.n_points);
  const int64_t n_chunks = ((int64_t)n_rec + b.chunk - 1) / b.chunk;
  const int64_t wstride = (int64_t)gridDim.x * kFuseWarps;
  WarpCount wc;
  for (int64_t ch = (int64_t)blockIdx.x * kFuseWarps + (threadIdx.x >> 5); ch < n_chunks; ch += wstride)
    fuse_chunk(b, wc, ch, n_rec);
  warp_flush(b, wc);
}

cudaError_t launch_fuse(const BatchDev* b, int64_t n_points, int chunk, cudaStream_t s) {
  const int c = (chunk >= 64 && chunk <= 1024 && (chunk & (chunk - 1)) == 0) ? chunk : 256;
  const int64_t warps = n_points / c + 1;
  const int64_t want = (warps + kFuseWarps - 1) / kFuseWarps;
  const int64_t cap = (int64_t)sm_count() * kFuseBlocksPerSM;  // one resident wave
  const int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  k_fuse<<<grid, kFuseThreads, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace em
