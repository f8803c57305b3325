// fuse_pass.cuh -- the device pass of the per-cell fusion (k_fuse.cu): work
// items from the lists k_alloc writes, each a tile (or a piece of one) staged
// in shared memory, gated and fused into exact integer sums.  It runs on the
// blocks of its own kernel or of the persistent kernel (k_persist.cu).
#pragma once

#include "em_point.cuh"

namespace em {

// The cell's pre-update state as the cell update reads it.
struct CellCtx {
  float h, ve, href;
  bool valid;
};

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

// Per-cell accumulators of one tile in shared memory, and its staged state.
struct TileSmem {
  long long wh[kTile], th[kTile];            // fixed-point sums: high parts
  unsigned long long wl[kTile], tl[kTile];   // ... and low parts (value h 2^27 + l)
  unsigned long long n[kTile];               // accepted | rejected << 32
  float h[kTile], ve[kTile];                 // pre-update height, effective variance (+inf: empty)
  uint32_t cnt[kTile];                       // records per cell (the wall rule)
  FuseItem item;                             // this block's work (tile -1: none left)
  int last;                                  // this block finished its tile's last piece
  unsigned long long stat[4];                // accepted, rejected, wall, cells of the item
};

// A cell's new state from its complete sums (one thread; zero counts: untouched).
__device__ __forceinline__ uint32_t write_from_sums(const MapDev& m, int32_t cell, float h, float ve, __int128 qw,
                                                    __int128 qt, unsigned long long nn) {
  CellCtx cx;
  cx.h = h;
  cx.ve = ve;
  cx.valid = isfinite(ve);
  cx.href = cx.valid ? h : m.z_ref;
  return write_cell(m, cell, cx, qw, qt, (int)(uint32_t)nn, (int)(nn >> 32)) ? 1u : 0u;
}

// Work item w of the three lists (pieces, heavy tiles, light tiles), checked
// against the sizes of the batch; tile -1 when w is past the end.  A failed
// check records an internal error and also ends the block's work.
__device__ __forceinline__ FuseItem fetch_item(const BatchDev& b, int w, int n_pieces, int n_heavy, int n_light,
                                               int64_t n_tiles, int32_t rec_total) {
  FuseItem it{-1, 0, 0, 0, 0, 0, -1, 1};
  if (w >= 0 && w < n_pieces) it = b.pieces[w];
  else if (w >= n_pieces && w - n_pieces < n_heavy) it = b.heavy[w - n_pieces];
  else if (w >= n_pieces + n_heavy && w - n_pieces - n_heavy < n_light) it = b.light[w - n_pieces - n_heavy];
  else if (w >= 0) return it;
  const bool ok = it.tile >= 0 && it.tile < n_tiles && it.map >= 0 && it.map < b.n_maps && 0 <= it.r0 &&
                  it.r0 <= it.q0 && it.q0 <= it.q1 && it.q1 <= it.r1 && it.r1 <= rec_total && it.np >= 1 &&
                  it.slot >= -1 && it.slot < b.split_slots && w >= 0;
  if (!ok) {
    atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
    it.tile = -1;
  }
  return it;
}

template <int NT>
__device__ __forceinline__ void fuse_pass(const BatchDev& b, TileSmem& S) {
  const int lane = threadIdx.x & 31;
  const int64_t n_tiles = b.n_cells / kTile;
  const int n_pieces = b.ctl->n_pieces, n_heavy = b.ctl->n_heavy, n_light = b.ctl->n_light;
  const int32_t rec_total = b.ctl->rec_total;
  const int64_t n_items = (int64_t)n_pieces + n_heavy + n_light;
  // the accumulators start at zero and the write-out leaves them at zero
  for (int c = threadIdx.x; c < kTile; c += NT) {
    S.wh[c] = 0;
    S.th[c] = 0;
    S.wl[c] = 0;
    S.tl[c] = 0;
    S.n[c] = 0;
  }
  if (threadIdx.x == 0)
    S.item = fetch_item(b, atomicAdd(&b.ctl->fuse_next, 1), n_pieces, n_heavy, n_light, n_tiles, rec_total);
  __syncthreads();
  // every block takes work items from the counter until they run out; a block
  // takes at most all of them (a bound that holds whatever the counter reads)
  for (int64_t items = 0;; ++items) {
    const FuseItem it = S.item;
    if (it.tile < 0) break;  // block-uniform
    if (items >= n_items) {
      if (threadIdx.x == 0) atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
      break;
    }
    // the next item's index now, its entry after this one (the atomic's latency hides behind the work)
    int w_next = 0;
    if (threadIdx.x == 0) w_next = atomicAdd(&b.ctl->fuse_next, 1);
    const int64_t t = it.tile;
    const bool split = it.slot >= 0;
    const int32_t r0 = it.r0, r1 = it.r1, q0 = it.q0, q1 = it.q1;
    const MapDev& m = b.maps[it.map];
    const int32_t p0 = (int32_t)(t * kTile - m.cell_begin);
    const int32_t ncell = min(kTile, m.W * m.H - p0);
    const bool wall_on = m.wall > 0;
    // the first window of records, in flight while the tile's state is staged
    int32_t r = q0 + threadIdx.x;
    float z = 0.f, vp = 1.f;
    uint32_t c = 0;
    if (r < q1) { z = __ldg(b.rz + r); vp = __ldg(b.rv + r); c = __ldg(b.rc + r); }
    // ---- the tile's pre-update state; record counts to zero
    for (int c = threadIdx.x; c < kTile; c += NT) {
      float h = 0.f, ve = __int_as_float(0x7f800000);
      if (c < ncell) {
        const float var = __ldg(m.var + p0 + c);
        h = __ldg(m.h + p0 + c);
        const int32_t tl = __ldg(m.t_last + p0 + c);
        if (isfinite(var)) ve = var_eff(m, var, tl);
      }
      S.h[c] = h;
      S.ve[c] = ve;
      S.cnt[c] = 0;
    }
    if (threadIdx.x < 4) S.stat[threadIdx.x] = 0;
    __syncthreads();
    // records per cell of the whole tile first: the wall rule looks at the
    // cell's count (one atomic per cell and warp)
    if (wall_on) {
      for (int32_t cb = r0; cb < r1; cb += NT) {
        const int32_t rr = cb + threadIdx.x;
        const uint32_t key = rr < r1 ? (uint32_t)__ldg(b.rc + rr) : 0xffffffffu;
        const unsigned grp = __match_any_sync(kFull, key);
        if (rr < r1 && lane == __ffs(grp) - 1) atomicAdd(&S.cnt[key], (uint32_t)__popc(grp));
      }
      __syncthreads();
    }
    unsigned long long* const A = split ? b.split_acc + (size_t)it.slot * kSplitWords * kTile : nullptr;
    const float k2 = __fmul_rn(m.k, m.k);
    uint32_t acc = 0, rej = 0, wal = 0, cells = 0;
    // ---- records, NT at a time; the next window's loads in flight
    for (int32_t base = q0; base < q1; base += NT) {
      const bool live = r < q1;
      const int32_t rn = r + NT;
      float zn = 0.f, vpn = 1.f;
      uint32_t cn = 0;
      if (rn < q1) { zn = __ldg(b.rz + rn); vpn = __ldg(b.rv + rn); cn = __ldg(b.rc + rn); }
      Fix fw{0, 0u}, ft{0, 0u};
      uint8_t st = kPtFused;
      if (live) {
        const float h = S.h[c], ve = S.ve[c];
        const bool valid = isfinite(ve);
        if (wall_on && valid && (int32_t)S.cnt[c] > m.wall && z < h) {
          st = kPtWall;
        } else if (valid && m.k > 0.f && __fmul_rn(__fsub_rn(z, h), __fsub_rn(z, h)) > __fmul_rn(k2, __fadd_rn(ve, vp))) {
          // |z - h| / sqrt(sigma_m^2 + sigma_p^2) > k  <=>  (z - h)^2 > k^2 (sigma_m^2 + sigma_p^2)  (k > 0)
          st = kPtRejected;
        } else {
          const float wgt = __frcp_rn(vp);
          fw = to_fix(wgt);
          ft = to_fix(__fmul_rn(wgt, __fsub_rn(z, valid ? h : m.z_ref)));
        }
        acc += st == kPtFused;
        rej += st == kPtRejected;
        wal += st == kPtWall;
        if (b.tr_status) b.tr_status[b.idx_sorted[r]] = st;
      }
      // runs of equal cells in consecutive lanes: a segmented inclusive scan, as
      // many steps as the longest run needs; the run's last lane adds its sums.
      // Within a run of at most 32 lanes the 27-bit low parts and the counts
      // (accepted | rejected << 16) fit 32 bits.
      uint32_t nn = !live ? 0u : st == kPtFused ? 1u : st == kPtRejected ? (1u << 16) : 0u;
      const unsigned long long tag = live ? (unsigned long long)c : ~0ull;
      int head, len;
      key_runs(tag, head, len);
      // the run's last lane (every lane takes part in the shuffle)
      const unsigned long long next = __shfl_down_sync(kFull, tag, 1);
      const bool tail = lane == 31 || next != tag;
      const int maxrun = (int)__reduce_max_sync(kFull, live ? (unsigned)(lane - head + 1) : 1u);
      long long wh = fw.h, th = ft.h;
      uint32_t wl = fw.l, tl = ft.l;
      for (int o = 1; o < maxrun; o <<= 1) {
        const long long awh = __shfl_up_sync(kFull, wh, o), ath = __shfl_up_sync(kFull, th, o);
        const uint32_t awl = __shfl_up_sync(kFull, wl, o), atl = __shfl_up_sync(kFull, tl, o);
        const uint32_t an = __shfl_up_sync(kFull, nn, o);
        if (lane - o >= head) {
          wh += awh;
          th += ath;
          wl += awl;
          tl += atl;
          nn += an;
        }
      }
      if (live && tail) {
        const unsigned long long n64 = (unsigned long long)(nn & 0xffffu) | ((unsigned long long)(nn >> 16) << 32);
        const bool sums = (wh | th | (long long)(wl | tl)) != 0;
        if (split) {  // a piece: straight into the tile's slot
          if (nn) atomicAdd(&A[4 * kTile + c], n64);
          if (sums) {
            atomicAdd(&A[c], (unsigned long long)wh);
            atomicAdd(&A[kTile + c], (unsigned long long)wl);
            atomicAdd(&A[2 * kTile + c], (unsigned long long)th);
            atomicAdd(&A[3 * kTile + c], (unsigned long long)tl);
          }
        } else {
          if (nn) atomicAdd(&S.n[c], n64);
          if (sums) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&S.wh[c]), (unsigned long long)wh);
            atomicAdd(&S.wl[c], (unsigned long long)wl);
            atomicAdd(reinterpret_cast<unsigned long long*>(&S.th[c]), (unsigned long long)th);
            atomicAdd(&S.tl[c], (unsigned long long)tl);
          }
        }
      }
      r = rn;
      z = zn;
      vp = vpn;
      c = cn;
    }
    __syncthreads();
    if (!split) {
      // ---- every cell of the tile with accumulated sums, once; the accumulators back to zero
      for (int cc = threadIdx.x; cc < ncell; cc += NT) {
        const unsigned long long nn = S.n[cc];
        if (!nn) continue;
        const __int128 qw = fix128(S.wh[cc], S.wl[cc]), qt = fix128(S.th[cc], S.tl[cc]);
        S.wh[cc] = 0;
        S.th[cc] = 0;
        S.wl[cc] = 0;
        S.tl[cc] = 0;
        S.n[cc] = 0;
        cells += write_from_sums(m, p0 + cc, S.h[cc], S.ve[cc], qw, qt, nn);
      }
    } else {
      // ---- the last piece of the tile to finish writes the cells
      __threadfence();  // this block's sums before its count of done pieces
      __syncthreads();
      if (threadIdx.x == 0) {
        const int done = atomicAdd(&b.split_done[it.slot], 1);
        if (done >= it.np) atomicCAS(&b.maps[0].ctl->err, 0, kErrInternal);
        S.last = done == it.np - 1;
        __threadfence();  // the other pieces' sums before this block reads them
      }
      __syncthreads();
      if (S.last) {
        for (int cc = threadIdx.x; cc < ncell; cc += NT) {
          const unsigned long long nn = __ldcg(&A[4 * kTile + cc]);
          if (!nn) continue;
          const long long wh = (long long)__ldcg(&A[cc]), th = (long long)__ldcg(&A[2 * kTile + cc]);
          const unsigned long long wl = __ldcg(&A[kTile + cc]), tl = __ldcg(&A[3 * kTile + cc]);
#pragma unroll
          for (int k = 0; k < kSplitWords; ++k) A[k * kTile + cc] = 0ull;  // zero for the next update
          cells += write_from_sums(m, p0 + cc, S.h[cc], S.ve[cc], fix128(wh, wl), fix128(th, tl), nn);
        }
        if (threadIdx.x == 0) b.split_done[it.slot] = 0;
      }
    }
    // ---- the item's statistics: one atomic per counter
    const uint32_t v[4] = {acc, rej, wal, cells};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = __reduce_add_sync(kFull, v[k]);
      if (lane == 0 && x) atomicAdd(&S.stat[k], (unsigned long long)x);
    }
    __syncthreads();
    if (threadIdx.x < 4 && S.stat[threadIdx.x]) {
      const int idx = threadIdx.x == 0 ? kStAccepted : threadIdx.x == 1 ? kStRejected : threadIdx.x == 2 ? kStWall
                                                                                                     : kStCellsUpdated;
      atomicAdd(&m.ctl->stats[idx], S.stat[threadIdx.x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) S.item = fetch_item(b, w_next, n_pieces, n_heavy, n_light, n_tiles, rec_total);
    __syncthreads();
  }
  __syncthreads();  // the shared memory is free again
}

}  // namespace em
