// tensor.cu -- the iteration tensor of Section V: for every (rank, iteration)
// row, the exclusive time and sample count of each calling context the row
// holds, in ascending context order (rank prologues are rows too).
//
// Two passes over warp tiles with a scan in between; no tile waits for
// another.  A tile is TW consecutive samples; it owns the rows that START in
// it and reads past its end to finish its last row.  A warp streams a tile 128
// samples per step (4 per lane, 16-byte vector loads, the next steps already
// in flight in registers).
//   count pass (contexts only): rows and run heads of the tile's rows (a run
//     = consecutive samples of one context in a row; every row start is a
//     head).  A row has at most as many distinct contexts as runs, so the run
//     counts size the entry slots; also validates context ids.
//   scan: every tile's first row and first entry slot.
//   write pass (contexts and timestamps): validates timestamp order; each
//     step's run heads go to a per-warp ring (context, first timestamp,
//     offset); when a row ends, its runs (ring entries) are summed per context
//     and written in context order at the row's slots.  A run lasts until the
//     next head, so its time is a difference of two head timestamps (the
//     per-sample durations telescope) and its samples a difference of two
//     offsets.
//   compaction (only when some row holds a context in more than one run, so
//     that it fills fewer slots than it has runs): a scan of the rows'
//     distinct counts and a copy into exactly sized arrays.
#include <algorithm>

#include "ta_internal.h"

namespace ta {
namespace {

// Tile widths (samples per tile) the passes are built for: 4096 by default,
// 2048 for the batched form's autotuner.  Rank-start mask words cover
// positions 0 .. TW.
constexpr u32 TW_DEFAULT = 4096;
template <u32 TW>
struct TileW {
  static constexpr u32 MASKW = TW / 32 + 4;
};
constexpr u32 STEP = 128;           // samples per warp step (4 per lane)
constexpr int DEPTH_COUNT = 2;      // steps in flight, count pass (256 samples each)
constexpr int DEPTH_WRITE = 1;      // steps in flight in registers, write pass (timestamps too)
constexpr u32 RS = 128;             // staged entries per warp in shared memory
constexpr u32 TL = 128;             // touched bitmap words remembered
constexpr u32 RING = 256;           // run heads remembered per warp (power of two)
constexpr u32 FAST_RUNS = 128;      // longest row (in runs) of the direct-write path
constexpr u32 PF = 2;               // steps prefetched into L2 ahead (write pass)

struct Head {  // one run head: 16 bytes, one vector store
  u64 ts;
  u32 ctx;
  u32 pos;  // offset from the tile start
};

template <u32 TW>
struct WriteSmem {
  static constexpr u32 mask_off = 0;                      // u32[MASKW]
  static constexpr u32 tl_off = 4 * TileW<TW>::MASKW;     // u32[TL + 4] touched words, count
  static constexpr u32 time_off = tl_off + 4 * (TL + 4);  // u64[RS]
  static constexpr u32 ctx_off = time_off + 8 * RS;       // u32[RS]
  static constexpr u32 cnt_off = ctx_off + 4 * RS;        // u32[RS]
  static constexpr u32 stamp_off = cnt_off + 4 * RS;      // u32[RS] row ids (direct path)
  static constexpr u32 tctx_off = stamp_off + 4 * RS;     // u32[FAST_RUNS] template contexts
  static constexpr u32 tpos_off = tctx_off + 4 * FAST_RUNS;  // u8[FAST_RUNS] template positions
  static constexpr u32 ring_off = tpos_off + FAST_RUNS;   // Head[RING]
  static constexpr u32 fixed = ring_off + 16 * RING;      // bitmap words follow
};
static_assert(WriteSmem<4096>::time_off % 16 == 0 && WriteSmem<4096>::ring_off % 16 == 0 &&
                  WriteSmem<4096>::fixed % 16 == 0 && WriteSmem<2048>::time_off % 16 == 0 &&
                  WriteSmem<2048>::ring_off % 16 == 0 && WriteSmem<2048>::fixed % 16 == 0,
              "vector alignment of the write pass's shared memory");

// The tile's place in its trace set (a single experiment is one set).
struct Tile {
  u64 sbase, N, a, b, qrank;
  u32 lo, hi, rhi, C, m;
  bool last;
};

template <u32 TW>
__device__ __forceinline__ Tile tile_of(const TensorArgs& A, u64 t) {
  Tile T;
  T.sbase = 0;
  T.N = A.N;
  u64 t0 = 0, t1 = A.n_tiles;
  T.rhi = A.R;
  T.C = A.C;
  T.m = A.m;
  if (A.sets.S) {
    const u32 s = A.sets.tile_set[t];
    T.sbase = A.sets.set_rec0[s];
    T.N = A.sets.set_rec_end[s];
    t0 = A.sets.set_tile0[s];
    t1 = A.sets.set_tile0[s + 1];
    T.rhi = A.sets.set_rank0[s + 1];
    T.C = A.sets.set_C[s];
    T.m = A.sets.set_m[s];
  }
  T.a = T.sbase + (t - t0) * TW;
  T.b = min(T.a + (u64)TW, T.N);
  T.last = (t + 1 == t1);
  T.lo = A.tfr[t];
  T.hi = T.last ? T.rhi : A.tfr[t + 1];
  T.qrank = (T.hi < T.rhi) ? A.rank_off[T.hi] : T.N;  // first rank start >= b (or N)
  return T;
}

// Rank starts of the tile as a bit mask over positions 0 .. TW; returns the
// steps (bit s: samples s STEP .. s STEP + STEP - 1) that hold one.
template <u32 TW>
__device__ __forceinline__ u32 fill_mask(const TensorArgs& A, const Tile& T, u32* mask, int lane) {
  static_assert(TW <= 32 * STEP && TW % (2 * STEP) == 0, "one bit per step of a tile");
  for (u32 i = lane; i < TileW<TW>::MASKW; i += 32) mask[i] = 0;
  __syncwarp();
  u32 steps = 0;
  for (u32 r = T.lo + lane; r < T.hi; r += 32) {
    const u32 p = (u32)(A.rank_off[r] - T.a);
    atomicOr(&mask[p >> 5], 1u << (p & 31));
    if (p < TW) steps |= 1u << (p / STEP);
  }
  __syncwarp();
  return __reduce_or_sync(FULL, steps);
}

struct WStep {
  u32 c[4];
  u64 t[4];
};

__device__ __forceinline__ void load_w(const TensorArgs& A, u64 q0, int lane, WStep& s) {
  const u64 q = q0 + 4 * (u64)lane;
  if (q0 + STEP <= A.N) {
    const uint4 v = *reinterpret_cast<const uint4*>(A.ctx + q);
    const ulonglong2 t0 = *reinterpret_cast<const ulonglong2*>(A.ts + q);
    const ulonglong2 t1 = *reinterpret_cast<const ulonglong2*>(A.ts + q + 2);
    s.c[0] = v.x;
    s.c[1] = v.y;
    s.c[2] = v.z;
    s.c[3] = v.w;
    s.t[0] = t0.x;
    s.t[1] = t0.y;
    s.t[2] = t1.x;
    s.t[3] = t1.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s.c[j] = (q + j < A.N) ? A.ctx[q + j] : NONE32;
      s.t[j] = (q + j < A.N) ? A.ts[q + j] : 0ull;
    }
  }
}

// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, u32 bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One lane asks L2 for the samples of step q (contexts and timestamps) if
// the whole step lies inside the trace array; the register loads a few steps
// later then hit L2.  q is a multiple of 32, so both ranges are 16-byte
// aligned.
__device__ __forceinline__ void prefetch_step(const TensorArgs& A, u64 q) {
  if (q + STEP <= A.N) {
    prefetch_l2(A.ctx + q, STEP * 4);
    prefetch_l2(A.ts + q, STEP * 8);
  }
}

__device__ __forceinline__ u64 sel4(const u64* v, u32 j) {
  return j == 0 ? v[0] : j == 1 ? v[1] : j == 2 ? v[2] : v[3];
}

// Bits of this lane's 4 positions (4 lane + j) at or after position f.
__device__ __forceinline__ u32 from_mask(u32 f, int lane) {
  const int s = (int)f - 4 * lane;
  return s <= 0 ? 0xFu : (s >= 4 ? 0u : (0xFu << s) & 0xFu);
}

// Per-step row starts: rank starts (rs4, from the mask) and marker-run
// starts (ms4: the marker context after another context, or at a rank start).
__device__ __forceinline__ void step_bits(const u32* c, const u32* pc, u32 rs4, u32 valid4, u32 m,
                                          u32& ms4, u32& st4, u32& h4) {
  ms4 = 0;
  h4 = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool rs = (rs4 >> j) & 1u;
    ms4 |= ((c[j] == m && (pc[j] != m || rs)) ? 1u : 0u) << j;
    h4 |= ((pc[j] != c[j] || rs) ? 1u : 0u) << j;
  }
  ms4 &= valid4;
  st4 = (rs4 & valid4) | ms4;
  h4 = (h4 | st4) & valid4;
}

// ------------------------------------------------------------ count pass --
// 8 samples per lane, 256 per step: the pass does little per sample, so
// wider steps spread the per-step work (loop, shuffles, checks) thinner.
constexpr u32 KC = 8;
constexpr u32 STEPC = 32 * KC;
static_assert(STEPC == 2 * STEP, "a count step covers two rank-start mask steps");

struct CStep {
  u32 c[KC];
};

__device__ __forceinline__ void load_c(const TensorArgs& A, u64 q0, int lane, CStep& s) {
  const u64 q = q0 + KC * (u64)lane;
  if (q0 + STEPC <= A.N) {
    const uint4 v0 = *reinterpret_cast<const uint4*>(A.ctx + q);
    const uint4 v1 = *reinterpret_cast<const uint4*>(A.ctx + q + 4);
    s.c[0] = v0.x;
    s.c[1] = v0.y;
    s.c[2] = v0.z;
    s.c[3] = v0.w;
    s.c[4] = v1.x;
    s.c[5] = v1.y;
    s.c[6] = v1.z;
    s.c[7] = v1.w;
  } else {
#pragma unroll
    for (int j = 0; j < (int)KC; ++j) s.c[j] = (q + j < A.N) ? A.ctx[q + j] : NONE32;
  }
}

// Bits of this lane's KC positions (KC lane + j) at or after position f.
__device__ __forceinline__ u32 from_mask8(u32 f, int lane) {
  const int s = (int)f - (int)KC * lane;
  return s <= 0 ? 0xFFu : (s >= (int)KC ? 0u : (0xFFu << s) & 0xFFu);
}

// 64 registers (32 warps per SM): the rotating buffers would take 74 and
// leave room for 24.
template <int NW, u32 TW>
__global__ void __launch_bounds__(NW * 32, 32 / NW) k_tensor_count(const TensorArgs A) {
  constexpr int D = DEPTH_COUNT;
  __shared__ u32 masks[NW][TileW<TW>::MASKW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32* mask = masks[warp];
  const u64 gw = (u64)blockIdx.x * NW + warp;
  const u64 G = (u64)gridDim.x * NW;
  for (u64 t = gw; t < A.n_tiles; t += G) {
    const Tile T = tile_of<TW>(A, t);
    const u32 rsteps = fill_mask<TW>(A, T, mask, lane);
    u32 carry = (T.a > T.sbase) ? A.ctx[T.a - 1] : NONE32;
    u32 heads = 0, ms = 0, cmax = 0;
    bool open = false;  // a row of this tile has started
    // three step buffers in turn (the step being read and the next two in
    // flight): the loop body runs three times per iteration, so no buffer is
    // copied from one step to the next
    static_assert(D == 2, "three step buffers");
    CStep r0, r1, r2;
#pragma unroll
    for (int j = 0; j < (int)KC; ++j) r0.c[j] = r1.c[j] = r2.c[j] = NONE32;
    if (T.a < A.N) load_c(A, T.a, lane, r0);
    if (T.a + STEPC < A.N) load_c(A, T.a + STEPC, lane, r1);
    u64 q0 = T.a;
    // one step from cur, nxt taking the step D ahead; true: the tile is done
    auto step = [&](CStep& cur, CStep& nxt) -> bool {
      const bool tile_step = q0 < T.b;
      if (!tile_step && !open) return true;
      const u64 lim = tile_step ? T.b : T.qrank;
      if (q0 >= lim) return true;
      {
        const u64 qd = q0 + (u64)D * STEPC;
        if (qd < A.N) load_c(A, qd, lane, nxt);
      }
      u32 pc0 = __shfl_up_sync(FULL, cur.c[KC - 1], 1);
      if (lane == 0) pc0 = carry;
      carry = __shfl_sync(FULL, cur.c[KC - 1], 31);
      const u32 si = (u32)(q0 - T.a) / STEP;  // first of the two mask steps
      if (open && q0 + STEPC <= T.b && !((rsteps >> si) & 3u)) {
        // a full tile step inside the tile's rows, no rank start: every
        // change of context is a head, every marker after another context
        // an iteration start
        const u32 m = T.m;
        u32 prev = pc0, h = 0, s2 = 0, cm = 0;
#pragma unroll
        for (int j = 0; j < (int)KC; ++j) {
          const u32 c = cur.c[j];
          const u32 hd = (u32)(c != prev);
          h += hd;
          s2 += (u32)(c == m) & hd;  // a marker after another context is a head
          cm = max(cm, c);
          prev = c;
        }
        heads += h;
        ms += s2;
        cmax = max(cmax, cm);
        if (q0 + STEPC >= T.b && T.b == T.N) return true;  // the set's last tile
      } else {
        const u32 nvalid = (u32)min(lim - q0, (u64)STEPC);
        const u32 rel = (u32)(q0 - T.a) + KC * (u32)lane;
        const u32 rs8 = tile_step ? ((mask[rel >> 5] >> (rel & 31)) & 0xFFu) : 0u;
        const u32 valid8 = (nvalid >= STEPC) ? 0xFFu : ~from_mask8(nvalid, lane) & 0xFFu;
        const u32 m = T.m;
        u32 ms8 = 0, h8 = 0, prev = pc0;
#pragma unroll
        for (int j = 0; j < (int)KC; ++j) {
          const u32 c = cur.c[j];
          const bool rs = (rs8 >> j) & 1u;
          ms8 |= (u32)(c == m && (prev != m || rs)) << j;
          h8 |= (u32)(prev != c || rs) << j;
          if (tile_step && ((valid8 >> j) & 1u)) cmax = max(cmax, c);
          prev = c;
        }
        ms8 &= valid8;
        const u32 st8 = (rs8 & valid8) | ms8;
        h8 = (h8 | st8) & valid8;
        u32 take = h8;
        bool stop = false;
        if (tile_step) ms += __popc(ms8);
        if (!open || !tile_step) {
          const u32 my = st8 ? KC * lane + __ffs(st8) - 1u : 0xFFFFu;
          const u32 f = __reduce_min_sync(FULL, my);
          if (!open) {  // heads from the tile's first row start on
            take = (f < STEPC) ? (h8 & from_mask8(f, lane)) : 0u;
            open = f < STEPC;
          } else {  // continuation: heads before the end of the last row
            take = h8 & ~from_mask8(f, lane);
            stop = f < STEPC || q0 + STEPC >= lim;
          }
        }
        heads += __popc(take);
        if (stop) return true;
        if (tile_step && q0 + STEPC >= T.b && T.b == T.N) return true;  // the set's last tile
      }
      q0 += STEPC;
      return false;
    };
    for (;;) {
      if (step(r0, r2)) break;
      if (step(r1, r0)) break;
      if (step(r2, r1)) break;
    }
    u32 fl = cmax >= T.C ? F_BAD_CTX : 0u;
    heads = __reduce_add_sync(FULL, heads);
    ms = __reduce_add_sync(FULL, ms);
    fl = __reduce_or_sync(FULL, fl);
    if (lane == 0) {
      A.tile_rows[t] = (T.hi - T.lo) + ms;
      A.tile_ents[t] = heads;
      if (fl) flag(A.status, fl);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ write pass --
// Bitmap marking that remembers which words became non-empty, so that the
// union can be cleared by visiting only those words.
struct Touched {
  u32* list;  // [TL]
  u32* cnt;   // [1]
};

__device__ __forceinline__ u32 bm_mark(const Bm& b, const Touched& tw, u32 c) {
  const u32 w = c >> 5, bit = 1u << (c & 31);
  const u32 old = atomicOr(&b.L1[w], bit);
  if (old == 0) {
    atomicOr(&b.L2[w >> 5], 1u << (w & 31));
    const u32 i = atomicAdd(tw.cnt, 1u);
    if (i < TL) tw.list[i] = w;
  }
  return (old & bit) ? 0u : 1u;
}

__device__ __forceinline__ void bm_clear_touched(const Bm& b, const Touched& tw, int lane) {
  __syncwarp();
  const u32 n = *tw.cnt;
  if (n <= TL) {
    for (u32 i = lane; i < n; i += 32) {
      const u32 w = tw.list[i];
      b.L1[w] = 0;
      b.L2[w >> 5] = 0;
    }
  } else {
    bm_clear_warp(b, lane);
  }
  __syncwarp();
  if (lane == 0) *tw.cnt = 0;
  __syncwarp();
}

struct Stage {
  u32* ctx;
  u64* time;
  u32* cnt;
};

// The open row as the write pass closes it.
struct RowEnd {
  u32 k0, k1;    // its runs: heads k0 .. k1 - 1 of the ring (mod RING)
  bool listed;   // all of them are still in the ring
  u64 ts_end;    // the timestamp its last run lasts until
  u32 end_pos;   // end offset from the tile start
  u64 s, e;      // its samples
  bool e_rs;     // e is a rank start (or N): the last sample's duration is 0
};

// Marks the row's contexts from the ring; returns this lane's new bits.
__device__ __forceinline__ u32 mark_ring(const Bm& bm, const Touched& tw, const Head* ring,
                                         const RowEnd& R, int lane) {
  u32 fresh = 0;
  for (u32 k = R.k0 + lane; k < R.k1; k += 32) fresh += bm_mark(bm, tw, ring[k & (RING - 1)].ctx);
  return fresh;
}

// Marks the contexts of row [s, e) by re-reading its samples (rows whose
// runs no longer fit the ring).
__device__ __forceinline__ u32 mark_samples(const TensorArgs& A, const Bm& bm, const Touched& tw,
                                            const RowEnd& R, u32 C, int lane) {
  u32 carry = NONE32, fresh = 0;
  for (u64 g0 = R.s & ~(u64)(STEP - 1); g0 < R.e; g0 += STEP) {
    WStep x;
    load_w(A, g0, lane, x);
    const u64 q = g0 + 4 * (u64)lane;
    u32 pc = __shfl_up_sync(FULL, x.c[3], 1);
    if (lane == 0) pc = carry;
    carry = __shfl_sync(FULL, x.c[3], 31);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 qj = q + j;
      const u32 prev = j ? x.c[j - 1] : pc;
      if (qj >= R.s && qj < R.e && (qj == R.s || prev != x.c[j]))
        fresh += bm_mark(bm, tw, x.c[j] < C ? x.c[j] : 0u);
    }
  }
  return fresh;
}

// Sums the row's runs at their contexts' ranks in the stage (from the ring).
__device__ __forceinline__ void accumulate_ring(const Bm& bm, const Stage& st, const Head* ring,
                                                const RowEnd& R, int lane) {
  for (u32 k = R.k0 + lane; k < R.k1; k += 32) {
    const Head h = ring[k & (RING - 1)];
    u64 t1 = R.ts_end;
    u32 p1 = R.end_pos;
    if (k + 1 < R.k1) {
      const Head n = ring[(k + 1) & (RING - 1)];
      t1 = n.ts;
      p1 = n.pos;
    }
    const u32 r = bm_rank(bm, h.ctx);
    atomicAdd((unsigned long long*)&st.time[r], (unsigned long long)(t1 >= h.ts ? t1 - h.ts : 0ull));
    atomicAdd(&st.cnt[r], p1 - h.pos);
    st.ctx[r] = h.ctx;
  }
}

// Sums the row's samples at their contexts' ranks (rows whose runs no longer
// fit the ring): consecutive equal contexts merged in registers first.
__device__ __forceinline__ void accumulate_samples(const TensorArgs& A, const Bm& bm,
                                                   const Stage& st, const RowEnd& R, u32 C,
                                                   int lane) {
  const u64 s = R.s, e = R.e;
  for (u64 g0 = s & ~(u64)(STEP - 1); g0 < e; g0 += STEP) {
    WStep x;
    load_w(A, g0, lane, x);
    const u64 q = g0 + 4 * (u64)lane;
    u64 t_after = __shfl_down_sync(FULL, x.t[0], 1);  // first timestamp of the next lane
    if (lane == 31 && q + 4 < e) t_after = A.ts[q + 4];
    u32 rc = NONE32, rn = 0;
    u64 rt = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 qj = q + j;
      if (qj < s || qj >= e) continue;
      u64 tn;
      if (qj + 1 < e) tn = (j < 3) ? x.t[j + 1] : t_after;
      else tn = R.e_rs ? x.t[j] : A.ts[e];
      const u64 d = tn >= x.t[j] ? tn - x.t[j] : 0;
      const u32 c = x.c[j] < C ? x.c[j] : 0u;
      if (c == rc) {
        rt += d;
        ++rn;
      } else {
        if (rn) {
          const u32 k = bm_rank(bm, rc);
          atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)rt);
          atomicAdd(&st.cnt[k], rn);
          st.ctx[k] = rc;
        }
        rc = c;
        rt = d;
        rn = 1;
      }
    }
    if (rn) {
      const u32 k = bm_rank(bm, rc);
      atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)rt);
      atomicAdd(&st.cnt[k], rn);
      st.ctx[k] = rc;
    }
  }
}

// Writes the row's distinct contexts in ascending order from slot eo;
// returns how many.  The warp's bitmap holds the union of the contexts of its
// recent rows, with prefix counts (ranks) over it: successive iterations of a
// rank mostly call the same contexts, so the ranks are recomputed only when a
// row brings a context the union lacks, and the union restarts from the row
// when it outgrows the shared-memory stage.
// Template: the run contexts of the warp's last row written by the direct
// path and each run's position; tn = its run count (0: none).
struct Template {
  u32* ctx;            // [FAST_RUNS]
  unsigned char* pos;  // [FAST_RUNS]
};

__device__ __forceinline__ u32 emit_row(const TensorArgs& A, const Bm& bm, const Touched& tw,
                                        const Stage& sm, const Stage& gl, const Head* ring,
                                        u32* stamp, u32 rowid, u32& nb, const Template& tp,
                                        u32& tn, const RowEnd& R, u64 eo, u32 C, int lane) {
  const u32 n = R.k1 - R.k0;
  // Template path: successive iterations of a rank mostly repeat their run
  // sequence exactly, and then every run goes where the template's did.  The
  // runs are written while they are compared; a row that differs anywhere is
  // rewritten below, over all of its positions (direct path) or within its
  // first slots (general path, whose remaining slots no one reads).
  if (R.listed && n == tn) {
    bool same = true;
    u32* const ec = A.e_ctx + eo;
    u64* const et = A.e_time + eo;
    u32* const en = A.e_cnt + eo;
    for (u32 i = lane; i < n; i += 32) {
      const Head h = ring[(R.k0 + i) & (RING - 1)];
      u64 t1 = R.ts_end;
      u32 p1 = R.end_pos;
      if (i + 1 < n) {
        const Head x = ring[(R.k0 + i + 1) & (RING - 1)];
        t1 = x.ts;
        p1 = x.pos;
      }
      same = same && h.ctx == tp.ctx[i];
      const u32 pos = tp.pos[i] < n ? tp.pos[i] : 0u;
      ec[pos] = h.ctx;
      et[pos] = t1 >= h.ts ? t1 - h.ts : 0ull;
      en[pos] = p1 - h.pos;
    }
    if (__all_sync(FULL, same)) return n;
  }
  // Direct path: every run's context is in the union and no two runs share
  // one (each run stamps its union rank with the row's id; finding the id
  // already there means a repeat).  A row holding the whole union writes
  // each run at its rank; otherwise the stamped ranks, as a 128-bit mask,
  // give every run its position.
  if (R.listed && nb > 0 && nb <= RS && n <= FAST_RUNS) {
    u32* const rkb = sm.ctx;  // each run's union rank (the stage is idle on this path)
    bool ok = true;
    for (u32 i = lane; i < n; i += 32) {
      const u32 c = ring[(R.k0 + i) & (RING - 1)].ctx;
      const u32 w = c >> 5, word = bm.L1[w];
      if ((word >> (c & 31)) & 1u) {
        const u32 r = bm.pre[w] + __popc(word & ((1u << (c & 31)) - 1u));
        rkb[i] = r;
        ok = ok && atomicExch(&stamp[r], rowid) != rowid;
      } else {
        ok = false;
      }
    }
    if (__all_sync(FULL, ok)) {
      __syncwarp();
      u32 pm0 = 0, pm1 = 0, pm2 = 0, pm3 = 0;
      const bool whole = n == nb;
      if (!whole) {
        pm0 = __ballot_sync(FULL, vld(&stamp[lane]) == rowid);
        if (nb > 32) pm1 = __ballot_sync(FULL, vld(&stamp[32 + lane]) == rowid);
        if (nb > 64) pm2 = __ballot_sync(FULL, vld(&stamp[64 + lane]) == rowid);
        if (nb > 96) pm3 = __ballot_sync(FULL, vld(&stamp[96 + lane]) == rowid);
      }
      const u32 b1 = __popc(pm0), b2 = b1 + __popc(pm1), b3 = b2 + __popc(pm2);
      u32* const ec = A.e_ctx + eo;
      u64* const et = A.e_time + eo;
      u32* const en = A.e_cnt + eo;
      for (u32 i = lane; i < n; i += 32) {
        const Head h = ring[(R.k0 + i) & (RING - 1)];
        u64 t1 = R.ts_end;
        u32 p1 = R.end_pos;
        if (i + 1 < n) {
          const Head x = ring[(R.k0 + i + 1) & (RING - 1)];
          t1 = x.ts;
          p1 = x.pos;
        }
        const u32 r = rkb[i];
        u32 pos = r;
        if (!whole) {
          const u32 q = r >> 5;
          const u32 pmq = q == 0 ? pm0 : q == 1 ? pm1 : q == 2 ? pm2 : pm3;
          const u32 bq = q == 0 ? 0u : q == 1 ? b1 : q == 2 ? b2 : b3;
          pos = bq + __popc(pmq & ((1u << (r & 31)) - 1u));
        }
        ec[pos] = h.ctx;
        et[pos] = t1 >= h.ts ? t1 - h.ts : 0ull;
        en[pos] = p1 - h.pos;
        tp.ctx[i] = h.ctx;
        tp.pos[i] = (unsigned char)pos;
      }
      tn = n;
      __syncwarp();
      return n;
    }
  }
  tn = 0;  // the general path keeps no template
  // General path: mark the row's contexts into the union (restart it if it
  // would outgrow the stage), recompute ranks if anything was new, sum runs
  // at their ranks, write the present ones in order.
  u32 fresh = R.listed ? mark_ring(bm, tw, ring, R, lane) : mark_samples(A, bm, tw, R, C, lane);
  fresh = __reduce_add_sync(FULL, fresh);
  if (fresh && nb + fresh > RS && nb > 0) {
    bm_clear_touched(bm, tw, lane);
    fresh = R.listed ? mark_ring(bm, tw, ring, R, lane) : mark_samples(A, bm, tw, R, C, lane);
    fresh = __reduce_add_sync(FULL, fresh);
    nb = 0;
  }
  if (fresh) {
    __syncwarp();
    nb = bm_prefix_warp(bm, lane);
  }
  const Stage& st = (nb <= RS) ? sm : gl;
  for (u32 k = lane; k < nb; k += 32) {
    st.time[k] = 0;
    st.cnt[k] = 0;
  }
  __syncwarp();
  if (R.listed) accumulate_ring(bm, st, ring, R, lane);
  else accumulate_samples(A, bm, st, R, C, lane);
  __syncwarp();
  const u32 below = (1u << lane) - 1u;
  u32 nnz = 0;
  for (u32 k0 = 0; k0 < nb; k0 += 32) {
    const u32 k = k0 + lane;
    const u32 cnt = (k < nb) ? st.cnt[k] : 0u;
    const u32 bal = __ballot_sync(FULL, cnt != 0);
    if (cnt) {
      const u64 g = eo + nnz + __popc(bal & below);
      A.e_ctx[g] = st.ctx[k];
      A.e_time[g] = st.time[k];
      A.e_cnt[g] = cnt;
    }
    nnz += __popc(bal);
  }
  __syncwarp();
  return nnz;
}

template <int NW, bool BMS, u32 TW>
__global__ void __launch_bounds__(NW * 32) k_tensor_write(const TensorArgs A) {
  using WriteSmem = ::ta::WriteSmem<TW>;
  constexpr int D = DEPTH_WRITE;
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.C);
  const u32 wbytes = WriteSmem::fixed + (BMS ? bmw * 4 : 0);
  unsigned char* ws = sm + (size_t)warp * wbytes;
  const u64 gw = (u64)blockIdx.x * NW + warp;
  const u64 G = (u64)gridDim.x * NW;
  u32* mask = (u32*)(ws + WriteSmem::mask_off);
  u32* stamp = (u32*)(ws + WriteSmem::stamp_off);
  const Template tpl{(u32*)(ws + WriteSmem::tctx_off), (unsigned char*)(ws + WriteSmem::tpos_off)};
  u32 tn = 0;  // runs of the template (0: none)
  Touched tw;
  tw.list = (u32*)(ws + WriteSmem::tl_off);
  tw.cnt = tw.list + TL;
  if (lane == 0) *tw.cnt = 0;
  for (u32 i = lane; i < RS; i += 32) stamp[i] = NONE32;
  const Bm bm = bm_at(BMS ? (u32*)(ws + WriteSmem::fixed) : A.gbm + gw * bmw, A.C);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  Head* ring = (Head*)(ws + WriteSmem::ring_off);
  Stage sst, gst;
  sst.time = (u64*)(ws + WriteSmem::time_off);
  sst.ctx = (u32*)(ws + WriteSmem::ctx_off);
  sst.cnt = (u32*)(ws + WriteSmem::cnt_off);
  gst.time = A.gst_time + gw * A.gst_cap;
  gst.ctx = A.gst_ctx + gw * A.gst_cap;
  gst.cnt = A.gst_cnt + gw * A.gst_cap;
  u32 nb = 0;        // contexts in the bitmap's union
  u32 rowid = 0;     // rows this warp has closed (stamps of the direct path)
  u64 nnz_warp = 0;  // entries this warp wrote
  __syncwarp();
  for (u64 t = gw; t < A.n_tiles; t += G) {
    const Tile T = tile_of<TW>(A, t);
    const u32 rsteps = fill_mask<TW>(A, T, mask, lane);
    u32 carry = (T.a > T.sbase) ? A.ctx[T.a - 1] : NONE32;
    u64 tcarry = (T.a > T.sbase) ? A.ts[T.a - 1] : 0ull;  // timestamp before the step
    const u64 PR = A.tile_row_off[t], PE = A.tile_ent_off[t];
    // the tile's rows and slots end where the next tile's begin: a count that
    // disagreed with the count pass is reported, never written past
    const u64 row_end = (t + 1 < A.n_tiles) ? A.tile_row_off[t + 1] : A.totals[0];
    const u64 slot_end = (t + 1 < A.n_tiles) ? A.tile_ent_off[t + 1] : A.totals[1];
    u32 rank_ptr = T.lo, rows_local = 0, fl = 0;
    u64 cum = 0;     // slots of this tile's closed rows (their runs)
    u32 nh = 0;      // heads captured in this tile
    bool row_open = false;
    RowEnd R;        // the open row: its start (k0, s) while open
    R.k0 = 0;
    R.s = 0;
    u64 open_row = 0;
    // closes the open row at e (k1 = its heads end); n_top = heads captured
    auto close = [&](u32 k1, u32 n_top, u64 e, bool e_rs, u64 ts_end) {
      R.k1 = k1;
      R.listed = n_top - R.k0 <= RING;
      R.ts_end = ts_end;
      R.end_pos = (u32)(e - T.a);
      R.e = e;
      R.e_rs = e_rs;
      u32 nnz = 0;
      if (PE + cum + (k1 - R.k0) <= slot_end) {
        nnz = emit_row(A, bm, tw, sst, gst, ring, stamp, rowid, nb, tpl, tn, R, PE + cum, T.C,
                       lane);
        if (lane == 0) A.row_nnz[open_row] = nnz;
      } else {
        fl |= F_INTERNAL;
      }
      ++rowid;
      cum += k1 - R.k0;
      nnz_warp += nnz;
      row_open = false;
    };
    WStep ring_s[D + 1];
#pragma unroll
    for (int d = 0; d <= D; ++d) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ring_s[d].c[j] = NONE32;
        ring_s[d].t[j] = 0;
      }
    }
    if (lane >= D && lane < (int)PF) prefetch_step(A, T.a + (u64)lane * STEP);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const u64 qd = T.a + (u64)d * STEP;
      if (qd < A.N) load_w(A, qd, lane, ring_s[d]);
    }
    for (u64 q0 = T.a;; q0 += STEP) {
      const bool tile_step = q0 < T.b;
      if (!tile_step && !row_open) break;
      const u64 lim = tile_step ? T.b : T.qrank;
      if (q0 >= lim) {  // the open row runs to a rank boundary (or N) on a step edge
        if (row_open) close(nh, nh, lim, true, tcarry);
        break;
      }
      if (lane == 0) prefetch_step(A, q0 + (u64)PF * STEP);
      {
        const u64 qd = q0 + (u64)D * STEP;
        if (qd < A.N) load_w(A, qd, lane, ring_s[D]);
      }
      const WStep& cur = ring_s[0];
      u32 pc[4];
      pc[0] = __shfl_up_sync(FULL, cur.c[3], 1);
      if (lane == 0) pc[0] = carry;
      pc[1] = cur.c[0];
      pc[2] = cur.c[1];
      pc[3] = cur.c[2];
      carry = __shfl_sync(FULL, cur.c[3], 31);
      const u64 tprev = tcarry;  // timestamp of sample q0 - 1
      u64 tp = __shfl_up_sync(FULL, cur.t[3], 1);
      if (lane == 0) tp = tprev;
      tcarry = __shfl_sync(FULL, cur.t[3], 31);
      const u32 rel = (u32)(q0 - T.a) + 4u * (u32)lane;
      // per slot j of the lane: run heads (h4), row starts (st4), of which
      // rank starts (rs4) and marker-run starts (ms4)
      u32 h4, st4, rs4 = 0, ms4 = 0;
      // Timestamp order within ranks: no sample earlier than the one before
      // it, except at a rank start (each pair is checked by the tile holding
      // its later sample).
      if (q0 + STEP <= T.b && !((rsteps >> ((u32)(q0 - T.a) / STEP)) & 1u)) {
        // a full tile step without a rank start (the common case)
        const u32 m = T.m;
        h4 = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          h4 |= (u32)(cur.c[j] != pc[j]) << j;
          ms4 |= (u32)(cur.c[j] == m && pc[j] != m) << j;
        }
        st4 = ms4;
        const bool bad = (cur.t[0] < tp) | (cur.t[1] < cur.t[0]) | (cur.t[2] < cur.t[1]) |
                         (cur.t[3] < cur.t[2]);
        if (bad) fl |= F_NOT_SORTED;
      } else {
        const u32 nvalid = (u32)min(lim - q0, (u64)STEP);
        rs4 = tile_step ? ((mask[rel >> 5] >> (rel & 31)) & 0xFu) : 0u;
        const u32 valid4 = (nvalid >= STEP) ? 0xFu : ~from_mask(nvalid, lane) & 0xFu;
        step_bits(cur.c, pc, rs4, valid4, T.m, ms4, st4, h4);
        rs4 &= valid4;
        if (tile_step) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const u64 before = j ? cur.t[j - 1] : tp;
            if (((valid4 >> j) & 1u) && !((rs4 >> j) & 1u) && cur.t[j] < before)
              fl |= F_NOT_SORTED;
          }
        }
      }
      const bool any_st = __any_sync(FULL, st4 != 0);
      if (!row_open && !any_st) {  // nothing of this tile's rows in this step
        if (tile_step && q0 + STEP >= T.b && T.b == T.N) break;
#pragma unroll
        for (int d = 0; d < D; ++d) ring_s[d] = ring_s[d + 1];
        continue;
      }
      // the step's run heads, in sample order, into the ring
      const u32 below = (1u << lane) - 1u;
      u32 before = 0, total = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const u32 hb = __ballot_sync(FULL, (h4 >> j) & 1u);
        before += __popc(hb & below);
      }
      total = __shfl_sync(FULL, before + __popc(h4), 31);
      const u32 base = nh;
      {
        u32 slot = base + before;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if ((h4 >> j) & 1u) {
            // contexts are < C here: the count pass validated every sample
            // before this pass is launched
            const u32 c = cur.c[j];
            *reinterpret_cast<uint4*>(ring + (slot & (RING - 1))) =
                make_uint4((u32)cur.t[j], (u32)(cur.t[j] >> 32), c, rel + (u32)j);
            ++slot;
          }
      }
      __syncwarp();
      const u32 n_top = base + total;
      bool stop = false;
      // row starts in order; each lane's pending starts, start kinds, heads
      // and heads of lower lanes travel in one word
      u32 pend = st4;
      const u32 info = rs4 | (ms4 << 4) | (h4 << 8) | (before << 12);
      for (;;) {
        const u32 lanes = __ballot_sync(FULL, pend != 0);
        if (!lanes) break;
        const u32 L = __ffs(lanes) - 1;
        const u32 in = __shfl_sync(FULL, info | (pend << 24), L);
        const u32 J = __ffs(in >> 24) - 1;
        if (lane == (int)L) pend &= ~(1u << J);
        const u32 prel = 4 * L + J;
        const bool p_rs = (in >> J) & 1u, p_ms = (in >> (4 + J)) & 1u;
        const u32 kp = base + ((in >> 12) & 0xFFu) + __popc((in >> 8) & ((1u << J) - 1u));
        const u64 p = q0 + prel;
        if (row_open) {
          u64 ts_end;
          if (p_rs) {  // the row ends with its rank: its last sample, p - 1
            const u32 n1 = prel - 1;
            const u64 tm = __shfl_sync(FULL, sel4(cur.t, n1 & 3), (n1 >> 2) & 31);
            ts_end = prel ? tm : tprev;
          } else {  // the next row's first sample (the head at p)
            ts_end = ring[kp & (RING - 1)].ts;
          }
          close(kp, n_top, p, p_rs, ts_end);
        }
        if (!tile_step) {  // the continuation found the end of the row
          stop = true;
          break;
        }
        const u64 row0 = PR + rows_local;
        if (!p_rs) {  // an iteration starts (the common case): one row
          if (row0 >= row_end) {
            fl |= F_INTERNAL;
            stop = true;
            break;
          }
          if (lane == 0) A.entry_off[row0] = PE + cum;
          rows_local += 1;
          open_row = row0;
        } else {  // ranks start here (empty ones first), then maybe an iteration
          const u32 r0 = rank_ptr;
          u32 rp = rank_ptr;
          if (lane == 0)
            while (rp < T.hi && A.rank_off[rp] == p) ++rp;
          rp = __shfl_sync(FULL, rp, 0);
          const u32 nrs = rp - rank_ptr;
          rank_ptr = rp;
          const u32 nrow = nrs + (p_ms ? 1u : 0u);
          if (row0 + nrow > row_end) {
            fl |= F_INTERNAL;
            stop = true;
            break;
          }
          for (u32 k = lane; k < nrow; k += 32) {
            A.entry_off[row0 + k] = PE + cum;
            if (k + 1 < nrow) A.row_nnz[row0 + k] = 0;  // empty prologue rows
          }
          for (u32 k = lane; k < nrs; k += 32) A.row_off_of_rank[r0 + k] = row0 + k;
          rows_local += nrow;
          open_row = row0 + nrow - 1;
        }
        row_open = true;
        R.k0 = kp;
        R.s = p;
      }
      nh = n_top;
      if (stop) break;
      if (!tile_step && q0 + STEP >= lim) {  // the row ends at the next rank start (or N)
        if (row_open) close(nh, nh, lim, true, A.ts[lim - 1]);
        break;
      }
      if (tile_step && q0 + STEP >= T.b && T.b == T.N) {  // the set's last tile: rows end at N
        if (row_open) close(nh, nh, T.N, true, A.ts[T.N - 1]);
        break;
      }
#pragma unroll
      for (int d = 0; d < D; ++d) ring_s[d] = ring_s[d + 1];
    }
    u32 n_end = T.last ? T.hi - rank_ptr : 0u;  // empty ranks starting at N
    const u64 row0 = PR + rows_local;
    if (row0 + n_end > row_end) {
      fl |= F_INTERNAL;
      n_end = 0;
    }
    for (u32 k = lane; k < n_end; k += 32) {
      A.entry_off[row0 + k] = PE + cum;
      A.row_nnz[row0 + k] = 0;
      A.row_off_of_rank[T.rhi - n_end + k] = row0 + k;
    }
    fl = __reduce_or_sync(FULL, fl);
    if (lane == 0 && fl) flag(A.status, fl);
    __syncwarp();
  }
  bm_clear_touched(bm, tw, lane);  // leave a global bitmap clean
  if (lane == 0 && nnz_warp) atomicAdd((unsigned long long*)A.nnz_sum, (unsigned long long)nnz_warp);
}

// ------------------------------------------------------------ compaction --
// Rows whose runs repeat a context fill fewer slots than they have runs:
// move every row's entries to their exact place (warp per row).
__global__ void k_compact_rows(const u64* __restrict__ slot_off, const u32* __restrict__ row_nnz,
                               const u64* __restrict__ new_off, u64 rows,
                               const u32* __restrict__ ctx_in, const u64* __restrict__ time_in,
                               const u32* __restrict__ cnt_in, u32* ctx_out, u64* time_out,
                               u32* cnt_out) {
  const int lane = threadIdx.x & 31;
  const u64 G = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 r = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += G) {
    const u64 src = slot_off[r], dst = new_off[r];
    const u32 n = row_nnz[r];
    for (u32 i = lane; i < n; i += 32) {
      ctx_out[dst + i] = ctx_in[src + i];
      time_out[dst + i] = time_in[src + i];
      cnt_out[dst + i] = cnt_in[src + i];
    }
  }
}

}  // namespace

template <u32 TW>
static const void* tensor_kernel_tw(bool write, int nw, bool bms) {
  if (!write) {
    switch (nw) {
      case 4: return (const void*)k_tensor_count<4, TW>;
      case 16: return (const void*)k_tensor_count<16, TW>;
      default: return (const void*)k_tensor_count<8, TW>;
    }
  }
  switch (nw) {
    case 4:
      return bms ? (const void*)k_tensor_write<4, true, TW> : (const void*)k_tensor_write<4, false, TW>;
    case 16:
      return bms ? (const void*)k_tensor_write<16, true, TW>
                 : (const void*)k_tensor_write<16, false, TW>;
    default:
      return bms ? (const void*)k_tensor_write<8, true, TW> : (const void*)k_tensor_write<8, false, TW>;
  }
}

static const void* tensor_kernel(bool write, int nw, bool bms, int tile) {
  return tile == 2048 ? tensor_kernel_tw<2048>(write, nw, bms)
                      : tensor_kernel_tw<TW_DEFAULT>(write, nw, bms);
}

static void set_smem(const void* k, size_t smem) {
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// The bitmap goes to shared memory when it fits beside the default tile's
// layout (the narrower tile's layout is smaller), so the choice does not
// depend on the tile width.
static bool tensor_bm_in_smem(u32 C) {
  return WriteSmem<TW_DEFAULT>::fixed + (size_t)bm_words(C) * 4 <= 14 * 1024;
}

// Dynamic shared memory of a pass (the count pass uses static memory only).
static size_t tensor_smem(u32 C, bool write, int nw, int tile) {
  if (!write) return 0;
  const size_t bm = tensor_bm_in_smem(C) ? (size_t)bm_words(C) * 4 : 0;
  const size_t fixed = tile == 2048 ? WriteSmem<2048>::fixed : WriteSmem<TW_DEFAULT>::fixed;
  return (fixed + bm) * nw;
}

int tensor_max_per_sm(u32 C, bool write, int nw, int tile) {
  const void* k = tensor_kernel(write, nw, write && tensor_bm_in_smem(C), tile);
  const size_t smem = tensor_smem(C, write, nw, tile);
  if (write) set_smem(k, smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nw * 32, smem);
  return std::max(1, occ);
}

TensorPlan plan_tensor(u32 C, u64 N, int num_sms, const TensorShape& shape) {
  TensorPlan P;
  P.tile = shape.tile == 2048 ? 2048 : (int)TW_DEFAULT;
  P.bm_in_smem = tensor_bm_in_smem(C);
  P.nw_count = shape.nw_count;
  P.nw_write = shape.nw_write;
  P.smem_count = tensor_smem(C, false, P.nw_count, P.tile);
  P.smem = tensor_smem(C, true, P.nw_write, P.tile);
  const u64 n_tiles = std::max<u64>(1, (N + P.tile - 1) / P.tile);
  auto grid = [&](bool write, int nw, int per_sm) {
    const int occ = tensor_max_per_sm(C, write, nw, P.tile);
    const int ps = per_sm > 0 ? std::min(per_sm, occ) : occ;
    return (int)std::max<u64>(1, std::min<u64>((u64)num_sms * ps, (n_tiles + nw - 1) / nw));
  };
  P.grid_count = grid(false, P.nw_count, shape.per_sm_count);
  P.grid_write = grid(true, P.nw_write, shape.per_sm_write);
  P.gst_cap = C;
  return P;
}

void launch_tensor_count(const Launch& L, const TensorPlan& P, const TensorArgs& A) {
  void* args[] = {(void*)&A};
  cudaLaunchKernel(tensor_kernel(false, P.nw_count, false, P.tile), P.grid_count,
                   P.nw_count * 32, args, P.smem_count, L.stream);
  L.count();
}

void launch_tile_scan(const Launch& L, const TensorArgs& A) {
  const u64 ns = scan_scratch_elems(A.n_tiles);
  scan_exclusive(L, A.tile_rows, A.n_tiles, A.tile_row_off, A.totals, A.scan_scratch);
  scan_exclusive(L, A.tile_ents, A.n_tiles, A.tile_ent_off, A.totals + 1, A.scan_scratch + ns);
}

void launch_tensor_write(const Launch& L, const TensorPlan& P, const TensorArgs& A) {
  void* args[] = {(void*)&A};
  cudaLaunchKernel(tensor_kernel(true, P.nw_write, P.bm_in_smem, P.tile), P.grid_write,
                   P.nw_write * 32, args, P.smem, L.stream);
  L.count();
}

void launch_tensor_compact(const Launch& L, const TensorCompact& K) {
  scan_exclusive(L, K.row_nnz, K.rows, K.new_off, K.new_off + K.rows, K.scan_scratch);
  const u64 warps = std::min<u64>(std::max<u64>(K.rows, 1), (u64)L.num_sms * 64);
  k_compact_rows<<<(unsigned)((warps + 7) / 8), 256, 0, L.stream>>>(
      K.slot_off, K.row_nnz, K.new_off, K.rows, K.ctx_in, K.time_in, K.cnt_in, K.ctx_out,
      K.time_out, K.cnt_out);
  L.count();
}

}  // namespace ta
