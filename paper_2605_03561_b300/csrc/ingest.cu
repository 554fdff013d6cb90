// ingest.cu -- kernels that turn raw traces into the resident products:
// rank-offset and span validation, calling-context-tree validation and depth,
// the fused validate + duration + iteration-cut + (rank, iteration, context)
// aggregation kernel (the iteration tensor of Section V), and the per-rank
// exclusive / inclusive CSR kernels (Sections II-A and VI-B).
#include <algorithm>

#include "ta_internal.h"

namespace ta {

// ---------------------------------------------------------------------------
// Rank offsets: rank_off[0] = 0, non-decreasing, rank_off[R] = N, every rank
// shorter than 2^32 samples; per-rank span ts_last - ts_first.
__global__ void k_rank_off(const u64* __restrict__ rank_off, u32 R, u64 N,
                           const u64* __restrict__ ts, u64* span, unsigned long long* max_span,
                           u32* status, SetMap sets) {
  const u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > R) return;
  if (r == 0 && rank_off[0] != 0) flag(status, F_INVALID);
  if (r == R) {
    if (rank_off[R] != N) flag(status, F_INVALID);
    return;
  }
  const u64 b = rank_off[r];
  u64 e = rank_off[r + 1];
  if (sets.S) {
    const u32 s = sets.rank_set[r];
    if (r + 1 == sets.set_rank0[s + 1]) e = sets.set_rec_end[s];
  }
  if (e < b || e > N || b > N) {
    flag(status, F_INVALID);
    span[r] = 0;
    return;
  }
  if (e - b > 0xFFFFFFFFull) flag(status, F_INVALID);
  u64 sp = 0;
  if (e > b) {
    const u64 t0 = ts[b], t1 = ts[e - 1];
    sp = t1 >= t0 ? t1 - t0 : 0;  // a decrease is reported by the tensor pass
  }
  span[r] = sp;
  atomicMax(max_span, (unsigned long long)sp);
}

void launch_rank_off(const Launch& L, const u64* rank_off, u32 R, u64 N, const u64* ts,
                     u64* span, u64* max_span, u32* status, const SetMap& sets) {
  const u64 n = (u64)R + 1;
  k_rank_off<<<(unsigned)((n + 255) / 256), 256, 0, L.stream>>>(
      rank_off, R, N, ts, span, (unsigned long long*)max_span, status, sets);
  L.count();
}

// First rank whose samples start at or after each tile start (tile = fixed
// number of samples, tiles never span sets); tfr[n_tiles] = R so the last tile
// also owns the ranks that start at N (empty trailing ranks).
__global__ void k_tile_first_rank(const u64* __restrict__ rank_off, u32 R, u32 tile,
                                  u32 n_tiles, u32* tfr, SetMap sets) {
  const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  if (t == n_tiles) {
    tfr[t] = R;
    return;
  }
  u64 x = (u64)t * tile;
  u32 lo = 0, hi = R;
  if (sets.S) {
    const u32 s = sets.tile_set[t];
    x = sets.set_rec0[s] + (u64)(t - sets.set_tile0[s]) * tile;
    lo = sets.set_rank0[s];
    hi = sets.set_rank0[s + 1];
  }
  while (lo < hi) {
    const u32 mid = lo + (hi - lo) / 2;
    if (rank_off[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  tfr[t] = lo;
}

void launch_tile_first_rank(const Launch& L, const u64* rank_off, u32 R, u32 tile, u32 n_tiles,
                            u32* tfr, const SetMap& sets) {
  const u32 n = n_tiles + 1;
  k_tile_first_rank<<<(n + 255) / 256, 256, 0, L.stream>>>(rank_off, R, tile, n_tiles, tfr, sets);
  L.count();
}

// ---------------------------------------------------------------------------
// Calling context tree: one root, parents in range, acyclic; depth of every
// node by pointer jumping (log2 C rounds); a node that has not reached the
// root after 2^rounds >= C jumps lies on a cycle.
__global__ void k_cct_init(const u32* __restrict__ parent, u32 C, u32* anc, u32* dep, u32* roots,
                           u32* status, SetMap sets) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  const u32 p = parent[v];
  u32 s = 0, base = 0, Cs = C;
  if (sets.S) {
    s = set_of_ctx(sets, v);
    base = sets.set_ctx0[s];
    Cs = sets.set_C[s];
  }
  if (p == NONE32) {
    atomicAdd(&roots[s], 1u);
    anc[v] = NONE32;
    dep[v] = 0;
  } else if (p >= Cs) {
    flag(status, F_BAD_CCT);
    anc[v] = NONE32;
    dep[v] = 0;
  } else {
    anc[v] = base + p;
    dep[v] = 1;
  }
}

__global__ void k_cct_jump(const u32* __restrict__ anc_in, const u32* __restrict__ dep_in,
                           u32* anc_out, u32* dep_out, u32 C) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  const u32 a = anc_in[v];
  if (a != NONE32) {
    dep_out[v] = min(dep_in[v] + dep_in[a], 0x7FFFFFFFu);
    anc_out[v] = anc_in[a];
  } else {
    dep_out[v] = dep_in[v];
    anc_out[v] = NONE32;
  }
}

__global__ void k_cct_final(const u32* __restrict__ anc, const u32* __restrict__ dep, u32 C,
                            u32* depth, u32* max_depth, u32* status) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  if (anc[v] != NONE32) flag(status, F_BAD_CCT);
  depth[v] = dep[v];
  atomicMax(max_depth, dep[v]);
}

void launch_cct(const Launch& L, const u32* parent, u32 C, u32* depth, u32* max_depth,
                u32* roots, u32* scratch, u32* status, const SetMap& sets) {
  u32* anc0 = scratch;
  u32* dep0 = scratch + C;
  u32* anc1 = scratch + 2 * (u64)C;
  u32* dep1 = scratch + 3 * (u64)C;
  const unsigned g = (C + 255) / 256;
  k_cct_init<<<g, 256, 0, L.stream>>>(parent, C, anc0, dep0, roots, status, sets);
  int rounds = 1;
  while (rounds < 40 && (1ull << rounds) < (u64)C) ++rounds;
  for (int i = 0; i < rounds; ++i) {
    k_cct_jump<<<g, 256, 0, L.stream>>>(anc0, dep0, anc1, dep1, C);
    std::swap(anc0, anc1);
    std::swap(dep0, dep1);
  }
  k_cct_final<<<g, 256, 0, L.stream>>>(anc0, dep0, C, depth, max_depth, status);
  L.count(2 + rounds);
}

__global__ void k_n_iter(const u64* __restrict__ row_off_of_rank, u32 R, u32* n_iter) {
  const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) n_iter[r] = (u32)(row_off_of_rank[r + 1] - row_off_of_rank[r] - 1);
}

// ---------------------------------------------------------------------------
// Ancestor lists: context v's list is v, parent(v), ..., the root.
__global__ void k_anc_len(const u32* __restrict__ depth, u32 C, u32* len) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < C) len[v] = depth[v] + 1;
}

__global__ void k_anc_fill(const u32* __restrict__ parent, u32 C, const u64* __restrict__ anc_off,
                           u32* anc, SetMap sets) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  const u32 base = sets.S ? sets.set_ctx0[set_of_ctx(sets, v)] : 0u;
  u64 q = anc_off[v];
  const u64 q1 = anc_off[v + 1];
  u32 c = v - base;  // local id
  while (q < q1) {
    anc[q++] = c;
    const u32 p = parent[base + c];
    if (p == NONE32) break;
    c = p;
  }
}

void launch_anc_offsets(const Launch& L, const u32* depth, u32 C, u32* len, u64* anc_off,
                        u64* total, u64* scratch) {
  k_anc_len<<<(C + 255) / 256, 256, 0, L.stream>>>(depth, C, len);
  L.count();
  scan_exclusive(L, len, C, anc_off, total, scratch);
  cudaMemcpyAsync(anc_off + C, total, 8, cudaMemcpyDeviceToDevice, L.stream);
}

void launch_anc_fill(const Launch& L, const u32* parent, u32 C, const u64* anc_off, u32* anc,
                     const SetMap& sets) {
  k_anc_fill<<<(C + 255) / 256, 256, 0, L.stream>>>(parent, C, anc_off, anc, sets);
  L.count();
}

void launch_n_iter(const Launch& L, const u64* row_off_of_rank, u32 R, u32* n_iter) {
  k_n_iter<<<(R + 255) / 256, 256, 0, L.stream>>>(row_off_of_rank, R, n_iter);
  L.count();
}

// ---------------------------------------------------------------------------
// The iteration tensor (Section V): two passes over warp tiles, no waiting.
//
// A tile is TW consecutive samples; it owns the rows (rank prologues and
// iterations) that START inside it and reads past its end to finish its last
// row.  Every warp takes tiles grid-stride and streams a tile 128 samples at a
// time (4 per lane, 16-byte vector loads, the next step prefetched while the
// current one is processed): rank starts and marker-run starts cut rows; each
// run head of a row sets its context's bit in the warp's two-level bitmap.
//   count pass (contexts only): per tile, rows and distinct entries (bitmap
//     popcount per row); also validates context ids.
//   a device scan of the per-tile counts gives every tile its row and entry
//     offsets and the exact output sizes.
//   write pass (contexts and timestamps): validates timestamp order; per row a
//     prefix over the bitmap ranks its contexts in ascending order, a second
//     pass over the row's samples (cache-resident, consecutive equal contexts
//     merged in registers first) accumulates time and count at those ranks in
//     shared memory, and the row is written straight to its final place.
// No tile ever waits for another, so uneven tiles (long rows, rank
// boundaries) cost only their own work.
namespace {

constexpr u32 TW = 4096;   // samples per tile
constexpr u32 MASKW = TW / 32 + 4;  // rank-start mask words (positions 0 .. TW)
constexpr int DEPTH = 3;   // steps prefetched ahead (count pass)
constexpr u32 STEP = 128;  // samples per warp step (4 per lane)
constexpr u32 RS = 128;    // staged entries per warp in shared memory

constexpr u32 TL = 128;    // touched bitmap words remembered per row
constexpr u32 RL = 128;    // run heads remembered per row (write pass)

struct WarpSmem {
  static constexpr u32 mask_off = 0;                  // u32[MASKW] rank-start mask
  static constexpr u32 tl_off = 4 * MASKW;            // u32[TL + 4] touched words, count
  static constexpr u32 time_off = tl_off + 4 * (TL + 4);  // u64[RS] (16-byte aligned)
  static constexpr u32 ctx_off = time_off + 8 * RS;
  static constexpr u32 cnt_off = ctx_off + 4 * RS;
  static constexpr u32 run_ts_off = cnt_off + 4 * RS;     // u64[RL] run-head timestamps
  static constexpr u32 run_ctx_off = run_ts_off + 8 * RL;  // u32[RL] run contexts
  static constexpr u32 run_pos_off = run_ctx_off + 4 * RL;  // u32[RL] offsets in the row
  static constexpr u32 bm_off = run_pos_off + 4 * RL;     // bitmap words (16-byte aligned)
  static constexpr u32 fixed_count = time_off;        // count pass: mask + touched list
  static constexpr u32 fixed_write = bm_off;
};

// Bitmap marking that also remembers which words became non-empty, so the
// row's bitmap can be cleared by visiting only those words.  The count pass
// keeps no summary level (with_l2 = false): it only needs the number of new
// bits, and a row that touches more than TL words is cleared in full.
struct Touched {
  u32* list;  // [TL]
  u32* cnt;   // [1]
};

template <bool WITH_L2>
__device__ __forceinline__ u32 bm_mark(const Bm& b, const Touched& tw, u32 c) {
  const u32 w = c >> 5, bit = 1u << (c & 31);
  const u32 old = atomicOr(&b.L1[w], bit);
  if (old == 0) {
    if (WITH_L2) atomicOr(&b.L2[w >> 5], 1u << (w & 31));
    const u32 i = atomicAdd(tw.cnt, 1u);
    if (i < TL) tw.list[i] = w;
  }
  return (old & bit) ? 0u : 1u;
}

template <bool WITH_L2>
__device__ __forceinline__ void bm_clear_touched(const Bm& b, const Touched& tw, int lane) {
  __syncwarp();
  const u32 n = *tw.cnt;
  if (n <= TL) {
    for (u32 i = lane; i < n; i += 32) {
      const u32 w = tw.list[i];
      b.L1[w] = 0;
      if (WITH_L2) b.L2[w >> 5] = 0;
    }
  } else if (WITH_L2) {
    bm_clear_warp(b, lane);
  } else {
    for (u32 i = lane; i < b.W1; i += 32) b.L1[i] = 0;
  }
  __syncwarp();
  if (lane == 0) *tw.cnt = 0;
  __syncwarp();
}

// Element j (warp-uniform or per-lane) of a 4-element register array without
// dynamic register indexing.
__device__ __forceinline__ u64 sel4(const u64* v, u32 j) {
  return j == 0 ? v[0] : j == 1 ? v[1] : j == 2 ? v[2] : v[3];
}

struct Step {
  u32 c[4];
  u64 t[4];
};

// Load samples q0 + 4 lane + j (j < 4); contexts always, timestamps if want_ts.
__device__ __forceinline__ void load_step(const TensorArgs& A, u64 q0, int lane, bool want_ts,
                                          Step& s) {
  const u64 q = q0 + 4 * (u64)lane;
  if (q + 3 < A.N) {
    const uint4 cv = *reinterpret_cast<const uint4*>(A.ctx + q);
    s.c[0] = cv.x;
    s.c[1] = cv.y;
    s.c[2] = cv.z;
    s.c[3] = cv.w;
    if (want_ts) {
      const ulonglong2 t0 = *reinterpret_cast<const ulonglong2*>(A.ts + q);
      const ulonglong2 t1 = *reinterpret_cast<const ulonglong2*>(A.ts + q + 2);
      s.t[0] = t0.x;
      s.t[1] = t0.y;
      s.t[2] = t1.x;
      s.t[3] = t1.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s.c[j] = (q + j < A.N) ? A.ctx[q + j] : NONE32;
      if (want_ts) s.t[j] = (q + j < A.N) ? A.ts[q + j] : 0ull;
    }
  }
}

// Distinct contexts of the row in the bitmap (count pass).
__device__ __forceinline__ u32 bm_count_warp(const Bm& b, int lane) {
  u32 sum = 0;
  for (u32 g = 0; g < b.W2; g += 32) {
    const u32 w2 = g + lane;
    const u32 bits = (w2 < b.W2) ? vld(&b.L2[w2]) : 0u;
    for (u32 x = bits; x; x &= x - 1) sum += __popc(vld(&b.L1[w2 * 32 + __ffs(x) - 1]));
  }
  return __reduce_add_sync(FULL, sum);
}

struct Stage {
  u32* ctx;
  u64* time;
  u32* cnt;
};

// The write pass remembers the run heads of the open row (a run = samples of
// one context in a row, in order): its context, first timestamp and offset in
// the row.  A run lasts until the next run head, the last one until the row
// end, so its time is a difference of two head timestamps (the per-sample
// durations telescope) and its samples a difference of two offsets.
struct RunList {
  u64* ts;
  u32* ctx;
  u32* pos;
};

// Appends this lane's run heads (bits j of h4 among its 4 samples at q..q+3)
// to the list after the nrun already there; returns the warp's head count.
__device__ __forceinline__ u32 capture_runs(const RunList& rl, u32 nrun, u32 h4, const u32* c,
                                            const u64* t, u64 q, u64 row_s, u32 C, int lane) {
  // heads of lower lanes, from one ballot per sample slot
  const u32 below = (1u << lane) - 1u;
  u32 before = 0, total = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const u32 b = __ballot_sync(FULL, (h4 >> j) & 1u);
    before += __popc(b & below);
    total += __popc(b);
  }
  u32 slot = nrun + before;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if ((h4 >> j) & 1u) {
      if (slot < RL) {
        rl.ctx[slot] = c[j] < C ? c[j] : 0u;
        rl.ts[slot] = t[j];
        rl.pos[slot] = (u32)(q + j - row_s);
      }
      ++slot;
    }
  return total;
}


// Accumulates the row's runs (nrun <= RL) at their contexts' ranks.
__device__ __forceinline__ void accumulate_runs(const Bm& bm, const Stage& st, const RunList& rl,
                                                u32 nrun, u64 ts_end, u32 len, int lane) {
  for (u32 k = lane; k < nrun; k += 32) {
    const u64 t0 = rl.ts[k];
    const u32 p0 = rl.pos[k];
    const bool more = k + 1 < nrun;
    const u64 t1 = more ? rl.ts[k + 1] : ts_end;
    const u32 p1 = more ? rl.pos[k + 1] : len;
    const u32 c = rl.ctx[k];
    const u32 r = bm_rank(bm, c);
    atomicAdd((unsigned long long*)&st.time[r], (unsigned long long)(t1 >= t0 ? t1 - t0 : 0ull));
    atomicAdd(&st.cnt[r], p1 - p0);
    st.ctx[r] = c;
  }
}

// Write pass, one row [s, e) whose ranks are in the bitmap: accumulate time
// and count at each context's rank in the stage, then write the row at entry
// eo.  The stage is shared memory or the warp's global region (compile time).
__device__ __forceinline__ void accumulate_row(const TensorArgs& A, const Bm& bm, const Stage& st,
                                               u64 s, u64 e, bool e_rs, u32 C, int lane) {
  for (u64 g0 = s & ~(u64)(STEP - 1); g0 < e; g0 += STEP) {
    Step x;
    load_step(A, g0, lane, true, x);
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
      else tn = e_rs ? x.t[j] : A.ts[e];
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

// Marks the contexts of row [s, e) by re-reading its samples (rows with more
// runs than the run list holds).
__device__ __forceinline__ u32 mark_row_samples(const TensorArgs& A, const Bm& bm,
                                                const Touched& tw, u64 s, u64 e, u32 C,
                                                int lane) {
  u32 carry = NONE32, fresh = 0;
  for (u64 g0 = s & ~(u64)(STEP - 1); g0 < e; g0 += STEP) {
    Step x;
    load_step(A, g0, lane, false, x);
    const u64 q = g0 + 4 * (u64)lane;
    u32 pc = __shfl_up_sync(FULL, x.c[3], 1);
    if (lane == 0) pc = carry;
    carry = __shfl_sync(FULL, x.c[3], 31);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 qj = q + j;
      const u32 prev = j ? x.c[j - 1] : pc;
      if (qj >= s && qj < e && (qj == s || prev != x.c[j]))
        fresh += bm_mark<true>(bm, tw, x.c[j] < C ? x.c[j] : 0u);
    }
  }
  return fresh;
}


// Marks the row's contexts from its run list; returns this lane's new bits.
__device__ __forceinline__ u32 mark_runs_new(const Bm& bm, const Touched& tw, const RunList& rl,
                                             u32 nrun, int lane) {
  u32 fresh = 0;
  for (u32 k = lane; k < nrun; k += 32) fresh += bm_mark<true>(bm, tw, rl.ctx[k]);
  return fresh;
}

// Writes the open row [s, e) (write pass).  The warp's bitmap holds the
// union of the contexts of its recent rows, not only this row's: successive
// iterations of a rank mostly call the same contexts, so the ranks (the
// prefix counts over the bitmap) are recomputed only when a row brings a
// context the union lacks, and the union restarts from the row when it
// outgrows the shared-memory stage.  Times and counts are staged at union
// ranks and the contexts the row has are written in order, compacted.  Runs
// come from the run list, or from re-reading the samples of rows with more
// runs than it holds.  ts_end is the timestamp the last run lasts until: the
// sample at e, or the last sample when e ends the rank.
__device__ __forceinline__ u32 write_row(const TensorArgs& A, const Bm& bm, const Touched& tw,
                                         const Stage& sm, const Stage& gl, const RunList& rl,
                                         u32& nb, u32 nrun, u64 ts_end, u64 s, u64 e, bool e_rs,
                                         u64 eo, u32 C, int lane) {
  const bool listed = nrun <= RL;
  // Fast path, the common case of iterations that repeat: every context of
  // the row is already in the union and each appears in one run only.  Then
  // the runs' union ranks are distinct (checked by storing each run's index
  // at its rank and reading it back), a 128-bit mask of the ranks present
  // gives each run its entry position, and every run is written straight to
  // its entry.
  if (listed && nb > 0 && nb <= RS) {
    u32* present = sm.ctx;  // 4 words of the stage serve as the rank mask
    if (lane < RS / 32) present[lane] = 0;
    __syncwarp();
    u32 rk[RL / 32];
    bool ok = true;
#pragma unroll
    for (u32 it = 0; it < RL / 32; ++it) {
      const u32 k = lane + 32 * it;
      rk[it] = 0;
      if (k < nrun) {
        const u32 c = rl.ctx[k], w = c >> 5, word = bm.L1[w];
        ok = ok && ((word >> (c & 31)) & 1u);
        rk[it] = bm.pre[w] + __popc(word & ((1u << (c & 31)) - 1u));
        if (ok) {
          sm.cnt[rk[it]] = k;
          atomicOr(&present[rk[it] >> 5], 1u << (rk[it] & 31));
        }
      }
    }
    if (__all_sync(FULL, ok)) {
      __syncwarp();
#pragma unroll
      for (u32 it = 0; it < RL / 32; ++it) {
        const u32 k = lane + 32 * it;
        if (k < nrun) ok = ok && sm.cnt[rk[it]] == k;
      }
      if (__all_sync(FULL, ok)) {
        u32 pm[RS / 32], before[RS / 32 + 1];
        before[0] = 0;
#pragma unroll
        for (u32 q = 0; q < RS / 32; ++q) {
          pm[q] = present[q];
          before[q + 1] = before[q] + __popc(pm[q]);
        }
#pragma unroll
        for (u32 it = 0; it < RL / 32; ++it) {
          const u32 k = lane + 32 * it;
          if (k < nrun) {
            const u32 r = rk[it];
            u32 pos = 0;
#pragma unroll
            for (u32 q = 0; q < RS / 32; ++q)
              if (q == (r >> 5)) pos = before[q] + __popc(pm[q] & ((1u << (r & 31)) - 1u));
            const u64 t0 = rl.ts[k];
            const u32 p0 = rl.pos[k];
            const bool more = k + 1 < nrun;
            const u64 t1 = more ? rl.ts[k + 1] : ts_end;
            const u32 p1 = more ? rl.pos[k + 1] : (u32)(e - s);
            const u64 g = eo + pos;
            A.e_ctx[g] = rl.ctx[k];
            A.e_time[g] = t1 >= t0 ? t1 - t0 : 0ull;
            A.e_cnt[g] = p1 - p0;
          }
        }
        __syncwarp();
        return before[RS / 32];
      }
    }
    __syncwarp();
  }
  u32 fresh = listed ? mark_runs_new(bm, tw, rl, nrun, lane)
                     : mark_row_samples(A, bm, tw, s, e, C, lane);
  fresh = __reduce_add_sync(FULL, fresh);
  if (fresh && nb + fresh > RS && nb > 0) {  // restart the union from this row
    bm_clear_touched<true>(bm, tw, lane);
    fresh = listed ? mark_runs_new(bm, tw, rl, nrun, lane)
                   : mark_row_samples(A, bm, tw, s, e, C, lane);
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
  if (listed) accumulate_runs(bm, st, rl, nrun, ts_end, (u32)(e - s), lane);
  else accumulate_row(A, bm, st, s, e, e_rs, C, lane);
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
  return nnz;
}

}  // namespace

template <int NW, bool WRITE, bool BMS>
__global__ void __launch_bounds__(NW * 32) k_tensor_pass(const TensorArgs A) {
  constexpr int D = WRITE ? 2 : DEPTH;  // steps in flight (the write pass holds timestamps too)
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.C);
  const u32 fixed = WRITE ? WarpSmem::fixed_write : WarpSmem::fixed_count;
  const u32 wbytes = fixed + (BMS ? bmw * 4 : 0);
  unsigned char* ws = sm + (size_t)warp * wbytes;
  const u64 gw = (u64)blockIdx.x * NW + warp;
  const u64 G = (u64)gridDim.x * NW;
  u32* mask = (u32*)(ws + WarpSmem::mask_off);
  Touched tw;
  tw.list = (u32*)(ws + WarpSmem::tl_off);
  tw.cnt = tw.list + TL;
  if (lane == 0) *tw.cnt = 0;
  const Bm bm = bm_at(BMS ? (u32*)(ws + fixed) : A.gbm + gw * bmw, A.C);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  Stage sst, gst;
  RunList rl;
  if (WRITE) {
    rl.ts = (u64*)(ws + WarpSmem::run_ts_off);
    rl.ctx = (u32*)(ws + WarpSmem::run_ctx_off);
    rl.pos = (u32*)(ws + WarpSmem::run_pos_off);
    sst.time = (u64*)(ws + WarpSmem::time_off);
    sst.ctx = (u32*)(ws + WarpSmem::ctx_off);
    sst.cnt = (u32*)(ws + WarpSmem::cnt_off);
    gst.time = A.gst_time + gw * A.gst_cap;
    gst.ctx = A.gst_ctx + gw * A.gst_cap;
    gst.cnt = A.gst_cnt + gw * A.gst_cap;
  }
  u32 nb = 0;  // write pass: contexts in the bitmap's union
  __syncwarp();
  for (u64 t = gw; t < A.n_tiles; t += G) {
    // the tile's trace set (a single experiment is one set)
    u64 sbase = 0, N = A.N, t0 = 0, t1 = A.n_tiles;
    u32 rlo = 0, rhi = A.R, C = A.C, m = A.m;
    if (A.sets.S) {
      const u32 s = A.sets.tile_set[t];
      sbase = A.sets.set_rec0[s];
      N = A.sets.set_rec_end[s];
      t0 = A.sets.set_tile0[s];
      t1 = A.sets.set_tile0[s + 1];
      rlo = A.sets.set_rank0[s];
      rhi = A.sets.set_rank0[s + 1];
      C = A.sets.set_C[s];
      m = A.sets.set_m[s];
    }
    const u64 a = sbase + (t - t0) * TW;
    const u64 b = min(a + (u64)TW, N);
    const bool last = (t + 1 == t1);
    const u32 lo = A.tfr[t], hi = last ? rhi : A.tfr[t + 1];
    const u64 qrank = (hi < rhi) ? A.rank_off[hi] : N;  // first rank start >= b (or N)
    u32 carry = (a > sbase) ? A.ctx[a - 1] : NONE32;
    u64 tcarry = (WRITE && a > sbase) ? A.ts[a - 1] : 0ull;  // timestamp before the step
    u64 PR = 0, PE = 0;
    if (WRITE) {
      PR = A.tile_row_off[t];
      PE = A.tile_ent_off[t];
    }
    for (u32 i = lane; i < MASKW; i += 32) mask[i] = 0;
    __syncwarp();
    for (u32 r = lo + lane; r < hi; r += 32) {
      const u32 p = (u32)(A.rank_off[r] - a);
      atomicOr(&mask[p >> 5], 1u << (p & 31));
    }
    __syncwarp();

    u32 rank_ptr = lo, rows_local = 0, fl = 0;
    u32 fresh = 0;  // count pass: contexts this lane saw first in the open row
    u32 nrun = 0;   // write pass: run heads of the open row so far
    u64 cum = 0;
    bool row_open = false;
    u64 row_s = 0;
    // ring of steps: ring[0] is processed while ring[1 .. D] are in flight
    Step ring[D + 1];
#pragma unroll
    for (int d = 0; d <= D; ++d) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ring[d].c[j] = NONE32;
        ring[d].t[j] = 0;
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const u64 qd = a + (u64)d * STEP;
      if (qd < A.N) load_step(A, qd, lane, WRITE, ring[d]);
    }
    for (u64 q0 = a;; q0 += STEP) {
      const bool tile_step = q0 < b;
      if (!tile_step && !row_open) break;
      const u64 lim = tile_step ? b : qrank;
      if (q0 >= lim) {  // the open row runs to a rank boundary (or N)
        if (row_open) {
          if (WRITE)
            cum += write_row(A, bm, tw, sst, gst, rl, nb, nrun, A.ts[lim - 1], row_s, lim, true,
                             PE + cum, C, lane);
          else {
            cum += __reduce_add_sync(FULL, fresh);
            fresh = 0;
            bm_clear_touched<false>(bm, tw, lane);
          }
        }
        row_open = false;
        break;
      }
      Step& cur = ring[0];
      const u64 q1 = q0 + STEP;
      {
        const u64 qd = q0 + (u64)D * STEP;
        if (qd < A.N) load_step(A, qd, lane, WRITE, ring[D]);
      }
      const u64 q = q0 + 4 * (u64)lane;
      // samples of this step that exist (tile steps: below b; continuation:
      // below the next rank start)
      const u32 nvalid = (u32)min(lim - q0, (u64)STEP);
      const u32 pos0 = 4u * (u32)lane;
      u32 pc[4];
      pc[0] = __shfl_up_sync(FULL, cur.c[3], 1);
      if (lane == 0) pc[0] = carry;
      pc[1] = cur.c[0];
      pc[2] = cur.c[1];
      pc[3] = cur.c[2];
      carry = __shfl_sync(FULL, cur.c[3], 31);
      const u64 tprev = tcarry;  // timestamp of sample q0 - 1
      if (WRITE) tcarry = __shfl_sync(FULL, cur.t[3], 31);
      const u32 rel = (u32)(q - a);
      // rank-start bits of this lane's 4 samples (positions rel .. rel + 3)
      const u32 rs4 = tile_step ? ((mask[rel >> 5] >> (rel & 31)) & 0xFu) : 0u;
      u32 ms4 = 0, valid4 = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool valid = pos0 + j < nvalid;
        valid4 |= (valid ? 1u : 0u) << j;
        const bool ms = cur.c[j] == m && (pc[j] != m || ((rs4 >> j) & 1u));
        ms4 |= (ms ? 1u : 0u) << j;
      }
      ms4 &= valid4;
      if (tile_step) {
        if (!WRITE) {
          u32 cmax = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if ((valid4 >> j) & 1u) cmax = max(cmax, cur.c[j]);
          if (cmax >= C) fl |= F_BAD_CTX;
        } else {
          // timestamp order within ranks: no sample earlier than the one
          // before it, except at a rank start (each pair is checked by the
          // tile holding its later sample)
          u64 tp = __shfl_up_sync(FULL, cur.t[3], 1);
          if (lane == 0) tp = tprev;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const u64 before = j ? cur.t[j - 1] : tp;
            if (((valid4 >> j) & 1u) && !((rs4 >> j) & 1u) && cur.t[j] < before)
              fl |= F_NOT_SORTED;
          }
        }
      }
      const u32 st4_any = (rs4 & valid4) | ms4;
      if (!__any_sync(FULL, st4_any != 0)) {
        // fast path: no row starts in this step; mark the run heads of the
        // open row
        if (row_open) {
          u32 h4 = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (((valid4 >> j) & 1u) && pc[j] != cur.c[j]) {
              h4 |= 1u << j;
              if (!WRITE) fresh += bm_mark<false>(bm, tw, cur.c[j] < C ? cur.c[j] : 0u);
            }
          if (WRITE) nrun += capture_runs(rl, nrun, h4, cur.c, cur.t, q, row_s, C, lane);
        }
        if (q1 >= b && b == N) {  // the last tile: rows end at N
          if (row_open) {
            if (WRITE)
              cum += write_row(A, bm, tw, sst, gst, rl, nb, nrun, A.ts[N - 1], row_s, N, true,
                               PE + cum, C, lane);
            else {
              cum += __reduce_add_sync(FULL, fresh);
              fresh = 0;
              bm_clear_touched<false>(bm, tw, lane);
            }
          }
          row_open = false;
          break;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) ring[d] = ring[d + 1];
        continue;
      }
      u32 cc[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) cc[j] = cur.c[j] < C ? cur.c[j] : 0u;
      const u32 st4 = st4_any;
      u32 seg_lo = 0, from = 0;
      bool stop = false;
      for (;;) {
        u32 mypos = 255;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
          const u32 pos = 4 * lane + j;
          if (((st4 >> j) & 1u) && pos >= from) mypos = pos;
        }
        const u32 nxt = __reduce_min_sync(FULL, mypos);
        const u32 end = nxt < STEP ? nxt : STEP;
        if (row_open) {
          u32 h4 = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const u32 pos = pos0 + j;
            if (((valid4 >> j) & 1u) && pos >= seg_lo && pos < end)
              if (q + j == row_s || pc[j] != cur.c[j]) {
                h4 |= 1u << j;
                if (!WRITE) fresh += bm_mark<false>(bm, tw, cc[j]);
              }
          }
          if (WRITE) nrun += capture_runs(rl, nrun, h4, cur.c, cur.t, q, row_s, C, lane);
        }
        if (nxt >= STEP) break;
        const u64 p = q0 + nxt;
        const u32 src = nxt >> 2, bj = nxt & 3;
        const bool p_rs = (__shfl_sync(FULL, rs4, src) >> bj) & 1u;
        const bool p_ms = (__shfl_sync(FULL, ms4, src) >> bj) & 1u;
        if (row_open) {
          if (WRITE) {
            // timestamp the last run lasts until: sample p, or p - 1 at a rank start
            const u32 n1 = nxt - 1;
            const u64 tp = __shfl_sync(FULL, sel4(cur.t, bj), src);
            const u64 tm = __shfl_sync(FULL, sel4(cur.t, n1 & 3), (n1 >> 2) & 31);
            const u64 ts_end = p_rs ? (nxt ? tm : tprev) : tp;
            cum += write_row(A, bm, tw, sst, gst, rl, nb, nrun, ts_end, row_s, p, p_rs, PE + cum, C,
                             lane);
          }
          else {
            cum += __reduce_add_sync(FULL, fresh);
            fresh = 0;
            bm_clear_touched<false>(bm, tw, lane);
          }
        }
        if (!tile_step) {  // the continuation found the end of the row
          row_open = false;
          stop = true;
          break;
        }
        u32 nrs = 0, r0 = rank_ptr;
        if (p_rs) {
          u32 rp = rank_ptr;
          if (lane == 0)
            while (rp < hi && A.rank_off[rp] == p) ++rp;
          rp = __shfl_sync(FULL, rp, 0);
          nrs = rp - rank_ptr;
          rank_ptr = rp;
        }
        const u32 nrow = nrs + (p_ms ? 1u : 0u);
        if (WRITE) {
          const u64 row0 = PR + rows_local;
          for (u32 k = lane; k < nrow; k += 32) A.entry_off[row0 + k] = PE + cum;
          for (u32 k = lane; k < nrs; k += 32) A.row_off_of_rank[r0 + k] = row0 + k;
        }
        rows_local += nrow;
        row_open = true;
        row_s = p;
        nrun = 0;
        seg_lo = nxt;
        from = nxt + 1;
      }
      if (stop) break;
      if (q1 >= b && b == N) {  // the last tile: rows end at N
        if (row_open) {
          if (WRITE)
            cum += write_row(A, bm, tw, sst, gst, rl, nb, nrun, A.ts[N - 1], row_s, N, true,
                             PE + cum, C, lane);
          else {
            cum += __reduce_add_sync(FULL, fresh);
            fresh = 0;
            bm_clear_touched<false>(bm, tw, lane);
          }
        }
        row_open = false;
        break;
      }
#pragma unroll
      for (int d = 0; d < D; ++d) ring[d] = ring[d + 1];
    }
    fl = __reduce_or_sync(FULL, fl);
    if (lane == 0 && fl) flag(A.status, fl);
    const u32 n_end = last ? hi - rank_ptr : 0u;  // empty ranks starting at N
    if (WRITE) {
      const u64 row0 = PR + rows_local;
      for (u32 k = lane; k < n_end; k += 32) {
        A.entry_off[row0 + k] = PE + cum;
        A.row_off_of_rank[rhi - n_end + k] = row0 + k;
      }
    } else if (lane == 0) {
      A.tile_rows[t] = rows_local + n_end;
      A.tile_ents[t] = cum;
    }
    __syncwarp();
  }
  if (WRITE) bm_clear_touched<true>(bm, tw, lane);  // leave a global bitmap clean
}

static void set_smem(const void* k, size_t smem) {
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <bool WRITE>
static const void* tensor_kernel(int nw, bool bms) {
  switch (nw) {
    case 4:
      return bms ? (const void*)k_tensor_pass<4, WRITE, true> : (const void*)k_tensor_pass<4, WRITE, false>;
    case 16:
      return bms ? (const void*)k_tensor_pass<16, WRITE, true> : (const void*)k_tensor_pass<16, WRITE, false>;
    default:
      return bms ? (const void*)k_tensor_pass<8, WRITE, true> : (const void*)k_tensor_pass<8, WRITE, false>;
  }
}

static bool tensor_bm_in_smem(u32 C) {
  return WarpSmem::fixed_write + (size_t)bm_words(C) * 4 <= 12 * 1024;
}

static size_t tensor_smem(u32 C, bool write, int nw) {
  const size_t bm = tensor_bm_in_smem(C) ? (size_t)bm_words(C) * 4 : 0;
  return (size_t)((write ? WarpSmem::fixed_write : WarpSmem::fixed_count) + bm) * nw;
}

int tensor_max_per_sm(u32 C, bool write, int nw) {
  const void* k = write ? tensor_kernel<true>(nw, tensor_bm_in_smem(C))
                        : tensor_kernel<false>(nw, tensor_bm_in_smem(C));
  const size_t smem = tensor_smem(C, write, nw);
  set_smem(k, smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nw * 32, smem);
  return std::max(1, occ);
}

TensorPlan plan_tensor(u32 C, u64 N, int num_sms, const TensorShape& shape) {
  TensorPlan P;
  P.tile = TW;
  P.bm_in_smem = tensor_bm_in_smem(C);
  P.nw_count = shape.nw_count;
  P.nw_write = shape.nw_write;
  P.smem_count = tensor_smem(C, false, P.nw_count);
  P.smem = tensor_smem(C, true, P.nw_write);
  const u64 n_tiles = std::max<u64>(1, (N + TW - 1) / TW);
  auto grid = [&](bool write, int nw, int per_sm) {
    const int occ = tensor_max_per_sm(C, write, nw);
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
  cudaLaunchKernel(tensor_kernel<false>(P.nw_count, P.bm_in_smem), P.grid_count,
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
  cudaLaunchKernel(tensor_kernel<true>(P.nw_write, P.bm_in_smem), P.grid_write, P.nw_write * 32,
                   args, P.smem, L.stream);
  L.count();
}

// ---------------------------------------------------------------------------
// Per-rank CSR of distinct contexts, one warp per rank (grid-stride), in two
// passes with a scan between them (no rank waits for another):
//  mode 0 (exclusive, Section V): the union of the rank's tensor rows, summed.
//  mode 1 (inclusive, Sections II-A / VI-B): the ancestor closure of the
//    rank's exclusive contexts; values rolled up level by level from the
//    rank's deepest level to the root (every node of depth d adds into its
//    parent before any node of depth d-1 is read: a level-synchronous sweep).
// count pass: distinct contexts per rank -> out_cnt[r].  write pass: offsets
// from the scan; rank, accumulate (and sweep) in shared memory; write.
namespace {

constexpr u32 RSR = 256;           // staged entries per warp in shared memory
constexpr u32 DEPTH_BUCKETS = 64;  // depth range handled by the bucket sweep
constexpr u32 BUCKET_MAX = 1024;   // closure size handled by the bucket sweep
constexpr int RU = 8;              // entries per lane in flight (exclusive)

struct RankSmem {
  static constexpr u32 time_off = 0;                 // u64[RSR]
  static constexpr u32 ctx_off = 8 * RSR;            // u32[RSR]
  static constexpr u32 cnt_off = ctx_off + 4 * RSR;  // u32[RSR]
  static constexpr u32 dep_off = cnt_off + 4 * RSR;  // u32[RSR] (inclusive)
  static constexpr u32 par_off = dep_off + 4 * RSR;  // u32[RSR] (inclusive)
  static constexpr u32 bucket_off = par_off + 4 * RSR;  // u32[DEPTH_BUCKETS + 1], u16[BUCKET_MAX]
  static constexpr u32 fixed_write =
      (bucket_off + 4 * (DEPTH_BUCKETS + 1) + 2 * BUCKET_MAX + 15) & ~15u;
  static constexpr u32 fixed_write0 = dep_off;  // exclusive: time, ctx, cnt only
};

// Inclusive through ancestor lists: a stage of time, ctx, cnt only, larger
// (an inclusive set is the closure of the exclusive one).
constexpr u32 RSR2 = 512;
struct RankSmem2 {
  static constexpr u32 time_off = 0;
  static constexpr u32 ctx_off = 8 * RSR2;
  static constexpr u32 cnt_off = ctx_off + 4 * RSR2;
  static constexpr u32 fixed_write = cnt_off + 4 * RSR2;
};

struct RStage {
  u64* time;
  u32* ctx;
  u32* cnt;
  u32* dep;
  u32* par;
};

}  // namespace

template <int NW, int MODE, bool WRITE, bool BMS>
__global__ void __launch_bounds__(NW * 32) k_rank_pass(const RankCsrArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.C);
  const u32 fixed = !WRITE ? 0u
                    : MODE == 0 ? RankSmem::fixed_write0
                    : MODE == 1 ? RankSmem::fixed_write
                                : RankSmem2::fixed_write;
  const u32 wbytes = fixed + (BMS ? bmw * 4 : 0);
  unsigned char* ws = sm + (size_t)warp * wbytes;
  const u64 gw = (u64)blockIdx.x * NW + warp;
  const u64 G = (u64)gridDim.x * NW;
  const Bm bm = bm_at(BMS ? (u32*)(ws + fixed) : A.gbm + gw * bmw, A.C);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  RStage ss, gs;
  u32* bucket_base = nullptr;
  if (WRITE && MODE == 2) {
    ss.time = (u64*)(ws + RankSmem2::time_off);
    ss.ctx = (u32*)(ws + RankSmem2::ctx_off);
    ss.cnt = (u32*)(ws + RankSmem2::cnt_off);
    const u64 gbase = gw * (u64)A.gst_cap;
    gs.time = A.gst_time + gbase;
    gs.ctx = A.gst_ctx + gbase;
    gs.cnt = A.gst_cnt + gbase;
  } else if (WRITE) {
    ss.time = (u64*)(ws + RankSmem::time_off);
    ss.ctx = (u32*)(ws + RankSmem::ctx_off);
    ss.cnt = (u32*)(ws + RankSmem::cnt_off);
    if (MODE == 1) {
      ss.dep = (u32*)(ws + RankSmem::dep_off);
      ss.par = (u32*)(ws + RankSmem::par_off);
      bucket_base = (u32*)(ws + RankSmem::bucket_off);
    }
    const u64 gbase = gw * (u64)A.gst_cap;
    gs.time = A.gst_time + gbase;
    gs.ctx = A.gst_ctx + gbase;
    gs.cnt = A.gst_cnt + gbase;
    gs.dep = A.gst_dep + gbase;
    gs.par = A.gst_par + gbase;
  }
  __syncwarp();
  for (u64 r = gw; r < A.R; r += G) {
    // context ids are local to the rank's set; tree arrays are concatenated
    const u32 cbase = A.sets.S ? A.sets.set_ctx0[A.sets.rank_set[r]] : 0u;
    u64 E0, E1;
    if (MODE == 0) {
      E0 = A.entry_off[A.row_off_of_rank[r]];
      E1 = A.entry_off[A.row_off_of_rank[r + 1]];
      for (u64 j0 = E0; j0 < E1; j0 += 32 * RU) {
        u32 c[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const u64 j = j0 + 32 * u + lane;
          c[u] = j < E1 ? A.in_ctx[j] : NONE32;
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
          if (c[u] != NONE32 && !bm_has(bm, c[u])) bm_set(bm, c[u]);
      }
    } else if (MODE == 1) {
      E0 = A.in_off[r];
      E1 = A.in_off[r + 1];
      for (u64 j = E0 + lane; j < E1; j += 32) {
        u32 c = A.in_ctx[j];
        for (u32 step = 0; c != NONE32 && step <= A.max_depth; ++step) {
          if (bm_test_set(bm, c)) break;
          c = A.parent[cbase + c];
        }
      }
    } else {  // the closure: every ancestor of every exclusive context
      E0 = A.in_off[r];
      E1 = A.in_off[r + 1];
      for (u64 j = E0 + lane; j < E1; j += 32) {
        const u32 x = A.in_ctx[j];
        const u64 a1 = A.anc_off[cbase + x + 1];
        for (u64 q = A.anc_off[cbase + x]; q < a1; q += 4) {
          u32 a[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = (q + u < a1) ? A.anc[q + u] : NONE32;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (a[u] != NONE32 && !bm_has(bm, a[u])) bm_set(bm, a[u]);
        }
      }
    }
    __syncwarp();
    if (!WRITE) {
      const u32 n = bm_count_warp(bm, lane);
      if (lane == 0) A.out_cnt[r] = n;
      bm_clear_warp(bm, lane);
      __syncwarp();
      continue;
    }
    const u32 nnz = bm_prefix_warp(bm, lane);
    auto run = [&](const RStage& st) {
    for (u32 k = lane; k < nnz; k += 32) {
      st.time[k] = 0;
      st.cnt[k] = 0;
    }
    __syncwarp();
    if (MODE == 0) {
      for (u64 j0 = E0; j0 < E1; j0 += 32 * RU) {
        u32 c[RU], n[RU];
        u64 t[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const u64 j = j0 + 32 * u + lane;
          const bool ok = j < E1;
          c[u] = ok ? A.in_ctx[j] : NONE32;
          t[u] = ok ? A.in_time[j] : 0ull;
          n[u] = ok ? A.in_cnt[j] : 0u;
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          if (c[u] == NONE32) continue;
          const u32 k = bm_rank(bm, c[u]);
          atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)t[u]);
          atomicAdd(&st.cnt[k], n[u]);
          st.ctx[k] = c[u];
        }
      }
    } else if (MODE == 2) {
      // each exclusive value goes to every context on its root path
      for (u64 j = E0 + lane; j < E1; j += 32) {
        const u32 x = A.in_ctx[j];
        const u64 t = A.in_time[j];
        const u32 n = A.in_cnt[j];
        const u64 a1 = A.anc_off[cbase + x + 1];
        for (u64 q = A.anc_off[cbase + x]; q < a1; q += 4) {
          u32 a[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = (q + u < a1) ? A.anc[q + u] : NONE32;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (a[u] == NONE32) continue;
            const u32 k = bm_rank(bm, a[u]);
            atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)t);
            atomicAdd(&st.cnt[k], n);
            st.ctx[k] = a[u];
          }
        }
      }
    } else {
      bm_enumerate_warp(bm, st.ctx, lane);
      __syncwarp();
      u32 maxd = 0;
      for (u32 k = lane; k < nnz; k += 32) {
        const u32 c = st.ctx[k];
        const u32 d = A.depth[cbase + c];
        st.dep[k] = d;
        st.par[k] = d > 0 ? bm_rank(bm, A.parent[cbase + c]) : NONE32;
        maxd = max(maxd, d);
      }
      maxd = __reduce_max_sync(FULL, maxd);
      for (u64 j = E0 + lane; j < E1; j += 32) {
        const u32 k = bm_rank(bm, A.in_ctx[j]);
        st.time[k] = A.in_time[j];
        st.cnt[k] = A.in_cnt[j];
      }
      __syncwarp();
      if (maxd < DEPTH_BUCKETS && nnz <= BUCKET_MAX) {
        // order the entries by depth (counting sort in shared memory), then
        // roll up one level at a time from the deepest: O(entries + depth)
        u32* hist = bucket_base;
        uint16_t* order = (uint16_t*)(bucket_base + DEPTH_BUCKETS + 1);
        for (u32 d = lane; d <= DEPTH_BUCKETS; d += 32) hist[d] = 0;
        __syncwarp();
        for (u32 k = lane; k < nnz; k += 32) atomicAdd(&hist[st.dep[k]], 1u);
        __syncwarp();
        if (lane == 0) {
          u32 run = 0;
          for (u32 d = 0; d <= maxd; ++d) {
            const u32 h = hist[d];
            hist[d] = run;
            run += h;
          }
          hist[maxd + 1] = run;
        }
        __syncwarp();
        for (u32 k = lane; k < nnz; k += 32) {
          const u32 slot = atomicAdd(&hist[st.dep[k]], 1u);
          order[slot] = (uint16_t)k;
        }
        __syncwarp();
        // after the scatter hist[d] is the end of bucket d = start of d + 1
        for (u32 d = maxd; d >= 1; --d) {
          const u32 b0 = hist[d - 1], b1 = hist[d];
          for (u32 i = b0 + lane; i < b1; i += 32) {
            const u32 k = order[i];
            const u32 kp = st.par[k];
            atomicAdd((unsigned long long*)&st.time[kp], (unsigned long long)vld(&st.time[k]));
            atomicAdd(&st.cnt[kp], vld(&st.cnt[k]));
          }
          __syncwarp();
        }
      } else {
        for (u32 d = maxd; d >= 1; --d) {
          for (u32 k = lane; k < nnz; k += 32) {
            if (st.dep[k] == d) {
              const u32 kp = st.par[k];
              atomicAdd((unsigned long long*)&st.time[kp], (unsigned long long)vld(&st.time[k]));
              atomicAdd(&st.cnt[kp], vld(&st.cnt[k]));
            }
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
    const u64 eo = A.out_off[r];
    for (u32 k = lane; k < nnz; k += 32) {
      A.out_ctx[eo + k] = vld(&st.ctx[k]);
      A.out_time[eo + k] = vld(&st.time[k]);
      A.out_cnt_e[eo + k] = vld(&st.cnt[k]);
    }
    };
    if (nnz <= (MODE == 2 ? RSR2 : RSR)) run(ss);
    else run(gs);
    bm_clear_warp(bm, lane);
    __syncwarp();
  }
}

constexpr int RANK_NW = 8;

RankCsrPlan plan_rank_csr(u32 R, u32 C, int num_sms) {
  RankCsrPlan P;
  P.threads = RANK_NW * 32;
  const size_t bm = (size_t)bm_words(C) * 4;
  P.bm_in_smem = RankSmem::fixed_write + bm <= 16 * 1024;
  const size_t bms = P.bm_in_smem ? bm : 0;
  P.smem[0][0] = P.smem[1][0] = P.smem[2][0] = bms * RANK_NW;
  P.smem[0][1] = (RankSmem::fixed_write0 + bms) * RANK_NW;
  P.smem[1][1] = (RankSmem::fixed_write + bms) * RANK_NW;
  P.smem[2][1] = (RankSmem2::fixed_write + bms) * RANK_NW;
  const void* ks[3][2];
  if (P.bm_in_smem) {
    ks[0][0] = (const void*)k_rank_pass<RANK_NW, 0, false, true>;
    ks[0][1] = (const void*)k_rank_pass<RANK_NW, 0, true, true>;
    ks[1][0] = (const void*)k_rank_pass<RANK_NW, 1, false, true>;
    ks[1][1] = (const void*)k_rank_pass<RANK_NW, 1, true, true>;
    ks[2][0] = (const void*)k_rank_pass<RANK_NW, 2, false, true>;
    ks[2][1] = (const void*)k_rank_pass<RANK_NW, 2, true, true>;
  } else {
    ks[0][0] = (const void*)k_rank_pass<RANK_NW, 0, false, false>;
    ks[0][1] = (const void*)k_rank_pass<RANK_NW, 0, true, false>;
    ks[1][0] = (const void*)k_rank_pass<RANK_NW, 1, false, false>;
    ks[1][1] = (const void*)k_rank_pass<RANK_NW, 1, true, false>;
    ks[2][0] = (const void*)k_rank_pass<RANK_NW, 2, false, false>;
    ks[2][1] = (const void*)k_rank_pass<RANK_NW, 2, true, false>;
  }
  for (int m = 0; m < 3; ++m)
    for (int w = 0; w < 2; ++w) {
      cudaFuncSetAttribute(ks[m][w], cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)P.smem[m][w]);
      int o = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, ks[m][w], P.threads, P.smem[m][w]);
      P.grid[m][w] = (int)std::max<u64>(
          1, std::min<u64>((u64)num_sms * std::max(o, 1), ((u64)R + RANK_NW - 1) / RANK_NW));
    }
  P.n_units = R;
  P.gst_cap = C;
  return P;
}

template <int MODE, bool WRITE>
static void rank_launch(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A) {
  const size_t smem = P.smem[MODE][WRITE ? 1 : 0];
  const int grid = P.grid[MODE][WRITE ? 1 : 0];
  if (P.bm_in_smem) k_rank_pass<RANK_NW, MODE, WRITE, true><<<grid, P.threads, smem, L.stream>>>(A);
  else k_rank_pass<RANK_NW, MODE, WRITE, false><<<grid, P.threads, smem, L.stream>>>(A);
}

void launch_rank_count(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A) {
  if (A.mode == 0) rank_launch<0, false>(L, P, A);
  else if (A.anc) rank_launch<2, false>(L, P, A);
  else rank_launch<1, false>(L, P, A);
  L.count();
  scan_exclusive(L, A.out_cnt, A.R, A.out_off, A.total, A.scan_scratch);
  cudaMemcpyAsync(A.out_off + A.R, A.total, 8, cudaMemcpyDeviceToDevice, L.stream);
}

void launch_rank_write(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A) {
  if (A.mode == 0) rank_launch<0, true>(L, P, A);
  else if (A.anc) rank_launch<2, true>(L, P, A);
  else rank_launch<1, true>(L, P, A);
  L.count();
}

}  // namespace ta
