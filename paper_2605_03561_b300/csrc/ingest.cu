// ingest.cu -- kernels that turn raw traces into the resident products:
// rank-offset and span validation, calling-context-tree validation and depth,
// ancestor lists, and the per-rank exclusive / inclusive CSR kernels
// (Sections II-A and VI-B).  The iteration tensor is in tensor.cu.
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

// Exclusive fast path: the iteration rows of rank r (its rows after the
// first) as one template block.  Returns true when every such row holds the
// first one's contexts -- rows are context-sorted, so entry p of every row is
// then the same context -- with at most 96 of them; tc holds them and tt / tn
// each position's time and samples summed over the rows, ql / qh the 128-bit
// sum of the squared times (lane l: positions l, l + 32, l + 64; four rows'
// loads in flight, one vote per row).  The rank's first row (its prologue)
// is [p0, p1), left to the caller.
constexpr u32 XT_P = 3;  // positions per lane
constexpr u32 XT_R = 4;  // rows in flight
__device__ __forceinline__ bool excl_template(const RankCsrArgs& A, u64 r, int lane,
                                              u32 (&tc)[XT_P], u64 (&tt)[XT_P],
                                              u32 (&tn)[XT_P], u64 (&ql)[XT_P],
                                              u64 (&qh)[XT_P], u64& p0, u64& p1) {
  const u64 R0 = A.row_off_of_rank[r], R1 = A.row_off_of_rank[r + 1];
  if (R1 < R0 + 3) return false;  // fewer than two iteration rows: nothing to gain
  p0 = A.entry_off[R0];
  p1 = A.entry_off[R0 + 1];
  const u64 b0 = p1;
  const u64 L64 = A.entry_off[R0 + 2] - b0;
  if (L64 == 0 || L64 > 32 * XT_P) return false;
  const u32 L = (u32)L64;
#pragma unroll
  for (u32 q = 0; q < XT_P; ++q) {
    const u32 p = (u32)lane + 32 * q;
    tc[q] = p < L ? A.in_ctx[b0 + p] : NONE32;
    tt[q] = 0;
    tn[q] = 0;
    ql[q] = 0;
    qh[q] = 0;
  }
  const u64 nrow = R1 - R0 - 1;
  for (u64 j0 = 0; j0 < nrow; j0 += 32) {
    const u32 m = (u32)(nrow - j0 < 32 ? nrow - j0 : 32);
    // every row of the block is L entries long: row j starts at b0 + j L
    const bool okl = (u32)lane > m ||
                     A.entry_off[R0 + 1 + j0 + lane] == b0 + (j0 + (u32)lane) * (u64)L;
    if (!__all_sync(FULL, okl)) return false;
    for (u32 w0 = 0; w0 < m; w0 += XT_R) {
      u32 c[XT_R][XT_P], n[XT_R][XT_P];
      u64 t[XT_R][XT_P];
#pragma unroll
      for (u32 w = 0; w < XT_R; ++w)
#pragma unroll
        for (u32 q = 0; q < XT_P; ++q) {
          const u32 p = (u32)lane + 32 * q;
          const bool live = w0 + w < m && p < L;
          const u64 e = b0 + (j0 + w0 + w) * (u64)L + p;
          c[w][q] = live ? A.in_ctx[e] : tc[q];
          t[w][q] = live ? A.in_time[e] : 0ull;
          n[w][q] = live ? A.in_cnt[e] : 0u;
        }
      bool ok = true;
#pragma unroll
      for (u32 w = 0; w < XT_R; ++w)
#pragma unroll
        for (u32 q = 0; q < XT_P; ++q) ok = ok && c[w][q] == tc[q];
      if (!__all_sync(FULL, ok)) return false;
#pragma unroll
      for (u32 w = 0; w < XT_R; ++w)
#pragma unroll
        for (u32 q = 0; q < XT_P; ++q) {
          tt[q] += t[w][q];
          tn[q] += n[w][q];
          const u64 lo = t[w][q] * t[w][q];
          ql[q] += lo;
          qh[q] += __umul64hi(t[w][q], t[w][q]) + (ql[q] < lo ? 1ull : 0ull);
        }
    }
  }
  return true;
}

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
  // inclusive through ancestor lists: a rank whose exclusive contexts equal
  // the warp's previous rank's (ranks of one program mostly call the same)
  // keeps that rank's closure bitmap and prefix counts
  u64 pE0 = 0, pE1 = 0;
  u32 p_cbase = NONE32, p_nnz = 0;
  bool kept = false;  // the bitmap holds the previous rank's closure
  for (u64 r = gw; r < A.R; r += G) {
    if (MODE == 0 && WRITE && A.only_over && A.out_cnt[r] <= A.xs_cap) continue;
    // context ids are local to the rank's set; tree arrays are concatenated
    const u32 cbase = A.sets.S ? A.sets.set_ctx0[A.sets.rank_set[r]] : 0u;
    bool same = false;
    if (MODE == 2 && kept) {
      const u64 q0 = A.in_off[r], q1 = A.in_off[r + 1];
      if (q1 - q0 == pE1 - pE0 && cbase == p_cbase) {
        bool eq = true;
        for (u64 j = lane; j < q1 - q0; j += 32) eq = eq && A.in_ctx[q0 + j] == A.in_ctx[pE0 + j];
        same = __all_sync(FULL, eq);
      }
      if (!same) {
        bm_clear_warp(bm, lane);
        __syncwarp();
        kept = false;
      }
    }
    u64 E0, E1;
    // exclusive: the iteration rows as a template block when they allow it
    u32 xtc[XT_P];
    u64 xtt[XT_P], xql[XT_P], xqh[XT_P], xp0 = 0, xp1 = 0;
    u32 xtn[XT_P];
    const bool tmpl =
        MODE == 0 && WRITE && excl_template(A, r, lane, xtc, xtt, xtn, xql, xqh, xp0, xp1);
    if (MODE == 0 && tmpl) {  // marks: the template's contexts and the first row's
      E0 = A.entry_off[A.row_off_of_rank[r]];
      E1 = A.entry_off[A.row_off_of_rank[r + 1]];
#pragma unroll
      for (u32 q = 0; q < XT_P; ++q)
        if (xtc[q] != NONE32 && !bm_has(bm, xtc[q])) bm_set(bm, xtc[q]);
      for (u64 j = xp0 + lane; j < xp1; j += 32) {
        const u32 c = A.in_ctx[j];
        if (!bm_has(bm, c)) bm_set(bm, c);
      }
    } else if (MODE == 0) {
      E0 = A.entry_off[A.row_off_of_rank[r]];
      E1 = A.entry_off[A.row_off_of_rank[r + 1]];
      // entries as 32-bit offsets from the rank's first (a rank holds fewer
      // than 2^32 samples, so fewer entries); the next batch's contexts are
      // loaded before this batch is marked
      const u32* const cx = A.in_ctx + E0;
      const u32 ne = (u32)(E1 - E0);
      u32 c[RU];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const u32 j = 32 * u + lane;
        c[u] = j < ne ? cx[j] : NONE32;
      }
      for (u32 j0 = 0; j0 < ne; j0 += 32 * RU) {
        u32 cn[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const u32 j = j0 + 32 * RU + 32 * u + lane;
          cn[u] = j < ne ? cx[j] : NONE32;
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
          if (c[u] != NONE32 && !bm_has(bm, c[u])) bm_set(bm, c[u]);
#pragma unroll
        for (int u = 0; u < RU; ++u) c[u] = cn[u];
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
      for (u64 j = E0 + lane; j < E1 && !same; j += 32) {
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
      const u32 n = same ? p_nnz : bm_count_warp(bm, lane);
      if (lane == 0) A.out_cnt[r] = n;
      if (MODE == 2) {
        pE0 = E0;
        pE1 = E1;
        p_cbase = cbase;
        p_nnz = n;
        kept = true;
      } else {
        bm_clear_warp(bm, lane);
      }
      __syncwarp();
      continue;
    }
    const u32 nnz = same ? p_nnz : bm_prefix_warp(bm, lane);
    const bool scratch = MODE == 0 && A.xs_cap && !A.only_over;
    if (scratch) {
      if (lane == 0) {
        A.out_cnt[r] = nnz;
        if (nnz > A.xs_cap) atomicAdd(A.n_over, 1ull);
      }
      if (nnz > A.xs_cap) {  // left to the write pass over the ranks above the cap
        bm_clear_warp(bm, lane);
        __syncwarp();
        continue;
      }
    }
    auto run = [&](const RStage& st) {
    for (u32 k = lane; k < nnz; k += 32) {
      st.time[k] = 0;
      st.cnt[k] = 0;
    }
    __syncwarp();
    if (MODE == 0 && tmpl) {  // the template block's sums, then the first row's entries
#pragma unroll
      for (u32 q = 0; q < XT_P; ++q) {
        if (xtc[q] == NONE32) continue;
        const u32 k = bm_rank(bm, xtc[q]);
        atomic_add_u64_lo32((unsigned long long*)&st.time[k], xtt[q]);
        atomicAdd(&st.cnt[k], xtn[q]);
        st.ctx[k] = xtc[q];
      }
      for (u64 j = xp0 + lane; j < xp1; j += 32) {
        const u32 c = A.in_ctx[j];
        const u32 k = bm_rank(bm, c);
        atomic_add_u64_lo32((unsigned long long*)&st.time[k], A.in_time[j]);
        atomicAdd(&st.cnt[k], A.in_cnt[j]);
        st.ctx[k] = c;
      }
    } else if (MODE == 0) {
      // two batches of RA entries per lane: the next is loaded while this
      // one is added
      constexpr int RA = RU / 2;
      const u32* const cx = A.in_ctx + E0;
      const u64* const tx = A.in_time + E0;
      const u32* const nx = A.in_cnt + E0;
      const u32 ne = (u32)(E1 - E0);
      u32 c[RA], n[RA];
      u64 t[RA];
      auto load = [&](u32 j0, u32* cc, u64* tt, u32* nn) {
#pragma unroll
        for (int u = 0; u < RA; ++u) {
          const u32 j = j0 + 32 * u + lane;
          const bool ok = j < ne;
          cc[u] = ok ? cx[j] : NONE32;
          tt[u] = ok ? tx[j] : 0ull;
          nn[u] = ok ? nx[j] : 0u;
        }
      };
      load(0, c, t, n);
      for (u32 j0 = 0; j0 < ne; j0 += 32 * RA) {
        u32 cn[RA], nn[RA];
        u64 tn[RA];
        load(j0 + 32 * RA, cn, tn, nn);
#pragma unroll
        for (int u = 0; u < RA; ++u) {
          if (c[u] == NONE32) continue;
          const u32 k = bm_rank(bm, c[u]);
          atomic_add_u64_lo32((unsigned long long*)&st.time[k], (u64)t[u]);
          atomicAdd(&st.cnt[k], n[u]);
          st.ctx[k] = c[u];
        }
#pragma unroll
        for (int u = 0; u < RA; ++u) {
          c[u] = cn[u];
          t[u] = tn[u];
          n[u] = nn[u];
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
            atomic_add_u64_lo32((unsigned long long*)&st.time[k], (u64)t);
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
            atomic_add_u64_lo32((unsigned long long*)&st.time[kp], (u64)vld(&st.time[k]));
            atomicAdd(&st.cnt[kp], vld(&st.cnt[k]));
          }
          __syncwarp();
        }
      } else {
        for (u32 d = maxd; d >= 1; --d) {
          for (u32 k = lane; k < nnz; k += 32) {
            if (st.dep[k] == d) {
              const u32 kp = st.par[k];
              atomic_add_u64_lo32((unsigned long long*)&st.time[kp], (u64)vld(&st.time[k]));
              atomicAdd(&st.cnt[kp], vld(&st.cnt[k]));
            }
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
    if (scratch) {
      const u64 eo = r * (u64)A.xs_cap;
      for (u32 k = lane; k < nnz; k += 32) {
        A.xs_ctx[eo + k] = vld(&st.ctx[k]);
        A.xs_time[eo + k] = vld(&st.time[k]);
        A.xs_cnt[eo + k] = vld(&st.cnt[k]);
      }
    } else {
      const u64 eo = A.out_off[r];
      for (u32 k = lane; k < nnz; k += 32) {
        A.out_ctx[eo + k] = vld(&st.ctx[k]);
        A.out_time[eo + k] = vld(&st.time[k]);
        A.out_cnt_e[eo + k] = vld(&st.cnt[k]);
      }
    }
    if (MODE == 0 && A.mom_ok) {  // iteration moments: the template's, 0 elsewhere
      if (lane == 0) A.mom_ok[r] = tmpl ? 1 : 0;
      if (tmpl) {
        const u64 eo = scratch ? r * (u64)A.xs_cap : A.out_off[r];
        u64* const m1 = (scratch ? A.xs_m1 : A.out_m1) + eo;
        ulonglong2* const m2 = reinterpret_cast<ulonglong2*>(scratch ? A.xs_m2 : A.out_m2) + eo;
        for (u32 k = lane; k < nnz; k += 32) {
          m1[k] = 0;
          m2[k] = make_ulonglong2(0, 0);
        }
        __syncwarp();
#pragma unroll
        for (u32 q = 0; q < XT_P; ++q) {
          if (xtc[q] == NONE32) continue;
          const u32 k = bm_rank(bm, xtc[q]);
          m1[k] = xtt[q];
          m2[k] = make_ulonglong2(xql[q], xqh[q]);
        }
      }
    }
    };
    if (nnz <= (MODE == 2 ? RSR2 : RSR)) run(ss);
    else run(gs);
    if (MODE == 2) {
      pE0 = E0;
      pE1 = E1;
      p_cbase = cbase;
      p_nnz = nnz;
      kept = true;
    } else {
      bm_clear_warp(bm, lane);
    }
    __syncwarp();
  }
  if (MODE == 2 && kept) bm_clear_warp(bm, lane);  // leave a global bitmap clean
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

// Scratch rows of at most xs_cap contexts to their CSR place, warp per rank.
__global__ void k_excl_copy(const RankCsrArgs A) {
  const int lane = threadIdx.x & 31;
  const u64 G = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 r = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < A.R; r += G) {
    const u32 n = A.out_cnt[r];
    if (n > A.xs_cap) continue;
    const u64 src = r * (u64)A.xs_cap, dst = A.out_off[r];
    for (u32 k = lane; k < n; k += 32) {
      A.out_ctx[dst + k] = A.xs_ctx[src + k];
      A.out_time[dst + k] = A.xs_time[src + k];
      A.out_cnt_e[dst + k] = A.xs_cnt[src + k];
    }
    if (A.mom_ok && A.mom_ok[r]) {
      const ulonglong2* m2s = reinterpret_cast<const ulonglong2*>(A.xs_m2) + src;
      ulonglong2* m2d = reinterpret_cast<ulonglong2*>(A.out_m2) + dst;
      for (u32 k = lane; k < n; k += 32) {
        A.out_m1[dst + k] = A.xs_m1[src + k];
        m2d[k] = m2s[k];
      }
    }
  }
}

void launch_excl_scratch(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A) {
  rank_launch<0, true>(L, P, A);
  L.count();
  scan_exclusive(L, A.out_cnt, A.R, A.out_off, A.total, A.scan_scratch);
  cudaMemcpyAsync(A.out_off + A.R, A.total, 8, cudaMemcpyDeviceToDevice, L.stream);
}

void launch_excl_copy(const Launch& L, const RankCsrArgs& A) {
  const u64 warps = std::min<u64>(std::max<u64>(A.R, 1), (u64)L.num_sms * 64);
  k_excl_copy<<<(unsigned)((warps + 7) / 8), 256, 0, L.stream>>>(A);
  L.count();
}

void launch_rank_write(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A) {
  if (A.mode == 0) rank_launch<0, true>(L, P, A);
  else if (A.anc) rank_launch<2, true>(L, P, A);
  else rank_launch<1, true>(L, P, A);
  L.count();
}

}  // namespace ta
