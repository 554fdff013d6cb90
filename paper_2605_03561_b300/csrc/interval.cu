// interval.cu -- time-window slices of the traces (Section III-A: queries
// over rank ranges and time ranges, answered on time-ordered calling-context
// events by binary search on time) and bottom-up calling contexts (Section
// VI-B, "Obtaining Calling Context").
//
// Window profile of ranks [r0, r1) over [t0, t1), one warp per rank.  A
// rank's iterations tile its time, and the iteration tensor already holds
// every iteration's exclusive profile; so the window is split into
//   - the iterations lying wholly inside it, whose tensor entries are added
//     as they are (an iteration is inside when its first sample is at or
//     after t0 and the sample that ends its last one is before t1), and
//   - the samples of the partial iterations at both edges (and the sample in
//     progress at t0), added one by one, clipped to the window.
// Both are exact integer sums, so the result equals the sum over samples.
//   count pass: a 32-ary warp search finds b (first sample at or after t0)
//     and u (first at or after t1) in the rank's timestamps, then the inner
//     iterations by the same search over the first-sample index of the rank's
//     rows; the contexts of the inner entries and of the edge samples are
//     marked in a two-level bitmap; their number is the rank's entry count.
//   scan of the counts, exact allocation.
//   write pass: the bitmap again, its prefix ranks every context; inner
//     entries add their time and count; edge samples are taken 32 at a time,
//     grouped into runs of one context across lanes, and each run adds its
//     telescoped duration (min(next ts after its last sample, t1) - ts of its
//     first) and its length; entries go out context-ascending.
// The inclusive window profile is the exclusive one rolled up the tree by
// the same passes as the experiment's inclusive rollup.
#include <algorithm>
#include <cstring>

#include "ta_api_internal.h"

#define TRY(x)                  \
  do {                          \
    const ta_status s_ = (x);   \
    if (s_ != TA_OK) return s_; \
  } while (0)

namespace ta {
namespace {

constexpr int IW = 8;      // warps per CTA
constexpr u32 WSR = 256;   // entries staged in shared memory per warp
constexpr int KU = 4;      // chunks of 32 samples in flight per warp
constexpr int EU = 8;      // entries per lane in flight
constexpr u32 kStageBytes = WSR * 16;  // time u64, ctx u32, cnt u32

struct WinArgs {
  const u64* rank_off;
  const u64* ts;
  const u32* ctx;
  const u64* row_off_of_rank;
  const u64* entry_off;
  const u32* e_ctx;
  const u64* e_time;
  const u32* e_cnt;
  const u64* row_first;  // [rows + 1] first sample of every row
  const u64* row_ts;     // [rows] its timestamp (rows of empty ranks: unused)
  u32 r0, n, C, bm_in_smem;
  u64 t0, t1;
  u64* win;  // [4n] b, u, first inner row, end of inner rows
  unsigned long long* units;  // [3] edge samples, inner entries read, max entries of a rank
  u32* cnt;  // [n] entries of every rank
  const u64* off;
  u32* out_ctx;
  u64* out_time;
  u32* out_cnt;
  u32* gbm;  // per-warp bitmaps when they do not fit in shared memory
  u32* gst_ctx;
  u64* gst_time;
  u32* gst_cnt;
  u32 gst_cap;
  u32* status;  // F_INTERNAL: the write pass found a count the count pass did not
};

// A rank's window: samples [rb, re), window samples [b, u), inner rows
// [k0, k1) covering samples [s0, s1) (k0 == k1: none, [b, u) all edge).
struct Win {
  u64 rb, re, b, u, k0, k1, s0, s1;
};

__device__ __forceinline__ void win_rows(const WinArgs& A, Win& w) {
  if (w.k1 > w.k0) {
    w.s0 = A.row_first[w.k0];
    w.s1 = A.row_first[w.k1];
  } else {
    w.s0 = w.s1 = w.u;
  }
}

__device__ __forceinline__ void mark_ids(const u32* __restrict__ ids, u64 lo, u64 hi, const Bm& bm,
                                         int lane) {
  for (u64 j0 = lo; j0 < hi; j0 += 32 * 8) {
    u32 c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const u64 i = j0 + 32 * q + lane;
      c[q] = i < hi ? ids[i] : NONE32;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (c[q] != NONE32 && !bm_has(bm, c[q])) bm_set(bm, c[q]);
  }
}

// Marks the contexts of the rank's window: the sample in progress at t0 (if
// it has time in the window), the edge samples and the inner rows' entries.
__device__ __forceinline__ void mark_window(const WinArgs& A, const Bm& bm, const Win& w,
                                            int lane) {
  if (lane == 0 && w.b > w.rb && head_time(A.ts, w.b, w.re, A.t0, A.t1))
    bm_set(bm, A.ctx[w.b - 1]);
  mark_ids(A.ctx, w.b, w.s0, bm, lane);
  mark_ids(A.ctx, w.s1, w.u, bm, lane);
  if (w.k1 > w.k0) mark_ids(A.e_ctx, A.entry_off[w.k0], A.entry_off[w.k1], bm, lane);
}

template <bool BMS>
__global__ void __launch_bounds__(IW * 32) k_win_count(const WinArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.C);
  const u64 gw = (u64)blockIdx.x * IW + warp, G = (u64)gridDim.x * IW;
  const Bm bm = bm_at(BMS ? (u32*)(sm + (size_t)warp * bmw * 4) : A.gbm + gw * bmw, A.C);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  __syncwarp();
  for (u64 k = gw; k < A.n; k += G) {
    const u64 r = (u64)A.r0 + k;
    Win w;
    w.rb = A.rank_off[r];
    w.re = A.rank_off[r + 1];
    const u64 q0 = A.row_off_of_rank[r], q1 = A.row_off_of_rank[r + 1];
    if (w.re == w.rb) {  // no samples: an empty window
      w.b = w.u = w.rb;
      w.k0 = w.k1 = q0;
    } else {
      // the rows tile the rank's time: find the first row starting at or
      // after the bound (row start times are contiguous per rank), then
      // the bound inside the row before it (a few hundred samples)
      const u64 f0 = warp_lower_bound(A.row_ts, q0, q1, A.t0, lane);
      const u64 f1 = warp_lower_bound(A.row_ts, q0, q1, A.t1, lane);
      w.b = f0 == q0 ? w.rb
                     : warp_lower_bound(A.ts, A.row_first[f0 - 1], A.row_first[f0], A.t0, lane);
      w.u = f1 == q0 ? w.rb
                     : warp_lower_bound(A.ts, A.row_first[f1 - 1], A.row_first[f1], A.t1, lane);
      // inner rows: from the first row starting at or after b (row f0) to
      // the row before the one holding u's predecessor (its last sample ends
      // at or after t1), or every row to the end when u is the rank's end
      w.k0 = f0;
      if (w.u <= w.b) {
        w.u = w.b;
        w.k1 = w.k0;
      } else if (w.u == w.re) {
        w.k1 = q1;
      } else {
        w.k1 = max(w.k0, f1 - 1);
      }
    }
    if (lane == 0) {
      A.win[4 * k] = w.b;
      A.win[4 * k + 1] = w.u;
      A.win[4 * k + 2] = w.k0;
      A.win[4 * k + 3] = w.k1;
    }
    win_rows(A, w);
    mark_window(A, bm, w, lane);
    __syncwarp();
    const u32 n = bm_count_warp(bm, lane);
    if (lane == 0) {
      A.cnt[k] = n;
      atomicMax(&A.units[2], (unsigned long long)n);
      atomicAdd(&A.units[0], (unsigned long long)((w.s0 - w.b) + (w.u - w.s1)));
      if (w.k1 > w.k0)
        atomicAdd(&A.units[1],
                  (unsigned long long)(A.entry_off[w.k1] - A.entry_off[w.k0]));
    }
    bm_clear_warp(bm, lane);
    __syncwarp();
  }
}

struct Stage {
  u64* time;
  u32* ctx;
  u32* cnt;
};

// Edge samples [lo, hi) of a rank ending at re: runs of one context across
// lanes add their telescoped durations (clipped at t1) and lengths.
__device__ __forceinline__ void add_samples(const WinArgs& A, const Bm& bm, const Stage& st, u64 lo,
                                            u64 hi, u64 re, int lane) {
  const u32 le = 0xFFFFFFFFu >> (31 - lane);  // lanes at or below this one
  for (u64 j0 = lo; j0 < hi; j0 += 32 * KU) {
    u32 c[KU];
    u64 t[KU];
#pragma unroll
    for (int q = 0; q < KU; ++q) {
      const u64 i = j0 + 32 * q + lane;
      const bool v = i < hi;
      c[q] = v ? A.ctx[i] : NONE32;
      t[q] = v ? A.ts[i] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < KU; ++q) {
      const u64 i = j0 + 32 * q + lane;
      const bool v = i < hi;
      // timestamp of the next sample: the next lane's, the next chunk's
      // first, or (the range's last sample, the last of a block) memory
      u64 nx = __shfl_down_sync(FULL, t[q], 1);
      const u64 nx_chunk = q + 1 < KU ? __shfl_sync(FULL, t[q + 1], 0) : 0ull;
      if (v && (lane == 31 || i + 1 == hi)) {
        if (i + 1 < hi && q + 1 < KU) nx = nx_chunk;
        else nx = i + 1 < re ? A.ts[i + 1] : t[q];
      }
      const u32 cp = __shfl_up_sync(FULL, c[q], 1);
      const u32 cn = __shfl_down_sync(FULL, c[q], 1);
      const bool head = v && (lane == 0 || cp != c[q]);
      const bool tail = v && (lane == 31 || i + 1 == hi || cn != c[q]);
      const u32 heads = __ballot_sync(FULL, head);
      const u32 hm = heads & le;
      const int h = hm ? 31 - __clz(hm) : 0;
      const u64 th = __shfl_sync(FULL, t[q], h);
      if (tail) {
        const u32 p = bm_rank(bm, c[q]);
        atomicAdd((unsigned long long*)&st.time[p], (unsigned long long)(min(nx, A.t1) - th));
        atomicAdd(&st.cnt[p], (u32)(lane - h + 1));
        st.ctx[p] = c[q];
      }
    }
  }
}

// Inner rows' tensor entries [lo, hi), added as they are.
__device__ __forceinline__ void add_entries(const WinArgs& A, const Bm& bm, const Stage& st, u64 lo,
                                            u64 hi, int lane) {
  for (u64 j0 = lo; j0 < hi; j0 += 32 * EU) {
    u32 c[EU], n[EU];
    u64 t[EU];
#pragma unroll
    for (int q = 0; q < EU; ++q) {
      const u64 j = j0 + 32 * q + lane;
      const bool ok = j < hi;
      c[q] = ok ? A.e_ctx[j] : NONE32;
      t[q] = ok ? A.e_time[j] : 0ull;
      n[q] = ok ? A.e_cnt[j] : 0u;
    }
#pragma unroll
    for (int q = 0; q < EU; ++q) {
      if (c[q] == NONE32) continue;
      const u32 p = bm_rank(bm, c[q]);
      atomicAdd((unsigned long long*)&st.time[p], (unsigned long long)t[q]);
      atomicAdd(&st.cnt[p], n[q]);
      st.ctx[p] = c[q];
    }
  }
}

template <bool BMS>
__global__ void __launch_bounds__(IW * 32, 3) k_win_write(const WinArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.C);
  const u32 wbytes = kStageBytes + (BMS ? bmw * 4 : 0);
  unsigned char* ws = sm + (size_t)warp * wbytes;
  const u64 gw = (u64)blockIdx.x * IW + warp, G = (u64)gridDim.x * IW;
  const Bm bm = bm_at(BMS ? (u32*)(ws + kStageBytes) : A.gbm + gw * bmw, A.C);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  const Stage sst{(u64*)ws, (u32*)(ws + 8 * WSR), (u32*)(ws + 12 * WSR)};
  const u64 gbase = gw * (u64)A.gst_cap;
  // the global stage exists only when some rank has more than WSR entries
  const Stage gst = A.gst_time ? Stage{A.gst_time + gbase, A.gst_ctx + gbase, A.gst_cnt + gbase}
                               : sst;
  __syncwarp();
  for (u64 k = gw; k < A.n; k += G) {
    const u64 r = (u64)A.r0 + k;
    Win w;
    w.rb = A.rank_off[r];
    w.re = A.rank_off[r + 1];
    w.b = A.win[4 * k];
    w.u = A.win[4 * k + 1];
    w.k0 = A.win[4 * k + 2];
    w.k1 = A.win[4 * k + 3];
    win_rows(A, w);
    mark_window(A, bm, w, lane);
    __syncwarp();
    const u32 nnz = bm_prefix_warp(bm, lane);
    // the count pass sized both the output and the stage: a rank whose count
    // differs (or would need a global stage that was not allocated) is
    // reported and skipped, never written past
    if (nnz != A.cnt[k] || (nnz > WSR && !A.gst_time)) {
      if (lane == 0) flag(A.status, F_INTERNAL);
      bm_clear_warp(bm, lane);
      __syncwarp();
      continue;
    }
    const Stage st = nnz <= WSR ? sst : gst;
    for (u32 q = lane; q < nnz; q += 32) {
      st.time[q] = 0;
      st.cnt[q] = 0;
    }
    __syncwarp();
    if (lane == 0 && w.b > w.rb) {
      const u64 hd = head_time(A.ts, w.b, w.re, A.t0, A.t1);
      if (hd) {
        const u32 c = A.ctx[w.b - 1];
        const u32 p = bm_rank(bm, c);
        atomicAdd((unsigned long long*)&st.time[p], (unsigned long long)hd);
        st.ctx[p] = c;
      }
    }
    add_samples(A, bm, st, w.b, w.s0, w.re, lane);
    add_samples(A, bm, st, w.s1, w.u, w.re, lane);
    if (w.k1 > w.k0) add_entries(A, bm, st, A.entry_off[w.k0], A.entry_off[w.k1], lane);
    __syncwarp();
    const u64 eo = A.off[k];
    for (u32 q = lane; q < nnz; q += 32) {
      A.out_ctx[eo + q] = vld(&st.ctx[q]);
      A.out_time[eo + q] = vld(&st.time[q]);
      A.out_cnt[eo + q] = vld(&st.cnt[q]);
    }
    bm_clear_warp(bm, lane);
    __syncwarp();
  }
}

struct WinPlan {
  bool bms;
  size_t smem_count, smem_write;
  int grid_count, grid_write;
  u64 warps() const { return (u64)std::max(grid_count, grid_write) * IW; }
};

WinPlan plan_window(u32 n, u32 C, int num_sms) {
  WinPlan P;
  const size_t bm = (size_t)bm_words(C) * 4;
  P.bms = kStageBytes + bm <= 16 * 1024;
  P.smem_count = P.bms ? bm * IW : 0;
  P.smem_write = (kStageBytes + (P.bms ? bm : 0)) * IW;
  const void* kc = P.bms ? (const void*)k_win_count<true> : (const void*)k_win_count<false>;
  const void* kw = P.bms ? (const void*)k_win_write<true> : (const void*)k_win_write<false>;
  cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem_count);
  cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem_write);
  int oc = 0, ow = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, kc, IW * 32, P.smem_count);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ow, kw, IW * 32, P.smem_write);
  const u64 need = std::max<u64>(1, ((u64)n + IW - 1) / IW);
  P.grid_count = (int)std::min<u64>((u64)num_sms * std::max(oc, 1), need);
  P.grid_write = (int)std::min<u64>((u64)num_sms * std::max(ow, 1), need);
  return P;
}

// Start time of every row.  The row of an empty rank points at the next
// rank's first sample (or at N: then the largest value); the window kernels
// skip empty ranks, so those values are never used.
__global__ void k_row_ts(const u64* __restrict__ row_first, const u64* __restrict__ ts, u64 rows,
                         u64 N, u64* row_ts) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < rows; k += G)
    row_ts[k] = row_first[k] < N ? ts[row_first[k]] : ~0ull;
}

// Samples of every tensor row (the sum of its entries' counts).
__global__ void k_row_samples(const u64* __restrict__ entry_off, const u32* __restrict__ e_cnt,
                              u64 rows, u32* n) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < rows; k += G) {
    u32 s = 0;
    for (u64 j = entry_off[k]; j < entry_off[k + 1]; ++j) s += e_cnt[j];
    n[k] = s;
  }
}

// Calling contexts: lengths (depth + 1; ids checked), then the walks.
__global__ void k_chain_len(const u32* __restrict__ ctxs, u32 n, const u32* __restrict__ depth,
                            u32 C, u32* len, u32* status) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32 c = ctxs[i];
  if (c >= C) {
    len[i] = 0;
    flag(status, F_INVALID);
    return;
  }
  len[i] = depth[c] + 1;
}

__global__ void k_chain_fill(const u32* __restrict__ ctxs, u32 n, const u32* __restrict__ parent,
                             const u64* __restrict__ off, u32* chain) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  u32 c = ctxs[i];
  const u64 e = off[i + 1];
  for (u64 q = off[i]; q < e; ++q) {  // exactly depth + 1 steps: ends at the root
    chain[q] = c;
    c = parent[c];
  }
}

}  // namespace
}  // namespace ta

using namespace ta;

namespace {

// First sample of every tensor row, once per experiment: the rows of all
// ranks are concatenated in rank order and every sample lies in exactly one
// row, so an exclusive scan of the rows' sample counts gives each row's
// global first-sample index (and the total, N, at the end).
ta_status ensure_row_first(ta_experiment* e, const Launch& L, Pool& tmp) {
  if (e->row_first) return TA_OK;
  ta_ctx* c = e->ctx;
  u64* rf;
  u32* n;
  u64* scratch;
  TRY(tmp.get_n(std::max<u64>(e->rows, 1), &n, "row samples"));
  TRY(tmp.get_n(scan_scratch_elems(e->rows), &scratch, "row scan"));
  TRY(e->own((e->rows + 1) * 8, (void**)&rf, "row first samples"));
  const u64 nb = std::min<u64>(std::max<u64>(1, (e->rows + 255) / 256), (u64)c->num_sms * 16);
  k_row_samples<<<(unsigned)nb, 256, 0, c->stream>>>(e->entry_off, e->e_cnt, e->rows, n);
  L.count();
  scan_exclusive(L, n, e->rows, rf, rf + e->rows, scratch);
  u64* rt = nullptr;
  if (e->ts) {
    TRY(e->own(std::max<u64>(e->rows, 1) * 8, (void**)&rt, "row start times"));
    k_row_ts<<<(unsigned)nb, 256, 0, c->stream>>>(rf, e->ts, e->rows, e->N, rt);
    L.count();
  }
  TRY(sync_check(c, "ta_interval_profile (row index)"));
  e->row_first = rf;
  e->row_ts = rt;
  return TA_OK;
}

}  // namespace

ta_status ta::ensure_row_index(ta_experiment* e) {
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  Pool tmp{c, {}};
  const ta_status s = ensure_row_first(e, L, tmp);
  cudaStreamSynchronize(c->stream);
  tmp.release();
  return s;
}

namespace {

bool same_window(const ta_interval_args& x, const ta_interval_args& y) {
  return x.t0 == y.t0 && x.t1 == y.t1 && x.r0 == y.r0 && x.r1 == y.r1 && x.metric == y.metric;
}

void drop_window(ta_experiment* e) {
  e->iv_valid = false;
  for (void* p : {(void*)e->iv.off, (void*)e->iv.ctx, (void*)e->iv.time, (void*)e->iv.cnt})
    if (p) e->disown(p);
  e->iv = Csr{};
}

// Computes the window profile into e->iv (experiment-owned).
ta_status compute_window(ta_experiment* e, const ta_interval_args* a, Pool& tmp) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  TRY(ensure_row_first(e, L, tmp));
  const u32 n = a->r1 - a->r0;
  WinPlan P = plan_window(n, e->C, c->num_sms);
  WinArgs A;
  std::memset(&A, 0, sizeof A);
  A.rank_off = e->rank_off;
  A.ts = e->ts;
  A.ctx = e->ctxv;
  A.row_off_of_rank = e->row_off;
  A.entry_off = e->entry_off;
  A.e_ctx = e->e_ctx;
  A.e_time = e->e_time;
  A.e_cnt = e->e_cnt;
  A.row_first = e->row_first;
  A.row_ts = e->row_ts;
  A.r0 = a->r0;
  A.n = n;
  A.C = e->C;
  A.bm_in_smem = P.bms ? 1u : 0u;
  A.t0 = a->t0;
  A.t1 = a->t1;
  const bool incl = a->metric == TA_INCLUSIVE;
  const AllocFn own = [e](size_t b, void** p, const char* w) { return e->own(b, p, w); };
  const AllocFn scratch = [&tmp](size_t b, void** p, const char* w) { return tmp.get(b, p, w); };
  const AllocFn& xalloc = incl ? scratch : own;  // the exclusive window is the result or a step
  Csr xtmp;
  Csr& x = incl ? xtmp : e->iv;  // exclusive: written in place as the result
  u64* total;  // [0] entries, [1..2] units read, [3] most entries of one rank, [4] status
  u64* scan_scratch;
  TRY(tmp.get_n(4 * std::max<u64>(n, 1), &A.win, "window bounds"));
  TRY(tmp.get_n(std::max<u64>(n, 1), &A.cnt, "window counts"));
  TRY(xalloc(((u64)n + 1) * 8, (void**)&x.off, "window offsets"));
  TRY(tmp.get_n(5, &total, "window total"));
  cudaMemsetAsync(total, 0, 40, c->stream);
  A.units = (unsigned long long*)(total + 1);
  A.status = (u32*)(total + 4);
  TRY(tmp.get_n(scan_scratch_elems(n), &scan_scratch, "window scan"));
  if (!P.bms) {
    const size_t gbm = (size_t)P.warps() * bm_words(e->C) * 4;
    TRY(tmp.get(gbm, (void**)&A.gbm, "window bitmaps"));
    cudaMemsetAsync(A.gbm, 0, gbm, c->stream);
  }
  A.gst_cap = e->C;
  {
    PhaseTimer timer(c, &c->prof.interval_ms);
    if (n) {
      if (P.bms) k_win_count<true><<<P.grid_count, IW * 32, P.smem_count, c->stream>>>(A);
      else k_win_count<false><<<P.grid_count, IW * 32, P.smem_count, c->stream>>>(A);
      L.count();
    }
    scan_exclusive(L, A.cnt, n, x.off, total, scan_scratch);
    cudaMemcpyAsync(x.off + n, total, 8, cudaMemcpyDeviceToDevice, c->stream);
    timer.stop();
  }
  u64 h[4];
  TRY(copy(c, h, total, sizeof h));
  TRY(sync_check(c, "ta_interval_profile (count)"));
  x.nnz = h[0];
  c->prof.interval_samples += h[1];
  c->prof.interval_entries += h[2];
  if (h[3] > WSR) {  // some rank's window overflows the shared-memory stage
    const size_t gn = (size_t)P.warps() * e->C;
    TRY(tmp.get_n(gn, &A.gst_ctx, "window stage"));
    TRY(tmp.get_n(gn, &A.gst_time, "window stage"));
    TRY(tmp.get_n(gn, &A.gst_cnt, "window stage"));
  }
  const u64 m = std::max<u64>(x.nnz, 1);
  TRY(xalloc(m * 4, (void**)&x.ctx, "window ctx"));
  TRY(xalloc(m * 8, (void**)&x.time, "window time"));
  TRY(xalloc(m * 4, (void**)&x.cnt, "window cnt"));
  A.off = x.off;
  A.out_ctx = x.ctx;
  A.out_time = x.time;
  A.out_cnt = x.cnt;
  if (n) {
    PhaseTimer timer(c, &c->prof.interval_ms);
    if (P.bms) k_win_write<true><<<P.grid_write, IW * 32, P.smem_write, c->stream>>>(A);
    else k_win_write<false><<<P.grid_write, IW * 32, P.smem_write, c->stream>>>(A);
    L.count();
    timer.stop();
  }
  u64 f = 0;
  TRY(copy(c, &f, total + 4, 8));
  TRY(sync_check(c, "ta_interval_profile (write)"));
  TRY(status_from_flags((u32)f, "ta_interval_profile"));
  if (!incl) return TA_OK;
  return build_inclusive(e, x, n, e->iv, own, tmp, &c->prof.interval_ms);
}

}  // namespace

extern "C" ta_status ta_interval_profile(ta_experiment* e, const ta_interval_args* a,
                                         ta_csr_out* o) {
  if (!e || !a || !o) return fail(TA_ERR_INVALID_ARG, "ta_interval_profile: NULL argument");
  if (a->r0 > a->r1 || a->r1 > e->R)
    return fail(TA_ERR_INVALID_ARG, "ta_interval_profile: ranks [%u, %u) of %u", a->r0, a->r1,
                e->R);
  if (a->metric != TA_EXCLUSIVE && a->metric != TA_INCLUSIVE)
    return fail(TA_ERR_INVALID_ARG, "ta_interval_profile: metric");
  if (o->mem_kind != TA_MEM_HOST && o->mem_kind != TA_MEM_DEVICE)
    return fail(TA_ERR_INVALID_ARG, "ta_interval_profile: mem_kind");
  if (!e->ts && e->N > 0)
    return fail(TA_ERR_STATE, "ta_interval_profile: the traces were released after loading "
                              "(load with TA_LOAD_KEEP_TRACES or borrow them)");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  if (!e->iv_valid || !same_window(e->iv_args, *a)) {
    drop_window(e);
    Pool tmp{c, {}};
    const ta_status s = compute_window(e, a, tmp);
    cudaStreamSynchronize(c->stream);
    tmp.release();
    if (s != TA_OK) {
      drop_window(e);
      return s;
    }
    e->iv_valid = true;
    e->iv_args = *a;
  }
  const Csr& out = e->iv;
  const u32 n = a->r1 - a->r0;
  o->nnz = out.nnz;
  if ((o->ctx || o->time || o->cnt) && o->nnz_cap < out.nnz)
    return fail(TA_ERR_CAPACITY, "ta_interval_profile needs %llu entries",
                (unsigned long long)out.nnz);
  if (o->off) TRY(copy(c, o->off, out.off, ((u64)n + 1) * 8));
  if (o->ctx) TRY(copy(c, o->ctx, out.ctx, out.nnz * 4));
  if (o->time) TRY(copy(c, o->time, out.time, out.nnz * 8));
  if (o->cnt) TRY(copy(c, o->cnt, out.cnt, out.nnz * 4));
  return sync_check(c, "ta_interval_profile");
}

extern "C" ta_status ta_call_chains(const ta_experiment* e, uint32_t mem_kind, const uint32_t* ctxs,
                                    uint32_t n, uint64_t* off, uint32_t* chain, uint64_t chain_cap,
                                    uint64_t* total) {
  if (!e || !total || (n && !ctxs)) return fail(TA_ERR_INVALID_ARG, "ta_call_chains: NULL argument");
  if (mem_kind != TA_MEM_HOST && mem_kind != TA_MEM_DEVICE)
    return fail(TA_ERR_INVALID_ARG, "ta_call_chains: mem_kind");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  Pool tmp{c, {}};
  struct Rel {
    Pool& p;
    ~Rel() {
      cudaStreamSynchronize(p.ctx->stream);
      p.release();
    }
  } rel{tmp};
  const u32* dctx = ctxs;
  if (n && mem_kind == TA_MEM_HOST) {
    u32* d;
    TRY(tmp.get_n(n, &d, "chain contexts"));
    TRY(copy(c, d, ctxs, (size_t)n * 4));
    dctx = d;
  }
  u32 *len, *status;
  u64 *doff, *scratch;
  TRY(tmp.get_n(std::max<u32>(n, 1), &len, "chain lengths"));
  TRY(tmp.get_n((u64)n + 1, &doff, "chain offsets"));
  TRY(tmp.get_n(2, &status, "chain status"));
  TRY(tmp.get_n(scan_scratch_elems(n), &scratch, "chain scan"));
  cudaMemsetAsync(status, 0, 8, c->stream);
  const unsigned nb = std::max(1u, (n + 255) / 256);
  if (n) {
    k_chain_len<<<nb, 256, 0, c->stream>>>(dctx, n, e->depth, e->C, len, status);
    L.count();
  }
  scan_exclusive(L, len, n, doff, doff + n, scratch);
  u32 f = 0;
  TRY(copy(c, &f, status, 4));
  TRY(copy(c, total, doff + n, 8));
  TRY(sync_check(c, "ta_call_chains (lengths)"));
  if (f) return fail(TA_ERR_INVALID_ARG, "ta_call_chains: a context id >= n_ctx (%u)", e->C);
  if (chain && chain_cap < *total)
    return fail(TA_ERR_CAPACITY, "ta_call_chains needs %llu entries", (unsigned long long)*total);
  if (off) TRY(copy(c, off, doff, ((u64)n + 1) * 8));
  if (chain && *total) {
    u32* dch = chain;
    if (mem_kind == TA_MEM_HOST) TRY(tmp.get_n(*total, &dch, "chains"));
    k_chain_fill<<<nb, 256, 0, c->stream>>>(dctx, n, e->parent, doff, dch);
    L.count();
    if (mem_kind == TA_MEM_HOST) TRY(copy(c, chain, dch, *total * 4));
  }
  return sync_check(c, "ta_call_chains");
}
