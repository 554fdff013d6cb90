// interval.cu -- time-window slices of the traces (Section III-A: queries
// over rank ranges and time ranges, answered on time-ordered calling-context
// events by binary search on time) and bottom-up calling contexts (Section
// VI-B, "Obtaining Calling Context").
//
// Window profile of ranks [r0, r1) over [t0, t1), one warp per rank:
//   count pass: a 32-ary warp search finds b (first sample at or after t0)
//     and u (first at or after t1); the contexts of samples [b, u) and of the
//     sample in progress at t0 (b - 1, if any of its interval lies in the
//     window) are marked in a two-level bitmap; their number is the rank's
//     entry count.
//   scan of the counts, exact allocation.
//   write pass: the bitmap again, its prefix ranks every context; samples
//     are taken 32 at a time, grouped into runs of one context across
//     lanes, and each run adds its telescoped duration
//     (min(next ts of its last sample, t1) - ts of its first) and its length
//     to the staged entry; the entries go out context-ascending.
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
constexpr u32 kStageBytes = WSR * 16;  // time u64, ctx u32, cnt u32

struct WinArgs {
  const u64* rank_off;
  const u64* ts;
  const u32* ctx;
  u32 r0, n, C, bm_in_smem;
  u64 t0, t1;
  u64* win;  // [2n] b, u of every rank
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
};

// First i in [lo, hi) with ts[i] >= t, or hi.  One warp; each step probes 32
// evenly spaced positions and keeps the gap between the last probe below t
// and the first at or above it (ts is non-decreasing).
__device__ __forceinline__ u64 warp_lower_bound(const u64* __restrict__ ts, u64 lo, u64 hi, u64 t,
                                                int lane) {
  while (hi - lo > 32) {
    const u64 n = hi - lo;
    const u64 s = (n + 31) / 32;
    const u64 q = lo + min((u64)(lane + 1) * s, n) - 1;
    const u32 ge = __ballot_sync(FULL, ts[q] >= t);
    if (ge == 0) return hi;
    const u64 k = (u64)(__ffs(ge) - 1);
    const u64 qk = lo + min((k + 1) * s, n) - 1;
    lo = k ? lo + min(k * s, n) : lo;
    hi = qk + 1;
  }
  const u64 i = lo + lane;
  const u32 ge = __ballot_sync(FULL, i < hi && ts[i] >= t);
  return ge ? lo + (u64)(__ffs(ge) - 1) : hi;
}

// Time inside [t0, t1) of the sample in progress at t0 (sample b - 1, b > rb).
__device__ __forceinline__ u64 head_time(const u64* __restrict__ ts, u64 b, u64 re, u64 t0,
                                         u64 t1) {
  const u64 nx = b < re ? ts[b] : ts[b - 1];
  const u64 hi = min(nx, t1);
  return hi > t0 ? hi - t0 : 0ull;
}

// Marks the contexts of the rank's window: the sample in progress at t0 (if
// it has time in the window) and every sample in [b, u).
__device__ __forceinline__ void mark_window(const WinArgs& A, const Bm& bm, u64 rb, u64 re, u64 b,
                                            u64 u, int lane) {
  if (lane == 0 && b > rb && head_time(A.ts, b, re, A.t0, A.t1)) bm_set(bm, A.ctx[b - 1]);
  for (u64 j0 = b; j0 < u; j0 += 32 * 8) {
    u32 c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const u64 i = j0 + 32 * q + lane;
      c[q] = i < u ? A.ctx[i] : NONE32;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (c[q] != NONE32 && !bm_has(bm, c[q])) bm_set(bm, c[q]);
  }
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
    const u64 rb = A.rank_off[r], re = A.rank_off[r + 1];
    const u64 b = warp_lower_bound(A.ts, rb, re, A.t0, lane);
    const u64 u = warp_lower_bound(A.ts, b, re, A.t1, lane);
    if (lane == 0) {
      A.win[2 * k] = b;
      A.win[2 * k + 1] = u;
    }
    mark_window(A, bm, rb, re, b, u, lane);
    __syncwarp();
    const u32 n = bm_count_warp(bm, lane);
    if (lane == 0) A.cnt[k] = n;
    bm_clear_warp(bm, lane);
    __syncwarp();
  }
}

template <bool BMS>
__global__ void __launch_bounds__(IW * 32) k_win_write(const WinArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.C);
  const u32 wbytes = kStageBytes + (BMS ? bmw * 4 : 0);
  unsigned char* ws = sm + (size_t)warp * wbytes;
  const u64 gw = (u64)blockIdx.x * IW + warp, G = (u64)gridDim.x * IW;
  const Bm bm = bm_at(BMS ? (u32*)(ws + kStageBytes) : A.gbm + gw * bmw, A.C);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  u64* s_time = (u64*)ws;
  u32* s_ctx = (u32*)(ws + 8 * WSR);
  u32* s_cnt = (u32*)(ws + 12 * WSR);
  const u32 le = 0xFFFFFFFFu >> (31 - lane);  // lanes at or below this one
  __syncwarp();
  for (u64 k = gw; k < A.n; k += G) {
    const u64 r = (u64)A.r0 + k;
    const u64 rb = A.rank_off[r], re = A.rank_off[r + 1];
    const u64 b = A.win[2 * k], u = A.win[2 * k + 1];
    mark_window(A, bm, rb, re, b, u, lane);
    __syncwarp();
    const u32 nnz = bm_prefix_warp(bm, lane);
    const bool in_smem = nnz <= WSR;
    u64* st_time = in_smem ? s_time : A.gst_time + gw * (u64)A.gst_cap;
    u32* st_ctx = in_smem ? s_ctx : A.gst_ctx + gw * (u64)A.gst_cap;
    u32* st_cnt = in_smem ? s_cnt : A.gst_cnt + gw * (u64)A.gst_cap;
    for (u32 q = lane; q < nnz; q += 32) {
      st_time[q] = 0;
      st_cnt[q] = 0;
    }
    __syncwarp();
    if (lane == 0 && b > rb) {
      const u64 hd = head_time(A.ts, b, re, A.t0, A.t1);
      if (hd) {
        const u32 c = A.ctx[b - 1];
        const u32 q = bm_rank(bm, c);
        atomicAdd((unsigned long long*)&st_time[q], (unsigned long long)hd);
        st_ctx[q] = c;
      }
    }
    for (u64 j0 = b; j0 < u; j0 += 32 * KU) {
      u32 c[KU];
      u64 t[KU];
#pragma unroll
      for (int q = 0; q < KU; ++q) {
        const u64 i = j0 + 32 * q + lane;
        const bool v = i < u;
        c[q] = v ? A.ctx[i] : NONE32;
        t[q] = v ? A.ts[i] : 0ull;
      }
#pragma unroll
      for (int q = 0; q < KU; ++q) {
        const u64 i = j0 + 32 * q + lane;
        const bool v = i < u;
        // timestamp of the next sample: the next lane's, the next chunk's
        // first, or (the window's last sample, the last of a block) memory
        u64 nx = __shfl_down_sync(FULL, t[q], 1);
        const u64 nx_chunk = q + 1 < KU ? __shfl_sync(FULL, t[q + 1], 0) : 0ull;
        if (v && (lane == 31 || i + 1 == u)) {
          if (i + 1 < u && q + 1 < KU) nx = nx_chunk;
          else nx = i + 1 < re ? A.ts[i + 1] : t[q];
        }
        const u32 cp = __shfl_up_sync(FULL, c[q], 1);
        const u32 cn = __shfl_down_sync(FULL, c[q], 1);
        const bool head = v && (lane == 0 || cp != c[q]);
        const bool tail = v && (lane == 31 || i + 1 == u || cn != c[q]);
        const u32 heads = __ballot_sync(FULL, head);
        const u32 hm = heads & le;
        const int h = hm ? 31 - __clz(hm) : 0;
        const u64 th = __shfl_sync(FULL, t[q], h);
        if (tail) {
          const u32 p = bm_rank(bm, c[q]);
          atomicAdd((unsigned long long*)&st_time[p], (unsigned long long)(min(nx, A.t1) - th));
          atomicAdd(&st_cnt[p], (u32)(lane - h + 1));
          st_ctx[p] = c[q];
        }
      }
    }
    __syncwarp();
    const u64 eo = A.off[k];
    for (u32 q = lane; q < nnz; q += 32) {
      A.out_ctx[eo + q] = vld(&st_ctx[q]);
      A.out_time[eo + q] = vld(&st_time[q]);
      A.out_cnt[eo + q] = vld(&st_cnt[q]);
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
  Launch L{c->stream, c->num_sms, &c->launches};
  Pool tmp{c, {}};
  struct Rel {
    Pool& p;
    ~Rel() {
      cudaStreamSynchronize(p.ctx->stream);
      p.release();
    }
  } rel{tmp};
  const u32 n = a->r1 - a->r0;
  WinPlan P = plan_window(n, e->C, c->num_sms);
  WinArgs A;
  std::memset(&A, 0, sizeof A);
  A.rank_off = e->rank_off;
  A.ts = e->ts;
  A.ctx = e->ctxv;
  A.r0 = a->r0;
  A.n = n;
  A.C = e->C;
  A.bm_in_smem = P.bms ? 1u : 0u;
  A.t0 = a->t0;
  A.t1 = a->t1;
  Csr x;
  u64* total;
  u64* scan_scratch;
  TRY(tmp.get_n(2 * std::max<u64>(n, 1), &A.win, "window bounds"));
  TRY(tmp.get_n(std::max<u64>(n, 1), &A.cnt, "window counts"));
  TRY(tmp.get_n((u64)n + 1, &x.off, "window offsets"));
  TRY(tmp.get_n(1, &total, "window total"));
  TRY(tmp.get_n(scan_scratch_elems(n), &scan_scratch, "window scan"));
  if (!P.bms) {
    const size_t gbm = (size_t)P.warps() * bm_words(e->C) * 4;
    TRY(tmp.get(gbm, (void**)&A.gbm, "window bitmaps"));
    cudaMemsetAsync(A.gbm, 0, gbm, c->stream);
  }
  const size_t gn = (size_t)P.warps() * e->C;
  TRY(tmp.get_n(gn, &A.gst_ctx, "window stage"));
  TRY(tmp.get_n(gn, &A.gst_time, "window stage"));
  TRY(tmp.get_n(gn, &A.gst_cnt, "window stage"));
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
    timer.stop_and_sync();
  }
  TRY(copy(c, &x.nnz, total, 8));
  TRY(sync_check(c, "ta_interval_profile (count)"));
  const u64 m = std::max<u64>(x.nnz, 1);
  TRY(tmp.get_n(m, &x.ctx, "window ctx"));
  TRY(tmp.get_n(m, &x.time, "window time"));
  TRY(tmp.get_n(m, &x.cnt, "window cnt"));
  A.off = x.off;
  A.out_ctx = x.ctx;
  A.out_time = x.time;
  A.out_cnt = x.cnt;
  if (n) {
    PhaseTimer timer(c, &c->prof.interval_ms);
    if (P.bms) k_win_write<true><<<P.grid_write, IW * 32, P.smem_write, c->stream>>>(A);
    else k_win_write<false><<<P.grid_write, IW * 32, P.smem_write, c->stream>>>(A);
    L.count();
    timer.stop_and_sync();
  }
  TRY(sync_check(c, "ta_interval_profile (write)"));
  Csr out = x;
  if (a->metric == TA_INCLUSIVE) {
    const AllocFn alloc = [&tmp](size_t b, void** p, const char* w) { return tmp.get(b, p, w); };
    TRY(build_inclusive(e, x, n, out, alloc, tmp, &c->prof.interval_ms));
  }
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
