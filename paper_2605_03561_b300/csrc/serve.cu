// serve.cu -- the serving form: an interactive query server over resident
// experiments with continuous batching.
//
// Device side: every batch runs three kernels over all of its queries.  A
// query is cut into work items (a chunk of ranks or of slice cells), so a
// large query spreads over many CTAs and small ones share a launch:
//   A  per-rank value lookup (stored with a presence bit) and exact partial
//      moments (u64 / u128 atomics); slice cells and time windows are
//      answered here;
//   B  everything that needs the finished moments: outlier counts and the
//      argmax of STATS, per-node outlier / rank / sum counts of RACKS, and
//      the whole top-k selection of TOPK (one CTA: radix select on the
//      values, ordered compaction of the ties, bitonic sort of the rest);
//   C  per-query epilogue: the STATS record, the node -> rack rollup.
// Host side: a worker thread admits queries in arrival order while slots
// and arena space are free, packs descriptors, work items and rank subsets
// into one pinned upload per batch, launches, downloads the batch's results
// into a pinned mirror and marks the queries done from a stream callback.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ta.h"
#include "ta_api_internal.h"

using namespace ta;

namespace {

constexpr int SV_NT = 256;
constexpr u32 CHUNK_R = 2048;      // ranks per work item
constexpr u32 CHUNK_CELLS = 8192;  // slice cells per work item
constexpr u32 CHUNK_WIN = 64;      // window ranks per work item (a warp per rank)
constexpr u32 TOPK_MAX = 1024;
constexpr u32 MAX_EXPS = 64;
constexpr u64 PRESENT = 1ull << 63;  // values are < 2^63 (R * span < 2^63)
constexpr u64 ALIGN = 256;

__host__ __device__ inline u64 align_up(u64 x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Scratch of a STATS / TOPK / RACKS query: Acc, values xs[n] (with the
// presence bit), then for RACKS per-node outlier ranks, ranks and sums.
__host__ __device__ inline u64 xs_off() { return align_up(64); }
__host__ __device__ inline u64 nodes_off(u32 n) { return xs_off() + align_up((u64)n * 8); }
__host__ __device__ inline u64 scratch_bytes_for(u32 kind, u32 n, u32 n_nodes) {
  if (kind == TA_Q_SLICE || kind == TA_Q_WINDOW) return 0;
  u64 b = nodes_off(n);
  if (kind == TA_Q_RACKS) b += 2 * align_up((u64)n_nodes * 8);
  return b;
}

struct ExpDev {
  u32 R, C, n_nodes, n_racks;
  const u32* n_iter;
  const u64* row_off;
  const u64* entry_off;
  const u32* e_ctx;
  const u64* e_time;
  const u32* e_cnt;
  // raw traces and the first sample of every tensor row (window queries;
  // null when the experiment released its traces)
  const u64* rank_off;
  const u64* ts;
  const u32* tctx;
  const u64* row_first;
  const u64* off[2];
  const u32* ctx[2];
  const u64* time[2];
  const u32* cnt[2];
  const u32* node_of_rank;
  const u32* rack_of_node;
};

struct QDev {
  u32 kind, exp, metric, ctx;
  u32 tau_num, tau_den, k, min_ranks;
  u32 r0, r1, i0, i1;
  u32 n, pad;  // ranks the query runs over (subset size or R)
  u64 t0, t1;  // window
  const u32* ranks;
  unsigned char* out;
  unsigned char* scratch;  // zeroed before phase A
};

struct Item {
  u32 q, part;
};

// Per-query accumulators at the start of its scratch (zero-initialised).
struct Acc {
  unsigned long long present, nmin, mx, s1, s2lo, s2hi, n_out;
  unsigned int argmax_inv, pad;  // ~lowest rank attaining max (0 = none)
};

// First position in [b, e) of a context-ascending list whose context is >= c.
__device__ __forceinline__ void csr_find(const u32* __restrict__ ctx, u64 b, u64 e, u32 c,
                                         u64* pos) {
  while (b < e) {
    const u64 mid = (b + e) >> 1;
    if (ctx[mid] < c) b = mid + 1;
    else e = mid;
  }
  *pos = b;
}

// Value of context c in rank r's CSR (metric m) and whether it is present.
__device__ __forceinline__ u64 lookup(const ExpDev& E, u32 m, u32 r, u32 c, bool* present) {
  const u64 b = E.off[m][r], e = E.off[m][r + 1];
  u64 p;
  csr_find(E.ctx[m], b, e, c, &p);
  if (p < e && E.ctx[m][p] == c) {
    *present = true;
    return E.time[m][p];
  }
  *present = false;
  return 0;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, (T)__shfl_xor_sync(FULL, v, o));
  return v;
}

// Block reductions (all threads get the result).
__device__ u64 block_sum(u64 v, u64* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  u64 t = 0;
  for (int i = 0; i < SV_NT / 32; ++i) t += sm[i];
  return t;
}
__device__ u64 block_max(u64 v, u64* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  u64 t = 0;
  for (int i = 0; i < SV_NT / 32; ++i) t = max(t, sm[i]);
  return t;
}
__device__ u128 block_sum128(u128 v, u64* sm) {
  // exact: the low 64 bits are summed as two 32-bit halves and the high 64
  // bits on their own; no part's block sum can overflow 64 bits (the whole
  // sum of squares stays below 2^126).
  const u64 lo = (u64)v, hi = (u64)(v >> 64);
  const u64 lo_lo = lo & 0xFFFFFFFFull, lo_hi = lo >> 32;
  const u64 a = block_sum(lo_lo, sm), b = block_sum(lo_hi, sm), c = block_sum(hi, sm);
  return (u128)a + ((u128)b << 32) + ((u128)c << 64);
}

// Moments of a query from its accumulators.
struct Moments {
  u64 n, s1, mx;
  u128 M;
  double sd;
};
__device__ __forceinline__ Moments moments(const QDev& q, const Acc* acc) {
  Moments m;
  m.n = q.n;
  m.s1 = acc->s1;
  m.mx = acc->mx;
  const u128 S2 = ((u128)acc->s2hi << 64) | acc->s2lo;
  m.M = (u128)m.n * S2 - (u128)m.s1 * m.s1;
  m.sd = (m.n < 2) ? 0.0 : sqrt(u128_to_f64(m.M) / u64_to_f64(m.n * (m.n - 1)));
  return m;
}

// ---- phase A ---------------------------------------------------------------
__global__ void __launch_bounds__(SV_NT) k_serve_a(const QDev* __restrict__ qs,
                                                   const Item* __restrict__ items,
                                                   const ExpDev* __restrict__ exps) {
  __shared__ u64 sm[SV_NT / 32];
  const Item it = items[blockIdx.x];
  const QDev q = qs[it.q];
  const ExpDev& E = exps[q.exp];
  if (q.kind == TA_Q_WINDOW) {
    // a warp per rank: the window's ends by 32-ary searches of the rank's
    // timestamps, its inner iterations by the same search of the rows'
    // first samples; inner rows add their tensor entry of ctx (a binary
    // search in the context-ascending row), edge samples of ctx their
    // clipped durations (the sample in progress at t0: its part after t0)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 n = q.r1 - q.r0;
    const u32 k0 = it.part * CHUNK_WIN, k1 = min(n, k0 + CHUNK_WIN);
    u64* out_t = (u64*)q.out;
    u64* out_n = out_t + n;
    for (u32 k = k0 + w; k < k1; k += SV_NT / 32) {
      const u32 r = q.r0 + k;
      const u64 rb = E.rank_off[r], re = E.rank_off[r + 1];
      const u64 b = warp_lower_bound(E.ts, rb, re, q.t0, lane);
      const u64 u = warp_lower_bound(E.ts, b, re, q.t1, lane);
      const u64 q1 = E.row_off[r + 1];
      const u64 a0 = warp_lower_bound(E.row_first, E.row_off[r], q1, b, lane);
      const u64 a1 = warp_lower_bound(E.row_first, a0 + 1, q1 + 1, u == re ? re + 1 : u, lane) - 1;
      const u64 s0 = a1 > a0 ? E.row_first[a0] : u, s1 = a1 > a0 ? E.row_first[a1] : u;
      u64 t = 0, c = 0;
      for (u64 row = a0 + lane; row < a1; row += 32) {
        const u64 eb = E.entry_off[row], ee = E.entry_off[row + 1];
        u64 p;
        csr_find(E.e_ctx, eb, ee, q.ctx, &p);
        if (p < ee && E.e_ctx[p] == q.ctx) {
          t += E.e_time[p];
          c += E.e_cnt[p];
        }
      }
      for (int side = 0; side < 2; ++side) {
        const u64 lo = side ? s1 : b, hi = side ? u : s0;
        for (u64 i = lo + lane; i < hi; i += 32) {
          if (E.tctx[i] != q.ctx) continue;
          const u64 ti = E.ts[i];
          const u64 nx = i + 1 < re ? E.ts[i + 1] : ti;
          t += min(nx, q.t1) - ti;
          ++c;
        }
      }
      if (lane == 0 && b > rb && E.tctx[b - 1] == q.ctx) t += head_time(E.ts, b, re, q.t0, q.t1);
      t = warp_sum(t);
      c = warp_sum(c);
      if (lane == 0) {
        out_t[k] = t;
        out_n[k] = c;
      }
    }
    return;
  }
  if (q.kind == TA_Q_SLICE) {
    const u64 W = q.i1 - q.i0;
    const u64 total = (u64)(q.r1 - q.r0) * W;
    const u64 g0 = (u64)it.part * CHUNK_CELLS, g1 = min(total, g0 + CHUNK_CELLS);
    u64* out = (u64*)q.out;
    for (u64 g = g0 + threadIdx.x; g < g1; g += SV_NT) {
      const u32 r = q.r0 + (u32)(g / W), i = q.i0 + (u32)(g % W);
      u64 v = 0;
      if (i < E.n_iter[r]) {
        const u64 row = E.row_off[r] + 1 + i;
        const u64 b = E.entry_off[row], e = E.entry_off[row + 1];
        u64 p;
        csr_find(E.e_ctx, b, e, q.ctx, &p);
        if (p < e && E.e_ctx[p] == q.ctx) v = E.e_time[p];
      }
      out[g] = v;
    }
    return;
  }
  Acc* acc = (Acc*)q.scratch;
  u64* xs = (u64*)(q.scratch + xs_off());
  const u32 b = it.part * CHUNK_R, e = min(q.n, b + CHUNK_R);
  u64 present = 0, nmin = 0, mx = 0, s1 = 0;
  u128 s2 = 0;
  for (u32 i = b + threadIdx.x; i < e; i += SV_NT) {
    const u32 r = q.ranks ? q.ranks[i] : i;
    bool pr;
    const u64 x = lookup(E, q.metric, r, q.ctx, &pr);
    xs[i] = x | (pr ? PRESENT : 0ull);
    if (pr) {
      ++present;
      nmin = max(nmin, ~x);
    }
    mx = max(mx, x);
    s1 += x;
    s2 += (u128)x * x;
  }
  present = block_sum(present, sm);
  nmin = block_max(nmin, sm);
  mx = block_max(mx, sm);
  s1 = block_sum(s1, sm);
  s2 = block_sum128(s2, sm);
  if (threadIdx.x == 0) {
    atomicAdd(&acc->present, (unsigned long long)present);
    atomicMax(&acc->nmin, (unsigned long long)nmin);
    atomicMax(&acc->mx, (unsigned long long)mx);
    atomicAdd(&acc->s1, (unsigned long long)s1);
    atomic_add_u128((u64*)&acc->s2lo, (u64*)&acc->s2hi, s2);
  }
}

// ---- top-k of one query (one CTA) --------------------------------------------
struct Cand {
  u64 x;
  u32 rank, pad;
};

__device__ __forceinline__ bool cand_before(const Cand& a, const Cand& b) {
  return a.x != b.x ? a.x > b.x : a.rank < b.rank;
}

__device__ void topk_select(const QDev& q, const Acc* acc) {
  __shared__ u32 hist[256];
  __shared__ u64 sh_prefix, sh_mask;
  __shared__ u32 sh_need, sh_ngt, sh_taken;
  __shared__ Cand cand[TOPK_MAX];
  __shared__ u32 wsum[SV_NT / 32];
  const u64* xs = (const u64*)(q.scratch + xs_off());
  const u32 n = q.n, kk = min(q.k, n);
  const u64 VAL = ~PRESENT;
  if (threadIdx.x == 0) {
    sh_prefix = 0;
    sh_mask = 0;
    sh_need = kk;
    sh_ngt = 0;
    sh_taken = 0;
  }
  __syncthreads();
  // radix select of the kk-th largest value, 8 bits at a time from the top
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (u32 d = threadIdx.x; d < 256; d += SV_NT) hist[d] = 0;
    __syncthreads();
    const u64 prefix = sh_prefix, mask = sh_mask;
    for (u32 i = threadIdx.x; i < n; i += SV_NT) {
      const u64 v = xs[i] & VAL;
      if ((v & mask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 need = sh_need;
      int d = 255;
      for (; d > 0; --d) {
        if (hist[d] >= need) break;
        need -= hist[d];
      }
      sh_need = need;
      sh_prefix = prefix | ((u64)d << shift);
      sh_mask = mask | (255ull << shift);
    }
    __syncthreads();
  }
  const u64 T = sh_prefix;
  const u32 need_eq = sh_need, n_gt = kk - need_eq;
  // values above T (fewer than kk), in any order
  for (u32 i = threadIdx.x; i < n; i += SV_NT) {
    const u64 v = xs[i] & VAL;
    if (v > T) {
      const u32 s = atomicAdd(&sh_ngt, 1u);
      cand[s].x = v;
      cand[s].rank = q.ranks ? q.ranks[i] : i;
      cand[s].pad = 0;
    }
  }
  __syncthreads();
  // bitonic sort of the n_gt values above T (descending value, ascending rank)
  u32 P = 1;
  while (P < n_gt) P <<= 1;
  for (u32 i = n_gt + threadIdx.x; i < P; i += SV_NT) {
    cand[i].x = 0;  // sorts after every value above T (>= 1)
    cand[i].rank = 0xFFFFFFFFu;
  }
  __syncthreads();
  for (u32 k = 2; k <= P; k <<= 1)
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      for (u32 i = threadIdx.x; i < P; i += SV_NT) {
        const u32 l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          Cand a = cand[i], b = cand[l];
          if (cand_before(b, a) == up) {
            cand[i] = b;
            cand[l] = a;
          }
        }
      }
      __syncthreads();
    }
  // the need_eq lowest ranks holding T, by an ordered block compaction
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (u32 base = 0; base < n; base += SV_NT) {
    if (sh_taken >= need_eq) break;  // uniform: read after a barrier
    const u32 i = base + threadIdx.x;
    const bool f = i < n && (xs[i] & VAL) == T;
    const u32 bal = __ballot_sync(FULL, f);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    u32 before = 0, total = 0;
    for (int j = 0; j < SV_NT / 32; ++j) {
      if (j < w) before += wsum[j];
      total += wsum[j];
    }
    const u32 pos = sh_taken + before + __popc(bal & ((1u << lane) - 1u));
    if (f && pos < need_eq) {
      cand[n_gt + pos].x = T;
      cand[n_gt + pos].rank = q.ranks ? q.ranks[i] : i;
      cand[n_gt + pos].pad = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) sh_taken += total;
    __syncthreads();
  }
  // ties with T follow the sorted values above T; write everything with z
  const Moments mo = moments(q, acc);
  u64* head = (u64*)q.out;
  ta_q_topk_entry* out = (ta_q_topk_entry*)(q.out + 8);
  if (threadIdx.x == 0) *head = kk;
  for (u32 j = threadIdx.x; j < kk; j += SV_NT) {
    const Cand c = cand[j];
    const long long D = (long long)(mo.n * c.x) - (long long)mo.s1;
    ta_q_topk_entry o;
    o.rank = c.rank;
    o.reserved = 0;
    o.x = c.x;
    o.z = (mo.n < 2 || mo.M == 0) ? 0.0 : i64_to_f64(D) / (u64_to_f64(mo.n) * mo.sd);
    out[j] = o;
  }
}

// ---- phase B ---------------------------------------------------------------
__global__ void __launch_bounds__(SV_NT) k_serve_b(const QDev* __restrict__ qs,
                                                   const Item* __restrict__ items,
                                                   const ExpDev* __restrict__ exps) {
  __shared__ u64 sm[SV_NT / 32];
  const Item it = items[blockIdx.x];
  const QDev q = qs[it.q];
  Acc* acc = (Acc*)q.scratch;
  if (q.kind == TA_Q_TOPK) {
    topk_select(q, acc);
    return;
  }
  const ExpDev& E = exps[q.exp];
  const u64* xs = (const u64*)(q.scratch + xs_off());
  const Moments mo = moments(q, acc);
  const u32 b = it.part * CHUNK_R, e = min(q.n, b + CHUNK_R);
  if (q.kind == TA_Q_STATS) {
    u64 n_out = 0;
    u32 amin = 0xFFFFFFFFu;
    for (u32 i = b + threadIdx.x; i < e; i += SV_NT) {
      const u64 v = xs[i];
      const u64 x = v & ~PRESENT;
      const u32 r = q.ranks[i];
      if (mo.mx > 0 && x == mo.mx) amin = min(amin, r);
      if (v & PRESENT) {
        const long long D = (long long)(mo.n * x) - (long long)mo.s1;
        if (is_outlier(D, mo.n, mo.M, q.tau_num, q.tau_den)) ++n_out;
      }
    }
    n_out = block_sum(n_out, sm);
    const u64 inv = block_max((u64)(u32)(~amin), sm);
    if (threadIdx.x == 0) {
      if (n_out) atomicAdd(&acc->n_out, (unsigned long long)n_out);
      atomicMax(&acc->argmax_inv, (unsigned int)inv);
    }
    return;
  }
  // RACKS: per node, outlier ranks, ranks and summed values (all ranks)
  unsigned char* nb = q.scratch + nodes_off(q.n);
  u32* node_out = (u32*)nb;
  u32* node_ranks = node_out + E.n_nodes;
  unsigned long long* node_sum = (unsigned long long*)(nb + align_up((u64)E.n_nodes * 8));
  for (u32 i = b + threadIdx.x; i < e; i += SV_NT) {
    const u64 v = xs[i];
    const u64 x = v & ~PRESENT;
    const u32 nd = E.node_of_rank[i];
    atomicAdd(&node_ranks[nd], 1u);
    if (x) atomicAdd(&node_sum[nd], (unsigned long long)x);
    if (v & PRESENT) {
      const long long D = (long long)(mo.n * x) - (long long)mo.s1;
      if (is_outlier(D, mo.n, mo.M, q.tau_num, q.tau_den)) atomicAdd(&node_out[nd], 1u);
    }
  }
}

// ---- phase C ---------------------------------------------------------------
__global__ void __launch_bounds__(SV_NT) k_serve_c(const QDev* __restrict__ qs,
                                                   const Item* __restrict__ items,
                                                   const ExpDev* __restrict__ exps) {
  __shared__ u32 wsum[SV_NT / 32];
  __shared__ u32 sh_base;
  const Item it = items[blockIdx.x];
  const QDev q = qs[it.q];
  const Acc* acc = (const Acc*)q.scratch;
  if (q.kind == TA_Q_STATS) {
    if (threadIdx.x != 0) return;
    const Moments mo = moments(q, acc);
    const u64 n = mo.n;
    const u32 present = (u32)acc->present;
    ta_q_stats r;
    ta_ctx_stats& st = r.stats;
    st.n = (u32)n;
    st.present = present;
    st.argmax = (mo.mx == 0) ? q.ranks[0] : ~acc->argmax_inv;
    st.reserved = 0;
    st.min = (present < n) ? 0ull : ~acc->nmin;
    st.max = mo.mx;
    st.s1 = mo.s1;
    st.s2_lo = acc->s2lo;
    st.s2_hi = acc->s2hi;
    st.mean = u64_to_f64(mo.s1) / u64_to_f64(n);
    st.std = mo.sd;
    st.cv = (st.mean == 0.0) ? 0.0 : mo.sd / st.mean;
    st.balance = (mo.mx == 0) ? 1.0 : st.mean / u64_to_f64(mo.mx);
    r.n_outliers = acc->n_out;
    *(ta_q_stats*)q.out = r;
    return;
  }
  // RACKS: node -> rack rollup and the ascending list of flagged racks
  const ExpDev& E = exps[q.exp];
  const u32 NR = E.n_racks, NN = E.n_nodes;
  unsigned char* nb = q.scratch + nodes_off(q.n);
  const u32* node_out = (const u32*)nb;
  const unsigned long long* node_sum =
      (const unsigned long long*)(nb + align_up((u64)NN * 8));
  ta_q_racks* head = (ta_q_racks*)q.out;
  unsigned long long* rack_sum = (unsigned long long*)(q.out + 8);
  u32* rack_flagged = (u32*)(q.out + 8 + 8 * (u64)NR);
  u32* rack_nodes = rack_flagged + NR;
  u32* flagged = rack_nodes + NR;
  for (u32 j = threadIdx.x; j < NR; j += SV_NT) {
    rack_sum[j] = 0;
    rack_flagged[j] = 0;
    rack_nodes[j] = 0;
  }
  __syncthreads();
  for (u32 nd = threadIdx.x; nd < NN; nd += SV_NT) {
    const u32 rk = E.rack_of_node[nd];
    if (node_out[nd] >= q.min_ranks) atomicAdd(&rack_flagged[rk], 1u);
    atomicAdd(&rack_nodes[rk], 1u);
    if (node_sum[nd]) atomicAdd(&rack_sum[rk], node_sum[nd]);
  }
  if (threadIdx.x == 0) sh_base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (u32 base = 0; base < NR; base += SV_NT) {
    const u32 j = base + threadIdx.x;
    const bool f = j < NR && rack_flagged[j] > 0;
    const u32 bal = __ballot_sync(FULL, f);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    u32 before = 0, total = 0;
    for (int i = 0; i < SV_NT / 32; ++i) {
      if (i < w) before += wsum[i];
      total += wsum[i];
    }
    if (f) flagged[sh_base + before + __popc(bal & ((1u << lane) - 1u))] = j;
    __syncthreads();
    if (threadIdx.x == 0) sh_base += total;
    __syncthreads();
  }
  for (u32 j = sh_base + threadIdx.x; j < NR; j += SV_NT) flagged[j] = 0;  // defined bytes
  if (threadIdx.x == 0) {
    head->n_racks = NR;
    head->n_flagged_racks = sh_base;
  }
}

// ---- host side ---------------------------------------------------------------
u64 now_ns() {
  return (u64)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over [0, cap) in ALIGN granules.
struct Arena {
  u64 cap = 0;
  std::map<u64, u64> free_;  // offset -> length
  void init(u64 c) {
    cap = c;
    free_.clear();
    if (c) free_[0] = c;
  }
  u64 largest() const {
    u64 m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  bool alloc(u64 n, u64* off) {
    n = align_up(std::max<u64>(n, 1));
    for (auto itr = free_.begin(); itr != free_.end(); ++itr) {
      if (itr->second >= n) {
        *off = itr->first;
        const u64 rest = itr->second - n, o = itr->first + n;
        free_.erase(itr);
        if (rest) free_[o] = rest;
        return true;
      }
    }
    return false;
  }
  void release(u64 off, u64 n) {
    n = align_up(std::max<u64>(n, 1));
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + n == nx->first) {
      n += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        pv->second += n;
        return;
      }
    }
    free_[off] = n;
  }
};

struct QState {
  ta_query q{};
  std::vector<u32> ranks;
  u32 status = TA_OK;
  u32 n = 0;
  u64 t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
  u64 res_bytes = 0, scr_bytes = 0, pay_bytes = 0, items_a = 0, items_b = 0, items_c = 0;
  u64 out_bytes = 0;  // payload size (res_bytes rounded up to the arena granule)
  u64 res_off = 0, block = 0;  // result offset and the batch block holding it
  bool done = false;
};

struct Slot {
  cudaStream_t st = nullptr;
  unsigned char* h_stage = nullptr;
  unsigned char* d_stage = nullptr;
  u64 cap = 0;
  bool busy = false;
  std::vector<u64> tickets;
  u64 scr_off = 0, scr_len = 0;
  ta_server* srv = nullptr;
};

}  // namespace

struct ta_server {
  ta_ctx* ctx = nullptr;
  ta_serve_config cfg{};
  std::vector<ExpDev> exps;
  std::vector<ta_experiment*> exp_handles;
  ExpDev* d_exps = nullptr;
  unsigned char* d_result = nullptr;
  unsigned char* h_result = nullptr;
  unsigned char* d_scratch = nullptr;
  Arena res, scr;
  std::map<u64, std::pair<u64, u32>> blocks;  // result block offset -> (length, live queries)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<u64> pending;
  std::unordered_map<u64, QState> qs;
  u64 next_ticket = 1;
  u32 inflight = 0;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  u64 resident = 0;
  std::vector<Block> owned;
  std::atomic<unsigned long long> launches{0};
};

namespace {

void CUDART_CB on_batch_done(void* p) {
  Slot* sl = (Slot*)p;
  ta_server* s = sl->srv;
  const u64 t = now_ns();
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (u64 tk : sl->tickets) {
      auto itr = s->qs.find(tk);
      if (itr == s->qs.end()) continue;
      itr->second.done = true;
      itr->second.t_done = t;
    }
    if (sl->scr_len) s->scr.release(sl->scr_off, sl->scr_len);
    sl->scr_len = 0;
    sl->tickets.clear();
    sl->busy = false;
  }
  s->cv.notify_all();
}

// Sizes a validated query needs.
void size_query(const ta_server* s, QState& st) {
  const ta_query& q = st.q;
  const ExpDev& E = s->exps[q.experiment];
  st.n = (q.kind == TA_Q_STATS) ? q.n_ranks : E.R;
  st.scr_bytes = scratch_bytes_for(q.kind, st.n, E.n_nodes);
  st.pay_bytes = (q.kind == TA_Q_STATS) ? align_up((u64)q.n_ranks * 4) : 0;
  switch (q.kind) {
    case TA_Q_STATS:
      st.res_bytes = sizeof(ta_q_stats);
      st.items_a = st.items_b = (st.n + CHUNK_R - 1) / CHUNK_R;
      st.items_c = 1;
      break;
    case TA_Q_SLICE: {
      const u64 cells = (u64)(q.r1 - q.r0) * (q.i1 - q.i0);
      st.res_bytes = cells * 8;
      st.items_a = (cells + CHUNK_CELLS - 1) / CHUNK_CELLS;
      st.items_b = st.items_c = 0;
      break;
    }
    case TA_Q_WINDOW: {
      const u64 n = q.r1 - q.r0;
      st.res_bytes = n * 16;
      st.items_a = (n + CHUNK_WIN - 1) / CHUNK_WIN;
      st.items_b = st.items_c = 0;
      break;
    }
    case TA_Q_TOPK:
      st.res_bytes = 8 + (u64)std::min(q.k, E.R) * sizeof(ta_q_topk_entry);
      st.items_a = (st.n + CHUNK_R - 1) / CHUNK_R;
      st.items_b = 1;
      st.items_c = 0;
      break;
    default:  // RACKS
      st.res_bytes = 8 + 20 * (u64)E.n_racks;
      st.items_a = st.items_b = (st.n + CHUNK_R - 1) / CHUNK_R;
      st.items_c = 1;
  }
  st.out_bytes = st.res_bytes;
  st.res_bytes = align_up(std::max<u64>(st.res_bytes, 8));
}

u64 stage_bytes(const QState& st) {
  return sizeof(QDev) + (st.items_a + st.items_b + st.items_c) * sizeof(Item) + st.pay_bytes;
}

// Runs one admitted batch on slot sl (called without the lock).
void launch_batch(ta_server* s, Slot& sl, std::vector<QState*>& B, u64 res_block, u64 res_len,
                  u64 scr_block) {
  // staging layout: QDev[nq] | Item A | Item B | Item C | rank subsets
  const u64 nq = B.size();
  u64 na = 0, nb = 0, nc = 0, pay = 0;
  for (auto* q : B) {
    na += q->items_a;
    nb += q->items_b;
    nc += q->items_c;
    pay += q->pay_bytes;
  }
  const u64 o_q = 0, o_a = align_up(nq * sizeof(QDev)), o_b = o_a + align_up(na * sizeof(Item)),
            o_c = o_b + align_up(nb * sizeof(Item)), o_p = o_c + align_up(nc * sizeof(Item));
  const u64 total = o_p + pay;
  QDev* hq = (QDev*)(sl.h_stage + o_q);
  Item* ha = (Item*)(sl.h_stage + o_a);
  Item* hb = (Item*)(sl.h_stage + o_b);
  Item* hc = (Item*)(sl.h_stage + o_c);
  u64 ia = 0, ib = 0, ic = 0, p = o_p, so = scr_block;
  for (u64 j = 0; j < nq; ++j) {
    QState& st = *B[j];
    const ta_query& q = st.q;
    QDev& d = hq[j];
    d.kind = q.kind;
    d.exp = q.experiment;
    d.metric = q.metric;
    d.ctx = q.ctx;
    d.tau_num = q.tau_num;
    d.tau_den = q.tau_den;
    d.k = q.k;
    d.min_ranks = q.min_ranks;
    d.r0 = q.r0;
    d.r1 = q.r1;
    d.i0 = q.i0;
    d.i1 = q.i1;
    d.n = st.n;
    d.pad = 0;
    d.t0 = q.t0;
    d.t1 = q.t1;
    d.ranks = nullptr;
    if (st.pay_bytes) {
      std::memcpy(sl.h_stage + p, st.ranks.data(), st.ranks.size() * 4);
      d.ranks = (const u32*)(sl.d_stage + p);
      p += st.pay_bytes;
    }
    d.out = s->d_result + st.res_off;
    d.scratch = st.scr_bytes ? s->d_scratch + so : nullptr;
    so += align_up(st.scr_bytes);
    for (u64 k = 0; k < st.items_a; ++k) ha[ia++] = Item{(u32)j, (u32)k};
    for (u64 k = 0; k < st.items_b; ++k) hb[ib++] = Item{(u32)j, (u32)k};
    for (u64 k = 0; k < st.items_c; ++k) hc[ic++] = Item{(u32)j, (u32)k};
  }
  const u64 t = now_ns();
  for (auto* q : B) q->t_launch = t;
  cudaStream_t st = sl.st;
  cudaMemcpyAsync(sl.d_stage, sl.h_stage, total, cudaMemcpyHostToDevice, st);
  if (sl.scr_len) cudaMemsetAsync(s->d_scratch + scr_block, 0, sl.scr_len, st);
  const QDev* dq = (const QDev*)(sl.d_stage + o_q);
  unsigned long long n_k = 0;
  if (na) {
    k_serve_a<<<(unsigned)na, SV_NT, 0, st>>>(dq, (const Item*)(sl.d_stage + o_a), s->d_exps);
    ++n_k;
  }
  if (nb) {
    k_serve_b<<<(unsigned)nb, SV_NT, 0, st>>>(dq, (const Item*)(sl.d_stage + o_b), s->d_exps);
    ++n_k;
  }
  if (nc) {
    k_serve_c<<<(unsigned)nc, SV_NT, 0, st>>>(dq, (const Item*)(sl.d_stage + o_c), s->d_exps);
    ++n_k;
  }
  s->launches += n_k;
  __atomic_fetch_add(&s->ctx->launches, n_k, __ATOMIC_RELAXED);
  cudaMemcpyAsync(s->h_result + res_block, s->d_result + res_block, res_len,
                  cudaMemcpyDeviceToHost, st);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    std::lock_guard<std::mutex> g(s->mu);
    for (auto* q : B) q->status = TA_ERR_CUDA;
  }
  cudaLaunchHostFunc(st, on_batch_done, &sl);
}

void worker_main(ta_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    int si = -1;
    s->cv.wait(lk, [&] {
      if (s->stop) return true;
      if (s->pending.empty()) return false;
      for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].busy) {
          si = (int)i;
          return true;
        }
      return false;
    });
    if (s->stop) break;
    Slot& sl = s->slots[si];
    // admission in arrival order while a slot, result space, scratch space
    // and staging room remain
    std::vector<QState*> B;
    std::vector<u64> tk;
    u64 res_total = 0, scr_total = 0, stage = 0;
    const u64 res_free = s->res.largest(), scr_free = s->scr.largest();
    while (!s->pending.empty() && B.size() < s->cfg.max_batch &&
           s->inflight < s->cfg.max_inflight) {
      QState& st = s->qs[s->pending.front()];
      const u64 sb = stage_bytes(st) + 3 * ALIGN;
      if (res_total + st.res_bytes > res_free || scr_total + align_up(st.scr_bytes) > scr_free ||
          stage + sb > sl.cap)
        break;
      res_total += st.res_bytes;
      scr_total += align_up(st.scr_bytes);
      stage += sb;
      B.push_back(&st);
      tk.push_back(s->pending.front());
      s->pending.pop_front();
      ++s->inflight;
    }
    if (B.empty()) {  // the head waits for results to be released or batches to end
      s->cv.wait(lk);
      continue;
    }
    u64 res_block = 0, scr_block = 0;
    s->res.alloc(res_total, &res_block);
    if (scr_total) s->scr.alloc(scr_total, &scr_block);
    s->blocks[res_block] = {res_total, (u32)B.size()};
    u64 o = res_block;
    const u64 t = now_ns();
    for (size_t j = 0; j < B.size(); ++j) {
      B[j]->res_off = o;
      B[j]->block = res_block;
      B[j]->t_admit = t;
      o += B[j]->res_bytes;
    }
    sl.busy = true;
    sl.tickets = tk;
    sl.scr_off = scr_block;
    sl.scr_len = scr_total;
    lk.unlock();
    launch_batch(s, sl, B, res_block, res_total, scr_block);
    lk.lock();
  }
}

ta_status validate_query(const ta_server* s, const ta_query* q) {
  if (q->experiment >= s->exps.size()) return fail(TA_ERR_INVALID_ARG, "query: experiment id");
  const ExpDev& E = s->exps[q->experiment];
  if (q->ctx >= E.C) return fail(TA_ERR_INVALID_ARG, "query: ctx >= n_ctx");
  if (q->kind != TA_Q_SLICE && q->kind != TA_Q_WINDOW) {
    if (q->metric > 1) return fail(TA_ERR_INVALID_ARG, "query: metric");
    if (E.off[q->metric] == nullptr)
      return fail(TA_ERR_INVALID_ARG, "query: the inclusive rollup was not built");
  }
  switch (q->kind) {
    case TA_Q_STATS:
      if (q->tau_den == 0 || !q->ranks || q->n_ranks == 0)
        return fail(TA_ERR_INVALID_ARG, "stats query: tau_den = 0 or empty rank subset");
      for (u32 i = 0; i < q->n_ranks; ++i)
        if (q->ranks[i] >= E.R || (i && q->ranks[i] <= q->ranks[i - 1]))
          return fail(TA_ERR_INVALID_ARG, "stats query: ranks must be sorted, unique, < R");
      return TA_OK;
    case TA_Q_SLICE:
      if (q->r0 > q->r1 || q->r1 > E.R || q->i0 > q->i1)
        return fail(TA_ERR_INVALID_ARG, "slice query: r0 <= r1 <= R and i0 <= i1");
      return TA_OK;
    case TA_Q_TOPK:
      if (q->k == 0 || q->k > TOPK_MAX) return fail(TA_ERR_INVALID_ARG, "top-k query: 1 <= k <= 1024");
      return TA_OK;
    case TA_Q_WINDOW:
      if (q->r0 > q->r1 || q->r1 > E.R)
        return fail(TA_ERR_INVALID_ARG, "window query: r0 <= r1 <= R");
      if (!E.row_first)
        return fail(TA_ERR_INVALID_ARG,
                    "window query: the experiment's traces were released when it was loaded");
      return TA_OK;
    case TA_Q_RACKS:
      if (q->tau_den == 0 || q->min_ranks == 0 || !E.node_of_rank)
        return fail(TA_ERR_INVALID_ARG, "rack query: tau_den, min_ranks or missing topology");
      return TA_OK;
    default:
      return fail(TA_ERR_INVALID_ARG, "query: unknown kind %u", q->kind);
  }
}

}  // namespace

extern "C" {

ta_status ta_serve_open(ta_ctx* c, const ta_serve_config* cfg, ta_server** out) {
  if (!c || !out) return fail(TA_ERR_INVALID_ARG, "ta_serve_open: NULL argument");
  *out = nullptr;
  cudaSetDevice(c->device);
  ta_server* s = new ta_server();
  s->ctx = c;
  if (cfg) s->cfg = *cfg;
  ta_serve_config& g = s->cfg;
  if (!g.max_batch) g.max_batch = 1024;
  if (!g.n_streams) g.n_streams = 3;
  if (!g.max_inflight) g.max_inflight = 8192;
  if (!g.result_bytes) g.result_bytes = 1ull << 30;
  if (!g.scratch_bytes) g.scratch_bytes = 256ull << 20;
  if (!g.staging_bytes) g.staging_bytes = 32ull << 20;
  g.result_bytes = align_up(g.result_bytes);
  g.scratch_bytes = align_up(g.scratch_bytes);
  g.staging_bytes = align_up(g.staging_bytes);
  auto bail = [&](ta_status st) {
    ta_serve_close(s);
    return st;
  };
  auto own = [&](u64 bytes, void** p, const char* what) -> ta_status {
    void* q = dalloc(c, bytes);
    if (!q) return fail(TA_ERR_OOM, "ta_serve_open: %s (%llu bytes)", what, (unsigned long long)bytes);
    s->owned.push_back({q, bytes});
    *p = q;
    return TA_OK;
  };
  ta_status st;
  if ((st = own(MAX_EXPS * sizeof(ExpDev), (void**)&s->d_exps, "experiment table")) != TA_OK) return bail(st);
  if ((st = own(g.result_bytes, (void**)&s->d_result, "result arena")) != TA_OK) return bail(st);
  if ((st = own(g.scratch_bytes, (void**)&s->d_scratch, "scratch arena")) != TA_OK) return bail(st);
  if (cudaHostAlloc((void**)&s->h_result, g.result_bytes, cudaHostAllocDefault) != cudaSuccess)
    return bail(fail(TA_ERR_OOM, "ta_serve_open: pinned result mirror"));
  s->res.init(g.result_bytes);
  s->scr.init(g.scratch_bytes);
  s->slots.resize(g.n_streams);
  for (auto& sl : s->slots) {
    sl.srv = s;
    sl.cap = g.staging_bytes;
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void**)&sl.h_stage, sl.cap, cudaHostAllocDefault) != cudaSuccess)
      return bail(fail(TA_ERR_CUDA, "ta_serve_open: stream or pinned staging"));
    if ((st = own(sl.cap, (void**)&sl.d_stage, "staging")) != TA_OK) return bail(st);
  }
  cudaStreamSynchronize(c->stream);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TA_OK;
}

ta_status ta_serve_close(ta_server* s) {
  if (!s) return TA_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& sl : s->slots) {
    if (sl.st) {
      cudaStreamSynchronize(sl.st);
      cudaStreamDestroy(sl.st);
    }
    if (sl.h_stage) cudaFreeHost(sl.h_stage);
  }
  if (s->h_result) cudaFreeHost(s->h_result);
  cudaStreamSynchronize(s->ctx->stream);
  for (auto& b : s->owned) dfree(s->ctx, b.p, b.n);
  for (ta_experiment* e : s->exp_handles) --e->serve_refs;
  delete s;
  return TA_OK;
}

ta_status ta_serve_add_experiment(ta_server* s, ta_experiment* e, const ta_topology* topo,
                                  uint32_t* id) {
  if (!s || !e || !id) return fail(TA_ERR_INVALID_ARG, "ta_serve_add_experiment: NULL argument");
  if (s->exps.size() >= MAX_EXPS) return fail(TA_ERR_CAPACITY, "ta_serve_add_experiment: 64 experiments");
  u64 extra = 0;
  ExpDev d{};
  d.R = e->R;
  d.C = e->C;
  d.n_iter = e->n_iter;
  d.row_off = e->row_off;
  d.entry_off = e->entry_off;
  d.e_ctx = e->e_ctx;
  d.e_time = e->e_time;
  d.e_cnt = e->e_cnt;
  if (e->ts || e->N == 0) {  // traces kept or borrowed: window queries
    const ta_status st = ensure_row_index(e);
    if (st != TA_OK) return st;
    d.rank_off = e->rank_off;
    d.ts = e->ts;
    d.tctx = e->ctxv;
    d.row_first = e->row_first;
  }
  d.off[0] = e->x.off;
  d.ctx[0] = e->x.ctx;
  d.time[0] = e->x.time;
  d.cnt[0] = e->x.cnt;
  if (e->has_incl) {
    d.off[1] = e->in.off;
    d.ctx[1] = e->in.ctx;
    d.time[1] = e->in.time;
    d.cnt[1] = e->in.cnt;
  }
  if (topo) {
    if (!topo->node_of_rank || !topo->rack_of_node || topo->n_nodes == 0 || topo->n_racks == 0)
      return fail(TA_ERR_INVALID_ARG, "ta_serve_add_experiment: topology");
    std::vector<u32> node((u64)e->R), rack(topo->n_nodes);
    ta_ctx* c = s->ctx;
    ta_status st;
    if ((st = copy(c, node.data(), topo->node_of_rank, node.size() * 4)) != TA_OK) return st;
    if ((st = copy(c, rack.data(), topo->rack_of_node, rack.size() * 4)) != TA_OK) return st;
    if ((st = sync_check(c, "ta_serve_add_experiment")) != TA_OK) return st;
    for (u32 v : node)
      if (v >= topo->n_nodes) return fail(TA_ERR_INVALID_ARG, "topology: node_of_rank >= n_nodes");
    for (u32 v : rack)
      if (v >= topo->n_racks) return fail(TA_ERR_INVALID_ARG, "topology: rack_of_node >= n_racks");
    const u64 bytes = node.size() * 4 + rack.size() * 4;
    void* p = dalloc(c, bytes);
    if (!p) return fail(TA_ERR_OOM, "ta_serve_add_experiment: topology");
    s->owned.push_back({p, bytes});
    u32* dn = (u32*)p;
    u32* dr = dn + node.size();
    if ((st = copy(c, dn, node.data(), node.size() * 4)) != TA_OK) return st;
    if ((st = copy(c, dr, rack.data(), rack.size() * 4)) != TA_OK) return st;
    d.node_of_rank = dn;
    d.rack_of_node = dr;
    d.n_nodes = topo->n_nodes;
    d.n_racks = topo->n_racks;
    extra = bytes;
  }
  std::lock_guard<std::mutex> g(s->mu);
  const u64 need = e->device_bytes + extra;
  if (s->cfg.device_budget && s->resident + need > s->cfg.device_budget)
    return fail(TA_ERR_OOM, "ta_serve_add_experiment: %llu resident + %llu > budget %llu",
                (unsigned long long)s->resident, (unsigned long long)need,
                (unsigned long long)s->cfg.device_budget);
  const u32 k = (u32)s->exps.size();
  ta_status st = copy(s->ctx, s->d_exps + k, &d, sizeof d);
  if (st == TA_OK) st = sync_check(s->ctx, "ta_serve_add_experiment");
  if (st != TA_OK) return st;
  s->exps.push_back(d);
  s->exp_handles.push_back(e);
  ++e->serve_refs;
  s->resident += need;
  *id = k;
  return TA_OK;
}

ta_status ta_serve_submit(ta_server* s, const ta_query* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return fail(TA_ERR_INVALID_ARG, "ta_serve_submit: NULL argument");
  QState st;
  st.q = *q;
  {
    std::lock_guard<std::mutex> g(s->mu);
    ta_status v = validate_query(s, q);
    if (v != TA_OK) return v;
    size_query(s, st);
  }
  if (st.res_bytes > s->cfg.result_bytes || align_up(st.scr_bytes) > s->cfg.scratch_bytes ||
      stage_bytes(st) + 3 * ALIGN > s->cfg.staging_bytes)
    return fail(TA_ERR_CAPACITY, "ta_serve_submit: query needs %llu result / %llu scratch / %llu "
                "staging bytes", (unsigned long long)st.res_bytes,
                (unsigned long long)st.scr_bytes, (unsigned long long)stage_bytes(st));
  if (q->kind == TA_Q_STATS) st.ranks.assign(q->ranks, q->ranks + q->n_ranks);
  st.q.ranks = nullptr;
  st.t_submit = now_ns();
  {
    std::lock_guard<std::mutex> g(s->mu);
    const u64 t = s->next_ticket++;
    s->qs.emplace(t, std::move(st));
    s->pending.push_back(t);
    *ticket = t;
  }
  s->cv.notify_all();
  return TA_OK;
}

ta_status ta_serve_poll(ta_server* s, uint64_t ticket, int64_t wait_ns, ta_query_result* r) {
  if (!s || !r) return fail(TA_ERR_INVALID_ARG, "ta_serve_poll: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto itr = s->qs.find(ticket);
  if (itr == s->qs.end()) return fail(TA_ERR_INVALID_ARG, "ta_serve_poll: unknown ticket");
  auto done = [&] {
    auto j = s->qs.find(ticket);
    return j == s->qs.end() || j->second.done;
  };
  if (wait_ns < 0) s->cv.wait(lk, done);
  else if (wait_ns > 0) s->cv.wait_for(lk, std::chrono::nanoseconds(wait_ns), done);
  itr = s->qs.find(ticket);
  if (itr == s->qs.end()) return fail(TA_ERR_INVALID_ARG, "ta_serve_poll: released ticket");
  const QState& st = itr->second;
  if (!st.done) return TA_ERR_STATE;
  r->status = st.status;
  r->kind = st.q.kind;
  r->t_submit_ns = st.t_submit;
  r->t_admit_ns = st.t_admit;
  r->t_launch_ns = st.t_launch;
  r->t_done_ns = st.t_done;
  r->bytes = st.out_bytes;
  r->data = s->h_result + st.res_off;
  return TA_OK;
}

ta_status ta_serve_release(ta_server* s, uint64_t ticket) {
  if (!s) return fail(TA_ERR_INVALID_ARG, "ta_serve_release: NULL argument");
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto itr = s->qs.find(ticket);
    if (itr == s->qs.end()) return fail(TA_ERR_INVALID_ARG, "ta_serve_release: unknown ticket");
    if (!itr->second.done) return fail(TA_ERR_STATE, "ta_serve_release: query not finished");
    auto bl = s->blocks.find(itr->second.block);
    if (bl != s->blocks.end() && --bl->second.second == 0) {
      s->res.release(bl->first, bl->second.first);
      s->blocks.erase(bl);
    }
    s->qs.erase(itr);
    --s->inflight;
  }
  s->cv.notify_all();
  return TA_OK;
}

ta_status ta_serve_replay(ta_server* s, const ta_query* qs, const uint64_t* arrival_ns,
                          uint64_t n, uint64_t* latency_ns, uint64_t* wall_ns) {
  if (!s || (n && (!qs || !arrival_ns || !latency_ns)))
    return fail(TA_ERR_INVALID_ARG, "ta_serve_replay: NULL argument");
  std::vector<std::atomic<u64>> tickets(n);
  for (auto& t : tickets) t.store(0);
  std::atomic<u64> submitted{0};
  std::atomic<u32> first_err{TA_OK};
  const u64 start = now_ns();
  u64 last_done = start;
  std::thread collector([&] {
    for (u64 i = 0; i < n; ++i) {
      u64 t;
      while ((t = tickets[i].load()) == 0) {
        if (first_err.load() != TA_OK && submitted.load() <= i) return;
        std::this_thread::yield();
      }
      if (t == ~0ull) continue;  // refused at submit
      ta_query_result r;
      if (ta_serve_poll(s, t, -1, &r) == TA_OK) {
        latency_ns[i] = r.t_done_ns - (start + arrival_ns[i]);
        last_done = std::max(last_done, r.t_done_ns);
        if (r.status != TA_OK) {
          u32 ok = TA_OK;
          first_err.compare_exchange_strong(ok, r.status);
        }
      }
      ta_serve_release(s, t);
    }
  });
  for (u64 i = 0; i < n; ++i) {
    const u64 due = start + arrival_ns[i];
    for (u64 t = now_ns(); t < due; t = now_ns())
      if (due - t > 200000) std::this_thread::sleep_for(std::chrono::microseconds(50));
    u64 t = 0;
    const ta_status st = ta_serve_submit(s, &qs[i], &t);
    if (st != TA_OK) {
      u32 ok = TA_OK;
      first_err.compare_exchange_strong(ok, (u32)st);
      latency_ns[i] = 0;
      tickets[i].store(~0ull);
    } else {
      tickets[i].store(t);
    }
    submitted.store(i + 1);
  }
  collector.join();
  if (wall_ns) *wall_ns = last_done - start;
  return (ta_status)first_err.load();
}

}  // extern "C"
