// batch.cu -- many independent trace sets analysed as one unit.
//
// All sets are copied into one device arena (ranks, samples and tree nodes
// concatenated, tiles never spanning two sets) and every kernel works on all
// sets at once, looking up each tile's or rank's set.  The launch sequence of
// the whole analysis is therefore fixed by the batch's shape: it is run once
// eagerly to size every product exactly, captured in a CUDA graph, and each
// ta_batch_run replays the graph (then sorts the outliers, whose number is
// only known afterwards, and splits them by set).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ta.h"
#include "ta_api_internal.h"

using namespace ta;

#define TRY(x)                  \
  do {                          \
    ta_status _s = (x);         \
    if (_s != TA_OK) return _s; \
  } while (0)

namespace {

__global__ void k_put_u64(u64* p, u64 v) { *p = v; }

// out[g] for g in [0, seg0[S] + S): element k of segment s (g = seg0[s] + s + k,
// k <= len_s) is in[seg0[s] + k] - in[seg0[s]]: per-set offsets starting at 0,
// each set with its own closing element.
__global__ void k_rel_offsets(const u64* in, u64* out, const u64* seg0, u32 S) {
  const u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= seg0[S] + S) return;
  u32 lo = 0, hi = S;  // last s with seg0[s] + s <= g
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) / 2;
    if (seg0[mid] + mid <= g) lo = mid;
    else hi = mid;
  }
  const u64 k = g - seg0[lo] - lo;
  out[g] = in[seg0[lo] + k] - in[seg0[lo]];
}

constexpr u64 SET_ALIGN = 32;

inline unsigned nblocks(u64 n) { return (unsigned)std::max<u64>(1, (n + 255) / 256); }

}  // namespace

struct ta_batch {
  ta_ctx* ctx = nullptr;
  u32 S = 0, R = 0, Ctot = 0, Cmax = 0, max_depth = 0;
  u64 N = 0, n_tiles = 0;
  u32 tau_num = 3, tau_den = 1;
  u64 outlier_cap = 0;
  // host copies of the set layout
  std::vector<u64> h_rec0, h_rec_end, h_tile0;
  u64 n_samples = 0;  // without alignment padding
  std::vector<u32> h_rank0, h_ctx0, h_C, h_m;
  std::vector<u64> h_row0, h_ent0, h_x0, h_i0, h_out0;
  // device arena
  u64* rank_off = nullptr;
  u64* ts = nullptr;
  u32* cx = nullptr;
  u32* parent = nullptr;
  u32* depth = nullptr;
  u64* span = nullptr;
  u32* n_iter = nullptr;
  u64* row_off = nullptr;
  u64* entry_off = nullptr;
  u32* e_ctx = nullptr;
  u64* e_time = nullptr;
  u32* e_cnt = nullptr;
  // tensor slots (one per run) and the compaction into the arrays above, when
  // some row repeats a context in several runs
  u64 slots = 0;
  bool compact = false;
  TensorCompact TC{};
  Csr x, in;
  // iteration moments of the exclusive entries (see the single-experiment
  // load): time over the iteration rows and its 128-bit sum of squares
  u64* x_m1 = nullptr;
  u64* x_m2 = nullptr;
  uint8_t* x_mom = nullptr;
  ta_ctx_stats* stats = nullptr;
  u64* keys = nullptr;
  double* zs = nullptr;
  ta_outlier* outl = nullptr;
  u64* set_out0 = nullptr;
  // per-set relative offsets
  u64* rel_row_off = nullptr;
  u64* rel_entry_off = nullptr;
  u64* rel_x_off = nullptr;
  u64* rel_i_off = nullptr;
  u64* d_row0 = nullptr;
  u64* d_rank0_64 = nullptr;
  // set map
  SetMap sets{};
  // kernel scratch
  TensorArgs T{};
  TensorPlan TP{};
  TensorShape shape{};
  u32 tune_trials = 0;
  double tune_ms = 0.0;
  u64 n_tiles_max = 0;       // tiles at the narrowest width (sizes the tile arrays)
  u32* d_tile_set = nullptr; // the set map's tile arrays, rewritten per tile width
  u64* d_tile0 = nullptr;
  RankCsrArgs X[2]{};
  RankCsrPlan XP{};
  u64* meta = nullptr;   // [0] status, [1..2] tensor totals, [3] excl total, [4] incl total,
                         // [5] max span, [6] max depth | pad, [7] n_out
  u32* roots = nullptr;  // [S]
  u32* cct_scratch = nullptr;
  unsigned char* stats_scratch = nullptr;
  u64 rows = 0, nnz = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  u64 graph_nodes = 0, graph_kernels = 0;
  u64 n_out = 0;
  u64 device_bytes = 0;
  std::vector<Block> owned;
  // optional per-set speedup and rack rollup
  const ta_batch_set_args* set_args = nullptr;
  BatchSpeedupArgs SP{};
  BatchTopoArgs RT{};
  bool has_sp = false, has_topo = false;
  u64 sp_cells = 0, sp_cv = 0, rt_nodes = 0, rt_chassis = 0, rt_racks = 0;
  std::vector<u32> h_k0, h_nflag;
  std::vector<u64> h_node0, h_ch0, h_rk0;

  ta_status own(size_t bytes, void** p, const char* what) {
    void* q = dalloc(ctx, bytes);
    if (!q) return fail(TA_ERR_OOM, "batch: allocation of %zu bytes for %s failed", bytes, what);
    owned.push_back({q, bytes});
    device_bytes += bytes;
    *p = q;
    return TA_OK;
  }
  template <class T_>
  ta_status own_n(u64 n, T_** p, const char* what) {
    return own(std::max<u64>(n, 1) * sizeof(T_), (void**)p, what);
  }
  void drop() {
    for (auto& b : owned) dfree(ctx, b.p, b.n);
    owned.clear();
  }
};

namespace {

Launch launch_of(ta_batch* b) { return Launch{b->ctx->stream, b->ctx->num_sms, &b->ctx->launches}; }

// Validation and tree depth for all sets (status bits in meta[0]).
void enqueue_validate(ta_batch* b) {
  const Launch L = launch_of(b);
  u32* status = (u32*)b->meta;
  cudaMemsetAsync(b->meta, 0, 64, L.stream);
  cudaMemsetAsync(b->roots, 0, (size_t)b->S * 4, L.stream);
  launch_rank_off(L, b->rank_off, b->R, b->N, b->ts, b->span, b->meta + 5, status, b->sets);
  launch_cct(L, b->parent, b->Ctot, b->depth, (u32*)(b->meta + 6), b->roots, b->cct_scratch, status,
             b->sets);
}

void enqueue_tensor_count(ta_batch* b) {
  const Launch L = launch_of(b);
  launch_tile_first_rank(L, b->rank_off, b->R, b->TP.tile, (u32)b->n_tiles, (u32*)b->T.tfr,
                         b->sets);
  launch_tensor_count(L, b->TP, b->T);
  launch_tile_scan(L, b->T);
}

void enqueue_tensor_write(ta_batch* b) {
  const Launch L = launch_of(b);
  k_put_u64<<<1, 1, 0, L.stream>>>(b->row_off + b->R, b->rows);
  L.count();
  if (!b->compact) {
    k_put_u64<<<1, 1, 0, L.stream>>>(b->entry_off + b->rows, b->slots);
    L.count();
  }
  cudaMemsetAsync(b->T.nnz_sum, 0, 8, L.stream);
  launch_tensor_write(L, b->TP, b->T);
  if (b->compact) launch_tensor_compact(L, b->TC);
  launch_n_iter(L, b->row_off, b->R, b->n_iter);
}

void enqueue_stats(ta_batch* b) {
  const Launch L = launch_of(b);
  launch_batch_stats(L, b->R, b->Ctot, b->x.off, b->x.ctx, b->x.time, b->sets, b->tau_num,
                     b->tau_den, b->stats_scratch, b->stats, b->keys, b->zs, b->outlier_cap,
                     (unsigned long long*)(b->meta + 7));
}

void enqueue_views(ta_batch* b) {
  const Launch L = launch_of(b);
  k_rel_offsets<<<nblocks((u64)b->R + b->S), 256, 0, L.stream>>>(b->row_off, b->rel_row_off,
                                                                   b->d_rank0_64, b->S);
  k_rel_offsets<<<nblocks(b->rows + b->S), 256, 0, L.stream>>>(b->entry_off, b->rel_entry_off,
                                                                b->d_row0, b->S);
  k_rel_offsets<<<nblocks((u64)b->R + b->S), 256, 0, L.stream>>>(b->x.off, b->rel_x_off,
                                                                   b->d_rank0_64, b->S);
  k_rel_offsets<<<nblocks((u64)b->R + b->S), 256, 0, L.stream>>>(b->in.off, b->rel_i_off,
                                                                   b->d_rank0_64, b->S);
  L.count(4);
}

// Everything that runs every time, in order (sizes fixed by the plan).
void enqueue_all(ta_batch* b) {
  const Launch L = launch_of(b);
  enqueue_validate(b);
  enqueue_tensor_count(b);
  enqueue_tensor_write(b);
  for (int mode = 0; mode < 2; ++mode) {
    launch_rank_count(L, b->XP, b->X[mode]);
    launch_rank_write(L, b->XP, b->X[mode]);
  }
  enqueue_stats(b);
  if (b->has_sp) launch_batch_speedup(L, b->SP, b->sp_cells, b->sp_cv);
  if (b->has_topo) launch_batch_topology(L, b->RT, b->rt_nodes, b->rt_chassis, b->rt_racks);
  enqueue_views(b);
}

ta_status check_flags(ta_batch* b, const char* where) {
  u64 h[8];
  TRY(copy(b->ctx, h, b->meta, sizeof h));
  TRY(sync_check(b->ctx, where));
  const u32 f = (u32)h[0];
  if (f & F_INVALID)
    return fail(TA_ERR_INVALID_ARG, "%s: rank offsets of a set are not a valid CSR", where);
  std::vector<u32> roots(b->S);
  TRY(copy(b->ctx, roots.data(), b->roots, (size_t)b->S * 4));
  TRY(sync_check(b->ctx, where));
  for (u32 s = 0; s < b->S; ++s)
    if (roots[s] != 1) return fail(TA_ERR_BAD_CCT, "%s: set %u has %u tree roots", where, s, roots[s]);
  if (f & F_BAD_CCT) return fail(TA_ERR_BAD_CCT, "%s: a set's parent array is invalid", where);
  if ((unsigned __int128)h[5] * b->R >= ((unsigned __int128)1 << 63))
    return fail(TA_ERR_INVALID_ARG, "%s: R * longest span >= 2^63", where);
  TRY(status_from_flags(f, where));
  b->max_depth = (u32)h[6];
  b->n_out = h[7];
  return TA_OK;
}

// Autotuner of the tensor passes' launch shape (warps per CTA, CTAs per SM):
// every candidate runs the pass on the batch's own data once to warm up and
// once timed with CUDA events; the fastest is kept for the captured graph.
// Repeated runs write the same results (the passes are deterministic).
constexpr int kTuneWarps[] = {4, 8, 16};

ta_status tune_tensor(ta_batch* b, bool write, float* best_ms = nullptr) {
  ta_ctx* c = b->ctx;
  const Launch L = launch_of(b);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(TA_ERR_CUDA, "batch: tuning events");
  float best = 3.4e38f;
  TensorShape pick = b->shape;
  for (int nw : kTuneWarps) {
    const int occ = tensor_max_per_sm(b->Cmax, write, nw);
    for (int ps = 1; ps <= occ; ++ps) {
      TensorShape sh = b->shape;
      if (write) {
        sh.nw_write = nw;
        sh.per_sm_write = ps;
      } else {
        sh.nw_count = nw;
        sh.per_sm_count = ps;
      }
      const TensorPlan P = plan_tensor(b->Cmax, b->N, c->num_sms, sh);
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, c->stream);
        if (write) launch_tensor_write(L, P, b->T);
        else launch_tensor_count(L, P, b->T);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      ++b->tune_trials;
      b->tune_ms += ms;
      if (ms < best) {
        best = ms;
        pick = sh;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TRY(sync_check(c, "batch: tuning"));
  b->shape = pick;
  b->TP = plan_tensor(b->Cmax, b->N, c->num_sms, b->shape);
  if (best_ms) *best_ms = best;
  return TA_OK;
}

// Tile widths the autotuner tries (samples per tile).
constexpr int kTuneTiles[] = {4096, 2048};

// The set layout's tiles at width tw: every set's first tile (host and
// device) and every tile's set; tiles never span two sets.
ta_status set_tiles(ta_batch* b, int tw) {
  ta_ctx* c = b->ctx;
  const u32 S = b->S;
  b->h_tile0.assign(S + 1, 0);
  for (u32 s = 0; s < S; ++s) {
    const u64 n = b->h_rec_end[s] - b->h_rec0[s];
    b->h_tile0[s + 1] = b->h_tile0[s] + std::max<u64>(1, (n + tw - 1) / tw);
  }
  b->n_tiles = b->h_tile0[S];
  if (b->n_tiles > b->n_tiles_max) return fail(TA_ERR_STATE, "batch: tile map");
  std::vector<u32> tile_set(b->n_tiles);
  for (u32 s = 0; s < S; ++s)
    for (u64 t = b->h_tile0[s]; t < b->h_tile0[s + 1]; ++t) tile_set[t] = s;
  TRY(copy(c, b->d_tile_set, tile_set.data(), tile_set.size() * 4));
  TRY(copy(c, b->d_tile0, b->h_tile0.data(), (S + 1) * 8));
  TRY(sync_check(c, "batch: tile map"));
  b->T.n_tiles = b->n_tiles;
  return TA_OK;
}

// Per-set speedup and rack-rollup requests: host-side layout of every set's
// share of the work and outputs, from the products of the plan's first run.
ta_status plan_rollups(ta_batch* b) {
  const ta_batch_set_args* sa = b->set_args;
  if (!sa) return TA_OK;
  ta_ctx* c = b->ctx;
  const u32 S = b->S;
  bool any_sp = false, any_topo = false;
  for (u32 s = 0; s < S; ++s) {
    any_sp = any_sp || (sa[s].speedup_ctxs && sa[s].n_speedup_ctxs);
    any_topo = any_topo || sa[s].node_of_rank;
  }
  std::vector<u32> n_iter(b->R);
  std::vector<u64> span(b->R);
  TRY(copy(c, n_iter.data(), b->n_iter, (u64)b->R * 4));
  TRY(copy(c, span.data(), b->span, (u64)b->R * 8));
  TRY(sync_check(c, "batch: rollup sizes"));
  if (any_sp) {
    constexpr u32 GROUP = 256;  // ranks per cells work item
    std::vector<u32> kmap(b->Ctot, NONE32), k0(S + 1, 0), istar(S, 0);
    std::vector<u64> cell0(S + 1, 0), cv0(S + 1, 0), item0(S + 1, 0), excl(S, 0), tapp(S, 0);
    for (u32 s = 0; s < S; ++s) {
      const u32 nk = (sa[s].speedup_ctxs) ? sa[s].n_speedup_ctxs : 0u;
      const u32 r0 = b->h_rank0[s], r1 = b->h_rank0[s + 1], n = r1 - r0;
      for (u32 k = 0; k < nk; ++k) {
        const u32 cx = sa[s].speedup_ctxs[k];
        if (cx >= b->h_C[s] || (k && cx <= sa[s].speedup_ctxs[k - 1]))
          return fail(TA_ERR_INVALID_ARG, "batch: set %u: speedup contexts must be sorted, "
                      "unique, < n_ctx", s);
        kmap[b->h_ctx0[s] + cx] = k;
      }
      k0[s + 1] = k0[s] + nk;
      u32 I = 0xFFFFFFFFu;
      u64 sum_it = 0, mspan = 0;
      for (u32 r = r0; r < r1; ++r) {
        I = std::min(I, n_iter[r]);
        sum_it += n_iter[r];
        mspan = std::max(mspan, span[r]);
      }
      if (nk == 0) I = 0;
      istar[s] = I;
      excl[s] = nk ? sum_it - (u64)n * I : 0;
      tapp[s] = sa[s].app_time_ns ? sa[s].app_time_ns : mspan;
      cell0[s + 1] = cell0[s] + (u64)I * nk;
      cv0[s + 1] = cv0[s] + (u64)n * nk;
      const u64 items = (nk && I) ? (u64)I * ((nk + 63) / 64) * ((n + GROUP - 1) / GROUP) : 0;
      item0[s + 1] = item0[s] + items;
    }
    BatchSpeedupArgs& P = b->SP;
    P.S = S;
    P.R = b->R;
    P.nk_total = k0[S];
    P.group = GROUP;
    P.n_items = item0[S];
    P.rank_set = b->sets.rank_set;
    P.set_rank0 = b->sets.set_rank0;
    P.set_ctx0 = b->sets.set_ctx0;
    P.row_off = b->row_off;
    P.entry_off = b->entry_off;
    P.e_ctx = b->e_ctx;
    P.e_time = b->e_time;
    P.x_off = b->x.off;
    P.x_ctx = b->x.ctx;
    P.x_m1 = b->x_m1;
    P.x_m2 = b->x_m2;
    P.mom_ok = b->x_mom;
    u32 *d_kmap = nullptr, *d_k0 = nullptr, *d_istar = nullptr;
    u64 *d_cell0 = nullptr, *d_cv0 = nullptr, *d_item0 = nullptr, *d_excl = nullptr,
        *d_tapp = nullptr;
    TRY(b->own_n(b->Ctot, &d_kmap, "speedup map"));
    TRY(b->own_n(S + 1, &d_k0, "speedup layout"));
    TRY(b->own_n(S, &d_istar, "speedup layout"));
    TRY(b->own_n(S + 1, &d_cell0, "speedup layout"));
    TRY(b->own_n(S + 1, &d_cv0, "speedup layout"));
    TRY(b->own_n(S + 1, &d_item0, "speedup layout"));
    TRY(b->own_n(S, &d_excl, "speedup layout"));
    TRY(b->own_n(S, &d_tapp, "speedup layout"));
    TRY(copy(c, d_kmap, kmap.data(), kmap.size() * 4));
    TRY(copy(c, d_k0, k0.data(), (S + 1) * 4));
    TRY(copy(c, d_istar, istar.data(), S * 4));
    TRY(copy(c, d_cell0, cell0.data(), (S + 1) * 8));
    TRY(copy(c, d_cv0, cv0.data(), (S + 1) * 8));
    TRY(copy(c, d_item0, item0.data(), (S + 1) * 8));
    TRY(copy(c, d_excl, excl.data(), S * 8));
    TRY(copy(c, d_tapp, tapp.data(), S * 8));
    P.kmap = d_kmap;
    P.k0 = d_k0;
    P.istar = d_istar;
    P.cell0 = d_cell0;
    P.cv0 = d_cv0;
    P.item0 = d_item0;
    P.excluded = d_excl;
    P.t_app = d_tapp;
    b->sp_cells = cell0[S];
    b->sp_cv = cv0[S];
    TRY(b->own_n(std::max<u64>(b->sp_cells, 1), &P.g_sum, "speedup cells"));
    TRY(b->own_n(std::max<u64>(b->sp_cells, 1), &P.g_max, "speedup cells"));
    TRY(b->own_n(std::max<u64>(b->sp_cells, 1), &P.g_sqlo, "speedup cells"));
    TRY(b->own_n(std::max<u64>(b->sp_cells, 1), &P.g_sqhi, "speedup cells"));
    TRY(b->own_n(std::max<u64>(b->sp_cv, 1), &P.cvw, "speedup cv terms"));
    TRY(b->own_n(std::max<u64>(b->sp_cv, 1), &P.cvw2, "speedup cv terms"));
    TRY(b->own_n(std::max<u32>(P.nk_total, 1), &P.wsum, "speedup sums"));
    TRY(b->own_n(std::max<u32>(P.nk_total, 1), &P.per, "speedup per context"));
    TRY(b->own_n(S, &P.tot, "speedup totals"));
    b->h_k0 = k0;
    b->has_sp = P.nk_total > 0;
  }
  if (any_topo) {
    std::vector<u32> has(S, 0), tctx(S, 0), tn(S, 1), td(S, 1), mr(S, 1), node(b->R, 0);
    std::vector<u64> node0(S + 1, 0), ch0(S + 1, 0), rk0(S + 1, 0);
    std::vector<u32> rack, chassis;
    for (u32 s = 0; s < S; ++s) {
      const ta_batch_set_args& a = sa[s];
      const u32 r0 = b->h_rank0[s], n = b->h_rank0[s + 1] - r0;
      if (a.node_of_rank) {
        if (!a.rack_of_node || !a.chassis_of_node || !a.n_nodes || !a.n_racks || !a.n_chassis ||
            a.topo_ctx >= b->h_C[s] || !a.topo_tau_den || !a.topo_min_ranks)
          return fail(TA_ERR_INVALID_ARG, "batch: set %u: rack rollup arguments", s);
        for (u32 i = 0; i < n; ++i) {
          if (a.node_of_rank[i] >= a.n_nodes)
            return fail(TA_ERR_INVALID_ARG, "batch: set %u: node_of_rank >= n_nodes", s);
          node[r0 + i] = a.node_of_rank[i];
        }
        for (u32 i = 0; i < a.n_nodes; ++i) {
          if (a.rack_of_node[i] >= a.n_racks || a.chassis_of_node[i] >= a.n_chassis)
            return fail(TA_ERR_INVALID_ARG, "batch: set %u: rack or chassis id out of range", s);
          rack.push_back(a.rack_of_node[i]);
          chassis.push_back(a.chassis_of_node[i]);
        }
        has[s] = 1;
        tctx[s] = a.topo_ctx;
        tn[s] = a.topo_tau_num;
        td[s] = a.topo_tau_den;
        mr[s] = a.topo_min_ranks;
      }
      node0[s + 1] = node0[s] + (has[s] ? a.n_nodes : 0);
      ch0[s + 1] = ch0[s] + (has[s] ? a.n_chassis : 0);
      rk0[s + 1] = rk0[s] + (has[s] ? a.n_racks : 0);
    }
    BatchTopoArgs& T = b->RT;
    T.S = S;
    T.R = b->R;
    T.rank_set = b->sets.rank_set;
    T.set_ctx0 = b->sets.set_ctx0;
    T.x_off = b->x.off;
    T.x_ctx = b->x.ctx;
    T.x_time = b->x.time;
    T.stats = b->stats;
    b->rt_nodes = node0[S];
    b->rt_chassis = ch0[S];
    b->rt_racks = rk0[S];
    u32 *d_has = nullptr, *d_ctx = nullptr, *d_tn = nullptr, *d_td = nullptr, *d_mr = nullptr,
        *d_node = nullptr, *d_rack = nullptr, *d_ch = nullptr;
    u64 *d_n0 = nullptr, *d_c0 = nullptr, *d_r0 = nullptr;
    TRY(b->own_n(S, &d_has, "rollup layout"));
    TRY(b->own_n(S, &d_ctx, "rollup layout"));
    TRY(b->own_n(S, &d_tn, "rollup layout"));
    TRY(b->own_n(S, &d_td, "rollup layout"));
    TRY(b->own_n(S, &d_mr, "rollup layout"));
    TRY(b->own_n(b->R, &d_node, "rollup nodes"));
    TRY(b->own_n(std::max<u64>(b->rt_nodes, 1), &d_rack, "rollup racks"));
    TRY(b->own_n(std::max<u64>(b->rt_nodes, 1), &d_ch, "rollup chassis"));
    TRY(b->own_n(S + 1, &d_n0, "rollup layout"));
    TRY(b->own_n(S + 1, &d_c0, "rollup layout"));
    TRY(b->own_n(S + 1, &d_r0, "rollup layout"));
    TRY(copy(c, d_has, has.data(), S * 4));
    TRY(copy(c, d_ctx, tctx.data(), S * 4));
    TRY(copy(c, d_tn, tn.data(), S * 4));
    TRY(copy(c, d_td, td.data(), S * 4));
    TRY(copy(c, d_mr, mr.data(), S * 4));
    TRY(copy(c, d_node, node.data(), (u64)b->R * 4));
    if (!rack.empty()) {
      TRY(copy(c, d_rack, rack.data(), rack.size() * 4));
      TRY(copy(c, d_ch, chassis.data(), chassis.size() * 4));
    }
    TRY(copy(c, d_n0, node0.data(), (S + 1) * 8));
    TRY(copy(c, d_c0, ch0.data(), (S + 1) * 8));
    TRY(copy(c, d_r0, rk0.data(), (S + 1) * 8));
    TRY(sync_check(c, "batch: rollup layout"));
    T.has = d_has;
    T.ctx = d_ctx;
    T.tau_num = d_tn;
    T.tau_den = d_td;
    T.min_ranks = d_mr;
    T.node_of_rank = d_node;
    T.rack_of_node = d_rack;
    T.chassis_of_node = d_ch;
    T.node0 = d_n0;
    T.chassis0 = d_c0;
    T.rack0 = d_r0;
    const u64 nn = std::max<u64>(b->rt_nodes, 1), nc = std::max<u64>(b->rt_chassis, 1),
              nr = std::max<u64>(b->rt_racks, 1);
    TRY(b->own_n(nn, &T.node_out, "rollup outputs"));
    TRY(b->own_n(nn, &T.node_sum, "rollup outputs"));
    TRY(b->own_n(nn, &T.node_ranks, "rollup outputs"));
    TRY(b->own_n(nn, &T.node_flag, "rollup outputs"));
    TRY(b->own_n(nc, &T.ch_flag, "rollup outputs"));
    TRY(b->own_n(nc, &T.ch_nodes, "rollup outputs"));
    TRY(b->own_n(nc, &T.ch_sum, "rollup outputs"));
    TRY(b->own_n(nr, &T.rk_flag, "rollup outputs"));
    TRY(b->own_n(nr, &T.rk_nodes, "rollup outputs"));
    TRY(b->own_n(nr, &T.rk_sum, "rollup outputs"));
    TRY(b->own_n(nr, &T.flagged, "rollup outputs"));
    TRY(b->own_n(S, &T.n_flagged, "rollup outputs"));
    b->h_node0 = node0;
    b->h_ch0 = ch0;
    b->h_rk0 = rk0;
    b->has_topo = b->rt_nodes > 0;
  }
  return TA_OK;
}

ta_status create_impl(ta_batch* b, const ta_trace_desc* sets, u32 S) {
  ta_ctx* c = b->ctx;
  const Launch L = launch_of(b);
  // ---- layout --------------------------------------------------------------
  b->S = S;
  b->h_rec0.assign(S + 1, 0);
  b->h_rec_end.assign(S, 0);
  b->h_tile0.assign(S + 1, 0);
  b->h_rank0.assign(S + 1, 0);
  b->h_ctx0.assign(S + 1, 0);
  b->h_C.resize(S);
  b->h_m.resize(S);
  for (u32 s = 0; s < S; ++s) {
    const ta_trace_desc& d = sets[s];
    if (d.n_ranks == 0 || d.n_ctx == 0 || d.marker_ctx >= d.n_ctx || !d.rank_off || !d.parent ||
        (d.n_records && (!d.ts || !d.ctx)) || d.mem_kind > 1)
      return fail(TA_ERR_INVALID_ARG, "batch: set %u: invalid description", s);
    if (d.n_ctx > 0x7FFFFFFFu) return fail(TA_ERR_INVALID_ARG, "batch: set %u: n_ctx", s);
    // every set starts on a 32-sample boundary: the sample passes read
    // 4-sample vectors at tile-relative offsets
    b->h_rec_end[s] = b->h_rec0[s] + d.n_records;
    b->h_rec0[s + 1] = (b->h_rec_end[s] + SET_ALIGN - 1) / SET_ALIGN * SET_ALIGN;
    b->n_samples += d.n_records;
    b->n_tiles_max += std::max<u64>(1, (d.n_records + 2047) / 2048);
    if ((u64)b->h_rank0[s] + d.n_ranks >= 0xFFFFFFFFull)
      return fail(TA_ERR_INVALID_ARG, "batch: too many ranks");
    b->h_rank0[s + 1] = b->h_rank0[s] + d.n_ranks;
    if ((u64)b->h_ctx0[s] + d.n_ctx >= 0x7FFFFFFFull)
      return fail(TA_ERR_INVALID_ARG, "batch: too many contexts");
    b->h_ctx0[s + 1] = b->h_ctx0[s] + d.n_ctx;
    b->h_C[s] = d.n_ctx;
    b->h_m[s] = d.marker_ctx;
    b->Cmax = std::max(b->Cmax, d.n_ctx);
  }
  b->N = b->h_rec0[S];
  b->R = b->h_rank0[S];
  b->Ctot = b->h_ctx0[S];
  // ---- inputs ---------------------------------------------------------------
  TRY(b->own_n((u64)b->R + 1, &b->rank_off, "rank_off"));
  TRY(b->own_n(b->N, &b->ts, "ts"));
  TRY(b->own_n(b->N, &b->cx, "ctx"));
  TRY(b->own_n(b->Ctot, &b->parent, "parent"));
  std::vector<u64> ro((u64)b->R + 1);
  for (u32 s = 0; s < S; ++s) {
    const ta_trace_desc& d = sets[s];
    std::vector<u64> local((u64)d.n_ranks + 1);
    TRY(copy(c, local.data(), d.rank_off, local.size() * 8));
    TRY(sync_check(c, "batch: rank offsets"));
    if (local[0] != 0 || local[d.n_ranks] != d.n_records)
      return fail(TA_ERR_INVALID_ARG, "batch: set %u: rank_off must start at 0 and end at n_records",
                  s);
    for (u32 r = 0; r <= d.n_ranks; ++r) ro[b->h_rank0[s] + r] = b->h_rec0[s] + local[r];
    TRY(copy(c, b->ts + b->h_rec0[s], d.ts, d.n_records * 8));
    TRY(copy(c, b->cx + b->h_rec0[s], d.ctx, d.n_records * 4));
    TRY(copy(c, b->parent + b->h_ctx0[s], d.parent, (u64)d.n_ctx * 4));
    const u64 pad = b->h_rec0[s + 1] - b->h_rec_end[s];
    if (pad) {  // padding samples belong to no rank; keep them defined
      cudaMemsetAsync(b->ts + b->h_rec_end[s], 0, pad * 8, c->stream);
      cudaMemsetAsync(b->cx + b->h_rec_end[s], 0, pad * 4, c->stream);
    }
  }
  ro[b->R] = b->N;
  TRY(copy(c, b->rank_off, ro.data(), ro.size() * 8));
  // ---- set map on the device ------------------------------------------------
  std::vector<u32> rank_set(b->R);
  for (u32 s = 0; s < S; ++s)
    for (u32 r = b->h_rank0[s]; r < b->h_rank0[s + 1]; ++r) rank_set[r] = s;
  u32 *d_rank_set, *d_rank0, *d_ctx0, *d_C, *d_m;
  u64 *d_rec0, *d_rec_end;
  TRY(b->own_n(b->n_tiles_max, &b->d_tile_set, "set map"));
  TRY(b->own_n(b->R, &d_rank_set, "set map"));
  TRY(b->own_n(S + 1, &d_rank0, "set map"));
  TRY(b->own_n(S + 1, &d_ctx0, "set map"));
  TRY(b->own_n(S, &d_C, "set map"));
  TRY(b->own_n(S, &d_m, "set map"));
  TRY(b->own_n(S + 1, &b->d_tile0, "set map"));
  TRY(b->own_n(S + 1, &d_rec0, "set map"));
  TRY(b->own_n(S, &d_rec_end, "set map"));
  TRY(b->own_n(S + 1, &b->d_rank0_64, "set map"));
  TRY(copy(c, d_rank_set, rank_set.data(), rank_set.size() * 4));
  TRY(copy(c, d_rank0, b->h_rank0.data(), (S + 1) * 4));
  TRY(copy(c, d_ctx0, b->h_ctx0.data(), (S + 1) * 4));
  TRY(copy(c, d_C, b->h_C.data(), S * 4));
  TRY(copy(c, d_m, b->h_m.data(), S * 4));
  TRY(copy(c, d_rec0, b->h_rec0.data(), (S + 1) * 8));
  TRY(copy(c, d_rec_end, b->h_rec_end.data(), S * 8));
  std::vector<u64> rank0_64(b->h_rank0.begin(), b->h_rank0.end());
  TRY(copy(c, b->d_rank0_64, rank0_64.data(), (S + 1) * 8));
  TRY(sync_check(c, "batch: upload"));
  b->sets.S = S;
  b->sets.tile_set = b->d_tile_set;
  b->sets.set_tile0 = b->d_tile0;
  b->sets.set_rec0 = d_rec0;
  b->sets.set_rec_end = d_rec_end;
  b->sets.set_rank0 = d_rank0;
  b->sets.set_ctx0 = d_ctx0;
  b->sets.set_C = d_C;
  b->sets.set_m = d_m;
  b->sets.rank_set = d_rank_set;
  // ---- products and scratch whose size is known now --------------------------
  TRY(b->own(64, (void**)&b->meta, "meta"));
  TRY(b->own_n(S, &b->roots, "roots"));
  TRY(b->own_n(4 * (u64)b->Ctot, &b->cct_scratch, "tree scratch"));
  TRY(b->own_n(b->Ctot, &b->depth, "depth"));
  TRY(b->own_n(b->R, &b->span, "span"));
  TRY(b->own_n((u64)b->R + 1, &b->n_iter, "n_iter"));
  TRY(b->own_n((u64)b->R + 1, &b->row_off, "row_off_of_rank"));
  enqueue_validate(b);
  TRY(check_flags(b, "ta_batch_plan"));
  // tensor: count, size, write -- tile width and launch shapes tuned on the
  // batch's own data (every width: its layout, the count pass's shapes, one
  // count, the write pass's shapes; the fastest width with its shapes wins)
  b->TP = plan_tensor(b->Cmax, b->N, c->num_sms);
  TensorArgs& A = b->T;
  std::memset(&A, 0, sizeof A);
  const u64 nt = b->n_tiles_max;
  TRY(b->own_n(nt + 1, (u32**)&A.tfr, "tile map"));
  TRY(b->own_n(nt, &A.tile_rows, "tile rows"));
  TRY(b->own_n(nt, &A.tile_ents, "tile entries"));
  TRY(b->own_n(nt, &A.tile_row_off, "tile row offsets"));
  TRY(b->own_n(nt, &A.tile_ent_off, "tile entry offsets"));
  TRY(b->own_n(2 * scan_scratch_elems(nt), &A.scan_scratch, "tile scan"));
  // per-warp scratch for the widest launch shape the autotuner may try
  u64 max_warps = 0, max_write_warps = 0;
  for (int tw : kTuneTiles)
    for (int nw : kTuneWarps) {
      max_warps = std::max<u64>(max_warps, (u64)c->num_sms * nw *
                                               tensor_max_per_sm(b->Cmax, false, nw, tw));
      max_write_warps = std::max<u64>(
          max_write_warps, (u64)c->num_sms * nw * tensor_max_per_sm(b->Cmax, true, nw, tw));
    }
  max_warps = std::max(max_warps, max_write_warps);
  if (!b->TP.bm_in_smem) {
    const u64 words = max_warps * bm_words(b->Cmax);
    TRY(b->own_n(words, &A.gbm, "tensor bitmaps"));
    cudaMemsetAsync(A.gbm, 0, words * 4, c->stream);
  }
  const u64 gn = max_write_warps * b->TP.gst_cap;
  TRY(b->own_n(gn, &A.gst_ctx, "tensor stage"));
  TRY(b->own_n(gn, &A.gst_cnt, "tensor stage"));
  TRY(b->own_n(gn, &A.gst_time, "tensor stage"));
  A.rank_off = b->rank_off;
  A.ts = b->ts;
  A.ctx = b->cx;
  A.R = b->R;
  A.C = b->Cmax;
  A.m = 0;
  A.N = b->N;
  A.status = (u32*)b->meta;
  A.totals = b->meta + 1;
  A.gst_cap = b->TP.gst_cap;
  A.bm_in_smem = b->TP.bm_in_smem ? 1u : 0u;
  A.sets = b->sets;
  TRY(b->own_n(1, &A.nnz_sum, "tensor entries"));
  float best_total = 3.4e38f;
  TensorShape best_shape = b->shape;
  bool sized = false;
  for (int tw : kTuneTiles) {
    TRY(set_tiles(b, tw));
    b->shape.tile = tw;
    b->TP = plan_tensor(b->Cmax, b->N, c->num_sms, b->shape);
    launch_tile_first_rank(L, b->rank_off, b->R, tw, (u32)b->n_tiles, (u32*)A.tfr, b->sets);
    float t_count = 0.f, t_write = 0.f;
    TRY(tune_tensor(b, false, &t_count));
    enqueue_tensor_count(b);
    u64 h[3];
    TRY(copy(c, h, b->meta, sizeof h));
    TRY(sync_check(c, "batch: tensor count"));
    TRY(status_from_flags((u32)h[0], "ta_batch_plan"));
    if (!sized) {  // rows and slots do not depend on the tile width
      b->rows = h[1];
      b->slots = h[2];
      TRY(b->own_n(b->rows + 1, &b->entry_off, "entry_off"));
      TRY(b->own_n(b->slots, &b->e_ctx, "e_ctx"));
      TRY(b->own_n(b->slots, &b->e_time, "e_time"));
      TRY(b->own_n(b->slots, &b->e_cnt, "e_cnt"));
      TRY(b->own_n(b->rows, &A.row_nnz, "row entries"));
      A.row_off_of_rank = b->row_off;
      A.entry_off = b->entry_off;
      A.e_ctx = b->e_ctx;
      A.e_time = b->e_time;
      A.e_cnt = b->e_cnt;
      sized = true;
    } else if (h[1] != b->rows || h[2] != b->slots) {
      return fail(TA_ERR_STATE, "batch: tile widths disagree on the tensor's size");
    }
    k_put_u64<<<1, 1, 0, L.stream>>>(b->row_off + b->R, b->rows);
    TRY(tune_tensor(b, true, &t_write));
    if (t_count + t_write < best_total) {
      best_total = t_count + t_write;
      best_shape = b->shape;
    }
  }
  // the chosen width's layout and offsets, then the plan's first write
  b->shape = best_shape;
  TRY(set_tiles(b, b->shape.tile));
  b->TP = plan_tensor(b->Cmax, b->N, c->num_sms, b->shape);
  enqueue_tensor_count(b);
  TRY(check_flags(b, "ta_batch_plan"));
  enqueue_tensor_write(b);
  TRY(check_flags(b, "ta_batch_plan"));
  TRY(copy(c, &b->nnz, A.nnz_sum, 8));
  TRY(sync_check(c, "batch: tensor entries"));
  if (b->nnz > b->slots) return fail(TA_ERR_STATE, "batch: %llu tensor entries in %llu slots",
                                     (unsigned long long)b->nnz, (unsigned long long)b->slots);
  if (b->nnz < b->slots) {  // rows that repeat a context: compact into exact arrays
    TensorCompact& K = b->TC;
    K.rows = b->rows;
    K.slot_off = b->entry_off;
    K.row_nnz = A.row_nnz;
    K.ctx_in = b->e_ctx;
    K.time_in = b->e_time;
    K.cnt_in = b->e_cnt;
    TRY(b->own_n(b->rows + 1, &b->entry_off, "entry_off"));
    TRY(b->own_n(b->nnz, &b->e_ctx, "e_ctx"));
    TRY(b->own_n(b->nnz, &b->e_time, "e_time"));
    TRY(b->own_n(b->nnz, &b->e_cnt, "e_cnt"));
    TRY(b->own_n(scan_scratch_elems(std::max<u64>(b->rows, 1)), &K.scan_scratch, "row scan"));
    K.new_off = b->entry_off;
    K.ctx_out = b->e_ctx;
    K.time_out = b->e_time;
    K.cnt_out = b->e_cnt;
    b->compact = true;
    launch_tensor_compact(L, K);
    TRY(sync_check(c, "batch: tensor compaction"));
  } else {
    k_put_u64<<<1, 1, 0, L.stream>>>(b->entry_off + b->rows, b->nnz);
  }
  // exclusive and inclusive CSR
  b->XP = plan_rank_csr(b->R, b->Cmax, c->num_sms);
  const u64 rg = b->XP.warps() * b->XP.gst_cap;
  u32 *xg_ctx, *xg_cnt, *xg_dep, *xg_par, *x_cnt_r, *xgbm = nullptr;
  u64 *xg_time, *x_scan;
  TRY(b->own_n(rg, &xg_ctx, "csr stage"));
  TRY(b->own_n(rg, &xg_cnt, "csr stage"));
  TRY(b->own_n(rg, &xg_time, "csr stage"));
  TRY(b->own_n(rg, &xg_dep, "csr stage"));
  TRY(b->own_n(rg, &xg_par, "csr stage"));
  TRY(b->own_n(b->R, &x_cnt_r, "csr counts"));
  TRY(b->own_n(scan_scratch_elems(b->R), &x_scan, "csr scan"));
  if (!b->XP.bm_in_smem) {
    const u64 words = b->XP.warps() * bm_words(b->Cmax);
    TRY(b->own_n(words, &xgbm, "csr bitmaps"));
    cudaMemsetAsync(xgbm, 0, words * 4, c->stream);
  }
  // ancestor lists of every set's tree for the inclusive rollup (the trees do
  // not change between runs), unless they would be too long
  u64* anc_off = nullptr;
  u32* anc = nullptr;
  {
    u32* len;
    u64 *aoff, *ascr, *atot;
    TRY(b->own_n(b->Ctot, &len, "ancestor lengths"));
    TRY(b->own_n((u64)b->Ctot + 1, &aoff, "ancestor offsets"));
    TRY(b->own_n(scan_scratch_elems(b->Ctot), &ascr, "ancestor scan"));
    TRY(b->own_n(1, &atot, "ancestor total"));
    launch_anc_offsets(L, b->depth, b->Ctot, len, aoff, atot, ascr);
    u64 total = 0;
    TRY(copy(c, &total, atot, 8));
    TRY(sync_check(c, "batch: ancestors"));
    if (total <= (1ull << 28)) {
      TRY(b->own_n(total, &anc, "ancestor lists"));
      launch_anc_fill(L, b->parent, b->Ctot, aoff, anc, b->sets);
      anc_off = aoff;
    } else {
      anc = nullptr;
    }
  }
  for (int mode = 0; mode < 2; ++mode) {
    RankCsrArgs& X = b->X[mode];
    std::memset(&X, 0, sizeof X);
    Csr& out = mode == 0 ? b->x : b->in;
    TRY(b->own_n((u64)b->R + 1, &out.off, "csr off"));
    X.mode = (u32)mode;
    X.R = b->R;
    X.C = b->Cmax;
    X.max_depth = b->max_depth;
    X.row_off_of_rank = b->row_off;
    X.entry_off = b->entry_off;
    if (mode == 0) {
      X.in_ctx = b->e_ctx;
      X.in_time = b->e_time;
      X.in_cnt = b->e_cnt;
    } else {
      X.in_off = b->x.off;
      X.in_ctx = b->x.ctx;
      X.in_time = b->x.time;
      X.in_cnt = b->x.cnt;
    }
    X.parent = b->parent;
    X.depth = b->depth;
    if (mode == 1) {
      X.anc_off = anc_off;
      X.anc = anc;
    }
    X.out_off = out.off;
    X.out_cnt = x_cnt_r;
    X.total = b->meta + 3 + mode;
    X.scan_scratch = x_scan;
    X.status = (u32*)b->meta;
    X.gbm = xgbm;
    X.gst_ctx = xg_ctx;
    X.gst_cnt = xg_cnt;
    X.gst_time = xg_time;
    X.gst_dep = xg_dep;
    X.gst_par = xg_par;
    X.gst_cap = b->XP.gst_cap;
    X.bm_in_smem = b->XP.bm_in_smem ? 1u : 0u;
    X.sets = b->sets;
    launch_rank_count(L, b->XP, X);
    u64 t = 0;
    TRY(copy(c, &t, b->meta + 3 + mode, 8));
    TRY(sync_check(c, "batch: csr count"));
    out.nnz = t;
    TRY(b->own_n(t, &out.ctx, "csr ctx"));
    TRY(b->own_n(t, &out.time, "csr time"));
    TRY(b->own_n(t, &out.cnt, "csr cnt"));
    X.out_ctx = out.ctx;
    X.out_time = out.time;
    X.out_cnt_e = out.cnt;
    if (mode == 0) {
      TRY(b->own_n(std::max<u64>(t, 1), &b->x_m1, "iteration moments"));
      TRY(b->own_n(std::max<u64>(2 * t, 2), &b->x_m2, "iteration moments"));
      TRY(b->own_n(std::max<u32>(b->R, 1), &b->x_mom, "iteration moments"));
      X.out_m1 = b->x_m1;
      X.out_m2 = b->x_m2;
      X.mom_ok = b->x_mom;
    }
    launch_rank_write(L, b->XP, X);
    TRY(check_flags(b, "ta_batch_plan"));
  }
  // statistics
  TRY(b->own(batch_stats_scratch_bytes(b->Ctot), (void**)&b->stats_scratch, "stats scratch"));
  TRY(b->own_n(b->Ctot, &b->stats, "stats"));
  u64 P2 = 1;
  while (P2 < std::max<u64>(b->outlier_cap, 1)) P2 <<= 1;
  TRY(b->own_n(P2, &b->keys, "outlier keys"));
  TRY(b->own_n(P2, &b->zs, "outlier z"));
  TRY(b->own_n(std::max<u64>(b->outlier_cap, 1), &b->outl, "outliers"));
  TRY(b->own_n(S + 1, &b->set_out0, "outlier offsets"));
  TRY(plan_rollups(b));
  // per-set relative offsets
  std::vector<u64> h_ro((u64)b->R + 1), h_xo((u64)b->R + 1), h_io((u64)b->R + 1);
  TRY(copy(c, h_ro.data(), b->row_off, h_ro.size() * 8));
  TRY(copy(c, h_xo.data(), b->x.off, h_xo.size() * 8));
  TRY(copy(c, h_io.data(), b->in.off, h_io.size() * 8));
  TRY(sync_check(c, "batch: offsets"));
  b->h_row0.resize(S + 1);
  b->h_x0.resize(S + 1);
  b->h_i0.resize(S + 1);
  b->h_ent0.resize(S + 1);
  std::vector<u64> h_ent0(S + 1);
  for (u32 s = 0; s <= S; ++s) {
    b->h_row0[s] = h_ro[b->h_rank0[s]];
    b->h_x0[s] = h_xo[b->h_rank0[s]];
    b->h_i0[s] = h_io[b->h_rank0[s]];
  }
  std::vector<u64> row0_dev(b->h_row0);
  for (u32 s = 0; s <= S; ++s) {
    u64 v = 0;
    TRY(copy(c, &v, b->entry_off + b->h_row0[s], 8));
    TRY(sync_check(c, "batch: offsets"));
    b->h_ent0[s] = v;
  }
  TRY(b->own_n(S + 1, &b->d_row0, "row starts"));
  TRY(copy(c, b->d_row0, row0_dev.data(), (S + 1) * 8));
  TRY(b->own_n((u64)b->R + S, &b->rel_row_off, "relative offsets"));
  TRY(b->own_n(b->rows + S, &b->rel_entry_off, "relative offsets"));
  TRY(b->own_n((u64)b->R + S, &b->rel_x_off, "relative offsets"));
  TRY(b->own_n((u64)b->R + S, &b->rel_i_off, "relative offsets"));
  // ---- capture the whole sequence once, then run it -------------------------
  cudaStream_t st = c->stream;
  bool own_stream = false;
  if (st == nullptr) {  // the legacy default stream cannot be captured
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
      return fail(TA_ERR_CUDA, "batch: stream");
    own_stream = true;
  }
  cudaStream_t saved = c->stream;
  const unsigned long long launches = c->launches;  // capture launches nothing
  c->stream = st;
  cudaError_t err = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (err != cudaSuccess) {
    c->stream = saved;
    return cuda_fail(err, "cudaStreamBeginCapture");
  }
  enqueue_all(b);
  err = cudaStreamEndCapture(st, &b->graph);
  c->stream = saved;
  c->launches = launches;
  if (own_stream) cudaStreamDestroy(st);
  if (err != cudaSuccess) return cuda_fail(err, "cudaStreamEndCapture");
  size_t nodes = 0;
  cudaGraphGetNodes(b->graph, nullptr, &nodes);
  b->graph_nodes = nodes;
  std::vector<cudaGraphNode_t> list(nodes);
  if (nodes) cudaGraphGetNodes(b->graph, list.data(), &nodes);
  for (auto n : list) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(n, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
      ++b->graph_kernels;
  }
  err = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGraphInstantiate");
  const ta_status s = ta_batch_run(b);  // too many outliers is reported by each run
  return s == TA_ERR_CAPACITY ? TA_OK : s;
}

}  // namespace

extern "C" {

ta_status ta_batch_plan(ta_ctx* c, const ta_trace_desc* sets, uint32_t n_sets,
                          const ta_batch_args* args, ta_batch** out) {
  if (!c || !sets || !out || n_sets == 0) return fail(TA_ERR_INVALID_ARG, "ta_batch_plan: arguments");
  *out = nullptr;
  cudaSetDevice(c->device);
  ta_batch* b = new ta_batch();
  b->ctx = c;
  if (args) {
    b->tau_num = args->tau_num;
    b->tau_den = args->tau_den;
    b->outlier_cap = args->outlier_cap;
    b->set_args = args->set_args;
  }
  if (b->tau_den == 0) {
    delete b;
    return fail(TA_ERR_INVALID_ARG, "ta_batch_plan: tau_den = 0");
  }
  if (b->outlier_cap == 0) b->outlier_cap = 1u << 20;
  ta_status s = create_impl(b, sets, n_sets);
  if (s != TA_OK) {
    std::string keep = ta_last_error_message();
    cudaStreamSynchronize(c->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->drop();
    cudaStreamSynchronize(c->stream);
    delete b;
    fail(s, "%s", keep.c_str());
    return s;
  }
  *out = b;
  return TA_OK;
}

ta_status ta_batch_run(ta_batch* b) {
  if (!b || !b->exec) return fail(TA_ERR_STATE, "ta_batch_run: batch not ready");
  ta_ctx* c = b->ctx;
  cudaSetDevice(c->device);
  cudaError_t err = cudaGraphLaunch(b->exec, c->stream);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGraphLaunch");
  c->launches += b->graph_kernels;
  TRY(check_flags(b, "ta_batch_run"));
  const u64 n = std::min(b->n_out, b->outlier_cap);
  const Launch L = launch_of(b);
  launch_batch_outliers(L, b->keys, b->zs, b->n_out <= b->outlier_cap ? n : 0, b->sets, b->outl,
                        b->set_out0);
  b->h_out0.resize(b->S + 1);
  TRY(copy(c, b->h_out0.data(), b->set_out0, (b->S + 1) * 8));
  if (b->has_topo) {
    b->h_nflag.resize(b->S);
    TRY(copy(c, b->h_nflag.data(), b->RT.n_flagged, (u64)b->S * 4));
  }
  TRY(sync_check(c, "ta_batch_run"));
  if (b->n_out > b->outlier_cap)
    return fail(TA_ERR_CAPACITY, "batch: %llu outliers, capacity %llu",
                (unsigned long long)b->n_out, (unsigned long long)b->outlier_cap);
  return TA_OK;
}

ta_status ta_batch_free(ta_batch* b) {
  if (!b) return TA_OK;
  cudaStreamSynchronize(b->ctx->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->drop();
  cudaStreamSynchronize(b->ctx->stream);
  delete b;
  return TA_OK;
}

ta_status ta_batch_get_info(const ta_batch* b, ta_batch_info* i) {
  if (!b || !i) return fail(TA_ERR_INVALID_ARG, "ta_batch_get_info: NULL argument");
  i->n_sets = b->S;
  i->n_ranks = b->R;
  i->n_records = b->n_samples;
  i->n_rows = b->rows;
  i->tensor_nnz = b->nnz;
  i->excl_nnz = b->x.nnz;
  i->incl_nnz = b->in.nnz;
  i->n_outliers = b->n_out;
  i->graph_nodes = b->graph_nodes;
  i->graph_kernels = b->graph_kernels;
  i->count_warps = (u32)b->TP.nw_count;
  i->count_grid = (u32)b->TP.grid_count;
  i->write_warps = (u32)b->TP.nw_write;
  i->write_grid = (u32)b->TP.grid_write;
  i->tune_trials = b->tune_trials;
  i->tile_width = (u32)b->TP.tile;
  i->tune_ms = b->tune_ms;
  i->device_bytes = b->device_bytes;
  return TA_OK;
}

ta_status ta_batch_get_set(const ta_batch* b, uint32_t s, ta_batch_set_view* v) {
  if (!b || !v || s >= b->S) return fail(TA_ERR_INVALID_ARG, "ta_batch_get_set: arguments");
  const u32 r0 = b->h_rank0[s];
  v->n_ranks = b->h_rank0[s + 1] - r0;
  v->n_ctx = b->h_C[s];
  v->tensor.n_iter = b->n_iter + r0;
  v->tensor.row_off_of_rank = b->rel_row_off + r0 + s;
  v->tensor.entry_off = b->rel_entry_off + b->h_row0[s] + s;
  v->tensor.e_ctx = b->e_ctx + b->h_ent0[s];
  v->tensor.e_time = b->e_time + b->h_ent0[s];
  v->tensor.e_cnt = b->e_cnt + b->h_ent0[s];
  v->tensor.span = b->span + r0;
  v->tensor.rows = b->h_row0[s + 1] - b->h_row0[s];
  v->tensor.nnz = b->h_ent0[s + 1] - b->h_ent0[s];
  v->exclusive.off = b->rel_x_off + r0 + s;
  v->exclusive.ctx = b->x.ctx + b->h_x0[s];
  v->exclusive.time = b->x.time + b->h_x0[s];
  v->exclusive.cnt = b->x.cnt + b->h_x0[s];
  v->exclusive.nnz = b->h_x0[s + 1] - b->h_x0[s];
  v->inclusive.off = b->rel_i_off + r0 + s;
  v->inclusive.ctx = b->in.ctx + b->h_i0[s];
  v->inclusive.time = b->in.time + b->h_i0[s];
  v->inclusive.cnt = b->in.cnt + b->h_i0[s];
  v->inclusive.nnz = b->h_i0[s + 1] - b->h_i0[s];
  v->stats = b->stats + b->h_ctx0[s];
  if (b->h_out0.size() == b->S + 1) {
    v->outliers = b->outl + b->h_out0[s];
    v->n_outliers = b->h_out0[s + 1] - b->h_out0[s];
  } else {
    v->outliers = nullptr;
    v->n_outliers = 0;
  }
  v->speedup = nullptr;
  v->speedup_total = nullptr;
  v->n_speedup = 0;
  if (b->has_sp && b->h_k0[s + 1] > b->h_k0[s]) {
    v->speedup = b->SP.per + b->h_k0[s];
    v->speedup_total = b->SP.tot + s;
    v->n_speedup = b->h_k0[s + 1] - b->h_k0[s];
  }
  v->n_flagged_racks = 0;
  v->n_nodes = v->n_chassis = v->n_racks = v->reserved = 0;
  v->node_outliers = v->node_ranks = v->chassis_flagged = v->chassis_nodes = nullptr;
  v->rack_flagged = v->rack_nodes = v->flagged_racks = nullptr;
  v->node_sum = v->chassis_sum = v->rack_sum = nullptr;
  v->node_flag = nullptr;
  if (b->has_topo && b->h_node0[s + 1] > b->h_node0[s]) {
    const BatchTopoArgs& T = b->RT;
    const u64 n0 = b->h_node0[s], c0 = b->h_ch0[s], r0s = b->h_rk0[s];
    v->n_nodes = (u32)(b->h_node0[s + 1] - n0);
    v->n_chassis = (u32)(b->h_ch0[s + 1] - c0);
    v->n_racks = (u32)(b->h_rk0[s + 1] - r0s);
    v->n_flagged_racks = b->h_nflag.size() == b->S ? b->h_nflag[s] : 0;
    v->node_outliers = T.node_out + n0;
    v->node_sum = (const uint64_t*)T.node_sum + n0;
    v->node_ranks = T.node_ranks + n0;
    v->node_flag = T.node_flag + n0;
    v->chassis_flagged = T.ch_flag + c0;
    v->chassis_nodes = T.ch_nodes + c0;
    v->chassis_sum = (const uint64_t*)T.ch_sum + c0;
    v->rack_flagged = T.rk_flag + r0s;
    v->rack_nodes = T.rk_nodes + r0s;
    v->rack_sum = (const uint64_t*)T.rk_sum + r0s;
    v->flagged_racks = T.flagged + r0s;
  }
  return TA_OK;
}

}  // extern "C"
