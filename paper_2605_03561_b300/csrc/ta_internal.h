// ta_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ta.h"
#include "ta_dev.cuh"

namespace ta {

struct Launch {
  cudaStream_t stream;
  int num_sms;
  unsigned long long* launches;  // counter of kernel launches
  void count(int k = 1) const {
    __atomic_fetch_add(launches, (unsigned long long)k, __ATOMIC_RELAXED);
  }
};

// Several independent trace sets analysed together: sets are concatenated
// (ranks, samples, contexts) and every kernel looks up its set.  All arrays
// are null for a single experiment.
struct SetMap {
  u32 S;                  // number of sets (0 = single experiment)
  const u32* tile_set;    // [n_tiles] set of each tile
  const u64* set_tile0;   // [S+1] first tile of each set
  const u64* set_rec0;    // [S+1] first sample of each set (aligned; [S] = arena end)
  const u64* set_rec_end; // [S] one past the last sample of each set (<= set_rec0[s+1])
  const u32* set_rank0;   // [S+1] first rank of each set
  const u32* set_ctx0;    // [S+1] first context of each set (tree arrays)
  const u32* set_C;       // [S] contexts of each set
  const u32* set_m;       // [S] marker of each set
  const u32* rank_set;    // [R] set of each rank
};

// Set of a (global) context id: the last set whose first context is <= v.
__device__ __forceinline__ u32 set_of_ctx(const SetMap& sets, u32 v) {
  u32 lo = 0, hi = sets.S;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) / 2;
    if (sets.set_ctx0[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------- ingest ----
struct TensorArgs {
  const u64* rank_off;
  const u64* ts;
  const u32* ctx;
  u32 R, C, m;
  u64 n_tiles;
  u64 N;
  const u32* tfr;  // [n_tiles + 1] first rank starting at or after tile start
  // per-tile counts (count pass: rows, run heads) and their exclusive prefix
  u32* tile_rows;
  u64* tile_ents;
  u64* tile_row_off;
  u64* tile_ent_off;
  u64* totals;  // [2] rows, entry slots (= run heads)
  u64* scan_scratch;  // 2 x scan_scratch_elems(n_tiles)
  // outputs (write pass): rows exactly sized, entries at slots (one per run;
  // a row's distinct contexts fill the first row_nnz[row] of its slots)
  u64* row_off_of_rank;
  u64* entry_off;  // first slot of each row
  u32* row_nnz;    // [rows] distinct contexts of each row
  u64* nnz_sum;    // [1] total of row_nnz (added to)
  u32* e_ctx;
  u64* e_time;
  u32* e_cnt;
  u32* gbm;  // global bitmaps (per warp) when not in shared memory
  u32* gst_ctx;
  u64* gst_time;
  u32* gst_cnt;
  u32 gst_cap;  // per warp: rows with more entries than shared staging holds
  u32 bm_in_smem;
  u32* status;
  SetMap sets;
};

// Launch shape of the two tensor passes: the tile width (samples per tile:
// 4096, or 2048), warps per CTA (4, 8 or 16) and CTAs per SM (0 = as many as
// fit), the latter two chosen separately for the count and the write pass
// (the batched form tunes all of them on its data).
struct TensorShape {
  int tile = 4096;
  int nw_count = 8, per_sm_count = 0, nw_write = 8, per_sm_write = 0;
};
struct TensorPlan {
  int tile;
  int nw_count, grid_count, nw_write, grid_write;
  size_t smem, smem_count;
  bool bm_in_smem;
  u32 gst_cap;
  u64 warps() const {
    return (u64)std::max(grid_count * nw_count, grid_write * nw_write);
  }
  u64 write_warps() const { return (u64)grid_write * nw_write; }
};
TensorPlan plan_tensor(u32 C, u64 N, int num_sms, const TensorShape& shape = TensorShape{});
// CTAs of a pass that fit on one SM (occupancy) for warps per CTA nw.
int tensor_max_per_sm(u32 C, bool write, int nw, int tile = 4096);
void launch_tensor_count(const Launch& L, const TensorPlan& P, const TensorArgs& A);
void launch_tile_scan(const Launch& L, const TensorArgs& A);
void launch_tensor_write(const Launch& L, const TensorPlan& P, const TensorArgs& A);
// When some row fills fewer slots than it has runs: exact offsets (scan of
// row_nnz into new_off[rows + 1]) and a copy into exactly sized arrays.
struct TensorCompact {
  u64 rows;
  const u64* slot_off;  // [rows] first slot of each row (the write pass's entry_off)
  const u32* row_nnz;   // [rows]
  u64* new_off;         // [rows + 1]
  u64* scan_scratch;    // scan_scratch_elems(rows)
  const u32* ctx_in;
  const u64* time_in;
  const u32* cnt_in;
  u32* ctx_out;
  u64* time_out;
  u32* cnt_out;
};
void launch_tensor_compact(const Launch& L, const TensorCompact& K);

// With sets, the last rank of set s ends at set_rec_end[s] (samples between
// set_rec_end[s] and set_rec0[s+1] are alignment padding of no rank).
void launch_rank_off(const Launch& L, const u64* rank_off, u32 R, u64 N, const u64* ts,
                     u64* span, u64* max_span, u32* status, const SetMap& sets);
void launch_tile_first_rank(const Launch& L, const u64* rank_off, u32 R, u32 tile, u32 n_tiles,
                            u32* tfr, const SetMap& sets);
// parent[C] -> depth[C], *max_depth; scratch: 4*C u32.
// With sets, parent ids are local to each set's tree and roots[s] counts the
// roots of set s (roots has S entries); depth is per tree.
void launch_cct(const Launch& L, const u32* parent, u32 C, u32* depth, u32* max_depth,
                u32* roots, u32* scratch, u32* status, const SetMap& sets);
void launch_n_iter(const Launch& L, const u64* row_off_of_rank, u32 R, u32* n_iter);

// Per-rank CSR of distinct contexts (mode 0: exclusive from the tensor,
// mode 1: inclusive from the exclusive CSR): count pass + scan, write pass.
struct RankCsrArgs {
  u32 mode, R, C, max_depth;
  // mode 0 input: tensor
  const u64* row_off_of_rank;
  const u64* entry_off;
  // mode 1 input: exclusive CSR offsets
  const u64* in_off;
  const u32* in_ctx;
  const u64* in_time;
  const u32* in_cnt;
  const u32* parent;
  const u32* depth;
  // inclusive: per context its ancestors, itself first ([anc_off[v],
  // anc_off[v+1]) of anc, ids local to the set); null: level-by-level sweep
  const u64* anc_off;
  const u32* anc;
  u32* out_cnt;  // [R] count pass
  u64* out_off;  // [R+1] scan
  u32* out_ctx;
  u64* out_time;
  u32* out_cnt_e;
  u64* total;  // [1]
  u64* scan_scratch;
  u32* gbm;
  u32* gst_ctx;
  u64* gst_time;
  u32* gst_cnt;
  u32* gst_dep;
  u32* gst_par;
  u32 gst_cap;
  u32 bm_in_smem;
  u32* status;
  SetMap sets;
  // exclusive in one pass (mode 0): the write pass runs first, records every
  // rank's distinct count in out_cnt and writes ranks of at most xs_cap
  // contexts to a per-rank scratch (r * xs_cap); with only_over set it
  // writes just the ranks above xs_cap, at out_off
  u32* xs_ctx;
  u64* xs_time;
  u32* xs_cnt;
  u32 xs_cap;
  u32 only_over;
  unsigned long long* n_over;  // [1] ranks above xs_cap
  // exclusive, optional (null: not written): per entry the iteration
  // moments (time summed over the rank's rows after its first, and the
  // 128-bit sum of squares as lo, hi), at out_off or in the scratch like
  // the entries; mom_ok[r] = 1 where they were taken (every iteration row of
  // the rank holds the same contexts), else 0
  u64* out_m1;
  u64* out_m2;
  u64* xs_m1;
  u64* xs_m2;
  uint8_t* mom_ok;
};
// Kernels of the rank passes by variant: 0 exclusive, 1 inclusive by a
// level-by-level sweep, 2 inclusive through ancestor lists.
struct RankCsrPlan {
  int threads;
  int grid[3][2];     // [variant][write]: CTAs of each kernel (its own occupancy)
  size_t smem[3][2];  // [variant][write]: dynamic shared memory per CTA
  bool bm_in_smem;
  u32 gst_cap;
  u32 n_units;
  u64 warps() const {  // per-warp scratch (bitmaps, stages) covers every kernel
    int g = 0;
    for (int m = 0; m < 3; ++m)
      for (int w = 0; w < 2; ++w) g = std::max(g, grid[m][w]);
    return (u64)g * (threads / 32);
  }
};
RankCsrPlan plan_rank_csr(u32 R, u32 C, int num_sms);
void launch_rank_count(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A);
void launch_rank_write(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A);
// Exclusive in one pass: the write pass into the per-rank scratch, the scan
// of the counts, then (after the caller allocates) the copy to the CSR.
void launch_excl_scratch(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A);
void launch_excl_copy(const Launch& L, const RankCsrArgs& A);

// Ancestor lists of every context (itself first, then up to the root):
// anc_off = exclusive scan of depth + 1 (total in *total; len and scratch:
// C u32 and scan_scratch_elems(C) u64), then the lists.  With sets, parent
// ids are local to each set's tree and so are the listed ids.
void launch_anc_offsets(const Launch& L, const u32* depth, u32 C, u32* len, u64* anc_off,
                        u64* total, u64* scratch);
void launch_anc_fill(const Launch& L, const u32* parent, u32 C, const u64* anc_off, u32* anc,
                     const SetMap& sets);

// Batch statistics (stats.cu).
u64 batch_stats_scratch_bytes(u32 Ctot);
void launch_batch_stats(const Launch& L, u32 R, u32 Ctot, const u64* off, const u32* ctx,
                        const u64* time, const SetMap& sets, u32 tau_num, u32 tau_den,
                        unsigned char* scratch, ta_ctx_stats* stats, u64* keys, double* zs,
                        u64 cap, unsigned long long* n_out);
void launch_batch_outliers(const Launch& L, u64* keys, double* zs, u64 n, const SetMap& sets,
                           ta_outlier* out, u64* set_off);

// Potential speedup and rack rollup of every set of a batch (batch_rollup.cu).
// Per set s: contexts k0[s] .. k0[s+1] of the global context index (kmap maps
// a set-local context, offset by the set's first context, to its index in
// the set's list), I* istar[s], cells at cell0[s] (I* x nk), CV terms at
// cv0[s] (nk x ranks), cells work items at item0[s].
struct BatchSpeedupArgs {
  u32 S, R, nk_total, group;
  u64 n_items;
  const u32* rank_set;
  const u32* set_rank0;
  const u32* set_ctx0;
  const u64* row_off;
  const u64* entry_off;
  const u32* e_ctx;
  const u64* e_time;
  // exclusive entries with their iteration moments (mom_ok[r]: rank r's are set)
  const u64* x_off;
  const u32* x_ctx;
  const u64* x_m1;
  const u64* x_m2;
  const uint8_t* mom_ok;
  const u32* kmap;
  const u32* k0;
  const u32* istar;
  const u64* cell0;
  const u64* cv0;
  const u64* item0;
  const u64* excluded;
  const u64* t_app;
  u64 *g_sum, *g_max, *g_sqlo, *g_sqhi;
  double *cvw, *cvw2, *wsum;
  ta_speedup_ctx* per;
  ta_speedup_total* tot;
};
struct BatchTopoArgs {
  u32 S, R;
  const u32* rank_set;
  const u32* set_ctx0;
  const u64* x_off;
  const u32* x_ctx;
  const u64* x_time;
  const ta_ctx_stats* stats;
  const u32* has;
  const u32* ctx;
  const u32* tau_num;
  const u32* tau_den;
  const u32* min_ranks;
  const u32* node_of_rank;     // [R] node within the rank's set
  const u32* rack_of_node;     // nodes of all sets, concatenated
  const u32* chassis_of_node;
  const u64* node0;            // [S+1]
  const u64* chassis0;         // [S+1]
  const u64* rack0;            // [S+1]
  u32* node_out;
  unsigned long long* node_sum;
  u32* node_ranks;
  uint8_t* node_flag;
  u32* ch_flag;
  u32* ch_nodes;
  unsigned long long* ch_sum;
  u32* rk_flag;
  u32* rk_nodes;
  unsigned long long* rk_sum;
  u32* flagged;
  u32* n_flagged;  // [S]
};
void launch_batch_speedup(const Launch& L, const BatchSpeedupArgs& P, u64 n_cells, u64 n_cv);
void launch_batch_topology(const Launch& L, const BatchTopoArgs& T, u64 n_nodes, u64 n_chassis,
                           u64 n_racks);

// Exclusive prefix sums (scan.cu); scratch holds scan_scratch_elems(n) u64.
u64 scan_scratch_elems(u64 n);
void scan_exclusive(const Launch& L, const u32* in, u64 n, u64* out, u64* total, u64* scratch);
void scan_exclusive(const Launch& L, const u64* in, u64 n, u64* out, u64* total, u64* scratch);
// Inclusive prefix sums (out[i] includes in[i]), same scratch.
void scan_inclusive(const Launch& L, const u64* in, u64 n, u64* out, u64* total, u64* scratch);

}  // namespace ta
