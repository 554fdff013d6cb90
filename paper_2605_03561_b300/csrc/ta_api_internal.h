// ta_api_internal.h -- the objects behind the opaque handles of ta.h.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "ta.h"
#include "ta_internal.h"

struct ta_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  ta_alloc_fn alloc = nullptr;
  ta_free_fn free_fn = nullptr;
  void* user = nullptr;
  unsigned long long launches = 0;
  ta_profile prof{};
  // phase timing: event pairs recorded on the stream and read only when the
  // profile is asked for (no synchronisation on the work path)
  struct PendingPhase {
    cudaEvent_t a, b;
    double* acc;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<PendingPhase> pending;
  // a second stream for independent kernels of one call (created on first
  // use), forked from and joined back to `stream` by events
  cudaStream_t aux = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace ta {

struct Block {
  void* p;
  size_t n;
};

struct Csr {
  u64* off = nullptr;
  u32* ctx = nullptr;
  u64* time = nullptr;
  u32* cnt = nullptr;
  u64 nnz = 0;
};

// Per-call temporaries, released after the call's last synchronisation.
struct Pool {
  ta_ctx* ctx;
  std::vector<Block> items;
  ta_status get(size_t bytes, void** out, const char* what);
  template <class T>
  ta_status get_n(size_t n, T** out, const char* what) {
    return get(n * sizeof(T), (void**)out, what);
  }
  void release();
};

ta_status fail(ta_status s, const char* fmt, ...);
// The context's auxiliary stream, made to wait for the work queued so far on
// its stream; null if it could not be created (then use the stream alone).
cudaStream_t fork_aux(ta_ctx* c);
// The context's stream waits for the work queued so far on the auxiliary one.
void join_aux(ta_ctx* c);
ta_status cuda_fail(cudaError_t e, const char* what);
void* dalloc(ta_ctx* c, size_t bytes);
void dfree(ta_ctx* c, void* p, size_t bytes);
ta_status sync_check(ta_ctx* c, const char* what);
ta_status copy(ta_ctx* c, void* dst, const void* src, size_t bytes);
ta_status status_from_flags(u32 f, const char* where);

// Adds the device time of every recorded phase to its profile field and
// recycles the events (waits for the last phase to finish).
void resolve_phases(ta_ctx* c);
cudaEvent_t take_event(ta_ctx* c);

// Device time between two points on the context's stream (profiling): two
// events on the stream, resolved by resolve_phases; nothing waits here.
struct PhaseTimer {
  ta_ctx* c;
  double* acc;
  cudaEvent_t a;
  bool done = false;
  PhaseTimer(ta_ctx* c_, double* acc_) : c(c_), acc(acc_), a(take_event(c_)) {
    if (a) cudaEventRecord(a, c->stream);
  }
  ~PhaseTimer() {
    if (!done) stop();
  }
  // Records the end of the phase on the stream.
  void stop() {
    done = true;
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) {
      c->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, c->stream);
    c->pending.push_back({a, b, acc});
    if (c->pending.size() > 4096) resolve_phases(c);
  }
};

}  // namespace ta

struct ta_experiment {
  ta_ctx* ctx = nullptr;
  ta::u32 R = 0, C = 0, m = 0, max_depth = 0;
  ta::u64 N = 0, max_span = 0;
  // inputs on the device (ts/ctx released after ingestion unless borrowed)
  ta::u64* rank_off = nullptr;
  ta::u32* parent = nullptr;
  const ta::u64* ts = nullptr;
  const ta::u32* ctxv = nullptr;
  bool owns_traces = false;
  // resident products
  ta::u32* depth = nullptr;
  ta::u64* span = nullptr;
  ta::u32* n_iter = nullptr;
  ta::u64* row_off = nullptr;
  ta::u64* entry_off = nullptr;
  ta::u32* e_ctx = nullptr;
  ta::u64* e_time = nullptr;
  ta::u32* e_cnt = nullptr;
  ta::u64 rows = 0, nnz = 0;
  ta::Csr x, in;
  // iteration moments of every exclusive entry (in x's order): the sum of its
  // time over the rank's iteration rows (every row after the first) and the
  // 128-bit sum of their squares (lo, hi pairs); set for the ranks whose
  // iteration rows all hold the same contexts (x_mom[r] = 1).  Null when not
  // built or no longer matching x.
  ta::u64* x_m1 = nullptr;
  ta::u64* x_m2 = nullptr;
  uint8_t* x_mom = nullptr;
  // over all ranks (from the load): I* = min n_iter and the sum of n_iter
  bool has_iter_summary = false;
  ta::u32 istar_all = 0;
  ta::u64 sum_iter_all = 0;
  bool has_incl = false;
  // first sample of every tensor row ([rows + 1], global sample index; built
  // by the first time-window call) and that call's last result
  ta::u64* row_first = nullptr;
  ta::u64* row_ts = nullptr;  // [rows] timestamp of each row's first sample
  bool iv_valid = false;
  ta_interval_args iv_args{};
  ta::Csr iv;
  ta::u32 serve_refs = 0;  // servers holding pointers into its products
  ta::u64 device_bytes = 0;
  std::vector<ta::Block> owned;

  ta_status own(size_t bytes, void** out, const char* what);
  void disown(void* p);
  void drop();
};

namespace ta {
// Device allocation for a product (experiment-owned or a call's temporary).
using AllocFn = std::function<ta_status(size_t, void**, const char*)>;
// Offsets of every context's ancestor list (exclusive scan of depth + 1) and
// their total, when already computed.
struct AncOffsets {
  u64* off;
  u64 total;
};
// Inclusive rollup (Section II-A) of the per-rank exclusive CSR `in` of R
// ranks over e's calling context tree into `out` (arrays from `alloc`);
// device time is added to *acc.  anc: precomputed ancestor-list offsets (or
// null); status_out: receives the device status word instead of a wait.
ta_status build_inclusive(ta_experiment* e, const Csr& in, u32 R, Csr& out, const AllocFn& alloc,
                          Pool& tmp, double* acc, const AncOffsets* anc = nullptr,
                          u64** status_out = nullptr);
// The first-sample index of every tensor row (e->row_first), built once.
ta_status ensure_row_index(ta_experiment* e);
// Bitonic sort of n (key, value) pairs ascending by key, in buffers of at
// least next_pow2(n) entries (stats.cu).
void sort_u64_pairs(const Launch& L, u64* keys, double* vals, u64 n);
// I* (min n_iter, u32), the sum of n_iter and the longest span over all R
// ranks into meta[0..2] (32 bytes of device scratch).
void launch_iter_summary(const Launch& L, u32 R, const u32* n_iter, const u64* span, u64* meta);
// The experiment's CSR of a metric, or null (inclusive not built).
const Csr* csr_of_metric(const ta_experiment* e, u32 metric);
// A caller rank subset on the device (null stays null), checked sorted,
// unique and below limit; status: one device u32 of scratch.
ta_status rank_subset_to_device(ta_ctx* c, Pool& tmp, const Launch& L, const u32* src, u32 n,
                                u32 kind, u32 limit, u32* status, const u32** out);
}  // namespace ta
