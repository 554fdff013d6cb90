// api.cu -- host implementation of the C ABI declared in include/ta.h:
// contexts, device memory, ingestion orchestration, output copies and views.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ta.h"
#include "ta_api_internal.h"

using namespace ta;

namespace {
thread_local std::string g_err = "no error";
}

ta_status ta::fail(ta_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = std::string(ta_status_string(s)) + ": " + buf;
  return s;
}

ta_status ta::cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(TA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------ memory -----
void* ta::dalloc(ta_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, (void*)c->stream, c->user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void ta::dfree(ta_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (c->free_fn) c->free_fn(p, bytes, (void*)c->stream, c->user);
  else cudaFreeAsync(p, c->stream);
}

ta_status Pool::get(size_t bytes, void** out, const char* what) {
  void* p = dalloc(ctx, bytes);
  if (!p) return fail(TA_ERR_OOM, "device allocation of %zu bytes for %s failed", bytes, what);
  items.push_back({p, bytes});
  *out = p;
  return TA_OK;
}

void Pool::release() {
  for (auto& it : items) dfree(ctx, it.p, it.n);
  items.clear();
}

cudaEvent_t ta::take_event(ta_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void ta::resolve_phases(ta_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      *p.acc += ms;
    cudaGetLastError();
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
}

cudaStream_t ta::fork_aux(ta_ctx* c) {
  if (!c->aux) {
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (c->aux) cudaStreamDestroy(c->aux);
      if (c->fork_ev) cudaEventDestroy(c->fork_ev);
      c->aux = nullptr;
      c->fork_ev = c->join_ev = nullptr;
      return nullptr;
    }
  }
  cudaEventRecord(c->fork_ev, c->stream);
  cudaStreamWaitEvent(c->aux, c->fork_ev, 0);
  return c->aux;
}

void ta::join_aux(ta_ctx* c) {
  if (!c->aux) return;
  cudaEventRecord(c->join_ev, c->aux);
  cudaStreamWaitEvent(c->stream, c->join_ev, 0);
}

ta_status ta::sync_check(ta_ctx* c, const char* what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return TA_OK;
}

ta_status ta::copy(ta_ctx* c, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return TA_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  return TA_OK;
}

// Map device status bits to the first error in the documented order.
ta_status ta::status_from_flags(u32 f, const char* where) {
  if (f & F_INVALID) return fail(TA_ERR_INVALID_ARG, "%s: invalid argument", where);
  if (f & F_BAD_CCT) return fail(TA_ERR_BAD_CCT, "%s: invalid calling context tree", where);
  if (f & F_BAD_CTX) return fail(TA_ERR_BAD_CTX, "%s: context id >= n_ctx", where);
  if (f & F_NOT_SORTED) return fail(TA_ERR_NOT_SORTED, "%s: timestamps decrease within a rank", where);
  if (f & F_TIMEOUT) return fail(TA_ERR_TIMEOUT, "%s: device wait gave up", where);
  if (f & F_INTERNAL) return fail(TA_ERR_CUDA, "%s: internal staging overflow", where);
  return TA_OK;
}

// ------------------------------------------------------------ context ----
extern "C" {

const char* ta_status_string(ta_status s) {
  switch (s) {
    case TA_OK: return "TA_OK";
    case TA_ERR_INVALID_ARG: return "TA_ERR_INVALID_ARG";
    case TA_ERR_NOT_SORTED: return "TA_ERR_NOT_SORTED";
    case TA_ERR_BAD_CTX: return "TA_ERR_BAD_CTX";
    case TA_ERR_BAD_CCT: return "TA_ERR_BAD_CCT";
    case TA_ERR_OOM: return "TA_ERR_OOM";
    case TA_ERR_CAPACITY: return "TA_ERR_CAPACITY";
    case TA_ERR_TIMEOUT: return "TA_ERR_TIMEOUT";
    case TA_ERR_CUDA: return "TA_ERR_CUDA";
    case TA_ERR_STATE: return "TA_ERR_STATE";
  }
  return "TA_ERR_UNKNOWN";
}

const char* ta_last_error_message(void) { return g_err.c_str(); }

ta_status ta_create(int device, void* stream, ta_ctx** out) {
  if (!out) return fail(TA_ERR_INVALID_ARG, "ta_create: out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(TA_ERR_INVALID_ARG, "ta_create: no device %d", device);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  ta_ctx* c = new ta_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return TA_OK;
}

ta_status ta_destroy(ta_ctx* c) {
  if (!c) return TA_OK;
  cudaStreamSynchronize(c->stream);
  resolve_phases(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
    cudaEventDestroy(c->fork_ev);
    cudaEventDestroy(c->join_ev);
  }
  delete c;
  return TA_OK;
}

ta_status ta_set_allocator(ta_ctx* c, ta_alloc_fn a, ta_free_fn f, void* user) {
  if (!c) return fail(TA_ERR_INVALID_ARG, "ta_set_allocator: ctx is NULL");
  if ((a == nullptr) != (f == nullptr))
    return fail(TA_ERR_INVALID_ARG, "ta_set_allocator: give both callbacks or neither");
  c->alloc = a;
  c->free_fn = f;
  c->user = user;
  return TA_OK;
}

ta_status ta_sync(ta_ctx* c) {
  if (!c) return fail(TA_ERR_INVALID_ARG, "ta_sync: ctx is NULL");
  return sync_check(c, "ta_sync");
}

uint64_t ta_kernel_launches(const ta_ctx* c) { return c ? c->launches : 0; }

ta_status ta_get_profile(ta_ctx* c, ta_profile* out, int reset) {
  if (!c) return fail(TA_ERR_INVALID_ARG, "ta_get_profile: ctx is NULL");
  resolve_phases(c);
  if (out) *out = c->prof;
  if (reset) c->prof = ta_profile{};
  return TA_OK;
}

}  // extern "C"

// --------------------------------------------------------- experiment ----
void ta_experiment::drop() {
  for (auto& b : owned) dfree(ctx, b.p, b.n);
  owned.clear();
}

ta_status ta_experiment::own(size_t bytes, void** out, const char* what) {
  void* p = dalloc(ctx, bytes);
  if (!p) return fail(TA_ERR_OOM, "device allocation of %zu bytes for %s failed", bytes, what);
  owned.push_back({p, bytes});
  device_bytes += bytes;
  *out = p;
  return TA_OK;
}

void ta_experiment::disown(void* p) {
  for (size_t i = 0; i < owned.size(); ++i)
    if (owned[i].p == p) {
      dfree(ctx, p, owned[i].n);
      device_bytes -= owned[i].n;
      owned.erase(owned.begin() + i);
      return;
    }
}

#define TRY(x)                        \
  do {                                \
    ta_status _s = (x);               \
    if (_s != TA_OK) return _s;       \
  } while (0)

namespace {

// Longest total of ancestor lists (entries) the inclusive rollup builds;
// deeper trees use the level-by-level sweep.
constexpr u64 kAncMax = 1ull << 28;
// Per-rank scratch entries of the one-pass exclusive CSR (ranks with more
// distinct contexts take a second write pass).
constexpr u64 kXsCap = 256;

// What the tensor's write pass leaves for its finish step.
struct TensorPending {
  u64* meta;  // [0] status, [1..2] rows, entry slots, [3] distinct entries
  u64 slots;
  u32* row_nnz;
};

// Tensor, first half: count pass, scan of per-tile counts, allocation (rows
// exactly, entries one slot per run), write pass.  Nothing waits for the
// write pass: tensor_finish reads its results.
ta_status tensor_begin(ta_experiment* e, Pool& tmp, TensorPending* tp) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  const u64 N = e->N;
  const u32 R = e->R;
  TensorPlan P = plan_tensor(e->C, N, c->num_sms);
  const u64 n_tiles = std::max<u64>(1, (N + P.tile - 1) / P.tile);
  TensorArgs A;
  std::memset(&A, 0, sizeof A);
  TRY(tmp.get_n(n_tiles + 1, (u32**)&A.tfr, "tile map"));
  launch_tile_first_rank(L, e->rank_off, R, P.tile, (u32)n_tiles, (u32*)A.tfr, SetMap{});
  TRY(tmp.get_n(n_tiles, &A.tile_rows, "tile rows"));
  TRY(tmp.get_n(n_tiles, &A.tile_ents, "tile entries"));
  TRY(tmp.get_n(n_tiles, &A.tile_row_off, "tile row offsets"));
  TRY(tmp.get_n(n_tiles, &A.tile_ent_off, "tile entry offsets"));
  u64* meta;
  TRY(tmp.get(64, (void**)&meta, "tensor meta"));
  TRY(tmp.get_n(2 * scan_scratch_elems(n_tiles), &A.scan_scratch, "tile scan"));
  cudaMemsetAsync(meta, 0, 64, c->stream);
  const size_t gbm_bytes = P.bm_in_smem ? 0 : (size_t)P.write_warps() * bm_words(e->C) * 4;
  if (gbm_bytes) {
    TRY(tmp.get(gbm_bytes, (void**)&A.gbm, "tensor bitmaps"));
    cudaMemsetAsync(A.gbm, 0, gbm_bytes, c->stream);
  }
  const size_t gn = (size_t)P.write_warps() * P.gst_cap;
  TRY(tmp.get_n(gn, &A.gst_ctx, "tensor stage"));
  TRY(tmp.get_n(gn, &A.gst_cnt, "tensor stage"));
  TRY(tmp.get_n(gn, &A.gst_time, "tensor stage"));
  A.rank_off = e->rank_off;
  A.ts = e->ts;
  A.ctx = e->ctxv;
  A.R = R;
  A.C = e->C;
  A.m = e->m;
  A.n_tiles = n_tiles;
  A.N = N;
  A.status = (u32*)meta;
  A.totals = meta + 1;
  A.nnz_sum = meta + 3;
  A.gst_cap = P.gst_cap;
  A.bm_in_smem = P.bm_in_smem ? 1u : 0u;
  {
    PhaseTimer timer(c, &c->prof.tensor_count_ms);
    launch_tensor_count(L, P, A);
    launch_tile_scan(L, A);
  }
  u64 h[4];
  TRY(copy(c, h, meta, sizeof h));
  TRY(sync_check(c, "iteration tensor (count)"));
  TRY(status_from_flags((u32)h[0], "ta_load_traces"));
  e->rows = h[1];
  const u64 slots = h[2];
  TRY(e->own((u64)(R + 1) * 8, (void**)&e->row_off, "row_off_of_rank"));
  TRY(e->own((e->rows + 1) * 8, (void**)&e->entry_off, "entry_off"));
  TRY(e->own(std::max<u64>(slots, 1) * 4, (void**)&e->e_ctx, "e_ctx"));
  TRY(e->own(std::max<u64>(slots, 1) * 8, (void**)&e->e_time, "e_time"));
  TRY(e->own(std::max<u64>(slots, 1) * 4, (void**)&e->e_cnt, "e_cnt"));
  TRY(tmp.get_n(std::max<u64>(e->rows, 1), &A.row_nnz, "row entries"));
  TRY(copy(c, e->row_off + R, &e->rows, 8));
  A.row_off_of_rank = e->row_off;
  A.entry_off = e->entry_off;
  A.e_ctx = e->e_ctx;
  A.e_time = e->e_time;
  A.e_cnt = e->e_cnt;
  {
    PhaseTimer timer(c, &c->prof.tensor_ms);
    launch_tensor_write(L, P, A);
  }
  tp->meta = meta;
  tp->slots = slots;
  tp->row_nnz = A.row_nnz;
  return TA_OK;
}

// Tensor, second half (h = the write pass's meta, read back): status, the
// distinct entry count, and the compaction when some row repeats a context.
ta_status tensor_finish(ta_experiment* e, Pool& tmp, const TensorPending& tp, const u64* h) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  TRY(status_from_flags((u32)h[0], "ta_load_traces"));
  e->nnz = h[3];
  const u64 slots = tp.slots;
  if (e->nnz > slots) return fail(TA_ERR_STATE, "iteration tensor: %llu entries in %llu slots",
                                  (unsigned long long)e->nnz, (unsigned long long)slots);
  if (e->nnz == slots) {  // every row's contexts are distinct across its runs
    TRY(copy(c, e->entry_off + e->rows, &e->nnz, 8));
  } else {
    TensorCompact K{};
    K.rows = e->rows;
    K.slot_off = e->entry_off;
    K.row_nnz = tp.row_nnz;
    K.ctx_in = e->e_ctx;
    K.time_in = e->e_time;
    K.cnt_in = e->e_cnt;
    u64* off;
    u32 *cx, *cn;
    u64* tm;
    TRY(e->own((e->rows + 1) * 8, (void**)&off, "entry_off"));
    TRY(e->own(std::max<u64>(e->nnz, 1) * 4, (void**)&cx, "e_ctx"));
    TRY(e->own(std::max<u64>(e->nnz, 1) * 8, (void**)&tm, "e_time"));
    TRY(e->own(std::max<u64>(e->nnz, 1) * 4, (void**)&cn, "e_cnt"));
    TRY(tmp.get_n(scan_scratch_elems(std::max<u64>(e->rows, 1)), &K.scan_scratch, "row scan"));
    K.new_off = off;
    K.ctx_out = cx;
    K.time_out = tm;
    K.cnt_out = cn;
    {
      PhaseTimer timer(c, &c->prof.tensor_ms);
      launch_tensor_compact(L, K);
    }
    TRY(sync_check(c, "iteration tensor (compaction)"));
    e->disown(e->entry_off);
    e->disown(e->e_ctx);
    e->disown(e->e_time);
    e->disown(e->e_cnt);
    e->entry_off = off;
    e->e_ctx = cx;
    e->e_time = tm;
    e->e_cnt = cn;
  }
  c->prof.tensor_launches += 1;
  c->prof.tensor_records += e->N;
  c->prof.tensor_entries += e->nnz;
  c->prof.tensor_rows += e->rows;
  return TA_OK;
}

// What the exclusive scratch pass leaves for its finish step.
struct ExclPending {
  RankCsrArgs A;
  RankCsrPlan P;
  u64* meta;  // [0] status, [1] total entries, [2] ranks above the scratch cap
};

// Exclusive per-rank CSR in one pass over the tensor's rows, first half: the
// write pass into a per-rank scratch with exact counts, and their scan.
// Nothing waits for it: excl_finish reads the meta.
ta_status excl_begin(ta_experiment* e, Pool& tmp, ExclPending* xq) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  const u32 R = e->R;
  RankCsrPlan P = plan_rank_csr(R, e->C, c->num_sms);
  RankCsrArgs A;
  std::memset(&A, 0, sizeof A);
  u64* meta;
  TRY(tmp.get(64, (void**)&meta, "csr meta"));
  cudaMemsetAsync(meta, 0, 64, c->stream);
  const size_t gbm_bytes = P.bm_in_smem ? 0 : (size_t)P.warps() * bm_words(e->C) * 4;
  if (gbm_bytes) {
    TRY(tmp.get(gbm_bytes, (void**)&A.gbm, "csr bitmaps"));
    cudaMemsetAsync(A.gbm, 0, gbm_bytes, c->stream);
  }
  const size_t gn = (size_t)P.warps() * P.gst_cap;
  TRY(tmp.get_n(gn, &A.gst_ctx, "csr stage"));
  TRY(tmp.get_n(gn, &A.gst_cnt, "csr stage"));
  TRY(tmp.get_n(gn, &A.gst_time, "csr stage"));
  TRY(tmp.get_n((u64)R, &A.out_cnt, "csr counts"));
  TRY(tmp.get_n(scan_scratch_elems(R), &A.scan_scratch, "csr scan"));
  Csr& out = e->x;
  TRY(e->own(((u64)R + 1) * 8, (void**)&out.off, "csr off"));
  A.mode = 0;
  A.R = R;
  A.C = e->C;
  A.max_depth = e->max_depth;
  A.row_off_of_rank = e->row_off;
  A.entry_off = e->entry_off;
  A.in_ctx = e->e_ctx;
  A.in_time = e->e_time;
  A.in_cnt = e->e_cnt;
  A.parent = e->parent;
  A.depth = e->depth;
  A.out_off = out.off;
  A.total = meta + 1;
  A.status = (u32*)meta;
  A.gst_cap = P.gst_cap;
  A.bm_in_smem = P.bm_in_smem ? 1u : 0u;
  const u64 cap = kXsCap;
  TRY(tmp.get_n((u64)R * cap, &A.xs_ctx, "exclusive scratch"));
  TRY(tmp.get_n((u64)R * cap, &A.xs_time, "exclusive scratch"));
  TRY(tmp.get_n((u64)R * cap, &A.xs_cnt, "exclusive scratch"));
  A.xs_cap = (u32)cap;
  A.n_over = (unsigned long long*)(meta + 2);
  // iteration moments beside the entries (the speedup's within-rank terms
  // read them instead of the rows)
  TRY(tmp.get_n((u64)R * cap, &A.xs_m1, "exclusive scratch"));
  TRY(tmp.get_n((u64)R * cap * 2, &A.xs_m2, "exclusive scratch"));
  TRY(e->own(std::max<u32>(R, 1), (void**)&e->x_mom, "iteration moments"));
  A.mom_ok = e->x_mom;
  {
    PhaseTimer timer(c, &c->prof.exclusive_ms);
    launch_excl_scratch(L, P, A);
  }
  xq->A = A;
  xq->P = P;
  xq->meta = meta;
  return TA_OK;
}

// Second half (h = the scratch pass's meta, read back): exact allocation, the
// copy of the scratch rows, the pass over ranks above the cap.  Its status
// word (meta[0]) is left for the caller to read at its next synchronisation.
ta_status excl_finish(ta_experiment* e, ExclPending& xq, const u64* h) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  TRY(status_from_flags((u32)h[0], "exclusive"));
  Csr& out = e->x;
  RankCsrArgs& A = xq.A;
  out.nnz = h[1];
  const u64 n = std::max<u64>(out.nnz, 1);
  TRY(e->own(n * 4, (void**)&out.ctx, "csr ctx"));
  TRY(e->own(n * 8, (void**)&out.time, "csr time"));
  TRY(e->own(n * 4, (void**)&out.cnt, "csr cnt"));
  A.out_ctx = out.ctx;
  A.out_time = out.time;
  A.out_cnt_e = out.cnt;
  TRY(e->own(n * 8, (void**)&e->x_m1, "iteration moments"));
  TRY(e->own(n * 16, (void**)&e->x_m2, "iteration moments"));
  A.out_m1 = e->x_m1;
  A.out_m2 = e->x_m2;
  PhaseTimer timer(c, &c->prof.exclusive_ms);
  launch_excl_copy(L, A);
  if (h[2]) {
    A.only_over = 1;
    launch_rank_write(L, xq.P, A);
  }
  return TA_OK;
}

}  // namespace

// Inclusive rollup of a per-rank exclusive CSR over the experiment's tree:
// ancestor lists (unless too long: level-by-level sweep), count, scan,
// exact allocation through `alloc`, write.  `anc` may carry the list offsets
// and their total already computed (the load computes them beside the tree
// checks); with `status_out` set, the final status word is left there for the
// caller to read at its next synchronisation instead of being waited for.
ta_status ta::build_inclusive(ta_experiment* e, const Csr& in, u32 R, Csr& out,
                              const AllocFn& alloc, Pool& tmp, double* acc, const AncOffsets* anc,
                              u64** status_out) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  RankCsrPlan P = plan_rank_csr(R, e->C, c->num_sms);
  RankCsrArgs A;
  std::memset(&A, 0, sizeof A);
  u64* meta;
  TRY(tmp.get(64, (void**)&meta, "csr meta"));
  cudaMemsetAsync(meta, 0, 64, c->stream);
  const size_t gbm_bytes = P.bm_in_smem ? 0 : (size_t)P.warps() * bm_words(e->C) * 4;
  if (gbm_bytes) {
    TRY(tmp.get(gbm_bytes, (void**)&A.gbm, "csr bitmaps"));
    cudaMemsetAsync(A.gbm, 0, gbm_bytes, c->stream);
  }
  const size_t gn = (size_t)P.warps() * P.gst_cap;
  TRY(tmp.get_n(gn, &A.gst_ctx, "csr stage"));
  TRY(tmp.get_n(gn, &A.gst_cnt, "csr stage"));
  TRY(tmp.get_n(gn, &A.gst_time, "csr stage"));
  TRY(tmp.get_n(gn, &A.gst_dep, "csr stage"));
  TRY(tmp.get_n(gn, &A.gst_par, "csr stage"));
  TRY(tmp.get_n(std::max<u64>(R, 1), &A.out_cnt, "csr counts"));
  TRY(tmp.get_n(scan_scratch_elems(R), &A.scan_scratch, "csr scan"));
  TRY(alloc(((u64)R + 1) * 8, (void**)&out.off, "csr off"));
  A.mode = 1;
  A.R = R;
  A.C = e->C;
  A.max_depth = e->max_depth;
  A.in_off = in.off;
  A.in_ctx = in.ctx;
  A.in_time = in.time;
  A.in_cnt = in.cnt;
  A.parent = e->parent;
  A.depth = e->depth;
  A.out_off = out.off;
  A.total = meta + 1;
  A.status = (u32*)meta;
  A.gst_cap = P.gst_cap;
  A.bm_in_smem = P.bm_in_smem ? 1u : 0u;
  {  // ancestor lists of the tree, unless they would be too long
    PhaseTimer timer(c, acc);
    AncOffsets own{};
    if (!anc) {
      u32* len;
      u64* ascr;
      TRY(tmp.get_n(std::max<u32>(e->C, 1), &len, "ancestor lengths"));
      TRY(tmp.get_n((u64)e->C + 1, &own.off, "ancestor offsets"));
      TRY(tmp.get_n(scan_scratch_elems(e->C), &ascr, "ancestor scan"));
      launch_anc_offsets(L, e->depth, e->C, len, own.off, meta + 2, ascr);
      TRY(copy(c, &own.total, meta + 2, 8));
      TRY(sync_check(c, "inclusive (ancestors)"));
      anc = &own;
    }
    if (anc->total <= kAncMax) {
      u32* lists;
      TRY(tmp.get_n(std::max<u64>(anc->total, 1), &lists, "ancestor lists"));
      launch_anc_fill(L, e->parent, e->C, anc->off, lists, SetMap{});
      A.anc_off = anc->off;
      A.anc = lists;
    }
  }
  {
    PhaseTimer timer(c, acc);
    launch_rank_count(L, P, A);
  }
  u64 h[2];
  TRY(copy(c, h, meta, sizeof h));
  TRY(sync_check(c, "inclusive (count)"));
  out.nnz = h[1];
  const u64 n = std::max<u64>(out.nnz, 1);
  TRY(alloc(n * 4, (void**)&out.ctx, "csr ctx"));
  TRY(alloc(n * 8, (void**)&out.time, "csr time"));
  TRY(alloc(n * 4, (void**)&out.cnt, "csr cnt"));
  A.out_ctx = out.ctx;
  A.out_time = out.time;
  A.out_cnt_e = out.cnt;
  {
    PhaseTimer timer(c, acc);
    launch_rank_write(L, P, A);
  }
  if (status_out) {
    *status_out = meta;
    return TA_OK;
  }
  u64 f = 0;
  TRY(copy(c, &f, meta, 8));
  TRY(sync_check(c, "inclusive"));
  return status_from_flags((u32)f, "inclusive");
}

namespace {

ta_status load_impl(ta_ctx* c, const ta_trace_desc* d, ta_experiment* e, Pool& tmp) {
  Launch L{c->stream, c->num_sms, &c->launches};
  const u32 R = d->n_ranks, C = d->n_ctx;
  const u64 N = d->n_records;
  const bool dev = d->mem_kind == TA_MEM_DEVICE;
  TRY(e->own(((u64)R + 1) * 8, (void**)&e->rank_off, "rank_off"));
  TRY(copy(c, e->rank_off, d->rank_off, ((u64)R + 1) * 8));
  TRY(e->own((u64)C * 4, (void**)&e->parent, "parent"));
  TRY(copy(c, e->parent, d->parent, (u64)C * 4));
  // the sample passes read ts and ctx in 16-byte vectors: borrow only aligned arrays
  const bool aligned = ((uintptr_t)d->ts % 16 == 0) && ((uintptr_t)d->ctx % 16 == 0);
  if (dev && (d->flags & TA_LOAD_BORROW) && aligned) {
    e->ts = d->ts;
    e->ctxv = d->ctx;
  } else {
    u64* ts;
    u32* cx;
    TRY(e->own(N * 8, (void**)&ts, "ts"));
    TRY(e->own(N * 4, (void**)&cx, "ctx"));
    TRY(copy(c, ts, d->ts, N * 8));
    TRY(copy(c, cx, d->ctx, N * 4));
    e->ts = ts;
    e->ctxv = cx;
    e->owns_traces = true;
  }
  TRY(e->own((u64)R * 8, (void**)&e->span, "span"));
  TRY(e->own((u64)C * 4, (void**)&e->depth, "depth"));
  TRY(e->own((u64)R * 4 + 4, (void**)&e->n_iter, "n_iter"));
  u64* meta;  // [0] status|pad, [1] max_span, [2] roots|max_depth, [3] ancestor-list total
  TRY(tmp.get(64, (void**)&meta, "load meta"));
  u32* scratch;
  TRY(tmp.get((u64)C * 16, (void**)&scratch, "tree scratch"));
  cudaMemsetAsync(meta, 0, 64, c->stream);
  u32* status = (u32*)meta;
  const bool incl = !(d->flags & TA_LOAD_NO_INCLUSIVE);
  AncOffsets anc{};
  {
    PhaseTimer timer(c, &c->prof.validate_ms);
    launch_rank_off(L, e->rank_off, R, N, e->ts, e->span, meta + 1, status, SetMap{});
    launch_cct(L, e->parent, C, e->depth, (u32*)(meta + 2) + 1, (u32*)(meta + 2), scratch, status,
               SetMap{});
    if (incl) {  // the inclusive rollup's ancestor-list offsets, read back with the checks
      u32* len;
      u64* ascr;
      TRY(tmp.get_n(std::max<u32>(C, 1), &len, "ancestor lengths"));
      TRY(tmp.get_n((u64)C + 1, &anc.off, "ancestor offsets"));
      TRY(tmp.get_n(scan_scratch_elems(C), &ascr, "ancestor scan"));
      launch_anc_offsets(L, e->depth, C, len, anc.off, meta + 3, ascr);
    }
  }
  u64 h[4];
  TRY(copy(c, h, meta, sizeof h));
  TRY(sync_check(c, "validation"));
  const u32 f = (u32)h[0];
  if (f & F_INVALID) return fail(TA_ERR_INVALID_ARG, "rank offsets are not a valid CSR of n_records samples "
                                                     "(rank_off[0] = 0, non-decreasing, rank_off[R] = N, < 2^32 per rank)");
  const u32 roots = (u32)h[2], maxd = (u32)(h[2] >> 32);
  if ((f & F_BAD_CCT) || roots != 1)
    return fail(TA_ERR_BAD_CCT, "parent array: %u roots, parents in range: %s, acyclic: %s", roots,
                (f & F_BAD_CCT) ? "no or cycle" : "yes", (f & F_BAD_CCT) ? "?" : "yes");
  if ((unsigned __int128)h[1] * R >= ((unsigned __int128)1 << 63))
    return fail(TA_ERR_INVALID_ARG, "R * longest rank span = %u * %llu >= 2^63 (exact moments)", R,
                (unsigned long long)h[1]);
  e->max_depth = maxd;
  e->max_span = h[1];
  anc.total = h[3];
  TensorPending tq;
  ExclPending xq;
  TRY(tensor_begin(e, tmp, &tq));
  u64 ht[8];
  TRY(copy(c, ht, tq.meta, 4 * 8));
  TRY(sync_check(c, "iteration tensor (write)"));
  TRY(tensor_finish(e, tmp, tq, ht));
  launch_n_iter(L, e->row_off, R, e->n_iter);
  u64* isum;  // I*, sum n_iter, max span over all ranks, read at the final wait
  TRY(tmp.get_n(4, &isum, "iteration summary"));
  launch_iter_summary(L, R, e->n_iter, e->span, isum);
  TRY(excl_begin(e, tmp, &xq));  // from the finished tensor's rows
  TRY(copy(c, ht + 4, xq.meta, 3 * 8));
  TRY(sync_check(c, "exclusive (scratch)"));
  TRY(excl_finish(e, xq, ht + 4));
  u64* incl_status = nullptr;
  if (incl) {
    const AllocFn own = [e](size_t n, void** p, const char* w) { return e->own(n, p, w); };
    TRY(build_inclusive(e, e->x, R, e->in, own, tmp, &c->prof.inclusive_ms, &anc, &incl_status));
    e->has_incl = true;
  }
  // the status words left by the last passes, read at the one final wait
  u64 fin[2] = {0, 0}, hi[3] = {0, 0, 0};
  TRY(copy(c, &fin[0], xq.meta, 8));
  if (incl_status) TRY(copy(c, &fin[1], incl_status, 8));
  TRY(copy(c, hi, isum, sizeof hi));
  TRY(sync_check(c, "ta_load_traces"));
  TRY(status_from_flags((u32)fin[0], "exclusive"));
  TRY(status_from_flags((u32)fin[1], "inclusive"));
  e->istar_all = (u32)hi[0];
  e->sum_iter_all = hi[1];
  e->has_iter_summary = true;
  // raw traces are not needed after ingestion unless kept for time windows
  if (e->owns_traces && !(d->flags & TA_LOAD_KEEP_TRACES)) {
    e->disown((void*)e->ts);
    e->disown((void*)e->ctxv);
    e->ts = nullptr;
    e->ctxv = nullptr;
  }
  return TA_OK;
}

}  // namespace

extern "C" {

ta_status ta_load_traces(ta_ctx* c, const ta_trace_desc* d, ta_experiment** out) {
  if (!c || !d || !out) return fail(TA_ERR_INVALID_ARG, "ta_load_traces: NULL argument");
  *out = nullptr;
  if (d->n_ranks == 0) return fail(TA_ERR_INVALID_ARG, "n_ranks = 0");
  if (d->n_ranks == 0xFFFFFFFFu) return fail(TA_ERR_INVALID_ARG, "n_ranks too large");
  if (d->n_ctx == 0) return fail(TA_ERR_INVALID_ARG, "n_ctx = 0");
  if (d->marker_ctx >= d->n_ctx) return fail(TA_ERR_INVALID_ARG, "marker_ctx >= n_ctx");
  if (d->mem_kind != TA_MEM_HOST && d->mem_kind != TA_MEM_DEVICE)
    return fail(TA_ERR_INVALID_ARG, "mem_kind");
  if (!d->rank_off || !d->parent) return fail(TA_ERR_INVALID_ARG, "rank_off / parent NULL");
  if (d->n_records > 0 && (!d->ts || !d->ctx)) return fail(TA_ERR_INVALID_ARG, "ts / ctx NULL");
  if (d->n_ctx > 0x7FFFFFFFu) return fail(TA_ERR_INVALID_ARG, "n_ctx too large");
  cudaSetDevice(c->device);
  ta_experiment* e = new ta_experiment();
  e->ctx = c;
  e->R = d->n_ranks;
  e->C = d->n_ctx;
  e->m = d->marker_ctx;
  e->N = d->n_records;
  Pool tmp{c, {}};
  ta_status s = load_impl(c, d, e, tmp);
  cudaStreamSynchronize(c->stream);
  tmp.release();
  if (s != TA_OK) {
    std::string keep = g_err;
    e->drop();
    cudaStreamSynchronize(c->stream);
    delete e;
    g_err = keep;
    return s;
  }
  *out = e;
  return TA_OK;
}

ta_status ta_experiment_free(ta_experiment* e) {
  if (!e) return TA_OK;
  cudaStreamSynchronize(e->ctx->stream);
  e->drop();
  cudaStreamSynchronize(e->ctx->stream);
  delete e;
  return TA_OK;
}

ta_status ta_experiment_get_info(const ta_experiment* e, ta_experiment_info* i) {
  if (!e || !i) return fail(TA_ERR_INVALID_ARG, "ta_experiment_get_info: NULL argument");
  i->n_ranks = e->R;
  i->n_ctx = e->C;
  i->marker_ctx = e->m;
  i->max_depth = e->max_depth;
  i->n_records = e->N;
  i->n_rows = e->rows;
  i->tensor_nnz = e->nnz;
  i->excl_nnz = e->x.nnz;
  i->incl_nnz = e->has_incl ? e->in.nnz : 0;
  i->device_bytes = e->device_bytes;
  return TA_OK;
}

ta_status ta_iteration_tensor(ta_experiment* e, ta_tensor_out* o) {
  if (!e || !o) return fail(TA_ERR_INVALID_ARG, "ta_iteration_tensor: NULL argument");
  ta_ctx* c = e->ctx;
  o->rows = e->rows;
  o->nnz = e->nnz;
  if (o->entry_off && o->rows_cap < e->rows + 1)
    return fail(TA_ERR_CAPACITY, "entry_off needs %llu elements", (unsigned long long)e->rows + 1);
  if ((o->e_ctx || o->e_time || o->e_cnt) && o->nnz_cap < e->nnz)
    return fail(TA_ERR_CAPACITY, "entries need %llu elements", (unsigned long long)e->nnz);
  if (o->n_iter) TRY(copy(c, o->n_iter, e->n_iter, (u64)e->R * 4));
  if (o->row_off_of_rank) TRY(copy(c, o->row_off_of_rank, e->row_off, ((u64)e->R + 1) * 8));
  if (o->entry_off) TRY(copy(c, o->entry_off, e->entry_off, (e->rows + 1) * 8));
  if (o->e_ctx) TRY(copy(c, o->e_ctx, e->e_ctx, e->nnz * 4));
  if (o->e_time) TRY(copy(c, o->e_time, e->e_time, e->nnz * 8));
  if (o->e_cnt) TRY(copy(c, o->e_cnt, e->e_cnt, e->nnz * 4));
  return sync_check(c, "ta_iteration_tensor");
}

static ta_status csr_out(ta_experiment* e, const Csr& s, ta_csr_out* o, const char* what) {
  ta_ctx* c = e->ctx;
  o->nnz = s.nnz;
  if ((o->ctx || o->time || o->cnt) && o->nnz_cap < s.nnz)
    return fail(TA_ERR_CAPACITY, "%s needs %llu entries", what, (unsigned long long)s.nnz);
  if (o->off) TRY(copy(c, o->off, s.off, ((u64)e->R + 1) * 8));
  if (o->ctx) TRY(copy(c, o->ctx, s.ctx, s.nnz * 4));
  if (o->time) TRY(copy(c, o->time, s.time, s.nnz * 8));
  if (o->cnt) TRY(copy(c, o->cnt, s.cnt, s.nnz * 4));
  return sync_check(c, what);
}

ta_status ta_exclusive(ta_experiment* e, ta_csr_out* o) {
  if (!e || !o) return fail(TA_ERR_INVALID_ARG, "ta_exclusive: NULL argument");
  return csr_out(e, e->x, o, "ta_exclusive");
}

ta_status ta_inclusive_rollup(ta_experiment* e, ta_csr_out* o) {
  if (!e || !o) return fail(TA_ERR_INVALID_ARG, "ta_inclusive_rollup: NULL argument");
  if (!e->has_incl) return fail(TA_ERR_STATE, "inclusive rollup was skipped at load");
  return csr_out(e, e->in, o, "ta_inclusive_rollup");
}

ta_status ta_tensor_get_view(const ta_experiment* e, ta_tensor_view* v) {
  if (!e || !v) return fail(TA_ERR_INVALID_ARG, "ta_tensor_get_view: NULL argument");
  v->n_iter = e->n_iter;
  v->row_off_of_rank = e->row_off;
  v->entry_off = e->entry_off;
  v->e_ctx = e->e_ctx;
  v->e_time = e->e_time;
  v->e_cnt = e->e_cnt;
  v->span = e->span;
  v->rows = e->rows;
  v->nnz = e->nnz;
  return TA_OK;
}

ta_status ta_csr_get_view(const ta_experiment* e, uint32_t metric, ta_csr_view* v) {
  if (!e || !v) return fail(TA_ERR_INVALID_ARG, "ta_csr_get_view: NULL argument");
  if (metric > 1) return fail(TA_ERR_INVALID_ARG, "metric");
  if (metric == 1 && !e->has_incl) return fail(TA_ERR_STATE, "inclusive rollup was skipped at load");
  const Csr& s = metric == 0 ? e->x : e->in;
  v->off = s.off;
  v->ctx = s.ctx;
  v->time = s.time;
  v->cnt = s.cnt;
  v->nnz = s.nnz;
  return TA_OK;
}

}  // extern "C"
