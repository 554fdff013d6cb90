// prune.cu -- pruning of the calling context tree on the summary profile
// (Section III-A, "Pruning Large Calling Context Trees": a strategy evaluated
// once on the summary profile, the aggregate of all parallel profiles, then
// propagated to every parallel profile; Section VI-B's 1 % rule and class
// drops).  Three steps: the summary inclusive time of every context over all
// ranks, the kept set by an exact threshold against the root's, and every
// rank's exclusive and inclusive CSR compacted in place to the kept contexts.
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

inline unsigned nblocks(u64 n, int nt = 256) {
  return (unsigned)std::max<u64>(1, std::min<u64>((n + nt - 1) / nt, 1u << 20));
}

// Summary profile: each inclusive entry adds its time to its context.  The
// sums are exact in 64 bits: loading guarantees R x longest span < 2^63.
__global__ void k_prune_summary(const u32* __restrict__ ctx, const u64* __restrict__ time, u64 nnz,
                                unsigned long long* summary) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += G)
    atomicAdd(&summary[ctx[j]], (unsigned long long)time[j]);
}

// The root: the one context without a parent (loading checked there is one).
__global__ void k_prune_root(const u32* __restrict__ parent, u32 C, u32* root) {
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C && parent[c] == NONE32) *root = c;
}

// Kept iff summary[c] * den >= total * num (128-bit products) and not dropped.
__global__ void k_prune_keep(const u64* __restrict__ summary, u32 C, u32 num, u32 den,
                             const uint8_t* __restrict__ drop, const u32* __restrict__ root,
                             uint8_t* kept, u32* n_kept) {
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const u64 total = summary[*root];
  const bool k = (u128)summary[c] * den >= (u128)total * num && !(drop && drop[c]);
  kept[c] = k ? 1 : 0;
  if (k) atomicAdd(n_kept, 1u);
}

// Kept entries of every rank (warp per rank).
__global__ void k_prune_count(const u64* __restrict__ off, const u32* __restrict__ ctx, u32 R,
                              const uint8_t* __restrict__ kept, u32* cnt) {
  const int lane = threadIdx.x & 31;
  const u64 G = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 r = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += G) {
    u32 n = 0;
    for (u64 j = off[r] + lane; j < off[r + 1]; j += 32) n += kept[ctx[j]];
    n = __reduce_add_sync(FULL, n);
    if (lane == 0) cnt[r] = n;
  }
}

// The kept entries of every rank, in order, at their new offsets.
__global__ void k_prune_write(const u64* __restrict__ off, const u32* __restrict__ ctx,
                              const u64* __restrict__ time, const u32* __restrict__ ecnt, u32 R,
                              const uint8_t* __restrict__ kept, const u64* __restrict__ new_off,
                              u32* octx, u64* otime, u32* ocnt) {
  const int lane = threadIdx.x & 31;
  const u32 below = (1u << lane) - 1u;
  const u64 G = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 r = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += G) {
    const u64 e = off[r + 1];
    u64 base = new_off[r];
    for (u64 j0 = off[r]; j0 < e; j0 += 32) {
      const u64 j = j0 + lane;
      const bool k = j < e && kept[ctx[j]];
      const u32 bal = __ballot_sync(FULL, k);
      if (k) {
        const u64 q = base + __popc(bal & below);
        octx[q] = ctx[j];
        otime[q] = time[j];
        ocnt[q] = ecnt[j];
      }
      base += __popc(bal);
    }
  }
}

}  // namespace
}  // namespace ta

using namespace ta;

extern "C" ta_status ta_prune_profiles(ta_experiment* e, const ta_prune_args* a, ta_prune_out* o) {
  if (!e || !a || !o) return fail(TA_ERR_INVALID_ARG, "ta_prune_profiles: NULL argument");
  if (a->keep_den == 0) return fail(TA_ERR_INVALID_ARG, "ta_prune_profiles: keep_den is 0");
  if (a->mem_kind > 1) return fail(TA_ERR_INVALID_ARG, "ta_prune_profiles: mem_kind");
  if (!e->has_incl)
    return fail(TA_ERR_STATE, "ta_prune_profiles: the experiment has no inclusive CSR");
  if (e->serve_refs)
    return fail(TA_ERR_STATE, "ta_prune_profiles: the experiment is registered with a server");
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
  const u32 C = e->C, R = e->R;
  const bool dev = a->mem_kind == TA_MEM_DEVICE;
  u64* summary;
  uint8_t* kept;
  u32* meta;  // [0] root, [1] kept contexts
  TRY(tmp.get_n(std::max<u32>(C, 1), &summary, "summary profile"));
  TRY(tmp.get_n(std::max<u32>(C, 1), &kept, "kept contexts"));
  TRY(tmp.get_n(2, &meta, "prune meta"));
  const uint8_t* drop = a->drop;
  if (drop && !dev) {
    uint8_t* d;
    TRY(tmp.get_n(std::max<u32>(C, 1), &d, "drop flags"));
    TRY(copy(c, d, a->drop, C));
    drop = d;
  }
  cudaMemsetAsync(summary, 0, (size_t)C * 8, c->stream);
  cudaMemsetAsync(meta, 0, 8, c->stream);
  k_prune_summary<<<nblocks(e->in.nnz), 256, 0, c->stream>>>(e->in.ctx, e->in.time, e->in.nnz,
                                                              (unsigned long long*)summary);
  k_prune_root<<<nblocks(C), 256, 0, c->stream>>>(e->parent, C, meta);
  k_prune_keep<<<nblocks(C), 256, 0, c->stream>>>(summary, C, a->keep_num, a->keep_den, drop, meta,
                                                  kept, meta + 1);
  L.count(3);
  const u64 warps = std::min<u64>(std::max<u64>(R, 1), (u64)c->num_sms * 64);
  const unsigned wblocks = (unsigned)((warps + 7) / 8);
  u32* cnt;
  u64* scan_scratch;
  TRY(tmp.get_n(std::max<u32>(R, 1), &cnt, "kept entries per rank"));
  TRY(tmp.get_n(scan_scratch_elems(R), &scan_scratch, "prune scan"));
  for (Csr* m : {&e->x, &e->in}) {
    u64* off;
    TRY(e->own(((u64)R + 1) * 8, (void**)&off, "csr off"));
    k_prune_count<<<wblocks, 256, 0, c->stream>>>(m->off, m->ctx, R, kept, cnt);
    L.count();
    scan_exclusive(L, cnt, R, off, off + R, scan_scratch);
    u64 nnz = 0;
    TRY(copy(c, &nnz, off + R, 8));
    TRY(sync_check(c, "ta_prune_profiles (count)"));
    u32 *cx, *cn;
    u64* tm;
    TRY(e->own(std::max<u64>(nnz, 1) * 4, (void**)&cx, "csr ctx"));
    TRY(e->own(std::max<u64>(nnz, 1) * 8, (void**)&tm, "csr time"));
    TRY(e->own(std::max<u64>(nnz, 1) * 4, (void**)&cn, "csr cnt"));
    k_prune_write<<<wblocks, 256, 0, c->stream>>>(m->off, m->ctx, m->time, m->cnt, R, kept, off, cx,
                                                   tm, cn);
    L.count();
    TRY(sync_check(c, "ta_prune_profiles (write)"));
    e->disown(m->off);
    e->disown(m->ctx);
    e->disown(m->time);
    e->disown(m->cnt);
    m->off = off;
    m->ctx = cx;
    m->time = tm;
    m->cnt = cn;
    m->nnz = nnz;
  }
  // the iteration moments follow the unpruned exclusive entries: dropped
  for (void* p : {(void*)e->x_m1, (void*)e->x_m2, (void*)e->x_mom})
    if (p) e->disown(p);
  e->x_m1 = e->x_m2 = nullptr;
  e->x_mom = nullptr;
  u32 h[2];
  TRY(copy(c, h, meta, 8));
  if (o->kept) TRY(copy(c, o->kept, kept, C));
  if (o->summary) TRY(copy(c, o->summary, summary, (size_t)C * 8));
  TRY(sync_check(c, "ta_prune_profiles"));
  o->n_kept = h[1];
  o->excl_nnz = e->x.nnz;
  o->incl_nnz = e->in.nnz;
  return TA_OK;
}
