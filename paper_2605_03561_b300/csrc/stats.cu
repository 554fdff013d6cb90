// stats.cu -- cross-rank statistics, outliers, topology rollup and the
// potential-speedup estimate (Sections VI-A and VI-B; Tables IV and V).
//
// Integer partials (present, min, max, sum, 128-bit sum of squares) are exact
// and order-independent; the FP64 values are computed from them once, by the
// same fixed sequence of correctly rounded operations for every context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
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

__device__ __forceinline__ u32 rank_at(const u32* S, u32 i) { return S ? S[i] : i; }

// sorted, unique, < limit
__global__ void k_check_sorted(const u32* __restrict__ v, u32 n, u32 limit, u32* status) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (v[i] >= limit || (i > 0 && v[i] <= v[i - 1])) flag(status, F_INVALID);
}

// slot_of_ctx[ctxs[i]] = i (ctxs NULL: identity over C).
__global__ void k_slot_map(const u32* __restrict__ ctxs, u32 n, u32 C, u32* slot_of_ctx) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (ctxs) {
    if (i < n && ctxs[i] < C) slot_of_ctx[ctxs[i]] = i;
  } else if (i < C) {
    slot_of_ctx[i] = i;
  }
}

__global__ void k_fill_u64(u64* p, u64 n, u64 v) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

struct Partials {
  u32* present;
  u64* mn;
  u64* mx;
  u64* s1;
  u64* s2lo;
  u64* s2hi;
  u32* argmax;
  double* sd;
  u64* Mlo;
  u64* Mhi;
};

// Per-CTA hash table of context slots in shared memory, flushed to the
// global partials once per CTA (low contention on popular contexts).
constexpr int HCAP = 1024;
constexpr int STATS_NT = 256;

__global__ void __launch_bounds__(STATS_NT)
    k_stats_partial(const u32* __restrict__ S, u32 n, const u64* __restrict__ off,
                    const u32* __restrict__ ctx, const u64* __restrict__ time,
                    const u32* __restrict__ slot_of_ctx, Partials P, SetMap sets) {
  __shared__ u32 hkey[HCAP];
  __shared__ u32 hpres[HCAP];
  __shared__ unsigned long long hmn[HCAP], hmx[HCAP], hs1[HCAP], hs2lo[HCAP], hs2hi[HCAP];
  for (int h = threadIdx.x; h < HCAP; h += STATS_NT) {
    hkey[h] = NONE32;
    hpres[h] = 0;
    hmn[h] = ~0ull;
    hmx[h] = 0;
    hs1[h] = 0;
    hs2lo[h] = 0;
    hs2hi[h] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const u32 gw = (blockIdx.x * STATS_NT + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * STATS_NT) >> 5;
  for (u32 i = gw; i < n; i += nw) {
    const u32 r = rank_at(S, i);
    const u32 cbase = sets.S ? sets.set_ctx0[sets.rank_set[r]] : 0u;
    const u64 E0 = off[r], E1 = off[r + 1];
    for (u64 j = E0 + lane; j < E1; j += 32) {
      const u32 slot = sets.S ? cbase + ctx[j] : slot_of_ctx[ctx[j]];
      if (slot == NONE32) continue;
      const u64 x = time[j];
      const u128 x2 = (u128)x * x;
      u32 h = (slot * 2654435761u) >> (32 - 10);
      int found = -1;
      for (int probe = 0; probe < 64; ++probe) {
        const u32 k = hkey[h];
        if (k == slot) {
          found = (int)h;
          break;
        }
        if (k == NONE32) {
          const u32 old = atomicCAS(&hkey[h], NONE32, slot);
          if (old == NONE32 || old == slot) {
            found = (int)h;
            break;
          }
        }
        h = (h + 1) & (HCAP - 1);
      }
      if (found >= 0) {
        atomicAdd(&hpres[found], 1u);
        atomicMin(&hmn[found], (unsigned long long)x);
        atomicMax(&hmx[found], (unsigned long long)x);
        atomicAdd(&hs1[found], (unsigned long long)x);
        atomic_add_u128((u64*)&hs2lo[found], (u64*)&hs2hi[found], x2);
      } else {
        atomicAdd(&P.present[slot], 1u);
        atomicMin((unsigned long long*)&P.mn[slot], (unsigned long long)x);
        atomicMax((unsigned long long*)&P.mx[slot], (unsigned long long)x);
        atomicAdd((unsigned long long*)&P.s1[slot], (unsigned long long)x);
        atomic_add_u128(&P.s2lo[slot], &P.s2hi[slot], x2);
      }
    }
  }
  __syncthreads();
  for (int h = threadIdx.x; h < HCAP; h += STATS_NT) {
    const u32 slot = hkey[h];
    if (slot == NONE32) continue;
    atomicAdd(&P.present[slot], hpres[h]);
    atomicMin((unsigned long long*)&P.mn[slot], hmn[h]);
    atomicMax((unsigned long long*)&P.mx[slot], hmx[h]);
    atomicAdd((unsigned long long*)&P.s1[slot], hs1[h]);
    atomic_add_u128(&P.s2lo[slot], &P.s2hi[slot], ((u128)hs2hi[h] << 64) | hs2lo[h]);
  }
}

// Index of context k in the context-sorted entries [E0, E1), or ~0.
__device__ __forceinline__ u64 find_ctx(const u32* __restrict__ ctx, u64 E0, u64 E1, u32 k) {
  u64 lo = E0, hi = E1;  // first entry >= k
  while (lo < hi) {
    const u64 mid = lo + (hi - lo) / 2;
    if (ctx[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return (lo < E1 && ctx[lo] == k) ? lo : ~0ull;
}

// The partials of one context (slot 0): a thread per rank finds the rank's
// entry by binary search (the entries are context-sorted) instead of a warp
// reading all of them; warp sums, then one set of atomics per warp.
__global__ void __launch_bounds__(STATS_NT)
    k_stats_partial_one(const u32* __restrict__ S, u32 n, const u64* __restrict__ off,
                        const u32* __restrict__ ctx, const u64* __restrict__ time, u32 k,
                        Partials P) {
  u32 pres = 0;
  u64 mn = ~0ull, mx = 0, s1 = 0, s2lo = 0, s2hi = 0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const u32 r = rank_at(S, i);
    const u64 j = find_ctx(ctx, off[r], off[r + 1], k);
    if (j == ~0ull) continue;
    const u64 x = time[j];
    const u128 x2 = (u128)x * x;
    ++pres;
    mn = min(mn, x);
    mx = max(mx, x);
    s1 += x;
    const u64 lo = s2lo + (u64)x2;
    s2hi += (u64)(x2 >> 64) + (lo < s2lo ? 1ull : 0ull);
    s2lo = lo;
  }
  pres = __reduce_add_sync(FULL, pres);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, (u64)__shfl_xor_sync(FULL, mn, o));
    mx = max(mx, (u64)__shfl_xor_sync(FULL, mx, o));
    s1 += __shfl_xor_sync(FULL, s1, o);
    const u64 ol = __shfl_xor_sync(FULL, s2lo, o), oh = __shfl_xor_sync(FULL, s2hi, o);
    const u64 lo = s2lo + ol;
    s2hi += oh + (lo < s2lo ? 1ull : 0ull);
    s2lo = lo;
  }
  if ((threadIdx.x & 31) == 0 && pres) {
    atomicAdd(&P.present[0], pres);
    atomicMin((unsigned long long*)&P.mn[0], (unsigned long long)mn);
    atomicMax((unsigned long long*)&P.mx[0], (unsigned long long)mx);
    atomicAdd((unsigned long long*)&P.s1[0], (unsigned long long)s1);
    atomic_add_u128(&P.s2lo[0], &P.s2hi[0], ((u128)s2hi << 64) | s2lo);
  }
}

// Per slot: mean, std (ddof 1), cv, balance from the exact partials.
__global__ void k_stats_finalize(u32 n_slots, u64 n_all, const u32* S, Partials P,
                                 ta_ctx_stats* out, SetMap sets) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  u64 n = n_all;
  u32 first_rank = 0;
  if (sets.S) {  // every context of a set is taken over that set's ranks
    const u32 set = set_of_ctx(sets, s);
    first_rank = sets.set_rank0[set];
    n = sets.set_rank0[set + 1] - first_rank;
  } else {
    first_rank = rank_at(S, 0);
  }
  const u32 present = P.present[s];
  const u64 mx = P.mx[s], s1 = P.s1[s];
  const u128 S2 = ((u128)P.s2hi[s] << 64) | P.s2lo[s];
  const u128 M = (u128)n * S2 - (u128)s1 * s1;
  const double mean = u64_to_f64(s1) / u64_to_f64(n);
  const double sd = (n < 2) ? 0.0 : sqrt(u128_to_f64(M) / u64_to_f64(n * (n - 1)));
  ta_ctx_stats st;
  st.n = (u32)n;
  st.present = present;
  st.argmax = 0;
  st.reserved = 0;
  st.min = (present < n) ? 0ull : P.mn[s];
  st.max = mx;
  st.s1 = s1;
  st.s2_lo = (u64)S2;
  st.s2_hi = (u64)(S2 >> 64);
  st.mean = mean;
  st.std = sd;
  st.cv = (mean == 0.0) ? 0.0 : sd / mean;
  st.balance = (mx == 0) ? 1.0 : mean / u64_to_f64(mx);
  out[s] = st;
  P.sd[s] = sd;
  P.Mlo[s] = (u64)M;
  P.Mhi[s] = (u64)(M >> 64);
  P.argmax[s] = (mx == 0) ? first_rank : NONE32;
}

// Argmax (lowest rank attaining max), z-scores and the exact outlier rule.
__global__ void k_stats_z(const u32* __restrict__ S, u32 n_all, const u64* __restrict__ off,
                          const u32* __restrict__ ctx, const u64* __restrict__ time,
                          const u32* __restrict__ slot_of_ctx, Partials P, u32 tn, u32 td,
                          double* z_out, u64* keys, double* zs, u64 cap,
                          unsigned long long* n_out, uint8_t* rank_flag, SetMap sets,
                          u64 n_stat, u32 single) {
  // entry j of rank r in slot `slot`, over n ranks
  auto entry = [&](u64 j, u32 r, u32 slot, u64 n) {
    const u64 x = time[j];
    const u64 mx = P.mx[slot];
    if (mx > 0 && x == mx) atomicMin(&P.argmax[slot], r);
    const u64 s1 = P.s1[slot];
    const u128 M = ((u128)P.Mhi[slot] << 64) | P.Mlo[slot];
    const long long D = (long long)((u64)n * x) - (long long)s1;
    const double z = (n < 2 || M == 0) ? 0.0 : i64_to_f64(D) / (u64_to_f64(n) * P.sd[slot]);
    if (z_out) z_out[j] = z;
    if (is_outlier(D, n, M, tn, td)) {
      const unsigned long long q = atomicAdd(n_out, 1ull);
      if (q < cap) {
        keys[q] = ((u64)slot << 32) | r;
        zs[q] = z;
      }
      if (rank_flag) rank_flag[r] = 1;
    }
  };
  if (single != NONE32) {  // one context (slot 0), no sets: a thread per rank
    const u64 n = n_stat ? n_stat : n_all;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += gridDim.x * blockDim.x) {
      const u32 r = rank_at(S, i);
      const u64 j = find_ctx(ctx, off[r], off[r + 1], single);
      if (j != ~0ull) entry(j, r, 0, n);
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 i = gw; i < n_all; i += nw) {
    const u32 r = rank_at(S, i);
    u64 n = n_stat ? n_stat : n_all;  // the moments' rank count (a shard's job: all shards)
    u32 cbase = 0;
    if (sets.S) {
      const u32 set = sets.rank_set[r];
      cbase = sets.set_ctx0[set];
      n = sets.set_rank0[set + 1] - sets.set_rank0[set];
    }
    const u64 E0 = off[r], E1 = off[r + 1];
    for (u64 j = E0 + lane; j < E1; j += 32) {
      const u32 c = ctx[j];
      const u32 slot = sets.S ? cbase + c : slot_of_ctx[c];
      if (slot == NONE32) continue;
      entry(j, r, slot, n);
    }
  }
}

// Argmax into the output; with sets, as a rank id local to the slot's set.
__global__ void k_stats_argmax(u32 n_slots, const u32* argmax, ta_ctx_stats* out,
                               SetMap sets = SetMap{}) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  out[s].argmax = argmax[s] - (sets.S ? sets.set_rank0[set_of_ctx(sets, s)] : 0u);
}

// ---- sort of (key, z) pairs by key: bitonic, in shared memory when small --
constexpr int SORT_SMEM = 2048;

__device__ __forceinline__ void cmp_swap(u64* k, double* v, u32 i, u32 j, bool up) {
  const u64 a = k[i], b = k[j];
  if ((a > b) == up) {
    k[i] = b;
    k[j] = a;
    const double t = v[i];
    v[i] = v[j];
    v[j] = t;
  }
}

__global__ void k_sort_small(u64* keys, double* vals, u32 n) {
  __shared__ u64 sk[SORT_SMEM];
  __shared__ double sv[SORT_SMEM];
  u32 P = 1;
  while (P < n) P <<= 1;
  for (u32 i = threadIdx.x; i < P; i += blockDim.x) {
    sk[i] = i < n ? keys[i] : ~0ull;
    sv[i] = i < n ? vals[i] : 0.0;
  }
  __syncthreads();
  for (u32 k = 2; k <= P; k <<= 1)
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      for (u32 i = threadIdx.x; i < P; i += blockDim.x) {
        const u32 l = i ^ j;
        if (l > i) cmp_swap(sk, sv, i, l, (i & k) == 0);
      }
      __syncthreads();
    }
  for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
    keys[i] = sk[i];
    vals[i] = sv[i];
  }
}

__global__ void k_sort_step(u64* keys, double* vals, u64 P, u64 j, u64 k) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const u64 l = i ^ j;
  if (l > i) {
    const bool up = (i & k) == 0;
    const u64 a = keys[i], b = keys[l];
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
      const double t = vals[i];
      vals[i] = vals[l];
      vals[l] = t;
    }
  }
}

// Bitonic stages of span below SORT_B inside blocks of SORT_B pairs, one
// block per CTA in shared memory: every stage k <= SORT_B (k_fixed = 0), or
// the spans j < SORT_B of stage k_fixed.  Directions follow global indices.
constexpr u32 SORT_B = 4096;

__global__ void __launch_bounds__(1024) k_sort_block(u64* keys, double* vals, u64 k_fixed) {
  extern __shared__ __align__(16) u64 sk[];
  double* sv = reinterpret_cast<double*>(sk + SORT_B);
  const u64 base = (u64)blockIdx.x * SORT_B;
  for (u32 i = threadIdx.x; i < SORT_B; i += blockDim.x) {
    sk[i] = keys[base + i];
    sv[i] = vals[base + i];
  }
  __syncthreads();
  const u64 k0 = k_fixed ? k_fixed : 2, k1 = k_fixed ? k_fixed : SORT_B;
  for (u64 k = k0; k <= k1; k <<= 1)
    for (u32 j = (u32)((k >> 1) < (SORT_B >> 1) ? (k >> 1) : (SORT_B >> 1)); j > 0; j >>= 1) {
      for (u32 i = threadIdx.x; i < SORT_B; i += blockDim.x) {
        const u32 l = i ^ j;
        if (l > i) cmp_swap(sk, sv, i, l, ((base + i) & k) == 0);
      }
      __syncthreads();
    }
  for (u32 i = threadIdx.x; i < SORT_B; i += blockDim.x) {
    keys[base + i] = sk[i];
    vals[base + i] = sv[i];
  }
}

// Keys are (slot << 32 | rank); slot_ctx maps a slot back to its context
// (null: the slot is the context).
__global__ void k_write_outliers(const u64* keys, const double* zs, u64 n, ta_outlier* out,
                                 const u32* slot_ctx, u32 rank_base) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ta_outlier o;
  const u32 slot = (u32)(keys[i] >> 32);
  o.ctx = slot_ctx ? slot_ctx[slot] : slot;
  o.rank = (u32)keys[i] + rank_base;
  o.z = zs[i];
  out[i] = o;
}

inline unsigned blocks(u64 n, int nt = 256) { return (unsigned)std::max<u64>(1, (n + nt - 1) / nt); }

// Sort n (key, z) pairs held in buffers of at least next_pow2(n) entries.
void sort_pairs(const Launch& L, u64* keys, double* vals, u64 n) {
  if (n <= 1) return;
  if (n <= SORT_SMEM) {
    k_sort_small<<<1, 1024, 0, L.stream>>>(keys, vals, (u32)n);
    L.count();
    return;
  }
  u64 P = 1;
  while (P < n) P <<= 1;
  k_fill_u64<<<blocks(P - n), 256, 0, L.stream>>>(keys + n, P - n, ~0ull);
  L.count();
  if (P < SORT_B) {
    for (u64 k = 2; k <= P; k <<= 1)
      for (u64 j = k >> 1; j > 0; j >>= 1) {
        k_sort_step<<<blocks(P), 256, 0, L.stream>>>(keys, vals, P, j, k);
        L.count();
      }
    return;
  }
  // spans below SORT_B in shared memory, longer ones one global step each
  const size_t smem = (size_t)SORT_B * 16;
  cudaFuncSetAttribute(k_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned nb = (unsigned)(P / SORT_B);
  k_sort_block<<<nb, 1024, smem, L.stream>>>(keys, vals, 0);
  L.count();
  for (u64 k = 2 * (u64)SORT_B; k <= P; k <<= 1) {
    for (u64 j = k >> 1; j >= SORT_B; j >>= 1) {
      k_sort_step<<<blocks(P), 256, 0, L.stream>>>(keys, vals, P, j, k);
      L.count();
    }
    k_sort_block<<<nb, 1024, smem, L.stream>>>(keys, vals, k);
    L.count();
  }
}

const Csr* metric_csr(const ta_experiment* e, u32 metric) {
  if (metric == TA_EXCLUSIVE) return &e->x;
  if (metric == TA_INCLUSIVE && e->has_incl) return &e->in;
  return nullptr;
}

// Device copy of a caller array (or the caller's device pointer itself).
template <class T>
ta_status to_device(ta_ctx* c, Pool& tmp, const T* src, u64 n, u32 kind, const T** out,
                    const char* what) {
  if (!src) {
    *out = nullptr;
    return TA_OK;
  }
  if (kind == TA_MEM_DEVICE) {
    *out = src;
    return TA_OK;
  }
  T* d;
  TRY(tmp.get_n(std::max<u64>(n, 1), &d, what));
  TRY(copy(c, d, src, n * sizeof(T)));
  *out = d;
  return TA_OK;
}

// Validate a sorted-unique subset on the device.
ta_status check_subset(ta_ctx* c, const Launch& L, const u32* dv, u32 n, u32 limit, u32* status,
                       const char* what) {
  if (!dv) return TA_OK;
  cudaMemsetAsync(status, 0, 4, c->stream);
  k_check_sorted<<<blocks(n), 256, 0, L.stream>>>(dv, n, limit, status);
  L.count();
  u32 h = 0;
  TRY(copy(c, &h, status, 4));
  TRY(sync_check(c, what));
  if (h) return fail(TA_ERR_INVALID_ARG, "%s must be sorted, unique and in range", what);
  return TA_OK;
}

struct StatsRun {
  u32 n_slots = 0;
  u64 n = 0;
  Partials P{};
  ta_ctx_stats* stats = nullptr;  // device [n_slots]
  u64* keys = nullptr;
  double* zs = nullptr;
  u64 n_out = 0;
  u64 kept = 0;
};

// Everything of ta_context_stats on device buffers.
ta_status stats_run(ta_experiment* e, Pool& tmp, u32 metric, const u32* dS, u32 n,
                    const u32* dK, u32 nk, u32 tn, u32 td, u64 cap, double* z_out,
                    uint8_t* rank_flag, StatsRun& R, bool count_outliers = true,
                    u32 single = NONE32) {
  ta_ctx* c = e->ctx;
  Launch L{c->stream, c->num_sms, &c->launches};
  const Csr* m = metric_csr(e, metric);
  R.n = n;
  R.n_slots = dK ? nk : e->C;
  const u32 ns = R.n_slots;
  u32* slot_of_ctx;
  TRY(tmp.get_n(e->C, &slot_of_ctx, "slot map"));
  cudaMemsetAsync(slot_of_ctx, 0xFF, (size_t)e->C * 4, c->stream);
  k_slot_map<<<blocks(dK ? nk : e->C), 256, 0, L.stream>>>(dK, nk, e->C, slot_of_ctx);
  L.count();
  Partials& P = R.P;
  TRY(tmp.get_n(ns, &P.present, "partials"));
  TRY(tmp.get_n(ns, &P.mn, "partials"));
  TRY(tmp.get_n(ns, &P.mx, "partials"));
  TRY(tmp.get_n(ns, &P.s1, "partials"));
  TRY(tmp.get_n(ns, &P.s2lo, "partials"));
  TRY(tmp.get_n(ns, &P.s2hi, "partials"));
  TRY(tmp.get_n(ns, &P.argmax, "partials"));
  TRY(tmp.get_n(ns, &P.sd, "partials"));
  TRY(tmp.get_n(ns, &P.Mlo, "partials"));
  TRY(tmp.get_n(ns, &P.Mhi, "partials"));
  TRY(tmp.get_n(ns, &R.stats, "stats"));
  cudaMemsetAsync(P.present, 0, (size_t)ns * 4, c->stream);
  cudaMemsetAsync(P.mn, 0xFF, (size_t)ns * 8, c->stream);
  cudaMemsetAsync(P.mx, 0, (size_t)ns * 8, c->stream);
  cudaMemsetAsync(P.s1, 0, (size_t)ns * 8, c->stream);
  cudaMemsetAsync(P.s2lo, 0, (size_t)ns * 8, c->stream);
  cudaMemsetAsync(P.s2hi, 0, (size_t)ns * 8, c->stream);
  const u64 kcap = std::max<u64>(1, cap);
  u64 P2 = 1;
  while (P2 < kcap) P2 <<= 1;
  TRY(tmp.get_n(P2, &R.keys, "outlier keys"));
  TRY(tmp.get_n(P2, &R.zs, "outlier z"));
  unsigned long long* n_out;
  TRY(tmp.get_n(1, &n_out, "outlier count"));
  cudaMemsetAsync(n_out, 0, 8, c->stream);
  if (z_out) cudaMemsetAsync(z_out, 0, m->nnz * 8, c->stream);
  const int grid = std::max(1, std::min<int>(c->num_sms * 4, (int)((n + 7) / 8)));
  // one context (given on the host): each rank's entry by binary search
  if (nk != 1 || !dK) single = NONE32;
  if (single != NONE32)
    k_stats_partial_one<<<blocks(n), STATS_NT, 0, L.stream>>>(dS, n, m->off, m->ctx, m->time,
                                                              single, P);
  else
    k_stats_partial<<<grid, STATS_NT, 0, L.stream>>>(dS, n, m->off, m->ctx, m->time, slot_of_ctx,
                                                     P, SetMap{});
  k_stats_finalize<<<blocks(ns), 256, 0, L.stream>>>(ns, n, dS, P, R.stats, SetMap{});
  k_stats_z<<<single != NONE32 ? blocks(n) : grid, 256, 0, L.stream>>>(
      dS, n, m->off, m->ctx, m->time, slot_of_ctx, P, tn, td, z_out, R.keys, R.zs, kcap, n_out,
      rank_flag, SetMap{}, 0, single);
  k_stats_argmax<<<blocks(ns), 256, 0, L.stream>>>(ns, P.argmax, R.stats);
  L.count(4);
  if (!count_outliers) return TA_OK;  // the caller needs the flags only
  u64 h = 0;
  TRY(copy(c, &h, n_out, 8));
  TRY(sync_check(c, "context statistics"));
  R.n_out = h;
  R.kept = std::min<u64>(h, cap);
  if (R.kept > 1 && h <= cap) sort_pairs(L, R.keys, R.zs, R.kept);
  return TA_OK;
}

// ------------------------------------------------------------- topology --
__global__ void k_topo_check(const u32* node_of_rank, u32 R, u32 nn, const u32* rack, u32 nr,
                             const u32* chassis, u32 nc, u32* status) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (node_of_rank && i < R && node_of_rank[i] >= nn) flag(status, F_INVALID);
  if (rack && chassis && i < nn && (rack[i] >= nr || chassis[i] >= nc)) flag(status, F_INVALID);
}

__device__ __forceinline__ u64 csr_lookup(const u64* off, const u32* ctx, const u64* time, u32 r,
                                          u32 c) {
  u64 lo = off[r], hi = off[r + 1];
  while (lo < hi) {
    const u64 mid = (lo + hi) / 2;
    if (ctx[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return (lo < off[r + 1] && ctx[lo] == c) ? time[lo] : 0ull;
}

__global__ void k_topo_nodes(const u32* S, u32 n, const u64* off, const u32* ctx, const u64* time,
                             u32 c, const uint8_t* rank_flag, const u32* node_of_rank,
                             u32* node_out, unsigned long long* node_sum, u32* node_ranks,
                             u32 nn) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32 r = rank_at(S, i);
  const u32 nd = node_of_rank[r];
  if (nd >= nn) return;  // reported by k_topo_check
  const u64 x = csr_lookup(off, ctx, time, r, c);
  if (rank_flag[r]) atomicAdd(&node_out[nd], 1u);
  atomicAdd(&node_sum[nd], (unsigned long long)x);
  atomicAdd(&node_ranks[nd], 1u);
}

__global__ void k_topo_up(u32 nn, const u32* node_out, const unsigned long long* node_sum,
                          u32 min_ranks, const u32* rack, const u32* chassis, uint8_t* node_flag,
                          u32* ch_flag, u32* ch_nodes, unsigned long long* ch_sum, u32* rk_flag,
                          u32* rk_nodes, unsigned long long* rk_sum, u32 nc, u32 nr) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const u32 f = node_out[i] >= min_ranks ? 1u : 0u;
  node_flag[i] = (uint8_t)f;
  const u32 ch = chassis[i], rk = rack[i];
  if (ch >= nc || rk >= nr) return;  // reported by k_topo_check
  atomicAdd(&ch_flag[ch], f);
  atomicAdd(&ch_nodes[ch], 1u);
  atomicAdd(&ch_sum[ch], node_sum[i]);
  atomicAdd(&rk_flag[rk], f);
  atomicAdd(&rk_nodes[rk], 1u);
  atomicAdd(&rk_sum[rk], node_sum[i]);
}

// One block: racks with a flagged node, ascending.
__global__ void k_topo_racks(u32 nr, const u32* rk_flag, u32* flagged, u32* count) {
  __shared__ u32 s_scan[32];
  __shared__ u32 s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (u32 b0 = 0; b0 < nr; b0 += blockDim.x) {
    const u32 i = b0 + threadIdx.x;
    const u32 f = (i < nr && rk_flag[i] > 0) ? 1u : 0u;
    const u32 x = warp_incl_scan(f, lane);
    if (lane == 31) s_scan[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const u32 nw = blockDim.x / 32;
      u32 y = lane < (int)nw ? s_scan[lane] : 0u;
      y = warp_incl_scan(y, lane);
      if (lane < (int)nw) s_scan[lane] = y;
    }
    __syncthreads();
    const u32 pos = s_base + (warp > 0 ? s_scan[warp - 1] : 0u) + x - f;
    if (f) flagged[pos] = i;
    __syncthreads();
    if (threadIdx.x == 0) s_base += s_scan[blockDim.x / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = s_base;
}

// -------------------------------------------------------------- speedup --
// I* = min over S of n_iter, their sum and the longest span: a warp
// reduction, then one set of atomics per warp.
__global__ void k_sp_istar(const u32* S, u32 n, const u32* n_iter, const u64* span, u32* istar,
                           unsigned long long* sum_iter, unsigned long long* max_span) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  u32 it = NONE32, sum = 0;
  u64 sp = 0;
  if (i < n) {
    const u32 r = rank_at(S, i);
    it = n_iter[r];
    sum = it;
    sp = span[r];
  }
  it = __reduce_min_sync(FULL, it);
  const u64 sum64 = warp_incl_scan((u64)sum, threadIdx.x & 31);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sp = max(sp, (u64)__shfl_xor_sync(FULL, sp, o));
  if ((threadIdx.x & 31) == 31) {
    if (it != NONE32) atomicMin(istar, it);
    atomicAdd(sum_iter, (unsigned long long)sum64);
    atomicMax(max_span, (unsigned long long)sp);
  }
}

constexpr int SP_NW = 8;
constexpr u32 SP_KC = 128;    // contexts per within-rank chunk (8-bit positions, 0xFF absent)
constexpr u32 SP_U = 4;       // entries per lane per batch (two batches in flight)
constexpr u32 SP_SMAP = 32768;  // context counts whose 8-bit map fits shared memory

// Context -> position in the requested set's chunk [k0, k0 + nkc) (0xFF:
// outside), built by every CTA in shared memory from the sorted set itself.
__device__ __forceinline__ void build_kmap8(unsigned char* kmap8, u32 C, const u32* kset, u32 k0,
                                            u32 nkc) {
  uint4* w = reinterpret_cast<uint4*>(kmap8);
  const uint4 ff = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (u32 i = threadIdx.x; i < (C + 15) / 16; i += blockDim.x) w[i] = ff;
  __syncthreads();
  for (u32 i = threadIdx.x; i < nkc; i += blockDim.x)
    if (kset[k0 + i] < C) kmap8[kset[k0 + i]] = (unsigned char)i;  // checked later
  __syncthreads();
}

// Chunk position of context c: the shared 8-bit map, or the global map for
// context counts beyond it.
struct KLookup {
  const unsigned char* kmap8;  // null: use kmap
  const u32* kmap;
  u32 k0, nkc;
  __device__ __forceinline__ u32 operator()(u32 c) const {
    if (kmap8) {
      const u32 k = kmap8[c];
      return k == 0xFFu ? NONE32 : k;
    }
    const u32 k = kmap[c];
    return (k == NONE32 || k < k0 || k >= k0 + nkc) ? NONE32 : k - k0;
  }
};

// (a) Within-rank CV terms: one warp per rank of S; over iterations i < I*,
// per context of the chunk: sum and 128-bit sum of squares of t[r][i][k] in
// warp-private shared memory (a context absent from a row adds 0), then the
// CV term of (r, k).  A rank with exactly I* iteration rows whose exclusive
// entries carry their iteration moments (mom_ok) takes both sums from them,
// one entry per context; any other rank reads its rows, which are contiguous
// entries, two batches in flight while one is summed.
__global__ void __launch_bounds__(SP_NW * 32)
    k_sp_within(const u32* S, u32 n, const u64* row_off, const u64* entry_off, const u32* e_ctx,
                const u64* e_time, const u32* kset, const u32* kmap, u32 C, u32 k0, u32 nkc,
                u32 I, const u64* x_off, const u32* x_ctx, const u64* x_m1, const u64* x_m2,
                const uint8_t* mom_ok, double* cvw) {
  __shared__ unsigned long long s_sum[SP_NW][SP_KC], s_lo[SP_NW][SP_KC], s_hi[SP_NW][SP_KC];
  extern __shared__ __align__(16) unsigned char kmap8[];
  const bool smap = C <= SP_SMAP;
  if (smap) build_kmap8(kmap8, C, kset, k0, nkc);
  const KLookup look{smap ? kmap8 : nullptr, kmap, k0, nkc};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* my_sum = s_sum[warp];
  unsigned long long* my_lo = s_lo[warp];
  unsigned long long* my_hi = s_hi[warp];
  for (u32 q = lane; q < SP_KC; q += 32) my_sum[q] = my_lo[q] = my_hi[q] = 0;
  __syncwarp();
  const u32 gw = blockIdx.x * SP_NW + warp, nw = gridDim.x * SP_NW;
  const double cI = cv_coef(I);
  for (u32 ri = gw; ri < n; ri += nw) {
    const u32 r = rank_at(S, ri);
    const u64 row0 = row_off[r] + 1;  // skip the prologue row
    if (mom_ok && mom_ok[r] && row_off[r + 1] - row_off[r] == (u64)I + 1) {
      const ulonglong2* m2 = reinterpret_cast<const ulonglong2*>(x_m2);
      for (u64 j = x_off[r] + lane; j < x_off[r + 1]; j += 32) {
        const u32 kk = look(x_ctx[j]);
        if (kk == NONE32) continue;
        const ulonglong2 q = m2[j];
        my_sum[kk] = x_m1[j];
        my_lo[kk] = q.x;
        my_hi[kk] = q.y;
      }
    } else {
      const u64 E0 = entry_off[row0], E1 = entry_off[row0 + I];
      u32 c[SP_U];
      u64 t[SP_U];
#pragma unroll
      for (u32 u = 0; u < SP_U; ++u) {
        const u64 j = E0 + u * 32 + lane;
        c[u] = j < E1 ? e_ctx[j] : NONE32;
        t[u] = j < E1 ? e_time[j] : 0ull;
      }
      for (u64 jb = E0; jb < E1; jb += 32 * SP_U) {
        u32 cn[SP_U];
        u64 tn[SP_U];
#pragma unroll
        for (u32 u = 0; u < SP_U; ++u) {  // the next batch
          const u64 j = jb + 32 * SP_U + u * 32 + lane;
          cn[u] = j < E1 ? e_ctx[j] : NONE32;
          tn[u] = j < E1 ? e_time[j] : 0ull;
        }
#pragma unroll
        for (u32 u = 0; u < SP_U; ++u) {
          const u32 kk = (c[u] != NONE32) ? look(c[u]) : NONE32;
          if (kk == NONE32) continue;
          atomic_add_u64_lo32(&my_sum[kk], t[u]);
          atomic_add_u128((u64*)&my_lo[kk], (u64*)&my_hi[kk], (u128)t[u] * t[u]);
        }
#pragma unroll
        for (u32 u = 0; u < SP_U; ++u) {
          c[u] = cn[u];
          t[u] = tn[u];
        }
      }
    }
    __syncwarp();
    for (u32 kk = lane; kk < nkc; kk += 32) {
      const u128 q = ((u128)my_hi[kk] << 64) | my_lo[kk];
      cvw[(u64)(k0 + kk) * n + ri] = cv_of_sums(my_sum[kk], q, I, cI);
      my_sum[kk] = my_lo[kk] = my_hi[kk] = 0;
    }
    __syncwarp();
  }
}

// (b) Cells (i, k) over ranks.  A warp owns the cells of SP_IB iterations
// [i0, i0 + SP_IB) and 64 contexts [k0, k0 + 64) for a group of ranks and
// keeps them in registers: lane l holds contexts k0 + l and k0 + l + 32
// (sum, max, 128-bit sum of squares).  A round is one rank: its SP_IB rows
// are one contiguous entry range, which the warp's lane 0 copies into a
// shared-memory stage with two bulk copies (contexts, times) completing on
// the stage's mbarrier; SPC_ST stages are in flight, so while one round is
// summed the next ones are on their way.  Each entry's time is scattered to
// a per-warp buffer indexed by (row, context) -- a row holds each context
// once, so plain stores suffice -- and every lane then folds its contexts'
// values into its registers, absent ones reading 0.  A rank whose iteration
// rows all hold the same contexts (the load's mom_ok) has only its first
// row's contexts copied: its values go to the buffer by position, through
// the warp's template (contexts by position and each chunk slot's position),
// rebuilt when a rank's first row differs from it.  A round too long for a
// stage is read from global memory directly.  The group's cells go to the
// global cells with one set of atomics per warp.
constexpr u32 SP_IB = 4;      // iterations per warp (one contiguous read per rank)
constexpr u32 SP_CU = 8;      // entries per lane in flight (rounds read directly)
constexpr u32 SPC_ST = 2;     // stages per warp
constexpr u32 SPC_CAP = 320;  // entries per stage
// per stage: contexts (cap + 4 for the 16-byte rounding), times (cap + 2)
constexpr u32 SPC_CTX_BYTES = 4 * (SPC_CAP + 4);
constexpr u32 SPC_TIME_BYTES = 8 * (SPC_CAP + 2);
constexpr u32 SPC_STAGE_BYTES = SPC_CTX_BYTES + SPC_TIME_BYTES;
constexpr u32 SPC_WARP_BYTES = SPC_ST * SPC_STAGE_BYTES + 16 * SPC_ST;  // + mbarriers
static_assert(SPC_CTX_BYTES % 16 == 0 && SPC_STAGE_BYTES % 16 == 0, "stage alignment");

__global__ void __launch_bounds__(SP_NW * 32, 2)
    k_sp_cells(const u32* __restrict__ S, u32 n, const u64* __restrict__ row_off,
               const u64* __restrict__ entry_off, const u32* __restrict__ e_ctx,
               const u64* __restrict__ e_time, const u32* __restrict__ kset,
               const u32* __restrict__ kmap, u32 C, u32 nk, u32 I, u32 n_ib, u32 n_kb, u32 group,
               u64 n_items, u32 map_bytes, u64* g_sum, u64* g_max, u64* g_sqlo, u64* g_sqhi,
               const uint8_t* __restrict__ mom_ok, u32* status) {
  __shared__ u64 rowbuf[SP_NW][SP_IB][64];
  __shared__ u32 tctx[SP_NW][96];             // the warp's template contexts by position
  __shared__ unsigned char pslot[SP_NW][64];  // and each chunk slot's position (0xFF: none)
  extern __shared__ __align__(16) unsigned char dsm[];
  unsigned char* kmap8 = dsm;  // [map_bytes]: one chunk of 64 contexts maps through it
  const bool smap = map_bytes > 0;
  if (smap) build_kmap8(kmap8, C, kset, 0, nk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* ws = dsm + map_bytes + (size_t)warp * SPC_WARP_BYTES;
  u64* bar = reinterpret_cast<u64*>(ws + SPC_ST * SPC_STAGE_BYTES);
  u64* buf = &rowbuf[warp][0][0];
  for (u32 q = lane; q < SP_IB * 64; q += 32) buf[q] = 0;
  const u64 item = (u64)blockIdx.x * SP_NW + warp;
  if (item >= n_items) return;
  if (lane == 0) {
    for (u32 s = 0; s < SPC_ST; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
  const u32 ib = (u32)(item % n_ib), kb = (u32)((item / n_ib) % n_kb);
  const u32 g = (u32)(item / ((u64)n_ib * n_kb));
  const u32 i0 = ib * SP_IB, k0 = kb * 64;
  const KLookup look{smap ? kmap8 : nullptr, kmap, k0, 64};
  const u32 nrow = min(SP_IB, I - i0);
  const u32 r_begin = g * group, r_end = min(n, r_begin + group);
  u64 csum[SP_IB][2], cmax[SP_IB][2], clo[SP_IB][2], chi[SP_IB][2];
#pragma unroll
  for (u32 il = 0; il < SP_IB; ++il)
#pragma unroll
    for (u32 h = 0; h < 2; ++h) csum[il][h] = cmax[il][h] = clo[il][h] = chi[il][h] = 0;
  constexpr u32 NB = SP_IB + 1;
  // entry boundaries of SPC_OB rounds at once: lane p NB + q holds the start
  // of row i0 + q of rank rb0 + p (q = nrow: the end of its last row); two
  // batches ahead of the round being summed are resolved or in flight, so a
  // stage is refilled without waiting on these loads
  constexpr u32 SPC_OB = 6;
  static_assert(SPC_OB * NB <= 32 && SPC_OB % SPC_ST == 0, "offset batch");
  // bit 63 of a round's first bound: every iteration row of its rank holds
  // the same contexts (mom_ok), so the stage copies the first row's contexts
  // only and the round is read by position (entry offsets are below 2^63)
  constexpr u64 TBIT = 1ull << 63;
  auto batch = [&](u32 rb0) -> u64 {
    const u32 p = (u32)lane / NB, q = (u32)lane % NB;
    u64 mine = 0;
    if (p < SPC_OB && rb0 + p < r_end) {
      const u32 rk = rank_at(S, rb0 + p);
      const u64 row = row_off[rk] + 1 + i0;
      mine = entry_off[row + min(q, nrow)];
      if (q == 0 && mom_ok && mom_ok[rk]) mine |= TBIT;
    }
    return mine;
  };
  u32 tp = 0;  // the template: L (bits 0-7, 0: none), slot positions (8-15, 16-23)
  // stage s takes round rb (its bounds in lanes p NB .. p NB + SP_IB of ob)
  u32 phase = 0;      // bit s: parity of stage s's next completion
  u32 staged = 0;     // bit s: stage s holds a copy in flight
  u64 sbase[SPC_ST];  // first entry of each stage's range
  auto issue = [&](u32 s, u32 rb, u64 ob, u32 p) {
    const u64 e0t = __shfl_sync(FULL, ob, p * NB), e1 = __shfl_sync(FULL, ob, p * NB + nrow);
    const u64 r1 = __shfl_sync(FULL, ob, p * NB + 1);  // end of the round's first row
    const u64 e0 = e0t & ~TBIT;
    staged &= ~(1u << s);
    if (rb >= r_end || e1 <= e0 || e1 - e0 > SPC_CAP) return;
    const u64 ce = (e0t & TBIT) ? r1 : e1;  // contexts: the first row only for a template rank
    const u64 c0 = e0 & ~(u64)3, c1 = (ce + 3) & ~(u64)3;  // 16-byte rounded ranges
    const u64 t0 = e0 & ~(u64)1, t1 = (e1 + 1) & ~(u64)1;
    sbase[s] = e0;
    staged |= 1u << s;
    if (lane == 0) {
      unsigned char* st = ws + s * SPC_STAGE_BYTES;
      fence_proxy_async_smem();  // the stage's last reads come before its refill
      mbar_arrive_expect_tx(&bar[s], (u32)((c1 - c0) * 4 + (t1 - t0) * 8));
      bulk_g2s(st, e_ctx + c0, (u32)((c1 - c0) * 4), &bar[s]);
      bulk_g2s(st + SPC_CTX_BYTES, e_time + t0, (u32)((t1 - t0) * 8), &bar[s]);
    }
  };
  bool failed = false;
  u64 ob0 = batch(r_begin), ob1 = batch(r_begin + SPC_OB);
#pragma unroll
  for (u32 s = 0; s < SPC_ST; ++s) issue(s, r_begin + s, ob0, s);
  for (u32 rb0 = r_begin; rb0 < r_end && !failed; rb0 += SPC_OB) {
    const u64 ob2 = batch(rb0 + 2 * SPC_OB);
#pragma unroll
    for (u32 p = 0; p < SPC_OB; ++p) {
      const u32 rb = rb0 + p, s = p % SPC_ST;
      if (rb >= r_end || failed) break;
      u64 bnd[NB];
#pragma unroll
      for (u32 q = 0; q < NB; ++q) bnd[q] = __shfl_sync(FULL, ob0, p * NB + q);
      const bool trank = (bnd[0] & TBIT) != 0;
      bnd[0] &= ~TBIT;
      const u64 total = bnd[SP_IB] - bnd[0];
      if ((staged >> s) & 1u) {
        if (!mbar_wait(&bar[s], (phase >> s) & 1u)) {
          failed = true;
          continue;
        }
        phase ^= 1u << s;
        const unsigned char* st = ws + s * SPC_STAGE_BYTES;
        const u32* sctx = reinterpret_cast<const u32*>(st) + (sbase[s] & 3);
        const u64* stime = reinterpret_cast<const u64*>(st + SPC_CTX_BYTES) + (sbase[s] & 1);
        if (trank) {  // every row is the first row's contexts: values by position
          const u32 L = (u32)(bnd[1] - bnd[0]);
          const bool h0 = (u32)lane < L, h1 = (u32)lane + 32 < L, h2 = (u32)lane + 64 < L;
          const u32 c0 = h0 ? sctx[lane] : NONE32, c1 = h1 ? sctx[lane + 32] : NONE32,
                    c2 = h2 ? sctx[lane + 64] : NONE32;
          bool same = (tp & 0xFFu) == L;
          if (same)
            same = c0 == tctx[warp][lane] && c1 == tctx[warp][lane + 32] &&
                   c2 == tctx[warp][lane + 64];
          if (!__all_sync(FULL, same)) {  // a new template: its contexts and slot positions
            tctx[warp][lane] = c0;
            tctx[warp][lane + 32] = c1;
            tctx[warp][lane + 64] = c2;
            pslot[warp][lane] = pslot[warp][lane + 32] = 0xFF;
            __syncwarp();
            const u32 k0s = h0 ? look(c0) : NONE32, k1s = h1 ? look(c1) : NONE32,
                      k2s = h2 ? look(c2) : NONE32;
            if (k0s != NONE32) pslot[warp][k0s] = (unsigned char)lane;
            if (k1s != NONE32) pslot[warp][k1s] = (unsigned char)(lane + 32);
            if (k2s != NONE32) pslot[warp][k2s] = (unsigned char)(lane + 64);
            __syncwarp();
            tp = L | (u32)pslot[warp][lane] << 8 | (u32)pslot[warp][lane + 32] << 16;
          }
          const u32 src0 = (tp >> 8) & 0xFFu, src1 = tp >> 16;
#pragma unroll
          for (u32 il = 0; il < SP_IB; ++il) {
            if (il >= nrow) continue;
            if (src0 != 0xFFu) buf[il * 64 + lane] = stime[il * L + src0];
            if (src1 != 0xFFu) buf[il * 64 + lane + 32] = stime[il * L + src1];
          }
        } else {
          // all of the stage's loads first (independent), then the lookups,
          // then the scatter: no chain of dependent shared-memory loads
          constexpr u32 SPC_U = SPC_CAP / 32;
          u32 kk[SPC_U];
#pragma unroll
          for (u32 u = 0; u < SPC_U; ++u) {
            const u32 v = (u32)lane + 32 * u;
            kk[u] = v < (u32)total ? sctx[v] : NONE32;
          }
#pragma unroll
          for (u32 u = 0; u < SPC_U; ++u) kk[u] = kk[u] != NONE32 ? look(kk[u]) : NONE32;
#pragma unroll
          for (u32 u = 0; u < SPC_U; ++u) {
            const u32 v = (u32)lane + 32 * u;
            if (kk[u] == NONE32) continue;
            const u64 jj = bnd[0] + v;
            u32 il = 0;
#pragma unroll
            for (u32 q = 1; q < SP_IB; ++q) il += (jj >= bnd[q]) ? 1u : 0u;
            buf[il * 64 + kk[u]] = stime[v];
          }
        }
      } else {
        for (u64 vb = 0; vb < total; vb += 32 * SP_CU) {
          u32 c[SP_CU], slot[SP_CU];
          u64 t[SP_CU];
#pragma unroll
          for (u32 u = 0; u < SP_CU; ++u) {
            const u64 v = vb + u * 32 + lane;
            const u64 jj = bnd[0] + v;
            u32 il = 0;
#pragma unroll
            for (u32 q = 1; q < SP_IB; ++q) il += (jj >= bnd[q]) ? 1u : 0u;
            slot[u] = il;
            c[u] = v < total ? e_ctx[jj] : NONE32;
            t[u] = v < total ? e_time[jj] : 0ull;
          }
#pragma unroll
          for (u32 u = 0; u < SP_CU; ++u) {
            const u32 kk = (c[u] != NONE32) ? look(c[u]) : NONE32;
            if (kk != NONE32) buf[slot[u] * 64 + kk] = t[u];
          }
        }
      }
      __syncwarp();
      // the stage is free: it takes the round SPC_ST ahead
      if (p + SPC_ST < SPC_OB) issue(s, rb + SPC_ST, ob0, p + SPC_ST);
      else issue(s, rb + SPC_ST, ob1, p + SPC_ST - SPC_OB);
#pragma unroll
      for (u32 il = 0; il < SP_IB; ++il)
#pragma unroll
        for (u32 h = 0; h < 2; ++h) {
          u64* cell = &buf[il * 64 + lane + 32 * h];
          const u64 v = *cell;
          *cell = 0;
          const u128 v2 = (u128)v * v;
          csum[il][h] += v;
          cmax[il][h] = max(cmax[il][h], v);
          const u64 lo = clo[il][h] + (u64)v2;
          chi[il][h] += (u64)(v2 >> 64) + (lo < clo[il][h] ? 1ull : 0ull);
          clo[il][h] = lo;
        }
      __syncwarp();
    }
    ob0 = ob1;
    ob1 = ob2;
  }
  if (failed) {  // report; let the copies still in flight land before leaving
    if (lane == 0) flag(status, F_TIMEOUT);
    for (u32 q = 0; q < SPC_ST; ++q)
      if ((staged >> q) & 1u) mbar_wait(&bar[q], (phase >> q) & 1u);
    return;
  }
#pragma unroll
  for (u32 il = 0; il < SP_IB; ++il)
#pragma unroll
    for (u32 h = 0; h < 2; ++h) {
      const u32 k = k0 + lane + 32 * h;
      if (il >= nrow || k >= nk) continue;
      const u64 gq = (u64)(i0 + il) * nk + k;
      if (csum[il][h]) atomicAdd((unsigned long long*)&g_sum[gq], (unsigned long long)csum[il][h]);
      if (cmax[il][h]) atomicMax((unsigned long long*)&g_max[gq], (unsigned long long)cmax[il][h]);
      if (clo[il][h] | chi[il][h])
        atomic_add_u128(&g_sqlo[gq], &g_sqhi[gq], ((u128)chi[il][h] << 64) | clo[il][h]);
    }
}

// Sum of each context's per-rank CV terms (a column of n values of cvw,
// context-major) in the fixed pairwise order of the definition: level by
// level, element i of the next level is v[2i] + v[2i+1], an odd last element
// moves up unchanged.  Element i of level l is the same rule applied to the
// values [i 2^l, min((i + 1) 2^l, n)) alone (a pair adds two such ranges, a
// carried element keeps its own), so the first PW_LEVELS levels are taken
// per block of 2^PW_LEVELS values in shared memory by many CTAs, and the
// rest by one CTA per context over the block values.
constexpr u32 PW_LEVELS = 11;
constexpr u32 PW_BLOCK = 1u << PW_LEVELS;

// Level PW_LEVELS of each context: CTA (k, y) reduces values
// [b PW_BLOCK, min((b + 1) PW_BLOCK, n)) of column k into blk[k nb + b] for
// the blocks b = y, y + gridDim.y, ...
__global__ void __launch_bounds__(256) k_sp_pair_blocks(const double* cvw, u32 n, u32 nb,
                                                        double* blk) {
  __shared__ double a[PW_BLOCK], b[PW_BLOCK];
  const u32 k = blockIdx.x;
  for (u32 bi = blockIdx.y; bi < nb; bi += gridDim.y) {
    const u64 base = (u64)k * n + (u64)bi * PW_BLOCK;
    u32 cnt = (u32)min((u64)PW_BLOCK, (u64)n - (u64)bi * PW_BLOCK);
    for (u32 i = threadIdx.x; i < cnt; i += blockDim.x) a[i] = cvw[base + i];
    __syncthreads();
    double *src = a, *dst = b;
    while (cnt > 1) {
      const u32 m = cnt / 2;
      for (u32 i = threadIdx.x; i < m; i += blockDim.x) dst[i] = src[2 * i] + src[2 * i + 1];
      if ((cnt & 1) && threadIdx.x == 0) dst[m] = src[cnt - 1];
      cnt = m + (cnt & 1);
      double* x = src;
      src = dst;
      dst = x;
      __syncthreads();
    }
    if (threadIdx.x == 0) blk[(u64)k * nb + bi] = src[0];
    __syncthreads();  // a and b are refilled for the next block
  }
}

// The remaining levels: one CTA per context over its n values of cvw (the
// block values), ping-ponging between cvw and tmp.
__global__ void __launch_bounds__(256) k_sp_pairwise(double* cvw, double* tmp, u32 n,
                                                     double* within) {
  const u32 k = blockIdx.x;
  double* src = cvw + (u64)k * n;
  double* dst = tmp + (u64)k * n;
  u32 cnt = n;
  while (cnt > 1) {
    const u32 m = cnt / 2;
    for (u32 i = threadIdx.x; i < m; i += blockDim.x) dst[i] = src[2 * i] + src[2 * i + 1];
    if ((cnt & 1) && threadIdx.x == 0) dst[m] = src[cnt - 1];
    cnt = m + (cnt & 1);
    double* x = src;
    src = dst;
    dst = x;
    __syncthreads();
  }
  if (threadIdx.x == 0) within[k] = (n == 0) ? 0.0 : src[0];
}

// One warp per context: the iteration sums in ascending order (the
// oracle's rounding; the lanes fetch 32 iterations at a time and every lane
// adds them in order from shuffles) and the finished per-context results.
__global__ void k_sp_final_k(u32 nk, u32 n, u32 I, const u64* g_sum, const u64* g_max,
                             const u64* g_sqlo, const u64* g_sqhi, const double* within,
                             ta_speedup_ctx* per) {
  const int lane = threadIdx.x & 31;
  const u32 k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= nk) return;
  u64 A = 0, B = 0;
  double across = 0.0;
  for (u32 i0 = 0; i0 < I; i0 += 32) {
    const u32 i = i0 + lane;
    u64 sum = 0, mx = 0;
    double term = 0.0;
    if (i < I) {
      const u64 q = (u64)i * nk + k;
      sum = g_sum[q];
      mx = g_max[q];
      const u128 sq = ((u128)g_sqhi[q] << 64) | g_sqlo[q];
      const double mean = u64_to_f64(sum) / u64_to_f64(n);
      const double sd = (n < 2) ? 0.0
                                : sqrt(u128_to_f64((u128)n * sq - (u128)sum * sum) /
                                       u64_to_f64((u64)n * (n - 1)));
      term = (mean == 0.0) ? 0.0 : sd / mean;
    }
    const u32 m = min(32u, I - i0);
    for (u32 x = 0; x < m; ++x) {
      A += __shfl_sync(FULL, mx, x);
      B += __shfl_sync(FULL, sum, x);
      across += __shfl_sync(FULL, term, x);
    }
  }
  const double w_sum = (I > 0) ? within[k] : 0.0;
  if (lane != 0) return;
  const u128 G = (u128)n * A - B;
  ta_speedup_ctx p;
  p.A = A;
  p.B = B;
  p.G_lo = (u64)G;
  p.G_hi = (u64)(G >> 64);
  if (I == 0) {
    p.avg_mean = p.avg_max = p.savings_per_iter = 0.0;
    p.cv_across = p.cv_within = 0.0;
  } else {
    p.avg_mean = u64_to_f64(B) / u128_to_f64((u128)n * I);
    p.avg_max = u64_to_f64(A) / u64_to_f64(I);
    p.savings_per_iter = u128_to_f64(G) / u128_to_f64((u128)n * I);
    p.cv_across = across / u64_to_f64(I);
    p.cv_within = w_sum / u64_to_f64(n);
  }
  p.total_reduction = u128_to_f64(G) / u64_to_f64(n);
  p.share = 0.0;
  per[k] = p;
}

__global__ void k_sp_total(u32 nk, u32 n, u32 I, u64 excluded, u64 t_app, ta_speedup_ctx* per,
                           ta_speedup_total* tot) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  u128 sumB = 0, sumG = 0;
  for (u32 k = 0; k < nk; ++k) {
    sumB += per[k].B;
    sumG += ((u128)per[k].G_hi << 64) | per[k].G_lo;
  }
  for (u32 k = 0; k < nk; ++k)
    per[k].share = (sumB == 0) ? 0.0 : u64_to_f64(per[k].B) / u128_to_f64(sumB);
  ta_speedup_total t;
  t.i_star = I;
  t.reserved = 0;
  t.excluded_iterations = excluded;
  t.sum_G_lo = (u64)sumG;
  t.sum_G_hi = (u64)(sumG >> 64);
  t.t_app = t_app;
  t.total_reduction = u128_to_f64(sumG) / u64_to_f64(n);
  t.speedup_fraction = (t_app == 0) ? 0.0 : u128_to_f64(sumG) / u128_to_f64((u128)n * t_app);
  *tot = t;
}

}  // namespace

namespace {

// The speedup's parts over ranks S (n of them), contexts dK[nk] and
// iterations i < I: the cells (per (i, k) sum, max and 128-bit sum of
// squares over ranks) and every context's pairwise sum of per-rank CV terms.
struct SpeedupParts {
  u64 *gs, *gm, *gl, *gh;
  double* wsum;
};

ta_status speedup_parts(ta_experiment* e, Pool& tmp, const Launch& L, const u32* dS, u32 n,
                        const u32* dK, u32 nk, u32 I, u32* status, SpeedupParts& sp) {
  ta_ctx* c = e->ctx;
  u32* kmap;
  TRY(tmp.get_n(e->C, &kmap, "kmap"));
  cudaMemsetAsync(kmap, 0xFF, (size_t)e->C * 4, c->stream);
  k_slot_map<<<blocks(nk), 256, 0, L.stream>>>(dK, nk, e->C, kmap);
  L.count();
  const u64 ncell = std::max<u64>(1, (u64)I * nk);
  u64 *&gs = sp.gs, *&gm = sp.gm, *&gl = sp.gl, *&gh = sp.gh;
  double* cvw;
  TRY(tmp.get_n(ncell, &gs, "cells"));
  TRY(tmp.get_n(ncell, &gm, "cells"));
  TRY(tmp.get_n(ncell, &gl, "cells"));
  TRY(tmp.get_n(ncell, &gh, "cells"));
  TRY(tmp.get_n(std::max<u64>(1, (u64)n * nk), &cvw, "cv terms"));
  cudaMemsetAsync(gs, 0, ncell * 8, c->stream);
  cudaMemsetAsync(gm, 0, ncell * 8, c->stream);
  cudaMemsetAsync(gl, 0, ncell * 8, c->stream);
  cudaMemsetAsync(gh, 0, ncell * 8, c->stream);
  if (I > 0) {
    const size_t map_smem = e->C <= SP_SMAP ? (size_t)(e->C + 15) / 16 * 16 : 0;
    const int grid = std::max(1, std::min<int>(c->num_sms * 4, (int)((n + SP_NW - 1) / SP_NW)));
    if (map_smem)
      cudaFuncSetAttribute(k_sp_within, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)map_smem);
    // the cells and the within-rank terms are independent: the latter run on
    // the auxiliary stream, launched second so that they fill the SMs the
    // cells' last wave leaves idle
    cudaStream_t ws = fork_aux(c);
    if (!ws) ws = L.stream;
    // cells: enough warps to fill the GPU, each with a sizeable group of ranks
    const u32 n_ib = (I + SP_IB - 1) / SP_IB, n_kb = (nk + 63) / 64;
    const u64 tiles = (u64)n_ib * n_kb;
    // at most `want` warps: three full waves of two 8-warp CTAs per SM (one
    // more item than that would start a fourth wave of a few CTAs)
    const u64 want = (u64)c->num_sms * 48;
    u64 groups = std::max<u64>(1, std::min<u64>(want / tiles, (n + 63) / 64));
    const u32 group = (u32)((n + groups - 1) / groups);
    groups = (n + group - 1) / group;
    const u64 n_items = tiles * groups;
    const size_t cmap_smem = (n_kb == 1) ? map_smem : 0;
    const size_t cells_smem = cmap_smem + (size_t)SP_NW * SPC_WARP_BYTES;
    cudaFuncSetAttribute(k_sp_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cells_smem);
    k_sp_cells<<<(unsigned)((n_items + SP_NW - 1) / SP_NW), SP_NW * 32, cells_smem, L.stream>>>(
        dS, n, e->row_off, e->entry_off, e->e_ctx, e->e_time, dK, kmap, e->C, nk, I, n_ib, n_kb,
        group, n_items, (u32)cmap_smem, gs, gm, gl, gh, e->x_mom, status);
    L.count();
    for (u32 k0 = 0; k0 < nk; k0 += SP_KC) {
      k_sp_within<<<grid, SP_NW * 32, map_smem, ws>>>(
          dS, n, e->row_off, e->entry_off, e->e_ctx, e->e_time, dK, kmap, e->C, k0,
          std::min(SP_KC, nk - k0), I, e->x.off, e->x.ctx, e->x_m1, e->x_m2, e->x_mom, cvw);
      L.count();
    }
    if (ws != L.stream) join_aux(c);
  }
  double* cvw2;
  double*& wsum = sp.wsum;
  const u32 nb = (u32)(((u64)n + PW_BLOCK - 1) / PW_BLOCK);
  TRY(tmp.get_n(std::max<u64>(1, 2ull * nk * nb), &cvw2, "cv block sums"));
  TRY(tmp.get_n(nk, &wsum, "within sums"));
  cudaMemsetAsync(wsum, 0, (size_t)nk * 8, c->stream);
  if (I > 0 && n > 0) {
    double* blk = cvw2;  // [nk nb] block values, then [nk nb] of ping-pong space
    k_sp_pair_blocks<<<dim3(nk, std::min(nb, 65535u)), 256, 0, L.stream>>>(cvw, n, nb, blk);
    k_sp_pairwise<<<nk, 256, 0, L.stream>>>(blk, blk + (u64)nk * nb, nb, wsum);
    L.count(2);
  }
  return TA_OK;
}

}  // namespace

extern "C" {

ta_status ta_context_stats(ta_experiment* e, const ta_stats_args* a, ta_stats_out* o) {
  if (!e || !a || !o) return fail(TA_ERR_INVALID_ARG, "ta_context_stats: NULL argument");
  if (a->metric > 1) return fail(TA_ERR_INVALID_ARG, "metric");
  if (!metric_csr(e, a->metric)) return fail(TA_ERR_STATE, "inclusive rollup was skipped at load");
  if (a->tau_den == 0) return fail(TA_ERR_INVALID_ARG, "tau_den = 0");
  if (a->mem_kind > 1) return fail(TA_ERR_INVALID_ARG, "mem_kind");
  if (a->ranks && a->n_ranks_subset == 0) return fail(TA_ERR_INVALID_ARG, "empty rank subset");
  if (!o->stats) return fail(TA_ERR_INVALID_ARG, "stats output is NULL");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.stats_ms);
  Pool tmp{c, {}};
  struct Rel {
    Pool& p;
    ~Rel() {
      cudaStreamSynchronize(p.ctx->stream);
      p.release();
    }
  } rel{tmp};
  const u32 n = a->ranks ? a->n_ranks_subset : e->R;
  const u32 nk = a->ctxs ? a->n_ctxs : e->C;
  const u32 *dS, *dK;
  TRY(to_device(c, tmp, a->ranks, a->ranks ? n : 0, a->mem_kind, &dS, "rank subset"));
  TRY(to_device(c, tmp, a->ctxs, a->ctxs ? nk : 0, a->mem_kind, &dK, "ctx subset"));
  u32* status;
  TRY(tmp.get_n(1, &status, "status"));
  TRY(check_subset(c, L, dS, n, e->R, status, "rank subset"));
  TRY(check_subset(c, L, dK, nk, e->C, status, "ctx subset"));
  const Csr* m = metric_csr(e, a->metric);
  double* dz = nullptr;
  if (o->z) {
    if (a->mem_kind == TA_MEM_DEVICE) dz = o->z;
    else TRY(tmp.get_n(std::max<u64>(m->nnz, 1), &dz, "z"));
  }
  StatsRun R;
  // one context given on the host (already checked against n_ctx): the
  // binary-search form
  const u32 single = (a->ctxs && nk == 1 && a->mem_kind == TA_MEM_HOST) ? a->ctxs[0] : NONE32;
  TRY(stats_run(e, tmp, a->metric, dS, n, dK, a->ctxs ? nk : 0, a->tau_num, a->tau_den,
                o->outlier_cap, dz, nullptr, R, true, single));
  o->n_outliers = R.n_out;
  const bool fits = R.n_out <= o->outlier_cap;
  ta_outlier* dout = nullptr;
  if (fits && R.kept > 0 && o->outliers) {
    if (a->mem_kind == TA_MEM_DEVICE) dout = o->outliers;
    else TRY(tmp.get_n(R.kept, &dout, "outliers"));
    k_write_outliers<<<blocks(R.kept), 256, 0, L.stream>>>(R.keys, R.zs, R.kept, dout, dK, 0);
    L.count();
    if (a->mem_kind == TA_MEM_HOST) TRY(copy(c, o->outliers, dout, R.kept * sizeof(ta_outlier)));
  }
  TRY(copy(c, o->stats, R.stats, (size_t)R.n_slots * sizeof(ta_ctx_stats)));
  if (o->z && a->mem_kind == TA_MEM_HOST) TRY(copy(c, o->z, dz, m->nnz * 8));
  TRY(sync_check(c, "ta_context_stats"));
  if (!fits)
    return fail(TA_ERR_CAPACITY, "%llu outliers, capacity %llu",
                (unsigned long long)R.n_out, (unsigned long long)o->outlier_cap);
  return TA_OK;
}

ta_status ta_topology_rollup(ta_experiment* e, const ta_topology* t, const ta_topo_args* a,
                             ta_topo_out* o) {
  if (!e || !t || !a || !o) return fail(TA_ERR_INVALID_ARG, "ta_topology_rollup: NULL argument");
  if (a->metric > 1 || !metric_csr(e, a->metric))
    return fail(a->metric > 1 ? TA_ERR_INVALID_ARG : TA_ERR_STATE, "metric");
  if (a->ctx >= e->C) return fail(TA_ERR_INVALID_ARG, "ctx >= n_ctx");
  if (a->min_ranks == 0) return fail(TA_ERR_INVALID_ARG, "min_ranks = 0");
  if (a->tau_den == 0) return fail(TA_ERR_INVALID_ARG, "tau_den = 0");
  if (!t->node_of_rank || !t->rack_of_node || !t->chassis_of_node || t->n_nodes == 0 ||
      t->n_racks == 0 || t->n_chassis == 0)
    return fail(TA_ERR_INVALID_ARG, "topology arrays");
  if (a->ranks && a->n_ranks_subset == 0) return fail(TA_ERR_INVALID_ARG, "empty rank subset");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.topology_ms);
  Pool tmp{c, {}};
  struct Rel {
    Pool& p;
    ~Rel() {
      cudaStreamSynchronize(p.ctx->stream);
      p.release();
    }
  } rel{tmp};
  const u32 n = a->ranks ? a->n_ranks_subset : e->R;
  const u32 nn = t->n_nodes, nc = t->n_chassis, nr = t->n_racks;
  const u32 *dS, *dnode, *drack, *dch;
  TRY(to_device(c, tmp, a->ranks, a->ranks ? n : 0, o->mem_kind, &dS, "rank subset"));
  TRY(to_device(c, tmp, t->node_of_rank, e->R, t->mem_kind, &dnode, "node_of_rank"));
  TRY(to_device(c, tmp, t->rack_of_node, nn, t->mem_kind, &drack, "rack_of_node"));
  TRY(to_device(c, tmp, t->chassis_of_node, nn, t->mem_kind, &dch, "chassis_of_node"));
  u32* status;
  TRY(tmp.get_n(1, &status, "status"));
  TRY(check_subset(c, L, dS, n, e->R, status, "rank subset"));
  cudaMemsetAsync(status, 0, 4, c->stream);
  // ids out of range are reported at the end (the kernels below skip them)
  k_topo_check<<<blocks(std::max(e->R, nn)), 256, 0, L.stream>>>(dnode, e->R, nn, drack, nr, dch,
                                                                  nc, status);
  L.count();
  uint8_t* rank_flag;
  TRY(tmp.get_n(e->R, &rank_flag, "rank flags"));
  cudaMemsetAsync(rank_flag, 0, e->R, c->stream);
  u32* dk;
  TRY(tmp.get_n(1, &dk, "ctx"));
  TRY(copy(c, dk, &a->ctx, 4));
  StatsRun R;
  TRY(stats_run(e, tmp, a->metric, dS, n, dk, 1, a->tau_num, a->tau_den, 0, nullptr, rank_flag, R,
                false, a->ctx));
  // outputs on the device (staged when the caller wants host memory)
  const bool dev = o->mem_kind == TA_MEM_DEVICE;
  u32 *no, *nrk, *cf, *cn, *rf, *rn, *fr, *cnt;
  unsigned long long *nsum, *csum, *rsum;
  uint8_t* nf;
  auto pick = [&](auto* user, auto** out, u64 cnt_, const char* w) -> ta_status {
    using T = std::remove_pointer_t<std::remove_reference_t<decltype(*out)>>;
    if (dev && user) {
      *out = (T*)user;
      return TA_OK;
    }
    return tmp.get_n(std::max<u64>(cnt_, 1), out, w);
  };
  TRY(pick(o->node_outliers, &no, nn, "node outliers"));
  TRY(pick((unsigned long long*)o->node_sum, &nsum, nn, "node sum"));
  TRY(pick(o->node_ranks, &nrk, nn, "node ranks"));
  TRY(pick(o->node_flag, &nf, nn, "node flag"));
  TRY(pick(o->chassis_flagged, &cf, nc, "chassis"));
  TRY(pick(o->chassis_nodes, &cn, nc, "chassis"));
  TRY(pick((unsigned long long*)o->chassis_sum, &csum, nc, "chassis"));
  TRY(pick(o->rack_flagged, &rf, nr, "rack"));
  TRY(pick(o->rack_nodes, &rn, nr, "rack"));
  TRY(pick((unsigned long long*)o->rack_sum, &rsum, nr, "rack"));
  TRY(pick(o->flagged_racks, &fr, nr, "flagged racks"));
  TRY(tmp.get_n(1, &cnt, "count"));
  cudaMemsetAsync(no, 0, (size_t)nn * 4, c->stream);
  cudaMemsetAsync(nsum, 0, (size_t)nn * 8, c->stream);
  cudaMemsetAsync(nrk, 0, (size_t)nn * 4, c->stream);
  cudaMemsetAsync(cf, 0, (size_t)nc * 4, c->stream);
  cudaMemsetAsync(cn, 0, (size_t)nc * 4, c->stream);
  cudaMemsetAsync(csum, 0, (size_t)nc * 8, c->stream);
  cudaMemsetAsync(rf, 0, (size_t)nr * 4, c->stream);
  cudaMemsetAsync(rn, 0, (size_t)nr * 4, c->stream);
  cudaMemsetAsync(rsum, 0, (size_t)nr * 8, c->stream);
  const Csr* m = metric_csr(e, a->metric);
  k_topo_nodes<<<blocks(n), 256, 0, L.stream>>>(dS, n, m->off, m->ctx, m->time, a->ctx, rank_flag,
                                                dnode, no, nsum, nrk, nn);
  k_topo_up<<<blocks(nn), 256, 0, L.stream>>>(nn, no, nsum, a->min_ranks, drack, dch, nf, cf, cn,
                                              csum, rf, rn, rsum, nc, nr);
  k_topo_racks<<<1, 256, 0, L.stream>>>(nr, rf, fr, cnt);
  L.count(3);
  u32 nfr = 0, hs = 0;
  TRY(copy(c, &nfr, cnt, 4));
  TRY(copy(c, &hs, status, 4));
  if (!dev) {
    if (o->node_outliers) TRY(copy(c, o->node_outliers, no, (size_t)nn * 4));
    if (o->node_sum) TRY(copy(c, o->node_sum, nsum, (size_t)nn * 8));
    if (o->node_ranks) TRY(copy(c, o->node_ranks, nrk, (size_t)nn * 4));
    if (o->node_flag) TRY(copy(c, o->node_flag, nf, nn));
    if (o->chassis_flagged) TRY(copy(c, o->chassis_flagged, cf, (size_t)nc * 4));
    if (o->chassis_nodes) TRY(copy(c, o->chassis_nodes, cn, (size_t)nc * 4));
    if (o->chassis_sum) TRY(copy(c, o->chassis_sum, csum, (size_t)nc * 8));
    if (o->rack_flagged) TRY(copy(c, o->rack_flagged, rf, (size_t)nr * 4));
    if (o->rack_nodes) TRY(copy(c, o->rack_nodes, rn, (size_t)nr * 4));
    if (o->rack_sum) TRY(copy(c, o->rack_sum, rsum, (size_t)nr * 8));
    if (o->flagged_racks) TRY(copy(c, o->flagged_racks, fr, (size_t)nr * 4));
  }
  TRY(sync_check(c, "ta_topology_rollup"));
  if (hs) return fail(TA_ERR_INVALID_ARG, "topology ids out of range");
  o->n_flagged_racks = nfr;
  return TA_OK;
}

ta_status ta_potential_speedup(ta_experiment* e, const ta_speedup_args* a, ta_speedup_out* o) {
  if (!e || !a || !o) return fail(TA_ERR_INVALID_ARG, "ta_potential_speedup: NULL argument");
  if (!a->ctxs || a->n_ctxs == 0) return fail(TA_ERR_INVALID_ARG, "empty context set");
  if (a->ranks && a->n_ranks_subset == 0) return fail(TA_ERR_INVALID_ARG, "empty rank subset");
  if (!o->per_ctx || !o->total) return fail(TA_ERR_INVALID_ARG, "outputs NULL");
  if (a->mem_kind > 1) return fail(TA_ERR_INVALID_ARG, "mem_kind");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.speedup_ms);
  Pool tmp{c, {}};
  struct Rel {
    Pool& p;
    ~Rel() {
      cudaStreamSynchronize(p.ctx->stream);
      p.release();
    }
  } rel{tmp};
  const u32 n = a->ranks ? a->n_ranks_subset : e->R;
  const u32 nk = a->n_ctxs;
  const u32 *dS, *dK;
  TRY(to_device(c, tmp, a->ranks, a->ranks ? n : 0, a->mem_kind, &dS, "rank subset"));
  TRY(to_device(c, tmp, a->ctxs, nk, a->mem_kind, &dK, "ctx set"));
  u32* status;  // [0] the cells kernel's stalled copies, [1] the context set's check
  TRY(tmp.get_n(2, &status, "status"));
  // rank ids index the tensor: checked before any kernel reads them
  TRY(check_subset(c, L, dS, n, e->R, status, "rank subset"));
  cudaMemsetAsync(status, 0, 8, c->stream);
  // context ids only select outputs (the maps skip ids >= C): checked on the
  // device here, read at the final wait
  k_check_sorted<<<blocks(nk), 256, 0, L.stream>>>(dK, nk, e->C, status + 1);
  L.count();
  u64 h[3];  // I*, sum n_iter, max span over S
  if (!dS && e->has_iter_summary) {  // all ranks: kept from the load
    h[0] = e->istar_all;
    h[1] = e->sum_iter_all;
    h[2] = e->max_span;
  } else {
    u64* meta;
    TRY(tmp.get_n(4, &meta, "speedup meta"));
    cudaMemsetAsync(meta, 0, 32, c->stream);
    cudaMemsetAsync(meta, 0xFF, 4, c->stream);
    k_sp_istar<<<blocks(n), 256, 0, L.stream>>>(dS, n, e->n_iter, e->span, (u32*)meta,
                                                (unsigned long long*)meta + 1,
                                                (unsigned long long*)meta + 2);
    L.count();
    TRY(copy(c, h, meta, sizeof h));
    TRY(sync_check(c, "speedup I*"));
  }
  const u32 I = (u32)h[0];
  const u64 excluded = h[1] - (u64)n * I;
  const u64 t_app = a->app_time_ns ? a->app_time_ns : h[2];
  SpeedupParts sp;
  TRY(speedup_parts(e, tmp, L, dS, n, dK, nk, I, status, sp));
  ta_speedup_ctx* dper;
  ta_speedup_total* dtot;
  if (a->mem_kind == TA_MEM_DEVICE) {
    dper = o->per_ctx;
    dtot = o->total;
  } else {
    TRY(tmp.get_n(nk, &dper, "per ctx"));
    TRY(tmp.get_n(1, &dtot, "total"));
  }
  k_sp_final_k<<<(unsigned)((nk + 3) / 4), 128, 0, L.stream>>>(nk, n, I, sp.gs, sp.gm, sp.gl,
                                                                  sp.gh, sp.wsum,
                                                                  dper);
  k_sp_total<<<1, 1, 0, L.stream>>>(nk, n, I, excluded, t_app, dper, dtot);
  L.count(2);
  if (a->mem_kind == TA_MEM_HOST) {
    TRY(copy(c, o->per_ctx, dper, (size_t)nk * sizeof(ta_speedup_ctx)));
    TRY(copy(c, o->total, dtot, sizeof(ta_speedup_total)));
  }
  u32 f[2] = {0, 0};
  TRY(copy(c, f, status, 8));
  TRY(sync_check(c, "ta_potential_speedup"));
  if (f[1]) return fail(TA_ERR_INVALID_ARG, "ctx set must be sorted, unique and in range");
  return status_from_flags(f[0], "ta_potential_speedup");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free statistics.  Callers that may not allocate device memory
// (a host runtime that owns all device memory and passes only its own
// buffers, or a fixed-budget allocator that forbids growth) get every temporary from one
// file-scope device array instead of the allocator.  The array lives in every
// GPU that loads this library until the process exits.
namespace {

constexpr u64 NA_MAX_CTX = 1u << 16;       // contexts
constexpr u64 NA_MAX_OUTLIERS = 1u << 16;  // outlier capacity (power of two)
// slot map u32[C] + ten per-context partial arrays (72 B per context) +
// outlier keys and z (16 B each) + counters.
constexpr u64 NA_BYTES = NA_MAX_CTX * 4 + NA_MAX_CTX * 72 + NA_MAX_OUTLIERS * 16 + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// The caller's CSR, checked before any kernel indexes the slot map or the
// partials with it: rank r's offsets non-decreasing (F_INVALID) and every
// context id below n_ctx (F_BAD_CTX).  Warp per rank of the subset.
__global__ void k_check_csr(const u32* __restrict__ S, u32 n, const u64* __restrict__ off,
                            const u32* __restrict__ ctx, u32 n_ctx, u32* status) {
  const int lane = threadIdx.x & 31;
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  u32 fl = 0;
  for (u32 i = gw; i < n; i += nw) {
    const u32 r = rank_at(S, i);
    const u64 E0 = off[r], E1 = off[r + 1];
    if (E1 < E0) {
      fl |= F_INVALID;
      continue;
    }
    for (u64 j = E0 + lane; j < E1; j += 32)
      if (ctx[j] >= n_ctx) fl |= F_BAD_CTX;
  }
  fl = __reduce_or_sync(FULL, fl);
  if (lane == 0 && fl) flag(status, fl);
}

constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_noalloc_ptr[NA_MAX_DEVICES];
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is not a device address).
ta_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
  if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(TA_ERR_INVALID_ARG, "device %d", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return TA_OK;
}

}  // namespace

extern "C" ta_status ta_context_stats_noalloc(void* cuda_stream, const uint64_t* off,
                                              const uint32_t* ctx, const uint64_t* time,
                                              uint32_t n_ranks, uint32_t n_ctx,
                                              const uint32_t* ranks, uint32_t n_ranks_subset,
                                              uint32_t tau_num, uint32_t tau_den,
                                              ta_ctx_stats* stats, ta_outlier* outliers,
                                              uint64_t outlier_cap, uint64_t* n_outliers) {
  if (!off || !ctx || !time || !stats || !n_outliers || (outlier_cap && !outliers))
    return fail(TA_ERR_INVALID_ARG, "ta_context_stats_noalloc: NULL argument");
  if (n_ranks == 0 || n_ctx == 0) return fail(TA_ERR_INVALID_ARG, "n_ranks and n_ctx must be > 0");
  if (n_ctx > NA_MAX_CTX)
    return fail(TA_ERR_INVALID_ARG,
                "ta_context_stats_noalloc: n_ctx = %u exceeds the fixed maximum %llu", n_ctx,
                (unsigned long long)NA_MAX_CTX);
  if (outlier_cap > NA_MAX_OUTLIERS)
    return fail(TA_ERR_INVALID_ARG,
                "ta_context_stats_noalloc: outlier_cap = %llu exceeds the fixed maximum %llu",
                (unsigned long long)outlier_cap, (unsigned long long)NA_MAX_OUTLIERS);
  if (tau_den == 0) return fail(TA_ERR_INVALID_ARG, "tau_den = 0");
  if (ranks && n_ranks_subset == 0) return fail(TA_ERR_INVALID_ARG, "empty rank subset");
  unsigned char* base;
  TRY(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long launches = 0;
  int num_sms = 1;
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr == cudaSuccess)
    derr = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (derr != cudaSuccess) return cuda_fail(derr, "ta_context_stats_noalloc (device)");
  Launch L{st, num_sms, &launches};
  const u64 C = n_ctx;
  // carve the scratch array
  u32* slot_of_ctx = (u32*)base;
  unsigned char* q = base + NA_MAX_CTX * 4;
  Partials P;
  P.present = (u32*)q;
  q += NA_MAX_CTX * 4;
  P.argmax = (u32*)q;
  q += NA_MAX_CTX * 4;
  P.mn = (u64*)q;
  q += NA_MAX_CTX * 8;
  P.mx = (u64*)q;
  q += NA_MAX_CTX * 8;
  P.s1 = (u64*)q;
  q += NA_MAX_CTX * 8;
  P.s2lo = (u64*)q;
  q += NA_MAX_CTX * 8;
  P.s2hi = (u64*)q;
  q += NA_MAX_CTX * 8;
  P.sd = (double*)q;
  q += NA_MAX_CTX * 8;
  P.Mlo = (u64*)q;
  q += NA_MAX_CTX * 8;
  P.Mhi = (u64*)q;
  q += NA_MAX_CTX * 8;
  u64* keys = (u64*)q;
  q += NA_MAX_OUTLIERS * 8;
  double* zs = (double*)q;
  q += NA_MAX_OUTLIERS * 8;
  unsigned long long* n_out = (unsigned long long*)q;
  u32* status = (u32*)(q + 8);
  const u32 n = ranks ? n_ranks_subset : n_ranks;
  // everything that accumulates starts from zero (the array keeps the last
  // call's contents)
  const int grid = std::max(1, std::min<int>(num_sms * 4, (int)((n + 7) / 8)));
  cudaError_t err = cudaMemsetAsync(q, 0, 16, st);
  if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
  // the subset and the caller's CSR are checked before any kernel reads
  // through them (a context id >= n_ctx would index past the slot map)
  if (ranks) {
    k_check_sorted<<<blocks(n), 256, 0, st>>>(ranks, n, n_ranks, status);
    L.count();
    err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc (subset check)");
    u32 hs = 0;
    err = cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc");
    if (hs) return fail(TA_ERR_INVALID_ARG, "rank subset must be sorted, unique and < n_ranks");
  }
  k_check_csr<<<grid, 256, 0, st>>>(ranks, n, off, ctx, n_ctx, status);
  L.count();
  err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc (CSR check)");
  {
    u32 hs = 0;
    err = cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc");
    if (hs & F_INVALID) return fail(TA_ERR_INVALID_ARG, "off decreases within the CSR");
    if (hs & F_BAD_CTX) return fail(TA_ERR_BAD_CTX, "a context id of the CSR is >= n_ctx");
  }
  struct Fill {
    void* p;
    int v;
    size_t bytes;
  };
  const Fill fills[] = {{slot_of_ctx, 0xFF, C * 4}, {P.present, 0, C * 4}, {P.mn, 0xFF, C * 8},
                        {P.mx, 0, C * 8},           {P.s1, 0, C * 8},      {P.s2lo, 0, C * 8},
                        {P.s2hi, 0, C * 8}};
  for (const Fill& f : fills) {
    err = cudaMemsetAsync(f.p, f.v, f.bytes, st);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
  }
  const u64 kcap = std::max<u64>(1, outlier_cap);
  k_slot_map<<<blocks(C), 256, 0, st>>>(nullptr, 0, n_ctx, slot_of_ctx);
  k_stats_partial<<<grid, STATS_NT, 0, st>>>(ranks, n, off, ctx, time, slot_of_ctx, P, SetMap{});
  k_stats_finalize<<<blocks(C), 256, 0, st>>>((u32)C, n, ranks, P, stats, SetMap{});
  k_stats_z<<<grid, 256, 0, st>>>(ranks, n, off, ctx, time, slot_of_ctx, P, tau_num, tau_den,
                                  nullptr, keys, zs, kcap, n_out, nullptr, SetMap{}, 0, NONE32);
  k_stats_argmax<<<blocks(C), 256, 0, st>>>((u32)C, P.argmax, stats);
  L.count(5);
  err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc (launch)");
  u64 h = 0;
  err = cudaMemcpyAsync(&h, n_out, 8, cudaMemcpyDeviceToHost, st);
  if (err != cudaSuccess) return cuda_fail(err, "cudaMemcpyAsync");
  err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc");
  *n_outliers = h;
  if (h > outlier_cap)
    return fail(TA_ERR_CAPACITY, "%llu outliers, capacity %llu", (unsigned long long)h,
                (unsigned long long)outlier_cap);
  if (h > 0) {
    sort_pairs(L, keys, zs, h);  // the key buffer holds NA_MAX_OUTLIERS (a power of two)
    k_write_outliers<<<blocks(h), 256, 0, st>>>(keys, zs, h, outliers, nullptr, 0);
    L.count();
  }
  err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc (sort)");
  err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return cuda_fail(err, "ta_context_stats_noalloc");
  return TA_OK;
}

// ---------------------------------------------------------------------------
// Sharded form: reducible partials of the cross-rank steps and their
// finishing from merged partials (one exchange: SUM, MIN or MAX element-wise;
// 128-bit sums as four 32-bit limbs in 64-bit words).
namespace {

__device__ __forceinline__ void put_limbs(u64* q, u128 v) {
  q[0] = (u64)(v & 0xFFFFFFFFull);
  q[1] = (u64)((v >> 32) & 0xFFFFFFFFull);
  q[2] = (u64)((v >> 64) & 0xFFFFFFFFull);
  q[3] = (u64)(v >> 96);
}
// Sum of limb l times 2^(32 l); merged limbs may exceed 32 bits (carried here).
__device__ __forceinline__ u128 get_limbs(const u64* q) {
  return (u128)q[0] + ((u128)q[1] << 32) + ((u128)q[2] << 64) + ((u128)q[3] << 96);
}

// Per context of the shard's partials: present, S1, S2 limbs; min (absent
// ranks count 0) and max.
__global__ void k_shard_export(u32 ns, Partials P, u32 R, u64* sums, u64* mins, u64* maxs) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const u32 present = P.present[s];
  sums[6 * (u64)s] = present;
  sums[6 * (u64)s + 1] = P.s1[s];
  put_limbs(sums + 6 * (u64)s + 2, ((u128)P.s2hi[s] << 64) | P.s2lo[s]);
  mins[s] = present < R ? 0ull : P.mn[s];
  maxs[s] = P.mx[s];
}

// Merged partials -> the finishing kernels' partials (slot s = ctx c0 + s).
__global__ void k_shard_import(u32 ns, u32 c0, const u64* sums, const u64* mins, const u64* maxs,
                               Partials P) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const u64 c = (u64)c0 + s;
  P.present[s] = (u32)sums[6 * c];
  P.s1[s] = sums[6 * c + 1];
  const u128 S2 = get_limbs(sums + 6 * c + 2);
  P.s2lo[s] = (u64)S2;
  P.s2hi[s] = (u64)(S2 >> 64);
  P.mn[s] = mins[c];
  P.mx[s] = maxs[c];
}

// Argmax candidates as global rank ids (none: 0xFFFFFFFF), also written into
// the statistics records.
__global__ void k_shard_argmax(u32 ns, const u32* argmax, u32 rank_base, u32* out,
                               ta_ctx_stats* stats) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const u32 a = argmax[s] == NONE32 ? NONE32 : argmax[s] + rank_base;
  out[s] = a;
  stats[s].argmax = a;
}

__global__ void k_set_argmax(u32 n, const u32* argmax, ta_ctx_stats* stats) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) stats[s].argmax = argmax[s];
}

// Node partials of one context over the shard's ranks: outlier ranks, sum of
// x, ranks (u64 SUM-reducible).
__global__ void k_shard_nodes(u32 R, const u64* off, const u32* ctx, const u64* time, u32 c,
                              const uint8_t* rank_flag, const u32* node_of_rank,
                              unsigned long long* parts, u32 nn) {
  const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const u32 nd = node_of_rank[r];
  const u64 x = csr_lookup(off, ctx, time, r, c);
  if (rank_flag[r]) atomicAdd(&parts[nd], 1ull);
  atomicAdd(&parts[(u64)nn + nd], (unsigned long long)x);
  atomicAdd(&parts[2 * (u64)nn + nd], 1ull);
}

__global__ void k_nodes_unpack(u32 nn, const u64* parts, u32* node_out,
                               unsigned long long* node_sum, u32* node_ranks) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  node_out[i] = (u32)parts[i];
  node_sum[i] = parts[(u64)nn + i];
  node_ranks[i] = (u32)parts[2 * (u64)nn + i];
}

// Speedup cells -> reducible (sum, sum of squares as limbs; max apart), and back.
__global__ void k_cells_export(u64 ncell, const u64* gs, const u64* gl, const u64* gh, u64* cells) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  cells[5 * i] = gs[i];
  put_limbs(cells + 5 * i + 1, ((u128)gh[i] << 64) | gl[i]);
}
__global__ void k_cells_import(u64 ncell, const u64* cells, u64* gs, u64* gl, u64* gh) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  gs[i] = cells[5 * i];
  const u128 q = get_limbs(cells + 5 * i + 1);
  gl[i] = (u64)q;
  gh[i] = (u64)(q >> 64);
}

// The finishing kernels' partial arrays for ns slots.
ta_status alloc_partials(Pool& tmp, u32 ns, Partials& P) {
  TRY(tmp.get_n(ns, &P.present, "partials"));
  TRY(tmp.get_n(ns, &P.mn, "partials"));
  TRY(tmp.get_n(ns, &P.mx, "partials"));
  TRY(tmp.get_n(ns, &P.s1, "partials"));
  TRY(tmp.get_n(ns, &P.s2lo, "partials"));
  TRY(tmp.get_n(ns, &P.s2hi, "partials"));
  TRY(tmp.get_n(ns, &P.argmax, "partials"));
  TRY(tmp.get_n(ns, &P.sd, "partials"));
  TRY(tmp.get_n(ns, &P.Mlo, "partials"));
  TRY(tmp.get_n(ns, &P.Mhi, "partials"));
  return TA_OK;
}

ta_status shard_check(const ta_experiment* e, const ta_shard_merged* m) {
  if (!m || !m->sums || !m->mins || !m->maxs) return fail(TA_ERR_INVALID_ARG, "merged partials NULL");
  if (m->metric > 1 || !metric_csr(e, m->metric))
    return fail(m->metric > 1 ? TA_ERR_INVALID_ARG : TA_ERR_STATE, "metric");
  if (m->tau_den == 0) return fail(TA_ERR_INVALID_ARG, "tau_den = 0");
  if (m->n_total < e->R || (u64)m->rank_base + e->R > m->n_total)
    return fail(TA_ERR_INVALID_ARG, "shard ranks [%u, %llu) outside the job's %u ranks",
                m->rank_base, (unsigned long long)m->rank_base + e->R, m->n_total);
  return TA_OK;
}

struct ShardCall {
  Pool tmp;
  explicit ShardCall(ta_ctx* c) : tmp{c, {}} {}
  ~ShardCall() {
    cudaStreamSynchronize(tmp.ctx->stream);
    tmp.release();
  }
};

}  // namespace

extern "C" {

ta_status ta_shard_stats_partials(ta_experiment* e, uint32_t metric, const ta_shard_stats_parts* o) {
  if (!e || !o || !o->sums || !o->mins || !o->maxs)
    return fail(TA_ERR_INVALID_ARG, "ta_shard_stats_partials: NULL argument");
  if (metric > 1 || !metric_csr(e, metric))
    return fail(metric > 1 ? TA_ERR_INVALID_ARG : TA_ERR_STATE, "metric");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.stats_ms);
  ShardCall call(c);
  Pool& tmp = call.tmp;
  const Csr* m = metric_csr(e, metric);
  const u32 C = e->C;
  Partials P;
  TRY(alloc_partials(tmp, C, P));
  u32* slot_of_ctx;
  TRY(tmp.get_n(C, &slot_of_ctx, "slot map"));
  k_slot_map<<<blocks(C), 256, 0, L.stream>>>(nullptr, 0, C, slot_of_ctx);
  cudaMemsetAsync(P.present, 0, (size_t)C * 4, c->stream);
  cudaMemsetAsync(P.mn, 0xFF, (size_t)C * 8, c->stream);
  cudaMemsetAsync(P.mx, 0, (size_t)C * 8, c->stream);
  cudaMemsetAsync(P.s1, 0, (size_t)C * 8, c->stream);
  cudaMemsetAsync(P.s2lo, 0, (size_t)C * 8, c->stream);
  cudaMemsetAsync(P.s2hi, 0, (size_t)C * 8, c->stream);
  const int grid = std::max(1, std::min<int>(c->num_sms * 4, (int)((e->R + 7) / 8)));
  k_stats_partial<<<grid, STATS_NT, 0, L.stream>>>(nullptr, e->R, m->off, m->ctx, m->time,
                                                   slot_of_ctx, P, SetMap{});
  k_shard_export<<<blocks(C), 256, 0, L.stream>>>(C, P, e->R, o->sums, o->mins, o->maxs);
  L.count(3);
  return sync_check(c, "ta_shard_stats_partials");
}

ta_status ta_shard_stats_finalize(ta_experiment* e, const ta_shard_merged* mg,
                                  ta_shard_stats_out* o) {
  if (!e || !o || !o->stats || !o->argmax || (o->outlier_cap && !o->outliers))
    return fail(TA_ERR_INVALID_ARG, "ta_shard_stats_finalize: NULL argument");
  TRY(shard_check(e, mg));
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.stats_ms);
  ShardCall call(c);
  Pool& tmp = call.tmp;
  const Csr* m = metric_csr(e, mg->metric);
  const u32 C = e->C;
  Partials P;
  TRY(alloc_partials(tmp, C, P));
  u32* slot_of_ctx;
  TRY(tmp.get_n(C, &slot_of_ctx, "slot map"));
  k_slot_map<<<blocks(C), 256, 0, L.stream>>>(nullptr, 0, C, slot_of_ctx);
  k_shard_import<<<blocks(C), 256, 0, L.stream>>>(C, 0, mg->sums, mg->mins, mg->maxs, P);
  k_stats_finalize<<<blocks(C), 256, 0, L.stream>>>(C, mg->n_total, nullptr, P, o->stats,
                                                    SetMap{});
  const u64 kcap = std::max<u64>(1, o->outlier_cap);
  u64 P2 = 1;
  while (P2 < kcap) P2 <<= 1;
  u64* keys;
  double* zs;
  unsigned long long* n_out;
  TRY(tmp.get_n(P2, &keys, "outlier keys"));
  TRY(tmp.get_n(P2, &zs, "outlier z"));
  TRY(tmp.get_n(1, &n_out, "outlier count"));
  cudaMemsetAsync(n_out, 0, 8, c->stream);
  const int grid = std::max(1, std::min<int>(c->num_sms * 4, (int)((e->R + 7) / 8)));
  k_stats_z<<<grid, 256, 0, L.stream>>>(nullptr, e->R, m->off, m->ctx, m->time, slot_of_ctx, P,
                                        mg->tau_num, mg->tau_den, nullptr, keys, zs, kcap, n_out,
                                        nullptr, SetMap{}, mg->n_total, NONE32);
  k_shard_argmax<<<blocks(C), 256, 0, L.stream>>>(C, P.argmax, mg->rank_base, o->argmax,
                                                  o->stats);
  L.count(5);
  u64 h = 0;
  TRY(copy(c, &h, n_out, 8));
  TRY(sync_check(c, "ta_shard_stats_finalize"));
  o->n_outliers = h;
  if (h > o->outlier_cap)
    return fail(TA_ERR_CAPACITY, "%llu outliers, capacity %llu", (unsigned long long)h,
                (unsigned long long)o->outlier_cap);
  if (h > 0) {
    sort_pairs(L, keys, zs, h);
    k_write_outliers<<<blocks(h), 256, 0, L.stream>>>(keys, zs, h, o->outliers, nullptr,
                                                      mg->rank_base);
    L.count();
  }
  return sync_check(c, "ta_shard_stats_finalize");
}

ta_status ta_shard_set_argmax(ta_ctx* c, ta_ctx_stats* stats, const uint32_t* argmax,
                              uint32_t n_ctx) {
  if (!c || !stats || !argmax) return fail(TA_ERR_INVALID_ARG, "ta_shard_set_argmax: NULL argument");
  cudaSetDevice(c->device);
  k_set_argmax<<<blocks(n_ctx), 256, 0, c->stream>>>(n_ctx, argmax, stats);
  ++c->launches;
  return sync_check(c, "ta_shard_set_argmax");
}

ta_status ta_shard_topology_partials(ta_experiment* e, const ta_shard_merged* mg, uint32_t ctx,
                                     const uint32_t* node_of_rank, uint32_t n_nodes,
                                     uint64_t* node_parts) {
  if (!e || !node_of_rank || !node_parts || n_nodes == 0)
    return fail(TA_ERR_INVALID_ARG, "ta_shard_topology_partials: NULL argument");
  TRY(shard_check(e, mg));
  if (ctx >= e->C) return fail(TA_ERR_INVALID_ARG, "ctx >= n_ctx");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.topology_ms);
  ShardCall call(c);
  Pool& tmp = call.tmp;
  const Csr* m = metric_csr(e, mg->metric);
  u32* status;
  TRY(tmp.get_n(1, &status, "status"));
  cudaMemsetAsync(status, 0, 4, c->stream);
  k_topo_check<<<blocks(e->R), 256, 0, L.stream>>>(node_of_rank, e->R, n_nodes, nullptr, 0,
                                                   nullptr, 0, status);
  L.count();
  u32 hs = 0;
  TRY(copy(c, &hs, status, 4));
  TRY(sync_check(c, "topology check"));
  if (hs) return fail(TA_ERR_INVALID_ARG, "node ids out of range");
  // the job's statistics of ctx (slot 0), then this shard's outlier ranks
  Partials P;
  TRY(alloc_partials(tmp, 1, P));
  u32* slot_of_ctx;
  TRY(tmp.get_n(e->C, &slot_of_ctx, "slot map"));
  cudaMemsetAsync(slot_of_ctx, 0xFF, (size_t)e->C * 4, c->stream);
  u32* dk;
  TRY(tmp.get_n(1, &dk, "ctx"));
  TRY(copy(c, dk, &ctx, 4));
  k_slot_map<<<1, 32, 0, L.stream>>>(dk, 1, e->C, slot_of_ctx);
  ta_ctx_stats* st;
  TRY(tmp.get_n(1, &st, "stats"));
  k_shard_import<<<1, 32, 0, L.stream>>>(1, ctx, mg->sums, mg->mins, mg->maxs, P);
  k_stats_finalize<<<1, 32, 0, L.stream>>>(1, mg->n_total, nullptr, P, st, SetMap{});
  uint8_t* rank_flag;
  TRY(tmp.get_n(std::max<u32>(e->R, 1), &rank_flag, "rank flags"));
  cudaMemsetAsync(rank_flag, 0, e->R, c->stream);
  u64* keys;
  double* zs;
  unsigned long long* n_out;
  TRY(tmp.get_n(1, &keys, "outlier keys"));
  TRY(tmp.get_n(1, &zs, "outlier z"));
  TRY(tmp.get_n(1, &n_out, "outlier count"));
  cudaMemsetAsync(n_out, 0, 8, c->stream);
  const int grid = std::max(1, std::min<int>(c->num_sms * 4, (int)((e->R + 7) / 8)));
  k_stats_z<<<grid, 256, 0, L.stream>>>(nullptr, e->R, m->off, m->ctx, m->time, slot_of_ctx, P,
                                        mg->tau_num, mg->tau_den, nullptr, keys, zs, 1, n_out,
                                        rank_flag, SetMap{}, mg->n_total, ctx);
  cudaMemsetAsync(node_parts, 0, (size_t)n_nodes * 24, c->stream);
  k_shard_nodes<<<blocks(e->R), 256, 0, L.stream>>>(e->R, m->off, m->ctx, m->time, ctx, rank_flag,
                                                    node_of_rank,
                                                    (unsigned long long*)node_parts, n_nodes);
  L.count(5);
  return sync_check(c, "ta_shard_topology_partials");
}

ta_status ta_topology_finalize(ta_ctx* c, const uint64_t* node_parts, const ta_topology* t,
                               uint32_t min_ranks, ta_topo_out* o) {
  if (!c || !node_parts || !t || !o || !t->rack_of_node || !t->chassis_of_node || t->n_nodes == 0 ||
      t->n_racks == 0 || t->n_chassis == 0)
    return fail(TA_ERR_INVALID_ARG, "ta_topology_finalize: NULL argument");
  if (min_ranks == 0) return fail(TA_ERR_INVALID_ARG, "min_ranks = 0");
  if (t->mem_kind != TA_MEM_DEVICE || o->mem_kind != TA_MEM_DEVICE)
    return fail(TA_ERR_INVALID_ARG, "ta_topology_finalize takes device arrays");
  if (!o->node_outliers || !o->node_sum || !o->node_ranks || !o->node_flag || !o->chassis_flagged ||
      !o->chassis_nodes || !o->chassis_sum || !o->rack_flagged || !o->rack_nodes || !o->rack_sum ||
      !o->flagged_racks)
    return fail(TA_ERR_INVALID_ARG, "ta_topology_finalize: output NULL");
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  ShardCall call(c);
  Pool& tmp = call.tmp;
  const u32 nn = t->n_nodes, nc = t->n_chassis, nr = t->n_racks;
  u32* status;
  TRY(tmp.get_n(2, &status, "status"));
  cudaMemsetAsync(status, 0, 8, c->stream);
  k_topo_check<<<blocks(nn), 256, 0, L.stream>>>(nullptr, 0, nn, t->rack_of_node, nr,
                                                 t->chassis_of_node, nc, status);
  L.count();
  u32 hs = 0;
  TRY(copy(c, &hs, status, 4));
  TRY(sync_check(c, "topology check"));
  if (hs) return fail(TA_ERR_INVALID_ARG, "topology ids out of range");
  cudaMemsetAsync(o->chassis_flagged, 0, (size_t)nc * 4, c->stream);
  cudaMemsetAsync(o->chassis_nodes, 0, (size_t)nc * 4, c->stream);
  cudaMemsetAsync(o->chassis_sum, 0, (size_t)nc * 8, c->stream);
  cudaMemsetAsync(o->rack_flagged, 0, (size_t)nr * 4, c->stream);
  cudaMemsetAsync(o->rack_nodes, 0, (size_t)nr * 4, c->stream);
  cudaMemsetAsync(o->rack_sum, 0, (size_t)nr * 8, c->stream);
  k_nodes_unpack<<<blocks(nn), 256, 0, L.stream>>>(nn, node_parts, o->node_outliers,
                                                  (unsigned long long*)o->node_sum, o->node_ranks);
  k_topo_up<<<blocks(nn), 256, 0, L.stream>>>(
      nn, o->node_outliers, (const unsigned long long*)o->node_sum, min_ranks, t->rack_of_node,
      t->chassis_of_node, o->node_flag, o->chassis_flagged, o->chassis_nodes,
      (unsigned long long*)o->chassis_sum, o->rack_flagged, o->rack_nodes,
      (unsigned long long*)o->rack_sum, nc, nr);
  k_topo_racks<<<1, 1024, 0, L.stream>>>(nr, o->rack_flagged, o->flagged_racks, status + 1);
  L.count(3);
  u32 nf = 0;
  TRY(copy(c, &nf, status + 1, 4));
  TRY(sync_check(c, "ta_topology_finalize"));
  o->n_flagged_racks = nf;
  return TA_OK;
}

ta_status ta_shard_speedup_bounds(ta_experiment* e, uint64_t* bounds) {
  if (!e || !bounds) return fail(TA_ERR_INVALID_ARG, "ta_shard_speedup_bounds: NULL argument");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  ShardCall call(c);
  Pool& tmp = call.tmp;
  u64* meta;  // [0] istar, [1] sum n_iter, [2] max span
  TRY(tmp.get_n(4, &meta, "speedup meta"));
  cudaMemsetAsync(meta, 0, 32, c->stream);
  cudaMemsetAsync(meta, 0xFF, 4, c->stream);
  k_sp_istar<<<blocks(e->R), 256, 0, L.stream>>>(nullptr, e->R, e->n_iter, e->span, (u32*)meta,
                                                 (unsigned long long*)meta + 1,
                                                 (unsigned long long*)meta + 2);
  L.count();
  u64 h[3];
  TRY(copy(c, h, meta, sizeof h));
  TRY(sync_check(c, "ta_shard_speedup_bounds"));
  bounds[0] = (u32)h[0];
  bounds[1] = h[1];
  bounds[2] = h[2];
  return TA_OK;
}

ta_status ta_shard_speedup_partials(ta_experiment* e, const uint32_t* ctxs, uint32_t nk,
                                    uint32_t i_star, const ta_shard_speedup_parts* o) {
  if (!e || !ctxs || nk == 0 || !o || !o->cells || !o->cell_max || !o->within)
    return fail(TA_ERR_INVALID_ARG, "ta_shard_speedup_partials: NULL argument");
  ta_ctx* c = e->ctx;
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  PhaseTimer call_timer(c, &c->prof.speedup_ms);
  ShardCall call(c);
  Pool& tmp = call.tmp;
  u32* status;
  TRY(tmp.get_n(1, &status, "status"));
  TRY(check_subset(c, L, ctxs, nk, e->C, status, "ctx set"));
  cudaMemsetAsync(status, 0, 4, c->stream);
  {  // every rank of the shard must hold i_star iterations
    u64 b[3];
    TRY(ta_shard_speedup_bounds(e, b));
    if (b[0] < i_star)
      return fail(TA_ERR_INVALID_ARG, "i_star = %u above the shard's fewest iterations %llu",
                  i_star, (unsigned long long)b[0]);
  }
  SpeedupParts sp;
  TRY(speedup_parts(e, tmp, L, nullptr, e->R, ctxs, nk, i_star, status, sp));
  const u64 ncell = (u64)i_star * nk;
  if (ncell) {
    k_cells_export<<<blocks(ncell), 256, 0, L.stream>>>(ncell, sp.gs, sp.gl, sp.gh, o->cells);
    L.count();
    cudaMemcpyAsync(o->cell_max, sp.gm, ncell * 8, cudaMemcpyDeviceToDevice, c->stream);
  }
  cudaMemcpyAsync(o->within, sp.wsum, (size_t)nk * 8, cudaMemcpyDeviceToDevice, c->stream);
  u32 f = 0;
  TRY(copy(c, &f, status, 4));
  TRY(sync_check(c, "ta_shard_speedup_partials"));
  return status_from_flags(f, "ta_shard_speedup_partials");
}

ta_status ta_speedup_finalize(ta_ctx* c, uint32_t nk, uint32_t n_total, uint32_t i_star,
                              uint64_t excluded, uint64_t t_app,
                              const ta_shard_speedup_parts* mg, ta_speedup_ctx* per,
                              ta_speedup_total* tot) {
  if (!c || nk == 0 || n_total == 0 || !mg || !mg->cells || !mg->cell_max || !mg->within || !per ||
      !tot)
    return fail(TA_ERR_INVALID_ARG, "ta_speedup_finalize: NULL argument");
  cudaSetDevice(c->device);
  Launch L{c->stream, c->num_sms, &c->launches};
  ShardCall call(c);
  Pool& tmp = call.tmp;
  const u64 ncell = std::max<u64>(1, (u64)i_star * nk);
  u64 *gs, *gl, *gh;
  TRY(tmp.get_n(ncell, &gs, "cells"));
  TRY(tmp.get_n(ncell, &gl, "cells"));
  TRY(tmp.get_n(ncell, &gh, "cells"));
  if (i_star) {
    k_cells_import<<<blocks(ncell), 256, 0, L.stream>>>((u64)i_star * nk, mg->cells, gs, gl, gh);
    L.count();
  }
  k_sp_final_k<<<(unsigned)((nk + 3) / 4), 128, 0, L.stream>>>(nk, n_total, i_star, gs,
                                                                  mg->cell_max, gl, gh,
                                                                  mg->within, per);
  k_sp_total<<<1, 1, 0, L.stream>>>(nk, n_total, i_star, excluded, t_app, per, tot);
  L.count(2);
  return sync_check(c, "ta_speedup_finalize");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Statistics of every context of every set of a batch (set-aware kernels).
namespace {

// Per set: index of the first outlier key whose slot is in the set.
__global__ void k_outlier_set_bounds(const u64* keys, u64 n, SetMap sets, u64* set_off) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > sets.S) return;
  const u64 key = (u64)sets.set_ctx0[s] << 32;
  u64 lo = 0, hi = n;
  while (lo < hi) {
    const u64 mid = (lo + hi) / 2;
    if (keys[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  set_off[s] = lo;
}

// Outliers of a batch with set-local contexts and ranks.
__global__ void k_write_batch_outliers(const u64* keys, const double* zs, u64 n, SetMap sets,
                                       ta_outlier* out) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32 slot = (u32)(keys[i] >> 32), r = (u32)keys[i];
  const u32 s = set_of_ctx(sets, slot);
  ta_outlier o;
  o.ctx = slot - sets.set_ctx0[s];
  o.rank = r - sets.set_rank0[s];
  o.z = zs[i];
  out[i] = o;
}

}  // namespace

namespace ta {

// Shared with the other entry points (declared in ta_api_internal.h).
void launch_iter_summary(const Launch& L, u32 R, const u32* n_iter, const u64* span, u64* meta) {
  cudaMemsetAsync(meta, 0, 32, L.stream);
  cudaMemsetAsync(meta, 0xFF, 4, L.stream);
  k_sp_istar<<<blocks(R), 256, 0, L.stream>>>(nullptr, R, n_iter, span, (u32*)meta,
                                              (unsigned long long*)meta + 1,
                                              (unsigned long long*)meta + 2);
  L.count();
}
void sort_u64_pairs(const Launch& L, u64* keys, double* vals, u64 n) { sort_pairs(L, keys, vals, n); }
const Csr* csr_of_metric(const ta_experiment* e, u32 metric) { return metric_csr(e, metric); }
ta_status rank_subset_to_device(ta_ctx* c, Pool& tmp, const Launch& L, const u32* src, u32 n,
                                u32 kind, u32 limit, u32* status, const u32** out) {
  TRY(to_device(c, tmp, src, src ? n : 0, kind, out, "rank subset"));
  return check_subset(c, L, *out, n, limit, status, "rank subset");
}

u64 batch_stats_scratch_bytes(u32 Ctot) { return (u64)Ctot * 72 + 64; }

// All ranks, all contexts of every set, threshold tau; outlier keys
// (global slot << 32 | global rank) and z go to keys/zs (capacity cap);
// *n_out receives the full count.  scratch: batch_stats_scratch_bytes.
void launch_batch_stats(const Launch& L, u32 R, u32 Ctot, const u64* off, const u32* ctx,
                        const u64* time, const SetMap& sets, u32 tau_num, u32 tau_den,
                        unsigned char* scratch, ta_ctx_stats* stats, u64* keys, double* zs,
                        u64 cap, unsigned long long* n_out) {
  Partials P;
  unsigned char* q = scratch;
  P.present = (u32*)q;
  q += (u64)Ctot * 4;
  P.argmax = (u32*)q;
  q += (u64)Ctot * 4;
  P.mn = (u64*)q;
  q += (u64)Ctot * 8;
  P.mx = (u64*)q;
  q += (u64)Ctot * 8;
  P.s1 = (u64*)q;
  q += (u64)Ctot * 8;
  P.s2lo = (u64*)q;
  q += (u64)Ctot * 8;
  P.s2hi = (u64*)q;
  q += (u64)Ctot * 8;
  P.sd = (double*)q;
  q += (u64)Ctot * 8;
  P.Mlo = (u64*)q;
  q += (u64)Ctot * 8;
  P.Mhi = (u64*)q;
  cudaMemsetAsync(P.present, 0, (u64)Ctot * 4, L.stream);
  cudaMemsetAsync(P.mn, 0xFF, (u64)Ctot * 8, L.stream);
  cudaMemsetAsync(P.mx, 0, (u64)Ctot * 8 * 4, L.stream);  // mx, s1, s2lo, s2hi
  cudaMemsetAsync(n_out, 0, 8, L.stream);
  const int grid = std::max(1, std::min<int>(L.num_sms * 4, (int)((R + 7) / 8)));
  k_stats_partial<<<grid, STATS_NT, 0, L.stream>>>(nullptr, R, off, ctx, time, nullptr, P, sets);
  k_stats_finalize<<<blocks(Ctot), 256, 0, L.stream>>>(Ctot, R, nullptr, P, stats, sets);
  k_stats_z<<<grid, 256, 0, L.stream>>>(nullptr, R, off, ctx, time, nullptr, P, tau_num, tau_den,
                                        nullptr, keys, zs, std::max<u64>(cap, 1), n_out, nullptr,
                                        sets, 0, NONE32);
  k_stats_argmax<<<blocks(Ctot), 256, 0, L.stream>>>(Ctot, P.argmax, stats, sets);
  L.count(4);
}

// Sort n (<= capacity, buffers of next_pow2(capacity)) keys and split them by set.
void launch_batch_outliers(const Launch& L, u64* keys, double* zs, u64 n, const SetMap& sets,
                           ta_outlier* out, u64* set_off) {
  sort_pairs(L, keys, zs, n);
  k_outlier_set_bounds<<<blocks(sets.S + 1), 256, 0, L.stream>>>(keys, n, sets, set_off);
  if (n) k_write_batch_outliers<<<blocks(n), 256, 0, L.stream>>>(keys, zs, n, sets, out);
  L.count(2);
}

}  // namespace ta
