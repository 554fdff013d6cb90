// cluster.cu -- groups of ranks by their value of one context (Section VI-B:
// DBSCAN over the ranks' times of a call site, the groups mapped to compute
// nodes, K-Means over a few groups as a stability check).
//
// Both methods work on the sorted values.  After a gather (every subset
// rank's value by a binary search of its CSR row), a sort of (value, index)
// pairs and a prefix sum of the sorted values:
//   DBSCAN in one dimension is exact with searches and scans: a point's
//     neighbourhood is the sorted range [lower_bound(x - eps),
//     upper_bound(x + eps)), so its size decides the core flag; a core
//     starts a new cluster iff no core lies in [lower_bound(x - eps), i)
//     (consecutive cores closer than eps are neighbours, and no chain of
//     cores can cross a wider gap); a scan of the start flags numbers the
//     clusters, a scan of the core flags locates the nearest core below and
//     above every non-core point.
//   K-Means runs in one CTA: in one dimension each cluster of a Lloyd step is
//     a range of the sorted values whose ends are found by a binary search
//     against the midpoints of consecutive distinct centroids (exact: the
//     comparison 2 x n_a n_b <= S_a n_b + S_b n_a in 128-bit integers), and
//     the new centroids come from the prefix sums.
// Clusters are ranges of the sorted values in both methods; their sums come
// from the prefix sums and the node view from per-node cluster bit masks.
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

constexpr u32 KM_MAX = 64;

inline unsigned nblk(u64 n, int nt = 256) {
  return (unsigned)std::max<u64>(1, std::min<u64>((n + nt - 1) / nt, 1u << 20));
}

// Value of ctx on every subset rank (0 where absent) with its subset index.
__global__ void k_cl_gather(const u32* __restrict__ S, u32 n, const u64* __restrict__ off,
                            const u32* __restrict__ ctx, const u64* __restrict__ time, u32 c,
                            u64* keys, double* vals) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) {
    const u32 r = S ? S[i] : (u32)i;
    const u64 e = off[r + 1];
    u64 lo = off[r], hi = e;
    while (lo < hi) {
      const u64 mid = (lo + hi) / 2;
      if (ctx[mid] < c) lo = mid + 1;
      else hi = mid;
    }
    keys[i] = (lo < e && ctx[lo] == c) ? time[lo] : 0ull;
    vals[i] = (double)i;
  }
}

__global__ void k_cl_check_nodes(const u32* __restrict__ S, u32 n,
                                 const u32* __restrict__ node_of_rank, u32 n_nodes, u32* status) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32 r = S ? S[i] : i;
  if (node_of_rank[r] >= n_nodes) flag(status, F_INVALID);
}

__device__ __forceinline__ u32 lower_bound_u64(const u64* __restrict__ k, u32 n, u64 v) {
  u32 lo = 0, hi = n;
  while (lo < hi) {
    const u32 m = (lo + hi) / 2;
    if (k[m] < v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

__device__ __forceinline__ u32 upper_bound_u64(const u64* __restrict__ k, u32 n, u64 v) {
  u32 lo = 0, hi = n;
  while (lo < hi) {
    const u32 m = (lo + hi) / 2;
    if (k[m] <= v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// ------------------------------------------------------------- DBSCAN ----
__global__ void k_db_core(const u64* __restrict__ keys, u32 n, u64 eps, u32 min_pts, u32* lo,
                          u32* hi, u32* core) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u64 x = keys[i];
  const u64 a = x >= eps ? x - eps : 0ull;
  const u64 b = x + eps < x ? ~0ull : x + eps;
  const u32 l = lower_bound_u64(keys, n, a), h = upper_bound_u64(keys, n, b);
  lo[i] = l;
  hi[i] = h;
  core[i] = (h - l >= min_pts) ? 1u : 0u;
}

// A core starts a cluster iff no core lies in [lo, i) (cex: cores before).
__global__ void k_db_start(u32 n, const u32* __restrict__ lo, const u32* __restrict__ core,
                           const u64* __restrict__ cex, u32* start, u32* corepos) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool c = core[i] != 0;
  start[i] = (c && cex[i] == cex[lo[i]]) ? 1u : 0u;
  if (c) corepos[cex[i]] = i;
}

__device__ __forceinline__ int core_cluster(u32 c, const u64* sex, const u32* start) {
  return (int)(sex[c] + start[c]) - 1;
}

// Cores take their component; a non-core takes the nearer of the last core
// below and the first core above it when within eps (equal: the lower).
__global__ void k_db_label(const u64* __restrict__ keys, u32 n, const u32* __restrict__ lo,
                           const u32* __restrict__ hi, const u32* __restrict__ core,
                           const u64* __restrict__ cex, const u64* __restrict__ sex,
                           const u32* __restrict__ start, const u32* __restrict__ corepos,
                           int* lab) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (core[i]) {
    lab[i] = core_cluster(i, sex, start);
    return;
  }
  const u64 m = cex[i], total = cex[n];
  const bool hp = m > 0 && corepos[m - 1] >= lo[i];
  const bool hq = m < total && corepos[m] < hi[i];
  int l = -1;
  if (hp && hq) {
    const u32 p = corepos[m - 1], q = corepos[m];
    l = core_cluster(keys[i] - keys[p] <= keys[q] - keys[i] ? p : q, sex, start);
  } else if (hp) {
    l = core_cluster(corepos[m - 1], sex, start);
  } else if (hq) {
    l = core_cluster(corepos[m], sex, start);
  }
  lab[i] = l;
}

// Every cluster is a range of sorted positions: its first and its end.
__global__ void k_cl_ranges(const int* __restrict__ lab, u32 n, u32* L, u32* U) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int l = lab[i];
  if (l < 0) return;
  if (i == 0 || lab[i - 1] != l) L[l] = i;
  if (i + 1 == n || lab[i + 1] != l) U[l] = i + 1;
}

// ------------------------------------------------------------ K-Means ----
struct KmState {
  u64 S[KM_MAX], N[KM_MAX];  // centroid S / N of every cluster (final order)
  u32 L[KM_MAX], U[KM_MAX];  // its range of sorted positions
  u32 iters;
};

__device__ __forceinline__ bool cent_lt(u64 Sa, u64 Na, u64 Sb, u64 Nb) {
  return (u128)Sa * Nb < (u128)Sb * Na;
}
__device__ __forceinline__ bool cent_eq(u64 Sa, u64 Na, u64 Sb, u64 Nb) {
  return (u128)Sa * Nb == (u128)Sb * Na;
}

// One CTA of KM_MAX threads; thread j owns cluster j.  Products stay in 128
// bits: x <= span < 2^63 / R and n_a + n_b <= R, so 2 x n_a n_b < 2^94 and
// S_a n_b < 2^95.
__global__ void __launch_bounds__(KM_MAX) k_kmeans(const u64* __restrict__ keys,
                                                   const u64* __restrict__ P, u32 n, u32 k,
                                                   u32 max_iter, KmState* out) {
  __shared__ u64 S[KM_MAX], N[KM_MAX];
  __shared__ u32 L[KM_MAX], U[KM_MAX], pL[KM_MAX], pU[KM_MAX];
  __shared__ int same;
  const u32 j = threadIdx.x;
  if (j < k) {
    S[j] = keys[((2ull * j + 1) * n) / (2ull * k)];
    N[j] = 1;
  }
  __syncthreads();
  auto assign = [&]() {
    if (j == 0) {  // clusters in ascending centroid order (stable insertion sort)
      for (u32 q = 1; q < k; ++q) {
        const u64 s = S[q], c = N[q];
        u32 p = q;
        while (p > 0 && cent_lt(s, c, S[p - 1], N[p - 1])) {
          S[p] = S[p - 1];
          N[p] = N[p - 1];
          --p;
        }
        S[p] = s;
        N[p] = c;
      }
    }
    __syncthreads();
    // the first cluster of every run of equal centroids takes the points up
    // to the midpoint with the next distinct centroid (ties stay below)
    if (j < k && !(j > 0 && cent_eq(S[j], N[j], S[j - 1], N[j - 1]))) {
      u32 nj = j + 1;
      while (nj < k && cent_eq(S[nj], N[nj], S[j], N[j])) ++nj;
      u32 u = n;
      if (nj < k) {
        const u128 rhs = (u128)S[j] * N[nj] + (u128)S[nj] * N[j];
        const u128 m = (u128)2 * N[j] * N[nj];
        u32 lo = 0, hi = n;
        while (lo < hi) {
          const u32 mid = (lo + hi) / 2;
          if ((u128)keys[mid] * m <= rhs) lo = mid + 1;
          else hi = mid;
        }
        u = lo;
      }
      U[j] = u;
    }
    __syncthreads();
    if (j == 0) {
      u32 prev = 0;
      for (u32 q = 0; q < k; ++q) {
        if (q > 0 && cent_eq(S[q], N[q], S[q - 1], N[q - 1])) {
          L[q] = prev;  // an equal centroid after the first: empty
          U[q] = prev;
        } else {
          L[q] = prev;
          prev = U[q];
        }
      }
    }
    __syncthreads();
  };
  assign();
  u32 it = 0;
  while (it < max_iter) {
    if (j < k && U[j] > L[j]) {
      S[j] = P[U[j]] - P[L[j]];
      N[j] = U[j] - L[j];
    }
    if (j < k) {
      pL[j] = L[j];
      pU[j] = U[j];
    }
    ++it;
    __syncthreads();
    assign();
    if (j == 0) {
      int s = 1;
      for (u32 q = 0; q < k; ++q) s &= (L[q] == pL[q] && U[q] == pU[q]) ? 1 : 0;
      same = s;
    }
    __syncthreads();
    if (same) break;
  }
  if (j < k) {
    out->S[j] = S[j];
    out->N[j] = N[j];
    out->L[j] = L[j];
    out->U[j] = U[j];
  }
  if (j == 0) out->iters = it;
}

__global__ void k_km_label(const KmState* __restrict__ st, u32 k, u32 n, int* lab) {
  __shared__ u32 U[KM_MAX];
  if (threadIdx.x < k) U[threadIdx.x] = st->U[threadIdx.x];
  __syncthreads();
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int q = 0;
  while (q < (int)k && U[q] <= i) ++q;  // the first range ending after i
  lab[i] = q;
}

// --------------------------------------------------------- both methods --
__global__ void k_cl_info(const u64* __restrict__ keys, const u64* __restrict__ P,
                          const u32* __restrict__ L, const u32* __restrict__ U, u32 nc,
                          const KmState* km, ta_cluster_info* info) {
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  ta_cluster_info o;
  const u32 l = L[c], u = U[c];
  o.n = u - l;
  o.sum = o.n ? P[u] - P[l] : 0ull;
  o.min = o.n ? keys[l] : 0ull;
  o.max = o.n ? keys[u - 1] : 0ull;
  o.mean = o.n ? u64_to_f64(o.sum) / u64_to_f64(o.n) : 0.0;
  o.centroid = !km ? o.mean : km->N[c] ? u64_to_f64(km->S[c]) / u64_to_f64(km->N[c]) : 0.0;
  info[c] = o;
}

__global__ void k_cl_scatter(const int* __restrict__ lab, const double* __restrict__ vals, u32 n,
                             int* out) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[(u32)vals[i]] = lab[i];
}

__global__ void k_cl_nodes(const u32* __restrict__ S, u32 n, const u32* __restrict__ node_of_rank,
                           const int* __restrict__ lab, unsigned long long* mask, u32* noise) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32 node = node_of_rank[S ? S[i] : i];
  const int l = lab[i];
  if (l >= 0) atomicOr(&mask[node], 1ull << l);
  else noise[node] = 1;
}

__global__ void k_cl_pairs(u32 n_nodes, const unsigned long long* __restrict__ mask,
                           const u32* __restrict__ noise, u32 cap, u32* per, u32* pair,
                           u32* noise_nodes) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_nodes) return;
  const unsigned long long m = mask[v];
  for (unsigned long long x = m; x; x &= x - 1) {
    const u32 a = __ffsll((long long)x) - 1;
    atomicAdd(&per[a], 1u);
    for (unsigned long long y = x & (x - 1); y; y &= y - 1)
      atomicAdd(&pair[a * cap + (__ffsll((long long)y) - 1)], 1u);
  }
  if (noise[v]) atomicAdd(noise_nodes, 1u);
}

}  // namespace
}  // namespace ta

using namespace ta;

extern "C" ta_status ta_cluster_ranks(ta_experiment* e, const ta_cluster_args* a,
                                      ta_cluster_out* o) {
  if (!e || !a || !o) return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: NULL argument");
  if (a->method != TA_CLUSTER_DBSCAN && a->method != TA_CLUSTER_KMEANS)
    return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: method");
  if (a->metric != TA_EXCLUSIVE && a->metric != TA_INCLUSIVE)
    return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: metric");
  const Csr* m = csr_of_metric(e, a->metric);
  if (!m) return fail(TA_ERR_STATE, "ta_cluster_ranks: the inclusive rollup was not built");
  if (a->ctx >= e->C) return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: ctx >= n_ctx");
  if (a->mem_kind != TA_MEM_HOST && a->mem_kind != TA_MEM_DEVICE)
    return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: mem_kind");
  const bool db = a->method == TA_CLUSTER_DBSCAN;
  if (db && a->min_pts == 0) return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: min_pts = 0");
  if (!db && (a->k == 0 || a->k > KM_MAX))
    return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: k must be 1..%u", KM_MAX);
  if (a->node_of_rank && a->n_nodes == 0)
    return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: n_nodes = 0");
  if (a->ranks && a->n_ranks_subset > e->R)
    return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: subset larger than the experiment");
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
  const bool dev = a->mem_kind == TA_MEM_DEVICE;
  u32* status;
  TRY(tmp.get_n(4, &status, "cluster status"));
  const u32* dS = nullptr;
  TRY(rank_subset_to_device(c, tmp, L, a->ranks, a->n_ranks_subset, a->mem_kind, e->R, status,
                            &dS));
  const u32 n = a->ranks ? a->n_ranks_subset : e->R;
  const u32* dnode = nullptr;
  if (a->node_of_rank) {
    if (dev) {
      dnode = a->node_of_rank;
    } else {
      u32* d;
      TRY(tmp.get_n(e->R, &d, "node of rank"));
      TRY(copy(c, d, a->node_of_rank, (size_t)e->R * 4));
      dnode = d;
    }
    cudaMemsetAsync(status, 0, 4, c->stream);
    if (n) {
      k_cl_check_nodes<<<nblk(n), 256, 0, c->stream>>>(dS, n, dnode, a->n_nodes, status);
      L.count();
    }
    u32 f = 0;
    TRY(copy(c, &f, status, 4));
    TRY(sync_check(c, "ta_cluster_ranks (nodes)"));
    if (f) return fail(TA_ERR_INVALID_ARG, "ta_cluster_ranks: a node id >= n_nodes");
  }
  u64 P2 = 1;
  while (P2 < n) P2 <<= 1;
  u64 *keys, *P, *scratch;
  double* vals;
  int *lab, *lab_out;
  TRY(tmp.get_n(P2, &keys, "cluster keys"));
  TRY(tmp.get_n(P2, &vals, "cluster values"));
  TRY(tmp.get_n((u64)n + 1, &P, "cluster prefix"));
  TRY(tmp.get_n(scan_scratch_elems(n), &scratch, "cluster scan"));
  TRY(tmp.get_n(std::max<u32>(n, 1), &lab, "cluster labels"));
  TRY(tmp.get_n(std::max<u32>(n, 1), &lab_out, "cluster labels"));
  if (n) {
    k_cl_gather<<<nblk(n), 256, 0, c->stream>>>(dS, n, m->off, m->ctx, m->time, a->ctx, keys,
                                                 vals);
    L.count();
    sort_u64_pairs(L, keys, vals, n);
  }
  scan_exclusive(L, keys, n, P, P + n, scratch);
  u32 nc = 0, iters = 0;
  u32 *rL, *rU;
  KmState* km = nullptr;
  const unsigned bn = nblk(n);
  if (db) {
    u32 *lo, *hi, *core, *start, *corepos;
    u64 *cex, *sex;
    TRY(tmp.get_n(std::max<u32>(n, 1), &lo, "dbscan"));
    TRY(tmp.get_n(std::max<u32>(n, 1), &hi, "dbscan"));
    TRY(tmp.get_n(std::max<u32>(n, 1), &core, "dbscan"));
    TRY(tmp.get_n(std::max<u32>(n, 1), &start, "dbscan"));
    TRY(tmp.get_n(std::max<u32>(n, 1), &corepos, "dbscan"));
    TRY(tmp.get_n((u64)n + 1, &cex, "dbscan"));
    TRY(tmp.get_n((u64)n + 1, &sex, "dbscan"));
    if (n) {
      k_db_core<<<bn, 256, 0, c->stream>>>(keys, n, a->eps, a->min_pts, lo, hi, core);
      L.count();
    }
    scan_exclusive(L, core, n, cex, cex + n, scratch);
    if (n) {
      k_db_start<<<bn, 256, 0, c->stream>>>(n, lo, core, cex, start, corepos);
      L.count();
    }
    scan_exclusive(L, start, n, sex, sex + n, scratch);
    if (n) {
      k_db_label<<<bn, 256, 0, c->stream>>>(keys, n, lo, hi, core, cex, sex, start, corepos, lab);
      L.count();
    }
    u64 h = 0;
    TRY(copy(c, &h, sex + n, 8));
    TRY(sync_check(c, "ta_cluster_ranks (dbscan)"));
    nc = (u32)h;
    TRY(tmp.get_n(std::max<u32>(nc, 1), &rL, "cluster ranges"));
    TRY(tmp.get_n(std::max<u32>(nc, 1), &rU, "cluster ranges"));
    cudaMemsetAsync(rL, 0, (size_t)std::max<u32>(nc, 1) * 4, c->stream);
    cudaMemsetAsync(rU, 0, (size_t)std::max<u32>(nc, 1) * 4, c->stream);
    if (n) {
      k_cl_ranges<<<bn, 256, 0, c->stream>>>(lab, n, rL, rU);
      L.count();
    }
  } else {
    TRY(tmp.get_n(1, &km, "k-means state"));
    nc = a->k;
    if (n) {
      k_kmeans<<<1, KM_MAX, 0, c->stream>>>(keys, P, n, a->k, a->max_iter ? a->max_iter : 300, km);
      k_km_label<<<bn, 256, 0, c->stream>>>(km, a->k, n, lab);
      L.count(2);
    } else {
      cudaMemsetAsync(km, 0, sizeof(KmState), c->stream);
    }
    rL = km->L;
    rU = km->U;
  }
  ta_cluster_info* info;
  TRY(tmp.get_n(std::max<u32>(nc, 1), &info, "cluster info"));
  if (nc) {
    k_cl_info<<<nblk(nc), 256, 0, c->stream>>>(keys, P, rL, rU, nc, km, info);
    L.count();
  }
  if (n) {
    k_cl_scatter<<<bn, 256, 0, c->stream>>>(lab, vals, n, lab_out);
    L.count();
  }
  if (km) {
    TRY(copy(c, &iters, &km->iters, 4));
  }
  TRY(sync_check(c, "ta_cluster_ranks"));
  o->n_clusters = nc;
  o->iterations = km ? iters : 0;
  o->node_view = 0;
  o->noise_nodes = 0;
  if (o->labels) TRY(copy(c, o->labels, lab_out, (size_t)n * 4));
  u64 in_clusters = 0;
  {
    std::vector<ta_cluster_info> h(nc);
    if (nc) TRY(copy(c, h.data(), info, (size_t)nc * sizeof(ta_cluster_info)));
    TRY(sync_check(c, "ta_cluster_ranks (info)"));
    for (const auto& x : h) in_clusters += x.n;
  }
  o->n_noise = n - in_clusters;
  if (o->clusters && nc > o->cluster_cap)
    return fail(TA_ERR_CAPACITY, "ta_cluster_ranks: %u clusters, cluster_cap %u", nc,
                o->cluster_cap);
  if (o->clusters && nc) TRY(copy(c, o->clusters, info, (size_t)nc * sizeof(ta_cluster_info)));
  if (dnode && nc <= KM_MAX && (o->cluster_nodes || o->pair_nodes)) {
    if (o->cluster_cap < nc)
      return fail(TA_ERR_CAPACITY, "ta_cluster_ranks: %u clusters, cluster_cap %u", nc,
                  o->cluster_cap);
    const u32 cap = std::max<u32>(nc, 1);  // device stride; the caller's is cluster_cap
    unsigned long long* mask;
    u32 *noise, *per, *pair, *nn;
    TRY(tmp.get_n(a->n_nodes, &mask, "node masks"));
    TRY(tmp.get_n(a->n_nodes, &noise, "node noise"));
    TRY(tmp.get_n(std::max<u32>(cap, 1), &per, "cluster nodes"));
    TRY(tmp.get_n(std::max<u64>((u64)cap * cap, 1), &pair, "pair nodes"));
    TRY(tmp.get_n(1, &nn, "noise nodes"));
    cudaMemsetAsync(mask, 0, (size_t)a->n_nodes * 8, c->stream);
    cudaMemsetAsync(noise, 0, (size_t)a->n_nodes * 4, c->stream);
    cudaMemsetAsync(per, 0, (size_t)std::max<u32>(cap, 1) * 4, c->stream);
    cudaMemsetAsync(pair, 0, (size_t)std::max<u64>((u64)cap * cap, 1) * 4, c->stream);
    cudaMemsetAsync(nn, 0, 4, c->stream);
    if (n) {
      k_cl_nodes<<<bn, 256, 0, c->stream>>>(dS, n, dnode, lab_out, mask, noise);
      L.count();
    }
    k_cl_pairs<<<nblk(a->n_nodes), 256, 0, c->stream>>>(a->n_nodes, mask, noise, cap, per, pair,
                                                        nn);
    L.count();
    if (o->cluster_nodes) TRY(copy(c, o->cluster_nodes, per, (size_t)nc * 4));
    if (o->pair_nodes) {
      const size_t dp = (size_t)o->cluster_cap * 4;
      if (dev) cudaMemset2DAsync(o->pair_nodes, dp, 0, dp, o->cluster_cap, c->stream);
      else std::memset(o->pair_nodes, 0, dp * o->cluster_cap);
      if (nc) {
        const cudaError_t ce = cudaMemcpy2DAsync(o->pair_nodes, dp, pair, (size_t)cap * 4,
                                                 (size_t)nc * 4, nc, cudaMemcpyDefault, c->stream);
        if (ce != cudaSuccess) return cuda_fail(ce, "ta_cluster_ranks (pair nodes)");
      }
    }
    TRY(copy(c, &o->noise_nodes, nn, 4));
    o->node_view = 1;
  }
  return sync_check(c, "ta_cluster_ranks");
}
