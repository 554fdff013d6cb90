// batch_rollup.cu -- the potential-speedup estimate (Section VI-A, Table V)
// and the node / chassis / rack rollup (Section VI-B) for every set of a
// batch at once: each kernel covers all sets, looking up its set per rank,
// context, node or work item.  Same arithmetic as the single-experiment
// kernels (exact integer sums; the FP64 steps in the same order), so every
// set's results equal a single-experiment call's bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "ta_internal.h"

namespace ta {

namespace {

constexpr int BNW = 8;
constexpr u32 BKC = 256;  // contexts per within-rank chunk
constexpr u32 BU = 8;     // entries per lane in flight
constexpr u32 BPR = 4;    // ranks per round (cells)
constexpr u32 BCU = 8;    // entries per lane per round (cells)

__device__ __forceinline__ u32 find_set(const u64* prefix, u32 S, u64 v) {
  u32 lo = 0, hi = S;  // last s with prefix[s] <= v
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) / 2;
    if (prefix[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ u32 find_set32(const u32* prefix, u32 S, u32 v) {
  u32 lo = 0, hi = S;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) / 2;
    if (prefix[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Within-rank CV terms: warp per rank of every set with a speedup request.
// A rank with exactly I* iteration rows and iteration moments takes its sums
// from its exclusive entries; any other rank reads its rows.
__global__ void __launch_bounds__(BNW * 32) k_bsp_within(const BatchSpeedupArgs P) {
  __shared__ unsigned long long s_sum[BNW][BKC], s_lo[BNW][BKC], s_hi[BNW][BKC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* ms = s_sum[warp];
  unsigned long long* ml = s_lo[warp];
  unsigned long long* mh = s_hi[warp];
  for (u32 q = lane; q < BKC; q += 32) ms[q] = ml[q] = mh[q] = 0;
  __syncwarp();
  const u32 gw = blockIdx.x * BNW + warp, nw = gridDim.x * BNW;
  for (u32 r = gw; r < P.R; r += nw) {
    const u32 s = P.rank_set[r];
    const u32 nk = P.k0[s + 1] - P.k0[s], I = P.istar[s];
    if (nk == 0 || I == 0) continue;
    const u32 n = P.set_rank0[s + 1] - P.set_rank0[s], ri = r - P.set_rank0[s];
    const u32 cb = P.set_ctx0[s];
    const u64 row0 = P.row_off[r] + 1;
    const u64 E0 = P.entry_off[row0], E1 = P.entry_off[row0 + I];
    const bool mom = P.mom_ok && P.mom_ok[r] && P.row_off[r + 1] - P.row_off[r] == (u64)I + 1;
    for (u32 kc0 = 0; kc0 < nk; kc0 += BKC) {
      const u32 nkc = min(BKC, nk - kc0);
      if (mom) {
        const ulonglong2* m2 = reinterpret_cast<const ulonglong2*>(P.x_m2);
        for (u64 j = P.x_off[r] + lane; j < P.x_off[r + 1]; j += 32) {
          const u32 k = P.kmap[cb + P.x_ctx[j]];
          if (k == NONE32 || k < kc0 || k >= kc0 + nkc) continue;
          const ulonglong2 q = m2[j];
          ms[k - kc0] = P.x_m1[j];
          ml[k - kc0] = q.x;
          mh[k - kc0] = q.y;
        }
      }
      for (u64 jb = mom ? E1 : E0; jb < E1; jb += 32 * BU) {
        u32 c[BU];
        u64 t[BU];
#pragma unroll
        for (u32 u = 0; u < BU; ++u) {
          const u64 j = jb + u * 32 + lane;
          c[u] = j < E1 ? P.e_ctx[j] : NONE32;
          t[u] = j < E1 ? P.e_time[j] : 0ull;
        }
#pragma unroll
        for (u32 u = 0; u < BU; ++u) {
          const u32 k = (c[u] != NONE32) ? P.kmap[cb + c[u]] : NONE32;
          if (k == NONE32 || k < kc0 || k >= kc0 + nkc) continue;
          const u32 kk = k - kc0;
          atomicAdd(&ms[kk], (unsigned long long)t[u]);
          atomic_add_u128((u64*)&ml[kk], (u64*)&mh[kk], (u128)t[u] * t[u]);
        }
      }
      __syncwarp();
      const double cI = cv_coef(I);
      for (u32 kk = lane; kk < nkc; kk += 32) {
        const u128 q = ((u128)mh[kk] << 64) | ml[kk];
        P.cvw[P.cv0[s] + (u64)(kc0 + kk) * n + ri] = cv_of_sums(ms[kk], q, I, cI);
        ms[kk] = ml[kk] = mh[kk] = 0;
      }
      __syncwarp();
    }
  }
}

// Cells (iteration, context) over each set's ranks: a work item is one
// iteration, 64 contexts and a group of ranks of one set (items of all sets
// concatenated); registers hold the cells, rows are scattered through shared
// memory (a row holds each context once).
__global__ void __launch_bounds__(BNW * 32, 3) k_bsp_cells(const BatchSpeedupArgs P) {
  __shared__ u64 rowbuf[BNW][BPR][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* buf = &rowbuf[warp][0][0];
  for (u32 q = lane; q < BPR * 64; q += 32) buf[q] = 0;
  __syncwarp();
  const u64 item = (u64)blockIdx.x * BNW + warp;
  if (item >= P.item0[P.S]) return;
  const u32 s = find_set(P.item0, P.S, item);
  const u64 li = item - P.item0[s];
  const u32 nk = P.k0[s + 1] - P.k0[s], I = P.istar[s];
  const u32 n_kb = (nk + 63) / 64;
  const u32 i0 = (u32)(li % I), kb = (u32)((li / I) % n_kb);
  const u32 g = (u32)(li / ((u64)I * n_kb));
  const u32 k0 = kb * 64;
  const u32 cb = P.set_ctx0[s];
  const u32 rank0 = P.set_rank0[s], rankN = P.set_rank0[s + 1];
  const u32 r_begin = rank0 + g * P.group, r_end = min(rankN, r_begin + P.group);
  u64 csum[2] = {0, 0}, cmax[2] = {0, 0}, clo[2] = {0, 0}, chi[2] = {0, 0};
  for (u32 rb = r_begin; rb < r_end; rb += BPR) {
    u64 myb = 0, mye = 0;
    if (lane < BPR && rb + lane < r_end) {
      const u64 row = P.row_off[rb + lane] + 1 + i0;
      myb = P.entry_off[row];
      mye = P.entry_off[row + 1];
    }
    u64 b[BPR], len[BPR + 1];
    len[0] = 0;
#pragma unroll
    for (u32 p = 0; p < BPR; ++p) {
      b[p] = __shfl_sync(FULL, myb, p);
      len[p + 1] = len[p] + (__shfl_sync(FULL, mye, p) - b[p]);
    }
    const u64 total = len[BPR];
    for (u64 vb = 0; vb < total; vb += 32 * BCU) {
      u32 c[BCU], slot[BCU];
      u64 t[BCU];
#pragma unroll
      for (u32 u = 0; u < BCU; ++u) {
        const u64 v = vb + u * 32 + lane;
        u32 p = 0;
#pragma unroll
        for (u32 q = 1; q < BPR; ++q) p += (v >= len[q]) ? 1u : 0u;
        u64 bp = b[0], lp = len[0];
#pragma unroll
        for (u32 q = 1; q < BPR; ++q)
          if (p == q) {
            bp = b[q];
            lp = len[q];
          }
        const u64 jj = bp + (v - lp);
        slot[u] = p;
        c[u] = v < total ? P.e_ctx[jj] : NONE32;
        t[u] = v < total ? P.e_time[jj] : 0ull;
      }
#pragma unroll
      for (u32 u = 0; u < BCU; ++u) {
        const u32 k = (c[u] != NONE32) ? P.kmap[cb + c[u]] : NONE32;
        if (k != NONE32 && k >= k0 && k < k0 + 64) buf[slot[u] * 64 + (k - k0)] = t[u];
      }
    }
    __syncwarp();
#pragma unroll
    for (u32 p = 0; p < BPR; ++p)
#pragma unroll
      for (u32 h = 0; h < 2; ++h) {
        u64* cell = &buf[p * 64 + lane + 32 * h];
        const u64 v = *cell;
        *cell = 0;
        const u128 v2 = (u128)v * v;
        csum[h] += v;
        cmax[h] = max(cmax[h], v);
        const u64 lo = clo[h] + (u64)v2;
        chi[h] += (u64)(v2 >> 64) + (lo < clo[h] ? 1ull : 0ull);
        clo[h] = lo;
      }
    __syncwarp();
  }
#pragma unroll
  for (u32 h = 0; h < 2; ++h) {
    const u32 k = k0 + lane + 32 * h;
    if (k >= nk) continue;
    const u64 gq = P.cell0[s] + (u64)i0 * nk + k;
    if (csum[h]) atomicAdd((unsigned long long*)&P.g_sum[gq], (unsigned long long)csum[h]);
    if (cmax[h]) atomicMax((unsigned long long*)&P.g_max[gq], (unsigned long long)cmax[h]);
    if (clo[h] | chi[h]) atomic_add_u128(&P.g_sqlo[gq], &P.g_sqhi[gq], ((u128)chi[h] << 64) | clo[h]);
  }
}

// Pairwise sum of each (set, context)'s per-rank CV terms (the definition's
// fixed order); one CTA per global context index.
__global__ void __launch_bounds__(256) k_bsp_pairwise(const BatchSpeedupArgs P) {
  const u32 gk = blockIdx.x;
  const u32 s = find_set32(P.k0, P.S, gk);
  const u32 k = gk - P.k0[s], I = P.istar[s];
  const u32 n = P.set_rank0[s + 1] - P.set_rank0[s];
  if (I == 0) {
    if (threadIdx.x == 0) P.wsum[gk] = 0.0;
    return;
  }
  double* src = P.cvw + P.cv0[s] + (u64)k * n;
  double* dst = P.cvw2 + P.cv0[s] + (u64)k * n;
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
  if (threadIdx.x == 0) P.wsum[gk] = (n == 0) ? 0.0 : src[0];
}

// Per (set, context): iteration sums in order and the finished ratios.
__global__ void k_bsp_final(const BatchSpeedupArgs P) {
  const int lane = threadIdx.x & 31;
  const u32 gk = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gk >= P.k0[P.S]) return;
  const u32 s = find_set32(P.k0, P.S, gk);
  const u32 nk = P.k0[s + 1] - P.k0[s], k = gk - P.k0[s], I = P.istar[s];
  const u64 n = P.set_rank0[s + 1] - P.set_rank0[s];
  u64 A = 0, B = 0;
  double across = 0.0;
  for (u32 i0 = 0; i0 < I; i0 += 32) {
    const u32 i = i0 + lane;
    u64 sum = 0, mx = 0;
    double term = 0.0;
    if (i < I) {
      const u64 q = P.cell0[s] + (u64)i * nk + k;
      sum = P.g_sum[q];
      mx = P.g_max[q];
      const u128 sq = ((u128)P.g_sqhi[q] << 64) | P.g_sqlo[q];
      const double mean = u64_to_f64(sum) / u64_to_f64(n);
      const double sd = (n < 2) ? 0.0
                                : sqrt(u128_to_f64((u128)n * sq - (u128)sum * sum) /
                                       u64_to_f64(n * (n - 1)));
      term = (mean == 0.0) ? 0.0 : sd / mean;
    }
    const u32 m = min(32u, I - i0);
    for (u32 x = 0; x < m; ++x) {
      A += __shfl_sync(FULL, mx, x);
      B += __shfl_sync(FULL, sum, x);
      across += __shfl_sync(FULL, term, x);
    }
  }
  if (lane != 0) return;
  const double w_sum = (I > 0) ? P.wsum[gk] : 0.0;
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
  P.per[gk] = p;
}

// Per set: totals, shares and the speedup fraction.
__global__ void k_bsp_total(const BatchSpeedupArgs P) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.S) return;
  const u32 k0 = P.k0[s], k1 = P.k0[s + 1];
  if (k0 == k1) return;
  const u64 n = P.set_rank0[s + 1] - P.set_rank0[s];
  u128 sumB = 0, sumG = 0;
  for (u32 k = k0; k < k1; ++k) {
    sumB += P.per[k].B;
    sumG += ((u128)P.per[k].G_hi << 64) | P.per[k].G_lo;
  }
  for (u32 k = k0; k < k1; ++k)
    P.per[k].share = (sumB == 0) ? 0.0 : u64_to_f64(P.per[k].B) / u128_to_f64(sumB);
  ta_speedup_total t;
  t.i_star = P.istar[s];
  t.reserved = 0;
  t.excluded_iterations = P.excluded[s];
  t.sum_G_lo = (u64)sumG;
  t.sum_G_hi = (u64)(sumG >> 64);
  t.t_app = P.t_app[s];
  t.total_reduction = u128_to_f64(sumG) / u64_to_f64(n);
  t.speedup_fraction =
      (P.t_app[s] == 0) ? 0.0 : u128_to_f64(sumG) / u128_to_f64((u128)n * P.t_app[s]);
  P.tot[s] = t;
}

// ---- rack rollup ------------------------------------------------------------
__global__ void k_btopo_nodes(const BatchTopoArgs T) {
  const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= T.R) return;
  const u32 s = T.rank_set[r];
  if (!T.has[s]) return;
  const u32 c = T.ctx[s];
  const ta_ctx_stats st = T.stats[T.set_ctx0[s] + c];
  const u64 n = st.n;
  const u128 S2 = ((u128)st.s2_hi << 64) | st.s2_lo;
  const u128 M = (u128)n * S2 - (u128)st.s1 * st.s1;
  // the rank's exclusive value of c (binary search in its context-ascending list)
  u64 lo = T.x_off[r], hi = T.x_off[r + 1];
  const u64 end = hi;
  while (lo < hi) {
    const u64 mid = (lo + hi) / 2;
    if (T.x_ctx[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  const bool present = lo < end && T.x_ctx[lo] == c;
  const u64 x = present ? T.x_time[lo] : 0ull;
  const long long D = (long long)(n * x) - (long long)st.s1;
  const bool out = present && is_outlier(D, n, M, T.tau_num[s], T.tau_den[s]);
  const u64 nd = T.node0[s] + T.node_of_rank[r];
  if (out) atomicAdd(&T.node_out[nd], 1u);
  atomicAdd(&T.node_sum[nd], (unsigned long long)x);
  atomicAdd(&T.node_ranks[nd], 1u);
}

__global__ void k_btopo_up(const BatchTopoArgs T) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.node0[T.S]) return;
  const u32 s = find_set(T.node0, T.S, i);
  const u32 f = T.node_out[i] >= T.min_ranks[s] ? 1u : 0u;
  T.node_flag[i] = (uint8_t)f;
  const u64 ch = T.chassis0[s] + T.chassis_of_node[i], rk = T.rack0[s] + T.rack_of_node[i];
  atomicAdd(&T.ch_flag[ch], f);
  atomicAdd(&T.ch_nodes[ch], 1u);
  atomicAdd(&T.ch_sum[ch], T.node_sum[i]);
  atomicAdd(&T.rk_flag[rk], f);
  atomicAdd(&T.rk_nodes[rk], 1u);
  atomicAdd(&T.rk_sum[rk], T.node_sum[i]);
}

// One CTA per set: its flagged racks in ascending order.
__global__ void k_btopo_racks(const BatchTopoArgs T) {
  __shared__ u32 wsum[8];
  __shared__ u32 base;
  const u32 s = blockIdx.x;
  if (!T.has[s]) {
    if (threadIdx.x == 0) T.n_flagged[s] = 0;
    return;
  }
  const u64 r0 = T.rack0[s];
  const u32 nr = (u32)(T.rack0[s + 1] - r0);
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (u32 b0 = 0; b0 < nr; b0 += 256) {
    const u32 j = b0 + threadIdx.x;
    const bool f = j < nr && T.rk_flag[r0 + j] > 0;
    const u32 bal = __ballot_sync(FULL, f);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    u32 before = 0, total = 0;
    for (int i = 0; i < 8; ++i) {
      if (i < w) before += wsum[i];
      total += wsum[i];
    }
    if (f) T.flagged[r0 + base + before + __popc(bal & ((1u << lane) - 1u))] = j;
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) T.n_flagged[s] = base;
}

inline unsigned nblk(u64 n, int t = 256) { return (unsigned)std::max<u64>(1, (n + t - 1) / t); }

}  // namespace

void launch_batch_speedup(const Launch& L, const BatchSpeedupArgs& P, u64 n_cells, u64 n_cv) {
  const u32 NK = P.nk_total;
  if (NK == 0) return;
  cudaMemsetAsync(P.g_sum, 0, std::max<u64>(n_cells, 1) * 8, L.stream);
  cudaMemsetAsync(P.g_max, 0, std::max<u64>(n_cells, 1) * 8, L.stream);
  cudaMemsetAsync(P.g_sqlo, 0, std::max<u64>(n_cells, 1) * 8, L.stream);
  cudaMemsetAsync(P.g_sqhi, 0, std::max<u64>(n_cells, 1) * 8, L.stream);
  (void)n_cv;
  k_bsp_within<<<std::max(1, std::min<int>(L.num_sms * 8, (int)((P.R + BNW - 1) / BNW))),
                 BNW * 32, 0, L.stream>>>(P);
  if (P.n_items) k_bsp_cells<<<nblk(P.n_items, BNW), BNW * 32, 0, L.stream>>>(P);
  k_bsp_pairwise<<<NK, 256, 0, L.stream>>>(P);
  k_bsp_final<<<nblk((u64)NK * 32, 128), 128, 0, L.stream>>>(P);
  k_bsp_total<<<nblk(P.S), 256, 0, L.stream>>>(P);
  L.count(P.n_items ? 5 : 4);
}

void launch_batch_topology(const Launch& L, const BatchTopoArgs& T, u64 n_nodes, u64 n_chassis,
                           u64 n_racks) {
  if (!n_nodes) return;
  cudaMemsetAsync(T.node_out, 0, n_nodes * 4, L.stream);
  cudaMemsetAsync(T.node_sum, 0, n_nodes * 8, L.stream);
  cudaMemsetAsync(T.node_ranks, 0, n_nodes * 4, L.stream);
  cudaMemsetAsync(T.ch_flag, 0, n_chassis * 4, L.stream);
  cudaMemsetAsync(T.ch_nodes, 0, n_chassis * 4, L.stream);
  cudaMemsetAsync(T.ch_sum, 0, n_chassis * 8, L.stream);
  cudaMemsetAsync(T.rk_flag, 0, n_racks * 4, L.stream);
  cudaMemsetAsync(T.rk_nodes, 0, n_racks * 4, L.stream);
  cudaMemsetAsync(T.rk_sum, 0, n_racks * 8, L.stream);
  k_btopo_nodes<<<nblk(T.R), 256, 0, L.stream>>>(T);
  k_btopo_up<<<nblk(n_nodes), 256, 0, L.stream>>>(T);
  k_btopo_racks<<<T.S, 256, 0, L.stream>>>(T);
  L.count(3);
}

}  // namespace ta
