// ingest.cu -- kernels that turn raw traces into the resident products:
// rank-offset and span validation, calling-context-tree validation and depth,
// the fused validate + duration + iteration-cut + (rank, iteration, context)
// aggregation kernel (the iteration tensor of Section V), and the per-rank
// exclusive / inclusive CSR kernels (Sections II-A and VI-B).
#include <algorithm>

#include "ta_internal.h"

namespace ta {

// ---------------------------------------------------------------------------
// Rank offsets: rank_off[0] = 0, non-decreasing, rank_off[R] = N, every rank
// shorter than 2^32 samples; per-rank span ts_last - ts_first.
__global__ void k_rank_off(const u64* __restrict__ rank_off, u32 R, u64 N,
                           const u64* __restrict__ ts, u64* span, unsigned long long* max_span,
                           u32* status) {
  const u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > R) return;
  if (r == 0 && rank_off[0] != 0) flag(status, F_INVALID);
  if (r == R) {
    if (rank_off[R] != N) flag(status, F_INVALID);
    return;
  }
  const u64 b = rank_off[r], e = rank_off[r + 1];
  if (e < b || e > N || b > N) {
    flag(status, F_INVALID);
    span[r] = 0;
    return;
  }
  if (e - b > 0xFFFFFFFFull) flag(status, F_INVALID);
  u64 sp = 0;
  if (e > b) {
    const u64 t0 = ts[b], t1 = ts[e - 1];
    sp = t1 >= t0 ? t1 - t0 : 0;  // a decrease is reported by the tensor pass
  }
  span[r] = sp;
  atomicMax(max_span, (unsigned long long)sp);
}

void launch_rank_off(const Launch& L, const u64* rank_off, u32 R, u64 N, const u64* ts,
                     u64* span, u64* max_span, u32* status) {
  const u64 n = (u64)R + 1;
  k_rank_off<<<(unsigned)((n + 255) / 256), 256, 0, L.stream>>>(
      rank_off, R, N, ts, span, (unsigned long long*)max_span, status);
  L.count();
}

// First rank whose samples start at or after each tile start (tile = fixed
// number of samples); tfr[n_tiles] = R so the last tile also owns the ranks
// that start at N (empty trailing ranks).
__global__ void k_tile_first_rank(const u64* __restrict__ rank_off, u32 R, u32 tile,
                                  u32 n_tiles, u32* tfr) {
  const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  if (t == n_tiles) {
    tfr[t] = R;
    return;
  }
  const u64 x = (u64)t * tile;
  u32 lo = 0, hi = R;
  while (lo < hi) {
    const u32 mid = lo + (hi - lo) / 2;
    if (rank_off[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  tfr[t] = lo;
}

void launch_tile_first_rank(const Launch& L, const u64* rank_off, u32 R, u32 tile, u32 n_tiles,
                            u32* tfr) {
  const u32 n = n_tiles + 1;
  k_tile_first_rank<<<(n + 255) / 256, 256, 0, L.stream>>>(rank_off, R, tile, n_tiles, tfr);
  L.count();
}

// ---------------------------------------------------------------------------
// Calling context tree: one root, parents in range, acyclic; depth of every
// node by pointer jumping (log2 C rounds); a node that has not reached the
// root after 2^rounds >= C jumps lies on a cycle.
__global__ void k_cct_init(const u32* __restrict__ parent, u32 C, u32* anc, u32* dep, u32* roots,
                           u32* status) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  const u32 p = parent[v];
  if (p == NONE32) {
    atomicAdd(roots, 1u);
    anc[v] = NONE32;
    dep[v] = 0;
  } else if (p >= C) {
    flag(status, F_BAD_CCT);
    anc[v] = NONE32;
    dep[v] = 0;
  } else {
    anc[v] = p;
    dep[v] = 1;
  }
}

__global__ void k_cct_jump(const u32* __restrict__ anc_in, const u32* __restrict__ dep_in,
                           u32* anc_out, u32* dep_out, u32 C) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  const u32 a = anc_in[v];
  if (a != NONE32) {
    dep_out[v] = min(dep_in[v] + dep_in[a], 0x7FFFFFFFu);
    anc_out[v] = anc_in[a];
  } else {
    dep_out[v] = dep_in[v];
    anc_out[v] = NONE32;
  }
}

__global__ void k_cct_final(const u32* __restrict__ anc, const u32* __restrict__ dep, u32 C,
                            u32* depth, u32* max_depth, u32* status) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= C) return;
  if (anc[v] != NONE32) flag(status, F_BAD_CCT);
  depth[v] = dep[v];
  atomicMax(max_depth, dep[v]);
}

void launch_cct(const Launch& L, const u32* parent, u32 C, u32* depth, u32* max_depth,
                u32* roots, u32* scratch, u32* status) {
  u32* anc0 = scratch;
  u32* dep0 = scratch + C;
  u32* anc1 = scratch + 2 * (u64)C;
  u32* dep1 = scratch + 3 * (u64)C;
  const unsigned g = (C + 255) / 256;
  k_cct_init<<<g, 256, 0, L.stream>>>(parent, C, anc0, dep0, roots, status);
  int rounds = 1;
  while (rounds < 40 && (1ull << rounds) < (u64)C) ++rounds;
  for (int i = 0; i < rounds; ++i) {
    k_cct_jump<<<g, 256, 0, L.stream>>>(anc0, dep0, anc1, dep1, C);
    std::swap(anc0, anc1);
    std::swap(dep0, dep1);
  }
  k_cct_final<<<g, 256, 0, L.stream>>>(anc0, dep0, C, depth, max_depth, status);
  L.count(2 + rounds);
}

__global__ void k_n_iter(const u64* __restrict__ row_off_of_rank, u32 R, u32* n_iter) {
  const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) n_iter[r] = (u32)(row_off_of_rank[r + 1] - row_off_of_rank[r] - 1);
}

void launch_n_iter(const Launch& L, const u64* row_off_of_rank, u32 R, u32* n_iter) {
  k_n_iter<<<(R + 255) / 256, 256, 0, L.stream>>>(row_off_of_rank, R, n_iter);
  L.count();
}

// ---------------------------------------------------------------------------
// Staging of aggregated entries: shared memory first, a per-CTA global region
// when a tile's rows do not fit (sized so that it cannot overflow).
constexpr u32 GBIT = 0x80000000u;

__device__ __forceinline__ u32 stage_alloc(u32 n, u32* top, u32* gtop, u32 cap, u32 gcap,
                                           u32* status, bool* ok) {
  *ok = true;
  const u32 o = atomicAdd(top, n);
  if (o + n <= cap) return o;
  const u32 g = atomicAdd(gtop, n);
  if (g + n > gcap) {
    flag(status, F_INTERNAL);
    *ok = false;
    return GBIT;
  }
  return g | GBIT;
}

struct Stage {
  u32* ctx;
  u64* time;
  u32* cnt;
};

__device__ __forceinline__ Stage stage_at(u32 soff, const Stage& sm, const Stage& gl) {
  Stage s;
  if (soff & GBIT) {
    const u32 o = soff & ~GBIT;
    s.ctx = gl.ctx + o;
    s.time = gl.time + o;
    s.cnt = gl.cnt + o;
  } else {
    s.ctx = sm.ctx + soff;
    s.time = sm.time + soff;
    s.cnt = sm.cnt + soff;
  }
  return s;
}

// ---------------------------------------------------------------------------
// The iteration tensor (Section V): one persistent kernel over tiles of T
// consecutive samples, claimed in order.  A tile owns the rows (rank prologues
// and iterations) that START inside it and reads past its end to finish its
// last row.  Per tile:
//   0. load samples to shared memory; validate contexts and timestamp order;
//      durations; rank starts; marker-run starts; prefix counts -> local rows
//   1. rows of at most LONG samples: one warp each, sorted distinct-context
//      aggregation with the warp's two-level bitmap
//   2. longer rows (and the row that runs past the tile): the whole CTA
//   3. prefix of entries; decoupled look-back gives the global row / entry
//      offsets; 4. write rows, rank offsets and entries.
template <int T, int NT>
__global__ void __launch_bounds__(NT) k_tensor(const TensorArgs A) {
  constexpr int W = NT / 32;
  constexpr int PER = T / NT;
  constexpr u32 CAP = T;
  constexpr u32 LONG = 1024;
  static_assert(T % NT == 0 && T <= 32768, "tile shape");
  extern __shared__ __align__(16) unsigned char sm[];
  u64* dur_s = (u64*)sm;                      // [T + 2] ts, then durations
  u32* ctx_s = (u32*)(dur_s + T + 2);         // [T]
  u32* nrs_s = ctx_s + T;                     // [T + 4] rank starts per position
  uint16_t* d_pos = (uint16_t*)(nrs_s + T + 4);  // [T] data-row start position
  uint16_t* d_mspre = d_pos + T;              // [T] marker starts before it
  u32* d_nrspre = (u32*)(d_mspre + T);        // [T] rank starts before it
  u32* d_nnz = d_nrspre + T;                  // [T] entries, then entry prefix
  u32* d_soff = d_nnz + T;                    // [T] stage offset
  Stage ss;
  ss.ctx = d_soff + T;                        // [CAP]
  ss.cnt = ss.ctx + CAP;                      // [CAP]
  ss.time = (u64*)(ss.cnt + CAP);             // [CAP]
  u32* bm_sm = (u32*)(ss.time + CAP);

  __shared__ u64 s_scan[W];
  __shared__ u32 s_tile, s_rs_lo, s_rs_hi, s_prevc, s_rank_at_b, s_ndata, s_ms_total, s_nend;
  __shared__ u32 s_stage_top, s_gtop, s_cnnz, s_csoff;
  __shared__ unsigned long long s_q;
  __shared__ u64 s_nrs_total, s_pre_rows, s_pre_ents;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 bmw = bm_words(A.C);
  u32* const bm_cta_base =
      A.bm_in_smem ? bm_sm : A.gbm + (u64)blockIdx.x * W * bmw;
  const Bm bm = bm_at(bm_cta_base + (u64)warp * bmw, A.C);
  const Bm bm0 = bm_at(bm_cta_base, A.C);
  if (A.bm_in_smem)
    for (u32 i = tid; i < W * bmw; i += NT) bm_sm[i] = 0;
  Stage gs;
  gs.ctx = A.gst_ctx + (u64)blockIdx.x * A.gst_cap;
  gs.time = A.gst_time + (u64)blockIdx.x * A.gst_cap;
  gs.cnt = A.gst_cnt + (u64)blockIdx.x * A.gst_cap;
  const u32 m = A.m, C = A.C;

  for (;;) {
    if (tid == 0) {
      s_tile = atomicAdd(A.unit_counter, 1u);
      s_q = ~0ull;
      s_stage_top = 0;
      s_gtop = 0;
    }
    __syncthreads();
    const u32 t = s_tile;
    if (t >= A.n_tiles) break;
    const u64 a = (u64)t * T;
    const u64 b = min(a + (u64)T, A.N);
    const u32 nrec = (u32)(b - a);
    const bool last = (t == A.n_tiles - 1);

    // ---- 0. load, validate, durations, row starts --------------------------
    if (tid == 0) {
      const u32 hi = A.tfr[t + 1];
      s_rs_lo = A.tfr[t];
      s_rs_hi = hi;
      s_prevc = a > 0 ? A.ctx[a - 1] : NONE32;
      s_rank_at_b = (!last && hi < A.R && A.rank_off[hi] == b) ? 1u : 0u;
      dur_s[nrec] = (b < A.N) ? A.ts[b] : 0ull;
    }
    for (u32 i = tid; i < T + 4; i += NT) nrs_s[i] = 0;
    for (u32 i = tid; i < nrec; i += NT) {
      ctx_s[i] = A.ctx[a + i];
      dur_s[i] = A.ts[a + i];
    }
    __syncthreads();
    const u32 rs_lo = s_rs_lo, rs_hi = s_rs_hi;
    for (u32 r = rs_lo + tid; r < rs_hi; r += NT) atomicAdd(&nrs_s[(u32)(A.rank_off[r] - a)], 1u);
    __syncthreads();

    u64 v[PER], du[PER];
    u32 cl[PER];
    {
      u32 fl = 0;
      const u32 prevc = s_prevc;
      const bool rab = s_rank_at_b != 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const u32 i = tid * PER + k;
        v[k] = 0;
        du[k] = 0;
        cl[k] = 0;
        if (i < nrec) {
          const u32 c = ctx_s[i];
          u32 cc = c;
          if (c >= C) {
            fl |= F_BAD_CTX;
            cc = 0;
          }
          const u32 pc = i > 0 ? ctx_s[i - 1] : prevc;
          const u32 nr = nrs_s[i];
          const bool nxt = (i + 1 < nrec) ? (nrs_s[i + 1] > 0) : ((b == A.N) || rab);
          if (!nxt) {
            const u64 t0 = dur_s[i], t1 = dur_s[i + 1];
            if (t1 < t0) fl |= F_NOT_SORTED;
            else du[k] = t1 - t0;
          }
          const u32 ms = (c == m && (nr > 0 || pc != m)) ? 1u : 0u;
          v[k] = ((u64)nr << 32) | ((nr + ms > 0) ? (1ull << 16) : 0ull) | ms;
          cl[k] = cc;
        }
      }
      if (fl) flag(A.status, fl);
    }
    u64 tsum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) tsum += v[k];
    u64 TOT;
    u64 run = block_excl_scan<NT>(tsum, s_scan, &TOT);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const u32 i = tid * PER + k;
      if (i < nrec) {
        dur_s[i] = du[k];
        ctx_s[i] = cl[k];
        if (v[k] & (1ull << 16)) {
          const u32 di = (u32)((run >> 16) & 0xFFFFu);
          d_pos[di] = (uint16_t)i;
          d_mspre[di] = (uint16_t)(run & 0xFFFFu);
          d_nrspre[di] = (u32)(run >> 32);
        }
      }
      run += v[k];
    }
    if (tid == 0) {
      s_ndata = (u32)((TOT >> 16) & 0xFFFFu);
      s_ms_total = (u32)(TOT & 0xFFFFu);
      s_nrs_total = TOT >> 32;
      s_nend = last ? nrs_s[nrec] : 0u;
    }
    __syncthreads();
    const u32 nd = s_ndata;

    // ---- end of the tile's last row: first row start at or after b --------
    u64 e = b;
    bool lz = true;  // the last row ends at a rank boundary (last sample 0 ns)
    if (nd > 0 && b < A.N) {
      const u64 qrank = (rs_hi < A.R) ? A.rank_off[rs_hi] : A.N;
      e = qrank;
      for (u64 q0 = b; q0 < qrank; q0 += NT) {
        const u64 q = q0 + tid;
        bool hit = false;
        if (q < qrank) hit = (A.ctx[q] == m) && (A.ctx[q - 1] != m);
        if (hit) atomicMin(&s_q, (unsigned long long)q);
        if (__syncthreads_or(hit)) break;
      }
      if (s_q != ~0ull) {
        e = s_q;
        lz = false;
      }
    }
    const u64 e_rel = e - a;

    // ---- 1. short rows, one warp each --------------------------------------
    for (u32 d = warp; d < nd; d += W) {
      const u32 s = d_pos[d];
      const u64 te = (d + 1 < nd) ? (u64)d_pos[d + 1] : e_rel;
      if (te > nrec || te - s > LONG) continue;
      const u32 tt = (u32)te;
      for (u32 j = s + lane; j < tt; j += 32) {
        const u32 c = ctx_s[j];
        if (j == s || ctx_s[j - 1] != c) bm_set(bm, c);
      }
      __syncwarp();
      const u32 nnz = bm_prefix_warp(bm, lane);
      u32 soff = 0;
      bool ok = true;
      if (lane == 0) soff = stage_alloc(nnz, &s_stage_top, &s_gtop, CAP, A.gst_cap, A.status, &ok);
      soff = __shfl_sync(FULL, soff, 0);
      ok = __shfl_sync(FULL, ok, 0);
      const Stage st = stage_at(soff, ss, gs);
      if (ok) {
        for (u32 k = lane; k < nnz; k += 32) {
          st.time[k] = 0;
          st.cnt[k] = 0;
        }
        __syncwarp();
        for (u32 j = s + lane; j < tt; j += 32) {
          const u32 c = ctx_s[j];
          const u32 k = bm_rank(bm, c);
          atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)dur_s[j]);
          atomicAdd(&st.cnt[k], 1u);
          st.ctx[k] = c;
        }
      }
      __syncwarp();
      bm_clear_warp(bm, lane);
      __syncwarp();
      if (lane == 0) {
        d_nnz[d] = ok ? nnz : 0u;
        d_soff[d] = soff;
      }
    }
    __syncthreads();

    // ---- 2. long rows and the row that continues past the tile: whole CTA --
    for (u32 d = 0; d < nd; ++d) {
      const u32 s = d_pos[d];
      const u64 te = (d + 1 < nd) ? (u64)d_pos[d + 1] : e_rel;
      if (!(te > nrec || te - s > LONG)) continue;
      for (u64 j = s + tid; j < te; j += NT) {
        u32 c = (j < nrec) ? ctx_s[j] : A.ctx[a + j];
        if (c >= C) c = 0;
        bool head = (j == s);
        if (!head) {
          u32 cp = (j - 1 < nrec) ? ctx_s[j - 1] : A.ctx[a + j - 1];
          if (cp >= C) cp = 0;
          head = cp != c;
        }
        if (head) bm_set(bm0, c);
      }
      __syncthreads();
      if (warp == 0) {
        const u32 nnz = bm_prefix_warp(bm0, lane);
        if (lane == 0) {
          bool ok = true;
          const u32 so = stage_alloc(nnz, &s_stage_top, &s_gtop, CAP, A.gst_cap, A.status, &ok);
          s_cnnz = ok ? nnz : 0u;
          s_csoff = so;
        }
      }
      __syncthreads();
      const u32 nnz = s_cnnz;
      const Stage st = stage_at(s_csoff, ss, gs);
      for (u32 k = tid; k < nnz; k += NT) {
        st.time[k] = 0;
        st.cnt[k] = 0;
      }
      __syncthreads();
      if (nnz > 0) {
        for (u64 j = s + tid; j < te; j += NT) {
          u32 c;
          u64 dd;
          if (j < nrec) {
            c = ctx_s[j];
            dd = dur_s[j];
          } else {
            const u64 gj = a + j;
            c = A.ctx[gj];
            if (c >= C) c = 0;
            const u64 t0 = A.ts[gj];
            if (j + 1 < te) {
              const u64 t1 = A.ts[gj + 1];
              dd = t1 >= t0 ? t1 - t0 : 0;
            } else if (lz) {
              dd = 0;
            } else {
              const u64 t1 = A.ts[a + te];
              dd = t1 >= t0 ? t1 - t0 : 0;
            }
          }
          const u32 k = bm_rank(bm0, c);
          atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)dd);
          atomicAdd(&st.cnt[k], 1u);
          st.ctx[k] = c;
        }
      }
      __syncthreads();
      if (warp == 0) bm_clear_warp(bm0, lane);
      if (tid == 0) {
        d_nnz[d] = nnz;
        d_soff[d] = s_csoff;
      }
      __syncthreads();
    }

    // ---- 3. entry prefix over the tile's data rows ---------------------------
    u64 EL;
    {
      u32 vals[PER];
      u64 nsum = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const u32 di = tid * PER + k;
        vals[k] = di < nd ? d_nnz[di] : 0u;
        nsum += vals[k];
      }
      u64 r2 = block_excl_scan<NT>(nsum, s_scan, &EL);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const u32 di = tid * PER + k;
        if (di < nd) d_nnz[di] = (u32)r2;
        r2 += vals[k];
      }
    }

    // ---- look-back: global row / entry offsets --------------------------------
    const u64 RL = s_nrs_total + s_ms_total + s_nend;
    if (tid == 0) {
      u64 pr, pe;
      lookback(A.ustat, t, RL, EL, &pr, &pe, A.status);
      s_pre_rows = pr;
      s_pre_ents = pe;
      if (last) {
        const u64 rows = pr + RL, nnz = pe + EL;
        A.totals[0] = rows;
        A.totals[1] = nnz;
        A.row_off_of_rank[A.R] = rows;
        if (rows + 1 > A.rows_cap || nnz > A.nnz_cap) flag(A.status, F_CAPACITY);
        else A.entry_off[rows] = nnz;
      }
    }
    __syncthreads();
    const u64 PR = s_pre_rows, PE = s_pre_ents;

    // ---- 4. outputs ----------------------------------------------------------
    for (u32 d = warp; d < nd; d += W) {
      const u32 pos = d_pos[d];
      const u32 nrs = nrs_s[pos];
      const u32 ms = (u32)((d + 1 < nd) ? d_mspre[d + 1] : s_ms_total) - d_mspre[d];
      const u64 row0 = PR + d_nrspre[d] + d_mspre[d];
      const u64 eo = PE + d_nnz[d];
      const u32 nrow = nrs + ms;
      for (u32 k = lane; k < nrow; k += 32)
        if (row0 + k < A.rows_cap) A.entry_off[row0 + k] = eo;
      for (u32 k = lane; k < nrs; k += 32)
        A.row_off_of_rank[rs_lo + d_nrspre[d] + k] = row0 + k;
      const u32 nnz = (u32)(((d + 1 < nd) ? (u64)d_nnz[d + 1] : EL) - d_nnz[d]);
      const Stage st = stage_at(d_soff[d], ss, gs);
      for (u32 k = lane; k < nnz; k += 32) {
        const u64 g = eo + k;
        if (g < A.nnz_cap) {
          A.e_ctx[g] = vld(&st.ctx[k]);
          A.e_time[g] = vld(&st.time[k]);
          A.e_cnt[g] = vld(&st.cnt[k]);
        }
      }
    }
    if (last) {  // empty ranks that start at N
      const u32 ne = s_nend;
      const u64 row0 = PR + s_nrs_total + s_ms_total;
      for (u32 k = tid; k < ne; k += NT) {
        if (row0 + k < A.rows_cap) A.entry_off[row0 + k] = PE + EL;
        A.row_off_of_rank[A.R - ne + k] = row0 + k;
      }
    }
    __syncthreads();
  }
}

constexpr int TENSOR_T = 1024;
constexpr int TENSOR_NT = 256;

static size_t tensor_smem_base(int T) {
  const int CAP = T;
  return (size_t)8 * (T + 2) + 4 * T + 4 * (T + 4) + 2 * T + 2 * T + 3 * 4 * T + 16 * (size_t)CAP;
}

TensorPlan plan_tensor(u32 C, u64 N, int num_sms) {
  TensorPlan P;
  P.tile = TENSOR_T;
  P.threads = TENSOR_NT;
  const size_t base = tensor_smem_base(TENSOR_T);
  const size_t bm = (size_t)(TENSOR_NT / 32) * bm_words(C) * 4;
  P.bm_in_smem = base + bm <= 110 * 1024;
  P.smem = base + (P.bm_in_smem ? bm : 0);
  auto kern = k_tensor<TENSOR_T, TENSOR_NT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TENSOR_NT, P.smem);
  if (occ < 1) occ = 1;
  const u64 n_tiles = std::max<u64>(1, (N + TENSOR_T - 1) / TENSOR_T);
  P.grid = (int)std::min<u64>((u64)num_sms * occ, n_tiles);
  P.gst_cap = TENSOR_T + C;
  return P;
}

void launch_tensor(const Launch& L, const TensorPlan& P, const TensorArgs& A) {
  k_tensor<TENSOR_T, TENSOR_NT><<<P.grid, P.threads, P.smem, L.stream>>>(A);
  L.count();
}

// ---------------------------------------------------------------------------
// Per-rank CSR of distinct contexts.  Work unit = W consecutive ranks (one
// per warp), claimed in order; look-back over units gives output offsets.
//  mode 0 (exclusive, Section V): union of the rank's tensor rows, summed.
//  mode 1 (inclusive, Sections II-A / VI-B): the ancestor closure of the
//    rank's exclusive contexts, values rolled up level by level from the
//    deepest level to the root (every node of depth d adds into its parent
//    before any node of depth d-1 is read).
template <int NT>
__global__ void __launch_bounds__(NT) k_rank_csr(const RankCsrArgs A) {
  constexpr int W = NT / 32;
  constexpr u32 CAP = 4096;
  extern __shared__ __align__(16) unsigned char sm[];
  Stage ss;
  ss.time = (u64*)sm;
  ss.ctx = (u32*)(ss.time + CAP);
  ss.cnt = ss.ctx + CAP;
  u32* bm_sm = ss.cnt + CAP;
  __shared__ u32 s_unit, s_top, s_gtop;
  __shared__ u32 s_nnz[W], s_soff[W];
  __shared__ u64 s_eoff[W];
  __shared__ u64 s_pre;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 bmw = bm_words(A.C);
  u32* const bm_cta_base = A.bm_in_smem ? bm_sm : A.gbm + (u64)blockIdx.x * W * bmw;
  const Bm bm = bm_at(bm_cta_base + (u64)warp * bmw, A.C);
  if (A.bm_in_smem)
    for (u32 i = tid; i < W * bmw; i += NT) bm_sm[i] = 0;
  Stage gs;
  gs.ctx = A.gst_ctx + (u64)blockIdx.x * A.gst_cap;
  gs.time = A.gst_time + (u64)blockIdx.x * A.gst_cap;
  gs.cnt = A.gst_cnt + (u64)blockIdx.x * A.gst_cap;
  const u32 n_units = (A.R + W - 1) / W;

  for (;;) {
    if (tid == 0) {
      s_unit = atomicAdd(A.unit_counter, 1u);
      s_top = 0;
      s_gtop = 0;
    }
    __syncthreads();
    const u32 g = s_unit;
    if (g >= n_units) break;
    const u32 r = g * W + warp;
    u32 nnz = 0, soff = 0;
    if (r < A.R) {
      u64 E0, E1;
      const u32* in_ctx = A.in_ctx;
      if (A.mode == 0) {
        E0 = A.entry_off[A.row_off_of_rank[r]];
        E1 = A.entry_off[A.row_off_of_rank[r + 1]];
        for (u64 j = E0 + lane; j < E1; j += 32) {
          const u32 c = in_ctx[j];
          if (!bm_has(bm, c)) bm_set(bm, c);
        }
      } else {
        E0 = A.in_off[r];
        E1 = A.in_off[r + 1];
        for (u64 j = E0 + lane; j < E1; j += 32) {
          u32 c = in_ctx[j];
          for (u32 step = 0; c != NONE32 && step <= A.max_depth; ++step) {
            if (bm_test_set(bm, c)) break;
            c = A.parent[c];
          }
        }
      }
      __syncwarp();
      nnz = bm_prefix_warp(bm, lane);
      bool ok = true;
      if (lane == 0) soff = stage_alloc(nnz, &s_top, &s_gtop, CAP, A.gst_cap, A.status, &ok);
      soff = __shfl_sync(FULL, soff, 0);
      ok = __shfl_sync(FULL, ok, 0);
      const Stage st = stage_at(soff, ss, gs);
      if (ok) {
        for (u32 k = lane; k < nnz; k += 32) {
          st.time[k] = 0;
          st.cnt[k] = 0;
        }
        __syncwarp();
        if (A.mode == 0) {
          for (u64 j = E0 + lane; j < E1; j += 32) {
            const u32 c = in_ctx[j];
            const u32 k = bm_rank(bm, c);
            atomicAdd((unsigned long long*)&st.time[k], (unsigned long long)A.in_time[j]);
            atomicAdd(&st.cnt[k], A.in_cnt[j]);
            st.ctx[k] = c;
          }
        } else {
          bm_enumerate_warp(bm, st.ctx, lane);
          for (u64 j = E0 + lane; j < E1; j += 32) {
            const u32 k = bm_rank(bm, in_ctx[j]);
            st.time[k] = A.in_time[j];
            st.cnt[k] = A.in_cnt[j];
          }
          __syncwarp();
          for (u32 d = A.max_depth; d >= 1; --d) {
            for (u32 k = lane; k < nnz; k += 32) {
              const u32 c = vld(&st.ctx[k]);
              if (A.depth[c] == d) {
                const u32 kp = bm_rank(bm, A.parent[c]);
                atomicAdd((unsigned long long*)&st.time[kp], (unsigned long long)vld(&st.time[k]));
                atomicAdd(&st.cnt[kp], vld(&st.cnt[k]));
              }
            }
            __syncwarp();
          }
        }
      } else {
        nnz = 0;
      }
      __syncwarp();
      bm_clear_warp(bm, lane);
      __syncwarp();
    }
    if (lane == 0) {
      s_nnz[warp] = nnz;
      s_soff[warp] = soff;
    }
    __syncthreads();
    if (warp == 0) {
      const u32 x = lane < W ? s_nnz[lane] : 0u;
      const u64 incl = warp_incl_scan((u64)x, lane);
      if (lane < W) s_eoff[lane] = incl - x;
      const u64 tot = __shfl_sync(FULL, incl, 31);
      if (lane == 0) {
        u64 pre, dummy;
        lookback(A.ustat, g, tot, 0, &pre, &dummy, A.status);
        s_pre = pre;
        if (g == n_units - 1) {
          A.total[0] = pre + tot;
          A.out_off[A.R] = pre + tot;
          if (pre + tot > A.nnz_cap) flag(A.status, F_CAPACITY);
        }
      }
    }
    __syncthreads();
    if (r < A.R) {
      const u64 eo = s_pre + s_eoff[warp];
      if (lane == 0) A.out_off[r] = eo;
      const Stage st = stage_at(s_soff[warp], ss, gs);
      const u32 n = s_nnz[warp];
      for (u32 k = lane; k < n; k += 32) {
        const u64 gk = eo + k;
        if (gk < A.nnz_cap) {
          A.out_ctx[gk] = vld(&st.ctx[k]);
          A.out_time[gk] = vld(&st.time[k]);
          A.out_cnt[gk] = vld(&st.cnt[k]);
        }
      }
    }
    __syncthreads();
  }
}

constexpr int RANK_NT = 256;

RankCsrPlan plan_rank_csr(u32 R, u32 C, int num_sms) {
  RankCsrPlan P;
  P.threads = RANK_NT;
  const size_t base = (size_t)4096 * 16;
  const size_t bm = (size_t)(RANK_NT / 32) * bm_words(C) * 4;
  P.bm_in_smem = base + bm <= 110 * 1024;
  P.smem = base + (P.bm_in_smem ? bm : 0);
  auto kern = k_rank_csr<RANK_NT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, RANK_NT, P.smem);
  if (occ < 1) occ = 1;
  P.n_units = (R + RANK_NT / 32 - 1) / (RANK_NT / 32);
  P.grid = (int)std::min<u64>((u64)num_sms * occ, P.n_units);
  P.gst_cap = (RANK_NT / 32) * C;
  return P;
}

void launch_rank_csr(const Launch& L, const RankCsrPlan& P, const RankCsrArgs& A) {
  k_rank_csr<RANK_NT><<<P.grid, P.threads, P.smem, L.stream>>>(A);
  L.count();
}

}  // namespace ta
