// columns.cu -- the operation classes the paper times its DataFrame backends
// with on trace events (Section IV, Tables I-III), as kernels over device
// columns: the events table of an experiment, sorting (LSD radix sort),
// filtering (stream compaction), grouping by (segment, key) (per-segment
// bitmaps, as the rank passes), merging (a gather join on row ids), and the
// elementwise / reduction / scan classes.
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

inline unsigned nblk(u64 n, int nt = 256, u64 cap = 1u << 20) {
  return (unsigned)std::max<u64>(1, std::min<u64>((n + nt - 1) / nt, cap));
}

// ---------------------------------------------------------- events table --
__global__ void k_events(const u64* __restrict__ rank_off, const u64* __restrict__ ts,
                         const u32* __restrict__ ctx, u32 r0, u32 n_ranks, u64 base, u32* orank,
                         u64* ots, u32* octx, u64* odur) {
  const int lane = threadIdx.x & 31;
  const u64 G = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 k = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_ranks; k += G) {
    const u32 r = r0 + (u32)k;
    const u64 b = rank_off[r], e = rank_off[r + 1];
    for (u64 i = b + lane; i < e; i += 32) {
      const u64 o = i - base;
      const u64 t = ts[i];
      if (orank) orank[o] = r;
      if (ots) ots[o] = t;
      if (octx) octx[o] = ctx[i];
      if (odur) odur[o] = i + 1 < e ? ts[i + 1] - t : 0ull;
    }
  }
}

// --------------------------------------------------------- radix sort ----
// A pass orders by one 8-bit digit, stably: per tile of 4096 rows a digit
// histogram (warp-aggregated shared atomics), a digit-major exclusive scan
// of all tiles' histograms (so tile t's rows of digit d follow every earlier
// tile's), then a scatter.  In the scatter each warp owns 512 consecutive
// rows of the tile: its digit counts, then per digit the
// tile-local start (a scan over digits) and each warp's start within it,
// then each row's rank among equal digits of its 32-row round (nine
// ballots) places it in a shared-memory copy of the tile ordered
// by digit; the copy is written out in order, so rows of one digit go to
// consecutive addresses (coalesced) instead of 4096 scattered stores.
constexpr int RS_NT = 256, RS_WARPS = RS_NT / 32, RS_PER_WARP = 512;
constexpr int RS_ITEMS = RS_PER_WARP / 32;
constexpr u32 RS_TILE = RS_WARPS * RS_PER_WARP;
constexpr size_t RS_SMEM = (size_t)RS_TILE * 12;  // keys u64 + values u32

// Lanes of the warp holding the same 8-bit digit (valid lanes only match
// valid lanes): nine ballots, constant time whatever the digit mix.
__device__ __forceinline__ u32 digit_peers(u32 d, bool v) {
  u32 peers = __ballot_sync(FULL, v);
  if (!v) peers = ~peers;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1u;
    const u32 bal = __ballot_sync(FULL, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

__global__ void __launch_bounds__(RS_NT) k_rs_count(const u64* __restrict__ keys, u64 n, u32 shift,
                                                    u64 n_tiles, u32* hist) {
  __shared__ u32 h[256];
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  h[threadIdx.x] = 0;
  __syncthreads();
  const u64 base = (u64)blockIdx.x * RS_TILE;
  for (u32 k = threadIdx.x; k < RS_TILE; k += RS_NT) {
    const u64 i = base + k;
    const bool v = i < n;
    const u32 d = v ? (u32)(keys[i] >> shift) & 255u : 0u;
    const u32 peers = digit_peers(d, v);
    if (v && (peers & lt) == 0) atomicAdd(&h[d], (u32)__popc(peers));
  }
  __syncthreads();
  hist[(u64)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_NT, 2) k_rs_scatter(const u64* __restrict__ keys_in,
                                                      const u32* __restrict__ vals_in, u64 n,
                                                      u32 shift, u64 n_tiles,
                                                      const u64* __restrict__ off, u64* keys_out,
                                                      u32* vals_out) {
  extern __shared__ __align__(16) unsigned char rs_sm[];
  u64* skey = (u64*)rs_sm;
  u32* sval = (u32*)(skey + RS_TILE);
  __shared__ u32 wh[RS_WARPS][256];
  __shared__ u32 lstart[256];
  __shared__ u32 gbase[256];  // n < 2^32: offsets fit 32 bits (3 CTAs per SM fit)
  __shared__ u32 wsum[RS_WARPS];
  __shared__ u32 speers[RS_WARPS][RS_ITEMS][32];  // each row's equal-digit lanes
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  for (u32 d = lane; d < 256; d += 32) wh[w][d] = 0;
  const u64 tbase = (u64)blockIdx.x * RS_TILE;
  const u64 wbase = tbase + (u64)w * RS_PER_WARP;
  __syncwarp();
#pragma unroll 4
  for (int rd = 0; rd < RS_ITEMS; ++rd) {
    const u64 i = wbase + (u64)rd * 32 + lane;
    const bool v = i < n;
    const u32 d = v ? (u32)(keys_in[i] >> shift) & 255u : 0u;
    const u32 peers = digit_peers(d, v);
    speers[w][rd][lane] = peers;
    if (v && (peers & lt) == 0) wh[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // thread t owns digit t: tile-local start (scan over digits), warp starts
    const u32 d = threadIdx.x;
    u32 cnt = 0;
    for (int q = 0; q < RS_WARPS; ++q) cnt += wh[q][d];
    const u32 incl = warp_incl_scan(cnt, lane);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    u32 before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    const u32 start = before + incl - cnt;
    lstart[d] = start;
    gbase[d] = (u32)off[(u64)d * n_tiles + blockIdx.x];
    u32 run = start;
    for (int q = 0; q < RS_WARPS; ++q) {
      const u32 c = wh[q][d];
      wh[q][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int rd = 0; rd < RS_ITEMS; ++rd) {
    const u64 i = wbase + (u64)rd * 32 + lane;
    const bool v = i < n;
    const u64 key = v ? keys_in[i] : 0ull;  // a second read of the tile, from L2
    const u32 d = (u32)(key >> shift) & 255u;
    const u32 peers = speers[w][rd][lane];  // own lane's entry: no barrier needed
    const u32 pos = v ? wh[w][d] + __popc(peers & lt) : 0u;
    __syncwarp();
    if (v && (peers & lt) == 0) wh[w][d] += __popc(peers);
    __syncwarp();
    if (v) {
      skey[pos] = key;
      sval[pos] = vals_in ? vals_in[i] : (u32)i;
    }
  }
  __syncthreads();
  const u32 m = (u32)min((u64)RS_TILE, n - tbase);
  for (u32 j = threadIdx.x; j < m; j += RS_NT) {
    const u64 key = skey[j];
    const u32 d = (u32)(key >> shift) & 255u;
    const u64 g = (u64)gbase[d] + (j - lstart[d]);
    keys_out[g] = key;
    vals_out[g] = sval[j];
  }
}

__global__ void k_max_u64(const u64* __restrict__ a, u64 n, unsigned long long* out) {
  u64 m = 0;
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) m = max(m, a[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, (u64)__shfl_xor_sync(FULL, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)m);
}

__global__ void k_iota(u32* p, u64 n) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) p[i] = (u32)i;
}

// ------------------------------------------------------------ filtering --
constexpr int FL_NT = 256, FL_ROUNDS = 16;
constexpr u32 FL_TILE = FL_NT * FL_ROUNDS;

__global__ void __launch_bounds__(FL_NT) k_flt_count(const u64* __restrict__ col, u64 n, u64 lo,
                                                     u64 hi, u32* cnt) {
  __shared__ u32 s[FL_NT / 32];
  const u64 base = (u64)blockIdx.x * FL_TILE;
  u32 c = 0;
  for (int r = 0; r < FL_ROUNDS; ++r) {
    const u64 i = base + (u64)r * FL_NT + threadIdx.x;
    if (i < n) {
      const u64 v = col[i];
      c += (v >= lo && v <= hi) ? 1u : 0u;
    }
  }
  c = __reduce_add_sync(FULL, c);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 t = 0;
    for (int q = 0; q < FL_NT / 32; ++q) t += s[q];
    cnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(FL_NT) k_flt_write(const u64* __restrict__ col, u64 n, u64 lo,
                                                     u64 hi, const u64* __restrict__ toff,
                                                     u32* out) {
  __shared__ u32 s[FL_NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  const u64 base = (u64)blockIdx.x * FL_TILE;
  u64 run = toff[blockIdx.x];
  for (int r = 0; r < FL_ROUNDS; ++r) {
    const u64 i = base + (u64)r * FL_NT + threadIdx.x;
    bool m = false;
    if (i < n) {
      const u64 v = col[i];
      m = v >= lo && v <= hi;
    }
    const u32 bal = __ballot_sync(FULL, m);
    if (lane == 0) s[w] = __popc(bal);
    __syncthreads();
    u32 before = 0, total = 0;
    for (int q = 0; q < FL_NT / 32; ++q) {
      const u32 c = s[q];
      before += q < w ? c : 0u;
      total += c;
    }
    if (m) out[run + before + __popc(bal & lt)] = (u32)i;
    run += total;
    __syncthreads();
  }
}

// ------------------------------------------------------------- grouping --
constexpr int GW = 8;       // warps per CTA
constexpr u32 GSR = 256;    // entries staged in shared memory per warp
constexpr u32 kGStage = GSR * 16;

struct GroupArgs {
  const u64* seg_off;
  const u32* key;
  const u64* val;
  u32 n_seg, n_keys;
  u32* cnt;
  const u64* off;
  u32* out_key;
  u64* out_sum;
  u32* out_cnt;
  u32* gbm;
  u32* gst_key;
  u64* gst_sum;
  u32* gst_cnt;
};

__device__ __forceinline__ void grp_mark(const GroupArgs& A, const Bm& bm, u64 b, u64 e, int lane) {
  for (u64 j0 = b; j0 < e; j0 += 32 * 8) {
    u32 c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const u64 j = j0 + 32 * q + lane;
      c[q] = j < e ? A.key[j] : NONE32;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (c[q] != NONE32 && !bm_has(bm, c[q])) bm_set(bm, c[q]);
  }
}

template <bool BMS>
__global__ void __launch_bounds__(GW * 32) k_grp_count(const GroupArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.n_keys);
  const u64 gw = (u64)blockIdx.x * GW + warp, G = (u64)gridDim.x * GW;
  const Bm bm = bm_at(BMS ? (u32*)(sm + (size_t)warp * bmw * 4) : A.gbm + gw * bmw, A.n_keys);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  __syncwarp();
  for (u64 s = gw; s < A.n_seg; s += G) {
    grp_mark(A, bm, A.seg_off[s], A.seg_off[s + 1], lane);
    __syncwarp();
    const u32 n = bm_count_warp(bm, lane);
    if (lane == 0) A.cnt[s] = n;
    bm_clear_warp(bm, lane);
    __syncwarp();
  }
}

template <bool BMS>
__global__ void __launch_bounds__(GW * 32) k_grp_write(const GroupArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 bmw = bm_words(A.n_keys);
  const u32 wbytes = kGStage + (BMS ? bmw * 4 : 0);
  unsigned char* ws = sm + (size_t)warp * wbytes;
  const u64 gw = (u64)blockIdx.x * GW + warp, G = (u64)gridDim.x * GW;
  const Bm bm = bm_at(BMS ? (u32*)(ws + kGStage) : A.gbm + gw * bmw, A.n_keys);
  if (BMS)
    for (u32 i = lane; i < bmw; i += 32) bm.L1[i] = 0;
  u64* s_sum = (u64*)ws;
  u32* s_key = (u32*)(ws + 8 * GSR);
  u32* s_cnt = (u32*)(ws + 12 * GSR);
  const u64 gbase = gw * (u64)A.n_keys;
  __syncwarp();
  for (u64 s = gw; s < A.n_seg; s += G) {
    const u64 b = A.seg_off[s], e = A.seg_off[s + 1];
    grp_mark(A, bm, b, e, lane);
    __syncwarp();
    const u32 nnz = bm_prefix_warp(bm, lane);
    const bool sh = nnz <= GSR;
    u64* st_sum = sh ? s_sum : A.gst_sum + gbase;
    u32* st_key = sh ? s_key : A.gst_key + gbase;
    u32* st_cnt = sh ? s_cnt : A.gst_cnt + gbase;
    for (u32 q = lane; q < nnz; q += 32) {
      st_sum[q] = 0;
      st_cnt[q] = 0;
    }
    __syncwarp();
    for (u64 j0 = b; j0 < e; j0 += 32 * 4) {
      u32 c[4];
      u64 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const u64 j = j0 + 32 * q + lane;
        const bool ok = j < e;
        c[q] = ok ? A.key[j] : NONE32;
        v[q] = ok ? A.val[j] : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (c[q] == NONE32) continue;
        const u32 p = bm_rank(bm, c[q]);
        atomicAdd((unsigned long long*)&st_sum[p], (unsigned long long)v[q]);
        atomicAdd(&st_cnt[p], 1u);
        st_key[p] = c[q];
      }
    }
    __syncwarp();
    const u64 eo = A.off[s];
    for (u32 q = lane; q < nnz; q += 32) {
      A.out_key[eo + q] = vld(&st_key[q]);
      A.out_sum[eo + q] = vld(&st_sum[q]);
      A.out_cnt[eo + q] = vld(&st_cnt[q]);
    }
    bm_clear_warp(bm, lane);
    __syncwarp();
  }
}

__global__ void k_grp_check(const u64* __restrict__ seg_off, u32 n_seg, u64 n,
                            const u32* __restrict__ key, u32 n_keys, u32* status) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n || i <= n_seg; i += G) {
    if (i < n && key[i] >= n_keys) flag(status, F_INVALID);
    if (i <= n_seg) {
      const u64 s = seg_off[i];
      if ((i == 0 && s != 0) || (i == n_seg && s != n) || (i > 0 && s < seg_off[i - 1]))
        flag(status, F_INVALID);
    }
  }
}

// ------------------------------------------------------ elementwise etc. --
__global__ void k_gather(const u32* __restrict__ key, u64 n, const u32* __restrict__ dim,
                         u32 n_dim, u32* out, u32* status) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) {
    const u32 k = key[i];
    if (k < n_dim) {
      out[i] = dim[k];
    } else {
      out[i] = 0;
      flag(status, F_INVALID);
    }
  }
}

__global__ void k_compare(const u64* __restrict__ a, u64 n, u64 c, uint8_t* m) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) m[i] = a[i] > c ? 1 : 0;
}

__global__ void k_add(const u64* __restrict__ a, const u64* __restrict__ b, u64 n, u64* out) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) out[i] = a[i] + b[i];
}

__global__ void k_scale(u64* a, u64 n, u64 s) {
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) a[i] *= s;
}

__global__ void k_sum(const u64* __restrict__ a, u64 n, unsigned long long* out) {
  u64 s = 0;
  const u64 G = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += G) s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)s);
}

struct Scope {
  ta_ctx* c;
  Launch L;
  Pool tmp;
  explicit Scope(ta_ctx* c_) : c(c_), L{c_->stream, c_->num_sms, &c_->launches}, tmp{c_, {}} {
    cudaSetDevice(c->device);
  }
  ~Scope() {
    cudaStreamSynchronize(c->stream);
    tmp.release();
  }
};

unsigned grid_for(const ta_ctx* c, u64 n) {
  return nblk(n, 256, (u64)c->num_sms * 16);
}

}  // namespace
}  // namespace ta

using namespace ta;

extern "C" ta_status ta_events_table(ta_experiment* e, uint32_t r0, uint32_t r1, uint32_t* rank,
                                     uint64_t* ts, uint32_t* ctx, uint64_t* dur,
                                     uint64_t* n_out) {
  if (!e || !n_out) return fail(TA_ERR_INVALID_ARG, "ta_events_table: NULL argument");
  if (r0 > r1 || r1 > e->R)
    return fail(TA_ERR_INVALID_ARG, "ta_events_table: ranks [%u, %u) of %u", r0, r1, e->R);
  if (!e->ts && e->N > 0)
    return fail(TA_ERR_STATE, "ta_events_table: the traces were released after loading");
  Scope S(e->ctx);
  u64 ro[2];
  TRY(copy(S.c, &ro[0], e->rank_off + r0, 8));
  TRY(copy(S.c, &ro[1], e->rank_off + r1, 8));
  TRY(sync_check(S.c, "ta_events_table"));
  *n_out = ro[1] - ro[0];
  if (r1 > r0 && (rank || ts || ctx || dur)) {
    const u64 warps = std::min<u64>(r1 - r0, (u64)S.c->num_sms * 64);
    k_events<<<(unsigned)((warps + 7) / 8), 256, 0, S.c->stream>>>(
        e->rank_off, e->ts, e->ctxv, r0, r1 - r0, ro[0], rank, ts, ctx, dur);
    S.L.count();
  }
  return sync_check(S.c, "ta_events_table");
}

extern "C" ta_status ta_col_sort(ta_ctx* c, const uint64_t* keys, uint64_t n, uint64_t* keys_out,
                                 uint32_t* perm) {
  if (!c || (n && (!keys || !keys_out || !perm)))
    return fail(TA_ERR_INVALID_ARG, "ta_col_sort: NULL argument");
  if (n >= (1ull << 32)) return fail(TA_ERR_INVALID_ARG, "ta_col_sort: n >= 2^32");
  if (n == 0) return TA_OK;
  Scope S(c);
  unsigned long long* mx;
  TRY(S.tmp.get_n(1, &mx, "sort max"));
  cudaMemsetAsync(mx, 0, 8, c->stream);
  k_max_u64<<<grid_for(c, n), 256, 0, c->stream>>>(keys, n, mx);
  S.L.count();
  u64 h = 0;
  TRY(copy(c, &h, mx, 8));
  TRY(sync_check(c, "ta_col_sort (max)"));
  int P = 0;
  while (P < 8 && (h >> (8 * P)) != 0) ++P;
  if (P == 0) {  // every key equal (0): already sorted
    TRY(copy(c, keys_out, keys, n * 8));
    k_iota<<<grid_for(c, n), 256, 0, c->stream>>>(perm, n);
    S.L.count();
    return sync_check(c, "ta_col_sort");
  }
  const u64 n_tiles = (n + RS_TILE - 1) / RS_TILE;
  u64 *tk, *off, *scratch;
  u32 *tv, *hist;
  TRY(S.tmp.get_n(n, &tk, "sort keys"));
  TRY(S.tmp.get_n(n, &tv, "sort values"));
  TRY(S.tmp.get_n(256 * n_tiles, &hist, "sort histograms"));
  TRY(S.tmp.get_n(256 * n_tiles + 1, &off, "sort offsets"));
  TRY(S.tmp.get_n(scan_scratch_elems(256 * n_tiles), &scratch, "sort scan"));
  cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM);
  u64* kb[2] = {keys_out, tk};
  u32* vb[2] = {perm, tv};
  for (int p = 0; p < P; ++p) {
    const int o = (P - 1 - p) & 1, i = (P - p) & 1;
    const u64* kin = p == 0 ? keys : kb[i];
    const u32* vin = p == 0 ? nullptr : vb[i];
    const u32 shift = 8u * p;
    k_rs_count<<<(unsigned)n_tiles, RS_NT, 0, c->stream>>>(kin, n, shift, n_tiles, hist);
    S.L.count();
    scan_exclusive(S.L, hist, 256 * n_tiles, off, off + 256 * n_tiles, scratch);
    k_rs_scatter<<<(unsigned)n_tiles, RS_NT, RS_SMEM, c->stream>>>(kin, vin, n, shift, n_tiles,
                                                                   off, kb[o], vb[o]);
    S.L.count();
  }
  return sync_check(c, "ta_col_sort");
}

extern "C" ta_status ta_col_filter(ta_ctx* c, const uint64_t* col, uint64_t n, uint64_t lo,
                                   uint64_t hi, uint32_t* idx_out, uint64_t* n_out) {
  if (!c || !n_out || (n && (!col || !idx_out)))
    return fail(TA_ERR_INVALID_ARG, "ta_col_filter: NULL argument");
  if (n >= (1ull << 32)) return fail(TA_ERR_INVALID_ARG, "ta_col_filter: n >= 2^32");
  *n_out = 0;
  if (n == 0) return TA_OK;
  Scope S(c);
  const u64 nt = (n + FL_TILE - 1) / FL_TILE;
  u32* cnt;
  u64 *toff, *scratch;
  TRY(S.tmp.get_n(nt, &cnt, "filter counts"));
  TRY(S.tmp.get_n(nt + 1, &toff, "filter offsets"));
  TRY(S.tmp.get_n(scan_scratch_elems(nt), &scratch, "filter scan"));
  k_flt_count<<<(unsigned)nt, FL_NT, 0, c->stream>>>(col, n, lo, hi, cnt);
  S.L.count();
  scan_exclusive(S.L, cnt, nt, toff, toff + nt, scratch);
  k_flt_write<<<(unsigned)nt, FL_NT, 0, c->stream>>>(col, n, lo, hi, toff, idx_out);
  S.L.count();
  TRY(copy(c, n_out, toff + nt, 8));
  return sync_check(c, "ta_col_filter");
}

extern "C" ta_status ta_col_group(ta_ctx* c, const uint64_t* seg_off, uint32_t n_seg,
                                  const uint32_t* key, uint32_t n_keys, const uint64_t* val,
                                  uint64_t n, uint64_t* off_out, uint32_t* key_out,
                                  uint64_t* sum_out, uint32_t* cnt_out, uint64_t out_cap,
                                  uint64_t* n_out) {
  if (!c || !seg_off || !n_out || (n && (!key || !val)) || n_keys == 0)
    return fail(TA_ERR_INVALID_ARG, "ta_col_group: NULL argument or n_keys = 0");
  if (n >= (1ull << 32)) return fail(TA_ERR_INVALID_ARG, "ta_col_group: n >= 2^32");
  Scope S(c);
  u32* status;
  TRY(S.tmp.get_n(1, &status, "group status"));
  cudaMemsetAsync(status, 0, 4, c->stream);
  k_grp_check<<<grid_for(c, std::max<u64>(n, (u64)n_seg + 1)), 256, 0, c->stream>>>(
      seg_off, n_seg, n, key, n_keys, status);
  S.L.count();
  u32 f = 0;
  TRY(copy(c, &f, status, 4));
  TRY(sync_check(c, "ta_col_group (check)"));
  if (f)
    return fail(TA_ERR_INVALID_ARG,
                "ta_col_group: segment offsets not 0..n non-decreasing, or a key >= n_keys");
  GroupArgs A;
  std::memset(&A, 0, sizeof A);
  A.seg_off = seg_off;
  A.key = key;
  A.val = val;
  A.n_seg = n_seg;
  A.n_keys = n_keys;
  const size_t bm = (size_t)bm_words(n_keys) * 4;
  const bool bms = kGStage + bm <= 16 * 1024;
  const size_t smc = bms ? bm * GW : 0, smw = (kGStage + (bms ? bm : 0)) * GW;
  const void* kc = bms ? (const void*)k_grp_count<true> : (const void*)k_grp_count<false>;
  const void* kw = bms ? (const void*)k_grp_write<true> : (const void*)k_grp_write<false>;
  cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
  cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
  int oc = 0, ow = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, kc, GW * 32, smc);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ow, kw, GW * 32, smw);
  const u64 need = std::max<u64>(1, ((u64)n_seg + GW - 1) / GW);
  const unsigned gc = (unsigned)std::min<u64>((u64)c->num_sms * std::max(oc, 1), need);
  const unsigned gwr = (unsigned)std::min<u64>((u64)c->num_sms * std::max(ow, 1), need);
  const u64 warps = (u64)std::max(gc, gwr) * GW;
  if (!bms) {
    TRY(S.tmp.get(warps * bm, (void**)&A.gbm, "group bitmaps"));
    cudaMemsetAsync(A.gbm, 0, warps * bm, c->stream);
  }
  u64 *off, *scratch;
  TRY(S.tmp.get_n(std::max<u32>(n_seg, 1), &A.cnt, "group counts"));
  TRY(S.tmp.get_n((u64)n_seg + 1, &off, "group offsets"));
  TRY(S.tmp.get_n(scan_scratch_elems(n_seg), &scratch, "group scan"));
  if (n_seg) {
    if (bms) k_grp_count<true><<<gc, GW * 32, smc, c->stream>>>(A);
    else k_grp_count<false><<<gc, GW * 32, smc, c->stream>>>(A);
    S.L.count();
  }
  scan_exclusive(S.L, A.cnt, n_seg, off, off + n_seg, scratch);
  u64 total = 0;
  std::vector<u32> hc(n_seg);
  TRY(copy(c, &total, off + n_seg, 8));
  if (n_seg) TRY(copy(c, hc.data(), A.cnt, (size_t)n_seg * 4));
  TRY(sync_check(c, "ta_col_group (count)"));
  const u32 max_cnt = n_seg ? *std::max_element(hc.begin(), hc.end()) : 0u;
  *n_out = total;
  if (off_out) TRY(copy(c, off_out, off, ((u64)n_seg + 1) * 8));
  if (!key_out && !sum_out && !cnt_out) return sync_check(c, "ta_col_group");
  if (!key_out || !sum_out || !cnt_out)
    return fail(TA_ERR_INVALID_ARG, "ta_col_group: key_out, sum_out and cnt_out go together");
  if (out_cap < total)
    return fail(TA_ERR_CAPACITY, "ta_col_group needs %llu groups", (unsigned long long)total);
  if (max_cnt > GSR) {  // some segment's groups overflow the shared-memory stage
    const u64 gn = warps * n_keys;
    TRY(S.tmp.get_n(gn, &A.gst_key, "group stage"));
    TRY(S.tmp.get_n(gn, &A.gst_sum, "group stage"));
    TRY(S.tmp.get_n(gn, &A.gst_cnt, "group stage"));
  }
  A.off = off;
  A.out_key = key_out;
  A.out_sum = sum_out;
  A.out_cnt = cnt_out;
  if (n_seg) {
    if (bms) k_grp_write<true><<<gwr, GW * 32, smw, c->stream>>>(A);
    else k_grp_write<false><<<gwr, GW * 32, smw, c->stream>>>(A);
    S.L.count();
  }
  return sync_check(c, "ta_col_group");
}

extern "C" ta_status ta_col_gather(ta_ctx* c, const uint32_t* key, uint64_t n, const uint32_t* dim,
                                   uint32_t n_dim, uint32_t* out) {
  if (!c || (n && (!key || !dim || !out)))
    return fail(TA_ERR_INVALID_ARG, "ta_col_gather: NULL argument");
  if (n == 0) return TA_OK;
  Scope S(c);
  u32* status;
  TRY(S.tmp.get_n(1, &status, "gather status"));
  cudaMemsetAsync(status, 0, 4, c->stream);
  k_gather<<<grid_for(c, n), 256, 0, c->stream>>>(key, n, dim, n_dim, out, status);
  S.L.count();
  u32 f = 0;
  TRY(copy(c, &f, status, 4));
  TRY(sync_check(c, "ta_col_gather"));
  if (f) return fail(TA_ERR_INVALID_ARG, "ta_col_gather: a key >= n_dim");
  return TA_OK;
}

extern "C" ta_status ta_col_compare(ta_ctx* c, const uint64_t* col, uint64_t n, uint64_t v,
                                    uint8_t* mask) {
  if (!c || (n && (!col || !mask))) return fail(TA_ERR_INVALID_ARG, "ta_col_compare: NULL argument");
  if (n == 0) return TA_OK;
  Scope S(c);
  k_compare<<<grid_for(c, n), 256, 0, c->stream>>>(col, n, v, mask);
  S.L.count();
  return sync_check(c, "ta_col_compare");
}

extern "C" ta_status ta_col_add(ta_ctx* c, const uint64_t* a, const uint64_t* b, uint64_t n,
                                uint64_t* out) {
  if (!c || (n && (!a || !b || !out))) return fail(TA_ERR_INVALID_ARG, "ta_col_add: NULL argument");
  if (n == 0) return TA_OK;
  Scope S(c);
  k_add<<<grid_for(c, n), 256, 0, c->stream>>>(a, b, n, out);
  S.L.count();
  return sync_check(c, "ta_col_add");
}

extern "C" ta_status ta_col_scale(ta_ctx* c, uint64_t* a, uint64_t n, uint64_t s) {
  if (!c || (n && !a)) return fail(TA_ERR_INVALID_ARG, "ta_col_scale: NULL argument");
  if (n == 0) return TA_OK;
  Scope S(c);
  k_scale<<<grid_for(c, n), 256, 0, c->stream>>>(a, n, s);
  S.L.count();
  return sync_check(c, "ta_col_scale");
}

extern "C" ta_status ta_col_sum(ta_ctx* c, const uint64_t* a, uint64_t n, uint64_t* sum) {
  if (!c || !sum || (n && !a)) return fail(TA_ERR_INVALID_ARG, "ta_col_sum: NULL argument");
  *sum = 0;
  if (n == 0) return TA_OK;
  Scope S(c);
  unsigned long long* d;
  TRY(S.tmp.get_n(1, &d, "sum"));
  cudaMemsetAsync(d, 0, 8, c->stream);
  k_sum<<<grid_for(c, n), 256, 0, c->stream>>>(a, n, d);
  S.L.count();
  TRY(copy(c, sum, d, 8));
  return sync_check(c, "ta_col_sum");
}

extern "C" ta_status ta_col_cumsum(ta_ctx* c, const uint64_t* a, uint64_t n, uint64_t* out) {
  if (!c || (n && (!a || !out))) return fail(TA_ERR_INVALID_ARG, "ta_col_cumsum: NULL argument");
  if (n == 0) return TA_OK;
  Scope S(c);
  u64 *scratch, *total;
  TRY(S.tmp.get_n(scan_scratch_elems(n), &scratch, "cumsum scan"));
  TRY(S.tmp.get_n(1, &total, "cumsum total"));
  scan_inclusive(S.L, a, n, out, total, scratch);
  return sync_check(c, "ta_col_cumsum");
}
