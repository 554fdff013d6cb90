// ta_dev.cuh -- device helpers of the trace-analysis kernels (sm_103a).
#pragma once
#include <cstdint>

namespace ta {

typedef uint32_t u32;
typedef uint64_t u64;
typedef unsigned __int128 u128;

constexpr u32 NONE32 = 0xFFFFFFFFu;
constexpr u32 FULL = 0xFFFFFFFFu;

// Device status bits (one u32 word per call, OR-ed by any thread).
enum : u32 {
  F_INVALID = 1u,
  F_BAD_CCT = 2u,
  F_BAD_CTX = 4u,
  F_NOT_SORTED = 8u,
  F_TIMEOUT = 16u,
  F_CAPACITY = 32u,
  F_INTERNAL = 64u
};


__device__ __forceinline__ void flag(u32* status, u32 bits) { atomicOr(status, bits); }

__device__ __forceinline__ u32 vld(const u32* p) { return *(const volatile u32*)p; }
__device__ __forceinline__ u64 vld(const u64* p) { return *(const volatile u64*)p; }

// ---- bulk copies (TMA, non-tensor form) into shared memory, completed on an
// mbarrier.  Addresses and sizes of cp.async.bulk must be multiples of 16 B.
__device__ __forceinline__ u32 smem_u32(const void* p) {
  return (u32)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// Makes initialised mbarriers visible to the async proxy (the bulk copies).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic accesses of shared memory before
// later async-proxy writes to it (a stage read, then refilled).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Copies bytes (a multiple of 16, both addresses 16-byte aligned) from global
// src to shared dst; completion is counted on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity) {
  u32 done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for phase `parity` of bar to complete, at most MBAR_SPIN polls (each
// poll may suspend the thread briefly; about a second in all); returns false
// if it gave up.
constexpr u32 MBAR_SPIN = 1u << 20;
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity) {
  for (u32 i = 0; i < MBAR_SPIN; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ u32 ld_acquire(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(u32* p, u32 v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ u64 ld_relaxed(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------------ scans --
__device__ __forceinline__ u32 warp_incl_scan(u32 x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__device__ __forceinline__ u64 warp_incl_scan(u64 x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one u64 per thread.  scratch: >= NT/32 u64 of
// shared memory.  Contains __syncthreads(); every thread must call it.
template <int NT>
__device__ __forceinline__ u64 block_excl_scan(u64 v, u64* scratch, u64* total) {
  constexpr int W = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 x = warp_incl_scan(v, lane);
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    u64 y = lane < W ? scratch[lane] : 0;
    y = warp_incl_scan(y, lane);
    if (lane < W) scratch[lane] = y;
  }
  __syncthreads();
  u64 base = warp > 0 ? scratch[warp - 1] : 0;
  if (total) *total = scratch[W - 1];
  __syncthreads();
  return base + x - v;
}

// --------------------------------------------------- two-level bitmap -----
// Sorted distinct aggregation over calling-context ids without sorting:
// set one bit per present context (L1 word w = c / 32, plus a summary bit per
// non-empty L1 word in L2), then a prefix count over the non-empty words
// gives every present context its rank among the present contexts, which is
// its position in the context-ascending output.  Cost per use is
// O(samples + present contexts + C/1024), independent of C otherwise.
struct Bm {
  u32* L1;   // [W1]
  u32* pre;  // [W1] prefix count of set bits before each non-empty word
  u32* L2;   // [W2]
  u32 W1, W2;
};

__host__ __device__ inline u32 bm_w1(u32 C) { return (C + 31) / 32; }
__host__ __device__ inline u32 bm_w2(u32 C) { return (bm_w1(C) + 31) / 32; }
// Words per bitmap, rounded to keep 16-byte alignment.
__host__ __device__ inline u32 bm_words(u32 C) { return ((2 * bm_w1(C) + bm_w2(C)) + 3) & ~3u; }

__device__ __forceinline__ Bm bm_at(u32* base, u32 C) {
  Bm b;
  b.W1 = bm_w1(C);
  b.W2 = bm_w2(C);
  b.L1 = base;
  b.pre = base + b.W1;
  b.L2 = base + 2 * b.W1;
  return b;
}

__device__ __forceinline__ void bm_set(const Bm& b, u32 c) {
  const u32 w = c >> 5, bit = 1u << (c & 31);
  const u32 old = atomicOr(&b.L1[w], bit);
  if (old == 0) atomicOr(&b.L2[w >> 5], 1u << (w & 31));
}

// Sets c; returns 1 if this call set a new bit (first occurrence).
__device__ __forceinline__ u32 bm_set_new(const Bm& b, u32 c) {
  const u32 w = c >> 5, bit = 1u << (c & 31);
  const u32 old = atomicOr(&b.L1[w], bit);
  if (old == 0) atomicOr(&b.L2[w >> 5], 1u << (w & 31));
  return (old & bit) ? 0u : 1u;
}

// Sets c; returns true if c was already set.
__device__ __forceinline__ bool bm_test_set(const Bm& b, u32 c) {
  const u32 w = c >> 5, bit = 1u << (c & 31);
  const u32 old = atomicOr(&b.L1[w], bit);
  if (old == 0) atomicOr(&b.L2[w >> 5], 1u << (w & 31));
  return (old & bit) != 0;
}

__device__ __forceinline__ bool bm_has(const Bm& b, u32 c) {
  return (vld(&b.L1[c >> 5]) >> (c & 31)) & 1u;
}

// One warp: fills pre[] for every non-empty L1 word; returns the number of
// set bits.  All set operations must be visible (syncwarp / syncthreads).
__device__ __forceinline__ u32 bm_prefix_warp(const Bm& b, int lane) {
  u32 base = 0;
  for (u32 g = 0; g < b.W2; g += 32) {
    const u32 w2 = g + lane;
    const u32 bits = (w2 < b.W2) ? vld(&b.L2[w2]) : 0u;
    u32 sum = 0;
    for (u32 x = bits; x; x &= x - 1) sum += __popc(vld(&b.L1[w2 * 32 + __ffs(x) - 1]));
    const u32 incl = warp_incl_scan(sum, lane);
    u32 run = base + incl - sum;
    for (u32 x = bits; x; x &= x - 1) {
      const u32 w1 = w2 * 32 + __ffs(x) - 1;
      b.pre[w1] = run;
      run += __popc(vld(&b.L1[w1]));
    }
    base += __shfl_sync(FULL, incl, 31);
  }
  __syncwarp();
  return base;
}

// Position of (present) context c among the present contexts.
__device__ __forceinline__ u32 bm_rank(const Bm& b, u32 c) {
  const u32 w = c >> 5;
  return vld(&b.pre[w]) + __popc(vld(&b.L1[w]) & ((1u << (c & 31)) - 1u));
}

// One warp: writes the context id of every set bit at its rank.
__device__ __forceinline__ void bm_enumerate_warp(const Bm& b, u32* out_ctx, int lane) {
  for (u32 g = 0; g < b.W2; g += 32) {
    const u32 w2 = g + lane;
    const u32 bits = (w2 < b.W2) ? vld(&b.L2[w2]) : 0u;
    for (u32 x = bits; x; x &= x - 1) {
      const u32 w1 = w2 * 32 + __ffs(x) - 1;
      u32 p = vld(&b.pre[w1]);
      for (u32 y = vld(&b.L1[w1]); y; y &= y - 1) out_ctx[p++] = w1 * 32 + __ffs(y) - 1;
    }
  }
}

// One warp: the number of set bits.
__device__ __forceinline__ u32 bm_count_warp(const Bm& b, int lane) {
  u32 sum = 0;
  for (u32 g = 0; g < b.W2; g += 32) {
    const u32 w2 = g + lane;
    const u32 bits = (w2 < b.W2) ? vld(&b.L2[w2]) : 0u;
    for (u32 x = bits; x; x &= x - 1) sum += __popc(vld(&b.L1[w2 * 32 + __ffs(x) - 1]));
  }
  return __reduce_add_sync(FULL, sum);
}

// One warp: zeroes every set word (cost proportional to what was set).
__device__ __forceinline__ void bm_clear_warp(const Bm& b, int lane) {
  for (u32 g = 0; g < b.W2; g += 32) {
    const u32 w2 = g + lane;
    if (w2 < b.W2) {
      const u32 bits = vld(&b.L2[w2]);
      for (u32 x = bits; x; x &= x - 1) b.L1[w2 * 32 + __ffs(x) - 1] = 0;
      b.L2[w2] = 0;
    }
  }
}

// ----------------------------------------------------- time searches ------
// First i in [lo, hi) with v[i] >= t, or hi.  One warp; each step probes 32
// evenly spaced positions and keeps the gap between the last probe below t
// and the first at or above it (v is non-decreasing).
__device__ __forceinline__ u64 warp_lower_bound(const u64* __restrict__ v, u64 lo, u64 hi, u64 t,
                                                int lane) {
  while (hi - lo > 32) {
    const u64 n = hi - lo;
    const u64 s = (n + 31) / 32;
    const u64 q = lo + min((u64)(lane + 1) * s, n) - 1;
    const u32 ge = __ballot_sync(FULL, v[q] >= t);
    if (ge == 0) return hi;
    const u64 k = (u64)(__ffs(ge) - 1);
    const u64 qk = lo + min((k + 1) * s, n) - 1;
    lo = k ? lo + min(k * s, n) : lo;
    hi = qk + 1;
  }
  const u64 i = lo + lane;
  const u32 ge = __ballot_sync(FULL, i < hi && v[i] >= t);
  return ge ? lo + (u64)(__ffs(ge) - 1) : hi;
}

// Time inside [t0, t1) of the sample in progress at t0 (sample b - 1, b > rb).
__device__ __forceinline__ u64 head_time(const u64* __restrict__ ts, u64 b, u64 re, u64 t0,
                                         u64 t1) {
  const u64 nx = b < re ? ts[b] : ts[b - 1];
  const u64 hi = min(nx, t1);
  return hi > t0 ? hi - t0 : 0ull;
}

// ------------------------------------------- exact integer -> double ------
// Correctly rounded (nearest, ties to even).  64-bit values use the CUDA
// conversion; wider values are first narrowed to 64 bits keeping a sticky
// bit below the rounding position, which preserves round-to-nearest-even.
__device__ __forceinline__ double u64_to_f64(u64 v) { return __ull2double_rn(v); }
__device__ __forceinline__ double i64_to_f64(long long v) { return __ll2double_rn(v); }
__device__ __forceinline__ double u128_to_f64(u128 v) {
  const u64 hi = (u64)(v >> 64);
  if (hi == 0) return __ull2double_rn((u64)v);
  const int s = 64 - __clzll(hi);  // bits to drop so the value fits in 64
  const u64 top = (u64)(v >> s);
  const u64 dropped = (u64)v & ((1ull << s) - 1ull);
  const double d = __ull2double_rn(top | (dropped ? 1ull : 0ull));
  return scalbn(d, s);
}

// Coefficient of variation (sample standard deviation over the mean) of m
// values from their sum s and exact sum of squares q.  The definition's
// mean = s / m and sd = sqrt((m q - s^2) / (m (m - 1))) give
// sd / mean = c_m sqrt(m q - s^2) / s with c_m = sqrt(m / (m - 1)), taken
// once per launch: one square root and one division per value instead of
// three divisions and a square root (a few units in the last place from the
// definition's rounding).  0 when the mean is 0 or m < 2.
__device__ __forceinline__ double cv_coef(u32 m) {
  return m < 2 ? 0.0 : sqrt(u64_to_f64(m) / u64_to_f64(m - 1));
}
__device__ __forceinline__ double cv_of_sums(u64 s, u128 q, u32 m, double c_m) {
  if (s == 0 || m < 2) return 0.0;
  const u128 d = (u128)m * q - (u128)s * s;
  return c_m * sqrt(u128_to_f64(d)) / u64_to_f64(s);
}

// a * b exactly as 256 bits (little-endian limbs), a, b < 2^128.
struct W256 {
  u64 w[4];
};
__device__ __forceinline__ W256 mul128(u128 a, u128 b) {
  const u64 a0 = (u64)a, a1 = (u64)(a >> 64), b0 = (u64)b, b1 = (u64)(b >> 64);
  const u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0,
             p11 = (u128)a1 * b1;
  W256 r;
  r.w[0] = (u64)p00;
  u128 mid = (p00 >> 64) + (u64)p01 + (u64)p10;
  r.w[1] = (u64)mid;
  u128 up = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (u64)p11;
  r.w[2] = (u64)up;
  r.w[3] = (u64)((up >> 64) + (p11 >> 64));
  return r;
}
__device__ __forceinline__ bool gt256(const W256& x, const W256& y) {
#pragma unroll
  for (int i = 3; i >= 0; --i)
    if (x.w[i] != y.w[i]) return x.w[i] > y.w[i];
  return false;
}

// Exact high-side outlier rule: D > 0 and D^2 (n-1) tau_den^2 > tau_num^2 n M,
// with D = n x - S1 (|D| < 2^63), M = n S2 - S1^2 (< 2^126), n < 2^32.
__device__ __forceinline__ bool is_outlier(long long D, u64 n, u128 M, u32 tn, u32 td) {
  if (D <= 0 || n < 2 || M == 0) return false;
  const u128 D2 = (u128)(u64)D * (u64)D;  // < 2^126
  const u128 lhs_f = (u128)(n - 1) * ((u64)td * td);  // < 2^96
  const u128 rhs_f = (u128)n * ((u64)tn * tn);        // < 2^96
  return gt256(mul128(D2, lhs_f), mul128(M, rhs_f));
}

// 128-bit accumulator updated with two 64-bit atomics (exact, any order).
// Adds v to the 64-bit word at p with 32-bit atomics: the low half's old
// value tells whether it wrapped, and the high half is touched only for a
// high part or a carry (rare for durations below 2^32 ns).  Exact in any
// order; the word is read only after every add (shared or global memory).
__device__ __forceinline__ void atomic_add_u64_lo32(unsigned long long* p, u64 v) {
  u32* w = reinterpret_cast<u32*>(p);
  const u32 lo = (u32)v, hi = (u32)(v >> 32);
  const u32 old = atomicAdd(&w[0], lo);
  const u32 up = hi + ((u32)(old + lo) < old ? 1u : 0u);
  if (up) atomicAdd(&w[1], up);
}

__device__ __forceinline__ void atomic_add_u128(u64* lo, u64* hi, u128 v) {
  const u64 vlo = (u64)v, vhi = (u64)(v >> 64);
  const u64 old = atomicAdd((unsigned long long*)lo, (unsigned long long)vlo);
  const u64 carry = (old + vlo < old) ? 1ull : 0ull;
  if (vhi + carry) atomicAdd((unsigned long long*)hi, (unsigned long long)(vhi + carry));
}

}  // namespace ta
