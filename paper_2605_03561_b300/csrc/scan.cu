// scan.cu -- device-wide exclusive prefix sums in three phases: per-block
// sums, one block scanning the block sums, then each block scanning its
// elements from its base.  Each thread owns SCAN_ITEMS consecutive elements.
#include <algorithm>

#include "ta_internal.h"

namespace ta {

namespace {

constexpr int SCAN_NT = 256;
constexpr int SCAN_ITEMS = 16;
constexpr u64 SCAN_TILE = (u64)SCAN_NT * SCAN_ITEMS;

__device__ __forceinline__ u64 warp_sum(u64 x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

template <class T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const T* __restrict__ in, u64 n,
                                                         u64* block_sums) {
  __shared__ u64 s[SCAN_NT / 32];
  const u64 base = (u64)blockIdx.x * SCAN_TILE + threadIdx.x;  // coalesced: order is free
  u64 sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + (u64)i * SCAN_NT < n) sum += in[base + (u64)i * SCAN_NT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  sum = warp_sum(sum);
  if (lane == 0) s[warp] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < SCAN_NT / 32; ++w) t += s[w];
    block_sums[blockIdx.x] = t;
  }
}

// One block: exclusive scan of nb block sums in place; total to *total.
__global__ void __launch_bounds__(1024) k_scan_blocks(u64* sums, u64 nb, u64* total) {
  __shared__ u64 s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 carry = 0;
  for (u64 b0 = 0; b0 < nb; b0 += 1024) {
    const u64 i = b0 + threadIdx.x;
    const u64 v = i < nb ? sums[i] : 0;
    const u64 x = warp_incl_scan(v, lane);
    if (lane == 31) s[warp] = x;
    __syncthreads();
    if (warp == 0) s[lane] = warp_incl_scan(s[lane], lane);
    __syncthreads();
    const u64 excl = carry + (warp ? s[warp - 1] : 0) + x - v;
    if (i < nb) sums[i] = excl;
    carry += s[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// The tile goes through shared memory twice so that global loads and stores
// are coalesced while each thread scans SCAN_ITEMS consecutive elements (one
// padding word per 16 keeps the per-thread runs on different banks).
__device__ __forceinline__ u32 scan_pad(u32 x) { return x + (x >> 4); }

template <class T, bool INCL = false>
__global__ void __launch_bounds__(SCAN_NT) k_scan_apply(const T* __restrict__ in, u64 n,
                                                        const u64* block_base, u64* out) {
  __shared__ u64 s[SCAN_NT / 32];
  __shared__ u64 t[SCAN_TILE + SCAN_TILE / 16];
  const u64 tile = (u64)blockIdx.x * SCAN_TILE;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const u32 j = (u32)i * SCAN_NT + threadIdx.x;
    t[scan_pad(j)] = (tile + j < n) ? (u64)in[tile + j] : 0ull;
  }
  __syncthreads();
  u64 v[SCAN_ITEMS];
  u64 sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = t[scan_pad(threadIdx.x * SCAN_ITEMS + i)];
    sum += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 x = warp_incl_scan(sum, lane);
  if (lane == 31) s[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const u64 y = lane < SCAN_NT / 32 ? s[lane] : 0;
    const u64 z = warp_incl_scan(y, lane);
    if (lane < SCAN_NT / 32) s[lane] = z;
  }
  __syncthreads();
  u64 run = block_base[blockIdx.x] + (warp ? s[warp - 1] : 0) + x - sum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    t[scan_pad(threadIdx.x * SCAN_ITEMS + i)] = INCL ? run + v[i] : run;
    run += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const u32 j = (u32)i * SCAN_NT + threadIdx.x;
    if (tile + j < n) out[tile + j] = t[scan_pad(j)];
  }
}

template <class T, bool INCL = false>
void scan_impl(const Launch& L, const T* in, u64 n, u64* out, u64* total, u64* scratch) {
  const u64 nb = std::max<u64>(1, (n + SCAN_TILE - 1) / SCAN_TILE);
  k_scan_reduce<T><<<(unsigned)nb, SCAN_NT, 0, L.stream>>>(in, n, scratch);
  k_scan_blocks<<<1, 1024, 0, L.stream>>>(scratch, nb, total);
  k_scan_apply<T, INCL><<<(unsigned)nb, SCAN_NT, 0, L.stream>>>(in, n, scratch, out);
  L.count(3);
}

}  // namespace

u64 scan_scratch_elems(u64 n) { return std::max<u64>(1, (n + SCAN_TILE - 1) / SCAN_TILE); }

void scan_exclusive(const Launch& L, const u32* in, u64 n, u64* out, u64* total, u64* scratch) {
  scan_impl<u32>(L, in, n, out, total, scratch);
}
void scan_exclusive(const Launch& L, const u64* in, u64 n, u64* out, u64* total, u64* scratch) {
  scan_impl<u64>(L, in, n, out, total, scratch);
}
void scan_inclusive(const Launch& L, const u64* in, u64 n, u64* out, u64* total, u64* scratch) {
  scan_impl<u64, true>(L, in, n, out, total, scratch);
}

}  // namespace ta
