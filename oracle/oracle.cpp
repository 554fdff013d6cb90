// oracle.cpp -- the plain CPU definition of the trace-analysis path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
// this file; only the tests, the smoke check and the benchmark's CPU-baseline
// leg do.  It is deliberately slow and obvious: one thread, rank by rank,
// std::map per iteration row, a literal ancestor walk for inclusive time, and
// the statistics written out from their definitions.  It shares no code,
// header or table with the CUDA path.
//
// What it computes, and where the paper defines it:
//  * A trace sample (t_i, c_i) means the rank was in calling context c_i from
//    t_i until the next sample (execution traces as timed CCT node events,
//    Section II-A); the last sample of a rank lasts 0 ns but still counts.
//  * Iterations (Section V, iteration-aware workflow; Section VI-A): a new
//    iteration starts at the first sample of every run of marker samples;
//    samples before the first marker form a prologue row.  Each iteration row
//    is a re-materialised profile: exclusive time and sample count per context.
//  * Exclusive time per (rank, context) (profiles collapse the time dimension,
//    Section V) and inclusive time rolled up the calling context tree
//    (inclusive/exclusive costs, Sections II-A and VI-B).
//  * Cross-rank statistics per context (the group-by of Section VI-A:
//    mean/min/max/std with ddof = 1), global balance ratio = mean / max
//    (Section VI-A, Table IV), coefficient of variation, z-scores and a
//    high-side outlier rule standing in for the paper's clustering
//    (Section VI-B).
//  * Node / chassis / rack rollup of outlier ranks (Section VI-B, the
//    rank -> node join and the Slingshot rack mapping).
//  * Potential savings per kernel = average over iterations of (max over
//    ranks) minus (mean over ranks); total = savings x iterations; speedup
//    fraction = total savings / application time (Section VI-A, Table V).
//
// Readings taken where the paper is silent (absent ranks count as 0, ddof 1,
// tau as a rational, ties -> lowest rank, the application-time default) are
// listed with the design notes of this repository.
//
// Parity pins: every function here is checked by tests against hand-worked
// examples, Table V's printed arithmetic, closed forms, brute force and
// invariants.  The per-group CV definitions (cv_across, cv_within) have no
// printed value to reproduce: parity unpinned against the paper's numbers
// (their arithmetic is pinned by closed-form cases only).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

namespace {

typedef unsigned __int128 u128;
typedef __int128 i128;

const uint32_t NONE = 0xFFFFFFFFu;

enum {
  OR_OK = 0,
  OR_INVALID = 1,
  OR_NOT_SORTED = 2,
  OR_BAD_CTX = 3,
  OR_BAD_CCT = 4
};

// ---- correctly rounded integer -> double (round to nearest, ties to even) --
// Written from the IEEE-754 definition: keep the 53 leading bits, round on the
// next bit with the OR of all lower bits as sticky.
double u128_to_double(u128 v) {
  if (v == 0) return 0.0;
  int msb = 127;
  while (((v >> msb) & 1) == 0) --msb;
  if (msb < 53) return (double)(uint64_t)v;  // exact
  int shift = msb - 52;                      // bits dropped
  u128 mant = v >> shift;                    // 53 bits
  u128 rest = v & ((((u128)1) << shift) - 1);
  u128 half = ((u128)1) << (shift - 1);
  if (rest > half || (rest == half && (mant & 1))) {
    mant += 1;
    if (mant >> 53) {  // carried into a new bit
      mant >>= 1;
      shift += 1;
    }
  }
  return std::ldexp((double)(uint64_t)mant, shift);
}

double i128_to_double(i128 v) {
  if (v < 0) return -u128_to_double((u128)(-v));
  return u128_to_double((u128)v);
}

// ---- 256-bit unsigned products for the exact outlier comparison ----------
struct U256 {
  uint64_t w[4];  // little endian
};

U256 u256_from(u128 a) {
  U256 r = {{(uint64_t)a, (uint64_t)(a >> 64), 0, 0}};
  return r;
}

U256 u256_mul64(const U256& a, uint64_t b) {
  U256 r = {{0, 0, 0, 0}};
  u128 carry = 0;
  for (int i = 0; i < 4; ++i) {
    u128 p = (u128)a.w[i] * b + carry;
    r.w[i] = (uint64_t)p;
    carry = p >> 64;
  }
  return r;  // callers keep products below 2^256
}

U256 u256_mul128(const U256& a, u128 b) {
  // a * (lo + hi * 2^64)
  U256 lo = u256_mul64(a, (uint64_t)b);
  U256 hi = u256_mul64(a, (uint64_t)(b >> 64));
  U256 r;
  u128 carry = 0;
  for (int i = 0; i < 4; ++i) {
    u128 s = (u128)lo.w[i] + (i > 0 ? hi.w[i - 1] : 0) + carry;
    r.w[i] = (uint64_t)s;
    carry = s >> 64;
  }
  return r;
}

bool u256_greater(const U256& a, const U256& b) {
  for (int i = 3; i >= 0; --i) {
    if (a.w[i] != b.w[i]) return a.w[i] > b.w[i];
  }
  return false;
}

struct Entry {
  uint32_t ctx;
  uint64_t time;
  uint64_t cnt;
};

struct RankResult {
  std::vector<std::vector<Entry>> rows;  // rows[0] = prologue, rows[1 + it]
  std::vector<Entry> excl, incl;
  uint32_t n_iter = 0;
  uint64_t span = 0;
};

struct Input {
  uint32_t R, C, marker;
  uint64_t N;
  const uint64_t* rank_off;
  const uint64_t* ts;
  const uint32_t* ctx;
  const uint32_t* parent;
};

struct Handle {
  Input in;
  uint32_t r0, r1;
  std::vector<RankResult> ranks;  // ranks[r - r0]
};

// ---- O0: input validation --------------------------------------------------
int validate(const Input& in) {
  if (in.R == 0 || in.C == 0 || !in.rank_off || !in.parent) return OR_INVALID;
  if (in.N > 0 && (!in.ts || !in.ctx)) return OR_INVALID;
  if (in.marker >= in.C) return OR_INVALID;
  if (in.rank_off[0] != 0 || in.rank_off[in.R] != in.N) return OR_INVALID;
  for (uint32_t r = 0; r < in.R; ++r) {
    if (in.rank_off[r + 1] < in.rank_off[r]) return OR_INVALID;
    if (in.rank_off[r + 1] - in.rank_off[r] > 0xFFFFFFFFull) return OR_INVALID;
  }
  // Calling context tree: one root, every other parent in range, and every
  // node reaches the root by walking parents in fewer than C steps.
  uint32_t roots = 0;
  for (uint32_t v = 0; v < in.C; ++v) {
    if (in.parent[v] == NONE) ++roots;
    else if (in.parent[v] >= in.C) return OR_BAD_CCT;
  }
  if (roots != 1) return OR_BAD_CCT;
  for (uint32_t v = 0; v < in.C; ++v) {
    uint32_t a = v;
    uint64_t steps = 0;
    while (in.parent[a] != NONE) {
      a = in.parent[a];
      if (++steps >= in.C) return OR_BAD_CCT;
    }
  }
  for (uint64_t i = 0; i < in.N; ++i)
    if (in.ctx[i] >= in.C) return OR_BAD_CTX;
  uint64_t max_span = 0;
  for (uint32_t r = 0; r < in.R; ++r) {
    uint64_t b = in.rank_off[r], e = in.rank_off[r + 1];
    for (uint64_t i = b; i + 1 < e; ++i)
      if (in.ts[i + 1] < in.ts[i]) return OR_NOT_SORTED;
    if (e > b && in.ts[e - 1] - in.ts[b] > max_span) max_span = in.ts[e - 1] - in.ts[b];
  }
  // Exactness contract of the 128-bit moments: R * (longest span) < 2^63.
  if ((u128)max_span * in.R >= ((u128)1 << 63)) return OR_INVALID;
  return OR_OK;
}

// ---- O1: durations, iteration cut, per-row and per-rank exclusive ---------
// ---- O2: inclusive by walking every present context up to the root ------
void analyze_rank(const Input& in, uint32_t r, RankResult& out, bool want_rows,
                  bool want_incl) {
  const uint64_t b = in.rank_off[r], e = in.rank_off[r + 1];
  std::vector<std::map<uint32_t, std::pair<uint64_t, uint64_t>>> rows(1);
  std::map<uint32_t, std::pair<uint64_t, uint64_t>> X;
  int64_t it = -1;
  for (uint64_t i = b; i < e; ++i) {
    const uint64_t d = (i + 1 < e) ? in.ts[i + 1] - in.ts[i] : 0;
    const bool starts = (in.ctx[i] == in.marker) && (i == b || in.ctx[i - 1] != in.marker);
    if (starts) {
      ++it;
      if (want_rows) rows.emplace_back();
    }
    if (want_rows) {
      auto& cell = rows[(size_t)(it + 1)][in.ctx[i]];
      cell.first += d;
      cell.second += 1;
    }
    auto& x = X[in.ctx[i]];
    x.first += d;
    x.second += 1;
  }
  out.n_iter = (uint32_t)(it + 1);
  out.span = (e > b) ? in.ts[e - 1] - in.ts[b] : 0;
  if (want_rows) {
    out.rows.resize(rows.size());
    for (size_t k = 0; k < rows.size(); ++k)
      for (auto& kv : rows[k]) out.rows[k].push_back({kv.first, kv.second.first, kv.second.second});
  }
  for (auto& kv : X) out.excl.push_back({kv.first, kv.second.first, kv.second.second});
  if (want_incl) {
    std::map<uint32_t, std::pair<uint64_t, uint64_t>> INC;
    for (auto& kv : X) {
      uint32_t a = kv.first;
      while (a != NONE) {
        auto& y = INC[a];
        y.first += kv.second.first;
        y.second += kv.second.second;
        a = in.parent[a];
      }
    }
    for (auto& kv : INC) out.incl.push_back({kv.first, kv.second.first, kv.second.second});
  }
}

const std::vector<Entry>& metric_of(const RankResult& rr, int metric) {
  return metric == 1 ? rr.incl : rr.excl;
}

// Value and count of context c in a ctx-ascending list (0, 0 if absent).
void lookup(const std::vector<Entry>& v, uint32_t c, uint64_t& x, uint64_t& cnt) {
  size_t lo = 0, hi = v.size();
  while (lo < hi) {
    size_t mid = (lo + hi) / 2;
    if (v[mid].ctx < c) lo = mid + 1;
    else hi = mid;
  }
  if (lo < v.size() && v[lo].ctx == c) {
    x = v[lo].time;
    cnt = v[lo].cnt;
  } else {
    x = 0;
    cnt = 0;
  }
}

uint64_t row_time(const RankResult& rr, size_t row, uint32_t c) {
  if (row >= rr.rows.size()) return 0;
  uint64_t x, cnt;
  lookup(rr.rows[row], c, x, cnt);
  return x;
}

// Sum of v in a fixed pairwise order: level by level, element i of the next
// level is v[2i] + v[2i+1]; an odd last element moves up unchanged.  (The
// order is part of the definition: with it the result does not depend on how
// the work is split.)
double pairwise_sum(std::vector<double> v) {
  size_t n = v.size();
  if (n == 0) return 0.0;
  while (n > 1) {
    const size_t m = n / 2;
    for (size_t i = 0; i < m; ++i) v[i] = v[2 * i] + v[2 * i + 1];
    if (n & 1) {
      v[m] = v[n - 1];
      n = m + 1;
    } else {
      n = m;
    }
  }
  return v[0];
}

bool check_subset(const uint32_t* s, uint32_t n, uint32_t limit) {
  for (uint32_t i = 0; i < n; ++i) {
    if (s[i] >= limit) return false;
    if (i > 0 && s[i] <= s[i - 1]) return false;
  }
  return true;
}

}  // namespace

extern "C" {

typedef struct or_input {
  uint32_t n_ranks, n_ctx, marker_ctx, pad;
  uint64_t n_records;
  const uint64_t* rank_off;
  const uint64_t* ts;
  const uint32_t* ctx;
  const uint32_t* parent;
} or_input;

static Input to_input(const or_input* p) {
  Input in;
  in.R = p->n_ranks;
  in.C = p->n_ctx;
  in.marker = p->marker_ctx;
  in.N = p->n_records;
  in.rank_off = p->rank_off;
  in.ts = p->ts;
  in.ctx = p->ctx;
  in.parent = p->parent;
  return in;
}

int or_validate(const or_input* p) {
  if (!p) return OR_INVALID;
  return validate(to_input(p));
}

// u128 -> double and the 256-bit comparison, exported for the pin tests.
double or_u128_to_double(uint64_t lo, uint64_t hi) {
  return u128_to_double(((u128)hi << 64) | lo);
}

// want: bit 0 = iteration rows, bit 1 = inclusive (exclusive is always kept).
// Ranks [r0, r1) are analysed; inputs are read, not copied, and must outlive
// the handle.  validate == 0 skips O0 (the caller validated already).
void* or_analyze(const or_input* p, uint32_t r0, uint32_t r1, int want, int do_validate,
                 int* status) {
  Input in = to_input(p);
  if (do_validate) {
    int s = validate(in);
    if (status) *status = s;
    if (s != OR_OK) return nullptr;
  }
  if (r1 > in.R || r0 > r1) {
    if (status) *status = OR_INVALID;
    return nullptr;
  }
  Handle* h = new Handle();
  h->in = in;
  h->r0 = r0;
  h->r1 = r1;
  h->ranks.resize(r1 - r0);
  for (uint32_t r = r0; r < r1; ++r) analyze_rank(in, r, h->ranks[r - r0], want & 1, want & 2);
  if (status) *status = OR_OK;
  return h;
}

void or_free(void* hp) { delete (Handle*)hp; }

// Sizes of the iteration tensor of the handle's ranks.
void or_tensor_sizes(void* hp, uint64_t* rows, uint64_t* nnz) {
  Handle* h = (Handle*)hp;
  uint64_t nr = 0, ne = 0;
  for (auto& rr : h->ranks) {
    nr += rr.rows.size();
    for (auto& row : rr.rows) ne += row.size();
  }
  *rows = nr;
  *nnz = ne;
}

// CSR of the tensor, offsets relative to the handle's first rank.
void or_tensor_get(void* hp, uint64_t* row_off_of_rank, uint64_t* entry_off, uint32_t* e_ctx,
                   uint64_t* e_time, uint32_t* e_cnt, uint32_t* n_iter) {
  Handle* h = (Handle*)hp;
  uint64_t row = 0, ent = 0;
  for (size_t k = 0; k < h->ranks.size(); ++k) {
    auto& rr = h->ranks[k];
    row_off_of_rank[k] = row;
    n_iter[k] = rr.n_iter;
    for (auto& rw : rr.rows) {
      entry_off[row++] = ent;
      for (auto& en : rw) {
        e_ctx[ent] = en.ctx;
        e_time[ent] = en.time;
        e_cnt[ent] = (uint32_t)en.cnt;
        ++ent;
      }
    }
  }
  row_off_of_rank[h->ranks.size()] = row;
  entry_off[row] = ent;
}

uint64_t or_csr_nnz(void* hp, int which) {
  Handle* h = (Handle*)hp;
  uint64_t n = 0;
  for (auto& rr : h->ranks) n += metric_of(rr, which).size();
  return n;
}

void or_csr_get(void* hp, int which, uint64_t* off, uint32_t* ctx, uint64_t* time,
                uint32_t* cnt) {
  Handle* h = (Handle*)hp;
  uint64_t e = 0;
  for (size_t k = 0; k < h->ranks.size(); ++k) {
    off[k] = e;
    for (auto& en : metric_of(h->ranks[k], which)) {
      ctx[e] = en.ctx;
      time[e] = en.time;
      cnt[e] = (uint32_t)en.cnt;
      ++e;
    }
  }
  off[h->ranks.size()] = e;
}

void or_span_get(void* hp, uint64_t* span) {
  Handle* h = (Handle*)hp;
  for (size_t k = 0; k < h->ranks.size(); ++k) span[k] = h->ranks[k].span;
}

typedef struct or_ctx_stats {
  uint32_t n, present, argmax, pad;
  uint64_t min, max, s1, s2_lo, s2_hi;
  double mean, std, cv, balance;
} or_ctx_stats;

typedef struct or_outlier {
  uint32_t ctx, rank;
  double z;
} or_outlier;

// O3.  Ranks S (sorted, unique; NULL = all ranks of the handle) must lie in
// the handle.  Contexts (sorted, unique; NULL = all C).  stats[i] describes
// ctxs[i].  Outliers are written sorted by (ctx, rank); *n_out is the full
// count even if it exceeds cap.  z (optional) receives, for the handle's CSR
// of the metric, the z-score of each entry whose rank is in S and whose ctx
// is requested, and 0 elsewhere.
int or_stats(void* hp, int metric, const uint32_t* ranks, uint32_t n_ranks,
             const uint32_t* ctxs, uint32_t n_ctxs, uint32_t tau_num, uint32_t tau_den,
             or_ctx_stats* stats, or_outlier* out, uint64_t cap, uint64_t* n_out, double* z) {
  Handle* h = (Handle*)hp;
  const Input& in = h->in;
  if (tau_den == 0) return OR_INVALID;
  std::vector<uint32_t> S, K;
  if (ranks) {
    if (!check_subset(ranks, n_ranks, in.R) || n_ranks == 0) return OR_INVALID;
    S.assign(ranks, ranks + n_ranks);
  } else {
    for (uint32_t r = h->r0; r < h->r1; ++r) S.push_back(r);
  }
  for (uint32_t r : S)
    if (r < h->r0 || r >= h->r1) return OR_INVALID;
  if (S.empty()) return OR_INVALID;
  if (ctxs) {
    if (!check_subset(ctxs, n_ctxs, in.C)) return OR_INVALID;
    K.assign(ctxs, ctxs + n_ctxs);
  } else {
    for (uint32_t c = 0; c < in.C; ++c) K.push_back(c);
  }
  // z output is laid out like the handle's CSR of the metric.
  std::vector<uint64_t> zoff(h->ranks.size() + 1, 0);
  for (size_t k = 0; k < h->ranks.size(); ++k)
    zoff[k + 1] = zoff[k] + metric_of(h->ranks[k], metric).size();
  if (z)
    for (uint64_t i = 0; i < zoff.back(); ++i) z[i] = 0.0;
  const uint64_t n = S.size();
  uint64_t count = 0;
  for (size_t ki = 0; ki < K.size(); ++ki) {
    const uint32_t c = K[ki];
    uint64_t present = 0, minp = UINT64_MAX, mx = 0, S1 = 0;
    uint32_t argmax = S[0];
    u128 S2 = 0;
    for (uint32_t r : S) {
      uint64_t x, cnt;
      lookup(metric_of(h->ranks[r - h->r0], metric), c, x, cnt);
      if (cnt > 0) {
        ++present;
        if (x < minp) minp = x;
      }
      if (x > mx) {
        mx = x;
        argmax = r;
      }
      S1 += x;
      S2 += (u128)x * x;
    }
    const u128 M = (u128)n * S2 - (u128)S1 * S1;
    or_ctx_stats& st = stats[ki];
    st.n = (uint32_t)n;
    st.present = (uint32_t)present;
    st.argmax = argmax;
    st.pad = 0;
    st.min = (present < n) ? 0 : minp;
    st.max = mx;
    st.s1 = S1;
    st.s2_lo = (uint64_t)S2;
    st.s2_hi = (uint64_t)(S2 >> 64);
    st.mean = u128_to_double(S1) / u128_to_double(n);
    st.std = (n < 2) ? 0.0 : std::sqrt(u128_to_double(M) / u128_to_double((u128)n * (n - 1)));
    st.cv = (st.mean == 0.0) ? 0.0 : st.std / st.mean;
    st.balance = (mx == 0) ? 1.0 : st.mean / u128_to_double(mx);
    // z-scores and the exact high-side outlier test for present ranks.
    for (uint32_t r : S) {
      const RankResult& rr = h->ranks[r - h->r0];
      const std::vector<Entry>& v = metric_of(rr, metric);
      uint64_t x, cnt;
      lookup(v, c, x, cnt);
      if (cnt == 0) continue;
      const i128 D = (i128)((u128)n * x) - (i128)S1;
      double zr = (n < 2 || M == 0) ? 0.0 : i128_to_double(D) / (u128_to_double(n) * st.std);
      if (z) {
        for (uint64_t e = 0; e < v.size(); ++e)
          if (v[e].ctx == c) z[zoff[r - h->r0] + e] = zr;
      }
      if (D > 0 && M > 0 && n >= 2) {
        // D^2 (n-1) tau_den^2  >  tau_num^2 n M
        U256 lhs = u256_mul64(u256_mul64(u256_from((u128)D * (u128)D), n - 1),
                              (uint64_t)tau_den * tau_den);
        U256 rhs = u256_mul128(u256_mul64(u256_from(M), n), (u128)tau_num * tau_num);
        if (u256_greater(lhs, rhs)) {
          if (count < cap && out) out[count] = {c, r, zr};
          ++count;
        }
      }
    }
  }
  if (n_out) *n_out = count;
  return OR_OK;
}

typedef struct or_topo_out {
  uint32_t n_flagged_racks, pad;
} or_topo_out;

// O4.  One context, its outlier ranks over S, then nodes, chassis and racks.
int or_topology(void* hp, int metric, uint32_t c, uint32_t tau_num, uint32_t tau_den,
                uint32_t min_ranks, const uint32_t* ranks, uint32_t n_ranks,
                const uint32_t* node_of_rank, uint32_t n_nodes, const uint32_t* rack_of_node,
                uint32_t n_racks, const uint32_t* chassis_of_node, uint32_t n_chassis,
                uint32_t* node_outliers, uint64_t* node_sum, uint32_t* node_ranks,
                uint8_t* node_flag, uint32_t* chassis_flagged, uint32_t* chassis_nodes,
                uint64_t* chassis_sum, uint32_t* rack_flagged, uint32_t* rack_nodes,
                uint64_t* rack_sum, uint32_t* flagged_racks, uint32_t* n_flagged_racks) {
  Handle* h = (Handle*)hp;
  const Input& in = h->in;
  if (c >= in.C || min_ranks == 0) return OR_INVALID;
  for (uint32_t nd = 0; nd < n_nodes; ++nd)
    if (rack_of_node[nd] >= n_racks || chassis_of_node[nd] >= n_chassis) return OR_INVALID;
  for (uint32_t r = 0; r < in.R; ++r)
    if (node_of_rank[r] >= n_nodes) return OR_INVALID;
  std::vector<uint32_t> S;
  if (ranks) {
    if (!check_subset(ranks, n_ranks, in.R) || n_ranks == 0) return OR_INVALID;
    S.assign(ranks, ranks + n_ranks);
  } else {
    for (uint32_t r = h->r0; r < h->r1; ++r) S.push_back(r);
  }
  or_ctx_stats st;
  std::vector<or_outlier> outl(S.size() + 1);
  uint64_t n_out = 0;
  int s = or_stats(hp, metric, S.data(), (uint32_t)S.size(), &c, 1, tau_num, tau_den, &st,
                   outl.data(), outl.size(), &n_out, nullptr);
  if (s != OR_OK) return s;
  std::vector<uint8_t> is_out(in.R, 0);
  for (uint64_t i = 0; i < n_out; ++i) is_out[outl[i].rank] = 1;
  for (uint32_t nd = 0; nd < n_nodes; ++nd) {
    node_outliers[nd] = 0;
    node_sum[nd] = 0;
    node_ranks[nd] = 0;
  }
  for (uint32_t r : S) {
    uint64_t x, cnt;
    lookup(metric_of(h->ranks[r - h->r0], metric), c, x, cnt);
    const uint32_t nd = node_of_rank[r];
    node_outliers[nd] += is_out[r];
    node_sum[nd] += x;
    node_ranks[nd] += 1;
  }
  for (uint32_t q = 0; q < n_chassis; ++q) {
    chassis_flagged[q] = 0;
    chassis_nodes[q] = 0;
    chassis_sum[q] = 0;
  }
  for (uint32_t q = 0; q < n_racks; ++q) {
    rack_flagged[q] = 0;
    rack_nodes[q] = 0;
    rack_sum[q] = 0;
  }
  for (uint32_t nd = 0; nd < n_nodes; ++nd) {
    node_flag[nd] = node_outliers[nd] >= min_ranks ? 1 : 0;
    chassis_flagged[chassis_of_node[nd]] += node_flag[nd];
    chassis_nodes[chassis_of_node[nd]] += 1;
    chassis_sum[chassis_of_node[nd]] += node_sum[nd];
    rack_flagged[rack_of_node[nd]] += node_flag[nd];
    rack_nodes[rack_of_node[nd]] += 1;
    rack_sum[rack_of_node[nd]] += node_sum[nd];
  }
  uint32_t nf = 0;
  for (uint32_t q = 0; q < n_racks; ++q)
    if (rack_flagged[q] > 0) flagged_racks[nf++] = q;
  *n_flagged_racks = nf;
  return OR_OK;
}

typedef struct or_speedup_ctx {
  uint64_t A, B, G_lo, G_hi;
  double avg_mean, avg_max, savings_per_iter, total_reduction, share, cv_across, cv_within;
} or_speedup_ctx;

typedef struct or_speedup_total {
  uint32_t i_star, pad;
  uint64_t excluded_iterations;
  uint64_t sum_G_lo, sum_G_hi;
  uint64_t t_app;
  double total_reduction;
  double speedup_fraction;
} or_speedup_total;

// O5.  Needs the handle's iteration rows for every rank of S.
int or_speedup(void* hp, const uint32_t* ctxs, uint32_t n_ctxs, const uint32_t* ranks,
               uint32_t n_ranks, uint64_t app_time_ns, or_speedup_ctx* per, or_speedup_total* tot) {
  Handle* h = (Handle*)hp;
  const Input& in = h->in;
  if (!ctxs || n_ctxs == 0 || !check_subset(ctxs, n_ctxs, in.C)) return OR_INVALID;
  std::vector<uint32_t> S;
  if (ranks) {
    if (!check_subset(ranks, n_ranks, in.R) || n_ranks == 0) return OR_INVALID;
    S.assign(ranks, ranks + n_ranks);
  } else {
    for (uint32_t r = h->r0; r < h->r1; ++r) S.push_back(r);
  }
  for (uint32_t r : S)
    if (r < h->r0 || r >= h->r1) return OR_INVALID;
  const uint64_t n = S.size();
  uint32_t I = UINT32_MAX;
  for (uint32_t r : S) I = std::min(I, h->ranks[r - h->r0].n_iter);
  uint64_t excluded = 0;
  for (uint32_t r : S) excluded += h->ranks[r - h->r0].n_iter - I;
  u128 sumB = 0, sumG = 0;
  for (uint32_t k = 0; k < n_ctxs; ++k) {
    const uint32_t c = ctxs[k];
    uint64_t A = 0, B = 0;
    double across = 0.0;
    for (uint32_t i = 0; i < I; ++i) {
      uint64_t sum = 0, mx = 0;
      u128 sq = 0;
      for (uint32_t r : S) {
        uint64_t t = row_time(h->ranks[r - h->r0], (size_t)i + 1, c);
        sum += t;
        if (t > mx) mx = t;
        sq += (u128)t * t;
      }
      A += mx;
      B += sum;
      double mean = u128_to_double(sum) / u128_to_double(n);
      double sd = (n < 2) ? 0.0
                          : std::sqrt(u128_to_double((u128)n * sq - (u128)sum * sum) /
                                      u128_to_double((u128)n * (n - 1)));
      across += (mean == 0.0) ? 0.0 : sd / mean;
    }
    std::vector<double> within_terms;  // per rank of S, in order
    for (uint32_t r : S) {
      uint64_t s = 0;
      u128 q = 0;
      for (uint32_t i = 0; i < I; ++i) {
        uint64_t t = row_time(h->ranks[r - h->r0], (size_t)i + 1, c);
        s += t;
        q += (u128)t * t;
      }
      if (I == 0) continue;
      double mean = u128_to_double(s) / u128_to_double(I);
      double sd = (I < 2) ? 0.0
                          : std::sqrt(u128_to_double((u128)I * q - (u128)s * s) /
                                      u128_to_double((u128)I * (I - 1)));
      within_terms.push_back((mean == 0.0) ? 0.0 : sd / mean);
    }
    const double within = pairwise_sum(within_terms);
    const u128 G = (u128)n * A - B;
    or_speedup_ctx& p = per[k];
    p.A = A;
    p.B = B;
    p.G_lo = (uint64_t)G;
    p.G_hi = (uint64_t)(G >> 64);
    if (I == 0) {
      p.avg_mean = p.avg_max = p.savings_per_iter = 0.0;
      p.cv_across = p.cv_within = 0.0;
    } else {
      p.avg_mean = u128_to_double(B) / u128_to_double((u128)n * I);
      p.avg_max = u128_to_double(A) / u128_to_double(I);
      p.savings_per_iter = u128_to_double(G) / u128_to_double((u128)n * I);
      p.cv_across = across / u128_to_double(I);
      p.cv_within = within / u128_to_double(n);
    }
    p.total_reduction = u128_to_double(G) / u128_to_double(n);
    sumB += B;
    sumG += G;
  }
  for (uint32_t k = 0; k < n_ctxs; ++k)
    per[k].share = (sumB == 0) ? 0.0 : u128_to_double(per[k].B) / u128_to_double(sumB);
  uint64_t T = app_time_ns;
  if (T == 0)
    for (uint32_t r : S) T = std::max(T, h->ranks[r - h->r0].span);
  tot->i_star = I;
  tot->pad = 0;
  tot->excluded_iterations = excluded;
  tot->sum_G_lo = (uint64_t)sumG;
  tot->sum_G_hi = (uint64_t)(sumG >> 64);
  tot->t_app = T;
  tot->total_reduction = u128_to_double(sumG) / u128_to_double(n);
  tot->speedup_fraction = (T == 0) ? 0.0 : u128_to_double(sumG) / u128_to_double((u128)n * T);
  return OR_OK;
}

// Q2, a slice of the tri-dimensional model (Section V; slicing by fixing a
// context, Section VI): out[(r - r0) * (i1 - i0) + (i - i0)] is the time of
// context c in iteration i of rank r (iteration rows only, the prologue is
// not an iteration), 0 where the context is absent or the rank has fewer
// iterations.  Ranks [r0, r1) must lie in the handle.
int or_slice(void* hp, uint32_t c, uint32_t r0, uint32_t r1, uint32_t i0, uint32_t i1,
             uint64_t* out) {
  Handle* h = (Handle*)hp;
  if (c >= h->in.C || r0 > r1 || i0 > i1 || r0 < h->r0 || r1 > h->r1) return OR_INVALID;
  const uint64_t w = i1 - i0;
  for (uint32_t r = r0; r < r1; ++r)
    for (uint32_t i = i0; i < i1; ++i)
      out[(uint64_t)(r - r0) * w + (i - i0)] = row_time(h->ranks[r - h->r0], (size_t)i + 1, c);
  return OR_OK;
}

// Q3, the k slowest ranks of context c over every rank of the handle (the
// ranks a per-context view ranks first, Section VI-B): ranks ordered by the
// metric's value x descending, equal values by rank ascending; the first
// min(k, n) are written with x and their z-score (n x - S1) / (n std) over all
// n ranks (0 when n < 2 or every value is equal), std with ddof 1 as in the
// statistics above.  Absent ranks take part with x = 0.
int or_topk(void* hp, int metric, uint32_t c, uint32_t k, uint32_t* out_rank, uint64_t* out_x,
            double* out_z, uint32_t* n_out) {
  Handle* h = (Handle*)hp;
  if (c >= h->in.C) return OR_INVALID;
  const uint64_t n = h->r1 - h->r0;
  std::vector<std::pair<uint64_t, uint32_t>> xs;
  uint64_t S1 = 0;
  u128 S2 = 0;
  for (uint32_t r = h->r0; r < h->r1; ++r) {
    uint64_t x, cnt;
    lookup(metric_of(h->ranks[r - h->r0], metric), c, x, cnt);
    xs.push_back({x, r});
    S1 += x;
    S2 += (u128)x * x;
  }
  const u128 M = (u128)n * S2 - (u128)S1 * S1;
  const double sd =
      (n < 2) ? 0.0 : std::sqrt(u128_to_double(M) / u128_to_double((u128)n * (n - 1)));
  std::sort(xs.begin(), xs.end(), [](const std::pair<uint64_t, uint32_t>& a,
                                     const std::pair<uint64_t, uint32_t>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  });
  const uint32_t m = (uint32_t)std::min<uint64_t>(k, n);
  for (uint32_t j = 0; j < m; ++j) {
    const i128 D = (i128)((u128)n * xs[j].first) - (i128)S1;
    out_rank[j] = xs[j].second;
    out_x[j] = xs[j].first;
    out_z[j] = (n < 2 || M == 0) ? 0.0 : i128_to_double(D) / (u128_to_double(n) * sd);
  }
  *n_out = m;
  return OR_OK;
}

// Finalize-only entry for the Table V pin: the paper prints per-kernel
// average mean and average max over ranks; savings per iteration is their
// difference, the kernel's total is that times the iteration count, and the
// speedup fraction is the summed totals over the application time.
void or_savings_from_averages(const double* avg_mean, const double* avg_max, uint32_t n_k,
                              uint32_t iterations, double app_time, double* savings,
                              double* totals, double* sum_total, double* fraction) {
  double s = 0.0;
  for (uint32_t k = 0; k < n_k; ++k) {
    savings[k] = avg_max[k] - avg_mean[k];
    totals[k] = savings[k] * iterations;
    s += totals[k];
  }
  *sum_total = s;
  *fraction = s / app_time;
}

}  // extern "C"
