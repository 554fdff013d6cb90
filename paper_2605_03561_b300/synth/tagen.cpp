// tagen.cpp -- seeded synthetic trace-set generator.  See tagen.h.
//
// Workload recipe (stand-in for the paper's AMG / GAMESS traces, Section VI):
//  * CCT: node 0 is the root; for v >= 1 the parent is uniform over the nodes
//    u < v whose depth is below max_depth.
//  * Iteration program: K segments, each a distinct context drawn uniformly
//    from the non-root, non-marker nodes, with weight w_k ~ U[1, 10];
//    round(comm_frac * K) of them (at least one) are "communication".
//  * A trace: prologue_len samples of a fixed prologue context, then I
//    iterations; an iteration is one marker sample followed, per segment, by a
//    run of samples whose sizes split the iteration by the weights (largest
//    remainder rounding).
//  * Timestamps: t0 ~ U[0, 1 ms); each sample's gap to the next is
//    max(1, round(Exp(gap_mean) * s)) with s the slowdown of the model.
#include "tagen.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace {

inline uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Xoshiro {  // xoshiro256** (Blackman & Vigna)
  uint64_t s[4];
  explicit Xoshiro(uint64_t seed) {
    uint64_t x = seed;
    for (auto& w : s) w = splitmix64(x);
  }
  static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  inline uint64_t next() {
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
  }
  inline double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }  // [0,1)
  inline double normal() {  // Box-Muller
    double u1 = uniform(), u2 = uniform();
    if (u1 < 1e-300) u1 = 1e-300;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  inline uint64_t below(uint64_t n) { return n ? next() % n : 0; }
};

uint64_t rank_seed(uint64_t seed, uint32_t r) {
  uint64_t x = seed ^ (uint64_t)r;
  return splitmix64(x);
}

// Everything that is shared by all ranks of one experiment.
struct Experiment {
  tagen_config c;
  uint32_t K = 0;
  uint32_t prologue_ctx = 0;
  std::vector<uint32_t> seg_ctx;
  std::vector<double> seg_w;
  std::vector<uint8_t> seg_comm;
  std::vector<uint8_t> slow_rank;   // model 1 or 2 (imbalanced ranks)
  std::vector<uint8_t> slow_rack;   // model 3
  uint32_t n_nodes = 0;
  std::vector<uint32_t> rack_of_node, chassis_of_node;
  uint32_t n_chassis = 0;

  explicit Experiment(const tagen_config& cfg) : c(cfg) {
    uint64_t es = cfg.seed ^ 0xA5A5F00DCAFEBEEFull;
    Xoshiro g(splitmix64(es));
    const uint32_t C = c.n_ctx;
    K = std::min<uint32_t>(c.n_segments, C > 2 ? C - 2 : 0);
    // Candidate contexts: all but the root (0) and the marker.
    std::vector<uint32_t> pool;
    pool.reserve(C);
    for (uint32_t v = 1; v < C; ++v)
      if (v != c.marker_ctx) pool.push_back(v);
    // Partial Fisher-Yates: the first K+1 entries become the program + prologue.
    uint32_t take = std::min<uint32_t>(K + 1, (uint32_t)pool.size());
    for (uint32_t i = 0; i < take; ++i) {
      uint32_t j = i + (uint32_t)g.below(pool.size() - i);
      std::swap(pool[i], pool[j]);
    }
    seg_ctx.assign(pool.begin(), pool.begin() + K);
    prologue_ctx = (take > K) ? pool[K] : (K ? seg_ctx[0] : 1);
    seg_w.resize(K);
    for (uint32_t k = 0; k < K; ++k) seg_w[k] = 1.0 + 9.0 * g.uniform();
    seg_comm.assign(K, 0);
    if (K) {
      uint32_t n_comm = (uint32_t)std::llround(c.comm_frac * K);
      if (c.comm_frac > 0 && n_comm == 0) n_comm = 1;
      n_comm = std::min(n_comm, K);
      std::vector<uint32_t> perm(K);
      for (uint32_t k = 0; k < K; ++k) perm[k] = k;
      for (uint32_t i = 0; i < n_comm; ++i) {
        uint32_t j = i + (uint32_t)g.below(K - i);
        std::swap(perm[i], perm[j]);
        seg_comm[perm[i]] = 1;
      }
    }
    const uint32_t R = c.n_ranks;
    slow_rank.assign(R, 0);
    auto pick_ranks = [&](uint32_t n) {
      n = std::min(n, R);
      std::vector<uint32_t> perm(R);
      for (uint32_t r = 0; r < R; ++r) perm[r] = r;
      for (uint32_t i = 0; i < n; ++i) {
        uint32_t j = i + (uint32_t)g.below(R - i);
        std::swap(perm[i], perm[j]);
        slow_rank[perm[i]] = 1;
      }
    };
    if (c.slow_model == TAGEN_SLOW_RANKS) pick_ranks(c.n_slow_ranks);
    if (c.slow_model == TAGEN_SLOW_JITTER)
      pick_ranks((uint32_t)std::llround(c.imb_rank_frac * R));
    // Topology.
    const uint32_t rpn = c.ranks_per_node ? c.ranks_per_node : 1;
    const uint32_t nr = c.n_racks ? c.n_racks : 1;
    const uint32_t npc = c.nodes_per_chassis ? c.nodes_per_chassis : 1;
    n_nodes = (R + rpn - 1) / rpn;
    rack_of_node.resize(n_nodes);
    chassis_of_node.resize(n_nodes);
    for (uint32_t n = 0; n < n_nodes; ++n)
      rack_of_node[n] = (uint32_t)((uint64_t)n * nr / std::max<uint32_t>(n_nodes, 1));
    uint32_t chassis_base = 0, first = 0;
    for (uint32_t n = 0; n <= n_nodes; ++n) {
      if (n == n_nodes || (n > 0 && rack_of_node[n] != rack_of_node[n - 1])) {
        uint32_t cnt = n - first;
        for (uint32_t m = first; m < n; ++m) chassis_of_node[m] = chassis_base + (m - first) / npc;
        chassis_base += (cnt + npc - 1) / npc;
        first = n;
      }
    }
    n_chassis = chassis_base;
    slow_rack.assign(nr, 0);
    if (c.slow_model == TAGEN_SLOW_RACK_COMM) {
      uint32_t n = std::min(c.n_slow_racks, nr);
      std::vector<uint32_t> perm(nr);
      for (uint32_t i = 0; i < nr; ++i) perm[i] = i;
      for (uint32_t i = 0; i < n; ++i) {
        uint32_t j = i + (uint32_t)g.below(nr - i);
        std::swap(perm[i], perm[j]);
        slow_rack[perm[i]] = 1;
      }
      for (uint32_t r = 0; r < R; ++r)
        if (slow_rack[rack_of_node[r / rpn]]) slow_rank[r] = 1;
    }
  }

  uint64_t min_len() const {
    return (uint64_t)c.n_iter * (K + 1) + c.prologue_len;
  }

  // Per-rank length: the first draws of the rank's stream.
  uint64_t length_of(Xoshiro& g) const {
    if (c.len_kind == TAGEN_LEN_FIXED) return std::max<uint64_t>((uint64_t)std::llround(c.len_mean), 0);
    double mu = std::log(c.len_mean) - 0.5 * c.len_sigma * c.len_sigma;
    double L = std::exp(mu + c.len_sigma * g.normal());
    double lo = (double)min_len(), hi = 20.0 * c.len_mean;
    L = std::min(std::max(std::round(L), lo), hi);
    return (uint64_t)L;
  }

  // Largest-remainder split of `body` samples over the K weights.
  void split(uint64_t body, std::vector<uint64_t>& n) const {
    n.assign(K, 0);
    if (!K) return;
    double W = 0;
    for (double w : seg_w) W += w;
    std::vector<std::pair<double, uint32_t>> frac(K);
    uint64_t used = 0;
    for (uint32_t k = 0; k < K; ++k) {
      double q = seg_w[k] / W * (double)body;
      n[k] = (uint64_t)std::floor(q);
      used += n[k];
      frac[k] = {q - std::floor(q), k};
    }
    std::stable_sort(frac.begin(), frac.end(),
                     [](const auto& a, const auto& b) { return a.first > b.first; });
    for (uint64_t i = 0; used < body; ++i, ++used) n[frac[i % K].second] += 1;
  }

  void fill_rank(uint32_t r, uint64_t len, uint64_t* ts, uint32_t* ctx) const {
    Xoshiro g(rank_seed(c.seed, r));
    (void)length_of(g);  // keep the stream aligned with tagen_plan
    uint64_t t = (uint64_t)(g.uniform() * 1.0e6);
    const uint32_t I = c.n_iter;
    const uint64_t P = std::min<uint64_t>(c.prologue_len, len);
    const uint64_t body = len - P;
    const double mean = c.gap_mean_ns;
    double rank_s = 1.0;
    if (c.slow_model == TAGEN_SLOW_RANKS && slow_rank[r]) rank_s = c.slow_factor;
    const bool rack_slow = (c.slow_model == TAGEN_SLOW_RACK_COMM) && slow_rank[r];
    uint64_t i = 0;
    auto emit = [&](uint32_t cx, double s) {
      ts[i] = t;
      ctx[i] = cx;
      double e = -std::log(1.0 - g.uniform()) * mean * s;
      uint64_t gap = (uint64_t)std::llround(e);
      t += gap < 1 ? 1 : gap;
      ++i;
    };
    for (uint64_t p = 0; p < P; ++p) emit(prologue_ctx, rank_s);
    if (I == 0 || body == 0) {
      while (i < len) emit(prologue_ctx, rank_s);
      return;
    }
    const uint64_t base = body / I, extra = body % I;
    std::vector<uint32_t> order(K);
    for (uint32_t k = 0; k < K; ++k) order[k] = k;
    std::vector<uint64_t> split_lo, split_hi;
    if (base >= 1) split(base - 1, split_lo);
    split(base, split_hi);  // used by the +1 iterations: (base + 1) - 1 samples
    for (uint32_t it = 0; it < I; ++it) {
      uint64_t L_it = base + (it < extra ? 1 : 0);
      double s = rank_s;
      if (c.slow_model == TAGEN_SLOW_JITTER) {
        double j = 1.0 + c.jitter_sigma * g.normal();
        j = std::min(std::max(j, 1.0 - c.jitter_clip), 1.0 + c.jitter_clip);
        double u = g.uniform(), f = c.imb_lo + (c.imb_hi - c.imb_lo) * g.uniform();
        if (slow_rank[r] && u < c.imb_iter_prob) j *= f;
        s *= j;
      }
      if (L_it == 0) continue;
      emit(c.marker_ctx, s);
      const std::vector<uint64_t>& n = (L_it == base) ? split_lo : split_hi;
      if (c.shuffle_segments)  // Fisher-Yates over the segment order
        for (uint32_t k = K; k > 1; --k) std::swap(order[k - 1], order[g.below(k)]);
      for (uint32_t kk = 0; kk < K; ++kk) {
        const uint32_t k = order[kk];
        double sk = (rack_slow && seg_comm[k]) ? s * c.slow_factor : s;
        for (uint64_t q = 0; q < n[k]; ++q) emit(seg_ctx[k], sk);
      }
    }
  }
};

void build_parent(const tagen_config& c, uint32_t* parent) {
  uint64_t es = c.seed ^ 0x5EEDC0DE12345678ull;
  Xoshiro g(splitmix64(es));
  const uint32_t C = c.n_ctx;
  std::vector<uint32_t> depth(C, 0), eligible;
  eligible.reserve(C);
  parent[0] = 0xFFFFFFFFu;
  if (c.max_depth > 0) eligible.push_back(0);
  for (uint32_t v = 1; v < C; ++v) {
    uint32_t p = eligible.empty() ? 0 : eligible[g.below(eligible.size())];
    parent[v] = p;
    depth[v] = depth[p] + 1;
    if (depth[v] < c.max_depth) eligible.push_back(v);
  }
}

}  // namespace

extern "C" {

int tagen_preset(int preset, tagen_config* c) {
  if (!c) return -1;
  std::memset(c, 0, sizeof(*c));
  c->seed = 1;
  c->max_depth = 12;
  c->n_segments = 64;
  c->prologue_len = 16;
  c->marker_ctx = 1;
  c->gap_mean_ns = 10000.0;
  c->jitter_sigma = 0.05;
  c->jitter_clip = 0.15;
  c->imb_rank_frac = 0.01;
  c->imb_iter_prob = 0.2;
  c->imb_lo = 1.2;
  c->imb_hi = 2.0;
  c->comm_frac = 0.1;
  c->ranks_per_node = 12;
  c->n_racks = 22;
  c->nodes_per_chassis = 8;
  c->n_slow_racks = 3;
  switch (preset) {
    case 0:  // tiny
      c->n_ranks = 8; c->n_ctx = 24; c->max_depth = 5; c->n_iter = 3; c->n_segments = 6;
      c->prologue_len = 4; c->len_kind = TAGEN_LEN_FIXED; c->len_mean = 60;
      c->slow_model = TAGEN_SLOW_RANKS; c->n_slow_ranks = 1; c->slow_factor = 1.5;
      c->ranks_per_node = 2; c->n_racks = 2; c->nodes_per_chassis = 1;
      return 0;
    case 1:  // 64 ranks x 20k samples, C = 200, depth <= 12, I = 10, 2 ranks 1.5x
      c->n_ranks = 64; c->n_ctx = 200; c->max_depth = 12; c->n_iter = 10;
      c->len_kind = TAGEN_LEN_FIXED; c->len_mean = 20000;
      c->slow_model = TAGEN_SLOW_RANKS; c->n_slow_ranks = 2; c->slow_factor = 1.5;
      c->ranks_per_node = 4; c->n_racks = 4; c->nodes_per_chassis = 2;
      return 0;
    case 2:  // 4096 ranks, C = 5000, depth <= 24, lognormal mean 100k sigma 0.5, I = 50
      c->n_ranks = 4096; c->n_ctx = 5000; c->max_depth = 24; c->n_iter = 50;
      c->len_kind = TAGEN_LEN_LOGNORMAL; c->len_mean = 100000; c->len_sigma = 0.5;
      c->slow_model = TAGEN_SLOW_JITTER;
      c->ranks_per_node = 12; c->n_racks = 22; c->nodes_per_chassis = 8;
      return 0;
    case 3:  // 100,000 ranks, C = 20,000, lognormal mean 20k sigma 0.7, I = 100
      c->n_ranks = 100000; c->n_ctx = 20000; c->max_depth = 24; c->n_iter = 100;
      c->len_kind = TAGEN_LEN_LOGNORMAL; c->len_mean = 20000; c->len_sigma = 0.7;
      c->slow_model = TAGEN_SLOW_RACK_COMM; c->slow_factor = 1.3; c->n_slow_racks = 3;
      c->ranks_per_node = 12; c->n_racks = 22; c->nodes_per_chassis = 8;
      return 0;
    default:
      return -1;
  }
}

int tagen_plan(const tagen_config* cfg, uint64_t* rank_off, uint32_t* parent,
               tagen_info* info) {
  if (!cfg || cfg->n_ctx < 3 || cfg->marker_ctx == 0 || cfg->marker_ctx >= cfg->n_ctx)
    return -1;
  Experiment e(*cfg);
  uint64_t off = 0;
  uint32_t max_len = 0;
  if (rank_off) rank_off[0] = 0;
  for (uint32_t r = 0; r < cfg->n_ranks; ++r) {
    Xoshiro g(rank_seed(cfg->seed, r));
    uint64_t L = e.length_of(g);
    off += L;
    max_len = std::max<uint32_t>(max_len, (uint32_t)L);
    if (rank_off) rank_off[r + 1] = off;
  }
  if (parent) build_parent(*cfg, parent);
  if (info) {
    info->n_segments = e.K;
    info->prologue_ctx = e.prologue_ctx;
    info->n_nodes = e.n_nodes;
    info->n_chassis = e.n_chassis;
    info->n_records = off;
    info->max_len = max_len;
  }
  return 0;
}

int tagen_fill(const tagen_config* cfg, const uint64_t* rank_off, uint32_t r0,
               uint32_t r1, uint64_t* ts, uint32_t* ctx, int n_threads) {
  if (!cfg || !rank_off || r1 < r0 || r1 > cfg->n_ranks) return -1;
  Experiment e(*cfg);
  const uint64_t base = rank_off[r0];
  int T = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  const uint32_t n = r1 - r0;
  if ((uint32_t)T > n) T = n ? (int)n : 1;
  auto work = [&](int t) {
    for (uint32_t r = r0 + t; r < r1; r += T) {
      uint64_t b = rank_off[r] - base, len = rank_off[r + 1] - rank_off[r];
      e.fill_rank(r, len, ts + b, ctx + b);
    }
  };
  if (T == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  return 0;
}

int tagen_topology(const tagen_config* cfg, uint32_t* node_of_rank,
                   uint32_t* rack_of_node, uint32_t* chassis_of_node) {
  if (!cfg) return -1;
  Experiment e(*cfg);
  const uint32_t rpn = cfg->ranks_per_node ? cfg->ranks_per_node : 1;
  if (node_of_rank)
    for (uint32_t r = 0; r < cfg->n_ranks; ++r) node_of_rank[r] = r / rpn;
  for (uint32_t n = 0; n < e.n_nodes; ++n) {
    if (rack_of_node) rack_of_node[n] = e.rack_of_node[n];
    if (chassis_of_node) chassis_of_node[n] = e.chassis_of_node[n];
  }
  return 0;
}

int tagen_truth(const tagen_config* cfg, uint8_t* slowed_rank, uint8_t* slowed_rack,
                uint8_t* comm_segment, uint32_t* segment_ctx) {
  if (!cfg) return -1;
  Experiment e(*cfg);
  if (slowed_rank) std::memcpy(slowed_rank, e.slow_rank.data(), e.slow_rank.size());
  if (slowed_rack) std::memcpy(slowed_rack, e.slow_rack.data(), e.slow_rack.size());
  if (comm_segment) std::memcpy(comm_segment, e.seg_comm.data(), e.seg_comm.size());
  if (segment_ctx) std::memcpy(segment_ctx, e.seg_ctx.data(), e.seg_ctx.size() * 4);
  return 0;
}

}  // extern "C"
