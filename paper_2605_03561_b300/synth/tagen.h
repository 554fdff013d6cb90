/*
 * tagen.h -- seeded synthetic trace-set generator (host C++, C ABI).
 *
 * The paper's workloads (an AMG run at 100,000 ranks on Aurora, a GAMESS run
 * on Frontier; Section VI) are not available, so this generator stands in for
 * them.  It produces what the paper's Read API would hand to the analysis
 * (Section II-A): per-rank execution traces, each a time-ordered list of
 * (u64 timestamp ns, u32 calling-context id) samples (Section II-A, trace
 * slices), a calling context tree given as a parent array, an iteration
 * marker context, and an integer rank -> node -> rack/chassis topology
 * (Section VI-B).
 *
 * This module holds none of the analysis method's arithmetic: it only draws
 * inputs.  Both the CUDA path and the CPU oracle consume its output; neither
 * includes this header.
 *
 * Randomness: every rank r draws from its own xoshiro256** stream seeded by
 * splitmix64(seed ^ r) (both are public, named generators), so ranks can be
 * generated independently, in any order, in parallel or in chunks.
 * Experiment-level choices (tree, iteration program, slowed ranks/racks) come
 * from a separate stream.
 */
#ifndef TAGEN_H
#define TAGEN_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum {
  TAGEN_LEN_FIXED = 0,     /* every trace has len_mean samples            */
  TAGEN_LEN_LOGNORMAL = 1  /* lognormal with arithmetic mean len_mean     */
};

enum {
  TAGEN_SLOW_NONE = 0,
  TAGEN_SLOW_RANKS = 1,      /* n_slow_ranks ranks run slow_factor slower      */
  TAGEN_SLOW_JITTER = 2,     /* per-(rank, iteration) Gaussian jitter, plus a   */
                             /* fraction of ranks slowed on random iterations   */
  TAGEN_SLOW_RACK_COMM = 3   /* ranks in n_slow_racks racks run slow_factor     */
                             /* slower in communication segments               */
};

typedef struct tagen_config {
  uint64_t seed;
  uint32_t n_ranks;           /* R                                           */
  uint32_t n_ctx;             /* C (>= 3)                                     */
  uint32_t max_depth;         /* deepest allowed node depth (root = 0)        */
  uint32_t n_iter;            /* I iterations per trace                       */
  uint32_t n_segments;        /* K segments per iteration (capped at C - 2)   */
  uint32_t prologue_len;      /* samples before the first marker              */
  uint32_t marker_ctx;        /* iteration marker context (1..C-1)            */
  uint32_t len_kind;          /* TAGEN_LEN_*                                  */
  double len_mean;            /* mean samples per trace                       */
  double len_sigma;           /* lognormal sigma                              */
  double gap_mean_ns;         /* mean of the exponential inter-sample gap     */
  uint32_t slow_model;        /* TAGEN_SLOW_*                                 */
  uint32_t n_slow_ranks;      /* TAGEN_SLOW_RANKS                             */
  double slow_factor;         /* TAGEN_SLOW_RANKS / TAGEN_SLOW_RACK_COMM      */
  double jitter_sigma;        /* TAGEN_SLOW_JITTER: N(0, sigma) jitter        */
  double jitter_clip;         /* ... clipped to +-clip                        */
  double imb_rank_frac;       /* ... fraction of imbalanced ranks             */
  double imb_iter_prob;       /* ... per-iteration probability                */
  double imb_lo, imb_hi;      /* ... U[lo, hi] extra factor                   */
  double comm_frac;           /* fraction of segments that are communication  */
  uint32_t ranks_per_node;
  uint32_t n_racks;
  uint32_t nodes_per_chassis;
  uint32_t n_slow_racks;      /* TAGEN_SLOW_RACK_COMM                         */
  uint32_t shuffle_segments;  /* 1: every iteration runs its segments in a    */
                              /* fresh random order (rows never repeat the     */
                              /* previous row's run sequence)                  */
} tagen_config;

/* Experiment description that does not depend on the record arrays. */
typedef struct tagen_info {
  uint32_t n_segments;        /* effective K                                  */
  uint32_t prologue_ctx;
  uint32_t n_nodes, n_chassis;
  uint64_t n_records;         /* N = sum of trace lengths                     */
  uint32_t max_len;           /* longest trace                                */
} tagen_info;

/* Fill the defaults of the config family named by `preset`
 * (1: 64 ranks x 20k, 2: 4096 ranks lognormal 100k, 3: 100,000 ranks
 * lognormal 20k with rack topology, 0: tiny).  Returns 0 on success. */
int tagen_preset(int preset, tagen_config* cfg);

/* Trace lengths -> rank_off[R+1] (CSR offsets), CCT parent[C]
 * (root = 0xFFFFFFFF), and info.  Either output pointer may be NULL. */
int tagen_plan(const tagen_config* cfg, uint64_t* rank_off, uint32_t* parent,
               tagen_info* info);

/* Records of ranks [r0, r1): ts/ctx are written at index
 * rank_off[r] - rank_off[r0].  n_threads <= 0 uses all hardware threads. */
int tagen_fill(const tagen_config* cfg, const uint64_t* rank_off, uint32_t r0,
               uint32_t r1, uint64_t* ts, uint32_t* ctx, int n_threads);

/* Integer topology: node_of_rank[R], rack_of_node[n_nodes],
 * chassis_of_node[n_nodes] (global chassis ids). */
int tagen_topology(const tagen_config* cfg, uint32_t* node_of_rank,
                   uint32_t* rack_of_node, uint32_t* chassis_of_node);

/* Ground truth of the injected slowdowns, for planted-structure tests:
 * slowed_rank[R] (1 if the rank was slowed in any way), slowed_rack[n_racks],
 * comm_segment_ctx[K] (1 if the k-th segment is communication) and
 * segment_ctx[K] (the ctx of segment k).  Any pointer may be NULL. */
int tagen_truth(const tagen_config* cfg, uint8_t* slowed_rank,
                uint8_t* slowed_rack, uint8_t* comm_segment,
                uint32_t* segment_ctx);

#ifdef __cplusplus
}
#endif
#endif
