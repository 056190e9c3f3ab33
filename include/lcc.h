/*
 * lcc.h -- C ABI of the GB300 LambdaCC library (liblcc.so).
 *
 * The library clusters an undirected weighted graph G = (V, E, w) under the
 * LambdaCC objective of Shi et al., "Scalable Community Detection via Parallel
 * Correlation Clustering" (arXiv 2108.01731):
 *
 *   CC(x) = sum over ordered pairs (i, j) in V x V of w'_ij (1 - x_ij),
 *   w'_uu = 0, w'_uv = w_uv - lambda k_u k_v on edges, -lambda k_u k_v off
 *   edges                                                   (Sec. 2)
 *
 * with the parallel Louvain method of Algorithm 1 run on the synchronous
 * schedule of Sec. 3.2.1: every round computes each vertex's best move from a
 * snapshot of the labels and cluster weights, then applies all moves at once;
 * rounds stop when nothing moves or after num_iter rounds; the clustering is
 * then compressed (Sec. 3.1, Appendix B) and the method recurses, flattens
 * and refines (Sec. 3.2.3).
 *
 * Arithmetic.  lambda is the rational p/q with p, q > 0.  Every gain is an
 * exact integer (gains are scaled by q), so labels are bit-identical from run
 * to run and independent of thread scheduling.  Exactness has a range: with
 * W = sum of |w| over all entries and Ktot = sum of the node weights, every
 * call that computes gains or the objective returns LCC_ERR_OVERFLOW unless
 * W < 2^62, Ktot < 2^62, q W < 2^125 and p Ktot^2 < 2^125 (q being q 2m in
 * LCC_NODEW_DEGREE mode).  Inside it every gain term, every comparison of two
 * gains and the objective fit a signed 128-bit integer on every level.  Ties between candidate
 * clusters go to the smallest cluster id, and a vertex moves only when the
 * best candidate is strictly better than staying.  Vertex v may also move to
 * cluster id v when that id has zero weight and none of v's neighbours is in
 * it (gain 0).  Final labels are the smallest vertex id of each cluster.
 *
 * Conventions for every entry point:
 *   - return an lcc_status; they never throw and never abort the process;
 *     lcc_last_error() gives a detail message for the calling thread;
 *   - host arrays are caller-owned and only read (or written, for outputs)
 *     during the call; the library copies what it keeps;
 *   - the GPU is the device current on the calling thread when the object is
 *     created; every later call on that object uses the same device;
 *   - `stream` is a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)
 *     or NULL for the legacy default stream.  Calls that return results on the
 *     host synchronise that stream before returning.
 *
 * Environment.  LCC_LAYOUT_MIN_BYTES (bytes, default 64 MiB): a level whose
 * packed label words (8 bytes per vertex) exceed it stores them in a
 * degree-ordered layout, at 4 bytes per vertex and 4 per CSR entry of extra
 * device memory.  When one contraction builds the coarse levels of several
 * graphs together, only the first graph's level takes it.  It moves storage
 * only, never a result.
 */
#ifndef LCC_H
#define LCC_H

#include <stdint.h>

#if defined(__GNUC__)
#define LCC_API __attribute__((visibility("default")))
#else
#define LCC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lcc_status {
  LCC_OK = 0,
  LCC_ERR_INVALID = 1,       /* bad argument or malformed CSR */
  LCC_ERR_NOT_SYMMETRIC = 2, /* the multiset {(u,v,w)} differs from {(v,u,w)};
                                lcc_load_csr compares two 128-bit hashes of the
                                multisets, so an asymmetric graph passes only
                                if the hashes collide (probability about
                                2^-64 or less) */
  LCC_ERR_SELF_LOOP = 3,     /* an entry u -> u */
  LCC_ERR_OOM = 4,           /* device or host allocation failed */
  LCC_ERR_OVERFLOW = 5,      /* a total exceeds the exact integer range */
  LCC_ERR_TIMEOUT = 6,       /* a bounded wait ran out */
  LCC_ERR_CUDA = 7,          /* a CUDA runtime call failed */
  LCC_ERR_BUSY = 8,          /* the result is not ready yet (serving API) */
  LCC_ERR_CANCELLED = 9      /* the job was cancelled (serving API) */
} lcc_status;

/* Node weights k (Sec. 2). */
typedef enum lcc_nodew_mode {
  LCC_NODEW_UNIT = 0,   /* k_v = 1; lambda = p / q */
  LCC_NODEW_DEGREE = 1, /* modularity: k_v = sum_u w_uv, lambda = gamma / 2m
                           with gamma = p / q and 2m = sum_v k_v (Sec. 2) */
  LCC_NODEW_CUSTOM = 2  /* k given at load time (non-negative); lambda = p/q */
} lcc_nodew_mode;

/* The vertex subset V' examined in the rounds after the first (Sec. 3.2.2). */
typedef enum lcc_vset {
  LCC_VSET_ALL = 0,           /* V' = V every round */
  LCC_VSET_NBR_VERTICES = 1,  /* neighbours of the vertices that moved */
  LCC_VSET_NBR_CLUSTERS = 2   /* neighbours of every vertex now in a cluster
                                 that some vertex moved out of */
} lcc_vset;

typedef enum lcc_memspace { LCC_MEM_HOST = 0, LCC_MEM_DEVICE = 1 } lcc_memspace;

/* Schedule flags. */
#define LCC_SCHED_TIMING 1 /* record per-phase device time in lcc_stats */
/* With LCC_VSET_NBR_VERTICES, V' of the next round is by default found in one
   of two ways with the same result on a symmetric graph: by marking the
   neighbours of every moved vertex, or, after a round whose movers' rows hold
   at least a quarter of the level's entries, by evaluating every vertex with
   an edge and keeping the label of each one none of whose neighbours moved.
   This flag always takes the first way. */
#define LCC_SCHED_MARK_ONLY 2
/* Symmetry-breaking coin.  The synchronous rounds have none, and the paper
   notes that they often end at very poor, even negative, objectives (Sec. 4).
   With this flag, a vertex whose best move differs from its cluster moves in
   round t of a Best-Moves call only if a coin allows it: the top bit of
   output key + 1 of the SplitMix64 stream seeded with `seed` (output i is the
   SplitMix64 finaliser of seed + i * 0x9e3779b97f4a7c15), with
   key = v + (t mod 2^16) 2^32 + (depth mod 2^8) 2^48 + phase 2^56, phase 1
   for the refinement call after Flatten, else 0.  A vertex held back keeps
   its label and is evaluated again in the next round; a call ends when no
   vertex wants to move (or after num_iter rounds).  Results stay
   deterministic for a given seed.  This schedule always marks V' (no pull
   rounds). */
#define LCC_SCHED_COIN 4

typedef struct lcc_schedule {
  int32_t num_iter;   /* max rounds per Best-Moves call (Algorithm 1); >= 0 */
  int32_t max_levels; /* max recursion depth incl. the input level; >= 1 */
  int32_t refine;     /* 1: Best-Moves again after each Flatten (Sec. 3.2.3) */
  int32_t vset;       /* lcc_vset */
  int32_t sync;       /* must be 1: the synchronous schedule (Sec. 3.2.1) */
  int32_t flags;      /* LCC_SCHED_* */
  uint64_t seed;      /* seed of the LCC_SCHED_COIN coin (ignored without it) */
} lcc_schedule;

typedef struct lcc_stats {
  int32_t levels;          /* levels visited, including the input level */
  int32_t rounds_total;    /* Best-Moves rounds over all levels */
  int64_t edges_scanned;   /* sum of deg(v) over every vertex evaluated */
  int64_t vertices_scanned;/* number of best-move evaluations */
  int64_t candidates;      /* distinct neighbouring clusters scored */
  int64_t num_clusters;    /* clusters in the final labelling */
  int64_t obj_num_hi;      /* exact objective: CC = num / den, num = hi:lo */
  uint64_t obj_num_lo;     /*   as a two's-complement 128-bit integer */
  int64_t obj_den;         /* q, or q * 2m in LCC_NODEW_DEGREE mode */
  double objective;        /* (double)num / den */
  /* device time in ms, filled when LCC_SCHED_TIMING is set */
  double ms_bestmove;      /* best-move kernels (all degree buckets, and the
                              pass that gathers the label words of a round
                              that reads every row: ms_gather) */
  double ms_round_other;   /* frontier, apply and marking kernels */
  double ms_contract;      /* compression (relabel, sort, reduce, CSR) */
  double ms_other;         /* flatten, refinement set-up, final labels */
  double ms_total;
  int64_t bytes_bestmove;  /* algorithmic bytes of the best-move kernels */
  int64_t pairs_sorted;    /* inter-cluster entries sorted by compression */
  int64_t kernel_launches; /* kernels launched by this call */
  /* best-move device time per degree bucket (rows of <=4, <=8, <=16, <=32,
     <=64, <=128, <=256, <=1024, <=2048, <=4096, <=8192, <=16384, <=32768,
     <=65536, <=131072 entries, and longer), filled when LCC_SCHED_TIMING is
     set; with the partitioned path on (lcc_tuning.part_min), its whole time
     is in the first bucket it takes */
  double ms_bucket[16];
  int64_t bucket_entries[16];  /* entries processed per degree bucket (after a
                                  round that marks no V', every row with an
                                  edge is processed) */
  int64_t bucket_vertices[16]; /* vertices processed per degree bucket */
  int64_t bytes_contract_min;  /* least bytes the contractions must move: each
                                  contracted level's offsets, neighbours, weights
                                  and labels read once, and the coarse offsets,
                                  neighbours, int64 weights and node weights
                                  written once (compare with ms_contract) */
  /* Best-Moves calls (each coarsening and each refinement call with at least
     one round), and those that stopped at num_iter rounds while some vertex
     still wanted to move.  The paper's run-to-convergence variant (Sec. 4,
     the ^CON runs) is a schedule whose num_iter is never reached:
     calls_capped == 0 shows that every call converged. */
  int64_t calls;
  int64_t calls_capped;
  double ms_gather;        /* the gathered-word passes (lcc_tuning.pregather),
                              included in ms_bestmove */
} lcc_stats;

typedef struct lcc_graph lcc_graph;

/*
 * lcc_load_csr -- copy a CSR graph into device memory and validate it.
 *
 * offsets [n+1] int64, monotone, offsets[0] = 0, offsets[n] = nnz;
 * nbrs    [nnz] int32 in [0, n);
 * weights [nnz] int32 or NULL for an unweighted graph (w = 1);
 * node_w  [n]   int64 >= 0, only read in LCC_NODEW_CUSTOM runs (may be NULL
 *               otherwise).
 * `memspace` says where the four arrays live (all in the same space).
 * Both directions of every undirected edge must be present with equal
 * weights (Sec. 2 graphs are undirected); there are no self loops.
 * Returns LCC_ERR_INVALID (sizes, ranges, offsets), LCC_ERR_SELF_LOOP,
 * LCC_ERR_NOT_SYMMETRIC, LCC_ERR_OVERFLOW (sum of |w| >= 2^62 or n >= 2^31)
 * or LCC_ERR_OOM.  On success *out owns a device copy; free it with
 * lcc_free_graph.
 */
LCC_API lcc_status lcc_load_csr(const int64_t *offsets, const int32_t *nbrs,
                        const int32_t *weights, int64_t n, int64_t nnz,
                        const int64_t *node_w, int32_t memspace, void *stream,
                        lcc_graph **out);

/* Sizes of a loaded graph. */
LCC_API lcc_status lcc_graph_info(const lcc_graph *g, int64_t *n, int64_t *nnz);

LCC_API void lcc_free_graph(lcc_graph *g);

/*
 * lcc_cluster -- Parallel-CC (Algorithm 1) on a loaded graph.
 *
 * lambda = lambda_p / lambda_q (gamma in LCC_NODEW_DEGREE mode); both > 0.
 * sched NULL means {num_iter 10, max_levels 64, refine 1, nbr-vertices, sync}.
 * labels_out [n] int32 receives the final labels (smallest vertex id of each
 * cluster); it lives in `labels_memspace`.  objective_out (nullable) gets the
 * objective CC as a double; stats_out (nullable) the exact value and counters.
 * Runs on the stream given at load time.
 */
LCC_API lcc_status lcc_cluster(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q,
                       int32_t mode, const lcc_schedule *sched,
                       int32_t *labels_out, int32_t labels_memspace,
                       double *objective_out, lcc_stats *stats_out);

/* One Best-Moves round of a run.  The paper plots the size of V' per round
 * for its vertex-subset rules (appendix); this is that record. */
typedef struct lcc_round {
  int32_t level;   /* depth of the level (0 = the input graph) */
  int32_t phase;   /* 0: the call that coarsens the level; 1: its refinement
                      after Flatten (Sec. 3.2.3) */
  int32_t round;   /* round within that Best-Moves call, from 0 */
  int32_t pad;
  int64_t vprime;  /* |V'|: vertices examined by the round (Sec. 3.2.2) */
  int64_t entries; /* CSR entries scanned: the sum of their degrees */
  int64_t moved;   /* vertices that moved */
  int64_t held;    /* vertices whose move the LCC_SCHED_COIN coin held back */
} lcc_round;

/*
 * lcc_cluster_trace -- lcc_cluster plus one lcc_round per Best-Moves round,
 * in the order the rounds ran (coarsening calls on the way down, refinement
 * calls on the way up).  trace [trace_cap] (host, caller-owned) receives the
 * first trace_cap records; *trace_len (nullable) the number of rounds run,
 * which may exceed trace_cap.  The other arguments are those of lcc_cluster.
 */
LCC_API lcc_status lcc_cluster_trace(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q,
                                     int32_t mode, const lcc_schedule *sched,
                                     int32_t *labels_out, int32_t labels_memspace,
                                     double *objective_out, lcc_stats *stats_out,
                                     lcc_round *trace, int64_t trace_cap, int64_t *trace_len);

/*
 * lcc_desired -- one synchronous best-move evaluation (Algorithm 1, the body
 * of the parallel loop, with the Appendix A gain) on the input level.
 *
 * labels [n] (host) is the snapshot; cluster weights are K_c = sum of k_v
 * over labels[v] = c.  frontier [n] (host, nullable = all) marks the vertices
 * evaluated.  desired_out [n] (host) receives D[v] for evaluated vertices and
 * labels[v] for the rest.
 */
LCC_API lcc_status lcc_desired(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q,
                       int32_t mode, const int32_t *labels,
                       const uint8_t *frontier, int32_t *desired_out);

/*
 * lcc_best_moves -- Best-Moves (Algorithm 1) on the input level, starting
 * from labels_inout (host [n]) with V' = V, for at most num_iter rounds.
 * Writes the labels back, the rounds run and whether anything moved.
 */
LCC_API lcc_status lcc_best_moves(const lcc_graph *g, int64_t lambda_p,
                          int64_t lambda_q, int32_t mode, int32_t num_iter,
                          int32_t vset, int32_t *labels_inout,
                          int32_t *rounds_out, int32_t *moved_out);

/*
 * lcc_compress -- Compress (Sec. 3.1, Appendix B): every occupied cluster
 * becomes a coarse vertex (ids ranked by cluster id) whose node weight is the
 * cluster weight; edges between different clusters are merged by summing
 * their weights; edges inside a cluster are dropped.  labels [n] (host).
 * map_out [n] (host) gets the coarse vertex of each vertex.  *coarse_out is a
 * new graph (int64 weights) whose node weights are the coarse k; free it with
 * lcc_free_graph.  `mode` selects the input node weights as in lcc_cluster.
 */
LCC_API lcc_status lcc_compress(const lcc_graph *g, int32_t mode,
                        const int32_t *labels, int32_t *map_out,
                        lcc_graph **coarse_out);

/*
 * lcc_graph_export -- copy a graph back to the host: off [n+1], nbr [nnz],
 * w [nnz] as int64, k [n] the node weights it was loaded or built with
 * (1 for a graph loaded without node weights).  Any pointer may be NULL.
 */
LCC_API lcc_status lcc_graph_export(const lcc_graph *g, int64_t *off, int32_t *nbr,
                            int64_t *w, int64_t *k);

/*
 * lcc_objective -- exact objective of labels [n] (host) on the input level:
 * CC = num / den with num = (*num_hi : *num_lo) as a signed 128-bit integer.
 */
LCC_API lcc_status lcc_objective(const lcc_graph *g, int64_t lambda_p,
                         int64_t lambda_q, int32_t mode, const int32_t *labels,
                         int64_t *num_hi, uint64_t *num_lo, int64_t *den);

/*
 * lcc_desired_noalloc -- the evaluation of lcc_desired (every vertex
 * evaluated, node weights given) on a graph, labels and cluster weights that
 * already live in device memory, without allocating any device memory.  The
 * paper has no counterpart: this entry point exists for callers that may not
 * allocate GPU memory at the point of the call, because their own runtime owns
 * every device allocation (a memory-budgeted host framework, or a process that
 * gave the rest of the GPU's memory to another allocator).  Every other entry
 * point allocates working memory from a stream-ordered pool.
 *
 * All pointers are device pointers owned by the caller:
 *   d_off [n+1] int64, d_nbr [nnz] int32, d_w [nnz] int32 or NULL (w = 1),
 *   d_k [n] int64 node weights, d_labels [n] int32 in [0, n),
 *   d_K [n] int64 cluster weights (K[c] = sum of d_k over vertices labelled c),
 *   d_desired [n] int32 output.
 * lambda = lambda_p / lambda_q > 0 (for modularity pass q * 2m).
 * Working memory is one fixed 16 MiB array inside the library, which every GPU
 * that loads the library keeps until the process exits; rows longer than 4096
 * entries do not fit and make the call return LCC_ERR_INVALID.  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress); under lazy module loading the first call on a device
 * is the one that loads the library's device code, and with it the 16 MiB
 * array, so make that first call during set-up, before any stream capture.
 * All calls on a device share the array and the call clears what it needs,
 * but calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it: order them.  Synchronises `stream` before returning.
 * The kernel checks what it reads and the call then returns, instead of
 * LCC_OK: LCC_ERR_INVALID for a neighbour id or label outside [0, n), a
 * negative node or cluster weight, or a cluster weight above the total node
 * weight; LCC_ERR_OVERFLOW outside the exact range stated at the top of this
 * file.  d_desired is unspecified after an error.
 */
LCC_API lcc_status lcc_desired_noalloc(const int64_t *d_off, const int32_t *d_nbr,
                                       const int32_t *d_w, const int64_t *d_k, int64_t n,
                                       int64_t lambda_p, int64_t lambda_q,
                                       const int32_t *d_labels, const int64_t *d_K,
                                       int32_t *d_desired, void *stream);

/* ----------------------------------------------------------------------
 * Batched and served clustering.
 *
 * Many graphs run through one engine: every round, one launch per kernel
 * covers the current level of every active graph, and each graph keeps its
 * own level stack, round counter and termination, so its labels are
 * bit-identical to an lcc_cluster run on it alone.
 * ---------------------------------------------------------------------- */

/*
 * lcc_cluster_batch -- cluster `count` loaded graphs together.  All graphs
 * must live on the same device.  lambda_p/lambda_q/mode are per graph
 * (arrays of `count`); labels_out[i] is a host array [n_i].  objectives_out
 * (nullable) [count].
 */
LCC_API lcc_status lcc_cluster_batch(const lcc_graph *const *graphs, int32_t count,
                             const int64_t *lambda_p, const int64_t *lambda_q,
                             const int32_t *mode, const lcc_schedule *sched,
                             int32_t *const *labels_out,
                             double *objectives_out);

/*
 * Kernel tuning of one device.  The paper routes rows by one fixed degree
 * threshold between a sequential scan and a parallel hash table (Appendix B);
 * here rows of 33..warp_max entries run in the kernels for rows up to 256
 * entries (one warp per row up to 128 entries, one 128-thread block per row
 * up to 256), and longer rows up to 1024 entries one 256-thread block per
 * row.  A tuning changes which kernel evaluates a vertex, never a result.  A
 * level keeps the routing it was bucketed with when it was built.
 */
typedef struct lcc_tuning {
  int32_t warp_max;    /* 32, 64, 128 or 256 (the default) */
  int32_t fuse_small;  /* 1 (the default): rows of at most 32 entries of every
                          graph in one resident launch whose warps take work
                          units from a device counter; 0: one launch per
                          bucket of <= 4, 8, 16 and 32 entries */
  int32_t prefetch;    /* 1: the block kernels for rows of 129..4096 entries
                          load the next vertex's neighbour positions while
                          they merge the current vertex and ask L2 for its
                          label words; 0 (the default): no pipeline (fewer
                          registers per thread) */
  int32_t pregather;   /* 1 (the default): a round that reads every row (V' =
                          V, or V' tested inside the best-move kernels) first
                          gathers the label word of every entry in one flat
                          pass (8 bytes per entry of extra device memory), and
                          the best-move kernels read those words as a stream;
                          0: every entry gathers its own word */
  int32_t part_min;    /* 1024, 4096, 8192 (the default) or 16384: rows of
                          more than part_min entries are hash-partitioned by
                          cluster id into parts of at most about 1024 entries, each
                          part merged in one 256-thread block's shared memory
                          and the parts' best clusters reduced per row (a
                          row whose part overflows its table falls back to
                          global tables).  0: no partitioning; rows up to 8192
                          entries in one block, up to 131072 in a thread-block
                          cluster's distributed shared memory, longer ones in
                          windowed global tables */
  int32_t reserved[3]; /* zero */
} lcc_tuning;

/* lcc_get_tuning / lcc_set_tuning -- the tuning used by later calls on CUDA
 * device `device`.  LCC_ERR_INVALID for a bad device or tuning. */
LCC_API lcc_status lcc_get_tuning(int32_t device, lcc_tuning *out);
LCC_API lcc_status lcc_set_tuning(int32_t device, const lcc_tuning *t);

/*
 * lcc_autotune -- choose the tuning of g's device.  With cache_path naming a
 * text file that has a line for this device (its name and SM count), that
 * line is applied.  Otherwise every warp_max is timed on three best-move
 * rounds of g from singletons (lambda and mode as in lcc_best_moves, V' of
 * moved vertices' neighbours), the fastest is applied and, with cache_path,
 * appended to the file as "<device name>|<SMs> <warp_max>".  The chosen
 * tuning goes to `out` (nullable).  LCC_ERR_INVALID for bad arguments or a
 * malformed line for this device; file errors are LCC_ERR_INVALID too.
 */
LCC_API lcc_status lcc_autotune(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q,
                                int32_t mode, const char *cache_path, lcc_tuning *out);

typedef struct lcc_server lcc_server;

typedef struct lcc_server_cfg {
  int64_t hbm_budget_bytes; /* admit while resident bytes stay under this */
  int32_t max_slots;        /* max graphs resident at once */
  int32_t reserved;
  lcc_schedule sched;       /* schedule of every job */
} lcc_server_cfg;

typedef struct lcc_job {
  const int64_t *offsets;   /* host CSR, copied at submit */
  const int32_t *nbrs;
  const int32_t *weights;   /* nullable */
  int64_t n, nnz;
  int64_t lambda_p, lambda_q;
  int32_t mode;             /* LCC_NODEW_UNIT or LCC_NODEW_DEGREE */
  /* Fault injection, for testing a serving deployment's error handling
     without a GPU fault: 0 (the normal value) does nothing; t > 0 makes the
     job fail with LCC_ERR_CUDA ("injected fault") at the start of its t-th
     engine tick, through the same path as a real error raised in a tick.
     Such an error belongs to one job, so only that job fails; the jobs that
     run with it continue and return their normal results. */
  int32_t inject_fault_tick;
} lcc_job;

/*
 * lcc_server_create -- start a serving engine on the current device with its
 * own worker thread and stream.  Jobs submitted while others run are admitted
 * between rounds as slots and HBM budget free up, and join the next round.
 */
LCC_API lcc_status lcc_server_create(const lcc_server_cfg *cfg, lcc_server **out);

/* lcc_submit -- copy a job's CSR to pinned host memory and queue it.
 * Returns LCC_ERR_INVALID for a malformed job, LCC_ERR_OOM if the job alone
 * exceeds the budget.  *ticket identifies it. */
LCC_API lcc_status lcc_submit(lcc_server *s, const lcc_job *job, uint64_t *ticket);

/*
 * lcc_poll -- LCC_ERR_BUSY while the job runs; then its status.  On LCC_OK
 * labels_out [n] (host, nullable) and obj_out (nullable) receive the result
 * and the ticket is released.  latency_ms_out (nullable) gets submit-to-done
 * time.
 */
LCC_API lcc_status lcc_poll(lcc_server *s, uint64_t ticket, int32_t *labels_out,
                    double *obj_out, double *latency_ms_out);

/* lcc_cancel -- drop a queued or running job; its poll returns
 * LCC_ERR_CANCELLED. */
LCC_API lcc_status lcc_cancel(lcc_server *s, uint64_t ticket);

/* lcc_server_wait_idle -- block until every submitted job has finished or
 * timeout_ms passes (LCC_ERR_TIMEOUT). */
LCC_API lcc_status lcc_server_wait_idle(lcc_server *s, int64_t timeout_ms);

/* Counters of the serving engine: [0] jobs done, [1] ticks, [2] peak resident
 * bytes, [3] peak concurrent jobs, [4] rejected jobs. */
LCC_API lcc_status lcc_server_counters(lcc_server *s, int64_t *out5);

/* Stops the worker (running jobs are cancelled) and frees everything. */
LCC_API lcc_status lcc_server_destroy(lcc_server *s);

LCC_API const char *lcc_status_str(lcc_status s);
LCC_API const char *lcc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LCC_H */
