// Internal declarations shared by the CUDA translation units of liblcc.
//
// Data layout in HBM (one "job" = one graph being clustered; a launch covers
// the current level of every job in a table):
//   CSR level : off int64[n+1] (absolute indices into nbr/w), nbr int32[nnz],
//               w int32[nnz] (input level, optional) or int64[nnz] (coarse
//               levels, merged weights), k int64[n] node weights;
//   state     : L int32[n] labels, K int64[n] cluster weights (indexed by
//               cluster id), D int32[n] desired clusters, fr uint8[n] next
//               frontier flags, cl uint8[n] "a vertex left this cluster";
//   work lists: uint64 items (job << 32 | vertex), one segment per degree
//               bucket.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lcc {

typedef __int128 i128;
typedef unsigned __int128 u128;

enum WType : int32_t { W_NONE = 0, W_I32 = 1, W_I64 = 2 };

// Job flags for a round.
enum : int32_t {
  JF_ALL = 1,       // evaluate every vertex this round (V' = V)
  JF_MARK_NBR = 2,  // next V' = neighbours of moved vertices
  JF_MARK_CL = 4,   // next V' = neighbours of clusters that lost a vertex
  JF_EVAL_ONLY = 8, // compute D only (no apply)
  // V' = neighbours of the previous round's moved vertices, tested by the
  // best-move kernels themselves: a vertex is evaluated in full and keeps its
  // label unless some entry of its row has LK_MOVED set.  On a symmetric
  // graph this is the same set as marking the neighbours of every mover.
  JF_PULL = 16
};
// Bit 31 of the label half of lk[u] (labels are non-negative int32): u moved
// in the previous round.  Set only for JF_PULL jobs.
constexpr uint32_t LK_MOVED = 0x80000000u;

// Degree buckets of the best-move kernels.  The tables hold at least two
// slots per entry of the row (power-of-two sizes) up to B_T4K, and 1.6 in
// the larger-row kernels (any size).
enum Bucket : int {
  B_G4 = 0,     // deg <= 4: 4 lanes per vertex, register aggregation
  B_G8 = 1,     // deg <= 8
  B_G16 = 2,    // deg <= 16
  B_G32 = 3,    // deg <= 32: one warp
  B_W64 = 4,    // deg <= 64: one warp, shared-memory table, 2 entries per lane
  B_W128 = 5,   // deg <= 128: 4 entries per lane
  B_WARP = 6,   // deg <= 256: one 128-thread block, 2 entries per thread
  B_BLK = 7,    // deg <= 1024: one 256-thread block, shared-memory table
  B_T2K = 8,    // deg <= 2048: one 512-thread block
  B_T4K = 9,    // deg <= 4096: one 1024-thread block
  B_T8K = 10,   // deg <= 8192: one 1024-thread block, two chunks per thread
  B_T16K = 11,  // deg <= 16384: cluster of 2 blocks, table in distributed shared memory
  B_T32K = 12,  // deg <= 32768: cluster of 4
  B_T64K = 13,  // deg <= 65536: cluster of 8
  B_T128K = 14, // deg <= 131072: cluster of 16 (a non-portable cluster size)
  B_HUB = 15,   // larger: global-memory table, many blocks per vertex
  NB = 16
};
constexpr int T_WARP = 256;
constexpr int T_BLK = 1024;
constexpr int TP_BLK = 2048;     // table slots of the B_BLK kernel (power of two, 2 per entry)
constexpr int TP_2K = 4096;      // of the B_T2K kernel (power of two, 2 per entry)
constexpr int TP_4K = 8192;      // of the B_T4K kernel (power of two, 2 per entry)
constexpr int TP_8K = 13312;     // per block of the larger-row kernels (>= 1.6 * 8192)
constexpr int WARP_CAP = 1024;   // of the B_WARP kernel (power of two, 4 per entry)
constexpr int HUB_CHUNK = 2048;  // edges per insertion unit
constexpr int HUB_SCHUNK = 4096; // table slots per scoring unit

// Rows of more than warp_max entries (a tuning: 32, 64, 128 or 256) and up
// to T_BLK go to the block kernel instead of the warp kernels.
__host__ __device__ inline int bucket_of(int64_t deg, int warp_max = T_WARP) {
  if (deg <= 4) return B_G4;
  if (deg <= 8) return B_G8;
  if (deg <= 16) return B_G16;
  if (deg <= 32) return B_G32;
  if (deg <= warp_max) {
    if (deg <= 64) return B_W64;
    if (deg <= 128) return B_W128;
    return B_WARP;
  }
  if (deg <= T_BLK) return B_BLK;
  if (deg <= 2048) return B_T2K;
  if (deg <= 4096) return B_T4K;
  if (deg <= 8192) return B_T8K;
  if (deg <= 16384) return B_T16K;
  if (deg <= 32768) return B_T32K;
  if (deg <= 65536) return B_T64K;
  if (deg <= 131072) return B_T128K;
  return B_HUB;
}

// A hash-table slot is a 64-bit word (cluster id in the low half, the
// cluster's weight K in the high half, or KNONE when the level's weights do
// not fit 32 bits) plus a 64-bit sum of edge weights.
constexpr uint32_t KNONE = 0xFFFFFFFFu;
constexpr unsigned long long SLOT_EMPTY = ~0ull;

__host__ __device__ inline int64_t next_pow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Global-table capacity of a hub row: a power of two >= 2 * deg.
__host__ __device__ inline int64_t hub_cap(int64_t deg) { return next_pow2(2 * deg); }

// Current level of one job, as seen by the round kernels.
struct JobDev {
  const int64_t *off;
  const int32_t *nbr;
  const void *w;
  const int64_t *k;
  int32_t *L;
  int64_t *K;
  int32_t *D;
  uint8_t *fr;
  uint8_t *cl;
  // per round: lk[pos[u]] = K[L[u]] << 32 | L[u]; null when K can reach 2^32 - 1
  unsigned long long *lk;
  // gather layout (null: identity): pos[u] is where u's packed word is kept,
  // and gnbr[e] = pos[nbr[e]] is what the best-move kernels gather through
  const int32_t *pos;
  const int32_t *gnbr;  // = nbr without a layout
  // this round's label words already gathered per entry (null: gather through
  // gnbr): gw[e - off[0]] = lk[gnbr[e]], written by k_gather_words in rounds
  // that read every row
  unsigned long long *gw;
  int64_t n;
  int64_t p, q;
  // the next round tests V' in the kernels (JF_PULL) instead of marking it
  // when the movers' rows hold at least this many entries (INT64_MAX: never)
  int64_t pull_min;
  int32_t wtype;
  int32_t flags;
  int32_t warp_max;  // degree routing of the level (see bucket_of)
  int32_t pad;
};

// Device counters of a round (int64 each).
enum Ctr : int {
  C_EDGES = 0,    // sum of deg over evaluated vertices
  C_VERTS = 1,    // evaluated vertices
  C_CANDS = 2,    // distinct candidate clusters scored
  C_MOVES = 3,    // vertices moved
  C_ERR = 4,      // error bits (see Err)
  C_MOVED_N = 5,  // entries in the moved list
  C_HUBS = 6,     // hubs handled this round
  C_WB = 7,       // sum of deg * (bytes per stored weight) over evaluated vertices
  C_BE = 8,       // [NB] entries per degree bucket
  C_BV = 8 + NB,  // [NB] vertices per degree bucket
  C_WORK = 8 + 2 * NB,  // work-unit counter of the fused small-row kernel
  NCTR = 9 + 2 * NB
};
enum Err : int64_t {
  E_BUCKET_OVERFLOW = 1,
  E_HUB_OVERFLOW = 2,
  E_MOVED_OVERFLOW = 4,
  E_PAIR_OVERFLOW = 8,
  E_BAD_LABEL = 16
};

struct Buckets {
  uint64_t *items;
  int64_t seg_start[NB];
  int64_t seg_cap[NB];
  int64_t *cnt;       // [NB] device counters
};

struct HubBufs {
  unsigned long long *keys;  // one window of tables: [window + largest table] slots
  int64_t *vals;
  int64_t window;     // hubs whose table starts in [lo, lo + window) share a pass
  int64_t *tbl_off;   // [max_hubs + 1]
  int64_t *unit_off;  // [max_hubs + 1]
  int64_t *sunit_off; // [max_hubs + 1]
  i128 *part_score;   // [max_sunits]
  int32_t *part_cid;  // [max_sunits]
  int64_t *stay;      // [max_hubs]
  int32_t *iso_seen;  // [max_hubs] bit 0: cluster id v occurs; bit 1: a neighbour moved
  int64_t max_hubs;
  int64_t max_sunits;
  // rows to process: the B_HUB segment, or (when set) list[0 .. *list_cnt)
  const uint64_t *list;
  const int64_t *list_cnt;
};

// One part of the partitioned path: its run of entries and its row.
struct PartDesc {
  int64_t st;   // first entry in pword / pw
  int32_t cnt;  // entries
  int32_t h;    // row
};

// The partitioned path's arrays (see PART_*): per row h < H of the long-row
// buckets, its item and prefix offsets of its parts, chunks and count cells;
// per part its best candidate; per row the stay weight and flags.
struct PartBufs {
  uint64_t *row;          // [max_rows]
  int64_t *part_off;      // [max_rows + 1]
  int64_t *chunk_off;     // [max_rows + 1]
  int64_t *cell_off;      // [max_rows + 1]
  int64_t *cells;         // [max_cells + 1] counts per (row, part, chunk), scanned in place
  unsigned long long *pword;  // [max_entries] entries grouped by (row, part): packed word
  int64_t *pw;            // [max_entries] and weight
  i128 *part_score;       // [max_parts]
  int32_t *part_cid;      // [max_parts]
  int64_t *stay;          // [max_rows]
  int32_t *flag;          // [max_rows] bit 0: cluster id v occurs; 1: a neighbour moved; 2: overflow
  uint64_t *fallback;     // [max_rows] rows whose part overflowed its table
  int64_t *nfallback;     // [1]
  int64_t *nrows;         // [1] rows this round (written by k_part_prep)
  int64_t *scan_tmp;      // [scan_tmp_elems(max(max_cells, max_rows) + 1)]
  int32_t *chunk_row;     // [max_chunks] row of each chunk
  PartDesc *desc;         // [max_parts]
  int64_t max_rows, max_parts, max_chunks, max_cells, max_entries;
  int32_t table_slots;    // slots of a part's table at most (a multiple of 32, <= PART_TP)
  int32_t seg0;           // first bucket taken by the path (PB0 .. B_HUB)
};

// Contraction view of one job's level.
struct CJob {
  const int64_t *off;
  const int32_t *nbr;
  const void *w;
  const int32_t *L;
  const int64_t *K;
  int32_t *map;  // out: coarse vertex of each vertex (local id)
  const int32_t *pos;   // gather layout of the level (null: identity)
  const int32_t *gnbr;  // neighbour positions (= nbr without a layout)
  int64_t n;
  int32_t wtype;
  int32_t pad;
};

// Level view for flatten / final / statistics kernels.
struct LJob {
  const int64_t *off;
  const int32_t *nbr;
  const void *w;
  const int64_t *k;
  int32_t *L;
  int64_t *K;
  int32_t *D;
  const int32_t *map;     // flatten: coarse vertex of each vertex
  const int32_t *Lcoarse; // flatten: labels of the coarse level
  int32_t *pos;           // gather layout (see JobDev)
  int32_t *gnbr;
  int64_t n;
  int32_t wtype;
  int32_t warp_max;       // degree routing of the level (see bucket_of)
};

// Degree classes of the gather layout: 0 for an isolated vertex, else
// 1 + floor(log2 deg); positions are handed out from the highest class down.
constexpr int LAYOUT_CLASSES = 34;
// Levels whose packed words take more than this many bytes get a layout.
constexpr int64_t LAYOUT_MIN_BYTES = (int64_t)64 << 20;

// Sizes of the partitioned best-move path over the rows of one degree
// bucket (B_T2K and above; see PART_*).
struct PartStat {
  int64_t rows, nnz;
  int64_t parts, chunks, cells;  // sums of P, of the rows' chunks, and of P * chunks
  int64_t cap, sunits, maxcap;   // the rows' global tables (the fallback)
};
constexpr int PB0 = B_T2K;           // first bucket the partitioned path can take
constexpr int NPB = B_HUB - PB0 + 1;

// Per-job results of the level statistics kernel.
struct LevelInfo {
  int64_t bcnt[NB];     // vertices per degree bucket
  int64_t hub_cap;      // sum of hub table capacities
  int64_t hub_units;    // insertion units over hubs
  int64_t hub_sunits;   // scoring units over hubs
  int64_t rmax;         // max over rows of sum |w|
  int64_t kmax;         // max node weight
  int64_t ksum;         // sum of node weights
  int64_t wabs;         // sum of |w| over entries
  int64_t pad;          // vertices with a negative node weight
  int64_t hub_maxcap;   // largest hub table
  int64_t nnz;          // entries (sum of deg)
  int64_t ksat;         // nonzero: the sum of node weights reached 2^62 (ksum is then not exact)
  // rows of the buckets B_T2K .. B_HUB, per bucket (the partitioned path)
  PartStat pst[NPB];
};

// Partitioned best-move path for the rows of the buckets from a tuned one
// (lcc_tuning.part_min) up: the entries of a row are split by a hash of
// their cluster into P = ceil(deg / PART_ENT) parts (at most PART_MAXP),
// counted and scattered in chunks of PART_CH entries, and each part is merged
// by one PART_T-thread block in a table of at most PART_TP slots.
constexpr int PART_ENT = 1024;
constexpr int PART_MAXP = 4096;
constexpr int PART_CH = 4096;
constexpr int PART_T = 256;
constexpr int PART_TP = 3328;  // table slots of a part's block (52 KB, 3.25 * PART_ENT)
// every row the path can take (more than T_BLK entries) has several parts
static_assert(PART_ENT <= T_BLK, "a row of the partitioned path must have more than one part");
__host__ __device__ inline int64_t part_count_of(int64_t deg) {
  const int64_t p = (deg + PART_ENT - 1) / PART_ENT;
  return p < PART_MAXP ? p : PART_MAXP;
}
// Chunks of the count and scatter passes.
__host__ __device__ inline int64_t part_chunks_of(int64_t deg) {
  return (deg + PART_CH - 1) / PART_CH;
}

// Per-job accumulators of the objective kernels.
struct ObjAcc {
  unsigned long long s_in;     // sum of w over same-cluster entries (two's complement)
  unsigned long long ksq_lo, ksq_hi;   // sum_C K_C^2 (128-bit)
  unsigned long long kself_lo, kself_hi; // sum_v k_v^2 (128-bit)
  unsigned long long nclus;    // vertices that are their cluster's label (canonical)
  unsigned long long pad[2];
};

__device__ __forceinline__ int64_t load_w(const void *w, int32_t wtype, int64_t e) {
  if (wtype == W_I32) return (int64_t)__ldg(((const int32_t *)w) + e);
  if (wtype == W_I64) return __ldg(((const int64_t *)w) + e);
  return 1;
}

// Largest j with vstart[j] <= i (vstart ascending, vstart[0] = 0).
__device__ __forceinline__ int find_job(const int64_t *__restrict__ vstart, int njobs, int64_t i) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(vstart + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void atomic_add_i64(int64_t *a, int64_t v) {
  atomicAdd((unsigned long long *)a, (unsigned long long)v);
}

// 128-bit accumulation from two 64-bit atomics: the carry of each low-word
// addition is decided by the value that addition saw, so the total is exact.
__device__ __forceinline__ void atomic_add_u128(unsigned long long *lo, unsigned long long *hi, u128 v) {
  unsigned long long vl = (unsigned long long)v;
  unsigned long long vh = (unsigned long long)(v >> 64);
  unsigned long long old = atomicAdd(lo, vl);
  unsigned long long carry = (old + vl < old) ? 1ull : 0ull;
  if (vh + carry) atomicAdd(hi, vh + carry);
}

template <typename S> struct ScoreOps;
template <> struct ScoreOps<int64_t> {
  __device__ static __forceinline__ int64_t lowest() { return INT64_MIN; }
  __device__ static __forceinline__ int64_t shfl_xor(int64_t x, int o, int width) {
    return __shfl_xor_sync(0xffffffffu, (long long)x, o, width);
  }
  __device__ static __forceinline__ int64_t shfl(int64_t x, int src, int width) {
    return __shfl_sync(0xffffffffu, (long long)x, src, width);
  }
};
template <> struct ScoreOps<i128> {
  __device__ static __forceinline__ i128 lowest() { return (i128)((u128)1 << 127); }
  __device__ static __forceinline__ i128 shfl_xor(i128 x, int o, int width) {
    long long lo = (long long)(uint64_t)x, hi = (long long)(x >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, o, width);
    hi = __shfl_xor_sync(0xffffffffu, hi, o, width);
    return ((i128)hi << 64) | (i128)(uint64_t)lo;
  }
  __device__ static __forceinline__ i128 shfl(i128 x, int src, int width) {
    long long lo = (long long)(uint64_t)x, hi = (long long)(x >> 64);
    lo = __shfl_sync(0xffffffffu, lo, src, width);
    hi = __shfl_sync(0xffffffffu, hi, src, width);
    return ((i128)hi << 64) | (i128)(uint64_t)lo;
  }
};

// (score, cluster) pair order: higher score first, then smaller cluster id.
template <typename S>
__device__ __forceinline__ bool better(S s1, int32_t c1, S s2, int32_t c2) {
  return s1 > s2 || (s1 == s2 && c1 < c2);
}

// ---- host-side launch helpers (defined in the .cu files) ----
struct Dev {
  int sms;
  int dev;
};

// Round kernels (k_round.cu).
// gw[f - estart[j]] of job j = its label word of entry off[0] + (f - estart[j])
// for f in [estart[j], estart[j+1]) (estart[njobs] = etot; jobs without a gw
// buffer have no entries there).
void launch_gather_words(const JobDev *jobs, const int64_t *estart, int njobs, int64_t etot,
                         cudaStream_t st, const Dev &d);
void launch_frontier(const JobDev *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                     const Buckets &b, int64_t *ctr, cudaStream_t st, const Dev &d);
// ev (nullable, NB events): ev[b] is recorded after degree bucket b's kernels.
// fuse_small: the <= 4 .. <= 32 buckets in one resident launch (k_bm_small);
// prefetch: the one-chunk table kernels pipeline their vertices; pb (nullable):
// rows of more than PART_MIN entries take the partitioned path, and h (with
// hub_passes) then serves its fallback rows.
void launch_bestmove(bool wide, const JobDev *jobs, const Buckets &b, const HubBufs &h,
                     int64_t hub_passes, int64_t *ctr, cudaStream_t st, const Dev &d,
                     int *launches, cudaEvent_t *ev, bool fuse_small, bool prefetch,
                     const PartBufs *pb);
// jmoves[2j] = moves of job j, jmoves[2j + 1] = entries of its movers' rows.
void launch_apply(const JobDev *jobs, const Buckets &b, int64_t *jmoves, uint64_t *moved,
                  int64_t moved_cap, int64_t *ctr, cudaStream_t st, const Dev &d);
void launch_mark(const JobDev *jobs, const uint64_t *moved, int64_t *ctr, const int64_t *jmoves,
                 bool any_cl, const int64_t *vstart, int njobs, int64_t vtot, cudaStream_t st,
                 const Dev &d, int *launches);

// Level kernels (k_level.cu).
void launch_level_stats(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                        LevelInfo *info, cudaStream_t st, const Dev &d);
// Gather layout of a level per job (k_level.cu): cnt is [njobs *
// LAYOUT_CLASSES] zeroed int64 scratch; estart[j] = first flat entry of job j
// (estart[njobs] = all entries).
void launch_layout(const LJob *jobs, const int64_t *vstart, const int64_t *estart, int njobs,
                   int64_t vtot, int64_t etot, int64_t *cnt, cudaStream_t st, const Dev &d);
void launch_init_level(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                       cudaStream_t st, const Dev &d);
void launch_degree_k(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                     int64_t *k_out_flat_unused, cudaStream_t st, const Dev &d);
void launch_fill_k_unit(int64_t *k, int64_t n, cudaStream_t st, const Dev &d);
void launch_recompute_K(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                        cudaStream_t st, const Dev &d);
void launch_flatten(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                    cudaStream_t st, const Dev &d);
void launch_canonical(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                      cudaStream_t st, const Dev &d);
void launch_objective(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                      ObjAcc *acc, cudaStream_t st, const Dev &d);
void launch_validate(const int64_t *off, int64_t n, int64_t nnz, unsigned long long *out8,
                     cudaStream_t st, const Dev &d);

// Symmetry-breaking coin of one job in one round (LCC_SCHED_COIN): the
// draws of vertex v use key = key_hi + v.
struct CoinJob {
  uint64_t seed;
  uint64_t key_hi;  // round 2^32 + depth 2^48 + phase 2^56
  int32_t on;
  int32_t pad;
};
// After the best-move kernels: every evaluated vertex of a coin job whose
// desired cluster differs from its own and whose coin forbids the move keeps
// its label (D[v] = L[v]) and is marked into the next V'; held[j] counts them.
void launch_coin(const JobDev *jobs, const CoinJob *coins, const Buckets &b, int64_t *held,
                 cudaStream_t st, const Dev &d);
void launch_validate_rows(const int64_t *off, const int32_t *nbr, const int32_t *w, int64_t n,
                          unsigned long long *out8, cudaStream_t st, const Dev &d);

// Contraction kernels (k_contract.cu).
void launch_occ(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vtot, int64_t *occ,
                int32_t *err, cudaStream_t st, const Dev &d);
// gmap[i] = global coarse id of flat vertex i; gmapp holds the same ids at
// the flat positions of the gather layout (gmapp[vstart_j + pos[v]]).
void launch_relabel(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                    const int64_t *rank, int32_t *gmap, int32_t *gmapp, cudaStream_t st,
                    const Dev &d);
void launch_knew(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                 const int64_t *rank, int64_t *knew, cudaStream_t st, const Dev &d);
void launch_job_counts(const int64_t *vstart, int njobs, const int64_t *rank, int64_t *out,
                       cudaStream_t st);
// Exclusive scan of int64 in place over [0, n]; a[n] receives the total.
// tmp must hold scan_tmp_elems(n) int64.
int64_t scan_tmp_elems(int64_t n);
void scan_exclusive_i64(int64_t *a, int64_t n, int64_t *tmp, cudaStream_t st, const Dev &d);

// Compress by rows (k_rows.cu).  Classes of coarse rows by the number of
// entries of their members.
enum RowClass : int {
  RC_G4 = 0, RC_G8, RC_G16, RC_G32, RC_WARP, RC_BLOCK, RC_BLOCK8K, RC_BIG, RC_N
};
constexpr int RC_WARP_MAX = 256;     // warp + shared table of 2 slots per entry
constexpr int RC_BLOCK_MAX = 4096;   // 512-thread block + shared table of 2 slots per entry
constexpr int RC_BLOCK8K_MAX = 8192; // 1024-thread block + 192 KB shared table
constexpr int RC_CHUNK = 4096;      // entries per insertion unit of a big row
constexpr int RC_SCHUNK = 4096;     // table slots per compaction unit of a big row

struct RowSpace {
  const CJob *jobs;
  const int64_t *vstart;    // [njobs + 1] first flat vertex of each job
  const int32_t *gmap;      // [vt] global coarse id of each flat vertex
  const int32_t *gmapp;     // global coarse id at the flat gather positions
  const int64_t *rank;      // rank[vstart_j] = first global coarse id of job j
  const int64_t *boff;      // [ntot + 1] region of coarse row C: [boff[C], boff[C+1])
  const int64_t *rpos;      // [vt] place of each fine vertex's entries in its region
  int32_t *tnbr;            // [entries] job-local coarse id of the far end, -1: a hole
  int64_t *tw;              // [entries] weight
  int64_t *ucnt;            // [ntot + 1] unique entries per row (zeroed)
  unsigned long long *intra;  // entries inside a cluster (counted)
  int32_t njobs;
  int32_t pad;
};

// Global tables of the rows of class RC_BIG (prefix arrays over those rows).
struct BigRows {
  int32_t *keys;            // window of tables, -1 = empty
  unsigned long long *vals;
  const int64_t *tbl_off;   // [H + 1] next_pow2(2 * bound) slots per row
  const int64_t *unit_off;  // [H + 1] ceil(bound / RC_CHUNK)
  const int64_t *sunit_off; // [H + 1] ceil(slots / RC_SCHUNK)
  int64_t H;
};

// rbound[gmap[i]] += deg(i) for every flat vertex (rbound zeroed); rpos[i]
// receives the value before the addition.
void launch_rbound(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vt,
                   const int32_t *gmap, int64_t *rbound, int64_t *rpos, cudaStream_t st,
                   const Dev &d);
// Writes every entry into its coarse row's region (intra-cluster ones as holes).
void launch_emit_rows(const RowSpace &R, int64_t vt, cudaStream_t st, const Dev &d);
void launch_rows_classify(const RowSpace &R, int64_t ntot, bool fill, unsigned long long *cnt,
                          const int64_t *seg, int32_t *items, cudaStream_t st, const Dev &d);
// seg and cnt: host arrays [RC_N]; items of class c at items + seg[c].
void launch_rows_small(const RowSpace &R, const int32_t *items, const int64_t *seg,
                       const int64_t *cnt, cudaStream_t st, const Dev &d, int *launches);
void launch_big_bounds(const RowSpace &R, const int32_t *items, int64_t H, int64_t *bound,
                       cudaStream_t st, const Dev &d);
// Rows [h0, h1) of the big class, whose tables start at or after slot lo
// (B.keys / B.vals hold that window, cleared).
void launch_big_window(const RowSpace &R, const int32_t *items, const BigRows &B, int64_t h0,
                       int64_t h1, int64_t lo, int64_t units, int64_t sunits, cudaStream_t st,
                       const Dev &d, int *launches);
void launch_rows_copy(const RowSpace &R, int64_t ntot, const int64_t *offg, int32_t *nbr_out,
                      int64_t *w_out, cudaStream_t st, const Dev &d);
// Sorting the rows of a CSR (offsets from 0) by neighbour: keys row << 32 |
// neighbour, then back.
void launch_row_keys(const int64_t *off, int64_t n, const int32_t *nbr, uint64_t *keys,
                     cudaStream_t st, const Dev &d);
void launch_row_unkey(const uint64_t *keys, int64_t nnz, int32_t *nbr, cudaStream_t st,
                      const Dev &d);

// LSD radix sort of (key, val) pairs on the given 8-bit digit positions.
int64_t radix_tmp_elems(int64_t n);
void radix_sort_pairs(uint64_t *keys, int64_t *vals, uint64_t *keys_alt, int64_t *vals_alt,
                      int64_t n, const int *shifts, int npasses, int64_t *tmp,
                      cudaStream_t st, const Dev &d, bool *result_in_alt, int *launches);
}  // namespace lcc
