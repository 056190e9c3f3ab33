/*
 * Multi-core CPU twin of the LambdaCC parallel Louvain method
 * (Shi, Dhulipala, Eisenstat, Lacki, Mirrokni, "Scalable Community Detection
 * via Parallel Correlation Clustering", arXiv 2108.01731), in OpenMP.
 *
 * MEASURED CPU BASELINE, not part of the library.  It runs the same
 * deterministic schedule as the GPU library on all host cores: Algorithm 1
 * with the synchronous best moves of Sec. 3.2.1, the vertex subsets V' of
 * Sec. 3.2.2, Compress and Flatten of Sec. 3.1 and Appendix B, and the
 * refinement of Sec. 3.2.3.  The benchmark times it beside the GPU; the tests
 * check that it returns the oracle's labels, objective and counters bit for
 * bit at every thread count.  The GPU library never calls it, and it shares
 * no code with the library or with the oracle.
 *
 * Exactness.  A move's gain (Appendix A) is compared after multiplying by q,
 * in __int128: a candidate cluster C scores q w(v,C) - p k_v K_C, staying
 * scores q w(v,L[v] minus v) - p k_v (K_L[v] - k_v).  Per-cluster edge sums
 * and cluster weights are int64: every partial sum is bounded by the total
 * absolute edge weight, which the entry points check.  Integer sums do not
 * depend on the order in which threads add them, so the result does not
 * depend on the thread count.
 *
 * Readings where the paper is silent (shared with the library and the
 * oracle): ties between candidates go to the smallest cluster id and a vertex
 * moves only when strictly better than staying; a vertex not in cluster v may
 * isolate itself into the empty cluster id v (score 0) when K[v] == 0 and no
 * neighbour is in cluster v; Compress drops intra-cluster edges and keeps
 * merged edges whose weights sum to 0; coarse ids are the occupied cluster
 * ids ranked in increasing order; a level whose compression does not shrink
 * the graph ends the recursion; final labels are the smallest vertex id of
 * each cluster.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

enum { TW_OK = 0, TW_ERR_INVALID = 1, TW_ERR_OOM = 4, TW_ERR_OVERFLOW = 5 };
enum { TW_VSET_ALL = 0, TW_VSET_NBR_VERTICES = 1, TW_VSET_NBR_CLUSTERS = 2 };
enum { TW_NODEW_UNIT = 0, TW_NODEW_DEGREE = 1, TW_NODEW_CUSTOM = 2 };

#define RELAXED __ATOMIC_RELAXED

/* One level: CSR with int32 weights (input level), int64 weights (coarse
 * levels) or none (all 1), and int64 node weights. */
typedef struct {
  int64_t n;
  const int64_t *off;
  const int32_t *nbr;
  const int32_t *w32;
  const int64_t *w64;
  const int64_t *k;
} tw_level;

static inline int64_t weight(const tw_level *g, int64_t e) {
  if (g->w64) return g->w64[e];
  return g->w32 ? (int64_t)g->w32[e] : 1;
}

/* ------------------------------------------------------------------------ */
/* Per-thread open-addressing table: cluster id -> int64 sum                 */
/* ------------------------------------------------------------------------ */

/* Every key slot is -1 between uses; `used` lists the slots a use filled so
 * that only those are cleared. */
typedef struct {
  int32_t *key;
  int64_t *sum;
  uint32_t *used;
  int64_t cap;
} tw_table;

static int64_t slots_for(int64_t entries) {
  int64_t c = 16;
  while (c < 2 * entries) c <<= 1;
  return c;
}

static int table_fit(tw_table *t, int64_t entries) {
  const int64_t cap = slots_for(entries);
  if (cap <= t->cap) return TW_OK;
  free(t->key); free(t->sum); free(t->used);
  t->key = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
  t->sum = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
  t->used = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
  if (!t->key || !t->sum || !t->used) {
    free(t->key); free(t->sum); free(t->used);
    t->key = NULL; t->sum = NULL; t->used = NULL; t->cap = 0;
    return TW_ERR_OOM;
  }
  memset(t->key, 0xff, (size_t)cap * sizeof(int32_t));
  t->cap = cap;
  return TW_OK;
}

static void table_free(tw_table *t) {
  free(t->key); free(t->sum); free(t->used);
  memset(t, 0, sizeof(*t));
}

/* 32-bit integer finaliser ("lowbias32", C. Wellons' hash-prospector). */
static inline uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du;
  x ^= x >> 15; x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

/* Adds s to the entry of cluster c, creating it on first sight. */
static inline void table_add(tw_table *t, uint32_t mask, int64_t *nused,
                             int32_t c, int64_t s) {
  uint32_t h = mix32((uint32_t)c) & mask;
  for (;;) {
    const int32_t kk = t->key[h];
    if (kk == c) { t->sum[h] += s; return; }
    if (kk < 0) {
      t->key[h] = c; t->sum[h] = s;
      t->used[(*nused)++] = h;
      return;
    }
    h = (h + 1) & mask;
  }
}

/* ------------------------------------------------------------------------ */
/* Symmetry-breaking coin                                                    */
/* ------------------------------------------------------------------------ */

/* With the coin on, a vertex whose best move differs from its cluster moves
 * in round t of a Best-Moves call only if the top bit of output key + 1 of
 * the SplitMix64 stream seeded with `seed` is 1 (Vigna's generator after
 * Steele, Lea and Flood 2014: output i is the finaliser applied to
 * seed + i * 0x9e3779b97f4a7c15), key = v + t 2^32 + depth 2^48 +
 * phase 2^56, phase 1 for the refinement call after Flatten.  A vertex held
 * back keeps its label and is evaluated again in the next round. */
typedef struct {
  int on;
  uint64_t seed;
  int phase, depth;
} tw_coin;

static inline int coin_allows(const tw_coin *c, int t, int64_t v) {
  uint64_t z = c->seed + ((uint64_t)v + ((uint64_t)(t & 0xffff) << 32) +
                          ((uint64_t)(c->depth & 0xff) << 48) +
                          ((uint64_t)(c->phase & 1) << 56) + 1) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (int)(z >> 63);
}

/* ------------------------------------------------------------------------ */
/* Best move of one vertex (Appendix A gain)                                 */
/* ------------------------------------------------------------------------ */

/* The cluster v wants under the snapshot (L, K).  The table must fit the
 * row (table_fit with the degree). */
static int32_t best_of(const tw_level *g, int64_t v, int64_t p, int64_t q,
                       const int32_t *L, const int64_t *K, tw_table *t) {
  const int64_t rb = g->off[v], re = g->off[v + 1];
  const uint32_t mask = (uint32_t)(slots_for(re - rb) - 1);
  int64_t nu = 0;
  for (int64_t e = rb; e < re; ++e) {
    if (e + 16 < re) __builtin_prefetch(&L[g->nbr[e + 16]]);  /* label gathers miss */
    table_add(t, mask, &nu, L[g->nbr[e]], weight(g, e));
  }
  const int32_t cv = L[v];
  const i128 kv = g->k[v];
  i128 w_stay = 0, best = 0;
  int have = 0, v_in_nbrs = 0;
  int32_t best_c = cv;
  for (int64_t i = 0; i < nu; ++i) {
    const uint32_t s = t->used[i];
    const int32_t c = t->key[s];
    const int64_t sum = t->sum[s];
    t->key[s] = -1;
    if ((int64_t)c == v) v_in_nbrs = 1;
    if (c == cv) { w_stay = sum; continue; }
    const i128 score = (i128)q * sum - (i128)p * kv * (i128)K[c];
    if (!have || score > best || (score == best && c < best_c)) {
      have = 1; best = score; best_c = c;
    }
  }
  if ((int64_t)cv != v && K[v] == 0 && !v_in_nbrs) {
    const int32_t c = (int32_t)v;  /* isolation: empty cluster id v, score 0 */
    if (!have || 0 > best || (0 == best && c < best_c)) {
      have = 1; best = 0; best_c = c;
    }
  }
  const i128 stay = (i128)q * w_stay - (i128)p * kv * ((i128)K[cv] - kv);
  return (have && best > stay) ? best_c : cv;
}

/* ------------------------------------------------------------------------ */
/* Shared helpers                                                            */
/* ------------------------------------------------------------------------ */

/* Optional per-round record (TW_TRACE_COLS int64 per round): level depth,
 * phase (0 coarsening, 1 refinement), round within the call, |V'|, entries
 * scanned, vertices moved, vertices held back by the coin. */
enum { TW_TRACE_COLS = 7 };

typedef struct {
  int64_t p, q;
  int num_iter, max_levels, refine, vset;
  int64_t levels, rounds, scanned;
  tw_table *tabs; /* one per thread */
  int ntabs;
  int coin;
  uint64_t seed;
  int64_t *trace;  /* [trace_cap][TW_TRACE_COLS] or NULL */
  int64_t trace_cap, trace_len;
} tw_run;

static int run_tables(tw_run *r) {
  r->ntabs = omp_get_max_threads();
  r->tabs = (tw_table *)calloc((size_t)r->ntabs, sizeof(tw_table));
  return r->tabs ? TW_OK : TW_ERR_OOM;
}

static void run_free(tw_run *r) {
  for (int i = 0; i < r->ntabs; ++i) table_free(&r->tabs[i]);
  free(r->tabs);
  r->tabs = NULL;
}

/* In-place exclusive prefix sum of a[0..len); returns the total. */
static int64_t scan_exclusive(int64_t *a, int64_t len) {
  const int T = omp_get_max_threads();
  int64_t part[T + 1];
  int used = 1;
  part[0] = 0;
#pragma omp parallel
  {
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
    const int64_t lo = len * t / nt, hi = len * (t + 1) / nt;
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a[i];
    part[t + 1] = s;
#pragma omp barrier
#pragma omp single
    {
      used = nt;
      for (int i = 1; i <= nt; ++i) part[i] += part[i - 1];
    }
    int64_t run = part[t];
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t x = a[i];
      a[i] = run;
      run += x;
    }
  }
  return part[used];
}

static int64_t max_degree(const tw_level *g) {
  int64_t m = 0;
#pragma omp parallel for reduction(max : m) schedule(static)
  for (int64_t v = 0; v < g->n; ++v) {
    const int64_t d = g->off[v + 1] - g->off[v];
    if (d > m) m = d;
  }
  return m;
}

/* Every gain fits __int128 and every per-cluster sum fits int64 when the
 * total absolute edge weight W < 2^62, Ktot < 2^62, q W < 2^125 and
 * p Ktot^2 < 2^125 (k_v <= Ktot and K_C <= Ktot at every level, as Compress
 * keeps both). */
static int check_bounds(const tw_level *g, int64_t p, int64_t q) {
  const int T = omp_get_max_threads();
  i128 wpart[T], kpart[T];
  int bad = 0;
  for (int i = 0; i < T; ++i) { wpart[i] = 0; kpart[i] = 0; }
#pragma omp parallel
  {
    const int t = omp_get_thread_num();
    i128 ws = 0, ks = 0;
#pragma omp for schedule(static)
    for (int64_t v = 0; v < g->n; ++v) {
      for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
        const int64_t x = weight(g, e);
        ws += x < 0 ? -(i128)x : (i128)x;
      }
      if (g->k[v] < 0) __atomic_store_n(&bad, 1, RELAXED);
      ks += g->k[v];
    }
    wpart[t] = ws;
    kpart[t] = ks;
  }
  if (bad) return TW_ERR_INVALID;
  i128 W = 0, Kt = 0;
  for (int i = 0; i < T; ++i) { W += wpart[i]; Kt += kpart[i]; }
  /* refused when q W or p Ktot^2 reaches 2^125 (the bound the oracle and the
   * library apply): q > (lim - 1) / W  <=>  q W >= lim for positive integers */
  const i128 lim = (i128)1 << 125;
  if (W >= ((i128)1 << 62) || Kt >= ((i128)1 << 62)) return TW_ERR_OVERFLOW;
  if (W > 0 && (i128)q > (lim - 1) / W) return TW_ERR_OVERFLOW;
  if (Kt > 0 && (i128)p > (lim - 1) / (Kt * Kt)) return TW_ERR_OVERFLOW;
  return TW_OK;
}

/* ------------------------------------------------------------------------ */
/* Best-Moves, synchronous (Algorithm 1, Sec. 3.2.1 and 3.2.2)               */
/* ------------------------------------------------------------------------ */

/* At most num_iter rounds from (L, K) with V' = V.  *any = 1 if some vertex
 * moved in some round.  With the coin on, rounds continue until no vertex
 * wants to move (or num_iter); phase and depth key its draws. */
static int best_moves(const tw_level *g, tw_run *r, int32_t *L, int64_t *K,
                      int *any, int phase, int depth) {
  const int64_t n = g->n;
  const size_t m = (size_t)(n > 0 ? n : 1);
  uint8_t *in = (uint8_t *)malloc(m), *nx = (uint8_t *)malloc(m);
  uint8_t *mv = (uint8_t *)malloc(m), *left = (uint8_t *)malloc(m);
  uint8_t *held = (uint8_t *)malloc(m);
  int32_t *D = (int32_t *)malloc(m * sizeof(int32_t));
  const tw_coin coin = {r->coin, r->seed, phase, depth};
  int err = (in && nx && mv && left && held && D) ? TW_OK : TW_ERR_OOM;
  const int64_t p = r->p, q = r->q;
  *any = 0;
  if (!err) {
    const int64_t dmax = max_degree(g);
#pragma omp parallel
    {
      if (table_fit(&r->tabs[omp_get_thread_num()], dmax) != TW_OK)
        __atomic_store_n(&err, TW_ERR_OOM, RELAXED);
    }
  }
  if (!err) memset(in, 1, m);
  for (int it = 0; !err && it < r->num_iter; ++it) {
    int64_t scanned = 0, nwant = 0, nmoves = 0, nvp = 0;
#pragma omp parallel reduction(+ : scanned, nwant, nmoves, nvp)
    {
      tw_table *t = &r->tabs[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 64)
      for (int64_t v = 0; v < n; ++v) {
        held[v] = 0;
        if (!in[v]) { D[v] = L[v]; continue; }
        D[v] = best_of(g, v, p, q, L, K, t);
        scanned += g->off[v + 1] - g->off[v];
        nvp += 1;
        if (D[v] != L[v]) {
          nwant += 1;
          if (coin.on && !coin_allows(&coin, it, v)) {
            D[v] = L[v];
            held[v] = 1;
          } else {
            nmoves += 1;
          }
        }
      }
    }
    r->rounds += 1;
    r->scanned += scanned;
    if (r->trace && r->trace_len < r->trace_cap) {
      int64_t *row = r->trace + r->trace_len * TW_TRACE_COLS;
      row[0] = depth; row[1] = phase; row[2] = it; row[3] = nvp;
      row[4] = scanned; row[5] = nmoves; row[6] = nwant - nmoves;
    }
    if (r->trace) r->trace_len += 1;
    if (nwant == 0) break;
    if (nmoves) *any = 1;
    /* every move at once; K follows by exact atomic sums */
    memset(left, 0, m);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
      const int32_t from = L[v], to = D[v];
      mv[v] = from != to;
      if (from != to) {
        __atomic_store_n(&left[from], 1, RELAXED);
        __atomic_fetch_add(&K[from], -g->k[v], RELAXED);
        __atomic_fetch_add(&K[to], g->k[v], RELAXED);
        L[v] = to;
      }
    }
    /* next V' */
    if (r->vset == TW_VSET_ALL) {
      memset(nx, 1, m);
    } else {
      memset(nx, 0, m);
      const int by_vertex = r->vset == TW_VSET_NBR_VERTICES;
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t x = 0; x < n; ++x) {
        if (by_vertex ? !mv[x] : !left[L[x]]) continue;
        for (int64_t e = g->off[x]; e < g->off[x + 1]; ++e)
          __atomic_store_n(&nx[g->nbr[e]], 1, RELAXED);
      }
    }
    if (coin.on) {
#pragma omp parallel for schedule(static)
      for (int64_t v = 0; v < n; ++v)
        if (held[v]) nx[v] = 1;  /* held back: evaluated again */
    }
    uint8_t *sw = in; in = nx; nx = sw;
  }
  free(in); free(nx); free(mv); free(left); free(held); free(D);
  return err;
}

/* ------------------------------------------------------------------------ */
/* Compress (Sec. 3.1, Appendix B)                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t *off, *w, *k;
  int32_t *nbr;
} tw_coarse;

static void coarse_free(tw_coarse *c) {
  free(c->off); free(c->w); free(c->k); free(c->nbr);
  memset(c, 0, sizeof(*c));
}

typedef struct {
  int32_t c;
  int64_t w;
} tw_pair;

static int cmp_pair(const void *a, const void *b) {
  const int32_t x = ((const tw_pair *)a)->c, y = ((const tw_pair *)b)->c;
  return (x > y) - (x < y);
}

/* The coarse graph of the clustering L: one vertex per occupied cluster
 * (ranked by id), node weight K_C, edges between clusters summed, rows
 * ascending.  map[v] = coarse vertex of v. */
static int compress(const tw_level *g, const int32_t *L, tw_run *r,
                    int32_t *map, tw_level *out, tw_coarse *cg) {
  const int64_t n = g->n;
  memset(cg, 0, sizeof(*cg));
  int64_t *rank = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!rank) return TW_ERR_OOM;
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) __atomic_store_n(&rank[L[v]], 1, RELAXED);
  const int64_t n2 = scan_exclusive(rank, n);
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) map[v] = (int32_t)rank[L[v]];
  free(rank);

  const size_t m2 = (size_t)n2 + 1;
  int64_t *mstart = (int64_t *)calloc(m2, sizeof(int64_t));
  int64_t *estart = (int64_t *)calloc(m2, sizeof(int64_t));
  int64_t *cursor = (int64_t *)malloc(m2 * sizeof(int64_t));
  int64_t *deg2 = (int64_t *)calloc(m2, sizeof(int64_t));
  int32_t *member = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  cg->k = (int64_t *)calloc(m2, sizeof(int64_t));
  int err = (mstart && estart && cursor && deg2 && member && cg->k) ? TW_OK : TW_ERR_OOM;
  int32_t *tn = NULL;
  int64_t *tw = NULL;
  if (!err) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
      const int32_t c = map[v];
      __atomic_fetch_add(&mstart[c], 1, RELAXED);
      __atomic_fetch_add(&estart[c], g->off[v + 1] - g->off[v], RELAXED);
      __atomic_fetch_add(&cg->k[c], g->k[v], RELAXED);
    }
    scan_exclusive(mstart, n2 + 1);
    const int64_t etot = scan_exclusive(estart, n2 + 1);
    memcpy(cursor, mstart, m2 * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v)
      member[__atomic_fetch_add(&cursor[map[v]], 1, RELAXED)] = (int32_t)v;
    tn = (int32_t *)malloc((size_t)(etot > 0 ? etot : 1) * sizeof(int32_t));
    tw = (int64_t *)malloc((size_t)(etot > 0 ? etot : 1) * sizeof(int64_t));
    if (!tn || !tw) err = TW_ERR_OOM;
  }
  if (!err) {
    /* each coarse row: sum its members' inter-cluster entries in a table,
     * sort the distinct neighbours, write them at the row's entry start */
#pragma omp parallel
    {
      tw_table *t = &r->tabs[omp_get_thread_num()];
      tw_pair *pairs = NULL;
      int64_t pcap = 0;
#pragma omp for schedule(dynamic, 16)
      for (int64_t cu = 0; cu < n2; ++cu) {
        if (__atomic_load_n(&err, RELAXED)) continue;
        int64_t need = estart[cu + 1] - estart[cu];
        if (need > n2) need = n2;
        if (table_fit(t, need) != TW_OK) { __atomic_store_n(&err, TW_ERR_OOM, RELAXED); continue; }
        const uint32_t mask = (uint32_t)(slots_for(need) - 1);
        int64_t nu = 0;
        for (int64_t i = mstart[cu]; i < mstart[cu + 1]; ++i) {
          const int32_t v = member[i];
          for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
            const int32_t cv = map[g->nbr[e]];
            if ((int64_t)cv != cu) table_add(t, mask, &nu, cv, weight(g, e));
          }
        }
        if (nu > pcap) {
          free(pairs);
          pcap = nu;
          pairs = (tw_pair *)malloc((size_t)pcap * sizeof(tw_pair));
          if (!pairs) {
            pcap = 0;
            __atomic_store_n(&err, TW_ERR_OOM, RELAXED);
            for (int64_t i = 0; i < nu; ++i) t->key[t->used[i]] = -1;
            continue;
          }
        }
        for (int64_t i = 0; i < nu; ++i) {
          const uint32_t s = t->used[i];
          pairs[i].c = t->key[s];
          pairs[i].w = t->sum[s];
          t->key[s] = -1;
        }
        qsort(pairs, (size_t)nu, sizeof(tw_pair), cmp_pair);
        const int64_t base = estart[cu];
        for (int64_t i = 0; i < nu; ++i) {
          tn[base + i] = pairs[i].c;
          tw[base + i] = pairs[i].w;
        }
        deg2[cu] = nu;
      }
      free(pairs);
    }
  }
  if (!err) {
    const int64_t nnz2 = scan_exclusive(deg2, n2 + 1);
    cg->nbr = (int32_t *)malloc((size_t)(nnz2 > 0 ? nnz2 : 1) * sizeof(int32_t));
    cg->w = (int64_t *)malloc((size_t)(nnz2 > 0 ? nnz2 : 1) * sizeof(int64_t));
    if (!cg->nbr || !cg->w) err = TW_ERR_OOM;
    if (!err) {
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t cu = 0; cu < n2; ++cu) {
        const int64_t d = deg2[cu + 1] - deg2[cu];
        memcpy(cg->nbr + deg2[cu], tn + estart[cu], (size_t)d * sizeof(int32_t));
        memcpy(cg->w + deg2[cu], tw + estart[cu], (size_t)d * sizeof(int64_t));
      }
      cg->off = deg2;
      deg2 = NULL;
      out->n = n2;
      out->off = cg->off;
      out->nbr = cg->nbr;
      out->w32 = NULL;
      out->w64 = cg->w;
      out->k = cg->k;
    }
  }
  free(mstart); free(estart); free(cursor); free(deg2); free(member);
  free(tn); free(tw);
  if (err) coarse_free(cg);
  return err;
}

/* ------------------------------------------------------------------------ */
/* Parallel-CC, Algorithm 1, with refinement (Sec. 3.2.3)                    */
/* ------------------------------------------------------------------------ */

static int run_level(const tw_level *g, int depth, tw_run *r, int32_t *L) {
  const int64_t n = g->n;
  const size_t m = (size_t)(n > 0 ? n : 1);
  if (r->levels < depth + 1) r->levels = depth + 1;
  int64_t *K = (int64_t *)malloc(m * sizeof(int64_t));
  if (!K) return TW_ERR_OOM;
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) { L[v] = (int32_t)v; K[v] = g->k[v]; }
  int any = 0;
  int err = best_moves(g, r, L, K, &any, 0, depth);
  if (err || !any || depth + 1 >= r->max_levels) { free(K); return err; }

  int32_t *map = (int32_t *)malloc(m * sizeof(int32_t));
  if (!map) { free(K); return TW_ERR_OOM; }
  tw_level g2;
  tw_coarse cg;
  err = compress(g, L, r, map, &g2, &cg);
  if (!err && g2.n < n) {
    int32_t *L2 = (int32_t *)malloc((size_t)(g2.n > 0 ? g2.n : 1) * sizeof(int32_t));
    err = L2 ? run_level(&g2, depth + 1, r, L2) : TW_ERR_OOM;
    if (!err) {
#pragma omp parallel for schedule(static)
      for (int64_t v = 0; v < n; ++v) L[v] = L2[map[v]];  /* Flatten */
      if (r->refine) {
        memset(K, 0, m * sizeof(int64_t));
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < n; ++v) __atomic_fetch_add(&K[L[v]], g->k[v], RELAXED);
        err = best_moves(g, r, L, K, &any, 1, depth);
      }
    }
    free(L2);
  }
  coarse_free(&cg);  /* compress leaves it empty when it fails */
  free(map);
  free(K);
  return err;
}

/* q * CC(labels) (Sec. 2, ordered pairs) = q S_in - p (sum_C K_C^2 -
 * sum_v k_v^2), S_in the weight of the ordered edge pairs inside clusters. */
static int objective(const tw_level *g, int64_t p, int64_t q,
                     const int32_t *labels, i128 *out) {
  const int64_t n = g->n;
  const int T = omp_get_max_threads();
  int64_t *K = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  if (!K) return TW_ERR_OOM;
  i128 part[T];
  for (int i = 0; i < T; ++i) part[i] = 0;
#pragma omp parallel
  {
    const int t = omp_get_thread_num();
    i128 s_in = 0, self_sq = 0, sq = 0;
#pragma omp for schedule(dynamic, 256)
    for (int64_t u = 0; u < n; ++u) {
      for (int64_t e = g->off[u]; e < g->off[u + 1]; ++e)
        if (labels[g->nbr[e]] == labels[u]) s_in += weight(g, e);
      self_sq += (i128)g->k[u] * g->k[u];
      __atomic_fetch_add(&K[labels[u]], g->k[u], RELAXED);
    }
#pragma omp for schedule(static)
    for (int64_t c = 0; c < n; ++c) sq += (i128)K[c] * K[c];
    part[t] = (i128)q * s_in - (i128)p * (sq - self_sq);
  }
  i128 tot = 0;
  for (int i = 0; i < T; ++i) tot += part[i];
  free(K);
  *out = tot;
  return TW_OK;
}

static int set_threads(int threads) {
  if (threads > 0) omp_set_num_threads(threads);
  return omp_get_max_threads();
}

/* ------------------------------------------------------------------------ */
/* Entry points                                                              */
/* ------------------------------------------------------------------------ */

/* Whole method.  Weights: w32 (int32) or w64 (int64) or neither (all 1).
 * mode UNIT (k = 1), DEGREE (k_v = weighted degree, lambda = p / (q 2m)) or
 * CUSTOM (k_custom).  Outputs: canonical labels, q' CC as an int128 in
 * (num_hi, num_lo) with q' in *den_out, stats = (levels, rounds, entries
 * scanned), the thread count used, and, if trace is not NULL, up to
 * trace_cap per-round rows (TW_TRACE_COLS each; *trace_len = rounds run).
 * Returns a TW_* status. */
int tw_cluster(int64_t n, const int64_t *off, const int32_t *nbr,
               const int32_t *w32, const int64_t *w64, const int64_t *k_custom,
               int mode, int64_t p, int64_t q, int num_iter, int max_levels,
               int refine, int vset, int coin, uint64_t seed, int threads,
               int64_t *trace, int64_t trace_cap, int64_t *trace_len,
               int32_t *labels_out,
               int64_t *num_hi, uint64_t *num_lo, int64_t *den_out,
               int64_t *stats_out, int *threads_used) {
  if (n < 0 || n >= ((int64_t)1 << 31) || p <= 0 || q <= 0 || num_iter < 0 ||
      max_levels < 1 || !off)
    return TW_ERR_INVALID;
  *threads_used = set_threads(threads);
  const size_t m = (size_t)(n > 0 ? n : 1);
  int64_t *k = (int64_t *)malloc(m * sizeof(int64_t));
  int32_t *L = (int32_t *)malloc(m * sizeof(int32_t));
  int32_t *minid = (int32_t *)malloc(m * sizeof(int32_t));
  if (!k || !L || !minid) { free(k); free(L); free(minid); return TW_ERR_OOM; }
  tw_level g = {n, off, nbr, w32, w64, k};
  int64_t qe = q;
  int err = TW_OK;
  if (mode == TW_NODEW_UNIT) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) k[v] = 1;
  } else if (mode == TW_NODEW_DEGREE) {
    int64_t two_m = 0;
    int neg = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : two_m)
    for (int64_t v = 0; v < n; ++v) {
      int64_t d = 0;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) d += weight(&g, e);
      if (d < 0) __atomic_store_n(&neg, 1, RELAXED);
      k[v] = d;
      two_m += d;
    }
    const i128 qq = (i128)q * two_m;
    if (neg || two_m <= 0 || qq > (i128)INT64_MAX) err = TW_ERR_INVALID;
    else qe = (int64_t)qq;
  } else if (mode == TW_NODEW_CUSTOM && k_custom) {
    memcpy(k, k_custom, m * sizeof(int64_t));
  } else {
    err = TW_ERR_INVALID;
  }
  if (!err) err = check_bounds(&g, p, qe);
  tw_run r = {p, qe, num_iter, max_levels, refine, vset, 0, 0, 0, NULL, 0, coin, seed,
              trace, trace_cap, 0};
  if (!err) err = run_tables(&r);
  if (!err) err = run_level(&g, 0, &r, L);
  run_free(&r);
  if (!err) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) minid[c] = INT32_MAX;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
      int32_t *slot = &minid[L[v]];
      int32_t cur = __atomic_load_n(slot, RELAXED);
      while ((int32_t)v < cur &&
             !__atomic_compare_exchange_n(slot, &cur, (int32_t)v, 1, RELAXED, RELAXED)) {
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) labels_out[v] = minid[L[v]];
    i128 tot = 0;
    err = objective(&g, p, qe, labels_out, &tot);
    *num_hi = (int64_t)(tot >> 64);
    *num_lo = (uint64_t)tot;
    *den_out = qe;
    stats_out[0] = r.levels;
    stats_out[1] = r.rounds;
    stats_out[2] = r.scanned;
    if (trace_len) *trace_len = r.trace_len;
  }
  free(k); free(L); free(minid);
  return err;
}

/* Best-Moves on one level from the labels L (updated in place), with
 * K = sum of k per label; node weights k given; the coin, if on, draws as
 * the coarsening call at depth 0.  *moved = 1 if a vertex moved, *rounds =
 * rounds evaluated. */
int tw_best_moves(int64_t n, const int64_t *off, const int32_t *nbr,
                  const int32_t *w32, const int64_t *w64, const int64_t *k,
                  int64_t p, int64_t q, int num_iter, int vset, int coin,
                  uint64_t seed, int threads, int32_t *L, int *moved,
                  int64_t *rounds) {
  if (n < 0 || n >= ((int64_t)1 << 31) || p < 0 || q <= 0 || num_iter < 0)
    return TW_ERR_INVALID;
  set_threads(threads);
  for (int64_t v = 0; v < n; ++v)
    if (L[v] < 0 || L[v] >= n) return TW_ERR_INVALID;
  tw_level g = {n, off, nbr, w32, w64, k};
  int err = check_bounds(&g, p, q);
  if (err) return err;
  int64_t *K = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  if (!K) return TW_ERR_OOM;
  for (int64_t v = 0; v < n; ++v) K[L[v]] += k[v];
  tw_run r = {p, q, num_iter, 1, 0, vset, 0, 0, 0, NULL, 0, coin, seed, NULL, 0, 0};
  err = run_tables(&r);
  if (!err) err = best_moves(&g, &r, L, K, moved, 0, 0);
  *rounds = r.rounds;
  run_free(&r);
  free(K);
  return err;
}

/* Compress of the clustering L: n', coarse CSR (malloc'd; release with
 * tw_free) and map[v] = coarse vertex of v. */
int tw_compress(int64_t n, const int64_t *off, const int32_t *nbr,
                const int32_t *w32, const int64_t *w64, const int64_t *k,
                const int32_t *L, int threads, int32_t *map, int64_t *n_out,
                int64_t *nnz_out, int64_t **off_out, int32_t **nbr_out,
                int64_t **w_out, int64_t **k_out) {
  if (n < 0 || n >= ((int64_t)1 << 31)) return TW_ERR_INVALID;
  set_threads(threads);
  for (int64_t v = 0; v < n; ++v)
    if (L[v] < 0 || L[v] >= n) return TW_ERR_INVALID;
  tw_level g = {n, off, nbr, w32, w64, k}, g2;
  tw_coarse cg;
  tw_run r = {1, 1, 0, 1, 0, 0, 0, 0, 0, NULL, 0, 0, 0, NULL, 0, 0};
  int err = run_tables(&r);
  if (!err) err = compress(&g, L, &r, map, &g2, &cg);
  run_free(&r);
  if (err) return err;
  *n_out = g2.n;
  *nnz_out = cg.off[g2.n];
  *off_out = cg.off;
  *nbr_out = cg.nbr;
  *w_out = cg.w;
  *k_out = cg.k;
  return TW_OK;
}

void tw_free(void *x) { free(x); }

/* One full-frontier best-move round from singletons (L[v] = v, K = k):
 * D[v] for every v, the entries scanned, and the wall time of the round
 * alone (tables are sized and touched before the clock starts).  k == NULL
 * selects modularity: k_v = weighted degree and lambda = p / (q 2m). */
int tw_first_round(int64_t n, const int64_t *off, const int32_t *nbr,
                   const int32_t *w32, const int64_t *k, int64_t p, int64_t q,
                   int threads, int32_t *D, int64_t *entries, double *secs,
                   int *threads_used) {
  if (n < 0 || n >= ((int64_t)1 << 31) || p < 0 || q <= 0) return TW_ERR_INVALID;
  *threads_used = set_threads(threads);
  const size_t m = (size_t)(n > 0 ? n : 1);
  int32_t *L = (int32_t *)malloc(m * sizeof(int32_t));
  int64_t *K = (int64_t *)malloc(m * sizeof(int64_t));
  int64_t *kd = k ? NULL : (int64_t *)malloc(m * sizeof(int64_t));
  tw_run r = {p, q, 1, 1, 0, TW_VSET_ALL, 0, 0, 0, NULL, 0, 0, 0, NULL, 0, 0};
  int err = (L && K && (k || kd)) ? run_tables(&r) : TW_ERR_OOM;
  tw_level g = {n, off, nbr, w32, NULL, k ? k : kd};
  if (!err && !k) {
    int64_t two_m = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : two_m)
    for (int64_t v = 0; v < n; ++v) {
      int64_t d = 0;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) d += weight(&g, e);
      kd[v] = d;
      two_m += d;
    }
    const i128 qq = (i128)q * two_m;
    if (two_m <= 0 || qq > (i128)INT64_MAX) err = TW_ERR_INVALID;
    else q = r.q = (int64_t)qq;
  }
  if (!err) err = check_bounds(&g, p, q);
  if (!err) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) { L[v] = (int32_t)v; K[v] = g.k[v]; }
    const int64_t dmax = max_degree(&g);
#pragma omp parallel
    {
      if (table_fit(&r.tabs[omp_get_thread_num()], dmax) != TW_OK)
        __atomic_store_n(&err, TW_ERR_OOM, RELAXED);
    }
  }
  if (!err) {
    int64_t scanned = 0;
    const double t0 = omp_get_wtime();
#pragma omp parallel reduction(+ : scanned)
    {
      tw_table *t = &r.tabs[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 64)
      for (int64_t v = 0; v < n; ++v) {
        D[v] = best_of(&g, v, p, q, L, K, t);
        scanned += off[v + 1] - off[v];
      }
    }
    *secs = omp_get_wtime() - t0;
    *entries = scanned;
  }
  run_free(&r);
  free(L); free(K); free(kd);
  return err;
}
