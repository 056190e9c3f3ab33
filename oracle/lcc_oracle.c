/*
 * Reference oracle for the LambdaCC parallel Louvain method
 * (Shi, Dhulipala, Eisenstat, Lacki, Mirrokni, "Scalable Community Detection
 * via Parallel Correlation Clustering", arXiv 2108.01731).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, single-threaded, slow and
 * deliberately unoptimised restatement of the method, used to check the CUDA
 * library.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Every gain and weight is an exact integer: lambda is the rational p/q and
 * all comparisons are done on q-scaled values in __int128, so the result is
 * independent of any rounding order.
 *
 * Sections followed (paper section / algorithm / equation):
 *   objective .......... Sec. 2 (CC(x) = sum over ordered pairs (i,j) in VxV
 *                        of w'_ij (1 - x_ij); w'_uu = 0, w'_uv = w_uv -
 *                        lambda k_u k_v on edges, -lambda k_u k_v otherwise)
 *   modularity mode .... Sec. 2 (k_v = degree, lambda = gamma / 2m)
 *   move gain .......... Appendix A (gain of moving v from c to c')
 *   Best-Moves ......... Algorithm 1, synchronous schedule of Sec. 3.2.1
 *   vertex subsets V' .. Sec. 3.2.2 (all / neighbours of moved vertices /
 *                        neighbours of clusters)
 *   Compress, Flatten .. Sec. 3.1 and Appendix B
 *   Parallel-CC ........ Algorithm 1 with the refinement of Sec. 3.2.3
 *   Sequential-CC ...... Sec. 3.1 (Algorithm 2 in the appendix): random-order
 *                        local moving to convergence, then Compress, recursion
 *                        and Flatten; the quality reference
 *
 * Readings where the paper is silent (kept identical on the CUDA side, and
 * listed with their reasons in the design notes):
 *   R1 ties between candidate clusters go to the smallest cluster id; a move
 *      happens only when strictly better than staying;
 *   R2 "isolate": if L[v] != v, cluster id v has weight K[v] == 0 in the
 *      round's snapshot and no neighbour of v is in cluster v, v may move to
 *      cluster v with score 0 (its exact gain: no edges into it and K = 0);
 *      when a neighbour is in cluster v, that cluster is already an ordinary
 *      candidate scored by the gain formula;
 *   R3 Compress drops intra-cluster edges (w'_uu = 0, so they never count)
 *      and keeps merged edges whose summed weight is 0;
 *   R4 coarse ids are the occupied cluster ids ranked in increasing order;
 *   R5 a level whose compression does not shrink the graph (n' == n) ends the
 *      recursion, and so does the level cap max_levels;
 *   R6 final labels are the smallest original vertex id of each cluster.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_OOM = 4, ORC_ERR_OVERFLOW = 5 };
enum { VSET_ALL = 0, VSET_NBR_VERTICES = 1, VSET_NBR_CLUSTERS = 2 };
enum { NODEW_UNIT = 0, NODEW_DEGREE = 1, NODEW_CUSTOM = 2 };

/* A graph level: CSR with int64 weights and int64 node weights. */
typedef struct {
  int64_t n;
  const int64_t *off; /* [n+1] */
  const int32_t *nbr; /* [off[n]] */
  const int64_t *w;   /* [off[n]] */
  const int64_t *k;   /* [n] */
} level_t;

typedef struct {
  int64_t rounds_total;
  int64_t edges_scanned;
  int64_t levels;
  /* optional per-round record (the paper's plot of |V'| per round, appendix):
   * rows of ORC_TRACE_COLS = depth, phase (1 = refinement after Flatten),
   * round of the Best-Moves call, |V'|, entries scanned, vertices moved,
   * vertices the coin held back */
  int64_t *trace;
  int64_t trace_cap, trace_len;
} orc_stats;
enum { ORC_TRACE_COLS = 7 };

/* SplitMix64 (S. Vigna's public-domain generator after Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
 * The stream seeded with s has state s + i gamma after i steps; its i-th
 * output (i >= 1) is splitmix64_mix(s + i gamma). */
static const uint64_t SPLITMIX_GAMMA = 0x9e3779b97f4a7c15ull;

static uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

/* Symmetry-breaking coin of the synchronous schedule (an extension: the
 * paper's synchronous rounds have none, and it notes their poor objectives
 * for lack of symmetry breaking, Sec. 4).  In round t of a Best-Moves call
 * (phase 0: the call that coarsens level `depth`; phase 1: its refinement
 * after Flatten), a vertex v whose desired cluster differs from its own may
 * move iff the top bit of output key + 1 of the stream seeded with `seed`
 * is 1, key = v + t 2^32 + depth 2^48 + phase 2^56.  A vertex the coin holds
 * back keeps its label and stays in the next V'. */
typedef struct {
  int on;
  uint64_t seed;
  int phase, depth;
} coin_t;

static int coin_allows(const coin_t *c, int round, int64_t v) {
  const uint64_t key = (uint64_t)v + ((uint64_t)(round & 0xffff) << 32) +
                       ((uint64_t)(c->depth & 0xff) << 48) + ((uint64_t)(c->phase & 1) << 56);
  return (int)(splitmix64_mix(c->seed + (key + 1) * SPLITMIX_GAMMA) >> 63);
}

/* ---------------------------------------------------------------------- */
/* Range of the exact arithmetic                                           */
/* ---------------------------------------------------------------------- */

/* Every q-scaled quantity is a difference of two terms: a gain (Appendix A)
 * is q w(v,C) - p k_v K_C (or the stay form with K_c - k_v), and q CC is
 * q S_in - p (sum_C K_C^2 - sum_v k_v^2) (Sec. 2).  With node weights k >= 0,
 * W = sum of |w| over all entries and Ktot = sum_v k_v, the first term is at
 * most q W and the second at most p Ktot^2 in magnitude.  Requiring
 *   W < 2^62 (so that merged coarse weights and K fit int64),
 *   q W < 2^125 and p Ktot^2 < 2^125
 * keeps each term below 2^125 and every difference, and every comparison of
 * two gains, inside a signed 128-bit integer.  Anything larger is refused
 * with ORC_ERR_OVERFLOW instead of being computed with a wrapped value. */
static int exact_range(i128 W, i128 Kt, int64_t p, int64_t q) {
  const i128 lim = (i128)1 << 125;
  if (W < 0 || Kt < 0) return ORC_ERR_INVALID;
  if (W >= ((i128)1 << 62) || Kt >= ((i128)1 << 62)) return ORC_ERR_OVERFLOW;
  if ((i128)q * W >= lim) return ORC_ERR_OVERFLOW;          /* < 2^63 * 2^62 */
  if (Kt > 0 && (i128)p > (lim - 1) / (Kt * Kt)) return ORC_ERR_OVERFLOW;
  return ORC_OK;
}

/* W over the entries [e0, e1) of w, and Ktot over k[0..n). */
static i128 abs_weight(const int64_t *w, int64_t e0, int64_t e1) {
  i128 W = 0;
  for (int64_t e = e0; e < e1; ++e) W += w[e] < 0 ? -(i128)w[e] : (i128)w[e];
  return W;
}
static i128 node_total(const int64_t *k, int64_t n) {
  i128 Kt = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (k[v] < 0) return -1;
    Kt += k[v];
  }
  return Kt;
}

/* ---------------------------------------------------------------------- */
/* Objective, Sec. 2                                                       */
/* ---------------------------------------------------------------------- */

/* q * CC(labels) by the literal definition: a double loop over all ordered
 * pairs (i, j) in V x V.  O(n^2); for small graphs only.  The edge weight of
 * a pair is looked up by scanning row i. */
int orc_objective_pairs(int64_t n, const int64_t *off, const int32_t *nbr,
                        const int64_t *w, const int64_t *k, int64_t p,
                        int64_t q, const int32_t *labels, int64_t *num_hi,
                        uint64_t *num_lo) {
  int rc = exact_range(abs_weight(w, 0, n > 0 ? off[n] : 0), node_total(k, n), p, q);
  if (rc != ORC_OK) return rc;
  i128 total = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      if (i == j) continue;                       /* w'_uu = 0 */
      if (labels[i] != labels[j]) continue;       /* (1 - x_ij) = 0 */
      i128 wij = 0;
      int is_edge = 0;
      for (int64_t e = off[i]; e < off[i + 1]; ++e)
        if (nbr[e] == j) { wij += w[e]; is_edge = 1; }
      /* q * w'_ij = q * w_ij - p * k_i * k_j   (w_ij = 0 off E) */
      i128 term = -(i128)p * k[i] * k[j];
      if (is_edge) term += (i128)q * wij;
      total += term;
    }
  }
  *num_hi = (int64_t)(total >> 64);
  *num_lo = (uint64_t)total;
  return ORC_OK;
}

/* q * CC(labels) grouped by cluster: the same sum, with the pairs of each
 * cluster C collected, i.e. q * S_in - p * sum_C (K_C^2 - sum_{v in C} k_v^2)
 * where S_in sums w over ordered edge pairs inside a cluster.  O(n + m). */
int orc_objective(int64_t n, const int64_t *off, const int32_t *nbr,
                  const int64_t *w, const int64_t *k, int64_t p, int64_t q,
                  const int32_t *labels, int64_t *num_hi, uint64_t *num_lo) {
  int rc = exact_range(abs_weight(w, 0, n > 0 ? off[n] : 0), node_total(k, n), p, q);
  if (rc != ORC_OK) return rc;
  i128 s_in = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = off[u]; e < off[u + 1]; ++e)
      if (labels[nbr[e]] == labels[u]) s_in += w[e];
  i128 *K = (i128 *)calloc((size_t)(n > 0 ? n : 1), sizeof(i128));
  if (!K) return ORC_ERR_OOM;
  i128 self_sq = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (labels[v] < 0 || labels[v] >= n) { free(K); return ORC_ERR_INVALID; }
    K[labels[v]] += k[v];
    self_sq += (i128)k[v] * k[v];
  }
  i128 sq = 0;
  for (int64_t c = 0; c < n; ++c) sq += K[c] * K[c];
  free(K);
  i128 total = (i128)q * s_in - (i128)p * (sq - self_sq);
  *num_hi = (int64_t)(total >> 64);
  *num_lo = (uint64_t)total;
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Best move of one vertex, Appendix A gain, readings R1 and R2            */
/* ---------------------------------------------------------------------- */

/* Scratch for the per-vertex aggregation: a dense accumulator over cluster
 * ids and the list of ids touched, reset after each vertex. */
typedef struct {
  i128 *acc;
  uint8_t *seen;
  int32_t *touched;
} scratch_t;

static int scratch_init(scratch_t *s, int64_t n) {
  size_t m = (size_t)(n > 0 ? n : 1);
  s->acc = (i128 *)calloc(m, sizeof(i128));
  s->seen = (uint8_t *)calloc(m, 1);
  s->touched = (int32_t *)malloc(m * sizeof(int32_t));
  return (s->acc && s->seen && s->touched) ? ORC_OK : ORC_ERR_OOM;
}
static void scratch_free(scratch_t *s) {
  free(s->acc); free(s->seen); free(s->touched);
}

/* The cluster vertex v (row [rb, re) of nbr/w) wants to join, given the
 * snapshot (L, K).  Moving v from c = L[v] to c' changes the objective by
 *   (w(v,c') - lambda k_v K_c') - (w(v, c minus v) - lambda k_v K_c + lambda k_v^2)
 * (Appendix A); times q, the candidate part is q w(v,c') - p k_v K_c' and the
 * stay part q w(v,c) - p k_v (K_c - k_v).  Returns the chosen id and adds
 * the number of distinct neighbouring clusters to *ncand. */
static int32_t desired_cluster(int64_t v, int64_t rb, int64_t re,
                               const int32_t *nbr, const int64_t *w,
                               const int64_t *k, int64_t p, int64_t q,
                               const int32_t *L, const int64_t *K,
                               scratch_t *s) {
  int64_t nt = 0;
  for (int64_t e = rb; e < re; ++e) {
    int32_t c = L[nbr[e]];
    if (!s->seen[c]) { s->seen[c] = 1; s->touched[nt++] = c; }
    s->acc[c] += w[e];
  }
  const int32_t cv = L[v];
  const i128 kv = k[v];
  const i128 w_stay = s->seen[cv] ? s->acc[cv] : 0;
  const i128 stay = (i128)q * w_stay - (i128)p * kv * ((i128)K[cv] - kv);
  int have = 0;
  i128 best = 0;
  int32_t best_c = cv;
  for (int64_t t = 0; t < nt; ++t) {
    int32_t c = s->touched[t];
    if (c == cv) continue;
    i128 score = (i128)q * s->acc[c] - (i128)p * kv * (i128)K[c];
    if (!have || score > best || (score == best && c < best_c)) {
      have = 1; best = score; best_c = c;
    }
  }
  /* R2: cluster id v, weight 0 and no edge into it: gain 0. */
  if ((int64_t)cv != v && K[v] == 0 && !s->seen[v]) {
    i128 score = 0;
    int32_t c = (int32_t)v;
    if (!have || score > best || (score == best && c < best_c)) {
      have = 1; best = score; best_c = c;
    }
  }
  for (int64_t t = 0; t < nt; ++t) {
    s->seen[s->touched[t]] = 0;
    s->acc[s->touched[t]] = 0;
  }
  if (have && best > stay) return best_c;
  return cv;
}

/* A scratch made once for many calls of orc_desired_scratch (the timed CPU
 * sample evaluates a large graph in windows): its pages are touched here, so
 * no timed window pays for allocating or first-touching them. */
void *orc_scratch_new(int64_t n) {
  scratch_t *s = (scratch_t *)calloc(1, sizeof(scratch_t));
  if (!s) return NULL;
  if (scratch_init(s, n) != ORC_OK) { scratch_free(s); free(s); return NULL; }
  size_t m = (size_t)(n > 0 ? n : 1);
  memset(s->acc, 0, m * sizeof(i128));
  memset(s->seen, 0, m);
  memset(s->touched, 0, m * sizeof(int32_t));
  return s;
}
void orc_scratch_free(void *s) {
  if (!s) return;
  scratch_free((scratch_t *)s);
  free(s);
}

/* One synchronous evaluation for the vertices v in [v0, v1): D[v - v0] is the
 * desired cluster of v under the snapshot (L, K) of all n vertices.  The rows
 * come as a window: row v is nbr_w[off_w[v-v0] .. off_w[v-v0+1]).  Used for the
 * parity checks of a single round and for the timed CPU sample.  `scratch`
 * comes from orc_scratch_new(n) (it is left empty after the call). */
int orc_desired_scratch(void *scratch, int64_t n, int64_t v0, int64_t v1,
                        const int64_t *off_w, const int32_t *nbr_w, const int64_t *w_w,
                        const int64_t *k, int64_t p, int64_t q, const int32_t *L,
                        const int64_t *K, int32_t *D) {
  if (!scratch || v0 < 0 || v1 > n || v0 > v1 || q <= 0 || p < 0) return ORC_ERR_INVALID;
  /* only the rows of the window are read: their |w| bounds every w(v,C) */
  int rc = exact_range(abs_weight(w_w, 0, off_w[v1 - v0]), node_total(k, n), p, q);
  if (rc != ORC_OK) return rc;
  for (int64_t v = v0; v < v1; ++v)
    D[v - v0] = desired_cluster(v, off_w[v - v0], off_w[v - v0 + 1], nbr_w,
                                w_w, k, p, q, L, K, (scratch_t *)scratch);
  return ORC_OK;
}

int orc_desired_range(int64_t n, int64_t v0, int64_t v1, const int64_t *off_w,
                      const int32_t *nbr_w, const int64_t *w_w,
                      const int64_t *k, int64_t p, int64_t q, const int32_t *L,
                      const int64_t *K, int32_t *D) {
  void *s = orc_scratch_new(n);
  if (!s) return ORC_ERR_OOM;
  const int rc = orc_desired_scratch(s, n, v0, v1, off_w, nbr_w, w_w, k, p, q, L, K, D);
  orc_scratch_free(s);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* Best-Moves, Algorithm 1, synchronous schedule (Sec. 3.2.1)              */
/* ---------------------------------------------------------------------- */

/* Runs at most num_iter rounds on level g, starting from (L, K) with V' = V.
 * Returns 1 if any vertex moved in any round, else 0.  With the coin on,
 * the rounds continue until no vertex wants to move (or num_iter). */
static int best_moves(const level_t *g, int64_t p, int64_t q, int num_iter,
                      int vset, int32_t *L, int64_t *K, orc_stats *st,
                      int *err, const coin_t *coin) {
  const int64_t n = g->n;
  size_t m = (size_t)(n > 0 ? n : 1);
  uint8_t *in_vp = (uint8_t *)malloc(m);
  uint8_t *next_vp = (uint8_t *)malloc(m);
  uint8_t *moved = (uint8_t *)malloc(m);
  uint8_t *left = (uint8_t *)malloc(m);
  uint8_t *held = (uint8_t *)malloc(m);
  int32_t *D = (int32_t *)malloc(m * sizeof(int32_t));
  scratch_t s;
  int rc = scratch_init(&s, n);
  int any = 0;
  if (!in_vp || !next_vp || !moved || !left || !held || !D || rc != ORC_OK) {
    *err = ORC_ERR_OOM;
    goto done;
  }
  for (int64_t v = 0; v < n; ++v) in_vp[v] = 1; /* V' <- V */
  for (int it = 0; it < num_iter; ++it) {
    /* parfor v in V': D[v] from the snapshot (L, K) of this round */
    int64_t nvp = 0, nent = 0;
    for (int64_t v = 0; v < n; ++v) {
      if (in_vp[v]) {
        D[v] = desired_cluster(v, g->off[v], g->off[v + 1], g->nbr, g->w,
                               g->k, p, q, L, K, &s);
        nvp += 1;
        nent += g->off[v + 1] - g->off[v];
      } else {
        D[v] = L[v];
      }
    }
    st->edges_scanned += nent;
    st->rounds_total += 1;
    int64_t nwant = 0, nmoved = 0, nheld = 0;
    for (int64_t v = 0; v < n; ++v) {
      held[v] = 0;
      if (D[v] != L[v]) {
        ++nwant;
        if (coin && coin->on && !coin_allows(coin, it, v)) {
          D[v] = L[v];
          held[v] = 1;
          ++nheld;
        }
      }
      moved[v] = (D[v] != L[v]);
      nmoved += moved[v];
      any |= moved[v];
    }
    if (st->trace && st->trace_len < st->trace_cap) {
      int64_t *row = st->trace + st->trace_len * ORC_TRACE_COLS;
      row[0] = coin ? coin->depth : 0;
      row[1] = coin ? coin->phase : 0;
      row[2] = it;
      row[3] = nvp;
      row[4] = nent;
      row[5] = nmoved;
      row[6] = nheld;
    }
    st->trace_len += 1;
    if (nwant == 0) break;
    /* move every v to D[v] at once; K follows the moves */
    memset(left, 0, m);
    for (int64_t v = 0; v < n; ++v) {
      if (!moved[v]) continue;
      left[L[v]] = 1;
      K[L[v]] -= g->k[v];
      K[D[v]] += g->k[v];
      L[v] = D[v];
    }
    /* next V' (Sec. 3.2.2) */
    memset(next_vp, 0, m);
    if (vset == VSET_ALL) {
      memset(next_vp, 1, m);
    } else if (vset == VSET_NBR_VERTICES) {
      for (int64_t v = 0; v < n; ++v)
        if (moved[v])
          for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e)
            next_vp[g->nbr[e]] = 1;
    } else { /* neighbours of the clusters that vertices moved out of */
      for (int64_t x = 0; x < n; ++x)
        if (left[L[x]])
          for (int64_t e = g->off[x]; e < g->off[x + 1]; ++e)
            next_vp[g->nbr[e]] = 1;
    }
    for (int64_t v = 0; v < n; ++v)
      if (held[v]) next_vp[v] = 1;  /* held back by the coin: evaluated again */
    memcpy(in_vp, next_vp, m);
  }
done:
  free(in_vp); free(next_vp); free(moved); free(left); free(held); free(D);
  scratch_free(&s);
  return any;
}

/* ---------------------------------------------------------------------- */
/* Compress and Flatten (Sec. 3.1, Appendix B)                             */
/* ---------------------------------------------------------------------- */

typedef struct {
  int64_t key_u, key_v, w;
} pair_t;

static int cmp_pair(const void *a, const void *b) {
  const pair_t *x = (const pair_t *)a, *y = (const pair_t *)b;
  if (x->key_u != y->key_u) return x->key_u < y->key_u ? -1 : 1;
  if (x->key_v != y->key_v) return x->key_v < y->key_v ? -1 : 1;
  return 0;
}

/* Each occupied cluster becomes a coarse vertex with node weight K_c; every
 * edge (u, v) becomes an edge between the coarse vertices of its endpoints'
 * clusters and parallel edges are summed (R3, R4).  map[v] is the coarse
 * vertex of v.  Outputs are malloc'd; release them with orc_free. */
int orc_compress(int64_t n, const int64_t *off, const int32_t *nbr,
                 const int64_t *w, const int64_t *k, const int32_t *L,
                 int32_t *map, int64_t *n_out, int64_t *nnz_out,
                 int64_t **off_out, int32_t **nbr_out, int64_t **w_out,
                 int64_t **k_out) {
  size_t m = (size_t)(n > 0 ? n : 1);
  /* merged weights and coarse node weights are int64 sums */
  if (abs_weight(w, 0, n > 0 ? off[n] : 0) >= ((i128)1 << 62)) return ORC_ERR_OVERFLOW;
  if (node_total(k, n) >= ((i128)1 << 62)) return ORC_ERR_OVERFLOW;
  int32_t *rank = (int32_t *)malloc(m * sizeof(int32_t));
  if (!rank) return ORC_ERR_OOM;
  for (int64_t c = 0; c < n; ++c) rank[c] = -1;
  for (int64_t v = 0; v < n; ++v) {
    if (L[v] < 0 || L[v] >= n) { free(rank); return ORC_ERR_INVALID; }
    rank[L[v]] = 0;
  }
  int64_t n2 = 0;
  for (int64_t c = 0; c < n; ++c)
    if (rank[c] == 0) rank[c] = (int32_t)(n2++);
  for (int64_t v = 0; v < n; ++v) map[v] = rank[L[v]];
  free(rank);

  int64_t *k2 = (int64_t *)calloc((size_t)(n2 > 0 ? n2 : 1), sizeof(int64_t));
  int64_t *off2 = (int64_t *)calloc((size_t)n2 + 1, sizeof(int64_t));
  if (!k2 || !off2) { free(k2); free(off2); return ORC_ERR_OOM; }
  for (int64_t v = 0; v < n; ++v) k2[map[v]] += k[v];

  int64_t np = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = off[u]; e < off[u + 1]; ++e)
      if (map[u] != map[nbr[e]]) ++np;
  pair_t *pairs = (pair_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(pair_t));
  if (!pairs) { free(k2); free(off2); return ORC_ERR_OOM; }
  int64_t t = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = off[u]; e < off[u + 1]; ++e)
      if (map[u] != map[nbr[e]]) {
        pairs[t].key_u = map[u];
        pairs[t].key_v = map[nbr[e]];
        pairs[t].w = w[e];
        ++t;
      }
  qsort(pairs, (size_t)np, sizeof(pair_t), cmp_pair);
  int64_t nnz2 = 0;
  for (int64_t i = 0; i < np; ++i)
    if (i == 0 || cmp_pair(&pairs[i], &pairs[i - 1]) != 0) ++nnz2;
  int32_t *nbr2 = (int32_t *)malloc((size_t)(nnz2 > 0 ? nnz2 : 1) * sizeof(int32_t));
  int64_t *w2 = (int64_t *)malloc((size_t)(nnz2 > 0 ? nnz2 : 1) * sizeof(int64_t));
  if (!nbr2 || !w2) {
    free(pairs); free(k2); free(off2); free(nbr2); free(w2);
    return ORC_ERR_OOM;
  }
  int64_t j = -1;
  for (int64_t i = 0; i < np; ++i) {
    if (i == 0 || cmp_pair(&pairs[i], &pairs[i - 1]) != 0) {
      ++j;
      nbr2[j] = (int32_t)pairs[i].key_v;
      w2[j] = 0;
      off2[pairs[i].key_u + 1] += 1;
    }
    w2[j] += pairs[i].w;
  }
  for (int64_t c = 0; c < n2; ++c) off2[c + 1] += off2[c];
  free(pairs);
  *n_out = n2;
  *nnz_out = nnz2;
  *off_out = off2;
  *nbr_out = nbr2;
  *w_out = w2;
  *k_out = k2;
  return ORC_OK;
}

void orc_free(void *p) { free(p); }

/* ---------------------------------------------------------------------- */
/* Parallel-CC, Algorithm 1 (recursive), with refinement (Sec. 3.2.3)      */
/* ---------------------------------------------------------------------- */

typedef struct {
  int64_t p, q;
  int num_iter, max_levels, refine, vset;
  orc_stats *st;
  int err;
  int coin;
  uint64_t seed;
} run_t;

/* Clusters level g (depth `depth`) and writes the labels to L. */
static void parallel_cc(const level_t *g, int depth, run_t *r, int32_t *L) {
  const int64_t n = g->n;
  size_t m = (size_t)(n > 0 ? n : 1);
  if (r->st->levels < depth + 1) r->st->levels = depth + 1;
  int64_t *K = (int64_t *)malloc(m * sizeof(int64_t));
  if (!K) { r->err = ORC_ERR_OOM; return; }
  for (int64_t v = 0; v < n; ++v) { L[v] = (int32_t)v; K[v] = g->k[v]; }
  const coin_t coarsen = {r->coin, r->seed, 0, depth};
  int moved = best_moves(g, r->p, r->q, r->num_iter, r->vset, L, K, r->st,
                         &r->err, &coarsen);
  if (r->err || !moved || depth + 1 >= r->max_levels) { free(K); return; }

  int32_t *map = (int32_t *)malloc(m * sizeof(int32_t));
  int64_t n2 = 0, nnz2 = 0;
  int64_t *off2 = NULL, *w2 = NULL, *k2 = NULL;
  int32_t *nbr2 = NULL;
  if (!map) { r->err = ORC_ERR_OOM; free(K); return; }
  int rc = orc_compress(n, g->off, g->nbr, g->w, g->k, L, map, &n2, &nnz2,
                        &off2, &nbr2, &w2, &k2);
  if (rc != ORC_OK) { r->err = rc; free(K); free(map); return; }
  if (n2 < n) {
    level_t g2 = {n2, off2, nbr2, w2, k2};
    int32_t *L2 = (int32_t *)malloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(int32_t));
    if (!L2) {
      r->err = ORC_ERR_OOM;
    } else {
      parallel_cc(&g2, depth + 1, r, L2);
      if (!r->err) {
        /* Flatten: v takes the cluster of its coarse vertex */
        for (int64_t v = 0; v < n; ++v) L[v] = L2[map[v]];
        if (r->refine) {
          for (int64_t v = 0; v < n; ++v) K[v] = 0;
          for (int64_t v = 0; v < n; ++v) K[L[v]] += g->k[v];
          const coin_t refine = {r->coin, r->seed, 1, depth};
          best_moves(g, r->p, r->q, r->num_iter, r->vset, L, K, r->st,
                     &r->err, &refine);
        }
      }
      free(L2);
    }
  }
  free(off2); free(nbr2); free(w2); free(k2); free(map); free(K);
}

/* Whole method on the input graph.  mode selects the node weights: UNIT
 * (k = 1), DEGREE (modularity: k_v = weighted degree and lambda = p / (q 2m)
 * with 2m = sum_v k_v) or CUSTOM (k given).  labels_out receives the
 * canonical labels (R6); num_hi/num_lo receive q' * CC where q' is the
 * effective denominator returned in *den_out. */
/* Node weights of the input level for a mode (Sec. 2): UNIT k = 1; DEGREE
 * (modularity) k_v = weighted degree, with lambda = p / (q 2m) carried as the
 * effective denominator *qe = q 2m; CUSTOM k given.  k is [n]. */
static int node_weights(int64_t n, const int64_t *off, const int64_t *w,
                        const int64_t *k_custom, int mode, int64_t q,
                        int64_t *k, int64_t *qe) {
  *qe = q;
  if (mode == NODEW_UNIT) {
    for (int64_t v = 0; v < n; ++v) k[v] = 1;
  } else if (mode == NODEW_DEGREE) {
    i128 two_m = 0;
    for (int64_t v = 0; v < n; ++v) {
      i128 d = 0;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) d += w[e];
      if (d < 0) return ORC_ERR_INVALID;
      k[v] = (int64_t)d;
      two_m += d;
    }
    if (two_m <= 0) return ORC_ERR_INVALID;
    i128 qq = (i128)q * two_m;
    if (qq > (i128)INT64_MAX) return ORC_ERR_OVERFLOW;
    *qe = (int64_t)qq;
  } else if (mode == NODEW_CUSTOM) {
    for (int64_t v = 0; v < n; ++v) {
      if (k_custom[v] < 0) return ORC_ERR_INVALID;
      k[v] = k_custom[v];
    }
  } else {
    return ORC_ERR_INVALID;
  }
  return ORC_OK;
}

/* R6 labels (smallest vertex id of each cluster of L) into labels_out, and
 * the exact objective of that clustering. */
static int finish_labels(int64_t n, const int64_t *off, const int32_t *nbr,
                         const int64_t *w, const int64_t *k, int64_t p,
                         int64_t qe, const int32_t *L, int32_t *labels_out,
                         int64_t *num_hi, uint64_t *num_lo) {
  int32_t *minid = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!minid) return ORC_ERR_OOM;
  for (int64_t c = 0; c < n; ++c) minid[c] = -1;
  for (int64_t v = 0; v < n; ++v)
    if (minid[L[v]] < 0) minid[L[v]] = (int32_t)v;
  for (int64_t v = 0; v < n; ++v) labels_out[v] = minid[L[v]];
  free(minid);
  return orc_objective(n, off, nbr, w, k, p, qe, labels_out, num_hi, num_lo);
}

int orc_cluster(int64_t n, const int64_t *off, const int32_t *nbr,
                const int64_t *w, const int64_t *k_custom, int mode,
                int64_t p, int64_t q, int num_iter, int max_levels, int refine,
                int vset, int coin, uint64_t seed, int32_t *labels_out,
                int64_t *num_hi, uint64_t *num_lo, int64_t *den_out,
                int64_t *stats_out, int64_t *trace, int64_t trace_cap,
                int64_t *trace_len) {
  if (n < 0 || p <= 0 || q <= 0 || num_iter < 0 || max_levels < 1)
    return ORC_ERR_INVALID;
  size_t m = (size_t)(n > 0 ? n : 1);
  int64_t *k = (int64_t *)malloc(m * sizeof(int64_t));
  if (!k) return ORC_ERR_OOM;
  int64_t qe = q;
  int rc = node_weights(n, off, w, k_custom, mode, q, k, &qe);
  if (rc == ORC_OK)
    rc = exact_range(abs_weight(w, 0, n > 0 ? off[n] : 0), node_total(k, n), p, qe);
  if (rc != ORC_OK) { free(k); return rc; }
  orc_stats st = {0, 0, 0, trace, trace_cap, 0};
  run_t r = {p, qe, num_iter, max_levels, refine, vset, &st, ORC_OK, coin, seed};
  level_t g = {n, off, nbr, w, k};
  int32_t *L = (int32_t *)malloc(m * sizeof(int32_t));
  if (!L) { free(k); return ORC_ERR_OOM; }
  parallel_cc(&g, 0, &r, L);
  if (r.err) { free(k); free(L); return r.err; }
  rc = finish_labels(n, off, nbr, w, k, p, qe, L, labels_out, num_hi, num_lo);
  *den_out = qe;
  if (stats_out) {
    stats_out[0] = st.levels;
    stats_out[1] = st.rounds_total;
    stats_out[2] = st.edges_scanned;
  }
  if (trace_len) *trace_len = st.trace_len;
  free(k);
  free(L);
  return rc;
}

/* One synchronous Best-Moves call on a single level from given labels, for
 * round-by-round checks: runs at most num_iter rounds from (L, K = sum of k
 * per label) with V' = V and returns 1 if anything moved.  With the coin on
 * it draws the coin of phase 0 at depth 0. */
int orc_best_moves(int64_t n, const int64_t *off, const int32_t *nbr,
                   const int64_t *w, const int64_t *k, int64_t p, int64_t q,
                   int num_iter, int vset, int coin, uint64_t seed, int32_t *L,
                   int64_t *rounds_out) {
  size_t m = (size_t)(n > 0 ? n : 1);
  if (q <= 0 || p <= 0) return -ORC_ERR_INVALID;
  const int range = exact_range(abs_weight(w, 0, n > 0 ? off[n] : 0), node_total(k, n), p, q);
  if (range != ORC_OK) return -range;
  int64_t *K = (int64_t *)calloc(m, sizeof(int64_t));
  if (!K) return -ORC_ERR_OOM;
  for (int64_t v = 0; v < n; ++v) {
    if (L[v] < 0 || L[v] >= n) { free(K); return -ORC_ERR_INVALID; }
    K[L[v]] += k[v];
  }
  orc_stats st = {0, 0, 0, NULL, 0, 0};
  int err = ORC_OK;
  level_t g = {n, off, nbr, w, k};
  const coin_t c = {coin, seed, 0, 0};
  int any = best_moves(&g, p, q, num_iter, vset, L, K, &st, &err, &c);
  free(K);
  if (rounds_out) *rounds_out = st.rounds_total;
  return err ? -err : any;
}

/* Sequential local moving (Algorithm 2 inner loop) with a fixed order
 * 0..n-1 instead of a random permutation: each vertex moves at once to its
 * desired cluster.  Stops after max_moves moves (or a full sweep); returns
 * the number of moves.  Used to check that every single move raises CC. */
int64_t orc_sequential_sweep(int64_t n, const int64_t *off,
                             const int32_t *nbr, const int64_t *w,
                             const int64_t *k, int64_t p, int64_t q,
                             int32_t *L, int64_t max_moves) {
  size_t m = (size_t)(n > 0 ? n : 1);
  if (exact_range(abs_weight(w, 0, n > 0 ? off[n] : 0), node_total(k, n), p, q) != ORC_OK)
    return -1;
  int64_t *K = (int64_t *)calloc(m, sizeof(int64_t));
  scratch_t s;
  if (!K || scratch_init(&s, n) != ORC_OK) { free(K); return -1; }
  for (int64_t v = 0; v < n; ++v) K[L[v]] += k[v];
  int64_t moves = 0;
  for (int64_t v = 0; v < n && moves < max_moves; ++v) {
    int32_t d = desired_cluster(v, off[v], off[v + 1], nbr, w, k, p, q, L, K, &s);
    if (d != L[v]) {
      K[L[v]] -= k[v];
      K[d] += k[v];
      L[v] = d;
      ++moves;
    }
  }
  free(K);
  scratch_free(&s);
  return moves;
}

/* ---------------------------------------------------------------------- */
/* Sequential-CC: the sequential Louvain method of Sec. 3.1 (Algorithm 2   */
/* in the appendix), the quality reference of the parallel method          */
/* ---------------------------------------------------------------------- */

/* The next output of the SplitMix64 stream whose state is *x. */
static uint64_t splitmix64(uint64_t *x) {
  *x += SPLITMIX_GAMMA;
  return splitmix64_mix(*x);
}

/* sigma = a random permutation of 0..n-1: Fisher-Yates, the swap partner of
 * position i taken as floor(r (i + 1) / 2^64) from the SplitMix64 stream
 * that starts at state `stream`. */
static void random_permutation(int64_t n, uint64_t stream, int32_t *sigma) {
  uint64_t x = stream;
  for (int64_t i = 0; i < n; ++i) sigma[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    const uint64_t r = splitmix64(&x);
    const int64_t j = (int64_t)(((unsigned __int128)r * (uint64_t)(i + 1)) >> 64);
    const int32_t t = sigma[i];
    sigma[i] = sigma[j];
    sigma[j] = t;
  }
}

typedef struct {
  int64_t p, q;
  uint64_t seed;
  int max_passes, max_levels;
  int64_t levels, passes, moves;
  int err;
} seq_run_t;

/* One level: from singletons, passes over a fresh random order move each
 * vertex at once to its best cluster (the Appendix A gain, readings R1 and
 * R2), until a pass moves nothing; every move raises CC, so "the objective
 * increased during the pass" is "the pass moved a vertex".  Then, if
 * anything moved, Compress, recurse and Flatten; there is no refinement.
 * The pass over level `depth` number `pass` draws its order from the stream
 * seed + depth 2^32 + pass. */
static void sequential_cc(const level_t *g, int depth, seq_run_t *r, int32_t *L) {
  const int64_t n = g->n;
  const size_t m = (size_t)(n > 0 ? n : 1);
  if (r->levels < depth + 1) r->levels = depth + 1;
  int64_t *K = (int64_t *)malloc(m * sizeof(int64_t));
  int32_t *sigma = (int32_t *)malloc(m * sizeof(int32_t));
  scratch_t s;
  int rc = scratch_init(&s, n);
  if (!K || !sigma || rc != ORC_OK) {
    r->err = ORC_ERR_OOM;
    free(K); free(sigma); scratch_free(&s);
    return;
  }
  for (int64_t v = 0; v < n; ++v) { L[v] = (int32_t)v; K[v] = g->k[v]; }
  int64_t level_moves = 0;
  for (int pass = 0; pass < r->max_passes; ++pass) {
    random_permutation(n, r->seed + ((uint64_t)depth << 32) + (uint64_t)pass, sigma);
    int64_t moves = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t v = sigma[i];
      const int32_t d = desired_cluster(v, g->off[v], g->off[v + 1], g->nbr,
                                        g->w, g->k, r->p, r->q, L, K, &s);
      if (d != L[v]) {
        K[L[v]] -= g->k[v];
        K[d] += g->k[v];
        L[v] = d;
        ++moves;
      }
    }
    r->passes += 1;
    level_moves += moves;
    if (moves == 0) break;
  }
  scratch_free(&s);
  free(sigma);
  free(K);
  r->moves += level_moves;
  if (level_moves == 0 || depth + 1 >= r->max_levels) return;

  int32_t *map = (int32_t *)malloc(m * sizeof(int32_t));
  int64_t n2 = 0, nnz2 = 0;
  int64_t *off2 = NULL, *w2 = NULL, *k2 = NULL;
  int32_t *nbr2 = NULL;
  if (!map) { r->err = ORC_ERR_OOM; return; }
  rc = orc_compress(n, g->off, g->nbr, g->w, g->k, L, map, &n2, &nnz2, &off2,
                    &nbr2, &w2, &k2);
  if (rc != ORC_OK) { r->err = rc; free(map); return; }
  if (n2 < n) {
    level_t g2 = {n2, off2, nbr2, w2, k2};
    int32_t *L2 = (int32_t *)malloc((size_t)(n2 > 0 ? n2 : 1) * sizeof(int32_t));
    if (!L2) {
      r->err = ORC_ERR_OOM;
    } else {
      sequential_cc(&g2, depth + 1, r, L2);
      if (!r->err)
        for (int64_t v = 0; v < n; ++v) L[v] = L2[map[v]];  /* Flatten */
      free(L2);
    }
  }
  free(off2); free(nbr2); free(w2); free(k2); free(map);
}

/* Sequential-CC on the input graph (node weights by `mode` as in
 * orc_cluster).  max_passes caps the passes of one level (a level whose cap
 * is reached proceeds as if it had converged); max_levels caps the depth.
 * Outputs: R6 labels, q' CC in (num_hi, num_lo) with q' in *den_out, and
 * stats = (levels, passes, moves). */
int orc_sequential_cc(int64_t n, const int64_t *off, const int32_t *nbr,
                      const int64_t *w, const int64_t *k_custom, int mode,
                      int64_t p, int64_t q, uint64_t seed, int max_passes,
                      int max_levels, int32_t *labels_out, int64_t *num_hi,
                      uint64_t *num_lo, int64_t *den_out, int64_t *stats_out) {
  if (n < 0 || p <= 0 || q <= 0 || max_passes < 1 || max_levels < 1)
    return ORC_ERR_INVALID;
  const size_t m = (size_t)(n > 0 ? n : 1);
  int64_t *k = (int64_t *)malloc(m * sizeof(int64_t));
  int32_t *L = (int32_t *)malloc(m * sizeof(int32_t));
  if (!k || !L) { free(k); free(L); return ORC_ERR_OOM; }
  int64_t qe = q;
  int rc = node_weights(n, off, w, k_custom, mode, q, k, &qe);
  if (rc == ORC_OK)
    rc = exact_range(abs_weight(w, 0, n > 0 ? off[n] : 0), node_total(k, n), p, qe);
  if (rc == ORC_OK) {
    seq_run_t r = {p, qe, seed, max_passes, max_levels, 0, 0, 0, ORC_OK};
    level_t g = {n, off, nbr, w, k};
    sequential_cc(&g, 0, &r, L);
    rc = r.err;
    if (rc == ORC_OK)
      rc = finish_labels(n, off, nbr, w, k, p, qe, L, labels_out, num_hi, num_lo);
    *den_out = qe;
    if (stats_out) {
      stats_out[0] = r.levels;
      stats_out[1] = r.passes;
      stats_out[2] = r.moves;
    }
  }
  free(k);
  free(L);
  return rc;
}

/* Modularity node weights (Sec. 2): k_v = sum_u w_uv, from int32 weights
 * (NULL = unweighted).  Returns the total 2m. */
int64_t orc_weighted_degrees_i32(int64_t n, const int64_t *off,
                                 const int32_t *w, int64_t *k_out) {
  int64_t total = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t d = 0;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) d += w ? (int64_t)w[e] : 1;
    k_out[v] = d;
    total += d;
  }
  return total;
}

/* Desired cluster of each vertex in a list (verts[0..nv)), whose rows are
 * given as a compact CSR: row i is nbr_l[off_l[i] .. off_l[i+1]).  Same rule
 * as orc_desired_range; used to check samples of very large graphs. */
int orc_desired_list(int64_t n, int64_t nv, const int64_t *verts,
                     const int64_t *off_l, const int32_t *nbr_l,
                     const int64_t *w_l, const int64_t *k, int64_t p,
                     int64_t q, const int32_t *L, const int64_t *K,
                     int32_t *D) {
  if (nv < 0 || q <= 0 || p < 0) return ORC_ERR_INVALID;
  int rc = exact_range(abs_weight(w_l, 0, off_l[nv]), node_total(k, n), p, q);
  if (rc != ORC_OK) return rc;
  scratch_t s;
  if (scratch_init(&s, n) != ORC_OK) { scratch_free(&s); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < nv; ++i) {
    if (verts[i] < 0 || verts[i] >= n) { scratch_free(&s); return ORC_ERR_INVALID; }
    D[i] = desired_cluster(verts[i], off_l[i], off_l[i + 1], nbr_l, w_l, k, p,
                           q, L, K, &s);
  }
  scratch_free(&s);
  return ORC_OK;
}
