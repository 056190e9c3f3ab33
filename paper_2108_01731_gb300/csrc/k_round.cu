// Kernels of one synchronous Best-Moves round (Algorithm 1, Sec. 3.2.1).
//
//   k_frontier  builds V' (Sec. 3.2.2) as per-degree-bucket work lists and
//               packs lk[u] = (K[L[u]], L[u]) for every vertex, so that one
//               gather yields both a neighbour's cluster and its weight;
//   k_bm_*      compute D[v] for every v in V' from the snapshot (L, K):
//               aggregate w(v, C) over the neighbouring clusters C, score
//               each with the Appendix A gain (times q, exact integers),
//               take the best (ties to the smallest id), move only if
//               strictly better than staying;
//   k_apply     moves every v to D[v] at once and updates K by exact
//               integer atomics (order-independent);
//   k_mark_*    marks the next V'.
//
// The gain of moving v from c = L[v] to c' (Appendix A), times q:
//   candidate  q * w(v, c')        - p * k_v * K_c'
//   stay       q * w(v, c minus v) - p * k_v * (K_c - k_v)
// S is int64_t when the host has proven both products stay below 2^62 for
// this level, else __int128.
//
// Aggregation by degree: up to 32 entries in registers (groups of 4..32
// lanes, equal clusters found with __match_any_sync); up to 256 in a per-warp
// shared-memory table; up to 4096 in a per-block table; up to 65536 in a table
// spread over the distributed shared memory of a 2..16-block cluster; above
// that in global-memory tables processed in bounded windows.
#include <cooperative_groups.h>
#include <type_traits>

#include "lcc_internal.cuh"

namespace cg = cooperative_groups;

namespace lcc {

namespace {
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Home slot of cluster c in a table of cap slots: the high half of a
// multiplicative (Fibonacci) hash scaled to [0, cap); for cap = 2^lg these
// are the hash's top lg bits.  Probing continues at the next slot, wrapping.
__device__ __forceinline__ uint32_t slot_in(int32_t c, uint32_t cap) {
  const uint32_t h = (uint32_t)(((uint64_t)(uint32_t)c * 0x9E3779B97F4A7C15ull) >> 32);
  return (uint32_t)(((uint64_t)h * cap) >> 32);
}
__device__ __forceinline__ uint32_t next_slot(uint32_t s, uint32_t cap) {
  return s + 1 < cap ? s + 1 : 0;
}


__device__ __forceinline__ int log2i(int64_t pow2) { return 63 - __clzll((long long)pow2); }

// Table geometry for the insert helpers: a power-of-two capacity (home slot
// = top bits of the hash, probing by masking) or any capacity.
struct Pow2Cap {
  uint32_t cap;
  int lg;
  __device__ __forceinline__ explicit Pow2Cap(uint32_t c) : cap(c), lg(log2i((int64_t)c)) {}
  __device__ __forceinline__ uint32_t home(int32_t c) const {
    return (uint32_t)(((uint64_t)(uint32_t)c * 0x9E3779B97F4A7C15ull) >> (64 - lg));
  }
  __device__ __forceinline__ uint32_t next(uint32_t s) const { return (s + 1) & (cap - 1); }
};
struct AnyCap {
  uint32_t cap;
  __device__ __forceinline__ explicit AnyCap(uint32_t c) : cap(c) {}
  __device__ __forceinline__ uint32_t home(int32_t c) const { return slot_in(c, cap); }
  __device__ __forceinline__ uint32_t next(uint32_t s) const { return next_slot(s, cap); }
};

__device__ __forceinline__ int64_t seg_count(const Buckets &b, int bk) {
  const int64_t c = b.cnt[bk];
  return c < b.seg_cap[bk] ? c : b.seg_cap[bk];
}

__device__ __forceinline__ long long warp_sum_ll(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

template <typename S>
__device__ __forceinline__ void warp_argmax(S &s, int32_t &c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const S os = ScoreOps<S>::shfl_xor(s, o, 32);
    const int32_t oc = __shfl_xor_sync(FULL, c, o);
    if (better<S>(os, oc, s, c)) { s = os; c = oc; }
  }
}

__device__ __forceinline__ unsigned long long slot_word(int32_t c, uint32_t k32) {
  return ((unsigned long long)k32 << 32) | (uint32_t)c;
}

// Fields of one job's current level, held in registers by the kernels (the
// job table lives in global memory; reading it once per vertex keeps the
// inner loops free of table loads).
struct JobView {
  const int64_t *off;
  const int32_t *nbr;
  const unsigned long long *gw;  // pre-gathered words from entry gw0 on (null: gather)
  int64_t gw0;
  const void *w;
  const int64_t *k;
  const int32_t *L;
  const int64_t *K;
  int32_t *D;
  const unsigned long long *lk;
  int64_t p, q;
  int32_t wtype;
  int32_t flags;
};

__device__ __forceinline__ JobView view_of(const JobDev *__restrict__ J) {
  JobView x;
  x.off = J->off;
  x.nbr = J->gnbr;  // neighbour positions in the gather layout
  x.gw = J->gw;
  x.gw0 = J->gw ? J->off[0] : 0;
  x.w = J->w;
  x.k = J->k;
  x.L = J->L;
  x.K = J->K;
  x.D = J->D;
  x.lk = J->lk;
  x.p = J->p;
  x.q = J->q;
  x.wtype = J->wtype;
  x.flags = J->flags;
  return x;
}

// L2 policies of the best-move loads.  A round streams every CSR entry of
// V' once (the neighbour ids and weights: read once, evicted first, not kept
// in L1), while the packed label words are gathered at data-dependent
// positions over and over; they are kept in L2 in preference to the streams.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *a) {
  int32_t x;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
      : "=r"(x) : "l"(a), "l"(l2_evict_first()));
  return x;
}
__device__ __forceinline__ int64_t ld_stream(const int64_t *a) {
  int64_t x;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b64 %0, [%1], %2;"
      : "=l"(x) : "l"(a), "l"(l2_evict_first()));
  return x;
}
__device__ __forceinline__ unsigned long long ld_keep(const unsigned long long *a) {
  unsigned long long x;
  asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(x) : "l"(a), "l"(l2_evict_last()));
  return x;
}

// Cluster of neighbour u and, when packed, its weight; `moved` collects the
// LK_MOVED bit.
__device__ __forceinline__ void label_of(const JobView &J, int32_t u, int32_t &c, uint32_t &k32,
                                         uint32_t &moved) {
  if (J.lk) {
    const unsigned long long x = ld_keep(J.lk + u);
    moved |= (uint32_t)x & LK_MOVED;
    c = (int32_t)((uint32_t)x & ~LK_MOVED);
    k32 = (uint32_t)(x >> 32);
  } else {
    c = J.L[u];
    k32 = KNONE;
  }
}

// The same from the word gathered for entry e by k_gather_words (a
// coalesced stream instead of a dependent random gather).
__device__ __forceinline__ void label_at(const JobView &J, int64_t e, int32_t &c, uint32_t &k32,
                                         uint32_t &moved) {
  const unsigned long long x = (unsigned long long)ld_stream((const int64_t *)(J.gw + (e - J.gw0)));
  moved |= (uint32_t)x & LK_MOVED;
  c = (int32_t)((uint32_t)x & ~LK_MOVED);
  k32 = (uint32_t)(x >> 32);
}

__device__ __forceinline__ long long weight_at(const JobView &J, int64_t e) {
  if (J.wtype == W_I32) return (long long)ld_stream((const int32_t *)J.w + e);
  if (J.wtype == W_I64) return (long long)ld_stream((const int64_t *)J.w + e);
  return 1;
}

__device__ __forceinline__ int64_t weight_of(const JobView &J, int32_t c, uint32_t k32) {
  return k32 != KNONE ? (int64_t)k32 : J.K[c];
}

template <typename S>
__device__ __forceinline__ S score_of(const JobView &J, int64_t kv, long long wsum, int32_t c,
                                      uint32_t k32) {
  return (S)J.q * (S)wsum - (S)J.p * (S)kv * (S)weight_of(J, c, k32);
}

// Final decision of one vertex: cluster id v when it has zero weight and no
// neighbour in it (gain 0), then the strict comparison with staying.
template <typename S>
__device__ __forceinline__ int32_t decide(const JobView &J, int32_t v, int32_t Lv, int64_t kv,
                                          int64_t KLv, S best, int32_t bc, long long w_stay,
                                          bool v_seen, int64_t Kv = -1) {
  const S p = (S)J.p, q = (S)J.q;
  if (Lv != v && !v_seen && (Kv >= 0 ? Kv : J.K[v]) == 0) {
    if (better<S>((S)0, v, best, bc)) { best = 0; bc = v; }
  }
  const S stay = q * (S)w_stay - p * (S)kv * ((S)KLv - (S)kv);
  return (bc != INT32_MAX && best > stay) ? bc : Lv;
}

// Weight of v's own cluster (K does not change during the best-move kernels).
__device__ __forceinline__ int64_t own_weight(const JobView &J, int32_t v, int32_t Lv) {
  return J.K[Lv];
}

// The scalars of v that the final decision needs.
struct Own {
  int32_t Lv;
  int64_t kv, KLv, Kv;
};
// Issued early so the loads overlap the row's gathers.
__device__ __forceinline__ Own own_of(const JobView &J, int32_t v) {
  Own o;
  o.Lv = J.L[v];
  o.KLv = J.K[o.Lv];
  o.kv = J.k[v];
  o.Kv = J.K[v];
  return o;
}

// V' work of JF_PULL jobs, counted where it is decided (the frontier kernel
// counts the vertices of the other jobs): entries, vertices and weight bytes,
// summed per block in shared memory so that no thread holds accumulators.
__shared__ unsigned long long s_pull[3];

struct PullCount {
  // every thread of the block, before the first add
  static __device__ __forceinline__ void init() {
    if (threadIdx.x < 3) s_pull[threadIdx.x] = 0;
    __syncthreads();
  }
  __device__ __forceinline__ void add(const JobView &J, int64_t deg) const {
    atomicAdd(&s_pull[0], (unsigned long long)deg);
    atomicAdd(&s_pull[1], 1ull);
    const int wb = J.wtype == W_I32 ? 4 : (J.wtype == W_I64 ? 8 : 0);
    if (wb) atomicAdd(&s_pull[2], (unsigned long long)(deg * wb));
  }
  // every thread of the block, after the last add
  static __device__ __forceinline__ void flush(int64_t *ctr) {
    __syncthreads();
    if (threadIdx.x == 0 && s_pull[1]) {
      atomicAdd((unsigned long long *)&ctr[C_EDGES], s_pull[0]);
      atomicAdd((unsigned long long *)&ctr[C_VERTS], s_pull[1]);
      if (s_pull[2]) atomicAdd((unsigned long long *)&ctr[C_WB], s_pull[2]);
    }
  }
};

// D[v] of an evaluated vertex.  A vertex of a JF_PULL job is in V' only when
// some neighbour moved in the previous round; otherwise it keeps its label.
template <typename S>
__device__ __forceinline__ void write_desired(const JobView &J, int32_t v, int64_t deg,
                                              int32_t Lv, int64_t kv, int64_t KLv, S best,
                                              int32_t bc, long long w_stay, bool v_seen,
                                              bool row_moved, int64_t Kv = -1) {
  if (J.flags & JF_PULL) {
    if (!row_moved) {
      J.D[v] = Lv;
      return;
    }
    PullCount().add(J, deg);
  }
  J.D[v] = decide<S>(J, v, Lv, kv, KLv, best, bc, w_stay, v_seen, Kv);
}

// Linear-probing insert of (c, k32) += sum.  The table has at least twice as
// many slots as keys, so a free or matching slot is found within cap probes.
// `at(s, kp, vp)` gives the key and value pointers of slot s.  `taken` is the
// slot when this call stored the key there first, else NOSLOT.
constexpr uint32_t NOSLOT = 0xFFFFFFFFu;
template <class At, class Cap>
__device__ __forceinline__ bool probe_insert(At at, Cap g, int32_t c, uint32_t k32,
                                             long long sum, uint32_t &taken) {
  const unsigned long long word = slot_word(c, k32);
  uint32_t s = g.home(c);
  taken = NOSLOT;
  for (uint32_t t = 0; t < g.cap; ++t) {
    unsigned long long *kp, *vp;
    at(s, kp, vp);
    const unsigned long long prev = atomicCAS(kp, SLOT_EMPTY, word);
    if (prev == SLOT_EMPTY || (int32_t)(uint32_t)prev == c) {
      atomicAdd(vp, (unsigned long long)sum);
      if (prev == SLOT_EMPTY) taken = s;
      return true;
    }
    s = g.next(s);
  }
  return false;
}
}  // namespace

// ------------------------------------------------------- gathered words ----

// The label word of every entry of the jobs that have a gw buffer, in one
// flat pass: each warp takes 256 consecutive entries, loads their neighbour
// positions (a coalesced stream) and then gathers all eight words a lane
// owns before storing them, so that every thread keeps eight gathers in
// flight and no gather waits on a table operation.
__global__ void __launch_bounds__(256) k_gather_words(const JobDev *__restrict__ jobs,
                                                      const int64_t *__restrict__ estart,
                                                      int njobs, int64_t etot) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 256;
       c0 < etot; c0 += warps * 256) {
    const int j0 = find_job(estart, njobs, c0);
    const int64_t jend = estart[j0 + 1];
    int32_t u[8];
    const JobDev *Js[8];
    int64_t dst[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t f = c0 + k * 32 + lane;
      u[k] = -1;
      Js[k] = nullptr;
      dst[k] = 0;
      if (f < etot) {
        const int jj = f < jend ? j0 : find_job(estart, njobs, f);
        const JobDev *J = jobs + jj;
        dst[k] = f - estart[jj];
        u[k] = ld_stream(J->gnbr + J->off[0] + dst[k]);
        Js[k] = J;
      }
    }
    unsigned long long x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = u[k] >= 0 ? ld_keep(Js[k]->lk + u[k]) : 0ull;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (u[k] >= 0) Js[k]->gw[dst[k]] = x[k];
  }
}

void launch_gather_words(const JobDev *jobs, const int64_t *estart, int njobs, int64_t etot,
                         cudaStream_t st, const Dev &d) {
  if (etot <= 0) return;
  int64_t g = (etot + 2047) / 2048;
  if (g > (int64_t)d.sms * 8) g = (int64_t)d.sms * 8;
  k_gather_words<<<(int)g, 256, 0, st>>>(jobs, estart, njobs, etot);
}

// ---------------------------------------------------------------- V' -----

// Sum of a non-negative value over the lanes of `peers` (each term below
// 2^43, so the high parts stay below 2^32), exact through two 32-bit
// reductions.
__device__ __forceinline__ unsigned long long peers_sum(unsigned peers, long long x) {
  const unsigned lo = __reduce_add_sync(peers, (unsigned)(x & 0xFFFF));
  const unsigned hi = __reduce_add_sync(peers, (unsigned)(x >> 16));
  return ((unsigned long long)hi << 16) + lo;
}

// Tiles of FR_T * FR_V vertices: the lanes of a warp that share a bucket take
// consecutive places of the tile's run of that bucket, and one global atomic
// per bucket and tile places the runs.
constexpr int FR_T = 256, FR_V = 4;

__global__ void __launch_bounds__(FR_T) k_frontier(const JobDev *__restrict__ jobs,
                                                   const int64_t *__restrict__ vstart, int njobs,
                                                   int64_t vtot, Buckets b, int64_t *ctr) {
  __shared__ unsigned t_cnt[NB];
  __shared__ unsigned long long t_base[NB];
  __shared__ unsigned long long s_be[NB], s_bv[NB];
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < NB) {
    t_cnt[tid] = 0;
    s_be[tid] = 0;
    s_bv[tid] = 0;
  }
  __syncthreads();
  long long my_deg = 0, my_cnt = 0, my_wb = 0;
  const int64_t tile = (int64_t)FR_T * FR_V;
  for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < vtot; t0 += (int64_t)gridDim.x * tile) {
    int bk[FR_V];
    uint64_t item[FR_V];
    unsigned place[FR_V];
#pragma unroll
    for (int r = 0; r < FR_V; ++r) {
      const int64_t i = t0 + (int64_t)r * FR_T + tid;
      bk[r] = -1;
      item[r] = 0;
      place[r] = 0;
      int64_t deg = 0;
      if (i < vtot) {
        const int j = find_job(vstart, njobs, i);
        const JobDev *J = jobs + j;
        const int64_t v = i - vstart[j];
        const int32_t Lv = J->L[v];
        // fr bit 0: v is in V' (marked); bit 1: v moved in the previous round
        const uint8_t m = J->fr[v];
        if (m) J->fr[v] = 0;
        const bool pull = (J->flags & JF_PULL) != 0;
        if (J->lk)
          J->lk[J->pos ? J->pos[v] : v] =
              slot_word(Lv, (uint32_t)J->K[Lv]) | (pull && (m & 2) ? LK_MOVED : 0u);
        deg = J->off[v + 1] - J->off[v];
        bool f;
        if (J->flags & JF_ALL)
          f = !(deg == 0 && Lv == (int32_t)v);  // alone with no neighbour: no candidate
        else if (pull)
          f = deg > 0;  // every vertex that can have a moved neighbour; the kernels test it
        else
          f = (m & 1) != 0;
        if (f) {
          bk[r] = bucket_of(deg, J->warp_max);
          item[r] = ((uint64_t)(uint32_t)j << 32) | (uint32_t)v;
          if (!pull) {
            my_deg += deg;
            my_cnt += 1;
            my_wb += deg * (J->wtype == W_I32 ? 4 : (J->wtype == W_I64 ? 8 : 0));
          }
        } else {
          // in V' = V but alone with no neighbour: it keeps its cluster
          // without an evaluation, and still counts as a member of V'
          if (J->flags & JF_ALL) my_cnt += 1;
          deg = 0;
        }
      }
      const unsigned peers = __match_any_sync(FULL, bk[r]);
      if (bk[r] >= 0) {
        const int leader = __ffs(peers) - 1;
        unsigned p0 = 0;
        if (lane == leader) p0 = atomicAdd(&t_cnt[bk[r]], (unsigned)__popc(peers));
        p0 = __shfl_sync(peers, p0, leader);
        place[r] = p0 + __popc(peers & lanemask_lt());
        const unsigned long long ents = peers_sum(peers, deg);
        if (lane == leader) {
          atomicAdd(&s_be[bk[r]], ents);
          atomicAdd(&s_bv[bk[r]], (unsigned long long)__popc(peers));
        }
      }
    }
    __syncthreads();
    if (tid < NB) {
      const unsigned c = t_cnt[tid];
      t_base[tid] = c ? atomicAdd((unsigned long long *)&b.cnt[tid], (unsigned long long)c) : 0ull;
      t_cnt[tid] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < FR_V; ++r) {
      if (bk[r] < 0) continue;
      const int64_t pos = (int64_t)(t_base[bk[r]] + place[r]);
      if (pos < b.seg_cap[bk[r]])
        b.items[b.seg_start[bk[r]] + pos] = item[r];
      else
        atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_BUCKET_OVERFLOW);
    }
  }
  my_deg = warp_sum_ll(my_deg);
  my_cnt = warp_sum_ll(my_cnt);
  my_wb = warp_sum_ll(my_wb);
  if (lane == 0 && my_cnt) {
    atomicAdd((unsigned long long *)&ctr[C_EDGES], (unsigned long long)my_deg);
    atomicAdd((unsigned long long *)&ctr[C_VERTS], (unsigned long long)my_cnt);
    if (my_wb) atomicAdd((unsigned long long *)&ctr[C_WB], (unsigned long long)my_wb);
  }
  __syncthreads();
  if (tid < NB && s_bv[tid]) {
    atomicAdd((unsigned long long *)&ctr[C_BE + tid], s_be[tid]);
    atomicAdd((unsigned long long *)&ctr[C_BV + tid], s_bv[tid]);
  }
}

void launch_frontier(const JobDev *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                     const Buckets &b, int64_t *ctr, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  const int64_t tile = (int64_t)FR_T * FR_V;
  int64_t blocks = (vtot + tile - 1) / tile;
  const int64_t maxb = (int64_t)d.sms * 8;
  if (blocks > maxb) blocks = maxb;
  k_frontier<<<(int)blocks, FR_T, 0, st>>>(jobs, vstart, njobs, vtot, b, ctr);
}

// ------------------------------------------------ deg <= G: G lanes/vertex --

// One step of a warp over items [wbase, wbase + 32 / G) of a bucket's list:
// each group of G lanes takes one vertex and lane t reads entry t.  Equal
// clusters are found with __match_any_sync on (group, cluster) and summed
// into the group leader's shared slot (accw: this warp's 32 words); the
// leaders' scores are then reduced inside the group with xor-shuffles of
// width G.
template <int G, typename S>
__device__ __forceinline__ void group_step(const JobDev *__restrict__ jobs,
                                           const uint64_t *__restrict__ items, int64_t count,
                                           int64_t wbase, unsigned long long *accw,
                                           long long &ncand) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int gsub = lane / G;
  const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (gsub * G));
  const int64_t it = wbase + gsub;
  const bool valid = it < count;
  const uint64_t item = valid ? items[it] : 0ull;
  const JobView J = view_of(jobs + (int)(item >> 32));
  const int32_t v = (int32_t)(uint32_t)item;
  int64_t beg = 0;
  int deg = 0;
  int32_t Lv = 0;
  int64_t kv = 0;
  if (valid) {
    beg = J.off[v];
    deg = (int)(J.off[v + 1] - beg);
    Lv = J.L[v];
    kv = J.k[v];
  }
  const bool has = valid && gl < deg;
  int32_t c = -1;
  uint32_t k32 = KNONE, mbit = 0;
  long long wt = 0;
  if (has) {
    wt = weight_at(J, beg + gl);
    if (J.gw) {
      label_at(J, beg + gl, c, k32, mbit);
    } else {
      const int32_t u = ld_stream(J.nbr + beg + gl);
      label_of(J, u, c, k32, mbit);
    }
  }
  const bool row_moved = (__ballot_sync(FULL, mbit != 0) & gmask) != 0;
  const unsigned long long key = ((unsigned long long)gsub << 32) | (uint32_t)c;
  const unsigned peers = __match_any_sync(FULL, key);
  const int leader = __ffs(peers) - 1;
  long long wsum = wt;
  if (!__all_sync(FULL, !has || __popc(peers) == 1)) {
    accw[lane] = 0;
    __syncwarp();
    if (has) atomicAdd(&accw[leader], (unsigned long long)wt);
    __syncwarp();
    wsum = (long long)accw[lane];
    __syncwarp();
  }
  const bool lead = has && lane == leader;
  const bool is_stay = lead && c == Lv;
  const unsigned sb = __ballot_sync(FULL, is_stay) & gmask;
  long long w_stay = __shfl_sync(FULL, wsum, sb ? (__ffs(sb) - 1) : lane);
  if (!sb) w_stay = 0;
  const bool v_seen = (__ballot_sync(FULL, lead && c == v) & gmask) != 0;
  const bool cand = lead && !is_stay;
  S score = ScoreOps<S>::lowest();
  int32_t cid = INT32_MAX;
  if (cand) {
    score = score_of<S>(J, kv, wsum, c, k32);
    cid = c;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const S os = ScoreOps<S>::shfl_xor(score, o, G);
    const int32_t oc = __shfl_xor_sync(FULL, cid, o, G);
    if (better<S>(os, oc, score, cid)) { score = os; cid = oc; }
  }
  if (valid && gl == 0)
    write_desired<S>(J, v, deg, Lv, kv, own_weight(J, v, Lv), score, cid, w_stay, v_seen,
                     row_moved);
  ncand += __popc(__ballot_sync(FULL, cand));
}

template <int G, typename S>
__global__ void __launch_bounds__(256) k_bm_group(const JobDev *__restrict__ jobs, Buckets b,
                                                  int bk, int64_t *ctr) {
  __shared__ unsigned long long acc[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  constexpr int GPW = 32 / G;
  const int64_t count = seg_count(b, bk);
  const uint64_t *items = b.items + b.seg_start[bk];
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  long long ncand = 0;
  PullCount::init();
  for (int64_t wbase = gw * GPW; wbase < count; wbase += warps_total * GPW)
    group_step<G, S>(jobs, items, count, wbase, acc[wib], ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
  PullCount::flush(ctr);
}

// Every row of at most 32 entries of every job in one resident launch: the
// four lane-group buckets (<= 4, 8, 16, 32 entries) are cut into warp-sized
// units (32 / G vertices each), and each warp takes the next unit from a
// device counter until all are done.  Units are handed out in bucket order,
// so warps that finish early move on to the next bucket's rows instead of
// waiting for a launch boundary, and the number of warps does not depend on
// the size of any one bucket or graph.
template <typename S>
__global__ void __launch_bounds__(256) k_bm_small(const JobDev *__restrict__ jobs, Buckets b,
                                                  int64_t *ctr) {
  __shared__ unsigned long long acc[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int64_t cnt[4], ends[4];
  int64_t tot = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    cnt[i] = seg_count(b, B_G4 + i);
    const int gpw = 8 >> i;  // 32 / G for G = 4, 8, 16, 32
    tot += (cnt[i] + gpw - 1) / gpw;
    ends[i] = tot;
  }
  long long ncand = 0;
  PullCount::init();
  while (true) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd((unsigned long long *)&ctr[C_WORK], 1ull);
    u = __shfl_sync(FULL, u, 0);
    if ((int64_t)u >= tot) break;
    const int64_t x = (int64_t)u;
    if (x < ends[0]) {
      group_step<4, S>(jobs, b.items + b.seg_start[B_G4], cnt[0], x * 8, acc[wib], ncand);
    } else if (x < ends[1]) {
      group_step<8, S>(jobs, b.items + b.seg_start[B_G8], cnt[1], (x - ends[0]) * 4, acc[wib],
                       ncand);
    } else if (x < ends[2]) {
      group_step<16, S>(jobs, b.items + b.seg_start[B_G16], cnt[2], (x - ends[1]) * 2,
                        acc[wib], ncand);
    } else {
      group_step<32, S>(jobs, b.items + b.seg_start[B_G32], cnt[3], x - ends[2], acc[wib],
                        ncand);
    }
  }
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
  PullCount::flush(ctr);
}

// ------------------------------------------------ preloaded row chunks -----

// E entries per thread, entry i of thread t at lo + i * stride + t: the
// neighbour ids and weights are loaded first and the labels gathered next,
// so that up to E independent gathers per thread are in flight.
template <int E>
struct Chunk {
  int32_t c[E];
  uint32_t k[E];
  long long w[E];
  uint32_t mv;  // LK_MOVED if some neighbour of the chunk moved
};

// (W = false: the weights are not loaded and read as 0)
template <int E, bool W = true>
__device__ __forceinline__ void load_chunk(const JobView &J, int64_t beg, int64_t lo, int64_t hi,
                                           int stride, int t, Chunk<E> &x) {
  if (J.gw) {
    x.mv = 0;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int64_t e = lo + (int64_t)i * stride + t;
      x.c[i] = -1;
      x.k[i] = KNONE;
      x.w[i] = 0;
      if (e < hi) {
        if (W) x.w[i] = weight_at(J, beg + e);
        label_at(J, beg + e, x.c[i], x.k[i], x.mv);
      }
    }
    return;
  }
  int32_t u[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int64_t e = lo + (int64_t)i * stride + t;
    u[i] = -1;
    x.w[i] = 0;
    if (e < hi) {
      u[i] = ld_stream(J.nbr + beg + e);
      if (W) x.w[i] = weight_at(J, beg + e);
    }
  }
  x.mv = 0;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    x.c[i] = -1;
    x.k[i] = KNONE;
    if (u[i] >= 0) label_of(J, u[i], x.c[i], x.k[i], x.mv);
  }
}

// The same chunk in two steps, for a pipeline over vertices: the neighbour
// positions first (load_pos), then, later, the weights and label words
// gathered through those positions (load_chunk_at).
template <int E>
__device__ __forceinline__ void load_pos(const JobView &J, int64_t beg, int64_t lo, int64_t hi,
                                         int stride, int t, int32_t (&u)[E]) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int64_t e = lo + (int64_t)i * stride + t;
    u[i] = (e < hi && !J.gw) ? ld_stream(J.nbr + beg + e) : -1;
  }
}

template <int E>
__device__ __forceinline__ void load_chunk_at(const JobView &J, int64_t beg, int64_t lo,
                                              int64_t hi, int stride, int t,
                                              const int32_t (&u)[E], Chunk<E> &x) {
  if (J.gw) {  // words already gathered: no positions were loaded
    load_chunk(J, beg, lo, hi, stride, t, x);
    return;
  }
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int64_t e = lo + (int64_t)i * stride + t;
    x.w[i] = e < hi ? weight_at(J, beg + e) : 0;
  }
  x.mv = 0;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    x.c[i] = -1;
    x.k[i] = KNONE;
    if (u[i] >= 0) label_of(J, u[i], x.c[i], x.k[i], x.mv);
  }
}

// Asks L2 for the label words the positions u will gather (no registers are
// held for the results): issued for the next vertex while the current one is
// merged, so that its gathers find the words in L2.
template <int E>
__device__ __forceinline__ void prefetch_words(const JobView &J, const int32_t (&u)[E]) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    if (u[i] < 0) continue;
    const void *a = J.lk ? (const void *)(J.lk + u[i]) : (const void *)(J.L + u[i]);
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(a));
  }
}

// Inserts a thread's chunk into a table.  The first probe of every entry is
// issued before any result is examined, so the compare-and-swaps overlap;
// entries whose home slot holds another cluster continue probing one by one.
// Equal clusters need no pre-aggregation: every inserter of a cluster finds
// its slot and adds to it (integer sums, so the order does not matter).
// won[i] is the slot where entry i's cluster was stored first (by this
// thread), else NOSLOT: each distinct cluster is won by exactly one thread.
template <int E, class At, class Cap>
__device__ __forceinline__ bool insert_chunk_won(const Chunk<E> &x, At at, Cap g,
                                                 uint32_t (&won)[E]) {
  unsigned long long prev[E];
  uint32_t home[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    prev[i] = 0;
    home[i] = 0;
    if (x.c[i] >= 0) {
      home[i] = g.home(x.c[i]);
      unsigned long long *kp, *vp;
      at(home[i], kp, vp);
      prev[i] = atomicCAS(kp, SLOT_EMPTY, slot_word(x.c[i], x.k[i]));
    }
  }
  bool ok = true;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    won[i] = NOSLOT;
    if (x.c[i] < 0) continue;
    if (prev[i] == SLOT_EMPTY || (int32_t)(uint32_t)prev[i] == x.c[i]) {
      unsigned long long *kp, *vp;
      at(home[i], kp, vp);
      atomicAdd(vp, (unsigned long long)x.w[i]);
      if (prev[i] == SLOT_EMPTY) won[i] = home[i];
    } else {
      ok &= probe_insert(at, g, x.c[i], x.k[i], x.w[i], won[i]);
    }
  }
  return ok;
}

template <int E, class At, class Cap>
__device__ __forceinline__ bool insert_chunk(const Chunk<E> &x, At at, Cap g) {
  uint32_t won[E];
  return insert_chunk_won(x, at, g, won);
}

// Scores the clusters a thread won (once the sums are complete) and empties
// their slots: best candidate, stay weight, and whether cluster id v occurs.
template <typename S, int E, class At>
__device__ __forceinline__ void scan_won(const JobView &J, const uint32_t (&won)[E], At at,
                                         int32_t v, int32_t Lv, int64_t kv, S &best, int32_t &bc,
                                         long long &w_stay, int &vseen, long long &ncand) {
  const S q = (S)J.q, pk = (S)J.p * (S)kv;
  unsigned long long word[E], val[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {  // all reads first (they may be remote)
    word[i] = SLOT_EMPTY;
    val[i] = 0;
    if (won[i] != NOSLOT) {
      unsigned long long *kp, *vp;
      at(won[i], kp, vp);
      word[i] = *kp;
      val[i] = *vp;
    }
  }
#pragma unroll
  for (int i = 0; i < E; ++i) {
    if (won[i] == NOSLOT) continue;
    unsigned long long *kp, *vp;
    at(won[i], kp, vp);
    *kp = SLOT_EMPTY;
    *vp = 0;
    const int32_t c = (int32_t)(uint32_t)word[i];
    if (c == Lv) {
      w_stay += (long long)val[i];
      continue;
    }
    vseen |= (c == v);
    ++ncand;
    const S sc = q * (S)(long long)val[i] - pk * (S)weight_of(J, c, (uint32_t)(word[i] >> 32));
    if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
  }
}

// Scans table slots s0, s0 + step, ... < s1 of a vertex: best candidate, stay
// weight, and whether cluster id v occurs.
template <typename S>
__device__ __forceinline__ void scan_slots(const JobView &J, const unsigned long long *keys,
                                           const unsigned long long *vals, int64_t s0, int64_t s1,
                                           int step, int32_t v, int32_t Lv, int64_t kv, S &best,
                                           int32_t &bc, long long &w_stay, int &vseen,
                                           long long &ncand) {
  const S q = (S)J.q, pk = (S)J.p * (S)kv;
  for (int64_t s = s0; s < s1; s += step) {
    const unsigned long long word = keys[s];
    if (word == SLOT_EMPTY) continue;
    const int32_t c = (int32_t)(uint32_t)word;
    const long long val = (long long)vals[s];
    if (c == Lv) {
      w_stay += val;
      continue;
    }
    vseen |= (c == v);
    ++ncand;
    const S sc = q * (S)val - pk * (S)weight_of(J, c, (uint32_t)(word >> 32));
    if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
  }
}

// The same over a block's own share of a table, emptying each slot as it is
// read (the next vertex finds the share empty after the closing sync).
template <typename S>
__device__ __forceinline__ void scan_slots_reset(const JobView &J, unsigned long long *keys,
                                                 unsigned long long *vals, int s0, int s1,
                                                 int step, int32_t v, int32_t Lv, int64_t kv,
                                                 S &best, int32_t &bc, long long &w_stay,
                                                 int &vseen, long long &ncand) {
  const S q = (S)J.q, pk = (S)J.p * (S)kv;
  for (int s = s0; s < s1; s += step) {
    const unsigned long long word = keys[s];
    if (word == SLOT_EMPTY) continue;
    const long long val = (long long)vals[s];
    keys[s] = SLOT_EMPTY;
    vals[s] = 0;
    const int32_t c = (int32_t)(uint32_t)word;
    if (c == Lv) {
      w_stay += val;
      continue;
    }
    vseen |= (c == v);
    ++ncand;
    const S sc = q * (S)val - pk * (S)weight_of(J, c, (uint32_t)(word >> 32));
    if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
  }
}

// ----------------------------------- deg <= T_WARP: warp + shared table --

// One warp per vertex, lane t reads entries t, t + 32, ...  The warp's table
// is emptied once at the start; afterwards every lane empties the slots it
// won while scoring them, so each vertex costs one step per distinct cluster.
// Blocks per SM are held to what the shared tables allow, so that the
// register allocation does not lower the occupancy.
template <typename S, int E, int BK>
__global__ void __launch_bounds__(128, E >= 8 ? 5 : (E >= 4 ? 7 : 8))
    k_bm_warp(const JobDev *__restrict__ jobs, Buckets b, int64_t *ctr) {
  constexpr int WPB = 4;
  // slots per entry, before rounding up to a power of two: 4 for rows of
  // up to 64 entries (fewer probes), 2 for longer ones (so that the
  // tables do not cap the blocks per SM)
  constexpr int SPREAD = E <= 2 ? 4 : 2;
  constexpr int CAP = SPREAD * 32 * E;
  __shared__ unsigned long long tkey[WPB][CAP];
  __shared__ unsigned long long tval[WPB][CAP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t count = seg_count(b, BK);
  const uint64_t *items = b.items + b.seg_start[BK];
  const int64_t warps_total = (int64_t)gridDim.x * WPB;
  long long ncand = 0;
  bool fail = false;
  PullCount::init();
  unsigned long long *K0 = tkey[wib], *V0 = tval[wib];
  auto at = [K0, V0](uint32_t s, unsigned long long *&kp, unsigned long long *&vp) {
    kp = K0 + s;
    vp = V0 + s;
  };
  for (int s = lane; s < CAP; s += 32) {
    K0[s] = SLOT_EMPTY;
    V0[s] = 0;
  }
  __syncwarp();
  for (int64_t it = (int64_t)blockIdx.x * WPB + wib; it < count; it += warps_total) {
    const uint64_t item = items[it];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J.off[v];
    const int deg = (int)(J.off[v + 1] - beg);
    Chunk<E> x;
    load_chunk(J, beg, 0, deg, 32, lane, x);
    const Own o = own_of(J, v);
    const int cap = (int)next_pow2(SPREAD * (int64_t)deg);
    uint32_t won[E];
    fail |= !insert_chunk_won(x, at, Pow2Cap((uint32_t)cap), won);
    const bool row_moved = __any_sync(FULL, x.mv != 0);  // after the gathers have landed
    __syncwarp();  // every lane's sums are in place
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    long long w_stay = 0, nc = 0;
    int vseen = 0;
    scan_won<S, E>(J, won, at, v, o.Lv, o.kv, best, bc, w_stay, vseen, nc);
    w_stay = warp_sum_ll(w_stay);
    const bool v_seen = __any_sync(FULL, vseen);
    ncand += nc;
    warp_argmax<S>(best, bc);
    if (lane == 0)
      write_desired<S>(J, v, deg, o.Lv, o.kv, o.KLv, best, bc, w_stay, v_seen, row_moved,
                       o.Kv);
    __syncwarp();  // the emptied slots are seen by the next vertex's inserts
  }
  ncand = warp_sum_ll(ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
  if (__any_sync(FULL, fail) && lane == 0)
    atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
  PullCount::flush(ctr);
}

// --------------- deg <= 65536: one block or a cluster of CS blocks ---------

// One vertex per cluster at a time; block r reads entries [r * per,
// (r + 1) * per) of the row in CH chunks of E per thread (the degree buckets
// keep per <= THREADS * E * CH).  The table has 1.6 slots per entry of the
// row (load <= 0.625, any size: home slots are scaled hashes), P slots in
// each block's shared memory (P <= TP), slot s in block s % CS, reached with
// distributed-shared-memory atomics when CS > 1.  The tables are emptied once
// at the start; after the inserts either the thread that first stored a
// cluster scores it and empties its slot (one chunk and CS <= 2: a vertex
// costs one step per distinct cluster), or each block scans and empties its
// own share, so no clearing pass is needed.  Block 0 combines the results.
// The 256-thread kernel is held to 5 blocks per SM worth of registers (its
// 32 KB tables allow 7; at 60 registers it ran 4), the 512-thread one to 2.
template <typename S, int CS, int THREADS, int TP, int E, int CH, bool POW2, int BK, bool PF = false>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 5 : (THREADS == 512 ? 2 : 1))
    k_bm_table(const JobDev *__restrict__ jobs, Buckets b,
                                                      int64_t *ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = THREADS / 32;
  // with several chunks, or with 4 or more blocks (most won slots remote),
  // each block scans (and empties) its own share of the table instead
  constexpr bool LOCAL_SCAN = CS >= 4 || CH > 1;
  constexpr int CSLG = CS >= 16 ? 4 : CS >= 8 ? 3 : CS >= 4 ? 2 : CS >= 2 ? 1 : 0;
  unsigned long long *tkey = (unsigned long long *)smem;
  unsigned long long *tval = tkey + TP;
  __shared__ S red_s[NW];
  __shared__ int32_t red_c[NW];
  __shared__ long long red_w[NW];
  __shared__ int red_v[NW];
  __shared__ S cl_s[CS];
  __shared__ int32_t cl_c[CS];
  __shared__ long long cl_w[CS];
  __shared__ int cl_v[CS];
  __shared__ int s_rowmv;  // a neighbour of the current vertex moved (this block's entries)
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int64_t count = seg_count(b, BK);
  const uint64_t *items = b.items + b.seg_start[BK];
  const int64_t ncl = gridDim.x / CS;
  const int64_t cid = blockIdx.x / CS;
  long long ncand = 0;
  bool fail = false;
  if (tid == 0) s_rowmv = 0;
  for (int s = tid; s < TP; s += THREADS) {
    tkey[s] = SLOT_EMPTY;
    tval[s] = 0;
  }
  PullCount::init();
  if (CS > 1) cluster.sync();  // every block's table is empty before any remote insert
  // This block's share [lo, hi) of the row of the vertex in item it.
  auto share = [&](const JobView &Jx, int32_t vx, int64_t &bx, int64_t &dx, int64_t &lx,
                   int64_t &hx) {
    bx = Jx.off[vx];
    dx = Jx.off[vx + 1] - bx;
    const int64_t px = (dx + CS - 1) / CS;
    lx = (int64_t)rank * px;
    hx = lx + px < dx ? lx + px : dx;
  };
  // One-chunk kernels pipeline the vertices: the next vertex's neighbour
  // positions are loaded while this one is merged, and its label words are
  // prefetched into L2 before the closing barriers.
  constexpr bool PIPE = PF && CH == 1;
  int32_t un[E];
  if (PIPE && cid < count) {
    const uint64_t item0 = items[cid];
    const JobView J0 = view_of(jobs + (int)(item0 >> 32));
    int64_t b0, d0, l0, h0;
    share(J0, (int32_t)(uint32_t)item0, b0, d0, l0, h0);
    load_pos<E>(J0, b0, l0, h0, THREADS, tid, un);
  }
  for (int64_t it = cid; it < count; it += ncl) {
    const uint64_t item = items[it];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    int64_t beg, deg, lo, hi;
    share(J, v, beg, deg, lo, hi);
    if (hi - lo > (int64_t)THREADS * E * CH) fail = true;  // excluded by the degree buckets
    Chunk<E> x;
    JobView Jn = J;
    const bool next = PIPE && it + ncl < count;
    if (PIPE) {
      load_chunk_at<E>(J, beg, lo, hi, THREADS, tid, un, x);
      if (next) {
        const uint64_t itemn = items[it + ncl];
        Jn = view_of(jobs + (int)(itemn >> 32));
        int64_t bn, dn, ln, hn;
        share(Jn, (int32_t)(uint32_t)itemn, bn, dn, ln, hn);
        load_pos<E>(Jn, bn, ln, hn, THREADS, tid, un);
      }
    } else {
      load_chunk(J, beg, lo, hi, THREADS, tid, x);
    }
    const Own o = own_of(J, v);
    // P slots per block: POW2, next_pow2(2 deg) / CS (at least 32); else 1.6
    // per entry of the row, a multiple of 32
    int64_t P;
    if (POW2) {
      // 4 slots per entry for rows of up to 256 entries (WARP_CAP), else 2
      constexpr int64_t SP = BK == B_WARP ? 4 : 2;
      P = next_pow2(SP * deg) / CS;
      if (P < 32) P = 32;
    } else {
      P = (deg * 8 + 5 * CS - 1) / (5 * CS);
      P = (P + 31) & ~(int64_t)31;
    }
    if (P > TP) {  // excluded by the degree buckets
      P = TP;
      fail = true;
    }
    const uint32_t part = (uint32_t)P;
    const uint32_t cap = part * CS;
    using Cap = typename std::conditional<POW2, Pow2Cap, AnyCap>::type;
    const Cap geo(cap);
    auto at = [&](uint32_t s, unsigned long long *&kp, unsigned long long *&vp) {
      if (CS == 1) {
        kp = tkey + s;
        vp = tval + s;
      } else {
        const unsigned r = s & (CS - 1), l = s >> CSLG;
        kp = cluster.map_shared_rank(tkey, r) + l;
        vp = cluster.map_shared_rank(tval, r) + l;
      }
    };
    uint32_t won[E];
    if (CH == 1) {
      fail |= !insert_chunk_won(x, at, geo, won);
      if (x.mv) s_rowmv = 1;
      if (next) prefetch_words<E>(Jn, un);
    } else {
      Chunk<E> y;  // the second chunk's gathers overlap the first chunk's inserts
      load_chunk(J, beg, lo + (int64_t)THREADS * E, hi, THREADS, tid, y);
      fail |= !insert_chunk(x, at, geo);
      fail |= !insert_chunk(y, at, geo);
      if (x.mv | y.mv) s_rowmv = 1;
    }
    if (CS > 1) cluster.sync(); else __syncthreads();  // sums complete
    const int32_t Lv = o.Lv;
    const int64_t kv = o.kv;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    long long w_stay = 0, nc = 0;
    int vseen = 0;
    if (LOCAL_SCAN)
      scan_slots_reset<S>(J, tkey, tval, tid, (int)part, THREADS, v, Lv, kv, best, bc, w_stay,
                          vseen, nc);
    else
      scan_won<S, E>(J, won, at, v, Lv, kv, best, bc, w_stay, vseen, nc);
    ncand += nc;
    w_stay = warp_sum_ll(w_stay);
    const int vs = __any_sync(FULL, vseen);
    warp_argmax<S>(best, bc);
    if (lane == 0) {
      red_s[wib] = best;
      red_c[wib] = bc;
      red_w[wib] = w_stay;
      red_v[wib] = vs;
    }
    __syncthreads();
    if (wib == 0) {
      S bs = lane < NW ? red_s[lane] : ScoreOps<S>::lowest();
      int32_t bcc = lane < NW ? red_c[lane] : INT32_MAX;
      long long ws = lane < NW ? red_w[lane] : 0;
      int vv = lane < NW ? red_v[lane] : 0;
      warp_argmax<S>(bs, bcc);
      ws = warp_sum_ll(ws);
      // bit 0: cluster id v occurs; bit 1: a neighbour moved (read, then
      // cleared for the next vertex: its writes come after the next sync)
      int vall = __any_sync(FULL, vv);
      if (lane == 0) {
        if (s_rowmv) vall |= 2;
        s_rowmv = 0;
        if (CS == 1) {
          write_desired<S>(J, v, deg, Lv, kv, o.KLv, bs, bcc, ws, (vall & 1) != 0,
                           (vall & 2) != 0, o.Kv);
        } else {
          *cluster.map_shared_rank(&cl_s[rank], 0) = bs;
          *cluster.map_shared_rank(&cl_c[rank], 0) = bcc;
          *cluster.map_shared_rank(&cl_w[rank], 0) = ws;
          *cluster.map_shared_rank(&cl_v[rank], 0) = vall;
        }
      }
    }
    // this sync also orders the emptied slots before the next vertex's inserts
    if (CS > 1) {
      cluster.sync();
      if (rank == 0 && tid == 0) {
        S bs = cl_s[0];
        int32_t bcc = cl_c[0];
        long long ws = cl_w[0];
        int vall = cl_v[0];
        for (int r = 1; r < CS; ++r) {
          if (better<S>(cl_s[r], cl_c[r], bs, bcc)) { bs = cl_s[r]; bcc = cl_c[r]; }
          ws += cl_w[r];
          vall |= cl_v[r];
        }
        write_desired<S>(J, v, deg, Lv, kv, o.KLv, bs, bcc, ws, (vall & 1) != 0,
                         (vall & 2) != 0, o.Kv);
      }
    } else {
      __syncthreads();
    }
  }
  ncand = warp_sum_ll(ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
  if (__any_sync(FULL, fail) && lane == 0)
    atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
  PullCount::flush(ctr);
}

// ------------------------------------- hubs: global-memory hash tables ----

__device__ __forceinline__ int find_seg(const int64_t *__restrict__ off, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return (int)lo;
}

// Lays out one table, insertion units and scoring units per hub (one block).
// Tables are placed back to back in a global slot space; the hubs whose table
// starts in [lo, lo + window) are processed together in one pass, their
// tables at (start - lo) in the scratch buffer.
__global__ void __launch_bounds__(1024) k_hub_prep(const JobDev *__restrict__ jobs, Buckets b,
                                                   HubBufs h, int64_t *ctr) {
  __shared__ int64_t s_a[1024], s_b[1024], s_c[1024];
  __shared__ int64_t run_a, run_b, run_c;
  const int tid = threadIdx.x;
  int64_t H = h.list ? *h.list_cnt : seg_count(b, B_HUB);
  if (H > h.max_hubs) {
    if (tid == 0) atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
    H = h.max_hubs;
  }
  const uint64_t *items = h.list ? h.list : b.items + b.seg_start[B_HUB];
  if (tid == 0) { run_a = 0; run_b = 0; run_c = 0; }
  __syncthreads();
  for (int64_t base = 0; base < H; base += 1024) {
    const int64_t i = base + tid;
    int64_t a = 0, u = 0, s = 0;
    if (i < H) {
      const uint64_t item = items[i];
      const JobDev *J = jobs + (int)(item >> 32);
      const int32_t v = (int32_t)(uint32_t)item;
      const int64_t deg = J->off[v + 1] - J->off[v];
      a = hub_cap(deg);
      u = (deg + HUB_CHUNK - 1) / HUB_CHUNK;
      s = (a + HUB_SCHUNK - 1) / HUB_SCHUNK;
      h.stay[i] = 0;
      h.iso_seen[i] = 0;
    }
    s_a[tid] = a; s_b[tid] = u; s_c[tid] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int64_t xa = 0, xb = 0, xc = 0;
      if (tid >= o) { xa = s_a[tid - o]; xb = s_b[tid - o]; xc = s_c[tid - o]; }
      __syncthreads();
      s_a[tid] += xa; s_b[tid] += xb; s_c[tid] += xc;
      __syncthreads();
    }
    if (i < H) {
      h.tbl_off[i] = run_a + s_a[tid] - a;
      h.unit_off[i] = run_b + s_b[tid] - u;
      h.sunit_off[i] = run_c + s_c[tid] - s;
    }
    __syncthreads();
    if (tid == 1023) { run_a += s_a[1023]; run_b += s_b[1023]; run_c += s_c[1023]; }
    __syncthreads();
  }
  if (tid == 0) {
    if (run_c > h.max_sunits) {
      atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
      H = 0;
      run_a = run_b = run_c = 0;
    }
    h.tbl_off[H] = run_a;
    h.unit_off[H] = run_b;
    h.sunit_off[H] = run_c;
    ctr[C_HUBS] = H;
  }
}

// First hub whose table starts at or after slot x.
__device__ __forceinline__ int64_t hub_lower(const int64_t *__restrict__ tbl_off, int64_t H,
                                             int64_t x) {
  int64_t lo = 0, hi = H;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (tbl_off[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_hub_clear(HubBufs h, const int64_t *ctr, int64_t lo) {
  const int64_t H = ctr[C_HUBS];
  const int64_t h1 = hub_lower(h.tbl_off, H, lo + h.window);
  const int64_t h0 = hub_lower(h.tbl_off, H, lo);
  if (h0 >= h1) return;
  const int64_t s0 = h.tbl_off[h0] - lo, s1 = h.tbl_off[h1] - lo;
  for (int64_t i = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s1;
       i += (int64_t)gridDim.x * blockDim.x) {
    h.keys[i] = SLOT_EMPTY;
    h.vals[i] = 0;
  }
}

__global__ void __launch_bounds__(256) k_hub_insert(const JobDev *__restrict__ jobs, Buckets b,
                                                    HubBufs h, int64_t *ctr, int64_t lo) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t H = ctr[C_HUBS];
  if (H == 0) return;
  const int64_t h0 = hub_lower(h.tbl_off, H, lo);
  const int64_t h1 = hub_lower(h.tbl_off, H, lo + h.window);
  if (h0 >= h1) return;
  const int64_t U0 = h.unit_off[h0], U1 = h.unit_off[h1];
  const uint64_t *items = h.list ? h.list : b.items + b.seg_start[B_HUB];
  bool fail = false;
  for (int64_t u = U0 + blockIdx.x; u < U1; u += gridDim.x) {
    const int hh = find_seg(h.unit_off, H, u);
    const uint64_t item = items[hh];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J.off[v];
    const int64_t deg = J.off[v + 1] - beg;
    const int64_t cap = hub_cap(deg);
    unsigned long long *tkey = h.keys + (h.tbl_off[hh] - lo);
    unsigned long long *tval = (unsigned long long *)(h.vals + (h.tbl_off[hh] - lo));
    auto at = [tkey, tval](uint32_t s, unsigned long long *&kp, unsigned long long *&vp) {
      kp = tkey + s;
      vp = tval + s;
    };
    const int64_t e_lo = (u - h.unit_off[hh]) * HUB_CHUNK;
    int64_t e_hi = e_lo + HUB_CHUNK;
    if (e_hi > deg) e_hi = deg;
    Chunk<HUB_CHUNK / 256> x;
    load_chunk(J, beg, e_lo, e_hi, 256, tid, x);
    if (__any_sync(FULL, x.mv != 0) && lane == 0) atomicOr(&h.iso_seen[hh], 2);
    fail |= !insert_chunk(x, at, AnyCap((uint32_t)cap));
  }
  if (__any_sync(FULL, fail) && lane == 0)
    atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
}

template <typename S>
__global__ void __launch_bounds__(256) k_hub_score(const JobDev *__restrict__ jobs, Buckets b,
                                                   HubBufs h, int64_t *ctr, int64_t lo) {
  __shared__ S red_s[8];
  __shared__ int32_t red_c[8];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int64_t H = ctr[C_HUBS];
  if (H == 0) return;
  const int64_t h0 = hub_lower(h.tbl_off, H, lo);
  const int64_t h1 = hub_lower(h.tbl_off, H, lo + h.window);
  if (h0 >= h1) return;
  const int64_t SU0 = h.sunit_off[h0], SU1 = h.sunit_off[h1];
  const uint64_t *items = h.list ? h.list : b.items + b.seg_start[B_HUB];
  long long ncand = 0;
  for (int64_t su = SU0 + blockIdx.x; su < SU1; su += gridDim.x) {
    const int hh = find_seg(h.sunit_off, H, su);
    const uint64_t item = items[hh];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t deg = J.off[v + 1] - J.off[v];
    const int64_t cap = hub_cap(deg);
    const int32_t Lv = J.L[v];
    const int64_t kv = J.k[v];
    const unsigned long long *tkey = h.keys + (h.tbl_off[hh] - lo);
    const unsigned long long *tval = (const unsigned long long *)(h.vals + (h.tbl_off[hh] - lo));
    const int64_t s_lo = (su - h.sunit_off[hh]) * HUB_SCHUNK;
    int64_t s_hi = s_lo + HUB_SCHUNK;
    if (s_hi > cap) s_hi = cap;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    long long w_stay = 0;
    int vseen = 0;
    scan_slots<S>(J, tkey, tval, s_lo + tid, s_hi, 256, v, Lv, kv, best, bc, w_stay, vseen,
                  ncand);
    if (w_stay) atomicAdd((unsigned long long *)&h.stay[hh], (unsigned long long)w_stay);
    if (vseen) atomicOr(&h.iso_seen[hh], 1);
    warp_argmax<S>(best, bc);
    if (lane == 0) { red_s[wib] = best; red_c[wib] = bc; }
    __syncthreads();
    if (wib == 0) {
      S bs = lane < 8 ? red_s[lane] : ScoreOps<S>::lowest();
      int32_t bcc = lane < 8 ? red_c[lane] : INT32_MAX;
      warp_argmax<S>(bs, bcc);
      if (lane == 0) {
        h.part_score[su] = (i128)bs;
        h.part_cid[su] = bcc;
      }
    }
    __syncthreads();
  }
  ncand = warp_sum_ll(ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
}

template <typename S>
__global__ void __launch_bounds__(256) k_hub_final(const JobDev *__restrict__ jobs, Buckets b,
                                                   HubBufs h, int64_t *ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t H = ctr[C_HUBS];
  const uint64_t *items = h.list ? h.list : b.items + b.seg_start[B_HUB];
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  PullCount::init();
  for (int64_t hh = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); hh < H;
       hh += warps_total) {
    const uint64_t item = items[hh];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    for (int64_t su = h.sunit_off[hh] + lane; su < h.sunit_off[hh + 1]; su += 32) {
      const S s = (S)h.part_score[su];
      const int32_t c = h.part_cid[su];
      if (better<S>(s, c, best, bc)) { best = s; bc = c; }
    }
    warp_argmax<S>(best, bc);
    if (lane == 0) {
      const int32_t Lv = J.L[v];
      const int fl = h.iso_seen[hh];
      write_desired<S>(J, v, J.off[v + 1] - J.off[v], Lv, J.k[v], own_weight(J, v, Lv), best,
                       bc, (long long)h.stay[hh], (fl & 1) != 0, (fl & 2) != 0);
    }
  }
  PullCount::flush(ctr);
}

// ------------------------- long rows: hash-partitioned shared-memory merges ----

// Rows of the buckets from P.seg0 up (a tuning).  A row's entries are split
// by a hash of their cluster into P parts, so that every cluster of the row
// lies in exactly one part; each part is then merged in one block's
// shared-memory table with no cluster barrier, no remote atomic and no
// global table, and the parts' best candidates are reduced per row.
// A part whose distinct clusters overflow the table (possible only when many
// clusters collide in the partition hash) marks its row, and such rows go
// through the global-table hub kernels instead.

// Part of cluster c among np parts: a multiplicative hash independent of the
// one that places clusters in a part's table.
__device__ __forceinline__ int part_of(int32_t c, int64_t np) {
  const uint32_t h = (uint32_t)(((uint64_t)(uint32_t)c * 0xD6E8FEB86659FD93ull) >> 32);
  return (int)(((uint64_t)h * (uint64_t)np) >> 32);
}

// One thread per row slot i <= max_rows: the row's item and its counts of
// parts, chunks and cells (zero past the round's rows), scanned afterwards
// into offsets.
__global__ void __launch_bounds__(256) k_part_fill(const JobDev *__restrict__ jobs, Buckets b,
                                                   PartBufs P, int64_t *ctr) {
  const int nseg = B_HUB - P.seg0 + 1;
  int64_t seg_o[NPB + 1];
  int64_t H = 0;
  for (int k = 0; k < nseg; ++k) {
    seg_o[k] = H;
    H += seg_count(b, P.seg0 + k);
  }
  seg_o[nseg] = H;
  if (H > P.max_rows) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
      atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
    H = P.max_rows;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *P.nrows = H;
    *P.nfallback = 0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= P.max_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = 0, u = 0;
    if (i < H) {
      int k = 0;
      while (i >= seg_o[k + 1]) ++k;
      const uint64_t item = b.items[b.seg_start[P.seg0 + k] + (i - seg_o[k])];
      const JobDev *J = jobs + (int)(item >> 32);
      const int32_t v = (int32_t)(uint32_t)item;
      const int64_t deg = J->off[v + 1] - J->off[v];
      a = part_count_of(deg);
      u = part_chunks_of(deg);
      P.row[i] = item;
      P.stay[i] = 0;
      P.flag[i] = 0;
    }
    P.part_off[i] = a;
    P.chunk_off[i] = u;
    P.cell_off[i] = a * u;
  }
}

// One warp per row: the row of each of its chunks (so that a chunk finds its
// row with one load instead of a search).
__global__ void __launch_bounds__(256) k_part_index(PartBufs P) {
  const int lane = threadIdx.x & 31;
  const int64_t H = *P.nrows;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t h = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); h < H;
       h += warps_total)
    for (int64_t u = P.chunk_off[h] + lane; u < P.chunk_off[h + 1]; u += 32)
      P.chunk_row[u] = (int32_t)h;
}

// Count (SCATTER = false) or scatter (true) pass over chunks of PART_CH
// entries of the rows of more than one part: each entry's part from its
// cluster.  The count pass writes the chunk's entries per part into
// cells[cell_off[h] + part * C + chunk] (part major, so that the scan groups
// each row's entries by part, chunks in order) and notes a moved neighbour;
// the scatter pass writes each entry to its part's run at the scanned cell
// plus its rank in the chunk.  With few parts, the lanes of a warp that hold
// the same part take their ranks from one shared atomic.
constexpr int PC_T = 256, PC_E = 4;  // a chunk in PART_CH / (PC_T * PC_E) sub-batches

template <bool SCATTER>
__global__ void __launch_bounds__(PC_T, 8) k_part_chunks(const JobDev *__restrict__ jobs, PartBufs P) {
  __shared__ int s_h[PART_MAXP];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t H = *P.nrows;
  if (H == 0) return;
  const int64_t NC = P.chunk_off[H];
  for (int64_t u = blockIdx.x; u < NC; u += gridDim.x) {
    const int64_t h = P.chunk_row[u];
    const uint64_t item = P.row[h];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J.off[v];
    const int64_t deg = J.off[v + 1] - beg;
    const int64_t np = P.part_off[h + 1] - P.part_off[h];
    const int64_t C = P.chunk_off[h + 1] - P.chunk_off[h];
    const int64_t ci = u - P.chunk_off[h];
    const int64_t lo = ci * PART_CH;
    const int64_t hi = lo + PART_CH < deg ? lo + PART_CH : deg;
    const bool agg = np <= 256;  // the same for the whole block
    const int64_t cb = P.cell_off[h] + ci;
    for (int p = tid; p < (int)np; p += PC_T) s_h[p] = 0;
    __syncthreads();
    uint32_t mv = 0;
    // ranks in the chunk are running counts, so each sub-batch is written
    // as soon as its ranks are known
    for (int64_t s0 = lo; s0 < hi; s0 += PC_T * PC_E) {
      const int64_t s1 = s0 + PC_T * PC_E < hi ? s0 + PC_T * PC_E : hi;
      Chunk<PC_E> x;
      load_chunk<PC_E, SCATTER>(J, beg, s0, s1, PC_T, tid, x);
      mv |= x.mv;
      int part[PC_E], rk[PC_E];
#pragma unroll
      for (int i = 0; i < PC_E; ++i) part[i] = x.c[i] >= 0 ? part_of(x.c[i], np) : -1;
      if (agg) {
#pragma unroll
        for (int i = 0; i < PC_E; ++i) {
          const unsigned peers = __match_any_sync(FULL, part[i]);
          const int leader = __ffs(peers) - 1;
          int base = 0;
          if (lane == leader && part[i] >= 0) base = atomicAdd(&s_h[part[i]], __popc(peers));
          base = __shfl_sync(FULL, base, leader);
          rk[i] = base + __popc(peers & ((1u << lane) - 1u));
        }
      } else {
#pragma unroll
        for (int i = 0; i < PC_E; ++i) rk[i] = part[i] >= 0 ? atomicAdd(&s_h[part[i]], 1) : 0;
      }
      if (SCATTER) {
#pragma unroll
        for (int i = 0; i < PC_E; ++i) {
          if (part[i] < 0) continue;
          const int64_t pos = P.cells[cb + (int64_t)part[i] * C] + rk[i];
          P.pword[pos] = slot_word(x.c[i], x.k[i]);
          P.pw[pos] = x.w[i];
        }
      }
    }
    const int anymv = __syncthreads_or(mv != 0);
    if (!SCATTER) {
      for (int p = tid; p < (int)np; p += PC_T) P.cells[cb + (int64_t)p * C] = s_h[p];
      if (tid == 0 && anymv) atomicOr(&P.flag[h], 2);
    }
    __syncthreads();  // s_h is rebuilt for the next chunk
  }
}

// One warp per row, after the scan of the count cells: each part's run of
// entries and its row in one 16-byte descriptor.
__global__ void __launch_bounds__(256) k_part_desc(PartBufs P) {
  const int lane = threadIdx.x & 31;
  const int64_t H = *P.nrows;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t h = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); h < H;
       h += warps_total) {
    const int64_t p0 = P.part_off[h], np = P.part_off[h + 1] - p0;
    const int64_t C = P.chunk_off[h + 1] - P.chunk_off[h];
    const int64_t cb = P.cell_off[h];
    for (int64_t pi = lane; pi < np; pi += 32) {
      const int64_t st = P.cells[cb + pi * C];
      PartDesc d;
      d.st = st;
      d.cnt = (int32_t)(P.cells[cb + (pi + 1) * C] - st);
      d.h = (int32_t)h;
      P.desc[p0 + pi] = d;
    }
  }
}

// One part per block iteration (PART_T threads): its entries merged in a
// shared table of 3.25 slots per entry (at most table_slots <= PART_TP),
// scored, and the used slots emptied as they are read.  Two barriers per part:
// after the inserts, and after the scan (the per-warp results go to one of
// two buffers, so that warp 0 reduces them while the next part's inserts
// run).  Several blocks per SM keep independent parts in flight.
template <typename S>
__global__ void __launch_bounds__(PART_T, 3) k_part_merge(const JobDev *__restrict__ jobs,
                                                          PartBufs P, int64_t *ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = PART_T / 32, E = 4, STEP = PART_T * E;
  unsigned long long *tkey = (unsigned long long *)smem;
  unsigned long long *tval = tkey + PART_TP;
  __shared__ S red_s[2][NW];
  __shared__ int32_t red_c[2][NW];
  __shared__ long long red_w[2][NW];
  __shared__ int red_v[2][NW];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  for (int sl = tid; sl < PART_TP; sl += PART_T) {
    tkey[sl] = SLOT_EMPTY;
    tval[sl] = 0;
  }
  __syncthreads();  // the empty table
  const int64_t H = *P.nrows;
  const int64_t NP = H > 0 ? P.part_off[H] : 0;
  long long ncand = 0;
  auto at = [&](uint32_t sl, unsigned long long *&kp, unsigned long long *&vp) {
    kp = tkey + sl;
    vp = tval + sl;
  };
  int par = 0;
  // the next part's descriptor is loaded while the current part is merged
  PartDesc nd;
  if (blockIdx.x < NP) nd = P.desc[blockIdx.x];
  for (int64_t q = blockIdx.x; q < NP; q += gridDim.x) {
    const PartDesc d = nd;
    if (q + gridDim.x < NP) nd = P.desc[q + gridDim.x];
    const int64_t h = d.h;
    const uint64_t item = P.row[h];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    // the row's own label and weight are needed only when the part is scored
    const int32_t Lv = J.L[v];
    const int64_t kv = J.k[v];
    // 3.25 slots per entry (at most table_slots): few probes per insert
    int64_t cap = ((int64_t)d.cnt * 13 + 3) / 4;
    cap = (cap + 31) & ~(int64_t)31;
    if (cap < 32) cap = 32;
    if (cap > P.table_slots) cap = P.table_slots;
    const AnyCap geo((uint32_t)cap);
    // a part of at most two sub-batches keeps the slots its threads stored
    // first in registers and scores only those; a longer one scans the table
    const bool two = d.cnt <= 2 * STEP;
    uint32_t won0[E], won1[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      won0[i] = NOSLOT;
      won1[i] = NOSLOT;
    }
    bool fail = false;
    for (int64_t t0 = 0; t0 < d.cnt; t0 += STEP) {
      const int64_t t1 = t0 + STEP < d.cnt ? t0 + STEP : d.cnt;
      Chunk<E> x;
      x.mv = 0;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int64_t e = t0 + (int64_t)i * PART_T + tid;
        x.c[i] = -1;
        x.k[i] = KNONE;
        x.w[i] = 0;
        if (e < t1) {
          const unsigned long long wd =
              (unsigned long long)ld_stream((const int64_t *)(P.pword + d.st + e));
          x.c[i] = (int32_t)(uint32_t)wd;
          x.k[i] = (uint32_t)(wd >> 32);
          x.w[i] = ld_stream(P.pw + d.st + e);
        }
      }
      if (!two)
        fail |= !insert_chunk(x, at, geo);
      else if (t0 == 0)
        fail |= !insert_chunk_won(x, at, geo, won0);
      else
        fail |= !insert_chunk_won(x, at, geo, won1);
    }
    fail = __syncthreads_or(fail) != 0;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    long long w_stay = 0;
    int vseen = 0;
    if (two) {
      scan_won<S, E>(J, won0, at, v, Lv, kv, best, bc, w_stay, vseen, ncand);
      scan_won<S, E>(J, won1, at, v, Lv, kv, best, bc, w_stay, vseen, ncand);
    } else {
      scan_slots_reset<S>(J, tkey, tval, tid, (int)cap, PART_T, v, Lv, kv, best, bc, w_stay,
                          vseen, ncand);
    }
    w_stay = warp_sum_ll(w_stay);
    const int vs = __any_sync(FULL, vseen);
    warp_argmax<S>(best, bc);
    if (lane == 0) {
      red_s[par][wib] = best;
      red_c[par][wib] = bc;
      red_w[par][wib] = w_stay;
      red_v[par][wib] = vs;
    }
    __syncthreads();  // the table is empty and the warps' results are in
    if (wib == 0) {
      S bs = lane < NW ? red_s[par][lane] : ScoreOps<S>::lowest();
      int32_t bcc = lane < NW ? red_c[par][lane] : INT32_MAX;
      long long ws = lane < NW ? red_w[par][lane] : 0;
      int vv = lane < NW ? red_v[par][lane] : 0;
      warp_argmax<S>(bs, bcc);
      ws = warp_sum_ll(ws);
      vv = __any_sync(FULL, vv);
      if (lane == 0) {
        P.part_score[q] = (i128)bs;
        P.part_cid[q] = bcc;
        if (ws) atomicAdd((unsigned long long *)&P.stay[h], (unsigned long long)ws);
        if (vv || fail) atomicOr(&P.flag[h], (vv ? 1 : 0) | (fail ? 4 : 0));
      }
    }
    par ^= 1;
  }
  ncand = warp_sum_ll(ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
}

// One warp per row: the best of its parts, then the
// decision; a row whose part overflowed goes to the fallback list for the
// global-table kernels.
template <typename S>
__global__ void __launch_bounds__(256) k_part_final(const JobDev *__restrict__ jobs, PartBufs P,
                                                    int64_t *ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t H = *P.nrows;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  PullCount::init();
  for (int64_t h = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); h < H;
       h += warps_total) {
    const int64_t q0 = P.part_off[h], q1 = P.part_off[h + 1];
    const uint64_t item = P.row[h];
    const JobView J = view_of(jobs + (int)(item >> 32));
    const int32_t v = (int32_t)(uint32_t)item;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const S sc = (S)P.part_score[q];
      const int32_t c = P.part_cid[q];
      if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
    }
    warp_argmax<S>(best, bc);
    if (lane == 0) {
      const int fl = P.flag[h];
      if (fl & 4) {
        const int64_t pos = (int64_t)atomicAdd((unsigned long long *)P.nfallback, 1ull);
        P.fallback[pos] = item;
      } else {
        const int32_t Lv = J.L[v];
        write_desired<S>(J, v, J.off[v + 1] - J.off[v], Lv, J.k[v], own_weight(J, v, Lv), best,
                         bc, (long long)P.stay[h], (fl & 1) != 0, (fl & 2) != 0);
      }
    }
  }
  PullCount::flush(ctr);
}

// ------------------------------------------------------------ dispatch ----

namespace {
template <typename K>
int occ_blocks(K kernel, int threads, size_t smem) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
  return nb > 0 ? nb : 1;
}

int grid_of_rows(int64_t n, const Dev &d) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)d.sms * 8) g = (int64_t)d.sms * 8;
  return (int)(g > 0 ? g : 1);
}

struct TableLaunch {
  int clusters = 0;  // clusters resident at once
  bool init = false;
};

template <typename S, int CS, int THREADS, int TP, int E, int CH, bool POW2, int BK, bool PF = false>
void launch_table(const JobDev *jobs, const Buckets &b, int64_t *ctr, cudaStream_t st,
                  TableLaunch &tl, int *launches) {
  auto kern = k_bm_table<S, CS, THREADS, TP, E, CH, POW2, BK, PF>;
  const size_t smem = (size_t)TP * 16;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!tl.init) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (CS > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cfg.gridDim = dim3(CS);
    int ncl = 0;
    cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
    tl.clusters = ncl > 0 ? ncl : 1;
    tl.init = true;
  }
  int64_t ncl = tl.clusters;
  if (b.seg_cap[BK] < ncl) ncl = b.seg_cap[BK];
  cfg.gridDim = dim3((unsigned)(ncl * CS));
  cudaLaunchKernelEx(&cfg, kern, jobs, b, ctr);
  ++*launches;
}

template <typename S>
void bestmove_impl(const JobDev *jobs, const Buckets &b, const HubBufs &h, int64_t hub_passes,
                   int64_t *ctr, cudaStream_t st, const Dev &d, int *launches, cudaEvent_t *ev,
                   bool fuse_small, bool prefetch, const PartBufs *pb) {
  auto mark = [&](int bk) {
    if (ev) cudaEventRecord(ev[bk], st);
  };
  static int occ[10] = {0};
  static bool init = false;
  static TableLaunch tl[9], tlp[4];
  if (!init) {
    occ[0] = occ_blocks(k_bm_group<4, S>, 256, 0);
    occ[1] = occ_blocks(k_bm_group<8, S>, 256, 0);
    occ[2] = occ_blocks(k_bm_group<16, S>, 256, 0);
    occ[3] = occ_blocks(k_bm_group<32, S>, 256, 0);
    occ[9] = occ_blocks(k_bm_small<S>, 256, 0);
    occ[7] = occ_blocks(k_bm_warp<S, 2, B_W64>, 128, 0);
    occ[8] = occ_blocks(k_bm_warp<S, 4, B_W128>, 128, 0);
    occ[5] = occ_blocks(k_hub_insert, 256, 0);
    occ[6] = occ_blocks(k_hub_score<S>, 256, 0);
    init = true;
  }
  auto grid = [&](int bk, int o, int per_block) {
    const int64_t need = (b.seg_cap[bk] + per_block - 1) / per_block;
    int64_t g = (int64_t)d.sms * o;
    if (need < g) g = need;
    return (int)(g > 0 ? g : 1);
  };
  if (fuse_small) {
    // one resident launch for the four lane-group buckets, timed as <= 32
    const int64_t small = b.seg_cap[B_G4] + b.seg_cap[B_G8] + b.seg_cap[B_G16] + b.seg_cap[B_G32];
    mark(B_G4);
    mark(B_G8);
    mark(B_G16);
    if (small > 0) {
      int64_t g = (small + 63) / 64;
      if (g > (int64_t)d.sms * occ[9]) g = (int64_t)d.sms * occ[9];
      k_bm_small<S><<<(int)g, 256, 0, st>>>(jobs, b, ctr);
      ++*launches;
    }
    mark(B_G32);
  } else {
    if (b.seg_cap[B_G4] > 0) {
      k_bm_group<4, S><<<grid(B_G4, occ[0], 64), 256, 0, st>>>(jobs, b, B_G4, ctr);
      ++*launches;
    }
    mark(B_G4);
    if (b.seg_cap[B_G8] > 0) {
      k_bm_group<8, S><<<grid(B_G8, occ[1], 32), 256, 0, st>>>(jobs, b, B_G8, ctr);
      ++*launches;
    }
    mark(B_G8);
    if (b.seg_cap[B_G16] > 0) {
      k_bm_group<16, S><<<grid(B_G16, occ[2], 16), 256, 0, st>>>(jobs, b, B_G16, ctr);
      ++*launches;
    }
    mark(B_G16);
    if (b.seg_cap[B_G32] > 0) {
      k_bm_group<32, S><<<grid(B_G32, occ[3], 8), 256, 0, st>>>(jobs, b, B_G32, ctr);
      ++*launches;
    }
    mark(B_G32);
  }
  if (b.seg_cap[B_W64] > 0) {
    k_bm_warp<S, 2, B_W64><<<grid(B_W64, occ[7], 4), 128, 0, st>>>(jobs, b, ctr);
    ++*launches;
  }
  mark(B_W64);
  if (b.seg_cap[B_W128] > 0) {
    k_bm_warp<S, 4, B_W128><<<grid(B_W128, occ[8], 4), 128, 0, st>>>(jobs, b, ctr);
    ++*launches;
  }
  mark(B_W128);
  if (b.seg_cap[B_WARP] > 0) {
    if (prefetch)
      launch_table<S, 1, 128, WARP_CAP, 2, 1, true, B_WARP, true>(jobs, b, ctr, st, tlp[0],
                                                                   launches);
    else
      launch_table<S, 1, 128, WARP_CAP, 2, 1, true, B_WARP>(jobs, b, ctr, st, tl[7], launches);
  }
  mark(B_WARP);
  if (b.seg_cap[B_BLK] > 0) {
    if (prefetch)
      launch_table<S, 1, 256, TP_BLK, 4, 1, true, B_BLK, true>(jobs, b, ctr, st, tlp[1],
                                                                launches);
    else
      launch_table<S, 1, 256, TP_BLK, 4, 1, true, B_BLK>(jobs, b, ctr, st, tl[0], launches);
  }
  mark(B_BLK);
  // buckets from seg0 up go to the partitioned path
  const int seg0 = pb ? pb->seg0 : NB;
  if (B_T2K < seg0 && b.seg_cap[B_T2K] > 0) {
    if (prefetch)
      launch_table<S, 1, 512, TP_2K, 4, 1, true, B_T2K, true>(jobs, b, ctr, st, tlp[3],
                                                               launches);
    else
      launch_table<S, 1, 512, TP_2K, 4, 1, true, B_T2K>(jobs, b, ctr, st, tl[8], launches);
  }
  if (B_T2K < seg0) mark(B_T2K);
  if (B_T4K < seg0 && b.seg_cap[B_T4K] > 0) {
    if (prefetch)
      launch_table<S, 1, 1024, TP_4K, 4, 1, true, B_T4K, true>(jobs, b, ctr, st, tlp[2],
                                                                launches);
    else
      launch_table<S, 1, 1024, TP_4K, 4, 1, true, B_T4K>(jobs, b, ctr, st, tl[1], launches);
  }
  if (B_T4K < seg0) mark(B_T4K);
  if (B_T8K < seg0 && b.seg_cap[B_T8K] > 0)
    launch_table<S, 1, 1024, TP_8K, 4, 2, false, B_T8K>(jobs, b, ctr, st, tl[2], launches);
  if (B_T8K < seg0) mark(B_T8K);
  if (B_T16K < seg0 && b.seg_cap[B_T16K] > 0)
    launch_table<S, 2, 1024, TP_8K, 4, 2, false, B_T16K>(jobs, b, ctr, st, tl[3], launches);
  if (B_T16K < seg0) mark(B_T16K);
  if (B_T32K < seg0 && b.seg_cap[B_T32K] > 0)
    launch_table<S, 4, 1024, TP_8K, 4, 2, false, B_T32K>(jobs, b, ctr, st, tl[4], launches);
  if (B_T32K < seg0) mark(B_T32K);
  if (B_T64K < seg0 && b.seg_cap[B_T64K] > 0)
    launch_table<S, 8, 1024, TP_8K, 4, 2, false, B_T64K>(jobs, b, ctr, st, tl[5], launches);
  if (B_T64K < seg0) mark(B_T64K);
  if (B_T128K < seg0 && b.seg_cap[B_T128K] > 0)
    launch_table<S, 16, 1024, TP_8K, 4, 2, false, B_T128K>(jobs, b, ctr, st, tl[6], launches);
  if (B_T128K < seg0) mark(B_T128K);
  if (pb) {
    // hash-partitioned merges, then the global-table kernels for the rows
    // whose part overflowed
    static int occ_merge = 0;
    if (!occ_merge) {
      cudaFuncSetAttribute(k_part_merge<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           PART_TP * 16);
      int nb = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_part_merge<S>, PART_T, PART_TP * 16);
      occ_merge = nb > 0 ? nb : 1;
    }
    const int64_t R = pb->max_rows;
    k_part_fill<<<grid_of_rows(R + 1, d), 256, 0, st>>>(jobs, b, *pb, ctr);
    scan_exclusive_i64(pb->part_off, R, pb->scan_tmp, st, d);
    scan_exclusive_i64(pb->chunk_off, R, pb->scan_tmp, st, d);
    scan_exclusive_i64(pb->cell_off, R, pb->scan_tmp, st, d);
    const int64_t rg0 = (R + 7) / 8;
    const int rg = (int)(rg0 < (int64_t)d.sms * 8 ? rg0 : (int64_t)d.sms * 8);
    int64_t g = pb->max_chunks < (int64_t)d.sms * 8 ? pb->max_chunks : (int64_t)d.sms * 8;
    if (pb->max_chunks > 0) {
      cudaMemsetAsync(pb->cells, 0, (pb->max_cells + 1) * sizeof(int64_t), st);
      k_part_index<<<rg, 256, 0, st>>>(*pb);
      k_part_chunks<false><<<(int)g, PC_T, 0, st>>>(jobs, *pb);
      scan_exclusive_i64(pb->cells, pb->max_cells, pb->scan_tmp, st, d);
      k_part_chunks<true><<<(int)g, PC_T, 0, st>>>(jobs, *pb);
      *launches += 6;
    }
    k_part_desc<<<rg, 256, 0, st>>>(*pb);
    g = pb->max_parts < (int64_t)d.sms * occ_merge ? pb->max_parts : (int64_t)d.sms * occ_merge;
    k_part_merge<S><<<(int)(g > 0 ? g : 1), PART_T, PART_TP * 16, st>>>(jobs, *pb, ctr);
    k_part_final<S><<<rg, 256, 0, st>>>(jobs, *pb, ctr);
    *launches += 13;
    HubBufs hf = h;
    hf.list = pb->fallback;
    hf.list_cnt = pb->nfallback;
    k_hub_prep<<<1, 1024, 0, st>>>(jobs, b, hf, ctr);
    for (int64_t p = 0; p < hub_passes; ++p) {
      const int64_t lo = p * hf.window;
      k_hub_clear<<<d.sms * 8, 256, 0, st>>>(hf, ctr, lo);
      k_hub_insert<<<d.sms * occ[5], 256, 0, st>>>(jobs, b, hf, ctr, lo);
      k_hub_score<S><<<d.sms * occ[6], 256, 0, st>>>(jobs, b, hf, ctr, lo);
      *launches += 3;
    }
    k_hub_final<S><<<rg, 256, 0, st>>>(jobs, b, hf, ctr);
    *launches += 2;
    for (int bk = seg0; bk <= B_HUB; ++bk) mark(bk);
    return;
  }
  if (b.seg_cap[B_HUB] > 0) {
    k_hub_prep<<<1, 1024, 0, st>>>(jobs, b, h, ctr);
    for (int64_t p = 0; p < hub_passes; ++p) {
      const int64_t lo = p * h.window;
      k_hub_clear<<<d.sms * 8, 256, 0, st>>>(h, ctr, lo);
      k_hub_insert<<<d.sms * occ[5], 256, 0, st>>>(jobs, b, h, ctr, lo);
      k_hub_score<S><<<d.sms * occ[6], 256, 0, st>>>(jobs, b, h, ctr, lo);
      *launches += 3;
    }
    int64_t fg = (b.seg_cap[B_HUB] + 7) / 8;
    if (fg > d.sms * 4) fg = d.sms * 4;
    k_hub_final<S><<<(int)(fg > 0 ? fg : 1), 256, 0, st>>>(jobs, b, h, ctr);
    *launches += 2;
  }
  mark(B_HUB);
}
}  // namespace

void launch_bestmove(bool wide, const JobDev *jobs, const Buckets &b, const HubBufs &h,
                     int64_t hub_passes, int64_t *ctr, cudaStream_t st, const Dev &d,
                     int *launches, cudaEvent_t *ev, bool fuse_small, bool prefetch,
                     const PartBufs *pb) {
  if (wide)
    bestmove_impl<i128>(jobs, b, h, hub_passes, ctr, st, d, launches, ev, fuse_small, prefetch,
                        pb);
  else
    bestmove_impl<int64_t>(jobs, b, h, hub_passes, ctr, st, d, launches, ev, fuse_small,
                           prefetch, pb);
}

// --------------------------------------------------------------- apply ----

// Sum of any 64-bit value over the lanes of `peers` (every lane of peers).
__device__ __forceinline__ unsigned long long peers_sum64(unsigned peers, unsigned long long x) {
  unsigned long long t = 0;
  for (unsigned m = peers; m; m &= m - 1) t += __shfl_sync(peers, x, __ffs(m) - 1);
  return t;
}

// Moves every evaluated vertex to D[v] and keeps K in step (Algorithm 1).
// Per job: moves and the movers' entries in jmoves[2j], jmoves[2j + 1],
// summed per lane while the lane stays on one job.  Movers of JF_MARK_NBR
// jobs get fr = 2 and a place in the moved list (one global atomic per tile).
constexpr int AP_T = 256, AP_V = 4;

__global__ void __launch_bounds__(AP_T) k_apply(const JobDev *__restrict__ jobs, Buckets b,
                                                int64_t *jmoves, uint64_t *moved,
                                                int64_t moved_cap, int64_t *ctr) {
  __shared__ unsigned t_cnt;
  __shared__ unsigned long long t_base;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) t_cnt = 0;
  __syncthreads();
  long long nmv = 0;
  int cur = -1;
  unsigned long long c_mv = 0, c_ents = 0;
  auto flush_lane = [&]() {
    if (cur >= 0 && c_mv) {
      atomicAdd((unsigned long long *)(jmoves + 2 * cur), c_mv);
      if (c_ents) atomicAdd((unsigned long long *)(jmoves + 2 * cur + 1), c_ents);
    }
    c_mv = c_ents = 0;
  };
  const int64_t tile = (int64_t)AP_T * AP_V;
  for (int bk = 0; bk < NB; ++bk) {
    const int64_t count = seg_count(b, bk);
    const uint64_t *items = b.items + b.seg_start[bk];
    for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < count; t0 += (int64_t)gridDim.x * tile) {
      unsigned place[AP_V];
      uint64_t mitem[AP_V];
#pragma unroll
      for (int r = 0; r < AP_V; ++r) {
        const int64_t i = t0 + (int64_t)r * AP_T + tid;
        bool mark = false;
        mitem[r] = 0;
        place[r] = ~0u;
        if (i < count) {
          const uint64_t item = items[i];
          const int j = (int)(item >> 32);
          const JobDev *J = jobs + j;
          const int32_t v = (int32_t)(uint32_t)item;
          if (!(J->flags & JF_EVAL_ONLY)) {
            const int32_t dv = J->D[v];
            const int32_t lv = J->L[v];
            if (dv != lv) {
              const int64_t kv = J->k[v];
              J->L[v] = dv;
              if (kv) {
                atomic_add_i64(J->K + lv, -kv);
                atomic_add_i64(J->K + dv, kv);
              }
              if (J->flags & JF_MARK_CL) J->cl[lv] = 1;
              int64_t deg = 0;
              if (J->flags & JF_MARK_NBR) {
                mark = true;
                mitem[r] = item;
                J->fr[v] = 2;  // moved: read by the frontier kernel when the next round pulls
                deg = J->off[v + 1] - J->off[v];
              }
              if (j != cur) {
                flush_lane();
                cur = j;
              }
              c_mv += 1;
              c_ents += (unsigned long long)deg;
              nmv += 1;
            }
          }
        }
        const unsigned mb = __ballot_sync(FULL, mark);
        if (mb) {
          unsigned p0 = 0;
          if (lane == __ffs(mb) - 1) p0 = atomicAdd(&t_cnt, (unsigned)__popc(mb));
          p0 = __shfl_sync(FULL, p0, __ffs(mb) - 1);
          if (mark) place[r] = p0 + __popc(mb & lanemask_lt());
        }
      }
      __syncthreads();
      if (tid == 0) {
        t_base = t_cnt ? atomicAdd((unsigned long long *)&ctr[C_MOVED_N],
                                   (unsigned long long)t_cnt)
                       : 0ull;
        t_cnt = 0;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < AP_V; ++r) {
        if (place[r] == ~0u) continue;
        const int64_t pos = (int64_t)(t_base + place[r]);
        if (pos < moved_cap)
          moved[pos] = mitem[r];
        else
          atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_MOVED_OVERFLOW);
      }
    }
  }
  // per-job sums: one atomic per warp and job where the lanes agree
  const unsigned peers = __match_any_sync(FULL, c_mv ? cur : -1);
  const unsigned long long s_mv = peers_sum64(peers, c_mv);
  const unsigned long long s_ents = peers_sum64(peers, c_ents);
  if (c_mv && lane == __ffs(peers) - 1) {
    atomicAdd((unsigned long long *)(jmoves + 2 * cur), s_mv);
    if (s_ents) atomicAdd((unsigned long long *)(jmoves + 2 * cur + 1), s_ents);
  }
  nmv = warp_sum_ll(nmv);
  if (lane == 0 && nmv) atomicAdd((unsigned long long *)&ctr[C_MOVES], (unsigned long long)nmv);
}

void launch_apply(const JobDev *jobs, const Buckets &b, int64_t *jmoves, uint64_t *moved,
                  int64_t moved_cap, int64_t *ctr, cudaStream_t st, const Dev &d) {
  int64_t tot = 0;
  for (int i = 0; i < NB; ++i) tot += b.seg_cap[i];
  if (tot == 0) return;
  const int64_t tile = (int64_t)AP_T * AP_V;
  int64_t g = (tot + tile - 1) / tile;
  if (g > d.sms * 8) g = d.sms * 8;
  k_apply<<<(int)g, AP_T, 0, st>>>(jobs, b, jmoves, moved, moved_cap, ctr);
}

// ---------------------------------------------------------------- mark ----

// V' <- neighbours of the moved vertices (Algorithm 1 / Sec. 3.2.2).  Jobs
// whose movers hold at least pull_min entries skip the marking: their next
// round runs with JF_PULL (the host takes the same decision from jmoves).
__global__ void __launch_bounds__(256) k_mark_nbr(const JobDev *__restrict__ jobs,
                                                  const uint64_t *__restrict__ moved,
                                                  const int64_t *ctr, const int64_t *jmoves,
                                                  int64_t moved_cap) {
  const int lane = threadIdx.x & 31;
  int64_t M = ctr[C_MOVED_N];
  if (M > moved_cap) M = moved_cap;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < M;
       i += warps_total) {
    const uint64_t item = moved[i];
    const int j = (int)(item >> 32);
    const JobDev *J = jobs + j;
    if (jmoves[2 * j + 1] >= J->pull_min) continue;
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J->off[v], end = J->off[v + 1];
    for (int64_t e = beg + lane; e < end; e += 32) J->fr[__ldg(J->nbr + e)] = 1;
  }
}

// V' <- neighbours of every vertex now in a cluster some vertex moved out of.
__global__ void __launch_bounds__(256) k_mark_cl(const JobDev *__restrict__ jobs,
                                                 const int64_t *__restrict__ vstart, int njobs,
                                                 int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const JobDev *J = jobs + j;
    if (!(J->flags & JF_MARK_CL)) continue;
    const int64_t x = i - vstart[j];
    if (!J->cl[J->L[x]]) continue;
    for (int64_t e = J->off[x]; e < J->off[x + 1]; ++e) J->fr[J->nbr[e]] = 1;
  }
}

__global__ void k_clear_cl(const JobDev *__restrict__ jobs, const int64_t *__restrict__ vstart,
                           int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const JobDev *J = jobs + j;
    if (J->flags & JF_MARK_CL) J->cl[i - vstart[j]] = 0;
  }
}

void launch_mark(const JobDev *jobs, const uint64_t *moved, int64_t *ctr, const int64_t *jmoves,
                 bool any_cl, const int64_t *vstart, int njobs, int64_t vtot, cudaStream_t st,
                 const Dev &d, int *launches) {
  k_mark_nbr<<<d.sms * 8, 256, 0, st>>>(jobs, moved, ctr, jmoves, vtot);
  ++*launches;
  if (any_cl && vtot > 0) {
    int64_t g = (vtot + 255) / 256;
    if (g > d.sms * 8) g = d.sms * 8;
    k_mark_cl<<<(int)g, 256, 0, st>>>(jobs, vstart, njobs, vtot);
    k_clear_cl<<<(int)g, 256, 0, st>>>(jobs, vstart, njobs, vtot);
    *launches += 2;
  }
}

}  // namespace lcc
