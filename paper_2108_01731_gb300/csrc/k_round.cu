// Kernels of one synchronous Best-Moves round (Algorithm 1, Sec. 3.2.1).
//
//   k_frontier  builds V' (Sec. 3.2.2) as per-degree-bucket work lists;
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
#include "lcc_internal.cuh"

namespace lcc {

namespace {
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t slot_of(int32_t c, int lg) {
  uint64_t h = (uint64_t)(uint32_t)c * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(h >> (64 - lg));
}

__device__ __forceinline__ int log2i(int64_t pow2) { return 63 - __clzll((long long)pow2); }

__device__ __forceinline__ int64_t seg_count(const Buckets &b, int bk) {
  int64_t c = b.cnt[bk];
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
    S os = ScoreOps<S>::shfl_xor(s, o, 32);
    int32_t oc = __shfl_xor_sync(FULL, c, o);
    if (better<S>(os, oc, s, c)) { s = os; c = oc; }
  }
}

// Final decision of one vertex: the empty cluster id v (reading of the
// paper's silence on empty clusters), then the strict comparison with staying.
template <typename S>
__device__ __forceinline__ int32_t decide(const JobDev *J, int32_t v, int32_t Lv, int64_t kv,
                                          S best, int32_t bc, long long w_stay, bool v_seen) {
  const S p = (S)J->p, q = (S)J->q;
  if (Lv != v && !v_seen && J->K[v] == 0) {
    if (better<S>((S)0, v, best, bc)) { best = 0; bc = v; }
  }
  const S stay = q * (S)w_stay - p * (S)kv * ((S)J->K[Lv] - (S)kv);
  return (bc != INT32_MAX && best > stay) ? bc : Lv;
}
}  // namespace

// ---------------------------------------------------------------- V' -----

__global__ void __launch_bounds__(256) k_frontier(const JobDev *__restrict__ jobs,
                                                  const int64_t *__restrict__ vstart, int njobs,
                                                  int64_t vtot, Buckets b, int64_t *ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  long long my_deg = 0, my_cnt = 0, my_wb = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < vtot;
       base += stride) {
    const int64_t i = base + lane;
    int bk = -1;
    uint64_t item = 0;
    if (i < vtot) {
      const int j = find_job(vstart, njobs, i);
      const JobDev *J = jobs + j;
      const int64_t v = i - vstart[j];
      bool f = (J->flags & JF_ALL) != 0;
      if (J->fr[v]) {
        J->fr[v] = 0;
        f = true;
      }
      if (f) {
        const int64_t deg = J->off[v + 1] - J->off[v];
        // A vertex with no neighbour in its own singleton has no candidate.
        if (!(deg == 0 && J->L[v] == (int32_t)v)) {
          bk = bucket_of(deg);
          item = ((uint64_t)(uint32_t)j << 32) | (uint32_t)v;
          my_deg += deg;
          my_cnt += 1;
          my_wb += deg * (J->wtype == W_I32 ? 4 : (J->wtype == W_I64 ? 8 : 0));
        }
      }
    }
    const unsigned active = __ballot_sync(FULL, bk >= 0);
    if (active) {
      const unsigned peers = __match_any_sync(FULL, bk);
      if (bk >= 0) {
        const int leader = __ffs(peers) - 1;
        unsigned long long basepos = 0;
        if (lane == leader)
          basepos = atomicAdd((unsigned long long *)&b.cnt[bk], (unsigned long long)__popc(peers));
        basepos = __shfl_sync(peers, basepos, leader);
        const int64_t pos = (int64_t)basepos + __popc(peers & lanemask_lt());
        if (pos < b.seg_cap[bk])
          b.items[b.seg_start[bk] + pos] = item;
        else
          atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_BUCKET_OVERFLOW);
      }
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
}

void launch_frontier(const JobDev *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                     const Buckets &b, int64_t *ctr, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  int64_t blocks = (vtot + 255) / 256;
  int64_t maxb = (int64_t)d.sms * 8;
  if (blocks > maxb) blocks = maxb;
  k_frontier<<<(int)blocks, 256, 0, st>>>(jobs, vstart, njobs, vtot, b, ctr);
}

// ------------------------------------------------ deg <= G: G lanes/vertex --

// Each group of G lanes takes one vertex; lane t reads edge t.  Equal
// clusters are found with __match_any_sync on (group, cluster) and summed
// into the group leader's shared slot; the leaders' scores are then reduced
// inside the group with xor-shuffles of width G.
template <int G, typename S>
__global__ void __launch_bounds__(256) k_bm_group(const JobDev *__restrict__ jobs, Buckets b,
                                                  int bk, int64_t *ctr) {
  __shared__ unsigned long long acc[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gl = lane & (G - 1);
  const int gsub = lane / G;
  constexpr int GPW = 32 / G;
  const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (gsub * G));
  const int64_t count = seg_count(b, bk);
  const uint64_t *items = b.items + b.seg_start[bk];
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  long long ncand = 0;
  for (int64_t wbase = gw * GPW; wbase < count; wbase += warps_total * GPW) {
    const int64_t it = wbase + gsub;
    const bool valid = it < count;
    const uint64_t item = valid ? items[it] : 0ull;
    const JobDev *J = jobs + (int)(item >> 32);
    const int32_t v = (int32_t)(uint32_t)item;
    int64_t beg = 0;
    int deg = 0;
    int32_t Lv = 0;
    int64_t kv = 0;
    if (valid) {
      beg = J->off[v];
      deg = (int)(J->off[v + 1] - beg);
      Lv = J->L[v];
      kv = J->k[v];
    }
    const bool has = valid && gl < deg;
    int32_t c = -1;
    long long wt = 0;
    if (has) {
      const int32_t u = __ldg(J->nbr + beg + gl);
      wt = load_w(J->w, J->wtype, beg + gl);
      c = J->L[u];
    }
    const unsigned long long key = ((unsigned long long)gsub << 32) | (uint32_t)c;
    const unsigned peers = __match_any_sync(FULL, key);
    const int leader = __ffs(peers) - 1;
    acc[wib][lane] = 0;
    __syncwarp();
    if (has) atomicAdd(&acc[wib][leader], (unsigned long long)wt);
    __syncwarp();
    const long long wsum = (long long)acc[wib][lane];
    __syncwarp();
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
      score = (S)J->q * (S)wsum - (S)J->p * (S)kv * (S)J->K[c];
      cid = c;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const S os = ScoreOps<S>::shfl_xor(score, o, G);
      const int32_t oc = __shfl_xor_sync(FULL, cid, o, G);
      if (better<S>(os, oc, score, cid)) { score = os; cid = oc; }
    }
    if (valid && gl == 0) J->D[v] = decide<S>(J, v, Lv, kv, score, cid, w_stay, v_seen);
    ncand += __popc(__ballot_sync(FULL, cand));
  }
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
}

// ----------------------------------- deg <= T_WARP: warp + shared table --

// Inserts (c, sum) into an open-addressing table (linear probing).  The
// table has at least twice as many slots as keys, so a free or matching slot
// is always found within `cap` probes.
__device__ __forceinline__ bool table_insert(int32_t *tkey, unsigned long long *tval, int cap,
                                             int lg, int32_t c, long long sum) {
  uint32_t s = slot_of(c, lg);
  for (int t = 0; t < cap; ++t) {
    const int32_t prev = atomicCAS(tkey + s, -1, c);
    if (prev == -1 || prev == c) {
      atomicAdd(tval + s, (unsigned long long)sum);
      return true;
    }
    s = (s + 1) & (uint32_t)(cap - 1);
  }
  return false;
}

template <typename S>
__global__ void __launch_bounds__(128) k_bm_warp(const JobDev *__restrict__ jobs, Buckets b,
                                                 int64_t *ctr) {
  constexpr int WPB = 4;
  __shared__ int32_t tkey[WPB][WARP_CAP];
  __shared__ unsigned long long tval[WPB][WARP_CAP];
  __shared__ unsigned long long acc[WPB][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t count = seg_count(b, B_WARP);
  const uint64_t *items = b.items + b.seg_start[B_WARP];
  const int64_t warps_total = (int64_t)gridDim.x * WPB;
  long long ncand = 0;
  bool fail = false;
  for (int64_t it = (int64_t)blockIdx.x * WPB + wib; it < count; it += warps_total) {
    const uint64_t item = items[it];
    const JobDev *J = jobs + (int)(item >> 32);
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J->off[v];
    const int deg = (int)(J->off[v + 1] - beg);
    const int32_t Lv = J->L[v];
    const int64_t kv = J->k[v];
    const int cap = (int)next_pow2(2 * (int64_t)deg);
    const int lg = log2i(cap);
    for (int s = lane; s < cap; s += 32) {
      tkey[wib][s] = -1;
      tval[wib][s] = 0;
    }
    __syncwarp();
    for (int e0 = 0; e0 < deg; e0 += 32) {
      const int e = e0 + lane;
      const bool has = e < deg;
      int32_t c = -1;
      long long wt = 0;
      if (has) {
        c = J->L[__ldg(J->nbr + beg + e)];
        wt = load_w(J->w, J->wtype, beg + e);
      }
      const unsigned peers = __match_any_sync(FULL, c);
      const int leader = __ffs(peers) - 1;
      acc[wib][lane] = 0;
      __syncwarp();
      if (has) atomicAdd(&acc[wib][leader], (unsigned long long)wt);
      __syncwarp();
      if (has && lane == leader)
        fail |= !table_insert(tkey[wib], tval[wib], cap, lg, c, (long long)acc[wib][lane]);
      __syncwarp();
    }
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    long long w_stay = 0;
    int vseen = 0, nc = 0;
    for (int s = lane; s < cap; s += 32) {
      const int32_t c = tkey[wib][s];
      if (c < 0) continue;
      const long long val = (long long)tval[wib][s];
      if (c == Lv) { w_stay = val; continue; }
      vseen |= (c == v);
      ++nc;
      const S sc = (S)J->q * (S)val - (S)J->p * (S)kv * (S)J->K[c];
      if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
    }
    w_stay = warp_sum_ll(w_stay);
    const bool v_seen = __any_sync(FULL, vseen);
    ncand += nc;
    warp_argmax<S>(best, bc);
    if (lane == 0) J->D[v] = decide<S>(J, v, Lv, kv, best, bc, w_stay, v_seen);
    __syncwarp();
  }
  ncand = warp_sum_ll(ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
  if (__any_sync(FULL, fail) && lane == 0)
    atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
}

// ------------------------------ deg <= T_BLKx: block + shared table --------

template <typename S, int CAP, int THREADS, int BK>
__global__ void __launch_bounds__(THREADS) k_bm_block(const JobDev *__restrict__ jobs, Buckets b,
                                                      int64_t *ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NW = THREADS / 32;
  unsigned long long *tval = (unsigned long long *)smem;
  int32_t *tkey = (int32_t *)(smem + (size_t)CAP * 8);
  __shared__ unsigned long long acc[NW][32];
  __shared__ S red_s[NW];
  __shared__ int32_t red_c[NW];
  __shared__ long long red_w[NW];
  __shared__ int red_v[NW];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int64_t count = seg_count(b, BK);
  const uint64_t *items = b.items + b.seg_start[BK];
  long long ncand = 0;
  bool fail = false;
  for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
    const uint64_t item = items[it];
    const JobDev *J = jobs + (int)(item >> 32);
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J->off[v];
    const int deg = (int)(J->off[v + 1] - beg);
    const int32_t Lv = J->L[v];
    const int64_t kv = J->k[v];
    int cap = (int)next_pow2(2 * (int64_t)deg);
    if (cap > CAP) cap = CAP;
    const int lg = log2i(cap);
    for (int s = tid; s < cap; s += THREADS) {
      tkey[s] = -1;
      tval[s] = 0;
    }
    __syncthreads();
    for (int e0 = 0; e0 < deg; e0 += THREADS) {
      const int e = e0 + tid;
      const bool has = e < deg;
      int32_t c = -1;
      long long wt = 0;
      if (has) {
        c = J->L[__ldg(J->nbr + beg + e)];
        wt = load_w(J->w, J->wtype, beg + e);
      }
      const unsigned peers = __match_any_sync(FULL, c);
      const int leader = __ffs(peers) - 1;
      acc[wib][lane] = 0;
      __syncwarp();
      if (has) atomicAdd(&acc[wib][leader], (unsigned long long)wt);
      __syncwarp();
      if (has && lane == leader)
        fail |= !table_insert(tkey, tval, cap, lg, c, (long long)acc[wib][lane]);
      __syncwarp();
    }
    __syncthreads();
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    long long w_stay = 0;
    int vseen = 0, nc = 0;
    for (int s = tid; s < cap; s += THREADS) {
      const int32_t c = tkey[s];
      if (c < 0) continue;
      const long long val = (long long)tval[s];
      if (c == Lv) { w_stay = val; continue; }
      vseen |= (c == v);
      ++nc;
      const S sc = (S)J->q * (S)val - (S)J->p * (S)kv * (S)J->K[c];
      if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
    }
    w_stay = warp_sum_ll(w_stay);
    const int vs = __any_sync(FULL, vseen);
    ncand += nc;
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
      const bool vseen_all = __any_sync(FULL, vv);
      if (lane == 0) J->D[v] = decide<S>(J, v, Lv, kv, bs, bcc, ws, vseen_all);
    }
    __syncthreads();
  }
  ncand = warp_sum_ll(ncand);
  if (lane == 0 && ncand) atomicAdd((unsigned long long *)&ctr[C_CANDS], (unsigned long long)ncand);
  if (__any_sync(FULL, fail) && lane == 0)
    atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
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
  int64_t H = seg_count(b, B_HUB);
  if (H > h.max_hubs) {
    if (tid == 0) atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_HUB_OVERFLOW);
    H = h.max_hubs;
  }
  const uint64_t *items = b.items + b.seg_start[B_HUB];
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
    h.keys[i] = -1;
    h.vals[i] = 0;
  }
}

__global__ void __launch_bounds__(256) k_hub_insert(const JobDev *__restrict__ jobs, Buckets b,
                                                    HubBufs h, int64_t *ctr, int64_t lo) {
  __shared__ unsigned long long acc[8][32];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int64_t H = ctr[C_HUBS];
  if (H == 0) return;
  const int64_t h0 = hub_lower(h.tbl_off, H, lo);
  const int64_t h1 = hub_lower(h.tbl_off, H, lo + h.window);
  if (h0 >= h1) return;
  const int64_t U0 = h.unit_off[h0], U1 = h.unit_off[h1];
  const uint64_t *items = b.items + b.seg_start[B_HUB];
  bool fail = false;
  for (int64_t u = U0 + blockIdx.x; u < U1; u += gridDim.x) {
    const int hh = find_seg(h.unit_off, H, u);
    const uint64_t item = items[hh];
    const JobDev *J = jobs + (int)(item >> 32);
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t beg = J->off[v];
    const int64_t deg = J->off[v + 1] - beg;
    const int64_t cap = hub_cap(deg);
    const int lg = log2i(cap);
    int32_t *tkey = h.keys + (h.tbl_off[hh] - lo);
    unsigned long long *tval = (unsigned long long *)(h.vals + (h.tbl_off[hh] - lo));
    const int64_t e_lo = (u - h.unit_off[hh]) * HUB_CHUNK;
    int64_t e_hi = e_lo + HUB_CHUNK;
    if (e_hi > deg) e_hi = deg;
    for (int64_t e0 = e_lo; e0 < e_hi; e0 += 256) {
      const int64_t e = e0 + tid;
      const bool has = e < e_hi;
      int32_t c = -1;
      long long wt = 0;
      if (has) {
        c = J->L[__ldg(J->nbr + beg + e)];
        wt = load_w(J->w, J->wtype, beg + e);
      }
      const unsigned peers = __match_any_sync(FULL, c);
      const int leader = __ffs(peers) - 1;
      acc[wib][lane] = 0;
      __syncwarp();
      if (has) atomicAdd(&acc[wib][leader], (unsigned long long)wt);
      __syncwarp();
      if (has && lane == leader) {
        const long long sum = (long long)acc[wib][lane];
        uint64_t s = slot_of(c, lg);
        bool done = false;
        for (int64_t t = 0; t < cap; ++t) {
          const int32_t prev = atomicCAS(tkey + s, -1, c);
          if (prev == -1 || prev == c) {
            atomicAdd(tval + s, (unsigned long long)sum);
            done = true;
            break;
          }
          s = (s + 1) & (uint64_t)(cap - 1);
        }
        fail |= !done;
      }
      __syncwarp();
    }
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
  const uint64_t *items = b.items + b.seg_start[B_HUB];
  long long ncand = 0;
  for (int64_t su = SU0 + blockIdx.x; su < SU1; su += gridDim.x) {
    const int hh = find_seg(h.sunit_off, H, su);
    const uint64_t item = items[hh];
    const JobDev *J = jobs + (int)(item >> 32);
    const int32_t v = (int32_t)(uint32_t)item;
    const int64_t deg = J->off[v + 1] - J->off[v];
    const int64_t cap = hub_cap(deg);
    const int32_t Lv = J->L[v];
    const int64_t kv = J->k[v];
    const int32_t *tkey = h.keys + (h.tbl_off[hh] - lo);
    const int64_t *tval = h.vals + (h.tbl_off[hh] - lo);
    const int64_t s_lo = (su - h.sunit_off[hh]) * HUB_SCHUNK;
    int64_t s_hi = s_lo + HUB_SCHUNK;
    if (s_hi > cap) s_hi = cap;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    for (int64_t s = s_lo + tid; s < s_hi; s += 256) {
      const int32_t c = tkey[s];
      if (c < 0) continue;
      const long long val = tval[s];
      if (c == Lv) { h.stay[hh] = val; continue; }
      if (c == v) h.iso_seen[hh] = 1;
      ++ncand;
      const S sc = (S)J->q * (S)val - (S)J->p * (S)kv * (S)J->K[c];
      if (better<S>(sc, c, best, bc)) { best = sc; bc = c; }
    }
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
                                                   HubBufs h, const int64_t *ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t H = ctr[C_HUBS];
  const uint64_t *items = b.items + b.seg_start[B_HUB];
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t hh = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); hh < H;
       hh += warps_total) {
    const uint64_t item = items[hh];
    const JobDev *J = jobs + (int)(item >> 32);
    const int32_t v = (int32_t)(uint32_t)item;
    S best = ScoreOps<S>::lowest();
    int32_t bc = INT32_MAX;
    for (int64_t su = h.sunit_off[hh] + lane; su < h.sunit_off[hh + 1]; su += 32) {
      const S s = (S)h.part_score[su];
      const int32_t c = h.part_cid[su];
      if (better<S>(s, c, best, bc)) { best = s; bc = c; }
    }
    warp_argmax<S>(best, bc);
    if (lane == 0)
      J->D[v] = decide<S>(J, v, J->L[v], J->k[v], best, bc, (long long)h.stay[hh],
                          h.iso_seen[hh] != 0);
  }
}

// ------------------------------------------------------------ dispatch ----

namespace {
template <typename K>
int occ_blocks(K kernel, int threads, size_t smem) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
  return nb > 0 ? nb : 1;
}

template <typename S>
void bestmove_impl(const JobDev *jobs, const Buckets &b, const HubBufs &h, int64_t hub_passes,
                   int64_t *ctr, cudaStream_t st, const Dev &d, int *launches) {
  static int occ[16] = {0};
  static bool init = false;
  const size_t smem1 = (size_t)BLK1_CAP * 12, smem2 = (size_t)BLK2_CAP * 12;
  if (!init) {
    cudaFuncSetAttribute(k_bm_block<S, BLK1_CAP, 256, B_BLK1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    cudaFuncSetAttribute(k_bm_block<S, BLK2_CAP, 512, B_BLK2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    occ[0] = occ_blocks(k_bm_group<4, S>, 256, 0);
    occ[1] = occ_blocks(k_bm_group<8, S>, 256, 0);
    occ[2] = occ_blocks(k_bm_group<16, S>, 256, 0);
    occ[3] = occ_blocks(k_bm_group<32, S>, 256, 0);
    occ[4] = occ_blocks(k_bm_warp<S>, 128, 0);
    occ[5] = occ_blocks(k_bm_block<S, BLK1_CAP, 256, B_BLK1>, 256, smem1);
    occ[6] = occ_blocks(k_bm_block<S, BLK2_CAP, 512, B_BLK2>, 512, smem2);
    occ[7] = occ_blocks(k_hub_insert, 256, 0);
    occ[8] = occ_blocks(k_hub_score<S>, 256, 0);
    init = true;
  }
  auto grid = [&](int bk, int o, int per_block) {
    int64_t need = (b.seg_cap[bk] + per_block - 1) / per_block;
    int64_t g = (int64_t)d.sms * o;
    if (need < g) g = need;
    return (int)(g > 0 ? g : 1);
  };
  if (b.seg_cap[B_G4] > 0) {
    k_bm_group<4, S><<<grid(B_G4, occ[0], 64), 256, 0, st>>>(jobs, b, B_G4, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_G8] > 0) {
    k_bm_group<8, S><<<grid(B_G8, occ[1], 32), 256, 0, st>>>(jobs, b, B_G8, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_G16] > 0) {
    k_bm_group<16, S><<<grid(B_G16, occ[2], 16), 256, 0, st>>>(jobs, b, B_G16, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_G32] > 0) {
    k_bm_group<32, S><<<grid(B_G32, occ[3], 8), 256, 0, st>>>(jobs, b, B_G32, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_WARP] > 0) {
    k_bm_warp<S><<<grid(B_WARP, occ[4], 4), 128, 0, st>>>(jobs, b, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_BLK1] > 0) {
    k_bm_block<S, BLK1_CAP, 256, B_BLK1><<<grid(B_BLK1, occ[5], 1), 256, smem1, st>>>(jobs, b, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_BLK2] > 0) {
    k_bm_block<S, BLK2_CAP, 512, B_BLK2><<<grid(B_BLK2, occ[6], 1), 512, smem2, st>>>(jobs, b, ctr);
    ++*launches;
  }
  if (b.seg_cap[B_HUB] > 0) {
    k_hub_prep<<<1, 1024, 0, st>>>(jobs, b, h, ctr);
    for (int64_t p = 0; p < hub_passes; ++p) {
      const int64_t lo = p * h.window;
      k_hub_clear<<<d.sms * 8, 256, 0, st>>>(h, ctr, lo);
      k_hub_insert<<<d.sms * occ[7], 256, 0, st>>>(jobs, b, h, ctr, lo);
      k_hub_score<S><<<d.sms * occ[8], 256, 0, st>>>(jobs, b, h, ctr, lo);
      *launches += 3;
    }
    int64_t fg = (b.seg_cap[B_HUB] + 7) / 8;
    if (fg > d.sms * 4) fg = d.sms * 4;
    k_hub_final<S><<<(int)(fg > 0 ? fg : 1), 256, 0, st>>>(jobs, b, h, ctr);
    *launches += 2;
  }
}
}  // namespace

void launch_bestmove(bool wide, const JobDev *jobs, const Buckets &b, const HubBufs &h,
                     int64_t hub_passes, int64_t *ctr, cudaStream_t st, const Dev &d,
                     int *launches) {
  if (wide)
    bestmove_impl<i128>(jobs, b, h, hub_passes, ctr, st, d, launches);
  else
    bestmove_impl<int64_t>(jobs, b, h, hub_passes, ctr, st, d, launches);
}

// --------------------------------------------------------------- apply ----

__global__ void __launch_bounds__(256) k_apply(const JobDev *__restrict__ jobs, Buckets b,
                                               int64_t *jmoves, uint64_t *moved, int64_t moved_cap,
                                               int64_t *ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  long long nmv = 0;
  for (int bk = 0; bk < NB; ++bk) {
    const int64_t count = seg_count(b, bk);
    const uint64_t *items = b.items + b.seg_start[bk];
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < count;
         base += stride) {
      const int64_t i = base + lane;
      int j = -1;
      bool mv = false, mark = false;
      uint64_t item = 0;
      if (i < count) {
        item = items[i];
        j = (int)(item >> 32);
        const JobDev *J = jobs + j;
        const int32_t v = (int32_t)(uint32_t)item;
        if (!(J->flags & JF_EVAL_ONLY)) {
          const int32_t dv = J->D[v];
          const int32_t lv = J->L[v];
          if (dv != lv) {
            mv = true;
            const int64_t kv = J->k[v];
            J->L[v] = dv;
            if (kv) {
              atomic_add_i64(J->K + lv, -kv);
              atomic_add_i64(J->K + dv, kv);
            }
            if (J->flags & JF_MARK_CL) J->cl[lv] = 1;
            mark = (J->flags & JF_MARK_NBR) != 0;
          }
        }
      }
      // per-job move counts, aggregated over the lanes of one job
      const unsigned peers = __match_any_sync(FULL, mv ? j : -1);
      if (mv && lane == __ffs(peers) - 1)
        atomicAdd((unsigned long long *)(jmoves + j), (unsigned long long)__popc(peers));
      nmv += mv;
      const unsigned mb = __ballot_sync(FULL, mark);
      if (mb) {
        unsigned long long basepos = 0;
        if (lane == __ffs(mb) - 1)
          basepos = atomicAdd((unsigned long long *)&ctr[C_MOVED_N], (unsigned long long)__popc(mb));
        basepos = __shfl_sync(FULL, basepos, __ffs(mb) - 1);
        if (mark) {
          const int64_t pos = (int64_t)basepos + __popc(mb & lanemask_lt());
          if (pos < moved_cap)
            moved[pos] = item;
          else
            atomicOr((unsigned long long *)&ctr[C_ERR], (unsigned long long)E_MOVED_OVERFLOW);
        }
      }
    }
  }
  nmv = warp_sum_ll(nmv);
  if (lane == 0 && nmv) atomicAdd((unsigned long long *)&ctr[C_MOVES], (unsigned long long)nmv);
}

void launch_apply(const JobDev *jobs, const Buckets &b, int64_t *jmoves, uint64_t *moved,
                  int64_t moved_cap, int64_t *ctr, cudaStream_t st, const Dev &d) {
  int64_t tot = 0;
  for (int i = 0; i < NB; ++i) tot += b.seg_cap[i];
  if (tot == 0) return;
  int64_t g = (tot + 255) / 256;
  if (g > d.sms * 8) g = d.sms * 8;
  k_apply<<<(int)g, 256, 0, st>>>(jobs, b, jmoves, moved, moved_cap, ctr);
}

// ---------------------------------------------------------------- mark ----

// V' <- neighbours of the moved vertices (Algorithm 1 / Sec. 3.2.2).
__global__ void __launch_bounds__(256) k_mark_nbr(const JobDev *__restrict__ jobs,
                                                  const uint64_t *__restrict__ moved,
                                                  const int64_t *ctr, int64_t moved_cap) {
  const int lane = threadIdx.x & 31;
  int64_t M = ctr[C_MOVED_N];
  if (M > moved_cap) M = moved_cap;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < M;
       i += warps_total) {
    const uint64_t item = moved[i];
    const JobDev *J = jobs + (int)(item >> 32);
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

void launch_mark(const JobDev *jobs, const uint64_t *moved, int64_t *ctr, bool any_cl,
                 const int64_t *vstart, int njobs, int64_t vtot, cudaStream_t st, const Dev &d,
                 int *launches) {
  k_mark_nbr<<<d.sms * 8, 256, 0, st>>>(jobs, moved, ctr, vtot);
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
