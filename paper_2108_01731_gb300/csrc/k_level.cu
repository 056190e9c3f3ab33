// Per-level kernels: level statistics, initial singletons, node weights,
// Flatten (Sec. 3.1 / Appendix B), canonical labels, the exact objective
// (Sec. 2) and input validation.  All of them run over a table of jobs in a
// flat vertex index space (vstart[j] is job j's first flat index).
#include "lcc_internal.cuh"

namespace lcc {

namespace {
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ long long wsum_ll(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

int grid_for(int64_t work, int threads, const Dev &d, int per_sm = 8) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t mx = (int64_t)d.sms * per_sm;
  if (g > mx) g = mx;
  return (int)(g > 0 ? g : 1);
}
}  // namespace

// ------------------------------------------------------- level statistics --

// A warp takes 32 consecutive vertices, one per lane: degree bucket, hub
// table sizes, row sum of |w|, node weight range.  A lane sums a short row's
// weights itself; the warp sums each long row together.  The warp keeps
// running totals for the job it is on (per lane, reduced when the job
// changes; bucket counts by ballot, in shared memory); a window that spans
// two jobs sends each vertex's figures to its own job directly.
namespace {
constexpr int64_t KSAT = (int64_t)1 << 62;

struct StatAcc {
  int64_t hcap, hun, hsu, hmax, rmax, kmax, ksum, wabs, kneg, ents, ksat;
};

__device__ __forceinline__ int64_t wmax_ll(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t y = __shfl_xor_sync(FULL, x, o);
    x = y > x ? y : x;
  }
  return x;
}

// Adds totals to job I's figures (the caller's lane holds the whole total;
// bucket counts go separately).
__device__ void stats_flush(LevelInfo *I, const StatAcc &a) {
  if (a.hcap) atomicAdd((unsigned long long *)&I->hub_cap, (unsigned long long)a.hcap);
  if (a.hun) atomicAdd((unsigned long long *)&I->hub_units, (unsigned long long)a.hun);
  if (a.hsu) atomicAdd((unsigned long long *)&I->hub_sunits, (unsigned long long)a.hsu);
  atomicMax((unsigned long long *)&I->rmax, (unsigned long long)a.rmax);
  atomicMax((unsigned long long *)&I->kmax, (unsigned long long)a.kmax);
  int64_t ksat = a.ksat;
  if (a.ksum) {
    // node weights are non-negative and every addend is below 2^62, so the
    // add that carries the total past 2^62 sees it before any wrap
    const unsigned long long old =
        atomicAdd((unsigned long long *)&I->ksum, (unsigned long long)a.ksum);
    if (old >= (unsigned long long)KSAT || old + (unsigned long long)a.ksum >= (unsigned long long)KSAT)
      ksat = 1;
  }
  if (ksat) atomicOr((unsigned long long *)&I->ksat, 1ull);
  if (a.wabs) atomicAdd((unsigned long long *)&I->wabs, (unsigned long long)a.wabs);
  if (a.kneg) atomicAdd((unsigned long long *)&I->pad, (unsigned long long)a.kneg);
  if (a.hmax) atomicMax((unsigned long long *)&I->hub_maxcap, (unsigned long long)a.hmax);
  if (a.ents) atomicAdd((unsigned long long *)&I->nnz, (unsigned long long)a.ents);
}

__device__ __forceinline__ void stats_clear(StatAcc &a) {
  a.hcap = a.hun = a.hsu = a.hmax = a.rmax = a.kmax = a.ksum = a.wabs = a.kneg = a.ents = a.ksat = 0;
}

// One vertex's figures into a lane's totals (its bucket is counted apart).
__device__ __forceinline__ void stats_add(StatAcc &a, int64_t deg, int b, long long ra,
                                          int64_t kv) {
  a.ents += deg;
  if (b == B_HUB) {
    const int64_t cap = hub_cap(deg);
    a.hcap += cap;
    if (cap > a.hmax) a.hmax = cap;
    a.hun += (deg + HUB_CHUNK - 1) / HUB_CHUNK;
    a.hsu += (cap + HUB_SCHUNK - 1) / HUB_SCHUNK;
  }
  if (ra > a.rmax) a.rmax = ra;
  a.wabs += ra;
  if (kv < 0) {
    a.kneg += 1;
  } else {
    if (kv > a.kmax) a.kmax = kv;
    if (kv >= KSAT - a.ksum) a.ksat = 1;  // the running total would reach 2^62
    else a.ksum += kv;
  }
}

// The rows of more than 1024 entries are few: their partitioned-path sizes
// go straight to the job's per-bucket totals.
__device__ __forceinline__ void part_stats_add(LevelInfo *I, int64_t deg, int b) {
  if (b < PB0) return;
  PartStat *ps = &I->pst[b - PB0];
  const int64_t P = part_count_of(deg), C = part_chunks_of(deg);
  const int64_t cap = hub_cap(deg);
  atomicAdd((unsigned long long *)&ps->rows, 1ull);
  atomicAdd((unsigned long long *)&ps->nnz, (unsigned long long)deg);
  atomicAdd((unsigned long long *)&ps->parts, (unsigned long long)P);
  if (C) {
    atomicAdd((unsigned long long *)&ps->chunks, (unsigned long long)C);
    atomicAdd((unsigned long long *)&ps->cells, (unsigned long long)(P * C));
  }
  atomicAdd((unsigned long long *)&ps->cap, (unsigned long long)cap);
  atomicAdd((unsigned long long *)&ps->sunits,
            (unsigned long long)((cap + HUB_SCHUNK - 1) / HUB_SCHUNK));
  atomicMax((unsigned long long *)&ps->maxcap, (unsigned long long)cap);
}
}  // namespace

__global__ void __launch_bounds__(256) k_level_stats(const LJob *__restrict__ jobs,
                                                     const int64_t *__restrict__ vstart,
                                                     int njobs, int64_t vtot, LevelInfo *info) {
  __shared__ long long s_bc[8][NB];  // the warp's bucket counts for job cur
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  int cur = -1;  // the job of the warp's running totals (warp-uniform)
  StatAcc acc;
  stats_clear(acc);
  if (lane < NB) s_bc[wib][lane] = 0;
  __syncwarp();
  // reduces the lanes' totals into lane 0 and adds them to job cur
  auto flush = [&]() {
    if (cur < 0) return;
    acc.hcap = wsum_ll(acc.hcap);
    acc.hun = wsum_ll(acc.hun);
    acc.hsu = wsum_ll(acc.hsu);
    acc.wabs = wsum_ll(acc.wabs);
    acc.kneg = wsum_ll(acc.kneg);
    acc.ents = wsum_ll(acc.ents);
    acc.hmax = wmax_ll(acc.hmax);
    acc.rmax = wmax_ll(acc.rmax);
    acc.kmax = wmax_ll(acc.kmax);
    // each lane's ksum is below 2^62: pairwise sums cannot wrap, and a sum
    // that reaches 2^62 saturates the flag
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t y = __shfl_xor_sync(FULL, acc.ksum, o);
      const int64_t ys = __shfl_xor_sync(FULL, acc.ksat, o);
      acc.ksum += y;
      acc.ksat |= ys;
      if (acc.ksum >= KSAT) {
        acc.ksum = KSAT - 1;
        acc.ksat = 1;
      }
    }
    if (lane == 0) stats_flush(info + cur, acc);
    __syncwarp();
    if (lane < NB) {
      const long long c = s_bc[wib][lane];
      if (c) atomicAdd((unsigned long long *)&info[cur].bcnt[lane], (unsigned long long)c);
      s_bc[wib][lane] = 0;
    }
    __syncwarp();
    stats_clear(acc);
  };
  for (int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * 32; i0 < vtot;
       i0 += warps_total * 32) {
    const int64_t i = i0 + lane;
    const bool valid = i < vtot;
    int j = 0;
    int64_t deg = 0, beg = 0, kv = 0;
    const LJob *J = jobs;
    if (valid) {
      j = find_job(vstart, njobs, i);
      J = jobs + j;
      const int64_t v = i - vstart[j];
      beg = J->off[v];
      deg = J->off[v + 1] - beg;
      kv = J->k[v];
    }
    // row sums of |w|: short rows by their lane, long rows by the warp
    long long ra = 0;
    const bool wt = valid && J->wtype != W_NONE;
    if (valid && !wt) ra = deg;
    if (wt && deg <= 32) {
#pragma unroll 4
      for (int64_t e = beg; e < beg + deg; ++e) {
        const long long x = load_w(J->w, J->wtype, e);
        ra += x < 0 ? -x : x;
      }
    }
    for (unsigned m = __ballot_sync(FULL, wt && deg > 32); m; m &= m - 1) {
      const int l = __ffs(m) - 1;
      const int jl = __shfl_sync(FULL, j, l);
      const int64_t bl = __shfl_sync(FULL, beg, l), dl = __shfl_sync(FULL, deg, l);
      const LJob *Jl = jobs + jl;
      long long sl = 0;
      for (int64_t e = bl + lane; e < bl + dl; e += 32) {
        const long long x = load_w(Jl->w, Jl->wtype, e);
        sl += x < 0 ? -x : x;
      }
      sl = wsum_ll(sl);
      if (lane == l) ra = sl;
    }
    const int b = valid ? bucket_of(deg, J->warp_max) : -1;
    if (valid) part_stats_add(info + j, deg, b);
    const int j0 = __shfl_sync(FULL, j, 0);
    if (__all_sync(FULL, !valid || j == j0)) {
      if (j0 != cur) {
        flush();
        cur = j0;
      }
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const int c = __popc(__ballot_sync(FULL, b == k));
        if (lane == k && c) s_bc[wib][k] += c;
      }
      if (valid) stats_add(acc, deg, b, ra, kv);
    } else if (valid) {
      // a window across two jobs: each vertex's figures to its own job
      StatAcc one;
      stats_clear(one);
      stats_add(one, deg, b, ra, kv);
      stats_flush(info + j, one);
      atomicAdd((unsigned long long *)&info[j].bcnt[b], 1ull);
    }
  }
  flush();
}

void launch_level_stats(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                        LevelInfo *info, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_level_stats<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, info);
}

// ---------------------------------------------------------- gather layout --

// Where each vertex's packed label word is kept for the best-move gathers:
// vertices in decreasing degree class, so that the words most rows refer to
// share a few L2-sized regions (on power-law graphs a small fraction of the
// vertices receives most entries).  Only storage positions change: labels,
// clusters and every result stay in terms of the vertex ids.

__device__ __forceinline__ int degree_class(int64_t deg) {
  return deg <= 0 ? 0 : 64 - __clzll((long long)deg);  // 1 + floor(log2 deg)
}

__device__ __forceinline__ unsigned lanemask_lt_l() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void k_layout_count(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                               int njobs, int64_t vtot, int64_t *cnt) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < vtot;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    int key = -1;
    if (i < vtot) {
      const int j = find_job(vstart, njobs, i);
      const int64_t v = i - vstart[j];
      key = j * LAYOUT_CLASSES + degree_class(jobs[j].off[v + 1] - jobs[j].off[v]);
    }
    const unsigned peers = __match_any_sync(FULL, key);
    if (key >= 0 && lane == __ffs(peers) - 1)
      atomicAdd((unsigned long long *)&cnt[key], (unsigned long long)__popc(peers));
  }
}

// One thread per job: class counts -> first position of each class, highest
// class first (in place).
__global__ void k_layout_base(int njobs, int64_t *cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= njobs) return;
  int64_t run = 0;
  for (int c = LAYOUT_CLASSES - 1; c >= 0; --c) {
    const int64_t x = cnt[j * LAYOUT_CLASSES + c];
    cnt[j * LAYOUT_CLASSES + c] = run;
    run += x;
  }
}

// pos[v] = next free position of v's class (positions within a class are
// taken in no particular order; any order is a valid layout).
__global__ void k_layout_place(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                               int njobs, int64_t vtot, int64_t *cur) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < vtot;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    int key = -1, j = 0;
    int64_t v = 0;
    if (i < vtot) {
      j = find_job(vstart, njobs, i);
      v = i - vstart[j];
      key = j * LAYOUT_CLASSES + degree_class(jobs[j].off[v + 1] - jobs[j].off[v]);
    }
    const unsigned peers = __match_any_sync(FULL, key);
    if (key >= 0) {
      const int leader = __ffs(peers) - 1;
      unsigned long long p0 = 0;
      if (lane == leader)
        p0 = atomicAdd((unsigned long long *)&cur[key], (unsigned long long)__popc(peers));
      p0 = __shfl_sync(peers, p0, leader);
      jobs[j].pos[v] = (int32_t)(p0 + __popc(peers & lanemask_lt_l()));
    }
  }
}

// gnbr[e] = pos[nbr[e]] over the flat entry space of all jobs.
__global__ void k_layout_nbr(const LJob *__restrict__ jobs, const int64_t *__restrict__ estart,
                             int njobs, int64_t etot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < etot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(estart, njobs, i);
    const LJob &J = jobs[j];
    const int64_t e = i - estart[j];
    J.gnbr[e] = __ldg(J.pos + __ldg(J.nbr + e));
  }
}

void launch_layout(const LJob *jobs, const int64_t *vstart, const int64_t *estart, int njobs,
                   int64_t vtot, int64_t etot, int64_t *cnt, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_layout_count<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, cnt);
  k_layout_base<<<(njobs + 127) / 128, 128, 0, st>>>(njobs, cnt);
  k_layout_place<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, cnt);
  if (etot > 0) k_layout_nbr<<<grid_for(etot, 256, d), 256, 0, st>>>(jobs, estart, njobs, etot);
}

// ------------------------------------------------------- per-vertex maps --

__global__ void k_init_level(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                             int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    J->L[v] = (int32_t)v;
    J->K[v] = J->k[v];
  }
}

void launch_init_level(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                       cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_init_level<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot);
}

// Modularity node weights (Sec. 2): k_v = sum_u w_uv, one warp per vertex.
// Written through LJob::K (the job's node-weight array for this purpose).
__global__ void __launch_bounds__(256) k_degree_k(const LJob *__restrict__ jobs,
                                                  const int64_t *__restrict__ vstart, int njobs,
                                                  int64_t vtot) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < vtot;
       i += warps_total) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    long long s = 0;
    for (int64_t e = J->off[v] + lane; e < J->off[v + 1]; e += 32) s += load_w(J->w, J->wtype, e);
    s = wsum_ll(s);
    if (lane == 0) J->K[v] = s;
  }
}

void launch_degree_k(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot, int64_t *,
                     cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_degree_k<<<grid_for(vtot * 32, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot);
}

__global__ void k_fill_one(int64_t *k, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    k[i] = 1;
}

void launch_fill_k_unit(int64_t *k, int64_t n, cudaStream_t st, const Dev &d) {
  if (n <= 0) return;
  k_fill_one<<<grid_for(n, 256, d), 256, 0, st>>>(k, n);
}

__global__ void k_zero_K(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                         int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    jobs[j].K[i - vstart[j]] = 0;
  }
}

// K_c = sum of k_v over the vertices labelled c (exact integer atomics).
__global__ void k_add_K(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                        int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    const int64_t kv = J->k[v];
    if (kv) atomic_add_i64(J->K + J->L[v], kv);
  }
}

void launch_recompute_K(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                        cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_zero_K<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot);
  k_add_K<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot);
}

// Flatten: v takes the cluster of its coarse vertex, L[v] = L'[map[v]].
__global__ void k_flatten(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                          int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    J->L[v] = J->Lcoarse[J->map[v]];
  }
}

void launch_flatten(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                    cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_flatten<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot);
}

// Canonical labels: the smallest vertex id of each cluster (D is scratch).
__global__ void k_canon_init(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                             int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    jobs[j].D[i - vstart[j]] = INT32_MAX;
  }
}
__global__ void k_canon_min(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                            int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    atomicMin(J->D + J->L[v], (int32_t)v);
  }
}
__global__ void k_canon_set(const LJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                            int njobs, int64_t vtot) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    J->L[v] = J->D[J->L[v]];
  }
}

void launch_canonical(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                      cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  const int g = grid_for(vtot, 256, d);
  k_canon_init<<<g, 256, 0, st>>>(jobs, vstart, njobs, vtot);
  k_canon_min<<<g, 256, 0, st>>>(jobs, vstart, njobs, vtot);
  k_canon_set<<<g, 256, 0, st>>>(jobs, vstart, njobs, vtot);
}

// ------------------------------------------------------------ objective --

// q * CC = q * S_in - p * (sum_C K_C^2 - sum_v k_v^2)   (Sec. 2, ordered
// pairs), with S_in the sum of w over entries whose ends share a label.
// This kernel accumulates S_in (one warp per vertex).
__global__ void __launch_bounds__(256) k_obj_edges(const LJob *__restrict__ jobs,
                                                   const int64_t *__restrict__ vstart, int njobs,
                                                   int64_t vtot, ObjAcc *acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  int cur = -1;
  long long run = 0;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < vtot;
       i += warps_total) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    const int32_t lv = J->L[v];
    long long s = 0;
    for (int64_t e = J->off[v] + lane; e < J->off[v + 1]; e += 32)
      if (J->L[J->nbr[e]] == lv) s += load_w(J->w, J->wtype, e);
    s = wsum_ll(s);
    if (lane == 0) {
      if (j != cur) {
        if (cur >= 0 && run) atomicAdd(&acc[cur].s_in, (unsigned long long)run);
        cur = j;
        run = 0;
      }
      run += s;
    }
  }
  if (lane == 0 && cur >= 0 && run) atomicAdd(&acc[cur].s_in, (unsigned long long)run);
}

// sum_C K_C^2 and sum_v k_v^2 (128-bit, one thread per cluster id / vertex).
__global__ void __launch_bounds__(256) k_obj_squares(const LJob *__restrict__ jobs,
                                                     const int64_t *__restrict__ vstart,
                                                     int njobs, int64_t vtot, ObjAcc *acc) {
  int cur = -1;
  u128 a = 0, b = 0;
  unsigned long long reps = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const LJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    if (j != cur) {
      if (cur >= 0) {
        atomic_add_u128(&acc[cur].ksq_lo, &acc[cur].ksq_hi, a);
        atomic_add_u128(&acc[cur].kself_lo, &acc[cur].kself_hi, b);
        if (reps) atomicAdd(&acc[cur].nclus, reps);
      }
      cur = j;
      a = b = 0;
      reps = 0;
    }
    reps += (J->L[v] == (int32_t)v);
    const u128 K = (u128)(uint64_t)J->K[v];
    const u128 k = (u128)(uint64_t)J->k[v];
    a += K * K;
    b += k * k;
  }
  if (cur >= 0) {
    atomic_add_u128(&acc[cur].ksq_lo, &acc[cur].ksq_hi, a);
    atomic_add_u128(&acc[cur].kself_lo, &acc[cur].kself_hi, b);
    if (reps) atomicAdd(&acc[cur].nclus, reps);
  }
}

void launch_objective(const LJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                      ObjAcc *acc, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  launch_recompute_K(jobs, vstart, njobs, vtot, st, d);
  k_obj_edges<<<grid_for(vtot * 32, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, acc);
  k_obj_squares<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, acc);
}

// ------------------------------------------------------------ validation --

// out[0] error bits (1 offsets, 2 range, 4 self loop), out[1..4] two pairs
// of order-independent hash sums over (u, v, w) and (v, u, w): equal sums
// for a symmetric multiset; out[5..6] sum of |w| as 128 bits.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

__global__ void k_validate_off(const int64_t *off, int64_t n, int64_t nnz,
                               unsigned long long *out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (off[v] > off[v + 1] || off[v] < 0 || off[v + 1] > nnz) atomicOr(out, 1ull);
  }
}

__global__ void __launch_bounds__(256) k_validate_rows(const int64_t *off, const int32_t *nbr,
                                                       const int32_t *w, int64_t n,
                                                       unsigned long long *out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long h1 = 0, h2 = 0, h3 = 0, h4 = 0, bits = 0;
  u128 wabs = 0;
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n;
       u += warps_total) {
    for (int64_t e = off[u] + lane; e < off[u + 1]; e += 32) {
      const int32_t v = nbr[e];
      if (v < 0 || v >= n) { bits |= 2; continue; }
      if (v == u) bits |= 4;
      const long long wt = w ? (long long)w[e] : 1;
      wabs += (u128)(unsigned long long)(wt < 0 ? -wt : wt);
      const unsigned long long uw = (unsigned long long)wt;
      const unsigned long long a = ((unsigned long long)u << 32) | (unsigned long long)(uint32_t)v;
      const unsigned long long b = ((unsigned long long)(uint32_t)v << 32) | (unsigned long long)u;
      h1 += mix64(a ^ mix64(uw));
      h2 += mix64(b ^ mix64(uw));
      h3 += mix64(mix64(a + 0x9e3779b97f4a7c15ull) + uw);
      h4 += mix64(mix64(b + 0x9e3779b97f4a7c15ull) + uw);
    }
  }
  // warp, then block sums: one set of atomics per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    h1 += __shfl_xor_sync(FULL, h1, o);
    h2 += __shfl_xor_sync(FULL, h2, o);
    h3 += __shfl_xor_sync(FULL, h3, o);
    h4 += __shfl_xor_sync(FULL, h4, o);
    bits |= __shfl_xor_sync(FULL, bits, o);
    const unsigned long long lo = __shfl_xor_sync(FULL, (unsigned long long)wabs, o);
    const unsigned long long hi = __shfl_xor_sync(FULL, (unsigned long long)(wabs >> 64), o);
    wabs += ((u128)hi << 64) | lo;
  }
  __shared__ unsigned long long part[8][7];
  const int wib = threadIdx.x >> 5;
  if (lane == 0) {
    part[wib][0] = bits;
    part[wib][1] = h1;
    part[wib][2] = h2;
    part[wib][3] = h3;
    part[wib][4] = h4;
    part[wib][5] = (unsigned long long)wabs;
    part[wib][6] = (unsigned long long)(wabs >> 64);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tb = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0;
    u128 tw = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      tb |= part[k][0];
      t1 += part[k][1];
      t2 += part[k][2];
      t3 += part[k][3];
      t4 += part[k][4];
      tw += ((u128)part[k][6] << 64) | part[k][5];
    }
    if (tb) atomicOr(out, tb);
    atomicAdd(out + 1, t1);
    atomicAdd(out + 2, t2);
    atomicAdd(out + 3, t3);
    atomicAdd(out + 4, t4);
    atomic_add_u128(out + 5, out + 6, tw);
  }
}

void launch_validate(const int64_t *off, int64_t n, int64_t nnz, unsigned long long *out8,
                     cudaStream_t st, const Dev &d) {
  if (n <= 0) return;
  k_validate_off<<<grid_for(n, 256, d), 256, 0, st>>>(off, n, nnz, out8);
}

void launch_validate_rows(const int64_t *off, const int32_t *nbr, const int32_t *w, int64_t n,
                          unsigned long long *out8, cudaStream_t st, const Dev &d) {
  if (n <= 0) return;
  k_validate_rows<<<grid_for(n * 32, 256, d), 256, 0, st>>>(off, nbr, w, n, out8);
}

// ------------------------------------------------------ symmetry breaking --

// SplitMix64 (Vigna's generator after Steele, Lea and Flood 2014): output
// i >= 1 of the stream seeded with `seed` is the finaliser applied to
// seed + i * 0x9e3779b97f4a7c15.  The coin of key allows a move when the top
// bit of output key + 1 is 1.
__device__ __forceinline__ bool coin_allows(uint64_t seed, uint64_t key) {
  uint64_t z = seed + (key + 1) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (z >> 63) != 0;
}

// Runs between the best-move kernels and k_apply over the same bucket items
// (the round's V').  Whole warps step together so the per-job counts of
// held-back vertices combine before their atomic.
__global__ void __launch_bounds__(256) k_coin(const JobDev *__restrict__ jobs,
                                              const CoinJob *__restrict__ coins, Buckets b,
                                              int64_t *held) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int bk = 0; bk < NB; ++bk) {
    int64_t count = b.cnt[bk];
    if (count > b.seg_cap[bk]) count = b.seg_cap[bk];
    const uint64_t *items = b.items + b.seg_start[bk];
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < count; base += stride) {
      const int64_t i = base + threadIdx.x;
      int hj = -1;
      if (i < count) {
        const uint64_t item = items[i];
        const int j = (int)(item >> 32);
        const CoinJob c = coins[j];
        if (c.on) {
          const JobDev *J = jobs + j;
          const int32_t v = (int32_t)(uint32_t)item;
          const int32_t lv = J->L[v];
          if (J->D[v] != lv && !coin_allows(c.seed, c.key_hi + (uint32_t)v)) {
            J->D[v] = lv;     // keeps its cluster this round
            J->fr[v] |= 1;    // and is evaluated again in the next
            hj = j;
          }
        }
      }
      const unsigned peers = __match_any_sync(FULL, hj);
      if (hj >= 0 && lane == __ffs(peers) - 1)
        atomicAdd((unsigned long long *)(held + hj), (unsigned long long)__popc(peers));
    }
  }
}

void launch_coin(const JobDev *jobs, const CoinJob *coins, const Buckets &b, int64_t *held,
                 cudaStream_t st, const Dev &d) {
  int64_t tot = 0;
  for (int i = 0; i < NB; ++i) tot += b.seg_cap[i];
  if (tot == 0) return;
  k_coin<<<grid_for(tot, 256, d), 256, 0, st>>>(jobs, coins, b, held);
}

}  // namespace lcc
