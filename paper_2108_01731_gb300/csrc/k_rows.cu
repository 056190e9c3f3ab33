// Compress (Sec. 3.1, Appendix B) by rows: the entries of every coarse
// vertex C are gathered into one region, the entries that stay inside C are
// dropped, and parallel edges (equal coarse neighbour) are merged by summing
// their weights in a hash table.  This is the paper's parallel aggregation of
// edges by endpoint clusters, done per coarse row, with no global sort.
//
//   bound    one atomic per fine vertex u adds deg(u) to rbound[C] for its
//            coarse vertex C and keeps the old value as u's place rpos[u]
//            in C's region; the scan of rbound gives each coarse row a region
//            [boff[C], boff[C+1]) of the flat entry space;
//   emit     a warp takes 32 consecutive fine vertices, whose rows are one
//            contiguous run of entries, reads them coalesced, looks up every
//            neighbour's coarse id and writes (local coarse id of the far
//            end, w) at boff[C] + rpos[u] + j; an entry inside C becomes a
//            hole (-1) that the merges skip;
//   classes  rows by region length: a single entry is already final (or a
//            hole); G lanes per row
//            (<= 4 .. 32 entries), a warp with a shared table (<= 256), a
//            block with a shared table (<= 4096, and <= 8192 with 1024
//            threads and 192 KB), global tables in bounded windows (more);
//   reduce   every row merges its region in place: its unique entries are
//            written back to the start of the region, their number to
//            ucnt[C]; a scan of ucnt gives the coarse offsets and the rows
//            are copied into place.
//
// The order of a coarse row's entries is not fixed (arrival and table
// order): no result depends on it, because every sum is an exact integer and
// ties between clusters go to the smallest id.  The exported graph of
// lcc_compress sorts its rows.
#include "lcc_internal.cuh"

namespace lcc {

namespace {
constexpr unsigned FULL = 0xffffffffu;

int grid_of(int64_t work, int threads, const Dev &d, int per_sm = 8) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t mx = (int64_t)d.sms * per_sm;
  if (g > mx) g = mx;
  return (int)(g > 0 ? g : 1);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Home slot of a coarse id in a power-of-two table of 2^lg slots.
__device__ __forceinline__ uint32_t row_home(int32_t c, int lg) {
  return (uint32_t)(((uint64_t)(uint32_t)c * 0x9E3779B97F4A7C15ull) >> (64 - lg));
}

__device__ __forceinline__ int lg_of(int64_t pow2) { return 63 - __clzll((long long)pow2); }

// One coarse row: its region and its number of entries there.
struct Row {
  int64_t rb;    // first entry of the region (and of its unique entries)
  int64_t cnt;   // entries in the region
  int32_t C;     // global coarse id
};

__device__ __forceinline__ Row row_of(const RowSpace &R, int32_t C) {
  Row r;
  r.C = C;
  r.rb = R.boff[C];
  r.cnt = R.boff[C + 1] - r.rb;
  return r;
}

__device__ __forceinline__ long long warp_sum(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}
}  // namespace

// ------------------------------------------------------- bound, emit ----

__global__ void k_rbound(const CJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                         int njobs, int64_t vt, const int32_t *__restrict__ gmap,
                         int64_t *rbound, int64_t *rpos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const CJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    const int64_t deg = J->off[v + 1] - J->off[v];
    rpos[i] = deg ? (int64_t)atomicAdd((unsigned long long *)&rbound[gmap[i]],
                                       (unsigned long long)deg)
                  : 0;
  }
}

void launch_rbound(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vt,
                   const int32_t *gmap, int64_t *rbound, int64_t *rpos, cudaStream_t st,
                   const Dev &d) {
  if (vt <= 0) return;
  k_rbound<<<grid_of(vt, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vt, gmap, rbound, rpos);
}

// One entry of fine vertex u (flat index i) of coarse row C, written at its
// place pos of C's region: the far end's job-local coarse id, or a hole.
__device__ __forceinline__ void emit_one(const RowSpace &R, const CJob *J, int64_t vs,
                                         int32_t cbase, int32_t C, int64_t e, int64_t pos,
                                         long long &nintra) {
  const int32_t cv = R.gmapp[vs + __ldg(J->gnbr + e)];
  const bool intra = cv == C;
  R.tnbr[pos] = intra ? -1 : cv - cbase;
  R.tw[pos] = load_w(J->w, J->wtype, e);
  nintra += intra ? 1 : 0;
}

// A warp takes 32 consecutive fine vertices.  Inside one job their rows are
// one contiguous run of entries [off[v0], off[v0 + 32]): the lanes stream it,
// each entry finding its vertex by a binary search over the 33 row starts in
// shared memory, and write it at its vertex's place in its coarse row's
// region.  A window that crosses into another job (at most one per job)
// walks each lane's own vertex instead.
__global__ void __launch_bounds__(256) k_emit_rows(RowSpace R, int64_t vt) {
  __shared__ int64_t s_e[8][33];
  __shared__ int64_t s_dst[8][32];
  __shared__ int32_t s_c[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  long long nintra = 0;
  for (int64_t i0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * 32; i0 < vt;
       i0 += warps_total * 32) {
    const int64_t i = i0 + lane;
    const bool valid = i < vt;
    int j = 0;
    int64_t eb = 0, ee = 0, dst = 0;
    int32_t C = 0;
    if (valid) {
      j = find_job(R.vstart, R.njobs, i);
      const CJob *J = R.jobs + j;
      const int64_t v = i - R.vstart[j];
      eb = J->off[v];
      ee = J->off[v + 1];
      C = R.gmap[i];
      if (ee > eb) dst = R.boff[C] + R.rpos[i];
    }
    const int j0 = __shfl_sync(FULL, j, 0);
    if (__all_sync(FULL, !valid || j == j0)) {
      // lanes past the end take the last vertex's end as an empty row
      const int last = vt - 1 - i0 < 31 ? (int)(vt - 1 - i0) : 31;
      const int64_t e_end = __shfl_sync(FULL, ee, last);
      if (!valid) eb = ee = e_end;
      s_e[wib][lane] = eb;
      if (lane == 31) s_e[wib][32] = ee;
      s_dst[wib][lane] = dst;
      s_c[wib][lane] = C;
      __syncwarp();
      const CJob *J = R.jobs + j0;
      const int64_t vs = R.vstart[j0];
      const int32_t cbase = (int32_t)R.rank[vs];
      const int64_t e1 = s_e[wib][32];
      const int32_t *__restrict__ gnbr = J->gnbr;
      const int32_t *__restrict__ gmapp = R.gmapp + vs;
      // EU entries per lane per step: all their loads are issued before
      // any of their stores
      constexpr int EU = 4;
      for (int64_t e0 = s_e[wib][0] + lane; e0 < e1; e0 += 32 * EU) {
        int32_t cv[EU], Cr[EU];
        int64_t pos[EU], wv[EU];
#pragma unroll
        for (int u = 0; u < EU; ++u) {
          const int64_t e = e0 + 32 * u;
          cv[u] = 0;
          Cr[u] = 0;
          pos[u] = -1;
          wv[u] = 0;
          if (e < e1) {
            int lo = 0, hi = 32;  // the last vertex whose row starts at or before e
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (s_e[wib][mid] <= e) lo = mid; else hi = mid;
            }
            Cr[u] = s_c[wib][lo];
            pos[u] = s_dst[wib][lo] + (e - s_e[wib][lo]);
            cv[u] = __ldg(gmapp + __ldg(gnbr + e));
            wv[u] = load_w(J->w, J->wtype, e);
          }
        }
#pragma unroll
        for (int u = 0; u < EU; ++u) {
          if (pos[u] < 0) continue;
          const bool intra = cv[u] == Cr[u];
          R.tnbr[pos[u]] = intra ? -1 : cv[u] - cbase;
          R.tw[pos[u]] = wv[u];
          nintra += intra ? 1 : 0;
        }
      }
      __syncwarp();
    } else if (valid) {
      const CJob *J = R.jobs + j;
      const int64_t vs = R.vstart[j];
      const int32_t cbase = (int32_t)R.rank[vs];
      for (int64_t e = eb; e < ee; ++e) emit_one(R, J, vs, cbase, C, e, dst + (e - eb), nintra);
    }
  }
  nintra = warp_sum(nintra);
  if (lane == 0 && nintra) atomicAdd(R.intra, (unsigned long long)nintra);
}

void launch_emit_rows(const RowSpace &R, int64_t vt, cudaStream_t st, const Dev &d) {
  if (vt <= 0) return;
  k_emit_rows<<<grid_of((vt + 31) / 32 * 32, 256, d), 256, 0, st>>>(R, vt);
}

// ------------------------------------------------------------ classes ----

__device__ __forceinline__ int row_class(int64_t cnt) {
  if (cnt <= 1) return -1;  // nothing to merge
  if (cnt <= 4) return RC_G4;
  if (cnt <= 8) return RC_G8;
  if (cnt <= 16) return RC_G16;
  if (cnt <= 32) return RC_G32;
  if (cnt <= RC_WARP_MAX) return RC_WARP;
  if (cnt <= RC_BLOCK_MAX) return RC_BLOCK;
  if (cnt <= RC_BLOCK8K_MAX) return RC_BLOCK8K;
  return RC_BIG;
}

// fill = false: rows per class into cnt[]; fill = true: the rows of class c
// into items[seg[c] ..] (cnt[] then serves as the cursors, zeroed first), and
// a row of one entry that is not a hole gets ucnt = 1 (it is already in
// place).
__global__ void __launch_bounds__(256) k_rows_classify(RowSpace R, int64_t ntot, bool fill,
                                                       unsigned long long *cnt,
                                                       const int64_t *__restrict__ seg,
                                                       int32_t *items) {
  __shared__ unsigned long long s_cnt[RC_N];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < RC_N) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ntot;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t C = base + threadIdx.x;
    const int64_t rc = C < ntot ? R.boff[C + 1] - R.boff[C] : 0;
    const int cls = row_class(rc);
    if (fill && rc == 1 && R.tnbr[R.boff[C]] >= 0) R.ucnt[C] = 1;  // one entry, not a hole
    const unsigned peers = __match_any_sync(FULL, cls);
    const int leader = __ffs(peers) - 1;
    if (cls >= 0) {
      if (!fill) {
        if (lane == leader) atomicAdd(&s_cnt[cls], (unsigned long long)__popc(peers));
      } else {
        unsigned long long p0 = 0;
        if (lane == leader) p0 = atomicAdd(&cnt[cls], (unsigned long long)__popc(peers));
        p0 = __shfl_sync(peers, p0, leader);
        items[seg[cls] + (int64_t)p0 + __popc(peers & lanemask_lt())] = (int32_t)C;
      }
    }
  }
  if (!fill) {
    __syncthreads();
    if (threadIdx.x < RC_N && s_cnt[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], s_cnt[threadIdx.x]);
  }
}

void launch_rows_classify(const RowSpace &R, int64_t ntot, bool fill, unsigned long long *cnt,
                          const int64_t *seg, int32_t *items, cudaStream_t st, const Dev &d) {
  if (ntot <= 0) return;
  k_rows_classify<<<grid_of(ntot, 256, d), 256, 0, st>>>(R, ntot, fill, cnt, seg, items);
}

// -------------------------------------------- rows of <= 32: G lanes each --

// G lanes per row, lane t reads entry t.  Equal coarse neighbours are found
// with __match_any_sync on (group, id) and summed into the first lane's
// shared slot; the first lane of each id writes it.
template <int G>
__global__ void __launch_bounds__(256) k_rows_group(RowSpace R, const int32_t *__restrict__ items,
                                                    int64_t count) {
  __shared__ unsigned long long acc[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gl = lane & (G - 1), gsub = lane / G;
  constexpr int GPW = 32 / G;
  const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (gsub * G));
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wbase = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW; wbase < count;
       wbase += warps_total * GPW) {
    const int64_t it = wbase + gsub;
    const bool valid = it < count;
    Row r;
    r.cnt = 0;
    r.rb = 0;
    r.C = 0;
    if (valid) r = row_of(R, items[it]);
    int32_t cv = -1;
    long long w = 0;
    if (valid && gl < r.cnt) {
      cv = R.tnbr[r.rb + gl];
      w = R.tw[r.rb + gl];
    }
    const bool has = cv >= 0;  // holes (entries inside the cluster) are skipped
    // every lane holds its entry before any lane writes the row back
    const unsigned long long key =
        ((unsigned long long)gsub << 32) | (uint32_t)(has ? cv : -1 - gl);
    const unsigned peers = __match_any_sync(FULL, key);
    const int leader = __ffs(peers) - 1;
    long long wsum = w;
    if (!__all_sync(FULL, !has || __popc(peers) == 1)) {
      acc[wib][lane] = 0;
      __syncwarp();
      if (has) atomicAdd(&acc[wib][leader], (unsigned long long)w);
      __syncwarp();
      wsum = (long long)acc[wib][lane];
      __syncwarp();
    }
    const bool lead = has && lane == leader;
    const unsigned lb = __ballot_sync(FULL, lead) & gmask;
    if (lead) {
      const int pos = __popc(lb & lanemask_lt());
      R.tnbr[r.rb + pos] = cv;
      R.tw[r.rb + pos] = wsum;
    }
    if (valid && gl == 0) R.ucnt[r.C] = __popc(lb);
  }
}

// ------------------------------------ rows of <= 256: warp + shared table --

// Inserts (cv, w) into a power-of-two table of cap slots (keys -1 = empty).
// The table has at least two slots per entry, so a slot is always found.
__device__ __forceinline__ void table_add(int32_t *keys, unsigned long long *vals, int lg,
                                          int32_t cv, long long w) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t s = row_home(cv, lg);
  for (uint32_t t = 0; t <= mask; ++t) {
    const int32_t prev = atomicCAS(keys + s, -1, cv);
    if (prev == -1 || prev == cv) {
      atomicAdd(vals + s, (unsigned long long)w);
      return;
    }
    s = (s + 1) & mask;
  }
}

template <int E>
__global__ void __launch_bounds__(128) k_rows_warp(RowSpace R, const int32_t *__restrict__ items,
                                                   int64_t count) {
  constexpr int WPB = 4, CAP = 64 * E;
  __shared__ int32_t tkey[WPB][CAP];
  __shared__ unsigned long long tval[WPB][CAP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t *K0 = tkey[wib];
  unsigned long long *V0 = tval[wib];
  for (int s = lane; s < CAP; s += 32) {
    K0[s] = -1;
    V0[s] = 0;
  }
  __syncwarp();
  for (int64_t it = (int64_t)blockIdx.x * WPB + wib; it < count; it += (int64_t)gridDim.x * WPB) {
    const Row r = row_of(R, items[it]);
    const int64_t cap = next_pow2(2 * r.cnt);
    const int lg = lg_of(cap);
    int32_t cv[E];
    long long w[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {  // every load first, then the inserts
      cv[i] = -1;
      w[i] = 0;
      const int64_t t = lane + 32 * i;
      if (t < r.cnt) {
        cv[i] = R.tnbr[r.rb + t];
        w[i] = R.tw[r.rb + t];
      }
    }
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (cv[i] >= 0) table_add(K0, V0, lg, cv[i], w[i]);
    __syncwarp();
    int base = 0;
    for (int s0 = 0; s0 < (int)cap; s0 += 32) {
      const int s = s0 + lane;
      const int32_t key = K0[s];
      const bool occ = key >= 0;
      const unsigned b = __ballot_sync(FULL, occ);
      if (occ) {
        const int64_t pos = r.rb + base + __popc(b & lanemask_lt());
        R.tnbr[pos] = key;
        R.tw[pos] = (int64_t)V0[s];
        K0[s] = -1;
        V0[s] = 0;
      }
      base += __popc(b);
    }
    if (lane == 0) R.ucnt[r.C] = base;
    __syncwarp();
  }
}

// ----------------------------------- rows of <= 4096: block + shared table --

// One block per row, THREADS x E entries, a table of 2 slots per entry in
// shared memory (int32 keys and int64 sums: 12 bytes a slot).
template <int THREADS, int E>
__global__ void __launch_bounds__(THREADS) k_rows_block(RowSpace R,
                                                        const int32_t *__restrict__ items,
                                                        int64_t count) {
  constexpr int CAP = 2 * THREADS * E;
  extern __shared__ __align__(16) unsigned char rb_smem[];
  unsigned long long *tval = (unsigned long long *)rb_smem;
  int32_t *tkey = (int32_t *)(tval + CAP);
  __shared__ int s_cnt;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int s = tid; s < CAP; s += THREADS) {
    tkey[s] = -1;
    tval[s] = 0;
  }
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
    const Row r = row_of(R, items[it]);
    const int64_t cap = next_pow2(2 * r.cnt);
    const int lg = lg_of(cap);
    int32_t cv[E];
    long long w[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      cv[i] = -1;
      w[i] = 0;
      const int64_t t = tid + (int64_t)THREADS * i;
      if (t < r.cnt) {
        cv[i] = R.tnbr[r.rb + t];
        w[i] = R.tw[r.rb + t];
      }
    }
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (cv[i] >= 0) table_add(tkey, tval, lg, cv[i], w[i]);
    __syncthreads();  // every entry is read and inserted before the row is rewritten
    for (int s0 = 0; s0 < (int)cap; s0 += THREADS) {
      const int s = s0 + tid;
      const bool occ = s < (int)cap && tkey[s] >= 0;
      const unsigned b = __ballot_sync(FULL, occ);
      int wbase = 0;
      if (lane == 0 && b) wbase = atomicAdd(&s_cnt, __popc(b));
      wbase = __shfl_sync(FULL, wbase, 0);
      if (occ) {
        const int64_t pos = r.rb + wbase + __popc(b & lanemask_lt());
        R.tnbr[pos] = tkey[s];
        R.tw[pos] = (int64_t)tval[s];
        tkey[s] = -1;
        tval[s] = 0;
      }
    }
    __syncthreads();
    if (tid == 0) {
      R.ucnt[r.C] = s_cnt;
      s_cnt = 0;
    }
    __syncthreads();
  }
}

template <int THREADS, int E>
void launch_rows_block(const RowSpace &R, const int32_t *items, int64_t count, int &occ,
                       cudaStream_t st, const Dev &d) {
  constexpr int smem = 2 * THREADS * E * 12;
  auto kern = k_rows_block<THREADS, E>;
  if (!occ) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, THREADS, smem);
    occ = nb > 0 ? nb : 1;
  }
  int64_t blocks = count;
  if (blocks > (int64_t)d.sms * occ) blocks = (int64_t)d.sms * occ;
  kern<<<(int)blocks, THREADS, smem, st>>>(R, items, count);
}

void launch_rows_small(const RowSpace &R, const int32_t *items, const int64_t *seg,
                       const int64_t *cnt, cudaStream_t st, const Dev &d, int *launches) {
  static int occ_b = 0, occ_b8 = 0;
  auto groups = [&](int c, int G, auto kern) {
    if (cnt[c] <= 0) return;
    const int64_t warps = (cnt[c] * G + 31) / 32;
    int64_t blocks = (warps + 7) / 8;
    if (blocks > (int64_t)d.sms * 8) blocks = (int64_t)d.sms * 8;
    kern<<<(int)blocks, 256, 0, st>>>(R, items + seg[c], cnt[c]);
    ++*launches;
  };
  groups(RC_G4, 4, k_rows_group<4>);
  groups(RC_G8, 8, k_rows_group<8>);
  groups(RC_G16, 16, k_rows_group<16>);
  groups(RC_G32, 32, k_rows_group<32>);
  if (cnt[RC_WARP] > 0) {
    int64_t blocks = (cnt[RC_WARP] + 3) / 4;
    if (blocks > (int64_t)d.sms * 10) blocks = (int64_t)d.sms * 10;
    k_rows_warp<RC_WARP_MAX / 32><<<(int)blocks, 128, 0, st>>>(R, items + seg[RC_WARP],
                                                                 cnt[RC_WARP]);
    ++*launches;
  }
  if (cnt[RC_BLOCK] > 0) {
    launch_rows_block<512, RC_BLOCK_MAX / 512>(R, items + seg[RC_BLOCK], cnt[RC_BLOCK], occ_b,
                                               st, d);
    ++*launches;
  }
  if (cnt[RC_BLOCK8K] > 0) {
    launch_rows_block<1024, RC_BLOCK8K_MAX / 1024>(R, items + seg[RC_BLOCK8K], cnt[RC_BLOCK8K],
                                                   occ_b8, st, d);
    ++*launches;
  }
}

// ----------------------------------------- longer rows: global tables ----

// The rows of the big class get tables of next_pow2(2 * bound) slots at
// tbl_off[h] (prefix over the class); insertion units of RC_CHUNK entries
// (unit_off) and compaction units of RC_SCHUNK slots (sunit_off).  A window
// covers the rows whose tables lie in [lo, lo + window) of that prefix.

__global__ void k_big_bounds(const RowSpace R, const int32_t *__restrict__ items, int64_t H,
                             int64_t *bound) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < H;
       h += (int64_t)gridDim.x * blockDim.x) {
    bound[h] = R.boff[items[h] + 1] - R.boff[items[h]];
  }
}

void launch_big_bounds(const RowSpace &R, const int32_t *items, int64_t H, int64_t *bound,
                       cudaStream_t st, const Dev &d) {
  if (H <= 0) return;
  k_big_bounds<<<grid_of(H, 256, d), 256, 0, st>>>(R, items, H, bound);
}

__device__ __forceinline__ int64_t seg_of(const int64_t *__restrict__ off, int64_t n, int64_t x) {
  // largest h in [0, n) with off[h] <= x
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_big_insert(RowSpace R, const int32_t *__restrict__ items,
                                                    BigRows B, int64_t h0, int64_t h1,
                                                    int64_t lo) {
  const int64_t U0 = B.unit_off[h0], U1 = B.unit_off[h1];
  for (int64_t u = U0 + blockIdx.x; u < U1; u += gridDim.x) {
    const int64_t h = seg_of(B.unit_off, B.H, u);
    const Row r = row_of(R, items[h]);
    const int64_t cap = next_pow2(2 * r.cnt);
    const int lg = lg_of(cap);
    int32_t *keys = B.keys + (B.tbl_off[h] - lo);
    unsigned long long *vals = B.vals + (B.tbl_off[h] - lo);
    const int64_t t0 = (u - B.unit_off[h]) * RC_CHUNK;
    const int64_t t1 = t0 + RC_CHUNK < r.cnt ? t0 + RC_CHUNK : r.cnt;
    constexpr int E = RC_CHUNK / 256;
    int32_t cv[E];
    long long w[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      cv[i] = -1;
      w[i] = 0;
      const int64_t t = t0 + threadIdx.x + 256 * i;
      if (t < t1) {
        cv[i] = R.tnbr[r.rb + t];
        w[i] = R.tw[r.rb + t];
      }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if (cv[i] < 0) continue;
      // the table (>= 2 slots per entry) always has room: this loop ends
      const uint64_t mask = (uint64_t)cap - 1;
      uint64_t s = row_home(cv[i], lg);
      for (uint64_t t = 0; t <= mask; ++t) {
        const int32_t prev = atomicCAS(keys + s, -1, cv[i]);
        if (prev == -1 || prev == cv[i]) {
          atomicAdd(vals + s, (unsigned long long)w[i]);
          break;
        }
        s = (s + 1) & mask;
      }
    }
  }
}

// Compaction: a block takes RC_SCHUNK slots of one row's table, counts the
// occupied ones, claims their places with one atomic on ucnt and writes them.
__global__ void __launch_bounds__(256) k_big_compact(RowSpace R, const int32_t *__restrict__ items,
                                                     BigRows B, int64_t h0, int64_t h1,
                                                     int64_t lo) {
  __shared__ int s_wcnt[8];
  __shared__ long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int64_t S0 = B.sunit_off[h0], S1 = B.sunit_off[h1];
  constexpr int PER = RC_SCHUNK / 256;
  for (int64_t su = S0 + blockIdx.x; su < S1; su += gridDim.x) {
    const int64_t h = seg_of(B.sunit_off, B.H, su);
    const Row r = row_of(R, items[h]);
    const int64_t cap = next_pow2(2 * r.cnt);
    const int32_t *keys = B.keys + (B.tbl_off[h] - lo);
    const unsigned long long *vals = B.vals + (B.tbl_off[h] - lo);
    const int64_t s0 = (su - B.sunit_off[h]) * RC_SCHUNK;
    // thread tid owns slots s0 + tid * PER .. + PER (in order)
    int mine = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int64_t s = s0 + (int64_t)tid * PER + i;
      if (s < cap && keys[s] >= 0) ++mine;
    }
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wcnt[wib] = incl;
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int k = 0; k < 8; ++k) {
        const int c = s_wcnt[k];
        s_wcnt[k] = tot;
        tot += c;
      }
      s_base = tot ? (long long)atomicAdd((unsigned long long *)&R.ucnt[r.C],
                                          (unsigned long long)tot)
                   : 0;
    }
    __syncthreads();
    int64_t pos = r.rb + s_base + s_wcnt[wib] + (incl - mine);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int64_t s = s0 + (int64_t)tid * PER + i;
      if (s < cap && keys[s] >= 0) {
        R.tnbr[pos] = keys[s];
        R.tw[pos] = (int64_t)vals[s];
        ++pos;
      }
    }
    __syncthreads();
  }
}

void launch_big_window(const RowSpace &R, const int32_t *items, const BigRows &B, int64_t h0,
                       int64_t h1, int64_t lo, int64_t units, int64_t sunits, cudaStream_t st,
                       const Dev &d, int *launches) {
  if (h1 <= h0) return;
  int64_t g = units < (int64_t)d.sms * 8 ? units : (int64_t)d.sms * 8;
  k_big_insert<<<(int)(g > 0 ? g : 1), 256, 0, st>>>(R, items, B, h0, h1, lo);
  g = sunits < (int64_t)d.sms * 8 ? sunits : (int64_t)d.sms * 8;
  k_big_compact<<<(int)(g > 0 ? g : 1), 256, 0, st>>>(R, items, B, h0, h1, lo);
  *launches += 2;
}

// ------------------------------------------------------------- copy ------

// The unique entries of every row, from the start of its region to offg[C].
// A warp takes 32 consecutive rows: their outputs are one contiguous segment
// [offg[r0], offg[r0 + 32]), written coalesced; each position finds its row
// by a binary search over the 33 offsets held in shared memory.
__global__ void __launch_bounds__(256) k_rows_copy(const RowSpace R, int64_t ntot,
                                                   const int64_t *__restrict__ offg,
                                                   int32_t *nbr_out, int64_t *w_out) {
  __shared__ int64_t s_off[8][33];
  __shared__ int64_t s_src[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * 32; r0 < ntot;
       r0 += warps_total * 32) {
    const int64_t r = r0 + lane;
    s_off[wib][lane] = offg[r < ntot ? r : ntot];
    if (lane == 0) s_off[wib][32] = offg[r0 + 32 < ntot ? r0 + 32 : ntot];
    s_src[wib][lane] = r < ntot ? R.boff[r] : 0;
    __syncwarp();
    const int64_t o0 = s_off[wib][0], o1 = s_off[wib][32];
    const int32_t *__restrict__ tnbr = R.tnbr;
    const int64_t *__restrict__ tw = R.tw;
    // CU positions per lane per step, loads before stores
    constexpr int CU = 4;
    for (int64_t p0 = o0 + lane; p0 < o1; p0 += 32 * CU) {
      int32_t nb[CU];
      int64_t wv[CU];
#pragma unroll
      for (int u = 0; u < CU; ++u) {
        const int64_t p = p0 + 32 * u;
        nb[u] = 0;
        wv[u] = 0;
        if (p < o1) {
          // the last row whose output starts at or before p (rows without
          // entries share their offset with the next row)
          int lo = 0, hi = 32;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[wib][mid] <= p) lo = mid; else hi = mid;
          }
          const int64_t src = s_src[wib][lo] + (p - s_off[wib][lo]);
          nb[u] = __ldcs(tnbr + src);
          wv[u] = __ldcs(tw + src);
        }
      }
#pragma unroll
      for (int u = 0; u < CU; ++u) {
        const int64_t p = p0 + 32 * u;
        if (p < o1) {
          nbr_out[p] = nb[u];
          w_out[p] = wv[u];
        }
      }
    }
    __syncwarp();
  }
}

void launch_rows_copy(const RowSpace &R, int64_t ntot, const int64_t *offg, int32_t *nbr_out,
                      int64_t *w_out, cudaStream_t st, const Dev &d) {
  if (ntot <= 0) return;
  k_rows_copy<<<grid_of((ntot + 31) / 32 * 32, 256, d), 256, 0, st>>>(R, ntot, offg, nbr_out,
                                                                      w_out);
}

// ------------------------------------------------ sorted rows (export) ----

// key = row << 32 | neighbour for every entry of a CSR whose offsets start
// at 0; after a sort of (key, w) the rows keep their ranges and come out
// ascending by neighbour.
__global__ void k_row_keys(const int64_t *__restrict__ off, int64_t n,
                           const int32_t *__restrict__ nbr, uint64_t *keys) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps)
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
      keys[e] = ((uint64_t)v << 32) | (uint32_t)nbr[e];
}

__global__ void k_row_unkey(const uint64_t *__restrict__ keys, int64_t nnz, int32_t *nbr) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    nbr[e] = (int32_t)(uint32_t)keys[e];
}

void launch_row_keys(const int64_t *off, int64_t n, const int32_t *nbr, uint64_t *keys,
                     cudaStream_t st, const Dev &d) {
  if (n <= 0) return;
  k_row_keys<<<grid_of(n * 32, 256, d), 256, 0, st>>>(off, n, nbr, keys);
}

void launch_row_unkey(const uint64_t *keys, int64_t nnz, int32_t *nbr, cudaStream_t st,
                      const Dev &d) {
  if (nnz <= 0) return;
  k_row_unkey<<<grid_of(nnz, 256, d), 256, 0, st>>>(keys, nnz, nbr);
}

}  // namespace lcc
