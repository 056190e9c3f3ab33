// Compress (Sec. 3.1, Appendix B) as relabel -> emit -> radix sort ->
// reduce by key -> CSR, over a table of jobs laid out in one flat vertex
// space (vstart[j] = first flat index of job j).
//
//   occ/rank   occupied cluster ids, exclusive scan -> dense coarse ids in
//              increasing cluster-id order; rank[vstart_j + c] is the global
//              coarse id of cluster c of job j;
//   emit       every entry (u, v) whose ends lie in different clusters gives
//              key = (global coarse id of u) << 32 | (local coarse id of v)
//              and value w, at its own entry position; entries inside a
//              cluster get a key that sorts last and are dropped there;
//   sort       LSD radix sort, 8-bit digits, only on the bits in use;
//   reduce     equal keys are summed (parallel edges merged): heads per tile,
//              a scan of the tile counts, then keys and sums per tile;
//   CSR        row r starts at the first unique key >= r << 32.
#include "lcc_internal.cuh"

namespace lcc {

namespace {
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

int grid_for(int64_t work, int threads, const Dev &d, int per_sm = 8) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t mx = (int64_t)d.sms * per_sm;
  if (g > mx) g = mx;
  return (int)(g > 0 ? g : 1);
}
}  // namespace

// --------------------------------------------------------- occupancy ------

__global__ void k_occ(const CJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                      int njobs, int64_t vtot, int64_t *occ, int32_t *err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const CJob *J = jobs + j;
    const int32_t c = J->L[i - vstart[j]];
    if (c < 0 || c >= J->n) {
      *err = 1;
      continue;
    }
    occ[vstart[j] + c] = 1;
  }
}

void launch_occ(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vtot, int64_t *occ,
                int32_t *err, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_occ<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, occ, err);
}

// gmap: global coarse id per flat vertex; gmapp: the same ids in the flat
// positions of the gather layout, so that the emission kernels look
// neighbours up through gnbr with the hot ids sharing an L2-sized region.
__global__ void k_relabel(const CJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                          int njobs, int64_t vtot, const int64_t *__restrict__ rank,
                          int32_t *gmap, int32_t *gmapp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(vstart, njobs, i);
    const CJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    const int64_t g = rank[vstart[j] + J->L[v]];
    gmap[i] = (int32_t)g;
    gmapp[vstart[j] + (J->pos ? J->pos[v] : v)] = (int32_t)g;
    J->map[v] = (int32_t)(g - rank[vstart[j]]);
  }
}

void launch_relabel(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                    const int64_t *rank, int32_t *gmap, int32_t *gmapp, cudaStream_t st,
                    const Dev &d) {
  if (vtot <= 0) return;
  k_relabel<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, rank, gmap,
                                                    gmapp);
}

// k' = K: the coarse vertex of occupied cluster c gets node weight K_c.
__global__ void k_knew(const CJob *__restrict__ jobs, const int64_t *__restrict__ vstart,
                       int njobs, int64_t vtot, const int64_t *__restrict__ rank, int64_t *knew) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vtot;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (rank[i + 1] == rank[i]) continue;
    const int j = find_job(vstart, njobs, i);
    knew[rank[i]] = jobs[j].K[i - vstart[j]];
  }
}

void launch_knew(const CJob *jobs, const int64_t *vstart, int njobs, int64_t vtot,
                 const int64_t *rank, int64_t *knew, cudaStream_t st, const Dev &d) {
  if (vtot <= 0) return;
  k_knew<<<grid_for(vtot, 256, d), 256, 0, st>>>(jobs, vstart, njobs, vtot, rank, knew);
}

__global__ void k_job_counts(const int64_t *vstart, int njobs, const int64_t *rank, int64_t *out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < njobs; j += gridDim.x * blockDim.x) {
    out[2 * j] = rank[vstart[j + 1]] - rank[vstart[j]];  // n'_j
    out[2 * j + 1] = rank[vstart[j]];                     // first global coarse id
  }
}

void launch_job_counts(const int64_t *vstart, int njobs, const int64_t *rank, int64_t *out,
                       cudaStream_t st) {
  if (njobs <= 0) return;
  k_job_counts<<<(njobs + 255) / 256, 256, 0, st>>>(vstart, njobs, rank, out);
}

// ------------------------------------------------------------- emission --

// Every entry (u, v) of every job is written at its flat entry position
// estart[j] + (e - off[0]) (a coarse level of a contraction batch indexes a
// shared entry array, so its offsets need not start at 0):
// key = (global coarse id of u) << 32 | (local coarse id of v)
// and value w; an entry inside a cluster gets the key EMIT_INTRA instead,
// which sorts after every real pair (the sort covers the high half on
// bits_for(ntot + 1) bits, on which no coarse id is all ones), so the sorted
// array ends with the intra entries and the reduction stops before them.
// `intra` counts them.
__global__ void __launch_bounds__(256) k_emit_all(const CJob *__restrict__ jobs,
                                                  const int64_t *__restrict__ vstart,
                                                  const int64_t *__restrict__ estart, int njobs,
                                                  int64_t vtot, const int32_t *__restrict__ gmap,
                                                  const int32_t *__restrict__ gmapp,
                                                  const int64_t *__restrict__ rank, uint64_t *keys,
                                                  int64_t *vals, unsigned long long *intra) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  long long my_intra = 0;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < vtot;
       i += warps_total) {
    const int j = find_job(vstart, njobs, i);
    const CJob *J = jobs + j;
    const int64_t v = i - vstart[j];
    const int64_t vs = vstart[j];
    const int64_t es = estart[j] - J->off[0];
    const int64_t cbase = rank[vs];
    const uint64_t cu = (uint64_t)(uint32_t)gmap[i];
    const int64_t beg = J->off[v], end = J->off[v + 1];
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t cv = gmapp[vs + __ldg(J->gnbr + e)];
      const bool in = (uint32_t)cv == (uint32_t)cu;
      keys[es + e] = in ? EMIT_INTRA : ((cu << 32) | (uint64_t)(uint32_t)(cv - cbase));
      vals[es + e] = load_w(J->w, J->wtype, e);
      my_intra += in ? 1 : 0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_intra += __shfl_xor_sync(FULL, my_intra, o);
  if (lane == 0 && my_intra) atomicAdd(intra, (unsigned long long)my_intra);
}

void launch_emit_all(const CJob *jobs, const int64_t *vstart, const int64_t *estart, int njobs,
                     int64_t vtot, const int32_t *gmap, const int32_t *gmapp, const int64_t *rank,
                     uint64_t *keys, int64_t *vals, unsigned long long *intra, cudaStream_t st,
                     const Dev &d) {
  if (vtot <= 0) return;
  k_emit_all<<<grid_for(vtot * 32, 256, d), 256, 0, st>>>(jobs, vstart, estart, njobs, vtot, gmap,
                                                          gmapp, rank, keys, vals, intra);
}

// ----------------------------------------------------------------- scan --

constexpr int SCAN_T = 256, SCAN_I = 16, SCAN_TILE = SCAN_T * SCAN_I;

__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t *total) {
  __shared__ int64_t wsum[SCAN_T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  int64_t wprefix = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < SCAN_T / 32; ++k) {
    const int64_t s = wsum[k];
    if (k < w) wprefix += s;
    tot += s;
  }
  __syncthreads();
  *total = tot;
  return wprefix + inc - x;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int64_t *a, int64_t n, int64_t *sums) {
  __shared__ int64_t red[SCAN_T / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
    const int64_t idx = base + i;
    if (idx < n) s += a[idx];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int k = 0; k < SCAN_T / 32; ++k) t += red[k];
    sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(int64_t *a, int64_t n,
                                                       const int64_t *tile_off) {
  __shared__ int64_t s[SCAN_TILE];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
    const int64_t idx = base + i;
    s[i] = idx < n ? a[idx] : 0;
  }
  __syncthreads();
  int64_t loc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) loc += s[threadIdx.x * SCAN_I + k];
  int64_t tot;
  int64_t run = block_excl_scan(loc, &tot) + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_I; ++k) {
    const int64_t t = s[threadIdx.x * SCAN_I + k];
    s[threadIdx.x * SCAN_I + k] = run;
    run += t;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
    const int64_t idx = base + i;
    if (idx < n) a[idx] = s[i];
  }
}

int64_t scan_tmp_elems(int64_t n) {
  int64_t tot = 0;
  int64_t m = n + 1;
  while (true) {
    const int64_t tiles = (m + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) break;
    tot += tiles + 1;
    m = tiles + 1;
  }
  return tot + 1;
}

static void scan_rec(int64_t *a, int64_t m, int64_t *tmp, cudaStream_t st) {
  const int64_t tiles = (m + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles <= 1) {
    k_scan_apply<<<1, SCAN_T, 0, st>>>(a, m, nullptr);
    return;
  }
  k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, st>>>(a, m, tmp);
  cudaMemsetAsync(tmp + tiles, 0, sizeof(int64_t), st);
  scan_rec(tmp, tiles + 1, tmp + tiles + 1, st);
  k_scan_apply<<<(unsigned)tiles, SCAN_T, 0, st>>>(a, m, tmp);
}

void scan_exclusive_i64(int64_t *a, int64_t n, int64_t *tmp, cudaStream_t st, const Dev &) {
  // a has n + 1 elements; the caller zeroes a[n] so that it receives the total
  scan_rec(a, n + 1, tmp, st);
}

// ----------------------------------------------------------- radix sort --

constexpr int RS_T = 256, RS_I = 16, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;
constexpr int RS_WRUN = RS_TILE / RS_W;  // contiguous elements ranked by one warp

// Per-tile digit counts (one shared atomic per element: this measured faster
// than aggregating equal digits across lanes first, even on skewed digits).
__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t *keys, int64_t n, int shift,
                                                  int64_t ntiles, int64_t *ghist) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_T) {
    const int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  ghist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  Warp w ranks elements [w * RS_WRUN, (w + 1) *
// RS_WRUN) of the tile in index order with warp-private digit counters; a
// per-digit prefix over the warps and an exclusive scan over the digits give
// every element its place in the tile sorted by digit (ties in index order).
// The tile is rearranged in shared memory and written out so that consecutive
// threads store consecutive places of one digit's run (coalesced), after
// everything of smaller digit or earlier tile (tile-major offsets goff).
__global__ void __launch_bounds__(RS_T, 3) k_rs_scatter(const uint64_t *__restrict__ keys,
                                                     const int64_t *__restrict__ vals, int64_t n,
                                                     int shift, int64_t ntiles,
                                                     const int64_t *__restrict__ goff,
                                                     uint64_t *keys_out, int64_t *vals_out) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t *s_key = (uint64_t *)rs_smem;
  int64_t *s_val = (int64_t *)(s_key + RS_TILE);
  __shared__ int wcnt[RS_W][256];
  __shared__ int dstart[256];
  __shared__ int wsum[RS_W];
  __shared__ int64_t gbase[256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int k = 0; k < RS_W; ++k) wcnt[k][tid] = 0;
  gbase[tid] = goff[(int64_t)tid * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t wbase = tile0 + (int64_t)w * RS_WRUN;
  uint64_t key[RS_I];
  int lr[RS_I];
#pragma unroll
  for (int r = 0; r < RS_I; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    const bool has = idx < n;
    key[r] = has ? keys[idx] : 0ull;
    const int dg = has ? (int)((key[r] >> shift) & 255u) : 256 + lane;
    const unsigned peers = __match_any_sync(FULL, dg);
    lr[r] = has ? wcnt[w][dg] + __popc(peers & lanemask_lt()) : 0;
    __syncwarp();
    if (has && lane == __ffs(peers) - 1) wcnt[w][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // digit tid: exclusive prefix over the warps, then the tile's digit starts
  int tot = 0;
#pragma unroll
  for (int k = 0; k < RS_W; ++k) {
    const int c = wcnt[k][tid];
    wcnt[k][tid] = tot;
    tot += c;
  }
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < w; ++k) before += wsum[k];
  dstart[tid] = before + incl - tot;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_I; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    if (idx < n) {
      const int dg = (int)((key[r] >> shift) & 255u);
      const int pos = dstart[dg] + wcnt[w][dg] + lr[r];
      s_key[pos] = key[r];
      s_val[pos] = vals[idx];
    }
  }
  __syncthreads();
  const int64_t rem = n - tile0;
  const int cnt = rem < RS_TILE ? (int)rem : RS_TILE;
#pragma unroll 4
  for (int p = tid; p < cnt; p += RS_T) {
    const uint64_t k = s_key[p];
    const int dg = (int)((k >> shift) & 255u);
    const int64_t g = gbase[dg] + (p - dstart[dg]);
    keys_out[g] = k;
    vals_out[g] = s_val[p];
  }
}

constexpr size_t RS_SMEM = (size_t)RS_TILE * 16;

int64_t radix_tmp_elems(int64_t n) {
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  const int64_t m = 256 * ntiles;
  return m + 1 + scan_tmp_elems(m);
}

void radix_sort_pairs(uint64_t *keys, int64_t *vals, uint64_t *keys_alt, int64_t *vals_alt,
                      int64_t n, const int *shifts, int npasses, int64_t *tmp, cudaStream_t st,
                      const Dev &d, bool *result_in_alt, int *launches) {
  *result_in_alt = false;
  if (n <= 1 || npasses == 0) return;
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  const int64_t m = 256 * ntiles;
  int64_t *ghist = tmp;
  int64_t *stmp = tmp + m + 1;
  uint64_t *ki = keys, *ko = keys_alt;
  int64_t *vi = vals, *vo = vals_alt;
  // (a refusal shows up as the launch error of the first scatter)
  (void)cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RS_SMEM);
  for (int p = 0; p < npasses; ++p) {
    k_rs_hist<<<(unsigned)ntiles, RS_T, 0, st>>>(ki, n, shifts[p], ntiles, ghist);
    cudaMemsetAsync(ghist + m, 0, sizeof(int64_t), st);
    scan_exclusive_i64(ghist, m, stmp, st, d);
    k_rs_scatter<<<(unsigned)ntiles, RS_T, RS_SMEM, st>>>(ki, vi, n, shifts[p], ntiles, ghist, ko,
                                                          vo);
    *launches += 3;
    uint64_t *tk = ki; ki = ko; ko = tk;
    int64_t *tv = vi; vi = vo; vo = tv;
  }
  *result_in_alt = (npasses & 1) != 0;
}

// ---------------------------------------------------- reduce by key ----

// Sorted keys in tiles of RB_TILE (16 rounds of 256 consecutive elements).  A
// head is the first element of a run of equal keys; run r of the whole array
// goes to ukeys[r] / uvals[r].
constexpr int RB_T = 256, RB_I = 16, RB_TILE = RB_T * RB_I, RB_W = RB_T / 32;

__device__ __forceinline__ bool is_head(const uint64_t *__restrict__ keys, int64_t i) {
  return i == 0 || keys[i] != keys[i - 1];
}

// Heads per tile (the scan of these gives each tile's first run).
__global__ void __launch_bounds__(RB_T) k_rb_count(const uint64_t *__restrict__ keys, int64_t n,
                                                   int64_t *tile_heads) {
  __shared__ int wsum[RB_W];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * RB_TILE;
  int c = 0;
#pragma unroll 4
  for (int r = 0; r < RB_I; ++r) {
    const int64_t i = t0 + r * RB_T + tid;
    c += (i < n && is_head(keys, i)) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
  if (lane == 0) wsum[w] = c;
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int k = 0; k < RB_W; ++k) t += wsum[k];
    tile_heads[blockIdx.x] = t;
  }
}

// Unique keys and sums.  Heads are ranked in index order from per-(round,
// warp) ballot counts; values are summed per run inside each 32-element chunk
// by a segmented warp scan.  A run wholly inside one chunk is stored; parts of
// runs that cross a chunk are added atomically (uvals is zeroed beforehand).
__global__ void __launch_bounds__(RB_T) k_rb_write(const uint64_t *__restrict__ keys,
                                                   const int64_t *__restrict__ vals, int64_t n,
                                                   const int64_t *__restrict__ tile_off,
                                                   uint64_t *ukeys, int64_t *uvals) {
  __shared__ int cnt[RB_I * RB_W];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * RB_TILE;
  unsigned hmask = 0;
#pragma unroll
  for (int r = 0; r < RB_I; ++r) {
    const int64_t i = t0 + r * RB_T + tid;
    const bool h = i < n && is_head(keys, i);
    hmask |= (h ? 1u : 0u) << r;
    const unsigned b = __ballot_sync(FULL, h);
    if (lane == 0) cnt[r * RB_W + w] = __popc(b);
  }
  __syncthreads();
  if (w == 0) {  // exclusive prefix of the 128 counts in index order (round, warp)
    int v[RB_I * RB_W / 32];
    int tot = 0;
#pragma unroll
    for (int k = 0; k < RB_I * RB_W / 32; ++k) {
      v[k] = cnt[lane * (RB_I * RB_W / 32) + k];
      tot += v[k];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    int run = incl - tot;
#pragma unroll
    for (int k = 0; k < RB_I * RB_W / 32; ++k) {
      cnt[lane * (RB_I * RB_W / 32) + k] = run;
      run += v[k];
    }
  }
  __syncthreads();
  const int64_t base = tile_off[blockIdx.x];
#pragma unroll 2
  for (int r = 0; r < RB_I; ++r) {
    const int64_t i = t0 + r * RB_T + tid;
    const bool valid = i < n;
    const bool h = (hmask >> r) & 1u;
    const unsigned b = __ballot_sync(FULL, h);
    const int64_t before = base + cnt[r * RB_W + w] + __popc(b & lanemask_lt());
    // run of element i (the previous tile's last run before this tile's first head)
    const int64_t run = valid ? before + (h ? 1 : 0) - 1 : INT64_MAX;
    uint64_t key = 0;
    long long v = 0;
    if (valid) {
      key = keys[i];
      v = vals[i];
      if (h) ukeys[before] = key;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(FULL, v, o);
      const int64_t ry = __shfl_up_sync(FULL, run, o);
      if (lane >= o && ry == run) v += y;
    }
    const int64_t nrun = __shfl_down_sync(FULL, run, 1);
    const unsigned same = __match_any_sync(FULL, run);
    if (valid && (lane == 31 || nrun != run)) {  // last element of the run in this chunk
      const bool starts = (b >> (__ffs(same) - 1)) & 1u;
      bool ends;
      if (lane < 31)
        ends = true;  // the next lane starts another run or lies past the end
      else
        ends = i + 1 >= n || keys[i + 1] != key;
      if (starts && ends)
        uvals[run] = v;
      else
        atomic_add_i64(uvals + run, v);
    }
  }
}

int64_t rb_tiles(int64_t n) { return (n + RB_TILE - 1) / RB_TILE; }

void launch_rb_count(const uint64_t *keys, int64_t n, int64_t *tile_heads, cudaStream_t st) {
  if (n <= 0) return;
  k_rb_count<<<(unsigned)rb_tiles(n), RB_T, 0, st>>>(keys, n, tile_heads);
}

void launch_rb_write(const uint64_t *keys, const int64_t *vals, int64_t n, const int64_t *tile_off,
                     uint64_t *ukeys, int64_t *uvals, cudaStream_t st) {
  if (n <= 0) return;
  k_rb_write<<<(unsigned)rb_tiles(n), RB_T, 0, st>>>(keys, vals, n, tile_off, ukeys, uvals);
}


__global__ void k_csr_rows(const uint64_t *__restrict__ ukeys, int64_t nu, int64_t nrows,
                           int64_t *offg, int32_t *nbr_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= nrows; r += stride) {
    const uint64_t target = (uint64_t)r << 32;
    int64_t lo = 0, hi = nu;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ukeys[mid] < target) lo = mid + 1; else hi = mid;
    }
    offg[r] = lo;
  }
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += stride)
    nbr_out[u] = (int32_t)(uint32_t)(ukeys[u] & 0xffffffffull);
}

void launch_csr_rows(const uint64_t *ukeys, int64_t nu, int64_t nrows, int64_t *offg,
                     int32_t *nbr_out, cudaStream_t st, const Dev &d) {
  const int64_t work = (nu > nrows + 1) ? nu : nrows + 1;
  k_csr_rows<<<grid_for(work, 256, d), 256, 0, st>>>(ukeys, nu, nrows, offg, nbr_out);
}

}  // namespace lcc
