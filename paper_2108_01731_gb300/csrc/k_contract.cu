// The first steps of Compress (Sec. 3.1, Appendix B) over a table of jobs
// laid out in one flat vertex space (vstart[j] = first flat index of job j),
// plus the scan and the radix sort they and the exported graphs use:
//
//   occ/rank   occupied cluster ids, exclusive scan -> dense coarse ids in
//              increasing cluster-id order; rank[vstart_j + c] is the global
//              coarse id of cluster c of job j;
//   relabel    the global coarse id of every vertex (gmap, and gmapp at the
//              positions of the gather layout) and its job-local one (map);
//   knew       the coarse node weights k' = K;
//   scan       exclusive scan of int64;
//   sort       LSD radix sort of (key, value) pairs, 8-bit digits, only on
//              the bits in use (the rows of an exported coarse graph).
//
// The aggregation of the coarse rows is in k_rows.cu.
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

}  // namespace lcc
