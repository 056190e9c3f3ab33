// lcc_desired_noalloc: one synchronous best-move evaluation that performs no
// device-memory allocation of any kind.
//
// Who needs this: callers that must not call cudaMalloc (or any allocating
// library routine) at the time they run the evaluation -- for example code
// running inside a memory-budgeted host runtime that owns every device
// allocation itself, or a process that has handed the rest of the GPU's
// memory to another allocator and only lends this library pre-allocated input
// and output buffers.  Every other entry point of the library allocates its
// working memory from a stream-ordered pool; this one does not.
//
// Its hash tables live in one fixed, file-scope device array (below) that is
// part of the loaded library image: every GPU that loads the library holds it
// until the process exits.  The array is shared by all calls on a device and
// keeps whatever the previous call left in it; the call clears what must start
// at zero.  Two calls whose kernels overlap on the GPU (for example on two
// streams) race on the array, so such calls must be ordered by the caller.
#include <cuda_runtime.h>

#include <string>

#include "engine.h"

namespace lcc {
void set_last_error(const std::string &m);
}

namespace {

// 16 MiB: a 256-byte control block, then one hash table per block of the
// kernel's fixed grid.
constexpr size_t NA_SCRATCH_BYTES = (size_t)16 << 20;
constexpr int NA_BLOCKS = 160;
constexpr int NA_THREADS = 256;
constexpr int NA_CAP = 8192;            // table slots per block
constexpr int NA_MAX_DEG = NA_CAP / 2;  // longest row the tables can aggregate
constexpr size_t NA_TABLE_BYTES = (size_t)NA_CAP * (4 + 8);
static_assert(256 + (size_t)NA_BLOCKS * NA_TABLE_BYTES <= NA_SCRATCH_BYTES,
              "scratch too small for the fixed grid");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t na_slot(int32_t c, int lg) {
  const uint64_t h = (uint64_t)(uint32_t)c * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(h >> (64 - lg));
}

__device__ __forceinline__ bool na_better(lcc::i128 s1, int32_t c1, lcc::i128 s2, int32_t c2) {
  return s1 > s2 || (s1 == s2 && c1 < c2);
}

// Words of the 256-byte control block at the start of the scratch array.
enum : int {
  NA_LONG_ROW = 0,  // a row is longer than NA_MAX_DEG
  NA_MAX_ROW = 1,   // the longest such row
  NA_BAD_ID = 2,    // a neighbour id or a label outside [0, n)
  NA_NEG = 3,       // a negative node weight or cluster weight
  NA_WABS = 4,      // sum of |w| over the rows evaluated
  NA_WSAT = 5,      // ... reached 2^62
  NA_KSUM = 6,      // sum of the node weights
  NA_KSAT = 7,      // ... reached 2^62
  NA_KMAX = 8       // largest cluster weight K[c]
};
constexpr unsigned long long NA_LIM62 = 1ull << 62;

// Adds a non-negative x < 2^62 to a running total, raising *sat instead once
// the total would reach 2^62.
__device__ __forceinline__ void na_add_sat(unsigned long long &acc, unsigned long long x,
                                           unsigned long long &sat) {
  if (x >= NA_LIM62 - acc) sat = 1;
  else acc += x;
}

// Adds a partial total (< 2^62) into a control word; the add that carries the
// word past 2^62 sees it, so wrapping cannot hide a large total.
__device__ __forceinline__ void na_flush_sat(unsigned long long *ctl, int word, int satword,
                                             unsigned long long acc, unsigned long long sat) {
  if (acc) {
    const unsigned long long old = atomicAdd(ctl + word, acc);
    if (old >= NA_LIM62 || old + acc >= NA_LIM62) sat = 1;
  }
  if (sat) atomicOr(ctl + satword, 1ull);
}

// Same rule as the library's best-move kernels (gain of moving v from its
// cluster to a neighbouring one, scaled by q, exact in 128 bits; ties to the
// smallest cluster id; strict improvement over staying; cluster id v with
// zero weight and no neighbour in it as a gain-0 candidate).  One block per
// vertex at a time; the block's table is its slice of the static array.
// Besides D, the kernel records in the control block what the host needs to
// refuse inputs it cannot handle exactly: ids out of range (those entries are
// skipped), negative weights, the totals sum|w| and sum k, and the largest K.
__global__ void __launch_bounds__(NA_THREADS)
    k_desired_noalloc(unsigned char *scratch, const int64_t *__restrict__ off,
                      const int32_t *__restrict__ nbr, const int32_t *__restrict__ w,
                      const int64_t *__restrict__ k, int64_t n, int64_t p, int64_t q,
                      const int32_t *__restrict__ L, const int64_t *__restrict__ K,
                      int32_t *__restrict__ D) {
  __shared__ lcc::i128 red_s[NA_THREADS / 32];
  __shared__ int32_t red_c[NA_THREADS / 32];
  __shared__ long long red_w[NA_THREADS / 32];
  __shared__ int red_v[NA_THREADS / 32];
  unsigned long long *ctl = (unsigned long long *)scratch;
  int32_t *tkey = (int32_t *)(scratch + 256 + (size_t)blockIdx.x * NA_TABLE_BYTES);
  unsigned long long *tval = (unsigned long long *)(tkey + NA_CAP);
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  unsigned long long wacc = 0, wsat = 0, kacc = 0, ksat = 0, kmaxK = 0;
  int bad = 0, neg = 0;
  for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
    const int64_t beg = off[v];
    const int64_t deg = off[v + 1] - beg;
    const int32_t Lv = L[v];
    const int64_t kv64 = k[v];
    if (tid == 0) {
      // node weight of v and cluster weight of id v: every id is visited once
      const int64_t Kv = K[v];
      if (kv64 < 0 || Kv < 0) neg = 1;
      else {
        na_add_sat(kacc, (unsigned long long)kv64, ksat);
        if ((unsigned long long)Kv > kmaxK) kmaxK = (unsigned long long)Kv;
      }
      if (Lv < 0 || (int64_t)Lv >= n) bad = 1;
    }
    if (deg > NA_MAX_DEG) {
      if (tid == 0) {
        atomicExch(ctl + NA_LONG_ROW, 1ull);
        atomicMax(ctl + NA_MAX_ROW, (unsigned long long)deg);
        D[v] = Lv;
      }
      continue;
    }
    if (Lv < 0 || (int64_t)Lv >= n) {  // uniform over the block
      if (tid == 0) D[v] = Lv;
      continue;
    }
    int cap = 2;
    while (cap < 2 * deg) cap <<= 1;
    const int lg = 63 - __clzll((long long)cap);
    for (int s = tid; s < cap; s += NA_THREADS) {
      tkey[s] = -1;
      tval[s] = 0;
    }
    __syncthreads();
    for (int64_t e = tid; e < deg; e += NA_THREADS) {
      const int32_t u = nbr[beg + e];
      const long long wt = w ? (long long)w[beg + e] : 1;
      na_add_sat(wacc, (unsigned long long)(wt < 0 ? -wt : wt), wsat);
      if (u < 0 || (int64_t)u >= n) {
        bad = 1;
        continue;
      }
      const int32_t c = L[u];
      if (c < 0 || (int64_t)c >= n) {
        bad = 1;
        continue;
      }
      uint32_t s = na_slot(c, lg);
      for (int t = 0; t < cap; ++t) {
        const int32_t prev = atomicCAS(tkey + s, -1, c);
        if (prev == -1 || prev == c) {
          atomicAdd(tval + s, (unsigned long long)wt);
          break;
        }
        s = (s + 1) & (uint32_t)(cap - 1);
      }
    }
    __syncthreads();
    const lcc::i128 kv = (lcc::i128)kv64;
    lcc::i128 best = (lcc::i128)((unsigned __int128)1 << 127);
    int32_t bc = INT32_MAX;
    long long w_stay = 0;
    int vseen = 0;
    for (int s = tid; s < cap; s += NA_THREADS) {
      const int32_t c = tkey[s];
      if (c < 0) continue;
      const long long val = (long long)tval[s];
      if (c == Lv) {
        w_stay = val;
        continue;
      }
      vseen |= (c == (int32_t)v);
      const lcc::i128 sc = (lcc::i128)q * val - (lcc::i128)p * kv * (lcc::i128)K[c];
      if (na_better(sc, c, best, bc)) {
        best = sc;
        bc = c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long lo = (long long)(uint64_t)best, hi = (long long)(best >> 64);
      lo = __shfl_xor_sync(FULL, lo, o);
      hi = __shfl_xor_sync(FULL, hi, o);
      const lcc::i128 os = ((lcc::i128)hi << 64) | (lcc::i128)(uint64_t)lo;
      const int32_t oc = __shfl_xor_sync(FULL, bc, o);
      if (na_better(os, oc, best, bc)) {
        best = os;
        bc = oc;
      }
      w_stay += __shfl_xor_sync(FULL, w_stay, o);
      vseen |= __shfl_xor_sync(FULL, vseen, o);
    }
    if (lane == 0) {
      red_s[wib] = best;
      red_c[wib] = bc;
      red_w[wib] = w_stay;
      red_v[wib] = vseen;
    }
    __syncthreads();
    if (tid == 0) {
      lcc::i128 bs = red_s[0];
      int32_t bcc = red_c[0];
      long long ws = red_w[0];
      int vs = red_v[0];
      for (int i = 1; i < NA_THREADS / 32; ++i) {
        if (na_better(red_s[i], red_c[i], bs, bcc)) {
          bs = red_s[i];
          bcc = red_c[i];
        }
        ws += red_w[i];
        vs |= red_v[i];
      }
      if (Lv != (int32_t)v && !vs && K[v] == 0 && na_better(0, (int32_t)v, bs, bcc)) {
        bs = 0;
        bcc = (int32_t)v;
      }
      const lcc::i128 stay = (lcc::i128)q * ws - (lcc::i128)p * kv * ((lcc::i128)K[Lv] - kv);
      D[v] = (bcc != INT32_MAX && bs > stay) ? bcc : Lv;
    }
    __syncthreads();
  }
  if (bad) atomicOr(ctl + NA_BAD_ID, 1ull);
  if (neg) atomicOr(ctl + NA_NEG, 1ull);
  na_flush_sat(ctl, NA_WABS, NA_WSAT, wacc, wsat);
  na_flush_sat(ctl, NA_KSUM, NA_KSAT, kacc, ksat);
  if (kmaxK) atomicMax(ctl + NA_KMAX, kmaxK);
}

}  // namespace

extern "C" lcc_status lcc_desired_noalloc(const int64_t *d_off, const int32_t *d_nbr,
                                          const int32_t *d_w, const int64_t *d_k, int64_t n,
                                          int64_t lambda_p, int64_t lambda_q,
                                          const int32_t *d_labels, const int64_t *d_K,
                                          int32_t *d_desired, void *stream) {
  try {
    if (n < 0 || n >= ((int64_t)1 << 31) - 1) throw lcc::Error(LCC_ERR_INVALID, "n out of range");
    if (lambda_p <= 0 || lambda_q <= 0)
      throw lcc::Error(LCC_ERR_INVALID, "lambda_p and lambda_q must be positive");
    if (!d_off || (n > 0 && (!d_nbr || !d_k || !d_labels || !d_K || !d_desired)))
      throw lcc::Error(LCC_ERR_INVALID, "NULL device pointer");
    // Device address of the static array on the current device.  In host code
    // the array's name only stands in for it; the address is looked up on
    // every call (a cheap query once the module is loaded), so it stays right
    // after a device reset reloads the module.  The first call on a device may
    // be the one that loads the module, and with it the array.
    void *base = nullptr;
    {
      const cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
      if (e != cudaSuccess || !base) {
        cudaGetLastError();
        throw lcc::Error(LCC_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") +
                                           cudaGetErrorString(e));
      }
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(base, 0, 256, st));  // control block
    if (n > 0) {
      k_desired_noalloc<<<NA_BLOCKS, NA_THREADS, 0, st>>>(
          (unsigned char *)base, d_off, d_nbr, d_w, d_k, n, lambda_p, lambda_q, d_labels, d_K,
          d_desired);
      CK(cudaGetLastError());
    }
    unsigned long long ctl[16] = {0};
    CK(cudaMemcpyAsync(ctl, base, sizeof(ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctl[NA_BAD_ID])
      throw lcc::Error(LCC_ERR_INVALID, "a neighbour id or a label is outside [0, n)");
    if (ctl[NA_NEG]) throw lcc::Error(LCC_ERR_INVALID, "negative node or cluster weight");
    if (ctl[NA_LONG_ROW])
      throw lcc::Error(LCC_ERR_INVALID,
                       "a row has " + std::to_string(ctl[NA_MAX_ROW]) + " entries; the "
                       "allocation-free path handles rows of at most " + std::to_string(NA_MAX_DEG));
    // the exact range of the library's other entry points: every gain term
    // (q w(v,C) and p k_v K_C, with K_C at most the total node weight) below 2^125
    {
      typedef lcc::i128 I;
      const I lim = (I)1 << 125;
      const I wa = (I)ctl[NA_WABS], kt = (I)ctl[NA_KSUM];
      if (ctl[NA_WSAT] || ctl[NA_KSAT] || wa >= ((I)1 << 62) || kt >= ((I)1 << 62) ||
          (I)lambda_q * wa >= lim || (kt > 0 && (I)lambda_p > (lim - 1) / (kt * kt)))
        throw lcc::Error(LCC_ERR_OVERFLOW,
                         "q * sum|w| or p * (sum k)^2 reaches 2^125: outside the exact integer range");
      if ((I)ctl[NA_KMAX] > kt)
        throw lcc::Error(LCC_ERR_INVALID, "a cluster weight exceeds the total node weight");
    }
    return LCC_OK;
  } catch (const lcc::Error &e) {
    lcc::set_last_error(e.what());
    return e.st;
  } catch (const std::exception &e) {
    lcc::set_last_error(e.what());
    return LCC_ERR_CUDA;
  }
}
