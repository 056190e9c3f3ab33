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

#include <mutex>
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

// Same rule as the library's best-move kernels (gain of moving v from its
// cluster to a neighbouring one, scaled by q, exact in 128 bits; ties to the
// smallest cluster id; strict improvement over staying; cluster id v with
// zero weight and no neighbour in it as a gain-0 candidate).  One block per
// vertex at a time; the block's table is its slice of the static array.
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
  for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
    const int64_t beg = off[v];
    const int64_t deg = off[v + 1] - beg;
    const int32_t Lv = L[v];
    if (deg > NA_MAX_DEG) {
      if (tid == 0) {
        atomicExch(ctl, 1ull);
        atomicMax(ctl + 1, (unsigned long long)deg);
        D[v] = Lv;
      }
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
      const int32_t c = L[nbr[beg + e]];
      const long long wt = w ? (long long)w[beg + e] : 1;
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
    const lcc::i128 kv = (lcc::i128)k[v];
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
}

std::mutex g_na_mu;
void *g_na_addr[256] = {nullptr};

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
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) throw lcc::Error(LCC_ERR_INVALID, "device index out of range");
    void *base = nullptr;
    {
      // First call on this device: look up where the static array lives.
      std::lock_guard<std::mutex> lk(g_na_mu);
      if (!g_na_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
          cudaGetLastError();
          throw lcc::Error(LCC_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") +
                                             cudaGetErrorString(e));
        }
        g_na_addr[dev] = p;
      }
      base = g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(base, 0, 256, st));  // control block: error flag, longest row
    if (n > 0) {
      k_desired_noalloc<<<NA_BLOCKS, NA_THREADS, 0, st>>>(
          (unsigned char *)base, d_off, d_nbr, d_w, d_k, n, lambda_p, lambda_q, d_labels, d_K,
          d_desired);
      CK(cudaGetLastError());
    }
    unsigned long long ctl[2] = {0, 0};
    CK(cudaMemcpyAsync(ctl, base, sizeof(ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctl[0])
      throw lcc::Error(LCC_ERR_INVALID,
                       "a row has " + std::to_string(ctl[1]) + " entries; the allocation-free "
                       "path handles rows of at most " + std::to_string(NA_MAX_DEG));
    return LCC_OK;
  } catch (const lcc::Error &e) {
    lcc::set_last_error(e.what());
    return e.st;
  } catch (const std::exception &e) {
    lcc::set_last_error(e.what());
    return LCC_ERR_CUDA;
  }
}
