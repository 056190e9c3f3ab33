// extern "C" entry points of liblcc (declared in include/lcc.h) and the
// serving engine's worker thread.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "engine.h"

using namespace lcc;

namespace lcc {
void launch_validate_rows(const int64_t *off, const int32_t *nbr, const int32_t *w, int64_t n,
                          unsigned long long *out8, cudaStream_t st, const Dev &d);
}

static thread_local std::string t_err;

namespace lcc {
void set_last_error(const std::string &m) { t_err = m; }
}

#define API_BEGIN try {
#define API_END                                   \
  }                                               \
  catch (const Error &e) {                        \
    t_err = e.what();                             \
    return e.st;                                  \
  }                                               \
  catch (const std::bad_alloc &) {                \
    t_err = "host allocation failed";             \
    return LCC_ERR_OOM;                           \
  }                                               \
  catch (const std::exception &e) {               \
    t_err = e.what();                             \
    return LCC_ERR_CUDA;                          \
  }                                               \
  catch (...) {                                   \
    t_err = "unknown error";                      \
    return LCC_ERR_CUDA;                          \
  }                                               \
  return LCC_OK;

static void fail(lcc_status s, const std::string &m) { throw Error(s, m); }

static lcc_schedule default_schedule() {
  lcc_schedule s;
  s.num_iter = 10;
  s.max_levels = 64;
  s.refine = 1;
  s.vset = LCC_VSET_NBR_VERTICES;
  s.sync = 1;
  s.flags = 0;
  s.seed = 0;
  return s;
}

static lcc_schedule check_schedule(const lcc_schedule *sched) {
  lcc_schedule s = sched ? *sched : default_schedule();
  if (s.num_iter < 0) fail(LCC_ERR_INVALID, "num_iter must be >= 0");
  if (s.max_levels < 1) fail(LCC_ERR_INVALID, "max_levels must be >= 1");
  if (s.vset < 0 || s.vset > 2) fail(LCC_ERR_INVALID, "unknown vertex-subset rule");
  if (s.sync != 1) fail(LCC_ERR_INVALID, "only the synchronous schedule is implemented");
  return s;
}

static void check_lambda(int64_t p, int64_t q, int32_t mode) {
  if (p <= 0 || q <= 0) fail(LCC_ERR_INVALID, "lambda_p and lambda_q must be positive");
  if (mode < 0 || mode > 2) fail(LCC_ERR_INVALID, "unknown node-weight mode");
}

static void check_graph(const lcc_graph *g) {
  if (!g) fail(LCC_ERR_INVALID, "graph is NULL");
  CK(cudaSetDevice(g->dev));
}

static void check_labels(const int32_t *labels, int64_t n) {
  if (!labels && n > 0) fail(LCC_ERR_INVALID, "labels is NULL");
  for (int64_t v = 0; v < n; ++v)
    if (labels[v] < 0 || labels[v] >= n) fail(LCC_ERR_INVALID, "label out of range [0, n)");
}

// Loads and validates a CSR graph on the current device.
static lcc_graph *load_graph(const int64_t *offsets, const int32_t *nbrs, const int32_t *weights,
                             int64_t n, int64_t nnz, const int64_t *node_w, int32_t memspace,
                             cudaStream_t st) {
  if (n < 0 || nnz < 0) fail(LCC_ERR_INVALID, "negative size");
  if (n >= ((int64_t)1 << 31) - 1) fail(LCC_ERR_OVERFLOW, "n must be below 2^31 - 1");
  if (!offsets) fail(LCC_ERR_INVALID, "offsets is NULL");
  if (nnz > 0 && !nbrs) fail(LCC_ERR_INVALID, "nbrs is NULL");
  if (memspace != LCC_MEM_HOST && memspace != LCC_MEM_DEVICE)
    fail(LCC_ERR_INVALID, "unknown memory space");
  int dev;
  CK(cudaGetDevice(&dev));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  Dev d{sms, dev};
  std::unique_ptr<lcc_graph> g(new lcc_graph());
  g->dev = dev;
  g->st = st;
  g->n = n;
  g->nnz = nnz;
  g->store = std::make_shared<Store>(st);
  g->off = g->store->alloc<int64_t>(n + 1);
  g->nbr = g->store->alloc<int32_t>(nnz);
  const cudaMemcpyKind kind =
      memspace == LCC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(g->off, offsets, (n + 1) * 8, kind, st));
  if (nnz > 0) CK(cudaMemcpyAsync(g->nbr, nbrs, nnz * 4, kind, st));
  if (weights) {
    int32_t *w = g->store->alloc<int32_t>(nnz);
    if (nnz > 0) CK(cudaMemcpyAsync(w, weights, nnz * 4, kind, st));
    g->w = w;
    g->wtype = W_I32;
  }
  if (node_w) {
    g->kc = g->store->alloc<int64_t>(n);
    if (n > 0) CK(cudaMemcpyAsync(g->kc, node_w, n * 8, kind, st));
  }
  Store tmp(st);
  unsigned long long *v = tmp.alloc<unsigned long long>(10);
  // results come back to pageable memory: each such copy returns once done
  // (a pinned buffer per call would cost more than the copies)
  unsigned long long h[10];
  CK(cudaMemsetAsync(v, 0, 64, st));
  launch_validate(g->off, n, nnz, v, st, d);
  CK(cudaMemcpyAsync(v + 8, g->off, 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(v + 9, g->off + n, 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h, v, 10 * 8, cudaMemcpyDeviceToHost, st));
  sync_checked(st);
  if ((int64_t)h[8] != 0 || (int64_t)h[9] != nnz)
    fail(LCC_ERR_INVALID, "offsets[0] must be 0 and offsets[n] must equal nnz");
  if (h[0] & 1) fail(LCC_ERR_INVALID, "offsets are not monotone");
  launch_validate_rows(g->off, g->nbr, (const int32_t *)g->w, n, v, st, d);
  CK(cudaMemcpyAsync(h, v, 8 * 8, cudaMemcpyDeviceToHost, st));
  sync_checked(st);
  note_launches(2);
  if (h[0] & 2) fail(LCC_ERR_INVALID, "neighbour id out of range [0, n)");
  if (h[0] & 4) fail(LCC_ERR_SELF_LOOP, "self loop in the input");
  if (h[1] != h[2] || h[3] != h[4])
    fail(LCC_ERR_NOT_SYMMETRIC, "the graph is not symmetric (w_uv != w_vu or a missing direction)");
  const unsigned __int128 wabs = ((unsigned __int128)h[6] << 64) | h[5];
  if (wabs >= ((unsigned __int128)1 << 62)) fail(LCC_ERR_OVERFLOW, "sum of |w| must stay below 2^62");
  g->wabs = (int64_t)wabs;
  return g.release();
}


extern "C" {

const char *lcc_status_str(lcc_status s) {
  switch (s) {
    case LCC_OK: return "ok";
    case LCC_ERR_INVALID: return "invalid argument";
    case LCC_ERR_NOT_SYMMETRIC: return "graph not symmetric";
    case LCC_ERR_SELF_LOOP: return "self loop";
    case LCC_ERR_OOM: return "out of memory";
    case LCC_ERR_OVERFLOW: return "exact-integer range exceeded";
    case LCC_ERR_TIMEOUT: return "timeout";
    case LCC_ERR_CUDA: return "CUDA error";
    case LCC_ERR_BUSY: return "busy";
    case LCC_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char *lcc_last_error(void) { return t_err.c_str(); }

lcc_status lcc_load_csr(const int64_t *offsets, const int32_t *nbrs, const int32_t *weights,
                        int64_t n, int64_t nnz, const int64_t *node_w, int32_t memspace,
                        void *stream, lcc_graph **out) {
  API_BEGIN
  if (!out) fail(LCC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  *out = load_graph(offsets, nbrs, weights, n, nnz, node_w, memspace, (cudaStream_t)stream);
  API_END
}

lcc_status lcc_graph_info(const lcc_graph *g, int64_t *n, int64_t *nnz) {
  API_BEGIN
  if (!g) fail(LCC_ERR_INVALID, "graph is NULL");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  API_END
}

void lcc_free_graph(lcc_graph *g) {
  if (!g) return;
  try {
    cudaSetDevice(g->dev);
    cudaStream_t st = g->st;
    g->store.reset();
    cudaStreamSynchronize(st);
  } catch (...) {
  }
  delete g;
}

static void fill_stats(const Job &J, const Engine &E, lcc_stats *s, double ms_total,
                       long long launches, int64_t nclusters) {
  memset(s, 0, sizeof(*s));
  s->levels = J.levels;
  s->rounds_total = J.rounds_total;
  s->edges_scanned = E.stats.edges;
  s->vertices_scanned = E.stats.verts;
  s->candidates = E.stats.cands;
  s->num_clusters = nclusters;
  s->obj_num_hi = (int64_t)(J.num >> 64);
  s->obj_num_lo = (uint64_t)J.num;
  s->obj_den = J.den;
  s->objective = (double)J.num / (double)J.den;
  s->ms_bestmove = E.stats.ms_bm;
  s->ms_round_other = E.stats.ms_round_other;
  s->ms_contract = E.stats.ms_contract;
  s->ms_other = E.stats.ms_other;
  s->ms_total = ms_total;
  s->bytes_bestmove = E.stats.edges * 8 + E.stats.wbytes + E.stats.verts * 32 + E.stats.cands * 8;
  s->pairs_sorted = E.stats.pairs;
  s->kernel_launches = launches;
  s->bytes_contract_min = E.stats.contract_min_bytes;
  s->calls = J.calls;
  s->calls_capped = J.calls_capped;
  s->ms_gather = E.stats.ms_gather;
  for (int i = 0; i < NB && i < 16; ++i) {
    s->ms_bucket[i] = E.stats.ms_bucket[i];
    s->bucket_entries[i] = E.stats.bucket_entries[i];
    s->bucket_vertices[i] = E.stats.bucket_vertices[i];
  }
}

static void cluster_one(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                        const lcc_schedule *sched, int32_t *labels_out, int32_t labels_memspace,
                        double *objective_out, lcc_stats *stats_out,
                        std::vector<lcc_round> *trace);

lcc_status lcc_cluster(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                       const lcc_schedule *sched, int32_t *labels_out, int32_t labels_memspace,
                       double *objective_out, lcc_stats *stats_out) {
  API_BEGIN
  cluster_one(g, lambda_p, lambda_q, mode, sched, labels_out, labels_memspace, objective_out,
              stats_out, nullptr);
  API_END
}

lcc_status lcc_cluster_trace(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q,
                             int32_t mode, const lcc_schedule *sched, int32_t *labels_out,
                             int32_t labels_memspace, double *objective_out,
                             lcc_stats *stats_out, lcc_round *trace, int64_t trace_cap,
                             int64_t *trace_len) {
  API_BEGIN
  if (trace_cap < 0 || (trace_cap > 0 && !trace)) fail(LCC_ERR_INVALID, "bad trace buffer");
  std::vector<lcc_round> rec;
  cluster_one(g, lambda_p, lambda_q, mode, sched, labels_out, labels_memspace, objective_out,
              stats_out, &rec);
  const int64_t m = std::min<int64_t>(trace_cap, (int64_t)rec.size());
  if (m > 0) memcpy(trace, rec.data(), m * sizeof(lcc_round));
  if (trace_len) *trace_len = (int64_t)rec.size();
  API_END
}

static void cluster_one(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                        const lcc_schedule *sched, int32_t *labels_out, int32_t labels_memspace,
                        double *objective_out, lcc_stats *stats_out,
                        std::vector<lcc_round> *trace) {
  check_graph(g);
  check_lambda(lambda_p, lambda_q, mode);
  const lcc_schedule sc = check_schedule(sched);
  if (!labels_out && g->n > 0) fail(LCC_ERR_INVALID, "labels_out is NULL");
  if (labels_memspace != LCC_MEM_HOST && labels_memspace != LCC_MEM_DEVICE)
    fail(LCC_ERR_INVALID, "unknown memory space");
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(g->dev, g->st, lk);
  E->stats = EngineStats();
  E->timing = (sc.flags & LCC_SCHED_TIMING) != 0;
  const long long l0 = g_launches.load();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (E->timing) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, g->st));
  }
  Job J;
  J.g = g;
  J.p = lambda_p;
  J.q = lambda_q;
  J.mode = mode;
  J.sc = sc;
  J.labels_out = labels_out;
  J.labels_space = labels_memspace;
  J.trace = trace;
  try {
    E->add_job(&J);
    while (!E->idle()) E->tick();
  } catch (...) {
    E->drop_job(&J);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    throw;
  }
  float ms = 0;
  if (E->timing) {
    CK(cudaEventRecord(e1, g->st));
    CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (objective_out) *objective_out = (double)J.num / (double)J.den;
  if (stats_out) fill_stats(J, *E, stats_out, ms, g_launches.load() - l0, J.nclusters);
  J.lv.clear();
  J.base.reset();
}

lcc_status lcc_desired(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                       const int32_t *labels, const uint8_t *frontier, int32_t *desired_out) {
  API_BEGIN
  check_graph(g);
  check_lambda(lambda_p, lambda_q, mode);
  check_labels(labels, g->n);
  if (!desired_out && g->n > 0) fail(LCC_ERR_INVALID, "desired_out is NULL");
  std::vector<uint8_t> all;
  if (!frontier) {
    all.assign((size_t)g->n, 1);
    frontier = all.data();
  }
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(g->dev, g->st, lk);
  E->stats = EngineStats();
  E->timing = false;
  Job J;
  J.g = g;
  J.p = lambda_p;
  J.q = lambda_q;
  J.mode = mode;
  J.sc = default_schedule();
  J.eval_only = true;
  J.kind = BM_ONLY;
  try {
    E->add_job(&J, labels, frontier);
    while (!E->idle()) E->tick();
    CK(cudaMemcpyAsync(desired_out, J.lv[0].D, g->n * 4, cudaMemcpyDeviceToHost, g->st));
    sync_checked(g->st);
  } catch (...) {
    E->drop_job(&J);
    throw;
  }
  J.lv.clear();
  J.base.reset();
  API_END
}

lcc_status lcc_best_moves(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                          int32_t num_iter, int32_t vset, int32_t *labels_inout,
                          int32_t *rounds_out, int32_t *moved_out) {
  API_BEGIN
  check_graph(g);
  check_lambda(lambda_p, lambda_q, mode);
  check_labels(labels_inout, g->n);
  lcc_schedule sc = default_schedule();
  sc.num_iter = num_iter;
  sc.vset = vset;
  sc = check_schedule(&sc);
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(g->dev, g->st, lk);
  E->stats = EngineStats();
  E->timing = false;
  Job J;
  J.g = g;
  J.p = lambda_p;
  J.q = lambda_q;
  J.mode = mode;
  J.sc = sc;
  J.kind = BM_ONLY;
  try {
    E->add_job(&J, labels_inout, nullptr);
    while (!E->idle()) E->tick();
    CK(cudaMemcpyAsync(labels_inout, J.lv[0].L, g->n * 4, cudaMemcpyDeviceToHost, g->st));
    sync_checked(g->st);
  } catch (...) {
    E->drop_job(&J);
    throw;
  }
  if (rounds_out) *rounds_out = J.rounds_total;
  if (moved_out) *moved_out = J.moved_any ? 1 : 0;
  J.lv.clear();
  J.base.reset();
  API_END
}

// ------------------------------------------------------------ tuning ----

static void check_tuning(const lcc_tuning *t) {
  if (!t) fail(LCC_ERR_INVALID, "tuning is NULL");
  const int w = t->warp_max;
  if (w != 32 && w != 64 && w != 128 && w != 256)
    fail(LCC_ERR_INVALID, "warp_max must be 32, 64, 128 or 256");
  if (t->fuse_small != 0 && t->fuse_small != 1) fail(LCC_ERR_INVALID, "fuse_small must be 0 or 1");
  if (t->prefetch != 0 && t->prefetch != 1) fail(LCC_ERR_INVALID, "prefetch must be 0 or 1");
  if (t->pregather != 0 && t->pregather != 1) fail(LCC_ERR_INVALID, "pregather must be 0 or 1");
  const int pm = t->part_min;
  if (pm != 0 && pm != 1024 && pm != 4096 && pm != 8192 && pm != 16384)
    fail(LCC_ERR_INVALID, "part_min must be 0, 1024, 4096, 8192 or 16384");
  for (int i = 0; i < 3; ++i)
    if (t->reserved[i]) fail(LCC_ERR_INVALID, "reserved tuning fields must be zero");
}

static void check_device(int32_t device) {
  int nd = 0;
  CK(cudaGetDeviceCount(&nd));
  if (device < 0 || device >= nd) fail(LCC_ERR_INVALID, "no such CUDA device");
}

lcc_status lcc_get_tuning(int32_t device, lcc_tuning *out) {
  API_BEGIN
  check_device(device);
  if (!out) fail(LCC_ERR_INVALID, "out is NULL");
  *out = tuning_for(device);
  API_END
}

lcc_status lcc_set_tuning(int32_t device, const lcc_tuning *t) {
  API_BEGIN
  check_device(device);
  check_tuning(t);
  set_tuning(device, *t);
  API_END
}

// Key of a device in the tuning file: its name and SM count.
static std::string tuning_key(int dev) {
  cudaDeviceProp pr;
  CK(cudaGetDeviceProperties(&pr, dev));
  std::string name(pr.name);
  for (char &c : name)
    if (c == '|' || c == '\n') c = ' ';
  return name + "|" + std::to_string(pr.multiProcessorCount);
}

// Best-move device time of `rounds` rounds of g from singletons.
static double time_rounds(const lcc_graph *g, int64_t p, int64_t q, int32_t mode, int rounds) {
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(g->dev, g->st, lk);
  E->stats = EngineStats();
  E->timing = true;
  Job J;
  J.g = g;
  J.p = p;
  J.q = q;
  J.mode = mode;
  J.sc = default_schedule();
  J.sc.num_iter = rounds;
  J.kind = BM_ONLY;
  try {
    E->add_job(&J, nullptr, nullptr);
    while (!E->idle()) E->tick();
    sync_checked(g->st);
  } catch (...) {
    E->drop_job(&J);
    E->timing = false;
    throw;
  }
  E->timing = false;
  const double ms = E->stats.ms_bm;
  J.lv.clear();
  J.base.reset();
  return ms;
}

lcc_status lcc_autotune(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                        const char *cache_path, lcc_tuning *out) {
  API_BEGIN
  check_graph(g);
  check_lambda(lambda_p, lambda_q, mode);
  const std::string key = tuning_key(g->dev);
  lcc_tuning t;
  memset(&t, 0, sizeof(t));
  if (cache_path) {
    if (FILE *f = fopen(cache_path, "r")) {
      char line[512];
      bool found = false;
      while (!found && fgets(line, sizeof(line), f)) {
        // "<device name>|<SMs> <warp_max> [<fuse_small> <prefetch> <pregather> <part_min>]"
        std::string l(line);
        if (l.size() <= key.size() || l.compare(0, key.size(), key) != 0 || l[key.size()] != ' ')
          continue;
        int wm = 0, fs = 1, pf = 0, pg = 1, pbg = 8192;
        const int nread =
            sscanf(l.c_str() + key.size() + 1, "%d %d %d %d %d", &wm, &fs, &pf, &pg, &pbg);
        if (nread < 1) fail(LCC_ERR_INVALID, "malformed tuning line for this device");
        t.warp_max = wm;
        t.fuse_small = nread >= 2 ? fs : 1;
        t.prefetch = nread >= 3 ? pf : 0;
        t.pregather = nread >= 4 ? pg : 1;
        t.part_min = nread >= 5 ? pbg : 8192;
        found = true;
      }
      fclose(f);
      if (found) {
        check_tuning(&t);
        set_tuning(g->dev, t);
        if (out) *out = t;
        return LCC_OK;
      }
    }
  }
  const lcc_tuning before = tuning_for(g->dev);
  double best_ms = 0;
  lcc_tuning best = before;
  bool first = true;
  auto trial = [&](const lcc_tuning &c) {
    set_tuning(g->dev, c);
    const double ms = time_rounds(g, lambda_p, lambda_q, mode, 3);
    if (first || ms < best_ms) {
      best_ms = ms;
      best = c;
      first = false;
    }
  };
  try {
    time_rounds(g, lambda_p, lambda_q, mode, 1);  // first-use costs outside the comparison
    // one field at a time, each from the best so far: warp_max, then
    // fuse_small, prefetch, pregather and part_min
    memset(&t, 0, sizeof(t));
    t.fuse_small = 1;
    t.pregather = 1;
    t.part_min = 8192;
    for (int c : {32, 64, 128, 256}) {
      t.warp_max = c;
      trial(t);
    }
    t = best;
    t.fuse_small = 1 - t.fuse_small;
    trial(t);
    t = best;
    t.prefetch = 1 - t.prefetch;
    trial(t);
    t = best;
    t.pregather = 1 - t.pregather;
    trial(t);
    {
      const lcc_tuning base = best;
      for (int c : {0, 1024, 4096, 16384}) {
        t = base;
        t.part_min = c;
        trial(t);
      }
    }
  } catch (...) {
    set_tuning(g->dev, before);
    throw;
  }
  t = best;
  set_tuning(g->dev, t);
  if (cache_path) {
    FILE *f = fopen(cache_path, "a");
    if (!f) fail(LCC_ERR_INVALID, std::string("cannot write the tuning file ") + cache_path);
    fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), t.warp_max, t.fuse_small, t.prefetch,
            t.pregather, t.part_min);
    fclose(f);
  }
  if (out) *out = t;
  API_END
}

lcc_status lcc_compress(const lcc_graph *g, int32_t mode, const int32_t *labels,
                        int32_t *map_out, lcc_graph **coarse_out) {
  API_BEGIN
  check_graph(g);
  check_lambda(1, 1, mode);
  check_labels(labels, g->n);
  if (!coarse_out) fail(LCC_ERR_INVALID, "coarse_out is NULL");
  *coarse_out = nullptr;
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(g->dev, g->st, lk);
  E->stats = EngineStats();
  E->timing = false;
  Job J;
  J.g = g;
  J.p = 1;
  J.q = 1;
  J.mode = mode;
  J.sc = default_schedule();
  J.keep_coarse = true;
  try {
    E->add_job(&J, labels, nullptr, false);
    E->compress_to_graph(&J, map_out, coarse_out);
  } catch (...) {
    E->drop_job(&J);
    throw;
  }
  J.lv.clear();
  J.base.reset();
  API_END
}

lcc_status lcc_graph_export(const lcc_graph *g, int64_t *off, int32_t *nbr, int64_t *w,
                            int64_t *k) {
  API_BEGIN
  check_graph(g);
  cudaStream_t st = g->st;
  if (off) CK(cudaMemcpyAsync(off, g->off, (g->n + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (nbr && g->nnz) CK(cudaMemcpyAsync(nbr, g->nbr, g->nnz * 4, cudaMemcpyDeviceToHost, st));
  std::vector<int32_t> w32;
  if (w && g->nnz) {
    if (g->wtype == W_I64) {
      CK(cudaMemcpyAsync(w, g->w, g->nnz * 8, cudaMemcpyDeviceToHost, st));
    } else if (g->wtype == W_I32) {
      w32.resize((size_t)g->nnz);
      CK(cudaMemcpyAsync(w32.data(), g->w, g->nnz * 4, cudaMemcpyDeviceToHost, st));
    }
  }
  if (k && g->kc && g->n) CK(cudaMemcpyAsync(k, g->kc, g->n * 8, cudaMemcpyDeviceToHost, st));
  sync_checked(st);
  if (w && g->nnz) {
    if (g->wtype == W_I32)
      for (int64_t e = 0; e < g->nnz; ++e) w[e] = w32[e];
    else if (g->wtype == W_NONE)
      for (int64_t e = 0; e < g->nnz; ++e) w[e] = 1;
  }
  if (k && !g->kc)
    for (int64_t v = 0; v < g->n; ++v) k[v] = 1;
  API_END
}

lcc_status lcc_objective(const lcc_graph *g, int64_t lambda_p, int64_t lambda_q, int32_t mode,
                         const int32_t *labels, int64_t *num_hi, uint64_t *num_lo, int64_t *den) {
  API_BEGIN
  check_graph(g);
  check_lambda(lambda_p, lambda_q, mode);
  check_labels(labels, g->n);
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(g->dev, g->st, lk);
  Job J;
  J.g = g;
  J.p = lambda_p;
  J.q = lambda_q;
  J.mode = mode;
  J.sc = default_schedule();
  try {
    E->add_job(&J, labels, nullptr, false);
    E->objective_of(&J);
    J.lv.clear();
    J.base.reset();
  } catch (...) {
    E->drop_job(&J);
    throw;
  }
  if (num_hi) *num_hi = (int64_t)(J.num >> 64);
  if (num_lo) *num_lo = (uint64_t)J.num;
  if (den) *den = J.den;
  API_END
}

lcc_status lcc_cluster_batch(const lcc_graph *const *graphs, int32_t count,
                             const int64_t *lambda_p, const int64_t *lambda_q,
                             const int32_t *mode, const lcc_schedule *sched,
                             int32_t *const *labels_out, double *objectives_out) {
  API_BEGIN
  if (count < 0 || (count > 0 && (!graphs || !lambda_p || !lambda_q || !mode || !labels_out)))
    fail(LCC_ERR_INVALID, "bad batch arguments");
  if (count == 0) return LCC_OK;
  const lcc_schedule sc = check_schedule(sched);
  for (int i = 0; i < count; ++i) {
    check_graph(graphs[i]);
    check_lambda(lambda_p[i], lambda_q[i], mode[i]);
    if (graphs[i]->dev != graphs[0]->dev) fail(LCC_ERR_INVALID, "graphs on different devices");
  }
  CK(cudaSetDevice(graphs[0]->dev));
  std::unique_lock<std::mutex> lk;
  Engine *E = engine_for(graphs[0]->dev, graphs[0]->st, lk);
  E->stats = EngineStats();
  E->timing = false;
  std::vector<Job> jobs((size_t)count);
  try {
    for (int i = 0; i < count; ++i) {
      Job &J = jobs[i];
      J.g = graphs[i];
      J.p = lambda_p[i];
      J.q = lambda_q[i];
      J.mode = mode[i];
      J.sc = sc;
      J.labels_out = labels_out[i];
      J.labels_space = LCC_MEM_HOST;
      E->add_job(&J);
    }
    while (!E->idle()) E->tick();
  } catch (...) {
    for (auto &J : jobs) E->drop_job(&J);
    throw;
  }
  for (int i = 0; i < count; ++i) {
    if (objectives_out) objectives_out[i] = (double)jobs[i].num / (double)jobs[i].den;
    jobs[i].lv.clear();
    jobs[i].base.reset();
  }
  API_END
}

}  // extern "C"

// ------------------------------------------------------------- serving ----

namespace {
enum SState { S_QUEUED, S_RUNNING, S_DONE };

struct SJob {
  uint64_t ticket = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> nbr, w;
  bool weighted = false;
  int64_t n = 0, nnz = 0, p = 1, q = 1;
  int32_t mode = 0;
  int32_t inject_fault_tick = 0;
  int64_t est = 0;
  SState state = S_QUEUED;
  bool cancel = false;
  lcc_status status = LCC_OK;
  std::string err;
  std::vector<int32_t> labels;
  double obj = 0;
  std::chrono::steady_clock::time_point t_submit, t_done;
  Job job;
  lcc_graph *g = nullptr;
};
}  // namespace

struct lcc_server {
  lcc_server_cfg cfg;
  int dev = 0;
  cudaStream_t st = nullptr;      // the engine's stream
  cudaStream_t st_adm = nullptr;  // copies and validation of arriving graphs
  std::unique_ptr<Engine> eng;
  std::thread worker, admitter;
  std::mutex mu;
  std::condition_variable cv, cv_adm, cv_idle;
  bool stop = false;
  std::deque<SJob *> queue;   // submitted, not yet admitted
  std::deque<SJob *> loaded;  // admitted and loaded, waiting for the next tick
  std::unordered_map<uint64_t, SJob *> all;
  std::vector<SJob *> running;  // admitted (loading, loaded or in the engine)
  uint64_t next = 1;
  int64_t resident = 0;
  int64_t c_done = 0, c_ticks = 0, c_peak_bytes = 0, c_peak_jobs = 0, c_rejected = 0;
  int64_t pending = 0;  // submitted and not yet finished
};

static int64_t job_estimate(int64_t n, int64_t nnz, bool weighted) {
  // CSR + level-0 state + the first level's contraction workspace, and the
  // gather layout (positions and remapped neighbours) of large levels
  const int64_t csr = (n + 1) * 8 + nnz * (weighted ? 8 : 4);
  const int64_t layout = n * 8 > layout_min_bytes() ? 2 * (n * 4 + nnz * 4) : 0;
  return 2 * csr + n * 64 + nnz * 56 + layout + (1 << 20);
}

// Releases a job's graph without waiting: its memory returns to the pool in
// the order of the stream it was allocated on, and nothing of the engine
// uses it any more (the tick that finished the job has completed).
static void release_graph(SJob *j) {
  if (j->g) {
    j->g->store.reset();
    delete j->g;
    j->g = nullptr;
  }
}

static void finish_job(lcc_server *s, SJob *j, lcc_status st, const std::string &err) {
  release_graph(j);
  std::lock_guard<std::mutex> lk(s->mu);
  j->status = st;
  j->err = err;
  j->state = S_DONE;
  j->t_done = std::chrono::steady_clock::now();
  s->resident -= j->est;
  s->running.erase(std::remove(s->running.begin(), s->running.end(), j), s->running.end());
  s->c_done += 1;
  s->pending -= 1;
  s->cv_idle.notify_all();
  s->cv_adm.notify_all();  // a slot and budget came free
}

// Admission: takes queued jobs while a slot and the HBM budget allow,
// copies and validates their graphs on its own stream (overlapping the
// engine's ticks), and hands them to the worker.
static void admit_loop(lcc_server *s) {
  cudaSetDevice(s->dev);
  while (true) {
    std::vector<SJob *> take;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_adm.wait_for(lk, std::chrono::milliseconds(20), [&] {
        return s->stop ||
               (!s->queue.empty() && (int64_t)s->running.size() < s->cfg.max_slots &&
                s->resident + s->queue.front()->est <= s->cfg.hbm_budget_bytes);
      });
      if (s->stop) break;
      while (!s->queue.empty() && (int64_t)s->running.size() < s->cfg.max_slots &&
             s->resident + s->queue.front()->est <= s->cfg.hbm_budget_bytes) {
        SJob *j = s->queue.front();
        s->queue.pop_front();
        if (j->cancel) {
          j->state = S_DONE;
          j->status = LCC_ERR_CANCELLED;
          j->t_done = std::chrono::steady_clock::now();
          s->pending -= 1;
          s->cv_idle.notify_all();
          continue;
        }
        j->state = S_RUNNING;
        s->running.push_back(j);
        s->resident += j->est;
        take.push_back(j);
      }
      s->c_peak_bytes = std::max(s->c_peak_bytes, s->resident);
      s->c_peak_jobs = std::max(s->c_peak_jobs, (int64_t)s->running.size());
    }
    for (SJob *j : take) {
      try {
        j->g = load_graph(j->off.data(), j->nbr.data(), j->weighted ? j->w.data() : nullptr, j->n,
                          j->nnz, nullptr, LCC_MEM_HOST, s->st_adm);
        std::lock_guard<std::mutex> lk(s->mu);
        s->loaded.push_back(j);
        s->cv.notify_all();
      } catch (const Error &e) {
        finish_job(s, j, e.st, e.what());
      } catch (const std::exception &e) {
        finish_job(s, j, LCC_ERR_CUDA, e.what());
      }
    }
  }
}

static void server_loop(lcc_server *s) {
  cudaSetDevice(s->dev);
  Engine &E = *s->eng;
  while (true) {
    std::vector<SJob *> admit;
    std::vector<SJob *> cancelled;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      while (!s->loaded.empty()) {
        SJob *j = s->loaded.front();
        s->loaded.pop_front();
        if (j->cancel)
          cancelled.push_back(j);
        else
          admit.push_back(j);
      }
      for (SJob *j : s->running)
        if (j->cancel && j->job.g && std::find(cancelled.begin(), cancelled.end(), j) == cancelled.end())
          cancelled.push_back(j);
      if (admit.empty() && cancelled.empty() && E.idle()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
    }
    for (SJob *j : cancelled) {
      E.drop_job(&j->job);
      finish_job(s, j, LCC_ERR_CANCELLED, "cancelled");
    }
    if (!admit.empty()) {
      std::vector<Job *> jobs;
      for (SJob *j : admit) {
        j->labels.resize((size_t)j->n);
        Job &J = j->job;
        J.g = j->g;
        J.p = j->p;
        J.q = j->q;
        J.mode = j->mode;
        J.sc = s->cfg.sched;
        J.labels_out = j->labels.data();
        J.labels_space = LCC_MEM_HOST;
        J.inject_fault_tick = j->inject_fault_tick;
        jobs.push_back(&J);
      }
      try {
        // one statistics pass for every newly admitted job; a job whose own
        // input fails a check comes back alone
        for (auto &f : E.add_jobs(jobs))
          for (SJob *j : admit)
            if (&j->job == f.first) finish_job(s, j, f.second.st, f.second.what());
      } catch (const std::exception &e) {
        const Error *le = dynamic_cast<const Error *>(&e);
        for (SJob *j : admit) {
          E.drop_job(&j->job);
          finish_job(s, j, le ? le->st : LCC_ERR_CUDA, e.what());
        }
      }
    }
    if (!E.idle()) {
      try {
        std::vector<Job *> done = E.tick();
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->c_ticks += 1;
        }
        for (Job *J : done) {
          SJob *j = nullptr;
          {
            std::lock_guard<std::mutex> lk(s->mu);
            for (SJob *r : s->running)
              if (&r->job == J) j = r;
          }
          if (!j) continue;
          j->obj = (double)J->num / (double)J->den;
          J->lv.clear();
          J->base.reset();
          finish_job(s, j, LCC_OK, "");
        }
      } catch (const std::exception &e) {
        std::vector<SJob *> run;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          run = s->running;
        }
        const Error *le = dynamic_cast<const Error *>(&e);
        SJob *culprit = nullptr;
        if (le && le->job)
          for (SJob *j : run)
            if (&j->job == le->job) culprit = j;
        if (culprit) {
          // raised before any job's state changed in this tick: only that job
          // fails, the others run on in the next tick
          E.drop_job(&culprit->job);
          finish_job(s, culprit, le->st, e.what());
        } else {
          // otherwise the tick's state is unknown: every job in it fails
          for (SJob *j : run) {
            if (!j->job.g) continue;  // still being loaded: not in the tick
            E.drop_job(&j->job);
            finish_job(s, j, le ? le->st : LCC_ERR_CUDA, e.what());
          }
        }
      }
    }
  }
}

extern "C" {

lcc_status lcc_server_create(const lcc_server_cfg *cfg, lcc_server **out) {
  API_BEGIN
  if (!cfg || !out) fail(LCC_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->hbm_budget_bytes <= 0)
    fail(LCC_ERR_INVALID, "max_slots and hbm_budget_bytes must be positive");
  check_schedule(&cfg->sched);
  std::unique_ptr<lcc_server> s(new lcc_server());
  s->cfg = *cfg;
  CK(cudaGetDevice(&s->dev));
  CK(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&s->st_adm, cudaStreamNonBlocking));
  s->eng.reset(new Engine(s->dev, s->st));
  lcc_server *raw = s.get();
  s->worker = std::thread(server_loop, raw);
  s->admitter = std::thread(admit_loop, raw);
  *out = s.release();
  API_END
}

lcc_status lcc_submit(lcc_server *s, const lcc_job *job, uint64_t *ticket) {
  API_BEGIN
  if (!s || !job || !ticket) fail(LCC_ERR_INVALID, "NULL argument");
  if (job->n < 0 || job->nnz < 0 || !job->offsets || (job->nnz > 0 && !job->nbrs))
    fail(LCC_ERR_INVALID, "malformed job");
  check_lambda(job->lambda_p, job->lambda_q, job->mode);
  if (job->mode == LCC_NODEW_CUSTOM) fail(LCC_ERR_INVALID, "custom node weights are not served");
  std::unique_ptr<SJob> j(new SJob());
  j->n = job->n;
  j->nnz = job->nnz;
  j->p = job->lambda_p;
  j->q = job->lambda_q;
  j->mode = job->mode;
  if (job->inject_fault_tick < 0) fail(LCC_ERR_INVALID, "inject_fault_tick must be >= 0");
  j->inject_fault_tick = job->inject_fault_tick;
  j->weighted = job->weights != nullptr;
  j->est = job_estimate(job->n, job->nnz, j->weighted);
  if (j->est > s->cfg.hbm_budget_bytes) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->c_rejected += 1;
    fail(LCC_ERR_OOM, "job larger than the HBM budget");
  }
  j->off.assign(job->offsets, job->offsets + job->n + 1);
  j->nbr.assign(job->nbrs, job->nbrs + job->nnz);
  if (j->weighted) j->w.assign(job->weights, job->weights + job->nnz);
  j->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    j->ticket = s->next++;
    *ticket = j->ticket;
    s->all[j->ticket] = j.get();
    s->queue.push_back(j.release());
    s->pending += 1;
  }
  s->cv_adm.notify_all();
  API_END
}

lcc_status lcc_poll(lcc_server *s, uint64_t ticket, int32_t *labels_out, double *obj_out,
                    double *latency_ms_out) {
  API_BEGIN
  if (!s) fail(LCC_ERR_INVALID, "NULL server");
  std::unique_ptr<SJob> j;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) fail(LCC_ERR_INVALID, "unknown ticket");
    if (it->second->state != S_DONE) return LCC_ERR_BUSY;
    j.reset(it->second);
    s->all.erase(it);
  }
  if (latency_ms_out)
    *latency_ms_out =
        std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
  if (j->status != LCC_OK) {
    t_err = j->err;
    return j->status;
  }
  if (labels_out && j->n) memcpy(labels_out, j->labels.data(), j->n * 4);
  if (obj_out) *obj_out = j->obj;
  API_END
}

lcc_status lcc_cancel(lcc_server *s, uint64_t ticket) {
  API_BEGIN
  if (!s) fail(LCC_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) fail(LCC_ERR_INVALID, "unknown ticket");
  it->second->cancel = true;
  s->cv.notify_all();
  s->cv_adm.notify_all();
  API_END
}

lcc_status lcc_server_wait_idle(lcc_server *s, int64_t timeout_ms) {
  API_BEGIN
  if (!s) fail(LCC_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_idle.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [&] { return s->pending == 0; });
  if (!ok) fail(LCC_ERR_TIMEOUT, "jobs still running");
  API_END
}

lcc_status lcc_server_counters(lcc_server *s, int64_t *out5) {
  API_BEGIN
  if (!s || !out5) fail(LCC_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out5[0] = s->c_done;
  out5[1] = s->c_ticks;
  out5[2] = s->c_peak_bytes;
  out5[3] = s->c_peak_jobs;
  out5[4] = s->c_rejected;
  API_END
}

lcc_status lcc_server_destroy(lcc_server *s) {
  API_BEGIN
  if (!s) return LCC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->cv_adm.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->admitter.joinable()) s->admitter.join();
  cudaSetDevice(s->dev);
  for (SJob *j : s->running) {
    s->eng->drop_job(&j->job);
    release_graph(j);
  }
  for (auto &kv : s->all) delete kv.second;
  s->eng.reset();
  cudaStreamSynchronize(s->st_adm);
  cudaStreamDestroy(s->st);
  cudaStreamDestroy(s->st_adm);
  delete s;
  API_END
}

}  // extern "C"
