// Host side of liblcc: device memory, graphs, per-job level stacks and the
// tick engine that runs many jobs through Algorithm 1 together.
#pragma once

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "lcc.h"
#include "lcc_internal.cuh"

namespace lcc {

struct Error : std::runtime_error {
  lcc_status st;
  // The one job this error belongs to, when it is raised before any other
  // job's state changed in the current tick (the others can go on); null
  // when the whole tick must be failed.
  const void *job = nullptr;
  Error(lcc_status s, const std::string &m, const void *j = nullptr)
      : std::runtime_error(m), st(s), job(j) {}
};

void check_cuda(cudaError_t e, const char *what, int line);
#define CK(x) ::lcc::check_cuda((x), #x, __LINE__)
// Waits for the stream, then reports any launch that the runtime refused
// (a bad launch configuration does not surface through the stream).
inline void sync_checked(cudaStream_t st) {
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
}

extern std::atomic<long long> g_launches;
int64_t layout_min_bytes();
// Kernel tuning per device (degree routing), shared by every engine there.
lcc_tuning tuning_for(int dev);
void set_tuning(int dev, const lcc_tuning &t);
inline void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Stream-ordered device allocation from a per-device pool that keeps freed
// memory cached.
void *dalloc(size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);

// A set of device allocations released together (stream-ordered).
struct Store {
  cudaStream_t st;
  std::vector<void *> ptrs;
  explicit Store(cudaStream_t s) : st(s) {}
  ~Store() {
    for (void *p : ptrs) dfree(p, st);
  }
  template <class T> T *alloc(int64_t n) {
    void *p = dalloc((size_t)(n > 0 ? n : 1) * sizeof(T), st);
    ptrs.push_back(p);
    return (T *)p;
  }
};

// Grow-only scratch buffer.
struct Scratch {
  void *p = nullptr;
  size_t bytes = 0;
  template <class T> T *get(int64_t n, cudaStream_t st) {
    size_t need = (size_t)(n > 0 ? n : 1) * sizeof(T);
    if (need > bytes) {
      if (p) dfree(p, st);
      size_t nb = need + need / 4;
      p = dalloc(nb, st);
      bytes = nb;
    }
    return (T *)p;
  }
  void release(cudaStream_t st) {
    if (p) dfree(p, st);
    p = nullptr;
    bytes = 0;
  }
};

}  // namespace lcc

struct lcc_graph {
  int dev = 0;
  cudaStream_t st = nullptr;
  int64_t n = 0, nnz = 0;
  int64_t *off = nullptr;
  int32_t *nbr = nullptr;
  void *w = nullptr;
  int32_t wtype = lcc::W_NONE;
  int64_t *kc = nullptr;  // node weights (custom or coarse); may be null
  int64_t wabs = 0;       // sum of |w| over entries
  std::shared_ptr<lcc::Store> store;
};

namespace lcc {

struct Level {
  int64_t n = 0;
  const int64_t *off = nullptr;
  const int32_t *nbr = nullptr;
  const void *w = nullptr;
  int32_t wtype = W_NONE;
  const int64_t *k = nullptr;
  int32_t *L = nullptr;
  int64_t *K = nullptr;
  int32_t *D = nullptr;
  uint8_t *fr = nullptr;
  uint8_t *cl = nullptr;
  unsigned long long *lk = nullptr;  // packed (K[L[u]], L[u]); null if K can exceed 32 bits
  int32_t *pos = nullptr;            // gather layout (null: identity), see JobDev
  int32_t *gnbr = nullptr;
  int32_t warp_max = T_WARP;         // degree routing the level was bucketed with
  // the level's entries start at position 0 of nbr (the input level, or the
  // first job of a contraction batch; the other jobs of a batch index a
  // shared entry array from off[0] > 0)
  bool entries_from_zero = true;
  int32_t *map = nullptr;  // vertex -> coarse vertex of the next level
  std::shared_ptr<Store> store;
  std::shared_ptr<Store> map_store;
  LevelInfo info{};
  bool wide = false;
};

enum Phase { P_BM, P_CONTRACT, P_UP, P_FINAL, P_DONE };
enum BMKind { BM_COARSEN, BM_REFINE, BM_ONLY };

struct Job {
  uint64_t id = 0;
  const lcc_graph *g = nullptr;
  int64_t p = 1, q = 1;  // effective lambda = p / q for this run
  int32_t mode = LCC_NODEW_UNIT;
  lcc_schedule sc{};
  std::vector<Level> lv;
  int depth = 0;
  Phase phase = P_BM;
  BMKind kind = BM_COARSEN;
  int round = 0;
  bool pull = false;  // the next round tests V' in the best-move kernels (JF_PULL)
  bool moved_level = false;
  bool moved_any = false;
  bool eval_only = false;
  bool canonical = true;
  bool keep_coarse = false;  // Compress keeps the coarse level even if it does not shrink
  int64_t nclusters = 0;
  int64_t ktot = 0;
  // results
  lcc_status status = LCC_OK;
  std::string err;
  i128 num = 0;
  int64_t den = 1;
  int32_t rounds_total = 0;
  int32_t levels = 1;
  int64_t calls = 0, calls_capped = 0;  // Best-Moves calls; those ended by num_iter
  // final labels copied here (host or device pointer) when done
  int32_t *labels_out = nullptr;
  int32_t labels_space = LCC_MEM_HOST;
  // owned node-weight / state storage of level 0
  std::shared_ptr<Store> base;
  // ticks this job has been in (Engine::tick), and the fault-injection hook
  // of the serving API: > 0 makes tick number inject_fault_tick raise an
  // error for this job alone
  int64_t ticks = 0;
  int64_t inject_fault_tick = 0;
  // per-round record of a job that runs alone (lcc_cluster_trace)
  std::vector<lcc_round> *trace = nullptr;
};

struct EngineStats {
  int64_t edges = 0, verts = 0, cands = 0, wbytes = 0, pairs = 0;
  int64_t contract_min_bytes = 0;  // least bytes of the contractions (lcc_stats)
  int64_t rounds = 0;
  double ms_bm = 0, ms_round_other = 0, ms_contract = 0, ms_other = 0;
  double ms_gather = 0;  // the gathered-word passes (part of ms_bm)
  double ms_bucket[NB] = {0};
  int64_t bucket_entries[NB] = {0};
  int64_t bucket_vertices[NB] = {0};
};

class Engine {
 public:
  Engine(int dev, cudaStream_t st);
  ~Engine();
  // Prepares level 0 of a job (node weights, singletons, statistics) and
  // adds it to the active set.
  void add_job(Job *j, const int32_t *init_labels_host = nullptr,
               const uint8_t *frontier_host = nullptr, bool activate = true);
  // Level 0 of several jobs at once (singletons, every job activated), with
  // one statistics pass for all; a job whose own input fails a check is
  // returned with its error and not added, the others are.
  std::vector<std::pair<Job *, Error>> add_jobs(const std::vector<Job *> &js);
  // One step of every active job; returns the jobs that finished.
  std::vector<Job *> tick();
  bool idle() const { return active_.empty(); }
  void drop_job(Job *j);
  EngineStats stats;
  bool timing = false;
  cudaStream_t stream() const { return st_; }
  int device() const { return dev_; }
  Dev dinfo() const { return d_; }
  // Labels / objective helpers used by the single-call API.
  void objective_of(Job *j);
  void compress_to_graph(Job *j, int32_t *map_host, lcc_graph **out);
  size_t scratch_bytes() const;

 private:
  void round(std::vector<Job *> &js);
  void contract(std::vector<Job *> &js);
  void up(std::vector<Job *> &js);
  void finalize(std::vector<Job *> &js);
  void level_stats(std::vector<Job *> &js, std::vector<Level *> &lvs);
  void prepare_level0(Job *j, std::vector<LJob> &deg);
  void degree_weights(const std::vector<LJob> &deg);
  void check_level0(Job *j);
  // Gather layout for the levels (with packed words) that are large enough;
  // its arrays come from stores[i].
  void build_layout(std::vector<Level *> &lvs, std::vector<Store *> &stores);
  void init_levels(std::vector<Level *> &lvs);
  void end_bm(Job *j);
  float elapsed(cudaEvent_t a, cudaEvent_t b);

  int dev_;
  cudaStream_t st_;
  Dev d_;
  std::vector<Job *> active_;
  // scratch
  Scratch s_jobs_, s_vstart_, s_items_, s_cnt_, s_ctr_, s_jmoves_, s_moved_;
  Scratch s_hkeys_, s_hvals_, s_hmeta_, s_hpart_s_, s_hpart_c_, s_hstay_, s_hiso_;
  Scratch s_ljobs_, s_info_, s_obj_, s_layout_;
  Scratch s_coin_, s_jheld_, s_gw_, s_gwoff_;
  Scratch s_pmeta_, s_prow_, s_pflag_, s_pword_, s_pw_, s_pscore_, s_pcid_, s_pdesc_;
  // pinned host staging
  void *h_stage_ = nullptr;
  size_t h_stage_bytes_ = 0;
  void *h_stage2_ = nullptr;
  size_t h_stage2_bytes_ = 0;
  cudaEvent_t ev_[8];
  cudaEvent_t ev_gw_;  // end of the gathered-word pass of a round
  cudaEvent_t bev_[NB];
  void *stage(size_t bytes);
  void *stage2(size_t bytes);
};

// Shared engine for the single-graph calls on (device, stream).
Engine *engine_for(int dev, cudaStream_t st, std::unique_lock<std::mutex> &lock);

}  // namespace lcc
