// Tick engine: runs a set of jobs through Parallel-CC (Algorithm 1) on the
// synchronous schedule (Sec. 3.2.1).  Each job is a state machine over its
// level stack:
//
//   BM        one Best-Moves round per tick, all BM jobs in one launch per
//             kernel; ends after a round without moves or num_iter rounds;
//   CONTRACT  Compress of every job that finished coarsening with moves,
//             batched into one relabel/emit/sort/reduce pass;
//   UP        Flatten into the level below, then refinement (another
//             Best-Moves on that level, Sec. 3.2.3) or the next Flatten;
//   FINAL     canonical labels and the exact objective.
//
// Every job's arithmetic depends only on its own arrays, so its labels are
// the same whether it runs alone or with others.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "engine.h"

namespace lcc {

std::atomic<long long> g_launches{0};

// Slots of hub hash tables processed per pass (12 bytes each); the
// LCC_HUB_WINDOW_SLOTS environment variable overrides it (tests use a small
// window to exercise many passes).
static int64_t hub_window() {
  const char *e = getenv("LCC_HUB_WINDOW_SLOTS");
  if (e) {
    const long long v = atoll(e);
    if (v >= 1024) return (int64_t)v;
  }
  return (int64_t)1 << 27;
}

// Shared-table slots of one part of the partitioned long-row path (at most
// PART_TP); the LCC_PART_TABLE_SLOTS environment variable lowers it (tests
// use a small table so that parts overflow and their rows take the fallback).
static int32_t part_table_slots() {
  const char *e = getenv("LCC_PART_TABLE_SLOTS");
  if (e) {
    const long long v = atoll(e);
    if (v >= 32 && v <= PART_TP) return (int32_t)(v & ~31LL);
  }
  return PART_TP;
}

// Table slots of the longest coarse rows processed per pass of Compress; the
// LCC_ROW_WINDOW_SLOTS environment variable overrides it (tests use a small
// window to exercise many passes).
static int64_t row_window() {
  const char *e = getenv("LCC_ROW_WINDOW_SLOTS");
  if (e) {
    const long long v = atoll(e);
    if (v >= 1024) return (int64_t)v;
  }
  return (int64_t)1 << 27;
}

// Packed-word bytes above which a level gets a gather layout; the
// LCC_LAYOUT_MIN_BYTES environment variable overrides it (tests use 0 so that
// small graphs run through the layout too).
int64_t layout_min_bytes() {
  const char *e = getenv("LCC_LAYOUT_MIN_BYTES");
  if (e && *e) {
    const long long v = atoll(e);
    if (v >= 0) return (int64_t)v;
  }
  return LAYOUT_MIN_BYTES;
}

static std::mutex g_tune_mu;
static std::unordered_map<int, lcc_tuning> g_tune;

lcc_tuning tuning_for(int dev) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(dev);
  if (it != g_tune.end()) return it->second;
  lcc_tuning t;
  memset(&t, 0, sizeof(t));
  t.warp_max = T_WARP;
  t.fuse_small = 1;
  t.pregather = 1;
  t.part_min = 8192;
  return t;
}

void set_tuning(int dev, const lcc_tuning &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[dev] = t;
}

void check_cuda(cudaError_t e, const char *what, int line) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    throw Error(LCC_ERR_OOM, std::string("out of device memory in ") + what);
  }
  throw Error(LCC_ERR_CUDA, std::string(what) + " (line " + std::to_string(line) +
                                "): " + cudaGetErrorString(e));
}

// ------------------------------------------------------------- memory ----

static std::mutex g_pool_mu;
static std::unordered_map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t pool_for(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  CK(cudaMemPoolCreate(&pool, &props));
  uint64_t thr = UINT64_MAX;
  CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  g_pools[dev] = pool;
  return pool;
}

void *dalloc(size_t bytes, cudaStream_t st) {
  int dev;
  CK(cudaGetDevice(&dev));
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool_for(dev), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? LCC_ERR_OOM : LCC_ERR_CUDA,
                std::string("device allocation of ") + std::to_string(bytes) +
                    " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

void dfree(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// -------------------------------------------------------------- engine ----

Engine::Engine(int dev, cudaStream_t st) : dev_(dev), st_(st) {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  d_.sms = sms;
  d_.dev = dev;
  for (auto &e : ev_) CK(cudaEventCreate(&e));
  for (auto &e : bev_) CK(cudaEventCreate(&e));
  CK(cudaEventCreate(&ev_gw_));
}

Engine::~Engine() {
  for (auto &e : ev_) cudaEventDestroy(e);
  for (auto &e : bev_) cudaEventDestroy(e);
  cudaEventDestroy(ev_gw_);
  Scratch *all[] = {&s_jobs_,  &s_vstart_, &s_items_,  &s_cnt_,    &s_ctr_,    &s_jmoves_,
                    &s_moved_, &s_hkeys_,  &s_hvals_,  &s_hmeta_,  &s_hpart_s_, &s_hpart_c_,
                    &s_hstay_, &s_hiso_,   &s_ljobs_,  &s_info_,   &s_obj_,    &s_layout_,
                    &s_coin_,  &s_jheld_,  &s_gw_,     &s_gwoff_, &s_pmeta_, &s_prow_,
                    &s_pflag_, &s_pword_,  &s_pw_,     &s_pscore_, &s_pcid_, &s_pdesc_};
  for (Scratch *s : all) s->release(st_);
  cudaStreamSynchronize(st_);
  if (h_stage_) cudaFreeHost(h_stage_);
  if (h_stage2_) cudaFreeHost(h_stage2_);
}

size_t Engine::scratch_bytes() const {
  const Scratch *all[] = {&s_jobs_,  &s_vstart_, &s_items_,  &s_cnt_,    &s_ctr_,    &s_jmoves_,
                          &s_moved_, &s_hkeys_,  &s_hvals_,  &s_hmeta_,  &s_hpart_s_, &s_hpart_c_,
                          &s_hstay_, &s_hiso_,   &s_ljobs_,  &s_info_,   &s_obj_,
                          &s_layout_, &s_coin_,  &s_jheld_,  &s_gw_,     &s_gwoff_,
                          &s_pmeta_, &s_prow_,  &s_pflag_, &s_pword_,  &s_pw_,
                          &s_pscore_, &s_pcid_, &s_pdesc_};
  size_t t = 0;
  for (const Scratch *s : all) t += s->bytes;
  return t;
}

void *Engine::stage(size_t bytes) {
  // the previous upload from this buffer may still be in flight
  sync_checked(st_);
  if (bytes > h_stage_bytes_) {
    if (h_stage_) {
      sync_checked(st_);
      cudaFreeHost(h_stage_);
    }
    size_t nb = bytes + bytes / 2 + 4096;
    CK(cudaMallocHost(&h_stage_, nb));
    h_stage_bytes_ = nb;
  }
  return h_stage_;
}

void *Engine::stage2(size_t bytes) {
  if (bytes > h_stage2_bytes_) {
    if (h_stage2_) {
      sync_checked(st_);
      cudaFreeHost(h_stage2_);
    }
    size_t nb = bytes + bytes / 2 + 4096;
    CK(cudaMallocHost(&h_stage2_, nb));
    h_stage2_bytes_ = nb;
  }
  return h_stage2_;
}

float Engine::elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

static LJob ljob_of(const Level &L) {
  LJob x;
  memset(&x, 0, sizeof(x));
  x.off = L.off;
  x.nbr = L.nbr;
  x.w = L.w;
  x.k = L.k;
  x.L = L.L;
  x.K = L.K;
  x.D = L.D;
  x.pos = L.pos;
  x.gnbr = L.gnbr;
  x.n = L.n;
  x.wtype = L.wtype;
  x.warp_max = L.warp_max;
  return x;
}

// Uploads a table of T plus vstart (host vectors) through pinned staging.
template <class T>
static void upload_table(const std::vector<T> &tab, const std::vector<int64_t> &vs, T *d_tab,
                         int64_t *d_vs, void *stage, cudaStream_t st) {
  char *h = (char *)stage;
  size_t a = tab.size() * sizeof(T);
  memcpy(h, tab.data(), a);
  memcpy(h + a, vs.data(), vs.size() * sizeof(int64_t));
  CK(cudaMemcpyAsync(d_tab, h, a, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_vs, h + a, vs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
}

static bool needs_wide(const Level &L, int64_t p, int64_t q, int64_t ktot) {
  const i128 lim = (i128)1 << 62;
  const i128 a = (i128)q * (i128)L.info.rmax;
  const i128 b = (i128)p * (i128)L.info.kmax * (i128)ktot;
  return a >= lim || b >= lim;
}

void Engine::level_stats(std::vector<Job *> &js, std::vector<Level *> &lvs) {
  const int nj = (int)lvs.size();
  if (nj == 0) return;
  std::vector<LJob> tab(nj);
  std::vector<int64_t> vs(nj + 1);
  int64_t vt = 0;
  for (int i = 0; i < nj; ++i) {
    tab[i] = ljob_of(*lvs[i]);
    vs[i] = vt;
    vt += lvs[i]->n;
  }
  vs[nj] = vt;
  LJob *dt = s_ljobs_.get<LJob>(nj, st_);
  int64_t *dv = s_vstart_.get<int64_t>(nj + 1, st_);
  LevelInfo *di = s_info_.get<LevelInfo>(nj, st_);
  upload_table(tab, vs, dt, dv, stage(nj * (sizeof(LJob) + 8) + 8), st_);
  CK(cudaMemsetAsync(di, 0, nj * sizeof(LevelInfo), st_));
  launch_level_stats(dt, dv, nj, vt, di, st_, d_);
  note_launches(1);
  LevelInfo *h = (LevelInfo *)stage2(nj * sizeof(LevelInfo));
  CK(cudaMemcpyAsync(h, di, nj * sizeof(LevelInfo), cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  for (int i = 0; i < nj; ++i) {
    lvs[i]->info = h[i];
    lvs[i]->wide = needs_wide(*lvs[i], js[i]->p, js[i]->q, js[i]->ktot);
  }
}

void Engine::build_layout(std::vector<Level *> &lvs, std::vector<Store *> &stores) {
  std::vector<LJob> tab;
  std::vector<int64_t> vs(1, 0), es(1, 0);
  for (size_t i = 0; i < lvs.size(); ++i) {
    Level &L = *lvs[i];
    // the layout kernels index a level's entries from 0
    if (!L.lk || !L.entries_from_zero ||
        L.n * (int64_t)sizeof(unsigned long long) <= layout_min_bytes())
      continue;
    L.pos = stores[i]->alloc<int32_t>(L.n);
    L.gnbr = stores[i]->alloc<int32_t>(L.info.nnz);
    tab.push_back(ljob_of(L));
    vs.push_back(vs.back() + L.n);
    es.push_back(es.back() + L.info.nnz);
  }
  const int nj = (int)tab.size();
  if (nj == 0) return;
  std::vector<int64_t> ves(vs);
  ves.insert(ves.end(), es.begin(), es.end());
  LJob *dt = s_ljobs_.get<LJob>(nj, st_);
  int64_t *dv = s_vstart_.get<int64_t>(2 * (nj + 1), st_);
  int64_t *cnt = s_layout_.get<int64_t>(nj * LAYOUT_CLASSES, st_);
  upload_table(tab, ves, dt, dv, stage(nj * sizeof(LJob) + ves.size() * 8), st_);
  CK(cudaMemsetAsync(cnt, 0, nj * LAYOUT_CLASSES * sizeof(int64_t), st_));
  launch_layout(dt, dv, dv + (nj + 1), nj, vs.back(), es.back(), cnt, st_, d_);
  note_launches(4);
  sync_checked(st_);  // staging reuse
}

void Engine::init_levels(std::vector<Level *> &lvs) {
  const int nj = (int)lvs.size();
  if (nj == 0) return;
  std::vector<LJob> tab(nj);
  std::vector<int64_t> vs(nj + 1);
  int64_t vt = 0;
  for (int i = 0; i < nj; ++i) {
    tab[i] = ljob_of(*lvs[i]);
    vs[i] = vt;
    vt += lvs[i]->n;
  }
  vs[nj] = vt;
  LJob *dt = s_ljobs_.get<LJob>(nj, st_);
  int64_t *dv = s_vstart_.get<int64_t>(nj + 1, st_);
  upload_table(tab, vs, dt, dv, stage(nj * (sizeof(LJob) + 8) + 8), st_);
  launch_init_level(dt, dv, nj, vt, st_, d_);
  note_launches(1);
  // the staging buffer is reused by the next upload: wait for the copies
  sync_checked(st_);
}

// ------------------------------------------------------------ add job ----

// Level 0 of a job: its arrays and node weights.  Degree-mode weights are
// left to the caller (deg collects the job's table entry).
void Engine::prepare_level0(Job *j, std::vector<LJob> &deg) {
  const lcc_graph *g = j->g;
  j->base = std::make_shared<Store>(st_);
  Level L0;
  L0.n = g->n;
  L0.warp_max = tuning_for(dev_).warp_max;
  L0.off = g->off;
  L0.nbr = g->nbr;
  L0.w = g->w;
  L0.wtype = g->wtype;
  const int64_t n = g->n;
  int64_t *k = nullptr;
  if (j->mode == LCC_NODEW_CUSTOM) {
    if (!g->kc) throw Error(LCC_ERR_INVALID, "LCC_NODEW_CUSTOM needs node weights at load time", j);
    k = g->kc;
  } else if (j->mode == LCC_NODEW_UNIT || j->mode == LCC_NODEW_DEGREE) {
    k = j->base->alloc<int64_t>(n);
    if (j->mode == LCC_NODEW_UNIT) {
      launch_fill_k_unit(k, n, st_, d_);
      note_launches(1);
    } else {
      LJob t = ljob_of(L0);
      t.K = k;  // output of the degree kernel
      deg.push_back(t);
    }
  } else {
    throw Error(LCC_ERR_INVALID, "unknown node-weight mode", j);
  }
  L0.k = k;
  L0.L = j->base->alloc<int32_t>(n);
  L0.K = j->base->alloc<int64_t>(n);
  L0.D = j->base->alloc<int32_t>(n);
  L0.fr = j->base->alloc<uint8_t>(n);
  L0.cl = j->base->alloc<uint8_t>(n);
  L0.lk = j->base->alloc<unsigned long long>(n);
  CK(cudaMemsetAsync(L0.fr, 0, n, st_));
  CK(cudaMemsetAsync(L0.cl, 0, n, st_));
  j->lv.clear();
  j->lv.push_back(L0);
  j->depth = 0;
}

// Node weights of the degree-mode jobs collected by prepare_level0.
void Engine::degree_weights(const std::vector<LJob> &deg) {
  const int nj = (int)deg.size();
  if (nj == 0) return;
  std::vector<int64_t> vs(nj + 1, 0);
  for (int i = 0; i < nj; ++i) vs[i + 1] = vs[i] + deg[i].n;
  LJob *dt = s_ljobs_.get<LJob>(nj, st_);
  int64_t *dv = s_vstart_.get<int64_t>(nj + 1, st_);
  upload_table(deg, vs, dt, dv, stage(nj * (sizeof(LJob) + 8) + 8), st_);
  launch_degree_k(dt, dv, nj, vs[nj], nullptr, st_, d_);
  note_launches(1);
}

// Checks on level 0's statistics: node-weight signs, the modularity scaling
// of lambda, the range of the exact arithmetic and the integer widths.
void Engine::check_level0(Job *j) {
  LevelInfo &I = j->lv[0].info;
  if (I.pad > 0) throw Error(LCC_ERR_INVALID, "negative node weight (degree) in the input", j);
  j->ktot = I.ksum;
  if (j->mode == LCC_NODEW_DEGREE) {
    if (I.ksum <= 0)
      throw Error(LCC_ERR_INVALID, "modularity mode needs a positive total weight", j);
    const i128 qq = (i128)j->q * (i128)I.ksum;
    if (qq > (i128)INT64_MAX) throw Error(LCC_ERR_OVERFLOW, "q * 2m exceeds int64", j);
    j->q = (int64_t)qq;
  }
  // Range of the exact arithmetic.  A q-scaled gain is q w(v,C) - p k_v K_C
  // and q CC is q S_in - p (sum K^2 - sum k^2); with k >= 0 the first terms
  // are at most q * sum|w| and the second at most p * (sum k)^2.  Both
  // below 2^125 keep every gain, every comparison of two gains and the
  // objective inside a signed 128-bit integer on every level (coarse levels
  // keep sum k and never raise sum|w|).
  const i128 lim = (i128)1 << 125;
  const i128 kt = (i128)I.ksum, wa = (i128)I.wabs;
  if (I.ksat || kt >= ((i128)1 << 62) || wa >= ((i128)1 << 62) || (i128)j->q * wa >= lim ||
      (kt > 0 && (i128)j->p > (lim - 1) / (kt * kt)))
    throw Error(LCC_ERR_OVERFLOW,
                "q * sum|w| or p * (sum k)^2 reaches 2^125: outside the exact integer range", j);
  j->lv[0].wide = needs_wide(j->lv[0], j->p, j->q, j->ktot);
  // cluster weights fit the 32-bit half of the packed label word
  if (j->ktot >= (int64_t)KNONE) j->lv[0].lk = nullptr;
}

void Engine::add_job(Job *j, const int32_t *init_labels_host, const uint8_t *frontier_host,
                     bool activate) {
  const int64_t n = j->g->n;
  {
    std::vector<LJob> deg;
    prepare_level0(j, deg);
    degree_weights(deg);
  }
  // statistics of level 0 (also gives sum k for the modularity scaling)
  {
    std::vector<Job *> js = {j};
    std::vector<Level *> lvs = {&j->lv[0]};
    j->ktot = 0;
    level_stats(js, lvs);
    check_level0(j);
    std::vector<Store *> stores = {j->base.get()};
    build_layout(lvs, stores);
  }
  Level &L = j->lv[0];
  if (init_labels_host) {
    CK(cudaMemcpyAsync(L.L, init_labels_host, n * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    LJob t = ljob_of(L);
    std::vector<LJob> tab(1, t);
    std::vector<int64_t> vs = {0, n};
    LJob *dt = s_ljobs_.get<LJob>(1, st_);
    int64_t *dv = s_vstart_.get<int64_t>(2, st_);
    upload_table(tab, vs, dt, dv, stage(sizeof(LJob) + 16), st_);
    launch_recompute_K(dt, dv, 1, n, st_, d_);
    note_launches(2);
    sync_checked(st_);
  } else {
    std::vector<Level *> lvs = {&L};
    init_levels(lvs);
  }
  if (frontier_host) {
    CK(cudaMemcpyAsync(L.fr, frontier_host, n, cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(L.D, L.L, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st_));
  }
  j->phase = P_BM;
  j->round = 0;
  j->moved_level = false;
  if (activate) active_.push_back(j);
}

std::vector<std::pair<Job *, Error>> Engine::add_jobs(const std::vector<Job *> &in) {
  std::vector<std::pair<Job *, Error>> failed;
  auto drop = [&](Job *J, const Error &e) {
    failed.emplace_back(J, e);
    J->lv.clear();
    J->base.reset();
  };
  std::vector<Job *> js;
  std::vector<LJob> deg;
  for (Job *J : in) {
    try {
      prepare_level0(J, deg);
      js.push_back(J);
    } catch (const Error &e) {
      if (!e.job) throw;
      drop(J, e);
    }
  }
  degree_weights(deg);
  std::vector<Level *> lvs;
  for (Job *J : js) {
    J->ktot = 0;
    lvs.push_back(&J->lv[0]);
  }
  level_stats(js, lvs);
  std::vector<Job *> ok;
  std::vector<Level *> oklv;
  std::vector<Store *> stores;
  for (Job *J : js) {
    try {
      check_level0(J);
      ok.push_back(J);
      oklv.push_back(&J->lv[0]);
      stores.push_back(J->base.get());
    } catch (const Error &e) {
      drop(J, e);
    }
  }
  build_layout(oklv, stores);
  init_levels(oklv);
  for (Job *J : ok) {
    J->phase = P_BM;
    J->round = 0;
    J->moved_level = false;
    active_.push_back(J);
  }
  return failed;
}

void Engine::drop_job(Job *j) {
  active_.erase(std::remove(active_.begin(), active_.end(), j), active_.end());
  j->lv.clear();
  j->base.reset();
}

// -------------------------------------------------------------- rounds ----

void Engine::end_bm(Job *j) {
  if (j->kind == BM_ONLY || j->eval_only) {
    j->phase = P_DONE;
    return;
  }
  if (j->kind == BM_REFINE) {
    j->phase = P_UP;
    return;
  }
  // coarsening Best-Moves at this level finished
  if (!j->moved_level || j->depth + 1 >= j->sc.max_levels)
    j->phase = P_UP;
  else
    j->phase = P_CONTRACT;
}

void Engine::round(std::vector<Job *> &js) {
  const int nj = (int)js.size();
  const lcc_tuning tun = tuning_for(dev_);
  const bool pregather = tun.pregather != 0;
  std::vector<int64_t> gw_start(nj + 1, 0);
  int64_t gw_tot = 0;
  std::vector<JobDev> tab(nj);
  std::vector<CoinJob> coins(nj);
  std::vector<int64_t> vs(nj + 1);
  int64_t vt = 0, caps[NB] = {0}, hubcap = 0, hubs = 0, hub_su = 0, hub_max = 0;
  // rows of the buckets from seg0 up take the partitioned path (tuning
  // part_min: 0 = none; 1024, 4096, 8192 or 16384 = rows longer than that)
  const int seg0 = tun.part_min == 0 ? NB
                   : tun.part_min <= 1024 ? B_T2K
                   : tun.part_min <= 4096 ? B_T8K
                   : tun.part_min <= 8192 ? B_T16K : B_T32K;
  PartStat big;
  memset(&big, 0, sizeof(big));
  bool wide = false, any_cl = false, any_mark = false, any_apply = false, any_coin = false;
  for (int i = 0; i < nj; ++i) {
    Job *J = js[i];
    Level &L = J->lv[J->depth];
    JobDev &x = tab[i];
    x.off = L.off;
    x.nbr = L.nbr;
    x.w = L.w;
    x.k = L.k;
    x.L = L.L;
    x.K = L.K;
    x.D = L.D;
    x.fr = L.fr;
    x.cl = L.cl;
    x.lk = L.lk;
    x.pos = L.pos;
    x.gnbr = L.gnbr ? L.gnbr : L.nbr;
    x.n = L.n;
    x.p = J->p;
    x.q = J->q;
    x.wtype = L.wtype;
    x.pull_min = INT64_MAX;
    x.warp_max = L.warp_max;
    // symmetry-breaking coin of this round (LCC_SCHED_COIN): draws keyed by
    // vertex, round, depth and phase (1 = refinement after Flatten)
    const bool coin = (J->sc.flags & LCC_SCHED_COIN) && !J->eval_only;
    CoinJob &cj = coins[i];
    cj.seed = J->sc.seed;
    cj.key_hi = ((uint64_t)(J->round & 0xffff) << 32) + ((uint64_t)(J->depth & 0xff) << 48) +
                ((uint64_t)(J->kind == BM_REFINE ? 1 : 0) << 56);
    cj.on = coin ? 1 : 0;
    cj.pad = 0;
    any_coin |= coin;
    int32_t f = 0;
    if (J->eval_only) {
      f |= JF_EVAL_ONLY;
    } else {
      if (J->round == 0 || J->sc.vset == LCC_VSET_ALL) f |= JF_ALL;
      if (J->sc.vset == LCC_VSET_NBR_VERTICES) {
        f |= JF_MARK_NBR;
        // When the movers' rows cover a quarter of the level's entries, their
        // neighbourhoods are most of the graph: the next round evaluates every
        // vertex with an edge and keeps the labels of those with no moved
        // neighbour, instead of marking V' entry by entry.
        // (a vertex the coin holds back is marked, so coin rounds always mark)
        if (L.lk && !(J->sc.flags & LCC_SCHED_MARK_ONLY) && !coin)
          x.pull_min = std::max<int64_t>(1, L.info.nnz / 4);
        if (J->round > 0 && J->pull) f |= JF_PULL;
      }
      if (J->sc.vset == LCC_VSET_NBR_CLUSTERS) f |= JF_MARK_CL;
      any_apply = true;
    }
    x.flags = f;
    // a round that reads every row (V' = V, or V' tested in the kernels)
    // gathers its label words in one flat pass first
    if (pregather && L.lk && !J->eval_only && (f & (JF_ALL | JF_PULL))) {
      gw_start[i] = gw_tot;
      gw_tot += L.info.nnz;
    }
    gw_start[i + 1] = gw_tot;
    any_cl |= (f & JF_MARK_CL) != 0;
    any_mark |= (f & (JF_MARK_NBR | JF_MARK_CL)) != 0;
    vs[i] = vt;
    vt += L.n;
    for (int b = 0; b < NB; ++b) caps[b] += L.info.bcnt[b];
    hubcap += L.info.hub_cap;
    hubs += L.info.bcnt[B_HUB];
    hub_su += L.info.hub_sunits;
    hub_max = std::max(hub_max, L.info.hub_maxcap);
    for (int bk = seg0; bk < NB; ++bk) {
      const PartStat &ps = L.info.pst[bk - PB0];
      big.rows += ps.rows;
      big.nnz += ps.nnz;
      big.parts += ps.parts;
      big.chunks += ps.chunks;
      big.cells += ps.cells;
      big.cap += ps.cap;
      big.sunits += ps.sunits;
      big.maxcap = std::max(big.maxcap, ps.maxcap);
    }
    wide |= L.wide;
  }
  vs[nj] = vt;
  // the hub tables are then sized for all the partitioned path's rows (they
  // serve its fallback rows)
  const bool part_mode = big.rows > 0;
  if (part_mode) {
    hubcap = big.cap;
    hubs = big.rows;
    hub_su = big.sunits;
    hub_max = big.maxcap;
  }

  Buckets b;
  int64_t tot = 0;
  for (int i = 0; i < NB; ++i) {
    b.seg_start[i] = tot;
    b.seg_cap[i] = caps[i];
    tot += caps[i];
  }
  b.items = s_items_.get<uint64_t>(tot, st_);
  b.cnt = s_cnt_.get<int64_t>(NB, st_);

  int64_t *ctr = s_ctr_.get<int64_t>(NCTR, st_);
  int64_t *jm = s_jmoves_.get<int64_t>(2 * nj, st_);
  uint64_t *moved = s_moved_.get<uint64_t>(vt, st_);
  HubBufs h;
  memset(&h, 0, sizeof(h));
  int64_t hub_passes = 0;
  if (hubs > 0) {
    // Hub tables are processed in windows of kHubWindow slots (plus the
    // largest table that may start near the end of a window).
    const int64_t win = std::min(hubcap, hub_window());
    hub_passes = (hubcap + win - 1) / win;
    h.keys = s_hkeys_.get<unsigned long long>(win + hub_max, st_);
    h.vals = s_hvals_.get<int64_t>(win + hub_max, st_);
    h.window = win;
    int64_t *meta = s_hmeta_.get<int64_t>(3 * (hubs + 1) + hubs, st_);
    h.tbl_off = meta;
    h.unit_off = meta + (hubs + 1);
    h.sunit_off = meta + 2 * (hubs + 1);
    h.stay = meta + 3 * (hubs + 1);
    h.part_score = s_hpart_s_.get<i128>(hub_su, st_);
    h.part_cid = s_hpart_c_.get<int32_t>(hub_su, st_);
    h.iso_seen = s_hiso_.get<int32_t>(hubs, st_);
    h.max_hubs = hubs;
    h.max_sunits = hub_su;
  }
  PartBufs pb;
  memset(&pb, 0, sizeof(pb));
  if (part_mode) {
    const int64_t R = big.rows, NPt = big.parts, NC = big.chunks;
    const int64_t NCe = big.cells, NE = big.nnz;
    int64_t *pm = s_pmeta_.get<int64_t>(3 * (R + 1) + (NCe + 1) + R + 2 +
                                            scan_tmp_elems(std::max(NCe, R) + 1), st_);
    pb.part_off = pm;
    pb.chunk_off = pm + (R + 1);
    pb.cell_off = pm + 2 * (R + 1);
    pb.cells = pm + 3 * (R + 1);
    pb.stay = pb.cells + (NCe + 1);
    pb.nfallback = pb.stay + R;
    pb.nrows = pb.nfallback + 1;
    pb.scan_tmp = pb.nrows + 1;
    pb.row = s_prow_.get<uint64_t>(2 * R, st_);
    pb.fallback = pb.row + R;
    pb.flag = s_pflag_.get<int32_t>(R, st_);
    pb.pword = s_pword_.get<unsigned long long>(NE, st_);
    pb.pw = s_pw_.get<int64_t>(NE, st_);
    pb.part_score = s_pscore_.get<i128>(NPt, st_);
    pb.part_cid = s_pcid_.get<int32_t>(NPt + NC, st_);
    pb.chunk_row = pb.part_cid + NPt;
    pb.desc = s_pdesc_.get<PartDesc>(NPt, st_);
    pb.max_rows = R;
    pb.max_parts = NPt;
    pb.max_chunks = NC;
    pb.max_cells = NCe;
    pb.max_entries = NE;
    pb.table_slots = part_table_slots();
    pb.seg0 = seg0;
  }
  unsigned long long *gwbuf = nullptr;
  int64_t *dgw = nullptr;
  if (gw_tot > 0) {
    gwbuf = s_gw_.get<unsigned long long>(gw_tot, st_);
    dgw = s_gwoff_.get<int64_t>(nj + 1, st_);
    for (int i = 0; i < nj; ++i)
      if (gw_start[i + 1] > gw_start[i]) tab[i].gw = gwbuf + gw_start[i];
  }
  JobDev *dt = s_jobs_.get<JobDev>(nj, st_);
  int64_t *dv = s_vstart_.get<int64_t>(nj + 1, st_);
  const size_t tab_bytes = nj * (sizeof(JobDev) + 8) + 8;
  const size_t gw_bytes = gw_tot > 0 ? (nj + 1) * sizeof(int64_t) : 0;
  char *hs = (char *)stage(tab_bytes + (any_coin ? nj * sizeof(CoinJob) : 0) + gw_bytes);
  upload_table(tab, vs, dt, dv, hs, st_);
  if (gw_tot > 0) {
    char *hg = hs + tab_bytes + (any_coin ? nj * sizeof(CoinJob) : 0);
    memcpy(hg, gw_start.data(), gw_bytes);
    CK(cudaMemcpyAsync(dgw, hg, gw_bytes, cudaMemcpyHostToDevice, st_));
  }
  CoinJob *dcoin = nullptr;
  int64_t *dheld = nullptr;
  if (any_coin) {
    dcoin = s_coin_.get<CoinJob>(nj, st_);
    dheld = s_jheld_.get<int64_t>(nj, st_);
    memcpy(hs + tab_bytes, coins.data(), nj * sizeof(CoinJob));
    CK(cudaMemcpyAsync(dcoin, hs + tab_bytes, nj * sizeof(CoinJob), cudaMemcpyHostToDevice, st_));
    CK(cudaMemsetAsync(dheld, 0, nj * sizeof(int64_t), st_));
  }
  CK(cudaMemsetAsync(b.cnt, 0, NB * sizeof(int64_t), st_));
  CK(cudaMemsetAsync(ctr, 0, NCTR * sizeof(int64_t), st_));
  CK(cudaMemsetAsync(jm, 0, 2 * nj * sizeof(int64_t), st_));

  int launches = 0;
  if (timing) CK(cudaEventRecord(ev_[0], st_));
  launch_frontier(dt, dv, nj, vt, b, ctr, st_, d_);
  ++launches;
  // the gathered-word pass does the best-move kernels' gathers: it is timed
  // with them (ms_bestmove), before the first degree bucket
  if (timing) CK(cudaEventRecord(ev_[1], st_));
  if (gw_tot > 0) {  // after the frontier kernel wrote this round's label words
    launch_gather_words(dt, dgw, nj, gw_tot, st_, d_);
    ++launches;
  }
  if (timing) CK(cudaEventRecord(ev_gw_, st_));
  launch_bestmove(wide, dt, b, h, hub_passes, ctr, st_, d_, &launches, timing ? bev_ : nullptr,
                  tun.fuse_small != 0, tun.prefetch != 0, part_mode ? &pb : nullptr);
  if (timing) CK(cudaEventRecord(ev_[2], st_));
  if (any_coin) {
    launch_coin(dt, dcoin, b, dheld, st_, d_);
    ++launches;
  }
  if (any_apply) {
    launch_apply(dt, b, jm, moved, vt, ctr, st_, d_);
    ++launches;
    if (any_mark) launch_mark(dt, moved, ctr, jm, any_cl, dv, nj, vt, st_, d_, &launches);
  }
  if (timing) CK(cudaEventRecord(ev_[3], st_));
  note_launches(launches);

  int64_t *hbuf = (int64_t *)stage2((NCTR + 3 * nj) * sizeof(int64_t));
  CK(cudaMemcpyAsync(hbuf, ctr, NCTR * sizeof(int64_t), cudaMemcpyDeviceToHost, st_));
  CK(cudaMemcpyAsync(hbuf + NCTR, jm, 2 * nj * sizeof(int64_t), cudaMemcpyDeviceToHost, st_));
  if (any_coin)
    CK(cudaMemcpyAsync(hbuf + NCTR + 2 * nj, dheld, nj * sizeof(int64_t), cudaMemcpyDeviceToHost,
                       st_));
  sync_checked(st_);
  if (hbuf[C_ERR])
    throw Error(LCC_ERR_CUDA, "best-move round overflowed a work buffer (code " +
                                  std::to_string(hbuf[C_ERR]) + ")");
  stats.edges += hbuf[C_EDGES];
  stats.verts += hbuf[C_VERTS];
  stats.cands += hbuf[C_CANDS];
  stats.wbytes += hbuf[C_WB];
  for (int i = 0; i < NB; ++i) {
    stats.bucket_entries[i] += hbuf[C_BE + i];
    stats.bucket_vertices[i] += hbuf[C_BV + i];
  }
  stats.rounds += 1;
  if (timing) {
    for (int i = 0; i < NB; ++i)
      stats.ms_bucket[i] += elapsed(i == 0 ? ev_gw_ : bev_[i - 1], bev_[i]);
    stats.ms_gather += elapsed(ev_[1], ev_gw_);
    stats.ms_bm += elapsed(ev_[1], ev_[2]);
    stats.ms_round_other += elapsed(ev_[0], ev_[1]) + elapsed(ev_[2], ev_[3]);
  }
  for (int i = 0; i < nj; ++i) {
    Job *J = js[i];
    const int64_t mv = hbuf[NCTR + 2 * i];
    const int64_t held = any_coin ? hbuf[NCTR + 2 * nj + i] : 0;
    // the mark kernel skipped this job under the same test
    J->pull = hbuf[NCTR + 2 * i + 1] >= tab[i].pull_min;
    J->round += 1;
    J->rounds_total += 1;
    if (J->eval_only) {
      end_bm(J);
      continue;
    }
    if (J->trace && nj == 1) {
      lcc_round rr;
      memset(&rr, 0, sizeof(rr));
      rr.level = J->depth;
      rr.phase = J->kind == BM_REFINE ? 1 : 0;
      rr.round = J->round - 1;
      rr.vprime = hbuf[C_VERTS];
      rr.entries = hbuf[C_EDGES];
      rr.moved = mv;
      rr.held = held;
      J->trace->push_back(rr);
    }
    if (mv > 0) {
      J->moved_level = true;
      J->moved_any = true;
    }
    // the call ends when no vertex wants to move: none moved and the coin
    // held none back (converged), or after num_iter rounds
    const bool converged = mv == 0 && held == 0;
    if (converged || J->round >= J->sc.num_iter) {
      J->calls += 1;
      if (!converged) J->calls_capped += 1;
      end_bm(J);
    }
  }
}

// ---------------------------------------------------------- contraction ----

static int bits_for(int64_t x) {  // bits needed for values in [0, x)
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) < x) ++b;
  return b;
}

void Engine::contract(std::vector<Job *> &js) {
  const int nj = (int)js.size();
  if (timing) CK(cudaEventRecord(ev_[4], st_));
  std::vector<CJob> tab(nj);
  std::vector<int64_t> vs(nj + 1);
  int64_t vt = 0, et = 0, read_min = 0;
  for (int i = 0; i < nj; ++i) {
    Level &L = js[i]->lv[js[i]->depth];
    et += L.info.nnz;
    // least reads: offsets, neighbours, weights and labels, once each
    const int64_t wb = L.wtype == W_I32 ? 4 : (L.wtype == W_I64 ? 8 : 0);
    read_min += (L.n + 1) * 8 + L.info.nnz * (4 + wb) + L.n * 4;
    CJob &c = tab[i];
    memset(&c, 0, sizeof(c));
    c.off = L.off;
    c.nbr = L.nbr;
    c.w = L.w;
    c.L = L.L;
    c.K = L.K;
    c.pos = L.pos;
    c.gnbr = L.gnbr ? L.gnbr : L.nbr;
    c.n = L.n;
    c.wtype = L.wtype;
    vs[i] = vt;
    vt += L.n;
  }
  vs[nj] = vt;
  auto store = std::make_shared<Store>(st_);
  int32_t *map_u = store->alloc<int32_t>(vt);
  for (int i = 0; i < nj; ++i) tab[i].map = map_u + vs[i];

  Store tmp(st_);
  CJob *dt = tmp.alloc<CJob>(nj);
  int64_t *dv = tmp.alloc<int64_t>(nj + 1);
  {
    char *h = (char *)stage(nj * sizeof(CJob) + (nj + 1) * 8);
    memcpy(h, tab.data(), nj * sizeof(CJob));
    memcpy(h + nj * sizeof(CJob), vs.data(), (nj + 1) * 8);
    CK(cudaMemcpyAsync(dt, h, nj * sizeof(CJob), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(dv, h + nj * sizeof(CJob), (nj + 1) * 8, cudaMemcpyHostToDevice, st_));
  }
  int64_t *rank = tmp.alloc<int64_t>(vt + 1);
  int32_t *gmap = tmp.alloc<int32_t>(vt);
  int32_t *gmapp = tmp.alloc<int32_t>(vt);
  int64_t *stmp = tmp.alloc<int64_t>(scan_tmp_elems(vt + 1));
  int64_t *jc = tmp.alloc<int64_t>(2 * nj);
  int32_t *err = tmp.alloc<int32_t>(1);
  unsigned long long *intra = tmp.alloc<unsigned long long>(1);
  CK(cudaMemsetAsync(rank, 0, (vt + 1) * 8, st_));
  CK(cudaMemsetAsync(err, 0, 4, st_));
  CK(cudaMemsetAsync(intra, 0, 8, st_));
  launch_occ(dt, dv, nj, vt, rank, err, st_, d_);
  scan_exclusive_i64(rank, vt, stmp, st_, d_);
  launch_job_counts(dv, nj, rank, jc, st_);
  launch_relabel(dt, dv, nj, vt, rank, gmap, gmapp, st_, d_);
  note_launches(8);
  int64_t *hb = (int64_t *)stage2((3 + 2 * nj) * 8);
  CK(cudaMemcpyAsync(hb, rank + vt, 8, cudaMemcpyDeviceToHost, st_));
  CK(cudaMemcpyAsync(hb + 2, err, 4, cudaMemcpyDeviceToHost, st_));
  CK(cudaMemcpyAsync(hb + 3, jc, 2 * nj * 8, cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  if ((int32_t)hb[2]) throw Error(LCC_ERR_INVALID, "label out of range in Compress");
  const int64_t ntot = hb[0];
  std::vector<int64_t> nprime(nj), cbase(nj);
  for (int i = 0; i < nj; ++i) {
    nprime[i] = hb[3 + 2 * i];
    cbase[i] = hb[3 + 2 * i + 1];
  }
  if (ntot >= ((int64_t)1 << 31) - 1) throw Error(LCC_ERR_OVERFLOW, "too many coarse vertices");
  int64_t *knew = store->alloc<int64_t>(ntot);
  launch_knew(dt, dv, nj, vt, rank, knew, st_, d_);
  note_launches(1);

  // Every coarse row gets a region of the flat entry space as large as the
  // sum of its members' degrees; each fine vertex appends its entries that
  // leave its cluster to its coarse row's region.
  int64_t *boff = tmp.alloc<int64_t>(ntot + 1);
  int64_t *rpos = tmp.alloc<int64_t>(vt);
  int64_t *stmp2 = tmp.alloc<int64_t>(scan_tmp_elems(ntot + 1));
  int32_t *tnbr = tmp.alloc<int32_t>(et);
  int64_t *tw = tmp.alloc<int64_t>(et);
  int64_t *offg = store->alloc<int64_t>(ntot + 1);
  CK(cudaMemsetAsync(boff, 0, (ntot + 1) * 8, st_));
  CK(cudaMemsetAsync(offg, 0, (ntot + 1) * 8, st_));
  launch_rbound(dt, dv, nj, vt, gmap, boff, rpos, st_, d_);
  scan_exclusive_i64(boff, ntot, stmp2, st_, d_);
  RowSpace R;
  memset(&R, 0, sizeof(R));
  R.jobs = dt;
  R.vstart = dv;
  R.njobs = nj;
  R.gmap = gmap;
  R.gmapp = gmapp;
  R.rank = rank;
  R.boff = boff;
  R.rpos = rpos;
  R.tnbr = tnbr;
  R.tw = tw;
  R.ucnt = offg;  // unique entries per row, scanned into the offsets below
  R.intra = intra;
  launch_emit_rows(R, vt, st_, d_);
  // rows by their number of entries
  unsigned long long *ccnt = tmp.alloc<unsigned long long>(RC_N);
  int64_t *dseg = tmp.alloc<int64_t>(RC_N);
  CK(cudaMemsetAsync(ccnt, 0, RC_N * 8, st_));
  launch_rows_classify(R, ntot, false, ccnt, nullptr, nullptr, st_, d_);
  note_launches(6);
  int64_t *hc = (int64_t *)stage2(RC_N * 8);
  CK(cudaMemcpyAsync(hc, ccnt, RC_N * 8, cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  int64_t cnt[RC_N], seg[RC_N], nrows = 0;
  for (int c = 0; c < RC_N; ++c) {
    cnt[c] = hc[c];
    seg[c] = nrows;
    nrows += cnt[c];
  }
  int32_t *items = tmp.alloc<int32_t>(nrows);
  {
    int64_t *hs = (int64_t *)stage(RC_N * 8);
    memcpy(hs, seg, sizeof(seg));
    CK(cudaMemcpyAsync(dseg, hs, RC_N * 8, cudaMemcpyHostToDevice, st_));
  }
  CK(cudaMemsetAsync(ccnt, 0, RC_N * 8, st_));
  launch_rows_classify(R, ntot, true, ccnt, dseg, items, st_, d_);
  // each row merges its region in place: unique entries at its start,
  // their number in offg[C] (rows of one entry were counted by the classes)
  int launches = 1;
  launch_rows_small(R, items, seg, cnt, st_, d_, &launches);
  const int64_t H = cnt[RC_BIG];
  if (H > 0) {
    // rows longer than a block's table: global tables, in windows of slots
    const int32_t *bitems = items + seg[RC_BIG];
    int64_t *bb = tmp.alloc<int64_t>(H);
    launch_big_bounds(R, bitems, H, bb, st_, d_);
    ++launches;
    int64_t *hbb = (int64_t *)stage2(H * 8);
    CK(cudaMemcpyAsync(hbb, bb, H * 8, cudaMemcpyDeviceToHost, st_));
    sync_checked(st_);
    const std::vector<int64_t> bnd(hbb, hbb + H);
    std::vector<int64_t> offs(3 * (H + 1));
    int64_t *to = offs.data(), *uo = to + (H + 1), *so = uo + (H + 1);
    int64_t maxcap = 0;
    to[0] = uo[0] = so[0] = 0;
    for (int64_t h = 0; h < H; ++h) {
      const int64_t cap = next_pow2(2 * bnd[h]);
      maxcap = std::max(maxcap, cap);
      to[h + 1] = to[h] + cap;
      uo[h + 1] = uo[h] + (bnd[h] + RC_CHUNK - 1) / RC_CHUNK;
      so[h + 1] = so[h] + (cap + RC_SCHUNK - 1) / RC_SCHUNK;
    }
    int64_t *doffs = tmp.alloc<int64_t>(3 * (H + 1));
    {
      int64_t *hs = (int64_t *)stage(offs.size() * 8);
      memcpy(hs, offs.data(), offs.size() * 8);
      CK(cudaMemcpyAsync(doffs, hs, offs.size() * 8, cudaMemcpyHostToDevice, st_));
    }
    const int64_t win = std::min(to[H], row_window());
    BigRows B;
    B.keys = tmp.alloc<int32_t>(win + maxcap);
    B.vals = tmp.alloc<unsigned long long>(win + maxcap);
    B.tbl_off = doffs;
    B.unit_off = doffs + (H + 1);
    B.sunit_off = doffs + 2 * (H + 1);
    B.H = H;
    for (int64_t h0 = 0; h0 < H;) {
      const int64_t lo = to[h0];
      int64_t h1 = h0 + 1;
      while (h1 < H && to[h1] < lo + win) ++h1;
      const int64_t slots = to[h1] - lo;
      CK(cudaMemsetAsync(B.keys, 0xFF, slots * 4, st_));
      CK(cudaMemsetAsync(B.vals, 0, slots * 8, st_));
      launch_big_window(R, bitems, B, h0, h1, lo, uo[h1] - uo[h0], so[h1] - so[h0], st_, d_,
                        &launches);
      h0 = h1;
    }
  }
  scan_exclusive_i64(offg, ntot, stmp2, st_, d_);
  note_launches(launches + 2);
  int64_t *hu = (int64_t *)stage2(16);
  CK(cudaMemcpyAsync(hu, offg + ntot, 8, cudaMemcpyDeviceToHost, st_));
  CK(cudaMemcpyAsync(hu + 1, intra, 8, cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  const int64_t U = hu[0];
  const int64_t nintra = hu[1];
  stats.pairs += et - nintra;
  // least writes: coarse offsets, neighbours, int64 weights and node weights
  stats.contract_min_bytes += read_min + (ntot + nj) * 8 + U * (4 + 8) + ntot * 8;
  int64_t *uvals = store->alloc<int64_t>(U);
  int32_t *unbr = store->alloc<int32_t>(U);
  launch_rows_copy(R, ntot, offg, unbr, uvals, st_, d_);
  note_launches(1);
  int32_t *Lu = store->alloc<int32_t>(ntot);
  int64_t *Ku = store->alloc<int64_t>(ntot);
  int32_t *Du = store->alloc<int32_t>(ntot);
  uint8_t *fru = store->alloc<uint8_t>(ntot);
  uint8_t *clu = store->alloc<uint8_t>(ntot);
  unsigned long long *lku = store->alloc<unsigned long long>(ntot);
  CK(cudaMemsetAsync(fru, 0, ntot > 0 ? ntot : 1, st_));
  CK(cudaMemsetAsync(clu, 0, ntot > 0 ? ntot : 1, st_));

  std::vector<Job *> grow;
  std::vector<Level *> newlv;
  for (int i = 0; i < nj; ++i) {
    Job *J = js[i];
    Level &Lf = J->lv[J->depth];
    if (nprime[i] >= Lf.n && !J->keep_coarse) {  // no shrink: the recursion ends here
      J->phase = P_UP;
      continue;
    }
    Lf.map = map_u + vs[i];
    Lf.map_store = store;
    Level nl;
    nl.n = nprime[i];
    nl.warp_max = tuning_for(dev_).warp_max;
    nl.entries_from_zero = cbase[i] == 0;
    nl.off = offg + cbase[i];
    nl.nbr = unbr;
    nl.w = uvals;
    nl.wtype = W_I64;
    nl.k = knew + cbase[i];
    nl.L = Lu + cbase[i];
    nl.K = Ku + cbase[i];
    nl.D = Du + cbase[i];
    nl.fr = fru + cbase[i];
    nl.cl = clu + cbase[i];
    nl.lk = J->ktot < (int64_t)KNONE ? lku + cbase[i] : nullptr;
    nl.store = store;
    J->lv.push_back(nl);
    J->depth += 1;
    J->levels = std::max(J->levels, J->depth + 1);
    J->phase = P_BM;
    J->kind = BM_COARSEN;
    J->round = 0;
    J->moved_level = false;
    grow.push_back(J);
  }
  for (Job *J : grow) newlv.push_back(&J->lv[J->depth]);
  level_stats(grow, newlv);
  {
    std::vector<Store *> stores(newlv.size(), store.get());
    build_layout(newlv, stores);
  }
  init_levels(newlv);
  if (timing) {
    CK(cudaEventRecord(ev_[5], st_));
    CK(cudaEventSynchronize(ev_[5]));
    stats.ms_contract += elapsed(ev_[4], ev_[5]);
  }
  // temporaries are released (stream-ordered) when `tmp` goes out of scope
}

// ------------------------------------------------------------------ up ----

void Engine::up(std::vector<Job *> &js) {
  if (timing) CK(cudaEventRecord(ev_[6], st_));
  std::vector<Job *> cur = js;
  while (!cur.empty()) {
    std::vector<Job *> fl;
    for (Job *J : cur) {
      if (J->depth == 0)
        J->phase = P_FINAL;
      else
        fl.push_back(J);
    }
    if (fl.empty()) break;
    const int nj = (int)fl.size();
    std::vector<LJob> tab(nj);
    std::vector<int64_t> vs(nj + 1);
    int64_t vt = 0;
    for (int i = 0; i < nj; ++i) {
      Job *J = fl[i];
      Level &Lf = J->lv[J->depth - 1];
      Level &Lc = J->lv[J->depth];
      tab[i] = ljob_of(Lf);
      tab[i].map = Lf.map;
      tab[i].Lcoarse = Lc.L;
      vs[i] = vt;
      vt += Lf.n;
    }
    vs[nj] = vt;
    LJob *dt = s_ljobs_.get<LJob>(nj, st_);
    int64_t *dv = s_vstart_.get<int64_t>(nj + 1, st_);
    upload_table(tab, vs, dt, dv, stage(nj * (sizeof(LJob) + 8) + 8), st_);
    launch_flatten(dt, dv, nj, vt, st_, d_);
    note_launches(1);
    std::vector<LJob> rtab;
    std::vector<int64_t> rvs(1, 0);
    std::vector<Job *> next;
    for (int i = 0; i < nj; ++i) {
      Job *J = fl[i];
      J->lv.pop_back();  // stream-ordered release of the coarse level
      J->depth -= 1;
      Level &Lf = J->lv[J->depth];
      Lf.map = nullptr;
      Lf.map_store.reset();
      if (J->sc.refine) {
        rtab.push_back(ljob_of(Lf));
        rvs.push_back(rvs.back() + Lf.n);
        J->phase = P_BM;
        J->kind = BM_REFINE;
        J->round = 0;
        J->moved_level = false;
      } else {
        next.push_back(J);
      }
    }
    sync_checked(st_);  // staging reuse
    if (!rtab.empty()) {
      const int nr = (int)rtab.size();
      LJob *rt = s_ljobs_.get<LJob>(nr, st_);
      int64_t *rv = s_vstart_.get<int64_t>(nr + 1, st_);
      upload_table(rtab, rvs, rt, rv, stage(nr * (sizeof(LJob) + 8) + 8), st_);
      launch_recompute_K(rt, rv, nr, rvs.back(), st_, d_);
      note_launches(2);
      sync_checked(st_);
    }
    cur.swap(next);
  }
  if (timing) {
    CK(cudaEventRecord(ev_[7], st_));
    CK(cudaEventSynchronize(ev_[7]));
    stats.ms_other += elapsed(ev_[6], ev_[7]);
  }
}

// --------------------------------------------------------------- final ----

void Engine::finalize(std::vector<Job *> &js) {
  const int nj = (int)js.size();
  if (nj == 0) return;
  if (timing) CK(cudaEventRecord(ev_[6], st_));
  std::vector<LJob> tab(nj);
  std::vector<int64_t> vs(nj + 1);
  int64_t vt = 0;
  for (int i = 0; i < nj; ++i) {
    tab[i] = ljob_of(js[i]->lv[0]);
    vs[i] = vt;
    vt += js[i]->lv[0].n;
  }
  vs[nj] = vt;
  LJob *dt = s_ljobs_.get<LJob>(nj, st_);
  int64_t *dv = s_vstart_.get<int64_t>(nj + 1, st_);
  ObjAcc *acc = s_obj_.get<ObjAcc>(nj, st_);
  upload_table(tab, vs, dt, dv, stage(nj * (sizeof(LJob) + 8) + 8), st_);
  CK(cudaMemsetAsync(acc, 0, nj * sizeof(ObjAcc), st_));
  launch_canonical(dt, dv, nj, vt, st_, d_);
  launch_objective(dt, dv, nj, vt, acc, st_, d_);
  note_launches(7);
  ObjAcc *h = (ObjAcc *)stage2(nj * sizeof(ObjAcc));
  CK(cudaMemcpyAsync(h, acc, nj * sizeof(ObjAcc), cudaMemcpyDeviceToHost, st_));
  for (int i = 0; i < nj; ++i) {
    Job *J = js[i];
    if (J->labels_out) {
      cudaMemcpyKind kind = J->labels_space == LCC_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                              : cudaMemcpyDeviceToHost;
      CK(cudaMemcpyAsync(J->labels_out, J->lv[0].L, J->lv[0].n * sizeof(int32_t), kind, st_));
    }
  }
  sync_checked(st_);
  for (int i = 0; i < nj; ++i) {
    Job *J = js[i];
    const i128 s_in = (i128)(int64_t)h[i].s_in;
    const u128 ksq = ((u128)h[i].ksq_hi << 64) | h[i].ksq_lo;
    const u128 kself = ((u128)h[i].kself_hi << 64) | h[i].kself_lo;
    J->num = (i128)J->q * s_in - (i128)J->p * (i128)(ksq - kself);
    J->den = J->q;
    J->nclusters = (int64_t)h[i].nclus;
    J->phase = P_DONE;
  }
  if (timing) {
    CK(cudaEventRecord(ev_[7], st_));
    CK(cudaEventSynchronize(ev_[7]));
    stats.ms_other += elapsed(ev_[6], ev_[7]);
  }
}

void Engine::objective_of(Job *J) {
  std::vector<Job *> js = {J};
  std::vector<LJob> tab(1, ljob_of(J->lv[0]));
  std::vector<int64_t> vs = {0, J->lv[0].n};
  LJob *dt = s_ljobs_.get<LJob>(1, st_);
  int64_t *dv = s_vstart_.get<int64_t>(2, st_);
  ObjAcc *acc = s_obj_.get<ObjAcc>(1, st_);
  upload_table(tab, vs, dt, dv, stage(sizeof(LJob) + 16), st_);
  CK(cudaMemsetAsync(acc, 0, sizeof(ObjAcc), st_));
  launch_objective(dt, dv, 1, vs[1], acc, st_, d_);
  note_launches(4);
  ObjAcc *h = (ObjAcc *)stage2(sizeof(ObjAcc));
  CK(cudaMemcpyAsync(h, acc, sizeof(ObjAcc), cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  const i128 s_in = (i128)(int64_t)h->s_in;
  const u128 ksq = ((u128)h->ksq_hi << 64) | h->ksq_lo;
  const u128 kself = ((u128)h->kself_hi << 64) | h->kself_lo;
  J->num = (i128)J->q * s_in - (i128)J->p * (i128)(ksq - kself);
  J->den = J->q;
}

void Engine::compress_to_graph(Job *J, int32_t *map_host, lcc_graph **out) {
  std::vector<Job *> js = {J};
  J->sc.max_levels = 2;
  contract(js);
  if (J->depth != 1) throw Error(LCC_ERR_CUDA, "internal: Compress produced no level");
  Level &Lf = J->lv[0];
  Level &Lc = J->lv[1];
  const int64_t n2 = Lc.n;
  int64_t first = 0, last = 0;
  CK(cudaMemcpyAsync(&first, Lc.off, 8, cudaMemcpyDeviceToHost, st_));
  CK(cudaMemcpyAsync(&last, Lc.off + n2, 8, cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  const int64_t nnz2 = last - first;
  lcc_graph *g = new lcc_graph();
  g->dev = dev_;
  g->st = st_;
  g->n = n2;
  g->nnz = nnz2;
  g->store = std::make_shared<Store>(st_);
  g->off = g->store->alloc<int64_t>(n2 + 1);
  g->nbr = g->store->alloc<int32_t>(nnz2);
  int64_t *w = g->store->alloc<int64_t>(nnz2);
  g->w = w;
  g->wtype = W_I64;
  g->kc = g->store->alloc<int64_t>(n2);
  CK(cudaMemcpyAsync(g->off, Lc.off, (n2 + 1) * 8, cudaMemcpyDeviceToDevice, st_));
  if (nnz2 > 0) {
    CK(cudaMemcpyAsync(g->nbr, Lc.nbr + first, nnz2 * 4, cudaMemcpyDeviceToDevice, st_));
    CK(cudaMemcpyAsync(w, (const int64_t *)Lc.w + first, nnz2 * 8, cudaMemcpyDeviceToDevice, st_));
  }
  CK(cudaMemcpyAsync(g->kc, Lc.k, n2 * 8, cudaMemcpyDeviceToDevice, st_));
  if (map_host) CK(cudaMemcpyAsync(map_host, Lf.map, Lf.n * 4, cudaMemcpyDeviceToHost, st_));
  sync_checked(st_);
  if (first != 0) {
    // offsets of a single-job level start at 0; keep the invariant explicit
    throw Error(LCC_ERR_CUDA, "internal: coarse offsets do not start at 0");
  }
  if (nnz2 > 1) {
    // Compress leaves a row's entries in table order; the exported graph has
    // every row ascending by neighbour: sort (row << 32 | neighbour, w)
    Store srt(st_);
    uint64_t *k1 = srt.alloc<uint64_t>(nnz2), *k2 = srt.alloc<uint64_t>(nnz2);
    int64_t *w2 = srt.alloc<int64_t>(nnz2);
    int64_t *rt = srt.alloc<int64_t>(radix_tmp_elems(nnz2));
    launch_row_keys(g->off, n2, g->nbr, k1, st_, d_);
    int shifts[16], np = 0;
    const int b = bits_for(n2);
    for (int sh = 0; sh < b; sh += 8) shifts[np++] = sh;
    for (int sh = 32; sh < 32 + b; sh += 8) shifts[np++] = sh;
    bool in_alt = false;
    int lc = 0;
    radix_sort_pairs(k1, w, k2, w2, nnz2, shifts, np, rt, st_, d_, &in_alt, &lc);
    launch_row_unkey(in_alt ? k2 : k1, nnz2, g->nbr, st_, d_);
    if (in_alt) CK(cudaMemcpyAsync(w, w2, nnz2 * 8, cudaMemcpyDeviceToDevice, st_));
    note_launches(lc + 2);
    sync_checked(st_);
  }
  // |w| total of the coarse graph never exceeds the input's
  g->wabs = J->g->wabs;
  *out = g;
}

// ---------------------------------------------------------------- tick ----

std::vector<Job *> Engine::tick() {
  // Per-job checks come first, while no job's state has changed in this
  // tick: an error raised here names its job, and the caller can drop that
  // job and tick the others again.
  for (Job *J : active_) {
    J->ticks += 1;
    if (J->inject_fault_tick > 0 && J->ticks >= J->inject_fault_tick)
      throw Error(LCC_ERR_CUDA, "injected fault (tick " + std::to_string(J->ticks) + ")", J);
  }
  std::vector<Job *> bm;
  for (Job *J : active_)
    if (J->phase == P_BM) bm.push_back(J);
  if (!bm.empty()) {
    // jobs that would run zero rounds end their Best-Moves at once
    std::vector<Job *> run;
    for (Job *J : bm) {
      if (J->sc.num_iter <= 0 && !J->eval_only)
        end_bm(J);
      else
        run.push_back(J);
    }
    if (!run.empty()) round(run);
  }
  std::vector<Job *> ct;
  for (Job *J : active_)
    if (J->phase == P_CONTRACT) ct.push_back(J);
  if (!ct.empty()) contract(ct);
  std::vector<Job *> u;
  for (Job *J : active_)
    if (J->phase == P_UP) u.push_back(J);
  if (!u.empty()) up(u);
  std::vector<Job *> fin;
  for (Job *J : active_)
    if (J->phase == P_FINAL) fin.push_back(J);
  if (!fin.empty()) finalize(fin);
  std::vector<Job *> done;
  for (Job *J : active_)
    if (J->phase == P_DONE) done.push_back(J);
  for (Job *J : done)
    active_.erase(std::remove(active_.begin(), active_.end(), J), active_.end());
  return done;
}

// ------------------------------------------------------- shared engines ----

static std::mutex g_eng_mu;
struct EngSlot {
  std::unique_ptr<Engine> eng;
  std::unique_ptr<std::mutex> mu;
};
static std::unordered_map<uint64_t, EngSlot> g_engines;

Engine *engine_for(int dev, cudaStream_t st, std::unique_lock<std::mutex> &lock) {
  std::mutex *m;
  Engine *e;
  {
    std::lock_guard<std::mutex> lk(g_eng_mu);
    const uint64_t key = ((uint64_t)dev << 56) ^ (uint64_t)(uintptr_t)st;
    EngSlot &s = g_engines[key];
    if (!s.eng) {
      s.eng.reset(new Engine(dev, st));
      s.mu.reset(new std::mutex());
    }
    m = s.mu.get();
    e = s.eng.get();
  }
  lock = std::unique_lock<std::mutex>(*m);
  return e;
}

}  // namespace lcc
