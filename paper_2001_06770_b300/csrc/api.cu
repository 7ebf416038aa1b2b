// C ABI of librpq (include/rpq.h): validation, graph load, search slots,
// CUDA graphs per query shape, batches over concurrent slots, tracing.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "rpq_host.h"

namespace rpq {

static thread_local std::string g_last_error;

void set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = std::string(rpq_strerror(code)) + ": " + buf;
}

int dev_err_to_status(uint32_t err) {
  if (!err) return RPQ_OK;
  if (err & kErrTimeout) { set_error(RPQ_ETIMEOUT, "a bounded device wait ran out"); return RPQ_ETIMEOUT; }
  if (err & kErrKeyword) { set_error(RPQ_EINVAL, "keyword id out of range (device check)"); return RPQ_EINVAL; }
  if (err & kErrOverflow) { set_error(RPQ_EINTERNAL, "a device work list overflowed"); return RPQ_EINTERNAL; }
  if (err & kErrBounds) { set_error(RPQ_EINTERNAL, "an index failed its bounds check (checked build)"); return RPQ_EINTERNAL; }
  set_error(RPQ_EINTERNAL, "device consistency check failed (flags 0x%x)", err);
  return RPQ_EINTERNAL;
}

// Levels per run launched as plain graph nodes before the WHILE node of a
// query graph: the tuning's flat_levels, or RPQ_GRAPH_LOOP=1 (none: the loop
// runs every level) / RPQ_GRAPH_LOOP=0 (all L+1: no loop).
static int flat_levels(const rpq_kg* kg, int L) {
  static int v = -2;
  if (v == -2) { const char* e = getenv("RPQ_GRAPH_LOOP"); v = (e && *e) ? (*e == '0' ? 0 : 1) : -1; }
  const int k = v == -1 ? kg->tune.flat_levels : (v == 1 ? 0 : L + 1);
  return std::min(k, L + 1);
}

// Slot parameters that follow the tuning.  Graphs captured with other values
// are dropped (kernel parameters are baked into them).
void apply_tuning(rpq_kg* kg, Slot* s) {
  const size_t n = size_t(kg->dev.n);
  const size_t div = size_t(std::max(1, kg->tune.queue_div));
  s->d.fq_limit = uint32_t(std::min<size_t>(s->d.cap, std::max<size_t>(n / div, std::min<size_t>(4096, s->d.cap))));
  s->d.fq_next_mult = uint32_t(std::max(1, kg->tune.next_queue_mult));
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

// RPQ_NO_GRAPH=1 launches every kernel directly (for launch lists and
// per-kernel profiles).  The host then waits after each Glevel to stop at the
// end of a run, so concurrent slots (batch, server) no longer overlap.
static bool use_graphs() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("RPQ_NO_GRAPH"); v = (e && *e && *e != '0') ? 0 : 1; }
  return v == 1;
}

void destroy_slot(Slot* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);            // h_res lies inside it
  if (s->lrec) cudaFree(s->lrec);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
}

// The V_C check of the marginal run (k_target) and the skipped final
// expansion it allows are on unless RPQ_NO_TARGET=1 (for comparisons).
static bool use_target() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("RPQ_NO_TARGET"); v = (e && *e == '1') ? 0 : 1; }
  return v == 1;
}

// Smallest expansion (work units) worth the V_C check (RPQ_TARGET_MIN_WORK
// overrides the default for comparisons).
static uint32_t target_min_work() {
  static long v = -1;
  if (v < 0) { const char* e = getenv("RPQ_TARGET_MIN_WORK"); v = (e && *e) ? std::max(0L, atol(e)) : (1L << 18); }
  return uint32_t(v);
}

// Device arrays of one slot: (destination, bytes) in allocation order.  With
// own_cols the slot holds all kMaxCols hit-level and recovery columns; a
// server slot holds none (its queries borrow column pages).
// Visited bytes and the three bit maps share one allocation (cleared per run
// by one memset): bytes of the visited part and of each bit map.
static void run_clear_layout(size_t n, size_t* vb, size_t* fb) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  *vb = up(((n + 3) / 4) * 4 + 16);
  *fb = up((n + 31) / 32 * 4 + 16);
}

static std::vector<std::pair<void**, size_t>> slot_arrays(const rpq_kg* kg, DevSlot& d, bool own_cols) {
  const size_t n = size_t(kg->dev.n);
  d.cap = uint32_t(std::max<size_t>(n, 1));
  d.hp = uint32_t((n + 15) / 16 * 16);
  d.tile_cap = uint32_t(uint64_t(kg->m2) / 128 + 2);
  d.tgt_cap = d.cap;
  size_t vb = 0, fb = 0;
  run_clear_layout(n, &vb, &fb);
  d.run_clear_bytes = 2 * vb + 3 * fb;         // visited bytes, seen bytes, F[0], F[1], cf
  std::vector<std::pair<void**, size_t>> v = {
      {&d.run_clear, d.run_clear_bytes},
      {(void**)&d.stopl, n + 16},
      {(void**)&d.items, sizeof(Item) * d.cap},
      {(void**)&d.imask, sizeof(uint16_t) * d.cap + 16},
      {(void**)&d.cg, sizeof(uint32_t) * d.cap},
      {(void**)&d.topk, sizeof(uint32_t) * size_t(num_sms()) * 2 * kMaxK},   // k_topk: 2 blocks per SM
      {(void**)&d.vmask, sizeof(unsigned long long) * d.cap},
      {(void**)&d.rcnt, sizeof(uint32_t) * kRecStride * kMaxCols},
      {(void**)&d.tile_first, sizeof(uint32_t) * d.tile_cap},
      {(void**)&d.fq[0], sizeof(uint32_t) * d.cap},       // any queue limit up to n fits
      {(void**)&d.fq[1], sizeof(uint32_t) * d.cap},
      {(void**)&d.ulist, sizeof(uint32_t) * d.cap},
      {(void**)&d.vcl, sizeof(uint32_t) * d.cap},
      {(void**)&d.tgt, sizeof(uint32_t) * d.tgt_cap},
      {(void**)&d.sticky, 16},
      {(void**)&d.ctl, kCtlBytes + sizeof(rpq_result) * kMaxK},   // the results follow the control block
      {(void**)&d.q, sizeof(QueryDev)},
      {(void**)&d.n_res, 16},
      {(void**)&d.bar, 16},
  };
  if (own_cols) {
    v.push_back({(void**)&d.H, size_t(d.hp) * kMaxCols + 16});
    v.push_back({(void**)&d.rmask, sizeof(unsigned long long) * d.cap * kMaxCols});
    v.push_back({(void**)&d.rlist, sizeof(uint32_t) * d.cap * kMaxCols});
  }
  return v;
}

int64_t slot_bytes(const rpq_kg* kg, bool own_cols) {
  DevSlot d{};
  int64_t t = 0;
  for (const auto& a : slot_arrays(kg, d, own_cols)) t += int64_t(a.second);
  return t;
}

// Clock cycles a block of the persistent kernel waits at a grid barrier
// before it reports RPQ_ETIMEOUT: about 1 s at 2 GHz, or RPQ_BARRIER_LIMIT
// (cycles, at least 1), which the timeout test sets small.
static long long barrier_limit() {
  static long long v = -1;
  if (v < 0) { const char* e = getenv("RPQ_BARRIER_LIMIT"); v = (e && *e) ? std::max(1LL, atoll(e)) : 2000000000LL; }
  return v;
}

int create_slot(rpq_kg* kg, Slot** out, bool own_cols) {
  Slot* s = new Slot();
  DevSlot& d = s->d;
  int rc = RPQ_OK;
  for (const auto& a : slot_arrays(kg, d, own_cols)) {
    rc = alloc_device(a.first, a.second, &s->bytes);
    if (rc != RPQ_OK) break;
    s->allocs.push_back(*a.first);
  }
  if (rc == RPQ_OK) {
    char* b = static_cast<char*>(d.run_clear);
    size_t vb = 0, fb = 0;
    run_clear_layout(size_t(kg->dev.n), &vb, &fb);
    d.vis = reinterpret_cast<uint32_t*>(b);
    d.vseen = reinterpret_cast<uint8_t*>(b + vb);
    d.F[0] = reinterpret_cast<uint32_t*>(b + 2 * vb);
    d.F[1] = reinterpret_cast<uint32_t*>(b + 2 * vb + fb);
    d.cf = reinterpret_cast<uint32_t*>(b + 2 * vb + 2 * fb);
    d.res = reinterpret_cast<char*>(d.ctl) + kCtlBytes;   // one copy returns control block and results
    // masks start at zero; the recovery kernel restores zero after each use
    if ((own_cols && cudaMemset(d.rmask, 0, sizeof(unsigned long long) * d.cap * kMaxCols) != cudaSuccess) ||
        cudaMemset(d.vmask, 0, sizeof(unsigned long long) * d.cap) != cudaSuccess ||
        cudaMemset(d.rcnt, 0, sizeof(uint32_t) * kRecStride * kMaxCols) != cudaSuccess ||
        cudaMemset(d.sticky, 0, 16) != cudaSuccess ||
        cudaMemset(d.bar, 0, 16) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_ctl, kCtlBytes + sizeof(rpq_result) * kMaxK) != cudaSuccess) {
      cudaGetLastError();
      set_error(RPQ_ENOMEM, "search slot set-up failed");
      rc = RPQ_ENOMEM;
    }
  }
  if (rc != RPQ_OK) { destroy_slot(s); return rc; }
  s->h_res = reinterpret_cast<rpq_result*>(reinterpret_cast<char*>(s->h_ctl) + kCtlBytes);
  d.qlog = nullptr;
  d.qcap = 0;
  d.target = use_target() ? 1u : 0u;
  d.tgt_min_work = target_min_work();
  d.bar_limit = barrier_limit();
  apply_tuning(kg, s);
  *out = s;
  return RPQ_OK;
}

// Slot 0 serves one query at a time (rpq_search, rpq_search_device).  With
// RPQ_PERSISTENT=1 its level loops run as one persistent cooperative kernel
// per run (grid barriers instead of kernel boundaries).  Measured on B300 it
// is not faster than kernel pairs replayed from a flat CUDA graph (fewer
// resident blocks, L2-only loads of cross-block state, two barriers per
// level), so it is off by default.  Other slots always use kernel pairs.
static bool persistent_slot0() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("RPQ_PERSISTENT"); v = (e && *e == '1') ? 1 : 0; }
  return v == 1;
}


int get_slot(rpq_kg* kg, size_t i, Slot** out) {
  while (kg->slots.size() <= i) {
    Slot* s = nullptr;
    const int rc = create_slot(kg, &s);
    if (rc != RPQ_OK) return rc;
    s->d.persistent = (kg->slots.empty() && persistent_slot0()) ? 1u : 0u;
    kg->slots.push_back(s);
    kg->device_bytes += s->bytes;
  }
  *out = kg->slots[i];
  return RPQ_OK;
}

// Host validation of a query; fills qv.  Returns RPQ_OK, or an error, and
// sets *empty when a keyword has no keyword node (no result is possible).
int check_query(const rpq_kg* kg, const rpq_query* q, QueryDev* qv, bool* empty) {
  if (!q) { set_error(RPQ_EINVAL, "query is NULL"); return RPQ_EINVAL; }
  if (q->n_c < 1 || q->n_c > kMaxCols || q->n_m < 0 || q->n_m > kMaxCols) {
    set_error(RPQ_EINVAL, "need 1 <= n_c <= %d and 0 <= n_m <= %d (got %d, %d)", kMaxCols, kMaxCols, q->n_c, q->n_m);
    return RPQ_EINVAL;
  }
  if (!q->central || (q->n_m > 0 && !q->marginal)) { set_error(RPQ_EINVAL, "keyword array is NULL"); return RPQ_EINVAL; }
  if (q->k < 1 || q->k > kMaxK) { set_error(RPQ_EINVAL, "need 1 <= k <= %d (got %d)", kMaxK, q->k); return RPQ_EINVAL; }
  if (q->max_depth < 0 || q->max_depth > kMaxLevel) {
    set_error(RPQ_EINVAL, "need 0 <= max_depth <= %d (got %d)", kMaxLevel, q->max_depth);
    return RPQ_EINVAL;
  }
  if (!(q->gamma >= 0.0 && q->gamma <= 1.0)) { set_error(RPQ_EINVAL, "need 0 <= gamma <= 1"); return RPQ_EINVAL; }
  if (q->w != 0 && (q->w < q->k || q->w > kMaxK)) {
    set_error(RPQ_EINVAL, "need w = 0 or k <= w <= %d (got k %d, w %d)", kMaxK, q->k, q->w);
    return RPQ_EINVAL;
  }
  if (q->score != RPQ_SCORE_SUM && q->score != RPQ_SCORE_PRODUCT) {
    set_error(RPQ_EINVAL, "unknown score combination %d", q->score);
    return RPQ_EINVAL;
  }
  memset(qv, 0, sizeof(*qv));
  *empty = false;
  for (int i = 0; i < q->n_c + q->n_m; ++i) {
    const int32_t kw = i < q->n_c ? q->central[i] : q->marginal[i - q->n_c];
    if (kw < 0 || kw >= kg->dev.n_kw) {
      set_error(RPQ_EINVAL, "keyword id %d out of range [0, %d)", kw, kg->dev.n_kw);
      return RPQ_EINVAL;
    }
    if (kg->kw_ptr[kw + 1] == kg->kw_ptr[kw]) *empty = true;
    qv->kw[i] = kw;
  }
  qv->n_c = q->n_c; qv->n_m = q->n_m; qv->k = q->k; qv->L = q->max_depth; qv->gamma = q->gamma;
  qv->w = q->w ? q->w : q->k;
  qv->product = q->score == RPQ_SCORE_PRODUCT;
  return RPQ_OK;
}

// Graph of one query shape.  The whole query is captured into one graph; the
// level loop of each run is its first K levels as plain nodes (a level after
// the run stopped costs an early-exit launch) followed, when K < L+1, by a
// WHILE conditional node whose body (the level kernels) repeats until
// k_expand clears the condition.  k_expand also clears it when the run stops
// inside the first K levels, so a short run never enters the loop.  On B300 a
// WHILE iteration costs more than the early-exit launches of a level, and
// most runs stop within a few levels, hence a small plain prefix.
static int build_query_graph(rpq_kg* kg, Slot* s, int n_m, int L, int K, cudaGraphExec_t* out) {
  cudaGraph_t main = nullptr;
  RPQ_CUDA(cudaGraphCreate(&main, 0));
  cudaStream_t side = nullptr;
  int rc = RPQ_OK;
  auto fail = [&](const char* what, cudaError_t e) {
    if (rc != RPQ_OK) return;
    cudaGetLastError();
    set_error(RPQ_ECUDA, "graph build (%s): %s", what, cudaGetErrorString(e));
    rc = RPQ_ECUDA;
  };
  bool capturing = false;
  auto check = [&](const char* what, cudaError_t e) { if (e != cudaSuccess) fail(what, e); return e == cudaSuccess; };
  auto add_run = [&](int run) {
    if (rc != RPQ_OK) return;
    if (K >= L + 1) {                                   // no loop: L+1 plain levels
      for (int l = 0; l <= L; ++l) launch_level(kg->dev, s->d, run, s->st, nullptr, 0, false);
      return;
    }
    cudaGraphConditionalHandle h = 0;
    if (!check("conditional handle", cudaGraphConditionalHandleCreate(&h, main, 1, cudaGraphCondAssignDefault))) return;
    for (int l = 0; l < K; ++l) launch_level(kg->dev, s->d, run, s->st, nullptr, h, true);
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if (!check("capture info", cudaStreamGetCaptureInfo(s->st, &status, nullptr, nullptr, &deps, nullptr, &ndeps))) return;
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (!check("conditional node", cudaGraphAddNode(&node, main, dv.empty() ? nullptr : dv.data(), nullptr,
                                                    dv.size(), &cp))) return;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (!side && !check("side stream", cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking))) return;
    if (!check("capture loop body", cudaStreamBeginCaptureToGraph(side, body, nullptr, nullptr, 0,
                                                                  cudaStreamCaptureModeThreadLocal))) return;
    launch_level(kg->dev, s->d, run, side, nullptr, h, true);
    cudaGraph_t got = nullptr;
    if (!check("end loop body", cudaStreamEndCapture(side, &got))) return;
    check("loop dependency", cudaStreamUpdateCaptureDependencies(s->st, &node, nullptr, 1,
                                                                  cudaStreamSetCaptureDependencies));
  };
  if (check("begin capture", cudaStreamBeginCaptureToGraph(s->st, main, nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal))) {
    capturing = true;
    launch_run_setup(kg->dev, s->d, 0, s->st, nullptr);
    add_run(0);
    launch_select_recover(kg->dev, s->d, n_m, s->st, nullptr);
    if (n_m > 0) {
      launch_run_setup(kg->dev, s->d, 1, s->st, nullptr);
      add_run(1);
    }
  }
  if (capturing) {
    cudaGraph_t got = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s->st, &got);
    if (e != cudaSuccess) fail("end capture", e);
  }
  if (side) cudaStreamDestroy(side);
  if (rc == RPQ_OK) {
    const cudaError_t e = cudaGraphInstantiate(out, main, 0);
    if (e != cudaSuccess) fail("instantiate", e);
  }
  cudaGraphDestroy(main);
  return rc;
}

// Enqueue the body of a query: replay (or build, then replay) the graph of
// its shape, or launch the kernels directly.
static int enqueue_body(rpq_kg* kg, Slot* s, int n_c, int n_m, int L) {
  if (kg->prof) {                                       // direct launches with per-level records
    RPQ_CUDA(cudaGetLastError());
    const size_t rb = sizeof(LevelRec) * 2 * kLogLevels;
    if (!s->lrec) RPQ_CUDA(cudaMalloc((void**)&s->lrec, rb));
    RPQ_CUDA(cudaMemsetAsync(s->lrec, 0, rb, s->st));
    DevSlot d = s->d;
    d.lrec = s->lrec;
    return launch_query_body(kg->dev, d, n_m, L, s->st, kg->prof, true);
  }
  if (!use_graphs()) {
    RPQ_CUDA(cudaGetLastError());
    return launch_query_body(kg->dev, s->d, n_m, L, s->st, nullptr, true);
  }
  (void)n_c;
  const int K = s->d.persistent ? L + 1 : flat_levels(kg, L);
  const uint64_t key = (uint64_t(L) << 16) | (uint64_t(K) << 8) | uint64_t(n_m > 0 ? 1 : 0);
  auto it = s->graphs.find(key);
  if (it == s->graphs.end()) {
    cudaGraphExec_t exec = nullptr;
    if (!s->d.persistent) {
      const int rc = build_query_graph(kg, s, n_m, L, K, &exec);
      if (rc != RPQ_OK) return rc;
    } else {                                            // one persistent kernel per run
      cudaGraph_t graph = nullptr;
      RPQ_CUDA(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
      const int rc = launch_query_body(kg->dev, s->d, n_m, L, s->st, nullptr, false);
      const cudaError_t ce = cudaStreamEndCapture(s->st, &graph);
      if (rc != RPQ_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        set_error(RPQ_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        return RPQ_ECUDA;
      }
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) { set_error(RPQ_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie)); return RPQ_ECUDA; }
    }
    it = s->graphs.emplace(key, exec).first;
  }
  RPQ_CUDA(cudaGraphLaunch(it->second, s->st));
  return RPQ_OK;
}

// Start a validated query on a slot (asynchronous).
int start_query(rpq_kg* kg, Slot* s, const QueryDev& qv) {
  int rc = launch_query_setup(s->d, qv, nullptr, s->st);
  if (rc != RPQ_OK) { set_error(RPQ_ECUDA, "launch failed: %s", cudaGetErrorString(cudaGetLastError())); return rc; }
  rc = enqueue_body(kg, s, qv.n_c, qv.n_m, qv.L);
  if (rc != RPQ_OK) return rc;
  RPQ_CUDA(cudaMemcpyAsync(s->h_ctl, s->d.ctl, kCtlBytes + sizeof(rpq_result) * size_t(qv.k),
                           cudaMemcpyDeviceToHost, s->st));      // control block and results
  s->busy = true;
  s->pending_k = qv.k;
  s->pending_nc = qv.n_c;
  s->pending_nm = qv.n_m;
  return RPQ_OK;
}

void fill_stats(const Ctl& c, rpq_stats* st) {
  if (!st) return;
  st->e_act_central = int64_t(c.e_act[0]);
  st->e_act_marginal = int64_t(c.e_act[1]);
  st->hits_central = int64_t(c.hits[0]);
  st->hits_marginal = int64_t(c.hits[1]);
  st->levels_central = c.levels[0];
  st->levels_marginal = c.levels[1];
  st->n_cg = int32_t(c.ncg);
  st->n_selected = int32_t(c.nsel);
  st->work_units = int64_t(c.units);
  st->work_items = int64_t(c.items);
  st->frontier_nodes = int64_t(c.frontier);
  st->e_act_skipped = int64_t(c.e_act_skip);
}

// Profiling mode: pair the level kernels' device times of the slot's
// finished query with its per-level records (the query's launches are
// complete once the slot's stream has been synchronised).
static int collect_level_profile(rpq_kg* kg, Slot* s) {
  Prof* pf = kg->prof;
  pf->collect(s->st);
  if (!s->lrec) return RPQ_OK;
  std::vector<LevelRec> rec(2 * kLogLevels);
  RPQ_CUDA(cudaMemcpy(rec.data(), s->lrec, sizeof(LevelRec) * rec.size(), cudaMemcpyDeviceToHost));
  size_t keep = 0;
  for (const Prof::LevelTimes& lt : pf->level_times) {
    if (lt.st != s->st) { pf->level_times[keep++] = lt; continue; }
    const LevelRec& r = rec[size_t(lt.run) * kLogLevels + size_t(lt.level)];
    if (!r.flags) continue;                         // a launch after the run had stopped
    rpq_level_profile p;
    memset(&p, 0, sizeof(p));
    p.run = lt.run;
    p.level = lt.level;
    p.flags = int32_t(r.flags);
    p.frontier = int32_t(r.frontier);
    p.columns = lt.run == 0 ? s->pending_nc : s->pending_nm;
    p.units = int64_t(r.units);
    p.items = int64_t(r.items);
    p.e_act = int64_t(r.eact);
    p.claims = int64_t(r.claims);
    p.enqueue_ms = lt.ms[kKindEnqueue];
    p.target_ms = lt.ms[kKindTarget];
    p.expand_ms = lt.ms[kKindExpand];
    pf->levels.push_back(p);
  }
  pf->level_times.resize(keep);
  return RPQ_OK;
}

// Wait for the slot's query and copy its results out.
int finish_query(rpq_kg* kg, Slot* s, rpq_result* out, int32_t* n_out, rpq_stats* stats) {
  s->busy = false;
  RPQ_CUDA(cudaStreamSynchronize(s->st));
  if (kg->prof) {
    const int prc = collect_level_profile(kg, s);
    if (prc != RPQ_OK) return prc;
  }
  const Ctl& c = *s->h_ctl;
  const int rc = dev_err_to_status(c.err);
  if (rc != RPQ_OK) return rc;
  const int32_t nr = int32_t(std::min<uint32_t>(c.n_res, uint32_t(s->pending_k)));
  if (out && nr) memcpy(out, s->h_res, sizeof(rpq_result) * size_t(nr));
  if (n_out) *n_out = nr;
  fill_stats(c, stats);
  if (stats) {
    const int runs = 1 + (s->pending_nm > 0 && c.levels[1] >= 0 ? 1 : 0);
    stats->kernels = kernels_fixed_per_query(s->pending_nm) +
                     (s->d.persistent ? runs : 2 * int64_t(c.iters[0]) + 3 * int64_t(c.iters[1]));
  }
  return RPQ_OK;
}

void empty_result(int32_t* n_out, rpq_stats* stats) {
  if (n_out) *n_out = 0;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->levels_central = stats->levels_marginal = -1;
  }
}

static int slot_count(const rpq_kg* kg) {
  const char* e = getenv("RPQ_SLOTS");
  if (e && atoi(e) > 0) return std::min(atoi(e), 256);
  return std::max(1, std::min(kg->tune.batch_slots, 256));
}

}  // namespace rpq

using namespace rpq;

extern "C" {

const char* rpq_strerror(int code) {
  switch (code) {
    case RPQ_OK: return "RPQ_OK";
    case RPQ_EINVAL: return "RPQ_EINVAL";
    case RPQ_ENOMEM: return "RPQ_ENOMEM";
    case RPQ_ETIMEOUT: return "RPQ_ETIMEOUT";
    case RPQ_ECUDA: return "RPQ_ECUDA";
    case RPQ_ELIMIT: return "RPQ_ELIMIT";
    case RPQ_EINTERNAL: return "RPQ_EINTERNAL";
    case RPQ_ESIZE: return "RPQ_ESIZE";
  }
  return "RPQ_E(unknown)";
}

const char* rpq_last_error(void) { return g_last_error.c_str(); }

int rpq_load_kg(const rpq_kg_desc* d, rpq_kg** out) {
  ApiRange nvtx_range("rpq_load_kg");
  if (!d || !out) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  *out = nullptr;
  if (d->n <= 0 || d->n > RPQ_MAX_NODES) { set_error(RPQ_ELIMIT, "n = %d outside (0, %d]", d->n, RPQ_MAX_NODES); return d->n <= 0 ? RPQ_EINVAL : RPQ_ELIMIT; }
  if (d->m2 < 0 || d->m2 >= (int64_t(1) << 32)) { set_error(RPQ_ELIMIT, "m2 = %lld outside [0, 2^32)", (long long)d->m2); return RPQ_ELIMIT; }
  if (!d->row_ptr || (d->m2 > 0 && (!d->col || !d->label)) || !d->kw_ptr || d->n_kw < 0) {
    set_error(RPQ_EINVAL, "missing graph array"); return RPQ_EINVAL;
  }
  if (d->n_labels < 1 || d->n_labels > RPQ_MAX_LABELS) { set_error(RPQ_ELIMIT, "n_labels = %d outside [1, %d]", d->n_labels, RPQ_MAX_LABELS); return RPQ_ELIMIT; }
  if (!(d->alpha > 0.0 && d->alpha < 1.0)) { set_error(RPQ_EINVAL, "alpha must lie in (0, 1)"); return RPQ_EINVAL; }
  if (!(d->abar > 0.0) || !(d->abar < 1e6)) { set_error(RPQ_EINVAL, "abar must be positive"); return RPQ_EINVAL; }
  if (d->row_ptr[0] != 0 || d->row_ptr[d->n] != d->m2) { set_error(RPQ_EINVAL, "row_ptr must start at 0 and end at m2"); return RPQ_EINVAL; }
  for (int64_t i = 0; i < d->n; ++i)
    if (d->row_ptr[i + 1] < d->row_ptr[i]) { set_error(RPQ_EINVAL, "row_ptr decreases at %lld", (long long)i); return RPQ_EINVAL; }
  if (d->kw_ptr[0] != 0) { set_error(RPQ_EINVAL, "kw_ptr[0] must be 0"); return RPQ_EINVAL; }
  for (int64_t i = 0; i < d->n_kw; ++i)
    if (d->kw_ptr[i + 1] < d->kw_ptr[i]) { set_error(RPQ_EINVAL, "kw_ptr decreases at %lld", (long long)i); return RPQ_EINVAL; }
  const int64_t npost = d->kw_ptr[d->n_kw];
  if (npost >= (int64_t(1) << 32)) { set_error(RPQ_ELIMIT, "too many postings"); return RPQ_ELIMIT; }
  if (npost > 0 && !d->kw_nodes) { set_error(RPQ_EINVAL, "kw_nodes is NULL"); return RPQ_EINVAL; }
  for (int64_t i = 0; i < npost; ++i)
    if (d->kw_nodes[i] < 0 || d->kw_nodes[i] >= d->n) { set_error(RPQ_EINVAL, "kw_nodes[%lld] out of range", (long long)i); return RPQ_EINVAL; }

  rpq_kg* kg = new rpq_kg();
  cudaGetDevice(&kg->device);
  kg->m2 = d->m2;
  kg->alpha = d->alpha;
  kg->abar = d->abar;
  kg->kw_ptr.assign(d->kw_ptr, d->kw_ptr + d->n_kw + 1);
  int rc = build_graph(kg, d);
  if (rc == RPQ_OK) {
    std::vector<uint32_t> kp(size_t(d->n_kw) + 1);
    for (int64_t i = 0; i <= d->n_kw; ++i) kp[i] = uint32_t(d->kw_ptr[i]);
    rc = alloc_device((void**)&kg->d_kw_ptr, sizeof(uint32_t) * kp.size(), &kg->device_bytes);
    if (rc == RPQ_OK) rc = alloc_device((void**)&kg->d_kw_nodes, sizeof(int32_t) * size_t(std::max<int64_t>(npost, 1)), &kg->device_bytes);
    std::vector<int32_t> kn(size_t(std::max<int64_t>(npost, 0)));
    for (int64_t i = 0; i < npost; ++i) kn[size_t(i)] = kg->int_of[size_t(d->kw_nodes[i])];   // internal ids
    if (rc == RPQ_OK && (cudaMemcpy(kg->d_kw_ptr, kp.data(), sizeof(uint32_t) * kp.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                         (npost > 0 && cudaMemcpy(kg->d_kw_nodes, kn.data(), sizeof(int32_t) * size_t(npost), cudaMemcpyHostToDevice) != cudaSuccess))) {
      set_error(RPQ_ECUDA, "postings upload failed");
      rc = RPQ_ECUDA;
    }
  }
  if (rc != RPQ_OK) { rpq_free_kg(kg); return rc; }
  kg->dev.n = d->n;
  kg->dev.m2 = uint32_t(d->m2);
  kg->dev.row_ptr = kg->d_row_ptr;
  kg->dev.adj = kg->d_adj;
  kg->dev.amax = kg->d_amax;
  kg->dev.lvx = kg->d_lvx;
  kg->dev.lvx_long = kg->d_lvx_long;
  kg->dev.n_kw = d->n_kw;
  kg->dev.kw_ptr = kg->d_kw_ptr;
  kg->dev.kw_nodes = kg->d_kw_nodes;
  kg->dev.ext_of = kg->d_ext_of;
  kg->dev.int_of = kg->d_int_of;
  *out = kg;
  return RPQ_OK;
}

int rpq_free_kg(rpq_kg* kg) {
  ApiRange nvtx_range("rpq_free_kg");
  if (!kg) return RPQ_OK;
  for (Slot* s : kg->slots) destroy_slot(s);
  free_subgraph_scratch(kg);
  delete kg->prof;
  cudaFree(kg->d_row_ptr); cudaFree(kg->d_adj); cudaFree(kg->d_amax); cudaFree(kg->d_lvx); cudaFree(kg->d_lvx_long);
  cudaFree(kg->d_kw_ptr); cudaFree(kg->d_kw_nodes); cudaFree(kg->d_ext_of); cudaFree(kg->d_int_of);
  delete kg;
  return RPQ_OK;
}

int rpq_kg_export(const rpq_kg* kg, uint32_t* adj, uint8_t* amax) {
  if (!kg) { set_error(RPQ_EINVAL, "NULL graph"); return RPQ_EINVAL; }
  return export_graph(kg, adj, amax);
}

int rpq_kg_info(const rpq_kg* kg, int32_t* n, int64_t* m2, int64_t* device_bytes) {
  if (!kg) { set_error(RPQ_EINVAL, "NULL graph"); return RPQ_EINVAL; }
  if (n) *n = kg->dev.n;
  if (m2) *m2 = kg->m2;
  if (device_bytes) *device_bytes = kg->device_bytes;
  return RPQ_OK;
}

int rpq_search(rpq_kg* kg, const rpq_query* q, rpq_result* out, int32_t* n_out, rpq_stats* stats) {
  ApiRange nvtx_range("rpq_search");
  if (!kg || !out || !n_out) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  QueryDev qv;
  bool empty = false;
  int rc = check_query(kg, q, &qv, &empty);
  if (rc != RPQ_OK) return rc;
  if (empty) { empty_result(n_out, stats); return RPQ_OK; }
  Slot* s = nullptr;
  rc = get_slot(kg, 0, &s);
  if (rc != RPQ_OK) return rc;
  rc = start_query(kg, s, qv);
  if (rc != RPQ_OK) { s->busy = false; cudaStreamSynchronize(s->st); return rc; }
  return finish_query(kg, s, out, n_out, stats);
}

int rpq_search_batch(rpq_kg* kg, const rpq_query* qs, int32_t nq, rpq_result* out, int32_t* n_out,
                     int32_t* status, rpq_stats* stats) {
  ApiRange nvtx_range("rpq_search_batch");
  if (!kg || (nq > 0 && (!qs || !out || !n_out || !status))) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  if (nq < 0) { set_error(RPQ_EINVAL, "nq < 0"); return RPQ_EINVAL; }
  int nslots = std::max(1, std::min<int>(slot_count(kg), nq));
  std::vector<Slot*> slots(size_t(nslots), nullptr);
  for (int i = 0; i < nslots; ++i) {          // slots 1..nslots: slot 0 serves single searches
    const int rc = get_slot(kg, size_t(i) + 1, &slots[size_t(i)]);
    if (rc == RPQ_ENOMEM && i > 0) {          // device memory for fewer slots only: use those
      nslots = i;
      slots.resize(size_t(i));
      break;
    }
    if (rc != RPQ_OK) return rc;
  }
  std::vector<int64_t> base(size_t(nq) + 1, 0);
  for (int32_t i = 0; i < nq; ++i) base[size_t(i) + 1] = base[size_t(i)] + std::max(qs[i].k, 0);
  std::vector<int32_t> owner(size_t(nslots), -1);   // query running on each slot
  auto collect = [&](int si) {
    const int32_t qi = owner[size_t(si)];
    if (qi < 0) return;
    status[qi] = finish_query(kg, slots[size_t(si)], out + base[size_t(qi)], &n_out[qi], stats ? &stats[qi] : nullptr);
    if (status[qi] != RPQ_OK) n_out[qi] = 0;
    owner[size_t(si)] = -1;
  };
  for (int32_t i = 0; i < nq; ++i) {
    QueryDev qv;
    bool empty = false;
    n_out[i] = 0;
    status[i] = check_query(kg, &qs[i], &qv, &empty);
    if (status[i] != RPQ_OK) continue;
    if (empty) { empty_result(&n_out[i], stats ? &stats[i] : nullptr); continue; }
    const int si = int(i % nslots);
    collect(si);
    status[i] = start_query(kg, slots[size_t(si)], qv);
    if (status[i] == RPQ_OK) owner[size_t(si)] = i;
  }
  for (int si = 0; si < nslots; ++si) collect(si);
  return RPQ_OK;
}

int rpq_search_batch_persistent(rpq_kg* kg, const rpq_query* qs, int32_t nq, rpq_result* out, int32_t* n_out,
                                int32_t* status, rpq_stats* stats) {
  ApiRange nvtx_range("rpq_search_batch_persistent");
  if (!kg || (nq > 0 && (!qs || !out || !n_out || !status))) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  if (nq < 0) { set_error(RPQ_EINVAL, "nq < 0"); return RPQ_EINVAL; }
  std::vector<int64_t> base(size_t(nq) + 1, 0);
  for (int32_t i = 0; i < nq; ++i) base[size_t(i) + 1] = base[size_t(i)] + std::max(qs[i].k, 0);
  std::vector<QueryDev> recs;
  std::vector<int32_t> idx;                   // batch record -> caller's query
  for (int32_t i = 0; i < nq; ++i) {
    QueryDev qv;
    bool empty = false;
    n_out[i] = 0;
    status[i] = check_query(kg, &qs[i], &qv, &empty);
    if (status[i] != RPQ_OK) continue;
    if (empty) { empty_result(&n_out[i], stats ? &stats[i] : nullptr); continue; }
    recs.push_back(qv);
    idx.push_back(i);
  }
  const int nv = int(recs.size());
  if (nv == 0) return RPQ_OK;
  int nslots = std::max(1, std::min({slot_count(kg), nv, kBatchMaxSlots}));
  std::vector<Slot*> slots(size_t(nslots), nullptr);
  for (int i = 0; i < nslots; ++i) {          // the slots of rpq_search_batch (slot 0 serves single searches)
    const int rc = get_slot(kg, size_t(i) + 1, &slots[size_t(i)]);
    if (rc == RPQ_ENOMEM && i > 0) { nslots = i; slots.resize(size_t(i)); break; }
    if (rc != RPQ_OK) return rc;
  }
  std::vector<DevSlot> ds(static_cast<size_t>(nslots));
  for (int i = 0; i < nslots; ++i) {
    ds[size_t(i)] = slots[size_t(i)]->d;
    ds[size_t(i)].lrec = nullptr;               // no per-level records in a persistent batch
    ds[size_t(i)].qlog = nullptr;
  }
  QueryDev* d_q = nullptr;
  uint8_t* d_out = nullptr;
  void* d_state = nullptr;
  auto release = [&]() { cudaFree(d_q); cudaFree(d_out); cudaFree(d_state); };
  int rc = alloc_device((void**)&d_q, sizeof(QueryDev) * size_t(nv), nullptr);
  if (rc == RPQ_OK) rc = alloc_device((void**)&d_out, kBatchRecBytes * size_t(nv), nullptr);
  if (rc == RPQ_OK) rc = alloc_device((void**)&d_state, batch_state_bytes(nslots), nullptr);
  if (rc != RPQ_OK) { release(); return rc; }
  cudaStream_t st = slots[0]->st;
  std::vector<uint8_t> h_out(kBatchRecBytes * size_t(nv));
  BatchCtl bc{};
  if (cudaMemcpyAsync(d_q, recs.data(), sizeof(QueryDev) * size_t(nv), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(d_out, 0, kBatchRecBytes * size_t(nv), st) != cudaSuccess) {
    release();
    set_error(RPQ_ECUDA, "batch upload failed");
    return RPQ_ECUDA;
  }
  rc = launch_batch(kg->dev, ds.data(), nslots, d_q, nv, d_out, d_state, barrier_limit(), st);
  if (rc != RPQ_OK) {
    release();
    set_error(RPQ_ECUDA, "batch launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return RPQ_ECUDA;
  }
  const cudaError_t ce = cudaStreamSynchronize(st);
  if (ce == cudaSuccess &&
      (cudaMemcpy(h_out.data(), d_out, h_out.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
       cudaMemcpy(&bc, static_cast<char*>(d_state) + sizeof(BatchSlotState) * size_t(nslots), sizeof(bc),
                  cudaMemcpyDeviceToHost) != cudaSuccess)) {
    release();
    set_error(RPQ_ECUDA, "batch download failed");
    return RPQ_ECUDA;
  }
  release();
  if (ce != cudaSuccess) { set_error(RPQ_ECUDA, "persistent batch: %s", cudaGetErrorString(ce)); return RPQ_ECUDA; }
  if (bc.err) {
    // the watchdog ended the kernel: queries in flight left recovery state
    // behind, which must be zero when a query starts
    for (Slot* s : slots) {
      cudaMemset(s->d.rcnt, 0, sizeof(uint32_t) * kRecStride * kMaxCols);
      cudaMemset(s->d.vmask, 0, sizeof(unsigned long long) * s->d.cap);
      cudaMemset(s->d.rmask, 0, sizeof(unsigned long long) * s->d.cap * kMaxCols);
    }
  }
  for (int r = 0; r < nv; ++r) {
    const int32_t i = idx[size_t(r)];
    const uint8_t* rec = h_out.data() + kBatchRecBytes * size_t(r);
    uint32_t flag = 0;
    memcpy(&flag, rec, sizeof(flag));
    if (flag != 1u) {                           // not finished when the watchdog ended the kernel
      status[i] = RPQ_ETIMEOUT;
      set_error(RPQ_ETIMEOUT, "persistent batch: no phase finished within the watchdog limit");
      continue;
    }
    Ctl c;
    memcpy(&c, rec + kBatchRecHead, sizeof(Ctl));
    status[i] = dev_err_to_status(c.err);
    if (status[i] != RPQ_OK) continue;
    const int32_t nr = int32_t(std::min<uint32_t>(c.n_res, uint32_t(qs[i].k)));
    if (nr) memcpy(out + base[size_t(i)], rec + kBatchRecHead + kCtlBytes, sizeof(rpq_result) * size_t(nr));
    n_out[i] = nr;
    if (stats) {
      fill_stats(c, &stats[i]);
      stats[i].kernels = 0;                     // the whole batch is one launch
    }
  }
  return bc.err ? RPQ_ETIMEOUT : RPQ_OK;
}

int rpq_trace(rpq_kg* kg, const rpq_query* q, rpq_result* out, int32_t* n_out, rpq_stats* stats, rpq_trace_buf* tr) {
  ApiRange nvtx_range("rpq_trace");
  if (!kg || !out || !n_out || !tr) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  QueryDev qv;
  bool empty = false;
  int rc = check_query(kg, q, &qv, &empty);
  if (rc != RPQ_OK) return rc;
  tr->n_cgs = 0; tr->n_vc = 0; tr->n_selected = 0; tr->frontier_c_levels = 0; tr->frontier_m_levels = 0;
  if (empty) { empty_result(n_out, stats); return RPQ_OK; }
  Slot* s = nullptr;
  rc = get_slot(kg, 0, &s);
  if (rc != RPQ_OK) return rc;
  const size_t n = size_t(kg->dev.n);
  const size_t qcap = std::min<size_t>(n * size_t(qv.L + 1), size_t(1) << 28);
  uint32_t* d_qlog = nullptr;
  rc = alloc_device((void**)&d_qlog, sizeof(uint32_t) * qcap, nullptr);
  if (rc != RPQ_OK) return rc;
  DevSlot d = s->d;
  d.qlog = d_qlog;
  d.qcap = uint32_t(qcap);
  d.target = 0;            // every level expanded in full: the frontiers are part of the trace
  std::vector<uint8_t> H(size_t(s->d.hp) * kMaxCols), vis(((n + 3) / 4) * 4);
  std::vector<uint32_t> qlog;
  Ctl c{};
  auto frontiers = [&](uint32_t from, uint32_t to, int64_t* ptr, int32_t* dst, int64_t cap, int32_t* levels) {
    std::vector<uint32_t> e(qlog.begin() + from, qlog.begin() + to);
    for (uint32_t& x : e) x = (x & ~kNodeMask) | uint32_t(kg->ext_of[x & kNodeMask]);   // caller ids
    std::sort(e.begin(), e.end());   // by level, then node
    int maxl = -1;
    for (uint32_t x : e) maxl = std::max<int>(maxl, int(x >> kNodeBits));
    *levels = maxl + 1;
    if (ptr) {
      size_t p = 0;
      for (int l = 0; l <= kMaxLevel + 1; ++l) {
        ptr[l] = int64_t(p);
        while (p < e.size() && int(e[p] >> kNodeBits) == l) {
          if (dst && int64_t(p) < cap) dst[p] = int32_t(e[p] & kNodeMask);
          ++p;
        }
      }
    }
  };
  auto hmat = [&](uint8_t* dst, int nt) {
    if (!dst) return;
    for (size_t v = 0; v < n; ++v) {
      const size_t u = size_t(kg->ext_of[v]);   // row of the caller's node
      for (int j = 0; j < nt; ++j)
        dst[u * size_t(nt) + size_t(j)] = ((vis[v] >> j) & 1) ? H[size_t(j) * d.hp + v] : kInf;
    }
  };
  auto fail = [&](int code) { cudaFree(d_qlog); return code; };
#define TC(call) do { const cudaError_t e_ = (call); if (e_ != cudaSuccess) { set_error(RPQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); return fail(RPQ_ECUDA); } } while (0)
  if (launch_query_setup(d, qv, nullptr, s->st) != RPQ_OK) return fail(RPQ_ECUDA);
  if (launch_central_part(kg->dev, d, qv.L, s->st, nullptr) != RPQ_OK) return fail(RPQ_ECUDA);
  TC(cudaStreamSynchronize(s->st));
  TC(cudaMemcpy(&c, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  TC(cudaMemcpy(H.data(), d.H, H.size(), cudaMemcpyDeviceToHost));
  TC(cudaMemcpy(vis.data(), d.vis, n, cudaMemcpyDeviceToHost));
  const uint32_t nqc = std::min<uint32_t>(c.qlog_n, uint32_t(qcap));
  qlog.resize(nqc);
  if (nqc) TC(cudaMemcpy(qlog.data(), d_qlog, sizeof(uint32_t) * nqc, cudaMemcpyDeviceToHost));
  hmat(tr->h_central, qv.n_c);
  frontiers(0, nqc, tr->frontier_c_ptr, tr->frontier_c, tr->frontier_c_cap, &tr->frontier_c_levels);
  {
    std::vector<uint32_t> cg(c.ncg);
    if (c.ncg) TC(cudaMemcpy(cg.data(), d.cg, sizeof(uint32_t) * c.ncg, cudaMemcpyDeviceToHost));
    std::vector<int64_t> cgs;
    for (uint32_t x : cg) cgs.push_back((int64_t(x & kNodeMask) << 8) | int64_t(x >> kNodeBits));
    std::sort(cgs.begin(), cgs.end());
    tr->n_cgs = int64_t(cgs.size());
    if (tr->cgs) for (size_t i = 0; i < cgs.size() && int64_t(i) < tr->cg_cap; ++i) tr->cgs[i] = cgs[i];
    tr->n_selected = int32_t(c.nsel);
    for (uint32_t i = 0; i < c.nsel; ++i) tr->selected[i] = c.sel[i];
  }
  if (launch_marginal_part(kg->dev, d, qv.n_m, qv.L, s->st, nullptr) != RPQ_OK) return fail(RPQ_ECUDA);
  TC(cudaStreamSynchronize(s->st));
  TC(cudaMemcpy(&c, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  {
    std::vector<uint32_t> vcl(std::min<uint32_t>(c.nvc, d.cap));
    if (!vcl.empty()) TC(cudaMemcpy(vcl.data(), d.vcl, sizeof(uint32_t) * vcl.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> vc;
    for (uint32_t x : vcl) vc.push_back(int64_t((x & ~kNodeMask) | uint32_t(kg->ext_of[x & kNodeMask])));
    std::sort(vc.begin(), vc.end());
    tr->n_vc = int64_t(vc.size());
    if (tr->vc) for (size_t i = 0; i < vc.size() && int64_t(i) < tr->vc_cap; ++i) tr->vc[i] = vc[i];
  }
  if (qv.n_m > 0 && c.levels[1] >= 0) {
    TC(cudaMemcpy(H.data(), d.H, H.size(), cudaMemcpyDeviceToHost));
    TC(cudaMemcpy(vis.data(), d.vis, n, cudaMemcpyDeviceToHost));
    hmat(tr->h_marginal, qv.n_m);
    const uint32_t nqa = std::min<uint32_t>(c.qlog_n, uint32_t(qcap));
    qlog.resize(nqa);
    if (nqa > nqc) TC(cudaMemcpy(qlog.data() + nqc, d_qlog + nqc, sizeof(uint32_t) * (nqa - nqc), cudaMemcpyDeviceToHost));
    frontiers(nqc, nqa, tr->frontier_m_ptr, tr->frontier_m, tr->frontier_m_cap, &tr->frontier_m_levels);
  }
  rpq_result res[kMaxK];
  TC(cudaMemcpy(res, d.res, sizeof(rpq_result) * size_t(qv.k), cudaMemcpyDeviceToHost));
#undef TC
  cudaFree(d_qlog);
  rc = dev_err_to_status(c.err);
  if (c.qlog_n > qcap) { set_error(RPQ_ELIMIT, "trace frontier log overflow"); rc = RPQ_ELIMIT; }
  if (rc != RPQ_OK) return rc;
  const int32_t nr = int32_t(std::min<uint32_t>(c.n_res, uint32_t(qv.k)));
  memcpy(out, res, sizeof(rpq_result) * size_t(nr));
  *n_out = nr;
  fill_stats(c, stats);
  return RPQ_OK;
}

int rpq_search_device(rpq_kg* kg, const int32_t* d_keywords, int32_t n_c, int32_t n_m, int32_t k, int32_t max_depth,
                      double gamma, rpq_result* d_out, int32_t* d_n_out) {
  ApiRange nvtx_range("rpq_search_device");
  if (!kg || !d_keywords || !d_out || !d_n_out) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  if (n_c < 1 || n_c > kMaxCols || n_m < 0 || n_m > kMaxCols || k < 1 || k > kMaxK || max_depth < 0 ||
      max_depth > kMaxLevel || !(gamma >= 0.0 && gamma <= 1.0)) {
    set_error(RPQ_EINVAL, "query parameter out of range");
    return RPQ_EINVAL;
  }
  Slot* s = nullptr;
  int rc = get_slot(kg, 0, &s);
  if (rc != RPQ_OK) return rc;
  QueryDev qv;
  memset(&qv, 0, sizeof(qv));
  qv.n_c = n_c; qv.n_m = n_m; qv.k = k; qv.L = max_depth; qv.gamma = gamma; qv.w = k;
  rc = launch_query_setup(s->d, qv, d_keywords, s->st);
  if (rc != RPQ_OK) { set_error(RPQ_ECUDA, "launch failed"); return rc; }
  rc = enqueue_body(kg, s, n_c, n_m, max_depth);
  if (rc != RPQ_OK) return rc;
  RPQ_CUDA(cudaMemcpyAsync(d_out, s->d.res, sizeof(rpq_result) * size_t(k), cudaMemcpyDeviceToDevice, s->st));
  RPQ_CUDA(cudaMemcpyAsync(d_n_out, s->d.n_res, sizeof(int32_t), cudaMemcpyDeviceToDevice, s->st));
  return RPQ_OK;
}

int rpq_get_tuning(const rpq_kg* kg, rpq_tuning* out) {
  if (!kg || !out) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  *out = kg->tune;
  return RPQ_OK;
}

int rpq_set_tuning(rpq_kg* kg, const rpq_tuning* t) {
  if (!kg || !t) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  if (t->queue_div < 1 || t->next_queue_mult < 1 || t->batch_slots < 1 || t->flat_levels < 0) {
    set_error(RPQ_EINVAL, "tuning values must be positive");
    return RPQ_EINVAL;
  }
  for (Slot* s : kg->slots) RPQ_CUDA(cudaStreamSynchronize(s->st));
  kg->tune = *t;
  for (Slot* s : kg->slots) apply_tuning(kg, s);
  return RPQ_OK;
}

int rpq_autotune(rpq_kg* kg, const rpq_query* qs, int32_t nq, int32_t repeats, rpq_tuning* best) {
  ApiRange nvtx_range("rpq_autotune");
  if (!kg || !qs || nq < 1 || repeats < 1) { set_error(RPQ_EINVAL, "bad argument"); return RPQ_EINVAL; }
  using Clock = std::chrono::steady_clock;
  std::vector<rpq_result> out(size_t(RPQ_MAX_K) * size_t(nq));
  std::vector<int32_t> n_out(static_cast<size_t>(nq)), status(static_cast<size_t>(nq));
  int rc = RPQ_OK;
  auto median = [](std::vector<double> v) { std::sort(v.begin(), v.end()); return v[v.size() / 2]; };
  auto time_single = [&](double* sec) -> int {
    std::vector<double> t;
    for (int pass = 0; pass <= repeats; ++pass) {
      const auto t0 = Clock::now();
      for (int32_t i = 0; i < nq; ++i) {
        int32_t nr = 0;
        const int r = rpq_search(kg, &qs[i], out.data(), &nr, nullptr);
        if (r != RPQ_OK && r != RPQ_EINVAL) return r;
      }
      if (pass > 0) t.push_back(std::chrono::duration<double>(Clock::now() - t0).count());
    }
    *sec = median(t);
    return RPQ_OK;
  };
  auto time_batch = [&](double* sec) -> int {
    std::vector<double> t;
    for (int pass = 0; pass <= repeats; ++pass) {
      const auto t0 = Clock::now();
      const int r = rpq_search_batch(kg, qs, nq, out.data(), n_out.data(), status.data(), nullptr);
      if (r != RPQ_OK) return r;
      if (pass > 0) t.push_back(std::chrono::duration<double>(Clock::now() - t0).count());
    }
    *sec = median(t);
    return RPQ_OK;
  };
  // one-at-a-time needs at most k records per query
  for (int32_t i = 0; i < nq; ++i)
    if (qs[i].k > RPQ_MAX_K) { set_error(RPQ_EINVAL, "k above RPQ_MAX_K"); return RPQ_EINVAL; }
  rpq_tuning cur = kg->tune, bestt = kg->tune;
  double best_s = 1e30;
  for (int qd : {8, 32, 128}) {
    for (int nm : {4, 16, 64}) {
      cur.queue_div = qd;
      cur.next_queue_mult = nm;
      if ((rc = rpq_set_tuning(kg, &cur)) != RPQ_OK) return rc;
      double sec = 0;
      if ((rc = time_single(&sec)) != RPQ_OK) return rc;
      if (sec < best_s) { best_s = sec; bestt = cur; }
    }
  }
  cur = bestt;
  for (int fl : {2, 3, 4, 6, 64}) {
    cur.flat_levels = fl;
    if ((rc = rpq_set_tuning(kg, &cur)) != RPQ_OK) return rc;
    double sec = 0;
    if ((rc = time_single(&sec)) != RPQ_OK) return rc;
    if (sec < best_s) { best_s = sec; bestt.flat_levels = fl; }
  }
  cur = bestt;
  best_s = 1e30;
  for (int bs : {4, 8, 16, 32}) {
    cur.batch_slots = bs;
    if ((rc = rpq_set_tuning(kg, &cur)) != RPQ_OK) return rc;
    double sec = 0;
    if ((rc = time_batch(&sec)) != RPQ_OK) return rc;
    if (sec < best_s) { best_s = sec; bestt.batch_slots = bs; }
  }
  if ((rc = rpq_set_tuning(kg, &bestt)) != RPQ_OK) return rc;
  if (best) *best = bestt;
  return RPQ_OK;
}

int rpq_slot_stream(rpq_kg* kg, int32_t slot, void** stream) {
  if (!kg || !stream || slot < 0 || slot > 255) { set_error(RPQ_EINVAL, "bad argument"); return RPQ_EINVAL; }
  Slot* s = nullptr;
  const int rc = get_slot(kg, size_t(slot), &s);
  if (rc != RPQ_OK) return rc;
  *stream = s->st;
  return RPQ_OK;
}

int rpq_set_profiling(rpq_kg* kg, int32_t enable) {
  if (!kg) { set_error(RPQ_EINVAL, "NULL graph"); return RPQ_EINVAL; }
  for (Slot* s : kg->slots) cudaStreamSynchronize(s->st);
  if (enable && !kg->prof) kg->prof = new Prof();
  if (!enable && kg->prof) { kg->prof->collect(); delete kg->prof; kg->prof = nullptr; }
  return RPQ_OK;
}

int rpq_profile_read(rpq_kg* kg, rpq_profile* out, int32_t reset) {
  if (!kg || !out) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  memset(out, 0, sizeof(*out));
  if (!kg->prof) return RPQ_OK;
  for (Slot* s : kg->slots) cudaStreamSynchronize(s->st);
  kg->prof->collect();
  for (int i = 0; i < RPQ_PROF_CLASSES; ++i) { out->ms[i] = kg->prof->ms[i]; out->launches[i] = kg->prof->launches[i]; }
  if (reset) {
    for (int i = 0; i < RPQ_PROF_CLASSES; ++i) { kg->prof->ms[i] = 0; kg->prof->launches[i] = 0; }
  }
  return RPQ_OK;
}

int rpq_profile_levels(rpq_kg* kg, rpq_level_profile* out, int32_t cap, int32_t* n_out, int32_t reset) {
  if (!kg || !n_out || cap < 0 || (cap > 0 && !out)) { set_error(RPQ_EINVAL, "bad argument"); return RPQ_EINVAL; }
  *n_out = 0;
  if (!kg->prof) return RPQ_OK;
  const std::vector<rpq_level_profile>& v = kg->prof->levels;
  const size_t n = std::min(v.size(), size_t(cap));
  if (n) memcpy(out, v.data(), sizeof(rpq_level_profile) * n);
  *n_out = int32_t(v.size());
  if (reset) kg->prof->levels.clear();
  return RPQ_OK;
}

int rpq_transfer_bytes(int32_t k, int64_t* h2d, int64_t* d2h) {
  if (k < 1 || k > kMaxK) { set_error(RPQ_EINVAL, "need 1 <= k <= %d", kMaxK); return RPQ_EINVAL; }
  if (h2d) *h2d = int64_t(sizeof(QueryDev));
  if (d2h) *d2h = int64_t(kCtlBytes + sizeof(rpq_result) * size_t(k));
  return RPQ_OK;
}

int rpq_sync_device(rpq_kg* kg) {
  ApiRange nvtx_range("rpq_sync_device");
  if (!kg) { set_error(RPQ_EINVAL, "NULL graph"); return RPQ_EINVAL; }
  if (kg->slots.empty()) return RPQ_OK;
  Slot* s = kg->slots[0];
  RPQ_CUDA(cudaStreamSynchronize(s->st));
  uint32_t err = 0;
  RPQ_CUDA(cudaMemcpy(&err, s->d.sticky, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (err) RPQ_CUDA(cudaMemset(s->d.sticky, 0, sizeof(uint32_t)));
  return dev_err_to_status(err);
}

}  // extern "C"
