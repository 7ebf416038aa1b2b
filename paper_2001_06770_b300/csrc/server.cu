// Serving loop of librpq: continuous batching of radial-pattern queries.
//
// A server owns search slots and two pools of column pages.  A slot holds the
// per-query state that does not depend on the keywords (visited bytes,
// frontier bit maps, work lists, about 45 bytes per graph node) and its own
// CUDA stream; a query's keyword columns are pages lent to it while it runs:
// max(|C|, |M|) pages of the Node-Keyword Matrix (one byte per node each) and
// |C| recovery pages (a CG mask and a list entry per node, 12 bytes per node
// each).  So a query is admitted by the memory its own hit table needs: it
// starts when a slot and its pages are free; otherwise it waits in a FIFO.
// Every submit and poll call collects finished queries (CUDA event per slot,
// no blocking), returns their pages and admits waiting queries, so queries
// that arrive while others run are overlapped on the device with them.  Each
// query runs exactly the same kernels as rpq_search, so its result is the
// same alone or in the mix.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "rpq_host.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  rpq::QueryDev qv;
  uint64_t tag;
  Clock::time_point t_submit;
  bool empty;  // a keyword without keyword nodes: no device work
};

}  // namespace

struct rpq_server {
  rpq_kg* kg = nullptr;
  std::vector<rpq::Slot*> slots;
  std::vector<cudaEvent_t> done_ev;
  std::vector<Pending> running;      // per slot
  std::vector<bool> busy;
  std::vector<std::vector<int32_t>> held_h, held_r;   // pages lent to each slot's query
  std::deque<Pending> waiting;
  std::deque<rpq_completion> finished;
  uint8_t* hpool = nullptr;          // h_pages pages of hp bytes (Node-Keyword Matrix columns)
  char* rpool = nullptr;             // r_pages pages: CG masks (8 * cap bytes) then node list (4 * cap)
  int32_t h_pages = 0, r_pages = 0;
  int64_t h_page_bytes = 0, r_page_bytes = 0, slot_fixed_bytes = 0;
  std::vector<int32_t> h_free, r_free;
  int32_t peak_running = 0;
  int64_t submitted = 0, completed = 0;
  int64_t starts = 0;                // queries started (or tried)
  int64_t fail_start_at = 0;         // host-side fault injection: start number k fails (0: never)
};

namespace rpq {

static double seconds(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

// Keyword columns a query occupies: Node-Keyword Matrix pages (both runs
// reuse them) and central recovery pages.
static int h_cols(const QueryDev& q) { return std::max(q.n_c, q.n_m); }

static int release_pages(rpq_server* sv, size_t i, bool failed);

// Start waiting queries (in arrival order) while a slot and the head
// query's pages are free.
static int admit(rpq_server* sv) {
  size_t i = 0;
  while (!sv->waiting.empty()) {
    Pending& p = sv->waiting.front();
    if (p.empty) {                                    // completes without device work
      rpq_completion c;
      memset(&c, 0, sizeof(c));
      c.tag = p.tag;
      c.status = RPQ_OK;
      empty_result(&c.n_res, &c.stats);
      c.latency_s = seconds(p.t_submit, Clock::now());
      sv->finished.push_back(c);
      ++sv->completed;
      sv->waiting.pop_front();
      continue;
    }
    while (i < sv->slots.size() && sv->busy[i]) ++i;
    if (i == sv->slots.size()) break;                 // every slot is busy
    const int nh = h_cols(p.qv), nr = p.qv.n_c;
    if (int(sv->h_free.size()) < nh || int(sv->r_free.size()) < nr) break;   // its pages are in use
    for (int j = 0; j < nh; ++j) {
      const int32_t pg = sv->h_free.back();
      sv->h_free.pop_back();
      sv->held_h[i].push_back(pg);
      p.qv.hc[j] = sv->hpool + size_t(pg) * size_t(sv->h_page_bytes);
    }
    for (int j = 0; j < nr; ++j) {
      const int32_t pg = sv->r_free.back();
      sv->r_free.pop_back();
      sv->held_r[i].push_back(pg);
      char* base = sv->rpool + size_t(pg) * size_t(sv->r_page_bytes);
      p.qv.rm[j] = reinterpret_cast<unsigned long long*>(base);
      p.qv.rl[j] = reinterpret_cast<uint32_t*>(base + sizeof(unsigned long long) * sv->slots[i]->d.cap);
    }
    int rc;
    if (++sv->starts == sv->fail_start_at) {         // injected on the host, before any launch
      set_error(RPQ_EINTERNAL, "injected failure of query start %lld", (long long)sv->starts);
      rc = RPQ_EINTERNAL;
    } else {
      rc = start_query(sv->kg, sv->slots[i], p.qv);
    }
    if (rc == RPQ_OK) {
      const cudaError_t e = cudaEventRecord(sv->done_ev[i], sv->slots[i]->st);
      if (e != cudaSuccess) { set_error(RPQ_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e)); rc = RPQ_ECUDA; }
    }
    if (rc != RPQ_OK) {
      // The query could not be started: it completes with its error as its
      // status, the slot's pages go back once whatever it launched has
      // finished, and the queries behind it are admitted as usual.
      sv->slots[i]->busy = false;
      rpq_completion c;
      memset(&c, 0, sizeof(c));
      c.tag = p.tag;
      c.status = rc;
      c.latency_s = seconds(p.t_submit, Clock::now());
      sv->finished.push_back(c);
      ++sv->completed;
      sv->waiting.pop_front();
      release_pages(sv, i, true);
      continue;
    }
    sv->running[i] = p;
    sv->busy[i] = true;
    sv->waiting.pop_front();
    int32_t r = 0;
    for (bool b : sv->busy) r += b;
    sv->peak_running = std::max(sv->peak_running, r);
  }
  return RPQ_OK;
}

// Return the pages of slot i's finished query.  Recovery pages come back with
// their CG masks at zero (the recovery clears every mask it set); after a
// failed query they are cleared here.
static int release_pages(rpq_server* sv, size_t i, bool failed) {
  int rc = RPQ_OK;
  if (failed) {
    for (int32_t pg : sv->held_r[i]) {
      const cudaError_t e = cudaMemsetAsync(sv->rpool + size_t(pg) * size_t(sv->r_page_bytes), 0,
                                            sizeof(unsigned long long) * sv->slots[i]->d.cap, sv->slots[i]->st);
      if (e != cudaSuccess && rc == RPQ_OK) { set_error(RPQ_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)); rc = RPQ_ECUDA; }
    }
    const cudaError_t e = cudaStreamSynchronize(sv->slots[i]->st);
    if (e != cudaSuccess && rc == RPQ_OK) { set_error(RPQ_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e)); rc = RPQ_ECUDA; }
  }
  // the pages go back to the pools in any case (after a failed clear the
  // device is unusable for the queries that would take them anyway)
  sv->h_free.insert(sv->h_free.end(), sv->held_h[i].begin(), sv->held_h[i].end());
  sv->r_free.insert(sv->r_free.end(), sv->held_r[i].begin(), sv->held_r[i].end());
  sv->held_h[i].clear();
  sv->held_r[i].clear();
  return rc;
}

// Collect finished queries; with `block`, wait for at least one if any runs.
static int collect(rpq_server* sv, bool block) {
  bool any = false;
  for (;;) {
    for (size_t i = 0; i < sv->slots.size(); ++i) {
      if (!sv->busy[i]) continue;
      const cudaError_t q = cudaEventQuery(sv->done_ev[i]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) { set_error(RPQ_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(q)); return RPQ_ECUDA; }
      rpq_completion c;
      memset(&c, 0, sizeof(c));
      c.tag = sv->running[i].tag;
      c.status = finish_query(sv->kg, sv->slots[i], c.res, &c.n_res, &c.stats);
      c.latency_s = seconds(sv->running[i].t_submit, Clock::now());
      const int prc = release_pages(sv, i, c.status != RPQ_OK);
      if (prc != RPQ_OK) return prc;
      sv->busy[i] = false;
      sv->finished.push_back(c);
      ++sv->completed;
      any = true;
    }
    if (any || !block) return RPQ_OK;
    bool running = false;
    for (size_t i = 0; i < sv->slots.size(); ++i) running |= sv->busy[i];
    if (!running) return RPQ_OK;
    std::this_thread::yield();
  }
}

}  // namespace rpq

using namespace rpq;

extern "C" {

// Slots and column pages a server holds: slots alone may not hold all
// columns of every query at once, so the budget is split for queries of
// about 4 central keywords and 6 Node-Keyword Matrix columns on average: each
// slot comes with 6 matrix pages and the rest of the budget buys recovery
// pages (at least kMaxCols of each kind, so that every query fits).
static void size_server(const rpq_kg* kg, int64_t budget, int32_t max_slots, int32_t* slots, int32_t* h_pages,
                        int32_t* r_pages) {
  const int64_t f = slot_bytes(kg, false);
  const int64_t h = int64_t((size_t(kg->dev.n) + 15) / 16 * 16);
  const int64_t r = (12 * int64_t(std::max<int32_t>(kg->dev.n, 1)) + 255) / 256 * 256;
  int64_t s = std::max<int64_t>(1, budget / (f + 6 * h + 4 * r));
  s = std::min<int64_t>(s, max_slots);
  const int64_t hp = std::max<int64_t>(kMaxCols, 6 * s);
  const int64_t rest = budget - s * f - hp * h - 16;
  const int64_t rp = std::min<int64_t>(std::max<int64_t>(kMaxCols, rest / r), int64_t(kMaxCols) * s);
  *slots = int32_t(s);
  *h_pages = int32_t(hp);
  *r_pages = int32_t(rp);
}

int rpq_server_create_sized(rpq_kg* kg, int32_t n_slots, int32_t h_pages, int32_t r_pages, rpq_server** out) {
  ApiRange nvtx_range("rpq_server_create_sized");
  if (!kg || !out || n_slots < 1 || n_slots > 4096 || h_pages < kMaxCols || r_pages < kMaxCols ||
      h_pages > (1 << 20) || r_pages > (1 << 20)) {
    set_error(RPQ_EINVAL, "bad argument (need 1 <= n_slots <= 4096 and %d <= pages <= 2^20)", kMaxCols);
    return RPQ_EINVAL;
  }
  *out = nullptr;
  rpq_server* sv = new rpq_server();
  sv->kg = kg;
  if (const char* e = getenv("RPQ_INJECT_START_FAILURE")) sv->fail_start_at = atoll(e);
  const size_t cap = size_t(std::max<int32_t>(kg->dev.n, 1));
  sv->h_page_bytes = int64_t((size_t(kg->dev.n) + 15) / 16 * 16);
  sv->r_page_bytes = int64_t((12 * cap + 255) / 256 * 256);
  sv->slot_fixed_bytes = slot_bytes(kg, false);
  int64_t pool_bytes = 0;
  int rc = alloc_device((void**)&sv->hpool, size_t(sv->h_page_bytes) * size_t(h_pages) + 16, &pool_bytes);
  if (rc == RPQ_OK) rc = alloc_device((void**)&sv->rpool, size_t(sv->r_page_bytes) * size_t(r_pages), &pool_bytes);
  if (rc == RPQ_OK && cudaMemset(sv->rpool, 0, size_t(sv->r_page_bytes) * size_t(r_pages)) != cudaSuccess) {
    cudaGetLastError();
    set_error(RPQ_ECUDA, "page pool clear failed");
    rc = RPQ_ECUDA;
  }
  sv->h_pages = h_pages;
  sv->r_pages = r_pages;
  for (int32_t i = h_pages - 1; i >= 0; --i) sv->h_free.push_back(i);
  for (int32_t i = r_pages - 1; i >= 0; --i) sv->r_free.push_back(i);
  while (rc == RPQ_OK && int32_t(sv->slots.size()) < n_slots) {
    Slot* s = nullptr;
    rc = create_slot(kg, &s, false);
    if (rc != RPQ_OK) break;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      destroy_slot(s);
      set_error(RPQ_ECUDA, "cudaEventCreate failed");
      rc = RPQ_ECUDA;
      break;
    }
    sv->slots.push_back(s);
    sv->done_ev.push_back(ev);
  }
  if (rc != RPQ_OK) {
    rpq_server_destroy(sv);
    return rc;
  }
  sv->running.resize(sv->slots.size());
  sv->busy.assign(sv->slots.size(), false);
  sv->held_h.resize(sv->slots.size());
  sv->held_r.resize(sv->slots.size());
  *out = sv;
  return RPQ_OK;
}

int rpq_server_create(rpq_kg* kg, int64_t budget_bytes, int32_t max_slots, rpq_server** out) {
  if (!kg || !out || max_slots < 1) { set_error(RPQ_EINVAL, "bad argument"); return RPQ_EINVAL; }
  int32_t s = 0, hp = 0, rp = 0;
  size_server(kg, budget_bytes, std::min(max_slots, 4096), &s, &hp, &rp);
  return rpq_server_create_sized(kg, s, hp, rp, out);
}

int rpq_server_info(const rpq_server* sv, int32_t* n_slots, int64_t* slot_bytes, int32_t* n_running, int32_t* n_waiting) {
  if (!sv) { set_error(RPQ_EINVAL, "NULL server"); return RPQ_EINVAL; }
  if (n_slots) *n_slots = int32_t(sv->slots.size());
  if (slot_bytes) *slot_bytes = sv->slot_fixed_bytes;
  int32_t r = 0;
  for (bool b : sv->busy) r += b;
  if (n_running) *n_running = r;
  if (n_waiting) *n_waiting = int32_t(sv->waiting.size());
  return RPQ_OK;
}

int rpq_server_pages(const rpq_server* sv, int32_t* h_pages, int64_t* h_page_bytes, int32_t* r_pages,
                     int64_t* r_page_bytes, int32_t* peak_running) {
  if (!sv) { set_error(RPQ_EINVAL, "NULL server"); return RPQ_EINVAL; }
  if (h_pages) *h_pages = sv->h_pages;
  if (h_page_bytes) *h_page_bytes = sv->h_page_bytes;
  if (r_pages) *r_pages = sv->r_pages;
  if (r_page_bytes) *r_page_bytes = sv->r_page_bytes;
  if (peak_running) *peak_running = sv->peak_running;
  return RPQ_OK;
}

int rpq_server_submit(rpq_server* sv, const rpq_query* q, uint64_t tag) {
  ApiRange nvtx_range("rpq_server_submit");
  if (!sv) { set_error(RPQ_EINVAL, "NULL server"); return RPQ_EINVAL; }
  Pending p;
  p.tag = tag;
  p.t_submit = Clock::now();
  p.empty = false;
  int rc = check_query(sv->kg, q, &p.qv, &p.empty);
  if (rc != RPQ_OK) return rc;
  sv->waiting.push_back(p);
  ++sv->submitted;
  rc = collect(sv, false);
  if (rc != RPQ_OK) return rc;
  return admit(sv);
}

int rpq_server_poll(rpq_server* sv, rpq_completion* out, int32_t max_done, int32_t* n_done, int32_t wait) {
  ApiRange nvtx_range("rpq_server_poll");
  if (!sv || !n_done || (max_done > 0 && !out)) { set_error(RPQ_EINVAL, "bad argument"); return RPQ_EINVAL; }
  *n_done = 0;
  int rc = collect(sv, false);
  if (rc == RPQ_OK) rc = admit(sv);
  if (rc == RPQ_OK && wait && sv->finished.empty()) {
    rc = collect(sv, true);
    if (rc == RPQ_OK) rc = admit(sv);
  }
  while (*n_done < max_done && !sv->finished.empty()) {
    out[*n_done] = sv->finished.front();
    sv->finished.pop_front();
    ++*n_done;
  }
  return rc;
}

int rpq_server_replay(rpq_server* sv, const rpq_query* qs, const double* arrival_s, int32_t nq,
                      double* latency_s, int32_t* status, int32_t* n_out, rpq_result* out, double* wall_s) {
  ApiRange nvtx_range("rpq_server_replay");
  if (!sv || nq < 0 || (nq > 0 && (!qs || !arrival_s || !latency_s || !status || !n_out))) {
    set_error(RPQ_EINVAL, "bad argument");
    return RPQ_EINVAL;
  }
  for (int32_t i = 1; i < nq; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) { set_error(RPQ_EINVAL, "arrival times must be non-decreasing"); return RPQ_EINVAL; }
  // completions are matched to the schedule by tag (the query index), so no
  // query submitted before the call may still be running, waiting or unpolled
  bool idle = sv->waiting.empty() && sv->finished.empty();
  for (bool b : sv->busy) idle = idle && !b;
  if (!idle) {
    set_error(RPQ_EINVAL, "replay needs an idle server: poll every submitted query first");
    return RPQ_EINVAL;
  }
  std::vector<int64_t> base(size_t(nq) + 1, 0);
  for (int32_t i = 0; i < nq; ++i) base[size_t(i) + 1] = base[size_t(i)] + std::max(qs[i].k, 0);
  const Clock::time_point t0 = Clock::now();
  int32_t next = 0, done = 0;
  // latency counts from the scheduled arrival, not from the (possibly later) submit
  while (done < nq) {
    const double now = seconds(t0, Clock::now());
    while (next < nq && arrival_s[next] <= now) {
      Pending p;
      p.tag = uint64_t(next);
      p.t_submit = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[next]));
      p.empty = false;
      const int rc = check_query(sv->kg, &qs[next], &p.qv, &p.empty);
      if (rc != RPQ_OK) {
        status[next] = rc; n_out[next] = 0; latency_s[next] = 0.0; ++done;
      } else {
        sv->waiting.push_back(p);
        ++sv->submitted;
      }
      ++next;
    }
    int rc = collect(sv, false);
    if (rc == RPQ_OK) rc = admit(sv);
    if (rc != RPQ_OK) return rc;
    while (!sv->finished.empty()) {
      const rpq_completion c = sv->finished.front();
      sv->finished.pop_front();
      const int32_t i = int32_t(c.tag);
      status[i] = c.status;
      n_out[i] = c.n_res;
      latency_s[i] = c.latency_s;
      if (out && c.n_res > 0) memcpy(out + base[size_t(i)], c.res, sizeof(rpq_result) * size_t(c.n_res));
      ++done;
    }
    if (done < nq && next < nq && sv->waiting.empty()) {
      bool running = false;
      for (bool b : sv->busy) running |= b;
      if (!running) {                                  // idle until the next arrival
        const double gap = arrival_s[next] - seconds(t0, Clock::now());
        if (gap > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(gap - 100e-6));
      }
    }
  }
  if (wall_s) *wall_s = seconds(t0, Clock::now());
  return RPQ_OK;
}

int rpq_server_destroy(rpq_server* sv) {
  ApiRange nvtx_range("rpq_server_destroy");
  if (!sv) return RPQ_OK;
  for (size_t i = 0; i < sv->slots.size(); ++i) {
    destroy_slot(sv->slots[i]);
    if (i < sv->done_ev.size()) cudaEventDestroy(sv->done_ev[i]);
  }
  cudaFree(sv->hpool);
  cudaFree(sv->rpool);
  delete sv;
  return RPQ_OK;
}

}  // extern "C"
