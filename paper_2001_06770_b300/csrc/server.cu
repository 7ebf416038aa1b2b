// Serving loop of librpq: continuous batching of radial-pattern queries.
//
// A server owns a set of search slots; each slot holds the device state of one
// in-flight query (hit-level table, visited bytes, frontier bit maps and work
// lists, about 60 bytes per graph node) and its own CUDA stream.  The number of
// slots follows from the caller's device-memory budget: queries are admitted by
// the memory their search state needs.  A submitted query starts at once when
// a slot is free, otherwise it waits in a FIFO; every submit and poll call
// collects finished queries (CUDA event per slot, no blocking) and admits
// waiting queries into the slots they freed, so queries that arrive while
// others run are overlapped on the device with them.  Each query runs exactly
// the same kernels as rpq_search, so its result is the same alone or in the mix.
#include <algorithm>
#include <chrono>
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
  std::deque<Pending> waiting;
  std::deque<rpq_completion> finished;
  int64_t submitted = 0, completed = 0;
};

namespace rpq {

static double seconds(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

// Start waiting queries on free slots (in arrival order).
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
    const int rc = start_query(sv->kg, sv->slots[i], p.qv);
    if (rc != RPQ_OK) return rc;
    const cudaError_t e = cudaEventRecord(sv->done_ev[i], sv->slots[i]->st);
    if (e != cudaSuccess) { set_error(RPQ_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e)); return RPQ_ECUDA; }
    sv->running[i] = p;
    sv->busy[i] = true;
    sv->waiting.pop_front();
  }
  return RPQ_OK;
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

int rpq_server_create(rpq_kg* kg, int64_t budget_bytes, int32_t max_slots, rpq_server** out) {
  if (!kg || !out || max_slots < 1) { set_error(RPQ_EINVAL, "bad argument"); return RPQ_EINVAL; }
  *out = nullptr;
  rpq_server* sv = new rpq_server();
  sv->kg = kg;
  int rc = RPQ_OK;
  int64_t used = 0;
  while (int32_t(sv->slots.size()) < max_slots) {
    Slot* s = nullptr;
    rc = create_slot(kg, &s);
    if (rc != RPQ_OK) break;
    if (!sv->slots.empty() && used + s->bytes > budget_bytes) { destroy_slot(s); break; }
    used += s->bytes;
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
  if (sv->slots.empty() || (rc != RPQ_OK && rc != RPQ_ENOMEM)) {
    rpq_server_destroy(sv);
    return rc != RPQ_OK ? rc : RPQ_ENOMEM;
  }
  sv->running.resize(sv->slots.size());
  sv->busy.assign(sv->slots.size(), false);
  *out = sv;
  return RPQ_OK;
}

int rpq_server_info(const rpq_server* sv, int32_t* n_slots, int64_t* slot_bytes, int32_t* n_running, int32_t* n_waiting) {
  if (!sv) { set_error(RPQ_EINVAL, "NULL server"); return RPQ_EINVAL; }
  if (n_slots) *n_slots = int32_t(sv->slots.size());
  if (slot_bytes) *slot_bytes = sv->slots.empty() ? 0 : sv->slots[0]->bytes;
  int32_t r = 0;
  for (bool b : sv->busy) r += b;
  if (n_running) *n_running = r;
  if (n_waiting) *n_waiting = int32_t(sv->waiting.size());
  return RPQ_OK;
}

int rpq_server_submit(rpq_server* sv, const rpq_query* q, uint64_t tag) {
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
  if (!sv || nq < 0 || (nq > 0 && (!qs || !arrival_s || !latency_s || !status || !n_out))) {
    set_error(RPQ_EINVAL, "bad argument");
    return RPQ_EINVAL;
  }
  for (int32_t i = 1; i < nq; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) { set_error(RPQ_EINVAL, "arrival times must be non-decreasing"); return RPQ_EINVAL; }
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
  if (!sv) return RPQ_OK;
  for (size_t i = 0; i < sv->slots.size(); ++i) {
    destroy_slot(sv->slots[i]);
    if (i < sv->done_ev.size()) cudaEventDestroy(sv->done_ev[i]);
  }
  delete sv;
  return RPQ_OK;
}

}  // extern "C"
