// Host-side internals of librpq shared by the translation units.
#pragma once
#include <cstdint>
#include <cstdio>
#include <unordered_map>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rpq.h"
#include "rpq_internal.cuh"

namespace rpq {

// An NVTX range over one call of the C ABI, so that NVIDIA's profilers can
// attribute the kernels and copies on their timelines to the call that
// issued them (ncu --nvtx --nvtx-include "rpq_search/" and the like).  With
// no profiler attached a range costs a branch on a null function pointer.
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange&) = delete;
  ApiRange& operator=(const ApiRange&) = delete;
};

void set_error(int code, const char* fmt, ...);
int dev_err_to_status(uint32_t err);
int alloc_device(void** p, size_t bytes, int64_t* counter);

#define RPQ_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::rpq::set_error(RPQ_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                       __FILE__, __LINE__);                                                \
      return e_ == cudaErrorMemoryAllocation ? RPQ_ENOMEM : RPQ_ECUDA;                     \
    }                                                                                      \
  } while (0)

// One search slot: device state of one in-flight query, its stream, pinned
// staging for results and the graphs captured for each query shape.
struct Slot {
  DevSlot d{};
  LevelRec* lrec = nullptr;      // per-level records of the current query (profiling mode)
  cudaStream_t st = nullptr;
  int64_t bytes = 0;
  Ctl* h_ctl = nullptr;
  rpq_result* h_res = nullptr;   // inside the h_ctl allocation, kCtlBytes after its start
  std::vector<void*> allocs;
  std::unordered_map<uint64_t, cudaGraphExec_t> graphs;
  bool busy = false;
  int32_t pending_k = 0;
  int32_t pending_nc = 0;
  int32_t pending_nm = 0;
};

// Optional per-launch timing with CUDA events (profiling mode, no graphs).
struct SgScratch;   // subgraph.cu

// Launch kinds of the level kernels in a Glevel record (profiling).
enum LaunchKind { kKindOther = 0, kKindEnqueue, kKindTarget, kKindExpand };

struct Prof {
  struct Rec { int cls; cudaEvent_t a, b; cudaStream_t st; int run, level, kind; };
  // Device times of the level kernels of one Glevel of one run of a query.
  struct LevelTimes { cudaStream_t st; int run, level; double ms[4]; };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  std::vector<LevelTimes> level_times;   // per Glevel, in launch order, until paired with its record
  std::vector<rpq_level_profile> levels; // finished Glevel profiles (rpq_profile_levels)
  double ms[RPQ_PROF_CLASSES] = {};
  int64_t launches[RPQ_PROF_CLASSES] = {};
  int tag_run = -1, tag_level = -1, tag_kind = kKindOther;   // set by the launcher before a level kernel
  cudaEvent_t take() {
    if (pool.empty()) { cudaEvent_t e; cudaEventCreate(&e); return e; }
    cudaEvent_t e = pool.back(); pool.pop_back(); return e;
  }
  void begin(cudaStream_t st, cudaEvent_t* a) { *a = take(); cudaEventRecord(*a, st); }
  void end(int cls, cudaStream_t st, cudaEvent_t a) {
    cudaEvent_t b = take(); cudaEventRecord(b, st);
    pending.push_back({cls, a, b, st, tag_run, tag_level, tag_kind});
    tag_kind = kKindOther;
  }
  // Timings of the launches of stream `st` (after it has been synchronised;
  // every stream when st is NULL).
  void collect(cudaStream_t st = nullptr) {
    size_t keep = 0;
    for (const Rec& r : pending) {
      if (st && r.st != st) { pending[keep++] = r; continue; }
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.cls] += t;
        launches[r.cls] += 1;
        if (r.kind != kKindOther && r.level >= 0) {
          LevelTimes* lt = nullptr;
          for (auto it = level_times.rbegin(); it != level_times.rend(); ++it)
            if (it->st == r.st && it->run == r.run && it->level == r.level) { lt = &*it; break; }
          if (!lt) { level_times.push_back({r.st, r.run, r.level, {0, 0, 0, 0}}); lt = &level_times.back(); }
          lt->ms[r.kind] += t;
        }
      }
      pool.push_back(r.a); pool.push_back(r.b);
    }
    pending.resize(keep);
  }
  ~Prof() { for (cudaEvent_t e : pool) cudaEventDestroy(e); }
};

}  // namespace rpq

// Opaque graph handle of the C ABI.
struct rpq_kg {
  rpq::DevKG dev{};
  int device = 0;
  int64_t m2 = 0;
  double alpha = 0.5, abar = 1.0;
  uint32_t* d_row_ptr = nullptr;
  uint32_t* d_adj = nullptr;
  uint8_t* d_amax = nullptr;
  uint16_t* d_lvx = nullptr;
  uint32_t* d_lvx_long = nullptr;
  uint32_t* d_kw_ptr = nullptr;
  int32_t* d_kw_nodes = nullptr;        // postings in internal ids
  int32_t* d_ext_of = nullptr;          // internal -> caller node id
  int32_t* d_int_of = nullptr;          // caller -> internal node id
  std::vector<int32_t> ext_of, int_of;  // host copies
  std::vector<uint32_t> row_ext;        // caller row offsets (for exports)
  int64_t device_bytes = 0;
  std::vector<int64_t> kw_ptr;   // host copy of the postings offsets
  std::vector<rpq::Slot*> slots; // search slots, created on first use
  rpq::Prof* prof = nullptr;      // profiling mode when non-NULL
  rpq_tuning tune{32, 16, 8, 4};  // work-split parameters (rpq_set_tuning / rpq_autotune)
  rpq::SgScratch* sg = nullptr;   // result-subgraph lists (rpq_search_subgraphs), grown on demand
};

namespace rpq {
// Fill d_row_ptr, d_adj and d_amax of kg from the host CSR (kg_build.cu).
int build_graph(rpq_kg* kg, const rpq_kg_desc* d);
// The packed adjacency and amax in caller ids (kg_build.cu).
int export_graph(const rpq_kg* kg, uint32_t* adj, uint8_t* amax);

// Search slots and query execution (api.cu).
int create_slot(rpq_kg* kg, Slot** out, bool own_cols = true);
int64_t slot_bytes(const rpq_kg* kg, bool own_cols);   // device bytes create_slot allocates
void destroy_slot(Slot* s);
int get_slot(rpq_kg* kg, size_t i, Slot** out);
int check_query(const rpq_kg* kg, const rpq_query* q, QueryDev* qv, bool* empty);
int start_query(rpq_kg* kg, Slot* s, const QueryDev& qv);      // asynchronous
int finish_query(rpq_kg* kg, Slot* s, rpq_result* out, int32_t* n_out, rpq_stats* stats);
void empty_result(int32_t* n_out, rpq_stats* stats);
void apply_tuning(rpq_kg* kg, Slot* s);   // slot parameters from kg->tune; drops captured graphs
void fill_stats(const Ctl& c, rpq_stats* st);
void free_subgraph_scratch(rpq_kg* kg);     // subgraph.cu

// Kernel launch sequences (search_kernels.cu).
int launch_query_setup(const DevSlot& s, const QueryDev& qv, const int32_t* d_kw, cudaStream_t st);
int launch_query_body(const DevKG& g, const DevSlot& s, int n_m, int L, cudaStream_t st, Prof* prof,
                      bool stop_early);
void launch_run_setup(const DevKG& g, const DevSlot& s, int run, cudaStream_t st, Prof* prof);
void launch_level(const DevKG& g, const DevSlot& s, int run, cudaStream_t st, Prof* prof,
                  cudaGraphConditionalHandle loop, bool in_graph);
void launch_select_recover(const DevKG& g, const DevSlot& s, int n_m, cudaStream_t st, Prof* prof);
void launch_results(const DevSlot& s, cudaStream_t st, Prof* prof);
int kernels_fixed_per_query(int n_m);
int launch_central_part(const DevKG& g, const DevSlot& s, int L, cudaStream_t st, Prof* prof);
int launch_marginal_part(const DevKG& g, const DevSlot& s, int n_m, int L, cudaStream_t st, Prof* prof);
// The multi-query persistent kernel: n_queries query records (keyword ids
// and parameters) run on n_slots slots (own columns), one record of
// kBatchRecBytes per query at d_out; d_state holds batch_state_bytes(n_slots)
// bytes (cleared here).  limit: watchdog, clock cycles without a finished
// phase.  Asynchronous on st.
size_t batch_state_bytes(int n_slots);
int launch_batch(const DevKG& g, const DevSlot* slots, int n_slots, const QueryDev* d_queries, int n_queries,
                 void* d_out, void* d_state, long long limit, cudaStream_t st);
}  // namespace rpq
