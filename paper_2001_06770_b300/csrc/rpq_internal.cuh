// Internal declarations of librpq (device structures, helpers).
//
// Device layout of a loaded graph (all in HBM, written once by rpq_load_kg):
//   row_ptr  uint32[n+1]   CSR offsets (m2 < 2^32)
//   adj      uint32[m2]    (a << 26) | neighbour, each row ascending, i.e.
//                          sorted by activation level a, then neighbour id
//   amax     uint8[n]      largest activation level of the row
//   kw_ptr   uint32[n_kw+1], kw_nodes int32[]   keyword postings (V_t)
//
// Per-search state (one "slot"; several slots run concurrently):
//   H        uint8[8][hp]  Node-Keyword Matrix (Section 4.2.1), column-major
//                          hit levels; a column's level is written by the
//                          enqueue that first sees its visited bit (the
//                          node's seen byte records which), and is read only
//                          after that, so H is never cleared
//   vis      uint8[n]      visited bits, bit j = column j reached (read as
//                          bytes, set with 32-bit atomicOr / red.or)
//   vseen    uint8[n]      the visited bits the enqueue has written H for
//   F[2]     uint32[n/32]  Frontier Flag Array, double buffered by level
//   cf       uint32[n/32]  Joining Flag Array (node stopped expanding)
//   stopl    uint8[n]      level at which the cf bit was set
//   items    Item[n]       expansion work list of the current level (8 B each,
//                          column masks in imask uint16[n])
//   cg       uint32[n]     identified CGs, (level << 26) | caller node id
// Node ids inside the device structures are internal (decreasing degree, see
// kg_build.cu); CG keys, selected CGs and results carry the caller's ids.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rpq {

constexpr uint32_t kNodeBits = 26;
constexpr uint32_t kNodeMask = (1u << kNodeBits) - 1u;
constexpr uint8_t kInf = 255;
constexpr int kMaxCols = 8;
constexpr int kMaxK = 64;
constexpr int kMaxLevel = 63;
constexpr int kRecStride = kMaxLevel + 3;   // recovery counters of one column
constexpr int kMaxLabels = 8192;

enum DevErr : uint32_t {
  kErrNone = 0,
  kErrBadCol = 1u << 0,    // neighbour id out of range or self-loop
  kErrUnsorted = 1u << 1,  // row not strictly ascending
  kErrBadLabel = 1u << 2,  // label >= n_labels
  kErrAsym = 1u << 3,      // missing reverse entry or label differs
  kErrLevel = 1u << 4,     // activation level above kMaxLevel
  kErrKeyword = 1u << 5,   // keyword id out of range (device queries)
  kErrOverflow = 1u << 6,  // a work list overflowed its capacity
  kErrInternal = 1u << 7,
  kErrTimeout = 1u << 8,   // a bounded grid barrier ran out
  kErrBounds = 1u << 9,    // checked build: an index failed its bounds check (the access was skipped)
};

// Checked build (-DRPQ_CHECKED, librpq_checked.so): the search kernels test
// the indices they derive from device data (queue and list entries, CSR
// offsets, neighbour ids, work-list positions) before using them; a failed
// test sets kErrBounds in *err and the access is skipped, so the query
// reports RPQ_EINTERNAL and nothing outside a buffer is touched.  In the
// normal build every test is the constant true and costs nothing.
#ifdef RPQ_CHECKED
#define RPQ_IN_BOUNDS(cond, err) ((cond) ? true : (atomicOr((err), ::rpq::kErrBounds), false))
#else
#define RPQ_IN_BOUNDS(cond, err) true
#endif

// Level index of every row, for x = 1..kLvxLevels: for a row with at most
// kLvxMaxDeg entries, lvx[x-1][v] is the offset (from the row start) of the
// first entry with level >= x; a longer row (a hub; there are fewer than
// 2^16 of them, as m2 < 2^32) stores its hub number h in every lvx[x-1][v],
// and the offsets go to lvx_long[h * kLvxLevels + x-1] (32-bit).  Higher
// levels use a binary search.
constexpr uint32_t kLvxLevels = 8;
constexpr uint32_t kLvxMaxDeg = 65535;

struct DevKG {
  int32_t n;
  uint32_t m2;
  const uint32_t* row_ptr;
  const uint32_t* adj;
  const uint8_t* amax;
  const uint16_t* lvx;        // kLvxLevels * n, level-major
  const uint32_t* lvx_long;   // kLvxLevels per row longer than kLvxMaxDeg
  int32_t n_kw;
  const uint32_t* kw_ptr;
  const int32_t* kw_nodes;    // internal ids
  const int32_t* ext_of;      // internal -> caller node id
  const int32_t* int_of;      // caller -> internal node id
};

// One expansion work item: the newly active segment of a frontier node.  The
// item's column masks (columns with h == level in the low byte, h < level in
// the high byte) are kept in a parallel uint16 array.
struct __align__(8) Item {
  uint32_t seg_begin;  // first CSR entry of the segment
  uint32_t off;        // exclusive prefix of segment lengths (work units)
};

// Query parameters as the kernels read them (device copy in the slot).
// The query's keyword columns live where the host placed them: column j of
// the Node-Keyword Matrix at hc[j] (one byte per node), and the recovery's
// CG masks and node list of central column j at rm[j] and rl[j] (cap
// entries each).  A slot that owns its columns points them at its own
// arrays; a server lends each query pages for just its |T| columns.
struct QueryDev {
  int32_t kw[2 * kMaxCols];  // central ids then marginal ids
  int32_t n_c, n_m, k, L;
  double gamma;
  int32_t w;                 // CG beam width, k <= w <= kMaxK
  int32_t product;           // multiplicative S^r = S^c * S^m
  uint8_t* hc[kMaxCols];
  unsigned long long* rm[kMaxCols];
  uint32_t* rl[kMaxCols];
};

// Control block of one slot, read and updated by the kernels of a search.
struct Ctl {
  unsigned long long work[2];  // per level parity: (items << 38) | work units
  uint32_t done;               // current run finished
  uint32_t exp_skip;           // the run had finished before this level's enqueue: its expansion exits
                               // at once (every block of the launch that stops the run still runs)
  uint32_t level;              // last identified level of the current run
  int32_t last_expanded;       // last level with an expansion (-1: none)
  uint32_t nq[2];              // |Q_l| per level parity
  uint32_t n_matched;          // selected CGs matched so far (marginal run)
  uint32_t rpg_stop;           // Theorem 4 ended the marginal run (w > k)
  uint32_t skip_lvl;           // l + 1: the expansion of Glevel l cannot change the outcome (k_target)
  uint32_t tgt_n, tgt_done;    // k_target: (column, node) hits found, blocks finished
  unsigned long long eact_lvl[2];  // E_act of the level being enqueued, per level parity
  unsigned long long e_act_skip;   // E_act of skipped expansions
  uint32_t qlog_n;             // entries of the frontier log (trace mode)
  uint32_t ncg;                // CGs identified (central run)
  uint32_t ncg_at;             // ncg after the last expanded level
  uint32_t cg_next[2];         // nodes the expansion of the previous level completed, per level parity
  uint32_t err;                // DevErr bits
  uint32_t n_items, n_work;    // expansion list of the current level
  uint32_t nsel;               // selected CGs
  uint32_t nvc;                // (g, node) pairs of V_C
  uint32_t ulist_n;            // recovery: nodes of the union list
  uint32_t lvl_enq, lvl_exp;   // Glevel of the next k_enqueue / the current k_expand
  uint32_t fq_n[2];            // frontier queue lengths per level parity
  uint32_t fq_over[2];         // queue abandoned (frontier too large): use the bitmap
  uint32_t iters[2];           // level kernel pairs executed per run
  uint32_t fq_use[2];          // the queue of this parity is being filled
  uint32_t n_res;
  uint32_t topk_done;          // k_topk: blocks finished
  uint32_t rec_done;           // recovery: CTAs finished
  unsigned long long e_act[2];  // per run
  unsigned long long hits[2];   // first hits, counted when the run stops
  unsigned long long seeded[2]; // (node, column) pairs seeded with h = 0
  unsigned long long units, items, frontier;  // work totals of both runs
  int32_t levels[2];           // last identified level per run
  int32_t sel[kMaxK];          // selected CGs, caller ids (ranking ties by caller id)
  int32_t sel_int[kMaxK];      // the same nodes, internal ids
  uint8_t sel_sc[kMaxK];
  uint8_t matched[kMaxK];
  uint8_t sm[kMaxK];
};

// Per-Glevel record of one query, kept while kernels are profiled: the level
// kernels of Glevel l of run r write entry r * kLogLevels + l.
constexpr int kLogLevels = kMaxLevel + 1;
enum LevelFlags : uint32_t {
  kLvlExpanded = 1u,   // the expansion ran
  kLvlSkipped = 2u,    // the V_C check skipped the expansion
  kLvlStop = 4u,       // the run stopped at this level
  kLvlQueue = 8u,      // the enqueue read the frontier queue (else the bit map)
};
struct LevelRec {
  unsigned long long units;    // work units (CSR entries of the items' segments)
  unsigned long long items;    // expansion items
  unsigned long long eact;     // (column, edge) activations the expansion executed
  unsigned long long claims;   // (node, column) claims written (h = l+1)
  uint32_t frontier;           // |Q_l|
  uint32_t flags;              // LevelFlags
};

// Bytes of the control block in a slot's control allocation; the results
// (rpq_result[kMaxK]) follow it there, so one copy returns both.
constexpr size_t kCtlBytes = (sizeof(Ctl) + 15) / 16 * 16;

struct DevSlot {
  uint8_t* H;                 // the slot's own columns (kMaxCols * hp bytes), or NULL (server slots)
  uint32_t* vis;
  uint8_t* vseen;             // per node: the visited bits the enqueue has written H for
  uint32_t* F[2];
  uint32_t* cf;
  uint8_t* stopl;
  Item* items;
  uint16_t* imask;            // column masks of the items
  uint32_t* cg;
  uint32_t* topk;             // k_topk: survivors of each block (w per block)
  unsigned long long* rmask;  // recovery: the slot's own per-column CG masks (kMaxCols * cap), or NULL
  unsigned long long* vmask;  // recovery: union over columns
  uint32_t* rlist;            // recovery: the slot's own per-column node lists (kMaxCols * cap), or NULL
  uint32_t* rcnt;             // recovery: per-column counters (kMaxCols * kRecStride), zero between uses
  uint32_t* tile_first;       // expansion: first item of each warp tile
  uint32_t tile_cap;
  uint32_t* fq[2];            // frontier queues (nodes of F), per level parity
  uint32_t fq_limit;          // queue used while it holds at most this many nodes
  uint32_t fq_next_mult;      // next queue kept while a level's work <= fq_next_mult * fq_limit
  uint32_t hp;                // column pitch of H (H[j * hp + v])
  uint32_t* ulist;
  uint32_t* vcl;              // V_C pairs (g << 26 | node)
  uint32_t cap;               // capacity (elements) of items/cg/lists
  uint32_t* qlog;             // trace mode: (level << 26 | node) of every Q_l entry
  uint32_t qcap;
  uint32_t* tgt;              // k_target: (column << 26 | node) hits of V_C nodes
  uint32_t tgt_cap;
  uint32_t target;            // marginal run: check V_C first and skip a final expansion
  uint32_t tgt_min_work;      // ... on levels with at least this many work units
  void* run_clear;            // vis, F[0], F[1], cf in one block, cleared per run
  unsigned long long run_clear_bytes;
  uint32_t* sticky;           // device error bits kept across queries
  unsigned* bar;              // grid barrier of the persistent run kernel: count, generation
  uint32_t persistent;        // run each level loop as one cooperative k_run launch
  long long bar_limit;        // clock cycles a block waits at a grid barrier before it gives up
  LevelRec* lrec;             // per-level records (2 * kLogLevels) while profiling, else NULL
  Ctl* ctl;
  QueryDev* q;
  void* res;                  // rpq_result[kMaxK] on the device
  int32_t* n_res;
};

// Multi-query persistent kernel: the work-queue state of one slot (device
// memory, zeroed before the launch).  A phase of a slot's query is split
// into chunks; a block takes chunk next of the current phase with one
// atomic add on word, and the block that finishes its last chunk moves the
// slot to its next phase.
constexpr int kBatchMaxSlots = 32;
struct BatchSlotState {
  unsigned long long word;   // the current phase (search_kernels.cu: batch_word) and the next chunk to hand out
  uint32_t done;             // chunks of the current phase finished
  uint32_t phase;            // current phase (search_kernels.cu)
  uint32_t run;              // its run (0 central, 1 marginal)
  uint32_t level;            // recovery level of a recovery sweep phase
  int32_t query;             // batch index of the slot's query, -1 when the slot is idle
  uint32_t pad[25];          // one 128-byte line per slot: polls and claims of one slot do not
                             // contend with another's
};
static_assert(sizeof(BatchSlotState) == 128, "one line per slot");
struct BatchCtl {
  uint32_t next_query;         // batch index of the next query to start
  uint32_t finished;           // queries whose record is written
  uint32_t err;                // kErrTimeout: no phase finished within the watchdog limit
  uint32_t pad;
  unsigned long long progress; // phases finished so far (watchdog)
};
// Record of one query of a persistent batch: a flag word (1 once the record
// is complete) padded to 16 bytes, the control block and the results.
constexpr size_t kBatchRecHead = 16;
constexpr size_t kBatchRecBytes = kBatchRecHead + kCtlBytes + 24 * kMaxK;   // 24 = sizeof(rpq_result)

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Column pointers of the current query.  Plain loads, not the read-only
// path: the multi-query persistent kernel rewrites a slot's query record
// while it runs.
__device__ __forceinline__ uint8_t* hcol(const QueryDev& q, int j) { return q.hc[j]; }
__device__ __forceinline__ unsigned long long* rmcol(const QueryDev& q, int j) { return q.rm[j]; }
__device__ __forceinline__ uint32_t* rlcol(const QueryDev& q, int j) { return q.rl[j]; }

__device__ __forceinline__ uint8_t vis_byte(const uint32_t* vis, uint32_t v) {
  return reinterpret_cast<const uint8_t*>(vis)[v];
}

// First index in [lo, hi) of a sorted packed row whose level is >= x.
__device__ __forceinline__ uint32_t seg_lower(const uint32_t* adj, uint32_t lo, uint32_t hi, uint32_t x) {
  const uint32_t key = x << kNodeBits;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(adj + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// First entry of row v (bounds rb, re) whose level is >= x.
__device__ __forceinline__ uint32_t seg_at(const DevKG& g, uint32_t v, uint32_t rb, uint32_t re, uint32_t x) {
  if (x == 0) return rb;
  if (x > kLvxLevels) return seg_lower(g.adj, rb, re, x);
  const uint32_t o = g.lvx[size_t(x - 1) * size_t(g.n) + v];
  return rb + (re - rb <= kLvxMaxDeg ? o : g.lvx_long[size_t(o) * kLvxLevels + (x - 1)]);
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
  const uint32_t lane = lane_id();
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= uint32_t(o)) v += t;
  }
  return v;
}

// Exclusive block scan of one 64-bit value per thread; *total gets the sum.
// s_warp must hold 33 entries.  Contains __syncthreads.
static __device__ uint64_t block_excl_scan(uint64_t v, uint64_t* s_warp, uint64_t* total) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t incl = warp_incl_scan(v);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t t = lane < nw ? s_warp[lane] : 0;
    const uint64_t ti = warp_incl_scan(t);
    if (lane < nw) s_warp[lane] = ti - t;
    if (lane == 31) s_warp[32] = ti;
  }
  __syncthreads();
  const uint64_t r = s_warp[warp] + incl - v;
  *total = s_warp[32];
  __syncthreads();
  return r;
}

int num_sms();

}  // namespace rpq
