// Search kernels of one radial-pattern query (Section 4).
//
// One query runs as a sequence of launches on the slot's stream:
//   k_set_query                       copy parameters, reset the control block
//   per run (central, then marginal):
//     k_run_start (marginal run; k_set_query prepares the central one), one
//     memset of vis / F / cf, k_seed (Section 4.2.1)
//     per Glevel l:  k_enqueue        frontier enqueue + reset (4.2.2) and
//                                     result identification (4.2.3,
//                                     Theorem 3; PTC stop; RPG match;
//                                     Theorem 4); E_act of the level
//                    k_target         marginal run only: hits of level l+1
//                                     on V_C, and whether they decide the run
//                    k_expand         termination decision + expansion
//                                     (Algorithm 1) of the newly active edges
//   after the central run: k_topk (top-w CGs),
//                          k_recover_cols (Algorithm 2 -> V_C)
//   the results (Eq. 6, top-k by (S^r, id)) are written by the kernel that
//   ends the search: k_topk when there is no marginal run, else the k_expand
//   that stops the marginal run (no launch of their own)
// The Glevel is kept in the control block, so the level kernels form the body
// of a CUDA-graph WHILE node that k_expand ends when the run stops, or the
// L+1 early-exit repetitions of a flat graph; the graph of each query shape
// (|C|, |M|, L) is built once and replayed.  Without a graph (profiling,
// tracing) the host launches the same sequence and the kernels of finished
// runs return at once.
//
// Exactness: the expansion at level l touches, for frontier node v and
// column j, only the edges with max(h[v][j], a) == l (the rows are sorted by
// a, so they form one segment).  An edge with a smaller max was already
// handled at that earlier level by the same node (which was in the frontier
// then, because it is retained while it has an edge with a > level), so
// skipping Algorithm 1's re-scan changes no h value.  A thread that finds a
// column of a neighbour unreached (its visited bit clear) at level l claims
// it: it sets the visited and frontier bits with reductions that return
// nothing.  The claimed column's level is l+1 whoever claims it (Theorem 6:
// the bits set before the launch are all visible, so the column was not
// reached at an earlier level), and the node is in F_{l+1}, so the enqueue
// of level l+1 writes h = l+1 for every column that is new since it last
// saw the node (its seen byte): the hit levels are written once, coalesced,
// instead of as scattered bytes by every claim.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include <cooperative_groups.h>

#include "rpq_host.h"

namespace rpq {

namespace cg = cooperative_groups;

namespace {

constexpr int kEnqThreads = 256;
constexpr int kEnqRounds = 4;
constexpr int kExpThreads = 256;
constexpr int kExpRounds = 4;                      // 32-unit rounds per warp tile
constexpr int kTgtThreads = 256;
constexpr uint32_t kTgtMaxTasks = 4096;             // (V_C node, column) pairs the V_C check takes on
constexpr int kWarpTile = 32 * kExpRounds;         // 128 work units per warp tile
constexpr int kRecThreads = 1024;
constexpr int kRecCluster = 8;                     // CTAs sweeping one keyword column
constexpr int kTopkThreads = 1024;
constexpr int kTopkChunk = 4096;                   // keys per block and round of the top-w selection
constexpr int kTopkBits = 11;                      // radix digit of the top-w selection
constexpr unsigned long long kWorkBits = 38;
constexpr unsigned long long kWorkMask = (1ull << kWorkBits) - 1ull;

__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t* s_warp) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  uint64_t t = 0;
  if (threadIdx.x == 0) for (uint32_t w = 0; w < nw; ++w) t += s_warp[w];
  return t;  // valid in thread 0
}

// Load of a value that other blocks may have written earlier in the same
// kernel.  The persistent run kernel (P) reads such values from L2; separate
// kernels, and the chunks of the multi-query persistent kernel (each taken
// with an acquire: an atomic, then a fence, after the release of the phases
// before it), use the cached path.
template <bool P, typename T>
__device__ __forceinline__ T ldx(const T* ptr) {
  if constexpr (P) return __ldcg(ptr);
  else return *ptr;
}

__device__ __forceinline__ void vis_or(uint32_t* vis, uint32_t v, uint32_t bits) {
  atomicOr(vis + (v >> 2), bits << ((v & 3u) * 8u));
}

// The block's share of a phase's work: block b of n.  A launched kernel is
// its own phase (blockIdx.x of gridDim.x); in the multi-query persistent
// kernel a block runs chunk b of the n chunks of one query's phase.
struct Part {
  uint32_t b, n;
};
__device__ __forceinline__ Part launch_part() { return Part{blockIdx.x, gridDim.x}; }

// ------------------------------------------------------------ query set-up
__global__ void k_set_query(DevSlot s, QueryDev qv, const int32_t* d_kw) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // the record goes to global memory first and the keyword ids are patched
  // there (with nvcc 13.0 for sm_103a, a modified local copy of the by-value
  // record stored back lost the patched ids)
  QueryDev* dst = s.q;
  *dst = qv;
  if (d_kw) for (int i = 0; i < qv.n_c + qv.n_m; ++i) dst->kw[i] = d_kw[i];
  Ctl* c = s.ctl;
  uint32_t* w = reinterpret_cast<uint32_t*>(c);
  for (size_t i = 0; i < sizeof(Ctl) / 4; ++i) w[i] = 0;
  c->levels[0] = c->levels[1] = -1;
  c->last_expanded = -1;
  c->fq_use[0] = 1;                  // the rest of k_run_start's state for the central run
  s.bar[0] = 0;
  *s.n_res = 0;
}

__global__ void k_run_start(DevSlot s, int run) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Ctl* c = s.ctl;
  c->done = (run == 1 && (s.q->n_m == 0 || c->nsel == 0)) ? 1u : 0u;
  c->work[0] = c->work[1] = 0;
  c->nq[0] = c->nq[1] = 0;
  c->fq_n[0] = c->fq_n[1] = 0;
  c->fq_over[0] = c->fq_over[1] = 0;
  c->fq_use[0] = 1;
  c->fq_use[1] = 0;
  c->lvl_enq = c->lvl_exp = 0;
  c->level = 0;
  c->eact_lvl[0] = c->eact_lvl[1] = 0;
  c->skip_lvl = 0;
  c->ncg_at = 0;
  c->cg_next[0] = c->cg_next[1] = 0;
  c->tgt_n = c->tgt_done = 0;
  s.bar[0] = 0;                      // barrier arrivals of the persistent kernel
  c->last_expanded = -1;
}

// Position of the n-th (0-based) set bit of w; n < popc(w).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t w, uint32_t n) {
  uint32_t pos = 0, c = __popc(w & 0xffffu);
  if (n >= c) { n -= c; w >>= 16; pos += 16; }
  c = __popc(w & 0xffu);
  if (n >= c) { n -= c; w >>= 8; pos += 8; }
  c = __popc(w & 0xfu);
  if (n >= c) { n -= c; w >>= 4; pos += 4; }
  c = __popc(w & 0x3u);
  if (n >= c) { n -= c; w >>= 2; pos += 2; }
  if (n >= (w & 1u)) pos += 1;
  return pos;
}

// Append the flagged lanes' nodes to frontier queue p (warp aggregated).  The
// queue is abandoned (flag set) once it would exceed its limit; the bitmap F
// stays complete either way.
__device__ __forceinline__ void queue_push(const DevSlot& s, Ctl* c, int p, bool enabled, bool flag, uint32_t v) {
  if (!enabled) return;                                  // same in every lane
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (!b) return;
  const uint32_t lane = lane_id();
  uint32_t base = 0;
  if (lane == 0) {
    if (*(volatile uint32_t*)&c->fq_over[p]) base = 0xffffffffu;
    else {
      base = atomicAdd(&c->fq_n[p], uint32_t(__popc(b)));
      if (base + uint32_t(__popc(b)) > s.fq_limit) { atomicExch(&c->fq_over[p], 1u); base = 0xffffffffu; }
    }
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (flag && base != 0xffffffffu) s.fq[p][base + __popc(b & ((1u << lane) - 1u))] = v;
}

// Eq. 6 scores and the top-k results of the query (defined below).
__device__ void write_results(const DevSlot& s);

// Initialisation (Section 4.2.1): keyword nodes get h = 0 and become frontiers.
__device__ __forceinline__ void seed_body(const DevKG& g, const DevSlot& s, int run, Part pt) {
  Ctl* c = s.ctl;
  if (c->done) return;
  const QueryDev& q = *s.q;
  const int nt = run == 0 ? q.n_c : q.n_m;
  const int kb = run == 0 ? 0 : q.n_c;
  uint32_t beg[kMaxCols], len[kMaxCols];
  uint32_t total = 0;
  for (int j = 0; j < nt; ++j) {
    const int32_t kw = q.kw[kb + j];
    if (kw < 0 || kw >= g.n_kw) {
      beg[j] = len[j] = 0;
      if (pt.b == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrKeyword);
      continue;
    }
    beg[j] = g.kw_ptr[kw];
    len[j] = g.kw_ptr[kw + 1] - beg[j];
    total += len[j];
  }
  if (pt.b == 0 && threadIdx.x == 0) c->seeded[run] = total;   // (node, column) pairs with h = 0
  uint32_t* F0 = s.F[0];
  const uint32_t stride = pt.n * blockDim.x;
  const uint32_t end = (total + 31u) & ~31u;            // whole warps for the queue push
  for (uint32_t i = pt.b * blockDim.x + threadIdx.x; i < end; i += stride) {
    bool fresh = false;
    uint32_t v = 0;
    if (i < total) {
      uint32_t r = i;
      int j = 0;
      while (r >= len[j]) { r -= len[j]; ++j; }
      const int32_t vv = g.kw_nodes[beg[j] + r];
      if (vv >= 0 && vv < g.n) {
        v = uint32_t(vv);
        hcol(q, j)[v] = 0;
        vis_or(s.vis, v, 1u << j);
        const uint32_t old = atomicOr(F0 + (v >> 5), 1u << (v & 31));
        fresh = !((old >> (v & 31)) & 1u);
      } else {
        atomicOr(&c->err, kErrInternal);
      }
    }
    queue_push(s, c, 0, true, fresh, v);
  }
}

__global__ void k_seed(DevKG g, DevSlot s, int run) { seed_body(g, s, run, launch_part()); }

// ------------------------------------------------------------- RPG scores
// S^r of Eq. 6, or the multiplicative combination S^c * S^m.  Explicit
// round-to-nearest products and sum (no fused multiply-add), the same
// operations as a plain double evaluation of the formula.
__device__ __forceinline__ double rpg_score(const QueryDev& q, uint32_t sc, uint32_t sm) {
  if (q.product) return double(sc * sm);
  return __dadd_rn(__dmul_rn(q.gamma, double(sc)), __dmul_rn(1.0 - q.gamma, double(sm)));
}

// Theorem 4 at Glevel l of the marginal run (called with k <= matched < nsel):
// a CG still unmatched matches at level l+1 or later, so its RPG scores at
// least rpg_score(S^c, l+1); the run may stop when every such bound ranks
// after the k-th matched RPG on (score, node id), the ranking order.
// `matched` and `sm` may be the control block's or a prospective copy.
__device__ bool theorem4_stop(const Ctl* c, const uint8_t* matched, const uint8_t* sm, const QueryDev& q,
                              uint32_t nsel, uint32_t l) {
  unsigned long long used = 0;
  double srk = 0.0;
  int32_t idk = -1;
  for (int r = 0; r < q.k; ++r) {                         // k-th smallest by repeated minimum
    int best = -1;
    double bs = 0.0;
    for (uint32_t gi = 0; gi < nsel; ++gi) {
      if (!matched[gi] || ((used >> gi) & 1ull)) continue;
      const double v = rpg_score(q, c->sel_sc[gi], sm[gi]);
      if (best < 0 || v < bs || (v == bs && c->sel[gi] < c->sel[best])) { best = int(gi); bs = v; }
    }
    if (best < 0) return false;
    used |= 1ull << best;
    srk = bs;
    idk = c->sel[best];
  }
  for (uint32_t gi = 0; gi < nsel; ++gi) {
    if (matched[gi]) continue;
    const double b = rpg_score(q, c->sel_sc[gi], l + 1);
    if (!(b > srk || (b == srk && c->sel[gi] > idk))) return false;
  }
  return true;
}

// ---------------------------------------------------------- level: enqueue
// Frontier enqueue (Section 4.2.2): every node of F_l is taken and its flag
// cleared - from the frontier queue when it is short (work proportional to
// |Q_l|), otherwise by scanning the bitmap (lane = node of a 32-bit word).
// Identification (Section 4.2.3): central run, a node reached by all central
// keywords is a CG with S^c = max_j h (Theorem 3) and stops expanding;
// marginal run with |M| >= 2, a node reached by all marginal keywords stops
// (PTC).  Nodes still expanding become work items with their newly active
// segment; retained nodes (an edge with a > l) go to F_{l+1}.  The last block of
// the marginal run also performs the RPG identification of the level.
// Items are compacted with warp ballots, a block scan and one 64-bit
// atomicAdd per block tile; each item also marks the warp tiles of the
// expansion that start inside it.
// NT is the run's number of keyword columns (1..kMaxCols), a compile-time
// constant so that the per-node column loops hold exactly the run's columns.
// Whether the enqueue of the level of parity p reads the frontier queue
// (else the bit map): the queue was filled, did not overflow and is short.
template <bool P>
__device__ __forceinline__ bool enqueue_sparse(const DevSlot& s, const Ctl* c, int p) {
  return ldx<P>(&c->fq_use[p]) && !ldx<P>(&c->fq_over[p]) && ldx<P>(&c->fq_n[p]) <= s.fq_limit;
}

// Shared memory of the enqueue, declared once for every column count.
struct EnqShared {
  uint64_t warp[33];
  unsigned long long base;
  uint32_t acc[kMaxK];
};

template <bool P, int NT>
__device__ __forceinline__ void enqueue_level(const DevKG& g, const DevSlot& s, int run, uint32_t l, Part pt,
                                              EnqShared& sh) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  constexpr int nt = NT;
  const uint32_t full = (1u << nt) - 1u;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const int p = int(l & 1u);
  uint32_t* Fc = s.F[p];
  uint32_t* Fn = s.F[p ^ 1];
  uint64_t* s_warp = sh.warp;
  unsigned long long& s_base = sh.base;
  uint32_t* s_acc = sh.acc;

  if (run == 1 && pt.b == pt.n - 1u) {
    // RPG identification: a selected CG matches when every marginal keyword
    // has reached some node of its V_C; then S^m = max_i min_{v in V_C} h = l.
    // (The last block: on a short level the first blocks hold the frontier.)
    const uint32_t nsel = ldx<P>(&c->nsel);
    for (uint32_t i = threadIdx.x; i < kMaxK; i += blockDim.x) s_acc[i] = 0;
    __syncthreads();
    const uint32_t nvc = min(ldx<P>(&c->nvc), s.cap);
    for (uint32_t i = threadIdx.x; i < nvc; i += blockDim.x) {
      const uint32_t pr = s.vcl[i];
      atomicOr(&s_acc[pr >> kNodeBits], uint32_t(ldx<P>(reinterpret_cast<const uint8_t*>(s.vis) + (pr & kNodeMask))));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t nm = 0;
      for (uint32_t gi = 0; gi < nsel; ++gi) {
        if (!c->matched[gi] && (s_acc[gi] & full) == full) { c->matched[gi] = 1; c->sm[gi] = uint8_t(l); }
        nm += c->matched[gi];
      }
      c->n_matched = nm;
      if (nm < nsel && nm >= uint32_t(q.k)) c->rpg_stop = theorem4_stop(c, c->matched, c->sm, q, nsel, l) ? 1u : 0u;
    }
  }

  // Central run: when the CGs found so far plus the nodes the last expansion
  // completed reach w, the run stops at this level, so the level only needs
  // its identification: no work items, no retained frontier.
  const bool ident_only = run == 0 && ldx<P>(&c->ncg_at) + ldx<P>(&c->cg_next[p]) >= uint32_t(q.w);
  // Marginal run: the V_C check of the previous level showed that the run
  // stops at this level, and the RPG match above is all of its
  // identification that can change the results (the PTC stops and work
  // items of a level that is not expanded are never used): count Q_l only.
  const bool count_only = run == 1 && l > 0 && ldx<P>(&c->skip_lvl) == l;
  if (pt.b == 0 && threadIdx.x == 0) c->cg_next[p ^ 1] = 0;   // counted by k_expand of this level
  const uint32_t fq_n = ldx<P>(&c->fq_n[p]);
  const bool sparse = enqueue_sparse<P>(s, c, p);
  // The next level's queue is kept only while this level is sparse (a dense
  // level is usually followed by a dense one, and its appends would all
  // contend on one counter).  Every block computes the same `sparse` from
  // values no kernel changes during this level; k_expand reads fq_use.
  if (pt.b == 0 && threadIdx.x == 0) {
    c->fq_use[p ^ 1] = sparse ? 1u : 0u;
    if (s.lrec && sparse) s.lrec[run * kLogLevels + l].flags |= kLvlQueue;
  }
  const uint32_t nwords = (uint32_t(g.n) + 31u) >> 5;
  const uint32_t nsrc = sparse ? fq_n : nwords * 32u;   // candidate slots
  // slots per block tile: one round per thread for the queue (short frontiers
  // spread over many blocks), kEnqRounds words per warp for the bitmap
  const uint32_t kTile = sparse ? uint32_t(kEnqThreads) : uint32_t(kEnqThreads * kEnqRounds);
  uint32_t qcount = 0;
  uint64_t eact = 0;                                   // E_act of this level (Algorithm 1's activations)
  for (uint32_t tile = pt.b * kTile; tile < nsrc; tile += pt.n * kTile) {
    uint32_t it_seg[kEnqRounds], it_len[kEnqRounds], it_msk[kEnqRounds];
    // Candidate node of each round.  Queue mode: entry tile + threadIdx, one
    // round.  Bit-map mode: the warp owns words w0 .. w0 + kEnqRounds - 1 of
    // F_l and packs their set bits onto its lanes, the k-th frontier node of
    // the warp going to round k / 32, lane k % 32: a warp runs one round per
    // 32 frontier nodes instead of one per word, so on a level where a few
    // bits in ten are set most rounds are not run at all.
    constexpr uint32_t kNone = 0xffffffffu;            // no node in this round and lane
    uint32_t cand[kEnqRounds];
    uint32_t total = 0;                                // the warp's frontier nodes (bit-map mode)
    const uint32_t w0 = tile / 32u + warp * kEnqRounds;
    if (sparse) {
      const uint32_t i = tile + threadIdx.x;
      cand[0] = i < nsrc ? ldx<P>(s.fq[p] + i) : kNone;
#pragma unroll
      for (int r = 1; r < kEnqRounds; ++r) cand[r] = kNone;
    } else {
      uint32_t wd[kEnqRounds], wpre[kEnqRounds + 1];   // the warp's words and their prefix counts
      wpre[0] = 0;
#pragma unroll
      for (int r = 0; r < kEnqRounds; ++r) {
        wd[r] = w0 + r < nwords ? ldx<P>(Fc + w0 + r) : 0u;
        wpre[r + 1] = wpre[r] + __popc(wd[r]);
      }
#pragma unroll
      for (int r = 0; r < kEnqRounds; ++r)
        if (lane == uint32_t(r) && wd[r]) Fc[w0 + r] = 0;   // reset F for its next use
      total = wpre[kEnqRounds];
#pragma unroll
      for (int r = 0; r < kEnqRounds; ++r) {
        const uint32_t k = uint32_t(r) * 32u + lane;
        uint32_t word = wd[0], base = 0, ww = 0;
#pragma unroll
        for (int x = 1; x < kEnqRounds; ++x)
          if (k >= wpre[x]) { word = wd[x]; base = wpre[x]; ww = uint32_t(x); }
        cand[r] = k < total ? (w0 + ww) * 32u + nth_set_bit(word, k - base) : kNone;
      }
    }
    // rounds this warp runs (the same in every lane)
    const uint32_t nr = sparse ? 1u : (total + 31u) >> 5;
    uint32_t my_items = 0, my_work = 0;
#pragma unroll
    for (int r = 0; r < kEnqRounds; ++r) {
      it_len[r] = 0;
      it_seg[r] = 0; it_msk[r] = 0;
      if (uint32_t(r) >= nr) continue;                 // the same in every lane
      const bool has = cand[r] != kNone && RPQ_IN_BOUNDS(cand[r] < uint32_t(g.n), &c->err);
      if (!__any_sync(0xffffffffu, has)) continue;
      const uint32_t v = has ? cand[r] : 0u;
      if (sparse && has) Fc[v >> 5] = 0;               // every set bit of F_l is in the queue
      qcount += has;
      if (s.qlog && has) {
        const uint32_t pq = atomicAdd(&c->qlog_n, 1u);
        if (pq < s.qcap) s.qlog[pq] = (l << kNodeBits) | v; else atomicOr(&c->err, kErrOverflow);
      }
      if (count_only) continue;                        // the same in every lane
      bool expand = false, is_cg = false, stop_now = false;
      uint32_t cg_key = 0;
      uint8_t eq = 0, lt = 0;
      // every load of the node first (they are independent), then the logic
      uint32_t cfw = 0, vb = 0, seen = 0, rb = 0, re = 0, o_lo = 0, o_hi = 0;
      if (has) {
        cfw = ldx<P>(s.cf + (v >> 5));
        vb = ldx<P>(reinterpret_cast<const uint8_t*>(s.vis) + v);
        seen = ldx<P>(s.vseen + v);
        if (!ident_only) {
          rb = g.row_ptr[v];
          re = g.row_ptr[v + 1];
          if (l + 1 <= kLvxLevels) o_hi = g.lvx[size_t(l) * size_t(g.n) + v];
          if (l >= 1 && l <= kLvxLevels) o_lo = g.lvx[size_t(l - 1) * size_t(g.n) + v];
        }
      }
      // Columns claimed since this node was last enqueued were reached at
      // this level: their hit level is l, written here once.  The columns it
      // had been seen with were reached earlier (h < l).  So the split the
      // expansion needs, h == l versus h < l, comes from the seen byte, and no
      // hit level is read.
      const uint32_t fresh = has ? (vb & ~seen & full) : 0u;
      if (fresh) {
#pragma unroll
        for (int j = 0; j < nt; ++j)
          if ((fresh >> j) & 1u) hcol(q, j)[v] = uint8_t(l);
        s.vseen[v] = uint8_t(vb);
      }
      if (has && !((cfw >> (v & 31u)) & 1u)) {
        eq = uint8_t(fresh);
        lt = uint8_t(vb & seen & full);
        if ((vb & full) == full && (run == 0 || nt >= 2)) {
          s.stopl[v] = uint8_t(l);
          stop_now = true;
          if (run == 0) {
            // a node is identified at the level its last column arrives
            // (it is in the frontier of that level), so S^c = max_j h = l
            // (Theorem 3)
            is_cg = true;
            cg_key = (l << kNodeBits) | uint32_t(g.ext_of[v]);   // ranked by (S^c, caller id)
            if (!fresh) atomicOr(&c->err, kErrInternal);
          }
        } else {
          expand = !ident_only;
        }
      }
      const unsigned cgb = __ballot_sync(0xffffffffu, is_cg);
      if (cgb) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&c->ncg, uint32_t(__popc(cgb)));
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t at = base + __popc(cgb & ((1u << lane) - 1u));
        if (is_cg && RPQ_IN_BOUNDS(at < s.cap, &c->err)) s.cg[at] = cg_key;
      }
      bool retain = false;
      if (expand) {
        if (re - rb > kLvxMaxDeg) {                     // a hub: o_hi / o_lo hold its number
          if (l + 1 <= kLvxLevels) o_hi = g.lvx_long[size_t(o_hi) * kLvxLevels + l];
          if (l >= 1 && l <= kLvxLevels) o_lo = g.lvx_long[size_t(o_lo) * kLvxLevels + (l - 1)];
        }
        const uint32_t hi = l + 1 <= kLvxLevels ? rb + o_hi : seg_lower(g.adj, rb, re, l + 1u);
        const uint32_t lo = eq ? rb : (l == 0 ? rb : (l <= kLvxLevels ? rb + o_lo : seg_lower(g.adj, rb, hi, l)));
        retain = hi < re;                              // an edge with a > l remains
        if (hi > lo) {
          it_seg[r] = lo; it_len[r] = hi - lo; it_msk[r] = uint32_t(eq) | (uint32_t(lt) << 8);
          ++my_items;
          my_work += hi - lo;
          // every eq column activates the prefix a <= l, every lt column the segment a == l
          uint32_t seg_l = lo;
          if (eq && lt) seg_l = l == 0 ? rb : (l <= kLvxLevels ? rb + o_lo : seg_lower(g.adj, rb, hi, l));
          eact += uint64_t(__popc(eq)) * (hi - rb) + uint64_t(__popc(lt)) * (hi - seg_l);
        }
      }
      if (sparse) {                                     // nodes of a warp lie in different words
        if (stop_now) atomicOr(s.cf + (v >> 5), 1u << (v & 31u));
        if (retain) atomicOr(Fn + (v >> 5), 1u << (v & 31u));
      } else {                                          // the warp owns words w0..: one update each
        // this round's nodes lie in the words of its first and last lanes with a node
        const uint32_t bit = 1u << (v & 31u), mw = v >> 5;
        const uint32_t last = min(31u, total - 1u - uint32_t(r) * 32u);
        const uint32_t wf = __shfl_sync(0xffffffffu, mw, 0), wl = __shfl_sync(0xffffffffu, mw, last);
        for (uint32_t x = wf; x <= wl; ++x) {
          const uint32_t sb = __reduce_or_sync(0xffffffffu, (stop_now && mw == x) ? bit : 0u);
          const uint32_t rbm = __reduce_or_sync(0xffffffffu, (retain && mw == x) ? bit : 0u);
          if (lane == 0 && sb) atomicOr(s.cf + x, sb);
          if (lane == 0 && rbm) atomicOr(Fn + x, rbm);   // F_{l+1} is empty before this level
        }
      }
      queue_push(s, c, p ^ 1, sparse, retain, v);
    }
    if (!__syncthreads_or(my_items != 0)) continue;    // no item in this tile
    const uint64_t packed = (uint64_t(my_items) << kWorkBits) | my_work;
    uint64_t tot = 0;
    const uint64_t pre = block_excl_scan(packed, s_warp, &tot);
    if (threadIdx.x == 0) s_base = atomicAdd(&c->work[p], (unsigned long long)tot);
    __syncthreads();
    {
      uint32_t idx = uint32_t((s_base >> kWorkBits) + (pre >> kWorkBits));
      uint32_t off = uint32_t((s_base & kWorkMask) + (pre & kWorkMask));
#pragma unroll
      for (int r = 0; r < kEnqRounds; ++r) {           // every lane runs every round (warp-wide fill)
        if (uint32_t(r) >= nr) break;                  // the same in every lane
        const bool has = it_len[r] != 0;
        uint32_t t0 = 1, t1 = 0;                       // warp tiles starting inside the item
        if (has) {
          Item it;
          it.seg_begin = it_seg[r];
          it.off = off;
          if (RPQ_IN_BOUNDS(idx < s.cap, &c->err)) {
            s.items[idx] = it;
            s.imask[idx] = uint16_t(it_msk[r]);
          }
          t0 = (off + kWarpTile - 1) / kWarpTile;
          t1 = (off + it_len[r] - 1) / kWarpTile;
        }
        const bool big = t0 + 2 <= t1;                 // three or more tiles: filled by the warp
        if (!big) {
          for (uint32_t t = t0; t <= t1; ++t) {
            if (t < s.tile_cap) s.tile_first[t] = idx; else atomicOr(&c->err, kErrOverflow);
          }
        }
        for (unsigned bb = __ballot_sync(0xffffffffu, big); bb; bb &= bb - 1) {
          const int src = __ffs(int(bb)) - 1;
          const uint32_t f0 = __shfl_sync(0xffffffffu, t0, src), f1 = __shfl_sync(0xffffffffu, t1, src);
          const uint32_t fi = __shfl_sync(0xffffffffu, idx, src);
          for (uint32_t t = f0 + lane; t <= f1; t += 32u) {
            if (t < s.tile_cap) s.tile_first[t] = fi; else atomicOr(&c->err, kErrOverflow);
          }
        }
        if (has) {
          ++idx;
          off += it_len[r];
        }
      }
    }
    __syncthreads();
  }
  const uint64_t qt = block_sum(qcount, s_warp);
  const uint64_t et = block_sum(eact, s_warp);
  if (threadIdx.x == 0 && qt) atomicAdd(&c->nq[p], uint32_t(qt));
  if (threadIdx.x == 0 && et) atomicAdd(&c->eact_lvl[p], (unsigned long long)et);
}

// The enqueue of the run's column count (the same in every thread).
template <bool P>
__device__ __forceinline__ void enqueue_columns(const DevKG& g, const DevSlot& s, int run, uint32_t l, Part pt) {
  const QueryDev& q = *s.q;
  __shared__ EnqShared sh;
  switch (run == 0 ? q.n_c : q.n_m) {
    case 1: enqueue_level<P, 1>(g, s, run, l, pt, sh); break;
    case 2: enqueue_level<P, 2>(g, s, run, l, pt, sh); break;
    case 3: enqueue_level<P, 3>(g, s, run, l, pt, sh); break;
    case 4: enqueue_level<P, 4>(g, s, run, l, pt, sh); break;
    case 5: enqueue_level<P, 5>(g, s, run, l, pt, sh); break;
    case 6: enqueue_level<P, 6>(g, s, run, l, pt, sh); break;
    case 7: enqueue_level<P, 7>(g, s, run, l, pt, sh); break;
    default: enqueue_level<P, kMaxCols>(g, s, run, l, pt, sh); break;
  }
}

template <bool P>
__device__ __forceinline__ void enqueue_body(const DevKG& g, const DevSlot& s, int run, Part pt) {
  Ctl* c = s.ctl;
  const bool done = ldx<P>(&c->done) != 0;
  if (pt.b == 0 && threadIdx.x == 0) c->exp_skip = done ? 1u : 0u;   // read by this level's k_expand
  if (done) return;
  const uint32_t l = ldx<P>(&c->lvl_enq);
  if (pt.b == 0 && threadIdx.x == 0) c->lvl_exp = l;
  enqueue_columns<P>(g, s, run, l, pt);
}

__global__ void __launch_bounds__(kEnqThreads, 6)      // at most 40 registers: 6 blocks per SM
k_enqueue(DevKG g, DevSlot s, int run) {
  enqueue_body<false>(g, s, run, launch_part());
}

// ------------------------------------------- level: V_C check (marginal run)
// Between the enqueue and the expansion of marginal Glevel l.  The first hits
// of level l+1 on the V_C nodes of still unmatched CGs are found from the
// receiving side: node v is first hit in column j at l+1 exactly when some
// neighbour u expands to it at level l, i.e. u was reached with
// max(h_uj, a_uv) = l and u had not stopped by then (Algorithm 1,
// Definition 8; the levels are symmetric; u's levels of the columns reached
// by level l were written by the enqueues up to this level's).  One warp per
// (V_C node, column) scans v's entries with a <= l and stops at the first
// such u; the scan writes nothing.  The last block to finish applies the
// hits (visited bit, F_{l+1} and the frontier queue of l+1 when it is in
// use, as a claim of the expansion would; and h = l+1, which the next
// enqueue writes again) and runs the identification of level l+1 on V_C
// alone.  When that shows the run stops at l+1 (every
// selected CG matched, Theorem 4, or l+1 = L) and some hit was applied (so
// Q_{l+1} is not empty), nothing else the expansion of level l would compute
// can reach the results, and k_expand skips it.  Levels with fewer than
// tgt_min_work work units, and queries whose V_C holds more than
// kTgtMaxTasks (node, column) pairs (keywords on hundreds of thousands of
// nodes: the single block applying the hits would dominate), are left alone.
// Off in trace mode, where every frontier is compared.
// Whether the V_C check runs at the current marginal Glevel: not when the
// run ends at this level anyway (the stop test of the expansion), nor when
// the level is too small for a skip to pay for the check.
template <bool P>
__device__ __forceinline__ bool target_runs(const DevSlot& s) {
  const Ctl* c = s.ctl;
  if (ldx<P>(&c->done) || !s.target) return false;
  const QueryDev& q = *s.q;
  const uint32_t l = ldx<P>(&c->lvl_exp);
  const int p = int(l & 1u);
  const int nm = q.n_m;
  if (nm == 0 || ldx<P>(&c->nq[p]) == 0 || ldx<P>(&c->n_matched) >= ldx<P>(&c->nsel) || ldx<P>(&c->rpg_stop) ||
      l >= uint32_t(q.L))
    return false;
  return (ldx<P>(&c->work[p]) & kWorkMask) >= s.tgt_min_work &&
         min(ldx<P>(&c->nvc), s.cap) * uint32_t(nm) <= kTgtMaxTasks;
}

__device__ __forceinline__ void target_body(const DevKG& g, const DevSlot& s, Part pt) {
  Ctl* c = s.ctl;
  if (!target_runs<false>(s)) return;
  const QueryDev& q = *s.q;
  const uint32_t l = c->lvl_exp;
  const int p = int(l & 1u);
  const uint32_t nsel = c->nsel;
  const int nm = q.n_m;
  const uint32_t nvc = min(c->nvc, s.cap);
  const uint32_t ntask = nvc * uint32_t(nm);
  const uint32_t lane = lane_id();
  const uint32_t gw = (pt.b * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (pt.n * blockDim.x) >> 5;
  for (uint32_t t = gw; t < ntask; t += nwarps) {
    const uint32_t pr = s.vcl[t / uint32_t(nm)];
    const uint32_t j = t % uint32_t(nm);
    const uint32_t gi = pr >> kNodeBits, v = pr & kNodeMask;
    if (!RPQ_IN_BOUNDS(v < uint32_t(g.n) && gi < uint32_t(kMaxK), &c->err)) continue;   // same in every lane
    if (c->matched[gi] || ((vis_byte(s.vis, v) >> j) & 1u)) continue;   // same in every lane
    const uint32_t rb = g.row_ptr[v];
    const uint32_t hi = seg_at(g, v, rb, g.row_ptr[v + 1], l + 1);      // entries with a <= l
    bool found = false;
    for (uint32_t e0 = rb; e0 < hi && !found; e0 += 32u) {
      const uint32_t e = e0 + lane;
      bool par = false;
      if (e < hi) {
        const uint32_t x = __ldg(g.adj + e);
        const uint32_t a = x >> kNodeBits, u0 = x & kNodeMask;
        const bool ok = RPQ_IN_BOUNDS(u0 < uint32_t(g.n), &c->err);
        const uint32_t u = ok ? u0 : 0u;
        const uint32_t vb = vis_byte(s.vis, u), hu = hcol(q, int(j))[u];
        const uint32_t cfw = s.cf[u >> 5], stl = s.stopl[u];
        if (ok && ((vb >> j) & 1u)) {
          const uint32_t lam = a > hu ? a : hu;
          par = lam == l && !(((cfw >> (u & 31u)) & 1u) && stl <= l);
        }
      }
      found = __any_sync(0xffffffffu, par);
    }
    if (found && lane == 0) {
      const uint32_t i = atomicAdd(&c->tgt_n, 1u);
      if (i < s.tgt_cap) s.tgt[i] = (j << kNodeBits) | v;
    }
  }
  __shared__ uint32_t s_last, s_hits;
  __shared__ uint32_t s_acc[kMaxK];
  __shared__ uint8_t s_matched[kMaxK], s_sm[kMaxK];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&c->tgt_done, 1u) == pt.n - 1u ? 1u : 0u;
    s_hits = 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const uint32_t nf = __ldcg(&c->tgt_n);
  const bool over = nf > s.tgt_cap;                     // too many to list: expand in full
  uint32_t* Fn = s.F[p ^ 1];
  const bool push = __ldcg(&c->fq_use[p ^ 1]) != 0;
  uint32_t hits = 0;
  for (uint32_t i = threadIdx.x; !over && i < nf; i += blockDim.x) {
    const uint32_t x = __ldcg(s.tgt + i), j = x >> kNodeBits, v = x & kNodeMask;
    hcol(q, int(j))[v] = uint8_t(l + 1);                 // a repeated (node, column) writes the same value
    const uint32_t old = atomicOr(s.vis + (v >> 2), (1u << j) << ((v & 3u) * 8u));
    if ((old >> ((v & 3u) * 8u + j)) & 1u) continue;
    ++hits;
    const uint32_t of = atomicOr(Fn + (v >> 5), 1u << (v & 31u));
    if (push && !((of >> (v & 31u)) & 1u) && !__ldcg(&c->fq_over[p ^ 1])) {
      const uint32_t b = atomicAdd(&c->fq_n[p ^ 1], 1u);
      if (b + 1u > s.fq_limit) atomicExch(&c->fq_over[p ^ 1], 1u); else s.fq[p ^ 1][b] = v;
    }
  }
  if (hits) atomicAdd(&s_hits, hits);
  for (uint32_t i = threadIdx.x; i < uint32_t(kMaxK); i += blockDim.x) s_acc[i] = 0;
  __syncthreads();
  // identification of level l+1 restricted to V_C (the RPG match of k_enqueue)
  for (uint32_t i = threadIdx.x; i < nvc; i += blockDim.x) {
    const uint32_t pr = s.vcl[i];
    atomicOr(&s_acc[pr >> kNodeBits], uint32_t(__ldcg(reinterpret_cast<const uint8_t*>(s.vis) + (pr & kNodeMask))));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t full = (1u << nm) - 1u;
    uint32_t cnt = 0;
    for (uint32_t gi = 0; gi < nsel; ++gi) {
      const bool was = c->matched[gi] != 0;
      s_matched[gi] = (was || (s_acc[gi] & full) == full) ? 1 : 0;
      s_sm[gi] = was ? c->sm[gi] : uint8_t(l + 1);
      cnt += s_matched[gi];
    }
    const bool stop_next = l + 1 >= uint32_t(q.L) || cnt >= nsel ||
                           (cnt >= uint32_t(q.k) && theorem4_stop(c, s_matched, s_sm, q, nsel, l + 1));
    if (!over && s_hits && stop_next) c->skip_lvl = l + 1;
    c->tgt_n = 0;
    c->tgt_done = 0;
  }
}

__global__ void __launch_bounds__(kTgtThreads) k_target(DevKG g, DevSlot s) { target_body(g, s, launch_part()); }

// ----------------------------------------------------------- level: expand
// Termination (every block reaches the same decision from the control block,
// which k_enqueue finished writing) and expansion (Algorithm 1) of the work
// items.  The work units (one per CSR entry of an item's segment) are cut
// into warp tiles of kWarpTile consecutive units: a hub's segment spans many
// tiles (split over the whole grid), short segments share a tile, and the 32
// lanes of each round read 32 consecutive CSR entries.  Each lane finds its
// item from a window of 32 items held in registers (one per lane): the item
// starts inside the round are OR-reduced into a bit mask and a popcount
// gives the lane's item, so no barrier and no search are needed.  When the
// kernel runs inside a graph WHILE node, block 0 ends the loop as the run stops.
template <bool P>
__device__ __forceinline__ void load_window(const Item* items, const uint16_t* imask, uint32_t n_items, uint32_t wb,
                                            uint32_t lane, uint32_t& woff, uint32_t& wseg, uint32_t& wmsk) {
  const uint32_t j = wb + lane;
  if (j < n_items) {
    const uint2 raw = ldx<P>(reinterpret_cast<const uint2*>(items + j));
    wseg = raw.x;
    woff = raw.y;
    wmsk = ldx<P>(imask + j);
  } else {
    woff = 0xffffffffu; wseg = 0; wmsk = 0;
  }
}

// First hits of a finished run: the (node, column) pairs its visited bits
// hold, less the seeds (h = 0).  Every block of the stopping launch takes a
// share of the visited words; the expansions themselves count no hits.
template <bool P>
__device__ void count_hits(const DevKG& g, const DevSlot& s, int run, uint64_t* s_warp, Part pt) {
  Ctl* c = s.ctl;
  const int nt = run == 0 ? s.q->n_c : s.q->n_m;
  const uint32_t colmask = ((1u << nt) - 1u) * 0x01010101u;      // the run's columns in each byte
  const uint32_t nwords = (uint32_t(g.n) + 3u) >> 2;
  uint64_t cnt = 0;
  for (uint32_t i = pt.b * blockDim.x + threadIdx.x; i < nwords; i += pt.n * blockDim.x)
    cnt += __popc(ldx<P>(s.vis + i) & colmask);
  const uint64_t tot = block_sum(cnt, s_warp);
  if (threadIdx.x == 0) {
    unsigned long long add = tot;
    if (pt.b == 0) add -= ldx<P>(&c->seeded[run]);        // modulo 2^64: the sum comes out right
    if (add) atomicAdd(&c->hits[run], add);
  }
}

// Termination decision of Glevel l, the same in every block (from the
// control block, which the enqueue and the V_C check finished writing): the
// run stops (empty frontier, enough CGs or every selected CG matched or
// Theorem 4, or l = L), or the V_C check showed that the V_C nodes alone
// decide the outcome at level l+1 (skip), else the level's work is expanded.
struct LevelPlan {
  bool stop, skip;
  uint32_t nq, n_items, n_work;
};
template <bool P>
__device__ __forceinline__ LevelPlan level_plan(const DevSlot& s, int run, uint32_t l) {
  const Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const int p = int(l & 1u);
  LevelPlan r;
  const unsigned long long wk = ldx<P>(&c->work[p]);
  r.n_items = uint32_t(wk >> kWorkBits);
  r.n_work = uint32_t(wk & kWorkMask);
  r.nq = ldx<P>(&c->nq[p]);
  const bool term = run == 0 ? (ldx<P>(&c->ncg) >= uint32_t(q.w))
                             : (ldx<P>(&c->n_matched) >= ldx<P>(&c->nsel) || ldx<P>(&c->rpg_stop));
  r.stop = (r.nq == 0) || term || (l >= uint32_t(q.L));
  r.skip = !r.stop && ldx<P>(&c->skip_lvl) == l + 1;
  return r;
}

// Returns true when the run stops at level l (no expansion then).
template <bool P>
__device__ __forceinline__ bool expand_level(const DevKG& g, const DevSlot& s, int run, uint32_t l,
                                             cudaGraphConditionalHandle loop, int in_graph, Part pt) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const int p = int(l & 1u);
  const LevelPlan plan = level_plan<P>(s, run, l);
  const uint32_t n_items = plan.n_items, n_work = plan.n_work, nq = plan.nq;
  const bool stop = plan.stop, skip = plan.skip;
  if (pt.b == 0 && threadIdx.x == 0) {
    c->level = l;
    c->frontier += nq;
    const unsigned long long ea = ldx<P>(&c->eact_lvl[p]);   // enqueued activations of this level
    c->eact_lvl[p] = 0;
    if (s.lrec) {                                  // profiling: the level's work
      LevelRec& lr = s.lrec[run * kLogLevels + l];
      const bool ran = !stop && !skip;
      lr.frontier = nq;
      lr.units = ran ? n_work : 0;
      lr.items = ran ? n_items : 0;
      lr.eact = ran ? ea : 0;
      lr.flags |= stop ? kLvlStop : (skip ? kLvlSkipped : kLvlExpanded);
    }
    if (stop) {
      c->done = 1;
      c->levels[run] = (nq == 0 && l > 0) ? int32_t(l) - 1 : int32_t(l);
      if (in_graph) cudaGraphSetConditional(loop, 0);
    } else {
      c->e_act[run] += ea;
      c->ncg_at = c->ncg;                            // CGs through level l (read by the next enqueue)
      if (skip) {
        c->e_act_skip += ea;
      } else {
        c->units += n_work;
        c->items += n_items;
      }
      c->last_expanded = int32_t(l);
      c->levels[run] = int32_t(l);   // provisional; final when the run stops
      c->lvl_enq = l + 1;
      c->work[p ^ 1] = 0;            // counters of level l+1 (nothing reads them now)
      c->nq[p ^ 1] = 0;
      c->fq_n[p] = 0;                // queue of level l was consumed by k_enqueue
      c->fq_over[p] = 0;
    }
  }
  __shared__ uint64_t s_warp[33];
  if (stop) count_hits<P>(g, s, run, s_warp, pt);
  if (stop && run == 1 && pt.b == 0) write_results(s);   // the marginal run ends here
  if (stop || skip || n_work == 0) return stop;

  uint32_t* Fn = s.F[p ^ 1];
  // The next level's queue (started by k_enqueue of this level) is kept only
  // if this level's work is small; a large level would overflow it anyway and
  // its appends would contend on one counter.
  const uint32_t fq_use_next = ldx<P>(&c->fq_use[p ^ 1]);
  const bool use_next = fq_use_next != 0 && uint64_t(n_work) <= uint64_t(s.fq_next_mult) * s.fq_limit;
  if (fq_use_next && !use_next && pt.b == 0 && threadIdx.x == 0) c->fq_over[p ^ 1] = 1;
  const uint32_t lane = lane_id();
  const uint32_t gw = (pt.b * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (pt.n * blockDim.x) >> 5;
  const uint32_t ntiles = (n_work + kWarpTile - 1) / kWarpTile;
  uint64_t claims = 0, completed = 0;                // completed: nodes that now hold every central column
  const uint32_t fullc = run == 0 ? (1u << q.n_c) - 1u : 0x100u;
  for (uint32_t t = gw; t < ntiles; t += nwarps) {
    if (!RPQ_IN_BOUNDS(t < s.tile_cap, &c->err)) break;   // the same in every lane
    const uint32_t t0 = t * kWarpTile;
    const uint32_t t1 = min(t0 + uint32_t(kWarpTile), n_work);
    uint32_t wb = ldx<P>(s.tile_first + t);
    uint32_t woff, wseg, wmsk;
    load_window<P>(s.items, s.imask, n_items, wb, lane, woff, wseg, wmsk);
    uint32_t e_r[kExpRounds], m_r[kExpRounds];
    bool v_r[kExpRounds];
#pragma unroll
    for (int r = 0; r < kExpRounds; ++r) {
      const uint32_t u0 = t0 + 32u * r;
      v_r[r] = false; e_r[r] = 0; m_r[r] = 0;
      if (u0 >= t1) continue;                      // same in every lane
      for (;;) {                                   // lane 0 must hold the item containing u0
        const unsigned le = __ballot_sync(0xffffffffu, woff <= u0);
        const int hb = 31 - __clz(le);
        if (hb == 0) break;
        wb += uint32_t(hb);
        load_window<P>(s.items, s.imask, n_items, wb, lane, woff, wseg, wmsk);
      }
      const uint32_t bit = (lane > 0 && woff < u0 + 32u) ? (1u << (woff - u0)) : 0u;
      const uint32_t starts = __reduce_or_sync(0xffffffffu, bit);
      const int k = __popc(starts & (0xffffffffu >> (31u - lane)));
      const uint32_t off = __shfl_sync(0xffffffffu, woff, k);
      const uint32_t seg = __shfl_sync(0xffffffffu, wseg, k);
      const uint32_t msk = __shfl_sync(0xffffffffu, wmsk, k);
      const uint32_t u = u0 + lane;
      if (u < t1 && RPQ_IN_BOUNDS(seg + (u - off) < g.m2, &c->err)) { e_r[r] = seg + (u - off); m_r[r] = msk; v_r[r] = true; }
    }
    uint32_t x_r[kExpRounds];
#pragma unroll
    // the adjacency is streamed (each entry read once per level): evict-first,
    // so that it does not push the visited and frontier lines out of L2
    for (int r = 0; r < kExpRounds; ++r) x_r[r] = v_r[r] ? __ldcs(g.adj + e_r[r]) : 0u;
#ifdef RPQ_CHECKED
    for (int r = 0; r < kExpRounds; ++r)
      if (v_r[r] && !RPQ_IN_BOUNDS((x_r[r] & kNodeMask) < uint32_t(g.n), &c->err)) v_r[r] = false;
#endif
    uint32_t vb_r[kExpRounds];
#pragma unroll
    for (int r = 0; r < kExpRounds; ++r) vb_r[r] = v_r[r] ? vis_byte(s.vis, x_r[r] & kNodeMask) : 0xffu;
    // candidate new columns of every round, then all atomics in flight together
    uint32_t nw_r[kExpRounds];
#pragma unroll
    for (int r = 0; r < kExpRounds; ++r) {
      nw_r[r] = 0;
      if (!v_r[r]) continue;
      const uint32_t a = x_r[r] >> kNodeBits;
      const uint32_t eq = m_r[r] & 0xffu, lt = m_r[r] >> 8;
      const uint32_t act = a < l ? eq : (eq | lt);   // columns for which the edge is new at level l
      nw_r[r] = act & ~vb_r[r];
    }
    // Claims: the visited and frontier bits of every column found unreached,
    // by reductions (the level l+1 is written by the next enqueue).  A
    // returning atomic only where its old
    // value is used: when this claim may complete a central node (the count
    // lets the next enqueue skip its work items if the run stops there; a
    // completion whose claims all looked incomplete is not counted, which
    // only forgoes that saving), and for the frontier bit while the next
    // level's queue is filled (a node is queued once).
#pragma unroll
    for (int r = 0; r < kExpRounds; ++r) {
      bool fresh = false;
      const uint32_t nb = x_r[r] & kNodeMask;
      const uint32_t nw = nw_r[r];
      if (nw) {
        const uint32_t sh = (nb & 3u) * 8u;
        if (((vb_r[r] | nw) & fullc) == fullc) {
          const uint32_t ob = (atomicOr(s.vis + (nb >> 2), nw << sh) >> sh) & 0xffu;
          completed += (ob & fullc) != fullc && ((ob | nw) & fullc) == fullc;   // one claim completes the node
        } else {
          atomicOr(s.vis + (nb >> 2), nw << sh);       // result unused: a reduction
        }
        if (use_next) {
          const uint32_t of = atomicOr(Fn + (nb >> 5), 1u << (nb & 31u));
          fresh = !((of >> (nb & 31u)) & 1u);
        } else {
          atomicOr(Fn + (nb >> 5), 1u << (nb & 31u));
        }
        claims += __popc(nw);
      }
      queue_push(s, c, p ^ 1, use_next, fresh, nb);
    }
  }
  const uint64_t cc = block_sum(claims | (completed << 40), s_warp);   // both counts in one reduction
  const uint64_t tcl = cc & ((1ull << 40) - 1ull), tc = cc >> 40;
  if (threadIdx.x == 0 && tc) atomicAdd(&c->cg_next[p ^ 1], uint32_t(tc));
  if (threadIdx.x == 0 && tcl && s.lrec) atomicAdd(&s.lrec[run * kLogLevels + l].claims, (unsigned long long)tcl);
  return false;
}

template <bool P>
__device__ __forceinline__ void expand_body(const DevKG& g, const DevSlot& s, int run, cudaGraphConditionalHandle loop,
                                            int in_graph, Part pt) {
  Ctl* c = s.ctl;
  if (pt.b == 0 && threadIdx.x == 0) c->iters[run] += 1;
  // exp_skip, not done: block 0 of the launch that stops the run sets done
  // while other blocks of that launch may still be starting, and they too
  // must take the stop path (their share of the hit count)
  if (ldx<P>(&c->exp_skip)) {
    if (in_graph && pt.b == 0 && threadIdx.x == 0) cudaGraphSetConditional(loop, 0);
    return;
  }
  expand_level<P>(g, s, run, ldx<P>(&c->lvl_exp), loop, in_graph, pt);
}

__global__ void __launch_bounds__(kExpThreads)
k_expand(DevKG g, DevSlot s, int run, cudaGraphConditionalHandle loop, int in_graph) {
  expand_body<false>(g, s, run, loop, in_graph, launch_part());
}

// ------------------------------------------------------ persistent run kernel
// All Glevels of one run in one cooperative launch (every block resident):
// the enqueue and expansion phases of a level are separated by a grid
// barrier instead of a kernel boundary.  The barrier is bounded: a block that
// waits longer than the slot's bar_limit clock cycles (about 1 s by default)
// sets kErrTimeout and every block leaves the kernel at its next barrier, so
// the kernel always ends.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, uint32_t* err, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g0 = *(volatile unsigned*)gen;
    __threadfence();
    if (atomicAdd(count, 1u) + 1u == nblocks) {
      *(volatile unsigned*)count = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*(volatile unsigned*)gen == g0) {
        if (*(volatile uint32_t*)err & kErrTimeout) { ok = 0; break; }
        if (clock64() - t0 > limit) { atomicOr(err, kErrTimeout); ok = 0; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kExpThreads)
k_run(DevKG g, DevSlot s, int run) {
  Ctl* c = s.ctl;
  if (c->done) return;
  for (;;) {
    const uint32_t l = *(volatile uint32_t*)&c->lvl_enq;
    if (blockIdx.x == 0 && threadIdx.x == 0) { c->lvl_exp = l; c->iters[run] += 1; }
    enqueue_columns<true>(g, s, run, l, launch_part());
    if (!grid_barrier(s.bar, s.bar + 1, gridDim.x, &c->err, s.bar_limit)) break;
    if (expand_level<true>(g, s, run, l, 0, 0, launch_part())) return;
    if (!grid_barrier(s.bar, s.bar + 1, gridDim.x, &c->err, s.bar_limit)) break;
  }
  // a barrier ran out: the run ends without results; the error reaches the
  // slot's sticky word (read by rpq_sync_device) as well as the control block
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->done = 1;
    atomicOr(s.sticky, __ldcg(&c->err));
  }
}

// ------------------------------------------------------ top-w CG selection
// One launch.  Keys are (S^c << 26) | node, so ascending order is the
// (S^c, node id) order of the selection.  Each block takes chunks of up to
// kTopkChunk CG keys and keeps the w smallest it has seen (the w-th smallest
// of a chunk is found by a radix select over the key offsets from the chunk's
// smallest key, up to 11 bits per round: two rounds when the keys share S^c
// and the node ids span up to 2^22; only keys up to it are kept); the last block
// to finish selects the w smallest of all blocks' survivors the same way,
// orders them by rank and writes the selected CGs.

// Smallest and largest valid key of keys[0..len) and their count (0xffffffff
// marks an empty entry); all threads of the block call it and get the result.
__device__ void block_key_range(const uint32_t* keys, uint32_t len, uint32_t* s_red, uint32_t& kmin,
                                uint32_t& kmax, uint32_t& cnt) {
  uint32_t mn = 0xffffffffu, mx = 0, n = 0;
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
    const uint32_t k = keys[i];
    if (k == 0xffffffffu) continue;
    mn = min(mn, k); mx = max(mx, k); ++n;
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  n = __reduce_add_sync(0xffffffffu, n);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { s_red[warp] = mn; s_red[32 + warp] = mx; s_red[64 + warp] = n; }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < nw;
    mn = __reduce_min_sync(0xffffffffu, in ? s_red[lane] : 0xffffffffu);
    mx = __reduce_max_sync(0xffffffffu, in ? s_red[32 + lane] : 0u);
    n = __reduce_add_sync(0xffffffffu, in ? s_red[64 + lane] : 0u);
    if (lane == 0) { s_red[96] = mn; s_red[97] = mx; s_red[98] = n; }
  }
  __syncthreads();
  kmin = s_red[96]; kmax = s_red[97]; cnt = s_red[98];
  __syncthreads();
}

// The K-th smallest (1-based, K <= number of valid keys) of keys[0..len),
// all of whose valid keys lie in [lo, lo + 2^span): a radix select over the
// offsets from lo, most significant digits first, up to BITS bits per round
// with a shared-memory histogram of 2^BITS bins.  All threads of the block
// call it.
template <int BITS>
__device__ uint32_t block_kth_key(const uint32_t* keys, uint32_t len, uint32_t K, uint32_t lo, uint32_t span,
                                  uint32_t* hist, uint64_t* s_warp, uint32_t* s_bin) {
  uint64_t prefix = 0;                                   // decided high bits of the offset
  uint32_t need = K;
  const uint32_t nt = blockDim.x;
#pragma unroll 1
  for (uint32_t rem = span; rem > 0;) {
    const uint32_t bits = min(rem, uint32_t(BITS)), sh = rem - bits;
    const uint32_t B = 1u << bits, per = (B + nt - 1) / nt;
    for (uint32_t i = threadIdx.x; i < B; i += nt) hist[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < len; i += nt) {
      const uint32_t k = keys[i];
      if (k == 0xffffffffu) continue;
      const uint64_t d = uint64_t(k - lo);
      if ((d >> rem) == (prefix >> rem)) atomicAdd(&hist[uint32_t(d >> sh) & (B - 1u)], 1u);
    }
    __syncthreads();
    uint32_t local = 0;
    for (uint32_t b = threadIdx.x * per; b < min(B, (threadIdx.x + 1) * per); ++b) local += hist[b];
    uint64_t tot = 0;
    uint32_t run = uint32_t(block_excl_scan(local, s_warp, &tot));
    for (uint32_t b = threadIdx.x * per; b < min(B, (threadIdx.x + 1) * per); ++b) {
      if (run < need && need <= run + hist[b]) { s_bin[0] = b; s_bin[1] = run; }
      run += hist[b];
    }
    __syncthreads();
    need -= s_bin[1];
    prefix |= uint64_t(s_bin[0]) << sh;
    rem = sh;
    __syncthreads();
  }
  return lo + uint32_t(prefix);
}

// Keep the (at most) K smallest valid keys of keys[0..len) in place; returns
// their count.  len <= PER * blockDim.x.
template <int PER, int BITS>
__device__ uint32_t block_keep_smallest(uint32_t* keys, uint32_t len, uint32_t K, uint32_t* hist,
                                        uint64_t* s_warp, uint32_t* s_bin, uint32_t* s_red) {
  if (threadIdx.x == 0) s_bin[3] = 0;
  uint32_t kmin, kmax, valid;
  block_key_range(keys, len, s_red, kmin, kmax, valid);   // ends with a barrier
  const uint32_t span = kmax > kmin ? 32u - uint32_t(__clz(kmax - kmin)) : 0u;
  const uint32_t t = valid > K ? block_kth_key<BITS>(keys, len, K, kmin, span, hist, s_warp, s_bin) : 0xfffffffeu;
  // compact keys <= t to the front (order is restored by the final ranking)
  uint32_t mine[PER];
  uint32_t nm = 0;
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
    if (keys[i] <= t) mine[nm++] = keys[i];
  __syncthreads();
  for (uint32_t r = 0; r < nm; ++r) keys[atomicAdd(&s_bin[3], 1u)] = mine[r];
  __syncthreads();
  return min(valid, K);
}

// key holds CHUNK + 2 kMaxK entries and hist 2^BITS; the block has NT threads.
template <int NT, int CHUNK, int BITS>
__device__ void topk_body(const DevKG& g, const DevSlot& s, Part pt, uint32_t* key, uint32_t* hist) {
  constexpr int PER = CHUNK / NT;
  Ctl* c = s.ctl;
  const uint32_t K = uint32_t(s.q->w);                   // beam width w
  const uint32_t n_in = min(c->ncg, s.cap);
  const uint32_t nchunks = (n_in + CHUNK - 1) / CHUNK;
  __shared__ uint64_t s_warp[33];
  __shared__ uint32_t s_bin[4];
  __shared__ uint32_t s_red[100];
  __shared__ uint32_t s_keep, s_last;
  uint32_t* keep = key + CHUNK;                          // survivors of this block (<= 2K while merging)
  if (threadIdx.x == 0) s_keep = 0;
  __syncthreads();
  for (uint32_t ch = pt.b; ch < nchunks; ch += pt.n) {
    const uint32_t b = ch * CHUNK;
    const uint32_t len = min(uint32_t(CHUNK), n_in - b);
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) key[i] = s.cg[b + i];
    __syncthreads();
    const uint32_t m = block_keep_smallest<PER, BITS>(key, len, K, hist, s_warp, s_bin, s_red);
    // merge with the survivors of earlier chunks
    const uint32_t k0 = s_keep;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) keep[k0 + i] = key[i];
    __syncthreads();
    const uint32_t mm = block_keep_smallest<PER, BITS>(keep, k0 + m, K, hist, s_warp, s_bin, s_red);
    if (threadIdx.x == 0) s_keep = mm;
    __syncthreads();
  }
  uint32_t* out = s.topk + size_t(pt.b) * K;
  for (uint32_t i = threadIdx.x; i < K; i += blockDim.x) out[i] = i < s_keep ? keep[i] : 0xffffffffu;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&c->topk_done, 1u) == pt.n - 1u ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: the K smallest of all survivors (blocks that had a chunk)
  const uint32_t nb = min(nchunks, pt.n);
  uint32_t total = 0;
  for (uint32_t blk = 0; blk < nb; ++blk) {            // gather, reducing whenever the buffer fills
    for (uint32_t i = threadIdx.x; i < K; i += blockDim.x) key[total + i] = __ldcg(s.topk + size_t(blk) * K + i);
    total += K;
    if (total + K > uint32_t(CHUNK) || blk + 1 == nb) {
      __syncthreads();
      total = block_keep_smallest<PER, BITS>(key, total, K, hist, s_warp, s_bin, s_red);
      __syncthreads();
    }
  }
  // rank the (at most K) selected keys: ascending (S^c, node id)
  __shared__ uint32_t s_sel[kMaxK];
  for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
    const uint32_t v = key[i];
    uint32_t rank = 0;
    for (uint32_t o = 0; o < total; ++o) rank += key[o] < v;
    s_sel[rank] = v;
  }
  __syncthreads();
  if (threadIdx.x < total) {
    const int32_t ext = int32_t(s_sel[threadIdx.x] & kNodeMask);
    c->sel[threadIdx.x] = ext;
    c->sel_int[threadIdx.x] = g.int_of[ext];
    c->sel_sc[threadIdx.x] = uint8_t(s_sel[threadIdx.x] >> kNodeBits);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c->nsel = total;
    c->ulist_n = 0;
    c->nvc = 0;
    c->topk_done = 0;
    __threadfence();
  }
  __syncthreads();
  if (s.q->n_m == 0 || total == 0) write_results(s);   // no marginal run follows
}

__global__ void __launch_bounds__(kTopkThreads) k_topk(DevKG g, DevSlot s) {
  __shared__ uint32_t key[kTopkChunk + 2 * kMaxK];
  __shared__ uint32_t hist[1 << kTopkBits];
  topk_body<kTopkThreads, kTopkChunk, kTopkBits>(g, s, launch_part(), key, hist);
}

// ---------------------------------------------------------------- recovery
// Recovering phase (Algorithm 2) for all selected CGs at once.  Central
// column j is swept by one thread-block cluster of kRecCluster CTAs: a
// backward sweep from the CG nodes, level by level downwards, follows the
// edges n -> q with h_q = max(a, h_n) + 1 (tight, Lemma 3) whose source n was
// still expanding at level max(a, h_n) (it had not stopped earlier).  Each
// node carries a bit mask of the CGs it belongs to, OR-ed along the tight
// edges; a node's mask is final once the level above it is done, since every
// tight edge into it starts one level higher or more.
//
// The column's node list (cap entries) holds each reached node once, filed
// when it is first reached: a node one level below the node that reached it
// (the usual case) goes into the segment of that level, the segments growing
// upwards in order of decreasing level; any other node (a CG node, or one
// reached over an edge whose activation level exceeds its own h) goes into
// the overflow part, which grows down from the end.  Level x visits its own
// segment and the overflow nodes with h = x, not the whole list.  Every CTA
// of the cluster scans those entries (the same block scan of row lengths) and
// the CSR entries are dealt round-robin over the cluster, so a hub's row is
// read by all of its CTAs at once; a cluster barrier separates the levels.
// The lists and counters live in global memory, read through L2 (__ldcg)
// because other CTAs append to them.  At the end every reached node that
// holds a central keyword ORs its column mask into the union mask (vmask),
// every column mask is cleared, and the last CTA of all columns turns the
// union masks into V_C of each CG.
// Node v holds a central keyword (h = 0 in a column it was reached in).
__device__ __forceinline__ bool holds_central(const DevSlot& s, const QueryDev& q, uint32_t v) {
  const uint32_t vb = vis_byte(s.vis, v);
  uint32_t h[kMaxCols];
#pragma unroll
  for (int jj = 0; jj < kMaxCols; ++jj) h[jj] = jj < q.n_c ? hcol(q, jj)[v] : 1u;
  bool holds = false;
#pragma unroll
  for (int jj = 0; jj < kMaxCols; ++jj) holds |= ((vb >> jj) & 1u) && h[jj] == 0;
  return holds;
}

// A node for the overflow part of column list rlist (cap entries).
__device__ __forceinline__ void rec_overflow(Ctl* c, uint32_t* rlist, uint32_t* ovf, uint32_t cap, uint32_t v) {
  const uint32_t p = atomicAdd(ovf, 1u);
  if (p < cap) rlist[cap - 1u - p] = v; else atomicOr(&c->err, kErrOverflow);
}

// Start of column j's sweep (one CTA): the CG nodes that do not hold keyword
// j start it with their CG bit; with j = 0 every CG node also enters V^c's
// union list.
__device__ void rec_start(const DevSlot& s, int j) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const uint32_t nsel = c->nsel;
  if (nsel == 0 || j >= q.n_c) return;
  const uint8_t* Hj = hcol(q, j);
  unsigned long long* rmask = rmcol(q, j);
  uint32_t* rlist = rlcol(q, j);
  uint32_t* ovf = s.rcnt + size_t(j) * kRecStride + (kMaxLevel + 2);
  for (uint32_t gi = threadIdx.x; gi < nsel; gi += blockDim.x) {
    const uint32_t v = uint32_t(c->sel_int[gi]);
    if (j == 0) {                                  // the CG nodes themselves belong to V^c
      const unsigned long long old = atomicOr(&s.vmask[v], 1ull << gi);
      if (old == 0) s.ulist[atomicAdd(&c->ulist_n, 1u)] = v;
    }
    if (Hj[v] == 0) continue;                      // the CG node holds keyword j
    if (atomicOr(&rmask[v], 1ull << gi) == 0) rec_overflow(c, rlist, ovf, s.cap, v);
  }
}

// Level x of column j's sweep, the share of CTA `rank` of the R CTAs on the
// column: every CTA scans the level's entries (segment of level x from
// entry `base`, then the overflow nodes with h = x), and the CSR entries
// with a <= x-1 of those nodes are dealt round-robin over the R CTAs.
// s_off and s_rb hold blockDim.x entries, s_m as many.
__device__ void rec_level(const DevKG& g, const DevSlot& s, int j, uint32_t rank, uint32_t R, int x, uint32_t base,
                          uint32_t* s_off, uint32_t* s_rb, unsigned long long* s_m) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const uint32_t cap = s.cap;
  const uint8_t* Hj = hcol(q, j);
  unsigned long long* rmask = rmcol(q, j);
  uint32_t* rlist = rlcol(q, j);
  uint32_t* sn = s.rcnt + size_t(j) * kRecStride;          // sn[y]: segment length of level y
  uint32_t* ovf = sn + (kMaxLevel + 2);                    // overflow length
  __shared__ uint64_t s_warp[33];
  __shared__ uint32_t s_total, s_cnt[2];
  const uint32_t stride = R * blockDim.x;
  // one read for the whole block: other CTAs append to the overflow while
  // this level runs, and every thread must run the same rounds (barriers)
  if (threadIdx.x == 0) { s_cnt[0] = __ldcg(&sn[x]); s_cnt[1] = min(__ldcg(ovf), cap); }
  __syncthreads();
  const uint32_t nseg = s_cnt[0], nov = s_cnt[1];
  const uint32_t next_base = base + nseg, cnt = nseg + nov;
  for (uint32_t c0 = 0; c0 < cnt; c0 += blockDim.x) {
    const uint32_t i = c0 + threadIdx.x;
    uint32_t len = 0, rb = 0;
    unsigned long long m = 0;
    if (i < cnt) {
      const uint32_t qn0 = i < nseg ? __ldcg(rlist + base + i) : __ldcg(rlist + cap - 1u - (i - nseg));
      const bool okq = RPQ_IN_BOUNDS(qn0 < uint32_t(g.n), &c->err);
      const uint32_t qn = okq ? qn0 : 0u;
      // every load of the node first (the addresses depend on qn alone)
      const uint32_t hq = Hj[qn];
      const uint32_t r0 = g.row_ptr[qn], r1 = g.row_ptr[qn + 1];
      const uint32_t o = uint32_t(x) <= kLvxLevels ? g.lvx[size_t(x - 1) * size_t(g.n) + qn] : 0u;
      const unsigned long long mq = __ldcg(rmask + qn);
      if (okq && (i < nseg || hq == uint32_t(x))) {
        uint32_t hi;                               // first entry with a >= x
        if (uint32_t(x) > kLvxLevels) hi = seg_lower(g.adj, r0, r1, uint32_t(x));
        else if (r1 - r0 <= kLvxMaxDeg) hi = r0 + o;
        else hi = r0 + g.lvx_long[size_t(o) * kLvxLevels + (x - 1)];
        rb = r0;
        len = hi - r0;                             // edges with a <= x-1
        m = mq;
      }
    }
    uint64_t tot = 0;
    const uint32_t pre = uint32_t(block_excl_scan(len, s_warp, &tot));
    s_off[threadIdx.x] = pre; s_rb[threadIdx.x] = rb; s_m[threadIdx.x] = m;
    if (threadIdx.x == 0) s_total = uint32_t(tot);
    __syncthreads();
    const uint32_t total = s_total;
    for (uint32_t u = rank * blockDim.x + threadIdx.x; u < total; u += stride) {
      uint32_t lo = 0, hi = blockDim.x - 1;       // last slot with s_off <= u
      while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo + 1) >> 1);
        if (s_off[mid] <= u) lo = mid; else hi = mid - 1;
      }
      if (!RPQ_IN_BOUNDS(s_rb[lo] + (u - s_off[lo]) < g.m2, &c->err)) continue;
      const uint32_t xe = __ldg(g.adj + s_rb[lo] + (u - s_off[lo]));
      const uint32_t a = xe >> kNodeBits, nb = xe & kNodeMask;
      if (!RPQ_IN_BOUNDS(nb < uint32_t(g.n), &c->err)) continue;
      // all loads of the neighbour at once, then the tests
      const uint32_t vb = vis_byte(s.vis, nb), hn = Hj[nb], cfw = s.cf[nb >> 5], stl = s.stopl[nb];
      if (!((vb >> j) & 1u)) continue;
      const uint32_t lam = a > hn ? a : hn;
      if (lam + 1 != uint32_t(x)) continue;                               // not tight
      if (((cfw >> (nb & 31u)) & 1u) && stl <= lam) continue;             // nb had stopped
      if (atomicOr(&rmask[nb], s_m[lo]) != 0) continue;                  // already listed
      if (hn + 1 == uint32_t(x)) {
        const uint32_t p = next_base + atomicAdd(&sn[hn], 1u);
        if (p < cap) rlist[p] = nb; else atomicOr(&c->err, kErrOverflow);
      } else {
        rec_overflow(c, rlist, ovf, cap, nb);
      }
    }
    __syncthreads();
  }
}

// End of column j's sweep (CTA `rank` of R, after its last level; `nseg`
// entries in the level segments): every reached node that holds a central
// keyword ORs its column mask into the union mask (vmask), and every column
// mask is cleared.  The last CTA of all columns (n_c * R of them) keeps the
// nodes of V^c that hold a central keyword: V_C of each CG, as
// (g << 26 | node) pairs; it also clears the list counters.
__device__ void rec_finish(const DevSlot& s, int j, uint32_t rank, uint32_t R, uint32_t nseg) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const uint32_t cap = s.cap;
  unsigned long long* rmask = rmcol(q, j);
  const uint32_t* rlist = rlcol(q, j);
  const uint32_t* ovf = s.rcnt + size_t(j) * kRecStride + (kMaxLevel + 2);
  const uint32_t stride = R * blockDim.x;
  const uint32_t nov = min(__ldcg(ovf), cap);
  for (uint32_t i = rank * blockDim.x + threadIdx.x; i < nseg + nov; i += stride) {
    const uint32_t v = i < nseg ? __ldcg(rlist + i) : __ldcg(rlist + cap - 1u - (i - nseg));
    if (!RPQ_IN_BOUNDS(v < uint32_t(s.cap), &c->err)) continue;
    const unsigned long long m = __ldcg(rmask + v);
    rmask[v] = 0;
    if (!holds_central(s, q, v)) continue;
    const unsigned long long old = atomicOr(&s.vmask[v], m);
    if (old == 0) {
      const uint32_t p = atomicAdd(&c->ulist_n, 1u);
      if (p < cap) s.ulist[p] = v; else atomicOr(&c->err, kErrOverflow);
    }
  }
  __shared__ uint32_t s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&c->rec_done, 1u) == uint32_t(q.n_c) * R - 1u ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (uint32_t i = threadIdx.x; i < uint32_t(q.n_c) * kRecStride; i += blockDim.x) s.rcnt[i] = 0;
  const uint32_t nu = min(__ldcg(&c->ulist_n), cap);
  for (uint32_t i = threadIdx.x; i < nu; i += blockDim.x) {
    const uint32_t v = __ldcg(s.ulist + i);
    unsigned long long m = __ldcg(s.vmask + v);
    s.vmask[v] = 0;
    if (!holds_central(s, q, v)) continue;
    for (; m; m &= m - 1) {
      const uint32_t gi = __ffsll(m) - 1;
      const uint32_t p = atomicAdd(&c->nvc, 1u);
      if (p < cap) s.vcl[p] = (gi << kNodeBits) | v; else atomicOr(&c->err, kErrOverflow);
    }
  }
  if (threadIdx.x == 0) c->rec_done = 0;
}

__global__ void __cluster_dims__(kRecCluster, 1, 1) __launch_bounds__(kRecThreads, 1)
k_recover_cols(DevKG g, DevSlot s) {
  cg::cluster_group cluster = cg::this_cluster();
  const int j = int(blockIdx.x / kRecCluster);
  const uint32_t rank = cluster.block_rank();
  if (s.ctl->nsel == 0 || j >= s.q->n_c) return;           // the same in every CTA of the cluster
  __shared__ uint32_t s_off[kRecThreads];
  __shared__ uint32_t s_rb[kRecThreads];
  __shared__ unsigned long long s_m[kRecThreads];
  if (rank == 0) rec_start(s, j);
  cluster.sync();
  const int maxlev = s.ctl->levels[0];
  uint32_t base = 0;                                 // first entry of the segment of level x
  for (int x = maxlev; x >= 1; --x) {
    const uint32_t nseg = __ldcg(&s.rcnt[size_t(j) * kRecStride + x]);
    rec_level(g, s, j, rank, kRecCluster, x, base, s_off, s_rb, s_m);
    cluster.sync();                                  // level x done everywhere before level x-1
    base += nseg;
  }
  rec_finish(s, j, rank, kRecCluster, base + __ldcg(&s.rcnt[size_t(j) * kRecStride]));
}

// --------------------------------------------------------------- results
// Eq. 6 (or product) scores and the top-k by (S^r, node id).  With M empty
// the results are the selected CGs with S^m = 0 and S^r = S^c.
// Needs at least kMaxK threads of one block; every thread of the block calls it.
// The control block is read through L2: inside one persistent launch other
// blocks wrote it.
__device__ void write_results(const DevSlot& s) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  rpq_result* out = reinterpret_cast<rpq_result*>(s.res);
  const uint32_t nsel = __ldcg(&c->nsel);
  __shared__ double s_sr[kMaxK];
  __shared__ uint32_t s_ok[kMaxK];
  __shared__ int32_t s_node[kMaxK];
  __shared__ uint32_t s_sc[kMaxK], s_sm[kMaxK];
  const uint32_t gi = threadIdx.x;
  if (gi < kMaxK) {
    s_ok[gi] = 0;
    if (gi < nsel) {
      s_node[gi] = __ldcg(&c->sel[gi]);
      s_sc[gi] = __ldcg(&c->sel_sc[gi]);
      s_sm[gi] = q.n_m == 0 ? 0u : uint32_t(__ldcg(&c->sm[gi]));
      if (q.n_m == 0) { s_ok[gi] = 1; s_sr[gi] = double(s_sc[gi]); }
      else if (__ldcg(&c->matched[gi])) {
        s_ok[gi] = 1;
        s_sr[gi] = rpg_score(q, s_sc[gi], s_sm[gi]);
      }
    }
  }
  __syncthreads();
  if (gi < nsel && s_ok[gi]) {
    const int32_t node = s_node[gi];
    uint32_t rank = 0;
    for (uint32_t o = 0; o < nsel; ++o) {
      if (!s_ok[o] || o == gi) continue;
      if (s_sr[o] < s_sr[gi] || (s_sr[o] == s_sr[gi] && s_node[o] < node)) ++rank;
    }
    if (rank < uint32_t(q.k)) {
      rpq_result r;
      r.node = node;
      r.s_c = int32_t(s_sc[gi]);
      r.s_m = int32_t(s_sm[gi]);
      r.reserved = 0;
      r.s_r = s_sr[gi];
      out[rank] = r;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t n = 0;
    for (uint32_t o = 0; o < nsel; ++o) n += s_ok[o];
    n = min(n, uint32_t(q.k));
    c->n_res = n;
    *s.n_res = int32_t(n);
    const uint32_t err = __ldcg(&c->err);
    if (err) atomicOr(s.sticky, err);
  }
}

// Standalone form (trace and subgraph paths); a query graph has no such node:
// the kernel that ends the search writes the results itself (k_topk when
// there is no marginal run, else the k_expand that stops the marginal run).
__global__ void k_results(DevSlot s) { write_results(s); }

// ------------------------------------------ multi-query persistent kernel
// A batch of queries runs in one launch of k_batch, one wave of blocks that
// stay resident until the batch is done, over a device work queue: every
// slot (the state of one query in flight) offers the chunks of its query's
// current phase, a block takes one chunk with an atomic add on the slot's
// phase word and runs it (the same device code as the launched kernels, with
// the chunk as its block of the phase; blocks prefer the oldest query with
// chunks left), and the block that finishes the phase's last chunk computes
// the next phase and publishes it; a slot whose
// query ends writes the query's record and takes the next query of the
// batch.  The phase boundaries take the place of the kernel boundaries of
// the launched sequence (release: fence, then the atomic that counts the
// chunk done; acquire: the atomic that takes a chunk, then a fence), and a
// phase has as many chunks as its work needs (one for a small frontier),
// so small levels of some queries leave the other blocks to the dense
// levels of others.  Recovery runs one phase per level of the sweep, in
// place of the cluster barrier between levels.  Blocks never wait for one
// another inside a phase; a block without work polls the slots, and a
// watchdog ends the kernel (kErrTimeout) when no phase finishes for `limit`
// clock cycles.
constexpr int kBatchThreads = 256;
constexpr int kBatchTopkChunk = 512;               // top-w selection: keys per chunk round, radix digit
constexpr int kBatchTopkBits = 8;
constexpr uint32_t kBatchRec = kRecCluster;   // chunks per central column of a recovery phase
static_assert(sizeof(rpq_result) == 24, "batch record layout");

enum BatchPhase : uint32_t {
  kPhClear = 1,      // zero the run's visited bytes and bit maps
  kPhSeed,           // k_seed
  kPhEnqueue,        // k_enqueue
  kPhTarget,         // k_target
  kPhExpand,         // k_expand
  kPhTopk,           // k_topk
  kPhRecStart,       // recovery: start of each column's sweep
  kPhRecLevel,       // recovery: one level of every column's sweep
  kPhRecFinish,      // recovery: union masks and V_C
};

struct BatchArgs {
  DevKG g;
  const QueryDev* queries;   // n_queries records (keyword ids and parameters)
  uint8_t* out;              // kBatchRecBytes per query
  BatchSlotState* bs;        // n_slots
  BatchCtl* bc;
  uint32_t n_queries, n_slots, n_sm;
  long long limit;
  DevSlot slot[kBatchMaxSlots];
};

// A slot's phase word: next chunk to hand out (bits 0-23), chunks of the
// phase (24-39), phase (40-43), run (44) and level (45-50), so that the
// atomic add that takes a chunk also returns what the chunk is.  Blocks add
// only after reading next < chunks, so next stays below chunks + blocks.
__device__ __forceinline__ unsigned long long batch_word(uint32_t phase, uint32_t run, uint32_t level, uint32_t nch) {
  return (uint64_t(level) << 45) | (uint64_t(run) << 44) | (uint64_t(phase) << 40) | (uint64_t(nch) << 24);
}
__device__ __forceinline__ uint32_t word_next(unsigned long long w) { return uint32_t(w) & 0xffffffu; }
__device__ __forceinline__ uint32_t word_chunks(unsigned long long w) { return uint32_t(w >> 24) & 0xffffu; }

__device__ __forceinline__ uint32_t clamp_chunks(uint64_t want, uint32_t most) {
  return uint32_t(want < 1 ? 1 : (want > most ? most : want));
}

// Thread 0: the slot's next phase; its chunks are handed out from here on.
__device__ __forceinline__ void batch_publish(BatchSlotState* b, BatchCtl* bc, uint32_t phase, uint32_t run,
                                              uint32_t level, uint32_t nch) {
  b->done = 0;
  b->phase = phase;
  b->run = run;
  b->level = level;
  __threadfence();
  atomicExch(&b->word, batch_word(phase, run, level, nch));
  atomicAdd(&bc->progress, 1ull);
}

// Chunks of the phases whose size is known from the control block, at most
// one per block: at least two frontier-queue tiles, four bit-map tiles or
// two warp tiles of work units per warp, so that the cost of taking a chunk
// stays small against its work; a small level gets few chunks and leaves
// the other blocks to other queries.
__device__ uint32_t clear_chunks(const DevSlot& s, uint32_t grid) {
  return clamp_chunks((s.run_clear_bytes + 65535ull) >> 16, grid);
}
__device__ uint32_t seed_chunks(const DevKG& g, const DevSlot& s, int run, uint32_t most) {
  const QueryDev& q = *s.q;
  const int nt = run == 0 ? q.n_c : q.n_m, kb = run == 0 ? 0 : q.n_c;
  uint64_t total = 0;
  for (int j = 0; j < nt; ++j) {
    const int32_t kw = q.kw[kb + j];
    if (kw >= 0 && kw < g.n_kw) total += g.kw_ptr[kw + 1] - g.kw_ptr[kw];
  }
  return clamp_chunks((total + kBatchThreads - 1) / kBatchThreads, most);
}
__device__ uint32_t enqueue_chunks(const DevKG& g, const DevSlot& s, uint32_t grid) {
  const Ctl* c = s.ctl;
  const int p = int(__ldcg(&c->lvl_enq) & 1u);
  if (enqueue_sparse<true>(s, c, p)) return clamp_chunks((uint64_t(__ldcg(&c->fq_n[p])) + 2 * kEnqThreads - 1) / (2 * kEnqThreads), grid);
  const uint64_t slots = uint64_t((uint32_t(g.n) + 31u) >> 5) * 32u;
  return clamp_chunks((slots + 4 * kEnqThreads * kEnqRounds - 1) / (4 * kEnqThreads * kEnqRounds), grid);
}
__device__ uint32_t expand_chunks(const DevSlot& s, int run, uint32_t grid) {
  const LevelPlan plan = level_plan<true>(s, run, __ldcg(&s.ctl->lvl_exp));
  if (plan.stop) return grid;                               // every block counts hits
  if (plan.skip || plan.n_work == 0) return 1;              // the bookkeeping of block 0 only
  const uint64_t tiles = (uint64_t(plan.n_work) + kWarpTile - 1) / kWarpTile;
  return clamp_chunks((tiles + kBatchThreads / 16 - 1) / (kBatchThreads / 16), grid);
}

// Thread 0: the first query of the batch not yet started goes to slot sl
// (k_set_query's work, with the slot's own columns), or the slot retires.
__device__ void batch_start_query(const BatchArgs& a, uint32_t sl) {
  BatchSlotState* b = a.bs + sl;
  const uint32_t qi = atomicAdd(&a.bc->next_query, 1u);
  if (qi >= a.n_queries) {
    b->query = -1;
    atomicExch(&b->word, 0ull);
    return;
  }
  const DevSlot& s = a.slot[sl];
  QueryDev* q = s.q;
  *q = a.queries[qi];
  for (int j = 0; j < kMaxCols; ++j) {
    q->hc[j] = s.H + size_t(j) * s.hp;
    q->rm[j] = s.rmask + size_t(j) * s.cap;
    q->rl[j] = s.rlist + size_t(j) * s.cap;
  }
  Ctl* c = s.ctl;
  uint32_t* w = reinterpret_cast<uint32_t*>(c);
  for (size_t i = 0; i < sizeof(Ctl) / 4; ++i) w[i] = 0;
  c->levels[0] = c->levels[1] = -1;
  c->last_expanded = -1;
  c->fq_use[0] = 1;
  s.bar[0] = 0;
  *s.n_res = 0;
  b->query = int32_t(qi);
  batch_publish(b, a.bc, kPhClear, 0, 0, clear_chunks(s, gridDim.x));
}

// k_run_start's work for the marginal run (thread 0).
__device__ void batch_run_start(const DevSlot& s) {
  Ctl* c = s.ctl;
  c->done = (s.q->n_m == 0 || c->nsel == 0) ? 1u : 0u;
  c->work[0] = c->work[1] = 0;
  c->nq[0] = c->nq[1] = 0;
  c->fq_n[0] = c->fq_n[1] = 0;
  c->fq_over[0] = c->fq_over[1] = 0;
  c->fq_use[0] = 1;
  c->fq_use[1] = 0;
  c->lvl_enq = c->lvl_exp = 0;
  c->level = 0;
  c->eact_lvl[0] = c->eact_lvl[1] = 0;
  c->skip_lvl = 0;
  c->ncg_at = 0;
  c->cg_next[0] = c->cg_next[1] = 0;
  c->tgt_n = c->tgt_done = 0;
  s.bar[0] = 0;
  c->last_expanded = -1;
}

// One chunk of the slot's current phase (every thread of the block).
__device__ void batch_chunk(const BatchArgs& a, const DevSlot& s, uint32_t phase, uint32_t run, uint32_t level,
                            Part pt, uint32_t* buf) {
  const DevKG& g = a.g;
  switch (phase) {
    case kPhClear: {
      uint4* p = static_cast<uint4*>(s.run_clear);
      const unsigned long long n16 = s.run_clear_bytes >> 4;
      const unsigned long long b0 = n16 * pt.b / pt.n, b1 = n16 * (pt.b + 1) / pt.n;
      for (unsigned long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) p[i] = make_uint4(0, 0, 0, 0);
      break;
    }
    case kPhSeed: seed_body(g, s, int(run), pt); break;
    case kPhEnqueue: enqueue_body<false>(g, s, int(run), pt); break;
    case kPhTarget: target_body(g, s, pt); break;
    case kPhExpand: expand_body<false>(g, s, int(run), 0, 0, pt); break;
    case kPhTopk:
      topk_body<kBatchThreads, kBatchTopkChunk, kBatchTopkBits>(g, s, pt, buf, buf + kBatchTopkChunk + 2 * kMaxK);
      break;
    case kPhRecStart: rec_start(s, int(pt.b)); break;
    case kPhRecLevel:
    case kPhRecFinish: {
      const int j = int(pt.b / kBatchRec);
      const uint32_t rank = pt.b % kBatchRec;
      if (s.ctl->nsel == 0 || j >= s.q->n_c) break;
      const int maxlev = s.ctl->levels[0];
      const uint32_t* sn = s.rcnt + size_t(j) * kRecStride;
      if (phase == kPhRecLevel) {
        uint32_t base = 0;                          // the segments of the levels above
        for (int y = maxlev; y > int(level); --y) base += __ldcg(&sn[y]);
        rec_level(g, s, j, rank, kBatchRec, int(level), base, buf, buf + kBatchThreads,
                  reinterpret_cast<unsigned long long*>(buf + 2 * kBatchThreads));
      } else {
        uint32_t nseg = 0;
        for (int y = maxlev; y >= 0; --y) nseg += __ldcg(&sn[y]);
        rec_finish(s, j, rank, kBatchRec, nseg);
      }
      break;
    }
    default: break;
  }
}

// The block that finished the slot's phase: the next phase, or the end of
// the query (its record, then the next query).  Every thread calls it.
__device__ void batch_advance(const BatchArgs& a, uint32_t sl) {
  BatchSlotState* b = a.bs + sl;
  const DevSlot& s = a.slot[sl];
  Ctl* c = s.ctl;
  const uint32_t grid = gridDim.x, small = 2u * a.n_sm;
  __shared__ uint32_t s_end;
  if (threadIdx.x == 0) {
    const uint32_t phase = __ldcg(&b->phase), run = __ldcg(&b->run), level = __ldcg(&b->level);
    const QueryDev& q = *s.q;
    bool end = false;
    switch (phase) {
      case kPhClear: batch_publish(b, a.bc, kPhSeed, run, 0, seed_chunks(a.g, s, int(run), small)); break;
      case kPhSeed: batch_publish(b, a.bc, kPhEnqueue, run, 0, enqueue_chunks(a.g, s, grid)); break;
      case kPhEnqueue:
        if (run == 1 && target_runs<true>(s)) {
          const uint32_t ntask = min(__ldcg(&c->nvc), s.cap) * uint32_t(q.n_m);
          batch_publish(b, a.bc, kPhTarget, run, 0, clamp_chunks((ntask + 7u) / 8u, small));
        } else {
          batch_publish(b, a.bc, kPhExpand, run, 0, expand_chunks(s, int(run), grid));
        }
        break;
      case kPhTarget: batch_publish(b, a.bc, kPhExpand, run, 0, expand_chunks(s, int(run), grid)); break;
      case kPhExpand:
        if (!__ldcg(&c->done) && __ldcg(&c->lvl_enq) <= uint32_t(q.L)) {
          batch_publish(b, a.bc, kPhEnqueue, run, 0, enqueue_chunks(a.g, s, grid));
        } else if (run == 0) {
          const uint32_t n_in = min(__ldcg(&c->ncg), s.cap);
          batch_publish(b, a.bc, kPhTopk, 0, 0, clamp_chunks((n_in + kBatchTopkChunk - 1) / kBatchTopkChunk, small));
        } else {
          end = true;
        }
        break;
      case kPhTopk:
        if (q.n_m == 0 || __ldcg(&c->nsel) == 0) end = true;   // k_topk wrote the results
        else batch_publish(b, a.bc, kPhRecStart, 0, 0, uint32_t(q.n_c));
        break;
      case kPhRecStart:
      case kPhRecLevel: {
        const int next = phase == kPhRecStart ? __ldcg(&c->levels[0]) : int(level) - 1;
        if (next >= 1) batch_publish(b, a.bc, kPhRecLevel, 0, uint32_t(next), uint32_t(q.n_c) * kBatchRec);
        else batch_publish(b, a.bc, kPhRecFinish, 0, 0, uint32_t(q.n_c) * kBatchRec);
        break;
      }
      case kPhRecFinish:
        batch_run_start(s);
        if (c->done) end = true;
        else batch_publish(b, a.bc, kPhClear, 1, 0, clear_chunks(s, grid));
        break;
      default: end = true; break;
    }
    s_end = end ? 1u : 0u;
  }
  __syncthreads();
  if (!s_end) return;
  // the query's record: control block and results, then the flag
  const int32_t qi = __ldcg(&b->query);
  uint32_t* rec = reinterpret_cast<uint32_t*>(a.out + size_t(qi) * kBatchRecBytes);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(c);            // the results follow the control block
  for (uint32_t i = threadIdx.x; i < (kCtlBytes + 24 * kMaxK) / 4; i += blockDim.x) rec[kBatchRecHead / 4 + i] = __ldcg(src + i);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    rec[0] = 1u;
    __threadfence();
    atomicAdd(&a.bc->finished, 1u);
    batch_start_query(a, sl);
  }
}

__global__ void __launch_bounds__(kBatchThreads, 6)
k_batch(const __grid_constant__ BatchArgs a) {
  // scratch of the top-w selection (keys, histogram) or of a recovery level (scan)
  constexpr int kBuf = kBatchTopkChunk + 2 * kMaxK + (1 << kBatchTopkBits) > 4 * kBatchThreads
                       ? kBatchTopkChunk + 2 * kMaxK + (1 << kBatchTopkBits) : 4 * kBatchThreads;
  __shared__ __align__(16) uint32_t buf[kBuf];
  __shared__ int s_slot;
  __shared__ uint32_t s_chunk, s_nch, s_phase, s_run, s_level, s_exit, s_last;
  if (blockIdx.x < a.n_slots && threadIdx.x == 0) batch_start_query(a, blockIdx.x);
  // thread 0's watchdog state (progress count last seen, and when), kept in
  // shared memory so that it holds no registers across the phase bodies
  __shared__ unsigned long long seen;
  __shared__ long long since;
  if (threadIdx.x == 0) { seen = ~0ull; since = clock64(); }
  for (;;) {
    __syncthreads();                               // every thread has read the last round's shared values
    if (threadIdx.x == 0) {
      int got = -1;
      // after a watchdog timeout no block takes further work
      const bool stopped = *(volatile uint32_t*)&a.bc->err != 0;
      // oldest query first: every block takes a chunk of the oldest query
      // with chunks left, so the blocks work on few queries at a time (their
      // per-node state shares L2) and younger queries fill the gaps
      for (int tries = 0; tries < 4 && got < 0 && !stopped; ++tries) {
        int best = -1;
        uint32_t best_q = 0xffffffffu;
        for (uint32_t sl = 0; sl < a.n_slots; ++sl) {
          const unsigned long long w = *(volatile unsigned long long*)&a.bs[sl].word;
          const uint32_t qi = *(volatile uint32_t*)&a.bs[sl].query;
          if (word_next(w) < word_chunks(w) && qi < best_q) { best = int(sl); best_q = qi; }
        }
        if (best < 0) break;
        const unsigned long long o = atomicAdd(&a.bs[best].word, 1ull);
        if (word_next(o) < word_chunks(o)) {
          got = best;
          s_chunk = word_next(o);
          s_nch = word_chunks(o);
          s_phase = uint32_t(o >> 40) & 0xfu;
          s_run = uint32_t(o >> 44) & 1u;
          s_level = uint32_t(o >> 45) & 0x3fu;
        }
      }
      s_exit = 0;
      if (got >= 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");   // acquire: the phase's inputs
      } else if (stopped || *(volatile uint32_t*)&a.bc->finished >= a.n_queries) {
        s_exit = 1;
      } else {
        const unsigned long long pr = *(volatile unsigned long long*)&a.bc->progress;
        const long long now = clock64();
        if (pr != seen) { seen = pr; since = now; }
        else if (now - since > a.limit) { atomicOr(&a.bc->err, kErrTimeout); s_exit = 1; }
        else __nanosleep(256);
      }
      s_slot = got;
    }
    __syncthreads();
    if (s_exit) break;
    const int sl = s_slot;
    if (sl < 0) continue;
    const uint32_t nch = s_nch;
    batch_chunk(a, a.slot[sl], s_phase, s_run, s_level, Part{s_chunk, nch}, buf);
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");    // release: this chunk's writes
      s_last = atomicAdd(&a.bs[sl].done, 1u) == nch - 1u ? 1u : 0u;
      if (s_last) asm volatile("fence.acq_rel.gpu;" ::: "memory");   // acquire: every chunk's writes
    }
    __syncthreads();
    if (s_last) batch_advance(a, uint32_t(sl));
  }
}

}  // namespace

// ------------------------------------------------------------ launchers

// Launch wrapper: brackets the launch with CUDA events in profiling mode.
template <typename F>
static void timed(Prof* prof, int cls, cudaStream_t st, F&& launch) {
  if (!prof) { launch(); return; }
  cudaEvent_t a;
  prof->begin(st, &a);
  launch();
  prof->end(cls, st, a);
}

int launch_query_setup(const DevSlot& s, const QueryDev& qv, const int32_t* d_kw, cudaStream_t st) {
  QueryDev q = qv;
  if (s.H) {                                  // the slot's own columns
    for (int j = 0; j < kMaxCols; ++j) {
      q.hc[j] = s.H + size_t(j) * s.hp;
      q.rm[j] = s.rmask + size_t(j) * s.cap;
      q.rl[j] = s.rlist + size_t(j) * s.cap;
    }
  } else {                                    // columns lent by a server: every used one is set
    const int nh = std::max(q.n_c, q.n_m);
    for (int j = 0; j < nh; ++j) if (!q.hc[j]) return RPQ_EINTERNAL;
    for (int j = 0; j < q.n_c; ++j) if (!q.rm[j] || !q.rl[j]) return RPQ_EINTERNAL;
  }
  k_set_query<<<1, 32, 0, st>>>(s, q, d_kw);
  return cudaGetLastError() == cudaSuccess ? RPQ_OK : RPQ_ECUDA;
}

// Reset and seed one run.
void launch_run_setup(const DevKG& g, const DevSlot& s, int run, cudaStream_t st, Prof* prof) {
  timed(prof, RPQ_PROF_SETUP, st, [&] {
    if (run != 0) k_run_start<<<1, 32, 0, st>>>(s, run);      // k_set_query prepared the central run
    cudaMemsetAsync(s.run_clear, 0, s.run_clear_bytes, st);   // visited bytes, F[0], F[1], cf
    k_seed<<<num_sms() * 2, 256, 0, st>>>(g, s, run);
  });
}

// Grid of a persistent-style kernel: SMs x blocks resident per SM (one wave).
template <typename K>
static int one_wave_grid(K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return num_sms() * per_sm;
}

size_t batch_state_bytes(int n_slots) { return sizeof(BatchSlotState) * size_t(n_slots) + sizeof(BatchCtl); }

int launch_batch(const DevKG& g, const DevSlot* slots, int n_slots, const QueryDev* d_queries, int n_queries,
                 void* d_out, void* d_state, long long limit, cudaStream_t st) {
  if (n_slots < 1 || n_slots > kBatchMaxSlots || n_queries < 1) return RPQ_EINVAL;
  static const int grid = one_wave_grid(k_batch, kBatchThreads);
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.queries = d_queries;
  a.out = static_cast<uint8_t*>(d_out);
  a.bs = static_cast<BatchSlotState*>(d_state);
  a.bc = reinterpret_cast<BatchCtl*>(a.bs + n_slots);
  a.n_queries = uint32_t(n_queries);
  a.n_slots = uint32_t(n_slots);
  a.n_sm = uint32_t(num_sms());
  a.limit = limit;
  for (int i = 0; i < n_slots; ++i) a.slot[i] = slots[i];
  if (cudaMemsetAsync(d_state, 0, batch_state_bytes(n_slots), st) != cudaSuccess) return RPQ_ECUDA;
  k_batch<<<grid, kBatchThreads, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? RPQ_OK : RPQ_ECUDA;
}

// One run as a single cooperative launch of k_run (one wave of blocks).
void launch_run_persistent(const DevKG& g, const DevSlot& s, int run, cudaStream_t st, Prof* prof) {
  static const int grid = one_wave_grid(k_run, kExpThreads);
  timed(prof, RPQ_PROF_EXPAND, st, [&] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(kExpThreads));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_run, g, s, run);
  });
}

// One Glevel: enqueue + identification, (marginal run) the V_C check, then
// termination + expansion.
void launch_level(const DevKG& g, const DevSlot& s, int run, cudaStream_t st, Prof* prof,
                  cudaGraphConditionalHandle loop, bool in_graph) {
  static const int enq_grid = one_wave_grid(k_enqueue, kEnqThreads);
  static const int exp_grid = one_wave_grid(k_expand, kExpThreads);
  static const int tgt_grid = num_sms() * 2;
  if (prof) prof->tag_kind = kKindEnqueue;
  timed(prof, RPQ_PROF_ENQUEUE, st, [&] { k_enqueue<<<enq_grid, kEnqThreads, 0, st>>>(g, s, run); });
  if (prof) prof->tag_kind = kKindTarget;
  if (run == 1) timed(prof, RPQ_PROF_ENQUEUE, st, [&] { k_target<<<tgt_grid, kTgtThreads, 0, st>>>(g, s); });
  if (prof) prof->tag_kind = kKindExpand;
  timed(prof, RPQ_PROF_EXPAND, st, [&] { k_expand<<<exp_grid, kExpThreads, 0, st>>>(g, s, run, loop, in_graph ? 1 : 0); });
  if (prof) prof->tag_kind = kKindOther;
}

// Top-w selection and, when the query has marginal keywords, the recovery.
void launch_select_recover(const DevKG& g, const DevSlot& s, int n_m, cudaStream_t st, Prof* prof) {
  const int sms = num_sms();
  timed(prof, RPQ_PROF_TOPK, st, [&] {
    k_topk<<<sms * 2, kTopkThreads, 0, st>>>(g, s);
  });
  if (n_m > 0) {
    timed(prof, RPQ_PROF_RECOVER, st, [&] {
      k_recover_cols<<<kMaxCols * kRecCluster, kRecThreads, 0, st>>>(g, s);
    });
  }
}

void launch_results(const DevSlot& s, cudaStream_t st, Prof* prof) {
  timed(prof, RPQ_PROF_RESULTS, st, [&] { k_results<<<1, kMaxK, 0, st>>>(s); });
}

// The whole query without a graph: one persistent launch or L+1 level pairs per run.
// With stop_early (direct launches, never under capture) the host waits after
// each Glevel and launches no further level once the run has stopped, like a
// query graph whose run ends inside its plain levels; kernel timings and
// launch lists then hold no early-exit launches.
int launch_query_body(const DevKG& g, const DevSlot& s, int n_m, int L, cudaStream_t st, Prof* prof,
                      bool stop_early) {
  auto levels = [&](int run) {
    for (int l = 0; l <= L; ++l) {
      if (prof) { prof->tag_run = run; prof->tag_level = l; }
      launch_level(g, s, run, st, prof, 0, false);
      if (prof) prof->tag_run = prof->tag_level = -1;
      if (!stop_early) continue;
      uint32_t done = 0;
      if (cudaStreamSynchronize(st) != cudaSuccess ||
          cudaMemcpy(&done, &s.ctl->done, sizeof(done), cudaMemcpyDeviceToHost) != cudaSuccess || done)
        break;
    }
  };
  launch_run_setup(g, s, 0, st, prof);
  if (s.persistent) launch_run_persistent(g, s, 0, st, prof);
  else levels(0);
  launch_select_recover(g, s, n_m, st, prof);
  if (n_m > 0) {
    launch_run_setup(g, s, 1, st, prof);
    if (s.persistent) launch_run_persistent(g, s, 1, st, prof);
    else levels(1);
  }
  return cudaGetLastError() == cudaSuccess ? RPQ_OK : RPQ_ECUDA;
}

int launch_central_part(const DevKG& g, const DevSlot& s, int L, cudaStream_t st, Prof* prof) {
  launch_run_setup(g, s, 0, st, prof);
  for (int l = 0; l <= L; ++l) launch_level(g, s, 0, st, prof, 0, false);
  const int sms = num_sms();
  timed(prof, RPQ_PROF_TOPK, st, [&] {
    k_topk<<<sms * 2, kTopkThreads, 0, st>>>(g, s);
  });
  return cudaGetLastError() == cudaSuccess ? RPQ_OK : RPQ_ECUDA;
}

int launch_marginal_part(const DevKG& g, const DevSlot& s, int n_m, int L, cudaStream_t st, Prof* prof) {
  if (n_m > 0) {
    timed(prof, RPQ_PROF_RECOVER, st, [&] {
      k_recover_cols<<<kMaxCols * kRecCluster, kRecThreads, 0, st>>>(g, s);
    });
    launch_run_setup(g, s, 1, st, prof);
    for (int l = 0; l <= L; ++l) launch_level(g, s, 1, st, prof, 0, false);
  }
  launch_results(s, st, prof);
  return cudaGetLastError() == cudaSuccess ? RPQ_OK : RPQ_ECUDA;
}

// Kernels launched by one query in a graph (for launch accounting): fixed
// kernels plus, per run, two per executed Glevel or one persistent launch.
int kernels_fixed_per_query(int n_m) {
  // k_set_query, k_seed, k_topk, [k_recover_cols, k_run_start, k_seed]
  return 1 + 1 + 1 + (n_m > 0 ? 3 : 0);
}

}  // namespace rpq
