// Result subgraphs of radial-pattern keyword search (rpq_search_subgraphs).
//
// The search itself (search_kernels.cu) keeps only what ranking needs: the
// CG nodes, V_C and the scores.  This file recovers the full result graphs
// G^r = G^c U G^m of Definition 5 on the device and checks the Pass Through
// Constraint on each of them.
//
//   after the central run  k_sg_sweep(0)  Algorithm 2 with Lemma 3, one block
//                                         per central column, backward from
//                                         the selected CG nodes
//                          k_sg_edges(0)  E^c (each edge once over columns)
//                          k_sg_nodes(0)  V^c, V_C (and the V_C pairs the
//                                         marginal run matches against)
//   after the marginal run k_sg_sweep(1)  the RPG variant of Section 4.3: the
//                                         sweep of marginal column i starts
//                                         at the nodes of V_C whose hit level
//                                         is min_{v in V_C} h^M[v][i]
//                          k_sg_edges(1), k_sg_nodes(1)   E^m, V^m
//   then                   k_sg_rank, k_sg_count, k_sg_offsets (list sizes),
//                          k_sg_scatter (per-result lists), k_sg_ptc
//
// Every node of a sweep carries a 64-bit mask of the selected CGs whose
// subgraph it belongs to (bit g = g-th selected CG), OR-ed backwards along
// the tight edges, so one sweep per column serves all CGs at once.  The
// masks of each column (rmask) are kept until the edge pass, which reads
// every row of a recovered node once and ORs the masks of all columns in
// which the edge is tight: an edge used by several keywords is reported
// once.  Nodes and edges are first written as (mask, ids) records; the
// scatter pass turns them into one list per (result, list kind).
//
// PTC (Definition 5) per result, one block each: the nodes of V^c U V^m go
// into an open-addressing hash table in global scratch, components of G^r
// without the nodes of V_C are found by min-label propagation along E^c U
// E^m, and the marginal keyword nodes are compared by component label (a
// node of V_C counts as its own component).
#include <algorithm>
#include <cstring>

#include "rpq_host.h"

namespace rpq {

namespace {

constexpr int kSwThreads = 1024;      // sweep: one block per keyword column
constexpr int kSgThreads = 256;       // edge / node passes
constexpr int kPtcThreads = 512;
constexpr uint32_t kEmptyKey = 0xffffffffu;
constexpr uint32_t kFlagVC = 1u << 8;      // hash flag: node of V_C
constexpr uint32_t kFlagTouch = 1u << 9;   // hash flag (label node): component adjacent to V_C

enum : uint32_t { kSgVc = 0, kSgVcKw = 1, kSgVm = 2, kSgEc = 3, kSgEm = 4, kSgKinds = 5 };

enum : uint32_t { kSgErrLookup = 1u, kSgErrLimit = 2u, kSgErrCap = 4u };

}  // namespace

// Node record: a = node, b = kind << 26.  Edge record: a = n, b = kind << 26 | q.
struct SgRec {
  unsigned long long mask;
  uint32_t a, b;
};

// Control block of the subgraph passes (device, copied to pinned host memory).
struct SgCtl {
  uint32_t nrec;                         // records written (beyond rec_cap: lost, grow and rerun)
  uint32_t err;                          // kSgErr* bits
  int32_t rank[kMaxK];                   // result rank of selected CG g, -1 if not a result
  uint32_t cnt[kSgKinds][kMaxK];         // list lengths per (kind, rank)
  uint32_t cur[kSgKinds][kMaxK];         // scatter cursors
  unsigned long long node_off[kMaxK * 3 + 1];
  unsigned long long edge_off[kMaxK * 2 + 1];
  unsigned long long hoff[kMaxK + 1];    // PTC hash table of rank r: [hoff[r], hoff[r+1])
  int32_t ptc[kMaxK];
};

struct SgDev {
  SgCtl* ctl;
  SgRec* rec;
  uint32_t rec_cap;
  uint32_t* nodes;
  unsigned long long nodes_cap;
  uint2* edges;
  unsigned long long edges_cap;
  uint32_t* hkey;                        // PTC hash tables: key, label, flags
  uint32_t* hlab;                        //   (one allocation, hash_cap entries each)
  uint32_t* hflag;
  unsigned long long hash_cap;
};

struct SgScratch {
  SgDev d{};
  SgCtl* h_ctl = nullptr;                // pinned
};

namespace {

__device__ __forceinline__ void emit(const SgDev& sg, unsigned long long mask, uint32_t a, uint32_t b) {
  const uint32_t p = atomicAdd(&sg.ctl->nrec, 1u);
  if (p < sg.rec_cap) {
    SgRec r;
    r.mask = mask;
    r.a = a;
    r.b = b;
    sg.rec[p] = r;
  }
}

__device__ __forceinline__ bool stopped_before(const DevSlot& s, uint32_t v, uint32_t lam) {
  return ((s.cf[v >> 5] >> (v & 31u)) & 1u) && s.stopl[v] <= lam;
}

// Add node v with CG bits m to the sweep of one column.
__device__ __forceinline__ void sweep_seed(const DevSlot& s, unsigned long long* rmask, uint32_t* rlist,
                                           uint32_t* s_n, uint32_t v, unsigned long long m) {
  const unsigned long long old = atomicOr(&rmask[v], m);
  if (old == 0) {
    const uint32_t p = atomicAdd(s_n, 1u);
    if (p < s.cap) rlist[p] = v; else atomicOr(&s.ctl->err, kErrOverflow);
  }
}

// Run 1 only: clear the union list before the marginal sweep.
__global__ void k_sg_begin(DevSlot s, SgDev sg, int run) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (run == 0) sg.ctl->nrec = 0, sg.ctl->err = 0;
  else s.ctl->ulist_n = 0;
}

// Backward sweep of column j = blockIdx.x (Algorithm 2 with Lemma 3): level
// by level downwards, node q at level x passes its CG mask to every n with an
// edge n -> q such that h_q = max(a, h_n) + 1 and n was still expanding at
// level max(a, h_n).  Run 0 starts at the selected CG nodes; run 1 at the
// nodes of V_C of each matched CG with the smallest marginal hit level.  The
// column masks stay set (the edge pass reads them); every swept node is
// OR-ed into the union mask vmask and listed once in ulist.
__global__ void __launch_bounds__(kSwThreads) k_sg_sweep(DevKG g, DevSlot s, int run) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const int nt = run == 0 ? q.n_c : q.n_m;
  const int j = int(blockIdx.x);
  const uint32_t nsel = c->nsel;
  if (j >= nt || nsel == 0) return;
  const uint8_t* Hj = hcol(*s.q, j);
  unsigned long long* rmask = rmcol(*s.q, j);
  uint32_t* rlist = rlcol(*s.q, j);
  __shared__ uint32_t s_off[kSwThreads];
  __shared__ uint32_t s_rb[kSwThreads];
  __shared__ unsigned long long s_m[kSwThreads];
  __shared__ uint64_t s_warp[33];
  __shared__ uint32_t s_n, s_cnt, s_total;
  __shared__ uint32_t s_d[kMaxK];
  if (threadIdx.x == 0) s_n = 0;
  for (uint32_t i = threadIdx.x; i < uint32_t(kMaxK); i += blockDim.x) s_d[i] = kInf;
  __syncthreads();
  const int maxlev = c->levels[run];
  if (run == 0) {
    for (uint32_t gi = threadIdx.x; gi < nsel; gi += blockDim.x)
      sweep_seed(s, rmask, rlist, &s_n, uint32_t(c->sel_int[gi]), 1ull << gi);
  } else {
    const uint32_t nvc = min(c->nvc, s.cap);
    for (uint32_t i = threadIdx.x; i < nvc; i += blockDim.x) {     // d_j(g) = min over V_C(g)
      const uint32_t pr = s.vcl[i], gi = pr >> kNodeBits, v = pr & kNodeMask;
      if (c->matched[gi] && ((vis_byte(s.vis, v) >> j) & 1u)) atomicMin(&s_d[gi], uint32_t(Hj[v]));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nvc; i += blockDim.x) {
      const uint32_t pr = s.vcl[i], gi = pr >> kNodeBits, v = pr & kNodeMask;
      if (c->matched[gi] && ((vis_byte(s.vis, v) >> j) & 1u) && uint32_t(Hj[v]) == s_d[gi])
        sweep_seed(s, rmask, rlist, &s_n, v, 1ull << gi);
    }
  }
  __syncthreads();
  for (int x = maxlev; x >= 1; --x) {
    if (threadIdx.x == 0) s_cnt = min(s_n, s.cap);
    __syncthreads();
    const uint32_t cnt = s_cnt;
    for (uint32_t c0 = 0; c0 < cnt; c0 += blockDim.x) {
      const uint32_t i = c0 + threadIdx.x;
      uint32_t len = 0, rb = 0;
      unsigned long long m = 0;
      if (i < cnt) {
        const uint32_t qn = rlist[i];
        if (Hj[qn] == uint8_t(x)) {
          rb = g.row_ptr[qn];
          len = seg_at(g, qn, rb, g.row_ptr[qn + 1], uint32_t(x)) - rb;   // edges with a <= x-1
          m = rmask[qn];
        }
      }
      uint64_t tot = 0;
      const uint32_t pre = uint32_t(block_excl_scan(len, s_warp, &tot));
      s_off[threadIdx.x] = pre;
      s_rb[threadIdx.x] = rb;
      s_m[threadIdx.x] = m;
      if (threadIdx.x == 0) s_total = uint32_t(tot);
      __syncthreads();
      const uint32_t total = s_total;
      for (uint32_t u = threadIdx.x; u < total; u += blockDim.x) {
        uint32_t lo = 0, hi = blockDim.x - 1;       // last slot with s_off <= u
        while (lo < hi) {
          const uint32_t mid = lo + ((hi - lo + 1) >> 1);
          if (s_off[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const uint32_t xe = __ldg(g.adj + s_rb[lo] + (u - s_off[lo]));
        const uint32_t a = xe >> kNodeBits, nb = xe & kNodeMask;
        if (!((vis_byte(s.vis, nb) >> j) & 1u)) continue;
        const uint32_t hn = Hj[nb];
        const uint32_t lam = a > hn ? a : hn;
        if (lam + 1 != uint32_t(x)) continue;                        // not tight
        if (stopped_before(s, nb, lam)) continue;                    // nb had stopped
        sweep_seed(s, rmask, rlist, &s_n, nb, s_m[lo]);
      }
      __syncthreads();
    }
  }
  const uint32_t nr = min(s_n, s.cap);
  for (uint32_t i = threadIdx.x; i < nr; i += blockDim.x) {
    const uint32_t v = rlist[i];
    const unsigned long long old = atomicOr(&s.vmask[v], rmask[v]);
    if (old == 0) {
      const uint32_t p = atomicAdd(&c->ulist_n, 1u);
      if (p < s.cap) s.ulist[p] = v; else atomicOr(&c->err, kErrOverflow);
    }
  }
}

// One record per recovered edge n -> q: q runs over the union list, n over
// q's row (entries with a below q's largest hit level); the record's mask is
// the OR over columns of q's column mask where the edge is tight and n had
// not stopped (the sweep's condition).
__global__ void __launch_bounds__(kSgThreads) k_sg_edges(DevKG g, DevSlot s, SgDev sg, int run) {
  const Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const int nt = run == 0 ? q.n_c : q.n_m;
  const uint32_t kind = run == 0 ? kSgEc : kSgEm;
  const uint32_t nu = min(c->ulist_n, s.cap);
  __shared__ uint32_t s_off[kSgThreads];
  __shared__ uint32_t s_rb[kSgThreads];
  __shared__ uint32_t s_q[kSgThreads];
  __shared__ uint64_t s_warp[33];
  __shared__ uint32_t s_total;
  for (uint32_t base = blockIdx.x * blockDim.x; base < nu; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    uint32_t len = 0, rb = 0, qn = 0;
    if (i < nu) {
      qn = s.ulist[i];
      const uint32_t vb = vis_byte(s.vis, qn);
      uint32_t hmax = 0;
      for (int j = 0; j < nt; ++j)
        if (((vb >> j) & 1u) && rmcol(q, j)[qn]) hmax = max(hmax, uint32_t(hcol(q, j)[qn]));
      if (hmax > 0) {
        rb = g.row_ptr[qn];
        len = seg_at(g, qn, rb, g.row_ptr[qn + 1], hmax) - rb;
      }
    }
    uint64_t tot = 0;
    const uint32_t pre = uint32_t(block_excl_scan(len, s_warp, &tot));
    s_off[threadIdx.x] = pre;
    s_rb[threadIdx.x] = rb;
    s_q[threadIdx.x] = qn;
    if (threadIdx.x == 0) s_total = uint32_t(tot);
    __syncthreads();
    const uint32_t total = s_total;
    for (uint32_t u = threadIdx.x; u < total; u += blockDim.x) {
      uint32_t lo = 0, hi = blockDim.x - 1;
      while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo + 1) >> 1);
        if (s_off[mid] <= u) lo = mid; else hi = mid - 1;
      }
      const uint32_t xe = __ldg(g.adj + s_rb[lo] + (u - s_off[lo]));
      const uint32_t a = xe >> kNodeBits, nb = xe & kNodeMask, qq = s_q[lo];
      const uint32_t vq = vis_byte(s.vis, qq), vn = vis_byte(s.vis, nb);
      unsigned long long mask = 0;
      for (int j = 0; j < nt; ++j) {
        if (!((vq >> j) & 1u) || !((vn >> j) & 1u)) continue;
        const unsigned long long m = rmcol(q, j)[qq];
        if (!m) continue;
        const uint32_t hq = hcol(q, j)[qq], hn = hcol(q, j)[nb];
        const uint32_t lam = a > hn ? a : hn;
        if (lam + 1 != hq || stopped_before(s, nb, lam)) continue;
        mask |= m;
      }
      if (mask) emit(sg, mask, nb, (kind << kNodeBits) | qq);
    }
    __syncthreads();
  }
}

// Node records of the union list (V^c or V^m with their CG masks); in run 0
// also V_C (nodes holding a central keyword) and the (g, node) pairs of V_C
// the marginal run matches against.  Clears the masks for the next sweep.
__global__ void k_sg_nodes(DevSlot s, SgDev sg, int run) {
  Ctl* c = s.ctl;
  const QueryDev& q = *s.q;
  const int nt = run == 0 ? q.n_c : q.n_m;
  const uint32_t nu = min(c->ulist_n, s.cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += gridDim.x * blockDim.x) {
    const uint32_t v = s.ulist[i];
    const unsigned long long m = s.vmask[v];
    s.vmask[v] = 0;
    for (int j = 0; j < nt; ++j) rmcol(q, j)[v] = 0;
    emit(sg, m, v, (run == 0 ? kSgVc : kSgVm) << kNodeBits);
    if (run != 0) continue;
    const uint32_t vb = vis_byte(s.vis, v);
    bool holds = false;
    for (int j = 0; j < nt; ++j) holds |= ((vb >> j) & 1u) && hcol(q, j)[v] == 0;
    if (!holds) continue;
    emit(sg, m, v, kSgVcKw << kNodeBits);
    for (unsigned long long b = m; b; b &= b - 1) {
      const uint32_t gi = uint32_t(__ffsll(static_cast<long long>(b)) - 1);
      const uint32_t p = atomicAdd(&c->nvc, 1u);
      if (p < s.cap) s.vcl[p] = (gi << kNodeBits) | v; else atomicOr(&c->err, kErrOverflow);
    }
  }
}

// Result rank of every selected CG (results are ranked by k_results).
__global__ void k_sg_rank(DevSlot s, SgDev sg) {
  const Ctl* c = s.ctl;
  const rpq_result* res = reinterpret_cast<const rpq_result*>(s.res);
  const uint32_t gi = threadIdx.x;
  if (gi >= uint32_t(kMaxK)) return;
  int32_t r = -1;
  const uint32_t nr = min(c->n_res, uint32_t(kMaxK));
  if (gi < c->nsel)
    for (uint32_t i = 0; i < nr; ++i)
      if (res[i].node == c->sel[gi]) r = int32_t(i);
  sg.ctl->rank[gi] = r;
  for (uint32_t k = 0; k < kSgKinds; ++k) sg.ctl->cnt[k][gi] = 0, sg.ctl->cur[k][gi] = 0;
}

// List lengths per (kind, rank).
__global__ void k_sg_count(SgDev sg) {
  __shared__ uint32_t h[kSgKinds * kMaxK];
  __shared__ int32_t rk[kMaxK];
  for (uint32_t t = threadIdx.x; t < kSgKinds * kMaxK; t += blockDim.x) h[t] = 0;
  for (uint32_t t = threadIdx.x; t < uint32_t(kMaxK); t += blockDim.x) rk[t] = sg.ctl->rank[t];
  __syncthreads();
  const uint32_t n = min(sg.ctl->nrec, sg.rec_cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const SgRec r = sg.rec[i];
    const uint32_t kind = r.b >> kNodeBits;
    for (unsigned long long b = r.mask; b; b &= b - 1) {
      const int32_t rr = rk[__ffsll(static_cast<long long>(b)) - 1];
      if (rr >= 0) atomicAdd(&h[kind * kMaxK + uint32_t(rr)], 1u);
    }
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < kSgKinds * kMaxK; t += blockDim.x)
    if (h[t]) atomicAdd(&sg.ctl->cnt[t / kMaxK][t % kMaxK], h[t]);
}

// Offsets of the per-result lists and of the PTC hash tables (one thread).
__global__ void k_sg_offsets(DevSlot s, SgDev sg) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  SgCtl* t = sg.ctl;
  const uint32_t nr = min(s.ctl->n_res, uint32_t(kMaxK));
  unsigned long long an = 0, ae = 0, ah = 0;
  for (uint32_t r = 0; r < uint32_t(kMaxK); ++r) {
    for (uint32_t l = 0; l < 3; ++l) {
      t->node_off[3 * r + l] = an;
      if (r < nr) an += t->cnt[kSgVc + l][r];
    }
    for (uint32_t l = 0; l < 2; ++l) {
      t->edge_off[2 * r + l] = ae;
      if (r < nr) ae += t->cnt[kSgEc + l][r];
    }
    t->hoff[r] = ah;
    if (r < nr) {
      const unsigned long long need = 2ull * (t->cnt[kSgVc][r] + t->cnt[kSgVm][r]) + 2ull;
      unsigned long long cap = 64;
      while (cap < need) cap <<= 1;
      ah += cap;
    }
    t->ptc[r] = -1;
  }
  t->node_off[3 * kMaxK] = an;
  t->edge_off[2 * kMaxK] = ae;
  t->hoff[kMaxK] = ah;
}

// Records -> per-result lists (node ids; (n, q) edge pairs).
__global__ void k_sg_scatter(SgDev sg) {
  SgCtl* t = sg.ctl;
  const uint32_t n = min(t->nrec, sg.rec_cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const SgRec r = sg.rec[i];
    const uint32_t kind = r.b >> kNodeBits;
    for (unsigned long long b = r.mask; b; b &= b - 1) {
      const int32_t rr = t->rank[__ffsll(static_cast<long long>(b)) - 1];
      if (rr < 0) continue;
      if (kind < kSgEc) {
        const unsigned long long pos = t->node_off[3 * rr + kind] + atomicAdd(&t->cur[kind][rr], 1u);
        if (pos < sg.nodes_cap) sg.nodes[pos] = r.a; else atomicOr(&t->err, kSgErrCap);
      } else {
        const unsigned long long pos = t->edge_off[2 * rr + (kind - kSgEc)] + atomicAdd(&t->cur[kind][rr], 1u);
        if (pos < sg.edges_cap) sg.edges[pos] = make_uint2(r.a, r.b & kNodeMask); else atomicOr(&t->err, kSgErrCap);
      }
    }
  }
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t v, uint32_t mask) { return (v * 2654435761u) & mask; }

// Slot of v in a table of hc (a power of two) slots, inserting it if absent.
__device__ __forceinline__ uint32_t hash_insert(uint32_t* key, uint32_t hc, uint32_t v) {
  uint32_t h = hash_slot(v, hc - 1);
  for (uint32_t probe = 0; probe < hc; ++probe) {
    const uint32_t k = atomicCAS(&key[h], kEmptyKey, v);
    if (k == kEmptyKey || k == v) return h;
    h = (h + 1) & (hc - 1);
  }
  return kEmptyKey;
}

__device__ __forceinline__ uint32_t hash_find(const uint32_t* key, uint32_t hc, uint32_t v) {
  uint32_t h = hash_slot(v, hc - 1);
  for (uint32_t probe = 0; probe < hc; ++probe) {
    const uint32_t k = __ldcg(&key[h]);
    if (k == v) return h;
    if (k == kEmptyKey) return kEmptyKey;
    h = (h + 1) & (hc - 1);
  }
  return kEmptyKey;
}

// Pass Through Constraint (Definition 5) of result r = blockIdx.x.  The
// marginal keyword nodes are the nodes of V^c U V^m holding a marginal
// keyword (marginal hit level 0, the marginal run being the last one).
__global__ void __launch_bounds__(kPtcThreads) k_sg_ptc(DevSlot s, SgDev sg) {
  SgCtl* t = sg.ctl;
  const uint32_t r = blockIdx.x;
  if (r >= min(s.ctl->n_res, uint32_t(kMaxK))) return;
  const int nm = s.q->n_m;
  if (nm == 0) return;                                   // ptc stays -1
  const unsigned long long hb = t->hoff[r];
  const uint32_t hc = uint32_t(t->hoff[r + 1] - hb);
  uint32_t* key = sg.hkey + hb;
  uint32_t* lab = sg.hlab + hb;
  uint32_t* flg = sg.hflag + hb;
  const unsigned long long vc0 = t->node_off[3 * r + kSgVc], vc1 = t->node_off[3 * r + kSgVc + 1];
  const unsigned long long kw0 = t->node_off[3 * r + kSgVcKw], kw1 = t->node_off[3 * r + kSgVcKw + 1];
  const unsigned long long vm0 = t->node_off[3 * r + kSgVm], vm1 = t->node_off[3 * r + kSgVm + 1];
  const unsigned long long e0 = t->edge_off[2 * r], e1 = t->edge_off[2 * r + 2];
  const uint32_t nvc = uint32_t(vc1 - vc0), nv = nvc + uint32_t(vm1 - vm0);
  __shared__ uint32_t s_cmin[kMaxCols], s_multi[kMaxCols], s_nonempty[kMaxCols];
  __shared__ uint32_t s_holds1, s_err;
  for (uint32_t i = threadIdx.x; i < hc; i += blockDim.x) key[i] = kEmptyKey, lab[i] = kEmptyKey, flg[i] = 0;
  if (threadIdx.x < uint32_t(kMaxCols)) s_cmin[threadIdx.x] = kEmptyKey, s_multi[threadIdx.x] = 0, s_nonempty[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_holds1 = 0, s_err = 0;
  __syncthreads();
  // nodes of G^r with their marginal keyword bits
  for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
    const uint32_t v = i < nvc ? sg.nodes[vc0 + i] : sg.nodes[vm0 + (i - nvc)];
    const uint32_t h = hash_insert(key, hc, v);
    if (h == kEmptyKey) { atomicOr(&s_err, kSgErrLookup); continue; }
    const uint32_t vb = vis_byte(s.vis, v);
    uint32_t hold = 0;
    for (int j = 0; j < nm; ++j)
      if (((vb >> j) & 1u) && hcol(*s.q, j)[v] == 0) hold |= 1u << j;
    atomicExch(&lab[h], v);
    if (hold) atomicOr(&flg[h], hold);
  }
  __syncthreads();
  for (unsigned long long i = kw0 + threadIdx.x; i < kw1; i += blockDim.x) {
    const uint32_t h = hash_find(key, hc, sg.nodes[i]);
    if (h == kEmptyKey) atomicOr(&s_err, kSgErrLookup); else atomicOr(&flg[h], kFlagVC);
  }
  __syncthreads();
  // components of G^r without V_C: min-label propagation along the edges
  const uint32_t limit = nv + 2;
  uint32_t iter = 0;
  for (; iter < limit; ++iter) {
    int changed = 0;
    for (unsigned long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const uint2 ed = sg.edges[e];
      const uint32_t hu = hash_find(key, hc, ed.x), hv = hash_find(key, hc, ed.y);
      if (hu == kEmptyKey || hv == kEmptyKey) { atomicOr(&s_err, kSgErrLookup); continue; }
      if ((__ldcg(&flg[hu]) | __ldcg(&flg[hv])) & kFlagVC) continue;
      const uint32_t lu = __ldcg(&lab[hu]), lv = __ldcg(&lab[hv]);
      if (lu < lv) { atomicMin(&lab[hv], lu); changed = 1; }
      else if (lv < lu) { atomicMin(&lab[hu], lv); changed = 1; }
    }
    if (!__syncthreads_or(changed)) break;
  }
  if (iter == limit && threadIdx.x == 0) atomicOr(&s_err, kSgErrLimit);
  // |M| = 1: mark the components that have an edge into V_C
  if (nm == 1) {
    for (unsigned long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const uint2 ed = sg.edges[e];
      const uint32_t hu = hash_find(key, hc, ed.x), hv = hash_find(key, hc, ed.y);
      if (hu == kEmptyKey || hv == kEmptyKey) continue;
      const bool cu = __ldcg(&flg[hu]) & kFlagVC, cv = __ldcg(&flg[hv]) & kFlagVC;
      if (cu == cv) continue;
      const uint32_t hl = hash_find(key, hc, __ldcg(&lab[cu ? hv : hu]));
      if (hl != kEmptyKey) atomicOr(&flg[hl], kFlagTouch);
    }
    __syncthreads();
  }
  // component label of every marginal keyword node (a node of V_C is its own component)
  for (uint32_t i = threadIdx.x; i < hc; i += blockDim.x) {
    const uint32_t v = __ldcg(&key[i]);
    if (v == kEmptyKey) continue;
    const uint32_t f = __ldcg(&flg[i]);
    const uint32_t hold = f & 0xffu;
    if (!hold) continue;
    const uint32_t l = (f & kFlagVC) ? v : __ldcg(&lab[i]);
    for (uint32_t b = hold; b; b &= b - 1) {
      const int j = __ffs(int(b)) - 1;
      atomicMin(&s_cmin[j], l);
      s_nonempty[j] = 1;
    }
    if (nm == 1) {
      const uint32_t hl = (f & kFlagVC) ? i : hash_find(key, hc, l);
      if ((f & kFlagVC) || (hl != kEmptyKey && (__ldcg(&flg[hl]) & kFlagTouch))) s_holds1 = 1;
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < hc; i += blockDim.x) {
    const uint32_t v = __ldcg(&key[i]);
    if (v == kEmptyKey) continue;
    const uint32_t f = __ldcg(&flg[i]);
    const uint32_t l = (f & kFlagVC) ? v : __ldcg(&lab[i]);
    for (uint32_t b = f & 0xffu; b; b &= b - 1) {
      const int j = __ffs(int(b)) - 1;
      if (l != s_cmin[j]) s_multi[j] = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t p = 0;
    if (nm == 1) {
      p = int32_t(s_holds1);
    } else {
      // two holders of different keywords in different components exist unless
      // both keywords' holders all share one and the same component
      for (int i = 0; i < nm && !p; ++i)
        for (int j = i + 1; j < nm && !p; ++j)
          if (s_nonempty[i] && s_nonempty[j] && (s_multi[i] || s_multi[j] || s_cmin[i] != s_cmin[j])) p = 1;
    }
    t->ptc[r] = p;
    if (s_err) atomicOr(&t->err, s_err);
  }
}

}  // namespace

// ------------------------------------------------------------- host side
void free_subgraph_scratch(rpq_kg* kg) {
  SgScratch* x = kg->sg;
  if (!x) return;
  cudaFree(x->d.ctl);
  cudaFree(x->d.rec);
  cudaFree(x->d.nodes);
  cudaFree(x->d.edges);
  cudaFree(x->d.hkey);                   // hlab and hflag live in the same block
  cudaFreeHost(x->h_ctl);
  delete x;
  kg->sg = nullptr;
}

// Grow a device array to at least `need` elements (contents dropped).
template <typename T, typename C>
static int grow(T** p, C* cap, unsigned long long need) {
  if (*p && static_cast<unsigned long long>(*cap) >= need) return RPQ_OK;
  unsigned long long n = std::max<unsigned long long>(need + need / 2, 1024);
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  RPQ_CUDA(cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * n));
  *cap = static_cast<C>(n);
  return RPQ_OK;
}

static int ensure_scratch(rpq_kg* kg) {
  if (kg->sg) return RPQ_OK;
  SgScratch* x = new SgScratch();
  kg->sg = x;
  RPQ_CUDA(cudaMalloc(reinterpret_cast<void**>(&x->d.ctl), sizeof(SgCtl)));
  RPQ_CUDA(cudaMallocHost(reinterpret_cast<void**>(&x->h_ctl), sizeof(SgCtl)));
  return grow(&x->d.rec, &x->d.rec_cap, 1ull << 16);
}

// Central run, its recovery, the marginal run and its recovery, list sizes.
// Returns the number of kernels launched.
static int enqueue_search(rpq_kg* kg, Slot* s, const QueryDev& qv, const SgDev& sg) {
  const DevKG& g = kg->dev;
  const DevSlot& d = s->d;
  cudaStream_t st = s->st;
  const int sms = num_sms();
  launch_query_setup(d, qv, nullptr, st);
  launch_central_part(g, d, qv.L, st, nullptr);
  k_sg_begin<<<1, 32, 0, st>>>(d, sg, 0);
  k_sg_sweep<<<kMaxCols, kSwThreads, 0, st>>>(g, d, 0);
  k_sg_edges<<<sms * 2, kSgThreads, 0, st>>>(g, d, sg, 0);
  k_sg_nodes<<<sms, kSgThreads, 0, st>>>(d, sg, 0);
  if (qv.n_m > 0) {
    launch_run_setup(g, d, 1, st, nullptr);
    for (int l = 0; l <= qv.L; ++l) launch_level(g, d, 1, st, nullptr, 0, false);
  }
  launch_results(d, st, nullptr);
  if (qv.n_m > 0) {
    k_sg_begin<<<1, 32, 0, st>>>(d, sg, 1);
    k_sg_sweep<<<kMaxCols, kSwThreads, 0, st>>>(g, d, 1);
    k_sg_edges<<<sms * 2, kSgThreads, 0, st>>>(g, d, sg, 1);
    k_sg_nodes<<<sms, kSgThreads, 0, st>>>(d, sg, 1);
  }
  k_sg_rank<<<1, kMaxK, 0, st>>>(d, sg);
  k_sg_count<<<sms, kSgThreads, 0, st>>>(sg);
  k_sg_offsets<<<1, 32, 0, st>>>(d, sg);
  // k_set_query, k_seed, levels (k_enqueue, k_expand; + k_target in the
  // marginal run), k_topk, 4 recovery passes, [k_run_start, k_seed, levels,
  // 4 recovery passes], k_results, k_sg_rank/count/offsets
  const int levels = qv.L + 1;
  return 1 + 1 + 2 * levels + 1 + 4 + (qv.n_m > 0 ? 2 + 3 * levels + 4 : 0) + 1 + 3;
}

}  // namespace rpq

using namespace rpq;

extern "C" int rpq_search_subgraphs(rpq_kg* kg, const rpq_query* q, rpq_result* out, int32_t* n_out,
                                    rpq_stats* stats, rpq_subgraphs* sgo) {
  ApiRange nvtx_range("rpq_search_subgraphs");
  if (!kg || !out || !n_out || !sgo) { set_error(RPQ_EINVAL, "NULL argument"); return RPQ_EINVAL; }
  if (sgo->nodes_cap < 0 || sgo->edges_cap < 0 || (sgo->nodes_cap > 0 && !sgo->nodes) ||
      (sgo->edges_cap > 0 && !sgo->edges)) {
    set_error(RPQ_EINVAL, "bad subgraph buffer");
    return RPQ_EINVAL;
  }
  QueryDev qv;
  bool empty = false;
  int rc = check_query(kg, q, &qv, &empty);
  if (rc != RPQ_OK) return rc;
  memset(sgo->node_off, 0, sizeof(sgo->node_off));
  memset(sgo->edge_off, 0, sizeof(sgo->edge_off));
  for (int r = 0; r < kMaxK; ++r) sgo->ptc[r] = -1;
  sgo->nodes_total = sgo->edges_total = 0;
  if (empty) { empty_result(n_out, stats); return RPQ_OK; }
  Slot* s = nullptr;
  rc = get_slot(kg, 0, &s);
  if (rc != RPQ_OK) return rc;
  rc = ensure_scratch(kg);
  if (rc != RPQ_OK) return rc;
  SgScratch* x = kg->sg;
  cudaStream_t st = s->st;
  const int sms = num_sms();
  int kernels = 0;
  for (int attempt = 0;; ++attempt) {
    kernels = enqueue_search(kg, s, qv, x->d);
    RPQ_CUDA(cudaGetLastError());
    RPQ_CUDA(cudaMemcpyAsync(s->h_ctl, s->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA(cudaMemcpyAsync(x->h_ctl, x->d.ctl, sizeof(SgCtl), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA(cudaStreamSynchronize(st));
    rc = dev_err_to_status(s->h_ctl->err);
    if (rc != RPQ_OK) return rc;
    if (x->h_ctl->nrec <= x->d.rec_cap) break;
    if (attempt >= 2) { set_error(RPQ_EINTERNAL, "subgraph record count unstable"); return RPQ_EINTERNAL; }
    rc = grow(&x->d.rec, &x->d.rec_cap, x->h_ctl->nrec);
    if (rc != RPQ_OK) return rc;
  }
  const Ctl c = *s->h_ctl;
  const int32_t nr = int32_t(std::min<uint32_t>(c.n_res, uint32_t(qv.k)));
  const unsigned long long nodes_total = x->h_ctl->node_off[3 * kMaxK];
  const unsigned long long edges_total = x->h_ctl->edge_off[2 * kMaxK];
  const unsigned long long hash_total = x->h_ctl->hoff[kMaxK];
  rc = grow(&x->d.nodes, &x->d.nodes_cap, nodes_total);
  if (rc == RPQ_OK) rc = grow(&x->d.edges, &x->d.edges_cap, edges_total);
  if (rc == RPQ_OK && x->d.hash_cap < hash_total) {   // key, label and flag arrays in one block
    unsigned long long words = 0;
    x->d.hash_cap = 0;
    rc = grow(&x->d.hkey, &words, 3 * hash_total);
    if (rc == RPQ_OK) {
      x->d.hash_cap = words / 3;
      x->d.hlab = x->d.hkey + x->d.hash_cap;
      x->d.hflag = x->d.hlab + x->d.hash_cap;
    }
  }
  if (rc != RPQ_OK) return rc;
  k_sg_scatter<<<sms, kSgThreads, 0, st>>>(x->d);
  k_sg_ptc<<<kMaxK, kPtcThreads, 0, st>>>(s->d, x->d);
  RPQ_CUDA(cudaGetLastError());
  RPQ_CUDA(cudaMemcpyAsync(x->h_ctl, x->d.ctl, sizeof(SgCtl), cudaMemcpyDeviceToHost, st));
  RPQ_CUDA(cudaMemcpyAsync(s->h_res, s->d.res, sizeof(rpq_result) * size_t(std::max(nr, 1)), cudaMemcpyDeviceToHost, st));
  RPQ_CUDA(cudaStreamSynchronize(st));
  if (x->h_ctl->err) {
    set_error(RPQ_EINTERNAL, "subgraph pass failed (flags 0x%x)", x->h_ctl->err);
    return RPQ_EINTERNAL;
  }
  memcpy(out, s->h_res, sizeof(rpq_result) * size_t(nr));
  *n_out = nr;
  fill_stats(c, stats);
  if (stats) stats->kernels = kernels + 2;      // + k_sg_scatter, k_sg_ptc
  for (int t = 0; t <= 3 * kMaxK; ++t) sgo->node_off[t] = int64_t(x->h_ctl->node_off[t]);
  for (int t = 0; t <= 2 * kMaxK; ++t) sgo->edge_off[t] = int64_t(x->h_ctl->edge_off[t]);
  for (int r = 0; r < kMaxK; ++r) sgo->ptc[r] = r < nr ? x->h_ctl->ptc[r] : -1;
  sgo->nodes_total = int64_t(nodes_total);
  sgo->edges_total = int64_t(edges_total);
  if (int64_t(nodes_total) > sgo->nodes_cap || int64_t(edges_total) > sgo->edges_cap) {
    set_error(RPQ_ESIZE, "subgraph lists need %llu nodes and %llu edges", nodes_total, edges_total);
    return RPQ_ESIZE;
  }
  if (nodes_total)
    RPQ_CUDA(cudaMemcpy(sgo->nodes, x->d.nodes, sizeof(uint32_t) * nodes_total, cudaMemcpyDeviceToHost));
  if (edges_total)
    RPQ_CUDA(cudaMemcpy(sgo->edges, x->d.edges, sizeof(uint2) * edges_total, cudaMemcpyDeviceToHost));
  // the lists hold internal ids: give them back in the caller's ids
  for (uint64_t i = 0; i < nodes_total; ++i) sgo->nodes[i] = kg->ext_of[size_t(sgo->nodes[i])];
  for (uint64_t i = 0; i < 2 * edges_total; ++i) sgo->edges[i] = kg->ext_of[size_t(sgo->edges[i])];
  return RPQ_OK;
}
