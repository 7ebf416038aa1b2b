// Graph load: edge activation levels on the device (Section 3.1, Eq. 1-3).
//
// For every CSR entry u->v with label l the fine-grained weight is
//   w = log(#out-edges of u labelled l + #in-edges of v labelled l).
// On the bi-directed graph (every edge has its reverse with the same label,
// Section 2) the in-edges of v labelled l are exactly v's out-edges labelled
// l, so the count is dl(u->v) + dl(v->u), where dl(e) is the number of
// entries in e's row that share e's label.  The weight depends only on this
// integer count; the host evaluates log, the min-max rescale and Eq. 1-3 in
// IEEE double once per distinct count and the device looks the level up.
//
// Kernels, in order:
//   k_rows_small   rows of <= 32 entries: validation + dl via __match_any_sync
//   k_rows_large   rows of > 32 entries: validation + dl via a shared-memory
//                  label histogram (one block per row)
//   k_count        cnt(e) = dl(e) + dl(reverse(e)); reverse found by binary
//                  search in the neighbour's ascending row; checks symmetry;
//                  global min/max of cnt
//   k_presence     marks the counts that occur
//   k_pack         adj(e) = level(cnt(e)) << 26 | neighbour
//   k_relabel      rows and neighbours renumbered to the internal ids
//   k_sort_small / k_sort_pass   per-row sort by (level, neighbour): rank
//                  sort in a warp; for longer rows, stable counting sorts by
//                  6-bit digits in a block (neighbour bits, then the level);
//                  both also write amax(u)
//
// Internal node ids.  The search numbers nodes by decreasing degree (ties by
// the caller's id): on a power-law graph most CSR entries point at the few
// high-degree nodes, and with this numbering their visited bytes, hit levels
// and bit-map words share a few hundred kilobytes of cache lines instead of
// being scattered over the whole per-node arrays.  Node ids cross the
// boundary in the caller's numbering: postings are renumbered at load, and
// results, traces, subgraphs and exports are given back in caller ids.  The
// identification keys of CGs carry caller ids, so every tie between equal
// scores is still broken by the caller's node id.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rpq_host.h"

namespace rpq {

namespace {

constexpr int kSortWarps = 8;

__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

// Rows with at most 32 entries: one warp per row.
__global__ void k_rows_small(int32_t n, const uint32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const uint16_t* __restrict__ label, int32_t n_labels, uint32_t* __restrict__ dl,
                             uint32_t* err) {
  const uint32_t lane = lane_id();
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    const uint32_t rb = row_ptr[u], re = row_ptr[u + 1];
    const uint32_t d = re - rb;
    if (d > 32 || d == 0) continue;
    const unsigned active = __ballot_sync(0xffffffffu, lane < d);
    if (lane < d) {
      const int32_t c = col[rb + lane];
      const uint32_t lab = label[rb + lane];
      const int32_t prev = __shfl_up_sync(active, c, 1);
      uint32_t bad = 0;
      if (c < 0 || c >= n || c == u) bad |= kErrBadCol;
      if (lane > 0 && c <= prev) bad |= kErrUnsorted;
      if (lab >= uint32_t(n_labels)) bad |= kErrBadLabel;
      if (bad) set_err(err, bad);
      dl[rb + lane] = __popc(__match_any_sync(active, lab));
    }
  }
}

// Rows with more than 32 entries: one block per row, label histogram in
// shared memory (n_labels <= kMaxLabels counters).
__global__ void k_rows_large(int32_t n, const uint32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const uint16_t* __restrict__ label, int32_t n_labels, uint32_t* __restrict__ dl,
                             uint32_t* err) {
  extern __shared__ uint32_t hist[];
  for (int64_t u = blockIdx.x; u < n; u += gridDim.x) {
    const uint32_t rb = row_ptr[u], re = row_ptr[u + 1];
    if (re - rb <= 32) continue;  // same decision in every thread of the block
    for (int32_t i = threadIdx.x; i < n_labels; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    uint32_t bad = 0;
    for (uint32_t e = rb + threadIdx.x; e < re; e += blockDim.x) {
      const int32_t c = col[e];
      const uint32_t lab = label[e];
      if (c < 0 || c >= n || c == u) bad |= kErrBadCol;
      if (e > rb && c <= col[e - 1]) bad |= kErrUnsorted;
      if (lab >= uint32_t(n_labels)) bad |= kErrBadLabel;
      else atomicAdd(&hist[lab], 1u);
    }
    if (bad) set_err(err, bad);
    __syncthreads();
    for (uint32_t e = rb + threadIdx.x; e < re; e += blockDim.x) {
      const uint32_t lab = label[e];
      dl[e] = lab < uint32_t(n_labels) ? hist[lab] : 0u;
    }
    __syncthreads();
  }
}

// Row containing entry e: the last r in [lo, hi] with row_ptr[r] <= e.
__device__ __forceinline__ uint32_t row_of(const uint32_t* row_ptr, uint32_t lo, uint32_t hi, uint32_t e) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo + 1) >> 1);
    if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// cnt(e) = dl(e) + dl(reverse e); one warp per 32 consecutive entries.
__global__ void k_count(int32_t n, uint32_t m2, const uint32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                        const uint16_t* __restrict__ label, const uint32_t* __restrict__ dl,
                        uint32_t* __restrict__ cnt, uint32_t* cmin, uint32_t* cmax, uint32_t* err) {
  const uint32_t lane = lane_id();
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t lmin = 0xffffffffu, lmax = 0;
  for (int64_t base = warp * 32; base < m2; base += nwarps * 32) {
    // rows of the chunk's first and last entries (the same searches in every
    // lane); runs of empty rows may lie between them, so lanes search that range
    const uint32_t r0 = row_of(row_ptr, 0, uint32_t(n - 1), uint32_t(base));
    const uint32_t last = uint32_t(base + 31 < int64_t(m2) ? base + 31 : int64_t(m2) - 1);
    const uint32_t r1 = row_of(row_ptr, r0, uint32_t(n - 1), last);
    const uint32_t e = uint32_t(base) + lane;
    if (e < m2) {
      const uint32_t u = row_of(row_ptr, r0, r1, e);
      const int32_t v = col[e];
      uint32_t c = 0;
      if (v >= 0 && v < n) {
        uint32_t lo = row_ptr[v], h = row_ptr[v + 1];  // reverse entry v->u
        while (lo < h) {
          const uint32_t mid = lo + ((h - lo) >> 1);
          if (uint32_t(col[mid]) < u) lo = mid + 1; else h = mid;
        }
        if (lo < row_ptr[v + 1] && uint32_t(col[lo]) == u && label[lo] == label[e]) {
          c = dl[e] + dl[lo];
        } else {
          set_err(err, kErrAsym);
        }
      }
      cnt[e] = c;
      if (c) { lmin = min(lmin, c); lmax = max(lmax, c); }
    }
  }
  for (int o = 16; o; o >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  if (lane == 0) {
    if (lmin != 0xffffffffu) atomicMin(cmin, lmin);
    if (lmax) atomicMax(cmax, lmax);
  }
}

__global__ void k_presence(uint32_t m2, const uint32_t* __restrict__ cnt, uint32_t cmin, uint32_t ncnt,
                           uint8_t* present) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m2; e += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t c = cnt[e] - cmin;
    if (c < ncnt && !present[c]) present[c] = 1;
  }
}

// adj(e) = level << 26 | neighbour, written over cnt.
__global__ void k_pack(uint32_t m2, uint32_t* __restrict__ cnt_adj, const int32_t* __restrict__ col,
                       const uint8_t* __restrict__ table, uint32_t cmin, uint32_t ncnt) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m2; e += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t c = cnt_adj[e] - cmin;
    const uint32_t a = c < ncnt ? table[c] : 0u;
    cnt_adj[e] = (a << kNodeBits) | uint32_t(col[e]);
  }
}

// Renumbered rows: entry e of caller row u goes to row to_new[u] of the
// renumbered CSR (same offset in the row) with its neighbour renumbered.
// Also used the other way round (to_new = internal -> caller ids) for exports.
// One warp per 32 consecutive entries, rows located as in k_count.
__global__ void k_relabel(int32_t n, uint32_t m2, const uint32_t* __restrict__ row_ptr,
                          const uint32_t* __restrict__ new_row_ptr, const int32_t* __restrict__ to_new,
                          const uint32_t* __restrict__ in, uint32_t* __restrict__ out) {
  const uint32_t lane = lane_id();
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < m2; base += nwarps * 32) {
    const uint32_t r0 = row_of(row_ptr, 0, uint32_t(n - 1), uint32_t(base));
    const uint32_t last = uint32_t(base + 31 < int64_t(m2) ? base + 31 : int64_t(m2) - 1);
    const uint32_t r1 = row_of(row_ptr, r0, uint32_t(n - 1), last);
    const uint32_t e = uint32_t(base) + lane;
    if (e < m2) {
      const uint32_t u = row_of(row_ptr, r0, r1, e);
      const uint32_t x = in[e];
      const uint32_t nu = uint32_t(to_new[u]);
      out[new_row_ptr[nu] + (e - row_ptr[u])] = (x & ~kNodeMask) | uint32_t(to_new[x & kNodeMask]);
    }
  }
}

// Rows of <= 32 entries: rank sort in a warp (values are distinct in a row);
// in place is allowed (every lane reads before any lane writes).
__global__ void k_sort_small(int32_t n, const uint32_t* __restrict__ row_ptr, const uint32_t* in,
                             uint32_t* out, uint8_t* __restrict__ amax) {
  const uint32_t lane = lane_id();
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps) {
    const uint32_t rb = row_ptr[u], d = row_ptr[u + 1] - rb;
    if (d > 32) continue;
    const uint32_t x = lane < d ? in[rb + lane] : 0xffffffffu;
    uint32_t rank = 0;
    for (int j = 0; j < 32; ++j) rank += (__shfl_sync(0xffffffffu, x, j) < x);
    if (lane < d) out[rb + rank] = x;
    uint32_t lv = lane < d ? (x >> kNodeBits) : 0u;
    for (int o = 16; o; o >>= 1) lv = max(lv, __shfl_xor_sync(0xffffffffu, lv, o));
    if (lane == 0 && amax) amax[u] = uint8_t(lv);
  }
}

// Rows of > 32 entries: stable counting sort by the 6-bit digit at `shift`
// (a pass of a least-significant-digit radix sort: the neighbour bits at
// shifts 0, 6, 12, 18, 24, then the level at 26 gives (level, neighbour)
// order; the level pass also writes amax when it is given).  One block of
// kSortWarps warps per row; chunks of blockDim entries are placed in order.
__global__ void __launch_bounds__(kSortWarps * 32)
k_sort_pass(int32_t n, const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ in,
            uint32_t* __restrict__ out, uint32_t shift, uint8_t* __restrict__ amax) {
  __shared__ uint32_t base[64];
  __shared__ uint32_t wcnt[kSortWarps][64];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  for (int64_t u = blockIdx.x; u < n; u += gridDim.x) {
    const uint32_t rb = row_ptr[u], re = row_ptr[u + 1];
    if (re - rb <= 32) continue;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) base[i] = 0;
    for (int i = threadIdx.x; i < kSortWarps * 64; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    for (uint32_t e = rb + threadIdx.x; e < re; e += blockDim.x) atomicAdd(&base[(in[e] >> shift) & 63u], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t s = 0, top = 0;
      for (int b = 0; b < 64; ++b) { const uint32_t c = base[b]; base[b] = s; s += c; if (c) top = b; }
      if (amax) amax[u] = uint8_t(top);
    }
    __syncthreads();
    for (uint32_t c0 = rb; c0 < re; c0 += blockDim.x) {
      const uint32_t e = c0 + threadIdx.x;
      const bool valid = e < re;
      const uint32_t x = valid ? in[e] : 0u;
      const uint32_t b = (x >> shift) & 63u;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      uint32_t r = 0;
      if (valid) {
        const unsigned m = __match_any_sync(act, b);
        r = __popc(m & ((1u << lane) - 1u));
        if (r == 0) wcnt[warp][b] = __popc(m);
      }
      __syncthreads();
      if (valid) {
        uint32_t pos = base[b] + r;
        for (uint32_t w = 0; w < warp; ++w) pos += wcnt[w][b];
        out[rb + pos] = x;
      }
      __syncthreads();
      if (threadIdx.x < 64) {
        uint32_t t = 0;
        for (int w = 0; w < kSortWarps; ++w) { t += wcnt[w][threadIdx.x]; wcnt[w][threadIdx.x] = 0; }
        base[threadIdx.x] += t;
      }
      __syncthreads();
    }
  }
}

// Level index of each row (see kLvxLevels): one thread per row; the rows
// longer than kLvxMaxDeg are left to k_level_index_long.
__global__ void k_level_index(int32_t n, const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ adj,
                              uint16_t* __restrict__ lvx) {
  for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t rb = row_ptr[v], re = row_ptr[v + 1];
    if (re - rb > kLvxMaxDeg) continue;
    for (uint32_t x = 1; x <= kLvxLevels; ++x)
      lvx[size_t(x - 1) * size_t(n) + size_t(v)] = uint16_t(seg_lower(adj, rb, re, x) - rb);
  }
}

// Level index of the long rows: one thread per (long row h, level x); the
// row's lvx entries hold h.
__global__ void k_level_index_long(int32_t n, uint32_t n_long, const uint32_t* __restrict__ long_rows,
                                   const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ adj,
                                   uint16_t* __restrict__ lvx, uint32_t* __restrict__ lvx_long) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_long * kLvxLevels) return;
  const uint32_t h = t / kLvxLevels, x = t % kLvxLevels + 1u, v = long_rows[h];
  const uint32_t rb = row_ptr[v], re = row_ptr[v + 1];
  lvx_long[t] = seg_lower(adj, rb, re, x) - rb;
  lvx[size_t(x - 1) * size_t(n) + size_t(v)] = uint16_t(h);
}

int grid_for(int64_t work, int threads) {
  const int64_t cap = int64_t(num_sms()) * 16;
  const int64_t g = (work + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min(g, cap)));
}

// Sort every row of `b` by its packed value, (level, neighbour): rows of more
// than 32 entries by six stable digit passes through `a` and back, the short
// rows in place; amax (if given) receives each row's largest level.
void sort_rows(int32_t n, const uint32_t* d_row, uint32_t* a, uint32_t* b, uint8_t* amax) {
  const int T = 256;
  const uint32_t shifts[6] = {0, 6, 12, 18, 24, kNodeBits};
  uint32_t* src = b;
  uint32_t* dst = a;
  for (int i = 0; i < 6; ++i) {
    k_sort_pass<<<num_sms() * 8, kSortWarps * 32>>>(n, d_row, src, dst, shifts[i], i == 5 ? amax : nullptr);
    std::swap(src, dst);
  }
  // six passes: the long rows are back in b
  k_sort_small<<<grid_for(int64_t(n) * 32, T), T>>>(n, d_row, b, b, amax);
}

// Host: level of each count (Eq. 1-3, round half up), evaluated as printed:
// reward = abar*(alpha-w)/alpha, penalty = abar*(w-alpha)/(1-alpha).  The
// min-max rescale uses the logarithms of the counts that occur.
int level_table(uint32_t cmin, const std::vector<uint8_t>& present, double alpha, double abar,
                std::vector<uint8_t>& table) {
  double wmin = INFINITY, wmax = -INFINITY;
  for (size_t i = 0; i < present.size(); ++i) {
    if (!present[i]) continue;
    const double w = std::log(double(cmin + i));
    wmin = std::min(wmin, w);
    wmax = std::max(wmax, w);
  }
  table.assign(present.size(), 0);
  for (size_t i = 0; i < table.size(); ++i) {
    if (!present[i]) continue;
    const double w = std::log(double(cmin + i));
    const double ws = (wmax > wmin) ? (w - wmin) / (wmax - wmin) : 0.0;
    double x;
    if (ws <= alpha) {
      const double reward = abar * (alpha - ws) / alpha;
      x = abar - reward;
    } else {
      const double penalty = abar * (ws - alpha) / (1.0 - alpha);
      x = abar + penalty;
    }
    const double r = std::floor(x + 0.5);
    if (r < 0 || r > kMaxLevel) {
      set_error(RPQ_ELIMIT, "activation level %.0f outside [0, %d] (abar too large)", r, kMaxLevel);
      return RPQ_ELIMIT;
    }
    table[i] = uint8_t(r);
  }
  return RPQ_OK;
}

}  // namespace

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    sms = (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 148;
  }
  return sms;
}

int alloc_device(void** p, size_t bytes, int64_t* counter) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error(RPQ_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return RPQ_ENOMEM;
  }
  if (counter) *counter += int64_t(bytes);
  return RPQ_OK;
}

int build_graph(rpq_kg* kg, const rpq_kg_desc* d) {
  const int32_t n = d->n;
  const uint32_t m2 = uint32_t(d->m2);
  const int T = 256;
  int rc = RPQ_OK;
  uint32_t *d_row = nullptr, *d_dl = nullptr, *d_cnt = nullptr, *d_scal = nullptr, *d_newrow = nullptr;
  int32_t* d_col = nullptr;
  uint16_t* d_lab = nullptr;
  uint8_t *d_amax = nullptr, *d_present = nullptr, *d_table = nullptr;
  std::vector<uint32_t>& row32 = kg->row_ext;
  row32.resize(size_t(n) + 1);
  for (int64_t i = 0; i <= n; ++i) row32[i] = uint32_t(d->row_ptr[i]);
  // internal numbering: decreasing degree, ties by caller id (counting sort)
  std::vector<int32_t>& ext_of = kg->ext_of;
  std::vector<int32_t>& int_of = kg->int_of;
  ext_of.resize(size_t(n));
  int_of.resize(size_t(n));
  std::vector<uint32_t> new_row32(size_t(n) + 1, 0);
  {
    uint32_t maxd = 0;
    for (int64_t v = 0; v < n; ++v) maxd = std::max(maxd, row32[v + 1] - row32[v]);
    std::vector<int64_t> start(size_t(maxd) + 2, 0);
    for (int64_t v = 0; v < n; ++v) ++start[maxd - (row32[v + 1] - row32[v]) + 1];
    for (size_t b = 1; b < start.size(); ++b) start[b] += start[b - 1];
    for (int64_t v = 0; v < n; ++v) {
      const int64_t id = start[maxd - (row32[v + 1] - row32[v])]++;
      ext_of[size_t(id)] = int32_t(v);
      int_of[size_t(v)] = int32_t(id);
    }
    for (int64_t i = 0; i < n; ++i)
      new_row32[i + 1] = new_row32[i] + (row32[ext_of[i] + 1] - row32[ext_of[i]]);
  }
  int64_t bytes = 0;
  auto cleanup = [&]() {
    cudaFree(d_dl); cudaFree(d_scal); cudaFree(d_col); cudaFree(d_lab); cudaFree(d_present); cudaFree(d_table);
    cudaFree(d_row);
    kg->device_bytes += bytes;
  };
#define TRY(x) do { rc = (x); if (rc != RPQ_OK) { cleanup(); return rc; } } while (0)
#define TRYC(call) do { const cudaError_t e_ = (call); if (e_ != cudaSuccess) { \
    set_error(RPQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); cleanup(); return RPQ_ECUDA; } } while (0)
  TRY(alloc_device((void**)&d_row, sizeof(uint32_t) * (size_t(n) + 1), nullptr));   // caller row offsets
  TRY(alloc_device((void**)&d_newrow, sizeof(uint32_t) * (size_t(n) + 1), &bytes));
  kg->d_row_ptr = d_newrow;
  TRY(alloc_device((void**)&kg->d_ext_of, sizeof(int32_t) * size_t(std::max(n, 1)), &bytes));
  TRY(alloc_device((void**)&kg->d_int_of, sizeof(int32_t) * size_t(std::max(n, 1)), &bytes));
  TRYC(cudaMemcpy(d_newrow, new_row32.data(), sizeof(uint32_t) * (size_t(n) + 1), cudaMemcpyHostToDevice));
  TRYC(cudaMemcpy(kg->d_ext_of, ext_of.data(), sizeof(int32_t) * size_t(n), cudaMemcpyHostToDevice));
  TRYC(cudaMemcpy(kg->d_int_of, int_of.data(), sizeof(int32_t) * size_t(n), cudaMemcpyHostToDevice));
  TRY(alloc_device((void**)&d_amax, size_t(n), &bytes));
  kg->d_amax = d_amax;
  TRY(alloc_device((void**)&kg->d_lvx, sizeof(uint16_t) * kLvxLevels * size_t(n), &bytes));
  TRY(alloc_device((void**)&d_cnt, sizeof(uint32_t) * size_t(m2), &bytes));
  kg->d_adj = d_cnt;  // replaced by the sorted buffer below
  TRY(alloc_device((void**)&d_col, sizeof(int32_t) * size_t(m2), nullptr));
  TRY(alloc_device((void**)&d_lab, sizeof(uint16_t) * size_t(m2), nullptr));
  TRY(alloc_device((void**)&d_dl, sizeof(uint32_t) * size_t(m2), nullptr));
  TRY(alloc_device((void**)&d_scal, sizeof(uint32_t) * 4, nullptr));
  TRYC(cudaMemcpy(d_row, row32.data(), sizeof(uint32_t) * (size_t(n) + 1), cudaMemcpyHostToDevice));
  if (m2) {
    TRYC(cudaMemcpy(d_col, d->col, sizeof(int32_t) * size_t(m2), cudaMemcpyHostToDevice));
    TRYC(cudaMemcpy(d_lab, d->label, sizeof(uint16_t) * size_t(m2), cudaMemcpyHostToDevice));
  }
  TRYC(cudaMemset(d_amax, 0, size_t(n)));
  const uint32_t init[4] = {0, 0xffffffffu, 0, 0};  // err, cmin, cmax, spare
  TRYC(cudaMemcpy(d_scal, init, sizeof(init), cudaMemcpyHostToDevice));
  uint32_t* d_err = d_scal;
  if (m2) {
    k_rows_small<<<grid_for(int64_t(n) * 32, T), T>>>(n, d_row, d_col, d_lab, d->n_labels, d_dl, d_err);
    const size_t hist_bytes = sizeof(uint32_t) * size_t(d->n_labels);
    if (hist_bytes > 48 * 1024)
      TRYC(cudaFuncSetAttribute(k_rows_large, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hist_bytes)));
    k_rows_large<<<num_sms() * 8, T, hist_bytes>>>(n, d_row, d_col, d_lab, d->n_labels, d_dl, d_err);
    k_count<<<grid_for(m2, T), T>>>(n, m2, d_row, d_col, d_lab, d_dl, d_cnt, d_scal + 1, d_scal + 2, d_err);
    TRYC(cudaGetLastError());
  }
  uint32_t scal[4];
  TRYC(cudaMemcpy(scal, d_scal, sizeof(scal), cudaMemcpyDeviceToHost));
  if (scal[0]) {
    set_error(RPQ_EINVAL, "graph rejected by the device checks (flags 0x%x:%s%s%s%s)", scal[0],
              (scal[0] & kErrBadCol) ? " neighbour id out of range or self-loop;" : "",
              (scal[0] & kErrUnsorted) ? " row not strictly ascending;" : "",
              (scal[0] & kErrBadLabel) ? " label >= n_labels;" : "",
              (scal[0] & kErrAsym) ? " missing reverse edge or label mismatch;" : "");
    cleanup();
    return RPQ_EINVAL;
  }
  if (m2) {
    const uint32_t cmin = scal[1], cmax = scal[2];
    const uint32_t ncnt = cmax - cmin + 1;
    TRY(alloc_device((void**)&d_present, ncnt, nullptr));
    TRYC(cudaMemset(d_present, 0, ncnt));
    k_presence<<<grid_for(m2, T), T>>>(m2, d_cnt, cmin, ncnt, d_present);
    std::vector<uint8_t> present(ncnt);
    TRYC(cudaMemcpy(present.data(), d_present, ncnt, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> table;
    TRY(level_table(cmin, present, d->alpha, d->abar, table));
    TRY(alloc_device((void**)&d_table, ncnt, nullptr));
    TRYC(cudaMemcpy(d_table, table.data(), ncnt, cudaMemcpyHostToDevice));
    k_pack<<<grid_for(m2, T), T>>>(m2, d_cnt, d_col, d_table, cmin, ncnt);
    uint32_t* d_sorted = reinterpret_cast<uint32_t*>(d_col);  // the old col buffer becomes adj
    k_relabel<<<grid_for(m2, T), T>>>(n, m2, d_row, d_newrow, kg->d_int_of, d_cnt, d_sorted);
    sort_rows(n, d_newrow, d_cnt, d_sorted, d_amax);
    TRYC(cudaGetLastError());
    TRYC(cudaDeviceSynchronize());
    kg->d_adj = d_sorted;  // same size as d_cnt, which it replaces
    d_col = nullptr;
    cudaFree(d_cnt);
  }
  k_level_index<<<grid_for(n, T), T>>>(n, d_newrow, kg->d_adj, kg->d_lvx);
  {
    std::vector<uint32_t> long_rows;                   // fewer than 2^16: each holds > 2^16 of m2 < 2^32 entries
    for (int64_t v = 0; v < n; ++v)
      if (new_row32[v + 1] - new_row32[v] > kLvxMaxDeg) long_rows.push_back(uint32_t(v));
    const uint32_t n_long = uint32_t(long_rows.size());
    TRY(alloc_device((void**)&kg->d_lvx_long, sizeof(uint32_t) * kLvxLevels * size_t(n_long), &bytes));
    if (n_long) {
      // d_dl (m2 entries, no longer needed) holds the list of long rows
      TRYC(cudaMemcpy(d_dl, long_rows.data(), sizeof(uint32_t) * n_long, cudaMemcpyHostToDevice));
      const uint32_t tasks = n_long * kLvxLevels;
      k_level_index_long<<<(tasks + T - 1) / T, T>>>(n, n_long, d_dl, d_newrow, kg->d_adj, kg->d_lvx, kg->d_lvx_long);
    }
  }
  TRYC(cudaGetLastError());
  TRYC(cudaDeviceSynchronize());
  cleanup();
  return RPQ_OK;
#undef TRY
#undef TRYC
}

// The packed adjacency and amax in the caller's numbering: rows in caller
// order, each sorted by (level, caller neighbour id).
int export_graph(const rpq_kg* kg, uint32_t* adj, uint8_t* amax) {
  const int32_t n = kg->dev.n;
  const uint32_t m2 = uint32_t(kg->m2);
  if (adj && m2) {
    uint32_t *a = nullptr, *b = nullptr, *row = nullptr;
    int rc = alloc_device((void**)&a, sizeof(uint32_t) * size_t(m2), nullptr);
    if (rc == RPQ_OK) rc = alloc_device((void**)&b, sizeof(uint32_t) * size_t(m2), nullptr);
    if (rc == RPQ_OK) rc = alloc_device((void**)&row, sizeof(uint32_t) * (size_t(n) + 1), nullptr);
    cudaError_t e = cudaSuccess;
    if (rc == RPQ_OK) {
      const int T = 256;
      e = cudaMemcpy(row, kg->row_ext.data(), sizeof(uint32_t) * (size_t(n) + 1), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        k_relabel<<<grid_for(m2, T), T>>>(n, m2, kg->d_row_ptr, row, kg->d_ext_of, kg->d_adj, b);
        sort_rows(n, row, a, b, nullptr);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemcpy(adj, b, sizeof(uint32_t) * size_t(m2), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) { set_error(RPQ_ECUDA, "export: %s", cudaGetErrorString(e)); rc = RPQ_ECUDA; }
    }
    cudaFree(a); cudaFree(b); cudaFree(row);
    if (rc != RPQ_OK) return rc;
  }
  if (amax && n > 0) {
    std::vector<uint8_t> in(static_cast<size_t>(n));
    RPQ_CUDA(cudaMemcpy(in.data(), kg->d_amax, size_t(n), cudaMemcpyDeviceToHost));
    for (int64_t u = 0; u < n; ++u) amax[u] = in[size_t(kg->int_of[size_t(u)])];
  }
  return RPQ_OK;
}

}  // namespace rpq
