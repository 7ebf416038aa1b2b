// rpq_topk_keys_noalloc: top-k selection that allocates no memory.
//
// Some callers cannot call cudaMalloc at the moment they need a selection:
// code running inside another library's CUDA graph capture, a real-time
// serving loop that pre-plans every allocation, or a process whose device
// memory is fully reserved by another allocator (a framework's caching pool).
// For them this entry point runs the block-local top-K merge with its
// intermediate buffers in a fixed device array that is part of the library
// image, so the call itself allocates nothing (no cudaMalloc, cudaFree,
// cudaMallocHost or stream creation).  The array costs every GPU that loads
// the library kNoAllocScratchBytes until the process exits.
#include <cstring>

#include "rpq_host.h"

namespace rpq {
namespace {

constexpr int kNaThreads = 1024;
constexpr uint32_t kNaChunk = 4096;                       // keys sorted per block
constexpr uint32_t kNaMaxKeys = 1u << 24;                 // largest accepted input
constexpr uint32_t kNaPass0Cap = (kNaMaxKeys / kNaChunk) * kMaxK;          // 262,144 keys
constexpr uint32_t kNaPass1Cap = ((kNaPass0Cap + kNaChunk - 1) / kNaChunk) * kMaxK;  // 4,096 keys
constexpr uint32_t kNaCounters = 8;
constexpr size_t kNoAllocScratchWords = size_t(kNaPass0Cap) + kNaPass1Cap + kNaCounters;
constexpr size_t kNoAllocScratchBytes = kNoAllocScratchWords * sizeof(uint32_t);   // ~1.04 MB
static_assert(kNoAllocScratchBytes < (size_t(2) << 20), "the fixed scratch must stay small");

// The scratch: pass outputs and key counts.  Shared by every call on a device.
static __device__ __align__(256) uint32_t g_topk_scratch[kNoAllocScratchWords];

// One pass of the block-local top-K merge: each block sorts a chunk of up to
// kNaChunk keys in shared memory (bitonic network sized to the chunk) and
// writes its K smallest, padded with 0xffffffff; *n_out receives the count.
__global__ void __launch_bounds__(kNaThreads)
k_topk_pass_static(const uint32_t* __restrict__ src, const uint32_t* n_in_ptr, uint32_t n_in_given,
                   uint32_t* __restrict__ dst, uint32_t* n_out, uint32_t K) {
  const uint32_t n_in = n_in_ptr ? *n_in_ptr : n_in_given;
  const uint32_t nchunks = (n_in + kNaChunk - 1) / kNaChunk;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = min(n_in, nchunks * K);
  __shared__ uint32_t key[kNaChunk];
  for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const uint32_t b = ch * kNaChunk;
    const uint32_t len = min(kNaChunk, n_in - b);
    uint32_t sz = 32;
    while (sz < len) sz <<= 1;
    for (uint32_t i = threadIdx.x; i < sz; i += blockDim.x) key[i] = i < len ? src[b + i] : 0xffffffffu;
    __syncthreads();
    for (uint32_t k = 2; k <= sz; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < sz; i += blockDim.x) {
          const uint32_t p = i ^ j;
          if (p > i) {
            const uint32_t a = key[i], bb = key[p];
            if ((a > bb) == ((i & k) == 0)) { key[i] = bb; key[p] = a; }
          }
        }
        __syncthreads();
      }
    }
    const uint32_t keep = min(K, len);
    for (uint32_t i = threadIdx.x; i < K; i += blockDim.x) dst[ch * K + i] = i < keep ? key[i] : 0xffffffffu;
    __syncthreads();
  }
}

// Final step: copy the K smallest valid keys of the last pass to the caller.
__global__ void k_topk_final_static(const uint32_t* __restrict__ src, const uint32_t* n_ptr, uint32_t K,
                                    uint32_t* __restrict__ out, uint32_t* n_out) {
  const uint32_t n = min(*n_ptr, K);
  __shared__ uint32_t cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t v = src[i];
    out[i] = v;
    if (v != 0xffffffffu) atomicAdd(&cnt, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) *n_out = cnt;
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_ptr[kMaxDevices] = {nullptr};

int scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(RPQ_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); return RPQ_ECUDA; }
  if (dev < 0 || dev >= kMaxDevices) { set_error(RPQ_ELIMIT, "device index %d above %d", dev, kMaxDevices - 1); return RPQ_ELIMIT; }
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t ge = cudaGetSymbolAddress(&p, g_topk_scratch);
    if (ge != cudaSuccess || !p) {
      set_error(RPQ_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(ge));
      return RPQ_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return RPQ_OK;
}

}  // namespace
}  // namespace rpq

using namespace rpq;

extern "C" int rpq_topk_keys_noalloc(const uint32_t* d_keys, uint32_t n, int32_t k, uint32_t* d_out,
                                     uint32_t* d_n_out, void* stream) {
  if (!d_keys && n > 0) { set_error(RPQ_EINVAL, "d_keys is NULL"); return RPQ_EINVAL; }
  if (!d_out || !d_n_out) { set_error(RPQ_EINVAL, "output pointer is NULL"); return RPQ_EINVAL; }
  if (k < 1 || k > kMaxK) { set_error(RPQ_EINVAL, "need 1 <= k <= %d (got %d)", kMaxK, k); return RPQ_EINVAL; }
  if (n > kNaMaxKeys) {
    set_error(RPQ_ELIMIT, "%u keys exceed the no-allocation limit of %u keys", n, kNaMaxKeys);
    return RPQ_ELIMIT;
  }
  uint32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != RPQ_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* bufA = scratch;                               // pass 0 output
  uint32_t* bufB = scratch + kNaPass0Cap;                 // pass 1 output
  uint32_t* cnt = scratch + kNaPass0Cap + kNaPass1Cap;    // counts of each pass
  const uint32_t K = uint32_t(k);
  // counts left by an earlier call must not leak into this one
  RPQ_CUDA(cudaMemsetAsync(cnt, 0, kNaCounters * sizeof(uint32_t), st));
  const int grid = num_sms() * 2;
  // pass 0: keys -> bufA (<= 262,144 keys); pass 1: bufA -> bufB (<= 4,096);
  // pass 2: bufB -> bufA (<= K), then the final copy.
  k_topk_pass_static<<<grid, kNaThreads, 0, st>>>(d_keys, nullptr, n, bufA, cnt + 0, K);
  k_topk_pass_static<<<grid, kNaThreads, 0, st>>>(bufA, cnt + 0, 0, bufB, cnt + 1, K);
  k_topk_pass_static<<<grid, kNaThreads, 0, st>>>(bufB, cnt + 1, 0, bufA, cnt + 2, K);
  k_topk_final_static<<<1, 256, 0, st>>>(bufA, cnt + 2, K, d_out, d_n_out);
  RPQ_CUDA(cudaGetLastError());
  return RPQ_OK;
}
