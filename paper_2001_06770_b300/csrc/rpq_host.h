// Host-side internals of librpq shared by the translation units.
#pragma once
#include <cstdint>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/rpq.h"
#include "rpq_internal.cuh"

namespace rpq {

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

struct Slot;

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
  uint32_t* d_kw_ptr = nullptr;
  int32_t* d_kw_nodes = nullptr;
  int64_t device_bytes = 0;
  std::vector<int64_t> kw_ptr;   // host copy of the postings offsets
  std::vector<rpq::Slot*> slots; // search slots, created on first use
};

namespace rpq {
// Fill d_row_ptr, d_adj and d_amax of kg from the host CSR (kg_build.cu).
int build_graph(rpq_kg* kg, const rpq_kg_desc* d);
}  // namespace rpq
