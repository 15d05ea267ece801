// State transfer on the SMs between device fields and page-locked host
// memory seen through its mapped device address (k_simple.cu, api.cu).
#pragma once

#include <cuda_runtime.h>

#include "../../include/u1u1.h"

namespace u1u1 {

// entry f copies n16 16-byte words from src[f] to dst[f]; one side of each
// entry is mapped host memory, the other a device field
struct XferTable {
  const void* src[U1U1_NFIELDS];
  void* dst[U1U1_NFIELDS];
  int m;
};
cudaError_t launch_state_copy(const XferTable& t, long long n16, cudaStream_t st);

}  // namespace u1u1
