// common.h -- host helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include "genasis_hydro.h"

namespace gh {

// Record the message of a failure for genasis_hydro_last_error and return code.
int fail(int code, const char* fmt, ...);
// True for device (or managed) memory of the current device.
bool is_device_ptr(const void* p);

}  // namespace gh

#define GH_CK(call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return ::gh::fail(e_ == cudaErrorMemoryAllocation ? GENASIS_ENOMEM : GENASIS_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                      \
  } while (0)
