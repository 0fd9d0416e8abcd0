// Host helpers shared by the translation units that implement the C ABI:
// error recording for ts_last_error, checked CUDA calls, device allocation.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/tsgls.h"

namespace ts {

// records msg as the calling thread's ts_last_error and returns code
int fail(int code, const std::string& msg);

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return 0;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace ts

#define TS_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t err__ = (call);                                                         \
    if (err__ != cudaSuccess)                                                           \
      return ts::fail(err__ == cudaErrorMemoryAllocation ? TS_ERR_OOM : TS_ERR_CUDA,    \
                      std::string(#call) + ": " + cudaGetErrorString(err__));           \
  } while (0)

#define TS_TRY(...)               \
  do {                            \
    int rc__ = (__VA_ARGS__);     \
    if (rc__ != 0) return rc__;   \
  } while (0)
