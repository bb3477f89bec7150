// capi_common.h -- error plumbing shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include "../../include/tron.h"

namespace xt {

void set_error(const char* fmt, ...);
void clear_error();
int device_sm_count();

}  // namespace xt

#define XT_CUDA(call)                                                               \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      xt::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                      \
      return TRON_ECUDA;                                                            \
    }                                                                               \
  } while (0)

#define XT_REQUIRE(cond, code, ...) \
  do {                              \
    if (!(cond)) {                  \
      xt::set_error(__VA_ARGS__);   \
      return (code);                \
    }                               \
  } while (0)
