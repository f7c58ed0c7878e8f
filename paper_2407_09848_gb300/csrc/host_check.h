// Error reporting of the host side: every failure is a Fail carrying the
// status returned through the C ABI; CK wraps CUDA runtime calls and REQ
// validates arguments.
#pragma once

#include <string>

#include <cuda_runtime.h>

#include "amgps.h"

namespace amgps {

struct Fail {
  amgps_status st;
  std::string msg;
};

}  // namespace amgps

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::amgps::Fail{AMGPS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define REQ(cond, st, msg)                   \
  do {                                       \
    if (!(cond)) throw ::amgps::Fail{st, msg}; \
  } while (0)
