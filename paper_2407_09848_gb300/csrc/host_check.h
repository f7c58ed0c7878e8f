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

// the last kernel launch on this thread failed -> AMGPS_E_CUDA
inline void check_launch() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw Fail{AMGPS_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

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
