// Host drivers of the hierarchy set-up on the device (setup_host.cu): the
// Galerkin product and one smoothed-aggregation level, with host CSR in and
// library-allocated host CSR out.  Errors are thrown as Fail (host_check.h).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "amgps.h"

namespace amgps {

struct SetupEnv {
  cudaStream_t stream;
  int nsm;  // SMs of the device (grid sizes)
};

// A_c = P^T A P (amgps_galerkin)
void galerkin_on_device(const SetupEnv& env, const amgps_csr& A, const amgps_csr& P,
                        amgps_csr_buf* Ac);
// P = (I - omega D^{-1} A) P_hat and A_c = P^T A P (amgps_sa_level)
void sa_level_on_device(const SetupEnv& env, const amgps_csr& A, const int32_t* agg,
                        int64_t n_coarse, double* omega, amgps_csr_buf* P_out,
                        amgps_csr_buf* Ac_out);
// frees the three arrays of a library-allocated CSR and zeroes it
void csr_buf_release(amgps_csr_buf* m);

}  // namespace amgps
