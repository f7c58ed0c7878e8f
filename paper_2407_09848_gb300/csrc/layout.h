// Host-side layout planning: validation of caller CSR, conversion to the
// device SELL-32 layout (uniform and explicit slices), the TMA tile plan with
// its bounds and alignment checks, FP64 -> BF16 rounding, and the warps-per-
// slice rule of the split kernels.  Pure host code.
#pragma once

#include <cstdint>
#include <functional>
#include <vector>

#include "amgps_internal.h"

namespace amgps {

// Most column offsets a uniform slice may list (the pattern of the widest
// coarse operators of smoothed aggregation on a grid still fits).
constexpr int64_t kUniformMax = 1024;


struct HostSell {
  int64_t n = 0, nnz = 0, nslices = 0, stored = 0, explicit_entries = 0;
  std::vector<SliceDesc> sd;
  std::vector<double> val;
  std::vector<int32_t> col;
  std::vector<int32_t> off;
  bool any_explicit = false;
};

struct HostPlan {
  TmaPlan p;
  std::vector<TmaTile> tiles;
  std::vector<int32_t> gen;  // slices the TMA kernel does not cover
};

// Host threads for `count` independent items (1 below 4096 items, else the
// hardware concurrency, at most 32); parallel_for calls f(i, thread) for
// i in [0, count) in contiguous chunks and rethrows the first failure.
int parallel_threads(int64_t count);
void parallel_for(int64_t count, const std::function<void(int64_t, int)>& f);

// AMGPS_E_ARG (through Fail) unless A is a well-formed CSR (square if asked)
void validate_csr(const amgps_csr& A, const char* what, bool square);
// AMGPS_E_NOT_SPD unless every row holds a positive diagonal entry (a
// validated square CSR)
void require_positive_diagonal(const amgps_csr& A);
// Warps per slice for the split kernels of a level (1: no split)
int split_for(int64_t stored, int64_t nslices);
// SELL-32 form of A; allow_uniform = false keeps every slice explicit
HostSell build_sell(const amgps_csr& A, bool allow_uniform = true);
// FP64 -> BF16 bits, round to nearest even directly from the double
uint16_t dbl_to_bf16(double x);
// The TMA-fed step's tiles and stage layout for a level (element sizes of the
// matrix values and of the vectors, dynamic shared memory per CTA)
HostPlan build_tma_plan(const HostSell& h, size_t vsize, size_t xsize, int smem_budget);

}  // namespace amgps
