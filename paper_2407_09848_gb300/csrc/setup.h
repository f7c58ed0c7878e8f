// Device CSR and the launchers of the hierarchy set-up kernels
// (kernels_setup.cu): smoothed-aggregation prolongator and Galerkin product.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace amgps {

// Most distinct columns a row of a sparse product (or of a transpose) may
// have in the narrow and in the wide form of the kernels.
constexpr int kRowMaxNarrow = 768;
constexpr int kRowMaxWide = 6144;

struct DevCsr {
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

// C = A B.  fill = false: counts[i] = distinct columns of row i of C.
// fill = true: C.rowptr set from those counts; writes C.col (ascending per
// row) and C.val.  *err = 1 if a row exceeds the form's column limit
// (kRowMaxNarrow, or kRowMaxWide with wide = true).
void launch_spgemm(const DevCsr& A, const DevCsr& B, int32_t* counts, const DevCsr& C, int* err,
                   bool fill, bool wide, int nsm, cudaStream_t s);
// Dense form of C = A B for B.n_cols <= kDenseMaxCols: same results as the
// hashed forms (bitwise), no row limit.
constexpr int64_t kDenseMaxCols = 16384;
void launch_spgemm_dense(const DevCsr& A, const DevCsr& B, int32_t* counts, const DevCsr& C,
                         int* err, bool fill, int nsm, cudaStream_t s);
// diag[i] = a_ii and per-block maxima of sum_j |a_ij| / a_ii into part[];
// returns the number of blocks (partials)
int launch_rowstat(const DevCsr& A, double* diag, double* part, int nsm, cudaStream_t s);
// in place on A P_hat: entries become [j == agg_i] - omega (1/a_ii) (A P_hat)_ij
void launch_sa_combine(const DevCsr& AP, const int32_t* agg, const double* diag, double omega,
                       cudaStream_t s);
// transpose T = M^T: count entries per column, scatter with per-row cursors
// (from the prefix sums of the counts), then sort each row of T by column
void launch_col_count(int64_t nnz, const int32_t* col, int32_t* cnt, cudaStream_t s);
void launch_transpose_fill(const DevCsr& M, int32_t* cursor, const DevCsr& T, cudaStream_t s);
void launch_sort_rows(const DevCsr& T, int* err, bool wide, int nsm, cudaStream_t s);

}  // namespace amgps
