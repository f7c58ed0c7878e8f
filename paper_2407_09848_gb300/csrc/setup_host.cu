// Hierarchy set-up on the device (smoothed aggregation of Sec. 4, Galerkin
// products of Sec. 2): CSR inputs are uploaded, the products run in
// kernels_setup.cu, results come back as library-allocated host CSR.  Device
// scratch lives for one call.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "host_check.h"
#include "layout.h"
#include "setup.h"
#include "setup_host.h"

namespace amgps {
namespace {

struct DevScratch {
  std::vector<void*> ptrs;
  ~DevScratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    REQ(e == cudaSuccess, AMGPS_E_NOMEM, std::string("set-up scratch: ") + cudaGetErrorString(e));
    ptrs.push_back(p);
    return (T*)p;
  }
  template <class T>
  T* upload(const T* h, size_t count, cudaStream_t s) {
    T* d = alloc<T>(count);
    if (count) CK(cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
  }
};

// every row strictly ascending: the product kernels rely on distinct columns
void require_sorted_rows(const amgps_csr& A, const char* what) {
  for (int64_t i = 0; i < A.n_rows; ++i)
    for (int e = A.rowptr[i] + 1; e < A.rowptr[i + 1]; ++e)
      REQ(A.col[e] > A.col[e - 1], AMGPS_E_ARG,
          std::string(what) + ": columns of a row must be strictly ascending");
}

DevCsr upload_csr(DevScratch& B, const amgps_csr& A, cudaStream_t s) {
  DevCsr d;
  d.n_rows = A.n_rows;
  d.n_cols = A.n_cols;
  d.nnz = A.nnz;
  d.rowptr = B.upload(A.rowptr, (size_t)A.n_rows + 1, s);
  d.col = B.upload(A.col, (size_t)A.nnz, s);
  d.val = B.upload(A.val, (size_t)A.nnz, s);
  return d;
}

// reads and clears the device error flag of the set-up kernels
bool dev_err_set(int* derr, cudaStream_t s) {
  check_launch();
  int h = 0;
  CK(cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h) CK(cudaMemsetAsync(derr, 0, sizeof(int), s));
  return h != 0;
}

void check_dev_err(int* derr, cudaStream_t s, const char* what) {
  REQ(!dev_err_set(derr, s), AMGPS_E_ARG, what);
}

// rowptr from per-row counts (prefix on the host); allocates col and val
DevCsr from_counts(DevScratch& B, const int32_t* dcnt, int64_t rows, int64_t cols,
                   cudaStream_t s) {
  std::vector<int32_t> h((size_t)rows);
  if (rows) CK(cudaMemcpyAsync(h.data(), dcnt, rows * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int32_t> rp((size_t)rows + 1, 0);
  int64_t acc = 0;
  for (int64_t i = 0; i < rows; ++i) {
    acc += h[i];
    REQ(acc < (int64_t(1) << 31), AMGPS_E_ARG, "sparse product exceeds 2^31 entries");
    rp[i + 1] = (int32_t)acc;
  }
  DevCsr C;
  C.n_rows = rows;
  C.n_cols = cols;
  C.nnz = acc;
  C.rowptr = B.upload(rp.data(), rp.size(), s);
  C.col = B.alloc<int32_t>(acc);
  C.val = B.alloc<double>(acc);
  return C;
}

DevCsr dev_spgemm(const SetupEnv& env, DevScratch& B, const DevCsr& X, const DevCsr& Y, int* derr) {
  cudaStream_t s = env.stream;
  int32_t* cnt = B.alloc<int32_t>(X.n_rows);
  if (Y.n_cols <= kDenseMaxCols) {  // few columns: dense row accumulator
    launch_spgemm_dense(X, Y, cnt, DevCsr{}, derr, false, env.nsm, s);
    check_dev_err(derr, s, "sparse product: symbolic pass failed");
    DevCsr C = from_counts(B, cnt, X.n_rows, Y.n_cols, s);
    launch_spgemm_dense(X, Y, nullptr, C, derr, true, env.nsm, s);
    check_dev_err(derr, s, "sparse product: numeric pass failed");
    return C;
  }
  // narrow form first; the wide form when some row exceeds its limit
  bool wide = false;
  launch_spgemm(X, Y, cnt, DevCsr{}, derr, false, false, env.nsm, s);
  if (dev_err_set(derr, s)) {
    wide = true;
    launch_spgemm(X, Y, cnt, DevCsr{}, derr, false, true, env.nsm, s);
    check_dev_err(derr, s, "sparse product: a row has more than 6144 distinct columns");
  }
  DevCsr C = from_counts(B, cnt, X.n_rows, Y.n_cols, s);
  launch_spgemm(X, Y, nullptr, C, derr, true, wide, env.nsm, s);
  check_dev_err(derr, s, "sparse product: numeric pass failed");
  return C;
}

DevCsr dev_transpose(const SetupEnv& env, DevScratch& B, const DevCsr& M, int* derr) {
  cudaStream_t s = env.stream;
  int32_t* cnt = B.alloc<int32_t>(M.n_cols);
  CK(cudaMemsetAsync(cnt, 0, M.n_cols * sizeof(int32_t), s));
  launch_col_count(M.nnz, M.col, cnt, s);
  check_launch();
  DevCsr T = from_counts(B, cnt, M.n_cols, M.n_rows, s);
  int32_t* cursor = B.alloc<int32_t>(M.n_cols);
  CK(cudaMemcpyAsync(cursor, T.rowptr, M.n_cols * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  launch_transpose_fill(M, cursor, T, s);
  launch_sort_rows(T, derr, false, env.nsm, s);
  if (dev_err_set(derr, s)) {  // rows beyond the narrow limit were left unsorted
    launch_sort_rows(T, derr, true, env.nsm, s);
    check_dev_err(derr, s, "transpose: a row has more than 6144 entries");
  }
  return T;
}

DevCsr dev_galerkin(const SetupEnv& env, DevScratch& B, const DevCsr& A, const DevCsr& P, int* derr) {
  const DevCsr AP = dev_spgemm(env, B, A, P, derr);
  const DevCsr R = dev_transpose(env, B, P, derr);
  return dev_spgemm(env, B, R, AP, derr);
}

void download_csr(const DevCsr& M, amgps_csr_buf* out, cudaStream_t s) {
  amgps_csr_buf o{};
  o.n_rows = M.n_rows;
  o.n_cols = M.n_cols;
  o.nnz = M.nnz;
  o.rowptr = (int32_t*)std::malloc(((size_t)M.n_rows + 1) * sizeof(int32_t));
  o.col = (int32_t*)std::malloc(std::max<size_t>(M.nnz, 1) * sizeof(int32_t));
  o.val = (double*)std::malloc(std::max<size_t>(M.nnz, 1) * sizeof(double));
  if (!o.rowptr || !o.col || !o.val) {
    std::free(o.rowptr);
    std::free(o.col);
    std::free(o.val);
    throw std::bad_alloc();
  }
  CK(cudaMemcpyAsync(o.rowptr, M.rowptr, (M.n_rows + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (M.nnz) {
    CK(cudaMemcpyAsync(o.col, M.col, M.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(o.val, M.val, M.nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    std::free(o.rowptr);
    std::free(o.col);
    std::free(o.val);
    throw Fail{AMGPS_E_CUDA, std::string("download: ") + cudaGetErrorString(e)};
  }
  *out = o;
}

}  // namespace

void csr_buf_release(amgps_csr_buf* m) {
  if (!m) return;
  std::free(m->rowptr);
  std::free(m->col);
  std::free(m->val);
  *m = amgps_csr_buf{};
}

void galerkin_on_device(const SetupEnv& env, const amgps_csr& A, const amgps_csr& P,
                        amgps_csr_buf* Ac) {
  validate_csr(A, "A", true);
  validate_csr(P, "P", false);
  REQ(P.n_rows == A.n_rows, AMGPS_E_ARG, "P rows must equal A rows");
  require_sorted_rows(P, "P");
  cudaStream_t s = env.stream;
  DevScratch B;
  int* derr = B.alloc<int>(1);
  CK(cudaMemsetAsync(derr, 0, sizeof(int), s));
  const DevCsr dA = upload_csr(B, A, s), dP = upload_csr(B, P, s);
  download_csr(dev_galerkin(env, B, dA, dP, derr), Ac, s);
}

void sa_level_on_device(const SetupEnv& env, const amgps_csr& A, const int32_t* agg,
                        int64_t n_coarse, double* omega, amgps_csr_buf* P_out,
                        amgps_csr_buf* Ac_out) {
  validate_csr(A, "A", true);
  REQ(n_coarse >= 1 && n_coarse <= A.n_rows, AMGPS_E_ARG, "n_coarse out of range");
  require_positive_diagonal(A);
  std::vector<int32_t> used((size_t)n_coarse, 0);
  for (int64_t i = 0; i < A.n_rows; ++i) {
    REQ(agg[i] >= 0 && agg[i] < n_coarse, AMGPS_E_ARG, "aggregate index out of range");
    used[agg[i]] = 1;
  }
  for (int64_t I = 0; I < n_coarse; ++I)
    REQ(used[I], AMGPS_E_ARG, "empty aggregate (coarse index without a fine point)");
  cudaStream_t s = env.stream;
  const int64_t n = A.n_rows;
  DevScratch B;
  int* derr = B.alloc<int>(1);
  CK(cudaMemsetAsync(derr, 0, sizeof(int), s));
  const DevCsr dA = upload_csr(B, A, s);
  int32_t* dagg = B.upload(agg, (size_t)n, s);
  // omega = 4 / (3 lambda), lambda = max_i sum_j |a_ij| / a_ii
  double* diag = B.alloc<double>(n);
  double* part = B.alloc<double>((size_t)env.nsm * 4);
  const int np = launch_rowstat(dA, diag, part, env.nsm, s);
  check_launch();
  std::vector<double> hp(np);
  CK(cudaMemcpyAsync(hp.data(), part, np * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double lam = 0.0;
  for (double v : hp) lam = std::max(lam, v);
  REQ(std::isfinite(lam) && lam > 0.0, AMGPS_E_NAN, "row-sum bound not finite");
  const double om = 4.0 / (3.0 * lam);
  // P_hat (one unit entry per row), A P_hat, then P in place
  std::vector<int32_t> iota((size_t)n + 1);
  for (int64_t i = 0; i <= n; ++i) iota[i] = (int32_t)i;
  std::vector<double> ones((size_t)n, 1.0);
  DevCsr Ph;
  Ph.n_rows = n;
  Ph.n_cols = n_coarse;
  Ph.nnz = n;
  Ph.rowptr = B.upload(iota.data(), iota.size(), s);
  Ph.col = dagg;
  Ph.val = B.upload(ones.data(), ones.size(), s);
  const DevCsr P = dev_spgemm(env, B, dA, Ph, derr);
  launch_sa_combine(P, dagg, diag, om, s);
  check_launch();
  const DevCsr Ac = dev_galerkin(env, B, dA, P, derr);
  download_csr(P, P_out, s);
  try {
    download_csr(Ac, Ac_out, s);
  } catch (...) {
    csr_buf_release(P_out);
    throw;
  }
  *omega = om;
}

}  // namespace amgps
