// Hierarchy set-up on the device: the smoothed-aggregation prolongator
// P = (I - omega D^{-1} A) P_hat and the Galerkin product A_c = P^T A P of
// Sec. 4, built from CSR matrices with sparse products (SpGEMM).
//
// SpGEMM C = A B, one warp per row i of C, Gustavson order: for each entry
// (k, a_ik) of row i of A in storage order, the lanes stride over row k of B
// and add a_ik b_kj into a hash table in shared memory keyed by column j.  One
// such pass over a row of B is a "round"; the columns of a row of B are
// distinct, so within a round no two lanes touch the same slot, and rounds are
// separated by __syncwarp().  Every c_ij is therefore summed in the order of
// k along row i of A, whatever the scheduling: the product is bitwise
// reproducible.  A symbolic pass (FILL = false) counts the distinct columns
// per row; the numeric pass (FILL = true) writes each row sorted by column.
// Two table sizes: the narrow form (1024 slots, rows up to kRowMaxNarrow,
// two warps per block) and the wide form (8192 slots, rows up to
// kRowMaxWide, one warp per block in opt-in shared memory) that the host
// falls back to when a narrow pass reports an over-long row through *err.
#include "kernels_common.cuh"
#include "setup.h"

namespace amgps {
namespace {

template <int HASH, int ROWMAX, int WARPS>
struct GemmShape {
  static constexpr int kHash = HASH, kRowMax = ROWMAX, kWarps = WARPS;
  static constexpr int kLog2 = HASH == 1024 ? 10 : 13;
  static_assert((1 << kLog2) == HASH, "hash size must be 1024 or 8192");
  static_assert(ROWMAX < HASH, "hash table must exceed the row limit");
  // per warp: vals[HASH], lval[ROWMAX] (doubles first), keys[HASH], lkey[ROWMAX]
  static constexpr size_t kWarpBytes = (size_t)(HASH + ROWMAX) * 12;
  static constexpr size_t kSmem = kWarpBytes * WARPS;
};
using Narrow = GemmShape<1024, kRowMaxNarrow, 2>;
using Wide = GemmShape<8192, kRowMaxWide, 1>;

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class G, bool FILL>
__global__ void __launch_bounds__(32 * G::kWarps) k_spgemm(const DevCsr A, const DevCsr B,
                                                          int32_t* __restrict__ counts,
                                                          const DevCsr C, int* err) {
  extern __shared__ double smem_d[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* val = smem_d + (size_t)w * (G::kHash + G::kRowMax);
  double* lval = val + G::kHash;
  int32_t* key = (int32_t*)(smem_d + (size_t)G::kWarps * (G::kHash + G::kRowMax)) +
                 (size_t)w * (G::kHash + G::kRowMax);
  int32_t* lkey = key + G::kHash;
  const int64_t stride = (int64_t)gridDim.x * G::kWarps;
  for (int64_t i = (int64_t)blockIdx.x * G::kWarps + w; i < A.n_rows; i += stride) {
    for (int h = lane; h < G::kHash; h += 32) {
      key[h] = -1;
      if (FILL) val[h] = 0.0;
    }
    __syncwarp();
    bool over = false;
    for (int e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int32_t k = A.col[e];
      const double a = A.val[e];
      for (int f = B.rowptr[k] + lane; f < B.rowptr[k + 1] && !over; f += 32) {
        const int32_t j = B.col[f];
        uint32_t h = ((uint32_t)j * 2654435761u) >> (32 - G::kLog2);
        int probes = 0;
        for (;;) {
          const int32_t prev = atomicCAS(&key[h], -1, j);
          if (prev == -1 || prev == j) break;
          h = (h + 1) & (G::kHash - 1);
          if (++probes == G::kHash) {
            over = true;
            break;
          }
        }
        if (FILL && !over) val[h] += a * B.val[f];
      }
      __syncwarp();
    }
    int cnt = 0;
    for (int h = lane; h < G::kHash; h += 32) cnt += key[h] >= 0;
    cnt = warp_sum_int(cnt);
    over = __any_sync(0xffffffffu, over) || cnt > G::kRowMax;
    if (over) {
      if (lane == 0) atomicExch(err, 1);
      __syncwarp();
      continue;
    }
    if (!FILL) {
      if (lane == 0) counts[i] = cnt;
      __syncwarp();
      continue;
    }
    if (C.rowptr[i + 1] - C.rowptr[i] != cnt) {  // passes disagree: cannot happen
      if (lane == 0) atomicExch(err, 2);
      __syncwarp();
      continue;
    }
    // compact the occupied slots, then place each entry by its rank in column order
    int base = 0;
    for (int h0 = 0; h0 < G::kHash; h0 += 32) {
      const int h = h0 + lane;
      const bool occ = key[h] >= 0;
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      if (occ) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        lkey[pos] = key[h];
        lval[pos] = val[h];
      }
      base += __popc(m);
    }
    __syncwarp();
    const int64_t out0 = C.rowptr[i];
    for (int q = lane; q < cnt; q += 32) {
      const int32_t kq = lkey[q];
      int rank = 0;
      for (int t = 0; t < cnt; ++t) rank += lkey[t] < kq;
      C.col[out0 + rank] = kq;
      C.val[out0 + rank] = lval[q];
    }
    __syncwarp();
  }
}

// Dense form for products with at most kDenseMaxCols columns (the coarse
// levels): one warp per block owns a dense row accumulator (values and touch
// flags for every column) in shared memory.  Rounds add in the same order as
// the hashed forms, so the result is bitwise the same; one ordered scan per
// row emits the columns already sorted (no sort) and clears what it touched.
// No row limit applies.
__global__ void __launch_bounds__(32) k_spgemm_dense(const DevCsr A, const DevCsr B,
                                                    int32_t* __restrict__ counts,
                                                    const DevCsr C, int fill, int* err) {
  extern __shared__ double dval[];
  const int ncols = (int)B.n_cols;
  uint8_t* flag = reinterpret_cast<uint8_t*>(dval + ncols);
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < ncols; j += 32) {
    dval[j] = 0.0;
    flag[j] = 0;
  }
  __syncwarp();
  for (int64_t i = blockIdx.x; i < A.n_rows; i += gridDim.x) {
    for (int e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int32_t k = A.col[e];
      const double a = A.val[e];
      for (int f = B.rowptr[k] + lane; f < B.rowptr[k + 1]; f += 32) {
        const int32_t j = B.col[f];
        if (fill) {
          if (flag[j]) {
            dval[j] += a * B.val[f];
          } else {
            flag[j] = 1;
            dval[j] = 0.0;
            dval[j] += a * B.val[f];
          }
        } else {
          flag[j] = 1;
        }
      }
      __syncwarp();
    }
    // the row's column count first: the numeric pass writes only when it
    // equals the slot the symbolic pass reserved
    int total = 0;
    if (fill) {
      for (int j0 = 0; j0 < ncols; j0 += 32) {
        const int j = j0 + lane;
        total += __popc(__ballot_sync(0xffffffffu, j < ncols && flag[j]));
      }
    }
    const bool write = fill && (C.rowptr[i + 1] - C.rowptr[i] == total);
    if (fill && !write && lane == 0) atomicExch(err, 2);
    const int64_t out0 = fill ? C.rowptr[i] : 0;
    int base = 0;
    for (int j0 = 0; j0 < ncols; j0 += 32) {
      const int j = j0 + lane;
      const bool on = j < ncols && flag[j];
      const unsigned m = __ballot_sync(0xffffffffu, on);
      if (on) {
        if (write) {
          const int pos = base + __popc(m & ((1u << lane) - 1u));
          C.col[out0 + pos] = j;
          C.val[out0 + pos] = dval[j];
        }
        dval[j] = 0.0;
        flag[j] = 0;
      }
      base += __popc(m);
    }
    if (!fill && lane == 0) counts[i] = base;
    __syncwarp();
  }
}

// diag[i] = a_ii, part[block] = max over its rows of sum_j |a_ij| / a_ii
__global__ void __launch_bounds__(kBlock) k_rowstat(const DevCsr A, double* __restrict__ diag,
                                                    double* __restrict__ part) {
  __shared__ double sh[kBlock / 32];
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < A.n_rows;
       i += (int64_t)gridDim.x * kBlock) {
    double d = 0.0, s = 0.0;
    for (int e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const double v = A.val[e];
      s += fabs(v);
      if (A.col[e] == i) d = v;
    }
    diag[i] = d;
    mx = fmax(mx, s / d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kBlock / 32; ++k) mx = fmax(mx, sh[k]);
    part[blockIdx.x] = mx;
  }
}

// P = P_hat - omega D^{-1} (A P_hat), in place on the entries of A P_hat
__global__ void __launch_bounds__(kBlock) k_sa_combine(const DevCsr AP, const int32_t* __restrict__ agg,
                                                       const double* __restrict__ diag,
                                                       double omega) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= AP.n_rows) return;
  const double dinv = 1.0 / diag[i];
  const int32_t own = agg[i];
  for (int e = AP.rowptr[i]; e < AP.rowptr[i + 1]; ++e)
    AP.val[e] = (AP.col[e] == own ? 1.0 : 0.0) - omega * (dinv * AP.val[e]);
}

// transpose, step 1: entries per column
__global__ void __launch_bounds__(kBlock) k_col_count(int64_t nnz, const int32_t* __restrict__ col,
                                                      int32_t* __restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (e < nnz) atomicAdd(&cnt[col[e]], 1);
}

// transpose, step 2: scatter (order inside a row of the transpose arbitrary)
__global__ void __launch_bounds__(kBlock) k_transpose_fill(const DevCsr M, int32_t* __restrict__ cursor,
                                                           const DevCsr T) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= M.n_rows) return;
  for (int e = M.rowptr[i]; e < M.rowptr[i + 1]; ++e) {
    const int32_t pos = atomicAdd(&cursor[M.col[e]], 1);
    T.col[pos] = (int32_t)i;
    T.val[pos] = M.val[e];
  }
}

// transpose, step 3: sort every row by column (warp per row, rank placement;
// the columns of a row are distinct) -- makes the transpose deterministic.
// Rows longer than the form's limit set *err and are left as they are.
template <class G>
__global__ void __launch_bounds__(32 * G::kWarps) k_sort_rows(const DevCsr T, int* err) {
  extern __shared__ double smem_d[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* lval = smem_d + (size_t)w * G::kRowMax;
  int32_t* lkey = (int32_t*)(smem_d + (size_t)G::kWarps * G::kRowMax) + (size_t)w * G::kRowMax;
  const int64_t stride = (int64_t)gridDim.x * G::kWarps;
  for (int64_t i = (int64_t)blockIdx.x * G::kWarps + w; i < T.n_rows; i += stride) {
    const int32_t r0 = T.rowptr[i];
    const int m = T.rowptr[i + 1] - r0;
    if (m > G::kRowMax) {
      if (lane == 0) atomicExch(err, 1);
      continue;
    }
    for (int q = lane; q < m; q += 32) {
      lkey[q] = T.col[r0 + q];
      lval[q] = T.val[r0 + q];
    }
    __syncwarp();
    for (int q = lane; q < m; q += 32) {
      const int32_t kq = lkey[q];
      int rank = 0;
      for (int t = 0; t < m; ++t) rank += lkey[t] < kq;
      T.col[r0 + rank] = kq;
      T.val[r0 + rank] = lval[q];
    }
    __syncwarp();
  }
}

int gemm_grid(int64_t rows, int warps, int nsm) {
  int64_t g = (rows + warps - 1) / warps;
  const int64_t cap = (int64_t)nsm * 16;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

// the wide forms need more than the default 48 KB of dynamic shared memory
void wide_smem_optin() {
  static uint64_t done = 0;  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (done >> dev & 1u)) return;
  cudaFuncSetAttribute(k_spgemm<Wide, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)Wide::kSmem);
  cudaFuncSetAttribute(k_spgemm<Wide, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)Wide::kSmem);
  cudaFuncSetAttribute(k_sort_rows<Wide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(Wide::kRowMax * 12));
  if (dev < 64) done |= uint64_t(1) << dev;
}

}  // namespace

void launch_spgemm(const DevCsr& A, const DevCsr& B, int32_t* counts, const DevCsr& C, int* err,
                   bool fill, bool wide, int nsm, cudaStream_t s) {
  if (A.n_rows == 0) return;
  if (wide) {
    wide_smem_optin();
    const int g = gemm_grid(A.n_rows, Wide::kWarps, nsm);
    if (fill) k_spgemm<Wide, true><<<g, 32 * Wide::kWarps, Wide::kSmem, s>>>(A, B, counts, C, err);
    else k_spgemm<Wide, false><<<g, 32 * Wide::kWarps, Wide::kSmem, s>>>(A, B, counts, C, err);
  } else {
    const int g = gemm_grid(A.n_rows, Narrow::kWarps, nsm);
    if (fill) k_spgemm<Narrow, true><<<g, 32 * Narrow::kWarps, Narrow::kSmem, s>>>(A, B, counts, C, err);
    else k_spgemm<Narrow, false><<<g, 32 * Narrow::kWarps, Narrow::kSmem, s>>>(A, B, counts, C, err);
  }
  count_launch();
}

void launch_spgemm_dense(const DevCsr& A, const DevCsr& B, int32_t* counts, const DevCsr& C,
                         int* err, bool fill, int nsm, cudaStream_t s) {
  if (A.n_rows == 0) return;
  const size_t smem = (size_t)B.n_cols * 9;
  static uint64_t done = 0;  // opt-in once per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !(done >> dev & 1u)) {
    cudaFuncSetAttribute(k_spgemm_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((size_t)kDenseMaxCols * 9));
    done |= uint64_t(1) << dev;
  }
  const int g = gemm_grid(A.n_rows, 1, nsm);
  k_spgemm_dense<<<g, 32, smem, s>>>(A, B, counts, C, fill ? 1 : 0, err);
  count_launch();
}

int launch_rowstat(const DevCsr& A, double* diag, double* part, int nsm, cudaStream_t s) {
  int64_t g = (A.n_rows + kBlock - 1) / kBlock;
  g = std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)nsm * 4));
  k_rowstat<<<(unsigned)g, kBlock, 0, s>>>(A, diag, part);
  count_launch();
  return (int)g;
}

void launch_sa_combine(const DevCsr& AP, const int32_t* agg, const double* diag, double omega,
                       cudaStream_t s) {
  if (AP.n_rows == 0) return;
  k_sa_combine<<<(unsigned)((AP.n_rows + kBlock - 1) / kBlock), kBlock, 0, s>>>(AP, agg, diag,
                                                                                 omega);
  count_launch();
}

void launch_col_count(int64_t nnz, const int32_t* col, int32_t* cnt, cudaStream_t s) {
  if (nnz == 0) return;
  k_col_count<<<(unsigned)((nnz + kBlock - 1) / kBlock), kBlock, 0, s>>>(nnz, col, cnt);
  count_launch();
}

void launch_transpose_fill(const DevCsr& M, int32_t* cursor, const DevCsr& T, cudaStream_t s) {
  if (M.n_rows == 0) return;
  k_transpose_fill<<<(unsigned)((M.n_rows + kBlock - 1) / kBlock), kBlock, 0, s>>>(M, cursor, T);
  count_launch();
}

void launch_sort_rows(const DevCsr& T, int* err, bool wide, int nsm, cudaStream_t s) {
  if (T.n_rows == 0) return;
  if (wide) {
    wide_smem_optin();
    k_sort_rows<Wide><<<gemm_grid(T.n_rows, Wide::kWarps, nsm), 32 * Wide::kWarps,
                        Wide::kRowMax * 12, s>>>(T, err);
  } else {
    k_sort_rows<Narrow><<<gemm_grid(T.n_rows, Narrow::kWarps, nsm), 32 * Narrow::kWarps,
                          Narrow::kWarps * Narrow::kRowMax * 12, s>>>(T, err);
  }
  count_launch();
}

}  // namespace amgps
