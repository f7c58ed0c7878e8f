// Outer-solver kernels (preconditioned CG, Sec. 4), the coarsest-level dense
// solve, and the power-iteration estimate.  All reductions are deterministic
// (fixed grid, fixed summation tree: see grid_sum), so a solve repeated on
// the same input performs the same iterations bit for bit.
#include <atomic>

#include "kernels_common.cuh"

namespace amgps {

namespace {
// kernels enqueued by this process (all contexts, all host threads)
std::atomic<int64_t> g_launches{0};
}
int64_t launches_enqueued() { return g_launches.load(std::memory_order_relaxed); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int reduction_grid(int64_t work_items, int nsm, int per_sm) {
  int64_t g = (work_items + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)nsm * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// q = A p and p.q (S_PQ).  One warp per slice, grid-stride over slices.
__global__ void __launch_bounds__(kBlock) k_spmv_dot(const DevMat<double> A,
                                                     const double* __restrict__ p,
                                                     double* __restrict__ q, const RedWork w,
                                                     double* scal) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
  double acc = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); s < A.nslices;
       s += nw) {
    const int64_t row = s * kSlice + lane;
    const double t = row_spmv<1, double, double>(A, s, lane, row, p, 0.0);
    if (row < A.n) {
      q[row] = t;
      acc = fma(p[row], t, acc);
    }
  }
  grid_sum(acc, w, [&](double tot) {
    scal[S_PQ] = tot;
    scal[S_ALPHA] = scal[S_RZ] / tot;  // once per iteration, not once per thread
  });
}

void launch_spmv_dot(const DevMat<double>& A, const double* p, double* q, const RedWork& w,
                     double* scal, cudaStream_t s) {
  k_spmv_dot<<<w.grid, kBlock, 0, s>>>(A, p, q, w, scal);
  count_launch();
}

// Three sums in one pass (the one-reduction flexible CG): partials are laid
// out [v0 of every block | v1 ... | v2 ...] in w.part (3 x grid doubles); the
// last block adds each column in index order and calls fin(t0, t1, t2).
template <class Fin>
__device__ __forceinline__ void grid_sum3(double v0, double v1, double v2, const RedWork& w,
                                          Fin fin) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double b0 = block_sum(v0, sh);
  const double b1 = block_sum(v1, sh);
  const double b2 = block_sum(v2, sh);
  if (threadIdx.x == 0) {
    w.part[blockIdx.x] = b0;
    w.part[gridDim.x + blockIdx.x] = b1;
    w.part[2 * gridDim.x + blockIdx.x] = b2;
    __threadfence();
    const unsigned t = atomicAdd(w.counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double t[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
        s += __ldcg(w.part + j * gridDim.x + i);
      t[j] = block_sum(s, sh);
    }
    if (threadIdx.x == 0) {
      fin(t[0], t[1], t[2]);
      *w.counter = 0u;
    }
  }
}

// One-reduction flexible CG (the outer solver of Sec. 4): w = A z and the
// three inner products rho = z.r, gamma = z.q_old, delta = z.w in a single
// grid reduction.  The last block forms beta = gamma / eta_old (the
// A-orthogonalisation of z against p_old), eta = p.A p = delta - beta gamma
// (by symmetry of A, with q = A p), and alpha = rho / eta.
__global__ void __launch_bounds__(kBlock) k_spmv_dot3(const DevMat<double> A,
                                                      const double* __restrict__ z,
                                                      double* __restrict__ w,
                                                      const double* __restrict__ r,
                                                      const double* __restrict__ q, int first,
                                                      const RedWork rw, double* scal) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
  double zr = 0.0, zq = 0.0, zw = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); s < A.nslices;
       s += nw) {
    const int64_t row = s * kSlice + lane;
    const double t = row_spmv<1, double, double>(A, s, lane, row, z, 0.0);
    if (row < A.n) {
      w[row] = t;
      const double zi = z[row];
      zw = fma(zi, t, zw);
      zr = fma(zi, r[row], zr);
      if (!first) zq = fma(zi, q[row], zq);
    }
  }
  grid_sum3(zr, zq, zw, rw, [&](double rho, double gam, double del) {
    const double beta = first ? 0.0 : gam / scal[S_PQ];
    const double eta = first ? del : del - beta * gam;
    scal[S_RZ] = rho;
    scal[S_GAMMA] = gam;
    scal[S_DELTA] = del;
    scal[S_BETA] = beta;
    scal[S_PQ] = eta;
    scal[S_ALPHA] = rho / eta;
  });
}

void launch_spmv_dot3(const DevMat<double>& A, const double* z, double* w, const double* r,
                      const double* q, int first, const RedWork& rw, double* scal,
                      cudaStream_t s) {
  k_spmv_dot3<<<rw.grid, kBlock, 0, s>>>(A, z, w, r, q, first, rw, scal);
  count_launch();
}

// p = z - beta p, q = w - beta q (first: p = z, q = w), x += alpha p,
// r -= alpha q, r.r (S_RR)
__global__ void __launch_bounds__(kBlock) k_fcg_update(int64_t n, const double* __restrict__ z,
                                                       const double* __restrict__ w,
                                                       double* __restrict__ p,
                                                       double* __restrict__ q,
                                                       double* __restrict__ x,
                                                       double* __restrict__ r, int first,
                                                       const RedWork rw, double* scal) {
  const double alpha = scal[S_ALPHA], beta = scal[S_BETA];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock) {
    const double pi = first ? z[i] : fma(-beta, p[i], z[i]);
    const double qi = first ? w[i] : fma(-beta, q[i], w[i]);
    p[i] = pi;
    q[i] = qi;
    x[i] = fma(alpha, pi, x[i]);
    const double ri = fma(-alpha, qi, r[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  grid_sum(acc, rw, [&](double tot) { scal[S_RR] = tot; });
}

void launch_fcg_update(int64_t n, const double* z, const double* w, double* p, double* q,
                       double* x, double* r, int first, const RedWork& rw, double* scal,
                       cudaStream_t s) {
  k_fcg_update<<<rw.grid, kBlock, 0, s>>>(n, z, w, p, q, x, r, first, rw, scal);
  count_launch();
}

// r -= alpha q ; r.r (S_RR).  The x update of the same iteration is deferred
// to k_xpay_x, which reads p anyway.  WC: also c = M^{-1} r (the product the
// stored-operator smoother of the next V-cycle starts from, same operation
// as its own c pass).
template <bool WC>
__global__ void __launch_bounds__(kBlock) k_r_update(int64_t n, const double* __restrict__ q,
                                                     double* __restrict__ r, const RedWork w,
                                                     double* scal, const double* __restrict__ dinv,
                                                     double* __restrict__ cout) {
  const double alpha = scal[S_ALPHA];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock) {
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    if constexpr (WC) cout[i] = ri * dinv[i];
    acc = fma(ri, ri, acc);
  }
  grid_sum(acc, w, [&](double tot) { scal[S_RR] = tot; });
}

void launch_r_update(int64_t n, const double* q, double* r, const RedWork& w, double* scal,
                     cudaStream_t s, const double* dinv, double* cout) {
  if (cout)
    k_r_update<true><<<w.grid, kBlock, 0, s>>>(n, q, r, w, scal, dinv, cout);
  else
    k_r_update<false><<<w.grid, kBlock, 0, s>>>(n, q, r, w, scal, nullptr, nullptr);
  count_launch();
}

// x += alpha p with the previous alpha, then p = z + beta p (x_beta = 1), or
// only x += alpha p (x_beta = 0: the last iteration)
__global__ void __launch_bounds__(kBlock) k_xpay_x(int64_t n, const double* __restrict__ z,
                                                   double* __restrict__ p, double* __restrict__ x,
                                                   const double* __restrict__ scal, int with_p) {
  const double alpha = scal[S_ALPHA], beta = scal[S_BETA];
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  const double pi = p[i];
  x[i] = fma(alpha, pi, x[i]);
  if (with_p) p[i] = fma(beta, pi, z[i]);
}

void launch_xpay_x(int64_t n, const double* z, double* p, double* x, const double* scal,
                   int with_p, cudaStream_t s) {
  if (n == 0) return;
  k_xpay_x<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, z, p, x, scal, with_p);
  count_launch();
}

__global__ void __launch_bounds__(kBlock) k_dot(int64_t n, const double* __restrict__ a,
                                                const double* __restrict__ b, const RedWork w,
                                                double* scal, int slot, int rz_shift) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock)
    acc = fma(a[i], b[i], acc);
  grid_sum(acc, w, [&](double tot) {
    if (rz_shift) {
      scal[S_RZOLD] = scal[S_RZ];
      scal[S_RZ] = tot;
      scal[S_BETA] = (rz_shift == 2 ? tot - scal[S_RZP] : tot) / scal[S_RZOLD];
    } else {
      scal[slot] = tot;
    }
  });
}

void launch_dot(int64_t n, const double* a, const double* b, const RedWork& w, double* scal,
                int out_slot, int rz_mode, cudaStream_t s) {
  k_dot<<<w.grid, kBlock, 0, s>>>(n, a, b, w, scal, out_slot, rz_mode);
  count_launch();
}

__global__ void __launch_bounds__(kBlock) k_sub(int64_t n, const double* __restrict__ x,
                                                const double* __restrict__ y,
                                                double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) out[i] = x[i] - y[i];
}

void launch_sub(int64_t n, const double* x, const double* y, double* out, cudaStream_t s) {
  if (n == 0) return;
  k_sub<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, x, y, out);
  count_launch();
}

__global__ void __launch_bounds__(kBlock) k_scale_dev(int64_t n, const double* __restrict__ x,
                                                      double* __restrict__ out,
                                                      const double* __restrict__ sd,
                                                      double factor) {
  const double f = factor / sd[0];
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) out[i] = f * x[i];
}

void launch_scale_dev(int64_t n, const double* x, double* out, const double* s_dev, double factor,
                      cudaStream_t s) {
  if (n == 0) return;
  k_scale_dev<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, x, out, s_dev, factor);
  count_launch();
}

// Coarsest level: x = A_c^{-1} b with the inverse formed at load time from the
// Cholesky factor (FP64).  One warp per row, lanes stride the columns.
template <class XT>
__global__ void __launch_bounds__(kBlock) k_coarse_gemv(int nc, const double* __restrict__ ainv,
                                                        const XT* __restrict__ b,
                                                        XT* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (i >= nc) return;
  coarse_gemv_row<XT>(i, nc, ainv, b, x, lane);
}

template <class XT>
void launch_coarse_gemv(int nc, const double* ainv, const XT* b, XT* x, cudaStream_t s) {
  if (nc == 0) return;
  k_coarse_gemv<XT><<<(nc + kWarpsPerBlock - 1) / kWarpsPerBlock, kBlock, 0, s>>>(nc, ainv, b, x);
  count_launch();
}

// Dense Cholesky A = L L^T (right-looking, one block, in place in `work`,
// row-major), then A^{-1} column by column (forward and back substitution),
// written row-major into ainv (A^{-1} is symmetric).  status = 1 if a pivot is
// not positive.  Set-up only: runs once per hierarchy load.
__global__ void __launch_bounds__(1024) k_chol_inverse(int n, double* L, double* ainv,
                                                      int* status) {
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[(size_t)j * n + j];
      if (!(d > 0.0)) {
        *status = 1;
        piv = -1.0;
      } else {
        piv = sqrt(d);
        L[(size_t)j * n + j] = piv;
      }
    }
    __syncthreads();
    if (piv < 0.0) return;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) L[(size_t)i * n + j] /= piv;
    __syncthreads();
    const int64_t m = n - j - 1;
    const int64_t npairs = m * (m + 1) / 2;
    for (int64_t q = threadIdx.x; q < npairs; q += blockDim.x) {
      int64_t ii = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
      while (ii * (ii + 1) / 2 > q) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
      const int64_t kk = q - ii * (ii + 1) / 2;
      const int64_t i = j + 1 + ii, k = j + 1 + kk;
      L[i * n + k] -= L[i * n + j] * L[k * n + j];
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double* y = ainv + (size_t)c * n;
    for (int i = 0; i < n; ++i) {
      if (i < c) {
        y[i] = 0.0;
        continue;
      }
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
      y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * y[k];
      y[i] = s / L[(size_t)i * n + i];
    }
  }
}

void launch_chol_inverse(int n, double* work, double* ainv, int* status, cudaStream_t s) {
  k_chol_inverse<<<1, 1024, 0, s>>>(n, work, ainv, status);
  count_launch();
}

// w = M^{-1} A v and ||w||^2 into scal[S_NRM] (one power-iteration product).
template <class VT, class XT>
__global__ void __launch_bounds__(kBlock) k_power_step(const DevMat<VT> A,
                                                       const XT* __restrict__ v,
                                                       const XT* __restrict__ dinv,
                                                       XT* __restrict__ w, const RedWork rw,
                                                       double* scal) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
  double acc = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); s < A.nslices;
       s += nw) {
    const int64_t row = s * kSlice + lane;
    const XT t = row_spmv<1, VT, XT>(A, s, lane, row, v, XT(0));
    if (row < A.n) {
      const XT wi = t * dinv[row];
      w[row] = wi;
      acc += (double)wi * (double)wi;
    }
  }
  grid_sum(acc, rw, [&](double tot) { scal[S_NRM] = tot; });
}

template <class VT, class XT>
void launch_power_step(const DevMat<VT>& A, const XT* v, const XT* dinv, XT* w, const RedWork& rw,
                       double* scal, cudaStream_t s) {
  k_power_step<VT, XT><<<rw.grid, kBlock, 0, s>>>(A, v, dinv, w, rw, scal);
  count_launch();
}

template <class XT>
__global__ void __launch_bounds__(kBlock) k_scale_by_norm(int64_t n, const XT* __restrict__ w,
                                                          XT* __restrict__ v,
                                                          const double* __restrict__ scal,
                                                          int slot) {
  const double inv = 1.0 / sqrt(scal[slot]);
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) v[i] = XT((double)w[i] * inv);
}

template <class XT>
void launch_scale_by_norm(int64_t n, const XT* w, XT* v, const double* scal, int slot,
                          cudaStream_t s) {
  if (n == 0) return;
  k_scale_by_norm<XT><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, w, v, scal,
                                                                                slot);
  count_launch();
}

template <class XT>
__global__ void __launch_bounds__(kBlock) k_norm2(int64_t n, const XT* __restrict__ v,
                                                  const RedWork rw, double* scal, int slot) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock)
    acc += (double)v[i] * (double)v[i];
  grid_sum(acc, rw, [&](double tot) { scal[slot] = tot; });
}

template <class XT>
void launch_norm2(int64_t n, const XT* v, const RedWork& rw, double* scal, int slot,
                  cudaStream_t s) {
  k_norm2<XT><<<rw.grid, kBlock, 0, s>>>(n, v, rw, scal, slot);
  count_launch();
}

template void launch_coarse_gemv<double>(int, const double*, const double*, double*, cudaStream_t);
template void launch_coarse_gemv<float>(int, const double*, const float*, float*, cudaStream_t);
template void launch_power_step<double, double>(const DevMat<double>&, const double*, const double*,
                                                double*, const RedWork&, double*, cudaStream_t);
template void launch_power_step<float, float>(const DevMat<float>&, const float*, const float*,
                                                float*, const RedWork&, double*, cudaStream_t);
template void launch_power_step<__nv_bfloat16, float>(const DevMat<__nv_bfloat16>&, const float*,
                                                      const float*, float*, const RedWork&,
                                                      double*, cudaStream_t);
template void launch_scale_by_norm<double>(int64_t, const double*, double*, const double*, int,
                                           cudaStream_t);
template void launch_scale_by_norm<float>(int64_t, const float*, float*, const double*, int,
                                          cudaStream_t);
template void launch_norm2<double>(int64_t, const double*, const RedWork&, double*, int,
                                   cudaStream_t);
template void launch_norm2<float>(int64_t, const float*, const RedWork&, double*, int,
                                  cudaStream_t);

}  // namespace amgps
