// Smoother, transfer and conversion kernels of the V-cycle (Sec. 2 and 3).
//
// One launch of k_step is one degree step of a polynomial smoother: the SpMV
// with the current recurrence vector, the residual update, the l1-Jacobi
// scaling and the recurrence / solution updates share a single pass over A and
// the vectors (the fusion Sec. 3 obtains with its psb_upd_xyz kernel):
//
//   4th kind (Eq. polsmoother / polsmootheropt), step producing z_{j+1}:
//     t = A z_j ; r_j = r_{j-1} - t
//     z_{j+1} = c1 z_j + c2 M^{-1} r_j         c1 = (2j-1)/(2j+3), c2 = (8j+4)/(2j+3)/rho
//     x += beta_{j+1} z_{j+1}
//   1st kind (Algorithm 1), step producing d^(j):
//     t = A d^(j-1) ; r^(j) = r^(j-1) - (1/rho) M^{-1} t
//     d^(j) = rho_j rho_{j-1} d^(j-1) + (2 rho_j/delta) r^(j) ; x += d^(j)
//   l1-Jacobi sweep: x_new = x + M^{-1}(b - A x)
//
// D^{-1} = 1/M (Eq. l1smooth) is formed once per level (re-deriving M_i from
// the row plus an IEEE division every step would cost about four times the
// FP64 instructions of the whole step).  On FP64 and FP32 levels the
// polynomial steps go further and run on the row-scaled values a_ij / M_i with
// the residual kept as M^{-1} r (rho M^{-1} r for the 1st kind): the families
// FAM_CHEB4S/SR and FAM_CHEB1S/SR, which need no 1/M product or stream except
// where rin is still b.  The row's own vectors are loaded before the SpMV so
// their latency overlaps it.  z ping-pongs between two buffers because
// neighbouring rows gather z_j in the same launch that writes z_{j+1}.  Levels
// with wide rows use the split form (several warps per slice).
#include <type_traits>

#include "kernels_common.cuh"

namespace amgps {

template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN>
__global__ void __launch_bounds__(kBlock) k_step(const StepArgs<VT, XT> a) {
  const int lane = threadIdx.x & 31;
  int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (a.slices) {
    if (s >= a.nlist) return;
    s = a.slices[s];
  } else if (s >= a.A.nslices) {
    return;
  }
  step_slice<VT, XT, FAM, INIT, WR, ZOWN>(a, s, lane);
}

// Split form for levels with wide rows: one block per slice, a.split warps;
// warp g sums entries [g w / G, (g+1) w / G) of each row, warp 0 adds the
// partials in warp order (deterministic) and finishes the rows.
template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN>
__global__ void __launch_bounds__(32 * kMaxSplit) k_step_split(const StepArgs<VT, XT> a) {
  __shared__ XT part[kMaxSplit][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, G = blockDim.x >> 5;
  int64_t s = blockIdx.x;
  if (a.slices) {
    if (s >= a.nlist) return;
    s = a.slices[s];
  } else if (s >= a.A.nslices) {
    return;
  }
  const int64_t row = s * kSlice + lane;
  const bool live = row < a.A.n;
  using F = StepForm<FAM, INIT>;
  const XT rin = (live && g == 0) ? a.rin[row] : XT(0);
  const XT di = (live && g == 0 && step_needs_dinv<FAM>()) ? a.dinv[row] : XT(0);
  const int w = a.A.sd[s].w;
  const int k0 = (int)((int64_t)w * g / G), k1 = (int)((int64_t)w * (g + 1) / G);
  part[g][lane] = row_spmv_range<F::kSign, VT, XT>(
      a.A, s, lane, row, a.u, g == 0 ? step_init<FAM, F::kResidual>(rin, di) : XT(0), k0, k1);
  __syncthreads();
  if (g != 0 || !live) return;
  XT acc = part[0][lane];
  for (int q = 1; q < G; ++q) acc += part[q][lane];
  XT xin = XT(0), zo = XT(0);
  if (FAM != FAM_RES) xin = a.xin[row];
  if (ZOWN) zo = a.zown[row];
  step_finish<VT, XT, FAM, INIT, WR, ZOWN>(a, row, acc, rin, xin, di, zo);
}

template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN>
static void go(const StepArgs<VT, XT>& a, int64_t work, cudaStream_t s) {
  if (a.split > 1)
    k_step_split<VT, XT, FAM, INIT, WR, ZOWN><<<(unsigned)work, 32 * a.split, 0, s>>>(a);
  else
    k_step<VT, XT, FAM, INIT, WR, ZOWN>
        <<<(unsigned)((work + kWarpsPerBlock - 1) / kWarpsPerBlock), kBlock, 0, s>>>(a);
  count_launch();
}

template <class VT, class XT, int FAM, bool INIT>
static void dispatch_wr(const StepArgs<VT, XT>& a, int64_t work, cudaStream_t s) {
  const bool z = a.zown != nullptr;
  if (a.write_r) {
    if (z) go<VT, XT, FAM, INIT, true, true>(a, work, s);
    else go<VT, XT, FAM, INIT, true, false>(a, work, s);
  } else {
    if (z) go<VT, XT, FAM, INIT, false, true>(a, work, s);
    else go<VT, XT, FAM, INIT, false, false>(a, work, s);
  }
}

// Stored-operator steps (FP64 levels, one warp per slice): the flags of
// FAM_OP / FAM_OPT from the arguments.
template <class VT, class XT>
static void dispatch_op(const StepArgs<VT, XT>& a, int64_t work, cudaStream_t s) {
  if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
    const unsigned g = (unsigned)((work + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const bool s0 = a.rin != nullptr, s1 = a.xin != nullptr, wr = a.write_r;
    if (a.fam == FAM_OPT) {
      if (wr) k_step<VT, XT, FAM_OPT, true, true, false><<<g, kBlock, 0, s>>>(a);
      else k_step<VT, XT, FAM_OPT, true, false, false><<<g, kBlock, 0, s>>>(a);
    } else if (!s0) {
      k_step<VT, XT, FAM_OP, false, false, false><<<g, kBlock, 0, s>>>(a);
    } else if (!s1) {
      if (wr) k_step<VT, XT, FAM_OP, true, true, false><<<g, kBlock, 0, s>>>(a);
      else k_step<VT, XT, FAM_OP, true, false, false><<<g, kBlock, 0, s>>>(a);
    } else {
      if (wr) k_step<VT, XT, FAM_OP, true, true, true><<<g, kBlock, 0, s>>>(a);
      else k_step<VT, XT, FAM_OP, true, false, true><<<g, kBlock, 0, s>>>(a);
    }
    count_launch();
  }
}

template <class VT, class XT>
void launch_step(const StepArgs<VT, XT>& a, cudaStream_t s) {
  const int64_t work = a.slices ? a.nlist : a.A.nslices;
  if (work == 0) return;
  if (is_op(a.fam)) {
    dispatch_op<VT, XT>(a, work, s);
    return;
  }
  switch (a.fam) {
    case FAM_CHEB4:
      if (a.init) dispatch_wr<VT, XT, FAM_CHEB4, true>(a, work, s);
      else dispatch_wr<VT, XT, FAM_CHEB4, false>(a, work, s);
      break;
    case FAM_CHEB4S:
      dispatch_wr<VT, XT, FAM_CHEB4S, false>(a, work, s);
      break;
    case FAM_CHEB4SR:
      if (a.init) dispatch_wr<VT, XT, FAM_CHEB4SR, true>(a, work, s);
      else dispatch_wr<VT, XT, FAM_CHEB4SR, false>(a, work, s);
      break;
    case FAM_CHEB1S:
      dispatch_wr<VT, XT, FAM_CHEB1S, false>(a, work, s);
      break;
    case FAM_CHEB1SR:
      dispatch_wr<VT, XT, FAM_CHEB1SR, true>(a, work, s);
      break;
    case FAM_CHEB1:
      if (a.init) dispatch_wr<VT, XT, FAM_CHEB1, true>(a, work, s);
      else dispatch_wr<VT, XT, FAM_CHEB1, false>(a, work, s);
      break;
    case FAM_RES:
      go<VT, XT, FAM_RES, true, false, false>(a, work, s);
      break;
    default:
      go<VT, XT, FAM_JAC, true, false, false>(a, work, s);
  }
}

// First step from x = 0 (no product with A): first_row (kernels_common.cuh).
template <class XT, int FAM>
__global__ void __launch_bounds__(kBlock) k_first(int64_t n, const XT* __restrict__ b,
                                                  const XT* __restrict__ dinv,
                                                  XT* __restrict__ rout, XT* __restrict__ zout,
                                                  XT* __restrict__ xout, XT c2, XT beta,
                                                  XT rhoinv) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  first_row<XT, FAM>(i, b, dinv, rout, zout, xout, c2, beta, rhoinv);
}

template <class XT>
void launch_first(int fam, int64_t n, const XT* b, const XT* dinv, XT* rout, XT* zout, XT* xout,
                  XT c2, XT beta, XT rhoinv, cudaStream_t s) {
  if (n == 0) return;
  dim3 g((unsigned)((n + kBlock - 1) / kBlock));
  if (fam == FAM_CHEB4)
    k_first<XT, FAM_CHEB4><<<g, kBlock, 0, s>>>(n, b, dinv, rout, zout, xout, c2, beta, rhoinv);
  else if (fam == FAM_CHEB1)
    k_first<XT, FAM_CHEB1><<<g, kBlock, 0, s>>>(n, b, dinv, rout, zout, xout, c2, beta, rhoinv);
  else
    k_first<XT, FAM_JAC><<<g, kBlock, 0, s>>>(n, b, dinv, rout, zout, xout, c2, beta, rhoinv);
  count_launch();
}

// b_c = P^T res for an unsmoothed aggregation P (Sec. 2): one thread per coarse
// row adds the residuals of its children (cidx[cptr[I] .. cptr[I+1])) in list
// order, so the sum does not depend on scheduling.  The residual itself comes
// from the FAM_RES step (pipelined and coalesced like the smoother steps).
template <class XT>
__global__ void __launch_bounds__(kBlock) k_aggregate(const int32_t* __restrict__ cptr,
                                                      const int32_t* __restrict__ cidx, int64_t nc,
                                                      const XT* __restrict__ res,
                                                      XT* __restrict__ bc) {
  const int64_t I = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (I >= nc) return;
  aggregate_row<XT>(I, cptr, cidx, res, bc);
}

template <class XT>
void launch_aggregate(const int32_t* cptr, const int32_t* cidx, int64_t nc, const XT* res, XT* bc,
                      cudaStream_t s) {
  if (nc == 0) return;
  const unsigned g = (unsigned)((nc + kBlock - 1) / kBlock);
  k_aggregate<XT><<<g, kBlock, 0, s>>>(cptr, cidx, nc, res, bc);
  count_launch();
}

// x += P e_c (gather through the aggregate map).
template <class XT>
__global__ void __launch_bounds__(kBlock) k_prolong(int64_t n, const int32_t* __restrict__ agg,
                                                    const XT* __restrict__ ec, XT* x) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) prolong_row<XT>(i, agg, ec, x);
}

template <class XT>
void launch_prolong(int64_t n, const int32_t* agg, const XT* ec, XT* x, cudaStream_t s) {
  if (n == 0) return;
  k_prolong<XT><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, agg, ec, x);
  count_launch();
}

template <class XT>
__global__ void __launch_bounds__(kBlock) k_add(int64_t n, const XT* __restrict__ x,
                                                const XT* __restrict__ y, XT* out) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) out[i] = x[i] + y[i];
}

template <class XT>
void launch_add(int64_t n, const XT* x, const XT* y, XT* out, cudaStream_t s) {
  if (n == 0) return;
  k_add<XT><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, x, y, out);
  count_launch();
}

// 1/M_i with M_i of Eq. l1smooth (a_ii + sum_{j != i} |a_ij|), formed once per level.
template <class VT, class XT>
__global__ void __launch_bounds__(kBlock) k_l1diag(const DevMat<VT> A, XT* __restrict__ dinv) {
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (s >= A.nslices) return;
  const int64_t row = s * kSlice + lane;
  const SliceDesc d = A.sd[s];
  const int64_t nm1 = A.n - 1;
  XT m = XT(0);
  for (int k = 0; k < d.w; ++k) {
    const int64_t e = d.vbase + (int64_t)k * kSlice + lane;
    const XT a = XT(ldval(A.val + e));
    int64_t c;
    if (d.cref >= 0) {
      c = row + (int64_t)A.off[d.cref + k];
      c = c < 0 ? 0 : (c > nm1 ? nm1 : c);
    } else {
      c = A.col[e];
    }
    m += (c == row) ? a : absv(a);
  }
  if (row < A.n) dinv[row] = XT(1) / m;
}

template <class VT, class XT>
void launch_l1diag(const DevMat<VT>& A, XT* dinv, cudaStream_t s) {
  if (A.nslices == 0) return;
  dim3 g((unsigned)((A.nslices + kWarpsPerBlock - 1) / kWarpsPerBlock));
  k_l1diag<VT, XT><<<g, kBlock, 0, s>>>(A, dinv);
  count_launch();
}

// Operator values of one stored-operator step, m = tau I - sigma B, entry by
// entry of B's layout.  The row's diagonal slot: offset 0 of a uniform slice,
// else the first stored column equal to the row (explicit rows are sorted by
// column and padded after their entries).  Rows past n keep zeros.
__global__ void __launch_bounds__(kBlock) k_build_op(const DevMat<double> B, double tau,
                                                     double sigma, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (s >= B.nslices) return;
  const int64_t row = s * kSlice + lane;
  const SliceDesc d = B.sd[s];
  bool seen = false;
  for (int k = 0; k < d.w; ++k) {
    const int64_t e = d.vbase + (int64_t)k * kSlice + lane;
    bool dg;
    if (d.cref >= 0) {
      dg = B.off[d.cref + k] == 0;
    } else {
      dg = !seen && B.col[e] == row;
      seen = seen || dg;
    }
    const double v = B.val[e];
    out[e] = row < B.n ? (dg ? fma(-sigma, v, tau) : -sigma * v) : 0.0;
  }
}

void launch_build_op(const DevMat<double>& B, double tau, double sigma, double* out,
                     cudaStream_t s) {
  if (B.nslices == 0) return;
  dim3 g((unsigned)((B.nslices + kWarpsPerBlock - 1) / kWarpsPerBlock));
  k_build_op<<<g, kBlock, 0, s>>>(B, tau, sigma, out);
  count_launch();
}

template <class A, class B>
__global__ void __launch_bounds__(kBlock) k_convert(int64_t n, const A* __restrict__ in,
                                                    B* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (i < n) out[i] = B(in[i]);
}

template <class A, class B>
void launch_convert(int64_t n, const A* in, B* out, cudaStream_t s) {
  if (n == 0) return;
  k_convert<A, B><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, in, out);
  count_launch();
}

#define AMGPS_INST(VT, XT)                                                                   \
  template void launch_step<VT, XT>(const StepArgs<VT, XT>&, cudaStream_t);                  \
  template void launch_l1diag<VT, XT>(const DevMat<VT>&, XT*, cudaStream_t);
AMGPS_INST(double, double)
AMGPS_INST(float, float)
AMGPS_INST(__nv_bfloat16, float)
#undef AMGPS_INST

template void launch_first<double>(int, int64_t, const double*, const double*, double*, double*,
                                   double*, double, double, double, cudaStream_t);
template void launch_first<float>(int, int64_t, const float*, const float*, float*, float*,
                                  float*, float, float, float, cudaStream_t);
template void launch_aggregate<double>(const int32_t*, const int32_t*, int64_t, const double*,
                                       double*, cudaStream_t);
template void launch_aggregate<float>(const int32_t*, const int32_t*, int64_t, const float*, float*,
                                      cudaStream_t);
template void launch_prolong<double>(int64_t, const int32_t*, const double*, double*, cudaStream_t);
template void launch_add<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template void launch_prolong<float>(int64_t, const int32_t*, const float*, float*, cudaStream_t);
template void launch_convert<double, float>(int64_t, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(int64_t, const float*, double*, cudaStream_t);
template void launch_convert<double, double>(int64_t, const double*, double*, cudaStream_t);

// Transfers through a general prolongator (explicit SELL-32, FP64 values):
// y = M u (add = 0) or y += M u (add = 1).  M = R = P^T restricts
// (b_c = P^T r), M = P prolongs (x += P x_c).  One warp per slice, or with
// split > 1 one block per slice whose warps share the row's entries (partials
// added in warp order).
template <class XT>
__global__ void __launch_bounds__(kBlock) k_xfer(const DevMat<double> M, const XT* __restrict__ u,
                                                 XT* __restrict__ y, int add) {
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (s >= M.nslices) return;
  const int64_t row = s * kSlice + lane;
  const XT init = (add && row < M.n) ? y[row] : XT(0);
  const XT t = row_spmv<1, double, XT>(M, s, lane, row, u, init);
  if (row < M.n) y[row] = t;
}

template <class XT>
__global__ void __launch_bounds__(32 * kMaxSplit) k_xfer_split(const DevMat<double> M,
                                                               const XT* __restrict__ u,
                                                               XT* __restrict__ y, int add) {
  __shared__ XT part[kMaxSplit][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, G = blockDim.x >> 5;
  const int64_t s = blockIdx.x;
  if (s >= M.nslices) return;
  const int64_t row = s * kSlice + lane;
  const bool live = row < M.n;
  const XT init = (add && live && g == 0) ? y[row] : XT(0);
  const int w = M.sd[s].w;
  const int k0 = (int)((int64_t)w * g / G), k1 = (int)((int64_t)w * (g + 1) / G);
  part[g][lane] = row_spmv_range<1, double, XT>(M, s, lane, row, u, init, k0, k1);
  __syncthreads();
  if (g != 0 || !live) return;
  XT t = part[0][lane];
  for (int q = 1; q < G; ++q) t += part[q][lane];
  y[row] = t;
}

template <class XT>
void launch_xfer(const DevMat<double>& M, const XT* u, XT* y, int add, int split, cudaStream_t s) {
  if (M.nslices == 0) return;
  if (split > 1) {
    k_xfer_split<XT><<<(unsigned)M.nslices, 32 * split, 0, s>>>(M, u, y, add);
  } else {
    const unsigned grid = (unsigned)((M.nslices + kWarpsPerBlock - 1) / kWarpsPerBlock);
    k_xfer<XT><<<grid, kBlock, 0, s>>>(M, u, y, add);
  }
  count_launch();
}
template void launch_xfer<double>(const DevMat<double>&, const double*, double*, int, int,
                                  cudaStream_t);
template void launch_xfer<float>(const DevMat<double>&, const float*, float*, int, int,
                                 cudaStream_t);

}  // namespace amgps
