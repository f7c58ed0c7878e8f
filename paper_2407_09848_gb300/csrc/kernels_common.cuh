// Device helpers shared by the kernel translation units.
#pragma once

#include "amgps_internal.h"

namespace amgps {

// Matrix values are streamed once per step: cache-streaming loads (evict-first
// in L1 and L2) keep them from displacing the vectors that neighbouring rows
// gather.  BF16 values are widened to FP32.
__device__ __forceinline__ double ldval(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ldval(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float ldval(const __nv_bfloat16* p) {
  unsigned short s = __ldcs(reinterpret_cast<const unsigned short*>(p));
  return __bfloat162float(__ushort_as_bfloat16(s));
}

template <class T>
__device__ __forceinline__ T absv(T v) { return v < T(0) ? -v : v; }

// Load of a vector entry.  CG = false: a plain load, or for the gathered
// operand of a product the read-only path (__ldg), which is valid in kernels
// whose launch does not write that vector.  CG = true: an L2 (coherent) load,
// for the persistent kernel that reads in one phase what other blocks wrote in
// an earlier phase of the same launch.
template <bool CG, class T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}
template <bool CG, class T>
__device__ __forceinline__ T ldu(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

// init + SIGN * (A u)_row from one pass over the row (SIGN = +1 or -1, so a
// residual b - A u comes out of the same multiply-adds).  `lane` is the row's
// position in slice `s`.  Rows past n (tail of the last slice) see only zero
// padding and clamped, in-range columns.  FP64 arithmetic is the scarce
// resource on this GPU (its FP64 pipe issues about 2 FMAs per clock per SM),
// so the row costs exactly one multiply-add per stored entry and nothing else.
// Entries k in [k0, k1) of row `row` of slice s: init + SIGN * sum a_k u_{c_k}.
template <int SIGN, class VT, class XT, bool CG = false>
__device__ __forceinline__ XT row_spmv_range(const DevMat<VT>& A, int64_t s, int lane, int64_t row,
                                             const XT* __restrict__ u, XT init, int k0, int k1) {
  const SliceDesc d = A.sd[s];
  const int64_t nm1 = A.n - 1;
  XT t = init;
  if (k1 - k0 == 7) {
    // the seven entries of a 7-point row without guards: on GB300's narrow
    // FP64 pipe a predicated-off multiply-add still takes an issue slot
    // (same operations in the same order as the general loop below)
    XT a[7];
    int64_t c[7];
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) {
      const int k = k0 + kk;
      const int64_t e = d.vbase + (int64_t)k * kSlice + lane;
      a[kk] = XT(ldval(A.val + e));
      if (d.cref >= 0) {
        const int64_t cc = row + (int64_t)A.off[d.cref + k];
        c[kk] = cc < 0 ? 0 : (cc > nm1 ? nm1 : cc);
      } else {
        c[kk] = A.col[e];
      }
    }
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) t = fma(SIGN > 0 ? a[kk] : -a[kk], ldu<CG>(u + c[kk]), t);
    return t;
  }
  for (int kb = k0; kb < k1; kb += 8) {
    XT a[8];
    int64_t c[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = kb + kk;
      a[kk] = XT(0);
      c[kk] = 0;
      if (k < k1) {
        const int64_t e = d.vbase + (int64_t)k * kSlice + lane;
        a[kk] = XT(ldval(A.val + e));
        if (d.cref >= 0) {
          int64_t cc = row + (int64_t)A.off[d.cref + k];
          c[kk] = cc < 0 ? 0 : (cc > nm1 ? nm1 : cc);
        } else {
          c[kk] = A.col[e];
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
      if (kb + kk < k1) t = fma(SIGN > 0 ? a[kk] : -a[kk], ldu<CG>(u + c[kk]), t);
  }
  return t;
}

// The whole row: entries 0 .. w-1 of the slice.
template <int SIGN, class VT, class XT, bool CG = false>
__device__ __forceinline__ XT row_spmv(const DevMat<VT>& A, int64_t s, int lane, int64_t row,
                                       const XT* __restrict__ u, XT init) {
  return row_spmv_range<SIGN, VT, XT, CG>(A, s, lane, row, u, init, 0, A.sd[s].w);
}

// The SpMV of one smoother step is accumulated as init + SIGN * (A u):
// r_j = r_{j-1} - A z_j directly for the 4th kind, the 1st-kind initial step
// and Jacobi (init = r_in, SIGN = -1); the plain product t = A d for the
// other 1st-kind steps (init = 0, SIGN = +1).
// The stored-operator steps add their operator's products to the vector terms
// (FAM_OP) or subtract the row-scaled products from q (FAM_OPT).
template <int FAM, bool INIT>
struct StepForm {
  static constexpr bool kResidual = !(FAM == FAM_CHEB1 && !INIT);
  static constexpr int kSign = FAM == FAM_OP ? 1 : (kResidual ? -1 : 1);
};

// Whether a step reads 1/M: every step but the residual, the scaled
// 4th-kind step with scaled rin and the stored-operator steps.
template <int FAM>
__device__ __forceinline__ constexpr bool step_needs_dinv() {
  return FAM != FAM_RES && FAM != FAM_CHEB4S && FAM != FAM_CHEB1S && !is_op(FAM);
}

// Stored-operator steps: the vector terms the accumulation starts from
// (s0 = slot-0 entry of the row, s1 = slot-1 entry), then the stores.
template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN>
__device__ __forceinline__ XT op_init(const StepArgs<VT, XT>& a, XT s0, XT s1) {
  XT acc = XT(0);
  if constexpr (FAM == FAM_OPT) {
    acc = s0;
  } else {
    if constexpr (INIT) acc = WR ? s0 : a.c2 * s0;
    if constexpr (ZOWN) acc = INIT ? fma(a.c1, s1, acc) : a.c1 * s1;
  }
  return acc;
}
template <class VT, class XT, int FAM, bool WR>
__device__ __forceinline__ void op_finish(const StepArgs<VT, XT>& a, int64_t row, XT acc, XT ucen) {
  a.zout[row] = acc;
  if constexpr (FAM == FAM_OPT && WR) a.rout[row] = fma(a.beta, acc, ucen);
}

// Starting value of the accumulation: rin for the residual forms ((1/M) rin
// when a scaled step's rin is still unscaled), 0 otherwise.
template <int FAM, bool RESID, class XT>
__device__ __forceinline__ XT step_init(XT rin, XT di) {
  if constexpr (!RESID) return XT(0);
  else if constexpr (FAM == FAM_CHEB4SR || FAM == FAM_CHEB1SR) return rin * di;
  else return rin;
}

// Epilogue of one smoother step for one row, given the accumulated SpMV and
// the row's own vector entries (see kernels_smooth.cu for the recurrences).
template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN>
__device__ __forceinline__ void step_finish(const StepArgs<VT, XT>& a, int64_t row, XT acc, XT rin,
                                            XT xin, XT di, XT zo) {
  if constexpr (is_cheb4(FAM)) {
    const XT r = acc;  // r_j, or M^{-1} r_j in the scaled forms
    if (WR) a.rout[row] = r;
    XT z;
    if constexpr (FAM == FAM_CHEB4) z = a.c2 * (r * di);
    else z = a.c2 * r;
    if (ZOWN) z = fma(a.c1, zo, z);
    a.zout[row] = z;
    a.xout[row] = fma(a.beta, z, xin);
  } else if constexpr (FAM == FAM_CHEB1) {
    XT r;
    if (INIT) r = a.rhoinv * (acc * di);
    else r = fma(-(a.rhoinv * di), acc, rin);
    if (WR) a.rout[row] = r;
    XT z = a.c2 * r;
    if (ZOWN) z = fma(a.c1, zo, z);
    a.zout[row] = z;
    a.xout[row] = xin + z;
  } else if constexpr (FAM == FAM_CHEB1S || FAM == FAM_CHEB1SR) {
    const XT r = acc;  // rho M^{-1} r
    if (WR) a.rout[row] = r;
    XT z = a.c2 * r;  // c2 carries the 1/rho
    if (ZOWN) z = fma(a.c1, zo, z);
    a.zout[row] = z;
    a.xout[row] = xin + z;
  } else if constexpr (FAM == FAM_JAC) {
    a.xout[row] = fma(acc, di, xin);
  } else {
    a.zout[row] = acc;  // FAM_RES: the true residual b - A x
  }
}

// One smoother step on the 32 rows of slice s, one row per lane, operands
// read from global memory (the direct form of the step).
template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN, bool CG = false>
__device__ __forceinline__ void step_slice(const StepArgs<VT, XT>& a, int64_t s, int lane) {
  const int64_t row = s * kSlice + lane;
  const bool live = row < a.A.n;
  if constexpr (is_op(FAM)) {
    XT s0 = XT(0), s1 = XT(0), uc = XT(0);
    if (live) {
      if (reads_slot0<FAM, INIT>()) s0 = ldv<CG>(a.rin + row);
      if (reads_slot1<FAM, ZOWN>()) s1 = ldv<CG>(a.xin + row);
      if (FAM == FAM_OPT && WR) uc = ldv<CG>(a.u + row);
    }
    constexpr int kSign = StepForm<FAM, INIT>::kSign;
    const XT acc = row_spmv<kSign, VT, XT, CG>(a.A, s, lane, row, a.u,
                                               op_init<VT, XT, FAM, INIT, WR, ZOWN>(a, s0, s1));
    if (live) op_finish<VT, XT, FAM, WR>(a, row, acc, uc);
    return;
  }
  XT rin = XT(0), xin = XT(0), zo = XT(0), di = XT(0);
  if (live) {
    rin = ldv<CG>(a.rin + row);
    if (FAM != FAM_RES) xin = ldv<CG>(a.xin + row);
    if (step_needs_dinv<FAM>()) di = a.dinv[row];  // formed at set-up, never written here
    if (ZOWN) zo = ldv<CG>(a.zown + row);
  }
  using F = StepForm<FAM, INIT>;
  const XT acc = row_spmv<F::kSign, VT, XT, CG>(a.A, s, lane, row, a.u,
                                                 step_init<FAM, F::kResidual>(rin, di));
  if (!live) return;
  step_finish<VT, XT, FAM, INIT, WR, ZOWN>(a, row, acc, rin, xin, di, zo);
}

// Per-element bodies of the elementwise V-cycle kernels, shared by their own
// launches (kernels_smooth.cu, kernels_krylov.cu) and by the persistent
// coarse-level kernel (kernels_cycle.cu), so both give the same bits.

// First step from x = 0 (no product with A), row i:
//   4th kind: z_1 = c2 M^{-1} b, x = beta_1 z_1 (r_0 = b is not copied)
//   1st kind: r^(0) = (1/rho) M^{-1} b, d^(0) = r^(0)/theta, x = d^(0)
//   Jacobi:   x = M^{-1} b
template <class XT, int FAM, bool CG = false>
__device__ __forceinline__ void first_row(int64_t i, const XT* b, const XT* dinv, XT* rout,
                                          XT* zout, XT* xout, XT c2, XT beta, XT rhoinv) {
  const XT bm = ldv<CG>(b + i) * dinv[i];
  if constexpr (FAM == FAM_CHEB4) {
    const XT z = c2 * bm;
    zout[i] = z;
    xout[i] = beta * z;
  } else if constexpr (FAM == FAM_CHEB1) {
    const XT r = rhoinv * bm;
    rout[i] = r;
    const XT z = c2 * r;
    zout[i] = z;
    xout[i] = z;
  } else {
    xout[i] = bm;
  }
}

// b_c[I] = sum of res over the children of coarse row I, in list order
template <class XT, bool CG = false>
__device__ __forceinline__ void aggregate_row(int64_t I, const int32_t* cptr, const int32_t* cidx,
                                              const XT* res, XT* bc) {
  XT acc = XT(0);
  const int q1 = cptr[I + 1];
  for (int q = cptr[I]; q < q1; ++q) acc += ldv<CG>(res + cidx[q]);
  bc[I] = acc;
}

// x_i += e_c[agg_i]
template <class XT, bool CG = false>
__device__ __forceinline__ void prolong_row(int64_t i, const int32_t* agg, const XT* ec, XT* x) {
  x[i] = ldv<CG>(x + i) + ldv<CG>(ec + agg[i]);
}

// x_i = (A_c^{-1} b)_i for the coarsest level, one warp per row: lane l sums
// columns l, l + 32, ... in order, then a fixed butterfly adds the lanes
template <class XT, bool CG = false>
__device__ __forceinline__ void coarse_gemv_row(int i, int nc, const double* ainv, const XT* b,
                                                XT* x, int lane) {
  const double* row = ainv + (size_t)i * nc;
  double acc = 0.0;
  for (int j = lane; j < nc; j += 32) acc = fma(row[j], (double)ldv<CG>(b + j), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[i] = XT(acc);
}

// Sum over a block (any blockDim multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// Deterministic grid-wide sum: each block writes its partial, the last block to
// arrive adds the partials in index order with a fixed tree and calls
// fin(total) from thread 0, then re-arms the counter.  The grid size is a pure
// function of the problem size, so the result is bitwise reproducible.
template <class Fin>
__device__ __forceinline__ void grid_sum(double v, const RedWork& w, Fin fin) {
  __shared__ double sh[32];
  __shared__ bool last;
  double b = block_sum(v, sh);
  if (threadIdx.x == 0) {
    w.part[blockIdx.x] = b;
    __threadfence();
    const unsigned t = atomicAdd(w.counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(w.part + i);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      fin(s);
      *w.counter = 0u;
    }
  }
}

}  // namespace amgps
