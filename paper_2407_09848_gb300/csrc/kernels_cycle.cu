// Persistent kernel for the coarse levels of a V-cycle (Eq. amg).
//
// Below the levels that run the TMA-fed step, every kernel of a V-cycle
// (smoother steps, first steps, residual + restriction, prolongation, the
// coarsest solve) lasts a few microseconds, so launch latency dominated them
// even inside a CUDA graph.  Here one co-resident grid walks the recorded
// phase list: each phase spreads its slices (steps), rows (elementwise
// phases) or coarse rows over all warps or threads of the grid, then every
// block meets at a grid-wide barrier before the next phase reads what the
// previous one wrote.  The per-row code is that of the launched kernels
// (step_slice, first_row, aggregate_row, prolong_row, coarse_gemv_row in
// kernels_common.cuh), so the results are bit for bit those of the launched
// sequence.  Vectors written by an earlier phase are read with L2 (coherent)
// loads, never through the read-only path.
//
// The barrier's waits are bounded: a block that gives up sets the solver's
// error slot and leaves the kernel; the host reports AMGPS_E_TIMEOUT.
#include "kernels_common.cuh"

namespace amgps {
namespace {

constexpr int kCycleThreads = 512;
constexpr int kCycleMaxBlocksPerSm = 1;
constexpr uint32_t kBarrierSpins = 1u << 22;  // L2 polls (~0.5 us each): about two seconds at most

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All blocks of the grid meet for the q-th time (q = 1, 2, ...): one
// arrival counter that only grows (zeroed before the launch); a block's
// thread 0 publishes the block's writes (fence, then its arrival) and waits
// until the counter reaches q x blocks.  False if this block's wait gave up.
__device__ bool grid_barrier(const CycleSync& sy, unsigned target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(sy.count, 1u);
    uint32_t i = 0;
    while (ld_acquire(sy.count) < target) {
      if (++i > kBarrierSpins) {
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN>
__device__ __forceinline__ void cy_slices(const StepArgs<VT, XT>& a, int64_t gw, int64_t nw,
                                          int lane) {
  for (int64_t s = gw; s < a.A.nslices; s += nw)
    step_slice<VT, XT, FAM, INIT, WR, ZOWN, true>(a, s, lane);
}

template <class VT, class XT, int FAM, bool INIT>
__device__ __forceinline__ void cy_step_wr(const StepArgs<VT, XT>& a, int64_t gw, int64_t nw,
                                           int lane) {
  if (a.write_r) {
    if (a.zown) cy_slices<VT, XT, FAM, INIT, true, true>(a, gw, nw, lane);
    else cy_slices<VT, XT, FAM, INIT, true, false>(a, gw, nw, lane);
  } else {
    if (a.zown) cy_slices<VT, XT, FAM, INIT, false, true>(a, gw, nw, lane);
    else cy_slices<VT, XT, FAM, INIT, false, false>(a, gw, nw, lane);
  }
}

// the family dispatch of launch_step (kernels_smooth.cu)
template <class VT, class XT>
__device__ void cy_step(const StepArgs<VT, XT>& a, int64_t gw, int64_t nw, int lane) {
  switch (a.fam) {
    case FAM_CHEB4:
      if (a.init) cy_step_wr<VT, XT, FAM_CHEB4, true>(a, gw, nw, lane);
      else cy_step_wr<VT, XT, FAM_CHEB4, false>(a, gw, nw, lane);
      break;
    case FAM_CHEB4S:
      cy_step_wr<VT, XT, FAM_CHEB4S, false>(a, gw, nw, lane);
      break;
    case FAM_CHEB4SR:
      if (a.init) cy_step_wr<VT, XT, FAM_CHEB4SR, true>(a, gw, nw, lane);
      else cy_step_wr<VT, XT, FAM_CHEB4SR, false>(a, gw, nw, lane);
      break;
    case FAM_CHEB1S:
      cy_step_wr<VT, XT, FAM_CHEB1S, false>(a, gw, nw, lane);
      break;
    case FAM_CHEB1SR:
      cy_step_wr<VT, XT, FAM_CHEB1SR, true>(a, gw, nw, lane);
      break;
    case FAM_CHEB1:
      if (a.init) cy_step_wr<VT, XT, FAM_CHEB1, true>(a, gw, nw, lane);
      else cy_step_wr<VT, XT, FAM_CHEB1, false>(a, gw, nw, lane);
      break;
    case FAM_RES:
      cy_slices<VT, XT, FAM_RES, true, false, false>(a, gw, nw, lane);
      break;
    default:
      cy_slices<VT, XT, FAM_JAC, true, false, false>(a, gw, nw, lane);
  }
}

template <class VT, class XT>
__global__ void __launch_bounds__(kCycleThreads, kCycleMaxBlocksPerSm)
    k_cycle(const CyclePhase<VT, XT>* __restrict__ phases, int nph, const CycleSync sy,
            double* err) {
  __shared__ CyclePhase<VT, XT> P;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (kCycleThreads / 32) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * (kCycleThreads / 32);
  const int64_t gt = (int64_t)blockIdx.x * kCycleThreads + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * kCycleThreads;
  static_assert(sizeof(CyclePhase<VT, XT>) % 4 == 0, "phase copied as 32-bit words");
  constexpr int kWords = (int)(sizeof(CyclePhase<VT, XT>) / 4);
  for (int q = 0; q < nph; ++q) {
    // the phase descriptor into shared memory (the list is never written here)
    for (int w = threadIdx.x; w < kWords; w += kCycleThreads)
      reinterpret_cast<uint32_t*>(&P)[w] = __ldg(reinterpret_cast<const uint32_t*>(phases + q) + w);
    __syncthreads();
    switch (P.op) {
      case CY_STEP:
        cy_step<VT, XT>(P.a, gw, nw, lane);
        break;
      case CY_FIRST:
        for (int64_t i = gt; i < P.n; i += nt) {
          if (P.fam == FAM_CHEB4)
            first_row<XT, FAM_CHEB4, true>(i, P.in0, P.in1, P.out0, P.out1, P.out2, P.c2, P.beta,
                                           P.rhoinv);
          else if (P.fam == FAM_CHEB1)
            first_row<XT, FAM_CHEB1, true>(i, P.in0, P.in1, P.out0, P.out1, P.out2, P.c2, P.beta,
                                           P.rhoinv);
          else
            first_row<XT, FAM_JAC, true>(i, P.in0, P.in1, P.out0, P.out1, P.out2, P.c2, P.beta,
                                         P.rhoinv);
        }
        break;
      case CY_AGG:
        for (int64_t I = gt; I < P.n; I += nt)
          aggregate_row<XT, true>(I, P.i0, P.i1, P.in0, P.out0);
        break;
      case CY_PROLONG:
        for (int64_t i = gt; i < P.n; i += nt) prolong_row<XT, true>(i, P.i0, P.in0, P.out0);
        break;
      case CY_GEMV:
        for (int64_t i = gw; i < P.n; i += nw)
          coarse_gemv_row<XT, true>((int)i, (int)P.n, P.ainv, P.in0, P.out0, lane);
        break;
      default:  // CY_COPY
        for (int64_t i = gt; i < P.n; i += nt) P.out0[i] = __ldcg(P.in0 + i);
    }
    // the next phase reads what this one wrote (and overwrites P)
    if (!grid_barrier(sy, (unsigned)(q + 1) * gridDim.x)) {
      if (threadIdx.x == 0) *err = 1.0;
      return;
    }
  }
}

}  // namespace

template <class VT, class XT>
int cycle_grid(int nsm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cycle<VT, XT>, kCycleThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm > kCycleMaxBlocksPerSm) per_sm = kCycleMaxBlocksPerSm;
  return per_sm * nsm;
}

template <class VT, class XT>
cudaError_t launch_cycle(const CyclePhase<VT, XT>* phases, int nph, const CycleSync& sync, int grid,
                         double* err, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kCycleThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_cycle<VT, XT>, phases, nph, sync, err);
  if (e == cudaSuccess) count_launch();
  return e;
}

#define AMGPS_CYCLE_INST(VT, XT)                                                              \
  template int cycle_grid<VT, XT>(int);                                                       \
  template cudaError_t launch_cycle<VT, XT>(const CyclePhase<VT, XT>*, int, const CycleSync&, \
                                            int, double*, cudaStream_t);
AMGPS_CYCLE_INST(double, double)
AMGPS_CYCLE_INST(float, float)
AMGPS_CYCLE_INST(__nv_bfloat16, float)
#undef AMGPS_CYCLE_INST

}  // namespace amgps
