// TMA-fed fused smoother step: the k_step recurrences (Sec. 2.1, 2.2) with
// every global read staged by the Tensor Memory Accelerator.
//
// A persistent grid walks a list of tiles round-robin, so the tiles in flight
// at any moment form one contiguous band and the vector windows that
// neighbouring tiles share are read from HBM once and then from L2.  Warp 0 of
// each CTA is the producer: one lane issues cp.async.bulk copies of a tile's
// values, of its rows of r_in, x_in and (when the step needs it, FP32 vectors)
// 1/M, and of
// the contiguous windows of the multiplied vector u (one per group of nearby
// column offsets) into a shared-memory stage, completing on that stage's
// "full" mbarrier.  The other warps are consumers, in groups that take
// alternate tiles; a group's warps split the tile's 32-row slices: they wait
// on "full", evaluate the rows from shared memory, store r/z/x to global
// memory, and arrive on the stage's "empty" mbarrier so the producer may
// refill it.  Before the tiles, while the first copies land, all consumers
// run the slices outside the plan with direct loads.  The arithmetic and its
// order are those of k_step, so both paths give the same bits.  The same
// pipeline runs the recurrence steps and the stored-operator steps (FAM_OP,
// FAM_OPT), whose values are the step's own operator and whose per-row
// vectors are copied only when the step reads them.  Tile height, groups and
// CTAs per SM come from TmaShape<XT>: for FP64 one CTA per SM with two groups
// of 8 warps and four 512-row stages in flight (copies issued three tiles
// ahead of the FP64-bound consumers), for FP32 vectors two CTAs per SM of 16
// consumers on 1024-row tiles.
//
// Rows of the 7-point pattern (seven sorted offsets, the row itself in the
// middle) take a variant with the width fixed at compile time: exactly seven
// multiply-adds per row with no guarded eighth one (on GB300's narrow FP64
// pipe a predicated-off DFMA still costs an issue slot), and the centre entry
// multiplies the z_j value the row already loaded for its c1 term; a lane of
// that variant evaluates two rows of the tile with their multiply-add chains
// interleaved (8 consumer warps per group on 512-row tiles instead of 15 of
// one row each on 480-row tiles: 323 -> 318 us per 256^3 step).
//
// Every wait is bounded (kWaitSpins polls).  A wait that gives up sets the
// solver's error slot and makes all warps leave their loops; the producer
// still waits (bounded) for the copies it issued before it exits.
#include <type_traits>

#include "kernels_common.cuh"

namespace amgps {
namespace {

constexpr uint32_t kWaitSpins = 1u << 21;
constexpr int kBarrierBytes = 2 * kTmaMaxStages * 8;  // full[] and empty[] (128 B)

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// true when the phase of `parity` has completed; false after kWaitSpins polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitSpins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

template <class XT>
__device__ __forceinline__ XT widen(double v) { return XT(v); }
template <class XT>
__device__ __forceinline__ XT widen(float v) { return XT(v); }
template <class XT>
__device__ __forceinline__ XT widen(__nv_bfloat16 v) { return XT(__bfloat162float(v)); }

// consumer warps per CTA
template <class XT>
__host__ __device__ constexpr int tma_warps() {
  return TmaShape<XT>::kGroups * TmaShape<XT>::kConsumers;
}

// W = 0: up to kTmaMaxW entries per row (p.w at run time); W > 0: exactly W,
// with entry W / 2 the row itself (checked by the launcher)
template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN, int W>
__global__ void __launch_bounds__((tma_warps<XT>() + 1) * 32, TmaShape<XT>::kCtasPerSm)
    k_step_tma(const StepArgs<VT, XT> a, const TmaPlan p, const TmaTile* __restrict__ tiles,
               int ntiles, const int32_t* __restrict__ gen, int64_t ngen, double* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ volatile int abort_flag;
  __shared__ long long stage_r0[kTmaMaxStages];  // first row of the tile held by each stage
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kTmaMaxStages;
  unsigned char* stages = smem + kBarrierBytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ns = p.nstages;

  if (threadIdx.x == 0) {
    for (int i = 0; i < ns; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], TmaShape<XT>::kConsumers);  // one group consumes a tile
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    // The whole warp fetches the descriptors of this CTA's next 32 tiles in one
    // load; lane 0 then issues their copies without a global round trip per tile.
    int it = 0;
    for (int j0 = blockIdx.x; j0 < ntiles; j0 += 32 * gridDim.x) {
      if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) break;  // warp-uniform exit
      const int jl = j0 + lane * gridDim.x;
      TmaTile mine{0, 0};
      if (jl < ntiles) mine = tiles[jl];
      const int cnt = min(32, (ntiles - j0 + (int)gridDim.x - 1) / (int)gridDim.x);
      for (int q = 0; q < cnt; ++q) {
        const long long rq = __shfl_sync(0xffffffffu, (long long)mine.r0, q);
        const long long vq = __shfl_sync(0xffffffffu, (long long)mine.vbase, q);
        if (lane == 0) {
          const int st = it % ns;
          const uint32_t ph = (uint32_t)(it / ns) & 1u;
          if (abort_flag || !mbar_wait(&empty[st], ph ^ 1u)) {
            abort_flag = 1;
          } else {
            unsigned char* base = stages + (size_t)st * p.stage_bytes;
            const int64_t r0 = rq;
            stage_r0[st] = rq;
            // the residual needs no x_in or 1/M; a scaled step with scaled rin no
            // 1/M; FP64 stages hold no 1/M slot (read from global memory)
            // (a stored-operator step copies the slots it reads)
            constexpr bool wdi = step_needs_dinv<FAM>() && TmaShape<XT>::kVecSlots == 3;
            constexpr bool c0 = reads_slot0<FAM, INIT>(), c1 = reads_slot1<FAM, ZOWN>();
            constexpr int nvec = (c0 ? 1 : 0) + (c1 ? 1 : 0) + (wdi ? 1 : 0);
            mbar_expect_tx(&full[st], (uint32_t)(p.vals_bytes + nvec * p.vec_bytes + p.win_bytes));
            bulk_g2s(base, a.A.val + vq, (uint32_t)p.vals_bytes, &full[st]);
            XT* sv = reinterpret_cast<XT*>(base + p.vals_bytes);
            if (c0) bulk_g2s(sv, a.rin + r0, (uint32_t)p.vec_bytes, &full[st]);
            if (c1) bulk_g2s(sv + p.rows, a.xin + r0, (uint32_t)p.vec_bytes, &full[st]);
            if (wdi) bulk_g2s(sv + 2 * p.rows, a.dinv + r0, (uint32_t)p.vec_bytes, &full[st]);
            XT* sw = sv + TmaShape<XT>::kVecSlots * p.rows;
            for (int g = 0; g < p.ngroups; ++g)
              bulk_g2s(sw + p.g_smem[g], a.u + r0 + p.g_start[g],
                       (uint32_t)(p.g_elems[g] * (int)sizeof(XT)), &full[st]);
            ++it;  // lane 0 counts issued tiles only: the drain waits for these
          }
        }
        if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) break;
      }
    }
    if (lane == 0) {
      // the last fill of each stage must have landed before this CTA exits:
      // wait for the last ns issued tiles (a tile given up on was not issued;
      // counting it would wait on its stage's stale phase and miss the copy
      // of that stage's previous tile)
      const int first = it > ns ? it - ns : 0;
      for (int q = first; q < it; ++q)
        if (!mbar_wait(&full[q % ns], (uint32_t)(q / ns) & 1u)) abort_flag = 1;
      if (abort_flag) *err = 1.0;
    }
    return;
  }

  const int c = warp - 1;
  constexpr int kGroups = TmaShape<XT>::kGroups, kCons = TmaShape<XT>::kConsumers;
  const int grp = c / kCons, cw = c % kCons;
  const int spt = p.rows / kSlice;  // slices per tile
  using F = StepForm<FAM, INIT>;
  // First the slices outside the plan (pattern changes, windows leaving
  // [0, n)): direct loads, round-robin over all consumer warps, while the
  // producer's first copies are in flight.  Their rows are disjoint from the
  // tiles' rows, so the order changes no result.
  for (int64_t q = (int64_t)blockIdx.x * tma_warps<XT>() + c; q < ngen;
       q += (int64_t)gridDim.x * tma_warps<XT>())
    step_slice<VT, XT, FAM, INIT, WR, ZOWN>(a, gen[q], lane);
  // group g takes this CTA's tiles g, g + kGroups, ...  The stage of tile it
  // last held tile it - nstages; nstages is a multiple of kGroups, so that
  // tile belongs to this group and was consumed before this wait, and the
  // parity wait cannot pass on a stale phase (copies may land out of order).
  for (int it = grp;; it += kGroups) {
    const int j = blockIdx.x + it * (int)gridDim.x;
    if (j >= ntiles) break;
    const int st = it % ns;
    const uint32_t ph = (uint32_t)(it / ns) & 1u;
    if (abort_flag || !mbar_wait(&full[st], ph)) {
      abort_flag = 1;
      break;
    }
    const unsigned char* base = stages + (size_t)st * p.stage_bytes;
    const XT* sv = reinterpret_cast<const XT*>(base + p.vals_bytes);
    const XT* sw = sv + TmaShape<XT>::kVecSlots * p.rows;
    const int64_t r0 = stage_r0[st];
    if constexpr (is_op(FAM)) {
      // stored-operator step: vector terms, then the row's products; with W
      // fixed a lane takes two rows (slices cs and cs + kCons) interleaved, and
      // the row's own u entry is the centre product's operand
      constexpr int kSign = F::kSign;
      constexpr bool c0 = reads_slot0<FAM, INIT>(), c1 = reads_slot1<FAM, ZOWN>();
      constexpr int kStep = W > 0 ? 2 * kCons : kCons;
      for (int cs = cw; cs < spt; cs += kStep) {
        const int cs2 = cs + kCons;
        const bool two = W > 0 && cs2 < spt;
        const int r1 = cs * kSlice + lane, r2 = (two ? cs2 : cs) * kSlice + lane;
        const VT* v1 = reinterpret_cast<const VT*>(base) + (size_t)cs * p.w * kSlice + lane;
        const VT* v2 =
            reinterpret_cast<const VT*>(base) + (size_t)(two ? cs2 : cs) * p.w * kSlice + lane;
        XT acc1 = op_init<VT, XT, FAM, INIT, WR, ZOWN>(a, c0 ? sv[r1] : XT(0),
                                                       c1 ? sv[p.rows + r1] : XT(0));
        XT uc1 = XT(0), uc2 = XT(0);
        if constexpr (W > 0) {
          XT acc2 = op_init<VT, XT, FAM, INIT, WR, ZOWN>(a, c0 ? sv[r2] : XT(0),
                                                         c1 ? sv[p.rows + r2] : XT(0));
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const XT a1 = widen<XT>(v1[k * kSlice]), a2 = widen<XT>(v2[k * kSlice]);
            const XT u1 = sw[p.d[k] + r1], u2 = sw[p.d[k] + r2];
            if (k == W / 2) {
              uc1 = u1;
              uc2 = u2;
            }
            acc1 = fma(kSign > 0 ? a1 : -a1, u1, acc1);
            acc2 = fma(kSign > 0 ? a2 : -a2, u2, acc2);
          }
          op_finish<VT, XT, FAM, WR>(a, r0 + r1, acc1, uc1);
          if (two) op_finish<VT, XT, FAM, WR>(a, r0 + r2, acc2, uc2);
        } else {
#pragma unroll
          for (int k = 0; k < kTmaMaxW; ++k) {
            if (k < p.w) {
              const XT av = widen<XT>(v1[k * kSlice]);
              acc1 = fma(kSign > 0 ? av : -av, sw[p.d[k] + r1], acc1);
            }
          }
          if (FAM == FAM_OPT && WR) uc1 = sw[p.d0 + r1];
          op_finish<VT, XT, FAM, WR>(a, r0 + r1, acc1, uc1);
        }
      }
    } else if constexpr (W > 0 && std::is_same<XT, double>::value) {
      // FP64 rows of fixed width: a lane evaluates two rows of the tile,
      // slices cs and cs + kCons, with their multiply-add chains interleaved
      // (a slot past the tile repeats slice cs and is not stored); each row's
      // operations and their order are those of k_step
      for (int cs = cw; cs < spt; cs += 2 * kCons) {
        const int cs2 = cs + kCons;
        const bool two = cs2 < spt;
        const int r1 = cs * kSlice + lane, r2 = (two ? cs2 : cs) * kSlice + lane;
        const VT* v1 = reinterpret_cast<const VT*>(base) + (size_t)cs * p.w * kSlice + lane;
        const VT* v2 =
            reinterpret_cast<const VT*>(base) + (size_t)(two ? cs2 : cs) * p.w * kSlice + lane;
        const XT rin1 = sv[r1], rin2 = sv[r2];
        const XT xin1 = FAM == FAM_RES ? XT(0) : sv[p.rows + r1];
        const XT xin2 = FAM == FAM_RES ? XT(0) : sv[p.rows + r2];
        XT di1 = XT(0), di2 = XT(0);
        if constexpr (step_needs_dinv<FAM>()) {  // formed at set-up, never written here
          di1 = __ldg(a.dinv + r0 + r1);
          di2 = __ldg(a.dinv + r0 + r2);
        }
        const XT zo1 = ZOWN ? sw[p.d0 + r1] : XT(0), zo2 = ZOWN ? sw[p.d0 + r2] : XT(0);
        XT acc1 = step_init<FAM, F::kResidual>(rin1, di1);
        XT acc2 = step_init<FAM, F::kResidual>(rin2, di2);
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const XT a1 = widen<XT>(v1[k * kSlice]), a2 = widen<XT>(v2[k * kSlice]);
          const XT u1 = (ZOWN && k == W / 2) ? zo1 : sw[p.d[k] + r1];
          const XT u2 = (ZOWN && k == W / 2) ? zo2 : sw[p.d[k] + r2];
          acc1 = fma(F::kSign > 0 ? a1 : -a1, u1, acc1);
          acc2 = fma(F::kSign > 0 ? a2 : -a2, u2, acc2);
        }
        step_finish<VT, XT, FAM, INIT, WR, ZOWN>(a, r0 + r1, acc1, rin1, xin1, di1, zo1);
        if (two) step_finish<VT, XT, FAM, INIT, WR, ZOWN>(a, r0 + r2, acc2, rin2, xin2, di2, zo2);
      }
    } else {
      for (int cs = cw; cs < spt; cs += kCons) {
        const int it_row = cs * kSlice + lane;  // row inside the tile
        const VT* svals = reinterpret_cast<const VT*>(base) + (size_t)cs * p.w * kSlice + lane;
        const XT rin = sv[it_row];
        const XT xin = FAM == FAM_RES ? XT(0) : sv[p.rows + it_row];
        XT di = XT(0);
        if constexpr (step_needs_dinv<FAM>()) {
          if constexpr (TmaShape<XT>::kVecSlots == 3) di = sv[2 * p.rows + it_row];
          else di = __ldg(a.dinv + r0 + it_row);  // formed at set-up, never written here
        }
        const XT zo = ZOWN ? sw[p.d0 + it_row] : XT(0);
        XT acc = step_init<FAM, F::kResidual>(rin, di);
        if constexpr (W > 0) {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const XT av = widen<XT>(svals[k * kSlice]);
            const XT uk = (ZOWN && k == W / 2) ? zo : sw[p.d[k] + it_row];
            acc = fma(F::kSign > 0 ? av : -av, uk, acc);
          }
        } else {
#pragma unroll
          for (int k = 0; k < kTmaMaxW; ++k) {
            if (k < p.w) {
              const XT av = widen<XT>(svals[k * kSlice]);
              acc = fma(F::kSign > 0 ? av : -av, sw[p.d[k] + it_row], acc);
            }
          }
        }
        step_finish<VT, XT, FAM, INIT, WR, ZOWN>(a, r0 + it_row, acc, rin, xin, di, zo);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
  if (abort_flag && lane == 0) *err = 1.0;
}

template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN, int W>
void launch_inst(const StepArgs<VT, XT>& a, const TmaPlan& p, const TmaTile* tiles, int ntiles,
                 int grid, double* err, cudaStream_t s) {
  const int smem = kBarrierBytes + p.nstages * p.stage_bytes;
  k_step_tma<VT, XT, FAM, INIT, WR, ZOWN, W><<<grid, (tma_warps<XT>() + 1) * 32, smem, s>>>(
      a, p, tiles, ntiles, a.slices, a.slices ? a.nlist : 0, err);
  count_launch();
}

template <class VT, class XT, int FAM, bool INIT, int W>
void launch_wr(const StepArgs<VT, XT>& a, const TmaPlan& p, const TmaTile* tiles, int ntiles,
               int grid, double* err, cudaStream_t s) {
  const bool z = a.zown != nullptr;
  if (a.write_r) {
    if (z) launch_inst<VT, XT, FAM, INIT, true, true, W>(a, p, tiles, ntiles, grid, err, s);
    else launch_inst<VT, XT, FAM, INIT, true, false, W>(a, p, tiles, ntiles, grid, err, s);
  } else {
    if (z) launch_inst<VT, XT, FAM, INIT, false, true, W>(a, p, tiles, ntiles, grid, err, s);
    else launch_inst<VT, XT, FAM, INIT, false, false, W>(a, p, tiles, ntiles, grid, err, s);
  }
}

// stored-operator steps (FP64 levels): the flags from the arguments
template <class VT, class XT, int W>
void launch_op(const StepArgs<VT, XT>& a, const TmaPlan& p, const TmaTile* tiles, int ntiles,
               int grid, double* err, cudaStream_t s) {
  if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
    const bool s0 = a.rin != nullptr, s1 = a.xin != nullptr, wr = a.write_r;
    if (a.fam == FAM_OPT) {
      if (wr) launch_inst<VT, XT, FAM_OPT, true, true, false, W>(a, p, tiles, ntiles, grid, err, s);
      else launch_inst<VT, XT, FAM_OPT, true, false, false, W>(a, p, tiles, ntiles, grid, err, s);
    } else if (!s0) {
      launch_inst<VT, XT, FAM_OP, false, false, false, W>(a, p, tiles, ntiles, grid, err, s);
    } else if (!s1) {
      if (wr) launch_inst<VT, XT, FAM_OP, true, true, false, W>(a, p, tiles, ntiles, grid, err, s);
      else launch_inst<VT, XT, FAM_OP, true, false, false, W>(a, p, tiles, ntiles, grid, err, s);
    } else {
      if (wr) launch_inst<VT, XT, FAM_OP, true, true, true, W>(a, p, tiles, ntiles, grid, err, s);
      else launch_inst<VT, XT, FAM_OP, true, false, true, W>(a, p, tiles, ntiles, grid, err, s);
    }
  }
}

template <class VT, class XT, int FAM, bool INIT, bool WR, bool ZOWN, int W>
void set_smem_attr(int bytes) {
  cudaFuncSetAttribute(k_step_tma<VT, XT, FAM, INIT, WR, ZOWN, W>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <class VT, class XT, int FAM, bool INIT, int W>
void configure_wr(int bytes) {
  set_smem_attr<VT, XT, FAM, INIT, true, true, W>(bytes);
  set_smem_attr<VT, XT, FAM, INIT, true, false, W>(bytes);
  set_smem_attr<VT, XT, FAM, INIT, false, true, W>(bytes);
  set_smem_attr<VT, XT, FAM, INIT, false, false, W>(bytes);
}

template <class VT, class XT, int W>
void configure_all(int bytes) {
  configure_wr<VT, XT, FAM_CHEB4, true, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB4, false, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB1, true, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB1, false, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB4S, false, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB4SR, true, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB4SR, false, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB1S, false, W>(bytes);
  configure_wr<VT, XT, FAM_CHEB1SR, true, W>(bytes);
  set_smem_attr<VT, XT, FAM_JAC, true, false, false, W>(bytes);
  set_smem_attr<VT, XT, FAM_RES, true, false, false, W>(bytes);
  if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value) {
    set_smem_attr<VT, XT, FAM_OPT, true, true, false, W>(bytes);
    set_smem_attr<VT, XT, FAM_OPT, true, false, false, W>(bytes);
    set_smem_attr<VT, XT, FAM_OP, false, false, false, W>(bytes);
    set_smem_attr<VT, XT, FAM_OP, true, true, false, W>(bytes);
    set_smem_attr<VT, XT, FAM_OP, true, false, false, W>(bytes);
    set_smem_attr<VT, XT, FAM_OP, true, true, true, W>(bytes);
    set_smem_attr<VT, XT, FAM_OP, true, false, true, W>(bytes);
  }
}

// the family / INIT dispatch for one width variant
template <class VT, class XT, int W>
void launch_fam(const StepArgs<VT, XT>& a, const TmaPlan& p, const TmaTile* tiles, int ntiles,
                int grid, double* err, cudaStream_t s) {
  if (is_op(a.fam)) {
    launch_op<VT, XT, W>(a, p, tiles, ntiles, grid, err, s);
    return;
  }
  switch (a.fam) {
    case FAM_CHEB4:
      if (a.init) launch_wr<VT, XT, FAM_CHEB4, true, W>(a, p, tiles, ntiles, grid, err, s);
      else launch_wr<VT, XT, FAM_CHEB4, false, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    case FAM_CHEB4S:
      launch_wr<VT, XT, FAM_CHEB4S, false, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    case FAM_CHEB4SR:
      if (a.init) launch_wr<VT, XT, FAM_CHEB4SR, true, W>(a, p, tiles, ntiles, grid, err, s);
      else launch_wr<VT, XT, FAM_CHEB4SR, false, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    case FAM_CHEB1S:
      launch_wr<VT, XT, FAM_CHEB1S, false, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    case FAM_CHEB1SR:
      launch_wr<VT, XT, FAM_CHEB1SR, true, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    case FAM_CHEB1:
      if (a.init) launch_wr<VT, XT, FAM_CHEB1, true, W>(a, p, tiles, ntiles, grid, err, s);
      else launch_wr<VT, XT, FAM_CHEB1, false, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    case FAM_RES:
      launch_inst<VT, XT, FAM_RES, true, false, false, W>(a, p, tiles, ntiles, grid, err, s);
      break;
    default:
      launch_inst<VT, XT, FAM_JAC, true, false, false, W>(a, p, tiles, ntiles, grid, err, s);
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

void tma_configure() {
  configure_all<double, double, 0>(TmaShape<double>::kSmemBudget + kBarrierBytes);
  configure_all<double, double, 7>(TmaShape<double>::kSmemBudget + kBarrierBytes);
  configure_all<float, float, 0>(TmaShape<float>::kSmemBudget + kBarrierBytes);
  configure_all<__nv_bfloat16, float, 0>(TmaShape<float>::kSmemBudget + kBarrierBytes);
}

template <class VT, class XT>
bool launch_step_tma(const StepArgs<VT, XT>& a, const TmaPlan& p, const TmaTile* tiles,
                     int ntiles, int grid, double* err, cudaStream_t s) {
  if (ntiles <= 0 || p.nstages < 2 || p.nstages % TmaShape<XT>::kGroups != 0) return false;
  if (!aligned16(a.A.val) || !aligned16(a.u) || !aligned16(a.rin)) return false;
  if (a.fam != FAM_RES && (!aligned16(a.xin) || !aligned16(a.dinv))) return false;
  if (a.zown && a.zown != a.u) return false;  // z_j at the row is read from u's window
  if (is_op(a.fam) && !(std::is_same<VT, double>::value && std::is_same<XT, double>::value))
    return false;  // stored-operator steps exist for FP64 levels only
  // FP64 rows of the 7-point pattern: the fixed-width variant (its centre
  // entry, index 3, is the row itself)
  if constexpr (std::is_same<XT, double>::value) {
    if (p.w == 7 && p.d[3] == p.d0) {
      launch_fam<VT, XT, 7>(a, p, tiles, ntiles, grid, err, s);
      return true;
    }
  }
  launch_fam<VT, XT, 0>(a, p, tiles, ntiles, grid, err, s);
  return true;
}

template bool launch_step_tma<double, double>(const StepArgs<double, double>&, const TmaPlan&,
                                              const TmaTile*, int, int, double*, cudaStream_t);
template bool launch_step_tma<float, float>(const StepArgs<float, float>&, const TmaPlan&,
                                            const TmaTile*, int, int, double*, cudaStream_t);
template bool launch_step_tma<__nv_bfloat16, float>(const StepArgs<__nv_bfloat16, float>&,
                                                    const TmaPlan&, const TmaTile*, int, int,
                                                    double*, cudaStream_t);

}  // namespace amgps
