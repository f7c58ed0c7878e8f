// Internal declarations shared by the libamgps translation units.
//
// Device matrix layout (every level): sliced ELLPACK with slices of 32
// consecutive rows (SELL-32, no row sorting).  Entry k of row (32 s + lane) is
// stored at val[vbase(s) + 32 k + lane], so a warp that owns a slice reads each
// k-column of the slice as one coalesced 256-byte (FP64) line.  A slice is
//   * "uniform" when all its rows fit one shared list of column offsets
//     (col = row + off[k]); then no per-entry column index is stored and
//     entries absent from a row hold 0 (their clamped column is a valid
//     address).  Every level of a 7-point operator with geometric
//     aggregation is uniform, so the index stream disappears; so are the
//     wide coarse levels of smoothed aggregation (patterns up to 1024
//     offsets).
//   * "explicit" otherwise: col[vbase + 32 k + lane] as in plain SELL.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "amgps.h"

namespace amgps {

constexpr int kSlice = 32;          // rows per slice (one warp)
constexpr int kBlock = 256;         // threads per block of the row kernels
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kMaxDegree = 16;

struct SliceDesc {
  int64_t vbase;  // index of entry (k=0, lane=0) of the slice in val[] / col[]
  int32_t w;      // stored entries per row
  int32_t cref;   // >= 0: uniform slice, offsets at off[cref .. cref+w); < 0: explicit
};
static_assert(sizeof(SliceDesc) == 16, "slice descriptor is one 16-byte load");

template <class VT>
struct DevMat {
  int64_t n = 0;
  int64_t nslices = 0;
  const SliceDesc* sd = nullptr;
  const VT* val = nullptr;
  const int32_t* col = nullptr;  // null when every slice is uniform
  const int32_t* off = nullptr;
};

// FAM_RES is not a smoother: it writes the true residual b - A x (rin = b,
// u = x, result in zout) for the restriction of Eq. amg.
// FAM_CHEB4S / FAM_CHEB4SR are the 4th-kind step on FP64 levels in the
// row-scaled form: A holds a_ij / M_i and the recurrence residual is kept as
// M^{-1} r, so a row needs no 1/M product; in FAM_CHEB4SR rin is still
// unscaled (b: the first step after the initial one, or an initial step) and
// the accumulation starts from (1/M) rin.
// FAM_CHEB1S / FAM_CHEB1SR do the same for the 1st-kind steps, keeping the
// residual as rho M^{-1} r (the 1/rho goes into the coefficient of r).
// FAM_OP / FAM_OPT are the steps of the stored-operator form of a polynomial
// smoother on FP64 levels (the same polynomial evaluated backwards, Clenshaw's
// scheme, with each step's operator tau I - sigma M^{-1} A stored in A's
// layout; api.cu derives the coefficients):
//   FAM_OP:  out = [q | c2 s] + [c1 p] + sum_k m_ik u_k   (A = the step's operator)
//            rin = the slot-0 vector (q or s): read when INIT, added with
//            coefficient 1 when WR, else times c2; xin = the slot-1 vector p,
//            read (times c1) when ZOWN.
//   FAM_OPT: out = q - sum_k (a_ik / M_i) u_k              (A = the row-scaled values)
//            rin = q; when WR also rout = u_row + beta out.
enum Family { FAM_CHEB4 = 0, FAM_CHEB1 = 1, FAM_JAC = 2, FAM_RES = 3, FAM_CHEB4S = 4,
              FAM_CHEB4SR = 5, FAM_CHEB1S = 6, FAM_CHEB1SR = 7, FAM_OP = 8, FAM_OPT = 9 };
__host__ __device__ constexpr bool is_cheb4(int fam) {
  return fam == FAM_CHEB4 || fam == FAM_CHEB4S || fam == FAM_CHEB4SR;
}
__host__ __device__ constexpr bool is_op(int fam) { return fam == FAM_OP || fam == FAM_OPT; }
// per-row vectors of a step: slot 0 (rin) and slot 1 (xin)
template <int FAM, bool INIT>
__host__ __device__ constexpr bool reads_slot0() {
  return !is_op(FAM) || FAM == FAM_OPT || INIT;
}
template <int FAM, bool ZOWN>
__host__ __device__ constexpr bool reads_slot1() {
  return is_op(FAM) ? (FAM == FAM_OP && ZOWN) : FAM != FAM_RES;
}

// Arguments of one fused smoother step (see kernels_smooth.cu).
template <class VT, class XT>
struct StepArgs {
  DevMat<VT> A;
  const XT* u = nullptr;     // vector multiplied by A (gathered)
  const XT* rin = nullptr;   // r_{j-1}, or b on the initial / Jacobi step
  XT* rout = nullptr;        // r_j (may equal rin); unused when not written
  const XT* zown = nullptr;  // z_j at the row itself; null: no c1 term
  XT* zout = nullptr;        // z_{j+1}
  const XT* xin = nullptr;
  XT* xout = nullptr;        // may equal xin unless u == xin
  const XT* dinv = nullptr;  // 1 / M_i (Eq. l1smooth)
  XT c1 = 0, c2 = 0, beta = 0, rhoinv = 1;
  int fam = FAM_CHEB4;
  bool init = false;
  bool write_r = false;
  const int32_t* slices = nullptr;  // optional list of slices to process (null: all)
  int64_t nlist = 0;                // entries in `slices`
  int split = 1;  // > 1: one block of `split` warps per slice, entries split among them
  // host hint for the scaled form: rin is still unscaled (b)
  bool rin_raw = false;
};

// Most warps per slice in the split form of the step and transfer kernels
// (levels with wide rows; the factor per level is chosen at load).
constexpr int kMaxSplit = 32;

// ---- TMA-fed step (kernels_tma.cu) ----
// A tile is `rows` consecutive rows (whole 32-row slices) of one uniform
// pattern.  For each tile the producer warp copies into shared memory, with
// cp.async.bulk: the tile's values, its rows of r_in, x_in and 1/M, and for
// each group of nearby column offsets the contiguous window of the multiplied
// vector that the group reads.  Consumer warps then work from shared memory
// only; a group's warps split each tile's slices between them.  Fewer, larger
// copies keep the TMA unit streaming.  The launch shape depends on the vector
// type:
//   FP64: 512-row tiles (16 slices), one CTA per SM of 1 producer warp and two
//     groups of 8 consumer warps taking alternate tiles (544 threads; a lane
//     evaluates two rows of a 7-point tile, slices cw and cw + 8), with up
//     to 225 KB of stages -- four in flight, so a tile's copies are issued
//     three tiles ahead of the FP64-bound consumers;
//   FP32/BF16: 1024-row tiles (32 slices), two CTAs per SM, each 1 producer
//     warp and one group of 16 consumer warps, up to 112.5 KB of stages.
// kVecSlots: the tile's own rows copied into a stage -- r_in, x_in and, for
// FP32 vectors, 1/M (FP64 consumers read 1/M from global memory in the few
// steps that need it, which keeps a 512-wide grid's stage four deep).
template <class XT>
struct TmaShape {  // FP32 vectors (FP32 and BF16 levels)
  static constexpr int kRows = 1024, kGroups = 1, kConsumers = 16, kCtasPerSm = 2;
  static constexpr int kSmemBudget = 115200;
  static constexpr int kVecSlots = 3;
};
template <>
struct TmaShape<double> {
  static constexpr int kRows = 512, kGroups = 2, kConsumers = 8, kCtasPerSm = 1;
  static constexpr int kSmemBudget = 230400;
  static constexpr int kVecSlots = 2;
};
// the same figures by vector size, for the host-side planner
inline int tma_rows(size_t xsize) {
  return xsize == 8 ? TmaShape<double>::kRows : TmaShape<float>::kRows;
}
inline int tma_ctas_per_sm(size_t xsize) {
  return xsize == 8 ? TmaShape<double>::kCtasPerSm : TmaShape<float>::kCtasPerSm;
}
inline int tma_smem_budget(size_t xsize) {
  return xsize == 8 ? TmaShape<double>::kSmemBudget : TmaShape<float>::kSmemBudget;
}
inline int tma_vec_slots(size_t xsize) {
  return xsize == 8 ? TmaShape<double>::kVecSlots : TmaShape<float>::kVecSlots;
}
// Two offset groups share one window when the merged window holds at most
// this many elements more than the two separate ones (the +-nx offsets of a
// 513..577-wide grid against 512-row tiles).
constexpr int kTmaMergeSlack = 64;
// The stage count of a plan is a multiple of the group count: then the
// previous fill of the stage a group waits on is a tile of the same group,
// already consumed, so the parity wait cannot pass on a stale phase.  (With
// two groups and an odd count, a group could reach a stage whose previous
// tile -- the other group's -- had not landed yet.)
inline int tma_groups(size_t xsize) {
  return xsize == 8 ? TmaShape<double>::kGroups : TmaShape<float>::kGroups;
}
constexpr int kTmaMaxW = 8;
constexpr int kTmaMaxGroups = 4;
constexpr int kTmaMaxStages = 8;

struct TmaTile {
  int64_t r0;     // first row of the tile
  int64_t vbase;  // val[] index of the tile's first entry
};

struct TmaPlan {
  int rows = 0;                     // rows per tile
  int w = 0, ngroups = 0;
  int g_start[kTmaMaxGroups] = {};  // window start, elements relative to the tile's first row
  int g_elems[kTmaMaxGroups] = {};  // elements copied (multiple of 16 bytes)
  int g_smem[kTmaMaxGroups] = {};   // element offset of the window in the stage's window area
  int d[kTmaMaxW] = {};             // window-area index of row (tile start + offset_k)
  int d0 = 0;                       // same for offset 0 (the row itself)
  int vals_bytes = 0, vec_bytes = 0, win_bytes = 0, stage_bytes = 0, nstages = 0;
};

// ---- launchers (kernels_smooth.cu) ----
template <class VT, class XT>
void launch_step(const StepArgs<VT, XT>& a, cudaStream_t s);
// Returns false (nothing launched) when the kernel cannot take these arguments
// (a pointer not 16-byte aligned); the caller then uses launch_step.
template <class VT, class XT>
bool launch_step_tma(const StepArgs<VT, XT>& a, const TmaPlan& p, const TmaTile* tiles,
                     int ntiles, int grid, double* err_slot, cudaStream_t s);
template <class XT>
void launch_first(int fam, int64_t n, const XT* b, const XT* dinv, XT* rout, XT* zout, XT* xout,
                  XT c2, XT beta, XT rhoinv, cudaStream_t s);
// b_c[I] = sum of res over the children of coarse row I (children lists)
template <class XT>
void launch_aggregate(const int32_t* cptr, const int32_t* cidx, int64_t nc, const XT* res, XT* bc,
                      cudaStream_t s);
template <class XT>
void launch_prolong(int64_t n, const int32_t* agg, const XT* ec, XT* x, cudaStream_t s);
// general prolongator transfers: y = M u (add = 0) or y += M u (add = 1);
// split > 1: one block of `split` warps per slice
template <class XT>
void launch_xfer(const DevMat<double>& M, const XT* u, XT* y, int add, int split, cudaStream_t s);
// out = x + y ; out = x - y ; out = (factor / *s_dev) * x
template <class XT>
void launch_add(int64_t n, const XT* x, const XT* y, XT* out, cudaStream_t s);
void launch_sub(int64_t n, const double* x, const double* y, double* out, cudaStream_t s);
void launch_scale_dev(int64_t n, const double* x, double* out, const double* s_dev, double factor,
                      cudaStream_t s);

// ---- persistent kernel for the coarse levels of a V-cycle (kernels_cycle.cu) ----
// The levels below the TMA-fed ones are launch-latency-bound: their kernels
// last a few microseconds each.  The host records the kernel sequence of
// those levels once (the same calls, same arguments, same order) as a list of
// phases, and one co-resident grid runs the phases with a grid-wide barrier
// between consecutive ones.
enum CycleOp { CY_STEP = 0, CY_FIRST = 1, CY_AGG = 2, CY_PROLONG = 3, CY_GEMV = 4, CY_COPY = 5 };

template <class VT, class XT>
struct CyclePhase {
  int op = CY_STEP;
  int fam = FAM_CHEB4;   // CY_FIRST: FAM_CHEB4, FAM_CHEB1 or FAM_JAC
  int64_t n = 0;         // rows (CY_AGG: coarse rows)
  StepArgs<VT, XT> a;    // CY_STEP (direct form, every slice of the level)
  const int32_t* i0 = nullptr;  // CY_AGG: cptr; CY_PROLONG: agg
  const int32_t* i1 = nullptr;  // CY_AGG: cidx
  // CY_FIRST: b; CY_AGG: res; CY_PROLONG: e_c; CY_GEMV: b; CY_COPY: src
  const XT* in0 = nullptr;
  const XT* in1 = nullptr;      // CY_FIRST: 1/M
  XT* out0 = nullptr;           // CY_FIRST: r; CY_AGG: b_c; CY_PROLONG, CY_GEMV: x; CY_COPY: dst
  XT* out1 = nullptr;           // CY_FIRST: z
  XT* out2 = nullptr;           // CY_FIRST: x
  const double* ainv = nullptr;  // CY_GEMV
  XT c2 = 0, beta = 0, rhoinv = 1;
};

// grid-barrier word: arrivals, zeroed before each launch
struct CycleSync {
  unsigned* count = nullptr;
};
// Operator values of a stored-operator step: out = tau I - sigma B over B's
// layout (B = a level's row-scaled values), in FP64.
void launch_build_op(const DevMat<double>& B, double tau, double sigma, double* out,
                     cudaStream_t s);

// the persistent kernel takes levels of at most this many rows (larger ones
// keep their launches, whose grids hold more warps in flight)
constexpr int64_t kCycleMaxRows = 65536;

// Blocks of the persistent launch: all co-resident (occupancy x SMs, at most
// kCycleMaxBlocksPerSm per SM); 0 when the kernel cannot run.
template <class VT, class XT>
int cycle_grid(int nsm);
// Launches the phases (a cooperative launch: the driver refuses it if the grid
// cannot be co-resident).  Returns the launch's error code.
template <class VT, class XT>
cudaError_t launch_cycle(const CyclePhase<VT, XT>* phases, int nph, const CycleSync& sync, int grid,
                         double* err, cudaStream_t s);

// ---- weight-predicting MLP (kernels_mlp.cu) ----
constexpr int kMlpParams = 4996;
constexpr int kMlpActs = 132;
void mlp_forward(const float* th, const float* F, int batch, const float* ref, float* beta,
                 float* acts, cudaStream_t s);
void mlp_backward(const float* th, const float* F, const float* acts, const float* beta,
                  int batch, const float* gbeta, float* work, float* grads, cudaStream_t s);
void mlp_adam(float* th, const float* g, float* m, float* v, int step, float lr, float b1,
              float b2, float eps, cudaStream_t s);
template <class VT, class XT>
void launch_l1diag(const DevMat<VT>& A, XT* dinv, cudaStream_t s);
template <class A, class B>
void launch_convert(int64_t n, const A* in, B* out, cudaStream_t s);

void tma_configure();

// Kernels enqueued through the launchers above (graph captures included; the
// host driver corrects for captures and adds graph replays).
int64_t launches_enqueued();
void count_launch();

}  // namespace amgps

#include "krylov.h"
