// Scalar slots, reduction workspace and launchers of the outer Krylov solver,
// the coarsest-level solve and the power iteration (kernels_krylov.cu), kept
// apart from the smoother-step declarations.  Included at the end of
// amgps_internal.h (uses DevMat).
#pragma once

namespace amgps {

// Device scalar slots of the Krylov solver.
enum Scalar {
  S_PQ = 0, S_RR = 1, S_RZ = 2, S_RZOLD = 3, S_ALPHA = 4, S_BB = 5, S_NRM = 6, S_BETA = 7,
  S_ERR = 8,  // set non-zero by a kernel whose bounded wait gave up
  S_RZP = 9,  // r . z_old (flexible CG)
  S_GAMMA = 10,  // z . q_old (one-reduction flexible CG)
  S_DELTA = 11,  // z . A z (one-reduction flexible CG)
  S_COUNT = 16
};

struct RedWork {
  double* part = nullptr;       // per-block partial sums [grid] (3 x grid for grid_sum3)
  unsigned* counter = nullptr;  // arrival counter (reset by the last block)
  int grid = 0;
};

// ---- launchers (kernels_krylov.cu) ----
void launch_spmv_dot(const DevMat<double>& A, const double* p, double* q, const RedWork& w,
                     double* scal, cudaStream_t s);
// one-reduction flexible CG: w = A z with z.r, z.q, z.w in one reduction
// (first = 1: no q yet), then p = z - beta p, q = w - beta q, x += alpha p,
// r -= alpha q, r.r
void launch_spmv_dot3(const DevMat<double>& A, const double* z, double* w, const double* r,
                      const double* q, int first, const RedWork& rw, double* scal,
                      cudaStream_t s);
void launch_fcg_update(int64_t n, const double* z, const double* w, double* p, double* q,
                       double* x, double* r, int first, const RedWork& rw, double* scal,
                       cudaStream_t s);
// standard PCG with the x update deferred: r -= alpha q and r.r (with cout:
// also cout = dinv .* r); later x += alpha p together with p = z + beta p
// (with_p = 0: x only)
void launch_r_update(int64_t n, const double* q, double* r, const RedWork& w, double* scal,
                     cudaStream_t s, const double* dinv = nullptr, double* cout = nullptr);
void launch_xpay_x(int64_t n, const double* z, double* p, double* x, const double* scal,
                   int with_p, cudaStream_t s);
// rz_mode 0: scal[out_slot] = a.b.  1: scal[S_RZOLD] <- scal[S_RZ], scal[S_RZ] = a.b,
// scal[S_BETA] = S_RZ / S_RZOLD.  2: as 1 with the flexible (Polak-Ribiere)
// beta = (S_RZ - S_RZP) / S_RZOLD.
void launch_dot(int64_t n, const double* a, const double* b, const RedWork& w, double* scal,
                int out_slot, int rz_mode, cudaStream_t s);
template <class XT>
void launch_coarse_gemv(int nc, const double* ainv, const XT* b, XT* x, cudaStream_t s);
void launch_chol_inverse(int n, double* work, double* ainv, int* status, cudaStream_t s);
template <class VT, class XT>
void launch_power_step(const DevMat<VT>& A, const XT* v, const XT* dinv, XT* w, const RedWork& rw,
                       double* scal, cudaStream_t s);
template <class XT>
void launch_scale_by_norm(int64_t n, const XT* w, XT* v, const double* scal, int slot,
                          cudaStream_t s);
template <class XT>
void launch_norm2(int64_t n, const XT* v, const RedWork& rw, double* scal, int slot,
                  cudaStream_t s);

// Blocks of a grid-stride reduction over work_items: enough for the items,
// at most per_sm per SM (kRedBlocksPerSm for the streaming vector kernels,
// whose registers allow a full SM; 4 for the SpMV-class ones)
constexpr int kRedBlocksPerSm = 8;
int reduction_grid(int64_t work_items, int nsm, int per_sm = 4);

}  // namespace amgps
