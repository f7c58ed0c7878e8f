// libamgps host side: the C ABI of include/amgps.h.
//
// Responsibilities: input validation (no device fault is ever used to report
// bad input), uploading the SELL-32 layout planned in layout.cu, the
// transfer maps, the coarsest-level factorisation, and the host
// drivers that sequence the kernels of one smoother application (Sec. 2.1-2.2),
// one V-cycle (Eq. amg) and the outer PCG (Sec. 4).  The V-cycle below the
// finest level is captured once into a CUDA graph and replayed, since those
// levels are launch-bound; the finest level is launched eagerly so that its
// kernels can be timed with plain CUDA events.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "amgps_internal.h"
#include "amgps_tables.h"
#include "host_check.h"
#include "layout.h"
#include "setup.h"
#include "setup_host.h"

using namespace amgps;

namespace {

thread_local std::string g_err;
constexpr int kDotSlots = 32 * 32;  // 32 levels x (16 post + 16 pre) weight-gradient dots
constexpr int kMaxLossVectors = 4096;

struct Spec {
  int kind = AMGPS_CHEB4_OPT;
  int k = 4;
  double w[kMaxDegree] = {};
  double rho = 1.0;
};

// Step coefficients of one smoother application, computed in FP64 on the host.
struct Coefs {
  int fam = FAM_CHEB4;
  int k = 1;
  double c1[kMaxDegree + 1] = {}, c2[kMaxDegree + 1] = {}, beta[kMaxDegree + 1] = {};
  double rhoinv = 1.0;
};

Coefs make_coefs(int kind, int k, const double* w, double rho) {
  Coefs c;
  c.k = k;
  if (rho <= 0.0) rho = 1.0;
  if (kind == AMGPS_L1JACOBI) {
    c.fam = FAM_JAC;
    return c;
  }
  if (kind == AMGPS_CHEB1 || kind == AMGPS_CHEB1_OPT) {
    // Algorithm 1 with theta, delta of Eq. optimal_parameters on [a_k*, 1]
    c.fam = FAM_CHEB1;
    const double a = AMGPS_ASTAR[k - 1];
    const double theta = 0.5 * (1.0 + a), delta = 0.5 * (1.0 - a);
    const double sigma1 = theta / delta;
    double rho_prev = 1.0 / sigma1;
    c.c2[0] = 1.0 / theta;  // d^(0) = r^(0) / theta
    for (int j = 1; j < k; ++j) {
      const double rj = 1.0 / (2.0 * sigma1 - rho_prev);
      c.c1[j] = rj * rho_prev;
      c.c2[j] = 2.0 * rj / delta;
      rho_prev = rj;
    }
    c.rhoinv = (kind == AMGPS_CHEB1_OPT) ? 1.0 : 1.0 / rho;
    return c;
  }
  // Eq. polsmoother / polsmootheropt:
  //   z_j = (2j-3)/(2j+1) z_{j-1} + (8j-4)/(2j+1)/rho M^{-1} r_{j-1}
  c.fam = FAM_CHEB4;
  for (int j = 1; j <= k; ++j) {
    c.c1[j] = double(2 * j - 3) / double(2 * j + 1);
    c.c2[j] = double(8 * j - 4) / double(2 * j + 1) / rho;
    if (kind == AMGPS_CHEB4) c.beta[j] = 1.0;
    else if (kind == AMGPS_CHEB4_OPT) c.beta[j] = AMGPS_OPT4_BETA[k - 1][j - 1];
    else c.beta[j] = w[j - 1];
  }
  return c;
}

// ---- stored-operator form of the polynomial smoothers (FP64 levels) ----
// Both polynomial families and l1-Jacobi are, with s_j = M^{-1} r_j and
// B = M^{-1} A,
//   z_1 = c_1 s_0,  z_j = a_j z_{j-1} + c_j s_{j-1},  s_j = s_{j-1} - B z_j,
//   x = x_0 + sum_j beta_j z_j
// (4th kind, Eq. polsmoother / polsmootheropt: a_j = (2j-3)/(2j+1),
// c_j = (8j-4)/(2j+1)/rho; 1st kind, Algorithm 1: z_{j+1} = d^(j), c_1 =
// 1/(theta rho), a_{j+1} = rho_j rho_{j-1}, c_{j+1} = 2 rho_j/(delta rho),
// beta = 1; l1-Jacobi, Eq. l1smooth: a_j = 0, c_j = 1, beta = 1).
// Eliminating s gives the three-term recurrence
//   z_{j+1} = (al_j I - mu_j B) z_j - ga_j z_{j-1},
//   al_j = a_{j+1} + c_{j+1}/c_j,  mu_j = c_{j+1},  ga_j = c_{j+1} a_j / c_j,
// and Clenshaw's backward scheme evaluates the weighted sum with one product
// per step: u_{k+1} = u_{k+2} = 0,
//   u_j = beta_j s_0 + (al_j I - mu_j B) u_{j+1} - ga_{j+1} u_{j+2},
//   x = x_0 + c_1 u_1
// (the same polynomial in B applied to s_0, so the same result up to
// rounding).  Step q (q = 0 .. k-2) produces u_j, j = k-1-q, as
//   u_j = h s_0 + g u_{j+2} + (tau I - sigma B) u_{j+1}
// with u_k = beta_k s_0 folded in; the operator tau I - sigma B of each step
// is stored in A's layout, so a row costs one multiply-add per stored entry
// plus one per vector term: 7 to 9 FP64 operations on a 7-point row instead
// of the recurrence's 10, and two or three vector streams instead of five.
struct OpStep {
  double tau = 0, sigma = 0, h = 0, g = 0;
};

// The steps for the coefficients of one smoother application (k >= 2);
// returns k - 1.
int op_plan(const Coefs& cf, OpStep* st) {
  const int k = cf.k;
  double a[kMaxDegree + 2] = {}, cc[kMaxDegree + 2] = {}, be[kMaxDegree + 2] = {};
  for (int j = 1; j <= k; ++j) be[j] = 1.0;
  if (cf.fam == FAM_CHEB4) {
    for (int j = 1; j <= k; ++j) {
      a[j] = cf.c1[j];
      cc[j] = cf.c2[j];
      be[j] = cf.beta[j];
    }
  } else if (cf.fam == FAM_JAC) {  // x_j = x_{j-1} + M^{-1} r_{j-1}: z_j = s_{j-1}
    for (int j = 1; j <= k; ++j) cc[j] = 1.0;
  } else {
    cc[1] = cf.c2[0] * cf.rhoinv;
    for (int j = 1; j < k; ++j) {
      a[j + 1] = cf.c1[j];
      cc[j + 1] = cf.c2[j] * cf.rhoinv;
    }
  }
  double al[kMaxDegree + 2] = {}, mu[kMaxDegree + 2] = {}, ga[kMaxDegree + 2] = {};
  for (int j = 1; j < k; ++j) {
    al[j] = a[j + 1] + cc[j + 1] / cc[j];
    mu[j] = cc[j + 1];
    ga[j] = j >= 2 ? cc[j + 1] * a[j] / cc[j] : 0.0;  // z_0 = 0
  }
  for (int q = 0; q < k - 1; ++q) {
    const int j = k - 1 - q;
    OpStep o;
    if (j == k - 1) {  // u_{k-1} = beta_{k-1} s + (al I - mu B)(beta_k s): the product is of s
      o.tau = be[k - 1] + be[k] * al[k - 1];
      o.sigma = be[k] * mu[k - 1];
    } else if (j == k - 2) {  // the u_{j+2} = u_k = beta_k s term joins h
      o.tau = al[j];
      o.sigma = mu[j];
      o.h = be[j] - ga[j + 1] * be[k];
    } else {
      o.tau = al[j];
      o.sigma = mu[j];
      o.h = be[j];
      o.g = -ga[j + 1];
    }
    if (j == 1) {  // x = x_0 + c_1 u_1
      o.tau *= cc[1];
      o.sigma *= cc[1];
      o.h *= cc[1];
      o.g *= cc[1];
    }
    st[q] = o;
  }
  return k - 1;
}

bool same_coefs(const Coefs& x, const Coefs& y) {
  if (x.fam != y.fam || x.k != y.k || x.rhoinv != y.rhoinv) return false;
  for (int j = 0; j <= x.k; ++j)
    if (x.c1[j] != y.c1[j] || x.c2[j] != y.c2[j] || x.beta[j] != y.beta[j]) return false;
  return true;
}

struct Level {
  int64_t n = 0, nnz = 0, stored = 0, nslices = 0, explicit_entries = 0;
  SliceDesc* sd = nullptr;
  void* val = nullptr;
  int32_t* col = nullptr;
  int32_t* off = nullptr;
  // FP64 copy of A_0 for the outer solver when the smoother path is FP32/BF16
  SliceDesc* sd64 = nullptr;
  double* val64 = nullptr;
  int32_t* col64 = nullptr;
  int32_t* off64 = nullptr;
  int32_t* agg = nullptr;
  int32_t* cptr = nullptr;
  int32_t* cidx = nullptr;
  int64_t nc = 0;
  // general prolongator (not one unit entry per row): P (n x nc) and R = P^T
  // (nc x n), FP64 values, explicit SELL-32 slices
  bool xfer_general = false;
  DevMat<double> Pm, Rm;
  int64_t xfer_stored = 0;  // stored entries of P and R together
  int psplit = 1, rsplit = 1;
  int split = 1;  // warps per slice of the generic step kernel (wide rows)
  void* dinv = nullptr;   // 1 / M_i
  // FP64 and FP32 levels: the row-scaled values a_ij / M_i in the layout and
  // type of `val`, used by the polynomial steps (their residual is kept scaled)
  void* sval = nullptr;
  void *b = nullptr, *x = nullptr, *r = nullptr, *za = nullptr, *zb = nullptr, *xb = nullptr;
  double* ainv = nullptr;
  bool coarsest = false;
  Spec spec;
  // TMA-fed step: eligible tiles, the other slices, and the stage layout
  TmaPlan plan;
  TmaTile* tma_tiles = nullptr;
  int ntma = 0;
  int tma_grid = 0;
  int32_t* gen_slices = nullptr;
  int64_t ngen = 0;
  // reverse-mode buffers (allocated on the first backward call)
  void *bx2 = nullptr, *bgx = nullptr, *bgb = nullptr, *bt1 = nullptr, *bt2 = nullptr,
       *bt3 = nullptr;
  // stored-operator form: one operator per step (stored entries each), built
  // for the coefficients ops_cf; ops_ok when they match the level's spec
  std::vector<double*> ops;
  Coefs ops_cf;
  bool ops_ok = false;
};

}  // namespace

struct amgps_ctx {
  int device = 0;
  int nsm = 0;
  cudaStream_t ustream = nullptr, stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_sync = nullptr;
  std::string err;
  bool loaded = false;
  amgps_prec prec = AMGPS_F64;
  std::vector<Level> lv;
  std::vector<void*> allocs;
  double *pr = nullptr, *pp = nullptr, *pq = nullptr, *pz = nullptr, *pz2 = nullptr;
  double *stage_b = nullptr, *stage_x = nullptr;
  double* h_stage = nullptr;
  size_t h_stage_n = 0;
  double* dscal = nullptr;
  double* hscal = nullptr;
  double* ddots = nullptr;      // dots of the weight gradients: [level][post 0..15 | pre 16..31]
  double* dacc = nullptr;       // their sum over the error vectors of a loss evaluation
  double* dloss = nullptr;      // per error vector: <e0, A e0>, <e1, A e1>
  double* hdots = nullptr;
  bool bwd_ready = false;
  double* part = nullptr;
  unsigned* counters = nullptr;
  int red_grid = 0;
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  int64_t graph_kernels = 0;   // kernel nodes in gexec
  int use_tma = 1;             // AMGPS_OPT_TMA: TMA-fed step kernels 0 off, 1 auto, 2 always
  int flexible = 0;            // AMGPS_OPT_FLEXIBLE: 0 standard, 1 Polak-Ribiere, 2 one-reduction
  int coarse_sweeps = 0;       // AMGPS_OPT_COARSE_SWEEPS: 0 dense Cholesky, m l1-Jacobi sweeps
  int step_form = 1;           // AMGPS_OPT_STEP_FORM: 0 recurrence, 1 stored operators where built
  int64_t launch_adjust = 0;   // captured (not run) launches removed, replays added
  int64_t launch_base = 0;     // reset point of the launch counter
  bool prof = false;
  struct Pair {
    cudaEvent_t a, b;
    int cls;
    double bytes, flops, inst;
  };
  std::vector<Pair> pending;
  std::vector<cudaEvent_t> pool;
  int64_t prof_launches[5] = {};  // class 3 (kernel count) is kept apart
  void* noalloc = nullptr;        // device address of the allocation-free scratch array
  size_t alloc_limit = 0;         // AMGPS_OPT_ALLOC_LIMIT: hierarchy bytes allowed (0: no limit)
  size_t alloc_bytes = 0;         // hierarchy bytes allocated
  // persistent kernel for the coarse levels (option AMGPS_OPT_COARSE_KERNEL)
  int use_cycle = 0;
  bool tail_ok = false;
  int tail_level = -1;             // first level it runs
  int tail_nph = 0;                // recorded phases
  int tail_grid = 0;               // co-resident blocks
  void* tail_dev = nullptr;        // CyclePhase<VT, XT>[tail_cap] on the device
  size_t tail_cap = 0;             // bytes
  unsigned* tail_sync = nullptr;   // barrier word (arrivals)
  double prof_ms[5] = {};
  double prof_bytes[5] = {};
  double prof_flops[5] = {};
  double prof_inst[5] = {};
};

namespace {

template <class F>
amgps_status guard(amgps_ctx* c, F&& f) {
  try {
    f();
    if (c) c->err.clear();
    return AMGPS_OK;
  } catch (const Fail& e) {
    if (c) c->err = e.msg;
    else g_err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    else g_err = "host allocation failed";
    return AMGPS_E_NOMEM;
  } catch (...) {
    if (c) c->err = "unexpected C++ exception";
    else g_err = "unexpected C++ exception";
    return AMGPS_E_ARG;
  }
}

void* dalloc(amgps_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c->alloc_limit && c->alloc_bytes + bytes > c->alloc_limit)
    throw Fail{AMGPS_E_NOMEM, "allocation of " + std::to_string(bytes) + " bytes would pass the " +
                                  "context's limit of " + std::to_string(c->alloc_limit) +
                                  " bytes (AMGPS_OPT_ALLOC_LIMIT)"};
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{AMGPS_E_NOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) +
                                  " bytes failed: " + cudaGetErrorString(e)};
  }
  c->allocs.push_back(p);
  c->alloc_bytes += bytes;
  return p;
}

template <class T>
T* dupload(amgps_ctx* c, const T* h, size_t count) {
  T* d = (T*)dalloc(c, count * sizeof(T));
  if (count) CK(cudaMemcpy(d, h, count * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}

void free_hierarchy(amgps_ctx* c) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->graph_ok = false;
  c->tail_ok = false;
  if (!c->allocs.empty()) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->alloc_bytes = 0;
  c->lv.clear();
  c->loaded = false;
  c->bwd_ready = false;
  c->pr = c->pp = c->pq = c->pz = c->pz2 = c->stage_b = c->stage_x = nullptr;
}

void enter(amgps_ctx* c) {
  CK(cudaSetDevice(c->device));
  CK(cudaEventRecord(c->ev_in, c->ustream));
  CK(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
}

void leave(amgps_ctx* c) {
  CK(cudaEventRecord(c->ev_out, c->stream));
  CK(cudaStreamWaitEvent(c->ustream, c->ev_out, 0));
}

RedWork redwork(amgps_ctx* c, int slot, int64_t work, int per_sm = 4) {
  RedWork w;
  w.part = c->part;
  w.counter = c->counters + slot;
  w.grid = reduction_grid(work, c->nsm, per_sm);
  return w;
}

// ---- profiling: event pairs around selected launches, harvested on sync ----
cudaEvent_t take_event(amgps_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

void harvest(amgps_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    CK(cudaEventSynchronize(p.b));
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    c->prof_launches[p.cls] += 1;
    c->prof_ms[p.cls] += ms;
    c->prof_bytes[p.cls] += p.bytes;
    c->prof_flops[p.cls] += p.flops;
    c->prof_inst[p.cls] += p.inst;
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pending.clear();
}

struct ProfScope {
  amgps_ctx* c;
  bool on;
  cudaEvent_t a{}, b{};
  int cls;
  double bytes, flops, inst;
  // flops / inst: the launch's algorithmic FP64 flops and FP64 thread instructions
  ProfScope(amgps_ctx* c_, bool want, int cls_, double bytes_, double flops_ = 0.0,
            double inst_ = 0.0)
      : c(c_), on(want && c_->prof), cls(cls_), bytes(bytes_), flops(flops_), inst(inst_) {
    if (on) {
      a = take_event(c);
      b = take_event(c);
      CK(cudaEventRecord(a, c->stream));
    }
  }
  void done() {
    if (on) {
      CK(cudaEventRecord(b, c->stream));
      c->pending.push_back({a, b, cls, bytes, flops, inst});
      on = false;
    }
  }
};

template <class VT>
DevMat<VT> devmat(const Level& L) {
  DevMat<VT> m;
  m.n = L.n;
  m.nslices = L.nslices;
  m.sd = L.sd;
  m.val = (const VT*)L.val;
  m.col = L.col;
  m.off = L.off;
  return m;
}

DevMat<double> devmat64(const Level& L, amgps_prec prec) {
  if (prec == AMGPS_F64) return devmat<double>(L);
  DevMat<double> m;
  m.n = L.n;
  m.nslices = L.nslices;
  m.sd = L.sd64;
  m.val = L.val64;
  m.col = L.col64;
  m.off = L.off64;
  return m;
}

// Algorithmic bytes of one fused step: A's nonzeros and stored indices once,
// each live vector stream once.
template <class VT, class XT>
double step_bytes(const Level& L, int nvec) {
  return (double)L.nnz * sizeof(VT) + (double)L.explicit_entries * 4.0 +
         (double)L.n * sizeof(XT) * nvec;
}

// Algorithmic FP64 flops of one step (a multiply-add 2, a lone multiply or
// add 1; nnz products per launch).  Recurrence form (row-scaled FP64
// families): the SpMV with the residual folded in, c2 r, the c1 z term when
// present, the x update, and (1/M) rin where rin is still unscaled.
double step_flops(const Level& L, int fam, bool zown, bool raw) {
  const double nnz2 = 2.0 * (double)L.nnz, n = (double)L.n;
  if (fam == FAM_JAC) return nnz2 + 2.0 * n;
  double per = (fam == FAM_CHEB4 ? 2.0 : 1.0) + 1.0 + (zown ? 2.0 : 0.0);
  if (!L.sval || raw) per += 1.0;
  return nnz2 + per * n;
}
// Stored-operator step: the products (the first one a lone multiply when no
// vector term starts the sum), c2 s0 (a multiply) or q (nothing), c1 p, and
// for FAM_OPT the side output u + beta out.
double op_flops(const Level& L, int fam, bool s0, bool s0add, bool s1, bool wt) {
  const double nnz2 = 2.0 * (double)L.nnz, n = (double)L.n;
  if (fam == FAM_OPT) return nnz2 + (wt ? 2.0 * n : 0.0);
  double f = nnz2 + (s0 ? (s0add ? 0.0 : n) : -n);
  if (s1) f += 2.0 * n;
  return f;
}

// FP64 thread instructions the step kernels issue for one step: one
// multiply-add per stored entry (zeros included) and one per vector term of
// the row.  Recurrence form: c2 r, the c1 z term, the x update, and (1/M) rin
// where rin is unscaled (Jacobi: the x update only).
double step_inst(const Level& L, int fam, bool zown, bool raw) {
  const double n = (double)L.n;
  if (fam == FAM_JAC) return (double)L.stored + n;
  return (double)L.stored + n * (2.0 + (zown ? 1.0 : 0.0) + (raw ? 1.0 : 0.0));
}
double op_inst(const Level& L, int fam, bool s0, bool s0add, bool s1, bool wt) {
  const double n = (double)L.n;
  if (fam == FAM_OPT) return (double)L.stored + (wt ? n : 0.0);
  return (double)L.stored + n * ((s0 && !s0add ? 1.0 : 0.0) + (s1 ? 1.0 : 0.0));
}

// ---------------------------------------------------------------------------
// Engine: the kernel sequences, templated on matrix value type VT and vector
// type XT (FP64/FP64, FP32/FP32, BF16/FP32).
// ---------------------------------------------------------------------------
template <class VT, class XT>
struct Engine {
  // While a phase list is being recorded (build_tail), the kernel calls below
  // append their arguments to it instead of launching.
  static std::vector<CyclePhase<VT, XT>>*& rec() {
    thread_local std::vector<CyclePhase<VT, XT>>* r = nullptr;
    return r;
  }

  static void do_first(int fam, int64_t n, const XT* b, const XT* dinv, XT* r, XT* z, XT* x,
                       XT c2, XT beta, XT rhoinv, cudaStream_t s) {
    if (auto* R = rec()) {
      CyclePhase<VT, XT> p;
      p.op = CY_FIRST;
      p.fam = fam;
      p.n = n;
      p.in0 = b;
      p.in1 = dinv;
      p.out0 = r;
      p.out1 = z;
      p.out2 = x;
      p.c2 = c2;
      p.beta = beta;
      p.rhoinv = rhoinv;
      R->push_back(p);
      return;
    }
    launch_first<XT>(fam, n, b, dinv, r, z, x, c2, beta, rhoinv, s);
  }

  static void do_copy(XT* dst, const XT* src, int64_t n, cudaStream_t s) {
    if (auto* R = rec()) {
      CyclePhase<VT, XT> p;
      p.op = CY_COPY;
      p.n = n;
      p.in0 = src;
      p.out0 = dst;
      R->push_back(p);
      return;
    }
    CK(cudaMemcpyAsync(dst, src, n * sizeof(XT), cudaMemcpyDeviceToDevice, s));
  }

  static void do_aggregate(const Level& L, const XT* res, XT* bc, cudaStream_t s) {
    if (auto* R = rec()) {
      CyclePhase<VT, XT> p;
      p.op = CY_AGG;
      p.n = L.nc;
      p.i0 = L.cptr;
      p.i1 = L.cidx;
      p.in0 = res;
      p.out0 = bc;
      R->push_back(p);
      return;
    }
    launch_aggregate<XT>(L.cptr, L.cidx, L.nc, res, bc, s);
  }

  static void do_prolong(const Level& L, const XT* ec, XT* x, cudaStream_t s) {
    if (auto* R = rec()) {
      CyclePhase<VT, XT> p;
      p.op = CY_PROLONG;
      p.n = L.n;
      p.i0 = L.agg;
      p.in0 = ec;
      p.out0 = x;
      R->push_back(p);
      return;
    }
    launch_prolong<XT>(L.n, L.agg, ec, x, s);
  }

  static void do_gemv(const Level& L, const XT* b, XT* x, cudaStream_t s) {
    if (auto* R = rec()) {
      CyclePhase<VT, XT> p;
      p.op = CY_GEMV;
      p.n = L.n;
      p.ainv = L.ainv;
      p.in0 = b;
      p.out0 = x;
      R->push_back(p);
      return;
    }
    launch_coarse_gemv<XT>((int)L.n, L.ainv, b, x, s);
  }

  // One fused step on level L: the TMA-fed kernel over its tiles plus the
  // direct kernel over the remaining slices, or the direct kernel alone.
  static void run_step(amgps_ctx* c, const Level& L, StepArgs<VT, XT> a, cudaStream_t s) {
    a.split = L.split;
    if (L.sval && a.fam == FAM_CHEB4) {
      a.A.val = (const VT*)L.sval;
      a.fam = (a.rin_raw || a.init) ? FAM_CHEB4SR : FAM_CHEB4S;  // an initial step's rin is b
    } else if (L.sval && a.fam == FAM_CHEB1) {
      // residual kept as rho M^{-1} r: the 1/rho moves into the coefficient of r
      a.A.val = (const VT*)L.sval;
      a.fam = a.init ? FAM_CHEB1SR : FAM_CHEB1S;
      a.c2 = a.c2 * a.rhoinv;
    }
    // TMA option 1 (auto): only where the level has at least 4 tiles per SM
    // (two per CTA for FP32 vectors, four per CTA for FP64); below that the
    // persistent pipeline cannot fill and the direct kernel (more, smaller
    // blocks) is faster.  Option 2 takes it wherever planned.
    if (auto* R = rec()) {  // the persistent kernel runs the direct form
      CyclePhase<VT, XT> p;
      p.op = CY_STEP;
      p.a = a;
      p.a.slices = nullptr;
      p.a.nlist = 0;
      R->push_back(p);
      return;
    }
    if (level_uses_tma(c, L)) {
      // the TMA kernel also runs the slices outside its plan (slice list)
      StepArgs<VT, XT> t = a;
      t.slices = L.ngen > 0 ? L.gen_slices : nullptr;
      t.nlist = L.ngen;
      if (launch_step_tma<VT, XT>(t, L.plan, L.tma_tiles, L.ntma, L.tma_grid, c->dscal + S_ERR, s))
        return;
    }
    launch_step<VT, XT>(a, s);
  }

  static bool level_uses_tma(const amgps_ctx* c, const Level& L) {
    return L.ntma > 0 && (c->use_tma == 2 || (c->use_tma == 1 && L.ntma >= 4 * c->nsm));
  }

  // Whether this application on level L runs in the stored-operator form.
  static bool use_ops(const amgps_ctx* c, const Level& L, const Coefs& cf) {
    if constexpr (std::is_same<VT, double>::value && std::is_same<XT, double>::value)
      return c->step_form == 1 && L.ops_ok && !rec() && same_coefs(L.ops_cf, cf);
    else
      return false;
  }

  // One application in the stored-operator form (see op_plan).  Buffers: za
  // holds c = M^{-1} b (formed here unless c_ready: an application from zero
  // on the same b, or on level 0 the PCG r update, left it there), then
  // s_0 = M^{-1}(b - A x_0) in place; the
  // u_j alternate between zb and xb (u_j overwrites u_{j+2}, which only its
  // own row reads); r holds x_0 + h s_0 for the last step when k >= 3.
  static void smooth_ops(amgps_ctx* c, int l, const Coefs& cf, const XT* b, XT* x, bool xzero,
                         bool c_ready) {
    Level& L = c->lv[l];
    cudaStream_t s = c->stream;
    OpStep st[kMaxDegree];
    const int ns = op_plan(cf, st);
    const int k = cf.k;
    XT* cv = (XT*)L.za;
    XT* U[2] = {(XT*)L.zb, (XT*)L.xb};
    XT* t = (XT*)L.r;
    const bool profl = (l == 0);
    if (!c_ready)
      do_first(FAM_JAC, L.n, b, (const XT*)L.dinv, nullptr, nullptr, cv, XT(0), XT(0), XT(1), s);
    const DevMat<VT> A = devmat<VT>(L);
    if (!xzero) {
      StepArgs<VT, XT> a;
      a.A = A;
      a.A.val = (const VT*)L.sval;
      a.u = x;
      a.rin = cv;
      a.zout = cv;
      a.fam = FAM_OPT;
      a.write_r = k >= 3;
      a.rout = t;
      a.beta = XT(st[ns - 1].h);
      ProfScope ps(c, profl, 0, step_bytes<VT, XT>(L, a.write_r ? 4 : 3),
                   op_flops(L, FAM_OPT, true, true, false, a.write_r),
                   op_inst(L, FAM_OPT, true, true, false, a.write_r));
      run_step(c, L, a, s);
      ps.done();
    }
    for (int q = 0; q < ns; ++q) {
      const int j = k - 1 - q;
      StepArgs<VT, XT> a;
      a.A = A;
      a.A.val = (const VT*)L.ops[q];
      a.fam = FAM_OP;
      a.u = q == 0 ? cv : U[(q - 1) & 1];
      a.zout = j == 1 ? x : U[q & 1];
      if (j == 1 && !xzero) {
        a.rin = k >= 3 ? t : x;  // x_0 (+ h s_0), added with coefficient 1
        a.write_r = true;
      } else if (j <= k - 2) {
        a.rin = cv;
        a.c2 = XT(st[q].h);
      }
      if (j <= k - 3) {
        a.xin = U[q & 1];  // u_{j+2}
        a.c1 = XT(st[q].g);
      }
      const int nvec = 2 + (a.rin ? 1 : 0) + (a.xin ? 1 : 0);
      const bool s0 = a.rin != nullptr, s1 = a.xin != nullptr;
      ProfScope ps(c, profl, 0, step_bytes<VT, XT>(L, nvec),
                   op_flops(L, FAM_OP, s0, a.write_r, s1, false),
                   op_inst(L, FAM_OP, s0, a.write_r, s1, false));
      run_step(c, L, a, s);
      ps.done();
    }
    check_launch();
  }

  // One smoother application on level l: x <- S(b, x) (x = 0 when xzero).
  // Returns true when it ran in the stored-operator form (then, from zero,
  // the level's za holds M^{-1} b for a following application with x given:
  // pass c_ready there).
  static bool smooth(amgps_ctx* c, int l, const Coefs& cf, const XT* b, XT* x, bool xzero,
                     bool c_ready = false) {
    Level& L = c->lv[l];
    if (use_ops(c, L, cf)) {
      smooth_ops(c, l, cf, b, x, xzero, c_ready);
      return true;
    }
    cudaStream_t s = c->stream;
    const DevMat<VT> A = devmat<VT>(L);
    const XT* md = (const XT*)L.dinv;
    XT* r = (XT*)L.r;
    XT* zc = (XT*)L.za;
    XT* zn = (XT*)L.zb;
    XT* xb = (XT*)L.xb;
    const int k = cf.k;
    const bool profl = (l == 0);
    if (cf.fam == FAM_JAC) {
      XT* cur = x;
      XT* oth = xb;
      int j0 = 0;
      if (xzero) {
        do_first(FAM_JAC, L.n, b, md, nullptr, nullptr, cur, XT(0), XT(0), XT(1), s);
        j0 = 1;
      }
      for (int j = j0; j < k; ++j) {
        StepArgs<VT, XT> a;
        a.A = A;
        a.u = cur;
        a.rin = b;
        a.xin = cur;
        a.xout = oth;
        a.dinv = md;
        a.fam = FAM_JAC;
        a.init = true;
        ProfScope ps(c, profl, 0, step_bytes<VT, XT>(L, 4), step_flops(L, FAM_JAC, false, false),
                     step_inst(L, FAM_JAC, false, false));
        run_step(c, L, a, s);
        ps.done();
        std::swap(cur, oth);
      }
      if (cur != x) do_copy(x, cur, L.n, s);
      check_launch();
      return false;
    }
    const XT* rin_next;
    XT* xcur = x;
    if (xzero) {
      double c2 = (cf.fam == FAM_CHEB4) ? cf.c2[1] : cf.c2[0];
      double rhoinv = cf.rhoinv;
      if (L.sval && cf.fam == FAM_CHEB1) {  // scaled 1st-kind form: r = rho r^(0)
        c2 *= rhoinv;
        rhoinv = 1.0;
      }
      do_first(cf.fam, L.n, b, md, r, zc, x, XT(c2), XT(cf.beta[1]), XT(rhoinv), s);
      rin_next = (cf.fam == FAM_CHEB4) ? b : r;
    } else {
      StepArgs<VT, XT> a;
      a.A = A;
      a.u = x;
      a.rin = b;
      a.rout = r;
      a.write_r = k > 1;
      a.zout = zc;
      a.xin = x;
      a.xout = xb;
      a.dinv = md;
      a.c2 = XT(cf.fam == FAM_CHEB4 ? cf.c2[1] : cf.c2[0]);
      a.beta = XT(cf.beta[1]);
      a.rhoinv = XT(cf.rhoinv);
      a.fam = cf.fam;
      a.init = true;
      ProfScope ps(c, profl, 0, step_bytes<VT, XT>(L, a.write_r ? 6 : 5),
                   step_flops(L, cf.fam, false, true), step_inst(L, cf.fam, false, true));
      run_step(c, L, a, s);
      ps.done();
      xcur = xb;
      rin_next = r;
    }
    for (int j = 1; j < k; ++j) {
      StepArgs<VT, XT> a;
      a.A = A;
      a.u = zc;
      a.rin = rin_next;
      a.rout = r;
      a.write_r = (j < k - 1);
      a.zown = zc;
      a.zout = zn;
      a.xin = xcur;
      a.xout = x;
      a.dinv = md;
      if (cf.fam == FAM_CHEB4) {
        a.c1 = XT(cf.c1[j + 1]);
        a.c2 = XT(cf.c2[j + 1]);
        a.beta = XT(cf.beta[j + 1]);
      } else {
        a.c1 = XT(cf.c1[j]);
        a.c2 = XT(cf.c2[j]);
      }
      a.rhoinv = XT(cf.rhoinv);
      a.fam = cf.fam;
      a.init = false;
      a.rin_raw = (rin_next == b);  // first step after k_first: r_0 = b
      // streams: z_j, r in(/out), z_{j+1}, x in/out, and 1/M unless scaled
      const bool no_dinv = L.sval && ((cf.fam == FAM_CHEB4 && !a.rin_raw) || cf.fam == FAM_CHEB1);
      const bool raw = a.rin_raw && cf.fam == FAM_CHEB4;
      ProfScope ps(c, profl, 0, step_bytes<VT, XT>(L, (a.write_r ? 7 : 6) - (no_dinv ? 1 : 0)),
                   step_flops(L, cf.fam, true, raw), step_inst(L, cf.fam, true, raw));
      run_step(c, L, a, s);
      ps.done();
      xcur = x;
      rin_next = r;
      std::swap(zc, zn);
    }
    if (xcur != x) do_copy(x, xcur, L.n, s);
    check_launch();
    return false;
  }

  // Coarsest level: x = A_c^{-1} b (dense inverse), or with the coarse-sweeps
  // option x = m l1-Jacobi sweeps from zero (the coarse solver of Sec. 4);
  // both operators are symmetric.
  static void coarse_solve(amgps_ctx* c, int l, const XT* b, XT* x) {
    Level& L = c->lv[l];
    if (c->coarse_sweeps > 0) {
      Coefs cf;
      cf.fam = FAM_JAC;
      cf.k = c->coarse_sweeps;
      smooth(c, l, cf, b, x, true);
    } else {
      do_gemv(L, b, x, c->stream);
      check_launch();
    }
  }

  // record: keep each level's post-smoother input (for the reverse pass);
  // c_ready: the level's za already holds M^{-1} b (written by the PCG update)
  static void vcycle_level(amgps_ctx* c, int l, const XT* b, XT* x, bool record = false,
                           bool c_ready = false) {
    Level& L = c->lv[l];
    cudaStream_t s = c->stream;
    if (!record && !rec() && c->tail_ok && l == c->tail_level && b == (const XT*)L.b &&
        x == (XT*)L.x) {
      launch_tail(c);
      return;
    }
    if (L.coarsest) {
      coarse_solve(c, l, b, x);
      return;
    }
    const Coefs cf = make_coefs(L.spec.kind, L.spec.k, L.spec.w, L.spec.rho);
    // stored-operator form: za = M^{-1} b afterwards, for the post-smoother
    const bool c_kept = smooth(c, l, cf, b, x, true, c_ready);
    Level& C = c->lv[l + 1];
    {
      // b_{l+1} = P^T (b - A x): the true residual (into the level's r buffer,
      // free between the smoothers), then the children sums of each aggregate
      ProfScope ps(c, l == 0, 1,
                   (double)L.nnz * sizeof(VT) + (double)L.explicit_entries * 4.0 +
                       (double)L.n * sizeof(XT) * 4 + (double)L.n * 4 + (double)C.n * 12 +
                       (L.xfer_general ? (double)L.xfer_stored * 6.0 : 0.0));
      StepArgs<VT, XT> a;
      a.A = devmat<VT>(L);
      a.u = x;
      a.rin = b;
      a.zout = (XT*)L.r;
      a.fam = FAM_RES;
      a.init = true;
      run_step(c, L, a, s);
      if (L.xfer_general) launch_xfer<XT>(L.Rm, (const XT*)L.r, (XT*)C.b, 0, L.rsplit, s);
      else do_aggregate(L, (const XT*)L.r, (XT*)C.b, s);
      ps.done();
    }
    {
      // levels >= 1 of the cycle, timed as one class-4 interval from level 0
      ProfScope ps(c, l == 0, 4, 0.0);
      if (l + 1 == 1 && c->graph_ok && !record && !capturing(c)) {
        CK(cudaGraphLaunch(c->gexec, s));
        c->launch_adjust += c->graph_kernels;
      } else {
        vcycle_level(c, l + 1, (const XT*)C.b, (XT*)C.x, record);
      }
      ps.done();
    }
    if (L.xfer_general) launch_xfer<XT>(L.Pm, (const XT*)C.x, x, 1, L.psplit, s);
    else do_prolong(L, (const XT*)C.x, x, s);
    if (record) CK(cudaMemcpyAsync(L.bx2, x, L.n * sizeof(XT), cudaMemcpyDeviceToDevice, s));
    smooth(c, l, cf, b, x, false, c_kept);
    check_launch();
  }

  // ---- reverse mode (FP64 hierarchies) ----
  // One application x = x0 + Q (b - A x0) has Q = q(M^{-1}A) M^{-1}, a symmetric
  // operator, so dL/db = Q gx is one more application of the same smoother to
  // gx from zero, and dL/dx0 = gx - A dL/db one residual step.  For the
  // 4th-kind family x = x0 + sum_j beta_j z_j with z_j independent of beta, so
  // dL/dbeta_j = <gx, z_j>: the z recurrence is recomputed from (b, x0) (no
  // recurrence vector is stored) and each z_j is dotted with gx.

  // <gx, z_j> for j = 1..k into ddots[slot0 + j - 1]
  static void zdots(amgps_ctx* c, int l, const Coefs& cf, const XT* b, const XT* x0,
                    const XT* gx, int slot0) {
    Level& L = c->lv[l];
    cudaStream_t s = c->stream;
    const DevMat<VT> A = devmat<VT>(L);
    const XT* md = (const XT*)L.dinv;
    XT* r = (XT*)L.r;
    XT* zc = (XT*)L.za;
    XT* zn = (XT*)L.zb;
    XT* xs = (XT*)L.xb;
    const int64_t n = L.n;
    const int k = cf.k;
    RedWork rw = redwork(c, 5, n);
    const XT* rin_next;
    if (!x0) {
      launch_first<XT>(FAM_CHEB4, n, b, md, r, zc, xs, XT(cf.c2[1]), XT(0), XT(1), s);
      rin_next = b;
    } else {
      StepArgs<VT, XT> a;
      a.A = A;
      a.u = x0;
      a.rin = b;
      a.rout = r;
      a.write_r = k > 1;
      a.zout = zc;
      a.xin = x0;
      a.xout = xs;
      a.dinv = md;
      a.c2 = XT(cf.c2[1]);
      a.beta = XT(0);
      a.fam = FAM_CHEB4;
      a.init = true;
      run_step(c, L, a, s);
      rin_next = r;
    }
    launch_dot(n, (const double*)gx, (const double*)zc, rw, c->ddots, slot0, 0, s);
    for (int j = 1; j < k; ++j) {
      StepArgs<VT, XT> a;
      a.A = A;
      a.u = zc;
      a.rin = rin_next;
      a.rout = r;
      a.write_r = (j < k - 1);
      a.zown = zc;
      a.zout = zn;
      a.xin = xs;
      a.xout = xs;
      a.dinv = md;
      a.c1 = XT(cf.c1[j + 1]);
      a.c2 = XT(cf.c2[j + 1]);
      a.beta = XT(0);
      a.fam = FAM_CHEB4;
      a.rin_raw = (rin_next == b);
      run_step(c, L, a, s);
      launch_dot(n, (const double*)gx, (const double*)zn, rw, c->ddots, slot0 + j, 0, s);
      rin_next = r;
      std::swap(zc, zn);
    }
    check_launch();
  }

  // gb = dL/db, gx0 = dL/dx0 (nullable), weight dots into ddots[slot0..] (slot0 < 0: none)
  static void smooth_bwd(amgps_ctx* c, int l, const Coefs& cf, const XT* b, const XT* x0,
                         const XT* gx, XT* gb, XT* gx0, int slot0) {
    Level& L = c->lv[l];
    smooth(c, l, cf, gx, gb, true);
    if (gx0) {
      StepArgs<VT, XT> a;
      a.A = devmat<VT>(L);
      a.u = gb;
      a.rin = gx;
      a.zout = gx0;
      a.fam = FAM_RES;
      a.init = true;
      run_step(c, L, a, c->stream);
    }
    if (slot0 >= 0 && cf.fam == FAM_CHEB4) zdots(c, l, cf, b, x0, gx, slot0);
    check_launch();
  }

  // reverse pass of vcycle_level (after a recorded forward): gbout = dL/db_l
  static void vcycle_bwd(amgps_ctx* c, int l, const XT* bl, const XT* xbar, XT* gbout) {
    Level& L = c->lv[l];
    cudaStream_t s = c->stream;
    if (L.coarsest) {
      coarse_solve(c, l, xbar, gbout);  // the coarse operator is symmetric
      return;
    }
    const Coefs cf = make_coefs(L.spec.kind, L.spec.k, L.spec.w, L.spec.rho);
    Level& C = c->lv[l + 1];
    XT* t1 = (XT*)L.bt1;
    XT* t2 = (XT*)L.bt2;
    XT* t3 = (XT*)L.bt3;
    // post-smoother x = S(b, x2): t1 = dL/db (post part), t2 = dL/dx2
    smooth_bwd(c, l, cf, bl, (const XT*)L.bx2, xbar, t1, t2, l * 32);
    // x2 = x1 + P xc ; xc = V_{l+1}(P^T (b - A x1))
    if (L.xfer_general) launch_xfer<XT>(L.Rm, (const XT*)t2, (XT*)C.bgx, 0, L.rsplit, s);
    else launch_aggregate<XT>(L.cptr, L.cidx, L.nc, t2, (XT*)C.bgx, s);
    vcycle_bwd(c, l + 1, (const XT*)C.b, (const XT*)C.bgx, (XT*)C.bgb);
    CK(cudaMemsetAsync(t3, 0, L.n * sizeof(XT), s));
    // dL/dres = P dL/db_c
    if (L.xfer_general) launch_xfer<XT>(L.Pm, (const XT*)C.bgb, t3, 1, L.psplit, s);
    else launch_prolong<XT>(L.n, L.agg, (const XT*)C.bgb, t3, s);
    launch_add<XT>(L.n, t1, t3, gbout, s);
    {
      StepArgs<VT, XT> a;  // dL/dx1 = dL/dx2 - A dL/dres  -> t1
      a.A = devmat<VT>(L);
      a.u = t3;
      a.rin = t2;
      a.zout = t1;
      a.fam = FAM_RES;
      a.init = true;
      run_step(c, L, a, s);
    }
    // pre-smoother x1 = S(b, 0)
    smooth_bwd(c, l, cf, bl, nullptr, t1, t2, nullptr, l * 32 + 16);
    launch_add<XT>(L.n, gbout, t2, gbout, s);
    check_launch();
  }

  static void ensure_bwd(amgps_ctx* c) {
    if (c->bwd_ready) return;
    c->dacc = (double*)dalloc(c, kDotSlots * sizeof(double));
    c->dloss = (double*)dalloc(c, 2 * kMaxLossVectors * sizeof(double));
    for (auto& L : c->lv) {
      const size_t bytes = L.n * sizeof(XT);
      L.bgx = dalloc(c, bytes);
      L.bgb = dalloc(c, bytes);
      if (L.coarsest) continue;
      L.bx2 = dalloc(c, bytes);
      L.bt1 = dalloc(c, bytes);
      L.bt2 = dalloc(c, bytes);
      L.bt3 = dalloc(c, bytes);
    }
    c->bwd_ready = true;
  }

  static bool capturing(amgps_ctx* c) {
    cudaStreamCaptureStatus st;
    CK(cudaStreamIsCapturing(c->stream, &st));
    return st != cudaStreamCaptureStatusNone;
  }

  static void launch_tail(amgps_ctx* c) {
    CycleSync sy;
    sy.count = c->tail_sync;
    CK(cudaMemsetAsync(sy.count, 0, sizeof(unsigned), c->stream));
    const cudaError_t e = launch_cycle<VT, XT>((const CyclePhase<VT, XT>*)c->tail_dev, c->tail_nph,
                                               sy, c->tail_grid, c->dscal + S_ERR, c->stream);
    CK(e);
  }

  // The persistent kernel takes the levels from the first one (>= 1) that
  // runs no TMA-fed step and has at most kCycleMaxRows rows down to the
  // coarsest, when all of them use the direct step, one warp per slice, and
  // aggregation transfers.  Its phase list is the kernel sequence
  // vcycle_level would launch there, recorded.
  static void build_tail(amgps_ctx* c) {
    c->tail_ok = false;
    const int nl = (int)c->lv.size();
    if (!c->use_cycle || nl < 3) return;
    int lt = 1;
    while (lt < nl - 1 && (level_uses_tma(c, c->lv[lt]) || c->lv[lt].n > kCycleMaxRows)) ++lt;
    if (lt >= nl - 1) return;  // only the coarsest level left
    for (int l = lt; l < nl - 1; ++l) {
      const Level& L = c->lv[l];
      if (L.split > 1 || L.xfer_general || level_uses_tma(c, L)) return;
    }
    const int grid = cycle_grid<VT, XT>(c->nsm);
    if (grid <= 0) return;
    std::vector<CyclePhase<VT, XT>> ph;
    rec() = &ph;
    try {
      vcycle_level(c, lt, (const XT*)c->lv[lt].b, (XT*)c->lv[lt].x);
    } catch (...) {
      rec() = nullptr;
      throw;
    }
    rec() = nullptr;
    const size_t bytes = ph.size() * sizeof(CyclePhase<VT, XT>);
    if (bytes > c->tail_cap) {
      if (c->tail_dev) CK(cudaFree(c->tail_dev));
      c->tail_dev = nullptr;
      c->tail_cap = 0;
      CK(cudaMalloc(&c->tail_dev, bytes));
      c->tail_cap = bytes;
    }
    if (!c->tail_sync) {
      CK(cudaMalloc(&c->tail_sync, sizeof(unsigned)));
      CK(cudaMemset(c->tail_sync, 0, sizeof(unsigned)));
    }
    CK(cudaMemcpyAsync(c->tail_dev, ph.data(), bytes, cudaMemcpyHostToDevice, c->stream));
    c->tail_level = lt;
    c->tail_nph = (int)ph.size();
    c->tail_grid = grid;
    // one trial launch outside any capture: a grid the driver cannot make
    // co-resident is refused here, and the coarse levels keep their launches
    // (the trial works on the coarse levels' own buffers, which every
    // V-cycle overwrites before reading)
    CycleSync sy;
    sy.count = c->tail_sync;
    CK(cudaMemsetAsync(sy.count, 0, sizeof(unsigned), c->stream));
    const cudaError_t e = launch_cycle<VT, XT>((const CyclePhase<VT, XT>*)c->tail_dev, c->tail_nph,
                                               sy, grid, c->dscal + S_ERR, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    CK(cudaStreamSynchronize(c->stream));
    c->tail_ok = true;
  }

  // Capture levels >= 1 of the V-cycle into c->gexec; the capture's error code.
  static cudaError_t capture_graph(amgps_ctx* c) {
    if (c->gexec) {
      CK(cudaGraphExecDestroy(c->gexec));
      c->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    const int64_t before = launches_enqueued();
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    try {
      vcycle_level(c, 1, (const XT*)c->lv[1].b, (XT*)c->lv[1].x);
    } catch (const Fail&) {
      err = cudaErrorStreamCaptureInvalidated;
    }
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (err == cudaSuccess) err = ee;
    if (err != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return err;
    }
    const int64_t captured = launches_enqueued() - before;
    err = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) {
      c->gexec = nullptr;
      cudaGetLastError();
      return err;
    }
    c->graph_kernels = captured;
    c->launch_adjust -= captured;
    return cudaSuccess;
  }

  // Levels >= 1 of the V-cycle as a CUDA graph (fixed internal buffers),
  // holding the persistent coarse-level kernel when it is available; if that
  // kernel cannot be captured, the graph holds the coarse levels' launches.
  static void build_graph(amgps_ctx* c) {
    if (c->graph_ok || c->lv.size() < 2) return;
    if (!capturing(c)) build_tail(c);
    else c->tail_ok = false;
    cudaError_t e = capture_graph(c);
    if (e != cudaSuccess && c->tail_ok) {
      c->tail_ok = false;
      e = capture_graph(c);
    }
    CK(e);
    c->graph_ok = true;
  }

  // z = B r on level 0 with FP64 vectors at the boundary (c_ready: level 0's
  // za already holds M^{-1} r, see pcg_impl).
  static void vcycle(amgps_ctx* c, const double* r, double* z, bool c_ready = false) {
    build_graph(c);
    Level& L = c->lv[0];
    if constexpr (std::is_same<XT, double>::value) {
      vcycle_level(c, 0, r, z, false, c_ready);
    } else {
      launch_convert<double, XT>(L.n, r, (XT*)L.b, c->stream);
      vcycle_level(c, 0, (const XT*)L.b, (XT*)L.x);
      launch_convert<XT, double>(L.n, (const XT*)L.x, z, c->stream);
    }
    check_launch();
  }

  static void smooth_public(amgps_ctx* c, int l, const Coefs& cf, const double* b, double* x,
                            bool xzero) {
    if constexpr (std::is_same<XT, double>::value) {
      smooth(c, l, cf, b, x, xzero);
    } else {
      Level& L = c->lv[l];
      // the level's own rhs / solution buffers serve as FP32 staging here
      launch_convert<double, XT>(L.n, b, (XT*)L.b, c->stream);
      if (!xzero) launch_convert<double, XT>(L.n, x, (XT*)L.x, c->stream);
      smooth(c, l, cf, (const XT*)L.b, (XT*)L.x, xzero);
      launch_convert<XT, double>(L.n, (const XT*)L.x, x, c->stream);
      check_launch();
    }
  }

  static double lambda(amgps_ctx* c, int l, const double* v0, int iters) {
    Level& L = c->lv[l];
    cudaStream_t s = c->stream;
    XT* v = (XT*)L.za;
    XT* w = (XT*)L.zb;
    launch_convert<double, XT>(L.n, v0, w, s);
    RedWork rw = redwork(c, 3, L.n);
    launch_norm2<XT>(L.n, w, rw, c->dscal, S_NRM, s);
    launch_scale_by_norm<XT>(L.n, w, v, c->dscal, S_NRM, s);
    const DevMat<VT> A = devmat<VT>(L);
    RedWork rs = redwork(c, 4, L.n);
    for (int i = 0; i < iters; ++i) {
      launch_power_step<VT, XT>(A, v, (const XT*)L.dinv, w, rs, c->dscal, s);
      if (i + 1 < iters) launch_scale_by_norm<XT>(L.n, w, v, c->dscal, S_NRM, s);
    }
    check_launch();
    CK(cudaMemcpyAsync(c->hscal, c->dscal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return std::sqrt(c->hscal[S_NRM]);
  }
};

// Type dispatch on the context's precision.
template <class F>
void with_engine(amgps_ctx* c, F&& f) {
  switch (c->prec) {
    case AMGPS_F64:
      f(Engine<double, double>{});
      break;
    case AMGPS_F32:
      f(Engine<float, float>{});
      break;
    default:
      f(Engine<__nv_bfloat16, float>{});
  }
}

void need_loaded(amgps_ctx* c) {
  REQ(c != nullptr, AMGPS_E_ARG, "null context");
  REQ(c->loaded, AMGPS_E_STATE, "no hierarchy loaded");
}

void check_kind_degree(int kind, int degree) {
  REQ(kind >= AMGPS_L1JACOBI && kind <= AMGPS_WEIGHTS, AMGPS_E_ARG, "unknown smoother kind");
  REQ(degree >= 1 && degree <= kMaxDegree, AMGPS_E_ARG, "degree must be in 1..16");
}

// Levels that take the stored-operator form: FP64 values with the row-scaled
// copy, one warp per slice, and at least kOpMinRows rows (whichever step
// kernel runs them; the smaller levels are launch-bound, and their operators
// would only take memory).
constexpr int64_t kOpMinRows = 1 << 17;
bool op_level(const amgps_ctx* c, const Level& L) {
  return c->prec == AMGPS_F64 && L.sval && !L.coarsest && L.split == 1 && L.n >= kOpMinRows;
}

// Builds, on the library stream, the stored operators of every such level
// for its current smoother (degree >= 2), unless they are
// already built for it.  A level whose operators would not fit the device or
// the context's allocation limit keeps the recurrence form; so does every
// level while the library stream is being captured.
void prepare_ops(amgps_ctx* c) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(c->stream, &cap));
  for (size_t l = 0; l + 1 < c->lv.size(); ++l) {
    Level& L = c->lv[l];
    const Coefs cf = make_coefs(L.spec.kind, L.spec.k, L.spec.w, L.spec.rho);
    if (L.ops_ok && same_coefs(L.ops_cf, cf)) continue;
    L.ops_ok = false;
    if (c->step_form != 1 || cap != cudaStreamCaptureStatusNone || !op_level(c, L)) continue;
    if (cf.k < 2) continue;
    const int ns = cf.k - 1;
    try {
      while ((int)L.ops.size() < ns)
        L.ops.push_back((double*)dalloc(c, (size_t)L.stored * sizeof(double)));
    } catch (const Fail& f) {
      if (f.st != AMGPS_E_NOMEM) throw;
      continue;
    }
    OpStep st[kMaxDegree];
    op_plan(cf, st);
    DevMat<double> B = devmat<double>(L);
    B.val = (const double*)L.sval;
    for (int q = 0; q < ns; ++q) launch_build_op(B, st[q].tau, st[q].sigma, L.ops[q], c->stream);
    check_launch();
    L.ops_cf = cf;
    L.ops_ok = true;
  }
}

// Outer PCG (Sec. 4): one application of the preconditioner (a V-cycle unless
// `precond` is given) per iteration; beta = r.z / r_old.z_old, or with the
// flexible option the Polak-Ribiere beta = r.(z - z_old) / r_old.z_old.
using Precond = std::function<void(const double* r, double* z)>;

// One-reduction flexible CG (AMGPS_OPT_FLEXIBLE = 2): per iteration one
// preconditioner application z = B r, w = A z with the three inner products
// in one grid reduction, and one update kernel that keeps q = A p by the
// recurrence q = w - beta q_old.  The iteration count is the number of
// updates of x, as in the standard form.
void fcg1_impl(amgps_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters,
               double* relres, bool* converged, const Precond& M) {
  Level& L = c->lv[0];
  cudaStream_t s = c->stream;
  const int64_t n = L.n;
  const DevMat<double> A = devmat64(L, c->prec);
  RedWork rw_dot = redwork(c, 0, n, kRedBlocksPerSm), rw_spmv = redwork(c, 1, n),
          rw_upd = redwork(c, 2, n, kRedBlocksPerSm);
  rw_spmv.grid = reduction_grid(L.nslices * kSlice, c->nsm);
  double *z = c->pz, *w = c->pz2, *p = c->pp, *q = c->pq;
  CK(cudaMemcpyAsync(c->pr, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  launch_dot(n, b, b, rw_dot, c->dscal, S_BB, 0, s);
  CK(cudaMemcpyAsync(c->hscal, c->dscal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(c->hscal[S_BB]);
  *converged = false;
  *iters = 0;
  *relres = 0.0;
  if (bnorm == 0.0) {
    *converged = true;
    return;
  }
  REQ(std::isfinite(bnorm), AMGPS_E_NAN, "right-hand side is not finite");
  int it = 0;
  double rel = 1.0;
  for (it = 1; it <= maxit; ++it) {
    const int first = it == 1;
    M(c->pr, z);
    {
      ProfScope ps(c, true, 2, (double)L.nnz * 8 + (double)L.explicit_entries * 4.0 + n * 8.0 * 4);
      launch_spmv_dot3(A, z, w, c->pr, q, first, rw_spmv, c->dscal, s);
      ps.done();
    }
    launch_fcg_update(n, z, w, p, q, x, c->pr, first, rw_upd, c->dscal, s);
    check_launch();
    CK(cudaMemcpyAsync(c->hscal, c->dscal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev_sync, s));
    CK(cudaEventSynchronize(c->ev_sync));
    harvest(c);
    if (c->hscal[S_ERR] != 0.0) {
      CK(cudaMemsetAsync(c->dscal + S_ERR, 0, sizeof(double), s));
      throw Fail{AMGPS_E_TIMEOUT, "a bounded wait inside a pipelined kernel gave up"};
    }
    const double eta = c->hscal[S_PQ], rr = c->hscal[S_RR];
    REQ(std::isfinite(eta) && std::isfinite(rr) && std::isfinite(c->hscal[S_ALPHA]), AMGPS_E_NAN,
        "NaN/Inf in PCG scalars");
    REQ(eta > 0.0, AMGPS_E_NOT_SPD, "p^T A p <= 0 in PCG");
    rel = std::sqrt(rr) / bnorm;
    if (rel <= rtol || it == maxit) break;
  }
  *iters = std::min(it, maxit);
  *relres = rel;
  *converged = rel <= rtol;
}

void pcg_impl(amgps_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters,
              double* relres, bool* converged, const Precond& precond = nullptr) {
  const Precond vcyc = [c](const double* r, double* z) {
    with_engine(c, [&](auto eng) { decltype(eng)::vcycle(c, r, z); });
  };
  const Precond& M = precond ? precond : vcyc;
  if (c->flexible == 2) {
    fcg1_impl(c, b, x, rtol, maxit, iters, relres, converged, M);
    return;
  }
  Level& L = c->lv[0];
  // The V-cycle's level-0 smoother starts from c = M^{-1} r in the
  // stored-operator form: the r update writes it (one stream less than a
  // pass of its own), and the V-cycle skips its c pass.
  const bool fuse_c = !precond && c->prec == AMGPS_F64 && c->step_form == 1 && !L.coarsest &&
                      L.ops_ok &&
                      same_coefs(L.ops_cf, make_coefs(L.spec.kind, L.spec.k, L.spec.w, L.spec.rho));
  cudaStream_t s = c->stream;
  const int64_t n = L.n;
  const DevMat<double> A = devmat64(L, c->prec);
  RedWork rw_dot = redwork(c, 0, n, kRedBlocksPerSm), rw_spmv = redwork(c, 1, n),
          rw_upd = redwork(c, 2, n, kRedBlocksPerSm);
  rw_spmv.grid = reduction_grid(L.nslices * kSlice, c->nsm);
  CK(cudaMemcpyAsync(c->pr, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  double* z = c->pz;    // current preconditioned residual
  double* zo = c->pz2;  // previous one (flexible CG)
  launch_dot(n, b, b, rw_dot, c->dscal, S_BB, 0, s);
  M(c->pr, z);
  launch_dot(n, c->pr, z, rw_dot, c->dscal, S_RZ, 1, s);
  CK(cudaMemcpyAsync(c->pp, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->hscal, c->dscal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  harvest(c);
  const double bnorm = std::sqrt(c->hscal[S_BB]);
  *converged = false;
  *iters = 0;
  *relres = 0.0;
  if (bnorm == 0.0) {
    *converged = true;
    return;
  }
  REQ(std::isfinite(bnorm), AMGPS_E_NAN, "right-hand side is not finite");
  int it = 0;
  double rel = 1.0;
  for (it = 1; it <= maxit; ++it) {
    {
      ProfScope ps(c, true, 2, (double)L.nnz * 8 + (double)L.explicit_entries * 4.0 + n * 8.0 * 2);
      launch_spmv_dot(A, c->pp, c->pq, rw_spmv, c->dscal, s);
      ps.done();
    }
    // r -= alpha q now; x += alpha p is deferred to the direction update
    if (fuse_c)
      launch_r_update(n, c->pq, c->pr, rw_upd, c->dscal, s, (const double*)L.dinv, (double*)L.za);
    else
      launch_r_update(n, c->pq, c->pr, rw_upd, c->dscal, s);
    check_launch();
    CK(cudaMemcpyAsync(c->hscal, c->dscal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev_sync, s));
    CK(cudaEventSynchronize(c->ev_sync));
    harvest(c);
    if (c->hscal[S_ERR] != 0.0) {
      CK(cudaMemsetAsync(c->dscal + S_ERR, 0, sizeof(double), s));
      throw Fail{AMGPS_E_TIMEOUT, "a bounded wait inside a pipelined kernel gave up"};
    }
    const double pq = c->hscal[S_PQ], rr = c->hscal[S_RR];
    REQ(std::isfinite(pq) && std::isfinite(rr), AMGPS_E_NAN, "NaN/Inf in PCG scalars");
    REQ(pq > 0.0, AMGPS_E_NOT_SPD, "p^T A p <= 0 in PCG");
    rel = std::sqrt(rr) / bnorm;
    if (rel <= rtol || it == maxit) {
      launch_xpay_x(n, z, c->pp, x, c->dscal, 0, s);  // the last x update
      check_launch();
      break;
    }
    std::swap(z, zo);
    if (fuse_c)
      Engine<double, double>::vcycle(c, c->pr, z, true);
    else
      M(c->pr, z);
    if (c->flexible == 1) launch_dot(n, c->pr, zo, rw_dot, c->dscal, S_RZP, 0, s);
    launch_dot(n, c->pr, z, rw_dot, c->dscal, S_RZ, c->flexible == 1 ? 2 : 1, s);
    launch_xpay_x(n, z, c->pp, x, c->dscal, 1, s);  // x += alpha p; p = z + beta p
    check_launch();
  }
  *iters = std::min(it, maxit);
  *relres = rel;
  *converged = rel <= rtol;
}

}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free smoother application (amgps_smooth_noalloc).
//
// Its work vectors (the recurrence residual r, the two z buffers, the second
// x buffer and, for FP32/BF16 hierarchies, the FP32 copies of b and x) live in
// this file-scope device array instead of the context's per-level buffers, so
// the call itself allocates nothing.  kNoAllocRows rows x 6 vectors x 8 bytes
// = 3 MiB.  Host code must not pass the symbol itself to a kernel (on the host
// it is only a stand-in): amgps_create looks up its device address with the
// context's device current and keeps it in the context.  That lookup is also
// what brings this file's device module (which holds only the array) onto the
// device under the CUDA runtime's lazy module loading, so the array is claimed
// when a context is created, not by the first allocation-free call.  The
// address stays valid while that device's primary context lives, which the
// library context's own buffers need as well.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocRows = 65536;
constexpr int kNoAllocVectors = 6;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocVectors * kNoAllocRows];

// Device address of the scratch array on the current device.
void* noalloc_scratch_lookup() {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    throw Fail{AMGPS_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                 cudaGetErrorString(e)};
  }
  return p;
}

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

bool is_aggregation(const amgps_csr& P) {
  for (int64_t i = 0; i < P.n_rows; ++i)
    if (P.rowptr[i + 1] - P.rowptr[i] != 1 || P.val[P.rowptr[i]] != 1.0) return false;
  return true;
}

// P and R = P^T in explicit SELL-32 form for the sparse-product transfers
void load_general_transfer(amgps_ctx* c, Level& L, const amgps_csr& P) {
  const int64_t n = P.n_rows, nc = P.n_cols;
  // R = P^T by a counting sort over columns; rows of R come out in
  // ascending column order because P's rows are visited in order
  std::vector<int32_t> rptr(nc + 1, 0), rcol(P.nnz);
  std::vector<double> rval(P.nnz);
  for (int64_t e = 0; e < P.nnz; ++e) rptr[P.col[e] + 1]++;
  for (int64_t I = 0; I < nc; ++I) rptr[I + 1] += rptr[I];
  std::vector<int32_t> fill(rptr.begin(), rptr.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e) {
      const int32_t f = fill[P.col[e]]++;
      rcol[f] = (int32_t)i;
      rval[f] = P.val[e];
    }
  const amgps_csr R{nc, n, P.nnz, rptr.data(), rcol.data(), rval.data()};
  auto put = [&](const amgps_csr& M, DevMat<double>& d, int& split) {
    HostSell h = build_sell(M, false);
    split = split_for(h.stored, h.nslices);
    d.n = M.n_rows;
    d.nslices = h.nslices;
    d.sd = dupload(c, h.sd.data(), h.sd.size());
    d.val = dupload(c, h.val.data(), h.val.size());
    d.col = dupload(c, h.col.data(), h.col.size());
    const int32_t zero = 0;
    d.off = dupload(c, &zero, 1);  // never read: every slice is explicit
    L.xfer_stored += h.stored;
  };
  put(P, L.Pm, L.psplit);
  put(R, L.Rm, L.rsplit);
  L.xfer_general = true;
}

}  // namespace


namespace {
void load_levels(amgps_ctx* c, int n_levels, const amgps_csr* A, const amgps_csr* P,
                 amgps_prec prec);
}  // namespace

extern "C" {

int amgps_version(void) { return 1; }

const char* amgps_last_error(const amgps_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_err.c_str();
}

amgps_status amgps_create(amgps_ctx** out, int device, void* user_stream) {
  if (!out) {
    g_err = "null output pointer";
    return AMGPS_E_ARG;
  }
  *out = nullptr;
  amgps_ctx* c = nullptr;
  amgps_status st = guard(nullptr, [&] {
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    REQ(device >= 0 && device < ndev, AMGPS_E_ARG, "device index out of range");
    CK(cudaSetDevice(device));
    std::unique_ptr<amgps_ctx> u(new amgps_ctx());
    u->device = device;
    CK(cudaDeviceGetAttribute(&u->nsm, cudaDevAttrMultiProcessorCount, device));
    u->ustream = (cudaStream_t)user_stream;
    u->noalloc = noalloc_scratch_lookup();  // with `device` current (see above)
    CK(cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&u->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&u->ev_out, cudaEventDisableTiming));
    // the per-iteration convergence check spin-waits on this event: a
    // blocking wait left the GPU idle ~60 us per iteration (thread wake-up)
    CK(cudaEventCreateWithFlags(&u->ev_sync, cudaEventDisableTiming));
    CK(cudaMalloc(&u->dscal, S_COUNT * sizeof(double)));
    CK(cudaMemset(u->dscal, 0, S_COUNT * sizeof(double)));
    CK(cudaMallocHost(&u->hscal, S_COUNT * sizeof(double)));
    CK(cudaMalloc(&u->ddots, kDotSlots * sizeof(double)));
    CK(cudaMallocHost(&u->hdots, kDotSlots * sizeof(double)));
    const int maxgrid = u->nsm * kRedBlocksPerSm;
    CK(cudaMalloc(&u->part, (size_t)maxgrid * 3 * sizeof(double)));  // grid_sum3: 3 x grid
    CK(cudaMalloc(&u->counters, 8 * sizeof(unsigned)));
    CK(cudaMemset(u->counters, 0, 8 * sizeof(unsigned)));
    c = u.release();
  });
  if (st == AMGPS_OK) *out = c;
  return st;
}

amgps_status amgps_destroy(amgps_ctx* c) {
  if (!c) return AMGPS_OK;
  cudaSetDevice(c->device);
  free_hierarchy(c);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->hscal) cudaFreeHost(c->hscal);
  if (c->hdots) cudaFreeHost(c->hdots);
  if (c->ddots) cudaFree(c->ddots);
  if (c->dscal) cudaFree(c->dscal);
  if (c->part) cudaFree(c->part);
  if (c->counters) cudaFree(c->counters);
  if (c->tail_dev) cudaFree(c->tail_dev);
  if (c->tail_sync) cudaFree(c->tail_sync);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ev_sync) cudaEventDestroy(c->ev_sync);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return AMGPS_OK;
}

amgps_status amgps_hierarchy_load(amgps_ctx* c, int n_levels, const amgps_csr* A,
                                  const amgps_csr* P, amgps_prec prec) {
  return guard(c, [&] {
    REQ(c, AMGPS_E_ARG, "null context");
    REQ(A && n_levels >= 1 && n_levels <= 32, AMGPS_E_ARG, "bad level count or null A");
    REQ(n_levels == 1 || P, AMGPS_E_ARG, "null P");
    REQ(prec == AMGPS_F64 || prec == AMGPS_F32 || prec == AMGPS_BF16, AMGPS_E_ARG,
        "unknown precision");
    // validate everything before touching the device
    for (int l = 0; l < n_levels; ++l) {
      validate_csr(A[l], "A", true);
      // SPD needs a positive diagonal; M_i = sum |a_ij| then bounds rho(M^{-1}A) <= 1
      require_positive_diagonal(A[l]);
    }
    for (int l = 0; l + 1 < n_levels; ++l) {
      validate_csr(P[l], "P", false);
      REQ(P[l].n_rows == A[l].n_rows && P[l].n_cols == A[l + 1].n_rows, AMGPS_E_ARG,
          "P dimensions do not match A_l / A_{l+1}");
    }
    REQ(A[n_levels - 1].n_rows <= 1024, AMGPS_E_ARG, "coarsest level larger than 1024 rows");
    enter(c);
    CK(cudaStreamSynchronize(c->stream));
    free_hierarchy(c);
    try {
      load_levels(c, n_levels, A, P, prec);
      prepare_ops(c);
    } catch (...) {
      free_hierarchy(c);  // a failed load keeps no buffers
      leave(c);
      throw;
    }
    leave(c);
  });
}

}  // extern "C"

namespace {
// The body of amgps_hierarchy_load after validation: upload and plan every level.
void load_levels(amgps_ctx* c, int n_levels, const amgps_csr* A, const amgps_csr* P,
                 amgps_prec prec) {
  tma_configure();
  check_launch();
  c->prec = prec;
  c->lv.resize(n_levels);
  const size_t xs = (prec == AMGPS_F64) ? sizeof(double) : sizeof(float);
  for (int l = 0; l < n_levels; ++l) {
    Level& L = c->lv[l];
    L.n = A[l].n_rows;
    L.nnz = A[l].nnz;
    L.coarsest = (l == n_levels - 1);
    L.b = dalloc(c, L.n * xs);
    L.x = dalloc(c, L.n * xs);
    if (L.coarsest) {
      std::vector<double> dense((size_t)L.n * L.n, 0.0);
      for (int64_t i = 0; i < L.n; ++i)
        for (int e = A[l].rowptr[i]; e < A[l].rowptr[i + 1]; ++e)
          dense[(size_t)i * L.n + A[l].col[e]] = A[l].val[e];
      double* work = dupload(c, dense.data(), dense.size());
      L.ainv = (double*)dalloc(c, dense.size() * sizeof(double));
      int* dstat = (int*)dalloc(c, sizeof(int));
      CK(cudaMemsetAsync(dstat, 0, sizeof(int), c->stream));
      launch_chol_inverse((int)L.n, work, L.ainv, dstat, c->stream);
      check_launch();
      int hstat = 0;
      CK(cudaMemcpyAsync(&hstat, dstat, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      REQ(hstat == 0, AMGPS_E_NOT_SPD, "coarsest matrix: Cholesky pivot not positive");
      // the coarsest level also keeps its SELL form and 1/M: for the PCG
      // SpMV of a single-level hierarchy and for l1-Jacobi coarse sweeps
    }
    HostSell h = build_sell(A[l]);
    L.split = split_for(h.stored, h.nslices);
    L.nslices = h.nslices;
    L.stored = h.stored;
    L.explicit_entries = h.explicit_entries;
    L.sd = dupload(c, h.sd.data(), h.sd.size());
    if (h.off.empty()) h.off.push_back(0);  // every slice explicit: keep a valid pointer
    L.off = dupload(c, h.off.data(), h.off.size());
    L.col = h.any_explicit ? dupload(c, h.col.data(), h.col.size()) : nullptr;
    if (prec == AMGPS_F64) {
      L.val = dupload(c, h.val.data(), h.val.size());
    } else if (prec == AMGPS_F32) {
      std::vector<float> f(h.val.size());
      for (size_t i = 0; i < f.size(); ++i) f[i] = (float)h.val[i];
      L.val = dupload(c, f.data(), f.size());
    } else {
      std::vector<uint16_t> f(h.val.size());
      for (size_t i = 0; i < f.size(); ++i) f[i] = dbl_to_bf16(h.val[i]);
      L.val = dupload(c, f.data(), f.size());
    }
    {
      const size_t vsz = prec == AMGPS_F64 ? 8 : (prec == AMGPS_F32 ? 4 : 2);
      HostPlan hp = build_tma_plan(h, vsz, xs, tma_smem_budget(xs));
      L.plan = hp.p;
      L.ntma = (int)hp.tiles.size();
      L.ngen = (int64_t)hp.gen.size();
      if (L.ntma > 0) {
        L.tma_tiles = dupload(c, hp.tiles.data(), hp.tiles.size());
        L.tma_grid = std::min<int>(L.ntma, tma_ctas_per_sm(xs) * c->nsm);
      }
      if (L.ngen > 0) L.gen_slices = dupload(c, hp.gen.data(), hp.gen.size());
    }
    if (l == 0 && prec != AMGPS_F64) {
      L.sd64 = L.sd;
      L.off64 = L.off;
      L.col64 = L.col;
      L.val64 = dupload(c, h.val.data(), h.val.size());
    }
    if ((prec == AMGPS_F64 || prec == AMGPS_F32) && !L.coarsest) {
      // row-scaled copy a_ij / M_i, M_i = sum_j |a_ij| (the l1 diagonal), in
      // the level's value type (BF16 levels keep A: a_ij / M_i is rarely exact
      // in BF16 where a_ij is)
      std::vector<double> m((size_t)L.n, 0.0);
      const amgps_csr& Al = A[l];
      parallel_for(L.n, [&](int64_t i, int) {
        double acc = 0.0;
        for (int e = Al.rowptr[i]; e < Al.rowptr[i + 1]; ++e) acc += std::fabs(Al.val[e]);
        m[i] = acc;
      });
      std::vector<double> sv(h.val.size(), 0.0);
      parallel_for(h.nslices, [&](int64_t sl, int) {
        const SliceDesc d = h.sd[sl];
        for (int k = 0; k < d.w; ++k)
          for (int ln = 0; ln < kSlice; ++ln) {
            const int64_t row = sl * kSlice + ln;
            const int64_t e = d.vbase + (int64_t)k * kSlice + ln;
            if (row < L.n) sv[e] = h.val[e] / m[row];
          }
      });
      if (prec == AMGPS_F64) {
        L.sval = dupload(c, sv.data(), sv.size());
      } else {
        std::vector<float> svf(sv.size());
        for (size_t i = 0; i < sv.size(); ++i) svf[i] = (float)sv[i];
        L.sval = dupload(c, svf.data(), svf.size());
      }
    }
    L.dinv = dalloc(c, L.n * xs);
    L.r = dalloc(c, L.n * xs);
    L.za = dalloc(c, L.n * xs);
    L.zb = dalloc(c, L.n * xs);
    L.xb = dalloc(c, L.n * xs);
    if (prec == AMGPS_F64)
      launch_l1diag<double, double>(devmat<double>(L), (double*)L.dinv, c->stream);
    else if (prec == AMGPS_F32)
      launch_l1diag<float, float>(devmat<float>(L), (float*)L.dinv, c->stream);
    else launch_l1diag<__nv_bfloat16, float>(devmat<__nv_bfloat16>(L), (float*)L.dinv, c->stream);
    check_launch();
    if (L.coarsest) continue;
    const amgps_csr& Pl = P[l];
    const int64_t nc = Pl.n_cols;
    L.nc = nc;
    L.spec = Spec{};
    if (!is_aggregation(Pl)) {
      load_general_transfer(c, L, Pl);
      continue;
    }
    // aggregation maps: agg[i] and the children lists of every coarse row
    std::vector<int32_t> agg(L.n), cptr(nc + 1, 0), cidx(L.n);
    for (int64_t i = 0; i < L.n; ++i) {
      agg[i] = Pl.col[Pl.rowptr[i]];
      cptr[agg[i] + 1]++;
    }
    for (int64_t I = 0; I < nc; ++I) {
      REQ(cptr[I + 1] > 0, AMGPS_E_ARG, "P has an empty aggregate (zero column)");
      cptr[I + 1] += cptr[I];
    }
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t i = 0; i < L.n; ++i) cidx[fill[agg[i]]++] = (int32_t)i;
    L.agg = dupload(c, agg.data(), agg.size());
    L.cptr = dupload(c, cptr.data(), cptr.size());
    L.cidx = dupload(c, cidx.data(), cidx.size());
  }
  const int64_t n0 = c->lv[0].n;
  c->pr = (double*)dalloc(c, n0 * sizeof(double));
  c->pp = (double*)dalloc(c, n0 * sizeof(double));
  c->pq = (double*)dalloc(c, n0 * sizeof(double));
  c->pz = (double*)dalloc(c, n0 * sizeof(double));
  c->pz2 = (double*)dalloc(c, n0 * sizeof(double));
  c->stage_b = (double*)dalloc(c, n0 * sizeof(double));
  c->stage_x = (double*)dalloc(c, n0 * sizeof(double));
  CK(cudaStreamSynchronize(c->stream));
  c->loaded = true;
}
}  // namespace

extern "C" {

amgps_status amgps_level_info(amgps_ctx* c, int level, int64_t* n, int64_t* nnz, int64_t* stored) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(level >= 0 && level < (int)c->lv.size(), AMGPS_E_ARG, "level out of range");
    if (n) *n = c->lv[level].n;
    if (nnz) *nnz = c->lv[level].nnz;
    if (stored) *stored = c->lv[level].stored;
  });
}

amgps_status amgps_set_smoother(amgps_ctx* c, int level, amgps_kind kind, int degree,
                                const double* weights, double rho) {
  return guard(c, [&] {
    need_loaded(c);
    check_kind_degree(kind, degree);
    const int nl = (int)c->lv.size();
    REQ(level == -1 || (level >= 0 && level < nl - 1), AMGPS_E_ARG,
        "level must be -1 or a non-coarsest level");
    REQ(kind != AMGPS_WEIGHTS || weights, AMGPS_E_ARG, "AMGPS_WEIGHTS needs weights");
    if (weights)
      for (int j = 0; j < degree; ++j)
        REQ(std::isfinite(weights[j]), AMGPS_E_ARG, "non-finite weight");
    REQ(std::isfinite(rho), AMGPS_E_ARG, "non-finite rho");
    for (int l = 0; l < nl - 1; ++l) {
      if (level != -1 && level != l) continue;
      Spec& s = c->lv[l].spec;
      s.kind = kind;
      s.k = degree;
      s.rho = rho > 0.0 ? rho : 1.0;
      std::fill(s.w, s.w + kMaxDegree, 0.0);
      if (weights) std::copy(weights, weights + degree, s.w);
    }
    c->graph_ok = false;
    enter(c);
    prepare_ops(c);
    leave(c);
  });
}

amgps_status amgps_estimate_lambda(amgps_ctx* c, int level, const double* v0, int iters,
                                   double* lambda_out) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(level >= 0 && level < (int)c->lv.size() - 1, AMGPS_E_ARG, "level out of range");
    REQ(v0 && lambda_out && iters >= 1 && iters <= 10000, AMGPS_E_ARG, "bad arguments");
    enter(c);
    double lam = 0.0;
    with_engine(c, [&](auto eng) { lam = decltype(eng)::lambda(c, level, v0, iters); });
    *lambda_out = lam;
    leave(c);
  });
}

amgps_status amgps_smooth(amgps_ctx* c, int level, amgps_kind kind, int degree, const double* b,
                          double* x, int x_is_zero) {
  return guard(c, [&] {
    need_loaded(c);
    check_kind_degree(kind, degree);
    REQ(level >= 0 && level < (int)c->lv.size() - 1, AMGPS_E_ARG,
        "level out of range (the coarsest level has no smoother)");
    REQ(b && x && (const void*)b != (const void*)x, AMGPS_E_ARG, "null or aliased vectors");
    const Spec& sp = c->lv[level].spec;
    REQ(kind != AMGPS_WEIGHTS || (sp.kind == AMGPS_WEIGHTS && sp.k == degree), AMGPS_E_STATE,
        "AMGPS_WEIGHTS: set the level's weights of this degree first");
    const Coefs cf = make_coefs(kind, degree, sp.w, sp.rho);
    enter(c);
    with_engine(c, [&](auto eng) {
      decltype(eng)::smooth_public(c, level, cf, b, x, x_is_zero != 0);
    });
    leave(c);
  });
}

amgps_status amgps_smooth_noalloc(amgps_ctx* c, int level, amgps_kind kind, int degree,
                                  const double* b, double* x, int x_is_zero) {
  return guard(c, [&] {
    need_loaded(c);
    check_kind_degree(kind, degree);
    REQ(level >= 0 && level < (int)c->lv.size() - 1, AMGPS_E_ARG,
        "level out of range (the coarsest level has no smoother)");
    REQ(b && x && (const void*)b != (const void*)x, AMGPS_E_ARG, "null or aliased vectors");
    Level& L = c->lv[level];
    REQ(L.n <= kNoAllocRows, AMGPS_E_ARG,
        "amgps_smooth_noalloc: level " + std::to_string(level) + " has " + std::to_string(L.n) +
            " rows; the static scratch holds at most 65536");
    const Spec& sp = L.spec;
    REQ(kind != AMGPS_WEIGHTS || (sp.kind == AMGPS_WEIGHTS && sp.k == degree), AMGPS_E_STATE,
        "AMGPS_WEIGHTS: set the level's weights of this degree first");
    const Coefs cf = make_coefs(kind, degree, sp.w, sp.rho);
    enter(c);
    REQ(c->noalloc != nullptr, AMGPS_E_STATE, "no scratch address in this context");
    char* base = (char*)c->noalloc;
    const size_t stride = (size_t)kNoAllocRows * sizeof(double);
    // Point the level's work vectors at the static scratch for this call only.
    struct Restore {
      Level& L;
      void *r, *za, *zb, *xb, *b, *x;
      ~Restore() { L.r = r; L.za = za; L.zb = zb; L.xb = xb; L.b = b; L.x = x; }
    } restore{L, L.r, L.za, L.zb, L.xb, L.b, L.x};
    L.r = base;
    L.za = base + stride;
    L.zb = base + 2 * stride;
    L.xb = base + 3 * stride;
    L.b = base + 4 * stride;
    L.x = base + 5 * stride;
    with_engine(c, [&](auto eng) {
      decltype(eng)::smooth_public(c, level, cf, b, x, x_is_zero != 0);
    });
    leave(c);
  });
}

amgps_status amgps_smooth_backward(amgps_ctx* c, int level, amgps_kind kind, int degree,
                                   const double* b, const double* x0, const double* gx, double* gb,
                                   double* gx0, double* gweights) {
  return guard(c, [&] {
    need_loaded(c);
    check_kind_degree(kind, degree);
    REQ(c->prec == AMGPS_F64, AMGPS_E_ARG, "the backward pass needs an FP64 hierarchy");
    REQ(level >= 0 && level < (int)c->lv.size() - 1, AMGPS_E_ARG,
        "level out of range (the coarsest level has no smoother)");
    REQ(b && gx, AMGPS_E_ARG, "null b or gx");
    const Spec& sp = c->lv[level].spec;
    REQ(kind != AMGPS_WEIGHTS || (sp.kind == AMGPS_WEIGHTS && sp.k == degree), AMGPS_E_STATE,
        "AMGPS_WEIGHTS: set the level's weights of this degree first");
    const Coefs cf = make_coefs(kind, degree, sp.w, sp.rho);
    using E = Engine<double, double>;
    enter(c);
    E::ensure_bwd(c);
    Level& L = c->lv[level];
    double* gbuf = gb ? gb : (double*)L.bgb;
    const bool want_w = gweights && cf.fam == FAM_CHEB4;
    E::smooth_bwd(c, level, cf, b, x0, gx, gbuf, gx0, want_w ? 0 : -1);
    if (gweights) {
      std::fill(gweights, gweights + degree, 0.0);
      if (want_w) {
        CK(cudaMemcpyAsync(c->hdots, c->ddots, degree * sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::copy(c->hdots, c->hdots + degree, gweights);
      }
    }
    leave(c);
  });
}

amgps_status amgps_vcycle_backward(amgps_ctx* c, const double* r, const double* gz, double* gr,
                                   double* gweights) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(c->prec == AMGPS_F64, AMGPS_E_ARG, "the backward pass needs an FP64 hierarchy");
    REQ(r && gz, AMGPS_E_ARG, "null r or gz");
    REQ(c->lv.size() <= 32, AMGPS_E_ARG, "too many levels");
    using E = Engine<double, double>;
    enter(c);
    E::ensure_bwd(c);
    Level& L0 = c->lv[0];
    if (L0.coarsest) {
      launch_coarse_gemv<double>((int)L0.n, L0.ainv, gz, gr ? gr : (double*)L0.bgb, c->stream);
      check_launch();
    } else {
      E::vcycle_level(c, 0, r, (double*)L0.x, true);  // forward, recording each level's x2
      E::vcycle_bwd(c, 0, r, gz, gr ? gr : (double*)L0.bgb);
    }
    if (gweights) {
      const int nl = (int)c->lv.size();
      CK(cudaMemcpyAsync(c->hdots, c->ddots, kDotSlots * sizeof(double), cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
      for (int l = 0; l < nl - 1; ++l) {
        const Spec& sp = c->lv[l].spec;
        const Coefs cf = make_coefs(sp.kind, sp.k, sp.w, sp.rho);
        for (int j = 0; j < kMaxDegree; ++j)
          gweights[l * kMaxDegree + j] =
              (cf.fam == FAM_CHEB4 && j < sp.k)
                  ? c->hdots[l * 32 + j] + c->hdots[l * 32 + 16 + j]
                  : 0.0;
      }
    }
    leave(c);
  });
}

amgps_status amgps_vcycle_loss_grad(amgps_ctx* c, const double* E0, int m, double* loss,
                                    double* gweights) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(c->prec == AMGPS_F64, AMGPS_E_ARG, "the loss gradient needs an FP64 hierarchy");
    REQ(E0 && loss && m >= 1 && m <= kMaxLossVectors, AMGPS_E_ARG,
        "null arguments or m outside 1..4096");
    REQ(c->lv.size() >= 2 && c->lv.size() <= 32, AMGPS_E_ARG, "needs 2..32 levels");
    using E = Engine<double, double>;
    enter(c);
    E::ensure_bwd(c);
    cudaStream_t s = c->stream;
    Level& L0 = c->lv[0];
    const int64_t n = L0.n;
    const DevMat<double> A = devmat64(L0, c->prec);
    RedWork rw = redwork(c, 1, n);
    rw.grid = reduction_grid(L0.nslices * kSlice, c->nsm);
    double *r = c->pp, *z = c->pz, *e1 = c->pr, *q1 = c->pq, *gz = c->stage_x;
    CK(cudaMemsetAsync(c->dacc, 0, kDotSlots * sizeof(double), s));
    for (int i = 0; i < m; ++i) {
      const double* e0 = E0 + (size_t)i * n;
      launch_spmv_dot(A, e0, r, rw, c->dscal, s);  // r = A e0, <e0, A e0>
      CK(cudaMemcpyAsync(c->dloss + 2 * i, c->dscal + S_PQ, sizeof(double),
                         cudaMemcpyDeviceToDevice, s));
      E::vcycle_level(c, 0, r, z, true);            // z = B r, recorded
      launch_sub(n, e0, z, e1, s);                  // e1 = (I - B A) e0
      launch_spmv_dot(A, e1, q1, rw, c->dscal, s);  // A e1, <e1, A e1>
      CK(cudaMemcpyAsync(c->dloss + 2 * i + 1, c->dscal + S_PQ, sizeof(double),
                         cudaMemcpyDeviceToDevice, s));
      launch_scale_dev(n, q1, gz, c->dloss + 2 * i, -2.0 / m, s);  // dL/dz
      E::vcycle_bwd(c, 0, r, gz, (double*)L0.bgb);
      launch_add<double>(kDotSlots, c->dacc, c->ddots, c->dacc, s);
      check_launch();
    }
    std::vector<double> hl(2 * (size_t)m);
    CK(cudaMemcpyAsync(hl.data(), c->dloss, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->hdots, c->dacc, kDotSlots * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int i = 0; i < m; ++i) acc += hl[2 * i + 1] / hl[2 * i] / m;
    *loss = acc;
    if (gweights) {
      const int nl = (int)c->lv.size();
      for (int l = 0; l < nl - 1; ++l) {
        const Spec& sp = c->lv[l].spec;
        const Coefs cf = make_coefs(sp.kind, sp.k, sp.w, sp.rho);
        for (int j = 0; j < kMaxDegree; ++j)
          gweights[l * kMaxDegree + j] =
              (cf.fam == FAM_CHEB4 && j < sp.k)
                  ? c->hdots[l * 32 + j] + c->hdots[l * 32 + 16 + j]
                  : 0.0;
      }
    }
    leave(c);
  });
}

amgps_status amgps_error_cycles(amgps_ctx* c, double* E, int m, int cycles) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(E && m >= 1 && cycles >= 0 && cycles <= 1000, AMGPS_E_ARG, "bad arguments");
    enter(c);
    cudaStream_t s = c->stream;
    Level& L0 = c->lv[0];
    const int64_t n = L0.n;
    const DevMat<double> A = devmat64(L0, c->prec);
    RedWork rw = redwork(c, 1, n);
    rw.grid = reduction_grid(L0.nslices * kSlice, c->nsm);
    for (int i = 0; i < m; ++i) {
      double* e = E + (size_t)i * n;
      for (int q = 0; q < cycles; ++q) {
        launch_spmv_dot(A, e, c->pp, rw, c->dscal, s);  // r = A e
        with_engine(c, [&](auto eng) { decltype(eng)::vcycle(c, c->pp, c->pz); });
        launch_sub(n, e, c->pz, e, s);                   // e <- (I - B A) e
      }
    }
    check_launch();
    leave(c);
  });
}

amgps_status amgps_mlp_forward(const float* params, const float* feats, int batch,
                               const float* beta_ref, float* beta, float* acts, void* stream) {
  return guard(nullptr, [&] {
    REQ(params && feats && beta_ref && beta && acts, AMGPS_E_ARG, "null argument");
    REQ(batch >= 1 && batch <= 65535, AMGPS_E_ARG, "batch outside 1..65535");
    mlp_forward(params, feats, batch, beta_ref, beta, acts, (cudaStream_t)stream);
    check_launch();
  });
}

amgps_status amgps_mlp_backward(const float* params, const float* feats, const float* acts,
                                const float* beta, int batch, const float* gbeta, float* work,
                                float* grads, void* stream) {
  return guard(nullptr, [&] {
    REQ(params && feats && acts && beta && gbeta && work && grads, AMGPS_E_ARG,
        "null argument");
    REQ(batch >= 1 && batch <= 65535, AMGPS_E_ARG, "batch outside 1..65535");
    mlp_backward(params, feats, acts, beta, batch, gbeta, work, grads, (cudaStream_t)stream);
    check_launch();
  });
}

amgps_status amgps_mlp_adam(float* params, const float* grads, float* m, float* v, int step,
                            float lr, float beta1, float beta2, float eps, void* stream) {
  return guard(nullptr, [&] {
    REQ(params && grads && m && v, AMGPS_E_ARG, "null argument");
    REQ(step >= 1, AMGPS_E_ARG, "Adam steps count from 1");
    mlp_adam(params, grads, m, v, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
    check_launch();
  });
}

amgps_status amgps_vcycle(amgps_ctx* c, const double* r, double* z) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(r && z && (const void*)r != (const void*)z, AMGPS_E_ARG, "null or aliased vectors");
    enter(c);
    with_engine(c, [&](auto eng) { decltype(eng)::vcycle(c, r, z); });
    leave(c);
  });
}

amgps_status amgps_pcg(amgps_ctx* c, const double* b, double* x, double rtol, int maxit,
                       int* iters, double* relres) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(b && x && iters && relres && (const void*)b != (const void*)x, AMGPS_E_ARG,
        "null or aliased arguments");
    REQ(rtol > 0.0 && maxit >= 1, AMGPS_E_ARG, "rtol must be > 0 and maxit >= 1");
    enter(c);
    bool conv = false;
    pcg_impl(c, b, x, rtol, maxit, iters, relres, &conv);
    leave(c);
    REQ(conv, AMGPS_E_NOCONV, "PCG did not reach rtol within maxit");
  });
}

amgps_status amgps_pcg_smoother(amgps_ctx* c, amgps_kind kind, int degree, const double* b,
                                double* x, double rtol, int maxit, int* iters, double* relres) {
  return guard(c, [&] {
    need_loaded(c);
    check_kind_degree(kind, degree);
    REQ(c->lv.size() >= 2, AMGPS_E_ARG, "level 0 must have a smoother (two or more levels)");
    REQ(b && x && iters && relres && (const void*)b != (const void*)x, AMGPS_E_ARG,
        "null or aliased arguments");
    REQ(rtol > 0.0 && maxit >= 1, AMGPS_E_ARG, "rtol must be > 0 and maxit >= 1");
    const Spec& sp = c->lv[0].spec;
    REQ(kind != AMGPS_WEIGHTS || (sp.kind == AMGPS_WEIGHTS && sp.k == degree), AMGPS_E_STATE,
        "AMGPS_WEIGHTS: set the level's weights of this degree first");
    const Coefs cf = make_coefs(kind, degree, sp.w, sp.rho);
    enter(c);
    bool conv = false;
    const Precond smoother = [&](const double* r, double* z) {
      with_engine(c, [&](auto eng) { decltype(eng)::smooth_public(c, 0, cf, r, z, true); });
    };
    pcg_impl(c, b, x, rtol, maxit, iters, relres, &conv, smoother);
    leave(c);
    REQ(conv, AMGPS_E_NOCONV, "PCG did not reach rtol within maxit");
  });
}

amgps_status amgps_pcg_host(amgps_ctx* c, const double* b_host, double* x_host, double rtol,
                            int maxit, int* iters, double* relres) {
  return guard(c, [&] {
    need_loaded(c);
    REQ(b_host && x_host && iters && relres, AMGPS_E_ARG, "null arguments");
    REQ(rtol > 0.0 && maxit >= 1, AMGPS_E_ARG, "rtol must be > 0 and maxit >= 1");
    const int64_t n = c->lv[0].n;
    enter(c);
    cudaPointerAttributes pa{};
    bool pinned_b = cudaPointerGetAttributes(&pa, b_host) == cudaSuccess &&
                    pa.type == cudaMemoryTypeHost;
    cudaGetLastError();
    cudaPointerAttributes px{};
    bool pinned_x = cudaPointerGetAttributes(&px, x_host) == cudaSuccess &&
                    px.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if ((!pinned_b || !pinned_x) && c->h_stage_n < (size_t)n) {
      if (c->h_stage) cudaFreeHost(c->h_stage);
      c->h_stage = nullptr;
      c->h_stage_n = 0;
      CK(cudaMallocHost(&c->h_stage, n * sizeof(double)));
      c->h_stage_n = n;
    }
    const double* src = b_host;
    if (!pinned_b) {
      std::memcpy(c->h_stage, b_host, n * sizeof(double));
      src = c->h_stage;
    }
    CK(cudaMemcpyAsync(c->stage_b, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    bool conv = false;
    pcg_impl(c, c->stage_b, c->stage_x, rtol, maxit, iters, relres, &conv);
    double* dst = pinned_x ? x_host : c->h_stage;
    CK(cudaMemcpyAsync(dst, c->stage_x, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!pinned_x) std::memcpy(x_host, c->h_stage, n * sizeof(double));
    leave(c);
    REQ(conv, AMGPS_E_NOCONV, "PCG did not reach rtol within maxit");
  });
}

amgps_status amgps_synchronize(amgps_ctx* c) {
  return guard(c, [&] {
    REQ(c, AMGPS_E_ARG, "null context");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(c->hscal + S_ERR, c->dscal + S_ERR, sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    harvest(c);
    if (c->hscal[S_ERR] != 0.0) {
      CK(cudaMemset(c->dscal + S_ERR, 0, sizeof(double)));
      throw Fail{AMGPS_E_TIMEOUT, "a bounded wait inside a pipelined kernel gave up"};
    }
  });
}

amgps_status amgps_set_option(amgps_ctx* c, int option, int64_t value) {
  return guard(c, [&] {
    REQ(c, AMGPS_E_ARG, "null context");
    REQ(option == AMGPS_OPT_TMA || option == AMGPS_OPT_FLEXIBLE ||
            option == AMGPS_OPT_COARSE_SWEEPS || option == AMGPS_OPT_COARSE_KERNEL ||
            option == AMGPS_OPT_ALLOC_LIMIT || option == AMGPS_OPT_STEP_FORM,
        AMGPS_E_ARG, "unknown option");
    if (option == AMGPS_OPT_STEP_FORM) {
      REQ(value == 0 || value == 1, AMGPS_E_ARG, "AMGPS_OPT_STEP_FORM takes 0 or 1");
      c->step_form = (int)value;
      c->graph_ok = false;
      if (c->loaded) {
        enter(c);
        prepare_ops(c);
        leave(c);
      }
    } else if (option == AMGPS_OPT_TMA) {
      REQ(value >= 0 && value <= 2, AMGPS_E_ARG, "AMGPS_OPT_TMA takes 0, 1 or 2");
      c->use_tma = (int)value;
      c->graph_ok = false;
    } else if (option == AMGPS_OPT_FLEXIBLE) {
      REQ(value >= 0 && value <= 2, AMGPS_E_ARG, "AMGPS_OPT_FLEXIBLE takes 0, 1 or 2");
      c->flexible = (int)value;
    } else if (option == AMGPS_OPT_ALLOC_LIMIT) {
      REQ(value >= 0, AMGPS_E_ARG, "AMGPS_OPT_ALLOC_LIMIT takes a byte count >= 0");
      c->alloc_limit = (size_t)value;
    } else if (option == AMGPS_OPT_COARSE_KERNEL) {
      REQ(value == 0 || value == 1, AMGPS_E_ARG, "AMGPS_OPT_COARSE_KERNEL takes 0 or 1");
      c->use_cycle = (int)value;
      c->graph_ok = false;
    } else {
      REQ(value >= 0 && value <= 1000, AMGPS_E_ARG, "AMGPS_OPT_COARSE_SWEEPS takes 0..1000");
      c->coarse_sweeps = (int)value;
      c->graph_ok = false;  // the coarse-level graph holds the coarse solve
    }
  });
}

amgps_status amgps_tma_plan_stats(const amgps_csr* A, amgps_prec prec, int64_t* tiles,
                                  int64_t* generic_slices, int* stage_bytes, int* nstages) {
  return guard(nullptr, [&] {
    REQ(A, AMGPS_E_ARG, "null matrix");
    REQ(prec == AMGPS_F64 || prec == AMGPS_F32 || prec == AMGPS_BF16, AMGPS_E_ARG,
        "unknown precision");
    validate_csr(*A, "A", true);
    HostSell h = build_sell(*A);
    const size_t vsz = prec == AMGPS_F64 ? 8 : (prec == AMGPS_F32 ? 4 : 2);
    const size_t xsz = prec == AMGPS_F64 ? 8 : 4;
    HostPlan hp = build_tma_plan(h, vsz, xsz, tma_smem_budget(xsz));
    if (tiles) *tiles = (int64_t)hp.tiles.size();
    if (generic_slices) *generic_slices = (int64_t)hp.gen.size();
    if (stage_bytes) *stage_bytes = hp.p.stage_bytes;
    if (nstages) *nstages = hp.p.nstages;
  });
}

amgps_status amgps_round_bf16(const double* x, int64_t n, uint16_t* out) {
  return guard(nullptr, [&] {
    REQ(n >= 0 && (n == 0 || (x && out)), AMGPS_E_ARG, "null argument");
    for (int64_t i = 0; i < n; ++i) {
      REQ(std::isfinite(x[i]), AMGPS_E_ARG, "non-finite value");
      out[i] = dbl_to_bf16(x[i]);
    }
  });
}

amgps_status amgps_step_coefs(amgps_kind kind, int degree, const double* weights, double rho,
                              double* c1, double* c2, double* beta, double* rhoinv) {
  return guard(nullptr, [&] {
    check_kind_degree(kind, degree);
    REQ(c1 && c2 && beta && rhoinv, AMGPS_E_ARG, "null argument");
    REQ(kind != AMGPS_WEIGHTS || weights, AMGPS_E_ARG, "AMGPS_WEIGHTS needs weights");
    REQ(std::isfinite(rho), AMGPS_E_ARG, "non-finite rho");
    const Coefs cf = make_coefs(kind, degree, weights, rho);
    for (int j = 0; j <= degree; ++j) {
      c1[j] = cf.c1[j];
      c2[j] = cf.c2[j];
      beta[j] = cf.beta[j];
    }
    *rhoinv = cf.rhoinv;
  });
}

amgps_status amgps_op_coefs(amgps_kind kind, int degree, const double* weights, double rho,
                            double* tau, double* sigma, double* h, double* g) {
  return guard(nullptr, [&] {
    check_kind_degree(kind, degree);
    REQ(degree >= 2, AMGPS_E_ARG, "the stored-operator form takes degrees >= 2");
    REQ(tau && sigma && h && g, AMGPS_E_ARG, "null argument");
    REQ(kind != AMGPS_WEIGHTS || weights, AMGPS_E_ARG, "AMGPS_WEIGHTS needs weights");
    REQ(std::isfinite(rho), AMGPS_E_ARG, "non-finite rho");
    const Coefs cf = make_coefs(kind, degree, weights, rho);
    OpStep st[kMaxDegree];
    const int ns = op_plan(cf, st);
    for (int q = 0; q < ns; ++q) {
      tau[q] = st[q].tau;
      sigma[q] = st[q].sigma;
      h[q] = st[q].h;
      g[q] = st[q].g;
    }
  });
}

amgps_status amgps_tma_plan(const amgps_csr* A, amgps_prec prec, int32_t* info, int64_t* ntiles,
                            int64_t* tiles, int64_t* ngen, int32_t* gen) {
  return guard(nullptr, [&] {
    REQ(A && info && ntiles && ngen, AMGPS_E_ARG, "null argument");
    REQ(prec == AMGPS_F64 || prec == AMGPS_F32 || prec == AMGPS_BF16, AMGPS_E_ARG,
        "unknown precision");
    validate_csr(*A, "A", true);
    const HostSell h = build_sell(*A);
    const size_t vsz = prec == AMGPS_F64 ? 8 : (prec == AMGPS_F32 ? 4 : 2);
    const size_t xsz = prec == AMGPS_F64 ? 8 : 4;
    const HostPlan hp = build_tma_plan(h, vsz, xsz, tma_smem_budget(xsz));
    const TmaPlan& p = hp.p;
    static_assert(kTmaMaxGroups == 4 && kTmaMaxW == 8, "info layout");
    std::fill(info, info + 32, 0);
    const int32_t head[9] = {p.rows, p.w, p.ngroups, p.d0, p.vals_bytes, p.vec_bytes,
                             p.win_bytes, p.stage_bytes, p.nstages};
    std::copy(head, head + 9, info);
    for (int g = 0; g < kTmaMaxGroups; ++g) {
      info[9 + g] = p.g_start[g];
      info[13 + g] = p.g_elems[g];
      info[17 + g] = p.g_smem[g];
    }
    for (int k = 0; k < kTmaMaxW; ++k) info[21 + k] = p.d[k];
    *ntiles = (int64_t)hp.tiles.size();
    *ngen = (int64_t)hp.gen.size();
    if (!tiles) return;  // size query
    REQ(gen || hp.gen.empty(), AMGPS_E_ARG, "null array");
    for (size_t t = 0; t < hp.tiles.size(); ++t) {
      tiles[2 * t] = hp.tiles[t].r0;
      tiles[2 * t + 1] = hp.tiles[t].vbase;
    }
    std::copy(hp.gen.begin(), hp.gen.end(), gen);
  });
}

amgps_status amgps_sell_layout(const amgps_csr* A, int64_t* nslices, int64_t* stored,
                               int64_t* noff, int64_t* vbase, int32_t* width, int32_t* cref,
                               double* val, int32_t* col, int32_t* off) {
  return guard(nullptr, [&] {
    REQ(A && nslices && stored && noff, AMGPS_E_ARG, "null argument");
    validate_csr(*A, "A", true);
    const HostSell h = build_sell(*A);
    *nslices = h.nslices;
    *stored = h.stored;
    *noff = (int64_t)h.off.size();
    if (!vbase) return;  // size query
    REQ(width && cref && val && col && (off || h.off.empty()), AMGPS_E_ARG, "null array");
    for (int64_t s = 0; s < h.nslices; ++s) {
      vbase[s] = h.sd[s].vbase;
      width[s] = h.sd[s].w;
      cref[s] = h.sd[s].cref;
      for (int64_t e = h.sd[s].vbase; e < h.sd[s].vbase + (int64_t)h.sd[s].w * kSlice; ++e)
        col[e] = h.sd[s].cref >= 0 ? -1 : h.col[e];
    }
    std::copy(h.val.begin(), h.val.end(), val);
    std::copy(h.off.begin(), h.off.end(), off);
  });
}

amgps_status amgps_opt4_weights(int degree, double* beta_out) {
  if (!beta_out || degree < 1 || degree > AMGPS_TABLE_KMAX) return AMGPS_E_ARG;
  for (int j = 0; j < degree; ++j) beta_out[j] = AMGPS_OPT4_BETA[degree - 1][j];
  return AMGPS_OK;
}

amgps_status amgps_cheb1_astar(int degree, double* a_out) {
  if (!a_out || degree < 1 || degree > AMGPS_TABLE_KMAX) return AMGPS_E_ARG;
  *a_out = AMGPS_ASTAR[degree - 1];
  return AMGPS_OK;
}

amgps_status amgps_profile_enable(amgps_ctx* c, int on) {
  return guard(c, [&] {
    REQ(c, AMGPS_E_ARG, "null context");
    c->prof = on != 0;
  });
}

amgps_status amgps_profile_read(amgps_ctx* c, int cls, int reset, int64_t* launches,
                                double* total_ms, double* bytes) {
  return guard(c, [&] {
    REQ(c, AMGPS_E_ARG, "null context");
    REQ(cls >= 0 && cls <= 4, AMGPS_E_ARG, "kernel class out of range");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    harvest(c);
    if (cls == 3) {
      const int64_t total = launches_enqueued() + c->launch_adjust;
      if (launches) *launches = total - c->launch_base;
      if (total_ms) *total_ms = 0.0;
      if (bytes) *bytes = 0.0;
      if (reset) c->launch_base = total;
      return;
    }
    if (launches) *launches = c->prof_launches[cls];
    if (total_ms) *total_ms = c->prof_ms[cls];
    if (bytes) *bytes = c->prof_bytes[cls];
    if (reset) {
      c->prof_launches[cls] = 0;
      c->prof_ms[cls] = 0.0;
      c->prof_bytes[cls] = 0.0;
      c->prof_flops[cls] = 0.0;
      c->prof_inst[cls] = 0.0;
    }
  });
}

amgps_status amgps_profile_flops(amgps_ctx* c, int cls, double* flops) {
  return guard(c, [&] {
    REQ(c && flops, AMGPS_E_ARG, "null argument");
    REQ(cls >= 0 && cls <= 4, AMGPS_E_ARG, "kernel class out of range");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    harvest(c);
    *flops = c->prof_flops[cls];
  });
}

amgps_status amgps_profile_fp64_inst(amgps_ctx* c, int cls, double* inst) {
  return guard(c, [&] {
    REQ(c && inst, AMGPS_E_ARG, "null argument");
    REQ(cls >= 0 && cls <= 4, AMGPS_E_ARG, "kernel class out of range");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    harvest(c);
    *inst = c->prof_inst[cls];
  });
}

void amgps_csr_buf_free(amgps_csr_buf* m) { csr_buf_release(m); }

amgps_status amgps_galerkin(amgps_ctx* c, const amgps_csr* A, const amgps_csr* P,
                            amgps_csr_buf* Ac) {
  return guard(c, [&] {
    REQ(c && A && P && Ac, AMGPS_E_ARG, "null argument");
    CK(cudaSetDevice(c->device));
    galerkin_on_device(SetupEnv{c->stream, c->nsm}, *A, *P, Ac);
  });
}

amgps_status amgps_sa_level(amgps_ctx* c, const amgps_csr* A, const int32_t* agg,
                            int64_t n_coarse, double* omega, amgps_csr_buf* P_out,
                            amgps_csr_buf* Ac_out) {
  return guard(c, [&] {
    REQ(c && A && agg && omega && P_out && Ac_out, AMGPS_E_ARG, "null argument");
    CK(cudaSetDevice(c->device));
    sa_level_on_device(SetupEnv{c->stream, c->nsm}, *A, agg, n_coarse, omega, P_out, Ac_out);
  });
}

}  // extern "C"
