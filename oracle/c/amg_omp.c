/* All-core CPU build of the oracle's smoother, V-cycle and PCG loops.
 *
 * TEST INFRASTRUCTURE ONLY: the benchmark's CPU baseline and its reference arm
 * time this build on every host core, and the CPU tests check it against the
 * numpy oracle (oracle/smoother.py, oracle/amg.py).  The CUDA path never links
 * or calls it, and it uses nothing of the CUDA path.
 *
 * It restates the numpy oracle in plain C: FP64 CSR, natural row order, one
 * pass per vector operation, no fusion, no blocking.  The only change is that
 * each row loop and each dot product is an OpenMP parallel loop (a dot product
 * is summed per thread, then over threads, so its rounding depends on the
 * thread count).  The steps follow the paper:
 *   l1 diagonal       M_i = a_ii + sum_{j != i} |a_ij|             (Eq. l1smooth)
 *   4th kind          z_j = (2j-3)/(2j+1) z_{j-1} + (8j-4)/(2j+1) (1/rho) M^{-1} r_{j-1},
 *                     x_j = x_{j-1} + beta_j z_j,  r_j = r_{j-1} - A z_j
 *                     (Eq. polsmoother; Eq. polsmootheropt with beta)
 *   1st kind          Algorithm 1 on [a, 1] with theta = (1+a)/2, delta = (1-a)/2
 *                     (Eq. optimal_parameters) and rho(M^{-1}A) := rho
 *   l1-Jacobi         x <- x + M^{-1}(b - A x)
 *   V-cycle           Eq. amg: pre-smooth from 0, P^T (b - A x), recurse,
 *                     x += P x_c, post-smooth from x; coarsest level by the
 *                     dense Cholesky factor L (A_c = L L^T) or m l1-Jacobi sweeps
 *   PCG               Hestenes-Stiefel with one V-cycle per iteration, x0 = 0,
 *                     stop at ||r||_2 <= rtol ||b||_2 (the outer solver of Sec. 4
 *                     in its textbook form)
 * The caller supplies P and its transpose (both CSR), the coarsest level's
 * Cholesky factor and the smoother scalars (beta_j, a_k*) from the numpy
 * oracle's parameter routines.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t n_rows, n_cols;
  const int32_t* rowptr; /* n_rows + 1 */
  const int32_t* col;
  const double* val;
} ora_csr;

/* kind: 0 l1-Jacobi, 1 4th kind (beta_j = 1 unless weights given), 2 1st kind */
typedef struct {
  int kind;
  int k;
  int has_beta;
  double beta[16];
  double a;   /* a_k* of Algorithm 1 */
  double rho; /* rho(M^{-1}A) */
} ora_spec;

typedef struct {
  int nlev;
  const ora_csr* A;  /* nlev */
  const ora_csr* P;  /* nlev - 1 */
  const ora_csr* PT; /* nlev - 1 */
  const ora_spec* spec;
  const double* Lc; /* nc x nc row-major lower Cholesky factor of the coarsest A */
  int coarse_sweeps;
  double** M;   /* l1 diagonal per level */
  double** wx;  /* per level, 6 vectors: x, b, a temporary, the smoother's r, z, t */
} ora_hier;

void ora_set_threads(int t) {
  if (t > 0) omp_set_num_threads(t);
}

int ora_get_threads(void) { return omp_get_max_threads(); }

/* y = A u */
static void spmv(const ora_csr* A, const double* u, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A->n_rows; ++i) {
    double s = 0.0;
    for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) s += A->val[e] * u[A->col[e]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double* x, const double* y) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

/* Eq. l1smooth */
void ora_l1diag(const ora_csr* A, double* M) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A->n_rows; ++i) {
    double m = 0.0;
    for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
      m += (A->col[e] == i) ? A->val[e] : fabs(A->val[e]);
    M[i] = m;
  }
}

/* One smoother application x <- S(b, x0) on A (x0 == NULL: from zero).
 * work: 3 n doubles (r, z, t). */
void ora_smooth(const ora_csr* A, const double* M, const ora_spec* sp, const double* b,
                const double* x0, double* x, double* work) {
  const int64_t n = A->n_rows;
  double* r = work;
  double* z = work + n;
  double* t = work + 2 * n;
  const int k = sp->k;
  if (x0) {
    if (x0 != x) memcpy(x, x0, (size_t)n * sizeof(double));
  } else {
    memset(x, 0, (size_t)n * sizeof(double));
  }
  if (sp->kind == 0) { /* k sweeps of x <- x + M^{-1}(b - A x) */
    for (int s = 0; s < k; ++s) {
      spmv(A, x, t);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + (b[i] - t[i]) / M[i];
    }
    return;
  }
  /* r^(0) = b - A x^(0) */
  if (x0) {
    spmv(A, x, t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
  } else {
    memcpy(r, b, (size_t)n * sizeof(double));
  }
  if (sp->kind == 1) { /* Eq. polsmoother / polsmootheropt */
    memset(z, 0, (size_t)n * sizeof(double));
    for (int j = 1; j <= k; ++j) {
      const double c1 = (double)(2 * j - 3) / (double)(2 * j + 1);
      const double c2 = (double)(8 * j - 4) / (double)(2 * j + 1) / sp->rho;
      const double bj = sp->has_beta ? sp->beta[j - 1] : 1.0;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        z[i] = c1 * z[i] + c2 * (r[i] / M[i]);
        x[i] = x[i] + bj * z[i];
      }
      if (j < k) {
        spmv(A, z, t);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - t[i];
      }
    }
    return;
  }
  /* Algorithm 1: r holds r^(j), z holds d^(j) */
  const double theta = 0.5 * (1.0 + sp->a), delta = 0.5 * (1.0 - sp->a);
  const double sigma1 = theta / delta;
  double rho_prev = 1.0 / sigma1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    r[i] = (r[i] / M[i]) / sp->rho;
    z[i] = r[i] / theta;
    x[i] = x[i] + z[i];
  }
  for (int j = 1; j < k; ++j) {
    spmv(A, z, t);
    const double rho_j = 1.0 / (2.0 * sigma1 - rho_prev);
    const double cd = rho_j * rho_prev, cr = 2.0 * rho_j / delta;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const double s = (t[i] / M[i]) / sp->rho;
      r[i] = r[i] - s;
      z[i] = cd * z[i] + cr * r[i];
      x[i] = x[i] + z[i];
    }
    rho_prev = rho_j;
  }
}

ora_hier* ora_hier_create(int nlev, const ora_csr* A, const ora_csr* P, const ora_csr* PT,
                          const ora_spec* spec, const double* Lc, int coarse_sweeps) {
  ora_hier* h = (ora_hier*)calloc(1, sizeof(ora_hier));
  if (!h) return NULL;
  h->nlev = nlev;
  h->A = A;
  h->P = P;
  h->PT = PT;
  h->spec = spec;
  h->Lc = Lc;
  h->coarse_sweeps = coarse_sweeps;
  h->M = (double**)calloc((size_t)nlev, sizeof(double*));
  h->wx = (double**)calloc((size_t)nlev, sizeof(double*));
  if (!h->M || !h->wx) return NULL;
  for (int l = 0; l < nlev; ++l) {
    const int64_t n = A[l].n_rows;
    h->M[l] = (double*)malloc((size_t)n * sizeof(double));
    h->wx[l] = (double*)malloc((size_t)n * 6 * sizeof(double));
    if (!h->M[l] || !h->wx[l]) return NULL;
    ora_l1diag(&A[l], h->M[l]);
  }
  return h;
}

void ora_hier_free(ora_hier* h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) {
    free(h->M[l]);
    free(h->wx[l]);
  }
  free(h->M);
  free(h->wx);
  free(h);
}

/* coarsest level: L y = b, L^T x = y; or m l1-Jacobi sweeps from zero */
static void coarse_solve(const ora_hier* h, const double* b, double* x) {
  const int l = h->nlev - 1;
  const int64_t n = h->A[l].n_rows;
  if (h->coarse_sweeps > 0) {
    ora_spec s;
    memset(&s, 0, sizeof s);
    s.kind = 0;
    s.k = h->coarse_sweeps;
    s.rho = 1.0;
    ora_smooth(&h->A[l], h->M[l], &s, b, NULL, x, h->wx[l] + 3 * n);
    return;
  }
  const double* L = h->Lc;
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t j = 0; j < i; ++j) s -= L[i * n + j] * x[j];
    x[i] = s / L[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t j = i + 1; j < n; ++j) s -= L[j * n + i] * x[j];
    x[i] = s / L[i * n + i];
  }
}

/* x = B_l b (Eq. amg) */
static void vcycle_level(const ora_hier* h, int l, const double* b, double* x) {
  if (l == h->nlev - 1) {
    coarse_solve(h, b, x);
    return;
  }
  const ora_csr* A = &h->A[l];
  const int64_t n = A->n_rows;
  const int64_t nc = h->A[l + 1].n_rows;
  double* r = h->wx[l] + 2 * n;    /* residual, then P x_c */
  double* work = h->wx[l] + 3 * n; /* 3 n for the smoother */
  double* xc = h->wx[l + 1];       /* the coarse level's x slot */
  double* bc = h->wx[l + 1] + nc;  /* the coarse level's b slot */
  ora_smooth(A, h->M[l], &h->spec[l], b, NULL, x, work);
  spmv(A, x, r);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  spmv(&h->PT[l], r, bc); /* b_c = P^T r */
  vcycle_level(h, l + 1, bc, xc);
  spmv(&h->P[l], xc, r); /* x += P x_c */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + r[i];
  ora_smooth(A, h->M[l], &h->spec[l], b, x, x, work);
}

void ora_vcycle(const ora_hier* h, const double* b, double* x) { vcycle_level(h, 0, b, x); }

/* PCG (x0 = 0).  Returns 0 when converged, 1 at maxit, 2 when p.Ap <= 0 or
 * non-finite. */
int ora_pcg(const ora_hier* h, const double* b, double* x, double rtol, int maxit, int* iters,
            double* relres) {
  const int64_t n = h->A[0].n_rows;
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* z = (double*)malloc((size_t)n * sizeof(double));
  double* p = (double*)malloc((size_t)n * sizeof(double));
  double* q = (double*)malloc((size_t)n * sizeof(double));
  int status = 1, it = 0;
  double rel = 1.0;
  if (!r || !z || !p || !q) {
    status = 3;
    goto done;
  }
  memset(x, 0, (size_t)n * sizeof(double));
  memcpy(r, b, (size_t)n * sizeof(double));
  const double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) {
    rel = 0.0;
    status = 0;
    goto done;
  }
  ora_vcycle(h, r, z);
  memcpy(p, z, (size_t)n * sizeof(double));
  double rz = dot(n, r, z);
  for (it = 1; it <= maxit; ++it) {
    spmv(&h->A[0], p, q);
    const double pq = dot(n, p, q);
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = 2;
      break;
    }
    const double alpha = rz / pq;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      x[i] = x[i] + alpha * p[i];
      r[i] = r[i] - alpha * q[i];
    }
    const double rn = sqrt(dot(n, r, r));
    rel = rn / bnorm;
    if (rn <= rtol * bnorm) {
      status = 0;
      break;
    }
    if (it == maxit) break;
    ora_vcycle(h, r, z);
    const double rz_new = dot(n, r, z);
    const double beta = rz_new / rz;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
  if (it > maxit) it = maxit;
done:
  free(r);
  free(z);
  free(p);
  free(q);
  *iters = it;
  *relres = rel;
  return status;
}
