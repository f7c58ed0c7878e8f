"""Symmetric multiplicative V-cycle (Eq. amg) and preconditioned CG (oracle).

Test infrastructure only.  FP64, recursive, no fusion.

Readings taken where the paper differs from the configuration built here:
coarsest level solved exactly by a dense Cholesky factorisation (the paper uses
30 l1-Jacobi sweeps there, Sec. 4); the outer solver is textbook
Hestenes-Stiefel PCG stopped on the recurrence residual
||r_k||_2 <= rtol ||b||_2 (the paper uses flexible CG with one reduction per
iteration, Sec. 4); ``fcg1`` gives that variant and ``pcg(flexible=True)`` the
two-reduction flexible form.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .smoother import SmootherSpec, l1_diag, smooth


class OracleAMG:
    """Hierarchy (A_l, P_l) of Sec. 2 plus one smoother spec per level (Eq. amg)."""

    def __init__(self, A_list, P_list, specs, coarse_sweeps=0):
        """coarse_sweeps = 0: the coarsest level is solved by a dense Cholesky
        factorisation; m > 0: by m l1-Jacobi sweeps from zero, the coarse
        solver of the paper's experiments (Sec. 4, 30 sweeps)."""
        self.A = [sp.csr_matrix(A) for A in A_list]
        self.P = [sp.csr_matrix(P) for P in P_list]
        if isinstance(specs, SmootherSpec):
            specs = [specs] * (len(self.A) - 1)
        self.specs = list(specs)
        self.M = [l1_diag(A) for A in self.A[:-1]]
        self.coarse_sweeps = int(coarse_sweeps)
        self.Mc = l1_diag(self.A[-1])
        Ac = self.A[-1].toarray()
        # Cholesky of the coarsest matrix; raises LinAlgError if not SPD
        self.L = np.linalg.cholesky(Ac)

    @property
    def n_levels(self):
        return len(self.A)

    def coarse_solve(self, b):
        """Coarsest level of Eq. amg: exact (Cholesky), or the l1-Jacobi sweeps
        of Sec. 4 when coarse_sweeps > 0."""
        if self.coarse_sweeps > 0:
            spec = SmootherSpec("l1jacobi", self.coarse_sweeps)
            return smooth(self.A[-1], b, None, spec, M=self.Mc)
        y = sla.solve_triangular(self.L, b, lower=True)
        return sla.solve_triangular(self.L.T, y, lower=False)

    def vcycle(self, b, level=0):
        """x = B_l b for the error propagation of Eq. amg:
        I - B_l A_l = G_post (I - P_l B_{l+1} P_l^T A_l) G_pre,
        pre-smoothing from x = 0, true residual b - A x restricted by P^T,
        coarse correction prolonged by P, then post-smoothing from the
        corrected x with the same kind, degree and weights."""
        if level == self.n_levels - 1:
            return self.coarse_solve(b)
        A, P, spec, M = self.A[level], self.P[level], self.specs[level], self.M[level]
        x = smooth(A, b, None, spec, M=M)
        r = b - A @ x
        bc = P.T @ r
        xc = self.vcycle(bc, level + 1)
        x = x + P @ xc
        x = smooth(A, b, x, spec, M=M)
        return x

    def pcg(self, b, rtol=1e-8, maxit=1000, flexible=False, precond=None):
        """Preconditioned CG, preconditioner = one V-cycle.

        flexible=True takes the Polak-Ribiere form of the direction update,
        beta = r_{k+1}.(z_{k+1} - z_k) / (r_k.z_k), the flexible CG that Sec. 4
        uses as its outer solver (there in a one-reduction variant), which
        stays robust when the preconditioner is not exactly a fixed symmetric
        operator.  precond (optional) replaces the V-cycle, e.g. one smoother
        application for the smoother-only experiment of the remark in
        Sec. 2.3.  Starts from x0 = 0.  Returns (x, iterations, recurrence
        residual ratio, history); the iteration count is the number of products
        A p performed."""
        B = self.vcycle if precond is None else precond
        A = self.A[0]
        b = np.asarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        r = b.copy()
        bnorm = np.linalg.norm(b)
        hist = [np.linalg.norm(r) / bnorm]
        if hist[-1] <= rtol:
            return x, 0, hist[-1], hist
        z = B(r)
        p = z.copy()
        rz = r @ z
        it = 0
        for it in range(1, maxit + 1):
            q = A @ p
            alpha = rz / (p @ q)
            x = x + alpha * p
            r = r - alpha * q
            rn = np.linalg.norm(r)
            hist.append(rn / bnorm)
            if rn <= rtol * bnorm or it == maxit:
                break
            z_old = z
            z = B(r)
            rz_new = r @ z
            if flexible:
                beta = (rz_new - r @ z_old) / rz
            else:
                beta = rz_new / rz
            p = z + beta * p
            rz = rz_new
        return x, it, hist[-1], hist

    def fcg1(self, b, rtol=1e-8, maxit=1000, precond=None):
        """Flexible CG needing one global reduction per iteration: the outer
        solver named in Sec. 4 (the paper cites the method and prints no
        algorithm; this is the textbook truncated flexible CG, FCG(1), with
        q = A p carried by recurrence).  Per iteration:
            z = B r;  w = A z
            rho = z.r,  gamma = z.q,  delta = z.w       (one reduction)
            beta = gamma / eta                          (A-orthogonalise z to p)
            p = z - beta p;  q = w - beta q;  eta = delta - beta gamma
            alpha = rho / eta;  x += alpha p;  r -= alpha q
        eta = p.A p follows from A being symmetric (p.w = q.z); rho stands for
        p.r because the previous update made r orthogonal to p.  x0 = 0;
        returns as pcg."""
        B = self.vcycle if precond is None else precond
        A = self.A[0]
        b = np.asarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        r = b.copy()
        bnorm = np.linalg.norm(b)
        hist = [1.0]
        if bnorm == 0.0:
            return x, 0, 0.0, [0.0]
        p = q = None
        eta = None
        it = 0
        for it in range(1, maxit + 1):
            z = B(r)
            w = A @ z
            rho, delta = z @ r, z @ w
            if p is None:
                p, q, eta = z.copy(), w.copy(), delta
            else:
                gamma = z @ q
                beta = gamma / eta
                p = z - beta * p
                q = w - beta * q
                eta = delta - beta * gamma
            alpha = rho / eta
            x = x + alpha * p
            r = r - alpha * q
            rn = np.linalg.norm(r)
            hist.append(rn / bnorm)
            if rn <= rtol * bnorm:
                break
        return x, it, hist[-1], hist
