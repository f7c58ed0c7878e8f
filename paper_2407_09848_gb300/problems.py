"""Seeded synthetic inputs: SPD model problems and their aggregation hierarchies.

This module produces the *inputs* of the solver and nothing else: the fine
matrix A, the per-level matrices A_l with prolongators P_l, right-hand sides
and random start vectors.  It holds none of the smoother, V-cycle or PCG
arithmetic.  Both the product path and the test oracle consume its output;
neither imports the other.

Problems (Sec. 4 of the paper uses a 7-point Poisson problem on the unit cube
with Dirichlet conditions, and a rotated anisotropic problem; the configurations
used here add a variable-coefficient diffusion problem):

* ``poisson``   : -Laplace, 7-point, Dirichlet nodes eliminated, unscaled
                  (diagonal 6, off-diagonals -1).
* ``aniso``     : 7-point with x/y face coefficient 1 and z face coefficient eps.
* ``varcoef``   : -div(k grad u), face coefficient = harmonic mean of the two
                  cell values, a boundary face uses the cell's own value,
                  k = exp(sigma * g) with g a Gaussian random field of
                  correlation length ell (cells).

The hierarchy is the host-side aggregation set-up of Sec. 2: P_l is the 0/1
piecewise-constant prolongator of 2x2x2 blocks, A_{l+1} = P_l^T A_l P_l
(Galerkin), coarsening until a level has at most ``coarse_max`` unknowns.
Ordering is lexicographic, x fastest.  Because aggregation is geometric, each
A_{l+1} is again a 7-point operator; it is assembled here directly in stencil
form (sums of fine couplings between blocks), which equals P^T A P exactly.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp

__all__ = [
    "Stencil7", "Level", "Hierarchy", "poisson", "aniso", "varcoef", "grf",
    "build_hierarchy", "rhs_uniform", "vec_normal", "vec_uniform", "to_csr",
]


@dataclasses.dataclass
class Stencil7:
    """A symmetric 7-point operator on an nx*ny*nz box.

    ``cx[z,y,x]`` couples (x,y,z) with (x+1,y,z) (shape nz,ny,nx-1), likewise
    ``cy`` (nz,ny-1,nx) and ``cz`` (nz-1,ny,nx).  Off-diagonal entries are
    ``-c``.  ``diag`` (nz,ny,nx) holds the full diagonal, including the
    coefficients of eliminated Dirichlet faces.
    """
    diag: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    cz: np.ndarray

    @property
    def shape(self):
        return self.diag.shape  # (nz, ny, nx)

    @property
    def n(self):
        return int(self.diag.size)


def _from_faces(fx, fy, fz):
    """Assemble a Dirichlet 7-point operator from face coefficients that include
    the boundary faces: fx has shape (nz,ny,nx+1) etc."""
    diag = fx[:, :, :-1] + fx[:, :, 1:] + fy[:, :-1, :] + fy[:, 1:, :] \
        + fz[:-1, :, :] + fz[1:, :, :]
    return Stencil7(diag=np.ascontiguousarray(diag),
                    cx=np.ascontiguousarray(fx[:, :, 1:-1]),
                    cy=np.ascontiguousarray(fy[:, 1:-1, :]),
                    cz=np.ascontiguousarray(fz[1:-1, :, :]))


def poisson(nx, ny=None, nz=None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _from_faces(np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)),
                       np.ones((nz + 1, ny, nx)))


def aniso(nx, eps=1e-3, ny=None, nz=None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _from_faces(np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)),
                       np.full((nz + 1, ny, nx), float(eps)))


def grf(shape, ell, seed):
    """Zero-mean, unit-sample-std Gaussian random field with covariance
    ~exp(-r^2/(2 ell^2)): white noise N(0,1) (PCG64, ``seed``) on a box padded
    by 4*ell per axis, filtered periodically in Fourier space by a Gaussian of
    std ell/sqrt(2), then cropped and normalised."""
    rng = np.random.default_rng(seed)
    pad = int(np.ceil(4 * ell))
    pshape = tuple(s + pad for s in shape)
    w = rng.standard_normal(pshape)
    s = ell / np.sqrt(2.0)
    fw = np.fft.rfftn(w)
    ks = [np.fft.fftfreq(m) for m in pshape[:-1]] + [np.fft.rfftfreq(pshape[-1])]
    filt = np.ones(fw.shape)
    for ax, k in enumerate(ks):
        sh = [1] * len(pshape)
        sh[ax] = -1
        filt = filt * np.exp(-0.5 * (2 * np.pi * k.reshape(sh) * s) ** 2)
    g = np.fft.irfftn(fw * filt, s=pshape, axes=tuple(range(len(pshape))))
    g = g[tuple(slice(0, m) for m in shape)]
    g = g - g.mean()
    g = g / g.std()
    return g


def varcoef(nx, sigma=1.0, ell=8.0, seed=0, ny=None, nz=None):
    """-div(k grad u) with k = exp(sigma*g), harmonic-mean face coefficients."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    kc = np.exp(sigma * grf((nz, ny, nx), ell, seed))

    def faces(axis):
        a = np.moveaxis(kc, axis, -1)
        inner = 2.0 * a[..., :-1] * a[..., 1:] / (a[..., :-1] + a[..., 1:])
        f = np.concatenate([a[..., :1], inner, a[..., -1:]], axis=-1)
        return np.moveaxis(f, -1, axis)

    return _from_faces(faces(2), faces(1), faces(0))


def to_csr(st: Stencil7) -> sp.csr_matrix:
    """CSR (int32 indices, sorted columns, FP64) of a 7-point operator."""
    nz, ny, nx = st.shape
    n = st.n
    idx = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    vals = np.zeros((nz, ny, nx, 7))
    cols = np.zeros((nz, ny, nx, 7), dtype=np.int64)
    mask = np.zeros((nz, ny, nx, 7), dtype=bool)
    # slot order = ascending column: -z, -y, -x, diag, +x, +y, +z
    vals[..., 3] = st.diag
    cols[..., 3] = idx
    mask[..., 3] = True
    vals[:, :, 1:, 2] = -st.cx
    cols[:, :, 1:, 2] = idx[:, :, :-1]
    mask[:, :, 1:, 2] = True
    vals[:, :, :-1, 4] = -st.cx
    cols[:, :, :-1, 4] = idx[:, :, 1:]
    mask[:, :, :-1, 4] = True
    vals[:, 1:, :, 1] = -st.cy
    cols[:, 1:, :, 1] = idx[:, :-1, :]
    mask[:, 1:, :, 1] = True
    vals[:, :-1, :, 5] = -st.cy
    cols[:, :-1, :, 5] = idx[:, 1:, :]
    mask[:, :-1, :, 5] = True
    vals[1:, :, :, 0] = -st.cz
    cols[1:, :, :, 0] = idx[:-1, :, :]
    mask[1:, :, :, 0] = True
    vals[:-1, :, :, 6] = -st.cz
    cols[:-1, :, :, 6] = idx[1:, :, :]
    mask[:-1, :, :, 6] = True
    mask = mask.reshape(n, 7)
    counts = mask.sum(axis=1)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    data = vals.reshape(n, 7)[mask]
    indices = cols.reshape(n, 7)[mask].astype(np.int32)
    if indptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return sp.csr_matrix((data, indices, indptr.astype(np.int32)), shape=(n, n))


def _block_sum(a, axis, n_in):
    """Sum consecutive pairs along ``axis`` (the last block is 1 wide when
    ``n_in`` is odd)."""
    starts = np.arange(0, n_in, 2)
    return np.add.reduceat(a, starts, axis=axis)


def _coarsen(st: Stencil7):
    """Galerkin product P^T A P for 2x2x2 piecewise-constant aggregation, in
    stencil form.  Returns the coarse stencil and the aggregate map agg
    (fine lexicographic index -> coarse lexicographic index)."""
    nz, ny, nx = st.shape
    cnx, cny, cnz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    # diagonal: sum of the block's diagonal entries minus twice the couplings
    # internal to the block (each internal face contributes -c to a_ij and a_ji)
    d = st.diag.copy()
    d = _block_sum(_block_sum(_block_sum(d, 2, nx), 1, ny), 0, nz)
    # internal x faces: faces between x=2X and 2X+1
    def internal(c, axis, n_ax):
        # faces along `axis` number n_ax-1; face f joins f and f+1; internal when f is even
        sel = [slice(None)] * 3
        sel[axis] = slice(0, n_ax - 1, 2)
        return c[tuple(sel)]
    ix = internal(st.cx, 2, nx)          # (nz, ny, floor(nx/2))
    iy = internal(st.cy, 1, ny)
    iz = internal(st.cz, 0, nz)
    ix_b = _block_sum(_block_sum(ix, 1, ny), 0, nz)
    iy_b = _block_sum(_block_sum(iy, 2, nx), 0, nz)
    iz_b = _block_sum(_block_sum(iz, 2, nx), 1, ny)
    d[:, :, :ix_b.shape[2]] -= 2 * ix_b
    d[:, :iy_b.shape[1], :] -= 2 * iy_b
    d[:iz_b.shape[0], :, :] -= 2 * iz_b

    # external faces: between blocks X and X+1 are fine faces f = 2X+1
    def external(c, axis, n_ax):
        sel = [slice(None)] * 3
        sel[axis] = slice(1, n_ax - 1, 2)
        return c[tuple(sel)]
    ex = _block_sum(_block_sum(external(st.cx, 2, nx), 1, ny), 0, nz)
    ey = _block_sum(_block_sum(external(st.cy, 1, ny), 2, nx), 0, nz)
    ez = _block_sum(_block_sum(external(st.cz, 0, nz), 2, nx), 1, ny)
    assert d.shape == (cnz, cny, cnx)
    assert ex.shape == (cnz, cny, cnx - 1)
    assert ey.shape == (cnz, cny - 1, cnx)
    assert ez.shape == (cnz - 1, cny, cnx)
    zz, yy, xx = np.meshgrid(np.arange(nz) // 2, np.arange(ny) // 2,
                             np.arange(nx) // 2, indexing="ij")
    agg = (xx + cnx * (yy + cny * zz)).reshape(-1).astype(np.int32)
    return Stencil7(diag=d, cx=ex, cy=ey, cz=ez), agg


@dataclasses.dataclass
class Level:
    A: sp.csr_matrix          # n_l x n_l, FP64, int32 indices
    shape: tuple              # grid shape (nz, ny, nx)
    agg: np.ndarray | None    # fine -> coarse aggregate (None on the coarsest)
    P: sp.csr_matrix | None   # n_l x n_{l+1} 0/1 prolongator


@dataclasses.dataclass
class Hierarchy:
    levels: list
    name: str = ""

    @property
    def n_levels(self):
        return len(self.levels)

    @property
    def A(self):
        return [lv.A for lv in self.levels]

    @property
    def P(self):
        return [lv.P for lv in self.levels[:-1]]


def build_hierarchy(st: Stencil7, coarse_max=512, name="") -> Hierarchy:
    levels = []
    cur = st
    while True:
        A = to_csr(cur)
        if cur.n <= coarse_max or min(cur.shape) < 2:
            levels.append(Level(A=A, shape=cur.shape, agg=None, P=None))
            break
        nxt, agg = _coarsen(cur)
        n, nc = cur.n, nxt.n
        P = sp.csr_matrix((np.ones(n), agg, np.arange(n + 1, dtype=np.int32)),
                          shape=(n, nc))
        levels.append(Level(A=A, shape=cur.shape, agg=agg, P=P))
        cur = nxt
    return Hierarchy(levels=levels, name=name)


def geometric_aggregates(shape, coarse_max=512):
    """Aggregate maps of 2x2x2 blocks of a lexicographic (x fastest) grid,
    level by level until a grid has <= coarse_max points (the same coarse grids
    as build_hierarchy).  Pure index maps -- the tentative prolongators of
    smoothed aggregation.  Returns [(agg, n_coarse, coarse_shape), ...] with
    agg[i] the coarse index of fine point i."""
    out = []
    nz, ny, nx = shape
    while nx * ny * nz > coarse_max and min(nx, ny, nz) >= 2:
        cnx, cny, cnz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
        zz, yy, xx = np.meshgrid(np.arange(nz) // 2, np.arange(ny) // 2,
                                 np.arange(nx) // 2, indexing="ij")
        agg = (xx + cnx * (yy + cny * zz)).reshape(-1).astype(np.int32)
        out.append((agg, cnx * cny * cnz, (cnz, cny, cnx)))
        nz, ny, nx = cnz, cny, cnx
    return out


def spectral_test_matrix(N, spectrum):
    """Dense SPD A = Q D Q^T of the smoother-only experiment (remark of
    Sec. 2.3): Q the orthonormal eigenvectors of the 1-D finite-difference
    second-derivative matrix (discrete sine basis), D one of three spectra:
      "equispaced": N points evenly spaced in [1/N, 1];
      "boundary":   1 - logspace(-8,-1,N/2) and logspace(-8,-1,N/2)
                    (accumulating at both ends of (0, 1));
      "gap":        logspace(-8,-1,N/2) and N/2 points log-spaced between
                    10 and pi.
    Returns (A as CSR with all N^2 entries, b = A 1)."""
    i = np.arange(1, N + 1)
    Q = np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, i) * np.pi / (N + 1))
    h = N // 2
    if spectrum == "equispaced":
        d = np.linspace(1.0 / N, 1.0, N)
    elif spectrum == "boundary":
        d = np.concatenate([1.0 - np.logspace(-8, -1, h), np.logspace(-8, -1, N - h)])
    elif spectrum == "gap":
        d = np.concatenate([np.logspace(-8, -1, h), np.logspace(1, np.log10(np.pi), N - h)])
    else:
        raise ValueError(spectrum)
    A = (Q * d) @ Q.T
    A = 0.5 * (A + A.T)
    Acsr = sp.csr_matrix(A)
    # keep every entry (the matrix is dense; scipy drops exact zeros only)
    return Acsr, Acsr @ np.ones(N)


def single_aggregate_hierarchy(A):
    """Two levels for a matrix without geometry: A and the 1x1 Galerkin
    coarse matrix of P = (1,...,1)^T (the level-0 smoother is what matters)."""
    n = A.shape[0]
    P = sp.csr_matrix((np.ones(n), np.zeros(n, dtype=np.int32), np.arange(n + 1, dtype=np.int32)),
                      shape=(n, 1))
    Ac = sp.csr_matrix(P.T @ A @ P)
    return [sp.csr_matrix(A), Ac], [P]


def rhs_uniform(n, seed=0):
    """b ~ U[-1,1]^n (PCG64 generator, ``seed``)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


vec_uniform = rhs_uniform


def vec_normal(n, seed=0, count=None):
    rng = np.random.default_rng(seed)
    if count is None:
        return rng.standard_normal(n)
    return rng.standard_normal((count, n))
