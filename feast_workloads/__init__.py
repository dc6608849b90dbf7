"""Seeded synthetic inputs for the FEAST contour-filter eigensolver.

This module only builds matrices, intervals and random start blocks.  It holds
none of the eigensolver's arithmetic, so both the CPU oracle (``oracle/``) and
the CUDA library can be fed from it without sharing any method code.

Every generator is deterministic: random numbers come from numpy's PCG64
(``numpy.random.default_rng(seed)``).  Matrices are returned as 0-based CSR
triples ``(indptr int32, indices int32, data float64)`` with sorted, duplicate
free rows.  The paper's own test matrix (the 4x4 "helloworld" system of the
FEAST v4.0 user guide, Sec. 2.4 and its IFEAST variant in Sec. 3.5) is the only
matrix taken from the paper; it stands in for the missing example data sets.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# CSR helpers
# --------------------------------------------------------------------------
@dataclass
class CSR:
    n: int
    indptr: np.ndarray  # int32 [n+1], 0-based
    indices: np.ndarray  # int32 [nnz]
    data: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.indptr[i], self.indptr[i + 1]
            d[i, self.indices[s:e]] += self.data[s:e]
        return d


def csr_from_coo(n: int, rows, cols, vals) -> CSR:
    """Sort (row, col) pairs, sum duplicates and return a 0-based CSR."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, r + 1, 1)
    indptr = np.cumsum(indptr).astype(np.int32)
    return CSR(n, indptr, c, summed.astype(np.float64))


def csr_from_dense(d: np.ndarray) -> CSR:
    r, c = np.nonzero(d)
    return csr_from_coo(d.shape[0], r, c, d[r, c])


def identity_csr(n: int) -> CSR:
    i = np.arange(n)
    return csr_from_coo(n, i, i, np.ones(n))


def diagonal_csr(d: np.ndarray) -> CSR:
    i = np.arange(len(d))
    return csr_from_coo(len(d), i, i, d)


# --------------------------------------------------------------------------
# Matrices
# --------------------------------------------------------------------------
def laplacian_1d(n: int) -> CSR:
    """tridiag(-1, 2, -1) of order n (Dirichlet)."""
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0), np.full(n - 1, -1.0)])
    return csr_from_coo(n, rows, cols, vals)


def _grid_laplacian(shape, potential) -> CSR:
    """(2d)-point Dirichlet Laplacian on a box grid plus a diagonal potential.

    Row index is lexicographic with the LAST axis fastest.
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 2.0 * len(shape)) + np.asarray(potential, dtype=np.float64).ravel()]
    for ax in range(len(shape)):
        lo = [slice(None)] * len(shape)
        hi = [slice(None)] * len(shape)
        lo[ax] = slice(0, shape[ax] - 1)
        hi[ax] = slice(1, shape[ax])
        a = idx[tuple(lo)].ravel()
        b = idx[tuple(hi)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, -1.0), np.full(a.size, -1.0)]
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def laplacian_2d(side: int, potential=None) -> CSR:
    pot = np.zeros((side, side)) if potential is None else potential
    return _grid_laplacian((side, side), pot)


def laplacian_3d(side: int, potential=None) -> CSR:
    pot = np.zeros((side, side, side)) if potential is None else potential
    return _grid_laplacian((side, side, side), pot)


def stencil27_spd(side: int, rng: np.random.Generator, shape=None) -> CSR:
    """27-point SPD stencil: off-diagonals -U[0.5,1.5] drawn once per undirected
    edge (so the matrix is symmetric), diagonal = row-abs-sum + U[0.1,1].  The
    grid is side^3, or `shape` = (nz, ny, nx) with x fastest."""
    shape = (side, side, side) if shape is None else tuple(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows, cols = [], []
    # each undirected edge once: offsets with the first nonzero component > 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                off = (dz, dy, dx)
                first = next((o for o in off if o != 0), 0)
                if first <= 0:
                    continue
                src = [slice(max(0, -o), m - max(0, o)) for o, m in zip(off, shape)]
                dst = [slice(max(0, o), m - max(0, -o)) for o, m in zip(off, shape)]
                rows.append(idx[tuple(src)].ravel())
                cols.append(idx[tuple(dst)].ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    w = -rng.uniform(0.5, 1.5, size=r.size)
    absum = np.zeros(n)
    np.add.at(absum, r, -w)
    np.add.at(absum, c, -w)
    diag = absum + rng.uniform(0.1, 1.0, size=n)
    i = np.arange(n)
    return csr_from_coo(n, np.concatenate([r, c, i]), np.concatenate([c, r, i]),
                        np.concatenate([w, w, diag]))


def mass_like_grid(shape, rng: np.random.Generator) -> CSR:
    """Non-diagonal SPD B for the generalized problem A x = lambda B x: the
    (2d+1)-point grid pattern of a box grid (last axis fastest) with diagonal
    U[1,2] and off-diagonals +U[0.05,0.15] drawn once per undirected edge
    (symmetric), like a finite-element mass matrix.  At most 2d <= 6
    off-diagonals of at most 0.15 per row against a diagonal of at least 1:
    strictly diagonally dominant with a positive diagonal, hence SPD
    (Gershgorin)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows, cols = [], []
    for ax in range(len(shape)):
        lo = [slice(None)] * len(shape)
        hi = [slice(None)] * len(shape)
        lo[ax] = slice(0, shape[ax] - 1)
        hi[ax] = slice(1, shape[ax])
        rows.append(idx[tuple(lo)].ravel())
        cols.append(idx[tuple(hi)].ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    w = rng.uniform(0.05, 0.15, size=r.size)
    i = np.arange(n)
    d = rng.uniform(1.0, 2.0, size=n)
    return csr_from_coo(n, np.concatenate([r, c, i]), np.concatenate([c, r, i]), np.concatenate([w, w, d]))


def mass_like_3d(side: int, rng: np.random.Generator) -> CSR:
    """mass_like_grid on a side^3 grid (7-point pattern)."""
    return mass_like_grid((side, side, side), rng)


def laplace3d_general_b(side: int = 10, count: int = 20, m0: int = 32, ne: int = 8, ratio: int = 100,
                        seed: int = 6) -> Problem:
    """Generalized problem with a non-diagonal sparse B: A = 7-point Laplacian +
    V ~ U[0, 0.5], B = mass_like_3d (same seed stream).  The interval is
    [0, Emax] with Emax midway between the count-th and (count+1)-th
    eigenvalues of the pencil (dense eigensolve: for small grids only)."""
    rng = np.random.default_rng(seed)
    pot = rng.uniform(0.0, 0.5, size=(side, side, side))
    A = laplacian_3d(side, pot)
    B = mass_like_3d(side, rng)
    import scipy.linalg

    ev = scipy.linalg.eigh(A.to_dense(), B.to_dense(), eigvals_only=True)
    emax = 0.5 * (ev[count - 1] + ev[count])
    return Problem(f"laplace3d_genB_{side}^3", A, B, 0.0, float(emax), m0, ne, ratio, seed,
                   {"target_count": count})


def helloworld_dense() -> np.ndarray:
    """The 4x4 real symmetric example of the FEAST v4.0 guide (Sec. 2.4),
    eigenvalues {0, 2, 4, 4}."""
    return np.array([[2.0, -1.0, -1.0, 0.0],
                     [-1.0, 3.0, -1.0, -1.0],
                     [-1.0, -1.0, 3.0, -1.0],
                     [0.0, -1.0, -1.0, 2.0]])


def helloworld_csr_1based():
    """The same matrix in the guide's 1-based CSR encoding (IFEAST example,
    Sec. 3.5): returns (sA, IA, JA) exactly as printed there."""
    sA = np.array([2.0, -1.0, -1.0, -1.0, 3.0, -1.0, -1.0, -1.0, -1.0, 3.0, -1.0, -1.0, -1.0, 2.0])
    IA = np.array([1, 4, 8, 12, 15], dtype=np.int32)
    JA = np.array([1, 2, 3, 1, 2, 3, 4, 1, 2, 3, 4, 2, 3, 4], dtype=np.int32)
    return sA, IA, JA


# --------------------------------------------------------------------------
# Start block and search-interval estimates
# --------------------------------------------------------------------------
# --------------------------------------------------------------------------
# complex Hermitian inputs (zfeast_hcsr-type problems)
# --------------------------------------------------------------------------
@dataclass
class ZCSR:
    """0-based CSR with complex128 values (full storage)."""
    n: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.complex128)
        for i in range(self.n):
            s, e = self.indptr[i], self.indptr[i + 1]
            d[i, self.indices[s:e]] += self.data[s:e]
        return d


def zcsr_from_dense(d: np.ndarray) -> ZCSR:
    n = d.shape[0]
    indptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(d[i])[0]
        cols.append(nz.astype(np.int32))
        vals.append(d[i, nz].astype(np.complex128))
        indptr[i + 1] = indptr[i] + len(nz)
    return ZCSR(n, indptr, np.concatenate(cols), np.concatenate(vals))


def flux_ring(n: int, phi: float) -> ZCSR:
    """Ring of n sites threaded by a magnetic flux: 2 on the diagonal,
    -exp(i phi) at (j, j+1 mod n) and its conjugate at (j+1 mod n, j)."""
    d = np.zeros((n, n), dtype=np.complex128)
    j = np.arange(n)
    d[j, j] = 2.0
    d[j, (j + 1) % n] = -np.exp(1j * phi)
    d[(j + 1) % n, j] = -np.exp(-1j * phi)
    return zcsr_from_dense(d)


def hermitian_banded(n: int, bw: int, rng: np.random.Generator, shift: float = 0.0) -> ZCSR:
    """Random complex Hermitian band matrix (half-bandwidth bw), plus shift * I."""
    d = np.zeros((n, n), dtype=np.complex128)
    for k in range(1, bw + 1):
        v = rng.standard_normal(n - k) + 1j * rng.standard_normal(n - k)
        d += np.diag(v, k) + np.diag(v.conj(), -k)
    d += np.diag(rng.standard_normal(n) + shift)
    return zcsr_from_dense(d)


def complex_gaussian_block(n: int, m0: int, seed: int) -> np.ndarray:
    """Y0 with independent N(0,1) real and imaginary parts, (n, m0), Fortran order."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m0)) + 1j * rng.standard_normal((n, m0)))


def gaussian_block(n: int, m0: int, seed: int) -> np.ndarray:
    """Y0 ~ N(0,1), shape (n, m0), Fortran (column-major) order."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m0)))


def _laplacian_levels(side: int, dim: int, count: int) -> np.ndarray:
    """Lowest `count`+ closed-form eigenvalues of the dim-D Dirichlet Laplacian
    on a side^dim grid (sums of 2-2cos(k pi/(side+1)))."""
    kmax = min(side, int(math.ceil((count * 2 ** dim) ** (1.0 / dim))) + 4)
    mu = 2.0 - 2.0 * np.cos(np.arange(1, kmax + 1) * np.pi / (side + 1))
    grids = np.meshgrid(*([mu] * dim), indexing="ij")
    return np.sort(np.sum(grids, axis=0).ravel())


def interval_estimate(side: int, dim: int, count: int, mean_potential: float) -> float:
    """Upper interval end placed in a gap of the closed-form spectrum of the
    constant-potential Laplacian (mean potential added), at the first gap after
    `count` eigenvalues.  For a random potential the true count is close to
    `count`, not exact; it is an input choice, not an expected value."""
    lev = _laplacian_levels(side, dim, count + 64)
    k = count
    while k < len(lev) - 1 and lev[k] - lev[k - 1] < 1e-9:
        k += 1
    return float(mean_potential + 0.5 * (lev[k - 1] + lev[k]))


# --------------------------------------------------------------------------
# Workloads of the evaluation configurations
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    A: CSR
    B: CSR | None  # None means B = I
    emin: float
    emax: float
    m0: int
    ne: int
    ratio: int  # fpm(18): ellipse ratio in percent
    y0_seed: int
    notes: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.n

    def y0(self) -> np.ndarray:
        return gaussian_block(self.n, self.m0, self.y0_seed)


def tridiag_1d(n: int = 1000, emin: float = 0.0, emax: float = 0.01, m0: int = 48,
               ne: int = 8, ratio: int = 30, seed: int = 0) -> Problem:
    """1D Laplacian tridiag(-1,2,-1), B = I.  At n=1000, [0,0.01] holds the 31
    eigenvalues 2-2cos(k pi/1001), k=1..31."""
    return Problem(f"laplace1d_n{n}", laplacian_1d(n), None, emin, emax, m0, ne, ratio, seed)


def laplace3d_potential(side: int = 64, count: int = 100, m0: int = 150, ne: int = 8,
                        ratio: int = 100, seed: int = 1, vmax: float = 0.5) -> Problem:
    """7-point 3D Laplacian on side^3 plus diagonal V ~ U[0, vmax] (seeded), B = I,
    interval [0, Emax] with Emax from the closed-form spectrum estimate."""
    rng = np.random.default_rng(seed)
    pot = rng.uniform(0.0, vmax, size=(side, side, side))
    A = laplacian_3d(side, pot)
    emax = interval_estimate(side, 3, count, 0.5 * vmax)
    return Problem(f"laplace3d_{side}^3", A, None, 0.0, emax, m0, ne, ratio, seed,
                   {"target_count": count})


def laplace3d_constant(side: int, v0: float, emax: float, m0: int, ne: int = 8,
                       ratio: int = 100, seed: int = 5) -> Problem:
    """Constant potential v0: spectrum is v0 + closed-form 3D Laplacian levels."""
    A = laplacian_3d(side, np.full((side, side, side), v0))
    return Problem(f"laplace3d_const_{side}^3", A, None, 0.0, emax, m0, ne, ratio, seed)


def stencil27_generalized(side: int = 96, count: int = 200, m0: int = 300, ne: int = 16,
                          ratio: int = 100, seed: int = 2, emax: float | None = None) -> Problem:
    """27-point SPD stencil with B = diag(U[1,2]); Emax must be supplied or is
    left to the extreme-eigenvalue estimate of the caller."""
    rng = np.random.default_rng(seed)
    A = stencil27_spd(side, rng)
    B = diagonal_csr(rng.uniform(1.0, 2.0, size=side ** 3))
    return Problem(f"stencil27_{side}^3", A, B, 0.0, -1.0 if emax is None else emax,
                   m0, ne, ratio, seed, {"target_count": count})


def gauge_phases(A: CSR, seed: int) -> ZCSR:
    """The complex Hermitian D A D^H with D = diag(exp(i theta_j)), theta_j ~
    U[0, 2 pi) (seeded): entry (j, k) gets the phase exp(i (theta_j - theta_k)),
    so every off-diagonal entry is complex while the spectrum stays A's (the
    eigenvectors are D x)."""
    rng = np.random.default_rng([seed, 7])
    theta = rng.uniform(0.0, 2.0 * np.pi, size=A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.indptr))
    data = A.data * np.exp(1j * (theta[rows] - theta[A.indices]))  # (k, j) is exactly the conjugate
    return ZCSR(A.n, A.indptr.copy(), A.indices.copy(), data.astype(np.complex128))


def laplace3d_gauge(side: int = 64, count: int = 100, m0: int = 150, ne: int = 8, ratio: int = 200,
                    seed: int = 1) -> Problem:
    """Complex Hermitian workload: the 7-point 3D Laplacian + V ~ U[0, 0.5] of
    laplace3d_potential with random gauge phases on every site (gauge_phases);
    same interval and same eigenvalues as the real problem.  y0() is complex."""
    p = laplace3d_potential(side=side, count=count, m0=m0, ne=ne, ratio=ratio, seed=seed)
    q = Problem(f"laplace3d_gauge_{side}^3", gauge_phases(p.A, seed), None, p.emin, p.emax, m0, ne, ratio, seed,
                dict(p.notes, real_problem=p))
    q.y0 = lambda: complex_gaussian_block(q.n, q.m0, q.y0_seed)  # type: ignore[method-assign]
    return q


def count_below(A: CSR, sigma: float) -> int:
    """Number of eigenvalues of the symmetric A below sigma, by Sylvester's law
    of inertia: negative pivots of a sparse symmetric LDL^T of A - sigma I
    (SuperLU with a symmetric ordering and diagonal pivots; a library
    factorisation used only to place search intervals)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    M = sp.csc_matrix((A.data, A.indices, A.indptr), shape=(A.n, A.n)) - sigma * sp.identity(A.n, format="csc")
    lu = sla.splu(M.tocsc(), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                  options={"SymmetricMode": True})
    return int(np.sum(lu.U.diagonal() < 0))


def _place_interval(A: CSR, k: int, e_est: float):
    """Emax with count_below(A, Emax) within [max(8, 3k/4), min(64, 5k/4)]:
    Illinois regula falsi on the count, bracketed below by 0 (all eigenvalues
    are positive) and above by the closed-form estimate (doubled if short)."""
    lo_c, hi_c = max(8, (3 * k) // 4), min(64, (5 * k + 3) // 4)
    target = 0.5 * (lo_c + hi_c)
    e_hi, c_hi = e_est, count_below(A, e_est)
    if lo_c <= c_hi <= hi_c:
        return e_hi, c_hi
    e_lo, c_lo = 0.0, 0
    while c_hi < lo_c:
        e_lo, c_lo = e_hi, c_hi
        e_hi *= 2.0
        c_hi = count_below(A, e_hi)
    if lo_c <= c_hi <= hi_c:
        return e_hi, c_hi
    side = 0
    e, c = e_hi, c_hi
    for _ in range(60):
        e = e_lo + (target - c_lo) * (e_hi - e_lo) / max(c_hi - c_lo, 1)
        c = count_below(A, e)
        if lo_c <= c <= hi_c:
            break
        if c > hi_c:
            e_hi, c_hi = e, c
            if side == -1:
                c_lo = c_lo + (target - c_lo) * 0.5  # Illinois: halve the stale end's weight
            side = -1
        else:
            e_lo, c_lo = e, c
            if side == 1:
                c_hi = c_hi - (c_hi - target) * 0.5
            side = 1
    return e, c


def _laplace2d_problem(args):
    p, seed, ne, ratio, side_lo, side_hi = args
    rng = np.random.default_rng([seed, p])
    side = int(math.floor(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
    side = max(side_lo, min(side_hi, side))
    k = int(rng.integers(8, 65))
    pot = rng.uniform(0.0, 1.0, size=(side, side))
    A = laplacian_2d(side, pot)
    emax, c = _place_interval(A, k, interval_estimate(side, 2, k, 0.5))
    # lower end just below the lowest eigenvalue: bisect the last energy with
    # an empty count, then leave a margin of 5% of the occupied width
    lam_lap = 2.0 * (2.0 - 2.0 * math.cos(math.pi / (side + 1)))  # lowest Laplacian eigenvalue
    lo, hi = lam_lap + float(pot.min()), emax  # Weyl: no eigenvalue below lo
    for _ in range(7):
        mid = 0.5 * (lo + hi)
        if count_below(A, mid) == 0:
            lo = mid
        else:
            hi = mid
    emin = max(0.0, lo - 0.05 * (emax - lo))
    m0 = int(math.ceil(1.5 * c))
    return Problem(f"laplace2d_{p}_{side}^2", A, None, emin, emax, m0, ne, ratio, 1000 * seed + p,
                   {"target_count": k, "count": c})


def batched_laplace2d(count: int = 512, seed: int = 3, ne: int = 8, ratio: int = 100,
                      side_lo: int = 32, side_hi: int = 256, workers: int | None = None) -> list[Problem]:
    """Independent 2D 5-point Laplacians with V ~ U[0,1]; grid side log-uniform in
    [side_lo, side_hi]; each problem draws a wanted count k ~ U{8..64}.  A
    random potential this strong pulls many more eigenvalues below the
    closed-form estimate on large grids, so Emax is placed by measured counts
    (count_below) until the interval holds about k of them (within
    [max(8, 3k/4), min(64, 5k/4)]), and Emin just below the lowest eigenvalue
    (so the contour is not much wider than the part of the spectrum it
    encloses); M0 = ceil(1.5 count).  Problem p draws from
    the PCG64 stream seeded by (seed, p).  Large batches are built by a pool of
    spawned worker processes."""
    args = [(p, seed, ne, ratio, side_lo, side_hi) for p in range(count)]
    if count < 32:
        return [_laplace2d_problem(a) for a in args]
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    nw = workers or min(32, os.cpu_count() or 4)
    with cf.ProcessPoolExecutor(max_workers=nw, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_laplace2d_problem, args, chunksize=4))


def laplace3d_grad(side: int = 48, count: int = 64, m0: int = 96, ne: int = 8,
                   ratio: int = 100, seed: int = 4) -> Problem:
    """Differentiation workload: 7-point 3D Laplacian + V ~ U[0,0.5]."""
    return laplace3d_potential(side, count, m0, ne, ratio, seed)


def loss_weights(m: int, seed: int) -> np.ndarray:
    """g_k ~ N(0,1) for the eigenvalue loss sum_k g_k lambda_k."""
    return np.random.default_rng([seed, 7]).standard_normal(m)
