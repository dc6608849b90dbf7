"""FP64 CPU oracle for the FEAST contour-filter eigensolver -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (``paper_2002_04807_gb300``) never
imports it and shares no code with it.

The arithmetic lives in ``feast_oracle.c`` (plain C, compiled with gcc by
:func:`build`); this module only marshals numpy arrays into it, except for
:func:`count_below_planes`, an inertia count written with numpy/scipy LAPACK
steps for grids too wide for the C banded count.  Each wrapper
names the step of the method it performs; the C file cites the guide's
sections and states the formulas.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "feast_oracle.c")
_SRC_HERM = os.path.join(_HERE, "feast_oracle_herm.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_HERM))
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_HERM, "-lm"],
                       check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_rho.restype = C.c_double
            _lib.orc_count_below.restype = C.c_long
            _lib.orc_ellipk.restype = C.c_double
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _csr_args(M):
    if M is None:
        return None, None, None
    return _c(M.indptr, np.int32), _c(M.indices, np.int32), _c(M.data, np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------- quadrature
def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_legendre(C.c_int(n), _ptr(x), _ptr(w)):
        raise ValueError("n must be >= 1")
    return x, w


def contour_gauss(ne: int, emin: float, emax: float, ratio: float):
    """Half-contour Gauss nodes z_e and weights w_e (complex arrays)."""
    z = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    lib().orc_contour_gauss(C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(ratio),
                            _ptr(z), _ptr(w))
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def contour_trapezoid(ne: int, emin: float, emax: float, ratio: float):
    """Half-contour trapezoidal (midpoint) nodes z_e and weights w_e (fpm(16)=1)."""
    z = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    lib().orc_contour_trapezoid(C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(ratio),
                                _ptr(z), _ptr(w))
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def contour_zolotarev(ne: int, emin: float, emax: float, eta: float = 0.05):
    """Zolotarev nodes z_e and weights w_e (fpm(16)=2) on the circle through
    Emin, Emax; eta = width of the edge transition band / half-width."""
    z = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    lib().orc_contour_zolotarev(C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(eta),
                                _ptr(z), _ptr(w))
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def ellipk(m: float) -> float:
    return float(lib().orc_ellipk(C.c_double(m)))


def ellipj(u: float, m: float):
    sn, cn = C.c_double(0), C.c_double(0)
    lib().orc_ellipj(C.c_double(u), C.c_double(m), C.byref(sn), C.byref(cn))
    return sn.value, cn.value


def rho(ne: int, emin: float, emax: float, ratio: float, lam, rule: int = 0):
    z = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    L = lib()
    if rule == 2:
        L.orc_contour_zolotarev(C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(0.05), _ptr(z), _ptr(w))
    else:
        nodes = L.orc_contour_trapezoid if rule == 1 else L.orc_contour_gauss
        nodes(C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(ratio), _ptr(z), _ptr(w))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    return np.array([L.orc_rho(C.c_int(ne), _ptr(z), _ptr(w), C.c_double(v)) for v in lam])


# ---------------------------------------------------------------- linear algebra
def csr_mm(A, X):
    X = np.asfortranarray(X, dtype=np.float64)
    m = X.shape[1]
    Y = np.zeros((A.n, m), order="F")
    ip, ix, v = _csr_args(A)
    lib().orc_csr_mm(C.c_int(A.n), _ptr(ip), _ptr(ix), _ptr(v), C.c_int(m), _ptr(X), _ptr(Y))
    return Y


def _cplx_block(R, n):
    R = np.asarray(R, dtype=np.complex128).reshape(n, -1, order="F")
    m = R.shape[1]
    buf = np.empty(2 * n * m)
    buf[0::2] = R.real.ravel(order="F")
    buf[1::2] = R.imag.ravel(order="F")
    return buf, m


def _unblock(buf, n, m):
    return (buf[0::2] + 1j * buf[1::2]).reshape(n, m, order="F")


def shifted_solve(A, B, z: complex, R, method: str = "direct", tol: float = 1e-13,
                  maxit: int = 100000):
    """Solve (z B - A) X = R for a block of right-hand sides (B None = identity)."""
    n = A.n
    rhs, m = _cplx_block(R, n)
    sol = np.zeros_like(rhs)
    ip, ix, v = _csr_args(A)
    bip, bix, bv = _csr_args(B)
    if method == "direct":
        st = lib().orc_shifted_solve_direct(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip),
                                            _ptr(bix), _ptr(bv), C.c_double(z.real),
                                            C.c_double(z.imag), C.c_int(m), _ptr(rhs), _ptr(sol))
        its = None
    else:
        its = np.zeros(m, dtype=np.int32)
        st = lib().orc_shifted_solve_cocg(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip),
                                          _ptr(bix), _ptr(bv), C.c_double(z.real),
                                          C.c_double(z.imag), C.c_int(m), _ptr(rhs), _ptr(sol),
                                          C.c_double(tol), C.c_int(maxit), _ptr(its))
    if st:
        raise RuntimeError(f"shifted solve failed ({st})")
    return _unblock(sol, n, m), its


def jacobi_eig(a):
    a = np.array(a, dtype=np.float64, order="F", copy=True)
    n = a.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    sweeps = lib().orc_jacobi_eig(C.c_int(n), _ptr(a), _ptr(w), _ptr(V))
    return w, V, int(sweeps)


def reduced_gev(Aq, Bq):
    Aq = np.asfortranarray(Aq, dtype=np.float64)
    Bq = np.asfortranarray(Bq, dtype=np.float64)
    m = Aq.shape[0]
    lam = np.zeros(m)
    V = np.zeros((m, m), order="F")
    mk = C.c_int(0)
    info = lib().orc_reduced_gev(C.c_int(m), _ptr(Aq), _ptr(Bq), _ptr(lam), _ptr(V), C.byref(mk))
    k = mk.value
    return info, lam[:k], np.asfortranarray(V[:, :k])


def count_below(A, B, sigma: float) -> int:
    """Number of eigenvalues of (A, B) below sigma (Sylvester inertia)."""
    ip, ix, v = _csr_args(A)
    bip, bix, bv = _csr_args(B)
    r = lib().orc_count_below(C.c_int(A.n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix),
                              _ptr(bv), C.c_double(sigma))
    if r < 0:
        raise RuntimeError("zero pivot in inertia count")
    return int(r)


def count_below_planes(A, B, sigma: float, nb: int) -> int:
    """Number of eigenvalues of (A, B) below sigma by Sylvester's law of
    inertia, for a matrix that is block tridiagonal in blocks of nb rows (the
    planes of a 3D grid): block Gaussian elimination
    S_1 = A_11 - sigma B_11,
    S_k = A_kk - sigma B_kk - C_k S_{k-1}^{-1} C_k^T,  C_k = A_{k,k-1} - sigma B_{k,k-1},
    is a congruence to blockdiag(S_k), so the count is the sum of the negative
    eigenvalues of the S_k (each from its symmetric indefinite LDL^T, whose D
    has 1x1 and 2x2 blocks).  Dense LAPACK steps on nb x nb blocks: for grids
    too wide for the banded count (N bw^2 work) and used only as a test pin.
    Raises if the matrix is not block tridiagonal or a block is singular."""
    import scipy.linalg as sl
    import scipy.sparse as sp

    n = A.n
    if n % nb:
        raise ValueError("nb must divide n")
    M = sp.csr_matrix((A.data, A.indices, A.indptr), shape=(n, n))
    if B is None:
        M = M - sigma * sp.identity(n, format="csr")
    else:
        M = M - sigma * sp.csr_matrix((B.data, B.indices, B.indptr), shape=(n, n))
    M = M.tocsr()
    rows = np.repeat(np.arange(n), np.diff(M.indptr))
    if np.abs(rows // nb - M.indices // nb).max(initial=0) > 1:
        raise ValueError("matrix is not block tridiagonal in blocks of nb rows")
    neg, Sinv = 0, None
    for k in range(n // nb):
        S = M[k * nb:(k + 1) * nb, k * nb:(k + 1) * nb].toarray()
        if k > 0:
            Ck = M[k * nb:(k + 1) * nb, (k - 1) * nb:k * nb]
            S -= np.asarray(Ck @ (Ck @ Sinv).T)  # C S^{-1} C^T (S^{-1} symmetric)
        _, d, _ = sl.ldl(S, lower=True)
        sub = np.diag(d, -1)
        i = 0
        while i < nb:  # eigenvalue signs of the 1x1 and 2x2 pivots
            if i + 1 < nb and sub[i] != 0.0:
                a, b, c = d[i, i], sub[i], d[i + 1, i + 1]
                det = a * c - b * b
                neg += 1 if det < 0 else (2 if a + c < 0 else 0)
                i += 2
            else:
                if d[i, i] == 0.0:
                    raise RuntimeError("singular pivot in inertia count")
                neg += int(d[i, i] < 0)
                i += 1
        Sinv = np.linalg.inv(S)
        Sinv = 0.5 * (Sinv + Sinv.T)
    return int(neg)


def residuals(A, B, X, lam, emin, emax):
    X = np.asfortranarray(X, dtype=np.float64)
    lam = _c(lam, np.float64)
    m = X.shape[1]
    res = np.zeros(m)
    ip, ix, v = _csr_args(A)
    bip, bix, bv = _csr_args(B)
    lib().orc_residuals(C.c_int(A.n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv),
                        C.c_int(m), _ptr(X), _ptr(lam), C.c_double(emin), C.c_double(emax),
                        _ptr(res))
    return res


def filter_block(A, B, ne, emin, emax, ratio, Y, lam=None, rii=False, solver="direct",
                 solve_tol=1e-13, rule=0):
    """One quadrature filter pass on the block Y (n x m): classic form
    sum_e Re(w_e (z_e B - A)^{-1} B Y), or with rii the residual-inverse form
    on (X = Y, lam).  Returns Q (n x m, column-major)."""
    Y = np.asfortranarray(Y, dtype=np.float64)
    n, m = Y.shape
    Q = np.zeros((n, m), order="F")
    lam_a = np.zeros(m) if lam is None else _c(lam, np.float64)
    ip, ix, v = _csr_args(A)
    bip, bix, bv = _csr_args(B)
    st = lib().orc_filter(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv),
                          C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(ratio), C.c_int(m),
                          _ptr(Y), _ptr(lam_a), C.c_int(1 if rii else 0), _ptr(Q),
                          C.c_int(0 if solver == "direct" else 1), C.c_double(solve_tol), C.c_int(rule))
    if st:
        raise RuntimeError("oracle filter failed")
    return Q


def stochastic_count(A, B, ne, emin, emax, ratio, Y, solver="direct", solve_tol=1e-13, rule=0):
    """Stochastic estimate of the eigenvalue count inside the contour (fpm(14)=2;
    ratio = ellipse axis ratio, fpm(18)/100):
    mean over the probe columns of Y of y^T rho(B^{-1}A) y, with its standard
    error.  Returns (estimate, standard_error)."""
    Y = np.asfortranarray(Y, dtype=np.float64)
    n, m = Y.shape
    ip, ix, v = _csr_args(A)
    bip, bix, bv = _csr_args(B)
    est, sem = C.c_double(0.0), C.c_double(0.0)
    st = lib().orc_stochastic_count(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv),
                                    C.c_int(ne), C.c_double(emin), C.c_double(emax), C.c_double(ratio),
                                    C.c_int(m), _ptr(Y), C.c_int(0 if solver == "direct" else 1),
                                    C.c_double(solve_tol), C.byref(est), C.byref(sem), C.c_int(rule))
    if st:
        raise RuntimeError("oracle stochastic count failed")
    return est.value, sem.value


def eig_grad(A, X, w):
    """grad[p] = sum_k w_k X[i_p,k] X[j_p,k] over the stored entries of A."""
    X = np.asfortranarray(X, dtype=np.float64)
    w = _c(w, np.float64)
    ip, ix, _ = _csr_args(A)
    grad = np.zeros(A.nnz)
    lib().orc_eig_grad(C.c_int(A.n), _ptr(ip), _ptr(ix), C.c_int(X.shape[1]), _ptr(X), _ptr(w), _ptr(grad))
    return grad


# ---------------------------------------------------------------- FEAST
def feastinit():
    """fpm defaults of the guide's parameter table (C indexing fpm[i-1])."""
    fpm = np.zeros(64, dtype=np.int32)
    defaults = {1: 0, 2: 8, 3: 12, 4: 20, 5: 0, 6: 1, 8: 16, 10: 1, 14: 0, 15: 2, 16: 0, 18: 30,
                19: 0, 40: 0, 41: 1, 42: 1, 43: 0, 45: 1, 46: 40}
    for i, v in defaults.items():
        fpm[i - 1] = v
    return fpm


def feast_scsr(A, B, emin, emax, m0, Y0=None, X0=None, ne=8, ratio=30, tol_exp=10, maxloop=20,
               solver="direct", solve_tol=1e-13, rii=False, rule=0):
    """Plain FP64 FEAST on a real symmetric CSR problem.

    Returns a dict with E (inside first, ascending), X (n x m0', column-major),
    res, M, loop, epsout, info, m0 (kept size), per-loop trace and max-residual.
    """
    n = A.n
    fpm = feastinit()
    fpm[1] = ne
    fpm[2] = tol_exp
    fpm[3] = maxloop
    fpm[17] = ratio
    fpm[15] = rule
    X = np.zeros((n, m0), order="F")
    if X0 is not None:
        fpm[4] = 1
        X[:] = X0
        Y = np.zeros((n, m0), order="F")
    else:
        Y = np.asfortranarray(Y0, dtype=np.float64)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M = C.c_int(0)
    loop = C.c_int(0)
    eps = C.c_double(0)
    m0io = C.c_int(m0)
    th = np.zeros(maxloop + 2)
    mh = np.zeros(maxloop + 2)
    it = C.c_long(0)
    ip, ix, v = _csr_args(A)
    bip, bix, bv = _csr_args(B)
    info = lib().orc_feast_scsr(
        C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv), _ptr(fpm),
        C.c_double(emin), C.c_double(emax), C.byref(m0io), _ptr(Y), _ptr(E), _ptr(X), _ptr(res),
        C.byref(M), C.byref(loop), C.byref(eps), C.c_int(0 if solver == "direct" else 1),
        C.c_double(solve_tol), C.c_int(1 if rii else 0), _ptr(th), _ptr(mh), C.byref(it))
    k = m0io.value
    return {"info": int(info), "E": E[:k].copy(), "X": np.asfortranarray(X[:, :k]),
            "res": res[:k].copy(), "M": M.value, "loop": loop.value, "epsout": eps.value,
            "m0": k, "trace": th[: loop.value + 1].copy(), "maxres": mh[: loop.value + 1].copy(),
            "inner_iters": it.value}


# ---------------------------------------------------------------- complex Hermitian (feast_oracle_herm.c)
def _zcsr_args(M):
    if M is None:
        return None, None, None
    return _c(M.indptr, np.int32), _c(M.indices, np.int32), _c(M.data, np.complex128)


def _zf(a):
    return np.asfortranarray(a, dtype=np.complex128)


def h_jacobi_eig(a):
    """Hermitian Jacobi: (w ascending, V unitary, status)."""
    a = _zf(a).copy(order="F")
    n = a.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().orc_h_jacobi_eig(C.c_int(n), _ptr(a), _ptr(w), _ptr(V))
    return w, V, int(st)


def h_reduced_gev(Aq, Bq):
    """Reduced generalized Hermitian problem: (info, lam[:mk], V[:, :mk])."""
    m = Aq.shape[0]
    Aq, Bq = _zf(Aq), _zf(Bq)
    lam = np.zeros(m)
    V = np.zeros((m, m), dtype=np.complex128, order="F")
    mk = C.c_int(0)
    info = lib().orc_h_reduced_gev(C.c_int(m), _ptr(Aq), _ptr(Bq), _ptr(lam), _ptr(V), C.byref(mk))
    k = mk.value
    return int(info), lam[:k].copy(), V[:, :k].copy()


def h_shifted_solve(A, B, z: complex, R):
    """(z B - A) X = R by banded LU without pivoting."""
    R = _zf(R)
    n, m = R.shape
    X = np.zeros((n, m), dtype=np.complex128, order="F")
    ip, ix, v = _zcsr_args(A)
    bip, bix, bv = _zcsr_args(B)
    st = lib().orc_h_shifted_solve(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv),
                                   C.c_double(z.real), C.c_double(z.imag), C.c_int(m), _ptr(R), _ptr(X))
    if st:
        raise RuntimeError("oracle Hermitian shifted solve failed")
    return X


def h_filter(A, B, ne, emin, emax, ratio, Y, rule=0):
    """Q = sum_e (1/2)[w_e G(z_e) + conj(w_e) G(conj z_e)] B Y (ratio = fpm(18)/100)."""
    Y = _zf(Y)
    n, m = Y.shape
    Q = np.zeros((n, m), dtype=np.complex128, order="F")
    ip, ix, v = _zcsr_args(A)
    bip, bix, bv = _zcsr_args(B)
    st = lib().orc_h_filter(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv), C.c_int(ne),
                            C.c_double(emin), C.c_double(emax), C.c_double(ratio), C.c_int(rule), C.c_int(m),
                            _ptr(Y), _ptr(Q))
    if st:
        raise RuntimeError("oracle Hermitian filter failed")
    return Q


def feast_hcsr(A, B, emin, emax, m0, Y0=None, X0=None, ne=8, ratio=100, tol_exp=10, maxloop=20, rule=0):
    """Plain FP64 FEAST on a complex Hermitian CSR problem (classic filter).
    Returns a dict with E, X (n x m0', complex), res, M, loop, epsout, info, m0."""
    n = A.n
    fpm = feastinit()
    fpm[1], fpm[2], fpm[3], fpm[15], fpm[17] = ne, tol_exp, maxloop, rule, ratio
    X = np.zeros((n, m0), dtype=np.complex128, order="F")
    if X0 is not None:
        fpm[4] = 1
        X[:] = X0
        Y = np.zeros((n, m0), dtype=np.complex128, order="F")
    else:
        Y = _zf(Y0)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, eps, m0io = C.c_int(0), C.c_int(0), C.c_double(0), C.c_int(m0)
    ip, ix, v = _zcsr_args(A)
    bip, bix, bv = _zcsr_args(B)
    info = lib().orc_feast_hcsr(C.c_int(n), _ptr(ip), _ptr(ix), _ptr(v), _ptr(bip), _ptr(bix), _ptr(bv), _ptr(fpm),
                                C.c_double(emin), C.c_double(emax), C.byref(m0io), _ptr(Y), _ptr(E), _ptr(X),
                                _ptr(res), C.byref(M), C.byref(loop), C.byref(eps))
    k = m0io.value
    return {"info": int(info), "E": E[:k].copy(), "X": np.asfortranarray(X[:, :k]), "res": res[:k].copy(),
            "M": M.value, "loop": loop.value, "epsout": eps.value, "m0": k}
