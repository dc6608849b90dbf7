"""Pins of the FP64 CPU oracle against facts fixed outside it.

Each test checks one oracle step against a closed form, a worked example the
FEAST guide prints, brute force or a library routine on small inputs, so that a
dropped term, a wrong sign, index or transposed operand fails somewhere.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import feast_workloads as fw
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _angles(U, V):
    """Sine of the largest principal angle between two column spaces of equal
    dimension: ||(I - P_V) Q_U||_2 with orthonormal bases (no arccos round-off)."""
    qu, _ = np.linalg.qr(U)
    qv, _ = np.linalg.qr(V)
    return float(np.linalg.norm(qu - qv @ (qv.T @ qu), 2))


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 24, 56])
def test_gauss_legendre_exact_on_polynomials(n):
    x, w = O.gauss_legendre(n)
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * x ** p) - exact) < 1e-13, p
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(x), xr, atol=1e-14) and np.allclose(w[np.argsort(x)], wr, atol=1e-14)


@pytest.mark.parametrize("ne", [1, 3, 8, 16])
def test_circle_filter_is_one_at_centre(ne):
    # on a circle (ratio 1) w_e/(z_e - c) = omega_e/2, so rho(c) = sum omega_e / 2 = 1
    assert abs(O.rho(ne, -2.0, 4.0, 1.0, 1.0)[0] - 1.0) < 1e-14


@pytest.mark.parametrize("ratio", [0.3, 1.0])
def test_filter_matches_contour_integral(ratio):
    # rho(lambda) approximates (1/pi) Im int_0^pi z'(t)/(z(t)-lambda) dt, an
    # independent adaptive quadrature of the same half-contour integral; for a
    # rule of many nodes it is the indicator of [Emin, Emax].
    emin, emax = 1.0, 3.0
    c, r = 2.0, 1.0

    def integral(lam):
        f = lambda t: ((-r * math.sin(t) + 1j * ratio * r * math.cos(t))
                       / (c + r * math.cos(t) + 1j * ratio * r * math.sin(t) - lam)).imag
        return scipy.integrate.quad(f, 0.0, math.pi, limit=400, epsabs=1e-13)[0] / math.pi

    for lam in [1.5, 2.0, 2.7, 0.0, 3.6, 10.0]:
        ref = integral(lam)
        ind = 1.0 if emin < lam < emax else 0.0
        assert abs(ref - ind) < 1e-9
        assert abs(O.rho(48, emin, emax, ratio, lam)[0] - ref) < 5e-6 * (1 if ratio == 1.0 else 20)


def test_filter_edges_and_decay():
    lam = np.array([-5.0, 0.0, 1.0, 2.0, 3.0, 4.0, 8.0])
    rho = O.rho(8, 1.0, 3.0, 1.0, lam)
    assert abs(rho[2] - 0.5) < 1e-12 and abs(rho[4] - 0.5) < 1e-12  # ends of the interval
    assert abs(rho[3] - 1.0) < 1e-14
    assert abs(rho[0]) < 1e-4 and abs(rho[-1]) < 1e-4


@pytest.mark.parametrize("ne", [1, 2, 3, 4, 8, 16])
def test_trapezoid_filter_closed_form_on_circle(ne):
    """The 2 ne equally spaced midpoints of a circle are the roots of
    t^(2 ne) = -1, and the trapezoidal sum of the resolvent is then exactly
    rho(lambda) = 1 / (1 + t^(2 ne)), t = (lambda - c) / r."""
    emin, emax = -1.0, 3.0
    c, r = 1.0, 2.0
    lam = np.linspace(-3.0, 5.0, 41)
    t = (lam - c) / r
    ref = 1.0 / (1.0 + t ** (2 * ne))
    got = O.rho(ne, emin, emax, 1.0, lam, rule=1)
    assert np.abs(got - ref).max() < 1e-13


@pytest.mark.parametrize("ratio", [0.3, 1.0])
def test_trapezoid_filter_converges_to_contour_integral(ratio):
    """On an ellipse the trapezoidal sum converges (geometrically, the
    integrand being periodic and analytic) to the same half-contour integral."""
    emin, emax = 1.0, 3.0
    c, r = 2.0, 1.0
    for lam in [1.5, 2.0, 2.7, 0.0, 3.6, 10.0]:
        f = lambda t: ((-r * math.sin(t) + 1j * ratio * r * math.cos(t))
                       / (c + r * math.cos(t) + 1j * ratio * r * math.sin(t) - lam)).imag
        ref = scipy.integrate.quad(f, 0.0, math.pi, limit=400, epsabs=1e-13)[0] / math.pi
        assert abs(O.rho(400, emin, emax, ratio, lam, rule=1)[0] - ref) < 1e-6


def test_trapezoid_weights_sum():
    """sum_e Re(w_e) = (r a / ne) sum cos(theta_e) = 0 and sum Im(w_e) equals the
    midpoint rule of (r/pi) int_0^pi sin = 2 r / pi up to its O(ne^-2) error."""
    z, w = O.contour_trapezoid(64, 0.0, 2.0, 0.5)
    assert abs(w.real.sum()) < 1e-14
    assert abs(w.imag.sum() - 2.0 / math.pi) < 1e-4
    assert np.all(z.imag > 0) and np.all(np.diff(z.real) < 0)


def test_feast_with_trapezoid_rule_matches_closed_form():
    """1D Laplacian, 31 eigenvalues in [0, 0.01] (closed form), trapezoidal
    nodes (fpm(16)=1)."""
    p = fw.tridiag_1d(n=1000, emin=0.0, emax=0.01, m0=48, ratio=30)
    ref = O.feast_scsr(p.A, None, 0.0, 0.01, 48, Y0=p.y0(), ne=8, ratio=30, tol_exp=11, rule=1)
    lam = 2 - 2 * np.cos(np.arange(1, 32) * np.pi / 1001)
    assert ref["info"] == 0 and ref["M"] == 31
    assert np.abs(ref["E"][:31] - lam).max() < 1e-13


# ------------------------------------------------------------------ linear algebra
def _rand_sym_csr(n, bw, rng, shift=0.0):
    d = np.zeros((n, n))
    for k in range(bw + 1):
        v = rng.standard_normal(n - k)
        d += np.diag(v, k) + (np.diag(v, -k) if k else 0)
    d += shift * np.eye(n)
    return fw.csr_from_dense(d), d


def test_csr_mm_matches_dense():
    rng = np.random.default_rng(0)
    A, d = _rand_sym_csr(30, 3, rng)
    X = rng.standard_normal((30, 4))
    assert np.allclose(O.csr_mm(A, X), d @ X, atol=1e-13)


@pytest.mark.parametrize("method", ["direct", "cocg"])
@pytest.mark.parametrize("gen", [False, True])
def test_shifted_solve(method, gen):
    rng = np.random.default_rng(1)
    n = 40
    A, da = _rand_sym_csr(n, 2, rng)
    if gen:
        B = fw.diagonal_csr(rng.uniform(1, 2, n))
        db = B.to_dense()
    else:
        B, db = None, np.eye(n)
    z = 0.3 + 0.7j
    R = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    X, _ = O.shifted_solve(A, B, z, R, method=method, tol=1e-14)
    ref = np.linalg.solve(z * db - da, R)
    assert np.abs(X - ref).max() < 1e-10 * np.abs(ref).max()


def test_jacobi_matches_eigh():
    rng = np.random.default_rng(2)
    for n in [1, 2, 7, 40]:
        a = rng.standard_normal((n, n))
        a = a + a.T
        w, V, _ = O.jacobi_eig(a)
        wr = np.linalg.eigvalsh(a)
        assert np.allclose(w, wr, atol=1e-12 * max(1, abs(wr).max()))
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)
        assert np.allclose(a @ V, V * w, atol=1e-11 * max(1, abs(wr).max()))


def test_reduced_gev_matches_scipy():
    rng = np.random.default_rng(3)
    m = 12
    a = rng.standard_normal((m, m)); a = a + a.T
    g = rng.standard_normal((m, m)); b = g @ g.T + 0.5 * np.eye(m)
    info, lam, V = O.reduced_gev(a, b)
    assert info == 0 and len(lam) == m
    assert np.allclose(lam, scipy.linalg.eigh(a, b, eigvals_only=True), atol=1e-11)
    assert np.allclose(V.T @ b @ V, np.eye(m), atol=1e-11)


def test_reduced_gev_rank_deficient_and_indefinite():
    rng = np.random.default_rng(4)
    m = 8
    Q = rng.standard_normal((50, 5))
    Q = np.hstack([Q, Q[:, :3] @ rng.standard_normal((3, 3))])  # rank 5 of 8
    a = rng.standard_normal((50, 50)); a = a + a.T
    info, lam, V = O.reduced_gev(Q.T @ a @ Q, Q.T @ Q)
    assert info == 0 and len(lam) == 5
    # the Ritz values of the 5-dimensional span
    qq, _ = np.linalg.qr(Q[:, :5])
    assert np.allclose(lam, np.linalg.eigvalsh(qq.T @ a @ qq), atol=1e-8)
    info, _, _ = O.reduced_gev(np.eye(3), -np.eye(3))
    assert info == -3


def test_inertia_counts():
    rng = np.random.default_rng(5)
    A, d = _rand_sym_csr(60, 4, rng)
    B = fw.diagonal_csr(rng.uniform(1, 2, 60))
    ev = scipy.linalg.eigh(d, B.to_dense(), eigvals_only=True)
    for s in [-3.0, -0.1, 0.4, 2.5]:
        assert O.count_below(A, B, s) == int(np.sum(ev < s))
    L = fw.laplacian_1d(1000)
    k = np.arange(1, 1001)
    lam = 2 - 2 * np.cos(k * np.pi / 1001)
    assert O.count_below(L, None, 0.01) == 31 == int(np.sum(lam < 0.01))


def test_residual_formula():
    rng = np.random.default_rng(6)
    A, d = _rand_sym_csr(20, 2, rng)
    B = fw.diagonal_csr(rng.uniform(1, 2, 20))
    X = rng.standard_normal((20, 3))
    lam = np.array([0.1, -0.5, 2.0])
    res = O.residuals(A, B, X, lam, -1.0, 4.0)
    db = B.to_dense()
    ref = np.linalg.norm(d @ X - db @ X * lam, axis=0) / (4.0 * np.linalg.norm(db @ X, axis=0))
    assert np.allclose(res, ref, rtol=1e-13)


# ------------------------------------------------------------------ FEAST
def test_helloworld_worked_example():
    g = json.load(open(os.path.join(GOLD, "helloworld.json")))
    run, exp = g["run"], g["expected"]
    dense = np.array(g["matrix_dense_rows"], dtype=float)
    assert np.allclose(np.linalg.eigvalsh(dense), g["eigenvalues_all"])
    c = g["csr_1based"]
    IA = np.array(c["IA"]) - 1
    JA = np.array(c["JA"]) - 1
    A = fw.CSR(4, IA.astype(np.int32), JA.astype(np.int32), np.array(c["sA"], dtype=float))
    assert np.array_equal(A.to_dense(), dense)
    Y0 = fw.gaussian_block(4, run["M0"], 0)
    for solver in ["direct", "cocg"]:
        r = O.feast_scsr(A, None, run["Emin"], run["Emax"], run["M0"], Y0=Y0, ne=run["Ne"],
                         ratio=run["ratio_percent"], tol_exp=12, solver=solver)
        assert r["info"] == 0 and r["M"] == exp["M"]
        assert np.allclose(r["E"][:2], exp["E"], atol=1e-12)
        assert abs(r["E"][:2].sum() - exp["trace"]) < 1e-12
        assert r["res"][:2].max() < exp["max_residual_below"]


def test_laplacian_1d_closed_form():
    p = fw.tridiag_1d()
    r = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=p.ne, ratio=p.ratio,
                     tol_exp=10)
    assert r["info"] == 0 and r["M"] == 31
    k = np.arange(1, 32)
    lam = 2 - 2 * np.cos(k * np.pi / 1001)
    assert np.abs(r["E"][:31] - lam).max() <= 1e-10 * lam.max()
    assert r["res"][:31].max() <= 1e-10
    i = np.arange(1, 1001)[:, None]
    xs = np.sqrt(2 / 1001) * np.sin(i * k[None, :] * np.pi / 1001)
    X = r["X"][:, :31]
    assert np.abs(X.T @ X - np.eye(31)).max() < 1e-12
    # per-eigenvalue eigenvectors are unique here (simple spectrum): compare up to sign
    dots = np.abs(np.sum(X * xs, axis=0))
    assert np.all(1 - dots < 1e-8)
    # outside Ritz values lie outside the interval and inside ones are all found
    assert np.all((r["E"][31:] < p.emin) | (r["E"][31:] > p.emax))


def test_constant_potential_3d_degenerate_clusters():
    side, v0 = 10, 0.3
    mu = 2 - 2 * np.cos(np.arange(1, side + 1) * np.pi / (side + 1))
    lev = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel()) + v0
    # interval closing just above the 4th distinct level (includes 3-fold and 6-fold clusters)
    distinct = np.unique(np.round(lev, 12))
    emax = 0.5 * (distinct[3] + distinct[4])
    want = lev[lev <= emax]
    p = fw.laplace3d_constant(side, v0, emax, m0=int(1.6 * len(want)) + 4)
    r = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=100, tol_exp=11)
    assert r["info"] == 0 and r["M"] == len(want)
    assert np.abs(r["E"][: r["M"]] - want).max() < 1e-10 * want.max()
    # subspace of every cluster against the closed-form eigenvectors
    s = np.sin(np.arange(1, side + 1)[:, None] * np.arange(1, side + 1)[None, :] * np.pi / (side + 1))
    s *= np.sqrt(2 / (side + 1))
    full = np.einsum("ia,jb,kc->ijkabc", s, s, s).reshape(side ** 3, -1)
    eig = (mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel() + v0
    sel = eig <= emax
    assert _angles(r["X"][:, : r["M"]], full[:, sel]) < 1e-8


def test_generalized_problem_against_dense_and_inertia():
    rng = np.random.default_rng(7)
    A = fw.stencil27_spd(7, rng)
    B = fw.diagonal_csr(rng.uniform(1.0, 2.0, A.n))
    ev = scipy.linalg.eigh(A.to_dense(), B.to_dense(), eigvals_only=True)
    emax = 0.5 * (ev[19] + ev[20])
    assert O.count_below(A, B, emax) == 20
    Y0 = fw.gaussian_block(A.n, 32, 2)
    for solver in ["direct", "cocg"]:
        r = O.feast_scsr(A, B, 0.0, emax, 32, Y0=Y0, ne=16, ratio=100, tol_exp=11, solver=solver)
        assert r["info"] == 0 and r["M"] == 20
        assert np.abs(r["E"][:20] - ev[:20]).max() < 1e-10 * ev[19]
        X = r["X"][:, :20]
        assert np.abs(X.T @ B.to_dense() @ X - np.eye(20)).max() < 1e-11


def test_generalized_nondiagonal_b_against_dense_and_inertia():
    """A non-diagonal SPD B (7-point mass-like pattern): the oracle's FEAST
    (both solver modes) against the dense generalized eigensolve, its count
    against Sylvester inertia, and X^T B X = I."""
    p = fw.laplace3d_general_b(side=8, count=20, m0=32)
    Bd = p.B.to_dense()
    assert np.abs(Bd - np.diag(np.diag(Bd))).max() > 0.05  # genuinely non-diagonal
    ev = scipy.linalg.eigh(p.A.to_dense(), Bd, eigvals_only=True)
    assert O.count_below(p.A, p.B, p.emax) == 20 == int(np.sum(ev < p.emax))
    for solver in ["direct", "cocg"]:
        r = O.feast_scsr(p.A, p.B, 0.0, p.emax, 32, Y0=p.y0(), ne=8, ratio=100, tol_exp=11, solver=solver)
        assert r["info"] == 0 and r["M"] == 20
        assert np.abs(r["E"][:20] - ev[:20]).max() < 1e-10 * ev[19]
        X = r["X"][:, :20]
        assert np.abs(X.T @ Bd @ X - np.eye(20)).max() < 1e-11


@pytest.mark.parametrize("side,seed", [(6, 1), (8, 2), (10, 3)])
def test_count_below_planes_matches_banded_and_dense(side, seed):
    """The block-tridiagonal inertia count (planes of a 3D grid) equals the
    banded LDL^T count and the dense eigenvalue count, at shifts below the
    spectrum, between eigenvalues and deep inside it; also for a 27-point
    generalized pencil."""
    p = fw.laplace3d_potential(side=side, count=20, m0=30, seed=seed)
    ev = np.linalg.eigvalsh(p.A.to_dense())
    for s in [0.0, 0.5 * (ev[5] + ev[6]), p.emax, 1.3]:
        want = int(np.sum(ev < s))
        assert O.count_below_planes(p.A, None, s, side * side) == want == O.count_below(p.A, None, s)
    rng = np.random.default_rng(seed)
    A = fw.stencil27_spd(side, rng)
    B = fw.diagonal_csr(rng.uniform(1, 2, A.n))
    d = 1 / np.sqrt(B.data)
    evg = np.linalg.eigvalsh(d[:, None] * A.to_dense() * d[None, :])
    for k in (3, 25):
        s = 0.5 * (evg[k - 1] + evg[k])
        assert O.count_below_planes(A, B, s, side * side) == k == O.count_below(A, B, s)


def test_count_below_planes_rejects_wide_coupling():
    A = fw.laplacian_2d(4)  # couples rows i and i + 4: two blocks of 2 rows apart
    with pytest.raises(ValueError):
        O.count_below_planes(A, None, 1.0, 2)


def test_bench_workload_count_golden_is_current():
    """The stored eigenvalue count of the 64^3 bench workload
    (tests/golden/laplace3d_64_count.json, written by the committed
    make_laplace3d_64_count.py through the oracle's block inertia count) was
    taken on exactly the matrix and interval the generator builds today."""
    import hashlib

    g = json.load(open(os.path.join(GOLD, "laplace3d_64_count.json")))
    p = fw.laplace3d_potential(side=64, count=100, m0=150, ne=8, ratio=200, seed=1)
    h = hashlib.sha1()
    for a in (p.A.indptr, p.A.indices, p.A.data):
        h.update(a.tobytes())
    fp = g["fingerprint"]
    assert (fp["n"], fp["nnz"], fp["emin"], fp["emax"], fp["csr_sha1"]) == (
        p.n, p.A.nnz, repr(p.emin), repr(p.emax), h.hexdigest())
    # nothing lies below Emin = 0: A = L + diag(V), L SPD and V >= 0 (Weyl)
    assert g["count_below_emin"] == 0
    assert g["count_in_interval"] == g["count_below_emax"] > 0


def test_rii_form_equals_classic_form():
    p = fw.laplace3d_potential(side=8, count=20, m0=32, seed=11)
    Y0 = p.y0()
    a = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=Y0, ne=8, ratio=100, tol_exp=11)
    b = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=Y0, ne=8, ratio=100, tol_exp=11, rii=True)
    assert a["info"] == b["info"] == 0 and a["M"] == b["M"]
    assert np.abs(a["E"][: a["M"]] - b["E"][: b["M"]]).max() < 1e-11
    # with exact solves the two forms give the same iterates
    assert len(a["maxres"]) == len(b["maxres"])
    ev = np.linalg.eigvalsh(p.A.to_dense())
    assert np.abs(a["E"][: a["M"]] - ev[: a["M"]]).max() < 1e-11
    assert O.count_below(p.A, None, p.emax) == a["M"]


def test_initial_guess_converges_immediately():
    p = fw.tridiag_1d(n=200, emax=0.05)
    r = O.feast_scsr(p.A, None, p.emin, p.emax, 24, Y0=fw.gaussian_block(200, 24, 0), ratio=100)
    assert r["info"] == 0
    X0 = np.zeros((200, 24), order="F")
    X0[:, : r["m0"]] = r["X"]
    r2 = O.feast_scsr(p.A, None, p.emin, p.emax, 24, X0=X0, ratio=100)
    assert r2["info"] == 0 and r2["loop"] <= 1 and r2["M"] == r["M"]


def test_argument_errors():
    A = fw.laplacian_1d(10)
    assert O.feast_scsr(A, None, 1.0, 0.5, 4, Y0=np.zeros((10, 4)))["info"] == 200
    assert O.feast_scsr(A, None, 0.0, 0.5, 11, Y0=np.zeros((10, 11)))["info"] == 201


def test_no_eigenvalue_in_interval():
    A = fw.laplacian_1d(50)
    r = O.feast_scsr(A, None, 5.0, 6.0, 8, Y0=fw.gaussian_block(50, 8, 1), ratio=100)
    assert r["info"] == 1 and r["M"] == 0


def _sym_pair_indices(A, p):
    """Stored index of the transposed entry of entry p (same index on the diagonal)."""
    i = int(np.searchsorted(A.indptr, p, side="right") - 1)
    j = int(A.indices[p])
    row = slice(A.indptr[j], A.indptr[j + 1])
    q = A.indptr[j] + int(np.nonzero(A.indices[row] == i)[0][0])
    return i, j, q


@pytest.mark.parametrize("gen", [False, True])
def test_eig_grad_matches_finite_differences(gen):
    # d(sum_k g_k lambda_k)/d(a_ij) summed over the symmetric pair (i,j),(j,i)
    # equals the symmetric central difference of dense eigenvalues
    rng = np.random.default_rng(11)
    A = fw.laplace3d_potential(side=4, count=5, m0=8, seed=3).A
    n = A.n
    B = fw.diagonal_csr(rng.uniform(1, 2, n)) if gen else None
    db = np.eye(n) if B is None else B.to_dense()
    lam, X = scipy.linalg.eigh(A.to_dense(), db)
    k = 10
    g = rng.standard_normal(k)
    ga = O.eig_grad(A, X[:, :k], g)
    gb = O.eig_grad(B, X[:, :k], -g * lam[:k]) if gen else None
    h = 1e-6
    for p in rng.choice(A.nnz, 12, replace=False):
        i, j, q = _sym_pair_indices(A, p)
        E = np.zeros((n, n))
        E[i, j] += h
        if i != j:
            E[j, i] += h
        lp = scipy.linalg.eigh(A.to_dense() + E, db, eigvals_only=True)[:k]
        lm = scipy.linalg.eigh(A.to_dense() - E, db, eigvals_only=True)[:k]
        fd = np.dot(g, lp - lm) / (2 * h)
        an = ga[p] + (ga[q] if q != p else 0.0)
        assert abs(fd - an) < 1e-6 + 1e-6 * abs(fd), (p, fd, an)
    if gen:
        for i in rng.choice(n, 6, replace=False):
            E = np.zeros((n, n))
            E[i, i] = h
            lp = scipy.linalg.eigh(A.to_dense(), db + E, eigvals_only=True)[:k]
            lm = scipy.linalg.eigh(A.to_dense(), db - E, eigvals_only=True)[:k]
            fd = np.dot(g, lp - lm) / (2 * h)
            assert abs(fd - gb[i]) < 1e-6 + 1e-6 * abs(fd)


# ------------------------------------------------------------------ stochastic count (fpm(14)=2)
def _rho_dense(ne, emin, emax, ratio, lam):
    """rho(lambda) = sum_e Re(w_e / (z_e - lambda)) from the pinned nodes."""
    z, w = O.contour_gauss(ne, emin, emax, ratio)
    return np.array([np.sum((w / (z - l)).real) for l in lam])


@pytest.mark.parametrize("gen", [False, True])
def test_stochastic_count_matches_dense_trace_formula(gen):
    """y^T rho(B^{-1}A) y by contour solves equals the dense spectral formula
    y^T X diag(rho(lambda)) X^T B y (X^T B X = I) for every probe."""
    rng = np.random.default_rng(21)
    A = fw.laplacian_2d(12, rng.uniform(0, 1, (12, 12)))
    B = fw.diagonal_csr(rng.uniform(1, 2, A.n)) if gen else None
    db = np.eye(A.n) if B is None else B.to_dense()
    lam, X = scipy.linalg.eigh(A.to_dense(), db)
    emin, emax = 0.0, 0.5 * (lam[14] + lam[15])
    Y = rng.standard_normal((A.n, 10))
    est, sem = O.stochastic_count(A, B, 8, emin, emax, 1.0, Y)
    r = _rho_dense(8, emin, emax, 1.0, lam)
    t = np.einsum("ij,ij->j", Y, X @ (r[:, None] * (X.T @ (db @ Y))))
    assert abs(est - t.mean()) < 1e-11 * abs(t.mean())
    assert abs(sem - t.std(ddof=1) / np.sqrt(10)) < 1e-9 * t.std()


def test_stochastic_count_estimates_eigenvalue_count():
    """With many probes and a sharp filter the estimate lands on the count of
    eigenvalues inside (inertia), within five standard errors."""
    rng = np.random.default_rng(22)
    A = fw.laplacian_2d(20, rng.uniform(0, 1, (20, 20)))
    lam = np.linalg.eigvalsh(A.to_dense())
    emax = 0.5 * (lam[29] + lam[30])
    cnt = O.count_below(A, None, emax)
    assert cnt == 30
    Y = rng.standard_normal((A.n, 400))
    est, sem = O.stochastic_count(A, None, 32, 0.0, emax, 1.0, Y)
    trace = np.sum(_rho_dense(32, 0.0, emax, 1.0, lam))
    assert abs(trace - cnt) < 0.05
    assert 0.0 < sem < 1.0
    assert abs(est - cnt) < 5 * sem


# ------------------------------------------------------------------ complex Hermitian oracle (zfeast_hcsr)
def test_hermitian_jacobi_matches_eigh():
    rng = np.random.default_rng(41)
    m = 30
    g = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    a = g + g.conj().T
    w, V, st = O.h_jacobi_eig(a)
    assert st == 0
    ref = np.linalg.eigvalsh(a)
    assert np.abs(w - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(V.conj().T @ V - np.eye(m)).max() < 1e-13
    assert np.abs(a @ V - V * w).max() < 1e-12 * np.abs(ref).max()


def test_hermitian_shifted_solve_matches_dense():
    rng = np.random.default_rng(42)
    A = fw.hermitian_banded(60, 3, rng)
    B = fw.zcsr_from_dense(np.diag(rng.uniform(1, 2, 60)).astype(np.complex128))
    R = rng.standard_normal((60, 4)) + 1j * rng.standard_normal((60, 4))
    for z in (0.3 + 0.7j, 0.3 - 0.7j, -2.0 + 0.01j):
        X = O.h_shifted_solve(A, B, z, R)
        ref = np.linalg.solve(z * B.to_dense() - A.to_dense(), R)
        assert np.abs(X - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("gen", [False, True])
def test_hermitian_filter_matches_dense_spectral_formula(gen):
    """Q = rho(B^{-1}A) Y = X diag(rho(lambda)) X^H B Y (X^H B X = I): both
    halves of the contour are needed once A is complex."""
    rng = np.random.default_rng(43)
    A = fw.hermitian_banded(80, 4, rng, shift=6.0)
    B = fw.zcsr_from_dense(np.diag(rng.uniform(1, 2, 80)).astype(np.complex128)) if gen else None
    db = np.eye(80) if B is None else B.to_dense()
    lam, X = scipy.linalg.eigh(A.to_dense(), db)
    emin, emax = lam[10] - 0.3, 0.5 * (lam[25] + lam[26])
    Y = rng.standard_normal((80, 5)) + 1j * rng.standard_normal((80, 5))
    Q = O.h_filter(A, B, 8, emin, emax, 1.0, Y)
    r = _rho_dense(8, emin, emax, 1.0, lam)
    ref = X @ (r[:, None] * (X.conj().T @ (db @ Y)))
    assert np.abs(Q - ref).max() < 1e-11 * np.abs(ref).max()
    # dropping the conjugate half (as the real symmetric filter may) is wrong here
    z, w = O.contour_gauss(8, emin, emax, 1.0)
    half = sum(O.h_shifted_solve(A, B, complex(ze), db @ Y) * we for ze, we in zip(z, w))
    assert np.abs(half.real - ref.real).max() > 1e-3 * np.abs(ref).max()


def test_hermitian_feast_flux_ring_closed_form():
    """Ring of 200 sites with flux phi: lambda_m = 2 - 2 cos(2 pi m / n + phi),
    eigenvectors the plane waves exp(i (2 pi m / n) j) / sqrt(n)."""
    n, phi = 200, 0.013
    A = fw.flux_ring(n, phi)
    mm = np.arange(n)
    lam = 2 - 2 * np.cos(2 * np.pi * mm / n + phi)
    order = np.argsort(lam)
    lam_s = lam[order]
    emax = 0.5 * (lam_s[20] + lam_s[21])
    Y0 = fw.complex_gaussian_block(n, 32, 0)
    ref = O.feast_hcsr(A, None, 0.0, emax, 32, Y0=Y0, ne=8, ratio=100, tol_exp=12)
    assert ref["info"] == 0 and ref["M"] == 21
    assert np.abs(ref["E"][:21] - lam_s[:21]).max() < 1e-13
    assert ref["res"][:21].max() < 1e-12
    waves = np.exp(1j * np.outer(np.arange(n), 2 * np.pi * mm[order[:21]] / n)) / np.sqrt(n)
    X = ref["X"][:, :21]
    assert np.abs(X.conj().T @ X - np.eye(21)).max() < 1e-12
    qx, _ = np.linalg.qr(X)
    assert np.linalg.norm(waves - qx @ (qx.conj().T @ waves), 2) < 1e-9


def test_hermitian_feast_generalized_matches_dense():
    rng = np.random.default_rng(44)
    A = fw.hermitian_banded(300, 5, rng, shift=8.0)
    B = fw.zcsr_from_dense(np.diag(rng.uniform(1, 2, 300)).astype(np.complex128))
    lam = scipy.linalg.eigh(A.to_dense(), B.to_dense(), eigvals_only=True)
    emin, emax = lam[0] - 0.5, 0.5 * (lam[29] + lam[30])
    ref = O.feast_hcsr(A, B, emin, emax, 48, Y0=fw.complex_gaussian_block(300, 48, 1), ne=8, ratio=100,
                       tol_exp=12)
    assert ref["info"] == 0 and ref["M"] == 30
    assert np.abs(ref["E"][:30] - lam[:30]).max() < 1e-12 * np.abs(lam).max()
    X = ref["X"][:, :30]
    assert np.abs(X.conj().T @ B.to_dense() @ X - np.eye(30)).max() < 1e-12


def test_hermitian_feast_reduces_to_real_symmetric():
    """A real symmetric matrix stored as complex: same eigenvalues as the real
    oracle, trapezoidal rule included."""
    p = fw.laplace3d_potential(side=6, count=10, m0=16, seed=12)
    Az = fw.zcsr_from_dense(p.A.to_dense().astype(np.complex128))
    for rule in (0, 1):
        r = O.feast_scsr(p.A, None, p.emin, p.emax, 16, Y0=p.y0(), ne=8, ratio=100, tol_exp=12, rule=rule)
        h = O.feast_hcsr(Az, None, p.emin, p.emax, 16, Y0=p.y0().astype(np.complex128), ne=8, ratio=100,
                         tol_exp=12, rule=rule)
        assert r["info"] == h["info"] == 0 and r["M"] == h["M"]
        assert np.abs(r["E"][: r["M"]] - h["E"][: h["M"]]).max() < 1e-12


# ------------------------------------------------------------------ Zolotarev rule (fpm(16)=2)
@pytest.mark.parametrize("m", [0.1, 0.5, 0.9, 0.999, 1 - 1e-8])
def test_elliptic_functions_match_scipy(m):
    import scipy.special as sps

    assert abs(O.ellipk(m) - sps.ellipk(m)) < 1e-13 * sps.ellipk(m)
    K = sps.ellipk(m)
    for u in (0.0, 0.3, 0.5 * K, 0.9 * K, K):
        sn, cn = O.ellipj(u, m)
        ref = sps.ellipj(u, m)
        assert abs(sn - ref[0]) < 1e-12 and abs(cn - ref[1]) < 1e-12


def _refined_extrema(f, xs):
    """Local extrema of the sampled function f on the sorted grid xs, each
    refined by a bounded scalar search between its grid neighbours."""
    import scipy.optimize

    v = f(xs)
    d = np.diff(np.sign(np.diff(v)))
    out = []
    for i in np.nonzero(d)[0] + 1:
        sgn = -1.0 if d[i - 1] < 0 else 1.0  # -1: maximum, +1: minimum
        r = scipy.optimize.minimize_scalar(lambda t: sgn * f(np.array([t]))[0], bounds=(xs[i - 1], xs[i + 1]),
                                           method="bounded", options={"xatol": 1e-14 * max(1.0, abs(xs[i]))})
        out.append(f(np.array([r.x]))[0])
    return np.array(out)


@pytest.mark.parametrize("ne", [2, 4, 8])
def test_zolotarev_filter_is_equiripple(ne):
    """Zolotarev's filter is the best uniform approximation of the interval's
    indicator outside the edge bands (|x| <= 1/(1+eta) inside, |x| >= 1+eta
    outside, x = (lambda - c)/r, eta = 0.05): its error equioscillates with
    equal extrema, and the two ripples sit exactly 1 apart."""
    eta, emin, emax = 0.05, -1.0, 3.0
    c, r = 1.0, 2.0
    z, w = O.contour_zolotarev(ne, emin, emax, eta)
    assert np.allclose(np.abs((z - c) / r), 1.0, atol=1e-13) and np.all(z.imag > 0)
    f = lambda x: np.array([np.sum((w / (z - (c + r * t))).real) for t in x])
    xin = np.linspace(-1 / (1 + eta), 1 / (1 + eta), 4001)
    ein = np.concatenate([_refined_extrema(f, xin), f(xin[[0, -1]])])
    eout = np.concatenate([_refined_extrema(f, np.geomspace(1 + eta, 1e9, 4001)),
                           _refined_extrema(f, -np.geomspace(1e9, 1 + eta, 4001)), f(np.array([1 + eta, -1 - eta]))])
    ripple = ein.max() - ein.min()
    assert len(ein) >= ne + 2 and ripple > 0
    assert abs((eout.max() - eout.min()) - ripple) < 1e-9 * ripple
    assert abs((ein.max() + ein.min()) / 2 - (eout.max() + eout.min()) / 2 - 1.0) < 1e-12
    # every extremum sits on one of the two levels of its region
    for e in (ein, eout):
        assert np.all(np.minimum(np.abs(e - e.max()), np.abs(e - e.min())) < 1e-9 * ripple)


def test_feast_with_zolotarev_rule_matches_closed_form():
    """1D Laplacian n = 1000, the 5 eigenvalues of [-5e-4, (lambda_5 + lambda_6)/2]
    (closed form; none in the edge bands), Zolotarev nodes (fpm(16)=2)."""
    lam = 2 - 2 * np.cos(np.arange(1, 40) * np.pi / 1001)
    emin, emax = -5e-4, 0.5 * (lam[4] + lam[5])
    x = (lam - 0.5 * (emin + emax)) / (0.5 * (emax - emin))
    assert np.all((np.abs(x) < 1 / 1.05) | (np.abs(x) > 1.05))
    p = fw.tridiag_1d(n=1000, emin=emin, emax=emax, m0=10, ratio=30)
    ref = O.feast_scsr(p.A, None, emin, emax, 10, Y0=p.y0(), ne=8, ratio=30, tol_exp=11, rule=2)
    assert ref["info"] == 0 and ref["M"] == 5
    assert np.abs(ref["E"][:5] - lam[:5]).max() < 1e-15


# ------------------------------------------------------------------ filter block against the spectral formula
@pytest.mark.parametrize("solver", ["direct", "cocg"])
@pytest.mark.parametrize("gen", [False, True])
def test_filter_block_matches_dense_spectral_formula(gen, solver):
    """Classic form: Q = rho(B^{-1}A) Y = X diag(rho(lambda)) X^T B Y; the
    residual-inverse form applied to Ritz pairs of a random subspace gives the
    same rho(B^{-1}A) applied to that subspace's Ritz vectors."""
    rng = np.random.default_rng(51)
    A = fw.laplacian_2d(10, rng.uniform(0, 1, (10, 10)))
    B = fw.diagonal_csr(rng.uniform(1, 2, A.n)) if gen else None
    db = np.eye(A.n) if B is None else B.to_dense()
    lam, X = scipy.linalg.eigh(A.to_dense(), db)
    emin, emax = 0.0, 0.5 * (lam[11] + lam[12])
    r = _rho_dense(8, emin, emax, 0.3, lam)
    P = X @ (r[:, None] * (X.T @ db))  # rho(B^{-1} A)
    Y = rng.standard_normal((A.n, 7))
    tol = 1e-12 if solver == "direct" else 1e-10
    Q = O.filter_block(A, B, 8, emin, emax, 0.3, Y, solver=solver)
    assert np.abs(Q - P @ Y).max() < tol * np.abs(P @ Y).max()
    # Ritz pairs of a random 7-dimensional subspace (not eigenpairs)
    Z = np.linalg.qr(rng.standard_normal((A.n, 7)))[0]
    lr, W = scipy.linalg.eigh(Z.T @ A.to_dense() @ Z, Z.T @ db @ Z)
    XR = Z @ W
    Qr = O.filter_block(A, B, 8, emin, emax, 0.3, XR, lam=lr, rii=True, solver=solver)
    assert np.abs(Qr - P @ XR).max() < 10 * tol * np.abs(P @ XR).max()


def test_hermitian_feast_gauge_workload_matches_real_problem():
    """Random gauge phases D A D^H keep the spectrum of the real 3D workload and
    map its eigenvectors to D x: the Hermitian oracle on the gauged matrix gives
    the real oracle's eigenvalues."""
    p = fw.laplace3d_gauge(side=6, count=10, m0=16, ratio=100, seed=12)
    real = p.notes["real_problem"]
    r = O.feast_scsr(real.A, None, p.emin, p.emax, 16, Y0=real.y0(), ne=8, ratio=100, tol_exp=12)
    h = O.feast_hcsr(p.A, None, p.emin, p.emax, 16, Y0=p.y0(), ne=8, ratio=100, tol_exp=12)
    assert r["info"] == h["info"] == 0 and r["M"] == h["M"] >= 5
    M = r["M"]
    assert np.abs(r["E"][:M] - h["E"][:M]).max() < 1e-12
    d = p.A.to_dense()
    assert np.abs(d - d.conj().T).max() == 0.0 and np.abs(d.imag).max() > 0.5


def test_hermitian_reduced_gev_matches_eigh_and_drops_null_directions():
    """Reduced generalized Hermitian problem: full rank against scipy's eigh;
    a B_Q of rank 6 (Gram matrix of 6 independent vectors in 9 columns) keeps
    6 directions, whose pairs solve A_Q v = lambda B_Q v with V^H B_Q V = I."""
    rng = np.random.default_rng(61)
    m = 9
    H = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    H = (H + H.conj().T) / 2
    Z = rng.standard_normal((40, m)) + 1j * rng.standard_normal((40, m))
    Aq, Bq = Z.conj().T @ H @ Z, Z.conj().T @ Z
    info, lam, V = O.h_reduced_gev(Aq, Bq)
    assert info == 0 and len(lam) == m
    ref = scipy.linalg.eigh((Aq + Aq.conj().T) / 2, (Bq + Bq.conj().T) / 2, eigvals_only=True)
    assert np.abs(lam - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(V.conj().T @ Bq @ V - np.eye(m)).max() < 1e-10
    # rank-deficient: columns 6..8 are combinations of columns 0..5
    Z2 = Z.copy()
    Z2[:, 6:] = Z[:, :6] @ (rng.standard_normal((6, 3)) + 1j * rng.standard_normal((6, 3)))
    Aq2, Bq2 = Z2.conj().T @ H @ Z2, Z2.conj().T @ Z2
    info, lam2, V2 = O.h_reduced_gev(Aq2, Bq2)
    assert info == 0 and len(lam2) == 6
    Q6, _ = np.linalg.qr(Z[:, :6])
    ref6 = np.linalg.eigvalsh(Q6.conj().T @ H @ Q6)  # H projected on the span
    assert np.abs(np.sort(lam2) - ref6).max() < 1e-8 * np.abs(ref6).max()
    assert np.abs(Aq2 @ V2 - Bq2 @ V2 * lam2).max() < 1e-8 * np.abs(Aq2).max()


def test_hermitian_feast_zolotarev_rule_matches_dense():
    """fpm(16) = 2 in the Hermitian oracle, eigenvalues kept out of the rule's
    edge bands 1/1.05 < |x| < 1.05."""
    rng = np.random.default_rng(46)
    A = fw.hermitian_banded(300, 5, rng, shift=8.0)
    lam = np.linalg.eigvalsh(A.to_dense())
    emin, emax = lam[0] - 0.5, 0.5 * (lam[18] + lam[19])
    x = np.abs((lam - 0.5 * (emin + emax)) / (0.5 * (emax - emin)))
    assert not np.any((x > 1 / 1.05) & (x < 1.05))
    ref = O.feast_hcsr(A, None, emin, emax, 48, Y0=fw.complex_gaussian_block(300, 48, 3), ne=8, tol_exp=12, rule=2)
    assert ref["info"] == 0 and ref["M"] == 19
    assert np.abs(ref["E"][:19] - lam[:19]).max() < 1e-12 * np.abs(lam).max()
