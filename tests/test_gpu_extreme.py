"""One-pass modes (fpm(14) = 1, 2) and the extreme-eigenvalue mode (fpm(40) =
-1, +1) on the GPU.

The stochastic count and the one-pass block are compared element by element
with the oracle on the same probe block (FP64 solves to a tight tolerance).
The extreme mode's answer is a plain definition -- the k lowest (largest)
eigenpairs of (A, B) -- so it is checked against dense FP64 decompositions
(closed forms where they exist): eigenvalues to 1e-10 relative, residuals
below 1e-10, subspace angles below 1e-8, and the returned interval must hold
exactly those k eigenvalues."""
import numpy as np
import pytest
import scipy.linalg
import torch

import feast_workloads as fw
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_04807_gb300 import build

    build.build()
    import paper_2002_04807_gb300 as p

    p.library()
    assert torch.cuda.is_available()
    return p


def _dev(M):
    return (torch.as_tensor(M.indptr).cuda(), torch.as_tensor(M.indices).cuda(), torch.as_tensor(M.data).cuda())


def _fpm(pkg, mixed=1, tol=12, inner=2, cap=200, ratio=100):
    f = pkg.feast_init()
    f[1], f[2], f[3], f[17], f[41], f[44], f[45] = 8, tol, 40, ratio, mixed, inner, cap
    f[49] = 1
    return f


def _sine(U, V):
    qu, _ = np.linalg.qr(U)
    qv, _ = np.linalg.qr(V)
    return float(np.linalg.norm(qu - qv @ (qv.T @ qu), 2))


def _problem(gen, seed=31):
    rng = np.random.default_rng(seed)
    A = fw.laplacian_2d(24, rng.uniform(0, 1, (24, 24)))
    B = fw.diagonal_csr(rng.uniform(1, 2, A.n)) if gen else None
    db = np.eye(A.n) if B is None else B.to_dense()
    lam = scipy.linalg.eigh(A.to_dense(), db, eigvals_only=True)
    return A, B, lam


def _one_pass(pkg, A, B, emin, emax, Y, mode, mixed, inner):
    f = _fpm(pkg, mixed=mixed, inner=inner, cap=5000)
    f[4], f[13] = 1, mode
    ia, ja, av = _dev(A)
    kw = {}
    if B is not None:
        ib, jb, bv = _dev(B)
        kw = dict(ib=ib, jb=jb, b=bv)
    x = torch.as_tensor(np.ascontiguousarray(Y.T)).cuda()
    r = pkg.feast_scsr_solve_dev(A.n, ia, ja, av, fpm=f, emin=emin, emax=emax, m0=Y.shape[1], x=x, **kw)
    return r, x


@pytest.mark.parametrize("gen", [False, True])
def test_stochastic_count_matches_oracle_fp64(pkg, gen):
    A, B, lam = _problem(gen)
    emin, emax = 0.0, 0.5 * (lam[19] + lam[20])
    Y = np.random.default_rng(5).standard_normal((A.n, 24))
    x_before = Y.copy()
    r, x = _one_pass(pkg, A, B, emin, emax, Y, 2, mixed=0, inner=13)
    assert r.info == 5
    est, sem = O.stochastic_count(A, B, 8, emin, emax, 1.0, Y)
    assert abs(r.E[0] - est) < 1e-9 * abs(est)
    assert abs(r.E[1] - sem) < 1e-7 * sem
    assert r.M == int(np.floor(est + 0.5))
    assert np.array_equal(x.cpu().numpy().T, x_before)  # the probes are left alone


def test_stochastic_count_mixed_precision(pkg):
    """Complex FP32 solves (tolerance 1e-5): the estimate moves by far less
    than its own statistical error."""
    A, B, lam = _problem(False)
    emin, emax = 0.0, 0.5 * (lam[29] + lam[30])
    Y = np.random.default_rng(6).standard_normal((A.n, 32))
    r, _ = _one_pass(pkg, A, B, emin, emax, Y, 2, mixed=1, inner=5)
    est, sem = O.stochastic_count(A, B, 8, emin, emax, 1.0, Y)
    assert r.info == 5
    assert abs(r.E[0] - est) < 1e-3 * abs(est) and abs(r.E[0] - est) < 0.01 * sem


def test_random_probe_count_near_inertia(pkg):
    """Seeded device probes: the count lands within five standard errors of
    the inertia count of the interval."""
    A, _, lam = _problem(False, seed=32)
    emax = 0.5 * (lam[39] + lam[40])
    f = _fpm(pkg, mixed=1, inner=5, cap=2000)
    f[1] = 16
    f[13] = 2
    ia, ja, av = _dev(A)
    r = pkg.feast_scsr_solve_dev(A.n, ia, ja, av, fpm=f, emin=0.0, emax=emax, m0=128)
    assert r.info == 5
    cnt = O.count_below(A, None, emax)
    assert cnt == 40
    assert 0.0 < r.E[1] < 3.0 and abs(r.E[0] - cnt) < 5 * r.E[1]


@pytest.mark.parametrize("gen", [False, True])
def test_one_pass_block_matches_oracle_filter(pkg, gen):
    A, B, lam = _problem(gen)
    emin, emax = 0.0, 0.5 * (lam[9] + lam[10])
    Y = np.random.default_rng(7).standard_normal((A.n, 16))
    r, x = _one_pass(pkg, A, B, emin, emax, Y, 1, mixed=0, inner=13)
    assert r.info == 4
    Q = O.filter_block(A, B, 8, emin, emax, 1.0, Y)
    Qg = x.cpu().numpy().T
    assert np.abs(Qg - Q).max() < 1e-9 * np.abs(Q).max()


def _check_extreme(r, lam_all, vecs, k, lowest, B=None):
    assert r.info == 0 and r.M == k
    want = lam_all[:k] if lowest else lam_all[-k:]
    scale = np.abs(lam_all).max()
    assert np.abs(r.E[:k] - want).max() < 1e-10 * scale
    assert r.res[:k].max() < 1e-10
    # the interval holds exactly the k wanted eigenvalues
    inside = np.sum((lam_all >= r.emin) & (lam_all <= r.emax))
    assert inside == k
    assert (r.emin < want[0] and r.emax >= want[-1]) if lowest else (r.emax > want[-1] and r.emin <= want[0])
    X = r.X.cpu().numpy().T if isinstance(r.X, torch.Tensor) else np.asarray(r.X)
    X = X[:, :k]
    G = X.T @ (X if B is None else B.to_dense() @ X)
    assert np.abs(G - np.eye(k)).max() < 1e-10
    V = vecs[:, :k] if lowest else vecs[:, -k:]
    assert _sine(X, V) < 1e-8


@pytest.mark.parametrize("lowest", [True, False])
def test_extreme_mode_laplace3d(pkg, lowest):
    p = fw.laplace3d_potential(side=12, count=20, m0=32, seed=3)
    A = p.A
    lam, V = np.linalg.eigh(A.to_dense())
    k = 20
    f = _fpm(pkg)
    f[39] = -1 if lowest else 1
    ia, ja, av = _dev(A)
    r = pkg.feast_scsr_extreme_dev(A.n, ia, ja, av, fpm=f, m0=2 * k)
    _check_extreme(r, lam, V, k, lowest)


def test_extreme_mode_generalized_27pt(pkg):
    """Lowest eigenpairs of the 27-point generalized workload's generator
    (B diagonal, U[1,2]) on an 8^3 grid."""
    p = fw.stencil27_generalized(side=8, count=16, m0=32, ne=16, emax=1.0)
    lam, V = scipy.linalg.eigh(p.A.to_dense(), p.B.to_dense())
    k = 16
    f = _fpm(pkg)
    f[1] = 16
    f[39] = -1
    ia, ja, av = _dev(p.A)
    ib, jb, bv = _dev(p.B)
    r = pkg.feast_scsr_extreme_dev(p.A.n, ia, ja, av, ib=ib, jb=jb, b=bv, fpm=f, m0=2 * k)
    _check_extreme(r, lam, V, k, True, B=p.B)


def test_extreme_mode_host_entry_closed_form(pkg):
    """1D Laplacian n = 200: lambda_j = 2 - 2 cos(j pi / 201), lowest 10."""
    n, k = 200, 10
    A = fw.laplacian_1d(n)
    f = _fpm(pkg)
    f[39] = -1
    r = pkg.feast_scsr_extreme("F", n, A.data, A.indptr, A.indices, fpm=f, m0=2 * k)
    lam = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    i = np.arange(1, n + 1)[:, None]
    V = np.sqrt(2.0 / (n + 1)) * np.sin(i * np.arange(1, n + 1)[None, :] * np.pi / (n + 1))
    _check_extreme(r, lam, V, k, True)
