"""Complex Hermitian FEAST on the GPU (the guide's zfeast_hcsr{ev,gv}, Sec. 3.2)
through the C ABI, against closed forms and the FP64 CPU oracle.

Bars as for the real symmetric driver: eigenvalue relative error <= 1e-10,
relative residual <= 1e-10, subspace angles <= 1e-8."""
import numpy as np
import pytest
import scipy.linalg
import torch

import feast_workloads as fw
import oracle as O

pytestmark = pytest.mark.gpu
EIG_TOL, RES_TOL, ANG_TOL = 1e-10, 1e-10, 1e-8


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_04807_gb300 import build

    build.build()
    import paper_2002_04807_gb300 as p

    p.library()
    assert torch.cuda.is_available()
    return p


def sin_angle(U, V):
    qu, _ = np.linalg.qr(U)
    qv, _ = np.linalg.qr(V)
    return float(np.linalg.norm(qu - qv @ (qv.conj().T @ qu), 2))


def cluster_angles(E, X, Xo, scale):
    """Max subspace angle over clusters of eigenvalues closer than 1e-8 * scale."""
    worst, i = 0.0, 0
    while i < len(E):
        j = i + 1
        while j < len(E) and E[j] - E[j - 1] < 1e-8 * scale:
            j += 1
        worst = max(worst, sin_angle(X[:, i:j], Xo[:, i:j]))
        i = j
    return worst


def fpm_for(pkg, mixed, ne=8, ratio=100, tol_exp=10, inner=(2, 300), maxloop=30, nb=0, rule=0, start=True):
    f = pkg.feast_init()
    f[1], f[2], f[3], f[17], f[41] = ne, tol_exp, maxloop, ratio, mixed
    f[15], f[49] = rule, nb
    f[44], f[45] = inner
    f[4] = 1 if start else 0
    f[5] = 1
    return f


def flux_case(n=200, phi=0.013, count=21):
    A = fw.flux_ring(n, phi)
    lam = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n + phi))
    return A, lam, 0.5 * (lam[count - 1] + lam[count])


@pytest.mark.parametrize("mixed", [1, 0])
def test_flux_ring_closed_form(pkg, mixed):
    """lambda_m = 2 - 2 cos(2 pi m / n + phi); eigenvectors the plane waves."""
    n, phi = 200, 0.013
    A, lam, emax = flux_case(n, phi)
    r = pkg.feast_hcsr_solve("F", n, A.data, A.indptr, A.indices, fpm=fpm_for(pkg, mixed), emin=0.0, emax=emax,
                             m0=32, x0=fw.complex_gaussian_block(n, 32, 0))
    assert r.info == 0 and r.M == 21
    assert np.abs(r.E[:21] - lam[:21]).max() < EIG_TOL * 4.0
    assert r.res[:21].max() < RES_TOL
    X = r.X[:, :21]
    assert np.abs(X.conj().T @ X - np.eye(21)).max() < 1e-10
    mm = np.arange(n)
    lam_all = 2 - 2 * np.cos(2 * np.pi * mm / n + phi)
    order = np.argsort(lam_all)[:21]
    waves = np.exp(1j * np.outer(np.arange(n), 2 * np.pi * mm[order] / n)) / np.sqrt(n)
    assert cluster_angles(r.E[:21], X, waves, 4.0) < ANG_TOL


def banded_case(gen, n=300, seed=44):
    rng = np.random.default_rng(seed)
    A = fw.hermitian_banded(n, 5, rng, shift=8.0)
    B = None
    if gen:  # Hermitian positive definite tridiagonal B
        off = 0.2 * (rng.standard_normal(n - 1) + 1j * rng.standard_normal(n - 1))
        db = np.diag(rng.uniform(2.5, 3.5, n)) + np.diag(off, 1) + np.diag(off.conj(), -1)
        B = fw.zcsr_from_dense(db.astype(np.complex128))
    db = np.eye(n) if B is None else B.to_dense()
    lam = scipy.linalg.eigh(A.to_dense(), db, eigvals_only=True)
    return A, B, lam


@pytest.mark.parametrize("gen", [False, True])
@pytest.mark.parametrize("mixed", [1, 0])
def test_banded_matches_oracle(pkg, gen, mixed):
    n, m0 = 300, 48
    A, B, lam = banded_case(gen, n)
    emin, emax = lam[0] - 0.5, 0.5 * (lam[29] + lam[30])
    y0 = fw.complex_gaussian_block(n, m0, 1)
    ref = O.feast_hcsr(A, B, emin, emax, m0, Y0=y0, ne=8, ratio=100, tol_exp=12)
    assert ref["info"] == 0 and ref["M"] == 30
    kw = {} if B is None else dict(b=B.data, ib=B.indptr, jb=B.indices)
    r = pkg.feast_hcsr_solve("F", n, A.data, A.indptr, A.indices, fpm=fpm_for(pkg, mixed), emin=emin, emax=emax,
                             m0=m0, x0=y0, **kw)
    assert r.info == 0 and r.M == 30
    scale = np.abs(lam).max()
    assert np.abs(r.E[:30] - ref["E"][:30]).max() < EIG_TOL * scale
    assert r.res[:30].max() < RES_TOL
    db = np.eye(n) if B is None else B.to_dense()
    X = r.X[:, :30]
    assert np.abs(X.conj().T @ db @ X - np.eye(30)).max() < 1e-10
    assert cluster_angles(r.E[:30], X, ref["X"][:, :30], scale) < ANG_TOL


def test_lower_storage_and_one_based_match_full(pkg):
    """'L' storage (mirrored entries conjugated) and 1-based CSR give the full-storage result."""
    n, m0 = 300, 48
    A, _, lam = banded_case(False, n, seed=45)
    emin, emax = lam[0] - 0.5, 0.5 * (lam[19] + lam[20])
    d = A.to_dense()
    low = fw.zcsr_from_dense(np.tril(d))
    y0 = fw.complex_gaussian_block(n, m0, 2)
    f = fpm_for(pkg, 1)
    full = pkg.feast_hcsr_solve("F", n, A.data, A.indptr, A.indices, fpm=f, emin=emin, emax=emax, m0=m0, x0=y0)
    lo = pkg.feast_hcsr_solve("L", n, low.data, low.indptr + 1, low.indices + 1, fpm=f, emin=emin, emax=emax,
                              m0=m0, x0=y0)
    assert full.info == lo.info == 0 and full.M == lo.M == 20
    assert np.abs(full.E[:20] - lo.E[:20]).max() < EIG_TOL * np.abs(lam).max()
    assert np.abs(full.E[:20] - lam[:20]).max() < EIG_TOL * np.abs(lam).max()


@pytest.mark.parametrize("rule", [1, 2])
def test_quadrature_rules(pkg, rule):
    """Trapezoidal and Zolotarev nodes reach the same eigenpairs."""
    n, m0 = 300, 48
    A, _, lam = banded_case(False, n, seed=46)
    emin, emax = lam[0] - 0.5, 0.5 * (lam[18] + lam[19])
    # no eigenvalue in the Zolotarev rule's edge bands 1/1.05 < |x| < 1.05
    x = np.abs((lam - 0.5 * (emin + emax)) / (0.5 * (emax - emin)))
    assert not np.any((x > 1 / 1.05) & (x < 1.05))
    ne = 16 if rule == 1 else 8
    r = pkg.feast_hcsr_solve("F", n, A.data, A.indptr, A.indices, fpm=fpm_for(pkg, 1, ne=ne, rule=rule),
                             emin=emin, emax=emax, m0=m0, x0=fw.complex_gaussian_block(n, m0, 3))
    assert r.info == 0 and r.M == 19
    assert np.abs(r.E[:19] - lam[:19]).max() < EIG_TOL * np.abs(lam).max()
    assert r.res[:19].max() < RES_TOL


def test_random_start_and_node_batches(pkg):
    """fpm(5) = 0 (the library's own start block) and nodes split into batches of 3."""
    n, m0 = 300, 48
    A, _, lam = banded_case(False, n, seed=47)
    emin, emax = lam[0] - 0.5, 0.5 * (lam[24] + lam[25])
    r = pkg.feast_hcsr_solve("F", n, A.data, A.indptr, A.indices, fpm=fpm_for(pkg, 1, nb=3, start=False),
                             emin=emin, emax=emax, m0=m0)
    assert r.info == 0 and r.M == 25
    assert np.abs(r.E[:25] - lam[:25]).max() < EIG_TOL * np.abs(lam).max()
    assert r.res[:25].max() < RES_TOL


def test_device_entry_point(pkg):
    n, m0 = 300, 48
    A, B, lam = banded_case(True, n, seed=48)
    emin, emax = lam[0] - 0.5, 0.5 * (lam[14] + lam[15])
    dev = torch.device("cuda:0")
    t = lambda v, dt: torch.as_tensor(np.ascontiguousarray(v)).to(dev, dt)  # noqa: E731
    y0 = fw.complex_gaussian_block(n, m0, 4)
    x = torch.as_tensor(np.ascontiguousarray(y0.T)).to(dev)  # (m0, n) row-major = column-major n x m0
    r = pkg.feast_hcsr_solve_dev(n, t(A.indptr, torch.int32), t(A.indices, torch.int32), t(A.data, torch.complex128),
                                 ib=t(B.indptr, torch.int32), jb=t(B.indices, torch.int32),
                                 b=t(B.data, torch.complex128), fpm=fpm_for(pkg, 1), emin=emin, emax=emax, m0=m0, x=x)
    assert r.info == 0 and r.M == 15
    assert np.abs(r.E[:15] - lam[:15]).max() < EIG_TOL * np.abs(lam).max()
    X = x.cpu().numpy().T[:, :15]
    db = B.to_dense()
    R = A.to_dense() @ X - db @ X * r.E[:15]
    assert np.abs(R).max() < 1e-9 * np.abs(lam).max()
    # caller workspace: the same kernels in the same order give the same result;
    # one byte short is rejected before any device work
    f = fpm_for(pkg, 1)
    need = pkg.feast_hcsr_workspace_bytes(n, A.nnz, B.nnz, m0, f)
    work = torch.empty(need, dtype=torch.uint8, device=dev)
    x2 = torch.as_tensor(np.ascontiguousarray(y0.T)).to(dev)
    args = (n, t(A.indptr, torch.int32), t(A.indices, torch.int32), t(A.data, torch.complex128))
    kw = dict(ib=t(B.indptr, torch.int32), jb=t(B.indices, torch.int32), b=t(B.data, torch.complex128), emin=emin,
              emax=emax, m0=m0)
    r2 = pkg.feast_hcsr_solve_dev(*args, fpm=f.copy(), x=x2, work=work, **kw)
    assert r2.info == 0 and np.array_equal(r2.E, r.E)
    assert torch.equal(x2, x)
    short = pkg.feast_hcsr_solve_dev(*args, fpm=f.copy(), x=x2.clone(), work=work[: need - 1], **kw)
    assert short.info == -120


def test_gauge_workload_matches_real_spectrum(pkg):
    """The bench's Hermitian workload at 12^3: random gauge phases keep the real
    problem's spectrum, so the eigenvalues are checked against a dense real eigh."""
    p = fw.laplace3d_gauge(side=12, count=20, m0=32, ratio=200)
    lam = np.linalg.eigvalsh(p.notes["real_problem"].A.to_dense())
    emax = 0.5 * (lam[19] + lam[20])
    r = pkg.feast_hcsr_solve("F", p.n, p.A.data, p.A.indptr, p.A.indices, fpm=fpm_for(pkg, 1, ratio=200),
                             emin=p.emin, emax=emax, m0=32, x0=p.y0())
    assert r.info == 0 and r.M == 20
    assert np.abs(r.E[:20] - lam[:20]).max() < EIG_TOL * np.abs(lam).max()
    assert r.res[:20].max() < RES_TOL


def test_gauge_workload_wide_subspace_both_projection_arithmetics(pkg):
    """The gauge workload at 16^3 with M0 = 150 (the bench's subspace width):
    the projections split over several row blocks (the sliced products' two
    Gram forms take different split counts), with the sliced BF16 products
    (fpm(54) = 0) and with the FP64 tensor cores (1); both against the real
    problem's dense spectrum."""
    p = fw.laplace3d_gauge(side=16, count=100, m0=150, ratio=200)
    lam = np.linalg.eigvalsh(p.notes["real_problem"].A.to_dense())
    emax = 0.5 * (lam[99] + lam[100])
    Es = []
    for arith in (0, 1):
        f = fpm_for(pkg, 1, ratio=200)
        f[53] = arith
        r = pkg.feast_hcsr_solve("F", p.n, p.A.data, p.A.indptr, p.A.indices, fpm=f, emin=p.emin, emax=emax,
                                 m0=150, x0=p.y0())
        assert r.info == 0 and r.M == 100, (arith, r.info, r.M)
        assert np.abs(r.E[:100] - lam[:100]).max() < EIG_TOL * np.abs(lam[:100]).max()
        assert r.res[:100].max() < RES_TOL
        Es.append(r.E[:100])
    assert np.abs(Es[0] - Es[1]).max() < 1e-12 * np.abs(lam[:100]).max()
