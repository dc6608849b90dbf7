"""End-to-end GPU FEAST through the C ABI against the FP64 CPU oracle.

Bars (from the method's accuracy targets): eigenvalue relative error
<= 1e-10, relative residual <= 1e-10, subspace angles <= 1e-8."""
import json
import os

import numpy as np
import pytest
import torch

import feast_workloads as fw
import oracle as O

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
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
    return float(np.linalg.norm(qu - qv @ (qv.T @ qu), 2))


def cluster_angles(E, X, Eo, Xo, scale):
    """Max subspace angle over clusters of eigenvalues closer than 1e-8 * scale."""
    worst = 0.0
    i = 0
    while i < len(Eo):
        j = i + 1
        while j < len(Eo) and Eo[j] - Eo[j - 1] < 1e-8 * scale:
            j += 1
        worst = max(worst, sin_angle(X[:, i:j], Xo[:, i:j]))
        i = j
    return worst


def run_gpu(pkg, p, mixed, y0=None, tol_exp=10, inner=(2, 200), maxloop=30, B=None, uplo="F", csr=None,
            nb=0, rule=0):
    fpm = pkg.feast_init()
    fpm[1], fpm[2], fpm[3], fpm[17], fpm[41] = p.ne, tol_exp, maxloop, p.ratio, mixed
    fpm[15] = rule
    fpm[44], fpm[45] = inner
    fpm[49] = nb
    if y0 is None:
        y0 = p.y0()
    fpm[4] = 1
    A = p.A if csr is None else csr
    Bm = p.B if B is None else B
    kw = {}
    if Bm is not None:
        kw = dict(b=Bm.data, ib=Bm.indptr, jb=Bm.indices)
    return pkg.feast_scsr_solve(uplo, p.n, A.data, A.indptr, A.indices, fpm=fpm, emin=p.emin, emax=p.emax,
                                m0=p.m0, x0=y0, **kw)


def check_against(r, ref, scale, B=None):
    assert r.info == 0, r.info
    assert r.M == ref["M"], (r.M, ref["M"])
    M = r.M
    rel = np.abs(r.E[:M] - ref["E"][:M]) / np.maximum(np.abs(ref["E"][:M]), 1e-300)
    assert rel.max() <= EIG_TOL, rel.max()
    assert r.res[:M].max() <= RES_TOL
    ang = cluster_angles(r.E[:M], r.X[:, :M], ref["E"][:M], ref["X"][:, :M], scale)
    assert ang <= ANG_TOL, ang
    X = r.X[:, :M]
    BX = X if B is None else O.csr_mm(B, X)
    assert np.abs(X.T @ BX - np.eye(M)).max() < 1e-11


@pytest.mark.parametrize("mixed", [0, 1])
def test_helloworld_worked_example(pkg, mixed):
    g = json.load(open(os.path.join(GOLD, "helloworld.json")))
    c, run = g["csr_1based"], g["run"]
    a = np.array(c["sA"], dtype=float)
    ia = np.array(c["IA"], dtype=np.int32)
    ja = np.array(c["JA"], dtype=np.int32)
    fpm = pkg.feast_init()
    fpm[41] = mixed
    fpm[44], fpm[45] = 2, 100
    fpm[4] = 1
    y0 = fw.gaussian_block(4, run["M0"], 0)
    r = pkg.feast_scsr_solve("F", 4, a, ia, ja, fpm=fpm, emin=run["Emin"], emax=run["Emax"], m0=run["M0"], x0=y0)
    assert r.info == 0 and r.M == g["expected"]["M"]
    assert np.allclose(r.E[:2], g["expected"]["E"], atol=1e-12)
    assert r.res[:2].max() < g["expected"]["max_residual_below"]


@pytest.mark.parametrize("uplo", ["L", "U"])
def test_half_storage(pkg, uplo):
    d = fw.helloworld_dense()
    tri = np.tril(d) if uplo == "L" else np.triu(d)
    A = fw.csr_from_dense(tri)
    fpm = pkg.feast_init()
    fpm[4] = 1
    fpm[44], fpm[45] = 2, 100
    y0 = fw.gaussian_block(4, 3, 0)
    r = pkg.feast_scsr_solve(uplo, 4, A.data, A.indptr, A.indices, fpm=fpm, emin=3.0, emax=5.0, m0=3, x0=y0)
    assert r.info == 0 and r.M == 2 and np.allclose(r.E[:2], [4.0, 4.0], atol=1e-12)


@pytest.mark.parametrize("mixed", [0, 1])
def test_laplacian_1d_closed_form(pkg, mixed):
    p = fw.tridiag_1d()
    ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=p.ne, ratio=p.ratio, tol_exp=10)
    r = run_gpu(pkg, p, mixed, inner=(2, 400), maxloop=60)
    check_against(r, ref, 0.01)
    k = np.arange(1, 32)
    lam = 2 - 2 * np.cos(k * np.pi / 1001)
    assert np.abs(r.E[:31] - lam).max() <= EIG_TOL * lam.max()


@pytest.mark.parametrize("mixed", [0, 1])
def test_laplace3d_potential_vs_oracle(pkg, mixed):
    p = fw.laplace3d_potential(side=16, count=30, m0=48, seed=7)
    ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=100, tol_exp=10)
    assert ref["info"] == 0
    r = run_gpu(pkg, p, mixed)
    check_against(r, ref, p.emax)


def test_constant_potential_degenerate_clusters(pkg):
    side, v0 = 12, 0.3
    mu = 2 - 2 * np.cos(np.arange(1, side + 1) * np.pi / (side + 1))
    eig = (mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel() + v0
    lev = np.sort(eig)
    distinct = np.unique(np.round(lev, 12))
    emax = 0.5 * (distinct[4] + distinct[5])
    sel = eig <= emax
    p = fw.laplace3d_constant(side, v0, emax, m0=int(1.6 * sel.sum()) + 4)
    r = run_gpu(pkg, p, 1)
    assert r.info == 0 and r.M == sel.sum()
    assert np.abs(r.E[: r.M] - np.sort(eig[sel])).max() < EIG_TOL * emax
    s = np.sin(np.arange(1, side + 1)[:, None] * np.arange(1, side + 1)[None, :] * np.pi / (side + 1))
    s *= np.sqrt(2 / (side + 1))
    full = np.einsum("ia,jb,kc->ijkabc", s, s, s).reshape(side ** 3, -1)
    assert sin_angle(r.X[:, : r.M], full[:, sel]) < ANG_TOL


@pytest.mark.parametrize("mixed", [0, 1])
def test_generalized_27pt(pkg, mixed):
    rng = np.random.default_rng(7)
    A = fw.stencil27_spd(9, rng)
    B = fw.diagonal_csr(rng.uniform(1.0, 2.0, A.n))
    ev = np.linalg.eigvalsh(np.diag(1 / np.sqrt(B.data)) @ A.to_dense() @ np.diag(1 / np.sqrt(B.data)))
    emax = 0.5 * (ev[24] + ev[25])
    p = fw.Problem("s27", A, B, 0.0, emax, 40, 16, 100, 2)
    ref = O.feast_scsr(A, B, 0.0, emax, 40, Y0=p.y0(), ne=16, ratio=100, tol_exp=10)
    assert ref["M"] == 25 == O.count_below(A, B, emax)
    r = run_gpu(pkg, p, mixed)
    check_against(r, ref, emax, B=B)


@pytest.mark.parametrize("mixed", [0, 1])
def test_generalized_nondiagonal_b(pkg, mixed):
    """A non-diagonal SPD sparse B (7-point mass-like pattern, the guide's
    dfeast_scsrgv with a full {B, IB, JB}): the packed general-B gathers of the
    filter, the general-B residual and SpMM, in both precisions, against the
    oracle; 1-based CSR input for both matrices on the FP64 run."""
    p = fw.laplace3d_general_b(side=10, count=20, m0=32)
    ref = O.feast_scsr(p.A, p.B, 0.0, p.emax, 32, Y0=p.y0(), ne=8, ratio=100, tol_exp=10)
    assert ref["info"] == 0 and ref["M"] == 20 == O.count_below(p.A, p.B, p.emax)
    if mixed:
        r = run_gpu(pkg, p, mixed)
    else:
        one = lambda M: fw.CSR(M.n, M.indptr + 1, M.indices + 1, M.data)  # noqa: E731
        r = run_gpu(pkg, p, mixed, csr=one(p.A), B=one(p.B))
    check_against(r, ref, p.emax, B=p.B)


@pytest.fixture(scope="module")
def config3_shape():
    """The 27-point generalized workload's generator (off-diagonals -U[0.5,1.5],
    diagonal row-abs-sum + U[0.1,1], B = diag(U[1,2])) at 12^3 with its shape
    scaled: the 100 lowest eigenvalues, M0 = 150, Ne = 16; the oracle solves it
    with its banded LDL^T."""
    p = fw.stencil27_generalized(side=12, count=100, m0=150, ne=16, emax=1.0)
    d = 1 / np.sqrt(p.B.data)
    ev = np.linalg.eigvalsh(d[:, None] * p.A.to_dense() * d[None, :])
    emax = 0.5 * (ev[99] + ev[100])
    p = fw.Problem(p.name, p.A, p.B, 0.0, emax, 150, 16, 100, 2)
    ref = O.feast_scsr(p.A, p.B, 0.0, emax, 150, Y0=p.y0(), ne=16, ratio=100, tol_exp=10)
    assert ref["M"] == 100 == O.count_below(p.A, p.B, emax)
    return p, ref


@pytest.mark.parametrize("mixed", [0, 1])
def test_generalized_27pt_config3_shape(pkg, config3_shape, mixed):
    p, ref = config3_shape
    r = run_gpu(pkg, p, mixed)
    check_against(r, ref, p.emax, B=p.B)


@pytest.mark.parametrize("mixed", [0, 1])
def test_trapezoid_rule_matches_oracle(pkg, mixed):
    """fpm(16) = 1: trapezoidal nodes, 12 of them (a count the Gauss rule does
    not allow), against the oracle with the same rule."""
    p = fw.laplace3d_potential(side=10, count=20, m0=32, ne=12, ratio=100, seed=13)
    ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=12, ratio=100, tol_exp=10, rule=1)
    assert ref["info"] == 0 and ref["M"] == O.count_below(p.A, None, p.emax)
    r = run_gpu(pkg, p, mixed, rule=1)
    check_against(r, ref, p.emax)


@pytest.mark.parametrize("mixed", [0, 1])
def test_zolotarev_rule_matches_oracle(pkg, mixed):
    """fpm(16) = 2: 1D Laplacian n = 1000, the 5 eigenvalues of
    [-5e-4, (lambda_5 + lambda_6)/2] (none in the edge bands), against the
    oracle with the same rule."""
    lam = 2 - 2 * np.cos(np.arange(1, 40) * np.pi / 1001)
    emin, emax = -5e-4, 0.5 * (lam[4] + lam[5])
    p = fw.tridiag_1d(n=1000, emin=emin, emax=emax, m0=10, ratio=30)
    ref = O.feast_scsr(p.A, None, emin, emax, 10, Y0=p.y0(), ne=8, ratio=30, tol_exp=11, rule=2)
    assert ref["info"] == 0 and ref["M"] == 5
    r = run_gpu(pkg, p, mixed, inner=(6, 3000), rule=2)
    check_against(r, ref, emax)


@pytest.mark.parametrize("kind", ["tall_ellipse", "trapezoid"])
def test_custom_nodes_match_oracle(pkg, kind):
    """Expert entry points (custom half-contour nodes): nodes of a taller
    ellipse, or trapezoidal nodes, passed by the caller while fpm(16)/fpm(18)
    say otherwise, give the oracle's result for that contour."""
    p = fw.laplace3d_potential(side=10, count=20, m0=32, ne=8, ratio=100, seed=14)
    if kind == "tall_ellipse":
        z, w = O.contour_gauss(8, p.emin, p.emax, 3.0)
        ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=300, tol_exp=10)
    else:
        z, w = O.contour_trapezoid(8, p.emin, p.emax, 1.0)
        ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=100, tol_exp=10, rule=1)
    fpm = pkg.feast_init()
    fpm[1], fpm[2], fpm[3], fpm[4], fpm[17], fpm[41], fpm[44], fpm[45] = 8, 10, 30, 1, 100, 1, 2, 200
    r = pkg.feast_scsr_solve_x("F", p.n, p.A.data, p.A.indptr, p.A.indices, z, w, fpm=fpm, emin=p.emin,
                               emax=p.emax, m0=p.m0, x0=p.y0())
    check_against(r, ref, p.emax)
    ia, ja, av = (torch.as_tensor(p.A.indptr).cuda(), torch.as_tensor(p.A.indices).cuda(),
                  torch.as_tensor(p.A.data).cuda())
    x = torch.as_tensor(np.ascontiguousarray(p.y0().T)).cuda()
    rd = pkg.feast_scsr_solve_dev_x(p.n, ia, ja, av, z, w, fpm=fpm, emin=p.emin, emax=p.emax, m0=p.m0, x=x)
    assert rd.info == 0 and np.array_equal(rd.E, r.E)  # same kernels, same order


def test_node_batches_agree(pkg):
    """Solving the 16 nodes in batches of 4 gives the same eigenpairs."""
    p = fw.laplace3d_potential(side=12, count=16, m0=28, ne=16, seed=9)
    a = run_gpu(pkg, p, 1, nb=4)
    b = run_gpu(pkg, p, 1, nb=16)
    assert a.info == b.info == 0 and a.M == b.M
    assert np.abs(a.E[: a.M] - b.E[: b.M]).max() < 1e-10 * p.emax


def test_no_eigenvalue_and_small_subspace(pkg):
    p = fw.tridiag_1d(n=300, emin=5.0, emax=6.0, m0=8, ratio=100)
    r = run_gpu(pkg, p, 1)
    assert r.info == 1 and r.M == 0
    # interval holding more eigenvalues than M0: warning 3 (or no convergence)
    p2 = fw.tridiag_1d(n=300, emin=0.0, emax=0.2, m0=8, ratio=100)
    r2 = run_gpu(pkg, p2, 1, maxloop=5)
    assert r2.info in (2, 3)


def test_tiny_full_subspace(pkg):
    A = fw.laplacian_1d(6)
    lam = 2 - 2 * np.cos(np.arange(1, 7) * np.pi / 7)
    fpm = pkg.feast_init()
    fpm[4] = 1
    fpm[17] = 100
    fpm[44], fpm[45] = 2, 100
    r = pkg.feast_scsr_solve("F", 6, A.data, A.indptr, A.indices, fpm=fpm, emin=0.0, emax=1.0, m0=6,
                             x0=fw.gaussian_block(6, 6, 1))
    inside = lam[lam <= 1.0]
    assert r.M == len(inside) and np.abs(r.E[: r.M] - inside).max() < 1e-12


def test_restart_from_solution(pkg):
    p = fw.laplace3d_potential(side=12, count=16, m0=28, seed=9)
    r = run_gpu(pkg, p, 1)
    assert r.info == 0
    X0 = np.zeros((p.n, p.m0), order="F")
    X0[:, : r.m0] = r.X
    r2 = run_gpu(pkg, p, 1, y0=X0)
    assert r2.info == 0 and r2.loop <= 1 and r2.M == r.M


def test_device_driver_with_torch_stream(pkg):
    p = fw.laplace3d_potential(side=12, count=16, m0=28, seed=9)
    host = run_gpu(pkg, p, 1)
    fpm = host.fpm.copy()
    s = torch.cuda.Stream()
    ia = torch.as_tensor(p.A.indptr).cuda()
    ja = torch.as_tensor(p.A.indices).cuda()
    av = torch.as_tensor(p.A.data).cuda()
    x = torch.as_tensor(np.ascontiguousarray(p.y0().T)).cuda()  # (m0, n) row-major == column-major n x m0
    with torch.cuda.stream(s):
        r = pkg.feast_scsr_solve_dev(p.n, ia, ja, av, fpm=fpm, emin=p.emin, emax=p.emax, m0=p.m0, x=x, stream=s)
    assert r.info == 0 and r.M == host.M
    assert np.array_equal(r.E, host.E)  # deterministic: same kernels, same order
    Xd = x.cpu().numpy().T[:, : r.m0]
    assert np.array_equal(Xd, host.X)


def test_projection_arithmetic_fp64_dmma_agrees(pkg):
    """fpm(54) = 1 builds the reduced matrices on the FP64 tensor cores instead
    of from BF16 slice products: same eigenpairs within the parity bars, both
    against the oracle."""
    p = fw.laplace3d_potential(side=14, count=24, m0=40, seed=12)
    ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=100, tol_exp=10)
    out = []
    for arith in (0, 1):
        fpm = pkg.feast_init()
        fpm[1], fpm[2], fpm[3], fpm[4], fpm[17], fpm[44], fpm[45], fpm[53] = 8, 10, 30, 1, 100, 2, 200, arith
        r = pkg.feast_scsr_solve("F", p.n, p.A.data, p.A.indptr, p.A.indices, fpm=fpm, emin=p.emin, emax=p.emax,
                                 m0=p.m0, x0=p.y0())
        check_against(r, ref, p.emax)
        out.append(r)
    M = out[0].M
    assert out[1].M == M and np.abs(out[0].E[:M] - out[1].E[:M]).max() <= 1e-12 * p.emax


def test_random_start_block(pkg):
    p = fw.laplace3d_potential(side=12, count=16, m0=28, seed=9)
    fpm = pkg.feast_init()
    fpm[17], fpm[44], fpm[45] = 100, 2, 200
    fpm[2] = 10
    r = pkg.feast_scsr_solve("F", p.n, p.A.data, p.A.indptr, p.A.indices, fpm=fpm, emin=p.emin, emax=p.emax,
                             m0=p.m0)
    ev = np.linalg.eigvalsh(p.A.to_dense())
    want = ev[(ev >= p.emin) & (ev <= p.emax)]
    assert r.info == 0 and r.M == len(want)
    assert np.abs(r.E[: r.M] - want).max() < 1e-10 * p.emax


def test_bench_workload_properties(pkg):
    """The 64^3 Laplacian + potential workload at full size with the bench's
    exact settings (N = 262144, M0 = 150, Ne = 8, ellipse ratio 200, inner
    tolerance fpm(45) = 2, fpm(46) = 80 steps, one node per COCG batch): the
    eigenvalue count equals the Sylvester-inertia count stored by the
    oracle's golden script, residuals recomputed by the oracle,
    B-orthonormality, and agreement of the mixed and FP64 solvers."""
    p = fw.laplace3d_potential(side=64, count=100, m0=150, ne=8, ratio=200, seed=1)
    gold = json.load(open(os.path.join(GOLD, "laplace3d_64_count.json")))
    mixed = run_gpu(pkg, p, 1, inner=(2, 80), maxloop=40, nb=1)
    assert mixed.info == 0 and mixed.M == gold["count_in_interval"], (mixed.info, mixed.M)
    M = mixed.M
    res = O.residuals(p.A, None, mixed.X[:, :M], mixed.E[:M], p.emin, p.emax)
    assert res.max() <= RES_TOL
    X = mixed.X[:, :M]
    assert np.abs(X.T @ X - np.eye(M)).max() < 1e-11
    full = run_gpu(pkg, p, 0, inner=(2, 80), maxloop=40, nb=1)
    assert full.info == 0 and full.M == M
    assert (np.abs(mixed.E[:M] - full.E[:M]) / mixed.E[:M]).max() <= EIG_TOL
    assert cluster_angles(mixed.E[:M], X, full.E[:M], full.X[:, :M], p.emax) <= ANG_TOL


def _scattered_spd(n, per_row, seed):
    """SPD matrix whose rows read columns spread over the whole range (random
    symmetric off-diagonal pattern, diagonally dominant): its row blocks read
    far more than 16 separate column ranges."""
    rng = np.random.default_rng(seed)
    r = np.repeat(np.arange(n), per_row)
    c = rng.integers(0, n, size=n * per_row)
    keep = r != c
    r, c = r[keep], c[keep]
    v = -rng.uniform(0.1, 1.0, size=r.size)
    rows = np.concatenate([r, c])
    cols = np.concatenate([c, r])
    vals = np.concatenate([v, v])
    off = fw.csr_from_coo(n, rows, cols, vals)
    diag = np.zeros(n)
    np.add.at(diag, off.indices, 0.0)
    for i in range(n):
        diag[i] = -off.data[off.indptr[i]:off.indptr[i + 1]].sum() + rng.uniform(0.0, 1.0)
    i = np.arange(n)
    return fw.csr_from_coo(n, np.concatenate([rows, i]), np.concatenate([cols, i]), np.concatenate([vals, diag]))


def _step_a_problems():
    rng = np.random.default_rng(7)
    s27 = fw.stencil27_spd(12, rng)
    bd = fw.diagonal_csr(rng.uniform(1.0, 2.0, s27.n))
    ev = np.linalg.eigvalsh(np.diag(1 / np.sqrt(bd.data)) @ s27.to_dense() @ np.diag(1 / np.sqrt(bd.data)))
    p27 = fw.Problem("s27", s27, bd, 0.0, 0.5 * (ev[29] + ev[30]), 48, 8, 100, 3)
    sc = _scattered_spd(1200, 4, 11)
    evs = np.linalg.eigvalsh(sc.to_dense())
    k = 8 + int(np.argmax(np.diff(evs[8:26])))  # interval edge in the widest gap after the 9th eigenvalue
    psc = fw.Problem("scattered", sc, None, evs[0] - 1e-3, 0.5 * (evs[k] + evs[k + 1]), k + 12, 8, 100, 5)
    # 27-point box with 96-row lines: an inner 32-row block stages 9 windows of 34 rows,
    # the case the producer-warp form takes (complex FP32)
    box = fw.stencil27_spd(0, rng, shape=(4, 4, 96))
    bb = fw.diagonal_csr(rng.uniform(1.0, 2.0, box.n))
    evb = np.linalg.eigvalsh(np.diag(1 / np.sqrt(bb.data)) @ box.to_dense() @ np.diag(1 / np.sqrt(bb.data)))
    pbox = fw.Problem("s27box", box, bb, 0.0, 0.5 * (evb[29] + evb[30]), 48, 8, 100, 4)
    return {"laplace3d": (fw.laplace3d_potential(side=14, count=24, m0=40, seed=7), 1),
            "stencil27_diag_b": (p27, 1),
            "stencil27_box": (pbox, 1),
            "scattered": (psc, 0)}


@pytest.mark.parametrize("mixed", [0, 1])
@pytest.mark.parametrize("name", ["laplace3d", "stencil27_diag_b", "stencil27_box", "scattered"])
def test_step_a_staged_and_cached_gathers_agree(pkg, name, mixed):
    """COCG step A either stages the rows of r each work item reads (windows
    copied into shared memory by the bulk-copy engine; default when the row
    blocks read few contiguous column ranges) or gathers through the caches
    (fpm(51) > 0, and matrices whose rows scatter).  Both give the oracle's
    eigenpairs, and each choice is the one the profile reports."""
    p, staged = _step_a_problems()[name]
    if name == "scattered":  # dense reference (the oracle's COCG converges slowly on this pattern)
        ev, V = np.linalg.eigh(p.A.to_dense())
        sel = (ev >= p.emin) & (ev <= p.emax)
        ref = {"M": int(sel.sum()), "E": ev[sel], "X": V[:, sel]}
    else:
        ref = O.feast_scsr(p.A, p.B, p.emin, p.emax, p.m0, Y0=p.y0(), ne=p.ne, ratio=p.ratio, tol_exp=10)
        assert ref["info"] == 0
    out = []
    for rows in (0, 256):
        fpm = pkg.feast_init()
        fpm[1], fpm[2], fpm[3], fpm[4], fpm[17], fpm[41] = p.ne, 10, 30, 1, p.ratio, mixed
        fpm[44], fpm[45], fpm[50], fpm[52] = 2, 200, rows, 1
        kw = {} if p.B is None else dict(b=p.B.data, ib=p.B.indptr, jb=p.B.indices)
        r = pkg.feast_scsr_solve("F", p.n, p.A.data, p.A.indptr, p.A.indices, fpm=fpm, emin=p.emin,
                                 emax=p.emax, m0=p.m0, x0=p.y0(), **kw)
        prof = pkg.feast_last_profile()
        check_against(r, ref, max(abs(p.emax), abs(p.emin)), B=p.B)
        form = int(prof["step_a_staged"])
        if rows == 0 and staged:  # the producer-warp form (2): complex FP32 blocks staging many rows
            assert form == (2 if mixed and name == "stencil27_box" else 1), prof
        else:
            assert form == 0, prof
        if form:
            assert int(prof["step_a_rows_per_item"]) in (32, 48, 64, 80)
            assert 1 <= int(prof["step_a_grid"]) <= -(-p.n // int(prof["step_a_rows_per_item"]))
        else:
            assert int(prof["step_a_rows_per_item"]) == 256
        out.append(r)
    M = out[0].M
    assert out[1].M == M
    assert np.abs(out[0].E[:M] - out[1].E[:M]).max() <= 1e-11 * max(abs(p.emax), abs(p.emin))
