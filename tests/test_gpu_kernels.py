"""GPU parity of the individual kernels against the FP64 CPU oracle (or, for
plain contractions, numpy FP64), element by element, at sizes that span
several tiles plus a ragged tail."""
import numpy as np
import pytest
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def dcsr(M, dtype=torch.float64):
    return dev(M.indptr, torch.int32), dev(M.indices, torch.int32), dev(M.data, dtype)


def to_tiles(Pstd, nb, fp64, pkg):
    """Pstd[e, i, j] complex (nb x n x m) -> tiled layout tensor (complex64/128 viewed as real pairs)."""
    W, nbp, mt = pkg.feast_filter_layout(nb, fp64)
    nbn, n, m = Pstd.shape
    G = -(-m // mt)
    T = np.zeros((G, n, W), dtype=np.complex128)
    for j in range(m):
        g, jl = divmod(j, mt)
        for e in range(nb):
            T[g, :, jl * nbp + e] = Pstd[e, :, j]
    return T, (W, nbp, mt, G)


def from_tiles(T, nb, m, lay):
    W, nbp, mt, G = lay
    n = T.shape[1]
    out = np.zeros((nb, n, m), dtype=np.complex128)
    for j in range(m):
        g, jl = divmod(j, mt)
        for e in range(nb):
            out[e, :, j] = T[g, :, jl * nbp + e]
    return out


def shifted_ref(A, B, z, Pstd):
    out = np.zeros_like(Pstd)
    for e, ze in enumerate(z):
        Pe = Pstd[e]
        ar = O.csr_mm(A, Pe.real) + 1j * O.csr_mm(A, Pe.imag)
        br = Pe if B is None else O.csr_mm(B, Pe.real) + 1j * O.csr_mm(B, Pe.imag)
        out[e] = ze * br - ar
    return out


def make_b(kind, n, side, rng):
    """B = I (None), a diagonal SPD B, or a non-diagonal SPD B with the 7-point
    pattern (the packed general-B gather path of the filter kernels)."""
    if kind == "diag":
        return fw.diagonal_csr(rng.uniform(1, 2, n))
    if kind == "general":
        return fw.mass_like_3d(side, rng)
    return None


@pytest.mark.parametrize("fp64", [0, 1])
@pytest.mark.parametrize("bkind", [None, "diag", "general"])
@pytest.mark.parametrize("nb,m", [(8, 10), (16, 3), (5, 7)])
def test_shifted_spmm(pkg, fp64, bkind, nb, m):
    rng = np.random.default_rng(10 + nb + m)
    p = fw.laplace3d_potential(side=11, count=10, m0=m, seed=4)  # n = 1331: 5 row blocks + tail
    A = p.A
    B = make_b(bkind, A.n, 11, rng)
    n = A.n
    z = rng.uniform(0, 2, nb) + 1j * rng.uniform(0.05, 1, nb)
    Pstd = rng.standard_normal((nb, n, m)) + 1j * rng.standard_normal((nb, n, m))
    T, lay = to_tiles(Pstd, nb, fp64, pkg)
    cdt = torch.complex128 if fp64 else torch.complex64
    rdt = torch.float64 if fp64 else torch.float32
    Pd = torch.as_tensor(T).to(device="cuda", dtype=cdt).contiguous()
    Vd = torch.zeros_like(Pd)
    ia, ja, av = dcsr(A)
    ib = jb = bv = None
    if B is not None:
        ib, jb, bv = dcsr(B)
    pkg.feast_shifted_spmm_dev(n, ia, ja, av, ib, jb, bv, z, m, fp64, Pd, Vd)
    got = from_tiles(Vd.cpu().numpy().astype(np.complex128), nb, m, lay)
    if not fp64:  # reference on the same rounded inputs
        Pstd = from_tiles(Pd.cpu().numpy().astype(np.complex128), nb, m, lay)
        A = fw.CSR(A.n, A.indptr, A.indices, A.data.astype(np.float32).astype(np.float64))
        if B is not None:
            B = fw.CSR(B.n, B.indptr, B.indices, B.data.astype(np.float32).astype(np.float64))
        z = z.astype(np.complex64).astype(np.complex128)
    ref = shifted_ref(A, B, z, Pstd)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < (1e-14 if fp64 else 2e-6), err


def _filter_case(side=10, m=12, seed=5):
    p = fw.laplace3d_potential(side=side, count=8, m0=m, seed=seed)
    return p


@pytest.mark.parametrize("mixed", [0, 1])
@pytest.mark.parametrize("bkind", [None, "general"])
def test_filter_classic_matches_oracle(pkg, mixed, bkind):
    p = _filter_case()
    n, m = p.n, p.m0
    Y = p.y0()
    B = make_b(bkind, n, 10, np.random.default_rng(21))
    fpm = pkg.feast_init()
    fpm[1], fpm[17], fpm[41] = 8, 100, mixed
    fpm[44], fpm[45] = (12, 3000) if not mixed else (6, 3000)
    ia, ja, av = dcsr(p.A)
    ib = jb = bv = None
    if B is not None:
        ib, jb, bv = dcsr(B)
    # right-hand side of the first pass: B Y
    R = dev(Y if B is None else O.csr_mm(B, Y))  # row-major n x m == C-order copy
    Q = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    it = pkg.feast_filter_dev(n, ia, ja, av, ib, jb, bv, m, R, R, dev(np.zeros(m)), 0, fpm, p.emin, p.emax, Q)
    assert it > 0
    ref = O.filter_block(p.A, B, 8, p.emin, p.emax, 1.0, Y)
    err = np.abs(Q.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-8 if not mixed else 2e-3), err


@pytest.mark.parametrize("mixed", [0, 1])
def test_filter_rii_matches_oracle(pkg, mixed):
    p = _filter_case(side=9, m=10, seed=6)
    n, m = p.n, p.m0
    # a block near an invariant subspace, as in later FEAST passes
    ev, V = np.linalg.eigh(p.A.to_dense())
    rng = np.random.default_rng(0)
    X = V[:, :m] + 1e-3 * rng.standard_normal((n, m))
    lam = ev[:m] + 1e-4 * rng.standard_normal(m)
    fpm = pkg.feast_init()
    fpm[1], fpm[17], fpm[41] = 8, 100, mixed
    fpm[44], fpm[45] = (12, 3000) if not mixed else (6, 3000)
    ia, ja, av = dcsr(p.A)
    # right-hand side of the residual-inverse form: R = A X - X diag(lam)
    Rm = O.csr_mm(p.A, X) - X * lam
    Q = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    pkg.feast_filter_dev(n, ia, ja, av, None, None, None, m, dev(Rm), dev(X), dev(lam), 1, fpm, p.emin, p.emax, Q)
    ref = O.filter_block(p.A, None, 8, p.emin, p.emax, 1.0, X, lam=lam, rii=True)
    err = np.abs(Q.cpu().numpy() - ref).max() / np.abs(ref).max()
    # the solve error is relative to ||R|| << ||X||, so even FP32 solves give a tight Q
    assert err < (1e-10 if not mixed else 1e-5), err


@pytest.mark.parametrize("n,m", [(1000, 70), (4097, 150), (33, 1), (262144, 150)])
def test_gram(pkg, n, m):
    rng = np.random.default_rng(n + m)
    X = rng.standard_normal((n, m))
    Y = rng.standard_normal((n, m))
    C = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    pkg.feast_gram_dev(n, m, dev(X), dev(Y), C)
    got = C.cpu().numpy()
    # the upper triangle of X^T Y, mirrored
    scale = np.sqrt(n)
    assert np.abs(got - got.T).max() == 0.0
    full = X.T @ Y
    exp = np.where(np.arange(m)[:, None] <= np.arange(m)[None, :], full, full.T)
    assert np.abs(got - exp).max() < 1e-13 * scale, np.abs(got - exp).max()


@pytest.mark.parametrize("n,m", [(1000, 70), (4097, 150), (33, 1), (262144, 150), (300, 33), (20000, 300)])
def test_gram_sliced_bf16(pkg, n, m):
    """The projections' default arithmetic: X^T Y from exact BF16 slice
    products (8 slices of 7 bits under a power-of-two column scale) against
    numpy's FP64 product, at the FP64 Gram's tolerance; sizes with ragged
    32-column tiles, a single column and more rows than one split."""
    rng = np.random.default_rng(n + 3 * m)
    X = rng.standard_normal((n, m))
    Y = rng.standard_normal((n, m))
    C = torch.full((m, m), np.nan, dtype=torch.float64, device="cuda")
    pkg.feast_gram_oz_dev(n, m, dev(X), dev(Y), C)
    got = C.cpu().numpy()
    assert np.abs(got - got.T).max() == 0.0
    full = X.T @ Y
    exp = np.where(np.arange(m)[:, None] <= np.arange(m)[None, :], full, full.T)
    assert np.abs(got - exp).max() < 1e-13 * np.sqrt(n), np.abs(got - exp).max()


def test_gram_sliced_scaling_edge_cases(pkg):
    """Columns 1e-150 .. 1e150 apart, a zero column, a column with one huge
    entry among tiny ones, and the symmetric call X = Y: each element within
    FP64 rounding of its own column norms (the column scale is per column)."""
    rng = np.random.default_rng(42)
    n, m = 5000, 40
    X = rng.standard_normal((n, m)) * np.logspace(-150, 150, m)[None, :]
    X[:, 7] = 0.0
    X[:, 11] = 1e-8 * rng.standard_normal(n)
    X[123, 11] = 3.0
    Y = rng.standard_normal((n, m)) * np.logspace(100, -100, m)[None, :]
    for Yc, same in ((Y, False), (X, True)):
        C = torch.zeros((m, m), dtype=torch.float64, device="cuda")
        Xd = dev(X)
        pkg.feast_gram_oz_dev(n, m, Xd, Xd if same else dev(Yc), C)
        got = C.cpu().numpy()
        full = X.T @ Yc
        exp = np.where(np.arange(m)[:, None] <= np.arange(m)[None, :], full, full.T)
        nx, ny = np.linalg.norm(X, axis=0), np.linalg.norm(Yc, axis=0)
        lo, hi = np.minimum.outer(np.arange(m), np.arange(m)), np.maximum.outer(np.arange(m), np.arange(m))
        scale = nx[lo] * ny[hi]
        bad = np.abs(got - exp) > 1e-13 * scale + 1e-300
        assert not bad.any(), np.argwhere(bad)[:5]
        assert np.all(got[7, 7:] == 0.0)  # X's zero column: row 7 of the upper triangle
        if same:
            assert np.all(got[7, :] == 0.0) and np.all(got[:, 7] == 0.0)


@pytest.mark.parametrize("n,m,k", [(1000, 70, 65), (129, 150, 150), (7, 3, 2)])
def test_gemm(pkg, n, m, k):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, m))
    V = rng.standard_normal((m, k))
    C = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    pkg.feast_gemm_dev(n, m, k, dev(A), dev(V), C)
    assert np.abs(C.cpu().numpy() - A @ V).max() < 1e-13 * np.sqrt(m)


@pytest.mark.parametrize("n,m,k", [(1000, 70, 65), (129, 150, 150), (7, 3, 2), (262144, 150, 150), (3000, 300, 300),
                                   (500, 301, 33)])
def test_gemm_sliced_bf16(pkg, n, m, k):
    """X = Q V, the Ritz vectors' default arithmetic, from exact BF16 slice
    products under row and column power-of-two scales, against numpy FP64;
    rows of very different size and a zero row are included."""
    rng = np.random.default_rng(n + m + k)
    A = rng.standard_normal((n, m)) * np.logspace(-30, 30, n)[:, None]
    A[n // 2] = 0.0
    V = rng.standard_normal((m, k))
    C = torch.full((n, k), np.nan, dtype=torch.float64, device="cuda")
    pkg.feast_gemm_oz_dev(n, m, k, dev(A), dev(V), C)
    got = C.cpu().numpy()
    exp = A @ V
    scale = np.linalg.norm(A, axis=1)[:, None] * np.linalg.norm(V, axis=0)[None, :]
    err = np.abs(got - exp) / np.maximum(scale, 1e-300)
    assert err.max() < 1e-14, err.max()
    assert np.all(got[n // 2] == 0.0)


@pytest.mark.parametrize("m", [1, 2, 7, 64, 151, 300])
def test_sym_eig_matches_oracle(pkg, m):
    rng = np.random.default_rng(m)
    a = rng.standard_normal((m, m))
    a = a + a.T
    A = dev(a)
    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    V = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    sweeps = pkg.feast_sym_eig_dev(m, A, lam, V)
    w, _, _ = O.jacobi_eig(a)
    lg = lam.cpu().numpy()
    Vg = V.cpu().numpy()
    nrm = max(1.0, np.abs(w).max())
    assert np.abs(lg - w).max() < 1e-12 * nrm
    assert np.abs(Vg.T @ Vg - np.eye(m)).max() < 1e-12
    assert np.abs(a @ Vg - Vg * lg).max() < 1e-11 * nrm
    assert sweeps < 40


def test_sym_eig_degenerate_and_diagonal(pkg):
    m = 40
    rng = np.random.default_rng(1)
    Qm, _ = np.linalg.qr(rng.standard_normal((m, m)))
    d = np.repeat([1.0, 2.0, 5.0, -3.0], 10)
    a = Qm @ np.diag(d) @ Qm.T
    a = 0.5 * (a + a.T)
    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    V = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    pkg.feast_sym_eig_dev(m, dev(a), lam, V)
    assert np.abs(lam.cpu().numpy() - np.sort(d)).max() < 1e-12
    # already diagonal: no rotation needed
    lam2 = torch.zeros(m, dtype=torch.float64, device="cuda")
    sw = pkg.feast_sym_eig_dev(m, dev(np.diag(d)), lam2, V)
    assert sw <= 1 and np.array_equal(lam2.cpu().numpy(), np.sort(d))


def _reduced_case(kind, m, rng):
    a = rng.standard_normal((m, m)); a = a + a.T
    if kind == "random":
        g = rng.standard_normal((m, m)); b = g @ g.T + 0.5 * np.eye(m)
    elif kind == "near_identity":  # a filtered subspace after a few loops: B_Q = D (I + E) D
        e = 1e-3 * rng.standard_normal((m, m)); e = e + e.T
        dg = rng.uniform(1e-4, 1.0, m)
        b = dg[:, None] * (np.eye(m) + e) * dg[None, :]
        a = dg[:, None] * (np.diag(np.sort(rng.uniform(-1, 1, m))) + 1e-3 * a) * dg[None, :]
    else:  # full rank, condition 1e9: the Cholesky factor is rejected (||L^-1||_F^2 >= 1e9)
        qm, _ = np.linalg.qr(rng.standard_normal((m, m)))
        b = qm @ np.diag(np.logspace(0, -9, m)) @ qm.T
        b = 0.5 * (b + b.T)
    return a, b


@pytest.mark.parametrize("kind,m", [("random", 40), ("random", 150), ("random", 200), ("near_identity", 150),
                                    ("near_identity", 200), ("ill", 60)])
def test_reduced_eig_matches_oracle(pkg, kind, m):
    """Both routes of the reduced generalized solver (Cholesky factor in
    shared or global memory; Jacobi on B~ when the factor is rejected)."""
    rng = np.random.default_rng(3 + m)
    a, b = _reduced_case(kind, m, rng)
    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    V = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    mk = pkg.feast_reduced_eig_dev(m, dev(a), dev(b), lam, V)
    info, lo, Vo = O.reduced_gev(a, b)
    assert mk == len(lo) == m
    lg = lam.cpu().numpy()
    Vg = V.cpu().numpy()
    if kind == "ill":  # eigenvalue perturbations of order eps * cond(B) = 2e-7 of the largest
        assert np.abs(lg - lo).max() < 1e-6 * np.abs(lo).max()
        return
    assert np.abs(lg - lo).max() < 1e-11 * np.abs(lo).max()
    assert np.abs(Vg.T @ b @ Vg - np.eye(m)).max() < 1e-11
    assert np.abs(a @ Vg - (b @ Vg) * lg).max() < 1e-11 * np.abs(lo).max() * np.abs(b).max()


def test_reduced_eig_rank_deficient(pkg):
    rng = np.random.default_rng(4)
    Qb = rng.standard_normal((60, 7))
    Qb = np.hstack([Qb, Qb[:, :3] @ rng.standard_normal((3, 3))])  # rank 7 of 10
    a = rng.standard_normal((60, 60)); a = a + a.T
    Aq, Bq = Qb.T @ a @ Qb, Qb.T @ Qb
    m = 10
    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    V = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    mk = pkg.feast_reduced_eig_dev(m, dev(Aq), dev(Bq), lam, V)
    info, lo, _ = O.reduced_gev(Aq, Bq)
    assert mk == len(lo) == 7
    lg = lam.cpu().numpy()
    assert np.abs(lg[:7] - lo).max() < 1e-8 * np.abs(lo).max()
    assert np.all(lg[7:] >= 1e299)


@pytest.mark.parametrize("bkind", [None, "diag", "general"])
def test_residual_matches_oracle(pkg, bkind):
    rng = np.random.default_rng(8)
    p = fw.laplace3d_potential(side=13, count=10, m0=37, seed=2)
    A = p.A
    B = make_b(bkind, A.n, 13, rng)
    gen = B is not None
    X = rng.standard_normal((A.n, 37))
    lam = rng.uniform(0, 1, 37)
    R = torch.zeros((A.n, 37), dtype=torch.float64, device="cuda")
    res = torch.zeros(37, dtype=torch.float64, device="cuda")
    ia, ja, av = dcsr(A)
    ib = jb = bv = None
    if gen:
        ib, jb, bv = dcsr(B)
    pkg.feast_residual_dev(A.n, ia, ja, av, ib, jb, bv, 37, dev(X), dev(lam), 1.7, R, res)
    ref = O.residuals(A, B, X, lam, -1.7, 0.5)
    assert np.abs(res.cpu().numpy() - ref).max() < 1e-13 * ref.max()
    BX = X if B is None else O.csr_mm(B, X)
    assert np.abs(R.cpu().numpy() - (O.csr_mm(A, X) - BX * lam)).max() < 1e-12


def test_jacobi_barrier_time_limit_returns_error_and_recovers(pkg):
    """The reduced eigensolver's cooperative Jacobi waits at a bounded grid
    barrier.  With a one-cycle spin limit the barrier of a multi-CTA launch
    (m = 150, about 40 CTAs) gives up: the kernel-level call fails with -3 and
    a full solve returns info -3, with no hang.  With the default limit back,
    the same calls succeed on the same context and match the oracle."""
    from paper_2002_04807_gb300 import FeastError

    m = 150
    rng = np.random.default_rng(77)
    a = rng.standard_normal((m, m))
    a = a + a.T
    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    V = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    p = fw.laplace3d_potential(side=12, count=30, m0=100, seed=9)
    fpm = pkg.feast_init()
    fpm[1], fpm[2], fpm[4], fpm[17], fpm[44], fpm[45] = 8, 10, 1, 100, 2, 200

    def solve():
        return pkg.feast_scsr_solve("F", p.n, p.A.data, p.A.indptr, p.A.indices, fpm=fpm.copy(), emin=p.emin,
                                    emax=p.emax, m0=p.m0, x0=p.y0())

    prev = pkg.feast_set_wait_limit(1)
    try:
        with pytest.raises(FeastError, match="-3"):
            pkg.feast_sym_eig_dev(m, dev(a), lam, V)
        # the filter's staged-row waits share the limit: whichever bounded wait
        # gives up first ends the solve (-3 reduced solver, -4 filter copies)
        assert solve().info in (-3, -4)
    finally:
        restored = pkg.feast_set_wait_limit(0)
    assert prev == 4_000_000_000 and restored == 1
    torch.cuda.synchronize()  # the context is still usable
    pkg.feast_sym_eig_dev(m, dev(a), lam, V)
    w, _, _ = O.jacobi_eig(a)
    assert np.abs(lam.cpu().numpy() - w).max() < 1e-12 * np.abs(w).max()
    r = solve()
    ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=100, tol_exp=10)
    assert r.info == 0 and r.M == ref["M"]
    assert np.abs(r.E[: r.M] - ref["E"][: r.M]).max() <= 1e-10 * p.emax


@pytest.mark.parametrize("mixed", [0, 1])
@pytest.mark.parametrize("rows", [0, 256])
@pytest.mark.parametrize("cap", [1, 6])
def test_filter_iteration_cap_matches_capped_cocg(pkg, mixed, rows, cap):
    """With the inner tolerance out of reach, every column stops at the
    iteration cap fpm(46): the filter must equal the quadrature sum of the
    oracle's COCG iterates after exactly `cap` steps, with step A staging its
    gathered rows (fpm(51) = 0) or gathering through the caches (256)."""
    p = _filter_case()
    n, m = p.n, p.m0
    Y = p.y0()
    fpm = pkg.feast_init()
    fpm[1], fpm[17], fpm[41] = 8, 100, mixed
    fpm[44], fpm[45], fpm[50] = 16, cap, rows
    ia, ja, av = dcsr(p.A)
    R = dev(Y)
    Q = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    it = pkg.feast_filter_dev(n, ia, ja, av, None, None, None, m, R, R, dev(np.zeros(m)), 0, fpm, p.emin, p.emax, Q)
    assert it == cap
    z, w = O.contour_gauss(8, p.emin, p.emax, 1.0)
    ref = np.zeros((n, m))
    scale = np.zeros((n, m))
    for ze, we in zip(z, w):
        Ye, its = O.shifted_solve(p.A, None, complex(ze), Y, method="cocg", tol=0.0, maxit=cap)
        assert (its == cap).all()
        ref += np.real(we * Ye)
        scale += np.abs(we * Ye)
    # relative to the size of the quadrature terms: after one step the sum is
    # the filter value at each column's Rayleigh quotient, far outside the
    # interval, and cancels to a tiny fraction of its terms
    err = np.abs(Q.cpu().numpy() - ref).max() / scale.max()
    assert err < (1e-12 if not mixed else 1e-4), err


@pytest.mark.parametrize("mixed", [0, 1])
def test_staged_copy_wait_limit_is_bounded(pkg, mixed):
    """The staged gathering step waits for its bulk copies on an mbarrier with
    the library's spin limit.  With a one-cycle limit each wait either sees the
    copies land within the hardware's own try-wait interval or gives up: the
    filter call then returns with the error flag read by the host (-4), never
    hangs, and leaves the context usable; with the default limit restored the
    same call matches the oracle."""
    p = _filter_case(side=16, m=24, seed=3)
    n, m = p.n, p.m0
    Y = p.y0()
    fpm = pkg.feast_init()
    fpm[1], fpm[17], fpm[41] = 8, 100, mixed
    fpm[44], fpm[45] = (12, 3000) if not mixed else (6, 3000)
    ia, ja, av = dcsr(p.A)
    R = dev(Y)
    from paper_2002_04807_gb300 import FeastError

    Q = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    prev = pkg.feast_set_wait_limit(1)
    try:
        try:
            pkg.feast_filter_dev(n, ia, ja, av, None, None, None, m, R, R, dev(np.zeros(m)), 0, fpm, p.emin,
                                 p.emax, Q)
        except FeastError as exc:
            assert "-4" in str(exc), exc
    finally:
        pkg.feast_set_wait_limit(0)
    torch.cuda.synchronize()
    Q.zero_()
    pkg.feast_filter_dev(n, ia, ja, av, None, None, None, m, R, R, dev(np.zeros(m)), 0, fpm, p.emin, p.emax, Q)
    ref = O.filter_block(p.A, None, 8, p.emin, p.emax, 1.0, Y)
    err = np.abs(Q.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-8 if not mixed else 2e-3), err
