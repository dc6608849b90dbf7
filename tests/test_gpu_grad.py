"""Differentiation of FEAST eigenvalues on the GPU: the SDDMM backward kernel
against the oracle's gradient, the autograd wrapper against a dense FP64
reference gradient, and the 48^3 workload against central finite
differences (h = 1e-6) of the loss L = sum_k g_k lambda_k on 50 stored
entries."""
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


def _dcsr(M):
    return (torch.as_tensor(M.indptr).cuda(), torch.as_tensor(M.indices).cuda(),
            torch.as_tensor(M.data).cuda().requires_grad_(True))


def _fpm(pkg, ratio=100, tol=12, mixed=1):
    f = pkg.feast_init()
    f[1], f[2], f[3], f[17], f[41], f[44], f[45] = 8, tol, 40, ratio, mixed, 2, 200
    f[49] = 1
    return f


def test_grad_kernel_matches_oracle(pkg):
    rng = np.random.default_rng(5)
    A = fw.laplace3d_potential(side=13, count=10, m0=20, seed=2).A
    X = rng.standard_normal((A.n, 37))
    w = rng.standard_normal(37)
    ia, ja, _ = _dcsr(A)
    g = torch.zeros(A.nnz, dtype=torch.float64, device="cuda")
    pkg.feast_eig_grad_dev(A.n, ia, ja, 37, torch.as_tensor(X).cuda().contiguous(), torch.as_tensor(w).cuda(), g)
    ref = O.eig_grad(A, X, w)
    assert np.abs(g.cpu().numpy() - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("gen", [False, True])
def test_autograd_matches_dense_reference(pkg, gen):
    """12^3 instance of the differentiation workload: gradient of sum g_k lambda_k
    over all stored entries against a dense FP64 eigendecomposition."""
    from paper_2002_04807_gb300.autograd import feast_eigenvalues

    p = fw.laplace3d_grad(side=12, count=20, m0=32)
    A = p.A
    rng = np.random.default_rng(9)
    B = fw.diagonal_csr(rng.uniform(1, 2, A.n)) if gen else None
    db = np.eye(A.n) if B is None else B.to_dense()
    lam, V = scipy.linalg.eigh(A.to_dense(), db)
    emax = 0.5 * (lam[19] + lam[20])
    ia, ja, av = _dcsr(A)
    kw = {}
    if gen:
        ib, jb, bv = _dcsr(B)
        kw = dict(b=bv, ib=ib, jb=jb)
    x0 = torch.as_tensor(np.ascontiguousarray(fw.gaussian_block(A.n, 32, 4).T)).cuda()
    ev = feast_eigenvalues(av, ia, ja, A.n, 0.0, emax, 32, _fpm(pkg), x0=x0, **kw)
    assert ev.numel() == 20
    assert np.abs(ev.detach().cpu().numpy() - lam[:20]).max() < 1e-10 * emax
    g = fw.loss_weights(20, 4)
    (torch.as_tensor(g).cuda() * ev).sum().backward()
    ref_a = O.eig_grad(A, V[:, :20], g)
    assert np.abs(av.grad.cpu().numpy() - ref_a).max() < 1e-9 * np.abs(ref_a).max()
    if gen:
        ref_b = O.eig_grad(B, V[:, :20], -g * lam[:20])
        assert np.abs(bv.grad.cpu().numpy() - ref_b).max() < 1e-9 * np.abs(ref_b).max()


def test_gradient_finite_differences_48cube(pkg):
    """48^3 Laplacian + potential, lowest 64 eigenvalues, M0 = 96: backward
    against central differences on 50 random stored entries."""
    from paper_2002_04807_gb300.autograd import feast_eigenvalues

    p = fw.laplace3d_grad()
    A = p.A
    n = A.n
    ia, ja, av = _dcsr(A)
    f = _fpm(pkg, ratio=200, tol=13)
    x0 = torch.as_tensor(np.ascontiguousarray(p.y0().T)).cuda()
    ev = feast_eigenvalues(av, ia, ja, n, p.emin, p.emax, p.m0, f, x0=x0)
    M = ev.numel()
    assert 48 <= M <= 80
    g = fw.loss_weights(M, 4)
    (torch.as_tensor(g).cuda() * ev).sum().backward()
    grad = av.grad.cpu().numpy()
    # warm start every perturbed solve from the unperturbed eigenvectors
    r0 = pkg.feast_scsr_solve_dev(n, ia, ja, av.detach(), fpm=f, emin=p.emin, emax=p.emax, m0=p.m0, x=x0.clone())
    xw = torch.zeros((p.m0, n), dtype=torch.float64, device="cuda")
    xw[: r0.m0] = r0.X[: r0.m0]
    rng = np.random.default_rng(17)
    h = 1e-6
    worst = 0.0
    for pidx in rng.choice(A.nnz, 50, replace=False):
        i = int(np.searchsorted(A.indptr, pidx, side="right") - 1)
        j = int(A.indices[pidx])
        q = A.indptr[j] + int(np.nonzero(A.indices[A.indptr[j]:A.indptr[j + 1]] == i)[0][0])
        vals = []
        for sgn in (+1, -1):
            a2 = av.detach().clone()
            a2[pidx] += sgn * h
            if q != pidx:
                a2[q] += sgn * h
            fw_ = f.copy()
            fw_[4] = 1
            r = pkg.feast_scsr_solve_dev(n, ia, ja, a2, fpm=fw_, emin=p.emin, emax=p.emax, m0=p.m0, x=xw.clone())
            assert r.info == 0 and r.M == M
            vals.append(np.dot(g, r.E[:M]))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = grad[pidx] + (grad[q] if q != pidx else 0.0)
        worst = max(worst, abs(fd - an) / (1e-5 + 1e-4 * abs(an)))
        assert abs(fd - an) <= 1e-5 + 1e-4 * abs(an), (pidx, fd, an)
    assert worst <= 1.0


@pytest.mark.parametrize("bkind", [None, "general"])
def test_host_grad_entry_point_matches_dense_reference(pkg, bkind):
    """feast_scsr_grad (host buffers, the boundary's gradient call) on the
    eigenpairs feast_scsr_solve returns for a 12^3 problem: grad_a and grad_b
    against the oracle's gradient on a dense FP64 eigendecomposition, per
    stored entry of the full patterns (B = I, or a non-diagonal SPD B)."""
    p = fw.laplace3d_grad(side=12, count=20, m0=32)
    A = p.A
    B = fw.mass_like_3d(12, np.random.default_rng(3)) if bkind else None
    lam, V = scipy.linalg.eigh(A.to_dense(), np.eye(A.n) if B is None else B.to_dense())
    emax = 0.5 * (lam[19] + lam[20])
    f = _fpm(pkg)
    f[4] = 1
    kw = {} if B is None else dict(b=B.data, ib=B.indptr, jb=B.indices)
    r = pkg.feast_scsr_solve("F", A.n, A.data, A.indptr, A.indices, fpm=f, emin=0.0, emax=emax, m0=32,
                             x0=fw.gaussian_block(A.n, 32, 4), **kw)
    assert r.info == 0 and r.M == 20
    g = fw.loss_weights(20, 4)
    ga, gb = pkg.feast_scsr_grad("F", A.n, A.indptr, A.indices, r.X[:, :20], g,
                                 ib=None if B is None else B.indptr, jb=None if B is None else B.indices,
                                 e=r.E[:20])
    ref_a = O.eig_grad(A, V[:, :20], g)
    assert np.abs(ga - ref_a).max() < 1e-9 * np.abs(ref_a).max()
    if B is None:
        assert gb is None
    else:
        ref_b = O.eig_grad(B, V[:, :20], -g * lam[:20])
        assert np.abs(gb - ref_b).max() < 1e-9 * np.abs(ref_b).max()


def test_host_grad_half_storage_and_one_based(pkg):
    """'L' storage with 1-based indices: a stored off-diagonal value stands for
    both symmetric entries, so its derivative is the sum of the two full-
    storage derivatives; diagonal entries keep theirs.  Exact against the
    oracle's entry-wise gradient on the same eigenvectors."""
    rng = np.random.default_rng(12)
    A = fw.laplace3d_potential(side=9, count=10, m0=16, seed=3).A
    X = rng.standard_normal((A.n, 23))
    g = rng.standard_normal(23)
    full = O.eig_grad(A, X, g)
    L = fw.csr_from_dense(np.tril(A.to_dense()))
    ga, _ = pkg.feast_scsr_grad("L", A.n, L.indptr + 1, L.indices + 1, X, g)
    rows = np.repeat(np.arange(A.n), np.diff(A.indptr))
    want = []
    for i, j in zip(np.repeat(np.arange(A.n), np.diff(L.indptr)), L.indices):
        pij = np.nonzero((rows == i) & (A.indices == j))[0][0]
        pji = np.nonzero((rows == j) & (A.indices == i))[0][0]
        want.append(full[pij] + (full[pji] if i != j else 0.0))
    assert np.abs(ga - np.array(want)).max() < 1e-13 * np.abs(full).max()
