"""Batched FEAST (many independent problems in one launch sequence) against
the FP64 oracle, problem by problem."""
import numpy as np
import pytest
import torch

import feast_workloads as fw
import oracle as O

pytestmark = pytest.mark.gpu
EIG_TOL, RES_TOL = 1e-10, 1e-10


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_04807_gb300 import build

    build.build()
    import paper_2002_04807_gb300 as p

    p.library()
    assert torch.cuda.is_available()
    return p


def _fpm(pkg, mixed=1, tol=10):
    f = pkg.feast_init()
    f[1], f[2], f[3], f[17], f[41], f[44], f[45] = 8, tol, 40, 200, mixed, 2, 80
    return f


def _as_dicts(probs, B=None, with_x0=True):
    out = []
    for k, p in enumerate(probs):
        d = dict(n=p.n, a=p.A.data, ia=p.A.indptr, ja=p.A.indices, emin=p.emin, emax=p.emax, m0=p.m0,
                 x0=p.y0() if with_x0 else None)
        if B is not None:
            d.update(b=B[k].data, ib=B[k].indptr, jb=B[k].indices)
        out.append(d)
    return out


def _sin_angle(U, V):
    qu, _ = np.linalg.qr(U)
    qv, _ = np.linalg.qr(V)
    return float(np.linalg.norm(qu - qv @ (qv.T @ qu), 2))


@pytest.mark.parametrize("mixed", [1, 0])
def test_batch_matches_oracle(pkg, mixed):
    probs = fw.batched_laplace2d(count=12, seed=7, side_lo=12, side_hi=40)
    st, res = pkg.feast_scsr_solve_batched(_as_dicts(probs), _fpm(pkg, mixed))
    assert st == 0
    for p, r in zip(probs, res):
        ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=200, tol_exp=10)
        assert ref["info"] == 0
        assert r.info == 0 and r.M == ref["M"], (p.name, r.info, r.M, ref["M"])
        M = r.M
        assert np.abs(r.E[:M] - ref["E"][:M]).max() <= EIG_TOL * np.abs(ref["E"][:M]).max()
        assert r.res[:M].max() <= RES_TOL
        assert np.abs(r.X[:, :M].T @ r.X[:, :M] - np.eye(M)).max() < 1e-11
        assert O.count_below(p.A, None, p.emax) - O.count_below(p.A, None, p.emin) == M


def test_batch_generalized_and_random_starts(pkg):
    import scipy.linalg

    probs = fw.batched_laplace2d(count=5, seed=9, side_lo=10, side_hi=30)
    rng = np.random.default_rng(3)
    B = [fw.diagonal_csr(rng.uniform(1, 2, p.n)) for p in probs]
    spectra = []
    for p, b in zip(probs, B):  # interval around the wanted count of the (A, B) spectrum
        ev = scipy.linalg.eigh(p.A.to_dense(), b.to_dense(), eigvals_only=True)
        k = p.notes["target_count"]
        p.emax = 0.5 * (ev[k - 1] + ev[k])
        p.emin = ev[0] - 0.05 * (p.emax - ev[0])
        p.m0 = int(np.ceil(1.5 * k))
        spectra.append(ev)
    st, res = pkg.feast_scsr_solve_batched(_as_dicts(probs, B, with_x0=False), _fpm(pkg))
    assert st == 0
    for p, b, r, ev in zip(probs, B, res, spectra):
        want = ev[(ev >= p.emin) & (ev <= p.emax)]
        assert r.info == 0 and r.M == len(want)
        assert np.abs(r.E[: r.M] - want).max() <= EIG_TOL * np.abs(want).max()
        X = r.X[:, : r.M]
        assert np.abs(X.T @ b.to_dense() @ X - np.eye(r.M)).max() < 1e-11


@pytest.mark.parametrize("mixed", [1, 0])
def test_batch_nondiagonal_b_matches_oracle(pkg, mixed):
    """Every problem with its own non-diagonal SPD B (5-point mass-like
    pattern): the batched general-B filter gathers and Rayleigh-Ritz against
    the oracle problem by problem."""
    import scipy.linalg

    probs = fw.batched_laplace2d(count=6, seed=11, side_lo=10, side_hi=28)
    rng = np.random.default_rng(5)
    B = []
    for p in probs:
        side = int(round(np.sqrt(p.n)))
        b = fw.mass_like_grid((side, side), rng)
        ev = scipy.linalg.eigh(p.A.to_dense(), b.to_dense(), eigvals_only=True)
        k = p.notes["target_count"]
        p.emax = 0.5 * (ev[k - 1] + ev[k])
        p.emin = ev[0] - 0.05 * (p.emax - ev[0])
        p.m0 = int(np.ceil(1.5 * k))
        B.append(b)
    st, res = pkg.feast_scsr_solve_batched(_as_dicts(probs, B), _fpm(pkg, mixed))
    assert st == 0
    for p, b, r in zip(probs, B, res):
        ref = O.feast_scsr(p.A, b, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=200, tol_exp=10)
        assert ref["info"] == 0
        assert r.info == 0 and r.M == ref["M"] == p.notes["target_count"], (p.name, r.info, r.M, ref["M"])
        M = r.M
        assert np.abs(r.E[:M] - ref["E"][:M]).max() <= EIG_TOL * np.abs(ref["E"][:M]).max()
        assert r.res[:M].max() <= RES_TOL
        X = r.X[:, :M]
        assert np.abs(X.T @ O.csr_mm(b, X) - np.eye(M)).max() < 1e-11


def test_batched_workload_512_problems(pkg):
    """512 2D Laplacians + potential, sides log-uniform in [32, 256], 8-64
    wanted eigenvalues each, M0 = 1.5 x count: every problem converges, the
    oracle's residuals confirm every result, and a sample of problems matches
    the oracle's own FEAST run."""
    probs = fw.batched_laplace2d()
    st, res = pkg.feast_scsr_solve_batched(_as_dicts(probs, with_x0=False), _fpm(pkg))
    assert st == 0
    for p, r in zip(probs, res):
        assert r.info == 0, (p.name, r.info)
        assert r.res[: r.M].max() <= RES_TOL
        chk = O.residuals(p.A, None, r.X[:, : r.M], r.E[: r.M], p.emin, p.emax)
        assert chk.max() <= RES_TOL, p.name
    rng = np.random.default_rng(1)
    for k in rng.choice(len(probs), 6, replace=False):
        p, r = probs[k], res[k]
        if p.n > 20000:
            continue
        ref = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=p.y0(), ne=8, ratio=200, tol_exp=10)
        assert r.M == ref["M"]
        assert np.abs(r.E[: r.M] - ref["E"][: r.M]).max() <= EIG_TOL * np.abs(ref["E"][: r.M]).max()
