"""The allocation-free Gram entry point, for callers that cannot allocate
device memory when they call the library (a memory pool owned by another
runtime, no implicit cudaMalloc synchronisation allowed, no workspace
argument in their interface).  Its output must match the allocating
feast_gram_dev on consecutive calls, which also shows that the shared fixed
scratch carries nothing stale from one call to the next.  This file sorts
last so a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_04807_gb300 import build

    build.build()
    import paper_2002_04807_gb300 as p

    p.library()
    assert torch.cuda.is_available()
    return p


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def test_noalloc_gram_matches_allocating_entry_point(pkg):
    rng = np.random.default_rng(2024)
    # two calls in a row with different inputs and shapes: the second must not
    # see anything of the first
    for n, m in [(262144, 150), (4097, 70), (262144, 150)]:
        X = rng.standard_normal((n, m))
        Y = rng.standard_normal((n, m))
        Xd, Yd = _dev(X), _dev(Y)
        ref = torch.zeros((m, m), dtype=torch.float64, device="cuda")
        got = torch.full((m, m), np.nan, dtype=torch.float64, device="cuda")
        pkg.feast_gram_dev(n, m, Xd, Yd, ref)
        pkg.feast_gram_noalloc_dev(n, m, Xd, Yd, got)
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        # same tolerance as the Gram parity test
        assert np.abs(g - r).max() < 1e-13 * np.sqrt(n), np.abs(g - r).max()
        assert np.abs(g - g.T).max() == 0.0


@pytest.mark.parametrize("n,m", [(300, 1448), (20000, 400), (262144, 150)])
def test_noalloc_gram_at_limits_matches_numpy(pkg, n, m):
    """Against numpy's FP64 X^T Y (upper triangle mirrored, as the Rayleigh-
    Ritz projection uses it) at the sizes where the fixed array bounds the
    split: m = 1448 fills it with one split; at (20000, 400) and (262144, 150)
    the split count the allocating path would take (22, 102) is capped at what
    fits (13, 93)."""
    rng = np.random.default_rng(n + m)
    X = rng.standard_normal((n, m))
    Y = rng.standard_normal((n, m))
    got = torch.full((m, m), np.nan, dtype=torch.float64, device="cuda")
    pkg.feast_gram_noalloc_dev(n, m, _dev(X), _dev(Y), got)
    g = got.cpu().numpy()
    full = X.T @ Y
    exp = np.where(np.arange(m)[:, None] <= np.arange(m)[None, :], full, full.T)
    assert np.abs(g - exp).max() < 1e-13 * np.sqrt(n), np.abs(g - exp).max()


def test_noalloc_gram_rejects_oversized_subspace(pkg):
    from paper_2002_04807_gb300 import FeastError

    m = 1449
    X = torch.zeros((4, m), dtype=torch.float64, device="cuda")
    C = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    with pytest.raises(FeastError, match="-102"):
        pkg.feast_gram_noalloc_dev(4, m, X, X, C)
    assert "fixed scratch" in pkg.feast_last_error()
