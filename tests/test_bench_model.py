"""The bench's algorithmic-byte model of the two COCG launches (host logic,
no GPU): step A = 5 passes over the live lanes of a tile (r gathered, p and q
read and written) plus the matrix once per launch; step B = 4 passes plus the
quadrature accumulator's read and write.  Padded lanes are not counted."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _problem(n, nnz, m0, ne, B=None):
    return SimpleNamespace(n=n, m0=m0, ne=ne, A=SimpleNamespace(nnz=nnz), B=B)


def test_cocg_rates_full_tile():
    import bench

    # one group of 32 columns (no padding), one node per batch, complex FP32
    pr = dict(n=1000, W=32, mt=32, complex_bytes=8, groups=1, group_iterations=1, cocg_a_launches=1,
              cocg_a_ms=1.0, cocg_b_ms=1.0)
    a, b = bench.cocg_rates(pr, _problem(1000, 3000, 32, 8))
    tile = 1000 * 32 * 8                      # one pass over the tile, bytes
    csr = 3000 * (4 + 4) + 1001 * 4           # column index + FP32 value per entry, row pointers
    assert a == pytest.approx((5 * tile + csr) / 1e-3 / 1e9)
    acc = 1000 * 32 * 2 * 4                   # FP32 accumulator read and written
    assert b == pytest.approx((4 * tile + acc) / 1e-3 / 1e9)


def test_cocg_rates_excludes_padded_lanes_and_counts_diagonal_b():
    import bench

    # 150 columns in 5 groups of 32 lanes: 10 padded lanes; a diagonal B read once per launch
    pr = dict(n=4096, W=32, mt=32, complex_bytes=8, groups=5, group_iterations=10, cocg_a_launches=2,
              cocg_a_ms=2.0, cocg_b_ms=4.0)
    a, b = bench.cocg_rates(pr, _problem(4096, 28000, 150, 8, B=object()))
    live_tile = 4096 * 150 * 8                # the 150 live columns of a group-iteration's tile, summed over groups / 5
    per_gi = live_tile / 5
    csr = 28000 * 8 + 4097 * 4 + 4096 * 4     # + FP32 diagonal of B
    assert a == pytest.approx((10 * 5 * per_gi + 2 * csr) / 2e-3 / 1e9)
    acc = 4096 * 32 * 2 * 4 * (150 / 160)
    assert b == pytest.approx(10 * (4 * per_gi + acc) / 4e-3 / 1e9)
