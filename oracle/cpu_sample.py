"""Bounded CPU sample of the oracle's FEAST work on a workload -- TEST
INFRASTRUCTURE for the CPU baseline (bench.py's cpu_baseline leg and its
reference arm, and the calibration script full_solve_laplace3d_64.py).

The oracle's full FEAST solve of the 64^3 workload takes minutes, so the
baseline times a few of its shifted solves (FP64 COCG to 1e-13, the oracle's
iterative mode) on all host cores and scales them to every (node, column)
solve of every filter pass of a full solve."""
from __future__ import annotations

import time

import numpy as np

from . import contour_gauss, num_threads, shifted_solve


def sample_solve_seconds(p, seconds: float, passes: int):
    """Wall seconds of the oracle's shifted solves for a full solve of problem p
    with `passes` filter passes, extrapolated from solving `cores` start-block
    columns at the hardest node (smallest imaginary part) and at a middle node.
    Returns (seconds, cores, text)."""
    cores = num_threads()
    z, _ = contour_gauss(p.ne, p.emin, p.emax, p.ratio / 100.0)
    y = p.y0()
    nodes = [int(np.argmin(z.imag)), p.ne // 2]
    per = []
    t_all = time.time()
    for e in nodes:
        cols = y[:, :cores]
        t0 = time.time()
        shifted_solve(p.A, None, z[e], cols, method="cocg", tol=1e-13)
        per.append(time.time() - t0)  # wall s for `cores` columns with all cores busy
        if time.time() - t_all > seconds:
            break
    t_col = float(np.mean(per)) / cores
    total = t_col * p.ne * p.m0 * passes
    text = (f"COCG solves of {cores} columns at node(s) {nodes[:len(per)]} of N={p.n}, extrapolated to "
            f"{p.ne}x{p.m0} solves x {passes} filter passes")
    return total, cores, text
