"""Full FP64 oracle FEAST solve of the 64^3 Laplacian + potential workload
(N = 262144, V ~ U[0, 0.5] seed 1, B = I, [0, Emax] with Emax from the
closed-form estimate, M0 = 150, Ne = 8 Gauss nodes, ellipse ratio 200, start
block seed 1, stop at relative residual 1e-10), in the oracle's iterative mode
(FP64 COCG shifted solves to 1e-13), timed on all host cores.  TEST
INFRASTRUCTURE: it calibrates the CPU baseline, whose timed runs only sample
a few shifted solves and extrapolate (oracle/cpu_sample.py); it writes
full_solve_laplace3d_64.json (wall time, cores, refinement loops, eigenvalue
count, the sample's estimate on the same host and their ratio) next to this
file.

    python oracle/full_solve_laplace3d_64.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import feast_workloads as fw  # noqa: E402
import oracle as O  # noqa: E402


def main():
    p = fw.laplace3d_potential(side=64, count=100, m0=150, ne=8, ratio=200, seed=1)
    O.build()
    from oracle.cpu_sample import sample_solve_seconds

    y0 = p.y0()
    t0 = time.time()
    r = O.feast_scsr(p.A, None, p.emin, p.emax, p.m0, Y0=y0, ne=p.ne, ratio=p.ratio, tol_exp=10, maxloop=20,
                     solver="cocg", solve_tol=1e-13)
    wall = time.time() - t0
    M = r["M"]
    # the bounded sample the CPU baseline times, on the same host, for the
    # oracle's own number of filter passes: its ratio to the full solve is the
    # baseline's calibration factor
    est, _, text = sample_solve_seconds(p, 20.0, r["loop"] + 1)
    out = {"workload": "laplace3d_potential(side=64, count=100, m0=150, ne=8, ratio=200, seed=1)",
           "solver": "oracle FEAST, FP64 COCG shifted solves to 1e-13, Gauss Ne = 8, tol 1e-10",
           "cores": O.num_threads(), "wall_s": round(wall, 2), "info": r["info"], "M": M,
           "loops": r["loop"], "filter_passes": r["loop"] + 1, "cocg_iterations": int(r["inner_iters"]),
           "max_residual": float(np.max(r["res"][:M])) if M else None,
           "eigenpairs_per_s": M / wall if wall > 0 else None,
           "sample_estimate_s": round(est, 2), "sample": text,
           "calibration": round(wall / est, 4) if est > 0 else None,
           "host": os.uname().machine}
    with open(os.path.join(HERE, "full_solve_laplace3d_64.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
