"""Writes laplace3d_64_count.json: the number of eigenvalues of the 64^3
7-point Laplacian + potential workload (V ~ U[0, 0.5], seed 1) in its search
interval [Emin, Emax], counted by Sylvester's law of inertia with the oracle's
block-tridiagonal LDL^T over the 64 grid planes (oracle.count_below_planes).
Test infrastructure: calls only the oracle and the seeded generator.  Takes a
few minutes per interval end on 8 host cores.

    python tests/golden/make_laplace3d_64_count.py
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import feast_workloads as fw  # noqa: E402
import oracle as O  # noqa: E402


def fingerprint(p):
    h = hashlib.sha1()
    for a in (p.A.indptr, p.A.indices, p.A.data):
        h.update(a.tobytes())
    return {"n": p.n, "nnz": int(p.A.nnz), "emin": repr(p.emin), "emax": repr(p.emax), "csr_sha1": h.hexdigest()}


def main():
    side = 64
    p = fw.laplace3d_potential(side=side, count=100, m0=150, ne=8, ratio=200, seed=1)
    t0 = time.time()
    below_max = O.count_below_planes(p.A, None, p.emax, side * side)
    below_min = O.count_below_planes(p.A, None, p.emin, side * side)
    out = {"workload": "laplace3d_potential(side=64, count=100, seed=1): 7-point Dirichlet Laplacian 64^3 + "
                       "diag(V), V ~ U[0, 0.5]; B = I",
           "fingerprint": fingerprint(p),
           "count_below_emax": below_max, "count_below_emin": below_min,
           "count_in_interval": below_max - below_min,
           "method": "Sylvester inertia, block-tridiagonal LDL^T over 64 grid planes (oracle.count_below_planes)",
           "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "laplace3d_64_count.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
