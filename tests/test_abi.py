"""CPU checks of the C ABI: the library builds/loads, exports every symbol the
header declares, and its host-side logic (defaults, contour nodes, tile
layout, argument validation) agrees with the oracle and the guide.  None of
these calls reaches the GPU."""
import os
import re
import subprocess

import numpy as np
import pytest

import feast_workloads as fw
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "feast_gb300.h")


@pytest.fixture(scope="module")
def pkg():
    from paper_2002_04807_gb300 import build

    build.build()
    import paper_2002_04807_gb300 as p

    p.library()
    return p


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(feast_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(pkg):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (feast_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    from paper_2002_04807_gb300 import _lib

    assert sorted(_lib.exported_symbols()) == declared


def test_library_built_for_sm103a(pkg):
    from paper_2002_04807_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_fpm_defaults_match_guide_table(pkg):
    f = pkg.feast_init()
    ref = O.feastinit()
    assert np.array_equal(f, ref)
    assert f[1] == 8 and f[2] == 12 and f[3] == 20 and f[17] == 30 and f[41] == 1 and f[45] == 40


@pytest.mark.parametrize("ne,ratio", [(1, 100), (8, 30), (8, 100), (16, 100), (56, 30)])
def test_contour_nodes_match_oracle(pkg, ne, ratio):
    z, w = pkg.feast_contour_nodes(ne, -1.5, 2.5, ratio)
    zo, wo = O.contour_gauss(ne, -1.5, 2.5, ratio / 100.0)
    assert np.abs(z - zo).max() < 1e-14 and np.abs(w - wo).max() < 1e-14


@pytest.mark.parametrize("ne,ratio", [(1, 100), (3, 30), (8, 100), (37, 200), (1024, 50)])
def test_trapezoid_nodes_match_oracle(pkg, ne, ratio):
    z, w = pkg.feast_contour_nodes_rule(1, ne, -1.5, 2.5, ratio)
    zo, wo = O.contour_trapezoid(ne, -1.5, 2.5, ratio / 100.0)
    assert np.abs(z - zo).max() < 1e-14 and np.abs(w - wo).max() < 1e-14
    zg, wg = pkg.feast_contour_nodes_rule(0, 8, -1.5, 2.5, ratio)
    zg0, wg0 = pkg.feast_contour_nodes(8, -1.5, 2.5, ratio)
    assert np.abs(zg - zg0).max() < 1e-15 and np.abs(wg - wg0).max() < 1e-15


@pytest.mark.parametrize("ne", [1, 2, 8, 16, 56])
def test_zolotarev_nodes_match_oracle(pkg, ne):
    """fpm(16)=2: the library's Zolotarev nodes and weights against the
    oracle's, written separately from the same construction."""
    z, w = pkg.feast_contour_nodes_rule(2, ne, -1.5, 2.5, 100)
    zo, wo = O.contour_zolotarev(ne, -1.5, 2.5)
    assert np.abs(z - zo).max() < 1e-13 and np.abs(w - wo).max() < 1e-13 * np.abs(wo).max()


def test_rule_and_node_count_checks(pkg):
    from paper_2002_04807_gb300 import FeastError

    with pytest.raises(FeastError):
        pkg.feast_contour_nodes_rule(3, 8, 0.0, 1.0, 30)
    with pytest.raises(FeastError):
        pkg.feast_contour_nodes_rule(1, 1025, 0.0, 1.0, 30)
    with pytest.raises(FeastError):
        pkg.feast_contour_nodes_rule(2, 21, 0.0, 1.0, 30)  # Zolotarev takes the Gauss node counts
    A = fw.laplacian_1d(20)
    base = dict(uplo="F", n=20, a=A.data, ia=A.indptr, ja=A.indices, emin=0.0, emax=0.5, m0=6)
    f = pkg.feast_init()
    f[15], f[1] = 3, 8
    assert pkg.feast_scsr_solve(**base, fpm=f).info == 116
    f[15], f[1] = 1, 0
    assert pkg.feast_scsr_solve(**base, fpm=f).info == 102
    f[15], f[1] = 0, 21  # 21 nodes: allowed for the trapezoidal rule only
    assert pkg.feast_scsr_solve(**base, fpm=f).info == 102


def test_contour_node_errors(pkg):
    from paper_2002_04807_gb300 import FeastError

    with pytest.raises(FeastError):
        pkg.feast_contour_nodes(21, 0.0, 1.0, 30)
    with pytest.raises(FeastError):
        pkg.feast_contour_nodes(8, 1.0, 0.0, 30)


@pytest.mark.parametrize("nb,fp64,expect", [(8, 0, (32, 8, 4)), (16, 0, (32, 16, 2)), (8, 1, (16, 8, 2)),
                                            (16, 1, (16, 16, 1)), (5, 0, (32, 8, 4)), (20, 1, (32, 32, 1)),
                                            (1, 0, (32, 1, 32))])
def test_filter_layout(pkg, nb, fp64, expect):
    assert pkg.feast_filter_layout(nb, fp64) == expect


def test_argument_errors_are_host_side(pkg):
    A = fw.laplacian_1d(20)
    ok = dict(uplo="F", n=20, a=A.data, ia=A.indptr, ja=A.indices, emin=0.0, emax=0.5, m0=6)

    def run(**kw):
        args = dict(ok)
        args.update(kw)
        return pkg.feast_scsr_solve(**args).info

    assert run(uplo="X") == -101
    assert run(n=0) == 202
    assert run(emin=1.0, emax=0.5) == 200
    assert run(m0=0) == 201 and run(m0=21) == 201
    f = pkg.feast_init()
    f[1] = 21
    assert run(fpm=f) == 102
    f = pkg.feast_init()
    f[15] = 3
    assert run(fpm=f) == 116
    bad = A.indices.copy()
    bad[3] = 99
    assert run(ja=bad) == -105
    nan = A.data.copy()
    nan[0] = np.nan
    assert run(a=nan) == -103
    bad_ia = A.indptr.copy()
    bad_ia[5] = bad_ia[4] - 1
    assert run(ia=bad_ia) == -104
    # lower storage with an upper entry
    assert run(uplo="L") == -105


def test_one_pass_and_extreme_mode_argument_checks(pkg):
    """fpm(14) and fpm(40) validation of the solve and extreme-mode entry
    points (guide parameter table: fpm(14) in {0,1,2}, fpm(40) in {-1,0,1})."""
    A = fw.laplacian_1d(20)
    base = dict(uplo="F", n=20, a=A.data, ia=A.indptr, ja=A.indices)
    f = pkg.feast_init()
    f[13] = 3
    assert pkg.feast_scsr_solve(**base, fpm=f, emin=0.0, emax=0.5, m0=6).info == 114
    f = pkg.feast_init()
    f[39] = -1  # the interval-search mode has its own entry point
    assert pkg.feast_scsr_solve(**base, fpm=f, emin=0.0, emax=0.5, m0=6).info == 140
    f[39] = 2
    assert pkg.feast_scsr_extreme(**base, fpm=f, m0=6).info == 140
    f[39] = 0
    assert pkg.feast_scsr_extreme(**base, fpm=f, m0=6).info == 140
    f[39] = 1
    assert pkg.feast_scsr_extreme(**base, fpm=f, m0=1).info == 201
    f[13] = 2
    assert pkg.feast_scsr_extreme(**base, fpm=f, m0=6).info == 114
    lib = pkg.library()
    fz = pkg.feast_init()
    fz[39] = -1
    # NULL interval pointers
    import ctypes as C

    E, X, R = np.zeros(6), np.zeros((20, 6)), np.zeros(6)
    M, L, I, m0 = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(6)
    eps = C.c_double(0)
    ia, ja, a = (np.ascontiguousarray(A.indptr, np.int32), np.ascontiguousarray(A.indices, np.int32),
                 np.ascontiguousarray(A.data))
    p = lambda v: v.ctypes.data_as(C.c_void_p)
    r = lib.feast_scsr_extreme(b"F", 20, p(a), p(ia), p(ja), None, None, None, p(fz), None, None, C.byref(m0),
                               p(E), p(X), C.byref(M), p(R), C.byref(eps), C.byref(L), C.byref(I))
    assert r == -110
    lo = C.c_double(0)
    r = lib.feast_scsr_extreme(b"F", 20, p(a), p(ia), p(ja), None, None, None, p(fz), C.byref(lo), None,
                               C.byref(m0), p(E), p(X), C.byref(M), p(R), C.byref(eps), C.byref(L), C.byref(I))
    assert r == -111


def test_extreme_workspace_includes_search_buffers(pkg):
    f = pkg.feast_init()
    base = pkg.feast_scsr_workspace_bytes(4096, 20000, 0, 40, f)
    f[39] = 1
    ext = pkg.feast_scsr_workspace_bytes(4096, 20000, 0, 40, f)
    assert ext >= base + 20000 * 8 + 4096 * 8


def test_custom_node_checks(pkg):
    """Expert entry point: every node strictly in the upper half plane."""
    A = fw.laplacian_1d(20)
    base = dict(uplo="F", n=20, a=A.data, ia=A.indptr, ja=A.indices, emin=0.0, emax=0.5, m0=6)
    z, w = pkg.feast_contour_nodes(8, 0.0, 0.5, 100)
    zb = z.copy()
    zb[3] = zb[3].real - 0.1j
    assert pkg.feast_scsr_solve_x(**base, zne=zb, wne=w).info == -120
    zb[3] = zb[3].real + np.nan * 1j
    assert pkg.feast_scsr_solve_x(**base, zne=zb, wne=w).info == -120


def test_no_cpu_fallback_without_gpu(pkg):
    """With valid arguments the host driver goes to the GPU; without one it
    must fail with the CUDA error code, never compute on the CPU."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    A = fw.laplacian_1d(20)
    r = None
    from paper_2002_04807_gb300 import FeastError

    with pytest.raises(FeastError):
        r = pkg.feast_scsr_solve("F", 20, A.data, A.indptr, A.indices, emin=0.0, emax=0.5, m0=6)
    assert r is None


def test_workspace_size_grows_with_problem(pkg):
    f = pkg.feast_init()
    small = pkg.feast_scsr_workspace_bytes(1000, 3000, 0, 48, f)
    big = pkg.feast_scsr_workspace_bytes(262144, 1810432, 0, 150, f)
    assert 0 < small < big
    f64 = f.copy()
    f64[41] = 0
    assert pkg.feast_scsr_workspace_bytes(262144, 1810432, 0, 150, f64) > big


def test_host_block_argument_checks(pkg):
    """x_out must be a Fortran-ordered float64 (n, m0) array; x0 must have
    shape (n, m0).  Checked before the library is called."""
    from paper_2002_04807_gb300 import FeastError

    A = fw.laplacian_1d(20)
    base = dict(uplo="F", n=20, a=A.data, ia=A.indptr, ja=A.indices, emin=0.0, emax=0.5, m0=6)
    with pytest.raises(FeastError):
        pkg.feast_scsr_solve(**base, x_out=np.zeros((20, 6)))  # C order
    with pytest.raises(FeastError):
        pkg.feast_scsr_solve(**base, x_out=np.zeros((20, 5), order="F"))
    with pytest.raises(FeastError):
        pkg.feast_scsr_solve(**base, x_out=np.zeros((20, 6), dtype=np.float32, order="F"))
    with pytest.raises(FeastError):
        pkg.feast_scsr_solve(**base, x0=np.zeros((19, 6)))


def test_hermitian_argument_errors_are_host_side(pkg):
    """feast_hcsr_solve validates its arguments before any device work (guide
    info table; fpm(14), fpm(40) and m0 > 1024 are outside the Hermitian driver)."""
    A = fw.flux_ring(20, 0.1)
    ok = dict(uplo="F", n=20, a=A.data, ia=A.indptr, ja=A.indices, emin=0.0, emax=0.5, m0=6)

    def run(**kw):
        args = dict(ok)
        args.update(kw)
        return pkg.feast_hcsr_solve(**args).info

    assert run(uplo="X") == -101
    assert run(n=0) == 202
    assert run(emin=1.0, emax=0.5) == 200
    assert run(m0=0) == 201 and run(m0=21) == 201
    for slot, val, code in ((1, 21, 102), (15, 3, 116), (13, 1, 114), (39, 1, 140), (49, 33, 150)):
        f = pkg.feast_init()
        f[slot] = val
        assert run(fpm=f) == code
    bad = A.indices.copy()
    bad[3] = 99
    assert run(ja=bad) == -105
    nan = A.data.copy()
    nan[0] = complex(np.nan, 0.0)
    assert run(a=nan) == -103
    bad_ia = A.indptr.copy()
    bad_ia[5] = bad_ia[4] - 1
    assert run(ia=bad_ia) == -104
    assert run(uplo="L") == -105  # lower storage with an upper entry
    big = fw.flux_ring(1100, 0.1)
    assert pkg.feast_hcsr_solve("F", 1100, big.data, big.indptr, big.indices, emin=0.0, emax=0.5,
                                m0=1025).info == 201


def test_hermitian_input_must_be_hermitian(pkg):
    """The Hermitian driver's shadow system needs A = A^H: a complex diagonal
    entry (any storage) or a full-storage pair with a_ji != conj(a_ij) (or a
    missing mirror) is rejected with the values argument's code -103 (-106 for
    B) before any device work; a conjugated pair within rounding passes the
    check (and then fails only for want of a GPU here)."""
    A = fw.flux_ring(20, 0.3)
    ok = dict(n=20, ia=A.indptr, ja=A.indices, emin=0.0, emax=0.5, m0=6)
    rows = np.repeat(np.arange(20), np.diff(A.indptr))

    def code(uplo, a, **kw):
        args = dict(ok)
        args.update(kw)
        return pkg.feast_hcsr_solve(uplo, a=a, **args).info

    diag = np.nonzero(rows == A.indices)[0][0]
    off = np.nonzero(rows < A.indices)[0][0]
    d = A.data.copy()
    d[diag] += 1e-3j
    assert code("F", d) == -103
    L = fw.zcsr_from_dense(np.tril(A.to_dense()))
    dl = L.data.copy()
    dl[np.nonzero(np.repeat(np.arange(20), np.diff(L.indptr)) == L.indices)[0][0]] += 1e-3j
    assert code("L", dl, ia=L.indptr, ja=L.indices) == -103
    f = A.data.copy()
    f[off] = np.conj(f[off])  # a_ij no longer the conjugate of a_ji
    assert code("F", f) == -103
    g = A.data.copy()
    g[off] *= 1 + 1e-9
    assert code("F", g) == -103
    h = A.data.copy()
    h[off] *= 1 + 1e-15  # within rounding: accepted by the check
    import torch

    if not torch.cuda.is_available():
        from paper_2002_04807_gb300 import FeastError

        with pytest.raises(FeastError):
            code("F", h)
    B = fw.zcsr_from_dense(np.diag(np.full(20, 1.0 + 1e-3j)))
    assert code("F", A.data, b=B.data, ib=B.indptr, jb=B.indices) == -106


def test_hermitian_no_cpu_fallback_without_gpu(pkg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    A = fw.flux_ring(20, 0.1)
    from paper_2002_04807_gb300 import FeastError

    with pytest.raises(FeastError):
        pkg.feast_hcsr_solve("F", 20, A.data, A.indptr, A.indices, emin=0.0, emax=0.5, m0=6)


def test_grad_argument_errors_are_host_side(pkg):
    """feast_scsr_grad validates its host arguments before any device work."""
    from paper_2002_04807_gb300 import FeastError

    A = fw.laplacian_1d(20)
    x, g = np.zeros((20, 3)), np.ones(3)

    def code(**kw):
        args = dict(uplo="F", n=20, ia=A.indptr, ja=A.indices, x=x, g=g)
        args.update(kw)
        try:
            pkg.feast_scsr_grad(**args)
        except FeastError as err:
            return int(str(err).split("returned")[1].split()[0])
        return 0

    assert code(uplo="X") == -101
    assert code(n=0) == 202
    bad = A.indices.copy()
    bad[3] = 99
    assert code(ja=bad) == -104
    assert code(uplo="L") == -104  # upper entries in lower storage
    bad_ia = A.indptr.copy()
    bad_ia[5] = bad_ia[4] - 1
    assert code(ia=bad_ia) == -103
    assert code(ib=A.indptr, jb=A.indices) == -109  # B pattern without eigenvalues
    assert code(x=np.zeros((20, 2049)), g=np.ones(2049)) == -107
    B = fw.laplacian_1d(20)
    badb = B.indices.copy()
    badb[0] = -5
    assert code(ib=B.indptr, jb=badb, e=np.ones(3)) == -106


def test_grad_no_cpu_fallback_without_gpu(pkg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2002_04807_gb300 import FeastError

    A = fw.laplacian_1d(20)
    with pytest.raises(FeastError, match="-4"):
        pkg.feast_scsr_grad("F", 20, A.indptr, A.indices, np.zeros((20, 3)), np.ones(3))
