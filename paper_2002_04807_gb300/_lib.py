"""ctypes marshalling for libfeast_gb300.so.  Names match the C ABI."""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libfeast_gb300.so")
_lock = threading.Lock()
_lib = None

_i = C.c_int
_d = C.c_double
_p = C.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "feast_init": (_i, [_p]),
    "feast_last_error": (C.c_char_p, []),
    "feast_contour_nodes": (_i, [_i, _d, _d, _i, _p, _p]),
    "feast_contour_nodes_rule": (_i, [_i, _i, _d, _d, _i, _p, _p]),
    "feast_scsr_solve": (_i, [C.c_char, _i, _p, _p, _p, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p, _p,
                              _p]),
    "feast_scsr_workspace_bytes": (C.c_size_t, [_i, _i, _i, _i, _p]),
    "feast_scsr_solve_dev": (_i, [_i, _i, _p, _p, _p, _i, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p, _p,
                                  _p, _p, C.c_size_t, _p]),
    "feast_filter_layout": (_i, [_i, _i, _p, _p, _p]),
    "feast_shifted_spmm_dev": (_i, [_i, _i, _p, _p, _p, _i, _p, _p, _p, _i, _p, _i, _i, _p, _p, _p]),
    "feast_filter_dev": (_i, [_i, _i, _p, _p, _p, _i, _p, _p, _p, _i, _p, _p, _p, _i, _p, _d, _d, _p, _p, _p]),
    "feast_gram_dev": (_i, [_i, _i, _p, _p, _p, _p]),
    "feast_gemm_dev": (_i, [_i, _i, _i, _p, _p, _p, _p]),
    "feast_sym_eig_dev": (_i, [_i, _p, _p, _p, _p, _p]),
    "feast_reduced_eig_dev": (_i, [_i, _p, _p, _p, _p, _p, _p]),
    "feast_residual_dev": (_i, [_i, _p, _p, _p, _p, _p, _p, _i, _p, _p, _d, _p, _p, _p]),
    "feast_eig_grad_dev": (_i, [_i, _p, _p, _i, _p, _p, _p, _p]),
    "feast_scsr_grad": (_i, [C.c_char, _i, _p, _p, _p, _p, _i, _p, _p, _p, _p, _p]),
    "feast_set_wait_limit": (C.c_longlong, [C.c_longlong]),
    "feast_last_profile": (_i, [_p]),
    "feast_gram_noalloc_dev": (_i, [_i, _i, _p, _p, _p, _p]),
    "feast_gram_oz_dev": (_i, [_i, _i, _p, _p, _p, _p]),
    "feast_gemm_oz_dev": (_i, [_i, _i, _i, _p, _p, _p, _p]),
    "feast_scsr_solve_batched": (_i, [_i, _p, _p, _p]),
    "feast_scsr_solve_x": (_i, [C.c_char, _i, _p, _p, _p, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p, _p,
                                _p, _p, _p]),
    "feast_scsr_solve_dev_x": (_i, [_i, _i, _p, _p, _p, _i, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p, _p,
                                    _p, _p, C.c_size_t, _p, _p, _p]),
    "feast_scsr_extreme": (_i, [C.c_char, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p,
                                _p]),
    "feast_scsr_extreme_dev": (_i, [_i, _i, _p, _p, _p, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p,
                                    _p, _p, _p, C.c_size_t, _p]),
    "feast_hcsr_solve": (_i, [C.c_char, _i, _p, _p, _p, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p, _p,
                              _p]),
    "feast_hcsr_solve_dev": (_i, [_i, _i, _p, _p, _p, _i, _p, _p, _p, _p, _d, _d, _p, _p, _p, _p, _p, _p, _p,
                                  _p, _p, C.c_size_t, _p]),
    "feast_hcsr_workspace_bytes": (C.c_size_t, [_i, _i, _i, _i, _p]),
}


class _Problem(C.Structure):
    _fields_ = [("n", _i), ("a", _p), ("ia", _p), ("ja", _p), ("b", _p), ("ib", _p), ("jb", _p),
                ("emin", _d), ("emax", _d), ("m0", _i), ("x0", _p)]


class _Result(C.Structure):
    _fields_ = [("info", _i), ("m", _i), ("loop", _i), ("m0", _i), ("epsout", _d), ("e", _p), ("x", _p),
                ("res", _p)]


class FeastError(RuntimeError):
    pass


def library_path() -> str:
    return _LIBPATH


def library():
    """Load libfeast_gb300.so (built by paper_2002_04807_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIBPATH):
                raise FeastError(f"{_LIBPATH} is missing: build it with "
                                 "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(_LIBPATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def feast_last_error() -> str:
    return library().feast_last_error().decode()


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())  # torch tensor


def _stream(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _check(code: int, what: str):
    if code != 0:
        msg = feast_last_error() if code == -4 else ""
        raise FeastError(f"{what} returned {code} {msg}".strip())


def _dev(t, dtype):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise FeastError(f"expected a contiguous CUDA tensor of {dtype}")
    return t


# ---------------------------------------------------------------- host-side helpers
PROFILE_KEYS = ["cocg_a_ms", "cocg_b_ms", "cocg_a_launches", "cocg_b_launches", "group_iterations",
                "filter_ms", "project_ms", "reduce_ms", "ritz_ms", "W", "mt", "n", "complex_bytes", "groups",
                "loops", "launches", "step_a_rows_per_item", "step_a_staged", "step_a_grid",
                "step_a_staged_rows"]


def feast_last_profile() -> dict:
    out = np.zeros(20)
    library().feast_last_profile(_ptr(out))
    return dict(zip(PROFILE_KEYS, out.tolist()))


def feast_init() -> np.ndarray:
    fpm = np.zeros(64, dtype=np.int32)
    library().feast_init(_ptr(fpm))
    return fpm


def feast_contour_nodes(ne: int, emin: float, emax: float, ratio_pct: int):
    z = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    _check(library().feast_contour_nodes(ne, emin, emax, ratio_pct, _ptr(z), _ptr(w)), "feast_contour_nodes")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def feast_contour_nodes_rule(rule: int, ne: int, emin: float, emax: float, ratio_pct: int):
    """Nodes of quadrature rule fpm(16) = rule (0 Gauss-Legendre, 1 trapezoidal)."""
    z = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    _check(library().feast_contour_nodes_rule(rule, ne, emin, emax, ratio_pct, _ptr(z), _ptr(w)),
           "feast_contour_nodes_rule")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def feast_filter_layout(nb: int, fp64: bool):
    W, nbp, mt = _i(), _i(), _i()
    _check(library().feast_filter_layout(nb, int(fp64), C.byref(W), C.byref(nbp), C.byref(mt)),
           "feast_filter_layout")
    return W.value, nbp.value, mt.value


@dataclass
class FeastResult:
    info: int
    E: np.ndarray
    X: np.ndarray  # (n, m0') column-major
    res: np.ndarray
    M: int
    loop: int
    epsout: float
    m0: int
    fpm: np.ndarray
    emin: float = float("nan")  # interval found by the extreme-eigenvalue search
    emax: float = float("nan")


def _fpm(fpm):
    f = feast_init() if fpm is None else np.array(fpm, dtype=np.int32, copy=True)
    if f.shape != (64,):
        raise FeastError("fpm must have 64 entries")
    return np.ascontiguousarray(f)


def _host_block(n, m0, x0, x_out, f):
    """The host X block (column-major n x m0) handed to the library: x_out in
    place when given (filled from x0 if that is another array), else a new
    array holding x0, else zeros when the library reads or may not write it."""
    if x_out is not None:
        if x_out.shape != (n, m0) or x_out.dtype != np.float64 or not x_out.flags.f_contiguous:
            raise FeastError("x_out must be a Fortran-ordered float64 array of shape (n, m0)")
        if x0 is not None and x0 is not x_out:
            np.copyto(x_out, x0)
        return x_out
    if x0 is not None:
        x = np.array(x0, dtype=np.float64, order="F", copy=True)
        if x.shape != (n, m0):
            raise FeastError("x0 must have shape (n, m0)")
        return x
    if f[4] == 1 or f[13] != 0:
        return np.zeros((n, m0), order="F")
    return np.empty((n, m0), order="F")


def feast_scsr_solve(uplo: str, n: int, a, ia, ja, b=None, ib=None, jb=None, fpm=None, emin=0.0, emax=1.0,
                     m0: int = 1, x0=None, x_out=None) -> FeastResult:
    """Host driver: CSR arrays (numpy, base ia[0] in {0,1}), returns a FeastResult.
    x0 (n x m0) is the start subspace when fpm(5)=1.  x_out: optional
    Fortran-ordered float64 (n, m0) array used in place as the library's X
    (pinned host memory makes the copies faster); it receives the eigenvectors."""
    f = _fpm(fpm)
    a = np.ascontiguousarray(a, dtype=np.float64)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ja = np.ascontiguousarray(ja, dtype=np.int32)
    if b is not None:
        b = np.ascontiguousarray(b, dtype=np.float64)
        ib = np.ascontiguousarray(ib, dtype=np.int32)
        jb = np.ascontiguousarray(jb, dtype=np.int32)
    x = _host_block(n, m0, x0, x_out, f)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps = _d(0)
    library().feast_scsr_solve(uplo.encode(), n, _ptr(a), _ptr(ia), _ptr(ja), _ptr(b), _ptr(ib), _ptr(jb),
                               _ptr(f), emin, emax, C.byref(mm), _ptr(E), _ptr(x), C.byref(M), _ptr(res),
                               C.byref(eps), C.byref(loop), C.byref(info))
    k = mm.value
    if info.value == -4:
        raise FeastError("feast_scsr_solve: " + feast_last_error())
    return FeastResult(info.value, E[:k].copy(), np.asfortranarray(x[:, :k]), res[:k].copy(), M.value,
                       loop.value, eps.value, k, f)


def feast_scsr_workspace_bytes(n: int, nnz_a: int, nnz_b: int, m0: int, fpm) -> int:
    f = _fpm(fpm)
    return int(library().feast_scsr_workspace_bytes(n, nnz_a, nnz_b, m0, _ptr(f)))


def feast_scsr_solve_dev(n: int, ia, ja, a, ib=None, jb=None, b=None, fpm=None, emin=0.0, emax=1.0,
                         m0: int = 1, x=None, work=None, stream=None) -> FeastResult:
    """Device driver: 0-based CSR as torch CUDA tensors (int32 / float64), x a
    CUDA float64 tensor holding the column-major n x m0 block (in/out; shape
    (m0, n) row-major is the same memory).  work: optional preallocated uint8
    CUDA tensor."""
    import torch

    f = _fpm(fpm)
    ia, ja, a = _dev(ia, torch.int32), _dev(ja, torch.int32), _dev(a, torch.float64)
    nnzb = 0
    if b is not None:
        ib, jb, b = _dev(ib, torch.int32), _dev(jb, torch.int32), _dev(b, torch.float64)
        nnzb = b.numel()
    if x is None:
        x = torch.zeros((m0, n), dtype=torch.float64, device=a.device)
    x = _dev(x, torch.float64)
    need = feast_scsr_workspace_bytes(n, a.numel(), nnzb, m0, f)
    if work is None or work.numel() < need:
        work = torch.empty(need, dtype=torch.uint8, device=a.device)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps = _d(0)
    library().feast_scsr_solve_dev(n, a.numel(), _ptr(ia), _ptr(ja), _ptr(a), nnzb, _ptr(ib), _ptr(jb), _ptr(b),
                                   _ptr(f), emin, emax, C.byref(mm), _ptr(E), _ptr(x), C.byref(M), _ptr(res),
                                   C.byref(eps), C.byref(loop), C.byref(info), _ptr(work), work.numel(),
                                   _stream(stream))
    if info.value == -4:
        raise FeastError("feast_scsr_solve_dev: " + feast_last_error())
    k = mm.value
    return FeastResult(info.value, E[:k].copy(), x, res[:k].copy(), M.value, loop.value, eps.value, k, f)


def _nodes(zne, wne):
    zne = np.asarray(zne, dtype=np.complex128)
    wne = np.asarray(wne, dtype=np.complex128)
    z = np.ascontiguousarray(np.stack([zne.real, zne.imag], axis=1).ravel())
    w = np.ascontiguousarray(np.stack([wne.real, wne.imag], axis=1).ravel())
    return z, w


def feast_scsr_solve_x(uplo: str, n: int, a, ia, ja, zne, wne, b=None, ib=None, jb=None, fpm=None, emin=0.0,
                       emax=1.0, m0: int = 1, x0=None, x_out=None) -> FeastResult:
    """Host driver with custom half-contour nodes zne and weights wne (complex
    arrays of fpm(2) values, convention of feast_contour_nodes)."""
    f = _fpm(fpm)
    a = np.ascontiguousarray(a, dtype=np.float64)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ja = np.ascontiguousarray(ja, dtype=np.int32)
    if b is not None:
        b = np.ascontiguousarray(b, dtype=np.float64)
        ib = np.ascontiguousarray(ib, dtype=np.int32)
        jb = np.ascontiguousarray(jb, dtype=np.int32)
    z, w = _nodes(zne, wne)
    x = _host_block(n, m0, x0, x_out, f)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps = _d(0)
    library().feast_scsr_solve_x(uplo.encode(), n, _ptr(a), _ptr(ia), _ptr(ja), _ptr(b), _ptr(ib), _ptr(jb),
                                 _ptr(f), emin, emax, C.byref(mm), _ptr(E), _ptr(x), C.byref(M), _ptr(res),
                                 C.byref(eps), C.byref(loop), C.byref(info), _ptr(z), _ptr(w))
    k = mm.value
    if info.value == -4:
        raise FeastError("feast_scsr_solve_x: " + feast_last_error())
    return FeastResult(info.value, E[:k].copy(), np.asfortranarray(x[:, :k]), res[:k].copy(), M.value,
                       loop.value, eps.value, k, f)


def feast_scsr_solve_dev_x(n: int, ia, ja, a, zne, wne, ib=None, jb=None, b=None, fpm=None, emin=0.0, emax=1.0,
                           m0: int = 1, x=None, work=None, stream=None) -> FeastResult:
    """Device driver with custom half-contour nodes (see feast_scsr_solve_x)."""
    import torch

    f = _fpm(fpm)
    ia, ja, a = _dev(ia, torch.int32), _dev(ja, torch.int32), _dev(a, torch.float64)
    nnzb = 0
    if b is not None:
        ib, jb, b = _dev(ib, torch.int32), _dev(jb, torch.int32), _dev(b, torch.float64)
        nnzb = b.numel()
    if x is None:
        x = torch.zeros((m0, n), dtype=torch.float64, device=a.device)
    x = _dev(x, torch.float64)
    need = feast_scsr_workspace_bytes(n, a.numel(), nnzb, m0, f)
    if work is None or work.numel() < need:
        work = torch.empty(need, dtype=torch.uint8, device=a.device)
    z, w = _nodes(zne, wne)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps = _d(0)
    library().feast_scsr_solve_dev_x(n, a.numel(), _ptr(ia), _ptr(ja), _ptr(a), nnzb, _ptr(ib), _ptr(jb), _ptr(b),
                                     _ptr(f), emin, emax, C.byref(mm), _ptr(E), _ptr(x), C.byref(M), _ptr(res),
                                     C.byref(eps), C.byref(loop), C.byref(info), _ptr(work), work.numel(),
                                     _stream(stream), _ptr(z), _ptr(w))
    if info.value == -4:
        raise FeastError("feast_scsr_solve_dev_x: " + feast_last_error())
    k = mm.value
    return FeastResult(info.value, E[:k].copy(), x, res[:k].copy(), M.value, loop.value, eps.value, k, f)


def feast_scsr_extreme(uplo: str, n: int, a, ia, ja, b=None, ib=None, jb=None, fpm=None, m0: int = 2,
                       x0=None, x_out=None) -> FeastResult:
    """Host driver of the extreme-eigenvalue mode: fpm(40) = -1 (lowest) or +1
    (largest) selects the m0/2 wanted pairs; the returned FeastResult carries
    the interval found in emin/emax."""
    f = _fpm(fpm)
    a = np.ascontiguousarray(a, dtype=np.float64)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ja = np.ascontiguousarray(ja, dtype=np.int32)
    if b is not None:
        b = np.ascontiguousarray(b, dtype=np.float64)
        ib = np.ascontiguousarray(ib, dtype=np.int32)
        jb = np.ascontiguousarray(jb, dtype=np.int32)
    x = _host_block(n, m0, x0, x_out, f)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps, lo, hi = _d(0), _d(0), _d(0)
    library().feast_scsr_extreme(uplo.encode(), n, _ptr(a), _ptr(ia), _ptr(ja), _ptr(b), _ptr(ib), _ptr(jb),
                                 _ptr(f), C.byref(lo), C.byref(hi), C.byref(mm), _ptr(E), _ptr(x), C.byref(M),
                                 _ptr(res), C.byref(eps), C.byref(loop), C.byref(info))
    k = mm.value
    if info.value == -4:
        raise FeastError("feast_scsr_extreme: " + feast_last_error())
    return FeastResult(info.value, E[:k].copy(), np.asfortranarray(x[:, :k]), res[:k].copy(), M.value,
                       loop.value, eps.value, k, f, lo.value, hi.value)


def feast_scsr_extreme_dev(n: int, ia, ja, a, ib=None, jb=None, b=None, fpm=None, m0: int = 2, x=None,
                           work=None, stream=None) -> FeastResult:
    """Device driver of the extreme-eigenvalue mode (tensors as for
    feast_scsr_solve_dev); the interval found is in emin/emax."""
    import torch

    f = _fpm(fpm)
    ia, ja, a = _dev(ia, torch.int32), _dev(ja, torch.int32), _dev(a, torch.float64)
    nnzb = 0
    if b is not None:
        ib, jb, b = _dev(ib, torch.int32), _dev(jb, torch.int32), _dev(b, torch.float64)
        nnzb = b.numel()
    if x is None:
        x = torch.zeros((m0, n), dtype=torch.float64, device=a.device)
    x = _dev(x, torch.float64)
    need = feast_scsr_workspace_bytes(n, a.numel(), nnzb, m0, f)
    if work is None or work.numel() < need:
        work = torch.empty(need, dtype=torch.uint8, device=a.device)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps, lo, hi = _d(0), _d(0), _d(0)
    library().feast_scsr_extreme_dev(n, a.numel(), _ptr(ia), _ptr(ja), _ptr(a), nnzb, _ptr(ib), _ptr(jb),
                                     _ptr(b), _ptr(f), C.byref(lo), C.byref(hi), C.byref(mm), _ptr(E), _ptr(x),
                                     C.byref(M), _ptr(res), C.byref(eps), C.byref(loop), C.byref(info),
                                     _ptr(work), work.numel(), _stream(stream))
    if info.value == -4:
        raise FeastError("feast_scsr_extreme_dev: " + feast_last_error())
    k = mm.value
    return FeastResult(info.value, E[:k].copy(), x, res[:k].copy(), M.value, loop.value, eps.value, k, f,
                       lo.value, hi.value)


def feast_scsr_solve_batched(problems, fpm=None):
    """Solve many independent problems together.

    problems: list of dicts with keys n, a, ia, ja (CSR, numpy), optional b, ib,
    jb, emin, emax, m0 and optional x0 (n x m0).  Returns (status, [FeastResult])."""
    f = _fpm(fpm)
    keep = []
    P = (_Problem * len(problems))()
    R = (_Result * len(problems))()
    outs = []
    for k, q in enumerate(problems):
        n, m0 = int(q["n"]), int(q["m0"])
        arrs = [np.ascontiguousarray(q["a"], dtype=np.float64), np.ascontiguousarray(q["ia"], dtype=np.int32),
                np.ascontiguousarray(q["ja"], dtype=np.int32)]
        if q.get("b") is not None:
            arrs += [np.ascontiguousarray(q["b"], dtype=np.float64), np.ascontiguousarray(q["ib"], dtype=np.int32),
                     np.ascontiguousarray(q["jb"], dtype=np.int32)]
        else:
            arrs += [None, None, None]
        x0 = None if q.get("x0") is None else np.asfortranarray(q["x0"], dtype=np.float64)
        E, X, res = np.zeros(m0), np.zeros((n, m0), order="F"), np.zeros(m0)
        keep += arrs + [x0, E, X, res]
        P[k] = _Problem(n, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), _ptr(arrs[3]), _ptr(arrs[4]), _ptr(arrs[5]),
                        float(q["emin"]), float(q["emax"]), m0, _ptr(x0))
        R[k] = _Result(0, 0, 0, m0, 0.0, _ptr(E), _ptr(X), _ptr(res))
        outs.append((E, X, res))
    st = library().feast_scsr_solve_batched(len(problems), C.cast(P, C.c_void_p), _ptr(f), C.cast(R, C.c_void_p))
    if st == -4:
        raise FeastError("feast_scsr_solve_batched: " + feast_last_error())
    results = []
    for k, (E, X, res) in enumerate(outs):
        r = R[k]
        km = r.m0
        results.append(FeastResult(r.info, E[:km].copy(), np.asfortranarray(X[:, :km]), res[:km].copy(), r.m, r.loop,
                                    r.epsout, km, f))
    return st, results


# ---------------------------------------------------------------- kernel-level entry points
def feast_shifted_spmm_dev(n, ia, ja, a, ib, jb, b, z, m, fp64, P, V, stream=None):
    z = np.ascontiguousarray(np.column_stack([np.real(z), np.imag(z)]).ravel(), dtype=np.float64)
    nb = len(z) // 2
    _check(library().feast_shifted_spmm_dev(n, a.numel(), _ptr(ia), _ptr(ja), _ptr(a), 0 if b is None else b.numel(),
                                            _ptr(ib), _ptr(jb), _ptr(b), nb, _ptr(z), m, int(fp64), _ptr(P), _ptr(V),
                                            _stream(stream)), "feast_shifted_spmm_dev")


def feast_filter_dev(n, ia, ja, a, ib, jb, b, m, R, X, lam, rii, fpm, emin, emax, Q, stream=None) -> int:
    f = _fpm(fpm)
    it = _i(0)
    _check(library().feast_filter_dev(n, a.numel(), _ptr(ia), _ptr(ja), _ptr(a), 0 if b is None else b.numel(),
                                      _ptr(ib), _ptr(jb), _ptr(b), m, _ptr(R), _ptr(X), _ptr(lam), int(rii),
                                      _ptr(f), emin, emax, _ptr(Q), C.byref(it), _stream(stream)),
           "feast_filter_dev")
    return it.value


def feast_gram_dev(n, m, X, Y, Cm, stream=None):
    _check(library().feast_gram_dev(n, m, _ptr(X), _ptr(Y), _ptr(Cm), _stream(stream)), "feast_gram_dev")


def feast_gram_oz_dev(n, m, X, Y, Cm, stream=None):
    _check(library().feast_gram_oz_dev(n, m, _ptr(X), _ptr(Y), _ptr(Cm), _stream(stream)), "feast_gram_oz_dev")


def feast_gemm_oz_dev(n, m, k, A, V, Cm, stream=None):
    _check(library().feast_gemm_oz_dev(n, m, k, _ptr(A), _ptr(V), _ptr(Cm), _stream(stream)), "feast_gemm_oz_dev")


def feast_gram_noalloc_dev(n, m, X, Y, Cm, stream=None):
    """C = X^T Y like feast_gram_dev, with the library's fixed device scratch
    instead of any allocation (for callers that cannot allocate)."""
    _check(library().feast_gram_noalloc_dev(n, m, _ptr(X), _ptr(Y), _ptr(Cm), _stream(stream)),
           "feast_gram_noalloc_dev")


def feast_gemm_dev(n, m, k, A, V, Cm, stream=None):
    _check(library().feast_gemm_dev(n, m, k, _ptr(A), _ptr(V), _ptr(Cm), _stream(stream)), "feast_gemm_dev")


def feast_sym_eig_dev(m, A, lam, V, stream=None) -> int:
    sw = _i(0)
    _check(library().feast_sym_eig_dev(m, _ptr(A), _ptr(lam), _ptr(V), C.byref(sw), _stream(stream)),
           "feast_sym_eig_dev")
    return sw.value


def feast_reduced_eig_dev(m, Aq, Bq, lam, V, stream=None) -> int:
    mk = _i(0)
    _check(library().feast_reduced_eig_dev(m, _ptr(Aq), _ptr(Bq), _ptr(lam), _ptr(V), C.byref(mk),
                                           _stream(stream)), "feast_reduced_eig_dev")
    return mk.value


def feast_residual_dev(n, ia, ja, a, ib, jb, b, m, X, lam, alpha, R, res, stream=None):
    _check(library().feast_residual_dev(n, _ptr(ia), _ptr(ja), _ptr(a), _ptr(ib), _ptr(jb), _ptr(b), m, _ptr(X),
                                        _ptr(lam), alpha, _ptr(R), _ptr(res), _stream(stream)),
           "feast_residual_dev")


def feast_eig_grad_dev(n, ia, ja, m, X, w, grad, stream=None):
    _check(library().feast_eig_grad_dev(n, _ptr(ia), _ptr(ja), m, _ptr(X), _ptr(w), _ptr(grad), _stream(stream)),
           "feast_eig_grad_dev")


def feast_set_wait_limit(cycles: int) -> int:
    """Spin limit (SM clock cycles) of the library's bounded device waits;
    cycles < 1 restores the default.  Returns the previous limit."""
    return int(library().feast_set_wait_limit(int(cycles)))


def feast_scsr_grad(uplo: str, n: int, ia, ja, x, g, ib=None, jb=None, e=None):
    """Gradient of L = sum_k g_k lambda_k over the stored entries of A's (and
    B's) CSR pattern, host buffers: x is n x m (eigenvectors in columns,
    B-orthonormal), g [m] the loss weights, e [m] the eigenvalues (with B).
    Returns (grad_a, grad_b or None)."""
    ia_ = np.ascontiguousarray(ia, dtype=np.int32)
    ja_ = np.ascontiguousarray(ja, dtype=np.int32)
    x_ = np.asfortranarray(x, dtype=np.float64)
    m = x_.shape[1] if x_.ndim == 2 else 0
    g_ = np.ascontiguousarray(g, dtype=np.float64)
    hasB = ib is not None or jb is not None
    ib_ = None if ib is None else np.ascontiguousarray(ib, dtype=np.int32)
    jb_ = None if jb is None else np.ascontiguousarray(jb, dtype=np.int32)
    e_ = None if e is None else np.ascontiguousarray(e, dtype=np.float64)
    base = int(ia_[0]) if ia_.size else 0
    ga = np.zeros(max(1, int(ia_[-1]) - base))
    gb = np.zeros(max(1, int(ib_[-1]) - int(ib_[0]))) if hasB and ib_ is not None else None
    code = library().feast_scsr_grad(uplo.encode()[:1], n, _ptr(ia_), _ptr(ja_), _ptr(ib_), _ptr(jb_), m, _ptr(x_),
                                     _ptr(e_), _ptr(g_), _ptr(ga), _ptr(gb))
    _check(code, "feast_scsr_grad")
    nnz_a = int(ia_[-1]) - base
    return ga[:nnz_a], (None if gb is None else gb[: int(ib_[-1]) - int(ib_[0])])


def _cvals(v):
    """complex values -> contiguous interleaved (real, imaginary) float64"""
    v = np.ascontiguousarray(v, dtype=np.complex128)
    return v.view(np.float64)


def feast_hcsr_solve(uplo: str, n: int, a, ia, ja, b=None, ib=None, jb=None, fpm=None, emin=0.0, emax=1.0,
                     m0: int = 1, x0=None) -> FeastResult:
    """Host driver for complex Hermitian CSR problems: a (and b) complex
    values, CSR base ia[0] in {0,1}; x0 (n x m0 complex) is the start subspace
    when fpm(5)=1.  The result's X is complex n x k."""
    f = _fpm(fpm)
    av = _cvals(a)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ja = np.ascontiguousarray(ja, dtype=np.int32)
    bv = None
    if b is not None:
        bv = _cvals(b)
        ib = np.ascontiguousarray(ib, dtype=np.int32)
        jb = np.ascontiguousarray(jb, dtype=np.int32)
    x = np.zeros((n, m0), dtype=np.complex128, order="F")
    if x0 is not None:
        if np.shape(x0) != (n, m0):
            raise FeastError("x0 must have shape (n, m0)")
        x[:] = x0
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps = _d(0)
    library().feast_hcsr_solve(uplo.encode(), n, _ptr(av), _ptr(ia), _ptr(ja), _ptr(bv), _ptr(ib), _ptr(jb),
                               _ptr(f), emin, emax, C.byref(mm), _ptr(E), _ptr(x), C.byref(M), _ptr(res),
                               C.byref(eps), C.byref(loop), C.byref(info))
    k = mm.value
    if info.value == -4:
        raise FeastError("feast_hcsr_solve: " + feast_last_error())
    return FeastResult(info.value, E[:k].copy(), np.asfortranarray(x[:, :k]), res[:k].copy(), M.value,
                       loop.value, eps.value, k, f)


def feast_hcsr_workspace_bytes(n: int, nnz_a: int, nnz_b: int, m0: int, fpm) -> int:
    return int(library().feast_hcsr_workspace_bytes(n, nnz_a, nnz_b, m0, _ptr(_fpm(fpm))))


def feast_hcsr_solve_dev(n: int, ia, ja, a, ib=None, jb=None, b=None, fpm=None, emin=0.0, emax=1.0, m0: int = 1,
                         x=None, work=None, stream=None) -> FeastResult:
    """Device driver for complex Hermitian CSR problems: 0-based CSR as torch
    CUDA tensors (int32 indices, complex128 values); x a CUDA complex128
    tensor holding the column-major n x m0 block (shape (m0, n) row-major is
    the same memory), in/out.  work: optional CUDA uint8 tensor of at least
    feast_hcsr_workspace_bytes(...) bytes (else the library allocates)."""
    import torch

    f = _fpm(fpm)
    ia, ja, a = _dev(ia, torch.int32), _dev(ja, torch.int32), _dev(a, torch.complex128)
    nnzb = 0
    if b is not None:
        ib, jb, b = _dev(ib, torch.int32), _dev(jb, torch.int32), _dev(b, torch.complex128)
        nnzb = b.numel()
    if x is None:
        x = torch.zeros((m0, n), dtype=torch.complex128, device=a.device)
    x = _dev(x, torch.complex128)
    E = np.zeros(m0)
    res = np.zeros(m0)
    M, loop, info, mm = _i(0), _i(0), _i(0), _i(m0)
    eps = _d(0)
    library().feast_hcsr_solve_dev(n, a.numel(), _ptr(ia), _ptr(ja), _ptr(a), nnzb, _ptr(ib), _ptr(jb), _ptr(b),
                                   _ptr(f), emin, emax, C.byref(mm), _ptr(E), _ptr(x), C.byref(M), _ptr(res),
                                   C.byref(eps), C.byref(loop), C.byref(info), _ptr(work),
                                   0 if work is None else work.numel(), _stream(stream))
    if info.value == -4:
        raise FeastError("feast_hcsr_solve_dev: " + feast_last_error())
    k = mm.value
    return FeastResult(info.value, E[:k].copy(), x, res[:k].copy(), M.value, loop.value, eps.value, k, f)
