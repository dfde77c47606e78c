"""The FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow statement of SpAMM (Sec. 2, Eqs. 1-4; Algorithm 1 of Sec. 3.1)
and of the cited SP2 spectral projection (Sec. 4), used to check the CUDA
library.  Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU
baseline may import this package.  It shares no code with the CUDA path: the
arithmetic lives in `spamm_oracle.c`, compiled here with gcc, and this module
only marshals numpy arrays into it.

Every function here is pinned by `tests/test_oracle_*.py` against something
other than itself: exact rational arithmetic, brute-force enumeration,
closed forms, numpy's dense product and eigensolver, a worked example
derived by hand, and the counts the paper prints (`tests/golden/`).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spamm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

H_TR, H_TR2, H_IDEM, H_BRANCH, H_TASKS, H_TRNEW, H_COLS = range(7)
STOP_CONVERGED, STOP_STAGNATED, STOP_FIXED, STOP_MAXITER = range(4)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, no
    floating-point contraction, OpenMP if the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.ora_depth.argtypes = [i64]
    lib.ora_depth.restype = i32
    lib.ora_tier_offset.argtypes = [i32]
    lib.ora_tier_offset.restype = i64
    lib.ora_leaf_norms2.argtypes = [P, i64, i64, i32, P]
    lib.ora_leaf_norms2.restype = None
    lib.ora_norm_pyramid.argtypes = [P, i32, P]
    lib.ora_norm_pyramid.restype = None
    lib.ora_spamm.argtypes = [P, i64, P, i64, P, i64, i64, i32, dbl, P, i64,
                              ctypes.POINTER(i64), i32]
    lib.ora_spamm.restype = i32
    lib.ora_flat_tasks.argtypes = [P, P, i64, i64, dbl, P, i64]
    lib.ora_flat_tasks.restype = i64
    lib.ora_gemm.argtypes = [P, P, P, i64]
    lib.ora_gemm.restype = None
    lib.ora_gershgorin.argtypes = [P, i64, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.ora_gershgorin.restype = None
    lib.ora_sp2.argtypes = [P, i64, i32, dbl, dbl, i32, i32, dbl, dbl, i32, P, P,
                            ctypes.POINTER(i32), i32]
    lib.ora_sp2.restype = i32
    lib.ora_num_threads.argtypes = []
    lib.ora_num_threads.restype = i32
    _lib = lib
    return lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the oracle uses by default."""
    return int(_load().ora_num_threads())


def depth(nb: int) -> int:
    """Quadtree depth d, the smallest d with 2^d >= nb (virtual padding)."""
    return int(_load().ora_depth(nb))


def leaf_norms2(a: np.ndarray, leaf: int) -> np.ndarray:
    """Squared leaf Frobenius norms (Eq. 2), a 2^d x 2^d grid (padding 0)."""
    a = _c(a)
    n = a.shape[0]
    nb = -(-n // leaf)
    P = 1 << depth(nb)
    out = np.zeros((P, P))
    _load().ora_leaf_norms2(_ptr(a), n, a.shape[1], leaf, _ptr(out))
    return out


def norm_pyramid(a: np.ndarray, leaf: int) -> list[np.ndarray]:
    """Squared norms of tiers 0..d (Eq. 3), as a list of 2^t x 2^t grids."""
    ln = leaf_norms2(a, leaf)
    d = int(np.log2(ln.shape[0]))
    total = ((1 << (2 * (d + 1))) - 1) // 3
    tiers = np.zeros(total)
    _load().ora_norm_pyramid(_ptr(ln), d, _ptr(tiers))
    out = []
    for t in range(d + 1):
        off = ((1 << (2 * t)) - 1) // 3
        w = 1 << t
        out.append(tiers[off:off + w * w].reshape(w, w).copy())
    return out


def spamm(a: np.ndarray, b: np.ndarray, leaf: int, tau: float,
          want_tasks: bool = False, nthreads: int = 0):
    """C = SpAMM(A, B, tau) by the recursive walk of Algorithm 1.

    With want_tasks the walk runs on one thread and also returns the surviving
    (i, k, j) leaf triples in visit order as an (T, 3) int32 array."""
    a = _c(a)
    b = _c(b)
    n = a.shape[0]
    if a.shape != (n, n) or b.shape != (n, n):
        raise ValueError("square matrices of equal size expected")
    c = np.zeros((n, n))
    lib = _load()
    nt = ctypes.c_int64(0)
    if want_tasks:
        nb = -(-n // leaf)
        cap = max(nb ** 3, 1)
        tasks = np.zeros((cap, 3), dtype=np.int32)
        rc = lib.ora_spamm(_ptr(a), n, _ptr(b), n, _ptr(c), n, n, leaf, tau,
                           tasks.ctypes.data_as(ctypes.c_void_p), cap,
                           ctypes.byref(nt), 1)
        if rc:
            raise MemoryError("oracle out of memory")
        return c, tasks[:int(nt.value)]
    rc = lib.ora_spamm(_ptr(a), n, _ptr(b), n, _ptr(c), n, n, leaf, tau, None, 0,
                       None, nthreads)
    if rc:
        raise MemoryError("oracle out of memory")
    return c


def flat_tasks(n2a: np.ndarray, n2b: np.ndarray, nb: int, tau: float) -> np.ndarray:
    """All (i, k, j) with n2a[i,k] * n2b[k,j] > tau^2, in (i, j, k) order."""
    n2a = _c(n2a)
    n2b = _c(n2b)
    P = n2a.shape[0]
    lib = _load()
    cnt = lib.ora_flat_tasks(_ptr(n2a), _ptr(n2b), nb, P, tau, None, 0)
    tasks = np.zeros((max(cnt, 1), 3), dtype=np.int32)
    lib.ora_flat_tasks(_ptr(n2a), _ptr(n2b), nb, P, tau,
                       tasks.ctypes.data_as(ctypes.c_void_p), cnt)
    return tasks[:cnt]


def gemm(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense FP64 product, three loops."""
    a = _c(a)
    b = _c(b)
    n = a.shape[0]
    c = np.zeros((n, n))
    _load().ora_gemm(_ptr(a), _ptr(b), _ptr(c), n)
    return c


def gershgorin(f: np.ndarray):
    """(emin, emax) Gershgorin bounds of a square matrix."""
    f = _c(f)
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    _load().ora_gershgorin(_ptr(f), f.shape[0], ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def sp2(f: np.ndarray, leaf: int, ne: float, tau: float, max_iter: int = 100,
        rule: int = 0, trace_tol: float = 1e-10, idem_tol: float = 1e-8,
        fixed_iters: int = 0, nthreads: int = 0):
    """P = SP2(F, Ne, tau) with SpAMM products.  Returns (P, hist, stop) where
    hist is an (iterations, 6) array of [tr X, tr X^2, ||X^2 - X||_F, branch
    (1 = X^2), surviving leaf triples, tr X_new] and stop the stop reason."""
    f = _c(f)
    n = f.shape[0]
    p = np.zeros((n, n))
    limit = fixed_iters if fixed_iters > 0 else max_iter
    hist = np.zeros((max(limit, 1), H_COLS))
    stop = ctypes.c_int(0)
    it = _load().ora_sp2(_ptr(f), n, leaf, ne, tau, max_iter, rule, trace_tol,
                         idem_tol, fixed_iters, _ptr(p), _ptr(hist),
                         ctypes.byref(stop), nthreads)
    if it < 0:
        raise MemoryError("oracle out of memory")
    return p, hist[:it].copy(), int(stop.value)
