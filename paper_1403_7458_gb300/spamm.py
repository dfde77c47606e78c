"""Python binding of the C ABI in `include/spamm.h` (argument marshalling only).

Every operation runs in the CUDA library `_lib/libspamm.so`; this module
converts torch tensors / numpy arrays to pointers and the current torch CUDA
stream to a `cudaStream_t`.  There is no CPU fallback: `load()` raises when
the library has not been built.

Functions mirror the C entry points:
    tree_build(a, leaf=32)                     -> Matrix
    multiply(A, B, tau, C=None, prec=..)       -> (Matrix, dict stats)
    to_dense(M, out=None)                      -> tensor / array
    norms(M, tier)                             -> numpy (2^t x 2^t)
    task_list(A, B, tau)                       -> (off, k) numpy arrays
    sp2_solve(F, ne, tau, ...)                 -> (Matrix, dict report)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libspamm.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_CAPACITY, E_TIMEOUT, E_NOCONV, E_NOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
FP64, OZAKI_BF16, BF16, BF16X3, TF32, TF32X3 = 0, 1, 2, 3, 4, 5
F_TIMING = 1
F_NOSYM = 2
F_HEAVIEST = 4
F_NOGRAPH = 8
TUNE_MAX = 6
RULE_TRACE_DISTANCE, RULE_TRACE_ABOVE = 0, 1
STOP_CONVERGED, STOP_STAGNATED, STOP_FIXED, STOP_MAXITER = 0, 1, 2, 3
H_FILL, H_COLS = 6, 7

_lib = None


class SpammError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, _lib.spamm_strerror(status).decode(),
                                          _lib.spamm_last_error().decode()))


class _Opts(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("slices", ctypes.c_int32), ("flags", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("tasks", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("flops_useful", ctypes.c_double), ("flops_issued", ctypes.c_double),
                ("ms_cull", ctypes.c_float), ("ms_gemm", ctypes.c_float),
                ("ms_norm", ctypes.c_float), ("sums_rounded", ctypes.c_int32)]


class _Tune(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int32), ("flags", ctypes.c_int32), ("ms", ctypes.c_float),
                ("tried", ctypes.c_int32), ("cand_leaf", ctypes.c_int32 * TUNE_MAX),
                ("cand_flags", ctypes.c_int32 * TUNE_MAX), ("cand_ms", ctypes.c_float * TUNE_MAX),
                ("cand_tasks", ctypes.c_int64 * TUNE_MAX)]


class _Sp2Opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("rule", ctypes.c_int32),
                ("trace_tol", ctypes.c_double), ("idem_tol", ctypes.c_double),
                ("fixed_iters", ctypes.c_int32), ("leaf", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Sp2Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("stop_reason", ctypes.c_int32),
                ("trace_err", ctypes.c_double), ("idem_err", ctypes.c_double),
                ("emin", ctypes.c_double), ("emax", ctypes.c_double),
                ("tasks_total", ctypes.c_int64), ("flops_useful", ctypes.c_double),
                ("flops_tensor", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_cull", ctypes.c_double),
                ("ms_gemm", ctypes.c_double), ("ms_update", ctypes.c_double),
                ("launches", ctypes.c_int64), ("symmetric", ctypes.c_int32),
                ("graphed", ctypes.c_int32), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int32), ("sums_rounded", ctypes.c_int32)]


def load():
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library not built: %s (run __graft_entry__.build())" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    H = ctypes.POINTER(ctypes.c_void_p)
    lib.spamm_tree_build.argtypes = [P, i64, i64, dbl, ctypes.POINTER(_Opts), P, H]
    lib.spamm_multiply.argtypes = [P, P, dbl, H, ctypes.POINTER(_Opts), ctypes.POINTER(_Stats), P]
    lib.spamm_multiply_batched.argtypes = [i32, P, P, P, P, ctypes.POINTER(_Opts), ctypes.POINTER(_Stats), P]
    lib.spamm_autotune_batched.argtypes = [i32, P, P, P, P, ctypes.POINTER(_Opts), i32,
                                           ctypes.POINTER(_Tune), P]
    lib.spamm_to_dense.argtypes = [P, P, i64, P]
    lib.spamm_norms.argtypes = [P, i32, P, P]
    lib.spamm_info.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64),
                               ctypes.POINTER(i32), ctypes.POINTER(i64)]
    lib.spamm_task_list.argtypes = [P, P, dbl, P, P, i64, ctypes.POINTER(i64), P]
    lib.spamm_cull_noalloc.argtypes = [P, i64, P, i64, i64, dbl, P, P, i64, P]
    lib.spamm_watchdog_selftest.argtypes = [i32, P]
    lib.spamm_trim.argtypes = []
    lib.spamm_free.argtypes = [P]
    lib.spamm_free.restype = None
    lib.spamm_release_scratch.argtypes = [P, P]
    lib.spamm_release_scratch.restype = None
    lib.spamm_strerror.argtypes = [ctypes.c_int]
    lib.spamm_strerror.restype = ctypes.c_char_p
    lib.spamm_last_error.argtypes = []
    lib.spamm_last_error.restype = ctypes.c_char_p
    lib.sp2_solve.argtypes = [P, dbl, dbl, ctypes.POINTER(_Sp2Opts), H,
                              ctypes.POINTER(_Sp2Report), P]
    for name in ("spamm_tree_build", "spamm_multiply", "spamm_multiply_batched", "spamm_autotune_batched",
                 "spamm_to_dense", "spamm_norms",
                 "spamm_info", "spamm_task_list", "sp2_solve", "spamm_cull_noalloc", "spamm_watchdog_selftest",
                 "spamm_trim"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc, where, allow=()):
    if rc != OK and rc not in allow:
        raise SpammError(rc, where)
    return rc


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _data(a):
    """(pointer, n, ld, keepalive) of a square FP64 row-major matrix."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or a.dim() != 2 or a.shape[0] != a.shape[1]:
                raise ValueError("square float64 tensor expected")
            if a.stride(1) != 1:
                a = a.contiguous()
            return ctypes.c_void_p(a.data_ptr()), a.shape[0], a.stride(0), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a.ctypes.data_as(ctypes.c_void_p), a.shape[0], a.shape[0], a


class Matrix:
    """Owner of a `spamm_mat_t` handle."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        n, leaf, nb, depth = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        stored = ctypes.c_int64()
        _check(load().spamm_info(self._h, ctypes.byref(n), ctypes.byref(leaf), ctypes.byref(nb),
                                 ctypes.byref(depth), ctypes.byref(stored)), "spamm_info")
        self.n, self.leaf, self.nb, self.depth = n.value, leaf.value, nb.value, depth.value
        self.stored = stored.value  # leaves stored (nb * nb when dense)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            load().spamm_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tree_build(a, leaf: int = 32, drop: float = 0.0, stream=None) -> Matrix:
    """Leaf storage + norm quadtree of an n x n FP64 matrix (host or device).
    Leaves with ||leaf||_F <= drop are not stored (drop < 0: store all)."""
    ptr, n, ld, keep = _data(a)
    h = ctypes.c_void_p()
    opts = _Opts(leaf, FP64, 0, 0)
    _check(load().spamm_tree_build(ptr, n, ld, float(drop), ctypes.byref(opts), _stream(stream),
                                   ctypes.byref(h)), "spamm_tree_build")
    del keep
    return Matrix(h.value)


def multiply(A: Matrix, B: Matrix, tau: float, C: Matrix | None = None, prec: int = FP64,
             slices: int = 0, timing: bool = False, stats: bool = False, stream=None, flags: int = 0):
    """C = SpAMM(A, B, tau).  Returns (C, stats dict or None)."""
    h = ctypes.c_void_p(C.handle.value if C is not None else None)
    opts = _Opts(A.leaf, prec, slices, flags | (F_TIMING if timing else 0))
    st = _Stats()
    want = stats or timing
    _check(load().spamm_multiply(A.handle, B.handle, float(tau), ctypes.byref(h),
                                 ctypes.byref(opts), ctypes.byref(st) if want else None,
                                 _stream(stream)), "spamm_multiply")
    out = C if C is not None else Matrix(h.value)
    info = None
    if want:
        info = {k: getattr(st, k) for k, _ in _Stats._fields_ if k != "reserved"}
    return out, info


def multiply_batched(A, B, tau, C=None, prec: int = FP64, slices: int = 0, timing: bool = False,
                     stats: bool = False, stream=None, flags: int = 0):
    """C[m] = SpAMM(A[m], B[m], tau[m]) for every m, leaf products of the whole
    batch in one launch.  `tau` is a float or a sequence; `C` None or a list
    whose None entries are created.  Returns (list of C, stats dict or None:
    totals over the batch)."""
    count = len(A)
    if len(B) != count:
        raise ValueError("A and B differ in length")
    taus = [float(tau)] * count if np.isscalar(tau) else [float(t) for t in tau]
    if len(taus) != count:
        raise ValueError("tau has the wrong length")
    Cs = list(C) if C is not None else [None] * count
    if len(Cs) != count:
        raise ValueError("C has the wrong length")
    ha = (ctypes.c_void_p * max(count, 1))(*[a.handle.value for a in A])
    hb = (ctypes.c_void_p * max(count, 1))(*[b.handle.value for b in B])
    hc = (ctypes.c_void_p * max(count, 1))(*[c.handle.value if c is not None else None for c in Cs])
    ht = (ctypes.c_double * max(count, 1))(*taus)
    opts = _Opts(A[0].leaf if count else 32, prec, slices, flags | (F_TIMING if timing else 0))
    st = _Stats()
    want = stats or timing
    _check(load().spamm_multiply_batched(count, ha, hb, ht, hc, ctypes.byref(opts),
                                         ctypes.byref(st) if want else None, _stream(stream)),
           "spamm_multiply_batched")
    out = [Cs[m] if Cs[m] is not None else Matrix(hc[m]) for m in range(count)]
    info = None
    if want:
        info = {k: getattr(st, k) for k, _ in _Stats._fields_ if k != "reserved"}
    return out, info


def autotune_batched(a, b, tau, prec: int = FP64, slices: int = 0, reps: int = 3, stream=None):
    """Leaf size and tile schedule for a batch of products a[m] x b[m] (dense
    FP64 square matrices, host arrays or CUDA tensors) chosen by timing.
    Returns {"leaf", "flags", "ms", "candidates": [(leaf, flags, ms, tasks)]}."""
    count = len(a)
    if len(b) != count or count < 1:
        raise ValueError("a and b must be equal, non-empty lists")
    keep, pa, pb, ns = [], [], [], []
    for x, y in zip(a, b):
        px, nx, ldx, kx = _data(x)
        if y is x:
            py, ky = px, kx
        else:
            py, ny, ldy, ky = _data(y)
            if ny != nx or ldy != ny:
                raise ValueError("a[m] and b[m] must be contiguous and of equal size")
        if ldx != nx:
            raise ValueError("contiguous matrices expected")
        keep += [kx, ky]
        pa.append(px.value)
        pb.append(py.value)
        ns.append(nx)
    taus = [float(tau)] * count if np.isscalar(tau) else [float(t) for t in tau]
    ha = (ctypes.c_void_p * count)(*pa)
    hb = (ctypes.c_void_p * count)(*pb)
    hn = (ctypes.c_int64 * count)(*ns)
    ht = (ctypes.c_double * count)(*taus)
    opts = _Opts(0, prec, slices, 0)
    out = _Tune()
    _check(load().spamm_autotune_batched(count, ha, hb, hn, ht, ctypes.byref(opts), reps,
                                         ctypes.byref(out), _stream(stream)), "spamm_autotune_batched")
    del keep
    cands = [(out.cand_leaf[q], out.cand_flags[q], out.cand_ms[q], out.cand_tasks[q]) for q in range(out.tried)]
    return {"leaf": out.leaf, "flags": out.flags, "ms": out.ms, "candidates": cands}


def watchdog_selftest(ms: int = 100, stream=None) -> int:
    """Status of the watchdog self-test (E_TIMEOUT when the bounded wait gave
    up as it should)."""
    return load().spamm_watchdog_selftest(int(ms), _stream(stream))


def release_scratch(M: Matrix, stream=None):
    """Free the slices and task lists a handle keeps for later products."""
    load().spamm_release_scratch(M.handle, _stream(stream))


def trim():
    """Hand the device memory the library keeps cached back to the driver
    (waits for the device)."""
    _check(load().spamm_trim(), "spamm_trim")


def to_dense(M: Matrix, out=None, stream=None):
    """Dense copy (torch tensor on the current device unless `out` is given)."""
    if out is None:
        import torch
        out = torch.empty((M.n, M.n), dtype=torch.float64, device="cuda")
    ptr, n, ld, keep = _data(out)
    if n != M.n:
        raise ValueError("output has the wrong size")
    _check(load().spamm_to_dense(M.handle, ptr, ld, _stream(stream)), "spamm_to_dense")
    return keep


def norms(M: Matrix, tier: int, stream=None) -> np.ndarray:
    w = 1 << tier
    out = np.zeros((w, w))
    _check(load().spamm_norms(M.handle, tier, out.ctypes.data_as(ctypes.c_void_p),
                              _stream(stream)), "spamm_norms")
    return out


def task_list(A: Matrix, B: Matrix, tau: float, stream=None):
    """(off, k): surviving k of output leaf g = i*nb + j are k[off[g]:off[g+1]]."""
    lib = load()
    G = A.nb * A.nb
    off = np.zeros(G + 1, dtype=np.int64)
    nt = ctypes.c_int64()
    rc = lib.spamm_task_list(A.handle, B.handle, float(tau), off.ctypes.data_as(ctypes.c_void_p),
                             None, 0, ctypes.byref(nt), _stream(stream))
    _check(rc, "spamm_task_list", allow=(E_CAPACITY,))
    k = np.zeros(max(nt.value, 1), dtype=np.uint32)
    _check(lib.spamm_task_list(A.handle, B.handle, float(tau), off.ctypes.data_as(ctypes.c_void_p),
                               k.ctypes.data_as(ctypes.c_void_p), k.size, ctypes.byref(nt),
                               _stream(stream)), "spamm_task_list")
    return off, k[:nt.value]


def cull_noalloc(n2a, n2b, nb: int, tau: float, off, klist, stream=None):
    """spamm_cull_noalloc on caller-owned CUDA tensors: n2a, n2b (float64,
    >= nb x nb, rows contiguous), off (int64, >= nb*nb + 1 entries), klist
    (4-byte elements, contiguous, any length, or None).  Asynchronous;
    off[nb*nb] holds the total.  The tensors are checked here (device, type,
    layout, size), since the C call can only trust the pointers it gets."""
    import torch
    nb = int(nb)
    for name, t in (("n2a", n2a), ("n2b", n2b)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2):
            raise ValueError("%s: 2-D float64 CUDA tensor expected" % name)
        if t.stride(1) != 1 or t.shape[0] < nb or t.shape[1] < nb or t.stride(0) < nb:
            raise ValueError("%s: needs >= nb x nb with contiguous rows" % name)
    if not (isinstance(off, torch.Tensor) and off.is_cuda and off.dtype == torch.int64 and off.is_contiguous()
            and off.numel() >= nb * nb + 1):
        raise ValueError("off: contiguous int64 CUDA tensor of >= nb*nb + 1 entries expected")
    if klist is not None and not (isinstance(klist, torch.Tensor) and klist.is_cuda and klist.element_size() == 4
                                  and klist.is_contiguous()):
        raise ValueError("klist: contiguous CUDA tensor of 4-byte elements expected")
    cap = klist.numel() if klist is not None else 0
    _check(load().spamm_cull_noalloc(
        ctypes.c_void_p(n2a.data_ptr()), n2a.stride(0), ctypes.c_void_p(n2b.data_ptr()),
        n2b.stride(0), nb, float(tau), ctypes.c_void_p(off.data_ptr()),
        ctypes.c_void_p(klist.data_ptr() if cap else 0), cap, _stream(stream)),
        "spamm_cull_noalloc")


def sp2_solve(F: Matrix, ne: float, tau: float, P: Matrix | None = None, max_iter: int = 100,
              rule: int = RULE_TRACE_DISTANCE, trace_tol: float = 1e-10, idem_tol: float = 1e-8,
              fixed_iters: int = 0, prec: int = FP64, slices: int = 0, timing: bool = False,
              symmetric: bool = True, stream=None, flags: int = 0):
    """P = SP2(F, Ne, tau).  Returns (P, report dict with a 'history' array)."""
    opts = _Sp2Opts(max_iter, rule, trace_tol, idem_tol, fixed_iters, F.leaf, prec, slices,
                    flags | (F_TIMING if timing else 0) | (0 if symmetric else F_NOSYM), 0)
    cap = fixed_iters if fixed_iters > 0 else max_iter
    hist = np.zeros((max(cap, 1), H_COLS))
    rep = _Sp2Report()
    rep.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rep.history_cap = hist.shape[0]
    h = ctypes.c_void_p(P.handle.value if P is not None else None)
    rc = load().sp2_solve(F.handle, float(ne), float(tau), ctypes.byref(opts), ctypes.byref(h),
                          ctypes.byref(rep), _stream(stream))
    _check(rc, "sp2_solve", allow=(E_NOCONV,))
    out = P if P is not None else Matrix(h.value)
    report = {k: getattr(rep, k) for k, _ in _Sp2Report._fields_
              if k not in ("history", "history_cap", "reserved")}
    report["history"] = hist[:rep.iters].copy()
    report["converged"] = rc == OK
    return out, report
