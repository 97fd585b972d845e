"""KIOPS CPU oracle — TEST INFRASTRUCTURE ONLY.

Plain serial FP64 C implementation of the KIOPS method (Gaudreault, Rainwater & Tokman, JCP 372, 2018),
loaded through ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path in ``paper_1804_05126_gb300`` never does, and it
shares no code with the CUDA implementation.

Functions
---------
* :func:`kiops`  Algorithm 1 (Task II) with Algorithms 2-4 — the reference result of every parity test.
* :func:`expm`   diagonal Pade with scaling and squaring (section 3.3.1, Higham 2005).
* :func:`apply`  y = A x for an operator description.
* :func:`iop`    Algorithm 2 alone, returning V and H (for the eq 30 / Theorem 2 invariants).

Pins (checked in ``tests/test_oracle_pins.py`` against things other than the oracle itself): dense
``scipy.linalg.expm`` of the Theorem 1 augmented matrix, the tail of eq 15, DST-I closed forms for
Dirichlet Laplacians, scalar phi closed forms for diagonal A, A = 0, p = 0, happy breakdown, the
Arnoldi-like relation eq 30 and Theorem 2, and full-Arnoldi equivalence (m_o >= m).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kiops_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it runs on x86_64 and aarch64 hosts)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bc_code(op: dict) -> int:
    """Boundary of a stencil description: op["bc"] in {"dirichlet", "periodic", "neumann"}, else the
    boolean op["periodic"]."""
    if op.get("bc") is not None:
        return {"dirichlet": 0, "periodic": 1, "neumann": 2}[op["bc"]]
    return 1 if op.get("periodic") else 0


class _Op(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int64),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("vals", C.c_void_p),
                ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("nspecies", C.c_int), ("bc", C.c_int),
                ("coef", (C.c_double * 7) * 2), ("diag", (C.c_void_p * 2) * 2),
                ("dense", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("m_min", C.c_int), ("m_max", C.c_int), ("m_o", C.c_int), ("normalize", C.c_int),
                ("breakdown_tol", C.c_double), ("max_substeps", C.c_int64), ("max_iterations", C.c_int64),
                ("literal_last_row", C.c_int), ("scenario", C.c_int)]


class _Trace(C.Structure):
    _fields_ = [("substep", C.c_int64), ("j", C.c_int), ("tau", C.c_double), ("t_now", C.c_double),
                ("eps", C.c_double), ("omega", C.c_double), ("accepted", C.c_int), ("breakdown", C.c_int),
                ("m_new", C.c_int), ("tau_new", C.c_double), ("cost_a", C.c_double), ("cost_b", C.c_double),
                ("hnorm", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.oracle_apply.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_void_p]
            lib.oracle_apply.restype = None
            lib.oracle_expm.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
            lib.oracle_expm.restype = C.c_int
            lib.oracle_iop.argtypes = [C.POINTER(_Op), C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                       C.c_double, C.c_void_p, C.c_void_p, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)]
            lib.oracle_iop.restype = C.c_int
            lib.oracle_kiops.argtypes = [C.POINTER(_Op), C.c_double, C.c_int, C.c_void_p, C.c_double, C.c_int,
                                         C.POINTER(_Opts), C.c_void_p, C.c_void_p, C.POINTER(_Trace), C.c_int64,
                                         C.POINTER(C.c_int64)]
            lib.oracle_kiops.restype = C.c_int
            lib.oracle_kiops_task1.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_double,
                                               C.c_int, C.POINTER(_Opts), C.c_void_p, C.c_void_p, C.POINTER(_Trace),
                                               C.c_int64, C.POINTER(C.c_int64)]
            lib.oracle_kiops_task1.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _make_op(op: dict):
    """Build the C description; returns (struct, keepalive list)."""
    s = _Op()
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(np.asarray(x, dtype=dt))
        keep.append(a)
        return a.ctypes.data

    k = op["kind"]
    if k == "csr":
        s.kind, s.n = 0, int(op["n"])
        s.rowptr, s.colind, s.vals = arr(op["rowptr"], np.int32), arr(op["colind"], np.int32), arr(op["vals"], np.float64)
    elif k == "stencil2d":
        s.kind = 1
        s.nx, s.ny, s.nz = int(op["nx"]), int(op["ny"]), 1
        s.nspecies, s.bc = int(op["nspecies"]), _bc_code(op)
        s.n = s.nx * s.ny * s.nspecies
        for sp in range(s.nspecies):
            for c in range(5):
                s.coef[sp][c] = float(op["coef"][sp][c])
        for (r, c), d in op.get("diag", {}).items():
            if d is not None:
                s.diag[r][c] = arr(d, np.float64)
    elif k == "stencil3d":
        s.kind = 2
        s.nx, s.ny, s.nz = int(op["nx"]), int(op["ny"]), int(op["nz"])
        s.nspecies, s.bc = 1, _bc_code(op)
        s.n = s.nx * s.ny * s.nz
        for c in range(7):
            s.coef[0][c] = float(op["coef"][c])
        if op.get("diag") is not None:
            s.diag[0][0] = arr(op["diag"], np.float64)
    elif k == "dense":
        s.kind, s.n = 3, int(op["n"])
        s.dense = arr(op["a"], np.float64)
    else:
        raise ValueError(k)
    return s, keep


def apply(op: dict, x: np.ndarray) -> np.ndarray:
    lib = _load()
    s, keep = _make_op(op)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib.oracle_apply(C.byref(s), x.ctypes.data, y.ctypes.data)
    return y


def dense_matrix(op: dict) -> np.ndarray:
    """Columns A e_k assembled with :func:`apply` (tiny N only)."""
    from paper_1804_05126_gb300.workloads import op_size  # input-description helper, no arithmetic
    n = op_size(op)
    cols = [apply(op, np.eye(n)[:, k]) for k in range(n)]
    return np.stack(cols, axis=1)


def expm(a: np.ndarray) -> np.ndarray:
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    f = np.empty_like(a)
    rc = lib.oracle_expm(n, a.ctypes.data, f.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_expm failed ({rc})")
    return f


def iop(op: dict, b: np.ndarray, v: np.ndarray, m: int, m_o: int = 2, breakdown_tol: float = 1e-12):
    """Algorithm 2 from start vector v (length N+p) with B built from b[1..p]; returns (V, H, j, breakdown)
    with V of shape (N+p, m+1) and H of shape (m+2, m+2) (1-based H(i,k) at H[i-1, k-1])."""
    lib = _load()
    s, keep = _make_op(op)
    b = np.ascontiguousarray(b, dtype=np.float64)
    p = b.shape[0] - 1
    n = b.shape[1]
    v = np.ascontiguousarray(v, dtype=np.float64)
    V = np.zeros((m + 1, n + p))
    H = np.zeros((m + 2, m + 2))
    j, bd = C.c_int(0), C.c_int(0)
    rc = lib.oracle_iop(C.byref(s), p, b.ctypes.data, v.ctypes.data, m, m_o, breakdown_tol, V.ctypes.data,
                        H.ctypes.data, C.byref(j), C.byref(bd))
    if rc != 0:
        raise RuntimeError(f"oracle_iop failed ({rc})")
    return V.T.copy(), H, j.value, bool(bd.value)


def kiops(op: dict, tau: float, b: np.ndarray, tol: float, m_init: int = 10, m_min: int = 10, m_max: int = 128,
          m_o: int = 2, normalize: bool = True, breakdown_tol: float = 1e-12, max_substeps: int = 10**6,
          max_iterations: int = 10**7, literal_last_row: bool = False, trace_cap: int = 100000,
          scenario: int = 0):
    """Algorithm 1 (Task II).  b has shape (p+1, N) in natural order b_0..b_p.

    Returns (w, stats, trace): stats = dict(substeps, rejected, matvecs, m_last, iterations, status),
    trace = list of per-iteration dicts (j, tau, t_now, eps, omega, accepted, breakdown, m_new, tau_new, and
    the eq 40 costs cost_a / cost_b of the two scenarios).  scenario = 1 lets the cheaper scenario replace
    Algorithm 4's change of m (reading R9 of the C source).
    """
    lib = _load()
    s, keep = _make_op(op)
    b = np.ascontiguousarray(b, dtype=np.float64)
    p = b.shape[0] - 1
    n = b.shape[1]
    o = _Opts(m_min, m_max, m_o, int(normalize), breakdown_tol, max_substeps, max_iterations, int(literal_last_row),
              int(scenario))
    w = np.empty(n)
    st = np.zeros(5, dtype=np.int64)
    tr = (_Trace * max(trace_cap, 1))()
    tl = C.c_int64(0)
    rc = lib.oracle_kiops(C.byref(s), float(tau), p, b.ctypes.data, float(tol), int(m_init), C.byref(o),
                          w.ctypes.data, st.ctypes.data, tr, trace_cap, C.byref(tl))
    stats = dict(substeps=int(st[0]), rejected=int(st[1]), matvecs=int(st[2]), m_last=int(st[3]),
                 iterations=int(st[4]), status=int(rc))
    trace = [dict(substep=t.substep, j=t.j, tau=t.tau, t_now=t.t_now, eps=t.eps, omega=t.omega,
                  accepted=bool(t.accepted), breakdown=bool(t.breakdown), m_new=t.m_new, tau_new=t.tau_new,
                  cost_a=t.cost_a, cost_b=t.cost_b, hnorm=t.hnorm)
             for t in tr[: tl.value]]
    return w, stats, trace


def kiops_task1(op: dict, T, b: np.ndarray, tol: float, m_init: int = 10, m_min: int = 10, m_max: int = 128,
                m_o: int = 2, normalize: bool = True, breakdown_tol: float = 1e-12, max_substeps: int = 10**6,
                max_iterations: int = 10**7):
    """Task I (Algorithm 1 with Algorithm 3's intermediate outputs): returns (W, stats) with W[l] =
    (1/T[l])^p * (top N entries of e^{T[l] A~} v), T increasing and positive."""
    lib = _load()
    s, keep = _make_op(op)
    b = np.ascontiguousarray(b, dtype=np.float64)
    p = b.shape[0] - 1
    n = b.shape[1]
    T = np.ascontiguousarray(T, dtype=np.float64)
    o = _Opts(m_min, m_max, m_o, int(normalize), breakdown_tol, max_substeps, max_iterations, 0, 0)
    W = np.empty((len(T), n))
    st = np.zeros(5, dtype=np.int64)
    tr = (_Trace * 1)()
    tl = C.c_int64(0)
    rc = lib.oracle_kiops_task1(C.byref(s), T.ctypes.data, len(T), p, b.ctypes.data, float(tol), int(m_init),
                                C.byref(o), W.ctypes.data, st.ctypes.data, tr, 0, C.byref(tl))
    stats = dict(substeps=int(st[0]), rejected=int(st[1]), matvecs=int(st[2]), m_last=int(st[3]),
                 iterations=int(st[4]), status=int(rc))
    return W, stats
