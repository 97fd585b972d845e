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
* :func:`cost_eq40`, :func:`n_mult`, :func:`op_nonzeros`  the section 3.2 cost model's pieces.
* :class:`Alg4`  Algorithm 4 with eqs 39, 43-46 for one iteration at a time (the adaptivity memory of the
  substep is kept between calls), for scripted error-estimate sequences.

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
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc at -O3 (portable flags, no -march: it runs on x86_64 and aarch64 hosts and
    must give the same results on both).  openmp=True builds the all-core variant used only to time the CPU
    baseline (the parity oracle is the serial build)."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-std=c11", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


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


class _Alg4State(C.Structure):
    _fields_ = [("have_prev", C.c_int), ("prev_j", C.c_int), ("prev_tau", C.c_double), ("prev_omega", C.c_double),
                ("prev_eps", C.c_double), ("kappa", C.c_double), ("qp1_est", C.c_double)]


class _Alg4Out(C.Structure):
    _fields_ = [("omega", C.c_double), ("accepted", C.c_int), ("kappa", C.c_double), ("qp1", C.c_double),
                ("remaining", C.c_double), ("tau_new", C.c_double), ("m_new", C.c_int)]


def _load(parallel: bool = False):
    """The serial parity oracle, or (parallel=True) its OpenMP build for the all-core baseline timing."""
    global _lib, _lib_omp
    with _lock:
        if parallel:
            if _lib_omp is None:
                _lib_omp = _declare(C.CDLL(build(openmp=True)))
            return _lib_omp
        if _lib is None:
            _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(lib):
    """Argument and result types of the exported functions."""
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
    lib.oracle_alg4.argtypes = [C.POINTER(_Alg4State), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                C.POINTER(_Alg4Out)]
    lib.oracle_alg4.restype = None
    lib.oracle_cost_eq40.argtypes = [C.c_double] * 7
    lib.oracle_cost_eq40.restype = C.c_double
    lib.oracle_n_mult.argtypes = [C.c_double]
    lib.oracle_n_mult.restype = C.c_double
    lib.oracle_op_nonzeros.argtypes = [C.POINTER(_Op)]
    lib.oracle_op_nonzeros.restype = C.c_double
    return lib


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


def cost_eq40(remaining: float, tau: float, m: float, n: float, p: float, nz: float, n_mult: float) -> float:
    """Eq 40 with eqs 41-42: the cost of finishing `remaining` with steps tau and Krylov dimension m."""
    return float(_load().oracle_cost_eq40(remaining, tau, m, n, p, nz, n_mult))


def n_mult(x: float) -> float:
    """Multiplications of the scaling-and-squaring Pade method of [47] for a matrix of 1-norm x (eq 42)."""
    return float(_load().oracle_n_mult(x))


def op_nonzeros(op: dict) -> float:
    """nz of eq 41 for an operator description (reading R9: the operator's stored nonzeros)."""
    s, keep = _make_op(op)
    return float(_load().oracle_op_nonzeros(C.byref(s)))


class Alg4:
    """The oracle's Algorithm 4 (eq 39, sections 3.6.1-3.6.2, readings R2-R5) driven one iteration at a time:
    the same function Algorithm 1 calls after every exponential.  The adaptivity memory of the substep
    (kappa of eq 45, the order estimate of eq 43, the last rejected iteration) is kept between calls."""

    def __init__(self, m_min: int = 10, m_max: int = 128, T_end: float = 1.0, tol: float = 1e-8):
        self.m_min, self.m_max, self.T_end, self.tol = m_min, m_max, T_end, tol
        self._st = _Alg4State()

    def step(self, new_substep: bool, j: int, m: int, tau: float, t_now: float, eps: float,
             breakdown: bool = False) -> dict:
        out = _Alg4Out()
        _load().oracle_alg4(C.byref(self._st), int(new_substep), j, m, self.m_min, self.m_max, tau, t_now,
                            self.T_end, self.tol, eps, int(breakdown), C.byref(out))
        return {"omega": out.omega, "accepted": bool(out.accepted), "kappa": out.kappa, "qp1": out.qp1,
                "remaining": out.remaining, "tau_new": out.tau_new, "m_new": out.m_new}


def kiops(op: dict, tau: float, b: np.ndarray, tol: float, m_init: int = 10, m_min: int = 10, m_max: int = 128,
          m_o: int = 2, normalize: bool = True, breakdown_tol: float = 1e-12, max_substeps: int = 10**6,
          max_iterations: int = 10**7, literal_last_row: bool = False, trace_cap: int = 100000,
          scenario: int = 0, parallel: bool = False):
    """Algorithm 1 (Task II).  b has shape (p+1, N) in natural order b_0..b_p.

    Returns (w, stats, trace): stats = dict(substeps, rejected, matvecs, m_last, iterations, status),
    trace = list of per-iteration dicts (j, tau, t_now, eps, omega, accepted, breakdown, m_new, tau_new, and
    the eq 40 costs cost_a / cost_b of the two scenarios).  scenario = 1 lets the cheaper scenario replace
    Algorithm 4's change of m (reading R9 of the C source).  parallel=True runs the OpenMP build on the
    threads OMP_NUM_THREADS allows (CPU-baseline timing only; its sums are split over threads).
    """
    lib = _load(parallel)
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
