"""Thin Python binding of the C ABI in include/kiops.h (ctypes; argument marshalling only).

Every step of the solve runs in the CUDA library ``_build/libkiops.so``; this module only converts
arguments.  Functions with the C names (``kiops_create``, ``kiops_solve`` ...) map one to one onto the
C entry points; :class:`Solver` and :class:`Operator` wrap them for torch CUDA tensors (PyTorch supplies
device memory and streams).  There is no CPU fallback: :func:`lib` raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

KIOPS_MAX_P = 16
KIOPS_MAX_M = 256
STATUS = {0: "KIOPS_OK", 1: "KIOPS_EINVAL", 2: "KIOPS_ENOMEM", 3: "KIOPS_ENOTCONV", 4: "KIOPS_ETIMEOUT",
          5: "KIOPS_ECUDA", 6: "KIOPS_EBUSY"}
FP64, FP32_BASIS = 0, 1
ENGINE_AUTO, ENGINE_GRID, ENGINE_CTA = 0, 1, 2


class KiopsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class kiops_config(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("m_min", C.c_int), ("m_max", C.c_int),
                ("normalize_B", C.c_int), ("breakdown_tol", C.c_double), ("max_substeps", C.c_int64),
                ("max_iterations", C.c_int64), ("timeout_s", C.c_double), ("engine", C.c_int),
                ("grid_blocks", C.c_int), ("profile", C.c_int), ("fuse_stencil", C.c_int),
                ("batch_team_blocks", C.c_int), ("fused_smem", C.c_int), ("scenario", C.c_int),
                ("block_threads", C.c_int), ("tma", C.c_int), ("tile_w", C.c_int), ("tile_h", C.c_int),
                ("tma_stages", C.c_int), ("tma_prefetch", C.c_int), ("tma_fixed", C.c_int)]


class kiops_stats(C.Structure):
    _fields_ = [("substeps", C.c_int64), ("rejected", C.c_int64), ("matvecs", C.c_int64),
                ("iterations", C.c_int64), ("expm_calls", C.c_int64), ("m_last", C.c_int), ("engine", C.c_int),
                ("grid_blocks", C.c_int), ("status", C.c_int), ("err_est", C.c_double),
                ("phase_cycles", C.c_int64 * 16), ("tile_path", C.c_int), ("tile_w", C.c_int),
                ("tile_h", C.c_int)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["phase_cycles"] = list(self.phase_cycles)
        return d


class kiops_trace_rec(C.Structure):
    _fields_ = [("substep", C.c_int64), ("j", C.c_int), ("accepted", C.c_int), ("breakdown", C.c_int),
                ("m_new", C.c_int), ("tau", C.c_double), ("t_now", C.c_double), ("eps", C.c_double),
                ("omega", C.c_double), ("tau_new", C.c_double), ("cost_a", C.c_double), ("cost_b", C.c_double),
                ("hnorm", C.c_double)]


BC_DIRICHLET, BC_PERIODIC, BC_NEUMANN = 0, 1, 2


def bc_code(desc: dict) -> int:
    """KIOPS_BC_* of a stencil description: desc["bc"] in {"dirichlet", "periodic", "neumann"}, else the
    boolean desc["periodic"]."""
    if desc.get("bc") is not None:
        return {"dirichlet": BC_DIRICHLET, "periodic": BC_PERIODIC, "neumann": BC_NEUMANN}[desc["bc"]]
    return BC_PERIODIC if desc.get("periodic") else BC_DIRICHLET


class kiops_stencil2d_desc(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nspecies", C.c_int), ("bc", C.c_int),
                ("coef", (C.c_double * 5) * 2), ("diag", (C.c_void_p * 2) * 2), ("nfields", C.c_int),
                ("dfield", (C.c_int * 2) * 2), ("dconst", (C.c_double * 2) * 2), ("dweight", (C.c_double * 2) * 2),
                ("field", C.c_void_p * 2)]


class kiops_stencil3d_desc(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("bc", C.c_int),
                ("coef", C.c_double * 7), ("diag", C.c_void_p)]


class kiops_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("queue_slots", C.c_int), ("small_team_blocks", C.c_int),
                ("large_team_blocks", C.c_int), ("large_teams", C.c_int), ("large_work_threshold", C.c_double),
                ("idle_timeout_s", C.c_double), ("solo_min_unknowns", C.c_double)]


class kiops_request(C.Structure):
    _fields_ = [("A", C.c_void_p), ("tau", C.c_double), ("p", C.c_int), ("b", C.POINTER(C.c_void_p)),
                ("tol", C.c_double), ("m_init", C.c_int), ("m_o", C.c_int), ("prec", C.c_int), ("w", C.c_void_p)]


class kiops_pde(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int64), ("param", C.c_double * 4)]


class kiops_integrate_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("kiops_calls", C.c_int64), ("matvecs", C.c_int64), ("substeps", C.c_int64),
                ("rejected", C.c_int64), ("m_last", C.c_int * 3)]

    def as_dict(self) -> dict:
        return {"steps": self.steps, "kiops_calls": self.kiops_calls, "matvecs": self.matvecs,
                "substeps": self.substeps, "rejected": self.rejected, "m_last": list(self.m_last)}


PDE_ADR2D, PDE_GRAY_SCOTT2D = 0, 1
SCHEMES = {"epirk4s3": 0, "epirk4s3a": 1, "exprb5s3": 2}


def pde_struct(pde: dict) -> kiops_pde:
    """kiops_pde of a test-problem description {"pde": "adr2d", "n", "eps", "alpha", "gamma"} or
    {"pde": "gray_scott2d", "n", "du", "dv", "a", "b"}."""
    d = kiops_pde()
    d.n = int(pde["n"])
    if pde["pde"] == "adr2d":
        d.kind = PDE_ADR2D
        vals = [pde["eps"], pde["alpha"], pde["gamma"], 0.0]
    elif pde["pde"] == "gray_scott2d":
        d.kind = PDE_GRAY_SCOTT2D
        vals = [pde["du"], pde["dv"], pde["a"], pde["b"]]
    else:
        raise ValueError(f"unknown test problem {pde['pde']!r}")
    for k, v in enumerate(vals):
        d.param[k] = float(v)
    return d


_lock = threading.Lock()
_lib = None

_SIGS = {
    "kiops_config_default": ([C.POINTER(kiops_config)], C.c_int),
    "kiops_constants": ([C.POINTER(C.c_double)], C.c_int),
    "kiops_create": ([C.POINTER(C.c_void_p), C.POINTER(kiops_config)], C.c_int),
    "kiops_destroy": ([C.c_void_p], C.c_int),
    "kiops_last_error": ([C.c_void_p], C.c_char_p),
    "kiops_status_string": ([C.c_int], C.c_char_p),
    "kiops_attach_workspace": ([C.c_void_p, C.c_void_p, C.c_size_t], C.c_int),
    "kiops_workspace_size": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
    "kiops_op_csr": ([C.c_void_p, C.POINTER(C.c_void_p), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
                     C.c_int),
    "kiops_op_stencil2d": ([C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(kiops_stencil2d_desc)], C.c_int),
    "kiops_op_stencil3d": ([C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(kiops_stencil3d_desc)], C.c_int),
    "kiops_op_destroy": ([C.c_void_p], C.c_int),
    "kiops_op_size": ([C.c_void_p], C.c_int64),
    "kiops_op_apply": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "kiops_solve": ([C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_void_p), C.c_double, C.c_int, C.c_int,
                     C.c_int, C.c_void_p, C.POINTER(kiops_stats)], C.c_int),
    "kiops_solve_traced": ([C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_void_p), C.c_double, C.c_int,
                            C.c_int, C.c_int, C.c_void_p, C.POINTER(kiops_stats), C.POINTER(kiops_trace_rec),
                            C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "kiops_solve_host": ([C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_void_p), C.c_double, C.c_int,
                          C.c_int, C.c_int, C.c_void_p, C.POINTER(kiops_stats)], C.c_int),
    "kiops_solve_batch": ([C.c_void_p, C.c_int, C.POINTER(kiops_request), C.POINTER(kiops_stats)], C.c_int),
    "kiops_set_batch_team_blocks": ([C.c_void_p, C.c_int], C.c_int),
    "kiops_get_config": ([C.c_void_p, C.POINTER(kiops_config)], C.c_int),
    "kiops_set_config": ([C.c_void_p, C.POINTER(kiops_config)], C.c_int),
    "kiops_server_config_default": ([C.POINTER(kiops_server_config)], C.c_int),
    "kiops_server_start": ([C.c_void_p, C.POINTER(kiops_server_config)], C.c_int),
    "kiops_submit": ([C.c_void_p, C.POINTER(kiops_request), C.POINTER(C.c_uint64)], C.c_int),
    "kiops_poll": ([C.c_void_p, C.c_uint64, C.c_double, C.POINTER(C.c_int), C.POINTER(kiops_stats)], C.c_int),
    "kiops_server_info": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "kiops_server_stop": ([C.c_void_p], C.c_int),
    "kiops_server_selftest_abort": ([C.c_void_p], C.c_int),
    "kiops_expm": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "kiops_solve_task1": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                           C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p), C.POINTER(kiops_stats)], C.c_int),
    "kiops_solve_noalloc": ([C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_void_p), C.c_double, C.c_int,
                             C.c_int, C.c_void_p, C.POINTER(kiops_stats)], C.c_int),
    "kiops_pde_rhs": ([C.c_void_p, C.POINTER(kiops_pde), C.c_void_p, C.c_void_p], C.c_int),
    "kiops_selftest_wait_timeout": ([C.c_void_p, C.c_double], C.c_int),
    "kiops_probe_fp64": ([C.c_void_p, C.POINTER(C.c_double)], C.c_int),
    "kiops_integrate": ([C.c_void_p, C.POINTER(kiops_pde), C.c_int, C.c_double, C.c_double, C.c_int64, C.c_double,
                         C.c_int, C.c_void_p, C.POINTER(kiops_integrate_stats)], C.c_int),
}


def lib(build_if_missing: bool = False):
    """Load libkiops.so (raises if it is not built; never falls back to anything else)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library not built ({_build.LIB}); run paper_1804_05126_gb300.build.build()")
            L = C.CDLL(_build.LIB)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


# ---------------------------------------------------------------- same-name wrappers of the C ABI
def kiops_config_default() -> kiops_config:
    cfg = kiops_config()
    lib().kiops_config_default(C.byref(cfg))
    return cfg


def kiops_constants() -> list[float]:
    out = (C.c_double * 6)()
    lib().kiops_constants(out)
    return list(out)


def kiops_create(cfg: kiops_config | None = None) -> int:
    h = C.c_void_p()
    st = lib().kiops_create(C.byref(h), C.byref(cfg) if cfg is not None else None)
    if st:
        raise KiopsError(st, "kiops_create failed")
    return h.value


def kiops_destroy(ctx: int) -> None:
    lib().kiops_destroy(ctx)


def kiops_last_error(ctx: int) -> str:
    return lib().kiops_last_error(ctx).decode()


def _check(ctx, st, what):
    if st:
        raise KiopsError(st, f"{what}: {kiops_last_error(ctx)}")


def kiops_op_csr(ctx: int, n: int, nnz: int, rowptr: int, colind: int, vals: int) -> int:
    h = C.c_void_p()
    _check(ctx, lib().kiops_op_csr(ctx, C.byref(h), n, nnz, rowptr, colind, vals), "kiops_op_csr")
    return h.value


def kiops_op_stencil2d(ctx: int, desc: kiops_stencil2d_desc) -> int:
    h = C.c_void_p()
    _check(ctx, lib().kiops_op_stencil2d(ctx, C.byref(h), C.byref(desc)), "kiops_op_stencil2d")
    return h.value


def kiops_op_stencil3d(ctx: int, desc: kiops_stencil3d_desc) -> int:
    h = C.c_void_p()
    _check(ctx, lib().kiops_op_stencil3d(ctx, C.byref(h), C.byref(desc)), "kiops_op_stencil3d")
    return h.value


def kiops_op_destroy(op: int) -> None:
    lib().kiops_op_destroy(op)


def kiops_op_size(op: int) -> int:
    return int(lib().kiops_op_size(op))


def kiops_op_apply(ctx: int, op: int, x_ptr: int, y_ptr: int) -> None:
    _check(ctx, lib().kiops_op_apply(ctx, op, x_ptr, y_ptr), "kiops_op_apply")


def _ptr_array(ptrs):
    arr = (C.c_void_p * len(ptrs))(*ptrs)
    return arr


def kiops_solve(ctx, op, tau, p, b_ptrs, tol, m_init, m_o, prec, w_ptr) -> dict:
    st = kiops_stats()
    _check(ctx, lib().kiops_solve(ctx, op, tau, p, _ptr_array(b_ptrs), tol, m_init, m_o, prec, w_ptr, C.byref(st)),
           "kiops_solve")
    return st.as_dict()


def kiops_solve_traced(ctx, op, tau, p, b_ptrs, tol, m_init, m_o, prec, w_ptr, trace_cap=4096):
    st = kiops_stats()
    tr = (kiops_trace_rec * trace_cap)()
    n = C.c_int64(0)
    _check(ctx, lib().kiops_solve_traced(ctx, op, tau, p, _ptr_array(b_ptrs), tol, m_init, m_o, prec, w_ptr,
                                         C.byref(st), tr, trace_cap, C.byref(n)), "kiops_solve_traced")
    recs = [{f: getattr(r, f) for f, _ in kiops_trace_rec._fields_} for r in tr[: n.value]]
    for r in recs:
        r["accepted"] = bool(r["accepted"])
        r["breakdown"] = bool(r["breakdown"])
    return st.as_dict(), recs


def kiops_solve_task1(ctx, op, T, p, b_ptrs, tol, m_init, m_o, prec, w_ptrs) -> dict:
    st = kiops_stats()
    Ta = (C.c_double * len(T))(*T)
    _check(ctx, lib().kiops_solve_task1(ctx, op, Ta, len(T), p, _ptr_array(b_ptrs), tol, m_init, m_o, prec,
                                        _ptr_array(w_ptrs), C.byref(st)), "kiops_solve_task1")
    return st.as_dict()


def kiops_solve_host(ctx, op, tau, p, b_host_ptrs, tol, m_init, m_o, prec, w_host_ptr) -> dict:
    st = kiops_stats()
    _check(ctx, lib().kiops_solve_host(ctx, op, tau, p, _ptr_array(b_host_ptrs), tol, m_init, m_o, prec, w_host_ptr,
                                       C.byref(st)), "kiops_solve_host")
    return st.as_dict()


def kiops_solve_batch(ctx, reqs: list[kiops_request]) -> list[dict]:
    n = len(reqs)
    arr = (kiops_request * n)(*reqs)
    stats = (kiops_stats * max(n, 1))()
    _check(ctx, lib().kiops_solve_batch(ctx, n, arr, stats), "kiops_solve_batch")
    return [stats[i].as_dict() for i in range(n)]


def kiops_selftest_wait_timeout(ctx, timeout_s: float) -> int:
    """Status of the bounded-wait self-test (KIOPS_ETIMEOUT = 4 is the designed outcome)."""
    return int(lib().kiops_selftest_wait_timeout(ctx, timeout_s))


def kiops_probe_fp64(ctx) -> float:
    """Measured FP64 FMA throughput of the context's GPU (flop/s)."""
    v = C.c_double(0.0)
    _check(ctx, lib().kiops_probe_fp64(ctx, C.byref(v)), "kiops_probe_fp64")
    return v.value


def kiops_pde_rhs(ctx, pde: kiops_pde, u_ptr, f_ptr) -> None:
    _check(ctx, lib().kiops_pde_rhs(ctx, C.byref(pde), u_ptr, f_ptr), "kiops_pde_rhs")


def kiops_integrate(ctx, pde: kiops_pde, scheme: int, t0: float, t1: float, nsteps: int, tol: float, m_init: int,
                    u_ptr) -> dict:
    st = kiops_integrate_stats()
    _check(ctx, lib().kiops_integrate(ctx, C.byref(pde), scheme, t0, t1, nsteps, tol, m_init, u_ptr, C.byref(st)),
           "kiops_integrate")
    return st.as_dict()


def kiops_solve_noalloc(ctx, op, tau, p, b_ptrs, tol, m_init, m_o, w_ptr) -> dict:
    """The allocation-free solve (FP64, one thread block, fixed device scratch); see include/kiops.h."""
    st = kiops_stats()
    _check(ctx, lib().kiops_solve_noalloc(ctx, op, tau, p, _ptr_array(b_ptrs), tol, m_init, m_o, w_ptr, C.byref(st)),
           "kiops_solve_noalloc")
    return st.as_dict()


def kiops_get_config(ctx) -> kiops_config:
    cfg = kiops_config()
    _check(ctx, lib().kiops_get_config(ctx, C.byref(cfg)), "kiops_get_config")
    return cfg


def kiops_set_config(ctx, cfg: kiops_config) -> None:
    _check(ctx, lib().kiops_set_config(ctx, C.byref(cfg)), "kiops_set_config")


def kiops_set_batch_team_blocks(ctx, team_blocks: int) -> None:
    _check(ctx, lib().kiops_set_batch_team_blocks(ctx, team_blocks), "kiops_set_batch_team_blocks")


def kiops_server_config_default() -> kiops_server_config:
    cfg = kiops_server_config()
    lib().kiops_server_config_default(C.byref(cfg))
    return cfg


def kiops_server_start(ctx, cfg: kiops_server_config | None = None) -> None:
    _check(ctx, lib().kiops_server_start(ctx, C.byref(cfg) if cfg is not None else None), "kiops_server_start")


def kiops_submit(ctx, req: kiops_request) -> int:
    t = C.c_uint64(0)
    _check(ctx, lib().kiops_submit(ctx, C.byref(req), C.byref(t)), "kiops_submit")
    return t.value


def kiops_poll(ctx, ticket: int, timeout_s: float = 0.0):
    done = C.c_int(0)
    st = kiops_stats()
    _check(ctx, lib().kiops_poll(ctx, ticket, timeout_s, C.byref(done), C.byref(st)), "kiops_poll")
    return bool(done.value), (st.as_dict() if done.value else None)


def kiops_server_info(ctx) -> dict:
    v = (C.c_int64 * 8)()
    _check(ctx, lib().kiops_server_info(ctx, v), "kiops_server_info")
    return {"pending": v[0], "in_flight": v[1], "reserved_bytes": v[2], "small_teams": v[3], "large_teams": v[4],
            "large_team_blocks": v[5], "claimed_small": v[6], "claimed_large": v[7]}


def kiops_server_selftest_abort(ctx) -> None:
    """Raise the server's abort word from the host (recovery self-test; see include/kiops.h)."""
    _check(ctx, lib().kiops_server_selftest_abort(ctx), "kiops_server_selftest_abort")


def kiops_server_stop(ctx) -> None:
    _check(ctx, lib().kiops_server_stop(ctx), "kiops_server_stop")


def kiops_expm(ctx, n, a_ptr, f_ptr) -> None:
    _check(ctx, lib().kiops_expm(ctx, n, a_ptr, f_ptr), "kiops_expm")


def kiops_attach_workspace(ctx, ptr, nbytes) -> None:
    _check(ctx, lib().kiops_attach_workspace(ctx, ptr, nbytes), "kiops_attach_workspace")


def kiops_workspace_size(ctx, op, p, m_o, prec) -> int:
    out = C.c_size_t(0)
    _check(ctx, lib().kiops_workspace_size(ctx, op, p, m_o, prec, C.byref(out)), "kiops_workspace_size")
    return int(out.value)


# ---------------------------------------------------------------- torch convenience layer
class Operator:
    """A device operator built from a workload description (see workloads.py); owns its device arrays.
    A 2D description with "shared_fields" passes its coupling block in that form unless shared_fields is
    False (then its "diag" entries are passed)."""

    def __init__(self, solver: "Solver", desc: dict, shared_fields: bool = True):
        import torch
        self.solver = solver
        self.desc = desc
        self._keep = []
        dev = solver.device
        ctx = solver.ctx

        def put(a, dtype):
            t = torch.as_tensor(np.ascontiguousarray(a)).to(device=dev, dtype=dtype).contiguous()
            self._keep.append(t)
            return t.data_ptr()

        k = desc["kind"]
        if k == "csr":
            self.handle = kiops_op_csr(ctx, int(desc["n"]), len(desc["vals"]), put(desc["rowptr"], torch.int32),
                                       put(desc["colind"], torch.int32), put(desc["vals"], torch.float64))
        elif k == "stencil2d":
            d = kiops_stencil2d_desc()
            d.nx, d.ny, d.nspecies, d.bc = int(desc["nx"]), int(desc["ny"]), int(desc["nspecies"]), bc_code(desc)
            for s in range(d.nspecies):
                for c in range(5):
                    d.coef[s][c] = float(desc["coef"][s][c])
            shared = desc.get("shared_fields") if shared_fields else None
            if shared is not None:  # entries affine in fields that several entries share
                d.nfields = len(shared["fields"])
                for f, arr in enumerate(shared["fields"]):
                    d.field[f] = put(arr, torch.float64)
                for s in range(2):
                    for c in range(2):
                        d.dfield[s][c] = -1
                for (r, c), (f, const, weight) in shared["entries"].items():
                    d.dfield[r][c], d.dconst[r][c], d.dweight[r][c] = int(f), float(const), float(weight)
            else:
                for (r, c), arr in desc.get("diag", {}).items():
                    if arr is not None:
                        d.diag[r][c] = put(arr, torch.float64)
            self.handle = kiops_op_stencil2d(ctx, d)
        elif k == "stencil3d":
            d = kiops_stencil3d_desc()
            d.nx, d.ny, d.nz, d.bc = int(desc["nx"]), int(desc["ny"]), int(desc["nz"]), bc_code(desc)
            for c in range(7):
                d.coef[c] = float(desc["coef"][c])
            d.diag = put(desc["diag"], torch.float64) if desc.get("diag") is not None else None
            self.handle = kiops_op_stencil3d(ctx, d)
        else:
            raise ValueError(f"operator kind {k!r} has no device implementation")
        self.n = kiops_op_size(self.handle)

    def apply(self, x):
        import torch
        y = torch.empty_like(x)
        kiops_op_apply(self.solver.ctx, self.handle, x.data_ptr(), y.data_ptr())
        return y

    def close(self):
        if getattr(self, "handle", None):
            kiops_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """A kiops context on a torch CUDA device/stream."""

    def __init__(self, device: int = 0, stream=None, m_min: int = 10, m_max: int = 128, normalize_B: bool = True,
                 breakdown_tol: float = 1e-12, max_substeps: int = 10**6, max_iterations: int = 10**5,
                 timeout_s: float = 10.0, engine: int = ENGINE_AUTO, grid_blocks: int = 0, profile: bool = False,
                 fuse_stencil: bool = True, fused_smem: int = -1, scenario: int = 0, block_threads: int = 0,
                 tma: int = 1, tile: tuple[int, int] | None = None, tma_stages: int = 0,
                 tma_prefetch: int = -1, tma_fixed: int = 1):
        import torch
        self.device = torch.device("cuda", device)
        cfg = kiops_config_default()
        cfg.device = device
        cfg.stream = stream.cuda_stream if stream is not None else None
        cfg.m_min, cfg.m_max, cfg.normalize_B = m_min, m_max, int(normalize_B)
        cfg.breakdown_tol, cfg.max_substeps, cfg.max_iterations = breakdown_tol, max_substeps, max_iterations
        cfg.timeout_s, cfg.engine, cfg.grid_blocks, cfg.profile = timeout_s, engine, grid_blocks, int(profile)
        cfg.fuse_stencil = int(fuse_stencil)
        cfg.fused_smem = int(fused_smem)
        cfg.scenario = int(scenario)
        cfg.block_threads = int(block_threads)
        cfg.tma = int(tma)
        cfg.tile_w, cfg.tile_h = (int(tile[0]), int(tile[1])) if tile else (0, 0)
        cfg.tma_stages = int(tma_stages)
        cfg.tma_prefetch = int(tma_prefetch)
        cfg.tma_fixed = int(tma_fixed)
        self.cfg = cfg
        self.ctx = kiops_create(cfg)

    def configure(self, **fields) -> dict:
        """Change fields of the live context's configuration (e.g. tile_w, tile_h, tma, tma_stages, fused_smem,
        block_threads, grid_blocks); returns the previous values of those fields."""
        cfg = kiops_get_config(self.ctx)
        old = {k: getattr(cfg, k) for k in fields}
        for k, v in fields.items():
            setattr(cfg, k, v)
        kiops_set_config(self.ctx, cfg)
        self.cfg = cfg
        return old

    def operator(self, desc: dict, shared_fields: bool = True) -> Operator:
        return Operator(self, desc, shared_fields)

    @staticmethod
    def _prec(precision) -> int:
        return FP32_BASIS if precision in (FP32_BASIS, "fp32_basis", "fp32") else FP64

    def solve(self, op: Operator, tau: float, b, tol: float, m_init: int = 10, m_o: int = 2, precision="fp64",
              w=None, trace: bool = False, trace_cap: int = 4096):
        """b: (p+1, N) float64 CUDA tensor (natural order b_0..b_p); returns (w, stats[, trace])."""
        import torch
        assert b.is_cuda and b.dtype == torch.float64 and b.is_contiguous()
        p = b.shape[0] - 1
        if w is None:
            w = torch.empty(b.shape[1], dtype=torch.float64, device=b.device)
        ptrs = [b[k].data_ptr() for k in range(p + 1)]
        if trace:
            st, tr = kiops_solve_traced(self.ctx, op.handle, tau, p, ptrs, tol, m_init, m_o, self._prec(precision),
                                        w.data_ptr(), trace_cap)
            return w, st, tr
        st = kiops_solve(self.ctx, op.handle, tau, p, ptrs, tol, m_init, m_o, self._prec(precision), w.data_ptr())
        return w, st

    def solve_task1(self, op: Operator, T, b, tol: float, m_init: int = 10, m_o: int = 2, precision="fp64"):
        """Task I: returns ([w_l], stats) with w_l = (1/T_l)^p sum_k T_l^k phi_k(T_l A) b_k."""
        import torch
        p = b.shape[0] - 1
        ws = [torch.empty(b.shape[1], dtype=torch.float64, device=b.device) for _ in T]
        st = kiops_solve_task1(self.ctx, op.handle, [float(t) for t in T], p, [b[k].data_ptr() for k in range(p + 1)],
                               tol, m_init, m_o, self._prec(precision), [w.data_ptr() for w in ws])
        return ws, st

    def solve_host(self, op: Operator, tau: float, b: np.ndarray, tol: float, m_init: int = 10, m_o: int = 2,
                   precision="fp64", w: np.ndarray | None = None):
        """b: (p+1, N) float64 host array (pinned or pageable); w: host output."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        p = b.shape[0] - 1
        if w is None:
            w = np.empty(b.shape[1], dtype=np.float64)
        ptrs = [b[k].ctypes.data for k in range(p + 1)]
        st = kiops_solve_host(self.ctx, op.handle, tau, p, ptrs, tol, m_init, m_o, self._prec(precision), w.ctypes.data)
        return w, st

    def solve_batch(self, items, team_blocks: int | None = None):
        """items: list of (op, tau, b_tensor, tol, m_init, m_o, precision, w_tensor); team_blocks sets the
        batch team size (None keeps the context's setting, 0 = automatic, 1 = one block per request)."""
        if team_blocks is not None:
            kiops_set_batch_team_blocks(self.ctx, team_blocks)
        reqs, keep = [], []
        for (op, tau, b, tol, m_init, m_o, precision, w) in items:
            p = b.shape[0] - 1
            arr = _ptr_array([b[k].data_ptr() for k in range(p + 1)])
            keep.append(arr)
            reqs.append(kiops_request(op.handle, tau, p, C.cast(arr, C.POINTER(C.c_void_p)), tol, m_init, m_o,
                                      self._prec(precision), w.data_ptr()))
        return kiops_solve_batch(self.ctx, reqs)

    # ---- serving (continuous batching)
    def server_start(self, hbm_budget_bytes: float | None = None, **kw) -> None:
        cfg = kiops_server_config_default()
        if hbm_budget_bytes is not None:
            cfg.hbm_budget_bytes = float(hbm_budget_bytes)
        for k, v in kw.items():
            setattr(cfg, k, v)
        kiops_server_start(self.ctx, cfg)
        self._served = {}

    def submit(self, op: Operator, tau: float, b, tol: float, m_init: int = 10, m_o: int = 2, precision="fp64",
               w=None):
        """Queue one request; returns (ticket, w).  b and w stay borrowed until poll reports done."""
        import torch
        p = b.shape[0] - 1
        if w is None:
            w = torch.empty(b.shape[1], dtype=torch.float64, device=b.device)
        arr = _ptr_array([b[k].data_ptr() for k in range(p + 1)])
        req = kiops_request(op.handle, tau, p, C.cast(arr, C.POINTER(C.c_void_p)), tol, m_init, m_o,
                            self._prec(precision), w.data_ptr())
        t = kiops_submit(self.ctx, req)
        self._served[t] = (op, b, w)
        return t, w

    def poll(self, ticket: int, timeout_s: float = 0.0):
        done, st = kiops_poll(self.ctx, ticket, timeout_s)
        if done:
            self._served.pop(ticket, None)
        return done, st

    def server_info(self) -> dict:
        return kiops_server_info(self.ctx)

    def server_stop(self) -> None:
        kiops_server_stop(self.ctx)

    # ---- exponential integrators on the section 4 test problems
    def pde_rhs(self, pde: dict, u):
        """f(u) of the test problem (u: CUDA float64 tensor of N values)."""
        import torch
        u = u.contiguous()
        f = torch.empty_like(u)
        kiops_pde_rhs(self.ctx, pde_struct(pde), u.data_ptr(), f.data_ptr())
        return f

    def integrate(self, pde: dict, scheme: str, u, t0: float, t1: float, nsteps: int, tol: float = 1e-10,
                  m_init: int = 10):
        """Integrate in place (u: contiguous CUDA float64 tensor) from t0 to t1 in nsteps steps of the
        scheme ("epirk4s3", "epirk4s3a", "exprb5s3"); returns the statistics."""
        assert u.is_contiguous() and u.dtype.is_floating_point and u.element_size() == 8
        return kiops_integrate(self.ctx, pde_struct(pde), SCHEMES[scheme], t0, t1, nsteps, tol, m_init, u.data_ptr())

    def expm(self, a):
        import torch
        a = a.contiguous()
        f = torch.empty_like(a)
        kiops_expm(self.ctx, a.shape[0], a.data_ptr(), f.data_ptr())
        return f

    def close(self):
        if getattr(self, "ctx", None):
            kiops_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
