"""Seeded synthetic inputs: operators shaped like the paper's PDE Jacobians and the vectors b_0..b_p.

This module only generates inputs.  It holds none of the phi-function / Krylov arithmetic: both the
CPU oracle and the CUDA path receive the same operator description and vectors from here and apply
them with their own code.

An operator description is a plain dict:

* ``{"kind": "csr", "n", "rowptr" (int32), "colind" (int32), "vals" (float64)}``
* ``{"kind": "stencil2d", "nx", "ny", "nspecies" (1|2), "periodic" (bool) or "bc" ("dirichlet" |
  "periodic" | "neumann"), "coef" (nspecies x 5:
  centre, -x, +x, -y, +y), "diag" {(r, c): float64 array of nx*ny}}`` — unknowns are species-blocked
  ``[u; v]``, each x-fastest; ``diag[(r, c)]`` couples species c into species r pointwise.  Optionally
  ``"shared_fields": {"fields": [float64 arrays of nx*ny], "entries": {(r, c): (field index or -1, const,
  weight)}}``, the same block with entry (r, c) = const + weight * fields[index].
* ``{"kind": "stencil3d", "nx", "ny", "nz", "periodic", "coef" (7: centre, -x, +x, -y, +y, -z, +z),
  "diag": float64 array of nx*ny*nz or None}``
* ``{"kind": "dense", "n", "a" (n x n float64)}``

The test problems follow section 4 of the paper (2D advection-diffusion-reaction, 2D Gray-Scott, 1D
Dirichlet Laplacian) with second-order centred differences; the sizes and coefficients are those of
the workloads this package is measured on (a 400-point 1D Laplacian, a 512 x 512 ADR Jacobian, a
1024 x 1024 two-species Gray-Scott Jacobian, batches of 3D diffusion-reaction operators and a stream
of 3D advection-diffusion-reaction requests).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "laplacian_1d_csr", "smooth_field", "adr2d", "gray_scott2d", "adr3d", "op_size",
    "problem_lap1d", "problem_adr2d", "problem_gray_scott", "batch_3d", "request_stream",
]


@dataclass
class Problem:
    """One phi-combination problem: w = sum_k tau^k phi_k(tau A) b_k."""
    name: str
    op: dict
    b: np.ndarray          # (p+1, N) float64, natural order b_0..b_p
    tau: float
    tol: float
    m_init: int = 10
    m_o: int = 2
    precision: str = "fp64"  # "fp64" or "fp32_basis"
    meta: dict = field(default_factory=dict)

    @property
    def p(self) -> int:
        return self.b.shape[0] - 1

    @property
    def n(self) -> int:
        return op_size(self.op)


def op_size(op: dict) -> int:
    k = op["kind"]
    if k in ("csr", "dense"):
        return int(op["n"])
    if k == "stencil2d":
        return int(op["nx"] * op["ny"] * op["nspecies"])
    if k == "stencil3d":
        return int(op["nx"] * op["ny"] * op["nz"])
    raise ValueError(k)


def laplacian_1d_csr(n: int, coeff: float = 1.0) -> dict:
    """coeff * (1/h^2) tridiag(1, -2, 1) on n interior points, Dirichlet, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    s = coeff / (h * h)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        for c, v in ((i - 1, s), (i, -2.0 * s), (i + 1, s)):
            if 0 <= c < n:
                cols.append(c)
                vals.append(v)
        rowptr[i + 1] = len(cols)
    return {"kind": "csr", "n": n, "rowptr": rowptr, "colind": np.asarray(cols, dtype=np.int32),
            "vals": np.asarray(vals, dtype=np.float64)}


def smooth_field(rng: np.random.Generator, nx: int, ny: int, periodic: bool) -> np.ndarray:
    """u = 1/2 + 1/2 S / max|S| with S = sum_{i=1..4} c_i sin(2pi(k_i x + a_i)) cos(2pi(l_i y + b_i)).

    Values lie in [0, 1]; x-fastest, length nx*ny.  Grid points are x = (i+1) h (Dirichlet, h = 1/(n+1))
    or x = i h (periodic, h = 1/n).
    """
    c = rng.uniform(0.5, 1.0, 4)
    k = rng.integers(1, 4, 4)
    l_ = rng.integers(1, 4, 4)
    a = rng.uniform(0.0, 1.0, 4)
    b = rng.uniform(0.0, 1.0, 4)
    if periodic:
        x = np.arange(nx) / nx
        y = np.arange(ny) / ny
    else:
        x = (np.arange(nx) + 1.0) / (nx + 1)
        y = (np.arange(ny) + 1.0) / (ny + 1)
    X, Y = np.meshgrid(x, y, indexing="xy")  # shape (ny, nx): row = y, column = x
    S = np.zeros_like(X)
    for i in range(4):
        S += c[i] * np.sin(2 * np.pi * (k[i] * X + a[i])) * np.cos(2 * np.pi * (l_[i] * Y + b[i]))
    u = 0.5 + 0.5 * S / np.max(np.abs(S))
    return np.ascontiguousarray(u.reshape(-1))


def adr2d(n: int, rng: np.random.Generator, eps: float = 0.01, alpha: float = -10.0,
          gamma: float = 100.0) -> dict:
    """Jacobian eps*Lap_h - alpha*(Dx + Dy) + gamma*diag(1 - 2 u0) of the 2D ADR problem (section 4),
    n x n interior points, homogeneous Dirichlet, h = 1/(n+1), centred differences; u0 a smooth
    seeded field in [0, 1]."""
    h = 1.0 / (n + 1)
    d = eps / (h * h)
    a = alpha / (2.0 * h)
    coef = [[-4.0 * d, d + a, d - a, d + a, d - a]]
    u0 = smooth_field(rng, n, n, periodic=False)
    return {"kind": "stencil2d", "nx": n, "ny": n, "nspecies": 1, "periodic": False,
            "coef": np.asarray(coef, dtype=np.float64), "diag": {(0, 0): gamma * (1.0 - 2.0 * u0)},
            "u0": u0}


def gray_scott2d(n: int, rng: np.random.Generator, du: float = 2e-5, dv: float = 1e-5,
                 F: float = 0.04, k: float = 0.06) -> dict:
    """Jacobian of the 2D Gray-Scott system (section 4) linearised at smooth seeded (u0, v0) in [0, 1]:
    [[du Lap - diag(v0^2 + F), -diag(2 u0 v0)], [diag(v0^2), dv Lap + diag(2 u0 v0 - (F + k))]],
    periodic n x n grid, h = 1/n, unknowns [u; v]."""
    h = 1.0 / n
    cu, cv = du / (h * h), dv / (h * h)
    u0 = smooth_field(rng, n, n, periodic=True)
    v0 = smooth_field(rng, n, n, periodic=True)
    coef = [[-4.0 * cu, cu, cu, cu, cu], [-4.0 * cv, cv, cv, cv, cv]]
    diag = {(0, 0): -(v0 * v0 + F), (0, 1): -2.0 * u0 * v0, (1, 0): v0 * v0,
            (1, 1): 2.0 * u0 * v0 - (F + k)}
    # the same block from the two fields v0^2 and 2 u0 v0 that its entries share: entry (r, c) =
    # const + weight * field (weights +-1, so each entry equals the one above exactly)
    shared = {"fields": [v0 * v0, 2.0 * u0 * v0],
              "entries": {(0, 0): (0, -F, -1.0), (0, 1): (1, 0.0, -1.0), (1, 0): (0, 0.0, 1.0),
                          (1, 1): (1, -(F + k), 1.0)}}
    return {"kind": "stencil2d", "nx": n, "ny": n, "nspecies": 2, "periodic": True,
            "coef": np.asarray(coef, dtype=np.float64), "diag": diag, "shared_fields": shared, "u0": u0, "v0": v0}


def adr3d(n: int, shift: float, adv=(0.0, 0.0, 0.0), diff: float = 1.0) -> dict:
    """diff*Lap_h + sum_d adv_d D_d + shift*I on an n^3 interior grid, Dirichlet, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    d = diff / (h * h)
    coef = [-6.0 * d + shift]
    for ad in adv:
        a = ad / (2.0 * h)
        coef += [d - a, d + a]
    return {"kind": "stencil3d", "nx": n, "ny": n, "nz": n, "periodic": False,
            "coef": np.asarray(coef, dtype=np.float64), "diag": None}


def _normal_b(rng: np.random.Generator, p: int, n: int) -> np.ndarray:
    return np.ascontiguousarray(rng.standard_normal((p + 1, n)))


def problem_lap1d(n: int = 400, seed: int = 1001) -> Problem:
    """1D diffusion Jacobian, 3-point Laplacian, CSR, p = 2, tau = 1e-3, tol = 1e-8."""
    rng = np.random.default_rng(seed)
    op = laplacian_1d_csr(n)
    return Problem(f"lap1d_csr_n{n}", op, _normal_b(rng, 2, n), 1e-3, 1e-8)


def problem_adr2d(n: int = 512, seed: int = 1002, p: int = 4, tau: float = 1e-2, tol: float = 1e-8) -> Problem:
    """Matrix-free 2D ADR Jacobian (5-point), eps = 0.01, alpha = -10, gamma = 100, p = 4, tau = 1e-2."""
    rng = np.random.default_rng(seed)
    op = adr2d(n, rng)
    return Problem(f"adr2d_n{n}", op, _normal_b(rng, p, n * n), tau, tol)


def problem_gray_scott(n: int = 1024, seed: int = 1003, p: int = 3, tau: float = 1.0, tol: float = 1e-6,
                       precision: str = "fp32_basis") -> Problem:
    """Two-species Gray-Scott Jacobian, periodic n x n, p = 3, tau = 1, tol = 1e-6, FP32 basis."""
    rng = np.random.default_rng(seed)
    op = gray_scott2d(n, rng)
    return Problem(f"gray_scott_n{n}", op, _normal_b(rng, p, 2 * n * n), tau, tol, precision=precision)


def batch_3d(count: int = 256, seed: int = 1004, n_range=(10, 40)) -> list[Problem]:
    """Independent 3D 7-point diffusion-reaction instances: n ~ U{n_range}, shift ~ U[-50, 0],
    p ~ U{1..4}, tau log-uniform in [1e-4, 1e-1], tol = 1e-8; instance i uses seed + i."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        shift = float(rng.uniform(-50.0, 0.0))
        p = int(rng.integers(1, 5))
        tau = float(10.0 ** rng.uniform(-4.0, -1.0))
        op = adr3d(n, shift)
        out.append(Problem(f"dr3d_{i}_n{n}", op, _normal_b(rng, p, n ** 3), tau, 1e-8,
                           meta={"shift": shift, "n": n}))
    return out


def request_stream(count: int, seed: int = 1005, rate: float = 2000.0, n_range=(16, 160)) -> list[tuple[float, Problem]]:
    """Poisson arrivals (mean `rate` per second) of 3D 7-point advection-diffusion-reaction solves:
    n ~ U{n_range}, advection ~ U[-10, 10]^3, shift ~ U[-50, 0], p ~ U{0..4}, tau log-uniform in
    [1e-4, 1], tol 1e-6 with an FP32 basis or 1e-10 in FP64 with probability 1/2 each."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        adv = tuple(float(x) for x in rng.uniform(-10.0, 10.0, 3))
        shift = float(rng.uniform(-50.0, 0.0))
        p = int(rng.integers(0, 5))
        tau = float(10.0 ** rng.uniform(-4.0, 0.0))
        mixed = bool(rng.integers(0, 2))
        sub = np.random.default_rng(seed * 7919 + i)
        op = adr3d(n, shift, adv)
        prob = Problem(f"req{i}_n{n}", op, _normal_b(sub, p, n ** 3), tau, 1e-6 if mixed else 1e-10,
                       precision="fp32_basis" if mixed else "fp64", meta={"n": n, "adv": adv, "shift": shift})
        out.append((t, prob))
    return out


# ---------------------------------------------------------------- nonlinear test problems (section 4)
def pde_adr2d(n: int, eps: float = 0.01, alpha: float = -10.0, gamma: float = 100.0) -> dict:
    """The 2D advection-diffusion-reaction problem of section 4, u_t = eps Lap u - alpha (u_x + u_y) +
    gamma u (u - 1/2)(1 - u) on [0,1]^2 with homogeneous Neumann boundaries, on an n x n vertex grid
    that includes the boundary (spacing 1/(n-1))."""
    return {"pde": "adr2d", "n": n, "ns": 1, "bc": "neumann", "dx": 1.0 / (n - 1),
            "eps": eps, "alpha": alpha, "gamma": gamma}


def pde_gray_scott2d(n: int, du: float = 0.2, dv: float = 0.1, a: float = 0.04, b: float = 0.06) -> dict:
    """The 2D Gray-Scott problem of section 4, u_t = d_u Lap u - u v^2 + a (1 - u), v_t = d_v Lap v +
    u v^2 - (a + b) v, on the periodic unit square with the n x n grid x = i/n."""
    return {"pde": "gray_scott2d", "n": n, "ns": 2, "bc": "periodic", "dx": 1.0 / n,
            "du": du, "dv": dv, "a": a, "b": b}


def pde_initial_condition(pde: dict) -> np.ndarray:
    """Initial data of section 4 (species-blocked, x fastest): ADR u = 256 (x y (1-x)(1-y))^2 + 0.3;
    Gray-Scott u = 1 - exp(-150 ((x-1/2)^2 + (y-1/2)^2)), v = exp(-150 ((x-1/2)^2 + 2 (y-1/2)^2))."""
    n = pde["n"]
    x = np.arange(n) * pde["dx"]
    X, Y = np.meshgrid(x, x, indexing="xy")  # X[iy, ix] = x_ix
    if pde["pde"] == "adr2d":
        return (256.0 * (X * Y * (1 - X) * (1 - Y)) ** 2 + 0.3).ravel()
    u = 1.0 - np.exp(-150.0 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))
    v = np.exp(-150.0 * ((X - 0.5) ** 2 + 2.0 * (Y - 0.5) ** 2))
    return np.concatenate([u.ravel(), v.ravel()])
