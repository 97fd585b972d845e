"""Oracle for the exponential integrators of section 4 (test infrastructure only).

Plain, slow, FP64 CPU code.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline use it.  It is independent of the CUDA path: the right-hand sides and Jacobians below are
written from the PDEs of section 4 with numpy, and every phi-combination goes through this package's
KIOPS (``oracle.kiops`` for Task II, ``oracle.kiops_task1`` for Task I).

Schemes (section 4), each in the "mixed" form of section 2: one Task I call for the stage vectors,
then one Task II call (eq 10) for u_{n+1}; EXPRB5s3 needs a second Task I call for its third stage.
With A = h_n J_n and tau = 1 as in eqs 10-11:

* EPIRK4s3, eq 50 (grouping eqs 9-11): stages at 1/8 and 1/9; b_3 = h(1892 r2 + 1458 (r3 - 2 r2)),
  b_4 = h(-42336 r2 - 34992 (r3 - 2 r2)).
* EPIRK4s3A, eq 51: stages at 1/2 and 2/3; b_3 = h(32 r2 - 27/2 r3), b_4 = h(-144 r2 + 81 r3).
* EXPRB5s3, eq 53: stages at 1/2 and 9/10, the third stage adds (27/25 phi_3(A/2) + 729/125
  phi_3(9A/10)) h r2; b_3 = h(18 r2 - 250/81 r3), b_4 = h(-60 r2 + 500/27 r3).

r(U) = f(U) - f(u_n) - J_n (U - u_n) is the remainder defined below eq 2, computed literally.

Test problems (section 4): 2D advection-diffusion-reaction on [0,1]^2 with homogeneous Neumann
boundaries, u_t = eps Lap u - alpha (u_x + u_y) + gamma u (u - 1/2)(1 - u), eps = 1/100, alpha = -10,
gamma = 100, u(0) = 256 (x y (1-x)(1-y))^2 + 0.3; and 2D Gray-Scott on the periodic unit square,
u_t = d_u Lap u - u v^2 + a (1 - u), v_t = d_v Lap v + u v^2 - (a + b) v, d_u = 0.2, d_v = 0.1,
a = 0.04, b = 0.06, with the paper's Gaussian initial data.  Second-order centred differences; the
Neumann grid has n points per dimension including the boundary (spacing 1/(n-1), ghost values
mirrored), the periodic grid n points at x = i/n.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1804_05126_gb300 import workloads as WL

SCHEMES = ("epirk4s3", "epirk4s3a", "exprb5s3")


# ----------------------------------------------------------------------------------- test problems
# The problem descriptions and initial data are inputs, shared with the CUDA path's callers.
adr2d = WL.pde_adr2d
gray_scott2d = WL.pde_gray_scott2d
initial_condition = WL.pde_initial_condition


def _neighbours(pde: dict, z: np.ndarray):
    """West, east, south, north neighbour values of an n x n field under the problem's boundary."""
    if pde["bc"] == "periodic":
        return (np.roll(z, 1, axis=1), np.roll(z, -1, axis=1), np.roll(z, 1, axis=0), np.roll(z, -1, axis=0))
    zp = np.pad(z, 1, mode="reflect")  # ghost value = the value one point inside (x(-1) = x(1))
    return zp[1:-1, :-2], zp[1:-1, 2:], zp[:-2, 1:-1], zp[2:, 1:-1]


def linear_part(pde: dict, u: np.ndarray) -> np.ndarray:
    """L u: diffusion (and advection for ADR) with second-order centred differences."""
    n, dx = pde["n"], pde["dx"]
    out = []
    for s in range(pde["ns"]):
        z = u[s * n * n:(s + 1) * n * n].reshape(n, n)
        w, e, so, no = _neighbours(pde, z)
        lap = (w + e + so + no - 4.0 * z) / dx ** 2
        if pde["pde"] == "adr2d":
            adv = ((e - w) + (no - so)) / (2.0 * dx)
            out.append(pde["eps"] * lap - pde["alpha"] * adv)
        else:
            out.append((pde["du"] if s == 0 else pde["dv"]) * lap)
    return np.concatenate([o.ravel() for o in out])


def reaction(pde: dict, u: np.ndarray) -> np.ndarray:
    """The pointwise nonlinear part R(u) of f(u) = L u + R(u)."""
    if pde["pde"] == "adr2d":
        return pde["gamma"] * u * (u - 0.5) * (1.0 - u)
    m = pde["n"] ** 2
    uu, vv = u[:m], u[m:]
    return np.concatenate([-uu * vv ** 2 + pde["a"] * (1.0 - uu), uu * vv ** 2 - (pde["a"] + pde["b"]) * vv])


def reaction_jacobian(pde: dict, u: np.ndarray) -> dict:
    """Pointwise blocks dR_r/du_c as {(r, c): field}."""
    if pde["pde"] == "adr2d":
        return {(0, 0): pde["gamma"] * (-3.0 * u ** 2 + 3.0 * u - 0.5)}
    m = pde["n"] ** 2
    uu, vv = u[:m], u[m:]
    return {(0, 0): -vv ** 2 - pde["a"], (0, 1): -2.0 * uu * vv,
            (1, 0): vv ** 2, (1, 1): 2.0 * uu * vv - (pde["a"] + pde["b"])}


def rhs(pde: dict, u: np.ndarray) -> np.ndarray:
    """f(u) of the semi-discrete system (eq 1)."""
    return linear_part(pde, u) + reaction(pde, u)


def stencil_coefficients(pde: dict) -> list:
    """Centre, -x, +x, -y, +y coefficients of L for each species."""
    dx = pde["dx"]
    if pde["pde"] == "adr2d":
        d, a = pde["eps"] / dx ** 2, pde["alpha"] / (2.0 * dx)
        return [[-4.0 * d, d + a, d - a, d + a, d - a]]
    return [[-4.0 * k / dx ** 2] + [k / dx ** 2] * 4 for k in (pde["du"], pde["dv"])]


def jacobian_op(pde: dict, u: np.ndarray, scale: float = 1.0) -> dict:
    """scale * J(u) as a stencil operator description (J = L + dR/du)."""
    coef = [[scale * c for c in row] for row in stencil_coefficients(pde)]
    diag = {k: scale * v for k, v in reaction_jacobian(pde, u).items()}
    return {"kind": "stencil2d", "nx": pde["n"], "ny": pde["n"], "nspecies": pde["ns"], "bc": pde["bc"],
            "coef": coef, "diag": diag}


def remainder(pde: dict, U: np.ndarray, un: np.ndarray, fn: np.ndarray, Jn: dict) -> np.ndarray:
    """r(U) = f(U) - f(u_n) - J_n (U - u_n) (section 2, below eq 2)."""
    return rhs(pde, U) - fn - oracle.apply(Jn, U - un)


# --------------------------------------------------------------------------------------- schemes
def _scheme(name: str) -> dict:
    """Stage nodes and the b_3, b_4 weights of r2 and r3 (eqs 50, 51, 53, grouped as in eq 11)."""
    if name == "epirk4s3":
        # b_3 = 1892 r2 + 1458 (r3 - 2 r2), b_4 = -42336 r2 - 34992 (r3 - 2 r2)
        return {"c2": 1.0 / 8.0, "c3": 1.0 / 9.0, "b3": lambda r2, r3: 1892.0 * r2 + 1458.0 * (r3 - 2.0 * r2),
                "b4": lambda r2, r3: -42336.0 * r2 - 34992.0 * (r3 - 2.0 * r2)}
    if name == "epirk4s3a":
        return {"c2": 0.5, "c3": 2.0 / 3.0, "b3": lambda r2, r3: 32.0 * r2 - 13.5 * r3,
                "b4": lambda r2, r3: -144.0 * r2 + 81.0 * r3}
    if name == "exprb5s3":
        return {"c2": 0.5, "c3": 0.9, "b3": lambda r2, r3: 18.0 * r2 - (250.0 / 81.0) * r3,
                "b4": lambda r2, r3: -60.0 * r2 + (500.0 / 27.0) * r3}
    raise ValueError(name)


def step(pde: dict, scheme: str, un: np.ndarray, h: float, tol: float, m_init: list, stats: dict) -> np.ndarray:
    """One step u_n -> u_{n+1} of the scheme.  m_init holds, per KIOPS call of the step, the Krylov
    dimension to start from; it is overwritten with the calls' final m (section 3.6: the last m of the
    previous time step is the first guess of the next)."""
    sc = _scheme(scheme)
    N = un.size
    fn = rhs(pde, un)
    A = jacobian_op(pde, un, scale=h)           # A = h_n J_n, tau = 1 (eq 10)
    Jn = jacobian_op(pde, un)
    zero = np.zeros(N)

    def call(kind, T, b, slot):
        if kind == 1:
            out, st = oracle.kiops_task1(A, T, b, tol, m_init=m_init[slot])
        else:
            out, st = oracle.kiops(A, T, b, tol, m_init=m_init[slot])[:2]
        if st["status"] != 0:
            raise RuntimeError(f"oracle KIOPS failed in {scheme} call {slot}: status {st['status']}")
        m_init[slot] = st["m_last"]
        stats["kiops_calls"] += 1
        stats["matvecs"] += st["matvecs"]
        stats["substeps"] += st["substeps"]
        stats["rejected"] += st["rejected"]
        return out

    # first call, Task I: phi_1(c A) h f(u_n) at both stage nodes (scaled by 1/c, Algorithm 3)
    nodes = sorted([sc["c2"], sc["c3"]])
    W = call(1, nodes, np.stack([zero, h * fn]), 0)
    Wc = {c: W[i] for i, c in enumerate(nodes)}
    U2 = un + sc["c2"] * Wc[sc["c2"]]
    U3 = un + sc["c3"] * Wc[sc["c3"]]
    r2 = remainder(pde, U2, un, fn, Jn)
    if scheme == "exprb5s3":
        # second call, Task I: phi_3(c A) h r(U_n2) at c = 1/2 and 9/10 (scaled by 1/c^3)
        Z = call(1, nodes, np.stack([zero, zero, zero, h * r2]), 1)
        U3 = U3 + (27.0 / 25.0) * Z[0] + (729.0 / 125.0) * Z[1]
    r3 = remainder(pde, U3, un, fn, Jn)
    b = np.stack([zero, h * fn, zero, h * sc["b3"](r2, r3), h * sc["b4"](r2, r3)])
    w = call(2, 1.0, b, 2)  # Task II, eq 10 with tau = 1
    return un + w


def integrate(pde: dict, scheme: str, u0: np.ndarray, t0: float, t1: float, nsteps: int, tol: float,
              m_init: int = 10):
    """Constant-step integration (section 4) from t0 to t1 in nsteps steps; returns (u, stats)."""
    h = (t1 - t0) / nsteps
    u = np.array(u0, dtype=np.float64)
    stats = {"steps": 0, "kiops_calls": 0, "matvecs": 0, "substeps": 0, "rejected": 0}
    minit = [m_init, m_init, m_init]
    for _ in range(nsteps):
        u = step(pde, scheme, u, h, tol, minit, stats)
        stats["steps"] += 1
    return u, stats
