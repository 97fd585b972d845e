"""Pins for the oracle's exponential integrators (section 4) and its Neumann stencil, against facts that do
not come from the oracle: convergence orders against scipy's Radau integrator, exactness on a linear
problem against scipy's expm, the Jacobian against central differences of f, and the closed-form
spectrum of the reflected second difference."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm as scipy_expm

import oracle
from oracle import integrators as I


def _dense_jacobian(pde, u):
    return oracle.dense_matrix(I.jacobian_op(pde, u))


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


# ---------------------------------------------------------------- discrete operators
@pytest.mark.parametrize("n", [5, 9, 16])
@pytest.mark.parametrize("k,l", [(0, 0), (1, 0), (2, 3), (4, 1)])
def test_neumann_second_difference_eigenvectors(n, k, l):
    """With reflected ghost points the vertex-grid second difference has the eigenvectors
    cos(k pi x) cos(l pi y), eigenvalue -(4/dx^2)(sin^2(k pi dx/2) + sin^2(l pi dx/2))."""
    if k >= n or l >= n:
        pytest.skip("mode not on the grid")
    dx = 1.0 / (n - 1)
    x = np.arange(n) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    v = (np.cos(k * np.pi * X) * np.cos(l * np.pi * Y)).ravel()
    lam = -(4.0 / dx ** 2) * (np.sin(k * np.pi * dx / 2) ** 2 + np.sin(l * np.pi * dx / 2) ** 2)
    op = {"kind": "stencil2d", "nx": n, "ny": n, "nspecies": 1, "bc": "neumann",
          "coef": [[-4.0 / dx ** 2] + [1.0 / dx ** 2] * 4], "diag": {}}
    y = oracle.apply(op, v)          # the C oracle's stencil with bc = Neumann
    scale = 4.0 / dx ** 2
    assert np.max(np.abs(y - lam * v)) <= 1e-12 * scale
    pde = I.adr2d(n, eps=1.0, alpha=0.0, gamma=0.0)
    assert np.max(np.abs(I.linear_part(pde, v) - lam * v)) <= 1e-12 * scale


@pytest.mark.parametrize("make", [lambda: I.adr2d(7), lambda: I.gray_scott2d(6)])
def test_linear_part_annihilates_constants(make):
    pde = make()
    c = np.full(pde["ns"] * pde["n"] ** 2, 0.37)
    assert np.max(np.abs(I.linear_part(pde, c))) <= 1e-9
    assert np.allclose(I.rhs(pde, c), I.reaction(pde, c), rtol=0, atol=1e-9)


@pytest.mark.parametrize("make", [lambda: I.adr2d(9), lambda: I.gray_scott2d(8)])
def test_jacobian_matches_central_differences_of_f(make):
    """J(u) v against (f(u + d v) - f(u - d v)) / 2d; a dropped term or wrong sign in dR fails."""
    pde = make()
    rng = np.random.default_rng(5)
    u = I.initial_condition(pde) + 0.05 * rng.standard_normal(pde["ns"] * pde["n"] ** 2)
    v = rng.standard_normal(u.size)
    d = 1e-5
    fd = (I.rhs(pde, u + d * v) - I.rhs(pde, u - d * v)) / (2 * d)
    Jv = oracle.apply(I.jacobian_op(pde, u), v)
    assert np.linalg.norm(Jv - fd) <= 1e-7 * np.linalg.norm(fd)


def test_jacobian_op_matches_dense_finite_difference_matrix():
    pde = I.adr2d(5)
    u = I.initial_condition(pde)
    J = _dense_jacobian(pde, u)
    d = 1e-6
    cols = [(I.rhs(pde, u + d * e) - I.rhs(pde, u - d * e)) / (2 * d) for e in np.eye(u.size)]
    assert np.max(np.abs(J - np.stack(cols, axis=1))) <= 1e-5 * np.max(np.abs(J))


def test_remainder_vanishes_at_u_n_and_is_second_order():
    pde = I.gray_scott2d(6)
    rng = np.random.default_rng(8)
    un = I.initial_condition(pde)
    fn, Jn = I.rhs(pde, un), I.jacobian_op(pde, un)
    assert np.max(np.abs(I.remainder(pde, un, un, fn, Jn))) <= 1e-12
    v = rng.standard_normal(un.size)
    r1 = np.linalg.norm(I.remainder(pde, un + 1e-2 * v, un, fn, Jn))
    r2 = np.linalg.norm(I.remainder(pde, un + 5e-3 * v, un, fn, Jn))
    assert 3.5 <= r1 / r2 <= 4.5  # halving the offset quarters a quadratic remainder


# ---------------------------------------------------------------- integrators
@pytest.mark.parametrize("scheme", I.SCHEMES)
def test_linear_problem_is_integrated_exactly(scheme):
    """gamma = 0 makes f linear, so r = 0 and every scheme reduces to u_{n+1} = e^{h L} u_n."""
    pde = I.adr2d(6, gamma=0.0)
    u0 = I.initial_condition(pde)
    L = _dense_jacobian(pde, u0)
    T, ns = 0.02, 3
    u, st = I.integrate(pde, scheme, u0, 0.0, T, ns, 1e-12)
    ref = scipy_expm(T * L) @ u0
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    assert st["kiops_calls"] == ns * (3 if scheme == "exprb5s3" else 2)


@pytest.fixture(scope="module")
def radau_refs():
    out = {}
    for name, pde, T in [("adr", I.adr2d(10), 0.02), ("gs", I.gray_scott2d(8), 0.05)]:
        u0 = I.initial_condition(pde)
        sol = solve_ivp(lambda t, y: I.rhs(pde, y), (0.0, T), u0, method="Radau", rtol=1e-13, atol=1e-13,
                        jac=lambda t, y: _dense_jacobian(pde, y))
        assert sol.success
        out[name] = (pde, T, u0, sol.y[:, -1])
    return out


@pytest.mark.parametrize("name", ["adr", "gs"])
@pytest.mark.parametrize("scheme,order", [("epirk4s3", 4), ("epirk4s3a", 4), ("exprb5s3", 5)])
def test_convergence_order_against_radau(radau_refs, name, scheme, order):
    """Observed order over step halvings against scipy's Radau IIA solution at tight tolerance: a wrong
    coefficient, node or grouping in eqs 50, 51, 53 loses the order."""
    pde, T, u0, ref = radau_refs[name]
    errs = []
    for ns in (4, 8, 16):
        u, _ = I.integrate(pde, scheme, u0, 0.0, T, ns, 1e-13)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() >= order - 0.45, (errs, orders)
    assert errs[-1] <= 1e-5
