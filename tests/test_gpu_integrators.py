"""GPU parity for the exponential integrators (section 4) and the Neumann stencil, through the C ABI,
against the CPU oracle on the same seeded inputs.

Bars: f(u) and operator products to rounding (relative 1e-13); a KIOPS solve within 10 tol with the
same decisions; integrations within 1e-8 relative of the oracle with each solve at tol = 1e-10 (the
remainders r(U) are computed in different but equivalent forms on the two sides, so the b vectors of
the solves agree to rounding, not bit for bit).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import integrators as I  # noqa: E402
from paper_1804_05126_gb300 import kiops  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def solver():
    from paper_1804_05126_gb300 import build
    build.build()
    s = kiops.Solver(device=0)
    yield s
    s.close()


def _state(pde, seed):
    rng = np.random.default_rng(seed)
    return I.initial_condition(pde) + 0.05 * rng.standard_normal(pde["ns"] * pde["n"] ** 2)


@pytest.mark.parametrize("make", [lambda: I.adr2d(33), lambda: I.adr2d(2), lambda: I.gray_scott2d(32),
                                  lambda: I.gray_scott2d(3)])
def test_rhs_matches_oracle(solver, make):
    pde = make()
    u = _state(pde, 11)
    f = solver.pde_rhs(pde, torch.as_tensor(u, device="cuda:0")).cpu().numpy()
    ref = I.rhs(pde, u)
    assert rel(f, ref) <= 1e-13


@pytest.mark.parametrize("fuse", [True, False])
@pytest.mark.parametrize("n", [5, 61, 200])
def test_neumann_stencil_apply_and_solve(solver, n, fuse):
    """The reflected boundary in every stencil path: operator product and a full adaptive solve (the
    tiled path finalises its halo through the same reflection)."""
    pde = I.adr2d(n)
    u = _state(pde, 12)
    op = I.jacobian_op(pde, u, scale=1e-3)
    s = kiops.Solver(device=0, fuse_stencil=fuse)
    try:
        A = s.operator(op)
        x = np.random.default_rng(13).standard_normal(n * n)
        y = A.apply(torch.as_tensor(x, device="cuda:0")).cpu().numpy()
        assert rel(y, oracle.apply(op, x)) <= 1e-13
        b = np.random.default_rng(14).standard_normal((3, n * n))
        tol = 1e-9
        w, st, tr = s.solve(A, 1.0, torch.as_tensor(b, device="cuda:0"), tol, trace=True)
        torch.cuda.synchronize()
        w_ref, st_ref, tr_ref = oracle.kiops(op, 1.0, b, tol)
        assert st["status"] == 0 and rel(w.cpu().numpy(), w_ref) <= 10 * tol
        assert [(t["j"], t["accepted"]) for t in tr] == [(t["j"], t["accepted"]) for t in tr_ref]
    finally:
        s.close()


CASES = [(lambda: I.adr2d(24), 0.0, 0.01, 4), (lambda: I.gray_scott2d(20), 0.0, 0.05, 4)]


@pytest.mark.parametrize("scheme", I.SCHEMES)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_integrators_match_oracle(solver, scheme, case):
    make, t0, t1, nsteps = CASES[case]
    pde = make()
    u0 = I.initial_condition(pde)
    tol = 1e-10
    ref, st_ref = I.integrate(pde, scheme, u0, t0, t1, nsteps, tol)
    u = torch.as_tensor(u0, device="cuda:0").clone()
    st = solver.integrate(pde, scheme, u, t0, t1, nsteps, tol)
    got = u.cpu().numpy()
    assert st["steps"] == nsteps and st["kiops_calls"] == st_ref["kiops_calls"]
    assert rel(got, ref) <= 1e-8, rel(got, ref)
    assert abs(st["matvecs"] - st_ref["matvecs"]) <= 0.1 * st_ref["matvecs"]


def test_integrator_full_size_adr_400(solver):
    """The paper's ADR grid (400 x 400) for two EPIRK4s3A steps of h = 0.0025 against the oracle."""
    pde = I.adr2d(400)
    u0 = I.initial_condition(pde)
    tol = 1e-10
    ref, st_ref = I.integrate(pde, "epirk4s3a", u0, 0.0, 0.005, 2, tol)
    u = torch.as_tensor(u0, device="cuda:0").clone()
    st = solver.integrate(pde, "epirk4s3a", u, 0.0, 0.005, 2, tol)
    err = rel(u.cpu().numpy(), ref)
    print(f"ADR 400^2 EPIRK4s3A, 2 steps: rel diff {err:.2e}, matvecs {st['matvecs']} (oracle {st_ref['matvecs']})")
    assert err <= 1e-8


def test_integrate_rejects_bad_arguments(solver):
    u = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kiops.KiopsError):
        solver.integrate(I.adr2d(4), "epirk4s3", u, 1.0, 0.5, 2)   # t1 < t0
    with pytest.raises(kiops.KiopsError):
        solver.integrate(I.adr2d(4), "epirk4s3", u, 0.0, 1.0, 0)   # no steps
    with pytest.raises(kiops.KiopsError):
        solver.integrate(dict(I.adr2d(4), n=1), "epirk4s3", u, 0.0, 1.0, 1)
