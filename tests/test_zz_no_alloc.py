"""The allocation-free entry point kiops_solve_noalloc, checked on the GPU against kiops_solve and the oracle.

Some callers cannot let a library allocate device memory while they run: applications whose device
memory belongs to their own pool or allocator (a hidden cudaMalloc escapes their accounting and
synchronises the device) and hosts that forbid allocation after start-up.  kiops_solve_noalloc serves
them from a fixed device array instead of the context's workspace.  Each case makes two calls in a row
(the array keeps the previous call's contents) and compares both with kiops_solve and with the FP64 CPU
oracle of the method.
This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1804_05126_gb300 import kiops, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def solver():
    from paper_1804_05126_gb300 import build
    build.build()
    s = kiops.Solver(device=0)
    yield s
    s.close()


@pytest.mark.parametrize("make", [lambda: W.problem_lap1d(), lambda: W.problem_adr2d(n=40, seed=3),
                                  lambda: W.batch_3d(count=1, seed=5, n_range=(9, 9))[0]])
def test_noalloc_matches_kiops_solve_on_two_calls_in_a_row(solver, make):
    P = make()
    op = solver.operator(P.op)
    b = torch.as_tensor(P.b, device="cuda:0")
    w_ref, st_ref = solver.solve(op, P.tau, b, P.tol, m_init=P.m_init, m_o=P.m_o)
    ref = w_ref.cpu().numpy()
    w_or, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol, m_init=P.m_init, m_o=P.m_o)
    ptrs = [b[k].data_ptr() for k in range(P.p + 1)]
    for call in range(2):
        w = torch.full((P.n,), float("nan"), dtype=torch.float64, device="cuda:0")
        st = kiops.kiops_solve_noalloc(solver.ctx, op.handle, P.tau, P.p, ptrs, P.tol, P.m_init, P.m_o, w.data_ptr())
        got = w.cpu().numpy()
        assert st["status"] == 0 and st["matvecs"] > 0
        assert np.linalg.norm(got - ref) <= 10 * P.tol * np.linalg.norm(ref), call
        assert np.linalg.norm(got - w_or) <= 10 * P.tol * np.linalg.norm(w_or), call


def test_noalloc_rejects_a_solve_larger_than_its_scratch(solver):
    P = W.problem_lap1d(n=40000)
    op = solver.operator(P.op)
    b = torch.as_tensor(P.b, device="cuda:0")
    w = torch.empty(P.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(kiops.KiopsError) as e:
        kiops.kiops_solve_noalloc(solver.ctx, op.handle, P.tau, P.p, [b[k].data_ptr() for k in range(P.p + 1)],
                                  P.tol, P.m_init, P.m_o, w.data_ptr())
    assert e.value.status == 1 and "bytes" in str(e.value)
