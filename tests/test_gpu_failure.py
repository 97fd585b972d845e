"""Failure detection on the GPU without a fault: a bounded device-side wait is made to run out (a barrier
arrival that never comes), the kernel returns a timeout status that the host reads, and the context keeps
working afterwards."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1804_05126_gb300 import kiops, workloads as W  # noqa: E402


def test_barrier_wait_times_out_and_the_context_stays_usable():
    from paper_1804_05126_gb300 import build
    build.build()
    s = kiops.Solver(device=0)
    try:
        t0 = time.perf_counter()
        status = kiops.kiops_selftest_wait_timeout(s.ctx, 0.2)
        dt = time.perf_counter() - t0
        assert status == 4, kiops.lib().kiops_last_error(s.ctx)          # KIOPS_ETIMEOUT
        assert b"exceeded" in kiops.lib().kiops_last_error(s.ctx)
        assert 0.15 <= dt <= 5.0
        # the same context solves normally afterwards
        P = W.problem_lap1d()
        op = s.operator(P.op)
        w, st = s.solve(op, P.tau, torch.as_tensor(P.b, device="cuda:0"), P.tol)
        torch.cuda.synchronize()
        w_ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
        w = w.cpu().numpy()
        assert st["status"] == 0 and np.linalg.norm(w - w_ref) <= 10 * P.tol * np.linalg.norm(w_ref)
    finally:
        s.close()


def test_wait_self_test_rejects_bad_limits():
    s = kiops.Solver(device=0)
    try:
        assert kiops.kiops_selftest_wait_timeout(s.ctx, 0.0) == 1
        assert kiops.kiops_selftest_wait_timeout(s.ctx, 60.0) == 1
    finally:
        s.close()
