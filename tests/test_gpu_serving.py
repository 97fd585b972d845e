"""Continuous-batching server on the GPU: results alone and in the mix, admission under a budget, a
served stream checked against the oracle, recovery after a device-side wait gave up."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1804_05126_gb300 import kiops, serve, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def solver():
    from paper_1804_05126_gb300 import build
    build.build()
    s = kiops.Solver(device=0)
    s.server_start(hbm_budget_bytes=4e9, small_team_blocks=8, large_teams=1, large_team_blocks=64,
                   large_work_threshold=5e7)
    yield s
    s.server_stop()
    s.close()


def small_stream(count=24, seed=1005, n_range=(16, 32), rate=2000.0, tau_max=0.02):
    """The serving workload's request mix on small grids (tau capped so that the oracle stays fast)."""
    out = W.request_stream(count, seed=seed, rate=rate, n_range=n_range)
    for _, P in out:
        P.tau = min(P.tau, tau_max)
    return out


def test_served_stream_matches_oracle(solver):
    stream = small_stream(count=12)
    res = serve.run_stream(solver, stream)
    for (t, P), w, st in zip(stream, res["w"], res["stats"]):
        ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
        err = np.linalg.norm(w.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert st["status"] == 0
        assert err <= 10 * P.tol, (P.name, P.precision, err)
    assert res["p99_ms"] >= res["p50_ms"] > 0


def test_result_alone_equals_result_in_the_mix(solver):
    stream = small_stream(count=30, seed=77)
    mix = serve.run_stream(solver, stream)
    for k in (0, 11, 29):
        t, P = stream[k]
        alone = serve.run_stream(solver, [(0.0, P)])
        assert torch.equal(alone["w"][0], mix["w"][k]), k


def test_admission_waits_for_budget():
    """A budget that holds about one request at a time still completes a burst (requests queue on the
    host and are admitted as workspaces free up)."""
    s = kiops.Solver(device=0)
    stream = small_stream(count=6, seed=5, n_range=(28, 28))
    P0 = stream[0][1]
    need = (128 + 1) * (P0.n + 64) * 8 * 1.5
    s.server_start(hbm_budget_bytes=need, small_team_blocks=8, large_teams=0)
    res = serve.run_stream(s, [(0.0, P) for _, P in stream])
    for (_, P), w in zip(stream, res["w"]):
        ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
        assert np.linalg.norm(w.cpu().numpy() - ref) <= 10 * P.tol * np.linalg.norm(ref)
    s.server_stop()
    s.close()


def test_large_class_request(solver):
    """A request above the large-work threshold runs on the large team."""
    P = W.request_stream(1, seed=9, n_range=(64, 64))[0][1]
    P.tau = 0.01
    res = serve.run_stream(solver, [(0.0, P)])
    ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
    assert np.linalg.norm(res["w"][0].cpu().numpy() - ref) <= 10 * P.tol * np.linalg.norm(ref)


def test_server_recovers_after_an_abort():
    """The abort word a device-side wait raises when it gives up (here raised from the host, no GPU fault):
    the request the server had claimed reports KIOPS_ETIMEOUT instead of never finishing, and the next
    launch clears the word and serves a later request correctly."""
    s = kiops.Solver(device=0)
    s.server_start(hbm_budget_bytes=4e9, small_team_blocks=8, large_teams=0)
    P = W.problem_adr2d(n=512, seed=3)
    op = s.operator(P.op)
    b = torch.as_tensor(P.b, device="cuda:0")
    t, _ = s.submit(op, 0.1, b, P.tol)  # 1664 matvecs: far longer than the claim, on one team of 8 blocks
    t0 = time.time()
    while s.server_info()["claimed_small"] < 1:  # a team has taken the request
        assert time.time() - t0 < 30, "the request was never claimed"
        time.sleep(0.001)
    kiops.kiops_server_selftest_abort(s.ctx)
    with pytest.raises(kiops.KiopsError) as e:
        t0 = time.time()
        while not s.poll(t, 1.0)[0]:
            assert time.time() - t0 < 60, "the claimed request never finished"
    assert e.value.status == 4
    assert s.server_info()["in_flight"] == 0
    _, P2 = small_stream(count=1, seed=21)[0]
    res = serve.run_stream(s, [(0.0, P2)])
    ref, _, _ = oracle.kiops(P2.op, P2.tau, P2.b, P2.tol)
    assert res["stats"][0]["status"] == 0
    assert np.linalg.norm(res["w"][0].cpu().numpy() - ref) <= 10 * P2.tol * np.linalg.norm(ref)
    s.server_stop()
    s.close()


def test_large_requests_run_alone_between_launches():
    """Requests with at least solo_min_unknowns unknowns run alone on the whole GPU between launches of the
    server kernel (the server drains, runs them, resumes): in a mix with smaller requests each of them equals
    kiops_solve of the same request bit for bit (same kernel and grid), and the smaller ones match the oracle."""
    s = kiops.Solver(device=0)
    s.server_start(hbm_budget_bytes=4e9, solo_min_unknowns=30000)
    stream = small_stream(count=10, seed=31, n_range=(16, 40))
    big = [P.n >= 30000 for _, P in stream]
    assert any(big) and not all(big)
    res = serve.run_stream(s, stream)
    s.server_stop()
    for ((_, P), w, st), alone in zip(zip(stream, res["w"], res["stats"]), big):
        assert st["status"] == 0
        if alone:
            op = s.operator(P.op)
            w_direct, _ = s.solve(op, P.tau, torch.as_tensor(P.b, device="cuda:0"), P.tol, P.m_init, P.m_o,
                                  precision=P.precision)
            assert torch.equal(w, w_direct), P.name
        else:
            ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
            assert np.linalg.norm(w.cpu().numpy() - ref) <= 10 * P.tol * np.linalg.norm(ref), P.name
    s.close()
