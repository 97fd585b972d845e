"""Batch team engine on the GPU: parity with the oracle for every team size, bitwise equality of a request
alone and in the mix (fixed team size), and the autotuner."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_1804_05126_gb300 import kiops, tune, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def solver():
    from paper_1804_05126_gb300 import build
    build.build()
    s = kiops.Solver(device=0)
    yield s
    s.close()


def make_items(solver, probs, precision="fp64"):
    items = []
    for P in probs:
        op = solver.operator(P.op)
        b = torch.as_tensor(P.b, device="cuda:0")
        w = torch.full((P.n,), float("nan"), dtype=torch.float64, device="cuda:0")
        items.append((op, P.tau, b, P.tol, P.m_init, P.m_o, precision, w))
    return items


@pytest.mark.parametrize("team_blocks", [1, 2, 8, 0])
def test_team_engine_matches_oracle(solver, team_blocks):
    probs = W.batch_3d(count=12, seed=301, n_range=(6, 14))
    items = make_items(solver, probs)
    stats = solver.solve_batch(items, team_blocks=team_blocks)
    torch.cuda.synchronize()
    for P, it, st in zip(probs, items, stats):
        w_ref, st_ref, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
        w = it[7].cpu().numpy()
        assert st["status"] == 0
        assert np.linalg.norm(w - w_ref) <= 10 * P.tol * np.linalg.norm(w_ref)


def test_full_batch_sample_vs_oracle(solver):
    """The 256-instance 3D batch (n in 10..40) in one team-engine launch; every 16th instance checked
    against the oracle, every instance against its own single-request solve."""
    probs = W.batch_3d()
    items = make_items(solver, probs)
    stats = solver.solve_batch(items, team_blocks=0)
    torch.cuda.synchronize()
    for i in range(0, len(probs), 16):
        P = probs[i]
        w_ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
        w = items[i][7].cpu().numpy()
        assert np.linalg.norm(w - w_ref) <= 10 * P.tol * np.linalg.norm(w_ref), i
    assert all(st["status"] == 0 for st in stats)


def test_request_alone_equals_request_in_the_mix(solver):
    probs = W.batch_3d(count=20, seed=401, n_range=(8, 24))
    items = make_items(solver, probs)
    solver.solve_batch(items, team_blocks=4)
    mixed = [it[7].clone() for it in items]
    for k in (0, 7, 19):
        alone = make_items(solver, [probs[k]])
        solver.solve_batch(alone, team_blocks=4)
        torch.cuda.synchronize()
        assert torch.equal(alone[0][7], mixed[k]), k


def test_autotuner_picks_a_candidate(solver):
    probs = W.batch_3d(count=16, seed=501, n_range=(8, 20))
    items = make_items(solver, probs)
    best, timings = tune.tune_batch(solver, items, candidates=(1, 4, 16))
    assert best in (1, 4, 16) and timings[best] == min(timings.values())
    assert tune.cached_team_blocks(items) == best


@pytest.mark.parametrize("team_blocks", [2, 3])
def test_team_engine_2d_grids_with_several_tiles_per_block(solver, team_blocks):
    """2D stencil requests in the team engine with teams of 2 or 3 blocks: grids of 1.4-3 x 10^4 unknowns
    need several tiles per block, which each team takes in turn (Dirichlet ADR in FP64, periodic two-species
    Gray-Scott in FP64 and with the FP32 basis, mixed in one launch); every result within 10 tol of the
    oracle."""
    probs = [W.problem_adr2d(n=150, seed=41), W.problem_adr2d(n=121, seed=42, p=2),
             W.problem_gray_scott(n=97, seed=43, precision="fp64", tol=1e-8, tau=1.0),
             W.problem_gray_scott(n=128, seed=44, precision="fp32_basis", tol=1e-6, tau=1.0)]
    items = []
    for P in probs:
        items += make_items(solver, [P], precision=P.precision)
    stats = solver.solve_batch(items, team_blocks=team_blocks)
    torch.cuda.synchronize()
    for P, it, st in zip(probs, items, stats):
        w_ref, _, _ = oracle.kiops(P.op, P.tau, P.b, P.tol)
        w = it[7].cpu().numpy()
        assert st["status"] == 0
        assert np.linalg.norm(w - w_ref) <= 10 * P.tol * np.linalg.norm(w_ref), P.name
