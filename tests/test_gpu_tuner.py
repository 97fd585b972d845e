"""The launch-shape autotuner of single solves on the GPU: it times the candidate tile shapes of the 2D
stencil step (and the per-element path), keeps the fastest, and the tile shapes change the result only
through the order of partial sums."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1804_05126_gb300 import kiops, tune, workloads as W  # noqa: E402


def test_solve_tuner_chooses_among_tile_shapes():
    """2048^2 Gray-Scott with the FP32 basis (several tiles per block, the staged path): four tile shapes and
    the per-element path are timed; re-timed afterwards, the tuner's choice is within 2 % of the fastest
    candidate; the staged candidates agree with one another within the solve's tolerance (they differ in the
    order of partial sums), and the per-element path within 10 tol, the FP32 basis's parity bar (it rounds the
    coupling entries, written in FP64, to FP32, where the staged path forms them in FP32 from Gray-Scott's two
    shared fields, so its rounding errors are not those of the staged runs)."""
    from paper_1804_05126_gb300 import build
    build.build()
    P = W.problem_gray_scott(n=2048)
    s = kiops.Solver(device=0)
    op = s.operator(P.op)
    b = torch.as_tensor(P.b, device="cuda:0")
    best, timings = tune.tune_solve(s, op, P.tau, b, P.tol, precision="fp32_basis", reps=3)
    shapes = {(c["tile_w"], c["tile_h"]) for c in map(json.loads, timings) if c["tma"]}
    assert len(shapes) >= 3 and json.dumps(best, sort_keys=True) in timings
    assert tune.cached_solve_config(op, "fp32_basis", P.p, P.m_o) == best
    again, results = {}, {}
    for key in timings:
        s.configure(**json.loads(key))
        again[key] = tune.time_solve(s, op, P.tau, b, P.tol, precision="fp32_basis", reps=3)
        w, st = s.solve(op, P.tau, b, P.tol, precision="fp32_basis")
        assert st["status"] == 0
        results[key] = w.cpu().numpy()
    assert again[json.dumps(best, sort_keys=True)] <= 1.02 * min(again.values()), (best, again)
    ref = results[json.dumps(best, sort_keys=True)]
    for key, w in results.items():
        bar = P.tol if json.loads(key)["tma"] else 10 * P.tol
        assert np.linalg.norm(w - ref) <= bar * np.linalg.norm(ref), key
    s.close()
