"""CPU checks of the benchmark's work models against values worked out by hand: the algorithmic bytes of one
Krylov step on grids beyond L2 (the three workloads of the beyond-L2 pattern) and the eq 41 flop count of a
solve from its iteration trace, so that the reported fractions can be re-derived from the JSON line."""
import os
import sys
from types import SimpleNamespace

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_beyond_l2_step_bytes_match_hand_worked_values():
    # 2048^2 Gray-Scott, FP32 basis, p = 3: N = 2 * 2048^2 = 8388608; (3 + 3) 4 N = 201326592; two shared
    # field planes of 2048^2 floats = 33554432; total 234881024.  One-barrier schedule: + 2 * 4 N = 67108864.
    gs = SimpleNamespace(n=8388608, p=3, op={"nspecies": 2})
    assert bench.beyond_l2_bytes(gs, 4, 2) == (234881024, 301989888)
    # 2048^2 ADR, FP64, p = 4: N = 4194304; (4 + 3) 8 N = 234881024; the reaction field 8 N = 33554432.
    adr = SimpleNamespace(n=4194304, p=4, op={"nspecies": 1})
    assert bench.beyond_l2_bytes(adr, 8, 1) == (268435456, 335544320)
    # 160^3 ADR, FP32 basis, p = 4, no field: N = 4096000; 7 * 4 N = 114688000; + 8 N = 147456000.
    adr3 = SimpleNamespace(n=4096000, p=4, op={"kind": "stencil3d"})
    assert bench.beyond_l2_bytes(adr3, 4, 0) == (114688000, 147456000)


def test_solve_flop_model_matches_a_hand_worked_trace():
    """A 10 x 10 ADR stencil with its reaction field (nz = 5 * 100 + 100 = 600), p = 4, two substeps that each
    accept at j = 3 after one rejection at j = 2 (so 6 matvecs), every ||tau H~||_1 below theta_13 (s = 0).
    eq 41 per step: 2 * 600 + 7 * 100 + 4 + 8 * 104 + 3 * 104 = 3048; per substep -4 (N + p) = -416:
    6 * 3048 - 2 * 416 = 17456.  Update: 2 j N per accepted substep, 2 * 3 * 100 twice = 1200.  Exponentials:
    (8 + 0) * 2 * (j + 1)^3 per iteration, 2 * (432 + 1024) = 2912.  Total 17456 + 1200 + 2912 = 21568."""
    rng = np.random.default_rng(0)
    op = {"kind": "stencil2d", "nx": 10, "ny": 10, "nspecies": 1, "periodic": False,
          "coef": np.ones((1, 5)), "diag": {(0, 0): rng.standard_normal(100)}}
    P = SimpleNamespace(n=100, p=4, op=op)
    trace = []
    for sub in (0, 1):
        trace.append({"substep": sub, "j": 2, "accepted": False, "hnorm": 0.5})
        trace.append({"substep": sub, "j": 3, "accepted": True, "hnorm": 0.5})
    m = bench.algorithmic_model(P, {"matvecs": 6, "substeps": 2}, trace)
    assert m["nz"] == 600 and m["flops_per_step"] == 3048
    assert m["iop_flops_per_solve"] == 17456
    assert m["update_flops_per_solve"] == 1200
    assert m["expm_flops_per_solve"] == 2912
    assert m["fp64_flops_per_solve"] == 21568
