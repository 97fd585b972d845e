"""Pins of the oracle's adaptive control (Algorithm 4, eqs 39 and 43-46) and of its section 3.2 cost model
against values worked out by hand from the paper (tests/golden/alg4_scripted.txt, cost_model.txt; CPU only).

The scripted sequences drive the same Algorithm 4 function the oracle's Algorithm 1 calls after every
exponential, one iteration at a time, with error estimates chosen so that every branch, estimator and
clip of section 3.6 is reached; an inverted exponent in eq 43 or eq 45 contradicts the stored values (the
golden file gives, for each, the value the inverted formula would produce).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_05126_gb300 import workloads as W
from tests.golden_util import GOLDEN


def _scenarios():
    out, cur = [], None
    with open(os.path.join(GOLDEN, "alg4_scripted.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("scenario"):
                _, name, m_min, m_max, t_end, tol = line.split()
                cur = {"name": name, "m_min": int(m_min), "m_max": int(m_max), "T_end": float(t_end),
                       "tol": float(tol), "rows": []}
                out.append(cur)
                continue
            lhs, rhs = line.split("->")
            new, j, m, tau, t_now, eps, bd = lhs.split()
            om, acc, kap, qp1, rem, tau_new, m_new = rhs.split()
            cur["rows"].append(((int(new), int(j), int(m), float(tau), float(t_now), float(eps), int(bd)),
                                (float(om), int(acc), float(kap), float(qp1), float(rem), float(tau_new), int(m_new))))
    return out


SCEN = _scenarios()


def test_golden_file_covers_every_branch_of_algorithm_4():
    rows = [(s, r) for s in SCEN for r in s["rows"]]
    assert len(SCEN) == 5 and len(rows) == 14
    assert any(r[0][6] for _, r in rows)                                          # breakdown
    assert any(r[0][1] == s["m_max"] and not r[1][1] for s, r in rows)            # m_max, rejected (9-13)
    assert any(r[0][1] == s["m_max"] and r[1][1] and not r[0][6] for s, r in rows)  # m_max, accepted (15)
    assert any(r[0][1] < s["m_max"] and not r[0][6] for s, r in rows)              # vary m (18)


@pytest.mark.parametrize("scen", SCEN, ids=[s["name"] for s in SCEN])
def test_algorithm4_matches_the_hand_worked_sequence(scen):
    ctl = oracle.Alg4(m_min=scen["m_min"], m_max=scen["m_max"], T_end=scen["T_end"], tol=scen["tol"])
    for k, ((new, j, m, tau, t_now, eps, bd), (om, acc, kap, qp1, rem, tau_new, m_new)) in enumerate(scen["rows"]):
        d = ctl.step(bool(new), j, m, tau, t_now, eps, bool(bd))
        where = (scen["name"], k + 1)
        assert d["omega"] == pytest.approx(om, rel=1e-13, abs=0), where                 # eq 39
        assert d["accepted"] == bool(acc), where
        assert d["kappa"] == pytest.approx(kap, rel=1e-13), where                        # eq 45
        assert d["qp1"] == pytest.approx(qp1, rel=1e-12), where                          # eq 43 (R2)
        assert d["remaining"] == pytest.approx(rem, rel=1e-13, abs=1e-15), where         # R5
        assert d["tau_new"] == pytest.approx(tau_new, rel=1e-12, abs=0), where           # eq 44, Alg 4
        assert d["m_new"] == m_new, where                                                # eq 46, clips


def _cost_rows(kind):
    with open(os.path.join(GOLDEN, "cost_model.txt")) as f:
        return [list(map(float, ln.split()[1:])) for ln in f if ln.startswith(kind + " ")]


@pytest.mark.parametrize("row", _cost_rows("cost"))
def test_cost_of_eq40_matches_hand_worked_values(row):
    rem, tau, m, n, p, nz, nm, want = row
    assert oracle.cost_eq40(rem, tau, m, n, p, nz, nm) == want


@pytest.mark.parametrize("row", _cost_rows("nmult"))
def test_n_mult_of_eq42_follows_the_cited_pade_method(row):
    x, want = row
    assert oracle.n_mult(x) == want


def test_nz_of_eq41_counts_the_operators_stored_nonzeros():
    """Reading R9: CSR nnz; 5 (2D) or 7 (3D) per unknown and one per unknown and coupling field."""
    rng = np.random.default_rng(0)
    assert oracle.op_nonzeros(W.laplacian_1d_csr(400)) == 3 * 400 - 2               # tridiagonal
    assert oracle.op_nonzeros(W.adr2d(8, rng)) == 5 * 64 + 64                       # reaction field
    assert oracle.op_nonzeros(W.gray_scott2d(4, rng)) == 5 * 2 * 16 + 4 * 16         # four coupling fields
    assert oracle.op_nonzeros(W.adr3d(3, shift=-1.0)) == 7 * 27                      # constant shift: no field
