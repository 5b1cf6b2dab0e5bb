"""The stored expected values under tests/golden/ against independent pins (CPU).

objectives.json holds the float64 oracle's objective at rel. KKT 1e-6 for every
instance whose reduced-precision objective the GPU tests check (written by
make_golden.py from oracle/ only).  Each is pinned here by HiGHS's optimum,
stored beside it, and by the relative KKT the oracle reached.
"""
import json
import os

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load():
    return json.load(open(os.path.join(HERE, "objectives.json")))


@pytest.mark.parametrize("key", sorted(load()))
def test_stored_oracle_objective_matches_highs(key):
    g = load()[key]
    assert g["oracle_status"] == 1 and g["oracle_rel_kkt"] <= g["oracle_tol"]
    # a relative KKT of 1e-6 bounds the objective's distance from the optimum by a few 1e-6
    assert abs(g["oracle_obj"] - g["highs_obj"]) / (1 + abs(g["highs_obj"])) <= 5e-6, g
    # the 1e-4 solution: within the few 1e-4 its relative gap and residuals allow
    assert g["oracle_rel_kkt_tol"] <= 1e-4
    assert abs(g["oracle_obj_tol"] - g["highs_obj"]) / (1 + abs(g["highs_obj"])) <= 5e-4, g


def test_every_checked_instance_has_a_stored_objective():
    import sys
    sys.path.insert(0, HERE)
    import make_golden
    assert set(make_golden.OBJECTIVES) <= set(load())
