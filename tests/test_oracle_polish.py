"""Pins of the oracle's primal and dual feasibility polishing (A13).

Facts fixed outside the oracle: two PDHG steps of the objective-free problem
and two of the dual feasibility problem worked by hand; a strictly feasible
point (the generator's x0) and a dual-feasible point are fixed points; HiGHS
says which LPs are feasible and every polished point is checked row by row (or
reduced cost by reduced cost) on the original data; an infeasible LP ends with
a Farkas ray and an unbounded one with a ray of descent.  Planted mistakes at
the end are each caught.
"""
import sys

import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from test_oracle_infeasibility import (INFEASIBLE, UNBOUNDED, _highs_status, _lp, descent_ray_margin,
                                      farkas_ray_margin)
from test_oracle_mutants import _mutant_module

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

NOSCALE = dict(ruiz_iters=0, pc_alpha=None, restarts=False, terminate=False)


def row_violation(lp, x):
    """Largest violation of a row, scaled by max(1, |b_i|), in dense numpy."""
    ax = lp.dense() @ x
    le, ge = lp.sense == ord("L"), lp.sense == ord("G")
    v = np.where(le, ax - lp.b, np.where(ge, lp.b - ax, np.abs(ax - lp.b)))
    return float(np.max(np.maximum(v, 0.0) / np.maximum(1.0, np.abs(lp.b)), initial=0.0))


def test_two_steps_by_hand():
    # x1 + x2 >= 3 in [0, 10]^2 from x = (1, 1), y = 0, eta = 0.5, omega = 1, K~ = K:
    # step 1: x+ = x - 0.5 (0 - K^T 0) = (1, 1); y+ = max(0 + 0.5 (3 - K(2x+ - x)), 0) = 0.5
    # step 2: x+ = (1, 1) - 0.5 (0 - (0.5, 0.5)) = (1.25, 1.25); 2x+ - x = (1.5, 1.5),
    #         K(2x+ - x) = 3, y+ = 0.5 + 0.5 (3 - 3) = 0.5
    lp = _lp([[1, 1]], [3], "G", [1, 1], [0, 0], [10, 10])
    r = O.polish_primal(lp, np.array([1.0, 1.0]),
                        O.Params(iter_limit=2, adaptive=False, fixed_eta=0.5, fixed_omega=1.0,
                                 **NOSCALE))
    assert r.iters == 2
    assert r.x_cur.tolist() == [1.25, 1.25]
    assert r.y_cur.tolist() == [0.5]


def test_strictly_feasible_point_is_a_fixed_point():
    # b = A x0 + U[0, 3] row by row: x0 satisfies every row with slack, so y stays 0
    lp = lpgen.mip_relaxation(4)
    x0 = lp.meta["x0"]
    assert row_violation(lp, x0) == 0.0
    r = O.polish_primal(lp, x0, O.Params(tol=1e-8))
    assert r.status == O.STATUS_OPTIMAL and r.iters == 64
    np.testing.assert_allclose(r.x, x0, rtol=1e-15, atol=0)
    assert np.all(r.y == 0.0)


@pytest.mark.parametrize("maker", [lambda: lpgen.mip_relaxation(1), lambda: lpgen.mip_relaxation(3),
                                   lambda: lpgen.set_cover(7, m=2000, n=8000),
                                   lambda: lpgen.random_sparse_lp(11, 300, 500)],
                         ids=["relaxation1", "relaxation3", "cover", "free_eq"])
def test_polishing_makes_a_loose_point_feasible(maker):
    lp = maker()
    assert _highs_status(lp) == 0
    r = O.solve(lp, O.Params(tol=1e-4))
    before = row_violation(lp, r.x)
    assert before > 1e-5  # a 1e-4 point misses rows
    p = O.polish_primal(lp, r.x, O.Params(tol=1e-8))
    assert p.status == O.STATUS_OPTIMAL
    assert row_violation(lp, p.x) <= 1e-8 * before + 1e-12
    assert np.all(p.x >= lp.l) and np.all(p.x <= lp.u)
    # the polished point moves the start by a distance of the order of its violation
    assert np.linalg.norm(p.x - r.x) <= 10.0 * max(1.0, np.linalg.norm(r.x)) * before


def test_polishing_an_infeasible_lp_returns_a_farkas_ray():
    lp = INFEASIBLE["contradiction1"]()
    p = O.polish_primal(lp, np.zeros(lp.n), O.Params(tol=1e-8, iter_limit=20000))
    assert p.status == O.STATUS_PRIMAL_INFEASIBLE
    margin, res = farkas_ray_margin(lp, p.y)
    assert margin > 0 and res <= 1e-8 * margin


def dual_violation(lp, y):
    """Relative dual residual of y on the original data in dense numpy: the parts of
    lambda = c - A^T y that no finite bound carries, ||.||_2 / (1 + ||c||_2); y must
    keep the caller's signs (<= 0 on <=-rows, >= 0 on >=-rows)."""
    assert np.all(y[lp.sense == ord("L")] <= 0) and np.all(y[lp.sense == ord("G")] >= 0)
    lam = lp.c - lp.dense().T @ y
    bad = np.where(np.isinf(lp.l), np.maximum(lam, 0.0), 0.0) + \
        np.where(np.isinf(lp.u), np.maximum(-lam, 0.0), 0.0)
    return float(np.linalg.norm(bad)) / (1.0 + float(np.linalg.norm(lp.c)))


DUAL_CASES = {
    "free_eq": lambda: lpgen.random_sparse_lp(11, 300, 500),
    "free_eq2": lambda: lpgen.random_sparse_lp(12, 400, 300),
    "energy": lambda: lpgen.energy_system(hours=24, regions=5, lines=6, techs=3, thermal=2),
}


def test_dual_two_steps_by_hand():
    # min x1 + x2, x1 + x2 >= 3, x in [1, inf)^2, from y = 2: the dual feasibility problem
    # has b = 0 and x in [0, inf)^2; from x = 0 with eta = 0.5, omega = 1, K~ = K:
    # step 1: x+ = max(0 - 0.5 (1 - 2), 0) = (0.5, 0.5); K(2x+ - x) = 2, y+ = 2 + 0.5 (0 - 2) = 1
    # step 2: x+ = 0.5 - 0.5 (1 - 1) = (0.5, 0.5); K(2x+ - x) = 1, y+ = 1 + 0.5 (0 - 1) = 0.5
    lp = _lp([[1, 1]], [3], "G", [1, 1], [1, 1], [np.inf, np.inf])
    r = O.polish_dual(lp, np.array([2.0]),
                      O.Params(iter_limit=2, adaptive=False, fixed_eta=0.5, fixed_omega=1.0,
                               **NOSCALE))
    assert r.iters == 2
    assert r.x_cur.tolist() == [0.5, 0.5]
    assert r.y_cur.tolist() == [0.5]


def test_dual_feasible_point_is_a_fixed_point():
    # every column of a covering LP has finite bounds, so every y >= 0 is dual feasible
    lp = lpgen.set_cover(7, m=2000, n=8000)
    y = np.random.default_rng(3).uniform(0.0, 5.0, lp.m)
    r = O.polish_dual(lp, y, O.Params(tol=1e-8))
    assert r.status == O.STATUS_OPTIMAL and r.iters == 64
    np.testing.assert_allclose(r.y, y, rtol=1e-15, atol=0)
    assert np.all(r.x == 0.0)


@pytest.mark.parametrize("name", list(DUAL_CASES))
def test_dual_polishing_makes_a_loose_dual_point_feasible(name):
    lp = DUAL_CASES[name]()
    assert _highs_status(lp) == 0
    r = O.solve(lp, O.Params(tol=1e-4))
    before = dual_violation(lp, r.y)
    assert before > 1e-8  # a 1e-4 dual point leaves reduced costs uncarried
    p = O.polish_dual(lp, r.y, O.Params(tol=1e-8))
    assert p.status == O.STATUS_OPTIMAL
    assert dual_violation(lp, p.y) <= 1e-8 * before + 1e-14
    # the polished point moves the start by a distance of the order of its violation
    assert np.linalg.norm(p.y - r.y) <= 100.0 * max(1.0, np.linalg.norm(r.y)) * before


@pytest.mark.parametrize("name", ["relaxation1", "relaxation2"])
def test_dual_polishing_of_an_unbounded_lp_returns_a_descent_ray(name):
    lp = UNBOUNDED[name]()
    p = O.polish_dual(lp, np.zeros(lp.m), O.Params(tol=1e-8, iter_limit=20000))
    assert p.status == O.STATUS_DUAL_INFEASIBLE
    descent, res = descent_ray_margin(lp, p.x)
    assert descent > 0 and res <= 1e-8 * descent


MUTANTS = [
    ("polishing keeps the objective", "lp0.c = np.zeros(lp.n)", "lp0.c = lp.c.copy()",
     ["test_two_steps_by_hand"]),
    ("polishing ignores the given point", "return solve(lp0, params, x0=x, y0=None)",
     "return solve(lp0, params, x0=None, y0=None)", ["test_two_steps_by_hand"]),
    ("dual polishing keeps b", "lp0.b = np.zeros(lp.m)", "lp0.b = lp.b.copy()",
     ["test_dual_two_steps_by_hand"]),
    ("dual polishing keeps the finite bounds", "lp0.l = np.where(np.isfinite(lp.l), 0.0, lp.l)",
     "lp0.l = lp.l.copy()", ["test_dual_two_steps_by_hand"]),
    ("dual polishing ignores the given point", "return solve(lp0, params, x0=None, y0=y)",
     "return solve(lp0, params, x0=None, y0=None)", ["test_dual_two_steps_by_hand"]),
]


@pytest.mark.parametrize("desc,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(desc, old, new, pins, monkeypatch):
    monkeypatch.setattr(sys.modules[__name__], "O", _mutant_module(old, new))
    caught = []
    for name in pins:
        try:
            globals()[name]()
        except Exception:
            caught.append(name)
    assert caught, f"mutant '{desc}' passed every pin in {pins}"
