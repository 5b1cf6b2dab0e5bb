"""GPU primal and dual feasibility polishing (A13) through the C ABI against the oracle.

* float64: the polished point after K PDHG steps of the objective-free problem
  (or of the dual feasibility problem) from the same loose point agrees with
  the oracle to 1e-9 relative;
* every precision mode makes a 1e-4 point row-feasible (checked row by row on
  the original data) and keeps it in its bounds, and a 1e-4 dual point dual
  feasible (checked reduced cost by reduced cost); strictly feasible and
  dual-feasible points come back unchanged;
* an infeasible LP ends with a Farkas ray, an unbounded one (dual side) with
  a ray of descent.
"""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from test_oracle_infeasibility import INFEASIBLE, UNBOUNDED, descent_ray_margin, farkas_ray_margin
from test_oracle_polish import DUAL_CASES, dual_violation, row_violation

pytestmark = pytest.mark.gpu

CASES = {
    "relaxation1": lambda: lpgen.mip_relaxation(1),
    "cover": lambda: lpgen.set_cover(7, m=2000, n=8000),
    "free_eq": lambda: lpgen.random_sparse_lp(11, 300, 500),
}
_cache = {}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


def loose(name):
    """The LP and the oracle's point at relative KKT 1e-4 (it misses rows)."""
    if name not in _cache:
        lp = CASES[name]()
        _cache[name] = (lp, O.solve(lp, O.Params(tol=1e-4)).x)
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("K", [1, 10, 100])
def test_fp64_polishing_matches_oracle(P, name, K):
    lp, x = loose(name)
    xg, yg, r = P.pdlp_polish_primal(lp, x, P.default_params(iter_limit=K, terminate=0))
    ref = O.polish_primal(lp, x, O.Params(iter_limit=K, terminate=False))
    assert r["iters"] == ref.iters == K
    for got, want in ((xg, ref.x), (yg, ref.y)):
        assert np.linalg.norm(got - want) <= 1e-9 * max(1.0, np.linalg.norm(want))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_polishing_makes_the_point_feasible(P, name, prec):
    lp, x = loose(name)
    before = row_violation(lp, x)
    assert before > 1e-5
    # float32 iterates resolve rows to ~1e-7 relative: polish to 1e-6 there
    tol = 1e-8 if prec == "fp64" else 1e-6
    xg, _, r = P.pdlp_polish_primal(lp, x, P.default_params(tol=tol, precision=prec))
    assert r["status"] == P.PDLP_OPTIMAL
    assert row_violation(lp, xg) <= (1e-6 if prec == "fp64" else 1e-5)
    assert np.all(xg >= lp.l) and np.all(xg <= lp.u)
    assert np.linalg.norm(xg - x) <= 10.0 * max(1.0, np.linalg.norm(x)) * before


def test_strictly_feasible_point_comes_back(P):
    lp = lpgen.mip_relaxation(4)
    x0 = lp.meta["x0"]
    xg, yg, r = P.pdlp_polish_primal(lp, x0, P.default_params(tol=1e-8))
    assert r["status"] == P.PDLP_OPTIMAL and r["iters"] == 64
    np.testing.assert_allclose(xg, x0, rtol=1e-15, atol=0)
    assert np.all(yg == 0.0)


def test_polishing_an_infeasible_lp(P):
    lp = INFEASIBLE["contradiction1"]()
    _, yg, r = P.pdlp_polish_primal(lp, np.zeros(lp.n), P.default_params(tol=1e-8, iter_limit=20000))
    assert r["status"] == P.PDLP_PRIMAL_INFEASIBLE
    margin, res = farkas_ray_margin(lp, yg)
    assert margin > 0 and res <= 1e-8 * margin


def loose_dual(name):
    """The LP and the oracle's dual point at relative KKT 1e-4 (it leaves reduced
    costs that no finite bound carries)."""
    key = ("dual", name)
    if key not in _cache:
        lp = DUAL_CASES[name]()
        _cache[key] = (lp, O.solve(lp, O.Params(tol=1e-4)).y)
    return _cache[key]


@pytest.mark.parametrize("name", list(DUAL_CASES))
@pytest.mark.parametrize("K", [1, 10, 100])
def test_fp64_dual_polishing_matches_oracle(P, name, K):
    lp, y = loose_dual(name)
    xg, yg, r = P.pdlp_polish_dual(lp, y, P.default_params(iter_limit=K, terminate=0))
    ref = O.polish_dual(lp, y, O.Params(iter_limit=K, terminate=False))
    assert r["iters"] == ref.iters == K
    for got, want in ((xg, ref.x), (yg, ref.y)):
        assert np.linalg.norm(got - want) <= 1e-9 * max(1.0, np.linalg.norm(want))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("name", list(DUAL_CASES))
def test_dual_polishing_makes_the_dual_point_feasible(P, name, prec):
    lp, y = loose_dual(name)
    before = dual_violation(lp, y)
    assert before > 1e-8
    tol = 1e-8 if prec == "fp64" else 1e-6
    _, yg, r = P.pdlp_polish_dual(lp, y, P.default_params(tol=tol, precision=prec))
    assert r["status"] == P.PDLP_OPTIMAL
    assert dual_violation(lp, yg) <= (1e-8 * before + 1e-14 if prec == "fp64" else 10 * tol)
    assert np.linalg.norm(yg - y) <= 100.0 * max(1.0, np.linalg.norm(y)) * max(before, tol)


def test_dual_feasible_point_comes_back(P):
    # every column of a covering LP has finite bounds: every y >= 0 is dual feasible
    lp = lpgen.set_cover(7, m=2000, n=8000)
    y = np.random.default_rng(3).uniform(0.0, 5.0, lp.m)
    xg, yg, r = P.pdlp_polish_dual(lp, y, P.default_params(tol=1e-8))
    assert r["status"] == P.PDLP_OPTIMAL and r["iters"] == 64
    np.testing.assert_allclose(yg, y, rtol=1e-15, atol=0)
    assert np.all(xg == 0.0)


def test_dual_polishing_an_unbounded_lp(P):
    lp = UNBOUNDED["relaxation1"]()
    xg, _, r = P.pdlp_polish_dual(lp, np.zeros(lp.m), P.default_params(tol=1e-8, iter_limit=20000))
    assert r["status"] == P.PDLP_DUAL_INFEASIBLE
    descent, res = descent_ray_margin(lp, xg)
    assert descent > 0 and res <= 1e-8 * descent
