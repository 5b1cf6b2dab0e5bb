"""Fix-and-propagate with its final LP on the GPU (the 200 x 400 MIP relaxation pipeline:
LP to rel. KKT 1e-4 on the GPU, then fp_run, whose final LP is pdlp_solve at 1e-8)."""
import numpy as np
import pytest

import lpgen
from oracle import fp_oracle as F
from oracle import pdlp_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


def milp_opt(lp):
    from scipy.optimize import Bounds, LinearConstraint, milp
    r = milp(lp.c, constraints=LinearConstraint(lp.dense(), -np.inf, lp.b), integrality=lp.is_int,
             bounds=Bounds(lp.l, lp.u), options={"time_limit": 60})
    return r.fun if r.status in (0, 1) and r.fun is not None else None


@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("strategy", ["frac", "redcost", "dual", "type"])
def test_pipeline_feasible_point(P, seed, strategy):
    lp = lpgen.mip_relaxation(seed)
    x_lp, y_lp, res = P.pdlp_solve(lp, P.default_params(tol=1e-4, precision="fp32"))
    assert res["status"] == P.PDLP_OPTIMAL
    x, fr = P.fp_run(lp, x_lp, y_lp, strategy=strategy, seed=seed)
    assert fr["status"] == P.FP_FEASIBLE, fr
    a = lp.dense()
    assert np.all(a @ x <= lp.b + 1e-6 * np.maximum(1, np.abs(lp.b)))
    assert np.all(x >= lp.l - 1e-9) and np.all(x <= lp.u + 1e-9)
    xi = x[lp.is_int == 1]
    np.testing.assert_array_equal(xi, np.round(xi))
    assert fr["obj"] == pytest.approx(float(lp.c @ x), rel=1e-12)
    opt = milp_opt(lp)
    if opt is not None:
        assert fr["obj"] >= opt - 1e-6 * (1 + abs(opt))


@pytest.mark.parametrize("strategy", [F.FRAC, F.TYPE])
def test_final_lp_matches_oracle(P, strategy):
    """Same LP point in, same integers out (the search is bit-exact); the final LP on the
    GPU and in the oracle then agree to 1e-6 relative in the objective."""
    lp = lpgen.mip_relaxation(3)
    r = O.solve(lp, O.Params(tol=1e-4))
    ref = F.fp_run(lp, r.x, r.y, lp.is_int, strategy, seed=11)
    name = {F.FRAC: "frac", F.TYPE: "type"}[strategy]
    x, fr = P.fp_run(lp, r.x, r.y, strategy=name, seed=11)
    assert fr["status"] == ref.status == F.FEASIBLE
    ints = lp.is_int == 1
    np.testing.assert_array_equal(x[ints], ref.x[ints])
    assert abs(fr["obj"] - ref.obj) <= 1e-6 * (1 + abs(ref.obj))


def test_check_points_match_oracle(P):
    """The current point of the last KKT checks (float64 path) equals the oracle's; a fixed
    step keeps the two runs on the same rounding over the 192 steps (with the adaptive step
    they part by ~1e-8 after ~150 steps, the method's own sensitivity)."""
    lp = lpgen.mip_relaxation(2)
    _, _, r, dg = P.pdlp_solve(lp, P.default_params(iter_limit=192, terminate=0, adaptive_step=0,
                                                    fixed_eta=0.9), check_points=2)
    ref = O.solve(lp, O.Params(iter_limit=192, terminate=False, adaptive=False, fixed_eta=0.9,
                               record_checks=2))
    assert r["kkt_checks"] == 3 and dg["check_points"].shape == (2, lp.n)
    for got, want in zip(dg["check_points"], ref.check_points):
        assert np.linalg.norm(got - want) <= 1e-9 * max(1.0, np.linalg.norm(want))


@pytest.mark.parametrize("seed", [4, 5])
def test_fp_from_several_reference_points_matches_oracle(P, seed):
    """fp_run_refs keeps the best feasible run over the references (the search is exact,
    the final LPs agree to their tolerance): the oracle's choice and objective."""
    lp = lpgen.mip_relaxation(seed)
    ref = O.solve(lp, O.Params(tol=1e-4, record_checks=4))
    x, res, k = P.fp_run_refs(lp, ref.check_points, ref.y, strategy="frac", final_lp_tol=1e-6)
    best, i = F.fp_run_refs(lp, ref.check_points, ref.y, lp.is_int, F.FRAC, 1, final_tol=1e-6)
    assert (k >= 0) == (i >= 0)
    if i >= 0:
        assert res["status"] == P.FP_FEASIBLE
        assert res["obj"] == pytest.approx(best.obj, rel=1e-6, abs=1e-6)
        objs = [F.fp_run(lp, x0, ref.y, lp.is_int, F.FRAC, 1, final_tol=1e-6).obj
                for x0 in ref.check_points]
        assert objs[k] == pytest.approx(min(objs), rel=1e-6, abs=1e-6)
        assert F.max_row_violation(lp, x) <= 1e-6
