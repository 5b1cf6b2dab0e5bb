"""GPU parity of the normalized-duality-gap restarts (pdlp_params.restart_metric = 1)
against the FP64 CPU oracle (reading A9b), through the C ABI.

* with a stable fixed step and restarts, the restart kind and primal weight of every
  check and the float64 iterates after 640 steps agree with the oracle (1e-9);
* the adaptive float64 solve to 1e-4 stops at the oracle's check with its restarts;
* every precision mode reaches relative KKT 1e-4 under the oracle's float64 KKT with the
  objective within 1e-4 of the float64 oracle's optimum; the other step forms
  (persistent, tiles) run the same restart rule.
"""
import numpy as np
import pytest

from oracle import pdlp_oracle as O
from test_gpu_pdlp import GOLDEN_KEY, OBJ_TOL, PARITY, assert_iterate_parity, inst, obj_err

pytestmark = pytest.mark.gpu

NAMES = ["mip_relaxation_200x400", "set_cover_2000x8000", "energy_system_24h",
         "random_free_eq_300x500", "skewed_6000x3000"]


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("K", [128, 640])
def test_ndg_restarts_with_a_fixed_step_match_oracle(P, name, K):
    lp = inst(name)
    _, _, res, dg = P.pdlp_solve(lp, P.default_params(restart_metric=1, iter_limit=K, terminate=0,
                                                      adaptive_step=0, fixed_eta=0.9),
                                 trace=K + 64)
    ref = O.solve(lp, O.Params(restart_metric="ndg", iter_limit=K, terminate=False,
                               adaptive=False, fixed_eta=0.9))
    assert res["iters"] == ref.iters == K
    assert list(dg["restart"]) == [c[0] for c in ref.check_trace]
    np.testing.assert_allclose(dg["omega"], [c[1] for c in ref.check_trace], rtol=1e-9)
    assert res["restarts"] == ref.restarts
    assert_iterate_parity(dg, ref)


@pytest.mark.parametrize("name", ["mip_relaxation_200x400", "random_free_eq_300x500"])
def test_ndg_adaptive_float64_solve_takes_the_oracle_checks(P, name):
    lp = inst(name)
    _, _, res = P.pdlp_solve(lp, P.default_params(restart_metric=1, tol=1e-4))
    ref = O.solve(lp, O.Params(restart_metric="ndg", tol=1e-4))
    assert res["status"] == ref.status == P.PDLP_OPTIMAL
    assert res["iters"] == ref.iters and res["restarts"] == ref.restarts


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_ndg_solve_reaches_tolerance(P, name, prec):
    lp = inst(name)
    x, y, res = P.pdlp_solve(lp, P.default_params(restart_metric=1, tol=1e-4, precision=prec))
    assert res["status"] == P.PDLP_OPTIMAL, res
    k = O.kkt_original(lp, x, y)
    assert k.rel_kkt <= 1.01e-4, (k, res)
    assert obj_err(res["primal_obj"], GOLDEN_KEY[name]) <= OBJ_TOL
    assert np.all(x >= lp.l) and np.all(x <= lp.u)


@pytest.mark.parametrize("form", [dict(persistent=1), dict(persistent=2),
                                  dict(tiles=1, precision="fp32"), dict(tiles=2, precision="fp32")])
def test_ndg_restarts_in_every_step_form(P, form):
    lp = inst("mip_relaxation_200x400")
    kw = dict(restart_metric=1, iter_limit=256, terminate=0, adaptive_step=0, fixed_eta=0.9)
    _, _, res, dg = P.pdlp_solve(lp, P.default_params(**kw, **form), trace=512)
    _, _, res0, dg0 = P.pdlp_solve(lp, P.default_params(**kw, precision=form.get("precision",
                                                                                    "fp64")),
                                   trace=512)
    assert list(dg["restart"]) == list(dg0["restart"])
    np.testing.assert_allclose(dg["omega"], dg0["omega"], rtol=1e-5)


def test_ndg_is_rejected_for_batches(P):
    import lpgen
    lps = [lpgen.mip_relaxation(s) for s in (1, 2)]
    with pytest.raises(P.PdlpError) as e:
        P.pdlp_solve_batch(lps, P.default_params(restart_metric=1))
    assert "restart_metric = 1 is for single LPs" in str(e.value)
