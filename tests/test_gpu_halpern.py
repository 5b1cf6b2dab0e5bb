"""GPU parity of the reflected restarted Halpern PDHG variant (pdlp_params.halpern)
against the FP64 CPU oracle (reading A14), through the C ABI.

* the power-iteration estimate of ||K~||_2 agrees with the oracle's to 1e-12;
* float64 candidates T(z^K) after K constant steps agree with the oracle's to 1e-9
  relative, without and with restarts (the restart kinds and primal weights of every
  check equal the oracle's), with the reflection 1 and 0, and together with the
  bound-objective rescaling;
* the fixed-point residual of every step (the decision trace's eta_bar slot) agrees
  with the oracle's to 1e-9 relative;
* every precision mode reaches relative KKT 1e-4 under the oracle's float64 KKT with
  the objective within 1e-4 of the float64 oracle's optimum.
"""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from test_gpu_pdlp import GOLDEN_KEY, OBJ_TOL, PARITY, inst, obj_err, rel

pytestmark = pytest.mark.gpu

NAMES = ["mip_relaxation_200x400", "set_cover_2000x8000", "energy_system_24h",
         "random_free_eq_300x500", "skewed_6000x3000"]


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


def candidate_parity(its, ref):
    for k, want in (("x_cur", ref.x_cur), ("y_cur", ref.y_cur)):
        assert rel(its[k], want) <= PARITY, (k, rel(its[k], want))
    # no averages: the average candidate is the current one
    np.testing.assert_array_equal(its["x_avg"], its["x_cur"])
    np.testing.assert_array_equal(its["y_avg"], its["y_cur"])


@pytest.mark.parametrize("name", NAMES)
def test_spectral_norm_estimate_matches_oracle(P, name):
    lp = inst(name)
    _, _, res = P.pdlp_solve(lp, P.default_params(halpern=1, iter_limit=0))
    ref = O.solve(lp, O.Params(halpern=True, iter_limit=0))
    assert res["spectral_norm"] == pytest.approx(ref.spectral_norm, rel=1e-12)
    assert res["eta"] == pytest.approx(0.998 / ref.spectral_norm, rel=1e-12)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("K", [1, 10, 100])
def test_halpern_steps_match_oracle(P, name, K):
    lp = inst(name)
    _, _, res, its = P.pdlp_solve(
        lp, P.default_params(halpern=1, iter_limit=K, restarts=0, terminate=0), iterates=True)
    ref = O.solve(lp, O.Params(halpern=True, iter_limit=K, restarts=False, terminate=False))
    assert res["iters"] == res["attempts"] == K == ref.iters
    candidate_parity(its, ref)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("K", [64, 640])
def test_restarted_halpern_matches_oracle(P, name, K):
    """Restarts at the checks (every 64 steps) on the fixed-point residual, the anchor
    moved to the candidate and the primal weight updated: the same decisions, residual
    trace and candidates as the oracle."""
    lp = inst(name)
    _, _, res, dg = P.pdlp_solve(lp, P.default_params(halpern=1, iter_limit=K, terminate=0),
                                 trace=K + 64)
    ref = O.solve(lp, O.Params(halpern=True, iter_limit=K, terminate=False))
    assert res["iters"] == ref.iters == K
    assert res["restarts"] == ref.restarts
    assert list(dg["restart"]) == [c[0] for c in ref.check_trace]
    np.testing.assert_allclose(dg["omega"], [c[1] for c in ref.check_trace], rtol=1e-9)
    r_ref = np.array([t[1] for t in ref.attempt_trace])
    np.testing.assert_allclose(dg["eta_bar"], r_ref, rtol=1e-9)
    assert np.all(dg["accepted"] == 1)
    assert np.all(dg["eta"] == dg["eta"][0])  # a constant step
    assert res["omega"] == pytest.approx(ref.omega, rel=1e-9)
    candidate_parity(dg, ref)


@pytest.mark.parametrize("name", ["mip_relaxation_200x400", "energy_system_24h"])
def test_plain_halpern_without_reflection_matches_oracle(P, name):
    lp = inst(name)
    _, _, res, its = P.pdlp_solve(
        lp, P.default_params(halpern=1, halpern_reflection=0.0, iter_limit=200, terminate=0),
        iterates=True)
    ref = O.solve(lp, O.Params(halpern=True, halpern_reflection=0.0, iter_limit=200,
                               terminate=False))
    assert res["restarts"] == ref.restarts
    candidate_parity(its, ref)


@pytest.mark.parametrize("name", ["mip_relaxation_200x400", "set_cover_2000x8000"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_halpern_with_bound_objective_rescaling(P, name, prec):
    lp = inst(name)
    if prec == "fp64":
        _, _, res, its = P.pdlp_solve(
            lp, P.default_params(halpern=1, bound_objective_rescaling=1, iter_limit=200,
                                 terminate=0), iterates=True)
        ref = O.solve(lp, O.Params(halpern=True, bound_objective_rescaling=True, iter_limit=200,
                                   terminate=False))
        assert res["restarts"] == ref.restarts
        candidate_parity(its, ref)
    else:
        x, y, res = P.pdlp_solve(lp, P.default_params(halpern=1, bound_objective_rescaling=1,
                                                      precision=prec, tol=1e-4))
        assert res["status"] == P.PDLP_OPTIMAL, res
        assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-4


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_halpern_solve_reaches_tolerance(P, name, prec):
    lp = inst(name)
    x, y, res = P.pdlp_solve(lp, P.default_params(halpern=1, tol=1e-4, precision=prec))
    assert res["status"] == P.PDLP_OPTIMAL, res
    k = O.kkt_original(lp, x, y)
    assert k.rel_kkt <= 1.01e-4, (k, res)
    assert res["rel_kkt"] == pytest.approx(k.rel_kkt, rel=1e-6, abs=1e-12)
    assert obj_err(res["primal_obj"], GOLDEN_KEY[name]) <= OBJ_TOL
    assert np.all(x >= lp.l) and np.all(x <= lp.u)


def test_halpern_float64_solve_takes_the_oracle_iterations(P):
    """To 1e-4 in float64 the GPU stops at the same check as the oracle."""
    lp = inst("mip_relaxation_200x400")
    _, _, res = P.pdlp_solve(lp, P.default_params(halpern=1, tol=1e-4))
    ref = O.solve(lp, O.Params(halpern=True, tol=1e-4))
    assert res["status"] == ref.status == P.PDLP_OPTIMAL
    assert res["iters"] == ref.iters and res["restarts"] == ref.restarts


def test_halpern_lanes_keep_float64_steps(P):
    lp = inst("set_cover_2000x8000")
    outs = []
    for la, lt in [(2, 2), (32, 8)]:
        _, _, _, its = P.pdlp_solve(
            lp, P.default_params(halpern=1, iter_limit=100, terminate=0, lanes_A=la, lanes_AT=lt),
            iterates=True)
        outs.append(its)
    assert rel(outs[0]["x_cur"], outs[1]["x_cur"]) <= PARITY
    assert rel(outs[0]["y_cur"], outs[1]["y_cur"]) <= PARITY


def test_halpern_is_rejected_for_batches(P):
    lps = [lpgen.mip_relaxation(s) for s in (1, 2)]
    with pytest.raises(P.PdlpError) as e:
        P.pdlp_solve_batch(lps, P.default_params(halpern=1))
    assert "halpern is for single LPs" in str(e.value)
