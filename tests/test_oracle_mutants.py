"""Plant plausible mistakes in a copy of the oracle and check that a pin catches each.

Each mutant is the oracle's source with one textual change, executed as a
fresh module on the CPU; the named pins from ``test_oracle_pins`` are re-run
against it and at least one of them must fail.  Nothing here touches a GPU.
"""
import os
import sys
import types

import numpy as np
import pytest

import lpgen
import test_oracle_pins as P

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "pdlp_oracle.py")

MUTANTS = [
    ("extrapolation 2x'-x dropped", "kt @ (2.0 * x_new - x)", "kt @ x_new",
     ["test_one_pdhg_step_by_hand"]),
    ("<=-row sign flip applied to >=-rows", "np.where(lp.sense == SENSE_LE, -1.0, 1.0)",
     "np.where(lp.sense == SENSE_GE, -1.0, 1.0)", ["test_mip_relaxation_matches_highs"]),
    ("upper-bound term of the dual objective with the wrong sign",
     "- u[ufin] @ lm[ufin]", "+ u[ufin] @ lm[ufin]", ["test_kkt_by_hand_with_infinite_bounds"]),
    ("dual residual charged on the wrong side of an infinite bound",
     "np.where(np.isinf(l), lp_, 0.0) + np.where(np.isinf(u), lm, 0.0)",
     "np.where(np.isinf(l), lm, 0.0) + np.where(np.isinf(u), lp_, 0.0)",
     ["test_kkt_by_hand_with_infinite_bounds"]),
    ("step-size growth exponent -0.6 replaced by -0.3", "(1.0 + (attempts + 1) ** -0.6)",
     "(1.0 + (attempts + 1) ** -0.3)", ["test_step_growth_when_eta_bar_is_infinite"]),
    ("step-size shrink exponent -0.3 replaced by -0.6", "(1.0 - (attempts + 1) ** -0.3)",
     "(1.0 - (attempts + 1) ** -0.6)", ["test_adaptive_step_rule_by_hand"]),
    ("Ruiz factor without the square root", "r = np.where(rmax > 0, np.sqrt(rmax), 1.0)",
     "r = np.where(rmax > 0, rmax, 1.0)", ["test_ruiz_on_powers_of_four_gives_identity_exactly"]),
    ("primal step with tau = eta * omega", "(eta / omega) * (ct - ktt @ y)",
     "(eta * omega) * (ct - ktt @ y)", ["test_one_pdhg_step_by_hand"]),
    ("dual projection clips equality rows", "np.where(is_eq, y, np.maximum(y, 0.0))",
     "np.maximum(y, 0.0)", ["test_one_pdhg_step_by_hand"]),
    ("unweighted average", "sum_x += eta_used * x", "sum_x += x",
     ["test_average_is_step_size_weighted"]),
    ("primal residual ignores violated >=-rows", "np.maximum(q - kx, 0.0)", "np.minimum(q - kx, 0.0)",
     ["test_kkt_primal_residual_senses_by_hand"]),
    ("primal-weight hint ratio inverted", "omega = nyh / nxh", "omega = nxh / nyh",
     ["test_primal_weight_hint_by_hand"]),
    ("primal-weight hint not projected onto the bounds",
     "xh = proj_box(np.asarray(p.omega_hint[0], dtype=np.float64) / dc, lt, ut)",
     "xh = np.asarray(p.omega_hint[0], dtype=np.float64) / dc", ["test_primal_weight_hint_by_hand"]),
    ("initial primal weight inverted", "omega = nc / nq if", "omega = nq / nc if",
     ["test_scaling_b_and_c_by_powers_of_two_scales_the_iterates_exactly"]),
    ("step bound weighs dy by omega and dx by 1/omega",
     "num = omega * float(dx @ dx) + float(dy @ dy) / omega",
     "num = float(dx @ dx) / omega + omega * float(dy @ dy)",
     ["test_scaling_b_and_c_by_powers_of_two_scales_the_iterates_exactly"]),
    ("dual step with sigma = eta / omega", "y + eta * omega * (qt - kt @", "y + eta / omega * (qt - kt @",
     ["test_scaling_b_and_c_by_powers_of_two_scales_the_iterates_exactly"]),
    ("restart candidate with the higher KKT", "use_avg = ma < mc", "use_avg = ma > mc",
     ["test_restarts_and_primal_weight_by_hand"]),
    ("primal weight ratio inverted", "math.log(ddy / ddx)", "math.log(ddx / ddy)",
     ["test_restarts_and_primal_weight_by_hand"]),
    ("primal weight without smoothing", "+ (1.0 - p.omega_smooth) * math.log(omega))",
     "+ p.omega_smooth * math.log(ddy / ddx))", ["test_restarts_and_primal_weight_by_hand"]),
    ("artificial restart fraction 0.36 read as 0.6", "beta_art: float = 0.36",
     "beta_art: float = 0.6", ["test_restarts_and_primal_weight_by_hand"]),
    ("necessary-decay restart without the rise over the previous candidate",
     "or (m_cand <= p.beta_nec * m_last and m_cand > kkt_prev_cand)",
     "or (m_cand <= p.beta_nec * m_last)", ["test_necessary_decay_restart_by_hand"]),
    ("necessary-decay factor 0.8 read as 0.5", "beta_nec: float = 0.8", "beta_nec: float = 0.5",
     ["test_necessary_decay_restart_by_hand"]),
    ("sufficient-decay restart dropped", "do_restart = (m_cand <= p.beta_suff * m_last\n",
     "do_restart = (False\n", ["test_sufficient_decay_restart_by_hand"]),
    ("eta0 from the unscaled matrix", "kmax = float(abs(kt).max()) if kt.nnz else 0.0",
     "kmax = float(abs(k).max()) if k.nnz else 0.0",
     ["test_eta0_is_one_over_the_largest_scaled_entry_by_hand"]),
    ("eta0 from the Frobenius norm of K~", "kmax = float(abs(kt).max()) if kt.nnz else 0.0",
     "kmax = float(sp.linalg.norm(kt)) if kt.nnz else 0.0",
     ["test_eta0_is_one_over_the_largest_scaled_entry_by_hand"]),
    ("eta0 from the spectral norm of K~", "kmax = float(abs(kt).max()) if kt.nnz else 0.0",
     "kmax = float(np.linalg.norm(kt.toarray(), 2)) if kt.nnz else 0.0",
     ["test_eta0_is_one_over_the_largest_scaled_entry_by_hand"]),
    ("restart metric KKT_omega on the unscaled point",
     "return kkt_canonical(kt, qt, is_eq, ct, lt, ut, xs, ys)", "return unscaled_kkt(xs, ys)",
     ["test_restart_metric_is_taken_in_scaled_space_by_hand"]),
    ("primal-weight distances measured unscaled",
     "ddx = float(np.linalg.norm(cand_x - x_last))\n"
     "                    ddy = float(np.linalg.norm(cand_y - y_last))",
     "ddx = float(np.linalg.norm(dc * (cand_x - x_last)))\n"
     "                    ddy = float(np.linalg.norm(dr * (cand_y - y_last)))",
     ["test_primal_weight_distances_are_taken_in_scaled_space_by_hand"]),
    ("rescaled variable bounds divided by gamma instead of beta",
     "lt = lt / beta\n        ut = ut / beta", "lt = lt / gamma\n        ut = ut / gamma",
     ["test_bound_objective_rescaling_is_the_same_pdhg_without_restarts"]),
    ("rescaled dual point not multiplied back by gamma", "dr = dr * gamma", "dr = dr",
     ["test_bound_objective_rescaling_one_step_by_hand"]),
    ("objective rescaled by beta", "ct = ct / gamma", "ct = ct / beta",
     ["test_bound_objective_rescaling_one_step_by_hand"]),
    ("Halpern weight k/(k+1) instead of (k+1)/(k+2)", "lam = (h_k + 1.0) / (h_k + 2.0)",
     "lam = (h_k + 0.0) / (h_k + 1.0)", ["test_halpern_steps_by_hand"]),
    ("Halpern reflection added instead of subtracted", "- rho * yh", "+ rho * yh",
     ["test_halpern_steps_by_hand"]),
    ("Halpern anchor kept at a restart",
     "xa0, ya0 = x.copy(), y.copy()\n                    h_k = 0", "h_k = 0",
     ["test_halpern_sufficient_decay_restart_by_hand"]),
    ("fixed-point residual with the cross term's sign flipped",
     "- 2.0 * float(dy @ (kt @ dx)))", "+ 2.0 * float(dy @ (kt @ dx)))",
     ["test_halpern_steps_by_hand"]),
    ("power iteration on K~ instead of K~^T K~", "w = kt.T @ (kt @ v)", "w = kt @ v",
     ["test_power_iteration_closed_forms"]),
    ("epoch residual r_0 replaced at every step",
     "if h_k == 0:\n                h_r0 = h_res", "h_r0 = h_res",
     ["test_halpern_necessary_decay_restart_by_hand"]),
    ("trust-region step of y scaled by 1/omega", "proj_dual(y + (t * omega) * gy, is_eq)",
     "proj_dual(y + (t / omega) * gy, is_eq)", ["test_trust_region_gap_closed_forms"]),
    ("gap gradient g_x with the wrong sign", "gx = ktt @ ys - ct", "gx = ct - ktt @ ys",
     ["test_normalized_gap_by_hand"]),
    ("gap not divided by the radius", "return val / r", "return val",
     ["test_normalized_gap_by_hand"]),
    ("reference gap not moved at a restart", "ndg_last = m_cand\n", "\n",
     ["test_ndg_restart_sequence_differs_from_kkt_and_restarts_less_on_a_relaxation"]),
    ("gap radius without the primal weight",
     "r = math.sqrt(omega * float(dx @ dx) + float(dy @ dy) / omega)\n    if r == 0.0:",
     "r = math.sqrt(float(dx @ dx) + float(dy @ dy))\n    if r == 0.0:",
     ["test_normalized_gap_by_hand"]),
    ("Halpern candidate taken at the mixed iterate instead of T(z)",
     "x, y = x_new, y_new\n            it += 1", "x, y = xh.copy(), yh.copy()\n            it += 1",
     ["test_halpern_steps_by_hand"]),
]


def _pin_args(name):
    """Arguments of a parametrised pin when it is called directly."""
    if name == "test_mip_relaxation_matches_highs":
        return {"seed": 1}
    if name == "test_scaling_b_and_c_by_powers_of_two_scales_the_iterates_exactly":
        return {"maker": lambda: lpgen.mip_relaxation(1)}
    if name == "test_bound_objective_rescaling_is_the_same_pdhg_without_restarts":
        return {"maker": lambda: lpgen.mip_relaxation(2)}
    return {}


def _mutant_module(old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) >= 1, old
    name = "pdlp_oracle_mutant"
    mod = types.ModuleType(name)
    mod.__file__ = ORACLE_SRC
    sys.modules[name] = mod  # dataclasses look their module up here
    try:
        exec(compile(src.replace(old, new), ORACLE_SRC, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


@pytest.mark.parametrize("desc,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(desc, old, new, pins, monkeypatch):
    mutant = _mutant_module(old, new)
    monkeypatch.setattr(P, "O", mutant)
    caught = []
    for name in pins:
        fn = getattr(P, name)
        try:
            fn(**_pin_args(name))
        except Exception:  # an assertion, or the mutant breaking outright
            caught.append(name)
    assert caught, f"mutant '{desc}' passed every pin in {pins}"


def test_unmutated_copy_passes_the_same_pins(monkeypatch):
    """Control: the exec'd copy without a change passes the pins used above."""
    mod = _mutant_module("import math", "import math")
    monkeypatch.setattr(P, "O", mod)
    for _, _, _, pins in MUTANTS:
        for name in pins:
            getattr(P, name)(**_pin_args(name))
