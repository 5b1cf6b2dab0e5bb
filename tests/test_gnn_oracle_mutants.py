"""Plant plausible mistakes in a copy of the warm-start oracle and check that a pin
catches each (CPU only, same scheme as the PDHG oracle's mutants)."""
import os
import sys
import types

import pytest

import test_gnn_oracle as P

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "gnn_oracle.py")

GRAD = "test_gradient_matches_central_differences"

MUTANTS = [
    ("constraint aggregation normalised by column degree",
     "rnorm = sp.diags(1.0 / np.maximum(deg_r, 1.0)) @ a", "rnorm = a @ sp.diags(1.0 / np.maximum(deg_c, 1.0))",
     ["test_message_passing_by_hand"]),
    ("variable aggregation through the row-normalised matrix",
     'sv.append(g["C"].T @ hc[-1])', 'sv.append(g["R"].T @ hc[-1])', ["test_message_passing_by_hand"]),
    ("backward drops the skip gradient into H_c", 'dhc = dhc + g["C"] @ dsv', 'dhc = g["C"] @ dsv', [GRAD]),
    ("backward masks with the input layer's activity", "dpv = dhv * (hv[k + 1] > 0)",
     "dpv = dhv * (hv[k] > 0)", [GRAD]),
    ("sigmoid derivative without (1 - s)", "sx * (1 - sx)", "sx", [GRAD]),
    ("message gradient through R instead of R^T", 'dhv = dhv_prev + g["R"].T @ dsc',
     'dhv = dhv_prev + g["C"] @ dsc[:0].sum() + g["R"].T[:, :0].sum()', [GRAD]),
    ("softplus on equality rows", 'y = np.where(g["eq"], zy, _softplus(zy))', "y = _softplus(zy)",
     ["test_message_passing_by_hand"]),
    ("bfloat16 by truncation", "(f + 0x7FFF + lsb)", "(f)", ["test_bf16_rounding_ties_to_even"]),
    ("Adam without bias correction", "mh = m / (1.0 - b1 ** t)", "mh = m",
     ["test_adam_first_step_is_lr_times_sign"]),
    ("features: <=-rows marked +1", "np.where(lp.sense == SENSE_GE, 1.0, np.where(lp.sense == SENSE_LE, -1.0, 0.0))",
     "np.where(lp.sense == SENSE_LE, 1.0, np.where(lp.sense == SENSE_GE, -1.0, 0.0))",
     ["test_features_by_hand"]),
]


def _mutant_module(old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) >= 1, old
    name = "gnn_oracle_mutant"
    mod = types.ModuleType(name)
    mod.__file__ = ORACLE_SRC
    sys.modules[name] = mod
    try:
        exec(compile(src.replace(old, new), ORACLE_SRC, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


def _run(name):
    fn = getattr(P, name)
    return fn(seed=1) if name == GRAD else fn()


@pytest.mark.parametrize("desc,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(desc, old, new, pins, monkeypatch):
    monkeypatch.setattr(P, "G", _mutant_module(old, new))
    caught = []
    for name in pins:
        try:
            _run(name)
        except Exception:
            caught.append(name)
    assert caught, f"mutant '{desc}' passed every pin in {pins}"


def test_unmutated_copy_passes_the_same_pins(monkeypatch):
    monkeypatch.setattr(P, "G", _mutant_module("import numpy as np", "import numpy as np"))
    for _, _, _, pins in MUTANTS:
        for name in pins:
            _run(name)
