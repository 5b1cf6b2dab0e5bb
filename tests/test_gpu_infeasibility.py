"""GPU certificates of primal infeasibility and unboundedness (A12), through the C ABI.

* float64 iterates: the status and, where the run is short enough for float64
  iterate parity to hold (a few hundred adaptive steps), the check at which it
  is found, the returned ray and its objective agree with the oracle;
* every precision mode and the batch return the oracle's status with a ray that
  passes the Farkas / descent check on the original data (written in the
  oracle's pin file with dense numpy, independent of both implementations);
* feasible LPs: the test never fires and switching it off changes no bit of
  the result; switched off, an infeasible LP runs to its iteration limit;
* a full-size covering LP (50,000 x 200,000) whose fixings leave a row with
  every column at 0, on the pattern matrix.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from oracle import pdlp_oracle as O
from test_oracle_infeasibility import INFEASIBLE, UNBOUNDED, descent_ray_margin, farkas_ray_margin

pytestmark = pytest.mark.gpu

CASES = {**{k: ("inf", f) for k, f in INFEASIBLE.items()},
         **{k: ("unb", f) for k, f in UNBOUNDED.items()}}
# float32 iterates cannot carry a ray whose certificate needs its growing
# components to cancel to 1e-8 (both columns free: A^T y^ must vanish)
FP32_CASES = [k for k in CASES if k != "free"]
_cache = {}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


def inst(name):
    if name not in _cache:
        _cache[name] = CASES[name][1]()
    return _cache[name]


def oracle(name):
    key = ("ref", name)
    if key not in _cache:
        _cache[key] = O.solve(inst(name), O.Params(tol=1e-8, iter_limit=20000))
    return _cache[key]


def check_certificate(P, lp, kind, x, y, r):
    if kind == "inf":
        assert r["status"] == P.PDLP_PRIMAL_INFEASIBLE, r
        margin, res = farkas_ray_margin(lp, y)
        assert margin > 0 and res <= 1e-8 * margin, (margin, res)
        assert r["ray_obj"] > 0
    else:
        assert r["status"] == P.PDLP_DUAL_INFEASIBLE, r
        descent, res = descent_ray_margin(lp, x)
        assert descent > 0 and res <= 1e-8 * descent, (descent, res)
        assert r["ray_obj"] < 0
    assert r["ray_res"] <= 1e-8 * abs(r["ray_obj"])


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_certificate_matches_oracle(P, name):
    kind, _ = CASES[name]
    lp = inst(name)
    ref = oracle(name)
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-8, iter_limit=20000))
    assert r["status"] == ref.status
    check_certificate(P, lp, kind, x, y, r)
    if ref.iters <= 256:
        assert r["iters"] == ref.iters and r["attempts"] == ref.attempts
        ray = ref.y if kind == "inf" else ref.x
        got = y if kind == "inf" else x
        assert np.linalg.norm(got - ray) <= 1e-6 * np.linalg.norm(ray)
        want = ref.rays[-1].dual_ray_obj if kind == "inf" else ref.rays[-1].primal_ray_obj
        assert r["ray_obj"] == pytest.approx(want, rel=1e-6)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("name", FP32_CASES)
def test_reduced_precision_certificate(P, name, prec):
    kind, _ = CASES[name]
    lp = inst(name)
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-8, iter_limit=20000, precision=prec))
    check_certificate(P, lp, kind, x, y, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_mixes_certificates_and_optima(P, prec):
    names = ["contradiction1", "relaxation1", "dead_cover", "box", "hand"]
    lps = [lpgen.mip_relaxation(1)] + [inst(k) for k in names] + [lpgen.set_cover(7, m=2000, n=8000)]
    kinds = ["opt"] + [CASES[k][0] for k in names] + ["opt"]
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-6, iter_limit=20000, precision=prec))
    for lp, kind, x, y, r in zip(lps, kinds, xs, ys, res):
        if kind == "opt":
            assert r["status"] == P.PDLP_OPTIMAL, (lp.name, r)
            assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-6
        else:
            check_certificate(P, lp, kind, x, y, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_batch_mixes_certificates_and_optima(P, prec):
    """The persistent kernel over a batch (persistent = 1): an LP that stops on a
    certificate leaves the launch's other LPs stepping."""
    names = ["contradiction1", "relaxation1", "dead_cover", "box", "hand"]
    lps = [lpgen.mip_relaxation(1)] + [inst(k) for k in names] + [lpgen.set_cover(7, m=2000, n=8000)]
    kinds = ["opt"] + [CASES[k][0] for k in names] + ["opt"]
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-6, iter_limit=20000, precision=prec,
                                                           persistent=1))
    for lp, kind, x, y, r in zip(lps, kinds, xs, ys, res):
        assert r["persistent_form"] == 1
        if kind == "opt":
            assert r["status"] == P.PDLP_OPTIMAL, (lp.name, r)
            assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-6
        else:
            check_certificate(P, lp, kind, x, y, r)


@pytest.mark.parametrize("name", FP32_CASES)
def test_shared_memory_kernel_certificates(P, name):
    """The one-block kernel (persistent = 2: the LP in shared memory where it fits, the
    covering LPs with a dead row from global memory) ends an infeasible or unbounded LP on
    the oracle's status with a valid ray."""
    kind, _ = CASES[name]
    lp = inst(name)
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-8, iter_limit=20000, persistent=2))
    assert r["persistent_form"] == (2 if name.startswith("dead_cover") else 3)
    check_certificate(P, lp, kind, x, y, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_switching_the_test_off_changes_nothing_on_feasible_lps(P, prec):
    lp = lpgen.random_sparse_lp(11, 300, 500)
    on = P.pdlp_solve(lp, P.default_params(tol=1e-6, precision=prec))
    off = P.pdlp_solve(lp, P.default_params(tol=1e-6, precision=prec, detect_infeasibility=0))
    assert on[2]["status"] == off[2]["status"] == P.PDLP_OPTIMAL
    assert on[2]["iters"] == off[2]["iters"]
    assert np.array_equal(on[0], off[0]) and np.array_equal(on[1], off[1])
    assert np.isnan(on[2]["ray_obj"]) and np.isnan(on[2]["ray_res"])


def test_switched_off_runs_to_the_limit(P):
    _, _, r = P.pdlp_solve(inst("box"), P.default_params(tol=1e-8, iter_limit=640,
                                                         detect_infeasibility=0))
    assert r["status"] == P.PDLP_ITER_LIMIT and r["iters"] == 640


def test_parity_mode_never_stops_on_a_certificate(P):
    # terminate = 0 runs to the limit whatever the checks find (as the oracle does); the
    # fixed step keeps float64 iterate parity on the diverging iterates (the adaptive
    # step feeds each rounding difference into the next step size)
    _, _, r, its = P.pdlp_solve(inst("box"), P.default_params(iter_limit=200, terminate=0,
                                                              adaptive_step=0, fixed_eta=0.9),
                                iterates=True)
    ref = O.solve(inst("box"), O.Params(iter_limit=200, terminate=False, adaptive=False,
                                        fixed_eta=0.9))
    assert r["status"] == ref.status == P.PDLP_ITER_LIMIT
    assert np.linalg.norm(its["y_cur"] - ref.y_cur) <= 1e-9 * max(1.0, np.linalg.norm(ref.y_cur))


def test_full_size_cover_with_a_dead_row(P):
    lp = lpgen.set_cover_dead(2025, 50_000, 200_000, dead=1)
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-4, iter_limit=100_000, precision="bf16"))
    assert r["status"] == P.PDLP_PRIMAL_INFEASIBLE, r
    # every bound is finite: the Farkas margin b^T y - sum_j max over [l_j, u_j] of (A^T y)_j x_j
    a = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    assert np.all(y >= 0)  # all rows are >=-rows
    g = a.T @ y
    margin = float(lp.b @ y) - float(np.maximum(g, 0) @ lp.u - np.maximum(-g, 0) @ lp.l)
    assert margin > 0
    assert r["ray_obj"] == pytest.approx(margin, rel=1e-6)


VARIANTS = {"halpern": ({"halpern": 1}, {"halpern": True}),
            "ndg_restarts": ({"restart_metric": 1}, {"restart_metric": "ndg"})}


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("name", list(CASES))
def test_variants_find_the_oracles_certificates(P, name, variant):
    """The algorithmic variants (Halpern PDHG, normalized-duality-gap restarts) end every
    infeasible or unbounded LP on the status the oracle reaches with the same variant, at
    the same check where float64 parity holds (short runs), with a valid ray."""
    kind, _ = CASES[name]
    lp = inst(name)
    gkw, okw = VARIANTS[variant]
    ref = O.solve(lp, O.Params(tol=1e-8, iter_limit=20000, **okw))
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-8, iter_limit=20000, **gkw))
    assert r["status"] == ref.status
    check_certificate(P, lp, kind, x, y, r)
    if ref.iters <= 256:
        assert r["iters"] == ref.iters
