"""Fix-and-propagate consumer (section 2 of the paper): oracle pins and C ABI parity.

CPU only: the C ABI's fp_run runs on the host, and with final_lp = 0 it never
touches the GPU, so its search (ordering, LP-based fixing, Alg. 1 branching,
propagation, backtracking) is compared with the oracle's, decision for
decision, here.  The final LP (pdlp_solve) is covered in test_gpu_fp.py.
"""
import math
import os

import numpy as np
import pytest

import lpgen
from oracle import fp_oracle as F
from oracle import pdlp_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _mip(a, b, sense, c, l, u, is_int):
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    rows, cols = np.nonzero(a)
    return lpgen._lp(m, n, rows, cols, a[rows, cols], np.asarray(b, float),
                     np.array([ord(s) for s in sense], dtype=np.uint8), np.asarray(c, float),
                     np.asarray(l, float), np.asarray(u, float), np.asarray(is_int, np.uint8), "hand")


# ---------------------------------------------------------------- pins
def test_splitmix64_published_vector():
    want = [int(v) for v in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if v.strip() and not v.startswith("#")]
    r = F.SplitMix64(1234567)
    assert [r.next() for _ in range(len(want))] == want


def test_uniform_draws_are_in_unit_interval_and_uniform():
    r = F.SplitMix64(7)
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=10, range=(0, 1))
    assert np.all(np.abs(hist - 2000) < 5 * np.sqrt(2000))


def test_alg1_branching_table():
    """Every case of Alg. 1 (increasing priority; the fixing value last)."""
    for line in open(os.path.join(GOLDEN, "alg1_branching.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split("|")
        l, u, a, c = (float(v) for v in lhs.split())
        want = [tuple(float(v) for v in ch.split(":")) for ch in rhs.strip().split(";")]
        assert F.branching(l, u, a, c) == want, line


def test_lp_fixing_rule():
    # d_i = 0.3: d > 0.3 -> floor (lower), otherwise ceil (upper)
    assert F.lp_fixing_value(2.3, 0, 5, 0.31) == 2.0
    assert F.lp_fixing_value(2.3, 0, 5, 0.29) == 3.0
    assert F.lp_fixing_value(2.25, 0, 5, 0.25) == 3.0         # d == d_i (exact) fixes up
    assert F.lp_fixing_value(4.0, 0, 5, 0.5) == 4.0           # integral value stays
    assert F.lp_fixing_value(-0.2, 0, 1, 0.9) == 0.0          # LP value clamped to the domain first
    assert F.lp_fixing_value(7.4, 0, 5, 0.1) == 5.0


def hand_mip():
    """rows: x0 + x1 <= 1;  x1 + x2 + x3 <= 2;  x3 + x4 <= 1 (all <=);
    c = (-1, -2, 1, 3, -1); x0, x1, x3 binary, x2 integer in [0,3], x4 continuous in [0,5];
    LP point x = (0.9, 0.5, 0.2, 0, 1), y = (-2, -0.5, -1)."""
    lp = _mip([[1, 1, 0, 0, 0], [0, 1, 1, 1, 0], [0, 0, 0, 1, 1]], [1, 2, 1], "LLL",
              [-1, -2, 1, 3, -1], [0, 0, 0, 0, 0], [1, 1, 3, 1, 5], [1, 1, 1, 1, 0])
    return lp, np.array([0.9, 0.5, 0.2, 0.0, 1.0]), np.array([-2.0, -0.5, -1.0])


def test_variable_orders_by_hand():
    """lambda = c - A^T y = (1, 0.5, 1.5, 4.5, 0).
    FRAC: fractionalities (0.1, 0.5, 0.2, 0) -> 3, 0, 2, 1.
    REDCOST: |lambda| (1, 0.5, 1.5, 4.5) -> 3, 2, 0, 1.
    DUAL: rows by |y|: 0 (2), 2 (1), 1 (0.5); row 0 gives 0, 1 (by |lambda|), row 2 gives 3,
          row 1 gives 2 -> 0, 1, 3, 2.
    TYPE: binaries 0, 1, 3 then the general integer 2."""
    lp, x, y = hand_mip()
    np.testing.assert_allclose(F.reduced_costs(lp, y), [1, 0.5, 1.5, 4.5, 0])
    ii = lp.is_int
    assert F.variable_order(lp, F.FRAC, x, y, ii) == [3, 0, 2, 1]
    assert F.variable_order(lp, F.REDCOST, x, y, ii) == [3, 2, 0, 1]
    assert F.variable_order(lp, F.DUAL, x, y, ii) == [0, 1, 3, 2]
    assert F.variable_order(lp, F.TYPE, x, y, ii) == [0, 1, 3, 2]


def tie_mip():
    """rows: x0 + x1 <= 1;  x2 + x3 <= 1;  x3 + x4 <= 1 (all <=); seven binaries, x5 and x6
    in no row; c = (-2, -1, -3, -4, -2, 0.5, 2); LP point x = (1, 0, 0.5, 0.5, 0, 0.3, 0.9),
    y = (-1, -2, -3).  Built so that every strategy meets ties."""
    a = [[1, 1, 0, 0, 0, 0, 0], [0, 0, 1, 1, 0, 0, 0], [0, 0, 0, 1, 1, 0, 0]]
    lp = _mip(a, [1, 1, 1], "LLL", [-2, -1, -3, -4, -2, 0.5, 2], [0] * 7, [1] * 7, [1] * 7)
    return lp, np.array([1.0, 0.0, 0.5, 0.5, 0.0, 0.3, 0.9]), np.array([-1.0, -2.0, -3.0])


def test_hybrid_orders_by_hand():
    """Section 2, "Tiebreaking and hybrid strategies": Frac with ties broken by Dual or by
    RedCost, and the reverse.  A^T y = (-1, -1, -2, -5, -3, 0, 0), so lambda = c - A^T y =
    (-1, 0, -1, 1, 1, 0.5, 2); |lambda| = (1, 0, 1, 1, 1, 0.5, 2); fractionality
    (0, 0, 0.5, 0.5, 0, 0.3, 0.1).
    FRAC:    0: {0, 1, 4} | 0.1: 6 | 0.3: 5 | 0.5: {2, 3}            -> 0 1 4 6 5 2 3
    REDCOST: 2: 6 | 1: {0, 2, 3, 4} | 0.5: 5 | 0: 1                   -> 6 0 2 3 4 5 1
    DUAL:    rows by |y|: r2, r1, r0; r2 -> 3, 4 (|lambda| tie, storage order); r1 -> 2;
             r0 -> 0, 1; no row: 5, 6 by index                        -> 3 4 2 0 1 5 6
    FRAC_DUAL:    {0, 1, 4} by DUAL rank (3, 4, 1) -> 4 0 1; 6; 5;
                  {2, 3} by rank (2, 0) -> 3 2                        -> 4 0 1 6 5 3 2
    FRAC_REDCOST: {0, 1, 4} by |lambda| (1, 0, 1) -> 0 4 1; 6; 5;
                  {2, 3} tie on both -> index                         -> 0 4 1 6 5 2 3
    DUAL_FRAC:    r2: 3, 4 tie on |lambda| -> by frac (0.5, 0) -> 4 3; r1 -> 2;
                  r0 -> 0 1; no row by frac (0.3, 0.1) -> 6 5        -> 4 3 2 0 1 6 5
    REDCOST_FRAC: 6; {0, 2, 3, 4} by frac (0, 0.5, 0.5, 0) -> 0 4 2 3; 5; 1
                                                                      -> 6 0 4 2 3 5 1"""
    lp, x, y = tie_mip()
    np.testing.assert_allclose(F.reduced_costs(lp, y), [-1, 0, -1, 1, 1, 0.5, 2])
    ii = lp.is_int
    want = {F.FRAC: [0, 1, 4, 6, 5, 2, 3], F.REDCOST: [6, 0, 2, 3, 4, 5, 1],
            F.DUAL: [3, 4, 2, 0, 1, 5, 6], F.FRAC_DUAL: [4, 0, 1, 6, 5, 3, 2],
            F.FRAC_REDCOST: [0, 4, 1, 6, 5, 2, 3], F.DUAL_FRAC: [4, 3, 2, 0, 1, 6, 5],
            F.REDCOST_FRAC: [6, 0, 4, 2, 3, 5, 1]}
    for strategy, order in want.items():
        assert F.variable_order(lp, strategy, x, y, ii) == order, strategy


def test_propagation_by_hand():
    """Fixing x0 = 1 forces x1 <= (1 - 1)/1 = 0 (row 0) and then x2 <= 2 - 0 - 0 = 2 (row 1)."""
    lp, _, _ = hand_mip()
    at_ptr, at_row = F.transpose_lists(lp)
    dom = F.Domains(lp.l, lp.u, [bool(v) for v in lp.is_int])
    assert F.propagate(lp, at_ptr, at_row, dom, range(lp.m))
    assert dom.hi[2] == 2.0  # root: x1 + x2 + x3 <= 2 already caps x2 at 2
    dom.set(0, 1.0, 1.0)
    assert F.propagate(lp, at_ptr, at_row, dom, at_row[at_ptr[0]:at_ptr[1]])
    assert (dom.lo[1], dom.hi[1]) == (0.0, 0.0)
    # and x3 = 1 with x4 continuous: x4 <= 0
    dom.set(3, 1.0, 1.0)
    assert F.propagate(lp, at_ptr, at_row, dom, at_row[at_ptr[3]:at_ptr[4]])
    assert dom.hi[4] == 0.0


def test_root_infeasibility_and_forced_values():
    # x0 + x1 >= 2 and x0 + x1 <= 1 with binaries: infeasible at the root
    lp = _mip([[1, 1], [1, 1]], [2, 1], "GL", [1, 1], [0, 0], [1, 1], [1, 1])
    st, _, nodes, _ = F.fp_search(lp, [0.5, 0.5], None, lp.is_int, F.FRAC, 1)
    assert st == F.INFEASIBLE and nodes == 0
    # x0 - x1 = 0 and x0 + x1 >= 1: whatever the first fixing, the search ends at (1, 1)
    lp = _mip([[1, -1], [1, 1]], [0, 1], "EG", [1, 1], [0, 0], [1, 1], [1, 1])
    for seed in range(20):
        st, dom, nodes, _ = F.fp_search(lp, [0.4, 0.4], None, lp.is_int, F.FRAC, seed)
        assert st == F.FEASIBLE and dom.lo[:2] == [1.0, 1.0] and nodes == 1


@pytest.mark.parametrize("seed", range(6))
def test_oracle_heuristic_returns_feasible_points(seed):
    """On small random MIPs every FEASIBLE answer satisfies the rows (1e-6 relative),
    the bounds and integrality, and is no better than the exact MIP optimum (scipy milp)."""
    from scipy.optimize import LinearConstraint, Bounds, milp
    lp = lpgen.mip_relaxation(100 + seed, m=12, n=16, density=0.3)
    r = O.solve(lp, O.Params(tol=1e-6))
    a = lp.dense()
    opt = milp(lp.c, constraints=LinearConstraint(a, -np.inf, lp.b), integrality=lp.is_int,
               bounds=Bounds(lp.l, lp.u))
    assert opt.status == 0
    for strategy in (F.FRAC, F.REDCOST, F.DUAL, F.TYPE):
        res = F.fp_run(lp, r.x, r.y, lp.is_int, strategy, seed=seed)
        if res.status != F.FEASIBLE:
            continue
        x = res.x
        assert np.all(a @ x <= lp.b + 1e-6 * np.maximum(1, np.abs(lp.b)))
        assert np.all(x >= lp.l - 1e-9) and np.all(x <= lp.u + 1e-9)
        xi = x[lp.is_int == 1]
        np.testing.assert_array_equal(xi, np.round(xi))
        assert res.obj >= opt.fun - 1e-6 * (1 + abs(opt.fun))


# ---------------------------------------------------------------- C ABI parity
@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


STRATEGY_IDS = {"frac": F.FRAC, "redcost": F.REDCOST, "dual": F.DUAL, "type": F.TYPE,
                "frac_dual": F.FRAC_DUAL, "frac_redcost": F.FRAC_REDCOST,
                "dual_frac": F.DUAL_FRAC, "redcost_frac": F.REDCOST_FRAC}


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("strategy", list(STRATEGY_IDS))
def test_cabi_search_matches_oracle(P, seed, strategy):
    """fp_run (final_lp = 0) takes exactly the oracle's decisions: the same integer
    assignment, node and backtrack counts and status, on 200 x 400 MIP relaxations."""
    lp = lpgen.mip_relaxation(seed)
    r = O.solve(lp, O.Params(tol=1e-4))
    sid = STRATEGY_IDS[strategy]
    for draw_seed in (1, 99):
        st, dom, nodes, backtracks = F.fp_search(lp, r.x, r.y, lp.is_int, sid, draw_seed)
        x, res = P.fp_run(lp, r.x, r.y, strategy=strategy, seed=draw_seed, final_lp=False)
        want = F.NO_FINAL_LP if st == F.FEASIBLE else st
        assert res["status"] == want
        assert res["nodes"] == nodes and res["backtracks"] == backtracks
        if st == F.FEASIBLE:
            ints = lp.is_int == 1
            np.testing.assert_array_equal(x[ints], np.array(dom.lo)[ints])


def _mixed_lp(seed):
    """Mixed-sense LP with free columns, half of the boxed columns integer."""
    lp = lpgen.random_sparse_lp(seed, 60, 90, density=0.08)
    ints = np.random.default_rng(seed).random(lp.n) < 0.5
    lp.is_int = (ints & np.isfinite(lp.l) & np.isfinite(lp.u)).astype(np.uint8)
    return lp


@pytest.mark.parametrize("maker", [lambda: lpgen.set_cover_fixed(20, 150), lambda: _mixed_lp(30),
                                   lambda: lpgen.mip_relaxation(5, m=120, n=240, density=0.04)],
                         ids=["cover_fixed", "mixed_free_eq", "denser_relaxation"])
@pytest.mark.parametrize("strategy", ["frac", "dual", "frac_dual", "dual_frac", "frac_redcost",
                                      "redcost_frac"])
def test_cabi_search_matches_oracle_on_other_shapes(P, maker, strategy):
    """The same node-for-node agreement on covering sub-LPs (fixed columns, >=-rows), mixed
    senses with free continuous columns, and a denser relaxation (the row filter of the
    C++ search, which skips rows whose slack covers every range, must not change a decision)."""
    lp = maker()
    r = O.solve(lp, O.Params(tol=1e-4, iter_limit=20000))
    sid = STRATEGY_IDS[strategy]
    for draw_seed in (1, 7):
        st, dom, nodes, backtracks = F.fp_search(lp, r.x, r.y, lp.is_int, sid, draw_seed)
        x, res = P.fp_run(lp, r.x, r.y, strategy=strategy, seed=draw_seed, final_lp=False)
        assert res["status"] == (F.NO_FINAL_LP if st == F.FEASIBLE else st)
        assert res["nodes"] == nodes and res["backtracks"] == backtracks
        if st == F.FEASIBLE:
            ints = lp.is_int == 1
            np.testing.assert_array_equal(x[ints], np.array(dom.lo)[ints])


def test_cabi_rejects_bad_arguments(P):
    lp, x, y = hand_mip()
    with pytest.raises(P.PdlpError, match="need y_lp"):
        P.fp_run(lp, x, None, strategy="dual", final_lp=False)  # Dual needs y
    with pytest.raises(P.PdlpError, match="unknown var_strategy"):
        P.fp_run(lp, x, y, strategy=8, final_lp=False)
    with pytest.raises(P.PdlpError, match="need y_lp"):
        P.fp_run(lp, x, None, strategy="frac_redcost", final_lp=False)
    with pytest.raises(P.PdlpError, match="nrefs >= 1"):
        P.fp_run_refs(lp, [], y, final_lp=False)


def tight_mip(seed, m=30, n=40):
    """0/1 MIP with slack below 0.5 and 30 % equality rows: the search backtracks."""
    rng = np.random.default_rng(seed)
    a = rng.integers(-3, 4, size=(m, n)).astype(float) * (rng.random((m, n)) < 0.25)
    x0 = rng.integers(0, 2, size=n).astype(float)
    sense = np.where(rng.random(m) < 0.3, ord("E"), ord("L")).astype(np.uint8)
    b = a @ x0 + np.where(sense == ord("E"), 0.0, rng.uniform(0, 0.5, size=m))
    rows, cols = np.nonzero(a)
    return lpgen._lp(m, n, rows, cols, a[rows, cols], b, sense, rng.uniform(-1, 1, size=n),
                     np.zeros(n), np.ones(n), np.ones(n, np.uint8), f"tight({seed})")


@pytest.mark.parametrize("seed", range(12))
def test_cabi_backtracking_matches_oracle(P, seed):
    lp = tight_mip(seed)
    r = O.solve(lp, O.Params(tol=1e-4, iter_limit=20000))
    total_bt = 0
    for sid, name in ((F.FRAC, "frac"), (F.REDCOST, "redcost"), (F.DUAL, "dual"), (F.TYPE, "type")):
        for limit in (0, 3):
            st, dom, nodes, bt = F.fp_search(lp, r.x, r.y, lp.is_int, sid, 5, node_limit=limit)
            x, res = P.fp_run(lp, r.x, r.y, strategy=name, seed=5, node_limit=limit, final_lp=False)
            assert res["status"] == (F.NO_FINAL_LP if st == F.FEASIBLE else st)
            assert res["nodes"] == nodes and res["backtracks"] == bt
            if st == F.FEASIBLE:
                np.testing.assert_array_equal(x, np.array(dom.lo))
            total_bt += bt
    if seed in (1, 3):
        assert total_bt > 0  # these instances do backtrack


def test_exhausted_search_is_infeasible(P):
    """x0 + x1 = 1 and x0 - x1 = 0: the LP point (0.5, 0.5) is feasible, no 0/1 point is;
    both branches of the first node fail, the search is exhausted."""
    lp = _mip([[1, 1], [1, -1]], [1, 0], "EE", [1, 1], [0, 0], [1, 1], [1, 1])
    st, _, nodes, bt = F.fp_search(lp, [0.5, 0.5], None, lp.is_int, F.FRAC, 3)
    assert st == F.INFEASIBLE and nodes == 1 and bt == 1
    x, res = P.fp_run(lp, [0.5, 0.5], None, strategy="frac", seed=3, final_lp=False)
    assert res["status"] == P.FP_INFEASIBLE and res["nodes"] == 1 and res["backtracks"] == 1


# ------------------------------------------------------- several reference points
def test_recorded_check_points_are_the_iterates_of_shorter_runs():
    """The oracle keeps the current point of the last checks; each is the current point of
    a run stopped at that check (the same steps, no termination test)."""
    lp = lpgen.mip_relaxation(2)
    r = O.solve(lp, O.Params(tol=1e-4, record_checks=3))
    k_last = r.iters // 64
    assert len(r.check_points) == 3
    for back, x in enumerate(reversed(r.check_points)):
        k = k_last - back
        ref = O.solve(lp, O.Params(iter_limit=64 * k, terminate=False))
        np.testing.assert_array_equal(x, ref.x_cur)


def test_fp_run_refs_keeps_the_best_feasible_run():
    lp = lpgen.mip_relaxation(5)
    r = O.solve(lp, O.Params(tol=1e-4, record_checks=4))
    runs = [F.fp_run(lp, x, r.y, lp.is_int, F.FRAC, 1, final_tol=1e-6) for x in r.check_points]
    best, i = F.fp_run_refs(lp, r.check_points, r.y, lp.is_int, F.FRAC, 1, final_tol=1e-6)
    objs = [q.obj if q.status == F.FEASIBLE else np.inf for q in runs]
    assert i == int(np.argmin(objs)) and best.obj == min(objs)
    # one reference is fp_run itself
    one, j = F.fp_run_refs(lp, [r.x], r.y, lp.is_int, F.FRAC, 1, final_tol=1e-6)
    direct = F.fp_run(lp, r.x, r.y, lp.is_int, F.FRAC, 1, final_tol=1e-6)
    assert j == (0 if direct.status == F.FEASIBLE else -1) and one.obj == direct.obj


def test_fp_run_refs_ties_go_to_the_earlier_point():
    # the same point twice: equal objectives, the first reference is kept
    lp = lpgen.mip_relaxation(5)
    r = O.solve(lp, O.Params(tol=1e-4))
    best, i = F.fp_run_refs(lp, [r.x, r.x.copy()], r.y, lp.is_int, F.FRAC, 1, final_tol=1e-6)
    assert best.status == F.FEASIBLE and i == 0


def test_cabi_refs_without_final_lp_returns_the_last_run(P):
    """Without the final LP no run is declared feasible: fp_run_refs reports index -1 and
    the last reference's search (the same as fp_run from it)."""
    lp = lpgen.mip_relaxation(3)
    r = O.solve(lp, O.Params(tol=1e-4, record_checks=2))
    x, res, k = P.fp_run_refs(lp, r.check_points, r.y, strategy="dual", final_lp=False)
    x1, res1 = P.fp_run(lp, r.check_points[-1], r.y, strategy="dual", final_lp=False)
    assert k == -1 and res["status"] == res1["status"] and res["nodes"] == res1["nodes"]
    ints = lp.is_int == 1
    np.testing.assert_array_equal(x[ints], x1[ints])
