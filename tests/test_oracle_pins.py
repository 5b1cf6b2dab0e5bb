"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a hand-computed worked example,
a closed form, an exact brute-force optimum, an independent library solver
(HiGHS), or an invariant of the LP.  Together they are chosen so that a
plausible slip in the oracle (a dropped extrapolation term, a wrong dual sign,
a transposed operand, a wrong bound term in the dual objective) fails at least
one of them; ``test_oracle_mutants.py`` plants such slips to show it.
"""
import math

import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from oracle import reference_lp as R

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _lp_from_dense(a, b, sense, c, l, u):
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    rows, cols = np.nonzero(a)
    return lpgen._lp(m, n, rows, cols, a[rows, cols], np.asarray(b, float),
                     np.array([ord(s) for s in sense], dtype=np.uint8), np.asarray(c, float),
                     np.asarray(l, float), np.asarray(u, float), np.zeros(n, np.uint8), "hand")


# ---------------------------------------------------------------- worked example
def _two_by_two():
    # row 0: -x0 - 2 x1 <= -1  (canonical: x0 + 2 x1 >= 1)
    # row 1:  3 x0 + 4 x1  = 2
    return _lp_from_dense([[-1, -2], [3, 4]], [-1, 2], "LE", [1, -1], [0, 0], [10, 1.2])


NOSCALE = dict(ruiz_iters=0, pc_alpha=None, restarts=False, terminate=False)


def test_one_pdhg_step_by_hand():
    """One PDHG step (A4/A5) with eta = 0.1, omega = 2, worked by hand.

    x = (1, 1), y_K = (0.5, 1)  [caller convention y = (-0.5, 1)]; tau = 0.05, sigma = 0.2
    K^T y = (1*0.5 + 3*1, 2*0.5 + 4*1) = (3.5, 5);  c - K^T y = (-2.5, -6)
    x - tau g = (1.125, 1.3) -> clip to u = (10, 1.2) -> x' = (1.125, 1.2)
    2x' - x = (1.25, 1.4);  K(2x' - x) = (1.25 + 2.8, 3.75 + 5.6) = (4.05, 9.35)
    q - that = (-3.05, -7.35);  y + sigma (...) = (0.5 - 0.61, 1 - 1.47) = (-0.11, -0.47)
    row 0 is an inequality -> max(-0.11, 0) = 0; row 1 is free -> -0.47
    y_K' = (0, -0.47) -> caller convention (-0, -0.47)
    """
    lp = _two_by_two()
    r = O.solve(lp, O.Params(iter_limit=1, adaptive=False, fixed_eta=0.1, fixed_omega=2.0,
                             **NOSCALE), x0=[1.0, 1.0], y0=[-0.5, 1.0])
    assert r.iters == 1
    np.testing.assert_allclose(r.x_cur, [1.125, 1.2], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.y_cur, [0.0, -0.47], rtol=0, atol=1e-15)
    # the average of a single accepted iterate is that iterate
    np.testing.assert_allclose(r.x_avg, r.x_cur, rtol=0, atol=1e-15)


def test_adaptive_step_rule_by_hand():
    """A6 on the same step: dx = (0.125, 0.2), dy = (0 - 0.5, -0.47 - 1) = (-0.5, -1.47).

    K dx = (0.125 + 0.4, 0.375 + 0.8) = (0.525, 1.175)
    dy^T K dx = -0.2625 - 1.72725 = -1.98975 -> denominator 2 * 1.98975 = 3.9795
    numerator = 2 * (0.015625 + 0.04) + (0.25 + 2.1609) / 2 = 0.11125 + 1.20545 = 1.3167
    eta_bar = 1.3167 / 3.9795 = 0.33087071240...  >= eta = 0.1  -> accepted
    eta_next = min((1 - 2^-0.3) eta_bar, (1 + 2^-0.6) 0.1)
             = min(0.1877476 * 0.3308707, 0.1659754) = 0.0621201833692...
    """
    lp = _two_by_two()
    r = O.solve(lp, O.Params(iter_limit=1, adaptive=True, fixed_eta=0.1, fixed_omega=2.0,
                             **NOSCALE), x0=[1.0, 1.0], y0=[-0.5, 1.0])
    assert r.attempts == 1 and r.iters == 1
    assert r.eta == pytest.approx(0.06212018336920332, rel=1e-13)


def test_adaptive_step_rejects_large_eta_and_retries_from_the_same_point():
    """With eta = 50 (far above 1/||K~||) the first attempt is rejected.  The retry
    starts from the same (x, y), so the accepted iterate equals the one a run
    started directly with the retried step size produces (attempt counter aside)."""
    lp = lpgen.mip_relaxation(1)
    r = O.solve(lp, O.Params(iter_limit=1, fixed_eta=50.0, terminate=False))
    assert r.iters == 1 and r.attempts == 2
    rej = [t for t in r.trace if t[0] == "reject"]
    assert len(rej) == 1 and rej[0][2] == 50.0 and rej[0][3] < 50.0
    eta_retry = min((1 - 2 ** -0.3) * rej[0][3], (1 + 2 ** -0.6) * 50.0)
    r2 = O.solve(lp, O.Params(iter_limit=1, fixed_eta=eta_retry, adaptive=False,
                              terminate=False))
    np.testing.assert_array_equal(r.x_cur, r2.x_cur)
    np.testing.assert_array_equal(r.y_cur, r2.y_cur)


# ---------------------------------------------------------------- scaling
def test_ruiz_on_powers_of_four_gives_identity_exactly():
    """Ruiz on diag(4, 16, 64): r = s = (2, 4, 8) in the first pass, so K~ = I exactly,
    and every later pass and the Pock-Chambolle pass (unit row/column sums) keep it."""
    k = O.sp.csr_matrix(np.diag([4.0, 16.0, 64.0]))
    dr, dc = O.ruiz_pock_chambolle(k, 10, 1.0)
    np.testing.assert_array_equal(dr, [0.5, 0.25, 0.125])
    np.testing.assert_array_equal(dc, [0.5, 0.25, 0.125])
    kt = (O.sp.diags(dr) @ k @ O.sp.diags(dc)).toarray()
    np.testing.assert_array_equal(kt, np.eye(3))


def test_pock_chambolle_sums_by_hand():
    """PC (alpha=1) without Ruiz on [[1,0,3],[0,9,0],[2,0,2]]:
    row sums (4, 9, 4) -> D_r = (1/2, 1/3, 1/2); column sums (3, 9, 5) -> D_c = (1/sqrt3, 1/3, 1/sqrt5)."""
    k = O.sp.csr_matrix(np.array([[1.0, 0, 3], [0, 9, 0], [2, 0, 2]]))
    dr, dc = O.ruiz_pock_chambolle(k, 0, 1.0)
    np.testing.assert_allclose(dr, [0.5, 1 / 3, 0.5], rtol=1e-15)
    np.testing.assert_allclose(dc, [1 / math.sqrt(3), 1 / 3, 1 / math.sqrt(5)], rtol=1e-15)


def test_ruiz_zero_row_and_column_get_factor_one():
    k = O.sp.csr_matrix(np.array([[0.0, 0, 0], [0, 4, 0], [0, 0, 0]]))
    dr, dc = O.ruiz_pock_chambolle(k, 3, None)
    assert dr[0] == 1.0 and dr[2] == 1.0 and dc[0] == 1.0 and dc[2] == 1.0
    assert dr[1] * 4 * dc[1] == 1.0


# ---------------------------------------------------------------- KKT (Part I)
def test_kkt_by_hand_with_infinite_bounds():
    """min x0 + 2 x1 - x2  s.t. x0 + x1 + x2 >= 1; x0 free, x1 in [0, inf), x2 in [0, 2].
    At x = (1, 0, 0), y = 0.5: lambda = c - A^T y = (0.5, 1.5, -1.5).
    r_d = (|0.5| for the free column, 0, 0) -> ||r_d|| = 0.5, ||c|| = sqrt(6).
    primal = 1; dual = q y + l1 lambda1+ - u2 lambda2- = 0.5 + 0 - 2*1.5 = -2.5.
    rel_p = 0, rel_d = 0.5 / (1 + sqrt 6), rel_gap = 3.5 / (1 + 1 + 2.5)."""
    lp = _lp_from_dense([[1, 1, 1]], [1], "G", [1, 2, -1], [-np.inf, 0, 0], [np.inf, np.inf, 2])
    k = O.kkt_original(lp, [1.0, 0.0, 0.0], [0.5])
    assert k.primal_obj == 1.0 and k.dual_obj == -2.5
    assert k.rel_p == 0.0
    assert k.rel_d == pytest.approx(0.5 / (1 + math.sqrt(6)), rel=1e-15)
    assert k.rel_gap == pytest.approx(3.5 / 4.5, rel=1e-15)


def test_kkt_primal_residual_senses_by_hand():
    """x = (1, 1): row L: 2 <= 1 violated by 1; row G: 2 >= 3 violated by 1;
    row E: 2 = 2.5 off by 0.5 -> ||r_p|| = 1.5, ||q|| = ||(-1, 3, 2.5)||."""
    lp = _lp_from_dense([[1, 1], [1, 1], [1, 1]], [1, 3, 2.5], "LGE", [0, 0], [0, 0], [5, 5])
    k = O.kkt_original(lp, [1.0, 1.0], [0.0, 0.0, 0.0])
    assert k.r_p == pytest.approx(1.5, rel=1e-15)
    assert k.rel_p == pytest.approx(1.5 / (1 + math.sqrt(1 + 9 + 6.25)), rel=1e-15)


@pytest.mark.parametrize("maker", [lambda: lpgen.mip_relaxation(1),
                                   lambda: lpgen.random_sparse_lp(7, 40, 60),
                                   lambda: lpgen.random_sparse_lp(8, 30, 50, free_frac=0.2)])
def test_kkt_vanishes_at_highs_optimum(maker):
    """At HiGHS's primal-dual optimum all three relative measures are ~0.
    This pins the dual sign convention and the bound terms of the dual objective."""
    lp = maker()
    obj, x, y, lam = R.highs(lp)
    k = O.kkt_original(lp, x, y)
    assert k.rel_p < 1e-9 and k.rel_d < 1e-9 and k.rel_gap < 1e-9
    assert k.primal_obj == pytest.approx(obj, rel=1e-12)


# ---------------------------------------------------------------- exact optima
@pytest.mark.parametrize("seed", range(8))
def test_tiny_lp_matches_vertex_enumeration(seed):
    lp = lpgen.tiny_lp(seed, m=5 + seed % 2, n=4 + seed % 2, eq_rows=seed % 2)
    best, verts = R.vertex_enumeration(lp)
    r = O.solve(lp, O.Params(tol=1e-10, iter_limit=400_000))
    assert r.status == O.STATUS_OPTIMAL
    assert r.kkt.primal_obj == pytest.approx(best, rel=1e-7, abs=1e-7)
    if len(verts) == 1 or np.ptp(np.array(verts), axis=0).max() < 1e-9:
        np.testing.assert_allclose(r.x, verts[0], atol=1e-5)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mip_relaxation_matches_highs(seed):
    lp = lpgen.mip_relaxation(seed)
    obj, _, _, _ = R.highs(lp)
    r = O.solve(lp, O.Params(tol=1e-8))
    assert r.status == O.STATUS_OPTIMAL
    assert r.kkt.rel_kkt <= 1e-8
    assert abs(r.kkt.primal_obj - obj) / (1 + abs(obj)) < 1e-7


def test_random_lp_with_free_columns_matches_highs_primal_and_dual():
    lp = lpgen.random_sparse_lp(11, 30, 45, free_frac=0.15)
    obj, xh, yh, lamh = R.highs(lp)
    r = O.solve(lp, O.Params(tol=1e-10, iter_limit=500_000))
    assert r.status == O.STATUS_OPTIMAL
    assert abs(r.kkt.primal_obj - obj) / (1 + abs(obj)) < 1e-8
    # the oracle's dual is a dual optimum: its own KKT and HiGHS's objective agree
    assert abs(r.kkt.dual_obj - obj) / (1 + abs(obj)) < 1e-8


def test_small_energy_system_matches_highs():
    lp = lpgen.energy_system(hours=24, regions=5, lines=6, techs=3, thermal=2)
    obj, _, _, _ = R.highs(lp)
    r = O.solve(lp, O.Params(tol=1e-7, iter_limit=400_000))
    assert r.status == O.STATUS_OPTIMAL
    assert abs(r.kkt.primal_obj - obj) / (1 + abs(obj)) < 1e-5


# ---------------------------------------------------------------- closed forms
def test_no_row_lp_closed_form():
    """With no rows the LP separates: x_j = l_j if c_j > 0, u_j if c_j < 0, proj(0) if c_j = 0."""
    n = 6
    c = np.array([1.0, -2.0, 0.0, 3.0, -0.5, 0.0])
    l = np.array([-1.0, 0.0, 0.5, -3.0, 2.0, -4.0])
    u = np.array([1.0, 2.0, 1.0, 5.0, 7.0, -1.0])
    lp = lpgen._lp(0, n, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0), np.zeros(0),
                   np.zeros(0, np.uint8), c, l, u, np.zeros(n, np.uint8), "norows")
    r = O.solve(lp, O.Params(tol=1e-12))
    assert r.status == O.STATUS_OPTIMAL
    np.testing.assert_array_equal(r.x, [-1.0, 2.0, 0.5, -3.0, 7.0, -1.0])


# ---------------------------------------------------------------- invariants
def test_iterates_stay_in_bounds_and_cone_every_step():
    lp = lpgen.random_sparse_lp(3, 25, 40)
    is_eq = lp.sense == ord("E")
    for it in (1, 2, 3, 17, 64, 65, 200):
        r = O.solve(lp, O.Params(iter_limit=it, terminate=False))
        assert np.all(r.x_cur >= lp.l) and np.all(r.x_cur <= lp.u)
        assert np.all(r.x_avg >= lp.l - 1e-12) and np.all(r.x_avg <= lp.u + 1e-12)
        yle = r.y_cur[lp.sense == ord("L")]
        yge = r.y_cur[lp.sense == ord("G")]
        assert np.all(yle <= 0) and np.all(yge >= 0)
        assert r.y_cur[is_eq].size == is_eq.sum()


def test_weak_duality_at_convergence():
    lp = lpgen.mip_relaxation(4)
    r = O.solve(lp, O.Params(tol=1e-6))
    k = r.kkt
    # with primal/dual feasibility at 1e-6 the dual bound sits below the primal
    assert k.dual_obj <= k.primal_obj + 1e-5 * (1 + abs(k.primal_obj))


def test_row_and_column_rescaling_keeps_the_solution():
    """Scaling row i by p_i > 0 and substituting x_j = z_j * t_j leaves the LP optimum unchanged."""
    lp = lpgen.mip_relaxation(5, m=60, n=120, density=0.06)
    rng = np.random.default_rng(0)
    p = rng.uniform(0.1, 10, size=lp.m)
    t = rng.uniform(0.1, 10, size=lp.n)
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    lp2 = lpgen._lp(lp.m, lp.n, rows, lp.col, lp.val * p[rows] * t[lp.col], lp.b * p, lp.sense,
                    lp.c * t, lp.l / t, lp.u / t, lp.is_int, "rescaled")
    r1 = O.solve(lp, O.Params(tol=1e-8))
    r2 = O.solve(lp2, O.Params(tol=1e-8))
    assert r1.kkt.primal_obj == pytest.approx(r2.kkt.primal_obj, rel=1e-6)


@pytest.mark.parametrize("maker", [lambda: lpgen.mip_relaxation(1),
                                   lambda: lpgen.random_sparse_lp(11, 300, 500)],
                         ids=["relaxation1", "free_eq"])
def test_scaling_b_and_c_by_powers_of_two_scales_the_iterates_exactly(maker):
    """Right-hand side and bounds times beta, costs times gamma (powers of two, so every
    product is exact): in exact arithmetic PDLP's iterates become (beta x, gamma y) -- the
    primal weight's start ||c~|| / ||q~|| moves by gamma / beta, which keeps tau * (c - K^T y)
    and sigma * (q - K x) in step, and the step bound eta_bar (omega on dx, 1/omega on dy) is
    unchanged.  With scalings by powers of two the run is the same bit for bit (adaptive
    steps, restarts off: the restart metric's gap term does not scale with the others)."""
    lp = maker()
    beta, gamma = 8.0, 0.25
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    lp2 = lpgen._lp(lp.m, lp.n, rows, lp.col, lp.val, lp.b * beta, lp.sense, lp.c * gamma,
                    lp.l * beta, lp.u * beta, lp.is_int, "scaled")
    prm = O.Params(iter_limit=150, terminate=False, restarts=False)
    r1, r2 = O.solve(lp, prm), O.solve(lp2, prm)
    assert r2.attempts == r1.attempts and r2.omega == r1.omega * gamma / beta
    for a, b, f in ((r2.x_cur, r1.x_cur, beta), (r2.y_cur, r1.y_cur, gamma),
                    (r2.x_avg, r1.x_avg, beta), (r2.y_avg, r1.y_avg, gamma)):
        np.testing.assert_array_equal(a, f * b)


def test_restarts_and_primal_weight_by_hand():
    """A9/A10 worked by hand: min x s.t. x >= 1, x in [0, 10], no scaling, eta = 0.5, a check
    after every step.  KKT_w(z) = sqrt(w r_p^2 + r_d^2 / w + gap^2); r_d = 0 (finite bounds).
    z0 = (0, 0): KKT 1.
    it 1: z = (0, 0.5): r_p = 1, gap 0.5, KKT sqrt(1.25) = 1.118; average = current (tie ->
      current); 1 - 0 >= 0.36: artificial restart; dx = 0: w stays 1.
    it 2: z = (0, 1), KKT sqrt(2) = 1.414 > 0.8 * 1.118; 2 - 1 >= 0.72: artificial restart.
    it 3: z = (0, 1.5): lambda = -0.5 on the upper bound 10, dual obj 1.5 - 5, gap 3.5,
      KKT 3.64; no criterion (1 < 1.08): no restart.
    it 4: z = (0.25, 1.75), KKT 6.05; average since it 2 = (0.125, 1.625), KKT 4.83 -> the
      candidate; 4 - 2 >= 1.44: restart to the average; dx = 0.125, dy = 0.625 from the
      anchor (0, 1): w = exp(0.5 ln 5 + 0.5 ln 1) = sqrt(5).
    it 5: x = 0.125 + (0.5 / sqrt5) 0.625, y = 1.625 + 0.5 sqrt5 (1 - (2x - 0.125))."""
    lp = _lp_from_dense([[1.0]], [1.0], "G", [1.0], [0.0], [10.0])
    r = O.solve(lp, O.Params(iter_limit=5, check_period=1, adaptive=False, fixed_eta=0.5,
                             ruiz_iters=0, pc_alpha=None, terminate=False))
    s5 = math.sqrt(5.0)
    kinds = [k for k, _ in r.check_trace]
    omegas = [w for _, w in r.check_trace]
    assert kinds == [1, 1, 0, 2, 0] and r.restarts == 3
    assert omegas[:3] == [1.0, 1.0, 1.0]
    assert omegas[3] == pytest.approx(s5, rel=1e-15) and omegas[4] == omegas[3]
    x5 = 0.125 + (0.5 / s5) * 0.625
    y5 = 1.625 + 0.5 * s5 * (1.0 - (2.0 * x5 - 0.125))
    assert r.x_cur[0] == pytest.approx(x5, rel=1e-14)
    assert r.y_cur[0] == pytest.approx(y5, rel=1e-14)


def test_sufficient_decay_restart_by_hand():
    """A9's sufficient-decay rule worked by hand: min x s.t. x >= 1, x in [0, inf), no
    scaling, eta = 1, a check after every step; r_d = lambda^- (u infinite).
    it 1: z = (0, 1), KKT sqrt(1 + 1) (r_p 1, gap 1): artificial restart (1 >= 0.36).
    it 2: z = (0, 2), lambda = -1: KKT sqrt(1 + 1 + 4) = 2.449: artificial restart (1 >= 0.72).
    it 3: z = (1, 1), the optimum: KKT 0.  The artificial rule does not fire (1 < 1.08) and
      the necessary one needs a previous candidate (there is none after a restart), so only
      sufficient decay (0 <= 0.2 * 2.449) restarts; dx = dy = 1 from the anchor (0, 2):
      w = exp(0.5 ln 1 + 0.5 ln 1) = 1.
    it 4: the last step, (1, 1) again."""
    lp = _lp_from_dense([[1.0]], [1.0], "G", [1.0], [0.0], [np.inf])
    r = O.solve(lp, O.Params(iter_limit=4, check_period=1, adaptive=False, fixed_eta=1.0,
                             ruiz_iters=0, pc_alpha=None, terminate=False))
    assert [k for k, _ in r.check_trace] == [1, 1, 1, 0] and r.restarts == 3
    assert all(w == 1.0 for _, w in r.check_trace)
    assert r.x_cur.tolist() == [1.0] and r.y_cur.tolist() == [1.0]


def test_necessary_decay_restart_by_hand():
    """A9's necessary-decay rule worked by hand (the artificial rule moved out of the way,
    beta_art = 1, so only the first check restarts by it): min 2x s.t. x >= 2, x in [0, 4],
    no scaling, w0 = ||c|| / ||q|| = 1, eta = 0.5, a check after every step;
    KKT = sqrt(r_p^2 + gap^2) (finite bounds: r_d = 0), dual obj 2y - 4 max(y - 2, 0).
    it 1: z = (0, 1), KKT sqrt(8): first check, restart; anchor (0, 1), last KKT 2.828.
    it 2: z = (0, 2), KKT sqrt(20) = 4.47: no rule (> 0.8 * 2.828 = 2.26).
    it 3: z = (0, 3), KKT sqrt(8) = 2.83 (average (0, 2.5): 3.61): no rule.
    it 4: z = (0.5, 3.5), KKT 1.5 <= 2.26 but below the previous candidate 2.83: no restart.
    it 5: z = (1.25, 3.5), KKT sqrt(2.8125) = 1.68 (average (0.4375, 3): 1.93): <= 2.26 and
      above the previous candidate 1.5: necessary decay restarts (sufficient decay would
      need <= 0.57); dx = 1.25, dy = 2.5 from the anchor: w = exp(0.5 ln 2 + 0.5 ln 1)."""
    lp = _lp_from_dense([[1.0]], [2.0], "G", [2.0], [0.0], [4.0])
    r = O.solve(lp, O.Params(iter_limit=6, check_period=1, adaptive=False, fixed_eta=0.5,
                             ruiz_iters=0, pc_alpha=None, terminate=False, beta_art=1.0))
    assert [k for k, _ in r.check_trace] == [1, 0, 0, 0, 1, 0] and r.restarts == 2
    assert r.check_trace[4][1] == pytest.approx(math.sqrt(2.0), rel=1e-15)


def test_looser_tolerance_never_needs_more_iterations():
    lp = lpgen.mip_relaxation(6)
    its = [O.solve(lp, O.Params(tol=t)).iters for t in (1e-2, 1e-4, 1e-6, 1e-8)]
    assert its == sorted(its)


def test_fixed_step_mode_accepts_every_attempt():
    lp = lpgen.mip_relaxation(1)
    r = O.solve(lp, O.Params(iter_limit=100, adaptive=False, restarts=False, terminate=False))
    assert r.iters == r.attempts == 100 and r.restarts == 0


def test_average_is_step_size_weighted():
    """A7: with the adaptive rule the two accepted steps use different step sizes
    eta_1 (given) and eta_2 (chosen after step 1); the average after two steps
    is (eta_1 x_1 + eta_2 x_2) / (eta_1 + eta_2), x_1 and x_2 taken from runs
    stopped after one and two iterations."""
    lp = lpgen.mip_relaxation(2)
    p1 = O.Params(iter_limit=1, fixed_eta=0.05, terminate=False, restarts=False)
    p2 = O.Params(iter_limit=2, fixed_eta=0.05, terminate=False, restarts=False)
    r1 = O.solve(lp, p1)
    r2 = O.solve(lp, p2)
    assert r1.attempts == 1 and r2.attempts == 2  # no rejection in either step
    eta1, eta2 = 0.05, r1.eta
    assert abs(eta2 - eta1) > 1e-3 * eta1
    expect = (eta1 * r1.x_cur + eta2 * r2.x_cur) / (eta1 + eta2)
    np.testing.assert_allclose(r2.x_avg, expect, rtol=1e-12, atol=1e-12)


def test_step_growth_when_eta_bar_is_infinite():
    """With no rows dy = 0, so dy^T K dx = 0 and eta_bar = inf: every attempt is
    accepted and eta grows by (1 + (k+1)^-0.6) per step (A6).
    From eta = 1: after one step 1 + 2^-0.6 = 1.6597539553864471; after two,
    (1 + 2^-0.6)(1 + 3^-0.6) = 1.6597539553864471 * 1.5172818579717866
    (3^0.6 = e^(0.6 ln 3) = e^0.6591674 = 1.9331820...)."""
    n = 3
    lp = lpgen._lp(0, n, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0), np.zeros(0),
                   np.zeros(0, np.uint8), np.array([1.0, -1.0, 0.5]), np.full(n, -1e3),
                   np.full(n, 1e3), np.zeros(n, np.uint8), "norows")
    r1 = O.solve(lp, O.Params(iter_limit=1, fixed_eta=1.0, terminate=False, restarts=False))
    r2 = O.solve(lp, O.Params(iter_limit=2, fixed_eta=1.0, terminate=False, restarts=False))
    assert r1.eta == pytest.approx(1.6597539553864471, rel=1e-15)
    assert r2.eta == pytest.approx(1.6597539553864471 * 1.5172818579717866, rel=1e-14)


def test_replaying_the_own_trace_reproduces_the_run():
    """The replay mode (step sizes and accept flags from a trace) is a pure
    substitution: replaying a run's own trace gives the same run bit for bit."""
    lp = lpgen.mip_relaxation(3)
    r = O.solve(lp, O.Params(iter_limit=700, terminate=False))
    eta = [t[0] for t in r.attempt_trace]
    acc = [t[2] for t in r.attempt_trace]
    r2 = O.solve(lp, O.Params(iter_limit=700, terminate=False, replay_eta=eta, replay_accepted=acc))
    assert r2.attempts == r.attempts and r2.restarts == r.restarts
    np.testing.assert_array_equal(r2.x_cur, r.x_cur)
    np.testing.assert_array_equal(r2.y_avg, r.y_avg)
    assert r2.check_trace == r.check_trace


def test_primal_weight_hint_by_hand():
    """K = I on two >=-rows: Ruiz and Pock-Chambolle leave D_r = D_c = I, so the hinted
    omega0 is the ratio of the projected hint's plain norms."""
    lp = _lp_from_dense(np.eye(2), [1.0, 1.0], "GG", [1.0, 1.0], [0.0, 0.0], [10.0, 4.0])
    k, _, _, _ = O.canonicalize(lp)
    dr, dc = O.ruiz_pock_chambolle(k)
    assert dr.tolist() == [1.0, 1.0] and dc.tolist() == [1.0, 1.0]
    fixed = dict(iter_limit=1, adaptive=False, restarts=False, terminate=False)
    # x = (3, 40) projects to (3, 4): norm 5; y = (-7, 10) projects to (0, 10): norm 10
    r = O.solve(lp, O.Params(omega_hint=(np.array([3.0, 40.0]), np.array([-7.0, 10.0])), **fixed))
    assert r.omega == 2.0
    # without a hint: ||c|| / ||b|| = 1; a hint with a zero part falls back to it
    assert O.solve(lp, O.Params(**fixed)).omega == 1.0
    r0 = O.solve(lp, O.Params(omega_hint=(np.zeros(2), np.array([0.0, 10.0])), **fixed))
    assert r0.omega == 1.0


# ---------------------------------------------------------------- exact non-identity scaling
# K = diag(4, 16): the first Ruiz pass takes r = s = (sqrt 4, sqrt 16) = (2, 4) from the same
# K~, so D_r = D_c = (1/2, 1/4) and K~ = I; every later pass and Pock-Chambolle (row and
# column sums of |K~| = 1) leave it there.  All of it is exact in floating point.
# K = [[1, 1], [1, 1]]: Ruiz keeps it (maxima 1); Pock-Chambolle divides rows and columns by
# sqrt(2), so K~ = [[1/2, 1/2], [1/2, 1/2]] up to one rounding of sqrt(2)^2.


def test_eta0_is_one_over_the_largest_scaled_entry_by_hand():
    """A3: eta0 = 1 / max |K~_ij| of the SCALED matrix, from the unforced start (no
    fixed_eta; with adaptive = False the step size stays eta0, which the result reports).
      diag(4, 16):  K~ = I                 -> eta0 = 1
                    (1/max|K| = 1/16, 1/||K~||_F = 1/sqrt 2: both wrong)
      ones(2, 2):   K~ = ones / 2          -> eta0 = 2
                    (1/||K~||_2 = 1, 1/||K~||_F = 1, 1/max|K| = 1: all wrong)"""
    fixed = dict(iter_limit=1, adaptive=False, restarts=False, terminate=False)
    lp = _lp_from_dense([[4.0, 0.0], [0.0, 16.0]], [1.0, 1.0], "GG", [1.0, 1.0], [0.0, 0.0],
                        [10.0, 10.0])
    k, _, _, _ = O.canonicalize(lp)
    dr, dc = O.ruiz_pock_chambolle(k)
    assert dr.tolist() == [0.5, 0.25] and dc.tolist() == [0.5, 0.25]
    assert O.solve(lp, O.Params(**fixed)).eta == 1.0
    lp = _lp_from_dense([[1.0, 1.0], [1.0, 1.0]], [1.0, 1.0], "GG", [1.0, 1.0], [0.0, 0.0],
                        [10.0, 10.0])
    assert O.solve(lp, O.Params(**fixed)).eta == pytest.approx(2.0, rel=1e-15)


def test_restart_metric_is_taken_in_scaled_space_by_hand():
    """A9 reads KKT_w on the SCALED iterate.  min 4x s.t. 4x >= 4, x in [0, 2]: K = [4]
    scales to K~ = [1] with D_r = D_c = 1/2 exactly, so q~ = 2, c~ = 2, u~ = 4, w0 =
    ||c~|| / ||q~|| = 1 -- in scaled space exactly the problem of
    test_necessary_decay_restart_by_hand (eta = 0.5, a check after every step, beta_art = 1),
    whose restarts are [1, 0, 0, 0, 1, 0] with w = sqrt 2 after the fifth check.
    In unscaled space r_p doubles (r_p = r_p~ / D_r) and the gap is unchanged, so the same
    checks would read: z1 = (0, 1): sqrt(16 + 4) = 4.47 (the restart anchor); z3 (0, 3):
    sqrt(16 + 4) = 4.47; z4 (0.5, 3.5): r_p 3, gap 0 -> 3 (<= 0.8 * 4.47 = 3.58 but below
    the previous 4.47); z5 (1.25, 3.5): r_p 1.5, gap 1.5 -> 2.12, below the previous
    candidate 3, so no necessary-decay restart there.  Unscaled, the returned iterate is
    x = D_c x~, y = D_r y~."""
    lp = _lp_from_dense([[4.0]], [4.0], "G", [4.0], [0.0], [2.0])
    k, _, _, _ = O.canonicalize(lp)
    assert [v.tolist() for v in O.ruiz_pock_chambolle(k)] == [[0.5], [0.5]]
    r = O.solve(lp, O.Params(iter_limit=6, check_period=1, adaptive=False, fixed_eta=0.5,
                             terminate=False, beta_art=1.0))
    assert [kd for kd, _ in r.check_trace] == [1, 0, 0, 0, 1, 0] and r.restarts == 2
    assert r.check_trace[4][1] == pytest.approx(math.sqrt(2.0), rel=1e-15)
    # z5 = (1.25, 3.5) scaled; the restart at check 5 keeps it, step 6 from it with
    # w = sqrt 2: x~ = 1.25 - (0.5 / sqrt 2)(2 - 3.5), y~ = 3.5 + 0.5 sqrt 2 (2 - (2 x~ - 1.25))
    s2 = math.sqrt(2.0)
    x6 = 1.25 - (0.5 / s2) * (2.0 - 3.5)
    y6 = 3.5 + 0.5 * s2 * (2.0 - (2.0 * x6 - 1.25))
    assert r.x_cur[0] == pytest.approx(0.5 * x6, rel=1e-14)
    assert r.y_cur[0] == pytest.approx(0.5 * y6, rel=1e-14)


def test_primal_weight_distances_are_taken_in_scaled_space_by_hand():
    """A10 measures the distances moved since the last restart in SCALED space.
    K = diag(4, 16) (D_r = D_c = (1/2, 1/4)), rows 4 x1 >= 0 and 16 x2 >= 8, c = (-2, 0),
    x in [0, 0.25] x [0, 1]: scaled q~ = (0, 2), c~ = (-1, 0), u~ = (0.5, 4), so
    w0 = ||c~|| / ||q~|| = 1/2; eta = 0.5 gives tau = eta / w = 1, sigma = eta w = 1/4.
      step 1 from 0: x~ = proj((0, 0) + (1, 0)) = (0.5, 0) (x1 at its bound);
                     y~ = proj_Y(0.25 ((0, 2) - (1, 0))) = (0, 0.5).
      check 1 (artificial restart, 1 >= 0.36; average = current): dx~ = 0.5, dy~ = 0.5,
        w1 = exp(0.5 ln(0.5 / 0.5) + 0.5 ln(1/2)) = sqrt(1/2).
        (Unscaled distances ||D_c dx~|| = 0.25, ||D_r dy~|| = 0.125 would give w = 1/2.)
      step 2, tau = 0.5 / w1 = sqrt(2)/2, sigma = sqrt(2)/4:
        x~ = proj((0.5, 0) - tau ((-1, 0) - (0, 0.5))) = (0.5, sqrt(2)/4),
        y~2 = 0.5 + sigma (2 - 2 sqrt(2)/4) = 0.25 + sqrt(2)/2, y~1 = max(0, -sigma/2) = 0.
      Unscaled: x = D_c x~ = (0.25, sqrt(2)/16), y = D_r y~ = (0, (0.25 + sqrt(2)/2)/4)."""
    lp = _lp_from_dense([[4.0, 0.0], [0.0, 16.0]], [0.0, 8.0], "GG", [-2.0, 0.0], [0.0, 0.0],
                        [0.25, 1.0])
    r1 = O.solve(lp, O.Params(iter_limit=1, check_period=1, adaptive=False, fixed_eta=0.5,
                              terminate=False))
    assert r1.x_cur.tolist() == [0.25, 0.0] and r1.y_cur.tolist() == [0.0, 0.125]
    r = O.solve(lp, O.Params(iter_limit=2, check_period=1, adaptive=False, fixed_eta=0.5,
                             terminate=False))
    s2 = math.sqrt(2.0)
    assert r.check_trace[0][0] == 1
    assert r.check_trace[0][1] == pytest.approx(math.sqrt(0.5), rel=1e-15)
    np.testing.assert_allclose(r.x_cur, [0.25, s2 / 16.0], rtol=1e-14, atol=0)
    np.testing.assert_allclose(r.y_cur, [0.0, (0.25 + s2 / 2.0) / 4.0], rtol=1e-14, atol=0)


# ---------------------------------------------------------------- A2b rescaling
def test_bound_objective_rescaling_one_step_by_hand():
    """A2b on min -3 x0 + 4 x1 s.t. x0 >= 1, x1 >= 0, x in [0, 10]^2 with K = I (no Ruiz,
    no Pock-Chambolle, so D = I): gamma = 1 + ||c|| = 6, beta = 1 + ||q|| = 2, the
    rescaled data c' = (-1/2, 2/3), q' = (1/2, 0), u' = 5, omega0' = ||c'|| / ||q'||
    = (5/6) / (1/2) = 5/3.  One step with eta = 1/2 from 0:
      x'1 = proj(0 - (0.5 / (5/3)) c') = proj(-0.3 c') = (0.15, 0),
      y'1 = proj_Y(0 + 0.5 (5/3) (q' - 2 x'1)) = (5/6)(0.2, 0) = (1/6, 0);
    unscaled x = beta x' = (0.3, 0), y = gamma y' = (1, 0) -- the unrescaled step with
    omega0 = ||c|| / ||q|| = 5 from 0 gives the same point."""
    lp = _lp_from_dense([[1.0, 0.0], [0.0, 1.0]], [1.0, 0.0], "GG", [-3.0, 4.0], [0.0, 0.0],
                        [10.0, 10.0])
    kw = dict(iter_limit=1, adaptive=False, fixed_eta=0.5, **NOSCALE)
    r = O.solve(lp, O.Params(bound_objective_rescaling=True, **kw))
    np.testing.assert_allclose(r.x_cur, [0.3, 0.0], rtol=1e-15, atol=0)
    np.testing.assert_allclose(r.y_cur, [1.0, 0.0], rtol=1e-15, atol=0)
    assert r.omega == pytest.approx(5.0 / 3.0, rel=1e-15)
    r0 = O.solve(lp, O.Params(**kw))
    np.testing.assert_allclose(r0.x_cur, r.x_cur, rtol=1e-15, atol=0)
    np.testing.assert_allclose(r0.y_cur, r.y_cur, rtol=1e-15, atol=0)
    assert r0.omega == pytest.approx(5.0, rel=1e-15)


@pytest.mark.parametrize("maker", [lambda: lpgen.mip_relaxation(2),
                                   lambda: lpgen.random_sparse_lp(3, 40, 60)])
def test_bound_objective_rescaling_is_the_same_pdhg_without_restarts(maker):
    """A2b changes the PDHG iteration only through the restart metric: with (x', y') =
    (x~ / beta, y~ / gamma) the step, the step bound eta_bar and the omega0 rule map onto
    the unrescaled ones with omega' = omega beta / gamma.  So with restarts off the
    adaptive runs take the same attempts and accept decisions and reach the same unscaled
    iterates (to the rounding the adaptive step amplifies), and the reported weights differ
    by beta / gamma exactly as the scaled norms give it."""
    lp = maker()
    kw = dict(iter_limit=60, restarts=False, terminate=False)
    r1 = O.solve(lp, O.Params(bound_objective_rescaling=True, **kw))
    r0 = O.solve(lp, O.Params(**kw))
    assert r1.iters == r0.iters == 60 and r1.attempts == r0.attempts
    assert [a[2] for a in r1.attempt_trace] == [a[2] for a in r0.attempt_trace]
    for a, b in ((r1.x_cur, r0.x_cur), (r1.y_cur, r0.y_cur), (r1.x_avg, r0.x_avg),
                 (r1.y_avg, r0.y_avg)):
        assert np.linalg.norm(a - b) <= 1e-9 * max(1.0, np.linalg.norm(b))
    k, q, _, _ = O.canonicalize(lp)
    dr, dc = O.ruiz_pock_chambolle(k)
    gamma = 1.0 + np.linalg.norm(dc * lp.c)
    beta = 1.0 + np.linalg.norm(dr * q)
    assert r1.omega == pytest.approx(r0.omega * beta / gamma, rel=1e-12)
    np.testing.assert_allclose([a[0] for a in r1.attempt_trace], [a[0] for a in r0.attempt_trace],
                               rtol=1e-9)


def test_bound_objective_rescaling_with_restarts_reaches_the_optimum():
    """With restarts the rescaled run is its own iteration (the restart metric weighs
    its gap term by 1 / (beta gamma)); it must still reach HiGHS's optimum."""
    lp = lpgen.mip_relaxation(1)
    r = O.solve(lp, O.Params(tol=1e-6, bound_objective_rescaling=True))
    assert r.status == O.STATUS_OPTIMAL and r.kkt.rel_kkt <= 1e-6
    obj, _, _, _ = R.highs(lp)
    assert abs(float(lp.c @ r.x) - obj) / (1 + abs(obj)) <= 1e-5


# ---------------------------------------------------------------- A14 Halpern
def _one_by_one():
    # min x  s.t.  x >= 1,  0 <= x (optimum x* = 1, y* = 1)
    return _lp_from_dense([[1.0]], [1.0], "G", [1.0], [0.0], [np.inf])


HALP = dict(ruiz_iters=0, pc_alpha=None, halpern=True, fixed_eta=0.5, fixed_omega=1.0,
            terminate=False)


def test_halpern_steps_by_hand():
    """Four reflected Halpern steps (rho = 1) on min x, x >= 1, eta = 0.5, omega = 1
    (tau = sigma = 0.5), from z^0 = (0, 0) = the anchor:
      k=0: T = (max(0 - 0.5*1, 0), 0 + 0.5*(1 - 0)) = (0, 0.5);  z1 = 1/2 (2T - z0) + 1/2 z0 = (0, 0.5)
      k=1: T = (max(0 - 0.5*0.5, 0), 0.5 + 0.5) = (0, 1);         z2 = 2/3 (0, 1.5) = (0, 1)
      k=2: T = (0, 1.5);                                           z3 = 3/4 (0, 2) = (0, 1.5)
      k=3: T = (0 + 0.5*0.5, 1.5 + 0.5*(1 - 0.5)) = (0.25, 1.75); z4 = 4/5 (0.5, 2) = (0.4, 1.6)
    Residuals ||z - T(z)||_P^2 = 2 dx^2 + 2 dy^2 - 2 dy dx: 0.5, 0.5, 0.5, then
    2/16 + 2/16 - 2/16 = 0.125."""
    r = O.solve(_one_by_one(), O.Params(iter_limit=4, restarts=False, **HALP))
    assert r.iters == 4 and r.attempts == 4
    np.testing.assert_allclose(r.x_cur, [0.25], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.y_cur, [1.75], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.x_halpern, [0.4], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.y_halpern, [1.6], rtol=0, atol=1e-15)
    np.testing.assert_allclose([t[1] for t in r.attempt_trace],
                               [math.sqrt(0.5)] * 3 + [math.sqrt(0.125)], rtol=1e-15)
    # no averages: the average candidate is the latest T(z^k)
    np.testing.assert_allclose(r.x_avg, r.x_cur, rtol=0, atol=0)


def test_plain_halpern_steps_by_hand():
    """rho = 0 (no reflection) on the same LP: z1 = 1/2 T(z0) = (0, 0.25);
    T(z1) = (max(0 - 0.5*(1 - 0.25), 0), 0.25 + 0.5) = (0, 0.75), z2 = 2/3 (0, 0.75) = (0, 0.5)."""
    r = O.solve(_one_by_one(), O.Params(iter_limit=2, restarts=False, halpern_reflection=0.0,
                                        **HALP))
    np.testing.assert_allclose(r.y_cur, [0.75], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.y_halpern, [0.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.x_halpern, [0.0], rtol=0, atol=1e-15)


def test_halpern_necessary_decay_restart_by_hand():
    """Checks after every step, the artificial rule out of reach (beta_art = 10).
    Residuals of the steps above: r = 0.7071 (r_0), 0.7071, 0.7071, 0.3536; step 5 from
    z4 = (0.4, 1.6): T = (0.4 + 0.5*0.6, 1.6 + 0.5*(1 - 1.0)) = (0.7, 1.6), r^2 = 2*0.09 = 0.18,
    r = 0.4243 <= 0.8 r_0 and above the previous check's 0.3536: a restart to (0.7, 1.6), with
    omega = exp(0.5 ln(1.6 / 0.7)) (distances from the anchor (0, 0)).  The sixth check is the
    iteration limit."""
    r = O.solve(_one_by_one(), O.Params(iter_limit=6, check_period=1, beta_art=10.0, **HALP))
    kinds = [k for k, _ in r.check_trace]
    assert kinds == [0, 0, 0, 0, 1, 0] and r.restarts == 1
    assert r.check_trace[4][1] == pytest.approx(math.sqrt(1.6 / 0.7), rel=1e-14)


def test_halpern_sufficient_decay_restart_by_hand():
    """beta_suff = 0.6: step 4's r = 0.3536 <= 0.6 * 0.7071 restarts to T(z3) = (0.25, 1.75);
    omega = exp(0.5 ln(1.75 / 0.25)) = sqrt(7).  Then, from the new anchor with
    tau = 0.5/sqrt(7), sigma = 0.5 sqrt(7), the first step of the epoch sets r_0 afresh."""
    r = O.solve(_one_by_one(), O.Params(iter_limit=5, check_period=1, beta_art=10.0,
                                        beta_suff=0.6, **HALP))
    assert [k for k, _ in r.check_trace][:4] == [0, 0, 0, 1]
    assert r.check_trace[3][1] == pytest.approx(math.sqrt(7.0), rel=1e-14)
    # step 5 starts from the anchor (0.25, 1.75): x' = 0.25 + tau*0.75, and with k = 0
    # z5 = 1/2 (2 T - z) + 1/2 z = T
    tau = 0.5 / math.sqrt(7.0)
    sigma = 0.5 * math.sqrt(7.0)
    xt = 0.25 + tau * 0.75
    yt = 1.75 + sigma * (1.0 - (2.0 * xt - 0.25))
    np.testing.assert_allclose(r.x_cur, [xt], rtol=1e-14)
    np.testing.assert_allclose(r.y_cur, [yt], rtol=1e-14)
    np.testing.assert_allclose(r.x_halpern, [xt], rtol=1e-14)
    np.testing.assert_allclose(r.y_halpern, [yt], rtol=1e-14)


def test_halpern_first_check_restarts_artificially():
    """check_period 2: at the first check (iteration 2) 2 - 0 >= 0.36 * 2 restarts to
    T(z1) = (0, 1) with omega unchanged (no primal distance); at iteration 4 the
    artificial rule (4 - 2 >= 1.44) restarts again, to T(z'1) where the epoch's first step
    T(0, 1) = (0, 1.5) and z'1 = 1/2 (2 (0, 1.5) - (0, 1)) + 1/2 (0, 1) = (0, 1.5), then
    T(z'1) = (0.25, 1.75): omega = exp(0.5 ln(0.75 / 0.25)) = sqrt(3)."""
    r = O.solve(_one_by_one(), O.Params(iter_limit=6, check_period=2, **HALP))
    assert [k for k, _ in r.check_trace] == [1, 1, 0]
    assert r.check_trace[0][1] == 1.0
    assert r.check_trace[1][1] == pytest.approx(math.sqrt(3.0), rel=1e-14)


def _diag_lp(d):
    n = len(d)
    return _lp_from_dense(np.diag(d), np.ones(n), "G" * n, np.ones(n), np.zeros(n),
                          np.full(n, np.inf))


def test_power_iteration_closed_forms():
    """||diag(2, 1)||_2 = 2 and ||u v^T||_2 = ||u|| ||v|| (rank one: exact after one
    pass); the power estimate never exceeds the true norm (LAPACK's 2-norm as the
    independent check) and the Halpern step is 0.998 / L."""
    import scipy.sparse as sps
    assert O.power_norm(sps.csr_matrix(np.diag([2.0, 1.0]))) == pytest.approx(2.0, rel=1e-14)
    u = np.array([1.0, 2.0, 2.0])
    v = np.array([3.0, 4.0])
    assert O.power_norm(sps.csr_matrix(np.outer(u, v))) == pytest.approx(15.0, rel=1e-14)
    rng = np.random.default_rng(5)
    for _ in range(5):
        a = sps.random(30, 20, density=0.2, random_state=rng, format="csr")
        true = np.linalg.norm(a.toarray(), 2)
        est = O.power_norm(a)
        assert est <= true * (1 + 1e-12) and est >= 0.9 * true
    r = O.solve(_diag_lp([2.0, 1.0]), O.Params(iter_limit=1, ruiz_iters=0, pc_alpha=None,
                                               halpern=True, terminate=False))
    assert r.spectral_norm == pytest.approx(2.0, rel=1e-14)
    assert r.eta == pytest.approx(0.998 / 2.0, rel=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_halpern_tiny_lp_matches_vertex_enumeration(seed):
    lp = lpgen.tiny_lp(seed, m=5 + seed % 2, n=4 + seed % 2, eq_rows=seed % 2)
    best, _ = R.vertex_enumeration(lp)
    r = O.solve(lp, O.Params(tol=1e-9, iter_limit=400_000, halpern=True))
    assert r.status == O.STATUS_OPTIMAL
    assert r.kkt.primal_obj == pytest.approx(best, rel=1e-6, abs=1e-6)


def test_halpern_mip_relaxation_matches_highs():
    lp = lpgen.mip_relaxation(2)
    obj, _, _, _ = R.highs(lp)
    r = O.solve(lp, O.Params(tol=1e-8, halpern=True))
    assert r.status == O.STATUS_OPTIMAL
    assert abs(r.kkt.primal_obj - obj) / (1 + abs(obj)) < 1e-7


# ---------------------------------------------------------------- A9b normalized duality gap
def _tr(gx, gy, x, y, lt, ut, is_eq, omega, r):
    f = lambda v: np.asarray(v, dtype=float)
    return O.trust_region_gap(f(gx), f(gy), f(x), f(y), f(lt), f(ut), np.asarray(is_eq, bool),
                              omega, r)[0]


def test_trust_region_gap_closed_forms():
    """Without active bounds the maximum of g^T d over ||d||_omega <= r is r times the dual
    norm sqrt(||g_x||^2 / omega + omega ||g_y||^2); a box that caps every direction inside
    the ball gives the box maximum; on [0, 1]^2 with g = (3, 4), omega = 1: r = 1 -> 5
    (interior), r = 1.3 -> b = 1, a = sqrt(1.69 - 1): 3 sqrt(0.69) + 4."""
    inf = np.inf
    v = _tr([1.0, -2.0], [0.5], [0.3, 0.1], [0.2], [-inf, -inf], [inf, inf], [True], 2.5, 0.7)
    assert v == pytest.approx(0.7 * math.sqrt((1 + 4) / 2.5 + 2.5 * 0.25), rel=1e-12)
    assert _tr([2.0], [], [0.0], [], [0.0], [1.0], [], 1.0, 5.0) == pytest.approx(2.0, rel=1e-12)
    assert _tr([3.0, 4.0], [], [0.0, 0.0], [], [0.0, 0.0], [1.0, 1.0], [], 1.0, 1.0) == \
        pytest.approx(5.0, rel=1e-12)
    assert _tr([3.0, 4.0], [], [0.0, 0.0], [], [0.0, 0.0], [1.0, 1.0], [], 1.0, 1.3) == \
        pytest.approx(3.0 * math.sqrt(0.69) + 4.0, rel=1e-12)
    # an inequality row's dual cannot go below 0: y = 0.5, g_y = -2 moves y to 0 at most
    assert _tr([], [-2.0], [], [0.5], [], [], [False], 1.0, 3.0) == pytest.approx(1.0, rel=1e-12)
    assert _tr([1.0], [2.0], [0.0], [0.0], [0.0], [1.0], [False], 1.0, 0.0) == 0.0


def test_trust_region_gap_matches_an_independent_solver():
    """Random boxes, cones, omega != 1: the bisection's maximum against SLSQP's on the
    same problem (maximise g^T d subject to the bounds and the omega-ball)."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(11)
    for trial in range(12):
        n, m = 3, 2
        omega = float(rng.uniform(0.3, 3.0))
        x = rng.uniform(-1, 1, n)
        lt = x - rng.uniform(0.0, 0.6, n)
        ut = x + rng.uniform(0.0, 0.6, n)
        lt[0], ut[1] = -np.inf, np.inf
        is_eq = np.array([trial % 2 == 0, False])
        y = np.where(is_eq, rng.normal(size=m), rng.uniform(0, 0.5, m))
        gx, gy = rng.normal(size=n), rng.normal(size=m)
        r = float(rng.uniform(0.2, 1.5))
        got = _tr(gx, gy, x, y, lt, ut, is_eq, omega, r)
        z0 = np.concatenate([x, y])
        lo = np.concatenate([lt, np.where(is_eq, -np.inf, 0.0)])
        hi = np.concatenate([ut, np.full(m, np.inf)])
        g = np.concatenate([gx, gy])
        w = np.concatenate([np.full(n, omega), np.full(m, 1.0 / omega)])
        cons = [{"type": "ineq", "fun": lambda z: r * r - float(w @ (z - z0) ** 2)}]
        bnds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
                for a, b in zip(lo, hi)]
        res = minimize(lambda z: -float(g @ (z - z0)), z0, jac=lambda z: -g, bounds=bnds,
                       constraints=cons, method="SLSQP", options={"ftol": 1e-12, "maxiter": 1000})
        zs = res.x
        # SLSQP's point is feasible (to 1e-9) and no better than the bisection's maximum
        assert float(w @ (zs - z0) ** 2) <= r * r * (1 + 1e-9)
        assert np.all(zs >= lo - 1e-9) and np.all(zs <= hi + 1e-9)
        assert got == pytest.approx(-res.fun, rel=1e-6, abs=1e-9)


def test_normalized_gap_by_hand():
    """min x s.t. x >= 1 (K = 1, q = 1, c = 1), omega = 1, from the restart point (0, 1):
    the current point (0.25, 1.75) is r = sqrt(0.625) away with g = (y - c, q - x) =
    (0.75, 0.75); nothing binds, so rho = ||g|| = 0.75 sqrt(2).  The point (0.125, 1.625):
    g = (0.625, 0.875), rho = sqrt(0.625^2 + 0.875^2).  With omega = 4 the gradient norm
    is sqrt(g_x^2 / 4 + 4 g_y^2).  At the restart point itself r = 0: rho = 0."""
    import scipy.sparse as sps
    kt = sps.csr_matrix(np.array([[1.0]]))
    args = (kt, kt.T.tocsr(), np.array([1.0]), np.array([1.0]), np.array([0.0]),
            np.array([np.inf]), np.array([False]))
    g = lambda om, xs, ys: O.normalized_gap(*args, om, np.array([xs]), np.array([ys]),
                                            np.array([0.0]), np.array([1.0]))
    assert g(1.0, 0.25, 1.75) == pytest.approx(0.75 * math.sqrt(2.0), rel=1e-12)
    assert g(1.0, 0.125, 1.625) == pytest.approx(math.hypot(0.625, 0.875), rel=1e-12)
    assert g(4.0, 0.25, 1.75) == pytest.approx(math.sqrt(0.75 ** 2 / 4 + 4 * 0.75 ** 2), rel=1e-12)
    assert g(1.0, 0.0, 1.0) == 0.0
    # omega = 4 with x <= 0.3 binding: r^2 = 4 (0.25)^2 + (0.75)^2 / 4 = 0.390625; x moves
    # 0.1875 t and stops at 0.3 (dx = 0.05), y moves 3 t; the ball then gives
    # 4 (0.05)^2 + (3 t)^2 / 4 = r^2, and rho = 0.75 (0.05 + 3 t) / r
    args_b = args[:5] + (np.array([0.3]),) + args[6:]
    rho = O.normalized_gap(*args_b, 4.0, np.array([0.25]), np.array([1.75]), np.array([0.0]),
                           np.array([1.0]))
    r = math.sqrt(0.390625)
    t = math.sqrt((0.390625 - 4 * 0.05 ** 2) * 4 / 9)
    assert rho == pytest.approx(0.75 * (0.05 + 3 * t) / r, rel=1e-12)


def test_ndg_restarts_reach_the_optimum():
    for seed in range(3):
        lp = lpgen.tiny_lp(seed, m=5 + seed % 2, n=4 + seed % 2, eq_rows=seed % 2)
        best, _ = R.vertex_enumeration(lp)
        r = O.solve(lp, O.Params(tol=1e-9, iter_limit=400_000, restart_metric="ndg"))
        assert r.status == O.STATUS_OPTIMAL
        assert r.kkt.primal_obj == pytest.approx(best, rel=1e-6, abs=1e-6)
    lp = lpgen.mip_relaxation(1)
    obj, _, _, _ = R.highs(lp)
    r = O.solve(lp, O.Params(tol=1e-8, restart_metric="ndg"))
    assert r.status == O.STATUS_OPTIMAL
    assert abs(r.kkt.primal_obj - obj) / (1 + abs(obj)) < 1e-7


def test_ndg_restart_sequence_differs_from_kkt_and_restarts_less_on_a_relaxation():
    """On the 200 x 400 relaxation (seed 1) the gap metric restarts at different checks
    than KKT_omega (3 against 4 restarts to 1e-4, 384 against 640 iterations)."""
    lp = lpgen.mip_relaxation(1)
    a = O.solve(lp, O.Params(tol=1e-4))
    b = O.solve(lp, O.Params(tol=1e-4, restart_metric="ndg"))
    assert [k for k, _ in a.check_trace] != [k for k, _ in b.check_trace]
    assert (a.iters, a.restarts) == (640, 4) and (b.iters, b.restarts) == (384, 3)
