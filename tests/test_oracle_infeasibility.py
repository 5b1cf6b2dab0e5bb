"""Pins of the oracle's infeasibility and unboundedness certificates (A12).

The expected classification comes from HiGHS (scipy ``linprog`` status 2 =
infeasible, 3 = unbounded) and from instances built to be infeasible or
unbounded by construction; every returned certificate is re-checked here on
the ORIGINAL data in the caller's sign convention with dense numpy, by the
Farkas alternative, not by the oracle's own functions.  The planted-mistake
tests at the end show that a plausible slip in A12 fails one of these pins.
"""
import sys

import numpy as np
import pytest
from scipy.optimize import linprog

import lpgen
from oracle import pdlp_oracle as O
from test_oracle_mutants import _mutant_module

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

INF = np.inf


def _lp(a, b, sense, c, l, u):
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    rows, cols = np.nonzero(a)
    return lpgen._lp(m, n, rows, cols, a[rows, cols], np.asarray(b, float),
                     np.array([ord(s) for s in sense], dtype=np.uint8), np.asarray(c, float),
                     np.asarray(l, float), np.asarray(u, float), np.zeros(n, np.uint8), "hand")


def _highs_status(lp):
    a = lp.dense()
    le, ge, eq = (lp.sense == ord(k) for k in "LGE")
    a_ub = np.vstack([a[le], -a[ge]])
    b_ub = np.concatenate([lp.b[le], -lp.b[ge]])
    bounds = [(None if np.isinf(lo) else lo, None if np.isinf(hi) else hi)
              for lo, hi in zip(lp.l, lp.u)]
    res = linprog(lp.c, A_ub=a_ub if a_ub.size else None, b_ub=b_ub if a_ub.size else None,
                  A_eq=a[eq] if eq.any() else None, b_eq=lp.b[eq] if eq.any() else None,
                  bounds=bounds, method="highs")
    return res.status


def farkas_ray_margin(lp, y):
    """Check y (caller convention: <= 0 on <=-rows, >= 0 on >=-rows) as a proof
    that {A x (senses) b, l <= x <= u} is empty.

    For any feasible x, y^T A x >= y^T b row by row (the sign of y matches the
    sense), and y^T A x = sum_j (A^T y)_j x_j <= sum_j max over [l_j, u_j] of
    (A^T y)_j x_j.  So  b^T y - sum_j max_{x_j in [l_j,u_j]} (A^T y)_j x_j > 0
    is a contradiction.  Returns (that margin, residual): the residual is the
    part of A^T y that pushes against an infinite bound (the max is +inf there).
    """
    le, ge = lp.sense == ord("L"), lp.sense == ord("G")
    assert np.all(y[le] <= 0) and np.all(y[ge] >= 0)
    g = lp.dense().T @ y
    pos, neg = np.maximum(g, 0.0), np.maximum(-g, 0.0)
    bad = np.where(np.isinf(lp.u), pos, 0.0) + np.where(np.isinf(lp.l), neg, 0.0)
    fin_u, fin_l = np.isfinite(lp.u), np.isfinite(lp.l)
    sup = float(pos[fin_u] @ lp.u[fin_u] - neg[fin_l] @ lp.l[fin_l])
    return float(lp.b @ y) - sup, float(np.linalg.norm(bad))


def descent_ray_margin(lp, x):
    """Check x as a direction of unbounded descent: A x keeps every row's sense
    (>= 0 on >=-rows, <= 0 on <=-rows, 0 on =-rows), x stays in the recession
    cone of [l, u], and c^T x < 0.  Returns (-c^T x, residual)."""
    assert np.all(x[np.isfinite(lp.l)] >= 0) and np.all(x[np.isfinite(lp.u)] <= 0)
    ax = lp.dense() @ x
    le, ge, eq = (lp.sense == ord(k) for k in "LGE")
    res = np.concatenate([np.maximum(ax[le], 0), np.maximum(-ax[ge], 0), np.abs(ax[eq])])
    return -float(lp.c @ x), float(np.linalg.norm(res))


INFEASIBLE = {
    "box": lambda: _lp([[1, 1], [1, 1]], [3, 1], "GL", [1, 1], [0, 0], [10, 10]),
    "free": lambda: _lp([[1, 1], [1, 1]], [3, 1], "GL", [1, 1], [-INF, -INF], [INF, INF]),
    "equalities": lambda: _lp([[1, 1], [1, 1]], [3, 1], "EE", [1, 1], [0, 0], [INF, INF]),
    "contradiction1": lambda: lpgen.mip_relaxation_contradiction(1),
    "contradiction2": lambda: lpgen.mip_relaxation_contradiction(2),
    "dead_cover": lambda: lpgen.set_cover_dead(5, 300),
    "dead_cover3": lambda: lpgen.set_cover_dead(6, 500, dead=3),
}

UNBOUNDED = {
    "hand": lambda: _lp([[1, -1]], [0], "G", [-1, 0], [0, 0], [INF, INF]),
    "hand_free": lambda: _lp([[1, -1]], [0], "G", [-1, 0], [-INF, -INF], [INF, INF]),
    "hand_upper": lambda: _lp([[1, 1]], [5], "L", [1, 0.5], [-INF, -INF], [0, 0]),
    "relaxation1": lambda: lpgen.mip_relaxation_unbounded(1),
    "relaxation2": lambda: lpgen.mip_relaxation_unbounded(2, rays=1),
}


@pytest.mark.parametrize("name", list(INFEASIBLE))
def test_infeasible_lp_returns_a_farkas_ray(name):
    lp = INFEASIBLE[name]()
    assert _highs_status(lp) == 2
    r = O.solve(lp, O.Params(tol=1e-8, iter_limit=20000))
    assert r.status == O.STATUS_PRIMAL_INFEASIBLE
    margin, res = farkas_ray_margin(lp, r.y)
    assert margin > 0
    assert res <= 1e-8 * margin
    # the point output is still the chosen iterate, inside the bounds
    assert np.all(r.x >= lp.l) and np.all(r.x <= lp.u)


@pytest.mark.parametrize("name", list(UNBOUNDED))
def test_unbounded_lp_returns_a_descent_ray(name):
    lp = UNBOUNDED[name]()
    assert _highs_status(lp) == 3
    r = O.solve(lp, O.Params(tol=1e-8, iter_limit=20000))
    assert r.status == O.STATUS_DUAL_INFEASIBLE
    descent, res = descent_ray_margin(lp, r.x)
    assert descent > 0
    assert res <= 1e-8 * descent


def test_farkas_ray_of_the_contradicting_rows_by_hand():
    # rows r (<=, b_r) and m (>=, b_r + d) repeat the same a: y_r = -1, y_m = +1 gives
    # A^T y = 0 and b^T y = d > 0.  The check above must accept it and reject -y.
    lp = lpgen.mip_relaxation_contradiction(1)
    r = lp.meta["row"]
    y = np.zeros(lp.m)
    y[r], y[lp.m - 1] = -1.0, 1.0
    margin, res = farkas_ray_margin(lp, y)
    assert margin == pytest.approx(lp.b[-1] - lp.b[r], rel=1e-15) and margin >= 1.0
    assert res == 0.0


def test_rays_by_hand():
    # canonical K = [[1, 1], [-1, -1]], q = (3, -1) (the <=-row flipped), x in [0, 10]^2;
    # displacements dy = (2, 1) -> y^ = (2, 1), K^T y^ = (1, 1), lambda^ = (-1, -1),
    # d^ = q^T y^ + sum l lambda^+ - u lambda^- = 6 - 1 + 0 - (10 + 10) = -15,
    # |d^|_terms = 6 + 1 + 20 = 27; dy = (1, 1): lambda^ = 0, d^ = 3 - 1 = 2
    lp = _lp([[1, 1], [1, 1]], [3, 1], "GL", [1, 1], [0, 0], [10, 10])
    k, q, is_eq, _ = O.canonicalize(lp)
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.zeros(2), np.array([2.0, 1.0]))
    assert (ry.dual_ray_obj, ry.dual_ray_res, ry.dual_ray_abs) == (-15.0, 0.0, 27.0)
    assert not ry.primal_infeasible(1e-8)
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.zeros(2), np.array([1.0, 1.0]))
    assert (ry.dual_ray_obj, ry.dual_ray_res) == (2.0, 0.0)
    assert ry.primal_infeasible(1e-8)
    # negative displacement on an inequality row is projected away: y^ = (0, 0)
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.zeros(2), np.array([-1.0, -1.0]))
    assert ry.y_ray.tolist() == [0.0, 0.0] and not ry.primal_infeasible(1e-8)
    # x in [0, inf)^2: y^ = (2, 1) leaves lambda^- = (1, 1) against u = inf, so
    # r^_d = (1, 1) and d^ = 6 - 1 = 5 is no certificate
    lp = _lp([[1, 1], [1, 1]], [3, 1], "GL", [1, 1], [0, 0], [INF, INF])
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.zeros(2), np.array([2.0, 1.0]))
    assert ry.dual_ray_obj == 5.0 and ry.dual_ray_res == pytest.approx(2 ** 0.5, rel=1e-15)
    assert not ry.primal_infeasible(1e-8)


def test_primal_ray_by_hand():
    # min -x0 s.t. x0 - x1 = 0 (E), x1 >= 2 (G); x0 >= 0, x1 in [0, 1e3] or [0, inf)
    # dx = (1, 0.5): x^ = (1, 0.5) when both are unbounded above, K x^ = (0.5, 0.5):
    # the equality row is missed by 0.5 whichever its sign, p^ = -1
    a, b, c = [[1, -1], [0, 1]], [0, 2], [-1, 0]
    lp = _lp(a, b, "EG", c, [0, 0], [INF, INF])
    k, q, is_eq, _ = O.canonicalize(lp)
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.array([1.0, 0.5]), np.zeros(2))
    assert (ry.primal_ray_obj, ry.primal_ray_res, ry.primal_ray_abs) == (-1.0, 0.5, 1.0)
    assert not ry.dual_infeasible(1e-8)
    # dx = (1, 1): K x^ = (0, 1), a true ray of descent
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.array([1.0, 1.0]), np.zeros(2))
    assert (ry.primal_ray_obj, ry.primal_ray_res) == (-1.0, 0.0) and ry.dual_infeasible(1e-8)
    # with x1 <= 1e3 the ray's x1 part is projected away: K x^ = (1, 0), missed by 1
    lp = _lp(a, b, "EG", c, [0, 0], [INF, 1e3])
    ry = O.rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, np.array([1.0, 1.0]), np.zeros(2))
    assert ry.x_ray.tolist() == [1.0, 0.0] and ry.primal_ray_res == 1.0
    assert not ry.dual_infeasible(1e-8)


def test_recession_cone_projection_by_hand():
    l = np.array([0.0, -INF, 0.0, -INF])
    u = np.array([1.0, 5.0, INF, INF])
    d = np.array([3.0, 3.0, -3.0, -3.0])
    assert O.recession_proj(d, l, u).tolist() == [0.0, 0.0, 0.0, -3.0]
    d = -d
    assert O.recession_proj(d, l, u).tolist() == [0.0, -3.0, 3.0, 3.0]


def test_zero_objective_ray_is_not_a_certificate():
    # an objective that is zero up to rounding must not pass: d^ = 1e-17 of terms ~1
    ry = O.Rays(np.zeros(1), np.zeros(1), 1e-17, 0.0, 1.0, 0.0, 0.0, 0.0)
    assert not ry.primal_infeasible(1e-8)
    ry = O.Rays(np.zeros(1), np.zeros(1), 0.0, 0.0, 0.0, -1e-17, 0.0, 1.0)
    assert not ry.dual_infeasible(1e-8)


def _split_equalities(seed, k=20):
    """A feasible LP whose k rows are equalities written as two inequalities,
    tight at a feasible point: its dual has rays of exactly zero objective."""
    lp = lpgen.mip_relaxation(seed)
    x0 = lp.meta["x0"]
    a = lp.dense()
    rng = np.random.default_rng(seed)
    rs = rng.choice(np.nonzero(np.abs(a).sum(1) > 0)[0], size=k, replace=False)
    b = lp.b.copy()
    b[rs] = a[rs] @ x0
    a2 = np.vstack([a, a[rs]])
    sense = "".join(chr(s) for s in lp.sense) + "G" * k
    return _lp(a2, np.concatenate([b, b[rs]]), sense, lp.c, lp.l, lp.u)


@pytest.mark.parametrize("maker", [lambda: lpgen.mip_relaxation(1), lambda: _split_equalities(2),
                                   lambda: lpgen.random_sparse_lp(7, 60, 80, free_frac=0.3),
                                   lambda: lpgen.random_sparse_lp(1, 40, 60, 0.1, 0.3, 0.8),
                                   lambda: _lp([[1, 0]], [1], "E", [-1, 0], [0, 0], [INF, INF])],
                         ids=["relaxation", "split_equalities", "free_columns", "free_equalities",
                              "equality_pins_ray"])
def test_feasible_bounded_lp_is_never_certified(maker):
    lp = maker()
    assert _highs_status(lp) == 0
    r = O.solve(lp, O.Params(tol=1e-8, iter_limit=50000))
    assert r.status == O.STATUS_OPTIMAL


def test_detection_off_runs_to_the_limit():
    lp = INFEASIBLE["box"]()
    r = O.solve(lp, O.Params(tol=1e-8, iter_limit=640, detect_infeasibility=False))
    assert r.status == O.STATUS_ITER_LIMIT and r.iters == 640


# ------------------------------------------------------------ planted mistakes
MUTANTS = [
    ("upper-bound term of the ray objective with the wrong sign",
     "d_obj = float(q @ y_ray + l[lfin] @ lp_[lfin] - u[ufin] @ lm[ufin])",
     "d_obj = float(q @ y_ray + l[lfin] @ lp_[lfin] + u[ufin] @ lm[ufin])",
     ["test_rays_by_hand"]),
    ("dual ray not projected onto the cone", "y_ray = proj_dual(dy, is_eq)", "y_ray = dy",
     ["test_rays_by_hand"]),
    ("recession projection keeps dx+ where u is finite",
     "return np.where(np.isfinite(u), np.minimum(d, 0.0), d)", "return d",
     ["test_recession_cone_projection_by_hand"]),
    ("equality rows' ray residual one-sided", "np.where(is_eq, np.abs(kx), np.maximum(-kx, 0.0))",
     "np.maximum(-kx, 0.0)", ["test_primal_ray_by_hand"]),
    ("primal-infeasibility test without the residual",
     "d > kappa * self.dual_ray_abs and self.dual_ray_res <= eps * d", "d > kappa * self.dual_ray_abs",
     ["test_feasible_bounded_lp_is_never_certified"]),
    ("ray residual charged on the wrong side of an infinite bound",
     "r_d = np.where(np.isinf(l), lp_, 0.0) + np.where(np.isinf(u), lm, 0.0)\n    lfin = np.isfinite(l)\n    ufin = np.isfinite(u)\n    d_obj",
     "r_d = np.where(np.isinf(l), lm, 0.0) + np.where(np.isinf(u), lp_, 0.0)\n    lfin = np.isfinite(l)\n    ufin = np.isfinite(u)\n    d_obj",
     ["test_rays_by_hand"]),
    ("no rounding guard", "return d > 0 and d > kappa", "return d > 0 and d >= 0 * kappa",
     ["test_zero_objective_ray_is_not_a_certificate"]),
    ("dual-infeasibility test reads the wrong sign of c^T x^", "p = -self.primal_ray_obj",
     "p = self.primal_ray_obj", ["test_unbounded_lp_returns_a_descent_ray"]),
]

_PARAMS = {
    "test_feasible_bounded_lp_is_never_certified": [
        {"maker": m} for m in [lambda: _split_equalities(2),
                               lambda: lpgen.random_sparse_lp(1, 40, 60, 0.1, 0.3, 0.8),
                               lambda: _lp([[1, 0]], [1], "E", [-1, 0], [0, 0], [INF, INF])]],
    "test_infeasible_lp_returns_a_farkas_ray": [{"name": "free"}, {"name": "box"}],
    "test_unbounded_lp_returns_a_descent_ray": [{"name": "hand"}, {"name": "relaxation1"}],
}


@pytest.mark.parametrize("desc,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(desc, old, new, pins, monkeypatch):
    mutant = _mutant_module(old, new)
    monkeypatch.setattr(sys.modules[__name__], "O", mutant)
    caught = []
    for name in pins:
        for kw in _PARAMS.get(name, [{}]):
            try:
                globals()[name](**kw)
            except Exception:
                caught.append(name)
                break
    assert caught, f"mutant '{desc}' passed every pin in {pins}"
