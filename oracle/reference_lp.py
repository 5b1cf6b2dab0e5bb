"""Independent LP references used to pin the oracle (test infrastructure only).

* :func:`vertex_enumeration` -- brute force over all n-subsets of the m + 2n
  constraint hyperplanes of a tiny LP with finite bounds: solve each n x n
  system, keep the feasible points, take the least objective.  This is the
  exact optimum of eq. (1) (section 1 of the paper) by the fundamental theorem
  of linear programming, with no iteration at all.
* :func:`highs` -- scipy's HiGHS (a library LP solver, dual simplex / IPM with
  crossover) on the same LP; returns the optimum, x, the row duals in the
  caller convention (y <= 0 on <=-rows, >= 0 on >=-rows) and reduced costs.

Neither shares code with the PDHG oracle or the CUDA path.
"""
from __future__ import annotations

import itertools

import numpy as np

SENSE_LE, SENSE_GE, SENSE_EQ = ord("L"), ord("G"), ord("E")


def vertex_enumeration(lp, feas_tol=1e-9):
    """Exact optimum of a tiny bounded LP: returns (obj, list of optimal vertices)."""
    a = lp.dense()
    m, n = a.shape
    assert np.all(np.isfinite(lp.l)) and np.all(np.isfinite(lp.u))
    # hyperplanes: rows, then x_j = l_j, then x_j = u_j
    planes = [(a[i], lp.b[i]) for i in range(m)]
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        planes.append((e, lp.l[j]))
        planes.append((e, lp.u[j]))
    best = np.inf
    verts = []
    for sub in itertools.combinations(range(len(planes)), n):
        mat = np.array([planes[i][0] for i in sub])
        rhs = np.array([planes[i][1] for i in sub])
        if abs(np.linalg.det(mat)) < 1e-12:
            continue
        x = np.linalg.solve(mat, rhs)
        ax = a @ x
        scale = 1.0 + np.abs(lp.b)
        ok = np.all(x >= lp.l - feas_tol) and np.all(x <= lp.u + feas_tol)
        ok &= np.all(np.where(lp.sense == SENSE_LE, ax - lp.b <= feas_tol * scale, True))
        ok &= np.all(np.where(lp.sense == SENSE_GE, lp.b - ax <= feas_tol * scale, True))
        ok &= np.all(np.where(lp.sense == SENSE_EQ, np.abs(ax - lp.b) <= feas_tol * scale, True))
        if not ok:
            continue
        obj = float(lp.c @ x)
        if obj < best - 1e-12:
            best = obj
            verts = [x]
        elif abs(obj - best) <= 1e-12:
            verts.append(x)
    return best, verts


def highs(lp, method="highs"):
    """HiGHS optimum of the LP: (obj, x, y in caller convention, reduced costs).

    ``method`` is scipy's HiGHS variant ("highs", "highs-ds" dual simplex,
    "highs-ipm" interior point with crossover)."""
    from scipy.optimize import linprog
    import scipy.sparse as sp

    a = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    le = np.nonzero(lp.sense == SENSE_LE)[0]
    ge = np.nonzero(lp.sense == SENSE_GE)[0]
    eq = np.nonzero(lp.sense == SENSE_EQ)[0]
    ub_rows = np.concatenate([le, ge])
    sgn = np.concatenate([np.ones(le.size), -np.ones(ge.size)])
    a_ub = sp.diags(sgn) @ a[ub_rows] if ub_rows.size else None
    b_ub = sgn * lp.b[ub_rows] if ub_rows.size else None
    a_eq = a[eq] if eq.size else None
    b_eq = lp.b[eq] if eq.size else None
    bounds = np.stack([np.where(np.isfinite(lp.l), lp.l, -np.inf),
                       np.where(np.isfinite(lp.u), lp.u, np.inf)], axis=1)
    bounds = [(None if not np.isfinite(lo) else lo, None if not np.isfinite(hi) else hi)
              for lo, hi in bounds]
    res = linprog(lp.c, A_ub=a_ub, b_ub=b_ub, A_eq=a_eq, b_eq=b_eq, bounds=bounds,
                  method=method)
    if res.status != 0:
        raise RuntimeError(f"HiGHS failed: {res.message}")
    y = np.zeros(lp.m)
    if ub_rows.size:
        # marginal of (sgn a) x <= sgn b w.r.t. its rhs; d obj / d b_i = sgn_i * marginal
        y[ub_rows] = sgn * res.ineqlin.marginals
    if eq.size:
        y[eq] = res.eqlin.marginals
    lam = lp.c - a.T @ y
    return float(res.fun), np.asarray(res.x), y, lam
