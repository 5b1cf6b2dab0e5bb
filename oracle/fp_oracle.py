"""CPU oracle of the fix-and-propagate consumer (section 2 of the paper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and nothing else.  Plain
Python loops over the CSR data, in the order the C ABI function ``fp_run``
must follow, so integer decisions can be compared exactly.

What it computes (section 2, "LP-based variable strategies", "LP-based
fixing", "Integer-aware branching strategy", Alg. 1):

* variable order of the integers:
    FRAC    ascending fractionality min(x - floor x, ceil x - x), stable;
    REDCOST descending |reduced cost| (lambda = c - A^T y), stable;
    DUAL    rows by descending |y| (stable); each row's integers not yet
            seen, by descending |lambda| (stable); remaining integers by index;
    TYPE    stable, binaries first, then general integers;
  and the hybrid strategies of section 2, "Tiebreaking and hybrid strategies"
  (Frac with ties broken by Dual or by RedCost, and the reverse): a variable
  strategy whose equal-ranked variables are ordered by a second one,
    FRAC_DUAL     ascending fractionality; ties by position in the DUAL order;
    FRAC_REDCOST  ascending fractionality; ties by descending |lambda|, then index;
    DUAL_FRAC     the DUAL order with each row's new integers by descending
                  |lambda| and then ascending fractionality (then storage order),
                  and the integers of no row by ascending fractionality, then index;
    REDCOST_FRAC  descending |lambda|; ties by ascending fractionality, then index;
* LP-based fixing: x = LP value clamped to the current domain,
  d_i = x - floor(x), d ~ U(0,1); fix to floor(x) if d > d_i, else ceil(x);
* Alg. 1 branching: bound changes in increasing priority,
    l < a < u, c > 0:  [(a+1, u), (l, a-1), (a, a)]
    l < a < u, c <= 0: [(l, a-1), (a+1, u), (a, a)]
    a = l:             [(u, u), (l, l)]
    otherwise:         [(l, l), (u, u)]
  the highest priority (last) is explored first;
* depth-first search: pick the first integer of the order whose domain is
  not a single value, draw d, branch, propagate, backtrack on conflict; when
  every integer is fixed, solve the final LP with the integers fixed.

Readings where the paper is silent: the random
generator is SplitMix64 (published by S. Vigna) with u = (r >> 11) * 2^-53,
one draw per branching node; the LP value is clamped to the current domain
before d_i is taken; the only propagator is linear activity bound tightening
(clique and implication propagators and repair are defined in the cited
Salvagnin 2024 code, not available); node limit 10 |I| by default; feasibility
tolerance 1e-6 (the paper's relative 1e-6 feasibility, section 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SENSE_LE, SENSE_GE, SENSE_EQ = ord("L"), ord("G"), ord("E")
FRAC, REDCOST, DUAL, TYPE = 0, 1, 2, 3
FRAC_DUAL, FRAC_REDCOST, DUAL_FRAC, REDCOST_FRAC = 4, 5, 6, 7
FEASIBLE, INFEASIBLE, NODE_LIMIT, NO_FINAL_LP = 1, 2, 3, 4
MASK = (1 << 64) - 1
INT_EPS = 1e-6   # rounding slack of integer bounds
FEAS_TOL = 1e-6  # row violation tolerance, relative to max(1, |b|)


# ------------------------------------------------------------------ RNG
class SplitMix64:
    """SplitMix64 (S. Vigna), 64-bit state, one output per call."""

    def __init__(self, seed: int):
        self.s = seed & MASK

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & MASK
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * (2.0 ** -53)


# ------------------------------------------------------------------ Alg. 1
def branching(l: float, u: float, a: float, c: float):
    """Alg. 1: the bound changes (lo, hi) of an integer, in increasing priority."""
    if l < a < u:
        if c > 0:
            return [(a + 1, u), (l, a - 1), (a, a)]
        return [(l, a - 1), (a + 1, u), (a, a)]
    if a == l:
        return [(u, u), (l, l)]
    return [(l, l), (u, u)]


def lp_fixing_value(x_lp: float, lo: float, hi: float, d: float) -> float:
    """LP-based fixing: floor of the clamped LP value if d > d_i, else its ceiling."""
    x = min(max(x_lp, lo), hi)
    fl = math.floor(x)
    di = x - fl
    return float(fl) if d > di else float(math.ceil(x))


# ------------------------------------------------------------------ strategies
def reduced_costs(lp, y):
    lam = lp.c.astype(np.float64).copy()
    for i in range(lp.m):
        for p in range(lp.row_ptr[i], lp.row_ptr[i + 1]):
            lam[lp.col[p]] -= lp.val[p] * y[i]
    return lam


def fractionality(v: float) -> float:
    return min(v - math.floor(v), math.ceil(v) - v)


def dual_order(lp, lam, y_lp, is_int, frac=None):
    """DUAL: rows by descending |y|; each row's integers not yet seen by descending
    |lambda| (and, given ``frac``, then ascending fractionality); the integers of no
    row last, in index order (or by ascending fractionality given ``frac``).  Python's
    sort is stable: remaining ties keep storage or index order."""
    rows = sorted(range(lp.m), key=lambda i: -abs(y_lp[i]))
    seen = [False] * lp.n
    out = []
    for i in rows:
        cols = [int(lp.col[p]) for p in range(lp.row_ptr[i], lp.row_ptr[i + 1])
                if is_int[lp.col[p]] and not seen[lp.col[p]]]
        if frac is None:
            cols = sorted(cols, key=lambda j: -abs(lam[j]))
        else:
            cols = sorted(cols, key=lambda j: (-abs(lam[j]), frac[j]))
        for j in cols:
            if not seen[j]:
                seen[j] = True
                out.append(j)
    rest = [j for j in range(lp.n) if is_int[j] and not seen[j]]
    if frac is not None:
        rest = sorted(rest, key=lambda j: frac[j])
    return out + rest


def variable_order(lp, strategy, x_lp, y_lp, is_int):
    ints = [j for j in range(lp.n) if is_int[j]]
    frac = [fractionality(x_lp[j]) for j in range(lp.n)]
    if strategy == FRAC:
        return sorted(ints, key=lambda j: frac[j])
    lam = reduced_costs(lp, y_lp) if strategy not in (TYPE,) else None
    if strategy == REDCOST:
        return sorted(ints, key=lambda j: -abs(lam[j]))
    if strategy == DUAL:
        return dual_order(lp, lam, y_lp, is_int)
    if strategy == FRAC_DUAL:
        rank = {j: k for k, j in enumerate(dual_order(lp, lam, y_lp, is_int))}
        return sorted(ints, key=lambda j: (frac[j], rank[j]))
    if strategy == FRAC_REDCOST:
        return sorted(ints, key=lambda j: (frac[j], -abs(lam[j])))
    if strategy == DUAL_FRAC:
        return dual_order(lp, lam, y_lp, is_int, frac=frac)
    if strategy == REDCOST_FRAC:
        return sorted(ints, key=lambda j: (-abs(lam[j]), frac[j]))
    if strategy == TYPE:
        binary = [j for j in ints if lp.l[j] == 0.0 and lp.u[j] == 1.0]
        general = [j for j in ints if not (lp.l[j] == 0.0 and lp.u[j] == 1.0)]
        return binary + general
    raise ValueError(strategy)


# ------------------------------------------------------------------ propagation
class Domains:
    """Bounds with a trail for undo."""

    def __init__(self, l, u, is_int):
        self.lo = [float(v) for v in l]
        self.hi = [float(v) for v in u]
        self.is_int = is_int
        self.trail = []
        for j in range(len(self.lo)):
            if is_int[j]:
                if math.isfinite(self.lo[j]):
                    self.lo[j] = float(math.ceil(self.lo[j] - INT_EPS))
                if math.isfinite(self.hi[j]):
                    self.hi[j] = float(math.floor(self.hi[j] + INT_EPS))

    def set(self, j, lo, hi):
        self.trail.append((j, self.lo[j], self.hi[j]))
        self.lo[j] = lo
        self.hi[j] = hi

    def undo(self, mark):
        while len(self.trail) > mark:
            j, lo, hi = self.trail.pop()
            self.lo[j] = lo
            self.hi[j] = hi


def _tighten(dom, j, new_lo, new_hi):
    """Apply a derived bound; returns (changed, infeasible)."""
    lo, hi = dom.lo[j], dom.hi[j]
    if dom.is_int[j]:
        if new_lo > -math.inf:
            new_lo = float(math.ceil(new_lo - INT_EPS))
        if new_hi < math.inf:
            new_hi = float(math.floor(new_hi + INT_EPS))
        nlo, nhi = max(lo, new_lo), min(hi, new_hi)
        changed = nlo > lo or nhi < hi
    else:
        nlo = new_lo if new_lo > lo + 1e-7 * max(1.0, abs(lo)) else lo
        nhi = new_hi if new_hi < hi - 1e-7 * max(1.0, abs(hi)) else hi
        changed = nlo != lo or nhi != hi
    if nlo > nhi + INT_EPS:
        return changed, True
    if changed:
        # a continuous domain squeezed below the tolerance collapses to a point
        dom.set(j, nlo, nhi if dom.is_int[j] else max(nhi, nlo))
    return changed, False


def propagate(lp, at_ptr, at_row, dom, rows):
    """Linear activity bound tightening to a fixpoint, rows processed FIFO from `rows`.
    Returns False on a detected infeasibility."""
    inq = [False] * lp.m
    queue = []
    for i in rows:
        if not inq[i]:
            inq[i] = True
            queue.append(i)
    head = 0
    while head < len(queue):
        i = queue[head]
        head += 1
        inq[i] = False
        s, e = int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])
        b = float(lp.b[i])
        sense = lp.sense[i]
        minact = maxact = 0.0
        ninf_min = ninf_max = 0
        for p in range(s, e):
            a = float(lp.val[p])
            j = int(lp.col[p])
            lo, hi = dom.lo[j], dom.hi[j]
            if a > 0:
                if lo == -math.inf:
                    ninf_min += 1
                else:
                    minact += a * lo
                if hi == math.inf:
                    ninf_max += 1
                else:
                    maxact += a * hi
            else:
                if hi == math.inf:
                    ninf_min += 1
                else:
                    minact += a * hi
                if lo == -math.inf:
                    ninf_max += 1
                else:
                    maxact += a * lo
        tol = FEAS_TOL * max(1.0, abs(b))
        if sense in (SENSE_LE, SENSE_EQ) and ninf_min == 0 and minact > b + tol:
            return False
        if sense in (SENSE_GE, SENSE_EQ) and ninf_max == 0 and maxact < b - tol:
            return False
        for p in range(s, e):
            a = float(lp.val[p])
            j = int(lp.col[p])
            lo, hi = dom.lo[j], dom.hi[j]
            new_lo, new_hi = -math.inf, math.inf
            if sense in (SENSE_LE, SENSE_EQ):
                # a x_j <= b - (min activity of the other entries)
                own = a * lo if a > 0 else a * hi
                own_inf = (lo == -math.inf) if a > 0 else (hi == math.inf)
                if ninf_min == 0 or (ninf_min == 1 and own_inf):
                    rest = minact - (0.0 if own_inf else own)
                    bound = (b - rest) / a
                    if a > 0:
                        new_hi = bound
                    else:
                        new_lo = bound
            if sense in (SENSE_GE, SENSE_EQ):
                own = a * hi if a > 0 else a * lo
                own_inf = (hi == math.inf) if a > 0 else (lo == -math.inf)
                if ninf_max == 0 or (ninf_max == 1 and own_inf):
                    rest = maxact - (0.0 if own_inf else own)
                    bound = (b - rest) / a
                    if a > 0:
                        new_lo = max(new_lo, bound)
                    else:
                        new_hi = min(new_hi, bound)
            changed, infeasible = _tighten(dom, j, new_lo, new_hi)
            if infeasible:
                return False
            if changed:
                for q in range(at_ptr[j], at_ptr[j + 1]):
                    r = at_row[q]
                    if r != i and not inq[r]:
                        inq[r] = True
                        queue.append(r)
    return True


def transpose_lists(lp):
    """Row lists per column, rows ascending (the order propagation enqueues them)."""
    cols = [[] for _ in range(lp.n)]
    for i in range(lp.m):
        for p in range(lp.row_ptr[i], lp.row_ptr[i + 1]):
            cols[lp.col[p]].append(i)
    at_ptr = [0]
    at_row = []
    for j in range(lp.n):
        at_row += cols[j]
        at_ptr.append(len(at_row))
    return at_ptr, at_row


# ------------------------------------------------------------------ the heuristic
@dataclass
class FPResult:
    status: int
    obj: float
    x: np.ndarray
    nodes: int
    backtracks: int
    fixed: np.ndarray       # integer values (NaN for continuous columns)


def fp_search(lp, x_lp, y_lp, is_int, strategy, seed, node_limit=None):
    """Order, fix, branch (Alg. 1), propagate, backtrack.  Returns (status, domains,
    nodes, backtracks); status FEASIBLE means every integer is fixed."""
    at_ptr, at_row = transpose_lists(lp)
    is_int = [bool(v) for v in is_int]
    n_int = sum(is_int)
    limit = 10 * n_int if node_limit is None or node_limit <= 0 else node_limit
    dom = Domains(lp.l, lp.u, is_int)
    if not propagate(lp, at_ptr, at_row, dom, range(lp.m)):
        return INFEASIBLE, dom, 0, 0
    order = variable_order(lp, strategy, x_lp, y_lp, is_int)
    rng = SplitMix64(seed)
    frames = []  # [mark, var, alternatives]
    nodes = backtracks = 0
    while True:
        j = next((v for v in order if dom.hi[v] - dom.lo[v] > 0.5), None)
        if j is None:
            return FEASIBLE, dom, nodes, backtracks
        if nodes >= limit:
            return NODE_LIMIT, dom, nodes, backtracks
        nodes += 1
        a = lp_fixing_value(float(x_lp[j]), dom.lo[j], dom.hi[j], rng.uniform())
        frames.append([len(dom.trail), j, branching(dom.lo[j], dom.hi[j], a, float(lp.c[j]))])
        while True:
            mark, v, alts = frames[-1]
            dom.undo(mark)
            if not alts:
                frames.pop()
                backtracks += 1
                if not frames:
                    return INFEASIBLE, dom, nodes, backtracks
                continue
            lo, hi = alts.pop()
            dom.set(v, lo, hi)
            if propagate(lp, at_ptr, at_row, dom, at_row[at_ptr[v]:at_ptr[v + 1]]):
                break


def fp_run(lp, x_lp, y_lp, is_int, strategy=TYPE, seed=1, node_limit=None, final_lp=True,
           final_tol=1e-8):
    """The whole heuristic: search, then the final LP with every integer fixed."""
    from oracle import pdlp_oracle as PO
    status, dom, nodes, backtracks = fp_search(lp, x_lp, y_lp, is_int, strategy, seed, node_limit)
    fixed = np.array([dom.lo[j] if is_int[j] else np.nan for j in range(lp.n)])
    if status != FEASIBLE:
        return FPResult(status, math.nan, np.full(lp.n, np.nan), nodes, backtracks, fixed)
    if not final_lp:
        return FPResult(NO_FINAL_LP, math.nan, np.full(lp.n, np.nan), nodes, backtracks, fixed)
    import copy
    lp2 = copy.copy(lp)
    lp2.l = np.where(is_int, fixed, lp.l)
    lp2.u = np.where(is_int, fixed, lp.u)
    # feasible when every row holds to FEAS_TOL max(1, |b_i|) (reading: the relative 1e-6
    # of section 4, per row); a first-order point that misses a row is polished (A13:
    # the same PDHG on the objective-free problem from that point, to final_tol)
    r = PO.solve(lp2, PO.Params(tol=final_tol, iter_limit=500_000))
    x = np.where(is_int, fixed, r.x)
    viol = max_row_violation(lp, x)
    if r.status == PO.STATUS_OPTIMAL and viol > FEAS_TOL:
        r = PO.polish_primal(lp2, r.x, PO.Params(tol=final_tol, iter_limit=500_000))
        x = np.where(is_int, fixed, r.x)
        viol = max_row_violation(lp, x)
    ok = r.status == PO.STATUS_OPTIMAL and viol <= FEAS_TOL
    return FPResult(FEASIBLE if ok else INFEASIBLE, float(lp.c @ x) if ok else math.nan, x, nodes,
                    backtracks, fixed)


def fp_run_refs(lp, x_refs, y_lp, is_int, strategy=TYPE, seed=1, node_limit=None,
                final_lp=True, final_tol=1e-8):
    """The heuristic from several LP reference points (the paper's suggestion to use
    PDLP's cycling for more than one reference, section 5): fp_run from each point in
    turn, the same strategy, seed and dual point; the feasible result with the lowest
    objective is kept (ties: the earlier point).  Returns (result, index), index -1 when
    no run is feasible (the result is then the last run's)."""
    best, best_i, last = None, -1, None
    for i, x in enumerate(x_refs):
        r = fp_run(lp, x, y_lp, is_int, strategy, seed, node_limit, final_lp, final_tol)
        last = r
        if r.status == FEASIBLE and (best is None or r.obj < best.obj):
            best, best_i = r, i
    return (best, best_i) if best is not None else (last, -1)


def max_row_violation(lp, x):
    """Largest row violation of x, each scaled by max(1, |b_i|)."""
    worst = 0.0
    for i in range(lp.m):
        act = sum(lp.val[p] * x[lp.col[p]] for p in range(lp.row_ptr[i], lp.row_ptr[i + 1]))
        bi = lp.b[i]
        if lp.sense[i] == SENSE_LE:
            v = act - bi
        elif lp.sense[i] == SENSE_GE:
            v = bi - act
        else:
            v = abs(act - bi)
        worst = max(worst, v / max(1.0, abs(bi)))
    return worst
