"""Seeded synthetic LP / MIP-relaxation generators.

This module is the only code shared by the FP64 CPU oracle (``oracle/``) and the
CUDA path (``paper_2503_10344_gb300``).  It builds problem data only: it holds
none of the solver's arithmetic (no scaling, no PDHG step, no KKT formula).

Every instance is an LP in the form of eq. (1) of the paper (section 1),

    min c^T x  s.t.  rows of A x compared with b by a per-row sense,
                     l <= x <= u,  l, u in R u {-inf, +inf},

plus an integrality mask (the MIP of section 1) for the fix-and-propagate
consumer.  The matrix is CSR with int64 row pointers, int32 column indices and
float64 values; senses are the bytes b'L' (<=), b'G' (>=) and b'E' (=).

Workload families (their shapes stand in for the paper's instances, which are
not available here: MIPLIB 2017 in section 4.1 and the UNSEEN/REMix energy
system models of section 3, Table 1):

* :func:`mip_relaxation` -- random MIP relaxation, 200 <=-rows x 400 columns.
* :func:`set_cover` -- covering LP, all coefficients 1 (exact in bf16).
* :func:`energy_system` -- hourly energy-system LP (demand balance, storage,
  transmission on a planar graph, ramping, integer capacity expansion).
* :func:`set_cover_batch` -- uneven covering sub-LPs with columns fixed to 0/1
  the way fix-and-propagate leaves them.
* :func:`tiny_lp` -- tiny LPs with finite bounds for brute-force checks.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SENSE_LE = ord("L")
SENSE_GE = ord("G")
SENSE_EQ = ord("E")


@dataclass
class LP:
    """An LP of eq. (1) with row senses, in CSR form (see module docstring)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    b: np.ndarray        # float64 [m]
    sense: np.ndarray    # uint8 [m], one of b'L', b'G', b'E'
    c: np.ndarray        # float64 [n]
    l: np.ndarray        # float64 [n], may hold -inf
    u: np.ndarray        # float64 [n], may hold +inf
    is_int: np.ndarray   # uint8 [n]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def validate(self) -> None:
        assert self.row_ptr.dtype == np.int64 and self.row_ptr.shape == (self.m + 1,)
        assert self.col.dtype == np.int32 and self.val.dtype == np.float64
        assert self.col.shape == self.val.shape == (self.nnz,)
        assert self.row_ptr[0] == 0 and np.all(np.diff(self.row_ptr) >= 0)
        if self.nnz:
            assert self.col.min() >= 0 and self.col.max() < self.n
        for a, k in ((self.b, self.m), (self.c, self.n), (self.l, self.n), (self.u, self.n)):
            assert a.dtype == np.float64 and a.shape == (k,)
        assert self.sense.dtype == np.uint8 and self.sense.shape == (self.m,)
        assert np.all(np.isin(self.sense, (SENSE_LE, SENSE_GE, SENSE_EQ)))
        assert np.all(self.l <= self.u)

    def dense(self) -> np.ndarray:
        """Dense copy of A (small instances only)."""
        a = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            a[i, self.col[s:e]] += self.val[s:e]
        return a


def csr_from_coo(m: int, n: int, rows, cols, vals):
    """Sorted CSR (row-major, ascending columns) from COO triplets without duplicates."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if np.any(dup):
            raise ValueError("duplicate (row, col) entries")
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals


def _lp(m, n, rows, cols, vals, b, sense, c, l, u, is_int, name, **meta) -> LP:
    row_ptr, col, val = csr_from_coo(m, n, rows, cols, vals)
    lp = LP(m, n, row_ptr, col, val,
            np.ascontiguousarray(b, dtype=np.float64),
            np.ascontiguousarray(sense, dtype=np.uint8),
            np.ascontiguousarray(c, dtype=np.float64),
            np.ascontiguousarray(l, dtype=np.float64),
            np.ascontiguousarray(u, dtype=np.float64),
            np.ascontiguousarray(is_int, dtype=np.uint8), name, dict(meta))
    lp.validate()
    return lp


# --------------------------------------------------------------------------
# Random MIP relaxation (stands in for MIPLIB 2017 relaxations, section 4.1)
# --------------------------------------------------------------------------
def mip_relaxation(seed: int = 1, m: int = 200, n: int = 400, density: float = 0.02) -> LP:
    """m <=-rows, n columns: the first n/2 binary in [0,1], the rest continuous in [0,10].

    A has a Bernoulli(density) pattern with values uniform on {-5..5}\\{0};
    b = A x0 + U[0,3] for a point x0 drawn inside the bounds (integer parts
    rounded to {0,1}), so the LP and the MIP are both feasible; c ~ U[-1,1].
    """
    rng = np.random.default_rng(seed)
    nint = n // 2
    mask = rng.random((m, n)) < density
    rows, cols = np.nonzero(mask)
    mag = rng.integers(1, 6, size=rows.size)
    sgn = np.where(rng.random(rows.size) < 0.5, -1, 1)
    vals = (mag * sgn).astype(np.float64)
    l = np.zeros(n)
    u = np.concatenate([np.ones(nint), np.full(n - nint, 10.0)])
    x0 = rng.random(n) * u
    x0[:nint] = np.round(x0[:nint])
    ax0 = np.zeros(m)
    np.add.at(ax0, rows, vals * x0[cols])
    b = ax0 + rng.uniform(0.0, 3.0, size=m)
    c = rng.uniform(-1.0, 1.0, size=n)
    is_int = np.zeros(n, dtype=np.uint8)
    is_int[:nint] = 1
    return _lp(m, n, rows, cols, vals, b, np.full(m, SENSE_LE), c, l, u, is_int,
               f"mip_relaxation(seed={seed},m={m},n={n})", x0=x0)


# --------------------------------------------------------------------------
# Set cover (covering-type MIP relaxation)
# --------------------------------------------------------------------------
def _cover_pattern(rng, m: int, n: int, kmin: int = 3, kmax: int = 10):
    """Each column covers k ~ U{kmin..kmax} distinct rows chosen uniformly."""
    k = rng.integers(kmin, kmax + 1, size=n)
    draw = rng.integers(0, m, size=(n, kmax))
    take = np.arange(kmax)[None, :] < k[:, None]
    # redraw the (rare) columns whose first k picks repeat a row
    srt = np.sort(np.where(take, draw, -1 - np.arange(kmax)[None, :]), axis=1)
    bad = np.nonzero(np.any(srt[:, 1:] == srt[:, :-1], axis=1))[0]
    for j in bad:
        draw[j, : k[j]] = rng.choice(m, size=k[j], replace=False)
    rows = draw[take]
    cols = np.repeat(np.arange(n), k)
    covered = np.zeros(m, dtype=bool)
    covered[rows] = True
    unc = np.nonzero(~covered)[0]
    if unc.size:  # an uncovered row gets one random column
        rows = np.concatenate([rows, unc])
        cols = np.concatenate([cols, rng.integers(0, n, size=unc.size)])
    return rows, cols


def set_cover(seed: int = 2025, m: int = 50_000, n: int = 200_000) -> LP:
    """Covering LP: m >=-rows with b = 1, n binary columns relaxed to [0,1].

    Each column covers 3..10 distinct rows chosen uniformly (E[nnz] = 6.5 n),
    all coefficients are 1, costs are uniform integers in [1,100].
    """
    rng = np.random.default_rng(seed)
    rows, cols = _cover_pattern(rng, m, n)
    c = rng.integers(1, 101, size=n).astype(np.float64)
    return _lp(m, n, rows, cols, np.ones(rows.size), np.ones(m), np.full(m, SENSE_GE), c,
               np.zeros(n), np.ones(n), np.ones(n, dtype=np.uint8),
               f"set_cover(seed={seed},m={m},n={n})")


def set_cover_fixed(seed: int, m: int, n: int | None = None) -> LP:
    """A covering sub-LP as fix-and-propagate leaves it.

    n = 4m; a random 10-50 % of the columns get l = u in {0,1}
    (Bernoulli 0.5).  Any row whose columns are all fixed to 0 gets one of them
    un-fixed so the sub-LP stays feasible.
    """
    n = 4 * m if n is None else n
    rng = np.random.default_rng(seed)
    rows, cols = _cover_pattern(rng, m, n)
    c = rng.integers(1, 101, size=n).astype(np.float64)
    l = np.zeros(n)
    u = np.ones(n)
    frac = rng.uniform(0.10, 0.50)
    fixed = rng.random(n) < frac
    one = rng.random(n) < 0.5
    l[fixed & one] = 1.0
    u[fixed & ~one] = 0.0
    # repair: a row whose every column is fixed to 0 un-fixes one of them
    dead = (u[cols] == 0.0)
    alive_rows = np.zeros(m, dtype=bool)
    alive_rows[rows[~dead]] = True
    for i in np.nonzero(~alive_rows)[0]:
        j = cols[rows == i][0]
        u[j] = 1.0
    return _lp(m, n, rows, cols, np.ones(rows.size), np.ones(m), np.full(m, SENSE_GE), c,
               l, u, np.ones(n, dtype=np.uint8), f"set_cover_fixed(seed={seed},m={m},n={n})",
               fixed_fraction=float(frac))


def set_cover_dead(seed: int, m: int, n: int | None = None, dead: int = 1) -> LP:
    """An infeasible covering sub-LP: ``set_cover_fixed`` whose fixings leave
    ``dead`` rows with every column fixed to 0 (the conflict fix-and-propagate
    runs into when its fixings contradict a covering row)."""
    lp = set_cover_fixed(seed, m, n)
    rng = np.random.default_rng(seed + 7919)
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    u = lp.u.copy()
    l = lp.l.copy()
    for i in rng.choice(lp.m, size=dead, replace=False):
        js = lp.col[lp.row_ptr[i]:lp.row_ptr[i + 1]]
        l[js] = 0.0
        u[js] = 0.0
    return _lp(lp.m, lp.n, rows, lp.col, lp.val, lp.b, lp.sense, lp.c, l, u, lp.is_int,
               f"set_cover_dead(seed={seed},m={lp.m},dead={dead})")


def mip_relaxation_contradiction(seed: int = 1, m: int = 200, n: int = 400,
                                 density: float = 0.02) -> LP:
    """An infeasible LP: ``mip_relaxation`` plus one >=-row that repeats the
    pattern and values of a random non-empty row r with right-hand side
    b_r + U[1,3], so that row r and the new row cannot both hold."""
    lp = mip_relaxation(seed, m, n, density)
    rng = np.random.default_rng(seed + 104729)
    nz = np.nonzero(np.diff(lp.row_ptr) > 0)[0]
    r = int(rng.choice(nz))
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    seg = slice(lp.row_ptr[r], lp.row_ptr[r + 1])
    rows = np.concatenate([rows, np.full(seg.stop - seg.start, lp.m)])
    cols = np.concatenate([lp.col, lp.col[seg]])
    vals = np.concatenate([lp.val, lp.val[seg]])
    b = np.append(lp.b, lp.b[r] + rng.uniform(1.0, 3.0))
    sense = np.append(lp.sense, SENSE_GE)
    return _lp(lp.m + 1, lp.n, rows, cols, vals, b, sense, lp.c, lp.l, lp.u, lp.is_int,
               f"mip_relaxation_contradiction(seed={seed},m={m},n={n})", row=r)


def mip_relaxation_unbounded(seed: int = 1, m: int = 200, n: int = 400, density: float = 0.02,
                             rays: int = 3) -> LP:
    """An unbounded LP: ``mip_relaxation`` where ``rays`` continuous columns
    lose their upper bound, get cost -U[0.5,1] and nonpositive coefficients
    (every <=-row stays satisfied as they grow, so each is a ray of descent)."""
    lp = mip_relaxation(seed, m, n, density)
    rng = np.random.default_rng(seed + 15485863)
    js = rng.choice(np.arange(n // 2, n), size=rays, replace=False)
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    vals = lp.val.copy()
    hit = np.isin(lp.col, js)
    vals[hit] = -np.abs(vals[hit])
    u = lp.u.copy()
    c = lp.c.copy()
    u[js] = np.inf
    c[js] = -rng.uniform(0.5, 1.0, size=rays)
    return _lp(lp.m, lp.n, rows, lp.col, vals, lp.b, lp.sense, c, lp.l, u, lp.is_int,
               f"mip_relaxation_unbounded(seed={seed},m={m},n={n})", ray_cols=js)


def set_cover_batch(count: int = 256, seed0: int = 4000, mmin: int = 2_000,
                    mmax: int = 40_000) -> list[LP]:
    """``count`` uneven covering sub-LPs, m ~ U[mmin, mmax], n = 4m, seeds seed0.."""
    out = []
    for s in range(seed0, seed0 + count):
        m = int(np.random.default_rng(s).integers(mmin, mmax + 1))
        out.append(set_cover_fixed(s, m))
    return out


# --------------------------------------------------------------------------
# Energy-system-shaped LP (stands in for the ESOMs of section 3, Table 1)
# --------------------------------------------------------------------------
def _planar_lines(rng, nodes: int, lines: int):
    """Greedy non-crossing shortest-edge graph on seeded points in the unit square."""

    def cross(p1, p2, p3, p4):
        def orient(a, b, c):
            return np.sign((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        return (orient(p1, p2, p3) * orient(p1, p2, p4) < 0) and \
               (orient(p3, p4, p1) * orient(p3, p4, p2) < 0)

    for _ in range(100):
        pts = rng.random((nodes, 2))
        pairs = [(np.hypot(*(pts[a] - pts[b])), a, b)
                 for a in range(nodes) for b in range(a + 1, nodes)]
        pairs.sort()
        edges = []
        for _, a, b in pairs:
            if len(edges) == lines:
                break
            if all(a in e or b in e or not cross(pts[a], pts[b], pts[e[0]], pts[e[1]])
                   for e in edges):
                edges.append((a, b))
        # connectivity check
        seen = {0}
        stack = [0]
        while stack:
            v = stack.pop()
            for a, b in edges:
                for s, t in ((a, b), (b, a)):
                    if s == v and t not in seen:
                        seen.add(t)
                        stack.append(t)
        if len(edges) == lines and len(seen) == nodes:
            return edges
    raise RuntimeError("no connected planar line graph found")


def energy_system(seed: int = 8760, hours: int = 8760, regions: int = 20, techs: int = 6,
                  lines: int = 40, thermal: int = 4) -> LP:
    """Hourly capacity-expansion LP (8760 h x 20 regions x 6 technologies by default).

    Columns: generation g[t,r,k] >= 0; storage charge ch[t,r] in [0,P_r],
    discharge dis[t,r] in [0,P_r], level s[t,r] in [0,E_r]; flows f+[t,l],
    f-[t,l] in [0,F_l] on ``lines`` lines of a planar graph; load shedding
    shed[t,r] >= 0; integer capacities cap[r,k] in [0,50].
    Rows: demand balance (=) per (t,r); availability g - a[t,r,k] U_k cap <= 0;
    cyclic storage s[t] - s[t-1] - 0.9 ch[t] + dis[t] = 0; ramping of the
    ``thermal`` technologies g[t] - g[t-1] - R_k cap <= 0 (cyclic in t).
    Demand D_r (1 + 0.3 sin(2 pi t/24 + phi_r) + 0.2 sin(2 pi t/8760 + psi_r))
    + U[0,0.2] D_r; availability a = clip(0.5 + 0.4 sin(...) + U[0,0.2], 0.1, 1).
    Costs: generation U[1,100], shedding 1e3, capacity U[1e3,1e4] per unit.
    """
    rng = np.random.default_rng(seed)
    T, R, Kt, L = hours, regions, techs, lines
    edges = _planar_lines(rng, R, L)
    t = np.arange(T)
    # column offsets
    o_g = 0
    o_ch = o_g + T * R * Kt
    o_dis = o_ch + T * R
    o_s = o_dis + T * R
    o_fp = o_s + T * R
    o_fm = o_fp + T * L
    o_shed = o_fm + T * L
    o_cap = o_shed + T * R
    n = o_cap + R * Kt

    def gi(tt, r, k):
        return o_g + (tt * R + r) * Kt + k

    # data
    D = rng.uniform(1.0, 10.0, size=R)
    phi = rng.uniform(0, 2 * np.pi, size=R)
    psi = rng.uniform(0, 2 * np.pi, size=R)
    dem = (D[None, :] * (1 + 0.3 * np.sin(2 * np.pi * t[:, None] / 24 + phi[None, :])
                         + 0.2 * np.sin(2 * np.pi * t[:, None] / 8760 + psi[None, :]))
           + rng.uniform(0, 0.2, size=(T, R)) * D[None, :])
    ph = rng.uniform(0, 2 * np.pi, size=(R, Kt))
    per = rng.choice([24.0, 168.0, 8760.0], size=(R, Kt))
    avail = np.clip(0.5 + 0.4 * np.sin(2 * np.pi * t[:, None, None] / per[None] + ph[None])
                    + rng.uniform(0, 0.2, size=(T, R, Kt)), 0.1, 1.0)
    U = rng.uniform(1.0, 10.0, size=Kt)          # unit size of one capacity step
    Rk = rng.uniform(0.1, 1.0, size=Kt) * U      # ramp limit per unit of capacity
    P = rng.uniform(1.0, 5.0, size=R)
    E = P * rng.uniform(4.0, 10.0, size=R)
    F = rng.uniform(1.0, 10.0, size=L)
    gcost = rng.uniform(1.0, 100.0, size=(R, Kt))
    capcost = rng.uniform(1e3, 1e4, size=(R, Kt))

    rows, cols, vals, b, sense = [], [], [], [], []
    r0 = 0
    # demand balance rows: index (t, r)
    TT, RR = np.meshgrid(t, np.arange(R), indexing="ij")
    tr_row = r0 + TT * R + RR
    for k in range(Kt):
        rows.append(tr_row.ravel()); cols.append(gi(TT, RR, k).ravel()); vals.append(np.ones(T * R))
    rows.append(tr_row.ravel()); cols.append((o_dis + TT * R + RR).ravel()); vals.append(np.ones(T * R))
    rows.append(tr_row.ravel()); cols.append((o_ch + TT * R + RR).ravel()); vals.append(-np.ones(T * R))
    rows.append(tr_row.ravel()); cols.append((o_shed + TT * R + RR).ravel()); vals.append(np.ones(T * R))
    for li, (a, bb) in enumerate(edges):
        fp = o_fp + t * L + li
        fm = o_fm + t * L + li
        ra = r0 + t * R + a
        rb = r0 + t * R + bb
        rows += [ra, ra, rb, rb]
        cols += [fp, fm, fp, fm]
        vals += [-np.ones(T), np.ones(T), np.ones(T), -np.ones(T)]
    b.append(dem.ravel()); sense.append(np.full(T * R, SENSE_EQ))
    r0 += T * R
    # availability rows: index (t, r, k)
    TT3, RR3, KK3 = np.meshgrid(t, np.arange(R), np.arange(Kt), indexing="ij")
    av_row = r0 + (TT3 * R + RR3) * Kt + KK3
    rows.append(av_row.ravel()); cols.append(gi(TT3, RR3, KK3).ravel()); vals.append(np.ones(T * R * Kt))
    rows.append(av_row.ravel()); cols.append((o_cap + RR3 * Kt + KK3).ravel())
    vals.append(-(avail * U[None, None, :]).ravel())
    b.append(np.zeros(T * R * Kt)); sense.append(np.full(T * R * Kt, SENSE_LE))
    r0 += T * R * Kt
    # cyclic storage rows: index (t, r)
    st_row = r0 + TT * R + RR
    tm1 = (TT - 1) % T
    rows += [st_row.ravel()] * 4
    cols += [(o_s + TT * R + RR).ravel(), (o_s + tm1 * R + RR).ravel(),
             (o_ch + TT * R + RR).ravel(), (o_dis + TT * R + RR).ravel()]
    vals += [np.ones(T * R), -np.ones(T * R), np.full(T * R, -0.9), np.ones(T * R)]
    b.append(np.zeros(T * R)); sense.append(np.full(T * R, SENSE_EQ))
    r0 += T * R
    # ramping rows of the thermal technologies: index (t, r, k<thermal)
    TT4, RR4, KK4 = np.meshgrid(t, np.arange(R), np.arange(thermal), indexing="ij")
    rp_row = r0 + (TT4 * R + RR4) * thermal + KK4
    rows += [rp_row.ravel()] * 3
    cols += [gi(TT4, RR4, KK4).ravel(), gi((TT4 - 1) % T, RR4, KK4).ravel(),
             (o_cap + RR4 * Kt + KK4).ravel()]
    vals += [np.ones(rp_row.size), -np.ones(rp_row.size), -np.broadcast_to(Rk[None, None, :thermal],
                                                                             rp_row.shape).ravel()]
    b.append(np.zeros(rp_row.size)); sense.append(np.full(rp_row.size, SENSE_LE))
    r0 += rp_row.size
    m = r0

    l = np.zeros(n)
    u = np.full(n, np.inf)
    for o in (o_ch, o_dis):
        u[o:o + T * R] = np.tile(P, T)
    u[o_s:o_s + T * R] = np.tile(E, T)
    u[o_fp:o_fp + T * L] = np.tile(F, T)
    u[o_fm:o_fm + T * L] = np.tile(F, T)
    u[o_cap:o_cap + R * Kt] = 50.0
    c = np.zeros(n)
    c[o_g:o_ch] = np.tile(gcost.ravel(), T)
    c[o_fp:o_shed] = 0.1
    c[o_shed:o_cap] = 1e3
    c[o_cap:] = capcost.ravel()
    is_int = np.zeros(n, dtype=np.uint8)
    is_int[o_cap:] = 1
    return _lp(m, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
               np.concatenate(b), np.concatenate(sense), c, l, u, is_int,
               f"energy_system(seed={seed},hours={hours})", edges=edges)


# --------------------------------------------------------------------------
# Tiny LPs for brute-force vertex enumeration
# --------------------------------------------------------------------------
def tiny_lp(seed: int, m: int = 4, n: int = 3, eq_rows: int = 0) -> LP:
    """Dense tiny LP with finite bounds [-2,3] and mixed senses; feasible by construction."""
    rng = np.random.default_rng(seed)
    a = rng.integers(-4, 5, size=(m, n)).astype(np.float64)
    x0 = rng.uniform(-1.0, 2.0, size=n)
    ax0 = a @ x0
    sense = rng.choice([SENSE_LE, SENSE_GE], size=m)
    sense[:eq_rows] = SENSE_EQ
    slack = rng.uniform(0.0, 2.0, size=m)
    b = np.where(sense == SENSE_LE, ax0 + slack, np.where(sense == SENSE_GE, ax0 - slack, ax0))
    c = rng.integers(-5, 6, size=n).astype(np.float64)
    rows, cols = np.nonzero(a)
    return _lp(m, n, rows, cols, a[rows, cols], b, sense, c, np.full(n, -2.0), np.full(n, 3.0),
               np.zeros(n, dtype=np.uint8), f"tiny_lp(seed={seed},m={m},n={n})")


def random_sparse_lp(seed: int, m: int, n: int, density: float = 0.05, free_frac: float = 0.1,
                     eq_frac: float = 0.2) -> LP:
    """Random feasible LP with mixed senses and some infinite bounds (for parity tests).

    Objective c = A^T w + (reduced-cost term) with w of the sign each row's
    sense allows, so the LP is bounded as well as feasible.
    """
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    rows, cols = np.nonzero(mask)
    vals = rng.normal(size=rows.size) * rng.choice([0.1, 1.0, 10.0], size=rows.size)
    l = rng.uniform(-5, 0, size=n)
    u = l + rng.uniform(0.5, 5.0, size=n)
    kind = rng.random(n)
    l[kind < free_frac] = -np.inf
    u[(kind >= free_frac) & (kind < 2 * free_frac)] = np.inf
    x0 = np.where(np.isfinite(l), l, np.where(np.isfinite(u), u, 0.0)) + \
        np.where(np.isfinite(l) & np.isfinite(u), rng.random(n) * (u - l), 0.0)
    x0 = np.where(np.isfinite(l) & ~np.isfinite(u), l + rng.random(n), x0)
    x0 = np.where(~np.isfinite(l) & np.isfinite(u), u - rng.random(n), x0)
    ax0 = np.zeros(m)
    np.add.at(ax0, rows, vals * x0[cols])
    sense = np.where(rng.random(m) < 0.5, SENSE_LE, SENSE_GE).astype(np.uint8)
    sense[rng.random(m) < eq_frac] = SENSE_EQ
    slack = rng.uniform(0.0, 1.0, size=m)
    b = np.where(sense == SENSE_LE, ax0 + slack, np.where(sense == SENSE_GE, ax0 - slack, ax0))
    # bounded objective: dual-feasible w, nonnegative reduced cost on columns with
    # an infinite upper bound, nonpositive on columns with an infinite lower bound
    w = rng.uniform(0.0, 1.0, size=m)
    w = np.where(sense == SENSE_LE, -w, np.where(sense == SENSE_GE, w, rng.normal(size=m)))
    atw = np.zeros(n)
    np.add.at(atw, cols, vals * w[rows])
    rc = rng.normal(size=n)
    rc = np.where(~np.isfinite(u) & np.isfinite(l), np.abs(rc), rc)
    rc = np.where(~np.isfinite(l) & np.isfinite(u), -np.abs(rc), rc)
    rc = np.where(~np.isfinite(l) & ~np.isfinite(u), 0.0, rc)
    c = atw + rc
    return _lp(m, n, rows, cols, vals, b, sense, c, l, u, np.zeros(n, dtype=np.uint8),
               f"random_sparse_lp(seed={seed},m={m},n={n})")


# --------------------------------------------------------------------------
# Structured parity cases: skewed rows and columns, long and very short rows
# --------------------------------------------------------------------------
def skewed_lp(seed: int = 3, m: int = 6000, n: int = 3000) -> LP:
    """Random LP with a dense row (n nnz), a column in every row (m nnz), a column in
    2/3 of the rows, and a sparse remainder; mixed senses, some infinite bounds;
    feasible by construction."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    rows.append(np.zeros(n, dtype=np.int64)); cols.append(np.arange(n))
    rows.append(np.arange(1, m)); cols.append(np.zeros(m - 1, dtype=np.int64))
    r2 = np.arange(1, m)[rng.random(m - 1) < 0.66]
    rows.append(r2); cols.append(np.ones(r2.size, dtype=np.int64))
    mask = rng.random((m, n)) < 0.002
    mask[0, :] = False
    mask[:, :2] = False
    rr, cc = np.nonzero(mask)
    rows.append(rr); cols.append(cc)
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = rng.uniform(0.5, 2.0, size=rows.size) * np.where(rng.random(rows.size) < 0.3, -1, 1)
    l = np.zeros(n); u = rng.uniform(1, 3, size=n)
    u[rng.random(n) < 0.1] = np.inf
    x0 = rng.random(n) * np.where(np.isfinite(u), u, 1.0)
    ax0 = np.zeros(m)
    np.add.at(ax0, rows, vals * x0[cols])
    sense = np.where(rng.random(m) < 0.5, SENSE_LE, SENSE_GE).astype(np.uint8)
    sense[rng.random(m) < 0.1] = SENSE_EQ
    slack = rng.uniform(0, 1, size=m)
    b = np.where(sense == SENSE_LE, ax0 + slack, np.where(sense == SENSE_GE, ax0 - slack, ax0))
    c = rng.uniform(0.1, 1.0, size=n)
    return _lp(m, n, rows, cols, vals, b, sense, c, l, u, np.zeros(n, np.uint8), "skewed")


def long_rows_lp(m: int = 6500, n: int = 3000, seed: int = 5) -> LP:
    """Covering-type LP with long rows and columns: column 0 in every row, column 1
    in two thirds of the rows, row 7 with over 900 entries, a sparse remainder;
    feasible (column 0 alone covers every row)."""
    rng = np.random.default_rng(seed)
    rows = [np.arange(m), np.arange(m)[rng.random(m) < 0.66], np.full(900, 7)]
    cols = [np.zeros(m, dtype=np.int64), np.ones(rows[1].size, dtype=np.int64),
            2 + rng.choice(n - 2, size=900, replace=False)]
    mask = rng.random((m, n)) < 0.002
    mask[:, :2] = False
    mask[7, :] = False
    rr, cc = np.nonzero(mask)
    rows.append(rr)
    cols.append(cc)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.uniform(0.5, 2.0, size=rows.size)
    vals[:m] = rng.uniform(1.0, 2.0, size=m)
    return _lp(m, n, rows, cols, vals, np.ones(m), np.full(m, SENSE_GE, dtype=np.uint8),
               rng.uniform(1, 10, size=n), np.zeros(n), np.ones(n), np.zeros(n, np.uint8),
               "long_rows")


def short_rows_lp(m: int = 3000, n: int = 40000, seed: int = 9) -> LP:
    """Covering LP whose columns have one or two entries (A^T has very short rows);
    all values 1, costs U{1..100}; every row covered."""
    rng = np.random.default_rng(seed)
    cols = np.arange(n)
    rows = rng.integers(0, m, size=n)
    extra = rng.random(n) < 0.3
    rows2 = rng.integers(0, m, size=int(extra.sum()))
    r = np.concatenate([rows, rows2])
    c = np.concatenate([cols, cols[extra]])
    key = r.astype(np.int64) * n + c
    _, keep = np.unique(key, return_index=True)
    r, c = r[keep], c[keep]
    cover = np.zeros(m, bool)
    cover[r] = True
    miss = np.nonzero(~cover)[0]
    r = np.concatenate([r, miss])
    c = np.concatenate([c, rng.integers(0, n, size=miss.size)])
    key = r.astype(np.int64) * n + c
    _, keep = np.unique(key, return_index=True)
    r, c = r[keep], c[keep]
    return _lp(m, n, r, c, np.ones(r.size), np.ones(m), np.full(m, SENSE_GE, dtype=np.uint8),
               rng.integers(1, 101, n).astype(float), np.zeros(n), np.ones(n),
               np.zeros(n, np.uint8), "short_rows")
