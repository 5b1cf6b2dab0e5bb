"""FP64 CPU oracle for the PDLP iteration (restarted, diagonally preconditioned PDHG).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA product path
never calls it and shares no code with it (the only common module is the
seeded input generator ``lpgen``).

What is computed, and from where
--------------------------------
The paper (Kempke & Koch, arXiv 2503.10344) solves the LP relaxation of eq. (1)
(section 1),  min c^T x  s.t.  A x <= b,  l <= x <= u,  with GPU PDLP to a
*relative* tolerance (section 4, "Hardware and software": relative primal/dual
tolerances; 1e-4 and 1e-6 in section 4.1 and Table "lp_results").  It runs PDLP
as a black box and does not restate its internals.  Every internal step below
is therefore the published PDLP method as this project reads it; each such
reading is marked "reading" where it is used below:

  A0  canonical form: flip <=-rows to >=, K = S A, q = S b; dual cone Y has
      y_i >= 0 on inequality rows and y_i free on equality rows.
  A2  Ruiz equilibration (10 passes, inf-norm) then Pock-Chambolle (alpha = 1)
      diagonal scaling, K~ = D_r K D_c.
  A2b optional bound-objective rescaling (one of the algorithmic variants of
      PDLP; off by default): after A2 the objective is divided by
      gamma = 1 + ||c~||_2 and the right-hand side and the variable bounds by
      beta = 1 + ||q~||_2, so PDHG runs on (K~, q~/beta, c~/gamma, l~/beta,
      u~/beta) and a point (x', y') of that problem is x = beta D_c x',
      y = gamma D_r y' in the original units (reading: the factors are the
      scaled norms plus one, both bounds and b share beta).  Everything in
      A3-A10 is taken in the rescaled space; A8, A11 and A12 measure the
      unscaled point as before.
  A3  x0 = proj_[l~,u~](0), y0 = 0, omega0 = ||c~|| / ||q~|| (if both > 1e-10,
      else 1), eta0 = 1 / max|K~_ij|.  With a primal-weight hint (x_h, y_h),
      omega0 = ||y~_h|| / ||x~_h|| of the hint projected and scaled like a
      start (if both > 1e-10) -- an addition for the learned warm start, not
      part of the paper's cold PDLP.
  A4/A5  PDHG step  x' = proj_X(x - (eta/omega)(c~ - K~^T y)),
                    y' = proj_Y(y + eta*omega (q~ - K~ (2x' - x))).
  A6  adaptive step size: eta_bar = (omega ||dx||^2 + ||dy||^2/omega)
      / (2 |dy^T K~ dx|); eta_next = min((1-(k+1)^-0.3) eta_bar,
      (1+(k+1)^-0.6) eta), k = attempt count (1-based); accept iff
      eta <= eta_bar, else retry from the same point with eta_next.
  A7  step-size-weighted averages since the last restart.
  A8  every ``check_period`` accepted iterations: relative KKT of the current
      and the average iterate on the unscaled data (Part I below).
  A9  KKT restart (beta_suff 0.2, beta_nec 0.8, beta_art 0.36) on the scaled
      KKT_omega = sqrt(omega ||r_p~||^2 + ||r_d~||^2 / omega + gap^2).
  A9b optional normalized-duality-gap restarts (the restart metric of the
      original PDLP; off by default; every detail is a reading): the same
      three rules with rho(r; z) in place of KKT_omega, where for a candidate
      z (current or average, scaled) r = ||z - z_last||_omega,
      ||(x, y)||_omega^2 = omega ||x||^2 + ||y||^2 / omega, and
        rho(r; z) = max{ L(x, y^) - L(x^, y) : z^ in X x Y,
                         ||z^ - z||_omega <= r } / r
      (0 when r = 0) with L(x, y) = c~^T x - y^T K~ x + q~^T y, i.e. the
      maximum of g^T (z^ - z), g = (K~^T y - c~, q~ - K~ x), over the
      trust region.  Its maximiser is z^(t) = (proj_X(x + t g_x / omega),
      proj_Y(y + t omega g_y)) with t the largest step whose distance
      d(t) = ||z^(t) - z||_omega is at most r (d is nondecreasing and
      d(t) <= t N, N^2 = ||g_x||^2 / omega + omega ||g_y||^2).  t is found
      by bisection from t0 = r / N: the smallest k in 0..63 with
      d(t0 2^k) >= r (bisection over k, 6 steps; t = t0 2^63 if none), then
      44 halvings of [t0 2^(k-1), t0 2^k], t the final lower end.  The
      candidate is the one with the smaller rho (tie: current); the restart
      point's rho (the one that triggered it, with the radius that brought it
      there) is the reference of the next epoch; before the first restart the
      reference is +inf.
  A10 primal weight omega <- exp(0.5 ln(dy/dx) + 0.5 ln omega) on restart.
  A11 stop when min(relKKT(current), relKKT(average)) <= tol; unscale.
  A12 infeasibility certificates (PDLP's test on iterate differences; the
      paper only says FP aborts when the LP is infeasible, section 2, so
      every detail is a reading): at each check, after the tolerance test,
      take the unscaled displacement since the last restart anchor,
      dx = x - x_last and dy = y - y_last (the points as A11 returns them).
      Dual ray y^ = proj_Y(dy), lambda^ = -K^T y^,
        d^ = q^T y^ + sum_{l finite} l lambda^+ - sum_{u finite} u lambda^-,
        r^_d = lambda^+ [l = -inf] + lambda^- [u = +inf];
      primal infeasible iff d^ > kappa |d^|_terms and ||r^_d|| <= eps d^
      (Farkas: no x in [l,u] with Kx >= q exists when r^_d = 0 and d^ > 0).
      Primal ray x^ = dx projected onto the recession cone of [l, u]
      (0 where both bounds are finite, dx+ where only l is, dx- where only u
      is), r^_p,i = max(0, -(Kx^)_i) on >=-rows, |(Kx^)_i| on =-rows,
        p^ = c^T x^;
      dual infeasible iff -p^ > kappa |p^|_terms and ||r^_p|| <= eps (-p^).
      eps = 1e-8; |.|_terms is the sum of the magnitudes of the terms the
      objective adds up, and kappa = 1e-9 keeps an objective that is zero up
      to rounding (a feasible LP whose ray objective is exactly 0) from
      passing.  The primal test is taken first.  The certificate is returned
      in place of the dual (primal infeasible) or primal (dual infeasible)
      output.
  A14 optional reflected restarted Halpern PDHG (one of the algorithmic
      variants of PDLP; off by default; every detail is a reading, the paper
      runs PDLP as a black box): a constant step eta = 0.998 / L, where L is
      the power-iteration estimate of ||K~||_2 (64 passes of
      v <- K~^T K~ v / ||K~^T K~ v|| from v = 1/sqrt(n), L = the square root of
      the last norm); no step-size search and no averages.  Each step maps the
      Halpern iterate z^k = (x^k, y^k) through the PDHG operator T (A4/A5 with
      tau = eta/omega, sigma = eta*omega) and mixes
        z^{k+1} = (k+1)/(k+2) ((1+rho) T(z^k) - rho z^k) + 1/(k+2) z^a,
      rho the reflection coefficient (1: reflected), z^a the anchor (the start,
      then the last restart point), k the steps since the last restart.  The
      candidate the checks (A8, A11, A12) evaluate and the solver returns is
      the latest T(z^k).  Restarts compare the fixed-point residual of the
      latest step, r = ||z^k - T(z^k)||_P with ||(dx, dy)||_P^2 =
      (omega/eta) ||dx||^2 + ||dy||^2 / (omega eta) - 2 dy^T K~ dx, with r_0,
      the residual of the epoch's first step, by the beta_suff / beta_nec /
      beta_art rules of A9 (r in place of KKT_omega; "no progress" = r above
      the previous check's r); a restart takes the candidate as the new
      anchor and iterate (k = 0) after the A10 primal-weight update from the
      candidate's scaled distance to the previous anchor.
  A13 primal feasibility polishing (``polish_primal``): the same iteration on
      the LP with its objective replaced by 0, from (x, 0).  Dual feasibility
      polishing (``polish_dual``): the same iteration on the LP with b = 0 and
      every finite bound moved to 0, from (0, y).

Part I (the definition every result is judged by): for a point x in [l,u] and
y in Y of the canonical problem,
  r_p,i = max(0, q_i - (Kx)_i) on >=-rows and q_i - (Kx)_i on =-rows,
  lambda = c - K^T y,  r_d,j = lambda+_j [l_j = -inf] + lambda-_j [u_j = +inf],
  primal = c^T x,  dual = q^T y + sum_{l finite} l lambda+ - sum_{u finite} u lambda-,
  rel_p = ||r_p|| / (1 + ||q||), rel_d = ||r_d|| / (1 + ||c||),
  rel_gap = |primal - dual| / (1 + |primal| + |dual|),
  rel_kkt = max(rel_p, rel_d, rel_gap).

Every step is written as its definition: scipy.sparse matrix-vector products
and numpy elementwise operations, no fusion and no reordering.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

SENSE_LE, SENSE_GE, SENSE_EQ = ord("L"), ord("G"), ord("E")

STATUS_OPTIMAL = 1
STATUS_ITER_LIMIT = 2
STATUS_TIME_LIMIT = 3
STATUS_PRIMAL_INFEASIBLE = 5
STATUS_DUAL_INFEASIBLE = 6


# ---------------------------------------------------------------- A0 -------
def canonicalize(lp):
    """A0: K = S A, q = S b with S_ii = -1 on <=-rows and +1 otherwise.

    Returns (K as scipy CSR, q, is_eq mask, S).  Eq. (1) of the paper states
    the LP with A x <= b; the row senses generalise it (reading).
    """
    a = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    s = np.where(lp.sense == SENSE_LE, -1.0, 1.0)
    k = sp.diags(s) @ a
    return sp.csr_matrix(k), s * lp.b, lp.sense == SENSE_EQ, s


def proj_box(x, l, u):
    """Projection onto [l, u] (infinite bounds allowed)."""
    return np.minimum(np.maximum(x, l), u)


def proj_dual(y, is_eq):
    """Projection onto Y: y_i >= 0 on inequality rows, free on equality rows."""
    return np.where(is_eq, y, np.maximum(y, 0.0))


# ---------------------------------------------------------------- A2 -------
def ruiz_pock_chambolle(k, ruiz_iters=10, pc_alpha=1.0):
    """A2: diagonal preconditioners D_r, D_c with K~ = D_r K D_c (reading).

    Ruiz pass: r_i = sqrt(max_j |K~_ij|), s_j = sqrt(max_i |K~_ij|), both taken
    from the same K~, a zero row/column gets factor 1, then D_r /= r, D_c /= s.
    Pock-Chambolle pass (alpha): r_i = sqrt(sum_j |K~_ij|^(2-alpha)),
    s_j = sqrt(sum_i |K~_ij|^alpha), applied the same way.
    """
    m, n = k.shape
    dr = np.ones(m)
    dc = np.ones(n)
    absk = abs(k).tocsr()
    for _ in range(ruiz_iters):
        kt = sp.diags(dr) @ absk @ sp.diags(dc)
        rmax = kt.max(axis=1).toarray().ravel() if m and n else np.zeros(m)
        cmax = kt.max(axis=0).toarray().ravel() if m and n else np.zeros(n)
        r = np.where(rmax > 0, np.sqrt(rmax), 1.0)
        s = np.where(cmax > 0, np.sqrt(cmax), 1.0)
        dr = dr / r
        dc = dc / s
    if pc_alpha is not None:
        kt = (sp.diags(dr) @ absk @ sp.diags(dc)).tocsr()
        rs = np.asarray(kt.power(2.0 - pc_alpha).sum(axis=1)).ravel()
        cs = np.asarray(kt.power(pc_alpha).sum(axis=0)).ravel()
        r = np.where(rs > 0, np.sqrt(rs), 1.0)
        s = np.where(cs > 0, np.sqrt(cs), 1.0)
        dr = dr / r
        dc = dc / s
    return dr, dc


# ----------------------------------------------------------- Part I --------
@dataclass
class KKT:
    primal_obj: float
    dual_obj: float
    r_p: float      # ||r_p||_2 (absolute)
    r_d: float      # ||r_d||_2 (absolute)
    gap: float      # |primal - dual| (absolute)
    rel_p: float
    rel_d: float
    rel_gap: float

    @property
    def rel_kkt(self) -> float:
        return max(self.rel_p, self.rel_d, self.rel_gap)

    def kkt_omega(self, omega: float) -> float:
        """A9: sqrt(omega ||r_p||^2 + ||r_d||^2 / omega + gap^2) (reading)."""
        return math.sqrt(omega * self.r_p ** 2 + self.r_d ** 2 / omega + self.gap ** 2)


def kkt_canonical(k, q, is_eq, c, l, u, x, y) -> KKT:
    """Part I residuals of (x, y) for the canonical LP (K, q, c, l, u)."""
    kx = k @ x
    r_p = np.where(is_eq, q - kx, np.maximum(q - kx, 0.0))
    lam = c - k.T @ y
    lp_ = np.maximum(lam, 0.0)
    lm = np.maximum(-lam, 0.0)
    r_d = np.where(np.isinf(l), lp_, 0.0) + np.where(np.isinf(u), lm, 0.0)
    primal = float(c @ x)
    lfin = np.isfinite(l)
    ufin = np.isfinite(u)
    dual = float(q @ y + l[lfin] @ lp_[lfin] - u[ufin] @ lm[ufin])
    nrp = float(np.linalg.norm(r_p))
    nrd = float(np.linalg.norm(r_d))
    gap = abs(primal - dual)
    return KKT(primal, dual, nrp, nrd, gap,
               nrp / (1.0 + float(np.linalg.norm(q))),
               nrd / (1.0 + float(np.linalg.norm(c))),
               gap / (1.0 + abs(primal) + abs(dual)))


def kkt_original(lp, x, y_orig) -> KKT:
    """Part I residuals on the original data, y in the caller's sign convention.

    Convention: y_i <= 0 on <=-rows, y_i >= 0 on >=-rows, free on =-rows,
    reduced costs lambda = c - A^T y (the signs the Dual / RedCost fixing
    strategies of section 2 consume).  x is first clipped to [l, u] and y to
    its cone, as every PDLP iterate already is.
    """
    k, q, is_eq, s = canonicalize(lp)
    x = proj_box(np.asarray(x, dtype=np.float64), lp.l, lp.u)
    y = proj_dual(s * np.asarray(y_orig, dtype=np.float64), is_eq)
    return kkt_canonical(k, q, is_eq, lp.c, lp.l, lp.u, x, y)


# ---------------------------------------------------------------- solver ---
@dataclass
class Params:
    tol: float = 1e-4
    iter_limit: int = 100_000
    time_limit_s: float = float("inf")
    check_period: int = 64
    ruiz_iters: int = 10
    pc_alpha: float | None = 1.0
    adaptive: bool = True           # A6; False = every step accepted with fixed eta
    restarts: bool = True           # A9/A10
    fixed_eta: float | None = None  # overrides eta0 (fixed-step mode)
    fixed_omega: float | None = None  # overrides omega0
    bound_objective_rescaling: bool = False  # A2b
    restart_metric: str = "kkt"     # A9 "kkt" | A9b "ndg" (normalized duality gap)
    halpern: bool = False           # A14: reflected restarted Halpern PDHG
    halpern_reflection: float = 1.0  # A14: rho
    halpern_eta_scale: float = 0.998  # A14: eta = scale / L
    power_iters: int = 64           # A14: passes of the power iteration for L
    terminate: bool = True          # stop at tol (False: run to iter_limit)
    beta_suff: float = 0.2
    beta_nec: float = 0.8
    beta_art: float = 0.36
    omega_smooth: float = 0.5
    omega_hint: object = None       # (x_h, y_h) caller convention: omega0 from their scaled norms
    detect_infeasibility: bool = True  # A12 (only where terminate is set)
    eps_infeasible: float = 1e-8
    record_checks: int = 0          # keep the unscaled current point of the last n checks
    # replay: step size and accept flag of every attempt taken from another run's
    # decision trace (eta_bar and all restart decisions are still computed here)
    replay_eta: object = None
    replay_accepted: object = None


@dataclass
class Result:
    status: int
    iters: int          # accepted iterations
    attempts: int       # all step attempts (k)
    restarts: int
    x: np.ndarray       # chosen output, unscaled
    y: np.ndarray       # chosen output, unscaled, caller sign convention
    kkt: KKT
    x_cur: np.ndarray   # unscaled current iterate
    y_cur: np.ndarray
    x_avg: np.ndarray   # unscaled average iterate (current iterate if the average is empty)
    y_avg: np.ndarray
    eta: float
    omega: float
    used_average: bool
    solve_s: float
    trace: list = field(default_factory=list)
    attempt_trace: list = field(default_factory=list)  # (eta, eta_bar, accepted) per attempt
    check_trace: list = field(default_factory=list)    # (restart kind, omega after) per check
    rays: list = field(default_factory=list)           # Rays of every check (A12)
    check_points: list = field(default_factory=list)   # unscaled current x of the last checks
    x_halpern: np.ndarray | None = None  # A14: the Halpern iterate z^k, unscaled (not clipped)
    y_halpern: np.ndarray | None = None
    spectral_norm: float | None = None   # A14: L, the estimate of ||K~||_2


@dataclass
class Rays:
    """A12: the two candidate certificates of one check, unscaled, canonical signs."""
    x_ray: np.ndarray
    y_ray: np.ndarray
    dual_ray_obj: float     # d^
    dual_ray_res: float     # ||r^_d||
    dual_ray_abs: float     # sum of |terms| of d^
    primal_ray_obj: float   # p^
    primal_ray_res: float   # ||r^_p||
    primal_ray_abs: float   # sum of |c_j x^_j|

    def primal_infeasible(self, eps, kappa=1e-9):
        d = self.dual_ray_obj
        return d > 0 and d > kappa * self.dual_ray_abs and self.dual_ray_res <= eps * d

    def dual_infeasible(self, eps, kappa=1e-9):
        p = -self.primal_ray_obj
        return p > 0 and p > kappa * self.primal_ray_abs and self.primal_ray_res <= eps * p


def power_norm(kt, iters=64) -> float:
    """A14: L = sqrt(||K~^T K~ v||) after ``iters`` passes of the power iteration
    v <- K~^T K~ v / ||K~^T K~ v|| from v = 1/sqrt(n) (0 for an empty K~ or when a
    pass gives the zero vector).  For a unit v, ||K~^T K~ v|| <= ||K~||_2^2, so L
    never exceeds ||K~||_2."""
    n = kt.shape[1]
    if n == 0 or kt.nnz == 0:
        return 0.0
    v = np.full(n, 1.0 / math.sqrt(n))
    s = 0.0
    for _ in range(iters):
        w = kt.T @ (kt @ v)
        s = float(np.linalg.norm(w))
        if s == 0.0:
            return 0.0
        v = w / s
    return math.sqrt(s)


NDG_K_STEPS = 6
NDG_HALVINGS = 44


def trust_region_gap(gx, gy, x, y, lt, ut, is_eq, omega, r):
    """A9b: max g^T (z^ - z) over z^ in X x Y with ||z^ - z||_omega <= r, by the
    bisection on t of the module docstring.  Returns (value, t)."""
    if r <= 0.0:
        return 0.0, 0.0
    nn = math.sqrt(float(gx @ gx) / omega + omega * float(gy @ gy))
    if nn == 0.0:
        return 0.0, 0.0

    def step(t):
        return proj_box(x + (t / omega) * gx, lt, ut) - x, proj_dual(y + (t * omega) * gy, is_eq) - y

    def dist(t):
        dx, dy = step(t)
        return math.sqrt(omega * float(dx @ dx) + float(dy @ dy) / omega)

    t0 = r / nn
    if dist(t0 * 2.0 ** 63) < r:
        t = t0 * 2.0 ** 63
    else:
        lo, hi = -1, 63            # d(t0 2^lo) < r <= d(t0 2^hi) (lo = -1: below k = 0)
        for _ in range(NDG_K_STEPS):
            mid = (lo + hi) // 2
            if mid == lo:
                break
            if dist(t0 * 2.0 ** mid) >= r:
                hi = mid
            else:
                lo = mid
        a, b = t0 * 2.0 ** (hi - 1), t0 * 2.0 ** hi
        for _ in range(NDG_HALVINGS):
            mid = 0.5 * (a + b)
            if dist(mid) >= r:
                b = mid
            else:
                a = mid
        t = a
    dx, dy = step(t)
    return float(gx @ dx) + float(gy @ dy), t


def normalized_gap(kt, ktt, ct, qt, lt, ut, is_eq, omega, xs, ys, x_last, y_last):
    """A9b: rho(r; z) for the scaled candidate z = (xs, ys), r its omega-distance from
    the last restart point (0 when r = 0)."""
    dx, dy = xs - x_last, ys - y_last
    r = math.sqrt(omega * float(dx @ dx) + float(dy @ dy) / omega)
    if r == 0.0:
        return 0.0
    gx = ktt @ ys - ct
    gy = qt - kt @ xs
    val, _ = trust_region_gap(gx, gy, xs, ys, lt, ut, is_eq, omega, r)
    return val / r


def recession_proj(dx, l, u):
    """Projection onto the recession cone of [l, u]: {d : d_j >= 0 where l_j is
    finite, d_j <= 0 where u_j is finite}."""
    d = np.where(np.isfinite(l), np.maximum(dx, 0.0), dx)
    return np.where(np.isfinite(u), np.minimum(d, 0.0), d)


def rays_canonical(k, q, is_eq, c, l, u, dx, dy) -> Rays:
    """A12 on the canonical LP from the displacements (dx, dy)."""
    y_ray = proj_dual(dy, is_eq)
    lam = -(k.T @ y_ray)
    lp_ = np.maximum(lam, 0.0)
    lm = np.maximum(-lam, 0.0)
    r_d = np.where(np.isinf(l), lp_, 0.0) + np.where(np.isinf(u), lm, 0.0)
    lfin = np.isfinite(l)
    ufin = np.isfinite(u)
    d_obj = float(q @ y_ray + l[lfin] @ lp_[lfin] - u[ufin] @ lm[ufin])
    d_abs = float(np.abs(q) @ np.abs(y_ray) + np.abs(l[lfin]) @ lp_[lfin]
                  + np.abs(u[ufin]) @ lm[ufin])
    x_ray = recession_proj(dx, l, u)
    kx = k @ x_ray
    r_p = np.where(is_eq, np.abs(kx), np.maximum(-kx, 0.0))
    return Rays(x_ray, y_ray, d_obj, float(np.linalg.norm(r_d)), d_abs,
                float(c @ x_ray), float(np.linalg.norm(r_p)), float(np.abs(c) @ np.abs(x_ray)))


def solve(lp, params: Params | None = None, x0=None, y0=None) -> Result:
    """PDLP (A0-A11) in FP64, step by step as listed in the module docstring."""
    p = params or Params()
    t0 = time.perf_counter()
    # A0
    k, q, is_eq, s = canonicalize(lp)
    # A2
    dr, dc = ruiz_pock_chambolle(k, p.ruiz_iters, p.pc_alpha)
    kt = sp.csr_matrix(sp.diags(dr) @ k @ sp.diags(dc))
    ktt = sp.csr_matrix(kt.T)
    ct = dc * lp.c
    qt = dr * q
    lt = lp.l / dc
    ut = lp.u / dc
    if p.bound_objective_rescaling:
        # A2b: gamma, beta from the scaled norms; the rescaled problem's point maps
        # back through D_c beta and D_r gamma (unscaling below uses dc, dr so folded)
        gamma = 1.0 + float(np.linalg.norm(ct))
        beta = 1.0 + float(np.linalg.norm(qt))
        ct = ct / gamma
        qt = qt / beta
        lt = lt / beta
        ut = ut / beta
        dc = dc * beta
        dr = dr * gamma
    # A3
    if x0 is None:
        x = proj_box(np.zeros(lp.n), lt, ut)
    else:
        x = proj_box(np.asarray(x0, dtype=np.float64) / dc, lt, ut)
    if y0 is None:
        y = np.zeros(lp.m)
    else:
        y = proj_dual(s * np.asarray(y0, dtype=np.float64) / dr, is_eq)
    nc, nq = float(np.linalg.norm(ct)), float(np.linalg.norm(qt))
    omega = nc / nq if (nc > 1e-10 and nq > 1e-10) else 1.0
    if p.omega_hint is not None:
        xh = proj_box(np.asarray(p.omega_hint[0], dtype=np.float64) / dc, lt, ut)
        yh = proj_dual(s * np.asarray(p.omega_hint[1], dtype=np.float64) / dr, is_eq)
        nxh, nyh = float(np.linalg.norm(xh)), float(np.linalg.norm(yh))
        if nxh > 1e-10 and nyh > 1e-10:
            omega = nyh / nxh
    kmax = float(abs(kt).max()) if kt.nnz else 0.0
    eta = 1.0 / kmax if kmax > 0 else 1.0
    spectral = None
    if p.halpern:
        # A14: a constant step from the power-iteration estimate of ||K~||_2
        spectral = power_norm(kt, p.power_iters)
        eta = p.halpern_eta_scale / spectral if spectral > 0 else 1.0
    if p.fixed_eta is not None:
        eta = p.fixed_eta
    if p.fixed_omega is not None:
        omega = p.fixed_omega

    def scaled_kkt(xs, ys):
        return kkt_canonical(kt, qt, is_eq, ct, lt, ut, xs, ys)

    def unscaled_kkt(xs, ys):
        # the unscaled point is clipped to [l, u] as the returned point is (A11)
        return kkt_canonical(k, q, is_eq, lp.c, lp.l, lp.u, proj_box(dc * xs, lp.l, lp.u), dr * ys)

    attempts = 0
    it = 0
    restarts = 0
    sum_x = np.zeros(lp.n)
    sum_y = np.zeros(lp.m)
    sum_w = 0.0
    x_last, y_last = x.copy(), y.copy()
    kkt_last = scaled_kkt(x, y)          # "last restart" KKT starts at z0
    kkt_prev_cand = math.inf
    ndg_last = math.inf                  # A9b: rho of the last restart point
    last_restart_it = 0
    status = STATUS_ITER_LIMIT
    trace = []
    chosen_avg = False
    chosen_kkt = None

    def average():
        if sum_w > 0:
            return sum_x / sum_w, sum_y / sum_w
        return x, y

    attempt_trace = []
    check_trace = []
    rays = []
    check_points = []
    cert = None

    def unscaled_point(xs, ys):
        return proj_box(dc * xs, lp.l, lp.u), dr * ys

    # A14 state: the Halpern iterate, its anchor, the steps since the last restart,
    # the residuals of the epoch's first step, of the latest step and of the last check
    xh, yh = x.copy(), y.copy()
    xa0, ya0 = x.copy(), y.copy()
    h_k = 0
    h_r0 = h_res = h_prev = math.inf

    while it < p.iter_limit:
        attempts += 1
        if p.halpern:
            # A14: the PDHG operator at the Halpern iterate (A4, A5 with the constant step)
            x_new = proj_box(xh - (eta / omega) * (ct - ktt @ yh), lt, ut)
            y_new = proj_dual(yh + eta * omega * (qt - kt @ (2.0 * x_new - xh)), is_eq)
            dx = x_new - xh
            dy = y_new - yh
            # fixed-point residual ||z^k - T(z^k)||_P
            r2 = (omega / eta * float(dx @ dx) + float(dy @ dy) / (omega * eta)
                  - 2.0 * float(dy @ (kt @ dx)))
            h_res = math.sqrt(max(r2, 0.0))
            if h_k == 0:
                h_r0 = h_res
            # the reflected Halpern mix with the anchor
            lam = (h_k + 1.0) / (h_k + 2.0)
            rho = p.halpern_reflection
            xh = lam * ((1.0 + rho) * x_new - rho * xh) + (1.0 - lam) * xa0
            yh = lam * ((1.0 + rho) * y_new - rho * yh) + (1.0 - lam) * ya0
            h_k += 1
            attempt_trace.append((eta, h_res, True))
            # the candidate: no averages (sum_w stays 0, so average() is the candidate)
            x, y = x_new, y_new
            it += 1
        else:
            if p.replay_eta is not None:
                eta = float(p.replay_eta[attempts - 1])
            # A4: primal step
            x_new = proj_box(x - (eta / omega) * (ct - ktt @ y), lt, ut)
            # A5: dual step with extrapolation 2x' - x
            y_new = proj_dual(y + eta * omega * (qt - kt @ (2.0 * x_new - x)), is_eq)
            eta_used = eta
            # A6: the step-size bound of this attempt
            dx = x_new - x
            dy = y_new - y
            denom = 2.0 * abs(float(dy @ (kt @ dx)))
            num = omega * float(dx @ dx) + float(dy @ dy) / omega
            eta_bar = num / denom if denom > 0 else math.inf
            accept = True
            if p.adaptive:
                eta_next = min((1.0 - (attempts + 1) ** -0.3) * eta_bar,
                               (1.0 + (attempts + 1) ** -0.6) * eta)
                accept = not (eta > eta_bar)
            if p.replay_accepted is not None:
                accept = bool(p.replay_accepted[attempts - 1])
            attempt_trace.append((eta_used, eta_bar, accept))
            if not accept:
                trace.append(("reject", attempts, eta, eta_bar))
                eta = eta_next
                continue
            if p.adaptive:
                eta = eta_next
            # accept; A7 running sums weighted by the step that produced the iterate
            x, y = x_new, y_new
            sum_x += eta_used * x
            sum_y += eta_used * y
            sum_w += eta_used
            it += 1
        last = it >= p.iter_limit
        if it % p.check_period == 0 or last:
            # A8
            xa, ya = average()
            kc = unscaled_kkt(x, y)
            ka = unscaled_kkt(xa, ya)
            chosen_avg = ka.rel_kkt < kc.rel_kkt
            chosen_kkt = ka if chosen_avg else kc
            trace.append(("check", it, kc.rel_kkt, ka.rel_kkt, eta, omega))
            if p.record_checks > 0:
                # the current point as the check sees it (A11's clipped unscaled point),
                # reference points for the heuristic from PDLP's cycling (section 5)
                check_points.append(proj_box(dc * x, lp.l, lp.u))
                del check_points[:-p.record_checks]
            if p.terminate and chosen_kkt.rel_kkt <= p.tol:
                status = STATUS_OPTIMAL
                check_trace.append((0, omega))
                break
            # A12
            xu, yu = unscaled_point(x, y)
            xl, yl = unscaled_point(x_last, y_last)
            ry = rays_canonical(k, q, is_eq, lp.c, lp.l, lp.u, xu - xl, yu - yl)
            rays.append(ry)
            if p.terminate and p.detect_infeasibility:
                if ry.primal_infeasible(p.eps_infeasible):
                    status = STATUS_PRIMAL_INFEASIBLE
                elif ry.dual_infeasible(p.eps_infeasible):
                    status = STATUS_DUAL_INFEASIBLE
                if status != STATUS_ITER_LIMIT:
                    cert = ry
                    check_trace.append((0, omega))
                    break
            if time.perf_counter() - t0 > p.time_limit_s:
                status = STATUS_TIME_LIMIT
                check_trace.append((0, omega))
                break
            if last:
                check_trace.append((0, omega))
                break
            kind = 0
            if p.restarts and p.halpern:
                # A14: the A9 rules on the fixed-point residual
                do_restart = (h_res <= p.beta_suff * h_r0
                              or (h_res <= p.beta_nec * h_r0 and h_res > h_prev)
                              or (it - last_restart_it) >= p.beta_art * it)
                if do_restart:
                    # A10 from the candidate's distance to the previous anchor
                    ddx = float(np.linalg.norm(x - x_last))
                    ddy = float(np.linalg.norm(y - y_last))
                    if ddx > 1e-10 and ddy > 1e-10:
                        omega = math.exp(p.omega_smooth * math.log(ddy / ddx)
                                         + (1.0 - p.omega_smooth) * math.log(omega))
                    x_last, y_last = x.copy(), y.copy()
                    xh, yh = x.copy(), y.copy()
                    xa0, ya0 = x.copy(), y.copy()
                    h_k = 0
                    h_prev = math.inf
                    last_restart_it = it
                    restarts += 1
                    kind = 1
                    trace.append(("restart", it, False, omega))
                else:
                    h_prev = h_res
            elif p.restarts:
                # A9
                sc = scaled_kkt(x, y)
                sa = scaled_kkt(xa, ya)
                if p.restart_metric == "ndg":
                    # A9b: the normalized duality gaps at the candidates' own radii
                    mc = normalized_gap(kt, ktt, ct, qt, lt, ut, is_eq, omega, x, y,
                                        x_last, y_last)
                    ma = normalized_gap(kt, ktt, ct, qt, lt, ut, is_eq, omega, xa, ya,
                                        x_last, y_last)
                    m_last = ndg_last
                else:
                    mc, ma = sc.kkt_omega(omega), sa.kkt_omega(omega)
                    m_last = kkt_last.kkt_omega(omega)
                use_avg = ma < mc
                cand_x, cand_y = (xa, ya) if use_avg else (x, y)
                cand_k = sa if use_avg else sc
                m_cand = ma if use_avg else mc
                do_restart = (m_cand <= p.beta_suff * m_last
                              or (m_cand <= p.beta_nec * m_last and m_cand > kkt_prev_cand)
                              or (it - last_restart_it) >= p.beta_art * it)
                if do_restart:
                    # A10
                    ddx = float(np.linalg.norm(cand_x - x_last))
                    ddy = float(np.linalg.norm(cand_y - y_last))
                    if ddx > 1e-10 and ddy > 1e-10:
                        omega = math.exp(p.omega_smooth * math.log(ddy / ddx)
                                         + (1.0 - p.omega_smooth) * math.log(omega))
                    x, y = cand_x.copy(), cand_y.copy()
                    x_last, y_last = x.copy(), y.copy()
                    kkt_last = cand_k
                    ndg_last = m_cand
                    kkt_prev_cand = math.inf
                    last_restart_it = it
                    sum_x[:] = 0.0
                    sum_y[:] = 0.0
                    sum_w = 0.0
                    restarts += 1
                    kind = 2 if use_avg else 1
                    trace.append(("restart", it, bool(use_avg), omega))
                else:
                    kkt_prev_cand = m_cand
            check_trace.append((kind, omega))
    xa, ya = average()
    if chosen_kkt is None:  # no check ran (iter_limit == 0)
        chosen_kkt = unscaled_kkt(x, y)
        chosen_avg = False
    xo, yo = (xa, ya) if chosen_avg else (x, y)

    def unscale_x(xs):
        # A11: x = D_c x~, clipped to [l, u] so the rounding of D_c (l / D_c)
        # cannot leave the box (reading)
        return proj_box(dc * xs, lp.l, lp.u)

    def unscale_y(ys):
        # A11: y = D_r y~, then back to the caller's sign convention
        return s * (dr * ys)

    x_out, y_out = unscale_x(xo), unscale_y(yo)
    if status == STATUS_PRIMAL_INFEASIBLE:
        y_out = s * cert.y_ray     # the Farkas ray, caller's sign convention
    elif status == STATUS_DUAL_INFEASIBLE:
        x_out = cert.x_ray
    return Result(status, it, attempts, restarts,
                  x_out, y_out, chosen_kkt,
                  unscale_x(x), unscale_y(y), unscale_x(xa), unscale_y(ya),
                  eta, omega, chosen_avg, time.perf_counter() - t0, trace, attempt_trace,
                  check_trace, rays, check_points,
                  dc * xh if p.halpern else None,
                  s * (dr * yh) if p.halpern else None, spectral)


# ---------------------------------------------------------------- A13 ------
def polish_primal(lp, x, params: Params | None = None) -> Result:
    """A13: primal feasibility polishing of a point x (reading of PDLP's feasibility
    polishing; the paper only needs feasible points for its heuristic, section 2).

    The same PDHG (A0-A12) on the primal feasibility problem -- the LP with its
    objective replaced by 0 -- started from (x, y = 0).  With c = 0 every dual
    iterate that stays 0 leaves x unchanged, so a feasible x is a fixed point;
    otherwise the iteration moves x onto the feasible set with y as the
    multipliers of the violated rows.  The result's x is the polished point
    (status OPTIMAL: relative KKT of the feasibility problem <= tol, so
    ||r_p|| <= tol (1 + ||q||)); an infeasible LP ends PRIMAL_INFEASIBLE.
    """
    import copy
    lp0 = copy.copy(lp)
    lp0.c = np.zeros(lp.n)
    return solve(lp0, params, x0=x, y0=None)


def polish_dual(lp, y, params: Params | None = None) -> Result:
    """A13, dual side: dual feasibility polishing of a dual point y (reading of
    PDLP's feasibility polishing, as for ``polish_primal``; y in the caller's
    sign convention of ``kkt_original``).

    The same PDHG (A0-A12) on the dual feasibility problem -- the LP with its
    right-hand side replaced by 0 and every finite bound by 0 (infinite bounds
    stay infinite) -- started from (x = 0, y).  The dual of that problem has the
    original dual's feasible set (y in Y, lambda = c - K^T y carried by the
    bounds that are finite) and a zero objective, so a dual-feasible y leaves
    x = 0 and is a fixed point; otherwise y moves onto the dual feasible set
    with x as the multipliers of the violated reduced costs.  The result's y is
    the polished dual point (status OPTIMAL: ||r_d|| <= tol (1 + ||c||)); an
    LP whose dual is infeasible ends DUAL_INFEASIBLE with a ray of descent.
    """
    import copy
    lp0 = copy.copy(lp)
    lp0.b = np.zeros(lp.m)
    lp0.l = np.where(np.isfinite(lp.l), 0.0, lp.l)
    lp0.u = np.where(np.isfinite(lp.u), 0.0, lp.u)
    return solve(lp0, params, x0=None, y0=y)
