"""Batched solves: many uneven LPs in one set of
launches, each with its own step size, restarts and termination."""
import numpy as np
import pytest

import lpgen
import test_gpu_pdlp as T
from oracle import pdlp_oracle as O
from oracle import reference_lp as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


MIXED_KEYS = ["mip_relaxation(1)", "set_cover(7,m=2000,n=8000)", "energy_system(hours=24)",
              "random_sparse_lp(11,300,500)", "skewed_lp()", "mip_relaxation(2,m=60,n=90)"]


def mixed_lps():
    return [lpgen.mip_relaxation(1), lpgen.set_cover(7, m=2000, n=8000), lpgen.energy_system(hours=24),
            lpgen.random_sparse_lp(11, 300, 500), lpgen.skewed_lp(), lpgen.mip_relaxation(2, m=60, n=90)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_mixed_batch_reaches_tolerance(P, prec):
    lps = mixed_lps()
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-4, precision=prec))
    for lp, key, x, y, r in zip(lps, MIXED_KEYS, xs, ys, res):
        assert r["status"] == P.PDLP_OPTIMAL, (lp.name, r)
        k = O.kkt_original(lp, x, y)
        assert k.rel_kkt <= 1.01e-4, (lp.name, k)
        assert r["rel_kkt"] == pytest.approx(k.rel_kkt, rel=1e-6, abs=1e-12)
        assert T.obj_err(r["primal_obj"], key) <= T.OBJ_TOL, lp.name
    assert len({r["iters"] for r in res}) > 1  # the LPs stop independently


@pytest.mark.parametrize("K", [1, 10, 60])
def test_fp64_batch_matches_oracle_per_lp(P, K):
    """Each LP of a float64 batch follows its own oracle run (the returned point, the
    better of current and average at the last check, to 1e-9)."""
    lps = mixed_lps()
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(iter_limit=K, terminate=0))
    for lp, x, y, r in zip(lps, xs, ys, res):
        ref = O.solve(lp, O.Params(iter_limit=K, terminate=False))
        assert r["iters"] == ref.iters == K and r["attempts"] == ref.attempts
        for got, want in ((x, ref.x), (y, ref.y)):
            err = np.linalg.norm(got - want) / max(1.0, np.linalg.norm(want))
            assert err <= 1e-9, (lp.name, err)


def test_batch_of_fixed_cover_subproblems(P):
    """Covering sub-LPs with 10-50 % of the columns fixed to 0/1 (as fix-and-propagate
    leaves them), float32 iterates on the pattern matrix."""
    sizes = [int(m) for m in np.random.default_rng(0).integers(2000, 6001, size=12)]
    lps = [lpgen.set_cover_fixed(4000 + k, m) for k, m in enumerate(sizes)]
    for tiles in (0, 1, 2):
        xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-4, precision="bf16", tiles=tiles))
        for k, (lp, x, y, r) in enumerate(zip(lps, xs, ys, res)):
            assert r["status"] == P.PDLP_OPTIMAL and r["precision_used"] == 3 and r["tiles"] == tiles
            assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-4
            assert np.all(x >= lp.l) and np.all(x <= lp.u)
            assert T.obj_err(r["primal_obj"], f"set_cover_fixed({4000 + k},{sizes[k]})") <= T.OBJ_TOL


def test_batch_rejects_an_invalid_member(P):
    lps = mixed_lps()[:3]
    bad = lpgen.mip_relaxation(5)
    bad.l = bad.l.copy()
    bad.l[0] = 2.0  # l > u
    with pytest.raises(P.PdlpError, match="LP 3"):
        P.pdlp_solve_batch(lps + [bad])


def test_autotuned_batch(P):
    """The tuner picks the lanes of the whole batch in dry mode: the float64 batch with
    autotune follows the batch run with the picked lanes set explicitly (to rounding: the
    long-row cut-off follows the lanes known at setup, so a long row may be summed by a
    block in one run and by a lane group in the other); a float32 autotuned batch reaches
    the tolerance."""
    lps = mixed_lps()
    kw = dict(iter_limit=60, terminate=0)
    xs1, ys1, r1 = P.pdlp_solve_batch(lps, P.default_params(autotune=1, **kw))
    la, lt = r1[0]["lanes_A"], r1[0]["lanes_AT"]
    assert la in (2, 4, 8, 16, 32) and lt in (2, 4, 8, 16, 32)  # float64: no one-lane form
    xs2, ys2, r2 = P.pdlp_solve_batch(lps, P.default_params(lanes_A=la, lanes_AT=lt, **kw))
    for a, b in zip(xs1 + ys1, xs2 + ys2):
        assert np.linalg.norm(a - b) <= 1e-11 * max(1.0, np.linalg.norm(b))
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-4, precision="bf16", autotune=1))
    for lp, x, y, r in zip(lps, xs, ys, res):
        assert r["status"] == P.PDLP_OPTIMAL, lp.name
        assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-4, lp.name


def test_batch_kernel_timing(P):
    """pdlp_time_kernels_batch times every fused kernel over the whole batch; the bytes are
    the single-LP formulas summed over the LPs' sizes, and a solve afterwards is unaffected."""
    lps = [lpgen.set_cover_fixed(4000 + k, m) for k, m in enumerate((2000, 3000, 4000))]
    prm = P.default_params(tol=1e-4, precision="bf16")
    kt = P.time_kernels_batch(lps, prm, reps=5)
    for k in ("primal_step", "dual_step", "attempt", "kkt_rows", "kkt_cols"):
        assert kt[k]["ms"] > 0 and kt[k]["bytes"] > 0, k
    assert kt["persistent_attempt"]["ms"] == 0.0 and kt["kkt_block"]["ms"] == 0.0
    one = [P.time_kernels(P.DeviceLP(lp), prm, reps=2) for lp in lps]
    for k in ("primal_step", "dual_step", "kkt_rows", "kkt_cols"):
        # the same formulas, up to the per-LP row-pointer terminators
        assert kt[k]["bytes"] == pytest.approx(sum(o[k]["bytes"] for o in one), rel=1e-5), k
    _, _, res = P.pdlp_solve_batch(lps, prm)
    assert all(r["status"] == P.PDLP_OPTIMAL for r in res)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_device_batch_equals_host_batch(P, prec):
    """pdlp_solve_batch_device (inputs and outputs on the device, the caller's stream)
    runs the same setup and iteration as the host entry point: the same points bit for
    bit, the same counts; no upload time."""
    lps = mixed_lps()
    prm = P.default_params(tol=1e-4, precision=prec)
    xh, yh, rh = P.pdlp_solve_batch(lps, prm)
    xd, yd, rd = P.pdlp_solve_batch_device([P.DeviceLP(lp) for lp in lps], prm)
    for a, b, c, d, r1, r2 in zip(xh, xd, yh, yd, rh, rd):
        assert np.array_equal(a, b.cpu().numpy()) and np.array_equal(c, d.cpu().numpy())
        assert r1["iters"] == r2["iters"] and r1["status"] == r2["status"]
        assert r2["upload_s"] == 0.0 and r1["upload_s"] > 0.0


def test_device_batch_rejects_an_invalid_member(P):
    lps = mixed_lps()[:3]
    bad = lpgen.mip_relaxation(5)
    bad.col = bad.col.copy()
    bad.col[3] = bad.n  # column index out of range
    with pytest.raises(P.PdlpError, match="LP 3: invalid input: column index"):
        P.pdlp_solve_batch_device([P.DeviceLP(lp) for lp in lps + [bad]])


# ---------------------------------------------------------------- persistent batch
@pytest.mark.parametrize("K", [1, 10, 60])
def test_persistent_batch_float64_equals_two_launch_form(P, K):
    """persistent = 1 over a batch: one cooperative kernel per check period walks both
    launch maps with the resident grid, three grid barriers per attempt.  Each virtual
    block keeps its rows and partial-sum slot and each LP's decision adds its slots in
    order, so float64 runs equal the two-launch form bit for bit (fixed step, K steps;
    adaptive steps with restarts below)."""
    lps = mixed_lps()
    kw = dict(iter_limit=K, terminate=0, adaptive_step=0, fixed_eta=0.9)
    x1, y1, r1 = P.pdlp_solve_batch(lps, P.default_params(persistent=1, **kw))
    x0, y0, r0 = P.pdlp_solve_batch(lps, P.default_params(persistent=0, **kw))
    for a, b, c, d, ra, rb in zip(x1, x0, y1, y0, r1, r0):
        assert ra["persistent_form"] == 1 and rb["persistent_form"] == 0
        assert ra["iters"] == rb["iters"] == K
        assert np.array_equal(a, b) and np.array_equal(c, d)


def test_persistent_batch_adaptive_matches_oracle_per_lp(P):
    lps = mixed_lps()
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(iter_limit=60, terminate=0, persistent=1))
    for lp, x, y, r in zip(lps, xs, ys, res):
        ref = O.solve(lp, O.Params(iter_limit=60, terminate=False))
        assert r["iters"] == ref.iters == 60 and r["attempts"] == ref.attempts
        for got, want in ((x, ref.x), (y, ref.y)):
            assert np.linalg.norm(got - want) <= 1e-9 * max(1.0, np.linalg.norm(want)), lp.name


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_persistent_batch_reaches_tolerance(P, prec):
    """Every LP stops on its own (its check due, then optimal) while the others keep
    stepping inside the same launch; fewer kernel launches than two per attempt."""
    lps = mixed_lps()
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-4, precision=prec, persistent=1))
    _, _, res0 = P.pdlp_solve_batch(lps, P.default_params(tol=1e-4, precision=prec))
    for lp, key, x, y, r in zip(lps, MIXED_KEYS, xs, ys, res):
        assert r["status"] == P.PDLP_OPTIMAL and r["persistent_form"] == 1, (lp.name, r)
        k = O.kkt_original(lp, x, y)
        assert k.rel_kkt <= 1.01e-4, (lp.name, k)
        assert T.obj_err(r["primal_obj"], key) <= T.OBJ_TOL, lp.name
    assert len({r["iters"] for r in res}) > 1
    assert res[0]["kernel_launches"] < res0[0]["kernel_launches"]


def test_persistent_batch_float32_iterates(P):
    """Float32 persistent and two-launch batch runs differ only in how rows are grouped
    into partial sums (the persistent kernel walks rows with the plain traversal): after
    30 fixed steps every LP's point agrees to float32 rounding."""
    lps = mixed_lps()
    kw = dict(iter_limit=30, terminate=0, adaptive_step=0, restarts=0, fixed_eta=0.9, precision="fp32")
    x1, y1, _ = P.pdlp_solve_batch(lps, P.default_params(persistent=1, **kw))
    x0, y0, _ = P.pdlp_solve_batch(lps, P.default_params(persistent=0, lanes_A=2, lanes_AT=2, **kw))
    for lp, a, b, c, d in zip(lps, x1, x0, y1, y0):
        assert np.linalg.norm(a - b) <= 2e-5 * max(1.0, np.linalg.norm(b)), lp.name
        assert np.linalg.norm(c - d) <= 2e-5 * max(1.0, np.linalg.norm(d)), lp.name


def test_persistent_two_is_rejected_for_batches(P):
    with pytest.raises(P.PdlpError, match="single LPs"):
        P.pdlp_solve_batch(mixed_lps()[:2], P.default_params(persistent=2))


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_with_degenerate_members(P, persistent):
    """A batch holding an LP without rows, a 1 x 1 LP and LPs of ordinary size: every member
    ends optimal with its own answer, in both batch forms."""
    n = 5
    norows = lpgen._lp(0, n, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0), np.zeros(0),
                       np.zeros(0, np.uint8), np.array([1.0, -2.0, 0.0, 3.0, -0.5]),
                       np.array([-1.0, 0.0, 0.5, -3.0, 2.0]), np.array([1.0, 2.0, 1.0, 5.0, 7.0]),
                       np.zeros(n, np.uint8), "norows")
    one = lpgen._lp(1, 1, np.zeros(1, np.int64), np.zeros(1, np.int64), np.array([2.0]),
                    np.array([1.0]), np.array([lpgen.SENSE_GE], np.uint8), np.array([1.0]),
                    np.array([0.0]), np.array([3.0]), np.zeros(1, np.uint8), "one")
    lps = [lpgen.mip_relaxation(1), norows, one, lpgen.set_cover(7, m=2000, n=8000)]
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-6, persistent=persistent))
    assert all(r["status"] == P.PDLP_OPTIMAL for r in res), [r["status"] for r in res]
    np.testing.assert_allclose(xs[1], [-1.0, 2.0, 0.5, -3.0, 7.0], atol=1e-6)
    assert xs[2][0] == pytest.approx(0.5, abs=1e-6) and ys[2][0] == pytest.approx(0.5, abs=1e-6)
    for lp, x, y in ((lps[0], xs[0], ys[0]), (lps[3], xs[3], ys[3])):
        assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-6
