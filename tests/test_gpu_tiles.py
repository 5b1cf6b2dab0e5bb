"""The staged tile step kernels (float32 iterates), through the C ABI.

The tile kernels compute the same attempt as the lanes-per-row kernels with
another summation order: in the fixed-step mode (every attempt accepted, no
restarts) their float32 iterates must agree with the lanes kernels' and with the
float64 oracle's to float32 rounding, on every row -- a row updated from the
wrong stage, index or slice would miss by the size of a step.  The instances
cover tiles cut by the row cap and by the nonzero window, empty rows and
columns, equality rows, infinite bounds, and rows longer than 256 entries (cut
into slices finished by a ticket, one of them over 6,000 entries), single LPs
and batches whose work items must not straddle two LPs.  Full solves with the
tile kernels reach the tolerance under the oracle's float64 KKT.
"""
import numpy as np
import pytest

import lpgen
import test_gpu_pdlp as T
from oracle import pdlp_oracle as O

pytestmark = pytest.mark.gpu

# float32 iterates against float64 / another float32 summation order, after at most
# 60 fixed steps: a few hundred float32 roundings of relative size 6e-8 each
F32 = 2e-5


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


long_rows_lp = lpgen.long_rows_lp
short_rows_lp = lpgen.short_rows_lp


INSTANCES = {
    "mip_relaxation_200x400": (lambda: lpgen.mip_relaxation(1), "fp32", "mip_relaxation(1)"),
    "set_cover_2000x8000_pattern": (lambda: lpgen.set_cover(7, m=2000, n=8000), "bf16",
                                    "set_cover(7,m=2000,n=8000)"),
    "mip_relaxation_bf16": (lambda: lpgen.mip_relaxation(3), "bf16", "mip_relaxation(3)"),
    "energy_system_48h": (lambda: lpgen.energy_system(hours=48), "fp32", "energy_system(hours=48)"),
    "random_free_eq_300x500": (lambda: lpgen.random_sparse_lp(11, 300, 500), "fp32",
                               "random_sparse_lp(11,300,500)"),
    "long_rows_6500x3000": (lambda: long_rows_lp(), "fp32", "long_rows_lp()"),
    "short_rows_3000x40000": (lambda: short_rows_lp(), "bf16", "short_rows_lp()"),
}
_cache = {}


def inst(name):
    if name not in _cache:
        _cache[name] = INSTANCES[name][0]()
    return _cache[name]


FIXED = dict(adaptive_step=0, restarts=0, terminate=0, fixed_eta=0.9)


FORMS = [1, 2]  # staged block tiles, warp tiles


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("K", [1, 10, 60])
def test_tile_iterates_match_lanes_and_oracle(P, name, K, form):
    lp = inst(name)
    prec = INSTANCES[name][1]
    _, _, rt, it_t = P.pdlp_solve(lp, P.default_params(iter_limit=K, precision=prec, tiles=form,
                                                       **FIXED), iterates=True)
    _, _, rl, it_l = P.pdlp_solve(lp, P.default_params(iter_limit=K, precision=prec, tiles=0, **FIXED),
                                  iterates=True)
    assert rt["tiles"] == form and rl["tiles"] == 0
    assert rt["iters"] == rl["iters"] == K
    ref = O.solve(lp, O.Params(iter_limit=K, adaptive=False, restarts=False, terminate=False,
                               fixed_eta=0.9))
    for k, want in (("x_cur", ref.x_cur), ("y_cur", ref.y_cur), ("x_avg", ref.x_avg),
                    ("y_avg", ref.y_avg)):
        assert rel(it_t[k], it_l[k]) <= F32, (k, rel(it_t[k], it_l[k]))
        assert rel(it_t[k], want) <= F32, (k, rel(it_t[k], want))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", list(INSTANCES))
def test_tile_solve_reaches_tolerance(P, name, form):
    lp = inst(name)
    prec = INSTANCES[name][1]
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-4, precision=prec, tiles=form))
    assert r["status"] == P.PDLP_OPTIMAL and r["tiles"] == form
    k = O.kkt_original(lp, x, y)
    assert k.rel_kkt <= 1.01e-4, k
    assert r["rel_kkt"] == pytest.approx(k.rel_kkt, rel=1e-6, abs=1e-12)
    assert T.obj_err(r["primal_obj"], INSTANCES[name][2]) <= T.OBJ_TOL


@pytest.mark.parametrize("form", FORMS)
def test_tiles_are_deterministic(P, form):
    lp = inst("long_rows_6500x3000")
    runs = [P.pdlp_solve(lp, P.default_params(iter_limit=300, terminate=0, precision="fp32",
                                              tiles=form), iterates=True) for _ in range(2)]
    for k in ("x_cur", "y_cur", "x_avg", "y_avg"):
        assert np.array_equal(runs[0][3][k], runs[1][3][k]), k
    assert runs[0][2]["attempts"] == runs[1][2]["attempts"]


def test_float64_ignores_tiles(P):
    lp = inst("mip_relaxation_200x400")
    _, _, r = P.pdlp_solve(lp, P.default_params(iter_limit=10, terminate=0, tiles=1))
    assert r["tiles"] == 0


def test_tiles_parameter_is_checked(P):
    with pytest.raises(P.PdlpError):
        P.pdlp_solve(inst("mip_relaxation_200x400"), P.default_params(tiles=3))


def batch_lps():
    return [lpgen.mip_relaxation(1), lpgen.set_cover(7, m=2000, n=8000),
            lpgen.energy_system(hours=24), lpgen.random_sparse_lp(11, 300, 500), long_rows_lp(),
            lpgen.mip_relaxation(2, m=60, n=90), short_rows_lp(m=500, n=3000, seed=4)]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("K", [1, 30])
def test_batch_tiles_match_lanes(P, K, form):
    """Every LP of a float32 batch ends at the same point with tiles and with lanes
    (fixed step, no restarts: the returned point of each LP after K steps)."""
    lps = batch_lps()
    xt, yt, rt = P.pdlp_solve_batch(lps, P.default_params(iter_limit=K, precision="fp32", tiles=form,
                                                          **FIXED))
    xl, yl, rl = P.pdlp_solve_batch(lps, P.default_params(iter_limit=K, precision="fp32", tiles=0,
                                                          **FIXED))
    for lp, a, b, c, d, r1, r2 in zip(lps, xt, xl, yt, yl, rt, rl):
        assert r1["tiles"] == form and r2["tiles"] == 0
        assert r1["iters"] == r2["iters"] == K
        assert rel(a, b) <= F32, (lp.name, rel(a, b))
        assert rel(c, d) <= F32, (lp.name, rel(c, d))


@pytest.mark.parametrize("form", FORMS)
def test_batch_tiles_reach_tolerance(P, form):
    lps = batch_lps()
    xs, ys, res = P.pdlp_solve_batch(lps, P.default_params(tol=1e-4, precision="fp32", tiles=form))
    for lp, x, y, r in zip(lps, xs, ys, res):
        assert r["status"] == P.PDLP_OPTIMAL and r["tiles"] == form, (lp.name, r)
        assert O.kkt_original(lp, x, y).rel_kkt <= 1.01e-4, lp.name
