"""Learned warm start on the GPU: features, forward, gradients, Adam and the start
KKT against the float64 oracle; training, save / load and the warm solve."""
import math
import os

import numpy as np
import pytest

import lpgen
import test_gpu_pdlp as T
from oracle import gnn_oracle as G
from oracle import pdlp_oracle as O
from oracle import reference_lp as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as E
    E.build()
    import paper_2503_10344_gb300 as P
    return P


def lps():
    # several 64-row tiles with ragged tails, mixed senses and infinite bounds; a covering LP
    return [lpgen.random_sparse_lp(21, 300, 517, density=0.02),
            lpgen.set_cover(5, m=1000, n=4000),
            lpgen.mip_relaxation(3)]


def biased_params(seed):
    """Oracle-initialised weights with positive biases, so most units are active."""
    rng = np.random.default_rng(seed)
    d = G.unpack(G.init_params(seed))
    for name, shape in G.param_shapes():
        if name.startswith("b"):
            d[name][...] = rng.uniform(0.05, 0.3, size=shape)
    return G.pack(d).astype(np.float32)


def labels(lp, seed):
    rng = np.random.default_rng(seed)
    box = np.isfinite(lp.l) & np.isfinite(lp.u)
    xs = np.where(box, np.where(box, lp.l, 0) + rng.random(lp.n) * np.where(box, lp.u - lp.l, 0),
                  rng.normal(size=lp.n))
    y = rng.random(lp.m) * float(np.max(np.abs(lp.c)))
    ys = np.where(lp.sense == ord("L"), -y, np.where(lp.sense == ord("G"), y, y - 0.5))
    return xs, ys


def test_init_matches_oracle_bit_for_bit(P):
    m = P.GnnModel(seed=1234)
    assert np.array_equal(m.params().astype(np.float64), G.init_params(1234))


@pytest.mark.parametrize("k", range(3))
def test_features_match_oracle(P, k):
    lp = lps()[k]
    m = P.GnnModel(seed=1)
    g = m.graph(lp)
    fv, fc = g.features()
    ref = G.graph(lp)
    # both sides compute in float64 and round once to float32
    np.testing.assert_allclose(fv, ref["fv"], rtol=2.4e-7, atol=1e-30)
    np.testing.assert_allclose(fc, ref["fc"], rtol=2.4e-7, atol=1e-30)


@pytest.mark.parametrize("k", range(3))
def test_forward_matches_oracle(P, k):
    lp = lps()[k]
    theta = biased_params(7 + k)
    m = P.GnnModel(seed=0)
    m.set_params(theta)
    xs, ys = labels(lp, k)
    g = m.graph(lp, xs, ys)
    x, y, loss = m.forward(g)
    xr, yr = G.predict(theta.astype(np.float64), lp)
    # float32 arithmetic through three layers against float64
    np.testing.assert_allclose(x, xr, rtol=1e-4, atol=1e-5 * (1 + np.max(np.abs(xr))))
    np.testing.assert_allclose(y, yr, rtol=1e-4, atol=1e-5 * (1 + np.max(np.abs(yr))))
    ycanon = np.where(lp.sense == ord("L"), -ys, ys)
    assert loss == pytest.approx(G.loss(theta.astype(np.float64), G.graph(lp), xs, ycanon), rel=1e-4)


@pytest.mark.parametrize("k", range(3))
def test_gradient_matches_oracle(P, k):
    """Every parameter block of the GPU backward pass against the float64 analytic
    gradient (itself pinned to central differences): relative 1e-3."""
    lp = lps()[k]
    theta = biased_params(11 + k)
    m = P.GnnModel(seed=0)
    m.set_params(theta)
    xs, ys = labels(lp, 100 + k)
    g = m.graph(lp, xs, ys)
    m.zero_grad()
    loss = m.backward(g, scale=1.0)
    got = m.grad().astype(np.float64)
    ycanon = np.where(lp.sense == ord("L"), -ys, ys)
    L, want = G.grad(theta.astype(np.float64), G.graph(lp), xs, ycanon)
    assert loss == pytest.approx(L, rel=1e-4)
    o = 0
    for name, shape in G.param_shapes():
        cnt = int(np.prod(shape))
        gw, ww = got[o:o + cnt], want[o:o + cnt]
        o += cnt
        nrm = np.linalg.norm(ww)
        if nrm == 0:
            assert np.linalg.norm(gw) <= 1e-6, name
            continue
        assert np.linalg.norm(gw - ww) / nrm <= 1e-3, (name, np.linalg.norm(gw - ww) / nrm)
    # the scale argument multiplies, and repeated calls accumulate
    m.backward(g, scale=-0.5)
    np.testing.assert_allclose(m.grad(), 0.5 * got, rtol=1e-5, atol=1e-6 * np.max(np.abs(got)))


def test_adam_matches_oracle(P):
    rng = np.random.default_rng(5)
    theta = biased_params(3).astype(np.float64)
    m = P.GnnModel(seed=0)
    m.set_params(theta)
    th, m1, v1 = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 4):
        gr = (rng.normal(size=theta.size) * 10.0 ** rng.uniform(-4, 0, size=theta.size)).astype(np.float32)
        m.set_grad(gr)
        m.adam_step(lr=1e-2)
        th, m1, v1 = G.adam(th, gr.astype(np.float64), m1, v1, t, lr=1e-2)
        np.testing.assert_allclose(m.params(), th, rtol=1e-5, atol=1e-6)
    # the forward pass uses the bfloat16 copy of the updated masters
    lp = lps()[0]
    x, y, _ = m.forward(m.graph(lp))
    xr, yr = G.predict(m.params().astype(np.float64), lp)
    np.testing.assert_allclose(x, xr, rtol=1e-4, atol=1e-5 * (1 + np.max(np.abs(xr))))


@pytest.mark.parametrize("k", range(3))
def test_start_kkt_matches_oracle(P, k):
    lp = lps()[k]
    rng = np.random.default_rng(40 + k)
    x0 = rng.normal(size=lp.n) * 3
    y0 = rng.normal(size=lp.m) * 3   # outside the cone on some rows: projected first
    got = P.start_kkt(lp, x0, y0)
    want = O.kkt_original(lp, x0, y0)
    for key, attr in (("rel_primal_res", "rel_p"), ("rel_dual_res", "rel_d"), ("rel_gap", "rel_gap"),
                      ("rel_kkt", "rel_kkt")):
        assert got[key] == pytest.approx(getattr(want, attr), rel=1e-12, abs=1e-300), key


def test_start_kkt_of_an_optimum_is_small(P):
    lp = lpgen.mip_relaxation(4)
    obj, x, y, _ = R.highs(lp)
    assert P.start_kkt(lp, x, y)["rel_kkt"] <= 1e-8


def test_save_load_roundtrip(P, tmp_path):
    m = P.GnnModel(seed=9)
    m.set_params(biased_params(9))
    lp = lps()[1]
    xs, ys = labels(lp, 3)
    g = m.graph(lp, xs, ys)
    m.zero_grad()
    m.backward(g)
    m.adam_step()
    path = str(tmp_path / "model.bin")
    m.save(path)
    m2 = P.GnnModel.load(path)
    assert np.array_equal(m.params(), m2.params())
    g2 = m2.graph(lp, xs, ys)
    assert np.array_equal(m.forward(g)[0], m2.forward(g2)[0])
    # Adam state travels too: the same gradient gives the same step
    for mm, gg in ((m, g), (m2, g2)):
        mm.zero_grad()
        mm.backward(gg)
        mm.adam_step()
    assert np.array_equal(m.params(), m2.params())


def test_invalid_inputs(P):
    m = P.GnnModel(seed=1)
    lp = lpgen.tiny_lp(1)
    bad = lpgen.tiny_lp(1)
    bad.col = bad.col.copy()
    bad.col[0] = lp.n + 5
    with pytest.raises(P.PdlpError):
        m.graph(bad)
    g = m.graph(lp)
    with pytest.raises(P.PdlpError):
        m.backward(g)          # no labels
    with pytest.raises(P.PdlpError):
        g.set_labels(np.full(lp.n, np.nan), np.zeros(lp.m))
    with pytest.raises(P.PdlpError):
        m.set_params(np.full(G.param_count(), np.inf, dtype=np.float32))
    with pytest.raises(P.PdlpError):
        P.GnnModel.load("/nonexistent/model.bin")


def test_training_is_deterministic_and_lowers_the_loss(P):
    lpl = [lpgen.set_cover(60 + k, m=800, n=3200) for k in range(6)]
    sols = []
    for lp in lpl:
        x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-6))
        assert r["status"] == P.PDLP_OPTIMAL
        sols.append((x, y))
    runs = []
    for _ in range(2):
        m = P.GnnModel(seed=3)
        gs = [m.graph(lp, x, y) for lp, (x, y) in zip(lpl, sols)]
        losses = m.train(gs, epochs=15, batch=2, lr=3e-3)
        runs.append((losses, m.params()))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    losses = runs[0][0]
    assert losses[-1] < 0.5 * losses[0], losses


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_warm_solve_reaches_tolerance(P, prec):
    lp = lpgen.set_cover(31, m=2000, n=8000)
    m = P.GnnModel(seed=4)
    x, y, r, info = P.pdlp_solve_warm(m, lp, P.default_params(tol=1e-4, precision=prec))
    assert r["status"] == P.PDLP_OPTIMAL
    k = O.kkt_original(lp, x, y)
    assert k.rel_kkt <= 1.01e-4
    assert T.obj_err(r["primal_obj"], "set_cover(31,m=2000,n=8000)") <= T.OBJ_TOL
    assert info["used_warm"] == int(info["warm_rel_kkt"] < info["cold_rel_kkt"])
    assert info["cold_rel_kkt"] == pytest.approx(O.kkt_original(lp, np.clip(0, lp.l, lp.u),
                                                                np.zeros(lp.m)).rel_kkt, rel=1e-12)
    # no model: the plain cold solve
    x0, y0, r0, info0 = P.pdlp_solve_warm(None, lp, P.default_params(tol=1e-4, precision=prec))
    assert r0["status"] == P.PDLP_OPTIMAL and info0["used_warm"] == 0


def test_warm_start_from_the_optimum_is_taken_and_fast(P):
    """A model is not needed to check the warm path's plumbing: the solver started
    from a float64 optimum (through pdlp_solve's own x0, y0) needs one check period."""
    lp = lpgen.set_cover(32, m=2000, n=8000)
    x, y, r = P.pdlp_solve(lp, P.default_params(tol=1e-8))
    x2, y2, r2 = P.pdlp_solve(lp, P.default_params(tol=1e-4), x0=x, y0=y)
    assert r2["status"] == P.PDLP_OPTIMAL and r2["iters"] <= 64
    assert P.start_kkt(lp, x, y)["rel_kkt"] <= 1e-8
    assert math.isfinite(r2["primal_obj"])


def test_trained_network_gains_over_cold_pdlp(P):
    """What the learned start buys: a network trained on float64 PDLP solutions of 64
    covering LPs (m in [2000, 6000], n = 4m) against plain cold PDLP on 12 held-out
    LPs of the family, to relative KKT 1e-4.  Records the geometric-mean iteration
    ratio (cold / warm) for the trained and the untrained network; the trained one
    must gain, and gain more than the untrained one."""
    from paper_2503_10344_gb300 import warmstart as W
    tr = [W.family(s, 2000, 6000) for s in range(10000, 10064)]
    te = [W.family(s, 2000, 6000) for s in range(20000, 20012)]
    labels = W.label(tr)
    trained = P.GnnModel(seed=1)
    graphs = [trained.graph(lp, x, y) for lp, (x, y) in zip(tr, labels)]
    losses = trained.train(graphs, epochs=60, batch=4, lr=1e-3)
    assert losses[-1] < 0.1 * losses[0]
    _, s_tr = W.evaluate(trained, te)
    _, s_un = W.evaluate(P.GnnModel(seed=1), te)
    print("trained", s_tr, "untrained", s_un)
    assert s_tr["all_optimal"] and s_un["all_optimal"]
    assert s_tr["max_rel_obj_diff"] <= 1e-3
    assert s_tr["iters_gain"] >= 1.08, s_tr
    assert s_tr["iters_gain"] > s_un["iters_gain"], (s_tr, s_un)
