"""Pins of the learned-warm-start oracle (CPU only).

The network's definition is the module docstring of ``oracle.gnn_oracle``; these
tests tie it to facts computed by hand, to textbook identities and to properties
every message-passing network over the bipartite graph must have.
"""
import math

import numpy as np
import pytest

import lpgen
from oracle import gnn_oracle as G


def _lp(m, n, rows, cols, vals, b, sense, c, l, u):
    return lpgen._lp(m, n, np.asarray(rows), np.asarray(cols), np.asarray(vals, dtype=float),
                     np.asarray(b, dtype=float), np.asarray([ord(s) for s in sense], dtype=np.uint8),
                     np.asarray(c, dtype=float), np.asarray(l, dtype=float), np.asarray(u, dtype=float),
                     np.zeros(n, dtype=np.uint8), "hand")


def test_bf16_rounding_ties_to_even():
    # spacing of bfloat16 at 1 is 2^-7; both inputs are exact ties
    got = G.to_bf16(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 0.0, 3.0]))
    assert got.tolist() == [1.0, 1 + 2.0 ** -6, -1.0, 0.0, 3.0]
    # just above a tie rounds up
    assert G.to_bf16(np.array([1 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1 + 2.0 ** -7


def test_param_count():
    per_layer = 4 * 64 * 64 + 2 * 64
    assert G.param_count() == 6 * 64 + 64 + 5 * 64 + 64 + 3 * per_layer + 64 + 1 + 64 + 1


def test_features_by_hand():
    # one >= row (1, 2) | b = 3; one <= row (4, 0) | b = -6
    lp = _lp(2, 2, [0, 0, 1], [0, 1, 0], [1, 2, 4], [3, -6], "GL", [1, -2], [0, -np.inf], [1, 5])
    g = G.graph(lp)
    # variables: c/cmax, signed log1p of l (inf clipped to -1e3) and u, ||A_:j|| / max, deg / max, 1
    np.testing.assert_allclose(g["fv"], [[0.5, 0, math.log(2), 1, 1, 1],
                                         [-1, -math.log(1001), math.log(6), 2 / math.sqrt(17), 0.5, 1]],
                               rtol=1e-15)
    # constraints: b/bmax, sense (+1 >=, -1 <=), ||A_i:|| / max, deg / max, 1
    np.testing.assert_allclose(g["fc"], [[0.5, 1, math.sqrt(5) / 4, 1, 1],
                                         [-1, -1, 1, 0.5, 1]], rtol=1e-15)


def _hand_net():
    """Weights that route the cost feature through unit 0 of every layer."""
    p = {name: np.zeros(shape) for name, shape in G.param_shapes()}
    p["W_vin"][0, 0] = 1.0      # H_v0[:,0] = relu(c / cmax)
    p["W_cv0"][0, 0] = 1.0      # H_c1[:,0] = S_c[:,0]
    p["W_vc0"][0, 0] = 1.0      # H_v1[:,0] = S_v[:,0]
    for k in (1, 2):
        p[f"W_vv{k}"][0, 0] = 1.0
        p[f"W_cc{k}"][0, 0] = 1.0
    p["w_x"][0] = 1.0
    p["w_y"][0] = 1.0
    return G.pack(p)


def test_message_passing_by_hand():
    # one >= row with a = (1, 2); c = (1, -2): H_v0 = (0.5, 0);
    # S_c = (1*0.5 + 2*0) / deg_row(2) = 0.25; S_v_j = a_j * 0.25 / deg_col(1) = (0.25, 0.5)
    lp = _lp(1, 2, [0, 0], [0, 1], [1, 2], [1], "G", [1, -2], [0, 0], [1, 1])
    x, y = G.forward(_hand_net(), G.graph(lp))
    sig = lambda z: 1 / (1 + math.exp(-z))
    np.testing.assert_allclose(x, [sig(0.25), sig(0.5)], rtol=1e-15)
    np.testing.assert_allclose(y, [math.log(1 + math.exp(0.25))], rtol=1e-15)
    # the same row as an equality: the dual head is the identity
    lp_eq = _lp(1, 2, [0, 0], [0, 1], [1, 2], [1], "E", [1, -2], [0, 0], [1, 1])
    _, y_eq = G.forward(_hand_net(), G.graph(lp_eq))
    np.testing.assert_allclose(y_eq, [0.25], rtol=1e-15)


def test_predict_sign_convention_and_units():
    lp = _lp(1, 2, [0, 0], [0, 1], [1, 2], [1], "L", [1, -2], [0, 0], [1, 1])
    x, y = G.predict(_hand_net(), lp)
    # canonical y is softplus(.) >= 0 in units of cmax = 2; a <=-row flips it
    _, yc = G.forward(_hand_net(), G.graph(lp))
    assert y[0] == -2.0 * yc[0] and y[0] < 0


def test_zero_weights_give_bias_heads():
    rng = np.random.default_rng(3)
    lp = lpgen.random_sparse_lp(5, 7, 9)
    theta = np.zeros(G.param_count())
    d = G.unpack(theta.copy())
    d["b_x"][0] = 0.75
    d["b_y"][0] = -0.5
    x, y = G.forward(G.pack(d), G.graph(lp))
    box = np.isfinite(lp.l) & np.isfinite(lp.u)
    sx = 1 / (1 + math.exp(-0.75))
    np.testing.assert_allclose(x[box], (lp.l + (lp.u - lp.l) * sx)[box], rtol=1e-15)
    np.testing.assert_allclose(x[~box], 0.75, rtol=1e-15)
    eq = lp.sense == ord("E")
    np.testing.assert_allclose(y[~eq], math.log(1 + math.exp(-0.5)), rtol=1e-15)
    np.testing.assert_allclose(y[eq], -0.5, rtol=1e-15)
    assert rng is not None


def test_permutation_equivariance():
    lp = lpgen.random_sparse_lp(11, 12, 15, density=0.3)
    theta = G.init_params(7)
    x, y = G.forward(theta, G.graph(lp))
    pr = np.random.default_rng(0).permutation(lp.m)
    pc = np.random.default_rng(1).permutation(lp.n)
    inv_r = np.argsort(pr)
    inv_c = np.argsort(pc)
    a = lp.dense()[pr][:, pc]
    r, c = np.nonzero(a)
    lp2 = lpgen._lp(lp.m, lp.n, r, c, a[r, c], lp.b[pr], lp.sense[pr], lp.c[pc], lp.l[pc], lp.u[pc],
                    lp.is_int[pc], "perm")
    x2, y2 = G.forward(theta, G.graph(lp2))
    np.testing.assert_allclose(x2[inv_c], x, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(y2[inv_r], y, rtol=1e-12, atol=1e-14)


def _case(seed):
    lp = lpgen.random_sparse_lp(seed, 14, 20, density=0.25)
    rng = np.random.default_rng(seed)
    theta = G.init_params(seed)
    # larger biases so that most units are active and every block carries gradient
    d = G.unpack(theta.copy())
    for name, shape in G.param_shapes():
        if name.startswith("b"):
            d[name][...] = rng.uniform(0.05, 0.3, size=shape)
    theta = G.to_bf16(G.pack(d))
    box = np.isfinite(lp.l) & np.isfinite(lp.u)
    xs = np.where(box, np.where(box, lp.l, 0) + rng.random(lp.n) * np.where(box, lp.u - lp.l, 0),
                  rng.normal(size=lp.n))
    ys = rng.normal(size=lp.m)
    return lp, theta, xs, ys


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_differences(seed):
    lp, theta, xs, ys = _case(seed)
    g = G.graph(lp)
    L, gr = G.grad(theta, g, xs, ys)
    assert abs(L - G.loss(theta, g, xs, ys)) <= 1e-15 * max(1.0, abs(L))
    # sample every parameter block
    idx, o = [], 0
    rng = np.random.default_rng(seed + 100)
    for _, shape in G.param_shapes():
        k = int(np.prod(shape))
        idx += list(o + rng.choice(k, size=min(k, 6), replace=False))
        o += k
    num = G.numeric_grad(theta, g, xs, ys, idx)
    ana = gr[idx]
    scale = np.max(np.abs(ana))
    assert scale > 0
    np.testing.assert_allclose(ana, num, rtol=1e-6, atol=1e-7 * scale)
    assert np.count_nonzero(ana) > len(idx) // 2


def test_gradient_descent_decreases_loss():
    lp, theta, xs, ys = _case(3)
    g = G.graph(lp)
    L0, gr = G.grad(theta, g, xs, ys)
    # on the exactly representable grid: step with a power of two times the gradient
    step = theta - 2.0 ** -10 * gr / np.max(np.abs(gr))
    assert G._loss_exact(step, g, xs, ys) < G._loss_exact(theta, g, xs, ys)
    assert L0 > 0


def test_adam_first_step_is_lr_times_sign():
    # at t = 1 the bias-corrected moments are g and g^2, so the step is lr * g / (|g| + eps)
    rng = np.random.default_rng(4)
    th = rng.normal(size=50)
    gr = rng.normal(size=50)
    t1, m1, v1 = G.adam(th, gr, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(t1, th - 0.01 * np.sign(gr), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * gr, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * gr * gr, rtol=1e-12)


def test_adam_constant_gradient_keeps_unit_step():
    # a constant gradient keeps mh / sqrt(vh) = sign(g) at every t
    th = np.array([1.0, -2.0])
    gr = np.array([0.3, -5.0])
    m = v = np.zeros(2)
    for t in range(1, 6):
        th_new, m, v = G.adam(th, gr, m, v, t, lr=0.1, eps=0.0)
        np.testing.assert_allclose(th - th_new, 0.1 * np.sign(gr), rtol=1e-12)
        th = th_new


def test_project_start_cones():
    lp = _lp(3, 2, [0, 1, 2], [0, 1, 0], [1, 1, 1], [0, 0, 0], "LGE", [1, 1], [0, -1], [1, 2])
    x, y = G.project_start(lp, np.array([-3.0, 5.0]), np.array([2.0, -2.0, -7.0]))
    assert x.tolist() == [0.0, 2.0]
    assert y.tolist() == [0.0, 0.0, -7.0]


def test_init_params_xavier_range_and_determinism():
    a = G.init_params(42)
    b = G.init_params(42)
    assert np.array_equal(a, b)
    d = G.unpack(a)
    lim = math.sqrt(6 / 128)
    assert np.max(np.abs(d["W_cc0"])) <= lim and np.max(np.abs(d["W_cc0"])) > 0.9 * lim
    assert np.all(d["b_v1"] == 0)
    assert a.dtype == np.float64 and np.array_equal(a.astype(np.float32).astype(np.float64), a)
