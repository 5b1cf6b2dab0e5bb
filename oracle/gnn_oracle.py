"""FP64 CPU oracle of the learned warm start: a bipartite message-passing network
over the LP's variable / constraint graph (test infrastructure only).

The network (hidden width H = 64, three layers).  The paper has no learned part:
this network is an addition that predicts a PDLP start point, and its
definition is this file:

  features  F_v[j] = (c_j / c_max, g(l_j), g(u_j), ||A_:j|| / max, deg_j / max, 1)
                      g(v) = sign(v) log(1 + |v|) of v clipped to [-1e3, 1e3] (infinite bounds too)
            F_c[i] = (b_i / b_max, s_i, ||A_i:|| / max, deg_i / max, 1)          (s = +1 >=, -1 <=, 0 =)
  embed     H_v0 = relu(F_v W_vin + b_vin),  H_c0 = relu(F_c W_cin + b_cin)
  layer l   S_c = R H_v(l-1)          R_ij = a_ij / deg_i   (mean over a row's columns)
            H_c(l) = relu(H_c(l-1) W_cc + S_c W_cv + b_c)
            S_v = C^T H_c(l)          C_ij = a_ij / deg_j   (mean over a column's rows)
            H_v(l) = relu(H_v(l-1) W_vv + S_v W_vc + b_v)
  heads     z_x = H_v3 w_x + b_x,  x^ = l + (u - l) sigmoid(z_x)    (finite boxes; else z_x)
            z_y = H_c3 w_y + b_y,  y^ = softplus(z_y) on inequality rows, z_y on equality rows
            (canonical duals, in units of c_max)
  loss      mean_j ((x^_j - x*_j) / (u_j - l_j))^2 + mean_i (y^_i - y*_i / c_max)^2

The parameter vector is flat, in the order of ``param_shapes``; the forward
pass uses the parameters rounded to bfloat16 (the GPU stores them so) and
float64 arithmetic.  ``grad`` is the analytic backward pass; ``numeric_grad``
is central differences, the pin of ``grad``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

H = 64
LAYERS = 3
NV, NC = 6, 5
SENSE_LE, SENSE_GE, SENSE_EQ = ord("L"), ord("G"), ord("E")
BOUND_CLIP = 1e3


def param_shapes():
    shapes = [("W_vin", (NV, H)), ("b_vin", (H,)), ("W_cin", (NC, H)), ("b_cin", (H,))]
    for k in range(LAYERS):
        shapes += [(f"W_cc{k}", (H, H)), (f"W_cv{k}", (H, H)), (f"b_c{k}", (H,)),
                   (f"W_vv{k}", (H, H)), (f"W_vc{k}", (H, H)), (f"b_v{k}", (H,))]
    shapes += [("w_x", (H,)), ("b_x", (1,)), ("w_y", (H,)), ("b_y", (1,))]
    return shapes


def param_count():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unpack(theta):
    out, o = {}, 0
    for name, shp in param_shapes():
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def to_bf16(theta):
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(theta, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def graph(lp):
    """Features and normalised adjacencies of an LP (float64)."""
    a = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    deg_r = np.diff(lp.row_ptr).astype(np.float64)
    deg_c = np.bincount(lp.col, minlength=lp.n).astype(np.float64)
    nr = np.sqrt(np.asarray(a.multiply(a).sum(axis=1)).ravel())
    nc = np.sqrt(np.asarray(a.multiply(a).sum(axis=0)).ravel())
    cmax = max(float(np.max(np.abs(lp.c))) if lp.n else 0.0, 1e-12)
    bmax = max(float(np.max(np.abs(lp.b))) if lp.m else 0.0, 1e-12)
    slog = lambda v: np.sign(v) * np.log1p(np.abs(v))
    l = slog(np.clip(lp.l, -BOUND_CLIP, BOUND_CLIP))
    u = slog(np.clip(lp.u, -BOUND_CLIP, BOUND_CLIP))
    fv = np.stack([lp.c / cmax, l, u, nc / max(nc.max(initial=0.0), 1e-12),
                   deg_c / max(deg_c.max(initial=0.0), 1.0), np.ones(lp.n)], axis=1)
    s = np.where(lp.sense == SENSE_GE, 1.0, np.where(lp.sense == SENSE_LE, -1.0, 0.0))
    fc = np.stack([lp.b / bmax, s, nr / max(nr.max(initial=0.0), 1e-12),
                   deg_r / max(deg_r.max(initial=0.0), 1.0), np.ones(lp.m)], axis=1)
    rnorm = sp.diags(1.0 / np.maximum(deg_r, 1.0)) @ a
    cnorm = a @ sp.diags(1.0 / np.maximum(deg_c, 1.0))
    return {"fv": fv, "fc": fc, "R": sp.csr_matrix(rnorm), "C": sp.csr_matrix(cnorm), "cmax": cmax,
            "l": lp.l, "u": lp.u, "eq": lp.sense == SENSE_EQ, "flip": lp.sense == SENSE_LE}


def _sig(z):
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def _softplus(z):
    return np.log1p(np.exp(-np.abs(z))) + np.maximum(z, 0.0)


def forward(theta, g, keep=False):
    p = unpack(to_bf16(theta))
    relu = lambda v: np.maximum(v, 0.0)
    hv = [relu(g["fv"] @ p["W_vin"] + p["b_vin"])]
    hc = [relu(g["fc"] @ p["W_cin"] + p["b_cin"])]
    sc, sv = [], []
    for k in range(LAYERS):
        sc.append(g["R"] @ hv[-1])
        hc.append(relu(hc[-1] @ p[f"W_cc{k}"] + sc[-1] @ p[f"W_cv{k}"] + p[f"b_c{k}"]))
        sv.append(g["C"].T @ hc[-1])
        hv.append(relu(hv[-1] @ p[f"W_vv{k}"] + sv[-1] @ p[f"W_vc{k}"] + p[f"b_v{k}"]))
    zx = hv[-1] @ p["w_x"] + p["b_x"][0]
    zy = hc[-1] @ p["w_y"] + p["b_y"][0]
    box = np.isfinite(g["l"]) & np.isfinite(g["u"])
    x = np.where(box, np.where(box, g["l"], 0) + np.where(box, g["u"] - g["l"], 0) * _sig(zx), zx)
    y = np.where(g["eq"], zy, _softplus(zy))
    if keep:
        return x, y, dict(p=p, hv=hv, hc=hc, sc=sc, sv=sv, zx=zx, zy=zy, box=box)
    return x, y


def predict(theta, lp):
    """Predicted (x0, y0) in the solver's caller convention (y <= 0 on <=-rows)."""
    g = graph(lp)
    x, y = forward(theta, g)
    yk = y * g["cmax"]
    return x, np.where(g["flip"], -yk, yk)


def loss(theta, g, x_star, y_star_canon):
    x, y, _ = forward(theta, g, keep=True)
    box = np.isfinite(g["l"]) & np.isfinite(g["u"])
    rng = np.where(box, g["u"] - g["l"], 1.0)
    rng = np.where(rng > 0, rng, 1.0)
    lx = np.mean(((x - x_star) / rng) ** 2) if len(x) else 0.0
    ly = np.mean((y - y_star_canon / g["cmax"]) ** 2) if len(y) else 0.0
    return lx + ly


def grad(theta, g, x_star, y_star_canon):
    """Loss and analytic gradient with respect to the (bfloat16-rounded) parameters."""
    x, y, c = forward(theta, g, keep=True)
    p, hv, hc, sc, sv = c["p"], c["hv"], c["hc"], c["sc"], c["sv"]
    n, m = len(x), len(y)
    box = c["box"]
    rng = np.where(box, g["u"] - g["l"], 1.0)
    rng = np.where(rng > 0, rng, 1.0)
    ex = (x - x_star) / rng
    ey = y - y_star_canon / g["cmax"]
    L = (np.mean(ex ** 2) if n else 0.0) + (np.mean(ey ** 2) if m else 0.0)
    sx = _sig(c["zx"])
    dzx = (2.0 / max(n, 1)) * ex / rng * np.where(box, np.where(box, g["u"] - g["l"], 0) * sx * (1 - sx), 1.0)
    dzy = (2.0 / max(m, 1)) * ey * np.where(g["eq"], 1.0, _sig(c["zy"]))
    gr = {k: np.zeros_like(v) for k, v in p.items()}
    gr["w_x"] = hv[-1].T @ dzx
    gr["b_x"] = np.array([dzx.sum()])
    gr["w_y"] = hc[-1].T @ dzy
    gr["b_y"] = np.array([dzy.sum()])
    dhv = np.outer(dzx, p["w_x"])
    dhc = np.outer(dzy, p["w_y"])
    for k in reversed(range(LAYERS)):
        dpv = dhv * (hv[k + 1] > 0)
        gr[f"W_vv{k}"] = hv[k].T @ dpv
        gr[f"W_vc{k}"] = sv[k].T @ dpv
        gr[f"b_v{k}"] = dpv.sum(axis=0)
        dhv_prev = dpv @ p[f"W_vv{k}"].T
        dsv = dpv @ p[f"W_vc{k}"].T
        dhc = dhc + g["C"] @ dsv
        dpc = dhc * (hc[k + 1] > 0)
        gr[f"W_cc{k}"] = hc[k].T @ dpc
        gr[f"W_cv{k}"] = sc[k].T @ dpc
        gr[f"b_c{k}"] = dpc.sum(axis=0)
        dhc = dpc @ p[f"W_cc{k}"].T
        dsc = dpc @ p[f"W_cv{k}"].T
        dhv = dhv_prev + g["R"].T @ dsc
    dpv0 = dhv * (hv[0] > 0)
    gr["W_vin"] = g["fv"].T @ dpv0
    gr["b_vin"] = dpv0.sum(axis=0)
    dpc0 = dhc * (hc[0] > 0)
    gr["W_cin"] = g["fc"].T @ dpc0
    gr["b_cin"] = dpc0.sum(axis=0)
    return L, pack(gr)


def numeric_grad(theta, g, x_star, y_star_canon, idx, h=1e-6):
    """Central differences of the loss in the bfloat16-rounded parameters (computed in
    float64 on the rounded vector, so the rounding does not enter the difference)."""
    base = to_bf16(theta)
    out = []
    for i in idx:
        tp = base.copy()
        tm = base.copy()
        tp[i] += h
        tm[i] -= h
        out.append((_loss_exact(tp, g, x_star, y_star_canon) - _loss_exact(tm, g, x_star, y_star_canon))
                   / (2 * h))
    return np.array(out)


def _loss_exact(theta64, g, x_star, y_star_canon):
    """The loss with the parameters used as given (no bfloat16 rounding)."""
    saved = globals()["to_bf16"]
    try:
        globals()["to_bf16"] = lambda t: np.asarray(t, dtype=np.float64)
        return loss(theta64, g, x_star, y_star_canon)
    finally:
        globals()["to_bf16"] = saved


def init_params(seed):
    """Xavier-uniform weights from SplitMix64 draws, zero biases (float32 values)."""
    from oracle.fp_oracle import SplitMix64
    r = SplitMix64(seed)
    out = []
    for name, shp in param_shapes():
        k = int(np.prod(shp))
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            out.append(np.array([(2.0 * r.uniform() - 1.0) * lim for _ in range(k)]))
        elif name in ("w_x", "w_y"):
            lim = np.sqrt(6.0 / (H + 1))
            out.append(np.array([(2.0 * r.uniform() - 1.0) * lim for _ in range(k)]))
        else:
            out.append(np.zeros(k))
    return np.concatenate(out).astype(np.float32).astype(np.float64)


def adam(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015, Algorithm 1), t 1-based; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def project_start(lp, x, y):
    """Projection of a predicted start onto the bounds and the dual sign cone, in the
    caller's convention (y <= 0 on <=-rows, y >= 0 on >=-rows, free on =-rows)."""
    x = np.minimum(np.maximum(x, lp.l), lp.u)
    y = np.where(lp.sense == SENSE_LE, np.minimum(y, 0.0),
                 np.where(lp.sense == SENSE_GE, np.maximum(y, 0.0), y))
    return x, y
