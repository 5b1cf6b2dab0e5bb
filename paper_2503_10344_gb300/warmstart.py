"""Learned warm start pipeline: instance family, labels, training and the warm-vs-cold
evaluation (host orchestration; every solve, forward, backward and optimiser step
runs in libpdlp.so).

Family: covering LPs shaped like the set-cover relaxation (every coefficient 1,
b = 1, costs uniform integers in [1, 100], each column covering 3-10 uniformly
chosen rows), m ~ U[mmin, mmax] drawn from the instance seed, n = 4m.  Labels are
float64 PDLP solutions at relative KKT 1e-6 from the batched solver.  The network
is trained on the GPU by gnn_train; evaluation solves each held-out LP cold and
warm (pdlp_solve_warm: the prediction is used only when its KKT beats the cold
start's) and reports iterations and times, with the shifted geometric mean of
the paper's measurement conventions (section 4, shift 1 s) and the unshifted one.

Usage (from the repository root, which holds the ``lpgen`` input generators):
    python -m paper_2503_10344_gb300.warmstart --train 2000 --test 100 --out result.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B
from . import gnn as N


def family(seed: int, mmin: int = 5_000, mmax: int = 50_000):
    import lpgen
    m = int(np.random.default_rng(seed).integers(mmin, mmax + 1))
    return lpgen.set_cover(seed, m=m, n=4 * m)


def label(lps, tol: float = 1e-6, nnz_budget: int = 60_000_000):
    """float64 PDLP solutions (x, y) of every LP, solved in batches of about nnz_budget."""
    out = [None] * len(lps)
    prm = B.default_params(tol=tol, precision="fp64")
    i = 0
    while i < len(lps):
        j, tot = i, 0
        while j < len(lps) and (j == i or tot + lps[j].nnz <= nnz_budget):
            tot += lps[j].nnz
            j += 1
        xs, ys, res = B.pdlp_solve_batch(lps[i:j], prm)
        for k, (x, y, r) in enumerate(zip(xs, ys, res)):
            if r["status"] != B.PDLP_OPTIMAL:
                raise RuntimeError(f"label solve of LP {i + k} ended with status {r['status']}")
            out[i + k] = (x, y)
        i = j
    return out


def shifted_geomean(v, shift: float) -> float:
    v = np.asarray(v, dtype=np.float64)
    return float(np.exp(np.mean(np.log(v + shift))) - shift)


def evaluate(model, lps, tol: float = 1e-4, precision: str = "bf16"):
    """Cold and warm solves of every LP; per-LP records and a summary."""
    prm = B.default_params(tol=tol, precision=precision)
    rows = []
    for lp in lps:
        t0 = time.perf_counter()
        _, _, rc = B.pdlp_solve(lp, prm)
        tc = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, _, rw, info = N.pdlp_solve_warm(model, lp, prm)
        tw = time.perf_counter() - t0
        rows.append({"m": lp.m, "n": lp.n, "cold_iters": rc["iters"], "warm_iters": rw["iters"],
                     "cold_s": rc["setup_s"] + rc["solve_s"],
                     "warm_s": rw["setup_s"] + rw["solve_s"] + info["predict_s"],
                     "cold_call_s": tc, "warm_call_s": tw,
                     "cold_status": rc["status"], "warm_status": rw["status"],
                     "cold_rel_kkt": rc["rel_kkt"], "warm_rel_kkt": rw["rel_kkt"],
                     "used_warm": info["used_warm"], "start_kkt_warm": info["warm_rel_kkt"],
                     "start_kkt_cold": info["cold_rel_kkt"],
                     "cold_obj": rc["primal_obj"], "warm_obj": rw["primal_obj"]})
    ci = [r["cold_iters"] for r in rows]
    wi = [r["warm_iters"] for r in rows]
    cs = [r["cold_s"] for r in rows]
    ws = [r["warm_s"] for r in rows]
    summary = {
        "instances": len(rows),
        "all_optimal": all(r["cold_status"] == B.PDLP_OPTIMAL and r["warm_status"] == B.PDLP_OPTIMAL
                           for r in rows),
        "fallback_rate": 1.0 - float(np.mean([r["used_warm"] for r in rows])),
        "iters_geomean": {"cold": shifted_geomean(ci, 0.0), "warm": shifted_geomean(wi, 0.0)},
        "time_s_geomean": {"cold": shifted_geomean(cs, 0.0), "warm": shifted_geomean(ws, 0.0)},
        "time_s_shifted_geomean_1s": {"cold": shifted_geomean(cs, 1.0), "warm": shifted_geomean(ws, 1.0)},
        "iters_gain": shifted_geomean(ci, 0.0) / max(shifted_geomean(wi, 0.0), 1e-300),
        "time_gain": shifted_geomean(cs, 0.0) / max(shifted_geomean(ws, 0.0), 1e-300),
        "max_rel_obj_diff": max(abs(r["warm_obj"] - r["cold_obj"]) / (1 + abs(r["cold_obj"]))
                                for r in rows),
    }
    return rows, summary


def run(train: int, test: int, mmin: int, mmax: int, epochs: int, batch: int, lr: float,
        seed0_train: int = 10_000, seed0_test: int = 20_000, model_path: str | None = None,
        precision: str = "bf16", label_tol: float = 1e-6, log=print):
    t0 = time.perf_counter()
    tr = [family(s, mmin, mmax) for s in range(seed0_train, seed0_train + train)]
    te = [family(s, mmin, mmax) for s in range(seed0_test, seed0_test + test)]
    t_gen = time.perf_counter() - t0
    log(f"generated {train} + {test} instances in {t_gen:.1f} s")
    t0 = time.perf_counter()
    labels = label(tr, tol=label_tol)
    t_lab = time.perf_counter() - t0
    log(f"labelled in {t_lab:.1f} s")
    model = N.GnnModel(seed=1)
    graphs = [model.graph(lp, x, y) for lp, (x, y) in zip(tr, labels)]
    t0 = time.perf_counter()
    losses = model.train(graphs, epochs=epochs, batch=batch, lr=lr)
    t_train = time.perf_counter() - t0
    log(f"trained {epochs} epochs in {t_train:.1f} s; loss {losses[0]:.4g} -> {losses[-1]:.4g}")
    for g in graphs:
        g.close()
    if model_path:
        model.save(model_path)
    rows, summary = evaluate(model, te, precision=precision)
    return {"train": train, "test": test, "m_range": [mmin, mmax], "epochs": epochs,
            "batch": batch, "lr": lr, "label_tol": label_tol, "precision": precision,
            "generate_s": t_gen, "label_s": t_lab, "train_s": t_train,
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
            "losses": [float(v) for v in losses], "summary": summary, "per_lp": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--mmin", type=int, default=5_000)
    ap.add_argument("--mmax", type=int, default=50_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--precision", default="bf16", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--model", default=None, help="save the trained model here")
    ap.add_argument("--out", default=None, help="write the result JSON here")
    a = ap.parse_args()
    res = run(a.train, a.test, a.mmin, a.mmax, a.epochs, a.batch, a.lr, model_path=a.model,
              precision=a.precision)
    s = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    print(json.dumps(res["summary"]))


if __name__ == "__main__":
    main()
