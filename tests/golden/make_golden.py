"""Write the stored expected values under tests/golden/ (run on the CPU).

Every number here comes from ``oracle/`` only: HiGHS through
``oracle.reference_lp.highs`` (the exact LP optimum) and the FP64 PDHG oracle
``oracle.pdlp_oracle.solve`` at the stated tolerance.  Inputs are the seeded
generators of ``lpgen``.  Usage:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lpgen  # noqa: E402
from oracle import pdlp_oracle as O  # noqa: E402
from oracle import reference_lp as R  # noqa: E402


def record(name, lp, oracle_tol=None, highs=True):
    out = {"instance": lp.name, "m": lp.m, "n": lp.n, "nnz": lp.nnz}
    if highs:
        t = time.time()
        obj, _, _, _ = R.highs(lp, method="highs-ipm")
        out.update({"highs_obj": obj, "highs_s": round(time.time() - t, 2)})
    if oracle_tol is not None:
        t = time.time()
        r = O.solve(lp, O.Params(tol=oracle_tol, iter_limit=200_000))
        out.update({"oracle_tol": oracle_tol, "oracle_status": r.status, "oracle_obj": r.kkt.primal_obj,
                    "oracle_rel_kkt": r.kkt.rel_kkt, "oracle_iters": r.iters,
                    "oracle_s": round(time.time() - t, 2)})
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out)


# Reference objectives of the reduced-precision checks: the FP64 oracle solved to the
# tolerance the reduced-precision solves use (rel. KKT 1e-4: "oracle_obj_tol"), and to
# 1e-6 ("oracle_obj": within a few 1e-6 of the optimum), with HiGHS's optimum beside
# them as the independent pin.  Keys are generator calls of lpgen.
OBJECTIVES = {
    "mip_relaxation(1)": lambda: lpgen.mip_relaxation(1),
    "mip_relaxation(2,m=60,n=90)": lambda: lpgen.mip_relaxation(2, m=60, n=90),
    "mip_relaxation(3)": lambda: lpgen.mip_relaxation(3),
    "set_cover(7,m=2000,n=8000)": lambda: lpgen.set_cover(7, m=2000, n=8000),
    "set_cover(31,m=2000,n=8000)": lambda: lpgen.set_cover(31, m=2000, n=8000),
    "energy_system(hours=24)": lambda: lpgen.energy_system(hours=24),
    "energy_system(hours=48)": lambda: lpgen.energy_system(hours=48),
    "random_sparse_lp(11,300,500)": lambda: lpgen.random_sparse_lp(11, 300, 500),
    "skewed_lp()": lambda: lpgen.skewed_lp(),
    "long_rows_lp()": lambda: lpgen.long_rows_lp(),
    "short_rows_lp()": lambda: lpgen.short_rows_lp(),
    "set_cover(2025)": lambda: lpgen.set_cover(2025),
}
# the batch of fixed covering sub-LPs the batch tests solve (sizes from a seeded draw)
for _k, _m in enumerate(np.random.default_rng(0).integers(2000, 6001, size=12)):
    OBJECTIVES[f"set_cover_fixed({4000 + _k},{int(_m)})"] = \
        (lambda k=_k, m=int(_m): lpgen.set_cover_fixed(4000 + k, m))
OBJ_TOL = 1e-6


def record_objective(key):
    lp = OBJECTIVES[key]()
    t = time.time()
    r = O.solve(lp, O.Params(tol=OBJ_TOL, iter_limit=400_000))
    out = {"instance": lp.name, "oracle_tol": OBJ_TOL, "oracle_status": r.status,
           "oracle_obj": r.kkt.primal_obj, "oracle_rel_kkt": r.kkt.rel_kkt, "oracle_iters": r.iters,
           "oracle_s": round(time.time() - t, 2)}
    r4 = O.solve(lp, O.Params(tol=1e-4, iter_limit=400_000))
    out.update({"oracle_tol_at": 1e-4, "oracle_obj_tol": r4.kkt.primal_obj,
                "oracle_rel_kkt_tol": r4.kkt.rel_kkt, "oracle_iters_tol": r4.iters})
    obj, _, _, _ = R.highs(lp, method="highs-ipm")
    out["highs_obj"] = obj
    return key, out


def add_tol_objectives(keys, procs=8):
    """Add the 1e-4 oracle objective to entries written before it was recorded."""
    import multiprocessing as mp
    path = os.path.join(HERE, "objectives.json")
    got = json.load(open(path))
    todo = [k for k in keys if "oracle_obj_tol" not in got.get(k, {})]
    with mp.get_context("spawn").Pool(procs) as pool:
        for key, extra in pool.imap_unordered(tol_objective, todo):
            got[key].update(extra)
            print(key, extra, flush=True)
            with open(path, "w") as f:
                json.dump(dict(sorted(got.items())), f, indent=1)


def tol_objective(key):
    lp = OBJECTIVES[key]()
    r4 = O.solve(lp, O.Params(tol=1e-4, iter_limit=400_000))
    return key, {"oracle_tol_at": 1e-4, "oracle_obj_tol": r4.kkt.primal_obj,
                 "oracle_rel_kkt_tol": r4.kkt.rel_kkt, "oracle_iters_tol": r4.iters}


def objectives(keys, procs=8):
    """Write objectives.json (merging into an existing file); one process per instance."""
    import multiprocessing as mp
    path = os.path.join(HERE, "objectives.json")
    got = json.load(open(path)) if os.path.exists(path) else {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for key, out in pool.imap_unordered(record_objective, keys):
            got[key] = out
            print(key, out, flush=True)
            with open(path, "w") as f:
                json.dump(dict(sorted(got.items())), f, indent=1)


if __name__ == "__main__":
    which = sys.argv[1:] or ["set_cover_2025", "energy_system_168h", "objectives"]
    if "objectives" in which:
        objectives(list(OBJECTIVES))
    if "tol_objectives" in which:
        add_tol_objectives(list(OBJECTIVES))
    if "set_cover_2025" in which:
        record("set_cover_2025", lpgen.set_cover(2025), oracle_tol=1e-4)
    if "energy_system_168h" in which:
        record("energy_system_168h", lpgen.energy_system(hours=168), oracle_tol=1e-4)
