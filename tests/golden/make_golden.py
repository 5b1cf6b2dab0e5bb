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


if __name__ == "__main__":
    which = sys.argv[1:] or ["set_cover_2025", "energy_system_168h"]
    if "set_cover_2025" in which:
        record("set_cover_2025", lpgen.set_cover(2025), oracle_tol=1e-4)
    if "energy_system_168h" in which:
        record("energy_system_168h", lpgen.energy_system(hours=168), oracle_tol=1e-4)
