"""pdlp_solve_device_noalloc, the solve for callers that cannot allocate device memory.

Such callers (device memory owned by another allocator, loops that must not
reach the CUDA driver's allocator, code with no workspace to hand over) get the
same solve with its scratch in the library's static 64 MiB device array.  This
file checks, through the C ABI, that two calls in a row give what
pdlp_solve_device gives on the same inputs (to the 1e-9 parity tolerance of
the other GPU tests), including an LP whose long columns take the device-built
transpose path and the persistent step kernel; that a call leaves the device's
allocated and free memory unchanged; that a request for the autotuner (which
needs its own stream, events and graphs) and a problem too large for the array
are refused.  It is named so pytest collects it last.
"""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

PARITY = 1e-9


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as G
    G.build()
    import paper_2503_10344_gb300 as P
    return P


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(1.0, np.linalg.norm(b)))


def long_column_lp(m=6000, n=3000, seed=5):
    """Feasible covering-type LP with one column in every row (two sort tiles) and
    one in two thirds of the rows, so the transpose sorts long column segments."""
    rng = np.random.default_rng(seed)
    rows = [np.arange(m), np.arange(m)[rng.random(m) < 0.66]]
    cols = [np.zeros(m, dtype=np.int64), np.ones(rows[1].size, dtype=np.int64)]
    mask = rng.random((m, n)) < 0.002
    mask[:, :2] = False
    rr, cc = np.nonzero(mask)
    rows.append(rr)
    cols.append(cc)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.uniform(0.5, 2.0, size=rows.size)
    vals[:m] = rng.uniform(1.0, 2.0, size=m)  # column 0 alone covers every row: feasible
    return lpgen._lp(m, n, rows, cols, vals, np.ones(m),
                     np.full(m, lpgen.SENSE_GE, dtype=np.uint8), rng.uniform(1, 10, size=n),
                     np.zeros(n), np.ones(n), np.zeros(n, np.uint8), "long_columns")


CASES = [(lambda: lpgen.mip_relaxation(1), "fp64", 0, {}),
         (lambda: lpgen.set_cover(7, m=2000, n=8000), "bf16", 0, {}),
         (lambda: long_column_lp(), "fp32", 0, {}),
         (lambda: lpgen.mip_relaxation(2), "fp64", 1, {}),
         (lambda: lpgen.set_cover(8, m=2000, n=8000), "fp32", 1, {}),
         # one block with the LP in shared memory; the algorithmic variants
         (lambda: lpgen.mip_relaxation(3), "fp64", 2, {}),
         (lambda: lpgen.mip_relaxation(4), "fp64", 0, {"bound_objective_rescaling": 1}),
         (lambda: lpgen.set_cover(9, m=2000, n=8000), "bf16", 0, {"bound_objective_rescaling": 1}),
         (lambda: lpgen.mip_relaxation(5), "fp64", 0, {"halpern": 1}),
         (lambda: lpgen.set_cover(10, m=2000, n=8000), "fp32", 0, {"halpern": 1}),
         (lambda: lpgen.mip_relaxation(6), "fp64", 0, {"restart_metric": 1}),
         (lambda: lpgen.set_cover(11, m=2000, n=8000), "bf16", 1, {"restart_metric": 1})]


@pytest.mark.parametrize("maker,prec,persistent,variant", CASES)
def test_noalloc_matches_solve_device_on_two_calls_in_a_row(P, maker, prec, persistent, variant):
    import torch
    lp = maker()
    d = P.DeviceLP(lp)
    prm = P.default_params(tol=1e-6, precision=prec, persistent=persistent, **variant)
    assert P.workspace_size(lp.m, lp.n, lp.nnz, prm) <= P.binding.NOALLOC_BYTES
    xr, yr, rr = P.pdlp_solve_device(d, prm)
    xr, yr = xr.cpu().numpy(), yr.cpu().numpy()
    xo = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    yo = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    for _ in range(2):
        x, y, r = P.pdlp_solve_device_noalloc(d, prm, x_out=xo, y_out=yo)
        torch.cuda.synchronize()
        assert r["status"] == rr["status"] == P.PDLP_OPTIMAL
        assert r["iters"] == rr["iters"] and r["restarts"] == rr["restarts"]
        assert rel(x.cpu().numpy(), xr) <= PARITY
        assert rel(y.cpu().numpy(), yr) <= PARITY
        assert r["rel_kkt"] == pytest.approx(rr["rel_kkt"], rel=PARITY)


@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_noalloc_call_leaves_device_memory_unchanged(P, persistent):
    """The property the entry point exists for: after a first call (which may load
    the library's module, and with it the static array), a call changes neither the
    memory PyTorch has allocated nor the device's free memory."""
    import torch
    # persistent = 2 on an LP that fits in shared memory (the kernel's dynamic shared
    # memory is no device allocation)
    lp = lpgen.mip_relaxation(1) if persistent == 2 else lpgen.set_cover(9, m=2000, n=8000)
    d = P.DeviceLP(lp)
    prm = P.default_params(tol=1e-4, precision="fp32", persistent=persistent)
    xo = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    yo = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    P.pdlp_solve_device_noalloc(d, prm, x_out=xo, y_out=yo)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    _, _, r = P.pdlp_solve_device_noalloc(d, prm, x_out=xo, y_out=yo)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert r["status"] == P.PDLP_OPTIMAL
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0


def test_noalloc_refuses_the_autotuner(P):
    lp = lpgen.set_cover(7, m=2000, n=8000)
    d = P.DeviceLP(lp)
    prm = P.default_params(tol=1e-4, precision="fp32", autotune=1)
    with pytest.raises(P.PdlpError, match="INVALID_INPUT.*autotune"):
        P.pdlp_solve_device_noalloc(d, prm)


def test_noalloc_refuses_a_problem_larger_than_its_array(P):
    lp = lpgen.set_cover(2025)  # needs well over 64 MiB in float64
    d = P.DeviceLP(lp)
    prm = P.default_params(precision="fp64")
    assert P.workspace_size(lp.m, lp.n, lp.nnz, prm) > P.binding.NOALLOC_BYTES
    with pytest.raises(P.PdlpError, match="OOM"):
        P.pdlp_solve_device_noalloc(d, prm)
