"""Host-side argument checks of the C ABI (no GPU needed: every call here is
rejected before the library touches CUDA).

Each entry point returns PDLP_ERR_INVALID_INPUT, with a message in
pdlp_last_error, for the malformed inputs its header comment names: invalid
parameter values, a params struct of another size, NULL result or vector
arguments, empty problems, l > u for dual polishing, an empty batch.
"""
import ctypes as C

import numpy as np
import pytest

import lpgen
import __graft_entry__ as G


@pytest.fixture(scope="module")
def P():
    G.build()
    import paper_2503_10344_gb300 as P
    return P


@pytest.fixture(scope="module")
def lp():
    return lpgen.mip_relaxation(1, m=20, n=40, density=0.2)


def _rejected(P, call, needle):
    with pytest.raises(P.PdlpError) as e:
        call()
    assert "PDLP_ERR_INVALID_INPUT" in str(e.value)
    assert needle in str(e.value)


@pytest.mark.parametrize("field,value,needle", [
    ("tol", 0.0, "invalid parameter value"),
    ("tol", float("nan"), "invalid parameter value"),
    ("iter_limit", -1, "invalid parameter value"),
    ("check_period", 0, "invalid parameter value"),
    ("ruiz_iters", -2, "invalid parameter value"),
    ("time_limit_s", 0.0, "invalid parameter value"),
    ("precision", 7, "unknown precision mode"),
    ("persistent", 3, "persistent must be 0, 1 or 2"),
    ("autotune", -1, "autotune must be 0 or 1"),
    ("tiles", 3, "tiles must be 0, 1 or 2"),
    ("lanes_A", 3, "step lanes must be"),
    ("lanes_AT", 64, "step lanes must be"),
    ("lanes_kkt_AT", 64, "KKT lanes must be"),
    ("lanes_kkt_A", 1, "KKT lanes must be"),  # one lane per row: step kernels only
])
def test_solve_rejects_invalid_parameters(P, lp, field, value, needle):
    _rejected(P, lambda: P.pdlp_solve(lp, P.default_params(**{field: value})), needle)


@pytest.mark.parametrize("persistent", [1, 2])
@pytest.mark.parametrize("field", ["lanes_A", "lanes_AT"])
def test_one_lane_per_row_needs_the_two_launch_form(P, lp, persistent, field):
    _rejected(P, lambda: P.pdlp_solve(lp, P.default_params(persistent=persistent, **{field: 1})),
              "one lane per row needs persistent = 0")


def test_solve_rejects_a_params_struct_of_another_size(P, lp):
    p = P.default_params()
    p.struct_size = C.sizeof(p) - 8
    _rejected(P, lambda: P.pdlp_solve(lp, p), "struct_size mismatch")


def test_solve_rejects_null_and_empty_arguments(P, lp):
    L = P.lib()
    p = P.default_params()
    res = P.binding.PdlpResult()
    x = np.empty(lp.n)
    y = np.empty(lp.m)
    f = np.zeros(lp.n)
    rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val = np.ascontiguousarray(lp.val, dtype=np.float64)
    b = np.ascontiguousarray(lp.b)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    ptr = P.binding._ptr
    csr = P.binding.PdlpCsr(lp.m, lp.n, int(rp[-1]), ptr(rp), ptr(col), ptr(val))
    args = [C.byref(csr), ptr(b), ptr(sense), ptr(f), ptr(f), ptr(f), C.byref(p), None, None,
            ptr(x), ptr(y)]
    INVALID = -1
    assert L.pdlp_solve(*args, None, None) == INVALID                       # no result
    assert b"NULL problem" in L.pdlp_last_error()
    for k in (1, 3, 9):                                                     # b, c, x_out
        bad = list(args)
        bad[k] = None
        assert L.pdlp_solve(*bad, C.byref(res), None) == INVALID
        assert b"NULL vector argument" in L.pdlp_last_error()
    empty = P.binding.PdlpCsr(lp.m, 0, 0, ptr(rp), ptr(col), ptr(val))
    assert L.pdlp_solve(C.byref(empty), *args[1:], C.byref(res), None) == INVALID
    assert b"n >= 1" in L.pdlp_last_error()
    nullcsr = P.binding.PdlpCsr(lp.m, lp.n, int(rp[-1]), None, ptr(col), ptr(val))
    assert L.pdlp_solve(C.byref(nullcsr), *args[1:], C.byref(res), None) == INVALID
    assert b"NULL CSR array" in L.pdlp_last_error()


def test_dual_polishing_rejects_l_above_u(P, lp):
    bad = lpgen.mip_relaxation(1, m=20, n=40, density=0.2)
    bad.l = bad.l.copy()
    bad.l[7] = bad.u[7] + 1.0
    _rejected(P, lambda: P.pdlp_polish_dual(bad, np.zeros(bad.m)), "l > u in column 7")


def test_polishing_needs_its_start_point(P, lp):
    L = P.lib()
    p = P.default_params()
    res = P.binding.PdlpResult()
    rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val = np.ascontiguousarray(lp.val, dtype=np.float64)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    f = np.zeros(max(lp.m, lp.n))
    ptr = P.binding._ptr
    csr = P.binding.PdlpCsr(lp.m, lp.n, int(rp[-1]), ptr(rp), ptr(col), ptr(val))
    assert L.pdlp_polish_primal(C.byref(csr), ptr(f), ptr(sense), ptr(f), ptr(f), C.byref(p),
                                None, ptr(f), ptr(f), C.byref(res)) == -1
    assert b"x_in" in L.pdlp_last_error()
    assert L.pdlp_polish_dual(C.byref(csr), ptr(sense), ptr(f), ptr(f), ptr(f), C.byref(p),
                              None, ptr(f), ptr(f), C.byref(res)) == -1
    assert b"y_in" in L.pdlp_last_error()


def test_batch_rejects_an_empty_batch_and_names_a_bad_lp(P, lp):
    _rejected(P, lambda: P.pdlp_solve_batch([]), "count >= 1")
    _rejected(P, lambda: P.pdlp_solve_batch([lp, lp], P.default_params(tol=-1.0)), "LP 0")


def test_bound_objective_rescaling_parameter_is_checked(P, lp):
    _rejected(P, lambda: P.pdlp_solve(lp, P.default_params(bound_objective_rescaling=2)),
              "bound_objective_rescaling must be 0 or 1")


@pytest.mark.parametrize("kw,needle", [
    (dict(halpern=2), "halpern must be 0 or 1"),
    (dict(halpern=1, halpern_reflection=1.5), "halpern_reflection must lie in [0, 1]"),
    (dict(halpern=1, halpern_reflection=-0.1), "halpern_reflection must lie in [0, 1]"),
    (dict(halpern=1, halpern_reflection=float("nan")), "halpern_reflection must lie in [0, 1]"),
    (dict(halpern=1, persistent=1), "halpern runs with persistent = 0 and tiles = 0 only"),
    (dict(halpern=1, persistent=2), "halpern runs with persistent = 0 and tiles = 0 only"),
    (dict(halpern=1, tiles=1, precision=1), "halpern runs with persistent = 0 and tiles = 0 only"),
])
def test_halpern_parameters_are_checked(P, lp, kw, needle):
    _rejected(P, lambda: P.pdlp_solve(lp, P.default_params(**kw)), needle)


@pytest.mark.parametrize("kw,needle", [
    (dict(restart_metric=2), "restart_metric must be 0 or 1"),
    (dict(restart_metric=1, halpern=1), "restart_metric = 1 runs without halpern"),
    (dict(restart_metric=1, bound_objective_rescaling=1), "restart_metric = 1 runs without halpern"),
])
def test_restart_metric_parameter_is_checked(P, lp, kw, needle):
    _rejected(P, lambda: P.pdlp_solve(lp, P.default_params(**kw)), needle)
