"""ctypes binding of the C ABI in ``include/pdlp.h`` (argument marshalling only).

Every step of the solve runs in the CUDA library ``libpdlp.so``; this module
only builds the C structs, passes pointers and converts results.  There is no
fallback: if the library is missing, :func:`lib` raises.

Host entry point :func:`pdlp_solve` takes numpy arrays; device entry point
:func:`pdlp_solve_device` takes CUDA torch tensors (PyTorch provides device
memory and the stream, nothing else).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdlp.so")

PDLP_OK = 0
ERRORS = {-1: "PDLP_ERR_INVALID_INPUT", -2: "PDLP_ERR_CUDA", -3: "PDLP_ERR_OOM",
          -4: "PDLP_ERR_TIMEOUT", -5: "PDLP_ERR_UNSUPPORTED"}
PDLP_OPTIMAL, PDLP_ITER_LIMIT, PDLP_TIME_LIMIT, PDLP_NUMERICAL = 1, 2, 3, 4
PDLP_PRIMAL_INFEASIBLE, PDLP_DUAL_INFEASIBLE = 5, 6
PDLP_FP64, PDLP_FP32, PDLP_FP32_BF16A = 0, 1, 2
PDLP_USED_BF16, PDLP_USED_PATTERN = 2, 3
PRECISION = {"fp64": PDLP_FP64, "fp32": PDLP_FP32, "bf16": PDLP_FP32_BF16A}


class PdlpCsr(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class PdlpParams(C.Structure):
    _fields_ = [("struct_size", C.c_size_t), ("tol", C.c_double), ("iter_limit", C.c_int64),
                ("time_limit_s", C.c_double), ("precision", C.c_int), ("check_period", C.c_int),
                ("ruiz_iters", C.c_int), ("pc_alpha", C.c_double), ("adaptive_step", C.c_int),
                ("restarts", C.c_int), ("fixed_eta", C.c_double), ("fixed_omega", C.c_double),
                ("terminate", C.c_int), ("lanes_A", C.c_int), ("lanes_AT", C.c_int),
                ("lanes_kkt_A", C.c_int), ("lanes_kkt_AT", C.c_int), ("verbose", C.c_int),
                ("persistent", C.c_int), ("autotune", C.c_int),
                ("detect_infeasibility", C.c_int), ("debug_skip_barrier", C.c_int),
                ("tiles", C.c_int), ("bound_objective_rescaling", C.c_int),
                ("halpern", C.c_int), ("halpern_reflection", C.c_double),
                ("restart_metric", C.c_int)]


class PdlpResult(C.Structure):
    _fields_ = [("status", C.c_int), ("precision_used", C.c_int), ("iters", C.c_int64),
                ("attempts", C.c_int64), ("restarts", C.c_int64), ("kkt_checks", C.c_int64),
                ("kernel_launches", C.c_int64), ("primal_obj", C.c_double),
                ("dual_obj", C.c_double), ("rel_primal_res", C.c_double),
                ("rel_dual_res", C.c_double), ("rel_gap", C.c_double), ("rel_kkt", C.c_double),
                ("eta", C.c_double), ("omega", C.c_double), ("used_average", C.c_int),
                ("setup_s", C.c_double), ("solve_s", C.c_double), ("lanes_A", C.c_int),
                ("lanes_AT", C.c_int), ("ray_obj", C.c_double), ("ray_res", C.c_double),
                ("tiles", C.c_int), ("upload_s", C.c_double), ("persistent_form", C.c_int),
                ("spectral_norm", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PdlpDiagnostics(C.Structure):
    _fields_ = [("x_cur", C.c_void_p), ("y_cur", C.c_void_p), ("x_avg", C.c_void_p),
                ("y_avg", C.c_void_p), ("attempt_capacity", C.c_int64), ("eta", C.c_void_p),
                ("eta_bar", C.c_void_p), ("accepted", C.c_void_p), ("check_capacity", C.c_int64),
                ("restart", C.c_void_p), ("omega", C.c_void_p), ("point_capacity", C.c_int64),
                ("check_points", C.c_void_p)]


_LIB = None


class PdlpError(RuntimeError):
    pass


def lib():
    """Load libpdlp.so (build it first with ``paper_2503_10344_gb300.build.build()``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise PdlpError(f"{LIB_PATH} is missing: run paper_2503_10344_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.pdlp_default_params.argtypes = [C.POINTER(PdlpParams)]
        L.pdlp_workspace_size.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.POINTER(PdlpParams)]
        L.pdlp_workspace_size.restype = C.c_size_t
        common = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 5 + [C.POINTER(PdlpParams)] + \
            [C.c_void_p] * 4 + [C.POINTER(PdlpResult), C.POINTER(PdlpDiagnostics)]
        L.pdlp_solve.argtypes = common
        L.pdlp_solve_hinted.argtypes = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 5 + \
            [C.POINTER(PdlpParams)] + [C.c_void_p] * 6 + [C.POINTER(PdlpResult),
                                                         C.POINTER(PdlpDiagnostics)]
        L.pdlp_solve_device.argtypes = common + [C.c_void_p, C.c_size_t, C.c_void_p]
        L.pdlp_solve_device_noalloc.argtypes = common + [C.c_void_p]
        L.pdlp_time_kernels.argtypes = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 5 + \
            [C.POINTER(PdlpParams), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
             C.c_void_p]
        L.pdlp_polish_primal.argtypes = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 4 + \
            [C.POINTER(PdlpParams)] + [C.c_void_p] * 3 + [C.POINTER(PdlpResult)]
        L.pdlp_polish_dual.argtypes = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 4 + \
            [C.POINTER(PdlpParams)] + [C.c_void_p] * 3 + [C.POINTER(PdlpResult)]
        L.pdlp_error_string.argtypes = [C.c_int]
        L.pdlp_error_string.restype = C.c_char_p
        L.pdlp_last_error.restype = C.c_char_p
        _LIB = L
    return _LIB


def default_params(**kw) -> PdlpParams:
    p = PdlpParams()
    lib().pdlp_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _check(rc: int):
    if rc != PDLP_OK:
        msg = lib().pdlp_last_error().decode()
        raise PdlpError(f"{ERRORS.get(rc, rc)}: {msg}")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


DIAG_ITERATES = ("x_cur", "y_cur", "x_avg", "y_avg")


def pdlp_solve(lp, params: PdlpParams | None = None, x0=None, y0=None, iterates: bool = False,
               trace: int = 0, omega_hint=None, check_points: int = 0):
    """Solve ``lp`` (an :class:`lpgen.LP`-like object) from host memory.

    Returns (x, y, result dict) or, with ``iterates`` or ``trace`` > 0,
    (x, y, result dict, diagnostics dict); ``trace`` is the capacity of the
    per-attempt decision trace (the per-check trace gets trace // 16 + 16).
    ``omega_hint`` = (x_h, y_h) calls pdlp_solve_hinted: the initial primal weight
    is the ratio of the hint's scaled norms.  ``check_points`` = R keeps the current
    point of the last R KKT checks: diagnostics["check_points"], oldest first.
    """
    p = params or default_params()
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val = f64(lp.val)
    b, c, l, u = f64(lp.b), f64(lp.c), f64(lp.l), f64(lp.u)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    csr = PdlpCsr(lp.m, lp.n, int(row_ptr[-1]), _ptr(row_ptr), _ptr(col), _ptr(val))
    x = np.empty(lp.n)
    y = np.empty(lp.m)
    x0a = None if x0 is None else f64(x0)
    y0a = None if y0 is None else f64(y0)
    res = PdlpResult()
    diag = None
    dgp = None
    if iterates or trace > 0 or check_points > 0:
        diag = {k: np.empty(lp.n if k[0] == "x" else lp.m) for k in DIAG_ITERATES}
        diag["check_points"] = np.zeros((check_points, lp.n))
        tc = trace // 16 + 16 if trace > 0 else 0
        diag.update(eta=np.full(trace, np.nan), eta_bar=np.full(trace, np.nan),
                    accepted=np.full(trace, -1, dtype=np.int8), restart=np.full(tc, -1, dtype=np.int8),
                    omega=np.full(tc, np.nan))
        dgp = PdlpDiagnostics(*[_ptr(diag[k]) for k in DIAG_ITERATES], trace, _ptr(diag["eta"]),
                              _ptr(diag["eta_bar"]), _ptr(diag["accepted"]), tc,
                              _ptr(diag["restart"]), _ptr(diag["omega"]), check_points,
                              _ptr(diag["check_points"]) if check_points > 0 else None)
    if omega_hint is None:
        rc = lib().pdlp_solve(C.byref(csr), _ptr(b), _ptr(sense), _ptr(c), _ptr(l), _ptr(u),
                              C.byref(p), _ptr(x0a), _ptr(y0a), _ptr(x), _ptr(y), C.byref(res),
                              C.byref(dgp) if dgp is not None else None)
    else:
        xh, yh = f64(omega_hint[0]), f64(omega_hint[1])
        rc = lib().pdlp_solve_hinted(C.byref(csr), _ptr(b), _ptr(sense), _ptr(c), _ptr(l), _ptr(u),
                                     C.byref(p), _ptr(x0a), _ptr(y0a), _ptr(xh), _ptr(yh), _ptr(x),
                                     _ptr(y), C.byref(res), C.byref(dgp) if dgp is not None else None)
    _check(rc)
    out = res.as_dict()
    if diag is None:
        return x, y, out
    if check_points > 0:  # ring buffer -> the last checks, oldest first
        kc = out["kkt_checks"]
        rows = [(k % check_points) for k in range(max(0, kc - check_points), kc)]
        diag["check_points"] = diag["check_points"][rows]
    if trace > 0:
        na = min(trace, out["attempts"])
        nc = min(tc, out["kkt_checks"])
        for k in ("eta", "eta_bar", "accepted"):
            diag[k] = diag[k][:na]
        for k in ("restart", "omega"):
            diag[k] = diag[k][:nc]
    return x, y, out, diag


def pdlp_polish_primal(lp, x, params: PdlpParams | None = None):
    """Primal feasibility polishing of ``x`` (host buffers): the PDHG on the
    objective-free problem from (x, 0).  Returns (x_polished, y, result dict)."""
    L = lib()
    p = params or default_params()
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val = f64(lp.val)
    b, l, u, xi = f64(lp.b), f64(lp.l), f64(lp.u), f64(x)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    csr = PdlpCsr(lp.m, lp.n, int(row_ptr[-1]), _ptr(row_ptr), _ptr(col), _ptr(val))
    xo = np.empty(lp.n)
    yo = np.empty(lp.m)
    res = PdlpResult()
    _check(L.pdlp_polish_primal(C.byref(csr), _ptr(b), _ptr(sense), _ptr(l), _ptr(u), C.byref(p),
                                _ptr(xi), _ptr(xo), _ptr(yo) if lp.m else None, C.byref(res)))
    return xo, yo, res.as_dict()


def pdlp_polish_dual(lp, y, params: PdlpParams | None = None):
    """Dual feasibility polishing of ``y`` (host buffers): the PDHG on the LP with
    b = 0 and finite bounds at 0, from (0, y).  Returns (x, y_polished, result
    dict); x is the multiplier of the violated reduced costs, or the ray of descent
    when the status is PDLP_DUAL_INFEASIBLE."""
    L = lib()
    p = params or default_params()
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val = f64(lp.val)
    c, l, u, yi = f64(lp.c), f64(lp.l), f64(lp.u), f64(y)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    csr = PdlpCsr(lp.m, lp.n, int(row_ptr[-1]), _ptr(row_ptr), _ptr(col), _ptr(val))
    xo = np.empty(lp.n)
    yo = np.empty(lp.m)
    res = PdlpResult()
    _check(L.pdlp_polish_dual(C.byref(csr), _ptr(sense), _ptr(c), _ptr(l), _ptr(u), C.byref(p),
                              _ptr(yi) if lp.m else None, _ptr(xo), _ptr(yo) if lp.m else None,
                              C.byref(res)))
    return xo, yo, res.as_dict()


def workspace_size(m: int, n: int, nnz: int, params: PdlpParams | None = None) -> int:
    p = params or default_params()
    return int(lib().pdlp_workspace_size(m, n, nnz, C.byref(p)))


class DeviceLP:
    """The arrays of an LP as CUDA torch tensors (inputs of pdlp_solve_device)."""

    def __init__(self, lp, device="cuda"):
        import torch
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        self.m, self.n, self.nnz = lp.m, lp.n, int(lp.row_ptr[-1])
        self.row_ptr = t(lp.row_ptr, torch.int64)
        self.col = t(lp.col, torch.int32)
        self.val = t(lp.val, torch.float64)
        self.b = t(lp.b, torch.float64)
        self.sense = t(lp.sense, torch.uint8)
        self.c = t(lp.c, torch.float64)
        self.l = t(lp.l, torch.float64)
        self.u = t(lp.u, torch.float64)


def pdlp_solve_device(dlp: DeviceLP, params: PdlpParams | None = None, x0=None, y0=None,
                      x_out=None, y_out=None, workspace=None, stream=None, iterates=None):
    # iterates: optional dict of float64 CUDA tensors named x_cur, y_cur, x_avg, y_avg
    """Solve from device tensors on ``stream`` (default: torch's current stream).

    ``x_out``/``y_out``/``iterates`` are float64 CUDA tensors (allocated if None);
    ``workspace`` is a uint8 CUDA tensor of at least :func:`workspace_size` bytes
    (allocated from torch's caching allocator if None).  Returns (x, y, result).
    """
    import torch
    p = params or default_params()
    dev = dlp.c.device
    if x_out is None:
        x_out = torch.empty(dlp.n, dtype=torch.float64, device=dev)
    if y_out is None:
        y_out = torch.empty(max(dlp.m, 1), dtype=torch.float64, device=dev)
    nbytes = workspace_size(dlp.m, dlp.n, dlp.nnz, p)
    if workspace is None:
        workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    avail = workspace.numel() - (aligned - base)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    dp = lambda t_: None if t_ is None else C.c_void_p(t_.data_ptr())
    csr = PdlpCsr(dlp.m, dlp.n, dlp.nnz, dlp.row_ptr.data_ptr(), dlp.col.data_ptr(),
                  dlp.val.data_ptr())
    res = PdlpResult()
    itp = None
    if iterates is not None:
        itp = PdlpDiagnostics(*[dp(iterates.get(k)) for k in DIAG_ITERATES], 0, None, None, None,
                              0, None, None)
    rc = lib().pdlp_solve_device(C.byref(csr), dp(dlp.b), dp(dlp.sense), dp(dlp.c), dp(dlp.l),
                                 dp(dlp.u), C.byref(p), dp(x0), dp(y0), dp(x_out), dp(y_out),
                                 C.byref(res), C.byref(itp) if itp is not None else None,
                                 C.c_void_p(aligned), avail, C.c_void_p(stream.cuda_stream))
    _check(rc)
    return x_out, y_out[: dlp.m], res.as_dict()


KERNELS = ("primal_step", "dual_step", "attempt", "kkt_rows", "kkt_cols", "persistent_attempt",
           "kkt_block")


def time_kernels(dlp: DeviceLP, params: PdlpParams | None = None, reps: int = 200,
                 workspace=None, stream=None) -> dict:
    """Average device ms and algorithmic bytes per launch of each fused kernel."""
    import torch
    p = params or default_params()
    dev = dlp.c.device
    nbytes = workspace_size(dlp.m, dlp.n, dlp.nnz, p)
    if workspace is None:
        workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    ms = np.zeros(len(KERNELS))
    by = np.zeros(len(KERNELS))
    csr = PdlpCsr(dlp.m, dlp.n, dlp.nnz, dlp.row_ptr.data_ptr(), dlp.col.data_ptr(),
                  dlp.val.data_ptr())
    dp = lambda t_: C.c_void_p(t_.data_ptr())
    rc = lib().pdlp_time_kernels(C.byref(csr), dp(dlp.b), dp(dlp.sense), dp(dlp.c), dp(dlp.l),
                                 dp(dlp.u), C.byref(p), reps, _ptr(ms), _ptr(by), C.c_void_p(aligned),
                                 workspace.numel() - (aligned - base), C.c_void_p(stream.cuda_stream))
    _check(rc)
    return {k: {"ms": float(ms[i]), "bytes": float(by[i])} for i, k in enumerate(KERNELS)}


NOALLOC_BYTES = 64 << 20


def pdlp_solve_device_noalloc(dlp: DeviceLP, params: PdlpParams | None = None, x0=None, y0=None,
                              x_out=None, y_out=None, stream=None):
    """pdlp_solve_device for callers that cannot allocate device memory: the library
    solves in its own static 64 MiB device array instead of a workspace.  Outputs
    must be passed in (float64 CUDA tensors) when the caller cannot allocate them
    either; they are allocated here only as a convenience when left as None."""
    import torch
    p = params or default_params()
    dev = dlp.c.device
    if x_out is None:
        x_out = torch.empty(dlp.n, dtype=torch.float64, device=dev)
    if y_out is None:
        y_out = torch.empty(max(dlp.m, 1), dtype=torch.float64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    dp = lambda t_: None if t_ is None else C.c_void_p(t_.data_ptr())
    csr = PdlpCsr(dlp.m, dlp.n, dlp.nnz, dlp.row_ptr.data_ptr(), dlp.col.data_ptr(),
                  dlp.val.data_ptr())
    res = PdlpResult()
    rc = lib().pdlp_solve_device_noalloc(C.byref(csr), dp(dlp.b), dp(dlp.sense), dp(dlp.c),
                                         dp(dlp.l), dp(dlp.u), C.byref(p), dp(x0), dp(y0),
                                         dp(x_out), dp(y_out), C.byref(res), None,
                                         C.c_void_p(stream.cuda_stream))
    _check(rc)
    return x_out, y_out[: dlp.m], res.as_dict()


# ------------------------------------------------------------------ fix-and-propagate
FP_FRAC, FP_REDCOST, FP_DUAL, FP_TYPE = 0, 1, 2, 3
FP_FEASIBLE, FP_INFEASIBLE, FP_NODE_LIMIT, FP_NO_FINAL_LP = 1, 2, 3, 4
FP_FRAC_DUAL, FP_FRAC_REDCOST, FP_DUAL_FRAC, FP_REDCOST_FRAC = 4, 5, 6, 7
FP_STRATEGY = {"frac": FP_FRAC, "redcost": FP_REDCOST, "dual": FP_DUAL, "type": FP_TYPE,
               "frac_dual": FP_FRAC_DUAL, "frac_redcost": FP_FRAC_REDCOST,
               "dual_frac": FP_DUAL_FRAC, "redcost_frac": FP_REDCOST_FRAC}


class FpParams(C.Structure):
    _fields_ = [("struct_size", C.c_size_t), ("var_strategy", C.c_int), ("seed", C.c_uint64),
                ("node_limit", C.c_int64), ("final_lp", C.c_int), ("final_lp_tol", C.c_double)]


class FpResult(C.Structure):
    _fields_ = [("status", C.c_int), ("obj", C.c_double), ("nodes", C.c_int64),
                ("backtracks", C.c_int64), ("final_lp_iters", C.c_int64),
                ("final_rel_primal", C.c_double), ("search_s", C.c_double), ("lp_s", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def fp_run(lp, x_lp, y_lp=None, is_int=None, strategy="type", seed: int = 1, node_limit: int = 0,
           final_lp: bool = True, final_lp_tol: float = 1e-8):
    """Fix-and-propagate on host buffers; returns (x, result dict)."""
    L = lib()
    if not getattr(L, "_fp_ready", False):
        L.fp_default_params.argtypes = [C.POINTER(FpParams)]
        L.fp_run.argtypes = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 8 + [C.POINTER(FpParams),
                                                                      C.c_void_p, C.POINTER(FpResult)]
        L._fp_ready = True
    p = FpParams()
    L.fp_default_params(C.byref(p))
    p.var_strategy = FP_STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    p.seed = seed
    p.node_limit = node_limit
    p.final_lp = 1 if final_lp else 0
    p.final_lp_tol = final_lp_tol
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val, b, c, l, u = f64(lp.val), f64(lp.b), f64(lp.c), f64(lp.l), f64(lp.u)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    ii = np.ascontiguousarray(lp.is_int if is_int is None else is_int, dtype=np.uint8)
    xl = f64(x_lp)
    yl = None if y_lp is None else f64(y_lp)
    csr = PdlpCsr(lp.m, lp.n, int(row_ptr[-1]), _ptr(row_ptr), _ptr(col), _ptr(val))
    x = np.empty(lp.n)
    r = FpResult()
    rc = L.fp_run(C.byref(csr), _ptr(b), _ptr(sense), _ptr(c), _ptr(l), _ptr(u), _ptr(xl), _ptr(yl),
                  _ptr(ii), C.byref(p), _ptr(x), C.byref(r))
    _check(rc)
    return x, r.as_dict()


def fp_run_refs(lp, x_refs, y_lp=None, is_int=None, strategy="type", seed: int = 1,
                node_limit: int = 0, final_lp: bool = True, final_lp_tol: float = 1e-8):
    """fp_run from each of several LP points (host buffers); returns (x, result dict, chosen
    index, -1 when no run is feasible)."""
    L = lib()
    if not getattr(L, "_fp_refs_ready", False):
        L.fp_run_refs.argtypes = [C.POINTER(PdlpCsr)] + [C.c_void_p] * 6 + [C.c_int] + \
            [C.c_void_p] * 2 + [C.POINTER(FpParams), C.c_void_p, C.POINTER(FpResult),
                                C.POINTER(C.c_int)]
        L.fp_default_params.argtypes = [C.POINTER(FpParams)]
        L._fp_refs_ready = True
    p = FpParams()
    L.fp_default_params(C.byref(p))
    p.var_strategy = FP_STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    p.seed = seed
    p.node_limit = node_limit
    p.final_lp = 1 if final_lp else 0
    p.final_lp_tol = final_lp_tol
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(lp.col, dtype=np.int32)
    val, b, c, l, u = f64(lp.val), f64(lp.b), f64(lp.c), f64(lp.l), f64(lp.u)
    sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
    ii = np.ascontiguousarray(lp.is_int if is_int is None else is_int, dtype=np.uint8)
    refs = [f64(x) for x in x_refs]
    rp = (C.c_void_p * len(refs))(*[_ptr(x) for x in refs])
    yl = None if y_lp is None else f64(y_lp)
    csr = PdlpCsr(lp.m, lp.n, int(row_ptr[-1]), _ptr(row_ptr), _ptr(col), _ptr(val))
    x = np.empty(lp.n)
    r = FpResult()
    chosen = C.c_int(-1)
    _check(L.fp_run_refs(C.byref(csr), _ptr(b), _ptr(sense), _ptr(c), _ptr(l), _ptr(u), rp,
                         len(refs), _ptr(yl), _ptr(ii), C.byref(p), _ptr(x), C.byref(r),
                         C.byref(chosen)))
    return x, r.as_dict(), chosen.value


def _batch_arrays(lps, xs=None, ys=None):
    """The pointer arrays of a batch call; `keep` holds the numpy arrays alive."""
    k = len(lps)
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    csrs = (PdlpCsr * k)()
    ptrs = {name: (C.c_void_p * k)() for name in ("b", "sense", "c", "l", "u", "x", "y")}
    for i, lp in enumerate(lps):
        rp = arr(lp.row_ptr, np.int64)
        csrs[i] = PdlpCsr(lp.m, lp.n, int(rp[-1]), _ptr(rp), _ptr(arr(lp.col, np.int32)),
                          _ptr(arr(lp.val, np.float64)))
        ptrs["b"][i] = _ptr(arr(lp.b, np.float64))
        ptrs["sense"][i] = _ptr(arr(lp.sense, np.uint8))
        ptrs["c"][i] = _ptr(arr(lp.c, np.float64))
        ptrs["l"][i] = _ptr(arr(lp.l, np.float64))
        ptrs["u"][i] = _ptr(arr(lp.u, np.float64))
        ptrs["x"][i] = _ptr(xs[i]) if xs is not None else None
        ptrs["y"][i] = _ptr(ys[i]) if ys is not None else None
    keep.append(csrs)
    csr_ptrs = (C.c_void_p * k)(*[C.cast(C.pointer(csrs[i]), C.c_void_p) for i in range(k)])
    return csr_ptrs, ptrs, keep


def pdlp_solve_batch(lps, params: PdlpParams | None = None, want_y: bool = True):
    """Solve a list of LPs together (host buffers); returns (xs, ys, results)."""
    L = lib()
    if not getattr(L, "_batch_ready", False):
        L.pdlp_solve_batch.argtypes = [C.c_int, C.c_void_p] + [C.c_void_p] * 5 + \
            [C.POINTER(PdlpParams), C.c_void_p, C.c_void_p, C.c_void_p]
        L._batch_ready = True
    p = params or default_params()
    k = len(lps)
    xs = [np.empty(lp.n) for lp in lps]
    ys = [np.empty(lp.m) for lp in lps]
    csr_ptrs, ptrs, keep = _batch_arrays(lps, xs, ys if want_y else None)
    res = (PdlpResult * k)()
    rc = L.pdlp_solve_batch(k, csr_ptrs, ptrs["b"], ptrs["sense"], ptrs["c"], ptrs["l"], ptrs["u"],
                            C.byref(p), ptrs["x"], ptrs["y"], res)
    _check(rc)
    del keep
    return xs, ys, [res[i].as_dict() for i in range(k)]


def pdlp_solve_batch_device(dlps, params: PdlpParams | None = None, stream=None):
    """Solve a list of DeviceLP together from device buffers (pdlp_solve_batch_device);
    returns (xs, ys, results) with xs / ys float64 CUDA tensors."""
    import torch
    L = lib()
    if not getattr(L, "_batch_dev_ready", False):
        L.pdlp_solve_batch_device.argtypes = [C.c_int, C.c_void_p] + [C.c_void_p] * 5 + \
            [C.POINTER(PdlpParams), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L._batch_dev_ready = True
    p = params or default_params()
    k = len(dlps)
    dev = dlps[0].c.device
    xs = [torch.empty(d.n, dtype=torch.float64, device=dev) for d in dlps]
    ys = [torch.empty(max(d.m, 1), dtype=torch.float64, device=dev) for d in dlps]
    csrs = (PdlpCsr * k)()
    ptrs = {name: (C.c_void_p * k)() for name in ("b", "sense", "c", "l", "u", "x", "y")}
    for i, d in enumerate(dlps):
        csrs[i] = PdlpCsr(d.m, d.n, d.nnz, d.row_ptr.data_ptr(), d.col.data_ptr(), d.val.data_ptr())
        for name, t in (("b", d.b), ("sense", d.sense), ("c", d.c), ("l", d.l), ("u", d.u),
                        ("x", xs[i]), ("y", ys[i])):
            ptrs[name][i] = t.data_ptr()
    csr_ptrs = (C.c_void_p * k)(*[C.cast(C.pointer(csrs[i]), C.c_void_p) for i in range(k)])
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    res = (PdlpResult * k)()
    rc = L.pdlp_solve_batch_device(k, csr_ptrs, ptrs["b"], ptrs["sense"], ptrs["c"], ptrs["l"],
                                   ptrs["u"], C.byref(p), ptrs["x"], ptrs["y"], res,
                                   C.c_void_p(stream.cuda_stream))
    _check(rc)
    return xs, [y[: d.m] for y, d in zip(ys, dlps)], [res[i].as_dict() for i in range(k)]


def time_kernels_batch(lps, params: PdlpParams | None = None, reps: int = 20) -> dict:
    """Average device ms and algorithmic bytes per launch of each fused kernel over a
    whole batch (every LP live), as :func:`time_kernels` for one LP."""
    L = lib()
    if not getattr(L, "_batch_timing_ready", False):
        L.pdlp_time_kernels_batch.argtypes = [C.c_int, C.c_void_p] + [C.c_void_p] * 5 + \
            [C.POINTER(PdlpParams), C.c_int, C.c_void_p, C.c_void_p]
        L._batch_timing_ready = True
    p = params or default_params()
    csr_ptrs, ptrs, keep = _batch_arrays(lps)
    ms = np.zeros(len(KERNELS))
    by = np.zeros(len(KERNELS))
    rc = L.pdlp_time_kernels_batch(len(lps), csr_ptrs, ptrs["b"], ptrs["sense"], ptrs["c"],
                                   ptrs["l"], ptrs["u"], C.byref(p), reps, _ptr(ms), _ptr(by))
    _check(rc)
    del keep
    return {k: {"ms": float(ms[i]), "bytes": float(by[i])} for i, k in enumerate(KERNELS)}
