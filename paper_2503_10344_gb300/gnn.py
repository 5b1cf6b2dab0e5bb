"""ctypes binding of the learned warm start in ``include/gnn.h`` (argument marshalling only).

Every forward, backward, optimiser and KKT step runs in ``libpdlp.so``; this
module builds the C structs, passes host pointers and converts results.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .binding import PdlpCsr, PdlpParams, PdlpResult, _check, _ptr, default_params, lib

_READY = False


class GnnAdam(C.Structure):
    _fields_ = [("struct_size", C.c_size_t), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double)]


class GnnTrainParams(C.Structure):
    _fields_ = [("struct_size", C.c_size_t), ("epochs", C.c_int), ("batch", C.c_int),
                ("adam", GnnAdam), ("lr_decay", C.c_double), ("seed", C.c_uint64)]


class GnnWarmInfo(C.Structure):
    _fields_ = [("used_warm", C.c_int), ("warm_rel_kkt", C.c_double),
                ("cold_rel_kkt", C.c_double), ("predict_s", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def _lib():
    global _READY
    L = lib()
    if not _READY:
        vp, ip = C.c_void_p, C.c_int
        L.gnn_param_count.restype = C.c_int64
        L.gnn_param_count.argtypes = []
        L.gnn_create.argtypes = [C.c_uint64, C.POINTER(vp)]
        L.gnn_free.argtypes = [vp]
        for f in (L.gnn_get_params, L.gnn_set_params, L.gnn_get_grad, L.gnn_set_grad):
            f.argtypes = [vp, vp]
        L.gnn_zero_grad.argtypes = [vp]
        L.gnn_save.argtypes = [vp, C.c_char_p]
        L.gnn_load.argtypes = [C.c_char_p, C.POINTER(vp)]
        L.gnn_graph_create.argtypes = [vp, C.POINTER(PdlpCsr)] + [vp] * 5 + [C.POINTER(vp)]
        L.gnn_graph_set_labels.argtypes = [vp, vp, vp]
        L.gnn_graph_features.argtypes = [vp, vp, vp]
        L.gnn_graph_free.argtypes = [vp]
        L.gnn_forward.argtypes = [vp, vp, vp, vp, vp]
        L.gnn_backward.argtypes = [vp, vp, C.c_double, vp]
        L.gnn_default_adam.argtypes = [C.POINTER(GnnAdam)]
        L.gnn_adam_step.argtypes = [vp, C.POINTER(GnnAdam)]
        L.gnn_default_train.argtypes = [C.POINTER(GnnTrainParams)]
        L.gnn_train.argtypes = [vp, vp, ip, C.POINTER(GnnTrainParams), vp]
        L.pdlp_start_kkt.argtypes = [C.POINTER(PdlpCsr)] + [vp] * 5 + [vp, vp, vp]
        L.pdlp_solve_warm.argtypes = [vp, C.POINTER(PdlpCsr)] + [vp] * 5 + \
            [C.POINTER(PdlpParams), vp, vp, C.POINTER(PdlpResult), C.POINTER(GnnWarmInfo)]
        _READY = True
    return L


class _LpArrays:
    """Contiguous host copies of an LP's arrays and its pdlp_csr (kept alive together)."""

    def __init__(self, lp):
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.row_ptr = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(lp.col, dtype=np.int32)
        self.val = f64(lp.val)
        self.b, self.c, self.l, self.u = f64(lp.b), f64(lp.c), f64(lp.l), f64(lp.u)
        self.sense = np.ascontiguousarray(lp.sense, dtype=np.uint8)
        self.m, self.n = lp.m, lp.n
        self.csr = PdlpCsr(lp.m, lp.n, int(self.row_ptr[-1]), _ptr(self.row_ptr), _ptr(self.col),
                           _ptr(self.val))

    def args(self):
        return (C.byref(self.csr), _ptr(self.b), _ptr(self.sense), _ptr(self.c), _ptr(self.l),
                _ptr(self.u))


def param_count() -> int:
    return int(_lib().gnn_param_count())


def default_adam(**kw) -> GnnAdam:
    a = GnnAdam()
    _lib().gnn_default_adam(C.byref(a))
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def default_train(**kw) -> GnnTrainParams:
    t = GnnTrainParams()
    _lib().gnn_default_train(C.byref(t))
    for k, v in kw.items():
        if k in ("lr", "beta1", "beta2", "eps"):
            setattr(t.adam, k, v)
        else:
            setattr(t, k, v)
    return t


class GnnModel:
    """Handle of a device-resident network (parameters, Adam state, scratch)."""

    def __init__(self, seed: int = 0, _handle=None):
        self.h = C.c_void_p()
        if _handle is not None:
            self.h = _handle
        else:
            _check(_lib().gnn_create(C.c_uint64(seed), C.byref(self.h)))

    @classmethod
    def load(cls, path: str) -> "GnnModel":
        h = C.c_void_p()
        _check(_lib().gnn_load(path.encode(), C.byref(h)))
        return cls(_handle=h)

    def save(self, path: str):
        _check(_lib().gnn_save(self.h, path.encode()))

    def close(self):
        if self.h:
            _lib().gnn_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(param_count(), dtype=np.float32)
        _check(_lib().gnn_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == param_count()
        _check(_lib().gnn_set_params(self.h, _ptr(a)))

    def grad(self) -> np.ndarray:
        out = np.empty(param_count(), dtype=np.float32)
        _check(_lib().gnn_get_grad(self.h, _ptr(out)))
        return out

    def set_grad(self, g):
        a = np.ascontiguousarray(g, dtype=np.float32)
        assert a.size == param_count()
        _check(_lib().gnn_set_grad(self.h, _ptr(a)))

    def zero_grad(self):
        _check(_lib().gnn_zero_grad(self.h))

    def graph(self, lp, x_star=None, y_star=None) -> "GnnGraph":
        return GnnGraph(self, lp, x_star, y_star)

    def forward(self, g: "GnnGraph"):
        """(x^, y^, loss) as float64 arrays in the caller's sign convention."""
        x = np.empty(g.n)
        y = np.empty(g.m)
        loss = C.c_double()
        _check(_lib().gnn_forward(self.h, g.h, _ptr(x), _ptr(y), C.byref(loss)))
        return x, y, loss.value

    def backward(self, g: "GnnGraph", scale: float = 1.0) -> float:
        loss = C.c_double()
        _check(_lib().gnn_backward(self.h, g.h, C.c_double(scale), C.byref(loss)))
        return loss.value

    def adam_step(self, **kw):
        a = default_adam(**kw)
        _check(_lib().gnn_adam_step(self.h, C.byref(a)))

    def train(self, graphs, **kw) -> np.ndarray:
        t = default_train(**kw)
        arr = (C.c_void_p * len(graphs))(*[g.h.value for g in graphs])
        losses = np.empty(t.epochs)
        _check(_lib().gnn_train(self.h, arr, len(graphs), C.byref(t), _ptr(losses)))
        return losses


class GnnGraph:
    """An LP's graph, features and optional labels on the model's device."""

    def __init__(self, model: GnnModel, lp, x_star=None, y_star=None):
        self.model = model
        self.arr = _LpArrays(lp)
        self.m, self.n = lp.m, lp.n
        self.h = C.c_void_p()
        _check(_lib().gnn_graph_create(model.h, *self.arr.args(), C.byref(self.h)))
        if x_star is not None:
            self.set_labels(x_star, y_star)

    def set_labels(self, x_star, y_star):
        xs = np.ascontiguousarray(x_star, dtype=np.float64)
        ys = np.ascontiguousarray(y_star, dtype=np.float64)
        _check(_lib().gnn_graph_set_labels(self.h, _ptr(xs), _ptr(ys)))

    def features(self):
        fv = np.empty((self.n, 6), dtype=np.float32)
        fc = np.empty((self.m, 5), dtype=np.float32)
        _check(_lib().gnn_graph_features(self.h, _ptr(fv), _ptr(fc)))
        return fv, fc

    def close(self):
        if self.h:
            _lib().gnn_graph_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def start_kkt(lp, x0, y0) -> dict:
    """Relative KKT of the projected start (x0, y0) (float64, on the device)."""
    a = _LpArrays(lp)
    xs = np.ascontiguousarray(x0, dtype=np.float64)
    ys = np.ascontiguousarray(y0, dtype=np.float64)
    out = np.empty(4)
    _check(_lib().pdlp_start_kkt(*a.args(), _ptr(xs), _ptr(ys), _ptr(out)))
    return dict(zip(("rel_primal_res", "rel_dual_res", "rel_gap", "rel_kkt"), out.tolist()))


def pdlp_solve_warm(model: GnnModel | None, lp, params: PdlpParams | None = None):
    """pdlp_solve from the learned start when its KKT beats the cold start's.
    Returns (x, y, result dict, warm-info dict)."""
    p = params or default_params()
    a = _LpArrays(lp)
    x = np.empty(lp.n)
    y = np.empty(lp.m)
    r = PdlpResult()
    info = GnnWarmInfo()
    _check(_lib().pdlp_solve_warm(model.h if model is not None else None, *a.args(), C.byref(p),
                                  _ptr(x), _ptr(y), C.byref(r), C.byref(info)))
    return x, y, r.as_dict(), info.as_dict()
