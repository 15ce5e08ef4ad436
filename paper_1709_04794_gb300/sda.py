"""Thin Python binding of libsda (include/sda.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own.  Arrays may be NumPy arrays (host memory) or torch
tensors (CUDA device memory); streams are torch.cuda.Stream objects, raw
cudaStream_t integers, or None for the legacy default stream.

The library must be built (``python -c "import __graft_entry__ as g;
g.build()"``); without it every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

SDA_OK = 0
SDA_NOT_CONVERGED = 1
SDA_ERR_INVALID_ARG = -1
SDA_ERR_SHAPE = -2
SDA_ERR_INDEX = -3
SDA_ERR_VALUE_NOT_EXACT = -4
SDA_ERR_NO_POSITIVE = -5
SDA_ERR_NO_NEGATIVE = -6
SDA_ERR_NOT_SYMMETRIC = -7
SDA_ERR_BREAKDOWN = -8
SDA_ERR_TIMEOUT = -9
SDA_ERR_CUDA = -10
SDA_ERR_OOM = -11
SDA_ERR_UNSUPPORTED = -12

SDA_F64, SDA_F32, SDA_F16, SDA_F8E4M3, SDA_PATTERN = 0, 1, 2, 3, 4
DTYPES = {"f64": SDA_F64, "f32": SDA_F32, "f16": SDA_F16, "f8e4m3": SDA_F8E4M3, "pattern": SDA_PATTERN}
SDA_RHS_CANONICAL, SDA_RHS_FROM_R, SDA_RHS_GIVEN = 0, 1, 2
SDA_SHIFTS_AUTO, SDA_SHIFTS_RECURRENCE, SDA_SHIFTS_BASIS = 0, 1, 2


class sda_csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("dtype", ctypes.c_int), ("on_device", ctypes.c_int32)]


class sda_labels(ctypes.Structure):
    _fields_ = [("n_targets", ctypes.c_int32), ("labels", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class sda_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("fixed_iters", ctypes.c_int32),
                ("rhs_mode", ctypes.c_int32), ("rhs", ctypes.c_void_p), ("rhs_on_device", ctypes.c_int32),
                ("target_begin", ctypes.c_int32), ("target_count", ctypes.c_int32),
                ("check_residual", ctypes.c_int32), ("out_on_device", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("iter_batch", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("scatter_weight", ctypes.c_double),
                ("refine_rounds", ctypes.c_int32), ("batch_targets", ctypes.c_int32), ("refine_tol", ctypes.c_double),
                ("shift_form", ctypes.c_int32)]


class sda_shift_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("est_residual", ctypes.c_double),
                ("true_residual", ctypes.c_double)]


class sda_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("shift_iterations", ctypes.c_int64),
                ("launches", ctypes.c_int64 * 5), ("ms", ctypes.c_double * 5), ("solve_ms", ctypes.c_double),
                ("shift_form", ctypes.c_int32), ("basis_slots", ctypes.c_int32)]


class sda_operator_info(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("graph_nnz", ctypes.c_int64), ("n_targets", ctypes.c_int32), ("compute", ctypes.c_int),
                ("alpha", ctypes.c_double), ("omega", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("col_ranges", ctypes.c_int32), ("row_head", ctypes.c_int32), ("col_entries", ctypes.c_int64),
                ("row_entries", ctypes.c_int64), ("head_cols", ctypes.c_int32), ("head_ranges", ctypes.c_int32),
                ("head_entries", ctypes.c_int64), ("tuned", ctypes.c_int32 * 4), ("exact_x_passes", ctypes.c_int32),
                ("x_frac_bits", ctypes.c_int16), ("x_int_bits", ctypes.c_int16)]


_vp = ctypes.c_void_p
_SIGS = {
    "sda_build_operator": (ctypes.c_int, [ctypes.POINTER(sda_csr), ctypes.POINTER(sda_csr),
                                          ctypes.POINTER(sda_labels), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "sda_build_regression": (ctypes.c_int, [ctypes.POINTER(sda_csr), ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "sda_build_sa": (ctypes.c_int, [ctypes.POINTER(sda_csr), ctypes.POINTER(sda_labels), ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "sda_default_opts": (None, [ctypes.POINTER(sda_solve_opts)]),
    "sda_solve_shifts": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.POINTER(sda_solve_opts), _vp,
                                        ctypes.POINTER(sda_shift_report), _vp]),
    "sda_project": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int32, ctypes.c_int32, _vp]),
    "sda_project_rows": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, ctypes.c_int64, _vp, ctypes.c_int32,
                                        ctypes.c_int32, _vp]),
    "sda_adjoint_grad": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp,
                                        ctypes.c_int64, ctypes.POINTER(sda_solve_opts), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), _vp, _vp]),
    "sda_adjoint_grad_batched": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp,
                                                ctypes.POINTER(sda_solve_opts), _vp, _vp, _vp,
                                                ctypes.POINTER(sda_shift_report), _vp]),
    "sda_heldout_logistic": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sda_operator_apply": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_double, _vp, _vp, _vp]),
    "sda_operator_apply_static": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_double, _vp, _vp, _vp]),
    "sda_knn_graph": (ctypes.c_int, [ctypes.POINTER(sda_csr), ctypes.c_int32, ctypes.c_int64, ctypes.c_double, _vp,
                                     _vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _vp]),
    "sda_get_operator_info": (ctypes.c_int, [_vp, ctypes.POINTER(sda_operator_info)]),
    "sda_get_target_counts": (ctypes.c_int, [_vp, _vp]),
    "sda_get_solve_stats": (ctypes.c_int, [_vp, ctypes.POINTER(sda_solve_stats)]),
    "sda_kernel_launch_count": (ctypes.c_int64, []),
    "sda_destroy_operator": (None, [_vp]),
    "sda_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sda_last_error_detail": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
}

_LIB = None


def lib_path() -> str:
    return _build.LIBSDA


def load():
    """Loads libsda.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libsda.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


class SDAError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        buf = ctypes.create_string_buffer(512)
        lib.sda_last_error_detail(buf, 512)
        self.code = code
        super().__init__("%s: %s (%s)" % (where, lib.sda_status_string(code).decode(), buf.value.decode()))


def _check(code: int, where: str) -> int:
    if code < 0:
        raise SDAError(code, where)
    return code


# ---------------------------------------------------------------------------
# marshalling
# ---------------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, on_device, keepalive) of a NumPy array or torch tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0, a
    a = np.ascontiguousarray(a)
    return a.ctypes.data, 0, a


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _csr(row_ptr, col_idx, values, n_rows, n_cols, keep):
    rp, dev, k1 = _ptr(row_ptr)
    ci, dev2, k2 = _ptr(col_idx)
    keep += [k1, k2]
    if values is None:
        vp, dt = None, SDA_PATTERN
    else:
        vp, dev3, k3 = _ptr(values)
        keep.append(k3)
        dt = SDA_F32 if str(getattr(values, "dtype", "")).endswith("float32") else SDA_F64
    nnz = int(col_idx.shape[0])
    return sda_csr(int(n_rows), int(n_cols), nnz, rp, ci, vp, dt, dev)


def sda_build_operator(x_ptr, x_col, x_val, n_cols, s_ptr, s_col, s_val, labels, alpha,
                       scatter_weight=float("nan"), compute="f64", stream=None):
    """Calls sda_build_operator; returns the opaque operator handle (int)."""
    lib = load()
    keep = []
    n = int(x_ptr.shape[0]) - 1
    X = _csr(x_ptr, x_col, x_val, n, n_cols, keep)
    S = _csr(s_ptr, s_col, s_val, n, n, keep)
    lp, ldev, lk = _ptr(labels)
    keep.append(lk)
    nt = int(labels.shape[0]) if len(labels.shape) == 2 else 1
    Y = sda_labels(nt, lp, ldev)
    out = _vp()
    comp = DTYPES[compute] if isinstance(compute, str) else int(compute)
    _check(lib.sda_build_operator(ctypes.byref(X), ctypes.byref(S), ctypes.byref(Y), float(alpha),
                                  float(scatter_weight), comp, _stream(stream), ctypes.byref(out)),
           "sda_build_operator")
    return out.value


def sda_build_regression(x_ptr, x_col, x_val, n_cols, compute="f64", stream=None):
    """Calls sda_build_regression (B = X^T X); returns the opaque operator handle (int)."""
    lib = load()
    keep = []
    n = int(x_ptr.shape[0]) - 1
    X = _csr(x_ptr, x_col, x_val, n, n_cols, keep)
    out = _vp()
    comp = DTYPES[compute] if isinstance(compute, str) else int(compute)
    _check(lib.sda_build_regression(ctypes.byref(X), comp, _stream(stream), ctypes.byref(out)),
           "sda_build_regression")
    return out.value


def sda_build_sa(s_ptr, s_col, s_val, labels, alpha, scatter_weight=float("nan"), compute="f64", stream=None):
    """Calls sda_build_sa (SA-SDA: the SDA operator with X = I_N); returns the operator handle (int)."""
    lib = load()
    keep = []
    n = int(s_ptr.shape[0]) - 1
    S = _csr(s_ptr, s_col, s_val, n, n, keep)
    lp, ldev, lk = _ptr(labels)
    keep.append(lk)
    nt = int(labels.shape[0]) if len(labels.shape) == 2 else 1
    Y = sda_labels(nt, lp, ldev)
    out = _vp()
    comp = DTYPES[compute] if isinstance(compute, str) else int(compute)
    _check(lib.sda_build_sa(ctypes.byref(S), ctypes.byref(Y), float(alpha), float(scatter_weight), comp,
                            _stream(stream), ctypes.byref(out)), "sda_build_sa")
    return out.value


def sda_default_opts() -> sda_solve_opts:
    o = sda_solve_opts()
    load().sda_default_opts(ctypes.byref(o))
    return o


def sda_solve_shifts(op, shifts, opts: sda_solve_opts | None = None, w_out=None, n_report: int = 0,
                     stream=None, rhs=None):
    """Calls sda_solve_shifts.  Returns (status, report array [targets][shifts] of dicts)."""
    lib = load()
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    o = opts if opts is not None else sda_default_opts()
    if n_report:
        # the report is [target_count][n_shifts]: refuse a buffer the call would overrun
        count = o.target_count if o.target_count >= 0 else sda_get_operator_info(op)["n_targets"] - o.target_begin
        if n_report < count:
            raise ValueError("n_report=%d is smaller than the %d targets this call solves" % (n_report, count))
    keep = [sh]
    if rhs is not None:
        rp, rdev, rk = _ptr(rhs)
        keep.append(rk)
        o.rhs = rp
        o.rhs_on_device = rdev
    wp = None
    if w_out is not None:
        wp, wdev, wk = _ptr(w_out)
        keep.append(wk)
        o.out_on_device = wdev
    rep = (sda_shift_report * max(1, n_report * sh.size))()
    code = _check(lib.sda_solve_shifts(op, sh.ctypes.data, sh.size, ctypes.byref(o), wp,
                                       rep if n_report else None, _stream(stream)), "sda_solve_shifts")
    out = []
    for t in range(n_report):
        out.append([dict(iters=rep[t * sh.size + s].iters, status=rep[t * sh.size + s].status,
                         est_residual=rep[t * sh.size + s].est_residual,
                         true_residual=rep[t * sh.size + s].true_residual) for s in range(sh.size)])
    return code, out


def sda_project(op, w, n_vec, scores, centred=0, target=0, stream=None):
    lib = load()
    wp, _, wk = _ptr(w)
    sp, _, sk = _ptr(scores)
    return _check(lib.sda_project(op, wp, int(n_vec), sp, int(centred), int(target), _stream(stream)),
                  "sda_project")


def sda_project_rows(op, w, n_vec, rows, scores, centred=0, target=0, stream=None):
    """Calls sda_project_rows: scores [n_vec][len(rows)] of the given rows only."""
    lib = load()
    wp, _, wk = _ptr(w)
    rp, _, rk = _ptr(rows)
    sp, _, sk = _ptr(scores)
    return _check(lib.sda_project_rows(op, wp, int(n_vec), rp, int(rows.shape[0]), sp, int(centred), int(target),
                                       _stream(stream)), "sda_project_rows")


def sda_adjoint_grad(op, target, alpha, beta, w, dloss_ds, rows, opts: sda_solve_opts | None = None,
                     lambda_out=None, stream=None):
    """Calls sda_adjoint_grad; returns (status, d_alpha, d_beta)."""
    lib = load()
    wp, _, wk = _ptr(w)
    gp, _, gk = _ptr(dloss_ds)
    rp, _, rk = _ptr(rows)
    lp, _, lk = _ptr(lambda_out)
    da, db = ctypes.c_double(), ctypes.c_double()
    code = _check(lib.sda_adjoint_grad(op, int(target), float(alpha), float(beta), wp, gp, rp, int(rows.shape[0]),
                                       ctypes.byref(opts) if opts is not None else None, ctypes.byref(da),
                                       ctypes.byref(db), lp, _stream(stream)), "sda_adjoint_grad")
    return code, da.value, db.value


def sda_adjoint_grad_batched(op, targets, alpha, betas, W, dloss_ds, rows, row_off, opts=None, lambda_out=None,
                             stream=None):
    """Calls sda_adjoint_grad_batched; returns (status, d_alpha [n], d_beta [n], reports)."""
    lib = load()
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    bt = np.ascontiguousarray(betas, dtype=np.float64)
    off = np.ascontiguousarray(row_off, dtype=np.int64)
    n = int(tg.size)
    if bt.size != n or off.size != n + 1:
        raise ValueError("targets, betas and row_off must describe the same number of gradients")
    wp, _, wk = _ptr(W)
    gp, _, gk = _ptr(dloss_ds)
    rp, _, rk = _ptr(rows)
    lp, _, lk = _ptr(lambda_out)
    da, db = np.zeros(n), np.zeros(n)
    rep = (sda_shift_report * max(1, n))()
    code = _check(lib.sda_adjoint_grad_batched(op, n, tg.ctypes.data, float(alpha), bt.ctypes.data, wp, gp, rp,
                                               off.ctypes.data, ctypes.byref(opts) if opts is not None else None,
                                               da.ctypes.data, db.ctypes.data, lp, rep, _stream(stream)),
                  "sda_adjoint_grad_batched")
    reps = [dict(iters=rep[i].iters, status=rep[i].status, est_residual=rep[i].est_residual,
                 true_residual=rep[i].true_residual) for i in range(n)]
    return code, da, db, reps


def sda_heldout_logistic(n_shifts, row_off, scores, y, loss, best, g, stream=None):
    """Calls sda_heldout_logistic: loss [n][n_shifts], best [n] (int32) and g
    (one entry per held-out row) into the given contiguous device tensors."""
    lib = load()
    off = np.ascontiguousarray(row_off, dtype=np.int64)
    n = int(off.size) - 1
    if n < 0:
        raise ValueError("row_off needs n_targets + 1 entries")
    for a in (loss, best, g):
        if _is_torch(a) and not a.is_contiguous():
            raise ValueError("output tensors must be contiguous")
    sp, _, sk = _ptr(scores)
    yp, _, yk = _ptr(y)
    lp, _, lk = _ptr(loss)
    bp, _, bk = _ptr(best)
    gp, _, gk = _ptr(g)
    return _check(lib.sda_heldout_logistic(n, int(n_shifts), off.ctypes.data, sp, yp, lp, bp, gp, _stream(stream)),
                  "sda_heldout_logistic")


def sda_operator_apply(op, target, sigma, p, q, stream=None):
    lib = load()
    pp, _, pk = _ptr(p)
    qp, _, qk = _ptr(q)
    return _check(lib.sda_operator_apply(op, int(target), float(sigma), pp, qp, _stream(stream)),
                  "sda_operator_apply")


def sda_operator_apply_static(op, target, sigma, p, q, stream=None):
    """The operator apply without device allocation (scratch in a fixed device array)."""
    lib = load()
    pp, _, pk = _ptr(p)
    qp, _, qk = _ptr(q)
    return _check(lib.sda_operator_apply_static(op, int(target), float(sigma), pp, qp, _stream(stream)),
                  "sda_operator_apply_static")


def sda_knn_graph(x_ptr, x_col, n_cols, k, cap, threshold=0.0, stream=None):
    """Calls sda_knn_graph; returns (row_ptr, col, val) as CUDA tensors (the
    output is sized for the union of the directed lists, 2 N k entries)."""
    import torch
    lib = load()
    keep = []
    n = int(x_ptr.shape[0]) - 1
    X = _csr(x_ptr, x_col, None, n, n_cols, keep)
    cap_out = 2 * n * int(k)
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(max(cap_out, 1), dtype=torch.int32, device="cuda")
    val = torch.empty(max(cap_out, 1), dtype=torch.float64, device="cuda")
    nnz = ctypes.c_int64()
    _check(lib.sda_knn_graph(ctypes.byref(X), int(k), int(cap), float(threshold), rp.data_ptr(), col.data_ptr(),
                             val.data_ptr(), cap_out, ctypes.byref(nnz), _stream(stream)), "sda_knn_graph")
    return rp, col[:nnz.value], val[:nnz.value]


def sda_get_operator_info(op) -> dict:
    info = sda_operator_info()
    _check(load().sda_get_operator_info(op, ctypes.byref(info)), "sda_get_operator_info")
    out = {f: getattr(info, f) for f, _ in sda_operator_info._fields_}
    out["tuned"] = list(info.tuned)
    return out


def sda_get_target_counts(op, n_targets: int) -> np.ndarray:
    c = np.zeros((n_targets, 3))
    _check(load().sda_get_target_counts(op, c.ctypes.data), "sda_get_target_counts")
    return c


def sda_get_solve_stats(op) -> dict:
    st = sda_solve_stats()
    _check(load().sda_get_solve_stats(op, ctypes.byref(st)), "sda_get_solve_stats")
    return dict(iterations=st.iterations, shift_iterations=st.shift_iterations,
                launches=list(st.launches), ms=list(st.ms), solve_ms=st.solve_ms, shift_form=st.shift_form,
                basis_slots=st.basis_slots)


def sda_kernel_launch_count() -> int:
    return int(load().sda_kernel_launch_count())


def sda_destroy_operator(op) -> None:
    if op:
        load().sda_destroy_operator(op)


def sda_status_string(code: int) -> str:
    return load().sda_status_string(int(code)).decode()


def exported_symbols() -> list:
    return sorted(_SIGS)


class Operator:
    """Owns one sda_operator handle (released on close / garbage collection)."""

    @classmethod
    def regression(cls, x_ptr, x_col, x_val, n_cols, compute="f64", stream=None):
        """The X^T X operator of CSR-SDA's regression step (sda_build_regression)."""
        self = cls.__new__(cls)
        self.handle = sda_build_regression(x_ptr, x_col, x_val, n_cols, compute, stream)
        self.info = sda_get_operator_info(self.handle)
        return self

    @classmethod
    def sa(cls, s_ptr, s_col, s_val, labels, alpha, scatter_weight=float("nan"), compute="f64", stream=None):
        """The SA-SDA operator (sda_build_sa): the SDA operator with X = I_N."""
        self = cls.__new__(cls)
        self.handle = sda_build_sa(s_ptr, s_col, s_val, labels, alpha, scatter_weight, compute, stream)
        self.info = sda_get_operator_info(self.handle)
        return self

    def __init__(self, prob=None, compute="f64", alpha=None, scatter_weight=float("nan"), stream=None,
                 device_inputs=False, targets=None, **arrays):
        if prob is not None:
            arrays = dict(x_ptr=prob.x_ptr, x_col=prob.x_col, x_val=prob.x_val, n_cols=prob.d,
                          s_ptr=prob.s_ptr, s_col=prob.s_col, s_val=prob.s_val,
                          labels=prob.labels if targets is None else prob.labels[targets])
            alpha = prob.alpha if alpha is None else alpha
        if device_inputs:
            import torch
            arrays = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
                      for k, v in arrays.items()}
        self.handle = sda_build_operator(arrays["x_ptr"], arrays["x_col"], arrays["x_val"], arrays["n_cols"],
                                         arrays["s_ptr"], arrays["s_col"], arrays["s_val"], arrays["labels"],
                                         alpha, scatter_weight, compute, stream)
        self.info = sda_get_operator_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sda_destroy_operator(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
