"""ctypes binding of libsa (include/sa.h): argument marshalling only.

Functions keep the C names.  Host arrays are numpy float64/int32/uint8;
device arrays are anything with ``data_ptr()`` (torch tensors) and are
passed with ``on_device=1``.  A non-zero status raises ``SAError``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsa.so")

SA_OK, SA_ERR_ARG, SA_ERR_GEOMETRY, SA_ERR_STATE, SA_ERR_CUDA, SA_ERR_OOM, \
    SA_ERR_NOT_CONVERGED, SA_ERR_TIMEOUT, SA_ERR_NAN = range(9)
SA_FP64, SA_MIXED = 0, 1
SA_PCG_AUTO, SA_PCG_SHARED, SA_PCG_GLOBAL = 0, 1, 2
SA_GUESS_PREVIOUS, SA_GUESS_EXTRAPOLATE = 0, 1
SA_PRECOND_AUTO, SA_PRECOND_JACOBI, SA_PRECOND_FD = 0, 1, 2
SA_HIST_AUTO, SA_HIST_PAIRWISE, SA_HIST_SEPARABLE = 0, 1, 2
SA_FACE_NONE, SA_FACE_NEUMANN, SA_FACE_DIRICHLET = 0, 1, 2
SA_FIELD_THAT, SA_FIELD_F, SA_FIELD_DTDN_LAT, SA_FIELD_TT_BOT, SA_FIELD_LAT_X, SA_FIELD_BOT_X = range(6)
STAGES = ("prologue", "history", "gather", "bottom", "rhs", "pcg", "finalize")


class sa_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("pcg_tol", C.c_double), ("pcg_max_iter", C.c_int),
                ("half_space_factor", C.c_double), ("cuda_stream", C.c_void_p),
                ("use_graph", C.c_int), ("device", C.c_int),
                ("hist_points_per_lane", C.c_int), ("hist_warps", C.c_int),
                ("stage_timing", C.c_int), ("pcg_variant", C.c_int),
                ("initial_guess", C.c_int), ("precond", C.c_int), ("hist_mode", C.c_int),
                ("hist_cutoff", C.c_double)]


class sa_step_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int), ("pcg_iters_last", C.c_int),
                ("pcg_iters_total", C.c_int), ("pcg_iters_max", C.c_int),
                ("bot_iters_total", C.c_int), ("rel_res_last", C.c_double),
                ("n_active_sources", C.c_int), ("step_index", C.c_longlong),
                ("ws_used_last", C.c_int), ("ws_ratio_last", C.c_double),
                ("hist_pairs_skipped", C.c_longlong)]


class sa_sizes(C.Structure):
    _fields_ = [("n_dof", C.c_int), ("n_free", C.c_int), ("n_dir", C.c_int),
                ("q_lat", C.c_int), ("q_bot", C.c_int), ("n_src", C.c_int),
                ("nnz_mk", C.c_longlong), ("nnz_a", C.c_longlong),
                ("step_index", C.c_longlong), ("n_elem", C.c_int),
                ("hist_separable", C.c_int), ("sep_factors", C.c_longlong)]


class sa_batch_shapes(C.Structure):
    _fields_ = [("hist_separable", C.c_int), ("tj_lat", C.c_int), ("tj_bot", C.c_int),
                ("units_per_tile", C.c_int), ("hist_P", C.c_int), ("hist_NW", C.c_int),
                ("pcg_grid", C.c_int), ("step_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsa.so not built ({LIB_PATH}); run "
                          "`python -m paper_2511_20432_gb300.build` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    P, I, D, LL, V = C.c_void_p, C.c_int, C.c_double, C.c_longlong, None
    sig = {
        "sa_options_default": (V, [C.POINTER(sa_options)]),
        "sa_create": (I, [C.POINTER(sa_options), C.POINTER(P)]),
        "sa_create_patch": (I, [P, P, P, P, P, P, P, I]),
        "sa_set_boundary": (I, [P, P]),
        "sa_set_material": (I, [P, D, D, D, D]),
        "sa_set_scan": (I, [P, P, I, P, D, D, D, D]),
        "sa_step": (I, [P, D, D, I, C.POINTER(sa_step_stats)]),
        "sa_eval_T": (I, [P, P, I, P, I]),
        "sa_eval_T_noalloc": (I, [P, P, I, P]),
        "sa_eval_T_superposed": (I, [P, I, P, I, P, I]),
        "sa_eval_flux": (I, [P, P, P, I, P, P, I]),
        "sa_get_sizes": (I, [P, C.POINTER(sa_sizes)]),
        "sa_get_field": (I, [P, I, P, LL, I]),
        "sa_get_matrix_nnz": (I, [P, C.POINTER(LL)]),
        "sa_get_matrix": (I, [P, I, P, P, P]),
        "sa_get_state": (I, [P, C.POINTER(LL), P, P]),
        "sa_set_state": (I, [P, LL, P, P]),
        "sa_get_stage_times": (I, [P, P, C.POINTER(LL)]),
        "sa_mlp_create": (I, [I, I, I, C.c_ulonglong, C.POINTER(P)]),
        "sa_mlp_destroy": (V, [P]),
        "sa_mlp_n_params": (LL, [P]),
        "sa_mlp_get_params": (I, [P, P]),
        "sa_mlp_set_params": (I, [P, P]),
        "sa_mlp_forward": (I, [P, P, I, P, P]),
        "sa_mlp_gradients": (I, [P, P, P, I, P, C.POINTER(D), P]),
        "sa_mlp_train_step": (I, [P, P, P, I, C.c_float, C.POINTER(D), P]),
        "sa_set_warm_start": (I, [P, P, I, P]),
        "sa_set_recorder": (I, [P, P, P, I, I, P]),
        "sa_get_recorded": (I, [P, C.POINTER(I)]),
        "sa_batch_create": (I, [P, I, C.POINTER(sa_options), C.POINTER(P)]),
        "sa_batch_step": (I, [P, D, D, I, C.POINTER(sa_step_stats)]),
        "sa_batch_get_field": (I, [P, I, I, P, LL]),
        "sa_batch_get_iters": (I, [P, P, P]),
        "sa_batch_autotune": (I, [P, C.c_char_p, C.POINTER(I), C.POINTER(I), C.POINTER(D)]),
        "sa_batch_tune": (I, [P, C.c_char_p, LL, C.POINTER(sa_batch_shapes)]),
        "sa_batch_get_shapes": (I, [P, C.POINTER(sa_batch_shapes)]),
        "sa_batch_last_error": (C.c_char_p, [P]),
        "sa_batch_destroy": (V, [P]),
        "sa_destroy": (V, [P]),
        "sa_status_str": (C.c_char_p, [I]),
        "sa_selftest_waits": (I, [C.POINTER(I), C.POINTER(I)]),
        "sa_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def status_name(s):
    return lib.sa_status_str(int(s)).decode()


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _check(ctx, status):
    if status != SA_OK:
        msg = lib.sa_last_error(ctx).decode() if ctx else ""
        raise SAError(status, msg)


def options(**kw) -> sa_options:
    o = sa_options()
    lib.sa_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = int(v.cuda_stream)
        setattr(o, k, v)
    return o


class Context:
    """Owns one sa_ctx.  Every method is one C call."""

    def __init__(self, opts: sa_options | None = None, **kw):
        self.ptr = C.c_void_p()
        o = opts if opts is not None else options(**kw)
        self._opts = o
        _check(None, lib.sa_create(C.byref(o), C.byref(self.ptr)))

    def close(self):
        if self.ptr:
            lib.sa_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- set-up -------------------------------------------------------------
    def set_boundary(self, face_kind):
        fk = np.ascontiguousarray(face_kind, dtype=np.int32)
        _check(self.ptr, lib.sa_set_boundary(self.ptr, _ptr(fk)))

    def create_patch(self, degree, n_ctrl, ctrl_xyz, weights, knots, seam_dir=-1):
        deg = np.ascontiguousarray(degree, dtype=np.int32)
        nc = np.ascontiguousarray(n_ctrl, dtype=np.int32)
        ctrl = np.ascontiguousarray(ctrl_xyz, dtype=np.float64)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        ks = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        kp = (C.c_void_p * 3)(*[k.ctypes.data for k in ks])
        nk = np.array([len(k) for k in ks], dtype=np.int32)
        _check(self.ptr, lib.sa_create_patch(self.ptr, _ptr(deg), _ptr(nc), _ptr(ctrl), _ptr(w),
                                             C.cast(kp, C.c_void_p), _ptr(nk), int(seam_dir)))

    def set_material(self, k, rho, cp, T_c):
        _check(self.ptr, lib.sa_set_material(self.ptr, k, rho, cp, T_c))

    def set_scan(self, path_xyz, seg_on, power, absorptivity, speed, spot_radius):
        path = np.ascontiguousarray(path_xyz, dtype=np.float64)
        on = None if seg_on is None else np.ascontiguousarray(seg_on, dtype=np.uint8)
        _check(self.ptr, lib.sa_set_scan(self.ptr, _ptr(path), int(path.shape[0]), _ptr(on),
                                         power, absorptivity, speed, spot_radius))

    # ---- stepping ---------------------------------------------------------------
    def step(self, theta, dt, n_steps=1, stats=True):
        st = sa_step_stats() if stats else None
        _check(self.ptr, lib.sa_step(self.ptr, theta, dt, int(n_steps),
                                     C.byref(st) if st is not None else None))
        return st

    def eval_T(self, pts, out=None, on_device=False):
        if on_device:
            n = pts.shape[0]
            _check(self.ptr, lib.sa_eval_T(self.ptr, _ptr(pts), int(n), _ptr(out), 1))
            return out
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        if out is not None:   # a caller's host buffer (e.g. pinned), n contiguous FP64
            if out.dtype != np.float64 or out.size != p.shape[0] or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out: a contiguous float64 array of one value per point")
            o = out
        else:
            o = np.empty(p.shape[0])
        _check(self.ptr, lib.sa_eval_T(self.ptr, _ptr(p), int(p.shape[0]), _ptr(o), 0))
        return o

    def eval_flux(self, pts, nrm):
        """Heat-loss rates (q~, q^) = (-k n . grad T~, -k n . grad T^) at host
        points with unit normals."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        nv = np.ascontiguousarray(nrm, dtype=np.float64).reshape(-1, 3)
        if nv.shape != p.shape:
            raise ValueError("pts and nrm differ in shape")
        qt = np.empty(p.shape[0])
        qh = np.empty(p.shape[0])
        _check(self.ptr, lib.sa_eval_flux(self.ptr, _ptr(p), _ptr(nv), int(p.shape[0]), _ptr(qt),
                                          _ptr(qh), 0))
        return qt, qh

    # ---- read-back --------------------------------------------------------------
    def sizes(self) -> sa_sizes:
        s = sa_sizes()
        _check(self.ptr, lib.sa_get_sizes(self.ptr, C.byref(s)))
        return s

    def field(self, which, count=None):
        s = self.sizes()
        n = {SA_FIELD_THAT: s.n_dof, SA_FIELD_F: s.n_dof, SA_FIELD_DTDN_LAT: s.q_lat,
             SA_FIELD_TT_BOT: s.q_bot, SA_FIELD_LAT_X: 7 * s.q_lat,
             SA_FIELD_BOT_X: 4 * s.q_bot}[which] if count is None else count
        o = np.empty(max(n, 1))
        _check(self.ptr, lib.sa_get_field(self.ptr, int(which), _ptr(o), int(n), 0))
        return o[:n]

    def matrix(self, which):
        nnz = C.c_longlong()
        _check(self.ptr, lib.sa_get_matrix_nnz(self.ptr, C.byref(nnz)))
        n = self.sizes().n_dof
        ptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value)
        _check(self.ptr, lib.sa_get_matrix(self.ptr, int(which), _ptr(ptr), _ptr(col), _ptr(val)))
        return ptr, col, val

    def stage_times(self):
        ms = np.zeros(len(STAGES))
        k = C.c_longlong()
        _check(self.ptr, lib.sa_get_stage_times(self.ptr, _ptr(ms), C.byref(k)))
        return dict(zip(STAGES, ms)), k.value

    def set_warm_start(self, net, in_idx):
        if net is None:
            _check(self.ptr, lib.sa_set_warm_start(self.ptr, None, 0, None))
            return
        idx = np.ascontiguousarray(in_idx, dtype=np.int32)
        _check(self.ptr, lib.sa_set_warm_start(self.ptr, net.ptr, int(idx.size), _ptr(idx)))

    def set_recorder(self, X, Y, in_idx):
        if X is None:
            _check(self.ptr, lib.sa_set_recorder(self.ptr, None, None, 0, 0, None))
            return
        idx = np.ascontiguousarray(in_idx, dtype=np.int32)
        _check(self.ptr, lib.sa_set_recorder(self.ptr, _ptr(X), _ptr(Y), int(X.shape[0]),
                                             int(idx.size), _ptr(idx)))

    def recorded(self):
        k = C.c_int()
        _check(self.ptr, lib.sa_get_recorded(self.ptr, C.byref(k)))
        return k.value

    def get_state(self):
        n = self.sizes().n_dof
        T = np.empty(n)
        F = np.empty(n)
        k = C.c_longlong()
        _check(self.ptr, lib.sa_get_state(self.ptr, C.byref(k), _ptr(T), _ptr(F)))
        return k.value, T, F

    def set_state(self, n, T, F):
        T = np.ascontiguousarray(T, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        _check(self.ptr, lib.sa_set_state(self.ptr, int(n), _ptr(T), _ptr(F)))


class MLP:
    """The warm-start network (sa_mlp): tensors are torch CUDA tensors."""

    def __init__(self, n_in, hidden, n_out, seed=1):
        self.ptr = C.c_void_p()
        st = lib.sa_mlp_create(int(n_in), int(hidden), int(n_out), int(seed), C.byref(self.ptr))
        if st != SA_OK:
            raise SAError(st, "sa_mlp_create")
        self.n_in, self.hidden, self.n_out = n_in, hidden, n_out

    def close(self):
        if self.ptr:
            lib.sa_mlp_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_params(self):
        return int(lib.sa_mlp_n_params(self.ptr))

    def params(self):
        out = np.empty(self.n_params(), dtype=np.float32)
        _check(None, lib.sa_mlp_get_params(self.ptr, _ptr(out)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(None, lib.sa_mlp_set_params(self.ptr, _ptr(p)))

    def forward(self, X, out, stream=None):
        s = None if stream is None else C.c_void_p(int(stream.cuda_stream))
        _check(None, lib.sa_mlp_forward(self.ptr, _ptr(X), int(X.shape[0]), _ptr(out), s))
        return out

    def gradients(self, X, Y, stream=None):
        g = np.empty(self.n_params(), dtype=np.float32)
        loss = C.c_double()
        s = None if stream is None else C.c_void_p(int(stream.cuda_stream))
        _check(None, lib.sa_mlp_gradients(self.ptr, _ptr(X), _ptr(Y), int(X.shape[0]), _ptr(g),
                                          C.byref(loss), s))
        return loss.value, g

    def train_step(self, X, Y, lr, want_loss=True, stream=None):
        loss = C.c_double()
        s = None if stream is None else C.c_void_p(int(stream.cuda_stream))
        _check(None, lib.sa_mlp_train_step(self.ptr, _ptr(X), _ptr(Y), int(X.shape[0]), float(lr),
                                           C.byref(loss) if want_loss else None, s))
        return loss.value if want_loss else None


class Batch:
    """Owns one sa_batch over existing Contexts (kept alive here)."""

    def __init__(self, contexts, opts: sa_options | None = None, **kw):
        self.contexts = list(contexts)
        self.ptr = C.c_void_p()
        o = opts if opts is not None else options(**kw)
        self._opts = o
        arr = (C.c_void_p * len(self.contexts))(*[c.ptr.value for c in self.contexts])
        st = lib.sa_batch_create(C.cast(arr, C.c_void_p), len(self.contexts), C.byref(o),
                                 C.byref(self.ptr))
        if st != SA_OK:
            raise SAError(st, "sa_batch_create")

    def _check(self, st):
        if st != SA_OK:
            raise SAError(st, lib.sa_batch_last_error(self.ptr).decode())

    def close(self):
        if self.ptr:
            lib.sa_batch_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, theta, dt, n_steps=1, stats=True):
        st = sa_step_stats() if stats else None
        self._check(lib.sa_batch_step(self.ptr, theta, dt, int(n_steps),
                                      C.byref(st) if st is not None else None))
        return st

    def field(self, inst, which):
        s = self.contexts[inst].sizes()
        n = {SA_FIELD_THAT: s.n_dof, SA_FIELD_F: s.n_dof, SA_FIELD_DTDN_LAT: s.q_lat,
             SA_FIELD_TT_BOT: s.q_bot}[which]
        o = np.empty(max(n, 1))
        self._check(lib.sa_batch_get_field(self.ptr, int(inst), int(which), _ptr(o), int(n)))
        return o[:n]

    def iters(self):
        m = np.zeros(len(self.contexts), dtype=np.int32)
        b = np.zeros(len(self.contexts), dtype=np.int32)
        self._check(lib.sa_batch_get_iters(self.ptr, _ptr(m), _ptr(b)))
        return m, b

    def autotune(self, cache_path=None):
        P, W, ms = C.c_int(), C.c_int(), C.c_double()
        path = cache_path.encode() if cache_path else None
        self._check(lib.sa_batch_autotune(self.ptr, path, C.byref(P), C.byref(W), C.byref(ms)))
        return P.value, W.value, ms.value

    def tune(self, cache_path=None, at_step=0):
        """sa_batch_tune: history tile shapes (sources active at at_step; 0:
        the next step) and solve grid; returns a dict."""
        sh = sa_batch_shapes()
        path = cache_path.encode() if cache_path else None
        self._check(lib.sa_batch_tune(self.ptr, path, int(at_step), C.byref(sh)))
        return sh.as_dict()

    def shapes(self):
        sh = sa_batch_shapes()
        self._check(lib.sa_batch_get_shapes(self.ptr, C.byref(sh)))
        return sh.as_dict()


def eval_T_superposed(ctxs, pts, out=None, on_device=False):
    """T at points for several lasers on one part: ctxs[l] carries laser l
    alone (same patch, material and step); sa_eval_T_superposed forms
    sum_l T_l - (L - 1) T_c on the device (see include/sa.h)."""
    arr = (C.c_void_p * len(ctxs))(*[c.ptr.value for c in ctxs])
    c0 = ctxs[0].ptr if ctxs else None
    if on_device:
        _check(c0, lib.sa_eval_T_superposed(arr, len(ctxs), _ptr(pts), int(pts.shape[0]), _ptr(out), 1))
        return out
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    o = np.empty(p.shape[0]) if out is None else out
    _check(c0, lib.sa_eval_T_superposed(arr, len(ctxs), _ptr(p), int(p.shape[0]), _ptr(o), 0))
    return o


def selftest_waits():
    """Run the bounded-wait self-test (see include/sa.h): returns whether the
    grid-barrier wait and the mbarrier wait gave up and flagged a timeout."""
    a, b = C.c_int(0), C.c_int(0)
    st = lib.sa_selftest_waits(C.byref(a), C.byref(b))
    if st != SA_OK:
        raise SAError(st, "sa_selftest_waits: " + status_name(st))
    return bool(a.value), bool(b.value)


def context_from_workload(wl, precision=SA_FP64, s_img=2.0, **opts):
    """Build a Context from a workloads.Workload description (marshalling)."""
    ctx = Context(precision=precision, half_space_factor=s_img, **opts)
    p = wl.patch
    ctx.set_boundary(p.faces)
    ctx.create_patch(p.degree, p.n_ctrl, p.ctrl.reshape(-1, 3), None if p.weights is None
                     else p.weights.ravel(), p.knots, getattr(p, "seam", -1))
    m = wl.material
    ctx.set_material(m.k, m.rho, m.cp, m.T_c)
    s = wl.scan
    ctx.set_scan(s.path, s.seg_on, s.power, s.absorptivity, s.speed, s.spot_radius)
    return ctx
