"""ctypes binding of libexpdg (C-ABI in include/expdg.h): argument marshalling
only, every step of the path runs in the CUDA library.

Arrays may be numpy float64 arrays (host memory: the library copies them in
and out inside the call) or torch float64 CUDA tensors (device memory, used
in place).  Importing this module loads the library and raises if it has not
been built; there is no fallback path.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("EXPDG_LIB", os.path.join(HERE, "libexpdg.so"))

EXPDG_OK, EXPDG_EINVAL, EXPDG_ENOMEM, EXPDG_EKRYLOV, EXPDG_ENONPHYSICAL, EXPDG_ETIMEOUT, EXPDG_ECUDA = range(7)
EXPDG_BURGERS, EXPDG_EULER = 1, 2
EXPDG_EPI2, EXPDG_EXPRB32, EXPDG_EXPRB42 = 2, 3, 4
EXPDG_FP64, EXPDG_MIXED, EXPDG_MIXED_FF = 0, 1, 2
EXPDG_BC_PERIODIC, EXPDG_BC_DIRICHLET = 0, 1
EXPDG_FLUX_LF, EXPDG_FLUX_ROE = 0, 1
EXPDG_TILE_AUTO, EXPDG_TILE_256, EXPDG_TILE_128, EXPDG_TILE_512, EXPDG_TILE_TC3, EXPDG_TILE_TC1 = 0, 1, 2, 3, 4, 5
EXPDG_MAX_ORDER, EXPDG_MAX_KRYLOV, EXPDG_MAX_PHI, EXPDG_MAX_IOP = 8, 64, 3, 8
STATUS_NAMES = {0: "EXPDG_OK", 1: "EXPDG_EINVAL", 2: "EXPDG_ENOMEM", 3: "EXPDG_EKRYLOV",
                4: "EXPDG_ENONPHYSICAL", 5: "EXPDG_ETIMEOUT", 6: "EXPDG_ECUDA"}


class expdg_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("ne", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("eq", ctypes.c_int),
                ("gamma", ctypes.c_double), ("scheme", ctypes.c_int), ("prec", ctypes.c_int),
                ("krylov_tol", ctypes.c_double), ("m_max", ctypes.c_int), ("m_step", ctypes.c_int),
                ("max_substeps", ctypes.c_int), ("iop", ctypes.c_int), ("kappa", ctypes.c_double),
                ("bc", ctypes.c_int), ("flux", ctypes.c_int), ("tile", ctypes.c_int)]


class expdg_stats(ctypes.Structure):
    _fields_ = [("krylov_iters", ctypes.c_int), ("substeps", ctypes.c_int), ("rejected", ctypes.c_int),
                ("jv_applies", ctypes.c_int), ("residual_applies", ctypes.c_int), ("err_est", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class expdg_trace_entry(ctypes.Structure):
    _fields_ = [("solve", ctypes.c_int), ("m", ctypes.c_int), ("sigma", ctypes.c_double), ("eta", ctypes.c_double)]


class expdg_kernel_prof(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


KERNEL_CLASSES = ["residual", "jv", "dots", "update", "phi", "combine", "vector"]


class expdg_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("workers", ctypes.c_int)]


class ExpdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libexpdg.so not found at {LIB_PATH}; build it with "
                           "'python -m paper_2011_01316_gb300.build' (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    vp = ctypes.POINTER
    sig = {
        "expdg_version": (ctypes.c_char_p, []),
        "expdg_default_config": (None, [vp(expdg_config)]),
        "expdg_create": (ctypes.c_int, [vp(expdg_config), vp(P)]),
        "expdg_destroy": (None, [P]),
        "expdg_set_stream": (ctypes.c_int, [P, P]),
        "expdg_num_unknowns": (ctypes.c_size_t, [P]),
        "expdg_tile_in_use": (ctypes.c_int, [P]),
        "expdg_num_fields": (ctypes.c_int, [P]),
        "expdg_num_elements": (ctypes.c_size_t, [P]),
        "expdg_nodes_per_element": (ctypes.c_int, [P]),
        "expdg_node_coords": (ctypes.c_int, [P, P]),
        "expdg_residual": (ctypes.c_int, [P, P, P]),
        "expdg_set_source": (ctypes.c_int, [P, P]),
        "expdg_jv": (ctypes.c_int, [P, P, P, P]),
        "expdg_phi": (ctypes.c_int, [P, P, ctypes.c_double, P, ctypes.c_int, P, vp(expdg_stats),
                                     P, ctypes.c_int, P, ctypes.c_int, vp(ctypes.c_int)]),
        "expdg_step": (ctypes.c_int, [P, P, ctypes.c_double, vp(expdg_stats), P, ctypes.c_int, P,
                                      ctypes.c_int, vp(ctypes.c_int)]),
        "expdg_advance": (ctypes.c_int, [P, P, ctypes.c_double, ctypes.c_int, vp(expdg_stats)]),
        "expdg_last_error": (ctypes.c_char_p, [P]),
        "expdg_profile_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "expdg_profile_get": (ctypes.c_int, [P, P, ctypes.c_int]),
        "expdg_residual_noalloc": (ctypes.c_int, [vp(expdg_config), P, P, P]),
        "expdg_config_node_coords": (ctypes.c_int, [vp(expdg_config), P]),
        "expdg_context_bytes": (ctypes.c_size_t, [vp(expdg_config)]),
        "expdg_server_create": (ctypes.c_int, [vp(expdg_server_config), vp(P)]),
        "expdg_server_destroy": (None, [P]),
        "expdg_server_submit": (ctypes.c_int, [P, vp(expdg_config), P, ctypes.c_double, ctypes.c_int,
                                               vp(ctypes.c_int64)]),
        "expdg_server_poll": (ctypes.c_int, [P, vp(ctypes.c_int64), ctypes.c_int, vp(ctypes.c_int)]),
        "expdg_server_fetch": (ctypes.c_int, [P, ctypes.c_int64, P, vp(expdg_stats), vp(ctypes.c_double)]),
        "expdg_server_info": (ctypes.c_int, [P, vp(ctypes.c_size_t), vp(ctypes.c_int), vp(ctypes.c_int)]),
        "expdg_batch_create": (ctypes.c_int, [P, ctypes.c_int, vp(P)]),
        "expdg_batch_advance": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
        "expdg_batch_result": (ctypes.c_int, [P, ctypes.c_int, vp(expdg_stats), vp(ctypes.c_int)]),
        "expdg_batch_launches": (ctypes.c_int, [P]),
        "expdg_batch_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
lib = _lib


def _ptr(a):
    """Raw pointer of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 numpy array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 torch tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def version():
    return _lib.expdg_version().decode()


def default_config(**kw):
    c = expdg_config()
    _lib.expdg_default_config(ctypes.byref(c))
    for k, v in kw.items():
        if k in ("ne", "lo", "hi"):
            arr = getattr(c, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(c, k, v)
    return c


def config_node_coords(cfg):
    """Node coordinates [dim, Ne, Np] of a configuration, without a context."""
    nelem = 1
    for d in range(cfg.dim):
        nelem *= cfg.ne[d]
    out = np.zeros((cfg.dim, nelem, (cfg.p + 1) ** cfg.dim))
    st = _lib.expdg_config_node_coords(ctypes.byref(cfg), _ptr(out))
    if st != EXPDG_OK:
        raise ExpdgError(st, "expdg_config_node_coords failed")
    return out


def context_bytes(cfg):
    return int(_lib.expdg_context_bytes(ctypes.byref(cfg)))


def _trace_array(trace):
    if trace is None:
        return None, 0
    arr = (expdg_trace_entry * max(1, len(trace)))()
    for i, (solve, m, sigma, eta) in enumerate(trace):
        arr[i] = expdg_trace_entry(int(solve), int(m), float(sigma), float(eta))
    return arr, len(trace)


class Context:
    """One expdg_ctx.  Methods mirror the C-ABI calls of the same names."""

    TRACE_CAP = 256

    def __init__(self, cfg=None, **kw):
        self.cfg = cfg if cfg is not None else default_config(**kw)
        h = ctypes.c_void_p()
        st = _lib.expdg_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if st != EXPDG_OK:
            raise ExpdgError(st, "expdg_create failed")
        self.h = h
        self.n = _lib.expdg_num_unknowns(h)
        self.m = _lib.expdg_num_fields(h)
        self.nelem = _lib.expdg_num_elements(h)
        self.np = _lib.expdg_nodes_per_element(h)
        self.tile = _lib.expdg_tile_in_use(h)  # expdg_tile of the operator apply (autotuned when AUTO)

    def close(self):
        if getattr(self, "h", None):
            _lib.expdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != EXPDG_OK:
            raise ExpdgError(st, _lib.expdg_last_error(self.h).decode())

    @property
    def shape(self):
        return (self.m, self.nelem, self.np)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(_lib.expdg_set_stream(self.h, ctypes.c_void_p(raw or 0)))

    def node_coords(self):
        out = np.zeros((self.cfg.dim, self.nelem, self.np))
        self._check(_lib.expdg_node_coords(self.h, _ptr(out)))
        return out

    def set_source(self, s):
        """Forcing added to R (canonical layout, N values); None removes it."""
        self._check(_lib.expdg_set_source(self.h, None if s is None else _ptr(s)))

    def residual(self, q, out=None):
        out = np.empty_like(q) if out is None else out
        self._check(_lib.expdg_residual(self.h, _ptr(q), _ptr(out)))
        return out

    def jv(self, qt, v, out=None):
        out = np.empty_like(v) if out is None else out
        self._check(_lib.expdg_jv(self.h, _ptr(qt), _ptr(v), _ptr(out)))
        return out

    def phi(self, qt, tau, c, out=None, replay=None):
        """sum_i phi_i(tau L(qt)) c_i; c is a list [c_0, ..., c_P] (None = zero).
        Returns (out, stats dict, trace list)."""
        P = len(c) - 1
        ptrs = (ctypes.c_void_p * len(c))(*[_ptr(x) for x in c])
        ref = next(x for x in c if x is not None) if any(x is not None for x in c) else qt
        out = np.empty_like(ref) if out is None else out
        st = expdg_stats()
        rep, nrep = _trace_array(replay)
        tr = (expdg_trace_entry * self.TRACE_CAP)()
        ntr = ctypes.c_int(0)
        self._check(_lib.expdg_phi(self.h, _ptr(qt), float(tau), ptrs, P, _ptr(out), ctypes.byref(st),
                                   rep, nrep, tr, self.TRACE_CAP, ctypes.byref(ntr)))
        trace = [(tr[i].solve, tr[i].m, tr[i].sigma, tr[i].eta) for i in range(min(ntr.value, self.TRACE_CAP))]
        return out, st.as_dict(), trace

    def step(self, q, dt, replay=None):
        """One exponential step in place; returns (stats dict, trace list)."""
        st = expdg_stats()
        rep, nrep = _trace_array(replay)
        tr = (expdg_trace_entry * self.TRACE_CAP)()
        ntr = ctypes.c_int(0)
        self._check(_lib.expdg_step(self.h, _ptr(q), float(dt), ctypes.byref(st), rep, nrep, tr,
                                    self.TRACE_CAP, ctypes.byref(ntr)))
        trace = [(tr[i].solve, tr[i].m, tr[i].sigma, tr[i].eta) for i in range(min(ntr.value, self.TRACE_CAP))]
        return st.as_dict(), trace

    def profile_enable(self, on=True):
        self._check(_lib.expdg_profile_enable(self.h, 1 if on else 0))

    def profile_get(self, reset=True):
        """Per kernel class: {name: {launches, ms, bytes}} since the last enable/reset."""
        arr = (expdg_kernel_prof * len(KERNEL_CLASSES))()
        self._check(_lib.expdg_profile_get(self.h, arr, 1 if reset else 0))
        return {n: {"launches": int(arr[i].launches), "ms": float(arr[i].ms), "bytes": float(arr[i].bytes)}
                for i, n in enumerate(KERNEL_CLASSES)}

    def advance(self, q, dt, nsteps):
        st = expdg_stats()
        self._check(_lib.expdg_advance(self.h, _ptr(q), float(dt), int(nsteps), ctypes.byref(st)))
        return st.as_dict()


BATCH_MAX_KRYLOV = 40   # EXPDG_BATCH_MAX_KRYLOV


class Batch:
    """One expdg_batch: n small EPI2 solves, one kernel launch per class of
    equal (eq, dim, p, prec).  Methods mirror the C-ABI calls."""

    def __init__(self, cfgs):
        self.n = len(cfgs)
        self._cfgs = (expdg_config * self.n)(*cfgs)
        h = ctypes.c_void_p()
        st = _lib.expdg_batch_create(self._cfgs, self.n, ctypes.byref(h))
        if st != EXPDG_OK:
            raise ExpdgError(st, "expdg_batch_create failed")
        self.h = h

    def launches(self):
        return int(_lib.expdg_batch_launches(self.h))

    def advance(self, qs, dts, nsteps, stream=None):
        """nsteps steps of instance i from device tensor qs[i] (float64,
        contiguous) with step dts[i], in place.  Returns the call's status
        (EXPDG_OK or the first failing instance's)."""
        if len(qs) != self.n or len(dts) != self.n:
            raise ValueError("one state and one dt per instance")
        ptrs = (ctypes.c_void_p * self.n)(*[_ptr(q) for q in qs])
        dt = (ctypes.c_double * self.n)(*[float(x) for x in dts])
        return _lib.expdg_batch_advance(self.h, ptrs, dt, int(nsteps), stream)

    def result(self, i):
        """(status, stats dict, steps done) of instance i after the last advance."""
        st = expdg_stats()
        done = ctypes.c_int(0)
        status = _lib.expdg_batch_result(self.h, int(i), ctypes.byref(st), ctypes.byref(done))
        return status, st.as_dict(), done.value

    def close(self):
        if self.h:
            _lib.expdg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
