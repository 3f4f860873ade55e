"""ctypes binding of libsadmm.so (include/sadmm.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  Host arrays are numpy; device arrays are torch CUDA tensors, whose
data pointers are passed straight through.  The library must have been built
(``paper_2307_08606_gb300.build.build()``); loading fails loudly otherwise.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTREADY, ENONFINITE = 0, -1, -2, -3, -4, -5, -6


class SadmmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"sadmm status {status}: {message}")
        self.status = status


class Criterion(C.Structure):
    _fields_ = [("mu", C.c_double), ("Kp", C.c_int), ("eps_p", C.c_double),
                ("eps_abs", C.c_double), ("eps_rel", C.c_double), ("elim", C.c_int),
                ("freeze_mode", C.c_int), ("stop", C.c_int), ("precision", C.c_int),
                ("correct_every", C.c_int), ("learn_every", C.c_int), ("learn_theta", C.c_double),
                ("readmit", C.c_double), ("ssc_every", C.c_int), ("consensus", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("stop_reason", C.c_int), ("refreshes", C.c_int),
                ("active_total", C.c_int), ("learned_steps", C.c_int), ("readmitted", C.c_int),
                ("r_pri", C.c_double), ("eps_pri", C.c_double),
                ("d", C.c_double), ("eps_dual", C.c_double), ("relchange", C.c_double),
                ("ms_total", C.c_double), ("ms_refresh", C.c_double), ("bytes_iter", C.c_double),
                ("proposed", C.c_int), ("proposed_readmitted", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IterRecord(C.Structure):
    _fields_ = [("k", C.c_int), ("gate", C.c_int), ("changed", C.c_int), ("active_total", C.c_int),
                ("learned", C.c_int), ("readmitted", C.c_int), ("r_pri", C.c_double), ("eps_pri", C.c_double), ("d", C.c_double),
                ("eps_dual", C.c_double), ("relchange", C.c_double)]


class BatchTuning(C.Structure):
    _fields_ = [("n_fwd", C.c_int), ("n_adj", C.c_int),
                ("fwd_splits", C.c_int * 8), ("adj_splits", C.c_int * 8),
                ("fwd_ms", C.c_double * 8), ("adj_ms", C.c_double * 8),
                ("fwd_choice", C.c_int), ("adj_choice", C.c_int),
                ("fwd_default", C.c_int), ("adj_default", C.c_int)]

    def as_dict(self):
        return {"forward": {int(self.fwd_splits[i]): float(self.fwd_ms[i]) for i in range(self.n_fwd)},
                "adjoint": {int(self.adj_splits[i]): float(self.adj_ms[i]) for i in range(self.n_adj)},
                "forward_splits": int(self.fwd_choice), "adjoint_splits": int(self.adj_choice),
                "forward_default": int(self.fwd_default), "adjoint_default": int(self.adj_default)}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_P = C.c_void_p
_SIGS = {
    "sadmm_default_criterion": (None, [C.POINTER(Criterion)]),
    "sadmm_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, _P]),
    "sadmm_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                               C.POINTER(Criterion), C.POINTER(_P)]),
    "sadmm_set_stream": (C.c_int, [_P, _P]),
    "sadmm_set_operator": (C.c_int, [_P, C.c_int, _P]),
    "sadmm_set_operator_delays": (C.c_int, [_P, C.c_int, _P, C.c_double, C.c_double]),
    "sadmm_set_products": (C.c_int, [_P, C.c_int]),
    "sadmm_backprojection": (C.c_int, [_P, _P, _P]),
    "sadmm_operator_tables": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _P, _P, _P, _P]),
    "sadmm_forward_factored": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P, _P, _P, _P]),
    "sadmm_adjoint_factored": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P, _P, _P]),
    "sadmm_prepare": (C.c_int, [_P]),
    "sadmm_solve": (C.c_int, [_P, C.POINTER(_P), _P, C.c_int, C.c_double, C.POINTER(Stats)]),
    "sadmm_resume": (C.c_int, [_P, _P, C.c_int, C.c_double, C.POINTER(Stats)]),
    "sadmm_get_xq": (C.c_int, [_P, C.c_int, _P]),
    "sadmm_get_active": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int)]),
    "sadmm_history": (C.c_int, [_P, C.POINTER(IterRecord), C.c_int]),
    "sadmm_get_state": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "sadmm_set_state": (C.c_int, [_P, _P, C.c_size_t]),
    "sadmm_set_profiling": (C.c_int, [_P, C.c_int]),
    "sadmm_set_eliminator": (C.c_int, [_P, _P, C.c_int, C.c_int]),
    "sadmm_features": (C.c_int, [_P, _P]),
    "sadmm_profile": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]),
    "sadmm_launch_count": (C.c_longlong, []),
    "sadmm_destroy": (None, [_P]),
    "sadmm_strerror": (C.c_char_p, [C.c_int]),
    "sadmm_last_error": (C.c_char_p, []),
    "sadmm_forward": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, _P, _P, _P, _P]),
    "sadmm_forward_noalloc": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, _P, _P, _P, _P]),
    "sadmm_adjoint": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, _P, _P, _P]),
    "sadmm_factor": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, C.c_double, C.c_double, _P,
                               C.c_int, C.POINTER(C.c_int), _P]),
    "sadmm_spd_apply": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "sadmm_set_wait_limit": (C.c_int, [C.c_longlong]),
    "sadmm_set_criterion": (C.c_int, [_P, _P]),
    "sadmm_set_lambda": (C.c_int, [_P, C.c_double]),
    "sadmm_digit_apply16": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "sadmm_gram": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, C.c_double, C.c_double, C.c_int, _P, C.c_int, _P,
                             _P]),
    "sadmm_factor_downdate": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_double, _P, _P]),
    "sadmm_factor_update": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_double, C.c_int, _P, _P]),
    "sadmm_forward16_tc": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "sadmm_adjoint16_tc": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "sadmm_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                     C.POINTER(C.c_double), C.POINTER(Criterion), C.POINTER(_P)]),
    "sadmm_batch_set_stream": (C.c_int, [_P, _P]),
    "sadmm_batch_set_operator": (C.c_int, [_P, C.c_int, _P]),
    "sadmm_batch_solve": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(Stats)]),
    "sadmm_batch_get_xq": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "sadmm_batch_destroy": (None, [_P]),
    "sadmm_batch_tune": (C.c_int, [_P, C.c_int, C.POINTER(BatchTuning)]),
    "sadmm_batch_group_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P)]),
    "sadmm_batch_group_set_stream": (C.c_int, [_P, _P]),
    "sadmm_batch_group_solve": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.c_int, C.POINTER(Stats)]),
    "sadmm_batch_group_destroy": (None, [_P]),
    "sadmm_cnn_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    "sadmm_cnn_num_params": (C.c_int, []),
    "sadmm_cnn_set_params": (C.c_int, [_P, _P]),
    "sadmm_cnn_get_params": (C.c_int, [_P, _P, C.c_int]),
    "sadmm_cnn_forward": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "sadmm_cnn_backward": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, _P, C.POINTER(C.c_double), _P]),
    "sadmm_cnn_adam_step": (C.c_int, [_P, _P, C.c_double, _P]),
    "sadmm_cnn_destroy": (None, [_P]),
    "sadmm_split_operator": (C.c_int, [_P, C.c_size_t, C.c_int, _P, _P, _P]),
    "sadmm_forward_split": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P, _P,
                                      _P, _P]),
    "sadmm_adjoint_split": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P, _P,
                                      _P]),
}

_lib = None


def library_path():
    return LIB


def load():
    """Load libsadmm.so and declare its signatures (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it with paper_2307_08606_gb300.build.build()")
    lib = C.CDLL(LIB)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def launch_count():
    """Kernels launched by the library in this process."""
    return int(load().sadmm_launch_count())


def check(status):
    if status != OK:
        lib = load()
        raise SadmmError(status, lib.sadmm_last_error().decode(errors="replace"))
    return status


def default_criterion(**kw):
    c = Criterion()
    load().sadmm_default_criterion(C.byref(c))
    names = {f for f, _ in Criterion._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown criterion field {k!r}")
        setattr(c, k, v)
    return c


# ------------------------------------------------------------------ torch glue
_torch_alloc = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc
    import torch

    def _alloc(nbytes, stream, user):
        dev = torch.cuda.current_device()
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    _torch_alloc = (ALLOC_FN(_alloc), FREE_FN(_free))
    check(load().sadmm_set_allocator(_torch_alloc[0], _torch_alloc[1], None))


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _as_c64(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.complex64)
    import torch
    return a.to(torch.complex64).contiguous()


class Solver:
    """One sadmm context (Eq. 3 with Algorithm 1 on one GPU)."""

    def __init__(self, Q, M, K, N, rho, lam, stream=None, **criterion):
        self.lib = load()
        self.Q, self.M, self.K, self.N, self.KM = Q, M, K, N, K * M
        self.crit = default_criterion(**criterion)
        h = C.c_void_p()
        check(self.lib.sadmm_create(Q, M, K, N, float(rho), float(lam), C.byref(self.crit), C.byref(h)))
        self.h = h
        if stream is not None:
            check(self.lib.sadmm_set_stream(self.h, C.c_void_p(stream)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sadmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        check(self.lib.sadmm_set_stream(self.h, C.c_void_p(stream)))

    def set_criterion(self, **criterion):
        """New method knobs (defaults for those not given) for the next solves,
        keeping the operators and factors (sadmm_set_criterion)."""
        crit = default_criterion(**criterion)
        check(self.lib.sadmm_set_criterion(self.h, C.byref(crit)))
        self.crit = crit

    def set_lambda(self, lam):
        """lambda of Eq. 2 for the next solves (the factors are kept)."""
        check(self.lib.sadmm_set_lambda(self.h, float(lam)))

    def set_operator(self, q, A):
        """A: (N, KM) complex64 pixel-major, numpy (host) or torch (host/cuda)."""
        A = _as_c64(A)
        assert tuple(A.shape) == (self.N, self.KM), A.shape
        check(self.lib.sadmm_set_operator(self.h, q, _ptr(A)))

    def set_operator_delays(self, q, tau, f0, df):
        """Operator of sensor q from its round-trip delays tau (M, N) seconds:
        A[(m, k), n] = exp(j 2 pi tau[m, n] (f0 + k df)) (sadmm_set_operator_delays)."""
        if isinstance(tau, np.ndarray):
            tau = np.ascontiguousarray(tau, dtype=np.float64)
        assert tuple(tau.shape) == (self.M, self.N)
        check(self.lib.sadmm_set_operator_delays(self.h, q, _ptr(tau), float(f0), float(df)))

    def backprojection(self, y, out=None):
        """Composite BP image sum_q |A_q^H y_q| (sadmm_backprojection); y: Q arrays of KM complex64."""
        ys = [_as_c64(v) for v in y]
        arr = (C.c_void_p * self.Q)(*[_ptr(v) for v in ys])
        if out is None:
            out = np.empty(self.N, dtype=np.float32)
        check(self.lib.sadmm_backprojection(self.h, arr, _ptr(out)))
        return out

    def set_products(self, mode):
        """0 auto (factored tables when every sensor has delays), 1 stored operator, 2 factored."""
        check(self.lib.sadmm_set_products(self.h, int(mode)))

    def prepare(self):
        check(self.lib.sadmm_prepare(self.h))

    def solve(self, y, iters, tol=0.0, out=None):
        """y: Q arrays of KM complex64 (host or device).  Returns (x_G, stats);
        x_G is written to `out` if given (numpy or torch), else a new numpy array."""
        ys = [_as_c64(v) for v in y]
        arr = (C.c_void_p * self.Q)(*[_ptr(v) for v in ys])
        if out is None:
            out = np.empty(self.N, dtype=np.float32)
        st = Stats()
        check(self.lib.sadmm_solve(self.h, arr, _ptr(out), int(iters), float(tol), C.byref(st)))
        return out, st.as_dict()

    def resume(self, iters, tol=0.0, out=None):
        if out is None:
            out = np.empty(self.N, dtype=np.float32)
        st = Stats()
        check(self.lib.sadmm_resume(self.h, _ptr(out), int(iters), float(tol), C.byref(st)))
        return out, st.as_dict()

    def xq(self, q):
        out = np.empty(self.N, dtype=np.float32)
        check(self.lib.sadmm_get_xq(self.h, q, _ptr(out)))
        return out

    def X(self):
        return np.stack([self.xq(q) for q in range(self.Q)])

    def active(self, q):
        idx = np.empty(self.N, dtype=np.int32)
        n = C.c_int()
        check(self.lib.sadmm_get_active(self.h, q, _ptr(idx), C.byref(n)))
        return idx[: n.value].copy()

    def history(self):
        n = self.lib.sadmm_history(self.h, None, 0)
        recs = (IterRecord * max(n, 1))()
        m = self.lib.sadmm_history(self.h, recs, n)
        return [{k: getattr(recs[i], k) for k, _ in IterRecord._fields_} for i in range(m)]

    PHASES = ("forward", "spd_woodbury", "adjoint_update", "adjoint_primal", "spd_update",
              "residuals", "ssc", "refresh")

    def set_profiling(self, on=True):
        check(self.lib.sadmm_set_profiling(self.h, int(on)))

    def profile(self):
        ms = (C.c_double * 8)()
        n = (C.c_longlong * 8)()
        k = self.lib.sadmm_profile(self.h, ms, n, 8)
        return {self.PHASES[i]: (ms[i], n[i]) for i in range(k)}

    def set_eliminator(self, params, H, W):
        """Proposal network for elim = 2: flat FP32 parameters (numpy or torch), or None."""
        if params is None:
            check(self.lib.sadmm_set_eliminator(self.h, None, 0, 0))
            return
        if isinstance(params, np.ndarray):
            params = np.ascontiguousarray(params, dtype=np.float32)
        check(self.lib.sadmm_set_eliminator(self.h, _ptr(params), int(H), int(W)))

    def features(self, out=None):
        """(6, N) features of the current state (numpy, or into `out`)."""
        if out is None:
            out = np.empty((6, self.N), dtype=np.float32)
        check(self.lib.sadmm_features(self.h, _ptr(out)))
        return out

    def get_state(self):
        n = C.c_size_t()
        check(self.lib.sadmm_get_state(self.h, None, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        check(self.lib.sadmm_get_state(self.h, _ptr(buf), C.byref(n)))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(self.lib.sadmm_set_state(self.h, _ptr(buf), buf.size))


class BatchSolver:
    """16 scenes sharing one geometry, iterated together (sadmm_batch_*)."""
    S = 16

    def __init__(self, Q, M, K, N, rho, lams, stream=None, **criterion):
        self.lib = load()
        self.Q, self.M, self.K, self.N, self.KM = Q, M, K, N, K * M
        lam = (C.c_double * self.S)(*[float(v) for v in lams])
        crit = default_criterion(**criterion)
        h = C.c_void_p()
        check(self.lib.sadmm_batch_create(Q, M, K, N, self.S, float(rho), lam, C.byref(crit), C.byref(h)))
        self.h = h
        if stream is not None:
            check(self.lib.sadmm_batch_set_stream(self.h, C.c_void_p(stream)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sadmm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_operator(self, q, A):
        A = _as_c64(A)
        assert tuple(A.shape) == (self.N, self.KM)
        check(self.lib.sadmm_batch_set_operator(self.h, q, _ptr(A)))

    def solve(self, y, iters, out=None):
        """y: (S, Q, KM) complex64 (numpy or torch); returns (x_G (S, N), stats)."""
        y = _as_c64(y)
        if out is None:
            out = np.empty((self.S, self.N), dtype=np.float32)
        st = Stats()
        check(self.lib.sadmm_batch_solve(self.h, _ptr(y), _ptr(out), int(iters), C.byref(st)))
        return out, st.as_dict()

    def xq(self, scene, q):
        out = np.empty(self.N, dtype=np.float32)
        check(self.lib.sadmm_batch_get_xq(self.h, scene, q, _ptr(out)))
        return out

    def tune(self, reps=5):
        """Time the candidate work splits of the two tensor-core products and keep
        the fastest (sadmm_batch_tune); returns the candidates' times and the choice."""
        t = BatchTuning()
        check(self.lib.sadmm_batch_tune(self.h, int(reps), C.byref(t)))
        return t.as_dict()


class BatchGroup:
    """Batches of different geometries iterated together, one graph branch per
    batch (sadmm_batch_group_*).  The batches stay owned by the caller."""

    def __init__(self, batches, stream=None):
        self.lib = load()
        self.batches = list(batches)
        hs = (_P * len(self.batches))(*[b.h for b in self.batches])
        h = C.c_void_p()
        check(self.lib.sadmm_batch_group_create(hs, len(self.batches), C.byref(h)))
        self.h = h
        if stream is not None:
            check(self.lib.sadmm_batch_group_set_stream(self.h, C.c_void_p(stream)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sadmm_batch_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, ys, iters, outs=None):
        """ys: one (S, Q_i, KM_i) complex64 array per batch; returns ([x_G (S, N_i)], [stats])."""
        n = len(self.batches)
        ys = [_as_c64(y) for y in ys]
        if outs is None:
            outs = [np.empty((b.S, b.N), dtype=np.float32) for b in self.batches]
        yp = (_P * n)(*[_ptr(y) for y in ys])
        xp = (_P * n)(*[_ptr(o) for o in outs])
        st = (Stats * n)()
        check(self.lib.sadmm_batch_group_solve(self.h, yp, xp, int(iters), st))
        return outs, [st[i].as_dict() for i in range(n)]


class CNN:
    """The learned elimination proposal network (sadmm_cnn_*); device tensors in and out."""

    def __init__(self, H, W, max_batch=1):
        self.lib = load()
        self.H, self.W, self.maxB = H, W, max_batch
        h = C.c_void_p()
        check(self.lib.sadmm_cnn_create(H, W, max_batch, C.byref(h)))
        self.h = h
        self.n = int(self.lib.sadmm_cnn_num_params())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sadmm_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32) if isinstance(p, np.ndarray) else p.contiguous()
        check(self.lib.sadmm_cnn_set_params(self.h, _ptr(p)))

    def params(self, rounded=False):
        out = np.empty(self.n, dtype=np.float32)
        check(self.lib.sadmm_cnn_get_params(self.h, _ptr(out), int(rounded)))
        return out

    def forward(self, x, stream=0):
        import torch
        B = x.shape[0]
        out = torch.empty((B, self.H, self.W), dtype=torch.float32, device=x.device)
        check(self.lib.sadmm_cnn_forward(self.h, _ptr(x), B, _ptr(out), C.c_void_p(stream)))
        return out

    def backward(self, x, labels, pos_weight=1.0, stream=0):
        import torch
        g = torch.empty(self.n, dtype=torch.float32, device=x.device)
        loss = C.c_double()
        check(self.lib.sadmm_cnn_backward(self.h, _ptr(x), _ptr(labels), x.shape[0], float(pos_weight), _ptr(g),
                                          C.byref(loss), C.c_void_p(stream)))
        return g, loss.value

    def adam_step(self, grad, lr, stream=0):
        check(self.lib.sadmm_cnn_adam_step(self.h, _ptr(grad), float(lr), C.c_void_p(stream)))


# ------------------------------------------------------ state blob conversion
def pack_state(Q, N, KM, Kp, k, x, xbar, zbar, s, ring, J, yprime, u=None):
    """Build a state blob (layout of sadmm_get_state) from host arrays; u: the
    consensus form's duals (Q, N), appended last."""
    hdr = np.array([0x31766174734d4453], dtype=np.uint64).tobytes() + np.array(
        [Q, N, KM, Kp, k, 0], dtype=np.int32).tobytes()
    cnt = np.array([len(j) for j in J], dtype=np.int32)
    Jpad = np.zeros((Q, N), dtype=np.int32)
    for q, j in enumerate(J):
        Jpad[q, : len(j)] = j
    parts = [hdr, np.asarray(x, np.float32).tobytes(), np.asarray(xbar, np.float32).tobytes(),
             np.asarray(zbar, np.float32).tobytes(), np.asarray(s, np.float32).tobytes(),
             np.asarray(ring, np.float32).tobytes(), cnt.tobytes(), Jpad.tobytes(),
             np.asarray(yprime, np.complex64).tobytes()]
    if u is not None:
        parts.append(np.asarray(u, np.float32).tobytes())
    return np.frombuffer(b"".join(parts), dtype=np.uint8).copy()


def unpack_state(buf, Q, N, KM, Kp):
    b = np.asarray(buf, dtype=np.uint8).tobytes()
    o = 8 + 24
    k = int(np.frombuffer(b[8:32], dtype=np.int32)[4])

    def take(n, dt):
        nonlocal o
        a = np.frombuffer(b[o:o + n * np.dtype(dt).itemsize], dtype=dt).copy()
        o += n * np.dtype(dt).itemsize
        return a
    x = take(Q * N, np.float32).reshape(Q, N)
    xbar, zbar, s = take(N, np.float32), take(N, np.float32), take(N, np.float32)
    ring = take(Kp * Q * N, np.float32).reshape(Kp, Q, N)
    cnt = take(Q, np.int32)
    Jp = take(Q * N, np.int32).reshape(Q, N)
    yp = take(Q * KM, np.complex64).reshape(Q, KM)
    return dict(k=k, x=x, xbar=xbar, zbar=zbar, s=s, ring=ring,
                J=[Jp[q, : cnt[q]].copy() for q in range(Q)], yprime=yp)


# ------------------------------------------------------------ kernel level
def forward(A, idx, v, base=None, out=None, stream=0):
    """r = base - A_idx v_idx on device tensors (see sadmm_forward)."""
    import torch
    KM = A.shape[1]
    if out is None:
        out = torch.empty(KM, dtype=torch.complex64, device=A.device)
    check(load().sadmm_forward(_ptr(A), KM, A.shape[0], _ptr(idx), int(idx.numel()), _ptr(v),
                               _ptr(base), _ptr(out), C.c_void_p(stream)))
    return out


def forward_noalloc(A, idx, v, base=None, out=None, stream=0):
    """As forward(), through the allocation-free entry point (fixed scratch)."""
    import torch
    KM = A.shape[1]
    if out is None:
        out = torch.empty(KM, dtype=torch.complex64, device=A.device)
    check(load().sadmm_forward_noalloc(_ptr(A), KM, A.shape[0], _ptr(idx), int(idx.numel()), _ptr(v),
                                       _ptr(base), _ptr(out), C.c_void_p(stream)))
    return out


def adjoint(A, idx, w, out=None, stream=0):
    import torch
    KM = A.shape[1]
    if out is None:
        out = torch.empty(int(idx.numel()), dtype=torch.float32, device=A.device)
    check(load().sadmm_adjoint(_ptr(A), KM, A.shape[0], _ptr(idx), int(idx.numel()), _ptr(w),
                               _ptr(out), C.c_void_p(stream)))
    return out


def operator_tables(tau, M, K, N, f0, df, with_entries=True, stream=0):
    """Device tables of the factored operator from delays tau (M, N) float64 on
    the device: returns (A (N, M K) complex64 or None, C (M, K/16, N), D (M, 16, N))."""
    import torch
    dev = tau.device
    A = torch.empty((N, M * K), dtype=torch.complex64, device=dev) if with_entries else None
    Ct = torch.empty((M, K // 16, N), dtype=torch.complex64, device=dev)
    Dt = torch.empty((M, 16, N), dtype=torch.complex64, device=dev)
    check(load().sadmm_operator_tables(_ptr(tau), M, K, N, float(f0), float(df), _ptr(A), _ptr(Ct), _ptr(Dt),
                                       C.c_void_p(stream)))
    return A, Ct, Dt


def forward_factored(Ct, Dt, K, idx, v, base=None, out=None, stream=0):
    """r = base - A_idx v_idx with A given by its factors (sadmm_forward_factored)."""
    import torch
    M, N = Ct.shape[0], Ct.shape[2]
    if out is None:
        out = torch.empty(M * K, dtype=torch.complex64, device=Ct.device)
    check(load().sadmm_forward_factored(_ptr(Ct), _ptr(Dt), M, K, N, _ptr(idx), int(idx.numel()), _ptr(v),
                                        _ptr(base), _ptr(out), C.c_void_p(stream)))
    return out


def adjoint_factored(Ct, Dt, K, idx, w, out=None, stream=0):
    """g = Re(A_idx^H w) with A given by its factors (sadmm_adjoint_factored)."""
    import torch
    M, N = Ct.shape[0], Ct.shape[2]
    if out is None:
        out = torch.empty(int(idx.numel()), dtype=torch.float32, device=Ct.device)
    check(load().sadmm_adjoint_factored(_ptr(Ct), _ptr(Dt), M, K, N, _ptr(idx), int(idx.numel()), _ptr(w),
                                        _ptr(out), C.c_void_p(stream)))
    return out


def factor(A, idx, mu, rho, stream=0):
    """Returns (F, form, n): F the padded FP64 factor as a torch tensor."""
    import torch
    KM = A.shape[1]
    nidx = int(idx.numel())
    n = 2 * KM if nidx > 2 * KM else nidx
    npad = (n + 63) // 64 * 64
    F = torch.empty((npad, npad), dtype=torch.float64, device=A.device)
    form = C.c_int()
    check(load().sadmm_factor(_ptr(A), KM, A.shape[0], _ptr(idx), nidx, float(mu), float(rho),
                              _ptr(F), npad, C.byref(form), C.c_void_p(stream)))
    return F, form.value, n


def adjoint16_tc(A, W, stream=0):
    """G (N x 16 float) = Re(A^H W) on the tensor cores; A (N, KM) complex64, W (KM, 16) complex64."""
    import torch
    N, KM = A.shape
    G = torch.empty((N, 16), dtype=torch.float32, device=A.device)
    check(load().sadmm_adjoint16_tc(_ptr(A), KM, N, _ptr(W), _ptr(G), C.c_void_p(stream)))
    return G


def factor_update(A, E, mu, sign, W, stream=0):
    """In place: W <- factor with the columns E removed (sign +1) or added (sign -1)."""
    KM = A.shape[1]
    check(load().sadmm_factor_update(_ptr(A), KM, _ptr(E), int(E.numel()), float(mu), int(sign), _ptr(W),
                                     C.c_void_p(stream)))
    return W


def factor_downdate(A, E, mu, W, stream=0):
    """In place: W <- factor of the active set without the columns E (Woodbury form)."""
    KM = A.shape[1]
    check(load().sadmm_factor_downdate(_ptr(A), KM, _ptr(E), int(E.numel()), float(mu), _ptr(W),
                                       C.c_void_p(stream)))
    return W


BF16, FP16 = 1, 2


def split_operator(A, kind, stream=0):
    """(hi, lo) int16 tensors holding the 16-bit planes of the complex64 operator A."""
    import torch
    hi = torch.empty(A.shape + (2,), dtype=torch.int16, device=A.device)
    lo = torch.empty_like(hi)
    check(load().sadmm_split_operator(_ptr(A), A.numel(), int(kind), _ptr(hi), _ptr(lo), C.c_void_p(stream)))
    return hi, lo


def forward_split(hi, lo, kind, planes, idx, v, base=None, stream=0):
    import torch
    N, KM = hi.shape[0], hi.shape[1]
    out = torch.empty(KM, dtype=torch.complex64, device=hi.device)
    check(load().sadmm_forward_split(_ptr(hi), _ptr(lo), int(kind), int(planes), KM, N, _ptr(idx),
                                     int(idx.numel()), _ptr(v), _ptr(base), _ptr(out), C.c_void_p(stream)))
    return out


def adjoint_split(hi, lo, kind, planes, idx, w, stream=0):
    import torch
    N, KM = hi.shape[0], hi.shape[1]
    out = torch.empty(int(idx.numel()), dtype=torch.float32, device=hi.device)
    check(load().sadmm_adjoint_split(_ptr(hi), _ptr(lo), int(kind), int(planes), KM, N, _ptr(idx),
                                     int(idx.numel()), _ptr(w), _ptr(out), C.c_void_p(stream)))
    return out


def spd_apply(F, n, u, out=None, stream=0):
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=F.device)
    check(load().sadmm_spd_apply(_ptr(F), n, F.shape[1], _ptr(u), _ptr(out), C.c_void_p(stream)))
    return out


def set_wait_limit(polls):
    """Polls of the factor apply's tile-copy wait before it reports
    SADMM_ETIMEOUT (failure-handling tests); polls < 0 restores the default."""
    check(load().sadmm_set_wait_limit(int(polls)))


def gram(A, idx, mu, rho, method=0, stream=0):
    """(F, form, n): F = mu G + rho I of the x-update system for the active
    columns idx of the pixel-major complex64 operator A (device tensors); the
    tensor-core digit method (0) or FP64 SIMT (1)."""
    import torch
    N, KM = A.shape
    nidx = int(idx.numel())
    n = 2 * KM if nidx > 2 * KM else nidx
    npad = (n + 63) // 64 * 64
    F = torch.empty((npad, npad), dtype=torch.float64, device=A.device)
    form = C.c_int(0)
    check(load().sadmm_gram(_ptr(A), KM, N, _ptr(idx), nidx, float(mu), float(rho), int(method), _ptr(F), npad,
                            C.byref(form), C.c_void_p(stream)))
    return F, form.value, n


def digit_apply16(F, U, stream=0):
    """F[:n, :n] @ U (n x 16) on the tensor cores through exact BF16 digit
    slices (the batched form's factor apply): F float64 (n x ld, row-major),
    U float32 (n x 16), device tensors; returns the float64 product (n x 16)."""
    import torch
    n = int(U.shape[0])
    if U.shape != (n, 16) or U.dtype != torch.float32 or F.dtype != torch.float64 or F.shape[0] < n:
        raise ValueError("digit_apply16: F float64 (n x ld), U float32 (n x 16)")
    F = F.contiguous()
    U = U.contiguous()
    out = torch.empty((n, 16), dtype=torch.float64, device=U.device)
    check(load().sadmm_digit_apply16(_ptr(F), int(F.shape[1]), n, _ptr(U), _ptr(out), C.c_void_p(stream)))
    return out


def forward16_tc(A, V, stream=0):
    """R = A^T V (KM x 16 complex64) for the pixel-major complex64 operator A
    (N x KM) and 16 real right-hand sides V (N x 16 float32), device tensors:
    the batched forward product on the tensor cores (3xTF32)."""
    import torch
    N, KM = A.shape
    if V.shape != (N, 16) or V.dtype != torch.float32 or A.dtype != torch.complex64:
        raise ValueError("forward16_tc: A complex64 (N x KM), V float32 (N x 16)")
    R = torch.empty((KM, 16), dtype=torch.complex64, device=A.device)
    check(load().sadmm_forward16_tc(_ptr(A.contiguous()), KM, N, _ptr(V.contiguous()), _ptr(R), C.c_void_p(stream)))
    return R
