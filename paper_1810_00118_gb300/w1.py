"""Thin ctypes binding of libw1.so (include/w1.h): argument marshalling only.

Every step of the solver runs in the library's sm_103a kernels.  Tensors are
torch CUDA float32, C-contiguous, shaped [ny, nx] (a flux is [2, ny, nx]);
streams are torch.cuda streams (default: the current stream).  There is no CPU
fallback: if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

from . import _build

NORM_L1 = 1
NORM_L2 = 2
NORM_LINF = 3
MAX_LEVELS = 16

OK = 0
ERR_INVALID_ARG = 1
ERR_SHAPE = 2
ERR_MASS = 3
ERR_NOMEM = 4
ERR_CUDA = 5
ERR_NOT_CONVERGED = 6
ERR_TIMEOUT = 7
PENDING = 8
ERR_BUDGET = 9
ERR_UNSUPPORTED = 10

_STATUS_NAMES = {
    OK: "OK", ERR_INVALID_ARG: "ERR_INVALID_ARG", ERR_SHAPE: "ERR_SHAPE", ERR_MASS: "ERR_MASS",
    ERR_NOMEM: "ERR_NOMEM", ERR_CUDA: "ERR_CUDA", ERR_NOT_CONVERGED: "ERR_NOT_CONVERGED",
    ERR_TIMEOUT: "ERR_TIMEOUT", PENDING: "PENDING", ERR_BUDGET: "ERR_BUDGET", ERR_UNSUPPORTED: "ERR_UNSUPPORTED",
}


class W1Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("check_every", ctypes.c_int), ("max_iters", ctypes.c_longlong), ("theta", ctypes.c_double),
                ("alpha", ctypes.c_double), ("time_budget_s", ctypes.c_double), ("path", ctypes.c_int),
                ("rows_per_thread", ctypes.c_int), ("eager", ctypes.c_int), ("tune", ctypes.c_int),
                ("algorithm", ctypes.c_int), ("tile", ctypes.c_int), ("step_ratio", ctypes.c_double),
                ("schedule", ctypes.c_int), ("estimate", ctypes.c_int)]


class LevelChoice(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("cluster", ctypes.c_int), ("batch", ctypes.c_int),
                ("us_per_step", ctypes.c_double), ("concurrent", ctypes.c_int), ("tile", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("opt", Options), ("latency_below", ctypes.c_int)]


class ServerInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in ("submitted", "completed", "rejected", "queued", "in_flight",
                                                  "slots", "evictions")] + [("bytes_in_use", ctypes.c_size_t)]


class _Stats(ctypes.Structure):
    L = MAX_LEVELS
    _fields_ = [("levels", ctypes.c_int), ("nx", ctypes.c_int * L), ("ny", ctypes.c_int * L),
                ("iters", ctypes.c_longlong * L), ("fpr", ctypes.c_double * L), ("tol", ctypes.c_double * L),
                ("path", ctypes.c_int * L), ("cluster", ctypes.c_int * L),
                ("w1", ctypes.c_double), ("dual", ctypes.c_double), ("lb", ctypes.c_double),
                ("ub", ctypes.c_double), ("route", ctypes.c_double), ("res_l1", ctypes.c_double),
                ("rho_l1", ctypes.c_double), ("gmax", ctypes.c_double), ("mass0", ctypes.c_double),
                ("mass1", ctypes.c_double), ("mass_shift", ctypes.c_double), ("converged", ctypes.c_int),
                ("primal", ctypes.c_double), ("saddle", ctypes.c_double)]


@dataclass
class Stats:
    levels: int = 0
    sizes: list = field(default_factory=list)
    iters: list = field(default_factory=list)
    fpr: list = field(default_factory=list)
    tol: list = field(default_factory=list)
    path: list = field(default_factory=list)
    cluster: list = field(default_factory=list)
    w1: float = 0.0
    dual: float = 0.0
    lb: float = 0.0
    ub: float = 0.0
    route: float = 0.0
    res_l1: float = 0.0
    rho_l1: float = 0.0
    gmax: float = 0.0
    mass0: float = 0.0
    mass1: float = 0.0
    mass_shift: float = 0.0
    converged: bool = False
    primal: float = 0.0
    saddle: float = 0.0

    @staticmethod
    def _from(s: _Stats) -> "Stats":
        L = s.levels
        return Stats(L, [(s.nx[k], s.ny[k]) for k in range(L)], [s.iters[k] for k in range(L)],
                     [s.fpr[k] for k in range(L)], [s.tol[k] for k in range(L)], [s.path[k] for k in range(L)],
                     [s.cluster[k] for k in range(L)], s.w1, s.dual, s.lb, s.ub, s.route, s.res_l1, s.rho_l1,
                     s.gmax, s.mass0, s.mass1, s.mass_shift, bool(s.converged), s.primal, s.saddle)


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path) or _build._stale():
        _build.build()
    lib = ctypes.CDLL(path)
    P, I, D, LL, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_float
    st = ctypes.c_int
    sig = {
        "w1_default_options": (None, [ctypes.POINTER(Options)]),
        "w1_calibrated_schedule": (st, [I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                        ctypes.POINTER(D)]),
        "w1_plan_create": (st, [I, I, D, I, I, D, ctypes.POINTER(P)]),
        "w1_plan_create_ex": (st, [I, I, D, I, I, D, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "w1_plan_create_batch": (st, [I, I, D, I, I, D, I, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "w1_plan_max_batch": (I, [P]),
        "w1_solve_batch": (st, [P, I, P, P, P, P, P, P, P]),
        "w1_solve_batch_host": (st, [P, I, P, P, P, P, P, P, P]),
        "w1_solve_async": (st, [P, I, P, P, P, P]),
        "w1_plan_results": (st, [P, P, P, P]),
        "w1_plan_destroy": (st, [P]),
        "w1_plan_workspace_bytes": (ctypes.c_size_t, [P]),
        "w1_plan_set_workspace": (st, [P, P, ctypes.c_size_t]),
        "w1_solve": (st, [P, P, P, P, ctypes.POINTER(D), P, ctypes.POINTER(_Stats)]),
        "w1_solve_host": (st, [P, P, P, P, ctypes.POINTER(D), P, ctypes.POINTER(_Stats)]),
        "w1_plan_potential": (st, [P, P, P]),
        "w1_cp_steps": (st, [I, I, D, I, F, F, P, P, P, P, LL, I, P, ctypes.POINTER(D)]),
        "w1_cp_steps_ex": (st, [I, I, D, I, F, F, P, P, P, P, LL, I, I, P, ctypes.POINTER(D)]),
        "w1_poisson": (st, [I, I, D, P, P, P]),
        "w1_pdhg_steps": (st, [I, I, D, I, F, F, P, P, P, P, P, P, P, LL, P, ctypes.POINTER(D)]),
        "w1_mixed_create": (st, [I, P, P, P, I, D, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "w1_mixed_destroy": (st, [P]),
        "w1_mixed_persistent": (I, [P, I]),
        "w1_mixed_launch_info": (st, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "w1_mixed_solve_async": (st, [P, P, P, P]),
        "w1_mixed_results": (st, [P, I, P, P, P]),
        "w1_restrict": (st, [I, I, P, P, P]),
        "w1_prolong": (st, [I, I, P, P, P, P, P, P, P]),
        "w1_state_stats": (st, [I, I, D, I, P, P, P, P, P, ctypes.POINTER(_Stats)]),
        "w1_state_stats_noalloc": (st, [I, I, D, I, P, P, P, P, P, ctypes.POINTER(_Stats)]),
        "w1_noalloc_last_error": (ctypes.c_char_p, []),
        "w1_solve3d": (st, [I, I, I, D, I, I, D, ctypes.POINTER(Options), P, P, P, ctypes.POINTER(D), P, P,
                            ctypes.POINTER(_Stats)]),
        "w1_cp_steps3d": (st, [I, I, I, D, I, F, F, P, P, P, P, P, LL, P, ctypes.POINTER(D)]),
        "w1_cp_steps3d_ex": (st, [I, I, I, D, I, F, F, P, P, P, P, P, LL, I, I, P, ctypes.POINTER(D)]),
        "w1_restrict3d": (st, [I, I, I, P, P, P]),
        "w1_prolong3d": (st, [I, I, I, P, P, P, P, P, P, P, P, P]),
        "w1_3d_last_error": (ctypes.c_char_p, []),
        "w1_3d_release_workspace": (None, []),
        "w1_plan_bytes": (ctypes.c_size_t, [I, I, D, I, I, D, I, ctypes.POINTER(Options)]),
        "w1_autotune_level": (st, [I, I, I, I, I, I, ctypes.POINTER(LevelChoice), ctypes.POINTER(LevelChoice),
                                   ctypes.POINTER(I)]),
        "w1_autotune_last_error": (ctypes.c_char_p, []),
        "w1_server_default_config": (None, [ctypes.POINTER(ServerConfig)]),
        "w1_server_create_ex": (st, [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]),
        "w1_server_create": (st, [ctypes.c_size_t, I, ctypes.POINTER(P)]),
        "w1_submit": (st, [P, I, I, D, I, I, D, P, P, ctypes.POINTER(ctypes.c_uint64)]),
        "w1_poll": (st, [P, ctypes.c_uint64, ctypes.POINTER(D), ctypes.POINTER(_Stats)]),
        "w1_poll_latency": (st, [P, ctypes.c_uint64, ctypes.POINTER(D), ctypes.POINTER(_Stats), ctypes.POINTER(D)]),
        "w1_wait": (st, [P, ctypes.c_uint64, D, ctypes.POINTER(D), ctypes.POINTER(_Stats)]),
        "w1_server_query": (st, [P, ctypes.POINTER(ServerInfo)]),
        "w1_server_destroy": (st, [P]),
        "w1_server_last_error": (ctypes.c_char_p, []),
        "w1_status_string": (ctypes.c_char_p, [st]),
        "w1_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _check(status: int, ok=(OK,)):
    if status not in ok:
        raise W1Error(status, _lib.w1_last_error().decode())
    return status


def default_options(**kw) -> Options:
    o = Options()
    _lib.w1_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def calibrated_schedule(norm) -> tuple:
    """(eps_L scale, alpha, theta, step ratio) of w1_options.schedule = 1 for a norm (host only)."""
    a, b, c, r = (ctypes.c_double(0.0) for _ in range(4))
    _check(_lib.w1_calibrated_schedule(norm, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(r)))
    return a.value, b.value, c.value, r.value


def _dev_ptr(t, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A solver plan for batches of up to `batch` nx x ny pairs (w1_plan_create_batch)."""

    def __init__(self, nx, ny, h=0.0, levels=0, norm=NORM_L1, tol=0.0, batch=1, **options):
        self._p = ctypes.c_void_p()
        self.nx, self.ny, self.batch = nx, ny, batch
        opt = default_options(**options)
        _check(_lib.w1_plan_create_batch(nx, ny, h, levels, norm, tol, batch, ctypes.byref(opt),
                                         ctypes.byref(self._p)))

    def close(self):
        if self._p:
            _lib.w1_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def workspace_bytes(self) -> int:
        return _lib.w1_plan_workspace_bytes(self._p)

    def set_workspace(self, tensor):
        _check(_lib.w1_plan_set_workspace(self._p, ctypes.c_void_p(tensor.data_ptr()),
                                          tensor.numel() * tensor.element_size()))

    def solve(self, rho0, rho1, flux=None, stream=None, allow=(OK,)):
        """Returns (W1 estimate, Stats, status).  Raises on statuses not in `allow`."""
        shape = (self.ny, self.nx)
        d = ctypes.c_double(0.0)
        s = _Stats()
        fp = _dev_ptr(flux, (2,) + shape) if flux is not None else None
        status = _lib.w1_solve(self._p, _dev_ptr(rho0, shape), _dev_ptr(rho1, shape), _stream_ptr(stream),
                               ctypes.byref(d), fp, ctypes.byref(s))
        _check(status, allow)
        return d.value, Stats._from(s), status

    def solve_host(self, rho0, rho1, flux=None, stream=None, allow=(OK,)):
        """Densities and flux as C-contiguous float32 numpy arrays (host memory)."""
        import numpy as np
        shape = (self.ny, self.nx)
        for a in (rho0, rho1):
            if a.dtype != np.float32 or a.shape != shape or not a.flags.c_contiguous:
                raise TypeError("expected C-contiguous float32 arrays of shape (ny, nx)")
        d = ctypes.c_double(0.0)
        s = _Stats()
        fp = None
        if flux is not None:
            if flux.dtype != np.float32 or flux.shape != (2,) + shape or not flux.flags.c_contiguous:
                raise TypeError("flux must be a C-contiguous float32 array of shape (2, ny, nx)")
            fp = ctypes.c_void_p(flux.ctypes.data)
        status = _lib.w1_solve_host(self._p, ctypes.c_void_p(rho0.ctypes.data), ctypes.c_void_p(rho1.ctypes.data),
                                    _stream_ptr(stream), ctypes.byref(d), fp, ctypes.byref(s))
        _check(status, allow)
        return d.value, Stats._from(s), status

    def solve_batch(self, rho0, rho1, flux=None, stream=None, allow=(OK,)):
        """rho0, rho1: [b, ny, nx] device tensors (b <= batch).  Returns
        (list of W1, list of Stats, list of per-pair statuses, status)."""
        b = rho0.shape[0]
        shape = (b, self.ny, self.nx)
        d = (ctypes.c_double * b)()
        s = (_Stats * b)()
        ps = (ctypes.c_int * b)()
        fp = _dev_ptr(flux, (b, 2, self.ny, self.nx)) if flux is not None else None
        status = _lib.w1_solve_batch(self._p, b, _dev_ptr(rho0, shape), _dev_ptr(rho1, shape), _stream_ptr(stream),
                                     ctypes.cast(d, ctypes.c_void_p), fp, ctypes.cast(s, ctypes.c_void_p),
                                     ctypes.cast(ps, ctypes.c_void_p))
        _check(status, allow)
        return list(d), [Stats._from(x) for x in s], list(ps), status

    def solve_batch_host(self, rho0, rho1, flux=None, stream=None, allow=(OK,)):
        """Host float32 arrays [b, ny, nx] (and flux [b, 2, ny, nx])."""
        import numpy as np
        b = rho0.shape[0]
        for a in (rho0, rho1):
            if a.dtype != np.float32 or a.shape != (b, self.ny, self.nx) or not a.flags.c_contiguous:
                raise TypeError("expected C-contiguous float32 arrays of shape (b, ny, nx)")
        d = (ctypes.c_double * b)()
        s = (_Stats * b)()
        ps = (ctypes.c_int * b)()
        fp = None
        if flux is not None:
            if flux.dtype != np.float32 or flux.shape != (b, 2, self.ny, self.nx) or not flux.flags.c_contiguous:
                raise TypeError("flux must be a C-contiguous float32 array of shape (b, 2, ny, nx)")
            fp = ctypes.c_void_p(flux.ctypes.data)
        status = _lib.w1_solve_batch_host(self._p, b, ctypes.c_void_p(rho0.ctypes.data),
                                          ctypes.c_void_p(rho1.ctypes.data), _stream_ptr(stream),
                                          ctypes.cast(d, ctypes.c_void_p), fp, ctypes.cast(s, ctypes.c_void_p),
                                          ctypes.cast(ps, ctypes.c_void_p))
        _check(status, allow)
        return list(d), [Stats._from(x) for x in s], list(ps), status

    def solve_async(self, rho0, rho1, flux=None, stream=None):
        """Enqueue a solve of rho0, rho1 ([ny, nx] or [b, ny, nx] device tensors)
        on `stream` without waiting; read it with results() once the stream is done."""
        b = 1 if rho0.dim() == 2 else rho0.shape[0]
        shape = tuple(rho0.shape)
        fshape = (2, self.ny, self.nx) if rho0.dim() == 2 else (b, 2, self.ny, self.nx)
        fp = _dev_ptr(flux, fshape) if flux is not None else None
        _check(_lib.w1_solve_async(self._p, b, _dev_ptr(rho0, shape), _dev_ptr(rho1, shape), _stream_ptr(stream), fp))
        self._pending = b

    def results(self, allow=(OK, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_MASS)):
        """(list of W1, list of Stats, list of statuses, status) of the last solve_async."""
        b = getattr(self, "_pending", 1)
        d = (ctypes.c_double * b)()
        s = (_Stats * b)()
        ps = (ctypes.c_int * b)()
        status = _lib.w1_plan_results(self._p, ctypes.cast(d, ctypes.c_void_p), ctypes.cast(s, ctypes.c_void_p),
                                      ctypes.cast(ps, ctypes.c_void_p))
        _check(status, allow)
        return list(d), [Stats._from(x) for x in s], list(ps), status

    def potential(self, out, stream=None):
        shape = (self.ny, self.nx) if out.dim() == 2 else (out.shape[0], self.ny, self.nx)
        _check(_lib.w1_plan_potential(self._p, _dev_ptr(out, shape), _stream_ptr(stream)))
        return out


class Mixed:
    """A batch of pairs of several grid sizes (w1_mixed_*).  classes: list of
    (nx, ny, count).  Classes whose levels fit one CTA run in one persistent
    launch; the others as batched plans overlapping it."""

    def __init__(self, classes, norm=NORM_L1, tol=0.0, **options):
        self.classes = [tuple(int(v) for v in c) for c in classes]
        n = len(self.classes)
        arr = lambda k: (ctypes.c_int * n)(*[c[k] for c in self.classes])  # noqa: E731
        self._nx, self._ny, self._cnt = arr(0), arr(1), arr(2)
        opt = default_options(**options)
        p = ctypes.c_void_p()
        _check(_lib.w1_mixed_create(n, ctypes.cast(self._nx, ctypes.c_void_p), ctypes.cast(self._ny, ctypes.c_void_p),
                                    ctypes.cast(self._cnt, ctypes.c_void_p), norm, tol, ctypes.byref(opt),
                                    ctypes.byref(p)))
        self._p = p

    def persistent(self, cls) -> bool:
        return _lib.w1_mixed_persistent(self._p, cls) == 1

    def launch_info(self) -> dict:
        """CTAs of the single-CTA persistent launch, clusters of the cluster
        launch and CTAs of the coarse launch (0 where unused)."""
        a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib.w1_mixed_launch_info(self._p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"ctas": a.value, "clusters": b.value, "coarse_ctas": c.value}

    def solve_async(self, rho0, rho1, stream=None):
        """rho0, rho1: lists (one per class) of device tensors [count, ny, nx]."""
        n = len(self.classes)
        if len(rho0) != n or len(rho1) != n:
            raise ValueError(f"expected {n} tensors per density")
        p0 = (ctypes.c_void_p * n)(*[_dev_ptr(t, (c[2], c[1], c[0])).value for t, c in zip(rho0, self.classes)])
        p1 = (ctypes.c_void_p * n)(*[_dev_ptr(t, (c[2], c[1], c[0])).value for t, c in zip(rho1, self.classes)])
        self._keep = (rho0, rho1)
        _check(_lib.w1_mixed_solve_async(self._p, ctypes.cast(p0, ctypes.c_void_p), ctypes.cast(p1, ctypes.c_void_p),
                                         _stream_ptr(stream)))

    def results(self, cls, allow=(OK, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_MASS)):
        """(list of W1, list of Stats, list of statuses, status) of class cls."""
        b = self.classes[cls][2]
        d = (ctypes.c_double * b)()
        s = (_Stats * b)()
        ps = (ctypes.c_int * b)()
        status = _lib.w1_mixed_results(self._p, cls, ctypes.cast(d, ctypes.c_void_p), ctypes.cast(s, ctypes.c_void_p),
                                       ctypes.cast(ps, ctypes.c_void_p))
        _check(status, allow)
        return list(d), [Stats._from(x) for x in s], list(ps), status

    def close(self):
        if getattr(self, "_p", None):
            _lib.w1_mixed_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cp_steps(rho, m1, m2, phi, h, norm, mu, tau, iters, path=2, stream=None, cluster=0) -> float:
    """`iters` steps of eq. primaldual in place on device state; returns R^k of the
    last step.  cluster: CTAs of the resident path (0: the library's choice)."""
    ny, nx = rho.shape
    f = ctypes.c_double(0.0)
    _check(_lib.w1_cp_steps_ex(nx, ny, h, norm, mu, tau, _dev_ptr(rho), _dev_ptr(m1, rho.shape),
                               _dev_ptr(m2, rho.shape), _dev_ptr(phi, rho.shape), int(iters), path, int(cluster),
                               _stream_ptr(stream), ctypes.byref(f)))
    return f.value


def poisson(r, psi, h, stream=None):
    """psi with -div grad psi = r - mean(r), mean(psi) = 0 (device tensors [ny, nx])."""
    ny, nx = r.shape
    _check(_lib.w1_poisson(nx, ny, h, _dev_ptr(r), _dev_ptr(psi, r.shape), _stream_ptr(stream)))
    return psi


def pdhg_steps(rho, m1, m2, phi1, phi2, phibar1, phibar2, h, norm, iters, mu=0.5, tau=0.5, stream=None) -> float:
    """`iters` steps of eq. pdhg in place on device state; returns G^k of the last step."""
    ny, nx = rho.shape
    g = ctypes.c_double(0.0)
    ptrs = [_dev_ptr(t, rho.shape) for t in (m1, m2, phi1, phi2, phibar1, phibar2)]
    _check(_lib.w1_pdhg_steps(nx, ny, h, norm, mu, tau, _dev_ptr(rho), *ptrs, int(iters), _stream_ptr(stream),
                              ctypes.byref(g)))
    return g.value


def restrict(fine, out, stream=None):
    ny, nx = fine.shape
    _check(_lib.w1_restrict(nx, ny, _dev_ptr(fine), _dev_ptr(out, (ny // 2, nx // 2)), _stream_ptr(stream)))
    return out


def prolong(m1c, m2c, phic, m1f, m2f, phif, stream=None):
    ncy, ncx = phic.shape
    fs = (2 * ncy, 2 * ncx)
    _check(_lib.w1_prolong(ncx, ncy, _dev_ptr(m1c, phic.shape), _dev_ptr(m2c, phic.shape), _dev_ptr(phic),
                           _dev_ptr(m1f, fs), _dev_ptr(m2f, fs), _dev_ptr(phif, fs), _stream_ptr(stream)))


def state_stats(rho, m1, m2, phi, h, norm, stream=None) -> Stats:
    ny, nx = rho.shape
    s = _Stats()
    _check(_lib.w1_state_stats(nx, ny, h, norm, _dev_ptr(rho), _dev_ptr(m1, rho.shape), _dev_ptr(m2, rho.shape),
                               _dev_ptr(phi, rho.shape), _stream_ptr(stream), ctypes.byref(s)))
    return Stats._from(s)


def _check3(status: int, ok=(OK,)):
    if status not in ok:
        raise W1Error(status, _lib.w1_3d_last_error().decode())
    return status


def solve3d(rho0, rho1, norm=NORM_L1, h=0.0, levels=0, tol=0.0, flux=None, potential=None, stream=None,
            **options):
    """Algorithm 3 on a 3-D grid (w1_solve3d).  rho0, rho1: [nz, ny, nx] device
    tensors; flux ([3, nz, ny, nx]) and potential ([nz, ny, nx]) receive the finest
    state when given.  Returns (W1, Stats, status); NOT_CONVERGED and TIMEOUT are
    returned, other errors raise."""
    nz, ny, nx = rho0.shape
    opt = default_options(**options)
    d = ctypes.c_double(0.0)
    s = _Stats()
    st = _lib.w1_solve3d(nx, ny, nz, h, levels, norm, tol, ctypes.byref(opt), _dev_ptr(rho0),
                         _dev_ptr(rho1, rho0.shape), _stream_ptr(stream), ctypes.byref(d),
                         _dev_ptr(flux, (3, nz, ny, nx)) if flux is not None else None,
                         _dev_ptr(potential, rho0.shape) if potential is not None else None, ctypes.byref(s))
    _check3(st, ok=(OK, ERR_NOT_CONVERGED, ERR_TIMEOUT))
    return d.value, Stats._from(s), st


def release_workspace3d():
    """Frees the device workspace w1_solve3d keeps between calls."""
    _lib.w1_3d_release_workspace()


def cp_steps3d(rho, m1, m2, m3, phi, h, norm, mu, tau, iters, path=2, cluster=0, stream=None) -> float:
    """`iters` steps of eq. primaldual on a 3-D level, in place; returns R^k of the
    last step.  path 2: two launches per step; 3: one launch per step; 1: on chip
    (cluster CTAs, 0: auto)."""
    nz, ny, nx = rho.shape
    f = ctypes.c_double(0.0)
    _check3(_lib.w1_cp_steps3d_ex(nx, ny, nz, h, norm, mu, tau, _dev_ptr(rho),
                                  *(_dev_ptr(t, rho.shape) for t in (m1, m2, m3, phi)), int(iters), int(path),
                                  int(cluster), _stream_ptr(stream), ctypes.byref(f)))
    return f.value


def restrict3d(fine, out, stream=None):
    nz, ny, nx = fine.shape
    _check3(_lib.w1_restrict3d(nx, ny, nz, _dev_ptr(fine), _dev_ptr(out, (nz // 2, ny // 2, nx // 2)),
                               _stream_ptr(stream)))
    return out


def prolong3d(m1c, m2c, m3c, phic, m1f, m2f, m3f, phif, stream=None):
    ncz, ncy, ncx = phic.shape
    fs = (2 * ncz, 2 * ncy, 2 * ncx)
    _check3(_lib.w1_prolong3d(ncx, ncy, ncz, *(_dev_ptr(t, phic.shape) for t in (m1c, m2c, m3c, phic)),
                              *(_dev_ptr(t, fs) for t in (m1f, m2f, m3f, phif)), _stream_ptr(stream)))


def status_string(status: int) -> str:
    return _lib.w1_status_string(status).decode()


def plan_bytes(nx, ny, h=0.0, levels=0, norm=NORM_L1, tol=0.0, batch=1, **options) -> int:
    opt = default_options(**options)
    return _lib.w1_plan_bytes(nx, ny, h, levels, norm, tol, batch, ctypes.byref(opt))


class Server:
    """Continuous-batching request loop (w1_server_create_ex)."""

    def __init__(self, hbm_budget_bytes=40 << 30, max_slots=32, max_batch=1, latency_below=0, **options):
        cfg = ServerConfig()
        _lib.w1_server_default_config(ctypes.byref(cfg))
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_slots = max_slots
        cfg.max_batch = max_batch
        cfg.latency_below = latency_below
        for k, v in options.items():
            setattr(cfg.opt, k, v)
        self._s = ctypes.c_void_p()
        st = _lib.w1_server_create_ex(ctypes.byref(cfg), ctypes.byref(self._s))
        if st != OK:
            raise W1Error(st, _lib.w1_server_last_error().decode())

    def submit(self, rho0, rho1, norm=NORM_L1, levels=0, tol=0.0, h=0.0) -> int:
        """Queue one pair ([ny, nx] device tensors, kept alive by the caller until done)."""
        ny, nx = rho0.shape
        t = ctypes.c_uint64(0)
        st = _lib.w1_submit(self._s, nx, ny, h, levels, norm, tol, _dev_ptr(rho0), _dev_ptr(rho1, (ny, nx)),
                            ctypes.byref(t))
        if st != OK:
            raise W1Error(st, _lib.w1_server_last_error().decode())
        return t.value

    def poll(self, ticket):
        """(status, W1, Stats, server latency in s); status PENDING while not finished."""
        d, lat = ctypes.c_double(0.0), ctypes.c_double(0.0)
        s = _Stats()
        st = _lib.w1_poll_latency(self._s, ticket, ctypes.byref(d), ctypes.byref(s), ctypes.byref(lat))
        if st == PENDING:
            return st, None, None, None
        return st, d.value, Stats._from(s), lat.value

    def wait(self, ticket, timeout_s=0.0):
        d = ctypes.c_double(0.0)
        s = _Stats()
        st = _lib.w1_wait(self._s, ticket, timeout_s, ctypes.byref(d), ctypes.byref(s))
        return st, d.value, Stats._from(s)

    def info(self) -> dict:
        i = ServerInfo()
        _lib.w1_server_query(self._s, ctypes.byref(i))
        return {n: getattr(i, n) for n, _ in ServerInfo._fields_}

    def close(self):
        if self._s:
            _lib.w1_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def autotune_level(nx, ny, norm=NORM_L1, objective=2, steps=256, batch=1):
    """(best, all candidates) as dicts: path, cluster, batch, us_per_step (one
    step of the whole batch; objective 1 times one pair alone), concurrent,
    tile (path 3: the tile variant, 0-based)."""
    best = LevelChoice()
    allc = (LevelChoice * 16)()  # W1_TUNE_MAX_CANDIDATES
    n = ctypes.c_int(0)
    st = _lib.w1_autotune_level(nx, ny, norm, batch, objective, steps, ctypes.byref(best), allc, ctypes.byref(n))
    if st != OK:
        raise W1Error(st, _lib.w1_autotune_last_error().decode())
    conv = lambda c: {f: getattr(c, f) for f, _ in LevelChoice._fields_}  # noqa: E731
    return conv(best), [conv(allc[k]) for k in range(n.value)]
