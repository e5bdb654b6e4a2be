"""FP64 CPU oracle for the multilevel primal-dual W1 solver (arXiv 1810.00118).

TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  The product path (``paper_1810_00118_gb300``) never does.

The arithmetic lives in ``w1_oracle.c`` (plain C loops, FP64, single thread);
this module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Every array is FP64, C-contiguous, shaped ``[ny, nx]`` (row j, column
i), matching the paper's grid of Sec. 2.2 restated on pixel centres.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "w1_oracle.c")
_SRC3 = os.path.join(_HERE, "w1_oracle3.c")
_LIB = os.path.join(_HERE, "libw1_oracle.so")
_lock = threading.Lock()
_lib = None

NORM_L1 = 1
NORM_L2 = 2
NORM_LINF = 3
STOP_GAP = 0
STOP_FPR = 1

OK = 0
NOT_CONVERGED = 1
ERR_ARG = -1
ERR_SHAPE = -2
ERR_MASS = -3
ERR_NOMEM = -4


class _Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in
                ("f", "dual", "res_l1", "rho_l1", "gmax", "lb", "route", "ub", "fpr", "saddle")]


@dataclass
class Stats:
    """Statistics of one state, see ``w1o_stats_t`` in w1_oracle.c."""
    f: float
    dual: float
    res_l1: float
    rho_l1: float
    gmax: float
    lb: float
    route: float
    ub: float
    fpr: float
    saddle: float

    @staticmethod
    def _from(s: _Stats) -> "Stats":
        return Stats(*(getattr(s, n) for n, _ in _Stats._fields_))

    @property
    def bracket_rel(self) -> float:
        """(UB - min(LB, f)) / UB, the certified relative gap the gap stop uses."""
        if self.ub <= 0:
            return 0.0
        return (self.ub - min(self.lb, self.f)) / self.ub


def build(force: bool = False) -> str:
    """Compile w1_oracle.c into libw1_oracle.so next to it (gcc, -O2, no -march)."""
    with _lock:
        stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in (_SRC, _SRC3))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, _SRC3, "-lm"],
                           check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = bind(ctypes.CDLL(_LIB))
    return _lib


def bind(lib):
    """Sets the ctypes signatures of the oracle's C functions on a loaded library
    (the built one, or a test's deliberately mutated copy of it)."""
    d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    lib.w1o_div.argtypes = [i, i, d, p, p, p]
    lib.w1o_grad.argtypes = [i, i, d, p, p, p]
    lib.w1o_prox.argtypes = [i, d, i, p, p, p, p]
    lib.w1o_cp_iterate.argtypes = [i, i, d, i, d, d, p, p, p, p, l, p]
    lib.w1o_cp_iterate.restype = i
    lib.w1o_route_bound.argtypes = [i, i, d, p]
    lib.w1o_route_bound.restype = d
    lib.w1o_stats.argtypes = [i, i, d, i, p, p, p, p, ctypes.POINTER(_Stats)]
    lib.w1o_restrict.argtypes = [i, i, p, p]
    lib.w1o_prolong.argtypes = [i, i, p, p, p, p, p, p]
    lib.w1o_step_size.argtypes = [d, d]
    lib.w1o_step_size.restype = d
    lib.w1o_solve_level.argtypes = [i, i, d, i, d, d, p, p, p, p, d, i, i, l, l, ctypes.POINTER(l),
                                    ctypes.POINTER(_Stats)]
    lib.w1o_solve_level.restype = i
    lib.w1o_multilevel.argtypes = [i, i, d, i, i, d, d, d, d, i, i, l, p, p, p, p, p, p, p,
                                   ctypes.POINTER(_Stats), ctypes.POINTER(d)]
    lib.w1o_multilevel.restype = i
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def div(m1, m2, h):
    """div^h of Sec. 2.2 (zero-flux boundary); m1, m2, result are [ny, nx]."""
    m1, m2 = _f64(m1), _f64(m2)
    ny, nx = m1.shape
    out = np.empty_like(m1)
    _load().w1o_div(nx, ny, h, _ptr(m1), _ptr(m2), _ptr(out))
    return out


def grad(phi, h):
    """Forward-difference gradient (= -A_h^*), zero where it would leave the grid."""
    phi = _f64(phi)
    ny, nx = phi.shape
    g1, g2 = np.empty_like(phi), np.empty_like(phi)
    _load().w1o_grad(nx, ny, h, _ptr(phi), _ptr(g1), _ptr(g2))
    return g1, g2


def prox(norm, mu, v1, v2):
    """Proximal map of mu*||.||_p applied node by node."""
    v1, v2 = _f64(v1), _f64(v2)
    o1, o2 = np.empty_like(v1), np.empty_like(v2)
    _load().w1o_prox(norm, mu, v1.size, _ptr(v1), _ptr(v2), _ptr(o1), _ptr(o2))
    return o1, o2


def step_size(h, theta=0.5):
    """mu = tau = theta / ||A_h|| with ||A_h|| <= 2 sqrt(2) / h."""
    return _load().w1o_step_size(h, theta)


def cp_iterate(rho, m1, m2, phi, h, norm, iters, mu=None, tau=None, theta=0.5):
    """Run `iters` steps of eq. primaldual; returns (m1, m2, phi, fpr_of_last_step)."""
    rho = _f64(rho)
    m1, m2, phi = _f64(m1).copy(), _f64(m2).copy(), _f64(phi).copy()
    ny, nx = rho.shape
    if mu is None:
        mu = step_size(h, theta)
    if tau is None:
        tau = mu
    fpr = ctypes.c_double(0.0)
    st = _load().w1o_cp_iterate(nx, ny, h, norm, mu, tau, _ptr(rho), _ptr(m1), _ptr(m2), _ptr(phi),
                                int(iters), ctypes.cast(ctypes.pointer(fpr), ctypes.c_void_p))
    if st != OK:
        raise RuntimeError(f"w1o_cp_iterate failed: {st}")
    return m1, m2, phi, fpr.value


def route_bound(e, h):
    """Cost of the explicit dyadic flux that carries a residual density e."""
    e = _f64(e)
    ny, nx = e.shape
    return _load().w1o_route_bound(nx, ny, h, _ptr(e))


def stats(rho, m1, m2, phi, h, norm) -> Stats:
    rho, m1, m2, phi = _f64(rho), _f64(m1), _f64(m2), _f64(phi)
    ny, nx = rho.shape
    s = _Stats()
    _load().w1o_stats(nx, ny, h, norm, _ptr(rho), _ptr(m1), _ptr(m2), _ptr(phi), ctypes.byref(s))
    return Stats._from(s)


def restrict(fine):
    """2x2 block mean (density), [ny, nx] -> [ny/2, nx/2]."""
    fine = _f64(fine)
    ny, nx = fine.shape
    out = np.empty((ny // 2, nx // 2))
    _load().w1o_restrict(nx, ny, _ptr(fine), _ptr(out))
    return out


def prolong(m1c, m2c, phic):
    """Interpolate of Sec. 3.3 restated for pixel grids; coarse [ncy, ncx] -> fine [2ncy, 2ncx]."""
    m1c, m2c, phic = _f64(m1c), _f64(m2c), _f64(phic)
    ncy, ncx = phic.shape
    m1f = np.empty((2 * ncy, 2 * ncx))
    m2f, phif = np.empty_like(m1f), np.empty_like(m1f)
    _load().w1o_prolong(ncx, ncy, _ptr(m1c), _ptr(m2c), _ptr(phic), _ptr(m1f), _ptr(m2f), _ptr(phif))
    return m1f, m2f, phif


@dataclass
class LevelResult:
    m1: np.ndarray
    m2: np.ndarray
    phi: np.ndarray
    iters: int
    stats: Stats
    status: int


def solve_level(rho, h, norm, m1=None, m2=None, phi=None, tol=1e-4, stop=STOP_GAP, check_every=32,
                max_iters=200000, replay=-1, theta=0.5, ratio=1.0) -> LevelResult:
    """Algorithm 1 on one grid from (m1, m2, phi) (zeros if None); step sizes
    mu = s / sqrt(ratio), tau = s sqrt(ratio) with s = theta / ||A_h||."""
    rho = _f64(rho)
    ny, nx = rho.shape
    z = np.zeros_like(rho)
    m1 = (z if m1 is None else _f64(m1)).copy()
    m2 = (z if m2 is None else _f64(m2)).copy()
    phi = (z if phi is None else _f64(phi)).copy()
    it = ctypes.c_long(0)
    s = _Stats()
    st = _load().w1o_solve_level(nx, ny, h, norm, theta, ratio, _ptr(rho), _ptr(m1), _ptr(m2), _ptr(phi), tol, stop,
                                 check_every, int(max_iters), int(replay), ctypes.byref(it), ctypes.byref(s))
    if st < 0:
        raise RuntimeError(f"w1o_solve_level failed: {st}")
    return LevelResult(m1, m2, phi, it.value, Stats._from(s), st)


@dataclass
class Result:
    w1: float
    m1: np.ndarray
    m2: np.ndarray
    phi: np.ndarray
    iters: list
    stats: Stats
    status: int


def multilevel(rho0, rho1, h=0.0, levels=1, norm=NORM_L1, tol=1e-4, alpha=-1.0, theta=0.5, stop=STOP_GAP,
               check_every=32, max_iters=200000, replay=None, estimate="saddle", ratio=1.0) -> Result:
    """Algorithm 3 (cascadic multilevel Algorithm 1).  Raises on argument errors;
    returns status NOT_CONVERGED (with the best result) if a level hit max_iters.
    Result.w1 is the W1 estimate of the returned finest pair (m, phi): the
    saddle value L(m, phi) of eq. minmax_cp (estimate="saddle", the default)
    or the primal objective f(m) that Sec. 5 prints (estimate="primal"); both
    are in Result.stats (.saddle, .f)."""
    rho0, rho1 = _f64(rho0), _f64(rho1)
    ny, nx = rho0.shape
    m1, m2, phi = np.empty_like(rho0), np.empty_like(rho0), np.empty_like(rho0)
    iters = (ctypes.c_long * 16)()
    rp = None
    if replay is not None:
        rp_arr = (ctypes.c_long * 16)(*[int(v) for v in replay])
        rp = ctypes.cast(rp_arr, ctypes.c_void_p)
    s = _Stats()
    w1 = ctypes.c_double(0.0)
    st = _load().w1o_multilevel(nx, ny, h, levels, norm, tol, alpha, theta, ratio, stop, check_every, int(max_iters),
                                _ptr(rho0), _ptr(rho1), rp, _ptr(m1), _ptr(m2), _ptr(phi),
                                ctypes.cast(iters, ctypes.c_void_p), ctypes.byref(s), ctypes.byref(w1))
    if st < 0:
        raise ValueError({ERR_ARG: "invalid argument", ERR_SHAPE: "shape not divisible by 2^(levels-1)",
                          ERR_MASS: "mass imbalance or non-finite input", ERR_NOMEM: "out of memory"}[st])
    stats_ = Stats._from(s)
    if estimate not in ("saddle", "primal"):
        raise ValueError("estimate must be 'saddle' or 'primal'")
    w = stats_.saddle if estimate == "saddle" else w1.value
    return Result(w, m1, m2, phi, [iters[k] for k in range(levels)], stats_, st)
