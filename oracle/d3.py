"""FP64 oracle of Algorithm 3 on three-dimensional grids (ctypes over
w1_oracle3.c).  TEST INFRASTRUCTURE ONLY, like the rest of this package.

Arrays are FP64 ``[nz, ny, nx]`` (x fastest), flux components (m1, m2, m3)
along x, y, z, zero flux through the boundary, inner products weighted by h^3.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _load as _load2d


class _Stats3(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in ("f", "dual", "res_l1", "rho_l1", "gmax", "lb", "route", "ub",
                                                      "saddle")]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = _load2d()
        d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        lib.w1o3_div.argtypes = [i, i, i, d, p, p, p, p]
        lib.w1o3_grad.argtypes = [i, i, i, d, p, p, p, p]
        lib.w1o3_prox.argtypes = [i, d, i, p, p, p, p, p, p]
        lib.w1o3_step_size.argtypes = [d, d]
        lib.w1o3_step_size.restype = d
        lib.w1o3_cp_iterate.argtypes = [i, i, i, d, i, d, d, p, p, p, p, p, l, p]
        lib.w1o3_cp_iterate.restype = i
        lib.w1o3_route_bound.argtypes = [i, i, i, d, p]
        lib.w1o3_route_bound.restype = d
        lib.w1o3_stats.argtypes = [i, i, i, d, i, p, p, p, p, p, ctypes.POINTER(_Stats3)]
        lib.w1o3_restrict.argtypes = [i, i, i, p, p]
        lib.w1o3_prolong.argtypes = [i, i, i, p, p, p, p, p, p, p, p]
        lib.w1o3_multilevel.argtypes = [i, i, i, d, i, i, d, d, d, i, l, p, p, p, p, p, p, p, p, p,
                                        ctypes.POINTER(_Stats3), ctypes.POINTER(d)]
        lib.w1o3_multilevel.restype = i
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def div(m1, m2, m3, h):
    m1, m2, m3 = _f64(m1), _f64(m2), _f64(m3)
    nz, ny, nx = m1.shape
    out = np.empty_like(m1)
    _load().w1o3_div(nx, ny, nz, h, _p(m1), _p(m2), _p(m3), _p(out))
    return out


def grad(phi, h):
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    g = [np.empty_like(phi) for _ in range(3)]
    _load().w1o3_grad(nx, ny, nz, h, _p(phi), *(_p(x) for x in g))
    return tuple(g)


def prox(norm, mu, v1, v2, v3):
    v = [_f64(x) for x in (v1, v2, v3)]
    o = [np.empty_like(v[0]) for _ in range(3)]
    _load().w1o3_prox(norm, mu, v[0].size, *(_p(x) for x in v), *(_p(x) for x in o))
    return tuple(o)


def step_size(h, theta=0.5):
    return _load().w1o3_step_size(h, theta)


def cp_iterate(rho, m1, m2, m3, phi, h, norm, iters, mu=None, tau=None, theta=0.5):
    rho = _f64(rho)
    st = [_f64(x).copy() for x in (m1, m2, m3, phi)]
    nz, ny, nx = rho.shape
    if mu is None:
        mu = step_size(h, theta)
    if tau is None:
        tau = mu
    f = ctypes.c_double(0.0)
    r = _load().w1o3_cp_iterate(nx, ny, nz, h, norm, mu, tau, _p(rho), *(_p(x) for x in st), int(iters),
                                ctypes.cast(ctypes.pointer(f), ctypes.c_void_p))
    if r != 0:
        raise RuntimeError(f"w1o3_cp_iterate failed: {r}")
    return (*st, f.value)


def route_bound(e, h):
    e = _f64(e)
    nz, ny, nx = e.shape
    return _load().w1o3_route_bound(nx, ny, nz, h, _p(e))


@dataclass
class Stats3:
    f: float
    dual: float
    res_l1: float
    rho_l1: float
    gmax: float
    lb: float
    route: float
    ub: float
    saddle: float


def stats(rho, m1, m2, m3, phi, h, norm) -> Stats3:
    a = [_f64(x) for x in (rho, m1, m2, m3, phi)]
    nz, ny, nx = a[0].shape
    s = _Stats3()
    _load().w1o3_stats(nx, ny, nz, h, norm, *(_p(x) for x in a), ctypes.byref(s))
    return Stats3(*(getattr(s, n) for n, _ in _Stats3._fields_))


def restrict(fine):
    fine = _f64(fine)
    nz, ny, nx = fine.shape
    out = np.empty((nz // 2, ny // 2, nx // 2))
    _load().w1o3_restrict(nx, ny, nz, _p(fine), _p(out))
    return out


def prolong(m1c, m2c, m3c, phic):
    c = [_f64(x) for x in (m1c, m2c, m3c, phic)]
    ncz, ncy, ncx = c[0].shape
    f = [np.empty((2 * ncz, 2 * ncy, 2 * ncx)) for _ in range(4)]
    _load().w1o3_prolong(ncx, ncy, ncz, *(_p(x) for x in c), *(_p(x) for x in f))
    return tuple(f)


@dataclass
class Result3:
    w1: float
    m1: np.ndarray
    m2: np.ndarray
    m3: np.ndarray
    phi: np.ndarray
    iters: list
    fpr: list
    stats: Stats3
    status: int


def multilevel(rho0, rho1, h=0.0, levels=1, norm=1, tol=1e-6, alpha=-1.0, theta=0.5, check_every=32,
               max_iters=1_000_000, replay=None, estimate="saddle") -> Result3:
    """Algorithm 3 on a 3-D grid with the FPR stop (R^k < eps_l after every K-th step).
    Result3.w1 is the saddle value (the Lagrangian of eq. minmax_cp at the
    returned pair) or, with estimate="primal", f(m); both are in .stats."""
    r0, r1 = _f64(rho0), _f64(rho1)
    nz, ny, nx = r0.shape
    out = [np.empty_like(r0) for _ in range(4)]
    iters = (ctypes.c_long * 16)()
    fprs = (ctypes.c_double * 16)()
    rp = None
    if replay is not None:
        arr = (ctypes.c_long * 16)(*[int(v) for v in replay])
        rp = ctypes.cast(arr, ctypes.c_void_p)
    s = _Stats3()
    w1 = ctypes.c_double(0.0)
    st = _load().w1o3_multilevel(nx, ny, nz, h, levels, norm, tol, alpha, theta, check_every, int(max_iters),
                                 _p(r0), _p(r1), rp, *(_p(x) for x in out), ctypes.cast(iters, ctypes.c_void_p),
                                 ctypes.cast(fprs, ctypes.c_void_p), ctypes.byref(s), ctypes.byref(w1))
    if st < 0:
        raise ValueError({-1: "invalid argument", -2: "shape not divisible by 2^(levels-1)",
                          -3: "mass imbalance or non-finite input", -4: "out of memory"}[st])
    s3 = Stats3(*(getattr(s, n) for n, _ in _Stats3._fields_))
    if estimate not in ("saddle", "primal"):
        raise ValueError("estimate must be 'saddle' or 'primal'")
    w = s3.saddle if estimate == "saddle" else w1.value
    return Result3(w, *out, [iters[k] for k in range(levels)], [fprs[k] for k in range(levels)], s3, st)
