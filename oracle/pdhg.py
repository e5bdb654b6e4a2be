"""FP64 oracle of Algorithms 2 and 4 (prox-PDHG on eq. minmax_pdhg and its
multilevel version), the reference the CUDA prox-PDHG path is checked against.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.

Arrays are FP64 ``[ny, nx]`` on the pixel-centre grid of the other oracle
(spacing h, zero-flux boundary: m1[:, nx-1] = m2[ny-1, :] = 0).  Steps follow
eq. pdhg in the paper's order:

    m^{k+1}   = Proj_{A m = rho}(m^k - mu phibar^k)       (the argmin over m)
    phi^{k+1} = Proj_{||.||_q <= 1}(phi^k + tau m^{k+1}) (the argmax over phi:
                f^* is the indicator of the dual-norm unit ball per node)
    phibar^{k+1} = 2 phi^{k+1} - phi^k

with A = div^h, A^* = -grad, so Proj_{A m = rho}(v) = v + grad psi where psi
solves (A A^*) psi = div v - rho, A A^* = -div grad the Neumann Laplacian.  That
Poisson solve uses scipy's DCT-II (a library primitive): on this grid the
5-point Neumann Laplacian is diagonal in the DCT-II basis with eigenvalues
(2 - 2 cos(pi k / nx)) / h^2 + (2 - 2 cos(pi l / ny)) / h^2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.fft as sf

from . import NORM_L1, NORM_L2, NORM_LINF, prolong, restrict

OK = 0
NOT_CONVERGED = 1


def div(m1, m2, h):
    """div^h of Sec. 2.2 (backward differences, zero flux through the boundary)."""
    a = np.array(m1, dtype=np.float64)
    b = np.array(m2, dtype=np.float64)
    a[:, -1] = 0.0
    b[-1, :] = 0.0
    d = a.copy()
    d[:, 1:] -= a[:, :-1]
    d += b
    d[1:, :] -= b[:-1, :]
    return d / h


def grad(p, h):
    """Forward differences, zero where they would leave the grid (= -A_h^*)."""
    p = np.asarray(p, dtype=np.float64)
    g1 = np.zeros_like(p)
    g2 = np.zeros_like(p)
    g1[:, :-1] = (p[:, 1:] - p[:, :-1]) / h
    g2[:-1, :] = (p[1:, :] - p[:-1, :]) / h
    return g1, g2


def laplacian_eigenvalues(nx, ny, h):
    lx = (2.0 - 2.0 * np.cos(np.pi * np.arange(nx) / nx)) / (h * h)
    ly = (2.0 - 2.0 * np.cos(np.pi * np.arange(ny) / ny)) / (h * h)
    return ly[:, None] + lx[None, :]


def poisson(r, h):
    """psi with (A A^*) psi = r - mean(r) and mean(psi) = 0 (Neumann, DCT-II)."""
    r = np.asarray(r, dtype=np.float64)
    ny, nx = r.shape
    lam = laplacian_eigenvalues(nx, ny, h)
    lam[0, 0] = 1.0
    rh = sf.dctn(r, type=2, norm="ortho")
    ph = rh / lam
    ph[0, 0] = 0.0
    return sf.idctn(ph, type=2, norm="ortho")


def project_affine(v1, v2, rho, h):
    """Euclidean projection of v onto {m : div^h m = rho} (rho of zero mean)."""
    v1 = np.array(v1, dtype=np.float64)
    v2 = np.array(v2, dtype=np.float64)
    v1[:, -1] = 0.0
    v2[-1, :] = 0.0
    psi = poisson(div(v1, v2, h) - rho, h)
    g1, g2 = grad(psi, h)
    return v1 + g1, v2 + g2


def project_dual_ball(f1, f2, norm):
    """Node-wise projection onto {||phi(x)||_q <= 1}, q the dual of p."""
    f1 = np.asarray(f1, dtype=np.float64)
    f2 = np.asarray(f2, dtype=np.float64)
    if norm == NORM_L1:  # q = infinity: clamp each component
        return np.clip(f1, -1.0, 1.0), np.clip(f2, -1.0, 1.0)
    if norm == NORM_L2:  # q = 2: scale back to the unit circle
        n = np.sqrt(f1 * f1 + f2 * f2)
        s = np.where(n > 1.0, 1.0 / np.maximum(n, 1e-300), 1.0)
        return f1 * s, f2 * s
    if norm == NORM_LINF:  # q = 1: the unit l1 ball; shrink both magnitudes by t
        a, b = np.abs(f1), np.abs(f2)
        t = np.where(np.abs(a - b) >= 1.0, np.maximum(a, b) - 1.0, 0.5 * (a + b - 1.0))
        inside = a + b <= 1.0
        o1 = np.where(inside, f1, np.sign(f1) * np.maximum(a - t, 0.0))
        o2 = np.where(inside, f2, np.sign(f2) * np.maximum(b - t, 0.0))
        return o1, o2
    raise ValueError("norm must be 1, 2 or 3")


def objective(m1, m2, h, norm):
    """f(m) = sum_x ||m(x)||_p h^2."""
    a, b = np.abs(m1), np.abs(m2)
    if norm == NORM_L1:
        v = a + b
    elif norm == NORM_L2:
        v = np.sqrt(a * a + b * b)
    else:
        v = np.maximum(a, b)
    return float(v.sum() * h * h)


def step_sizes(theta=0.5):
    """mu = tau = 1/2 (the paper's choice for Algorithm 2; mu tau < 1)."""
    return theta, theta


@dataclass
class State:
    m1: np.ndarray
    m2: np.ndarray
    f1: np.ndarray  # phi (the dual variable, a vector field)
    f2: np.ndarray
    g1: np.ndarray  # phibar
    g2: np.ndarray

    @staticmethod
    def zeros(ny, nx):
        z = lambda: np.zeros((ny, nx))  # noqa: E731
        return State(z(), z(), z(), z(), z(), z())

    def copy(self):
        return State(*(np.array(a) for a in (self.m1, self.m2, self.f1, self.f2, self.g1, self.g2)))


def step(rho, s: State, h, norm, mu, tau):
    """One pass of eq. pdhg; returns (new state, G^k of eq. pdhg_stop)."""
    n1, n2 = project_affine(s.m1 - mu * s.g1, s.m2 - mu * s.g2, rho, h)
    p1, p2 = project_dual_ball(s.f1 + tau * n1, s.f2 + tau * n2, norm)
    dm1, dm2 = n1 - s.m1, n2 - s.m2
    df1, df2 = p1 - s.f1, p2 - s.f2
    h2 = h * h
    G = ((dm1 * dm1 + dm2 * dm2).sum() / mu + (df1 * df1 + df2 * df2).sum() / tau
         + 2.0 * (df1 * dm1 + df2 * dm2).sum()) * h2
    return State(n1, n2, p1, p2, 2.0 * p1 - s.f1, 2.0 * p2 - s.f2), float(G)


@dataclass
class LevelResult:
    state: State
    iters: int
    G: float
    status: int


def solve_level(rho, h, norm, state=None, tol=1e-4, check_every=32, max_iters=100000, replay=-1, theta=0.5):
    """Algorithm 2 on one grid: steps until G^k < tol, tested after every
    check_every-th step (or exactly `replay` steps)."""
    rho = np.asarray(rho, dtype=np.float64)
    mu, tau = step_sizes(theta)
    s = State.zeros(*rho.shape) if state is None else state.copy()
    k, G = 0, 0.0
    while True:
        if replay >= 0 and k >= replay:
            return LevelResult(s, k, G, OK)
        if replay < 0 and k >= max_iters:
            return LevelResult(s, k, G, NOT_CONVERGED)
        s, G = step(rho, s, h, norm, mu, tau)
        k += 1
        if replay < 0 and k % check_every == 0 and G < tol:
            return LevelResult(s, k, G, OK)


def potential(f1, f2, h):
    """Kantorovich potential from phi (Appendix B): lambda = (A A^*)^{-1} A phi;
    returned with the sign of Algorithm 1's potential (dual value -<phi, rho>_h)."""
    return -poisson(div(f1, f2, h), h)


def stop_tolerance(h, levels_h=None):
    """eq. stop_tol for Algorithm 4: eps_L = min(2e-4, 1e-4 / 32 (h / (1/512))^2)."""
    return min(2e-4, 1e-4 / 32.0 * (h * 512.0) ** 2)


@dataclass
class Result:
    w1: float
    m1: np.ndarray
    m2: np.ndarray
    f1: np.ndarray
    f2: np.ndarray
    phi: np.ndarray
    iters: list
    G: list
    status: int


def interpolate(s: State):
    """Interpolate of Sec. 3.3: m and phi (both flux-like, eq. inter_m) to the next grid; phibar = phi."""
    z = np.zeros_like(s.m1)
    m1, m2, _ = prolong(s.m1, s.m2, z)
    f1, f2, _ = prolong(s.f1, s.f2, z)
    return State(m1, m2, f1, f2, f1.copy(), f2.copy())


def multilevel(rho0, rho1, h=0.0, levels=1, norm=NORM_L1, tol=None, alpha=-1.0, theta=0.5, check_every=32,
               max_iters=100000, replay=None) -> Result:
    """Algorithm 4: Algorithm 2 on levels h_l = 2^(L-l) h, coarse to fine, each
    level started from the interpolated coarser solution (zero on level 1),
    eps_l = eps_L (h_l / h)^alpha.  Same mass check and mean subtraction as the
    Algorithm 3 oracle."""
    rho0 = np.asarray(rho0, dtype=np.float64)
    rho1 = np.asarray(rho1, dtype=np.float64)
    ny, nx = rho0.shape
    if h <= 0:
        h = 1.0 / max(nx, ny)
    if levels < 1 or nx % (1 << (levels - 1)) or ny % (1 << (levels - 1)):
        raise ValueError("shape not divisible by 2^(levels-1)")
    M0, M1 = rho0.sum() * h * h, rho1.sum() * h * h
    if not (np.isfinite(rho0).all() and np.isfinite(rho1).all()) or abs(M0 - M1) > 1e-6 * max(abs(M0), abs(M1)):
        raise ValueError("mass imbalance or non-finite input")
    if tol is None:
        tol = stop_tolerance(h)
    rho = rho0 - rho1
    rho = rho - rho.mean()
    pyr = [rho]
    for _ in range(levels - 1):
        pyr.append(restrict(pyr[-1]))
    pyr = pyr[::-1]
    s = None
    iters, Gs, status = [], [], OK
    for lvl, rl in enumerate(pyr):
        hl = h * (1 << (levels - 1 - lvl))
        if s is not None:
            s = interpolate(s)
        r = solve_level(rl, hl, norm, s, tol=tol * (hl / h) ** alpha, check_every=check_every,
                        max_iters=max_iters, replay=-1 if replay is None else int(replay[lvl]), theta=theta)
        s = r.state
        iters.append(r.iters)
        Gs.append(r.G)
        if r.status != OK:
            status = r.status
    return Result(objective(s.m1, s.m2, h, norm), s.m1, s.m2, s.f1, s.f2, potential(s.f1, s.f2, h), iters, Gs,
                  status)
