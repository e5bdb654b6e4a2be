"""Independent exact solvers used to pin the oracle (library calls only).

The discrete problem of Sec. 2.2 with p = 1 is a min-cost flow on the
4-neighbour grid graph: every edge costs h per unit of mass moved (a flux m on
an edge moves mass |m| h across it and costs |m| h^2 in f).  These helpers
solve it with HiGHS (scipy.optimize.linprog) or networkx's network simplex, and
solve the tiny p = 2 problems by direct convex minimisation over the affine set
div m = rho.  None of this shares code with the oracle.
"""
from __future__ import annotations

import numpy as np


def _edges(nx, ny):
    """List of (node_a, node_b) for x-edges then y-edges, node = j*nx + i."""
    e = []
    for j in range(ny):
        for i in range(nx - 1):
            e.append((j * nx + i, j * nx + i + 1))
    for j in range(ny - 1):
        for i in range(nx):
            e.append((j * nx + i, (j + 1) * nx + i))
    return e


def w1_lp(rho: np.ndarray, h: float) -> float:
    """Exact discrete p = 1 W1 for a zero-mass density rho [ny, nx] (HiGHS LP)."""
    import scipy.sparse as sp
    from scipy.optimize import linprog

    ny, nx = rho.shape
    edges = _edges(nx, ny)
    E, N = len(edges), nx * ny
    rows, cols, vals = [], [], []
    for k, (a, b) in enumerate(edges):
        # a unit of flow a -> b leaves a and enters b
        rows += [a, b]
        cols += [k, k]
        vals += [1.0, -1.0]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(N, E))
    Aeq = sp.hstack([A, -A]).tocsr()
    b = (rho * h * h).ravel()
    cost = np.full(2 * E, h)
    r = linprog(cost, A_eq=Aeq, b_eq=b, bounds=(0, None), method="highs",
                options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert r.status == 0, r.message
    return float(r.fun)


def w1_network_simplex(q0: np.ndarray, q1: np.ndarray) -> int:
    """Exact min-cost (in edges) to move integer masses q0 onto q1 on the grid graph."""
    import networkx as nx_

    ny, nx = q0.shape
    G = nx_.DiGraph()
    for j in range(ny):
        for i in range(nx):
            G.add_node(j * nx + i, demand=int(q1[j, i]) - int(q0[j, i]))
    for a, b in _edges(nx, ny):
        G.add_edge(a, b, weight=1)
        G.add_edge(b, a, weight=1)
    return int(nx_.network_simplex(G)[0])


def _affine_param(rho, h):
    """Flux vectors m (edge order of _edges) with div m = rho: m = m0 + Z t."""
    import scipy.linalg as sl

    ny, nx = rho.shape
    edges = _edges(nx, ny)
    E, N = len(edges), nx * ny
    A = np.zeros((N, E))
    for k, (a, b) in enumerate(edges):
        A[a, k] += 1.0 / h  # div m at a gains m/h (outflow of the edge leaving a)
        A[b, k] -= 1.0 / h
    m0, *_ = np.linalg.lstsq(A, rho.ravel(), rcond=None)
    Z = sl.null_space(A)
    return edges, m0, Z


def _f_p2(mvec, edges, nx, ny, h):
    m1 = np.zeros((ny, nx))
    m2 = np.zeros((ny, nx))
    nxe = ny * (nx - 1)
    for k, (a, b) in enumerate(edges):
        j, i = divmod(a, nx)
        if k < nxe:
            m1[j, i] = mvec[k]
        else:
            m2[j, i] = mvec[k]
    return float(np.sqrt(m1 * m1 + m2 * m2).sum() * h * h)


def w1_p2_bruteforce(rho: np.ndarray, h: float) -> float:
    """Exact discrete p = 2 W1 on grids with at most two free flux parameters
    (2x2: one, 2x3 / 3x2: two), by nested bounded Brent minimisation of the
    convex objective over the affine set div m = rho."""
    from scipy.optimize import minimize_scalar

    ny, nx = rho.shape
    edges, m0, Z = _affine_param(rho, h)
    scale = 10.0 * (np.abs(m0).max() + 1.0)

    def f(t):
        return _f_p2(m0 + Z @ np.asarray(t), edges, nx, ny, h)

    if Z.shape[1] == 1:
        r = minimize_scalar(lambda t: f([t]), bounds=(-scale, scale), method="bounded",
                            options={"xatol": 1e-13, "maxiter": 2000})
        return float(r.fun)
    if Z.shape[1] == 2:
        def inner(t0):
            r = minimize_scalar(lambda t1: f([t0, t1]), bounds=(-scale, scale), method="bounded",
                                options={"xatol": 1e-13, "maxiter": 2000})
            return r.fun
        r = minimize_scalar(inner, bounds=(-scale, scale), method="bounded",
                            options={"xatol": 1e-12, "maxiter": 2000})
        return float(r.fun)
    raise ValueError("grid too large for the brute-force p=2 solver")


def w1_lp_linf(rho: np.ndarray, h: float) -> float:
    """Exact discrete p = infinity W1: min sum_x t_x h^2 with |m1(x)| <= t_x,
    |m2(x)| <= t_x and div m = rho (boundary flux components absent), an LP."""
    import scipy.sparse as sp
    from scipy.optimize import linprog

    ny, nx = rho.shape
    edges = _edges(nx, ny)
    E, N = len(edges), nx * ny
    # variables: flux per edge (free), t per node (>= 0)
    rows, cols, vals = [], [], []
    for k, (a, b) in enumerate(edges):
        rows += [a, b]
        cols += [k, k]
        vals += [1.0 / h, -1.0 / h]
    Aeq = sp.csr_matrix((vals, (rows, cols)), shape=(N, E + N))
    # |m_e| <= t_{tail node of e}: the edge (i,j)->(i+1,j) is m1 at (i,j), (i,j)->(i,j+1) is m2 at (i,j)
    ur, uc, uv = [], [], []
    r = 0
    for k, (a, b) in enumerate(edges):
        for sgn in (1.0, -1.0):
            ur += [r, r]
            uc += [k, E + a]
            uv += [sgn, -1.0]
            r += 1
    Aub = sp.csr_matrix((uv, (ur, uc)), shape=(r, E + N))
    cost = np.concatenate([np.zeros(E), np.full(N, h * h)])
    bounds = [(None, None)] * E + [(0, None)] * N
    res = linprog(cost, A_ub=Aub, b_ub=np.zeros(r), A_eq=Aeq, b_eq=rho.ravel(), bounds=bounds, method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert res.status == 0, res.message
    return float(res.fun)
