"""Exact discrete W1 for p = 1 and p = infinity, by linear programming.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only ``tests/``, the
smoke check, the benchmark's CPU-baseline leg and the script that writes the
stored converged values may use it.

The discrete problem of Sec. 2.2 (eq. opt_flux_dis) is

    W1_h = min_m  sum_x ||m(x)||_p h^2   s.t.  div^h m = rho,  zero-flux boundary,

with m1(i, j) on the x-edge (i, j) -> (i + 1, j) and m2(i, j) on the y-edge
(i, j) -> (i, j + 1), exactly the unknowns of the iteration.  For p = 1 and
p = infinity it is a linear program; this module writes that program out and
hands it to HiGHS (scipy.optimize.linprog, interior point with crossover to a
vertex, so the value is that of an exact basic solution).  No step of
Algorithm 1 or 3 is used: this is the definition the iteration converges to.

Scaling: the constraint rows are div^h m = rho multiplied by h, i.e.
m1(x) - m1(x - e1) + m2(x) - m2(x - e2) = h rho(x) (unit coefficients), and the
objective is sum ||m(x)||_p h^2.
"""
from __future__ import annotations

import numpy as np


def _incidence(nx: int, ny: int):
    """Sparse [nodes x edges] matrix of h * div^h: +1 where an edge leaves its
    node (its own m), -1 at the node it enters; x-edges first, then y-edges,
    each row-major over the nodes they leave."""
    import scipy.sparse as sp

    idx = np.arange(nx * ny).reshape(ny, nx)
    tail = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])  # (i, j)
    head = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])    # (i + 1, j) or (i, j + 1)
    e = tail.size
    rows = np.concatenate([tail, head])
    cols = np.concatenate([np.arange(e), np.arange(e)])
    vals = np.concatenate([np.ones(e), -np.ones(e)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nx * ny, e)), tail


def w1_exact(rho: np.ndarray, h: float, norm: int = 1) -> float:
    """Exact W1_h of a zero-sum density rho [ny, nx] for norm 1 (p = 1) or
    3 (p = infinity).  Raises if HiGHS does not report an optimal solution."""
    import scipy.sparse as sp
    from scipy.optimize import linprog

    rho = np.asarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    A, tail = _incidence(nx, ny)
    e = A.shape[1]
    b = rho.ravel() * h
    opts = {"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10}
    if norm == 1:
        # m = m+ - m-, m+/- >= 0: min sum (m+ + m-) h^2, at an optimum one of them is 0
        Aeq = sp.hstack([A, -A]).tocsr()
        cost = np.full(2 * e, h * h)
        r = linprog(cost, A_eq=Aeq, b_eq=b, bounds=(0, None), method="highs-ipm", options=opts)
    elif norm == 3:
        # per node t(x) >= |m1(x)|, t(x) >= |m2(x)| (the edges leaving x): min sum t h^2
        n = nx * ny
        T = sp.csr_matrix((np.ones(e), (np.arange(e), tail)), shape=(e, n))  # edge -> its node's t
        Aeq = sp.hstack([A, -A, sp.csr_matrix((n, n))]).tocsr()
        I = sp.identity(e, format="csr")
        Aub = sp.hstack([I, I, -T]).tocsr()  # m+ + m- - t(tail) <= 0
        cost = np.concatenate([np.zeros(2 * e), np.full(n, h * h)])
        r = linprog(cost, A_ub=Aub, b_ub=np.zeros(e), A_eq=Aeq, b_eq=b, bounds=(0, None), method="highs-ipm",
                    options=opts)
    else:
        raise ValueError("the exact LP covers norm 1 (p = 1) and 3 (p = infinity)")
    if r.status != 0:
        raise RuntimeError(f"HiGHS: {r.message}")
    return float(r.fun)
