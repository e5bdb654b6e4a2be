"""Pins of the FP64 3-D oracle (Algorithm 3 with d = 3) against exact LPs on the
6-neighbour grid graph, the 1-D closed form along each axis, translated bumps,
brute-force proximal maps and the identities of the operators."""
import numpy as np
import pytest

from oracle import d3

L1, L2, LINF = 1, 2, 3


def edges3(nx, ny, nz):
    idx = lambda i, j, k: (k * ny + j) * nx + i  # noqa: E731
    e = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if i + 1 < nx:
                    e.append((idx(i, j, k), idx(i + 1, j, k), 0))
                if j + 1 < ny:
                    e.append((idx(i, j, k), idx(i, j + 1, k), 1))
                if k + 1 < nz:
                    e.append((idx(i, j, k), idx(i, j, k + 1), 2))
    return e


def lp3(rho, h, norm):
    """Exact discrete W1 on the 6-neighbour grid (HiGHS): p = 1 min-cost flow
    (cost h per unit of mass per edge); p = infinity with a per-node bound t >= |m_c|."""
    import scipy.sparse as sp
    from scipy.optimize import linprog
    nz, ny, nx = rho.shape
    E = edges3(nx, ny, nz)
    N = nx * ny * nz
    if norm == L1:
        rows, cols, vals = [], [], []
        for k, (a, b, _) in enumerate(E):
            rows += [a, b]
            cols += [k, k]
            vals += [1.0, -1.0]
        A = sp.csr_matrix((vals, (rows, cols)), shape=(N, len(E)))
        r = linprog(np.full(2 * len(E), h), A_eq=sp.hstack([A, -A]).tocsr(), b_eq=(rho * h ** 3).ravel(),
                    bounds=(0, None), method="highs")
        assert r.status == 0
        return r.fun
    # p = infinity: flux variables per edge (value m = flow / h^2 per unit area), t per node
    rows, cols, vals = [], [], []
    for k, (a, b, _) in enumerate(E):
        rows += [a, b]
        cols += [k, k]
        vals += [1.0 / h, -1.0 / h]
    Aeq = sp.csr_matrix((vals, (rows, cols)), shape=(N, len(E) + N))
    ur, uc, uv, r_ = [], [], [], 0
    for k, (a, _, _) in enumerate(E):
        for sgn in (1.0, -1.0):
            ur += [r_, r_]
            uc += [k, len(E) + a]
            uv += [sgn, -1.0]
            r_ += 1
    Aub = sp.csr_matrix((uv, (ur, uc)), shape=(r_, len(E) + N))
    res = linprog(np.concatenate([np.zeros(len(E)), np.full(N, h ** 3)]), A_ub=Aub, b_ub=np.zeros(r_),
                  A_eq=Aeq, b_eq=rho.ravel(), bounds=[(None, None)] * len(E) + [(0, None)] * N, method="highs")
    assert res.status == 0
    return res.fun


def rand_zero_mass(rng, shape):
    r = rng.normal(size=shape)
    return r - r.mean()


def tight(rho, h, norm, tol=1e-15):
    r0 = np.maximum(rho, 0) + 1.0
    r1 = np.maximum(-rho, 0) + 1.0
    return d3.multilevel(r0, r1, h=h, levels=1, norm=norm, tol=tol, theta=1.0, check_every=64,
                         max_iters=2_000_000)


@pytest.mark.parametrize("shape", [(1, 1, 7), (6, 1, 1), (3, 4, 5)])
def test_adjoint_identity(shape):
    rng = np.random.default_rng(sum(shape))
    nz, ny, nx = shape
    h = 1.0 / max(shape)
    m1, m2, m3, p = rng.normal(size=(4,) + shape)
    g = d3.grad(p, h)
    lhs = (p * d3.div(m1, m2, m3, h)).sum()
    # the pinned boundary entries do not take part
    m1[..., -1] = 0
    m2[:, -1, :] = 0
    m3[-1] = 0
    rhs = -(g[0] * m1 + g[1] * m2 + g[2] * m3).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_prox_is_the_argmin(norm):
    from scipy.optimize import minimize
    rng = np.random.default_rng(norm)
    mu = 0.3
    nrm = {L1: 1, L2: 2, LINF: np.inf}[norm]
    for _ in range(12):
        v = rng.normal(size=3)
        got = np.array([x[0] for x in d3.prox(norm, mu, *(np.array([c]) for c in v))])
        obj = lambda u: mu * np.linalg.norm(u, ord=nrm) + 0.5 * np.sum((u - v) ** 2)  # noqa: E731
        best = minimize(obj, got + 1e-3, method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-14,
                                                                          "maxiter": 20000})
        assert obj(got) <= best.fun + 1e-10


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 3, 3), (2, 3, 4)])
@pytest.mark.parametrize("norm", [L1, LINF])
def test_matches_exact_lp(shape, norm):
    rng = np.random.default_rng(sum(shape) + norm)
    h = 1.0 / max(shape)
    rho = rand_zero_mass(rng, shape)
    exact = lp3(rho, h, norm)
    res = tight(rho, h, norm)
    assert res.status == 0
    assert res.w1 == pytest.approx(exact, rel=1e-6)
    assert res.stats.lb <= exact * (1 + 1e-9) and res.stats.ub >= exact * (1 - 1e-9)


def test_norms_order_the_distances():
    rng = np.random.default_rng(4)
    shape, h = (3, 3, 3), 1 / 3
    rho = rand_zero_mass(rng, shape)
    w = {n: tight(rho, h, n).w1 for n in (L1, L2, LINF)}
    assert w[LINF] <= w[L2] * (1 + 1e-6) and w[L2] <= w[L1] * (1 + 1e-6)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_strip_closed_form(axis, norm):
    n = 12
    rng = np.random.default_rng(10 * axis + norm)
    h = 1.0 / n
    r0 = rng.uniform(0.1, 1.0, n)
    r1 = rng.uniform(0.1, 1.0, n)
    r0 /= r0.sum() * h ** 3
    r1 /= r1.sum() * h ** 3
    C = np.cumsum((r0 - r1) * h ** 3)
    exact = np.abs(C[:-1]).sum() * h
    shape = [1, 1, 1]
    shape[2 - axis] = n  # axis 0 = x (last array axis)
    res = d3.multilevel(r0.reshape(shape), r1.reshape(shape), h=h, levels=1, norm=norm, tol=1e-24, theta=1.0,
                        check_every=64, max_iters=2_000_000)
    assert res.w1 == pytest.approx(exact, rel=1e-8)
    m = (res.m1, res.m2, res.m3)[axis].ravel()
    np.testing.assert_allclose(m[:-1], C[:-1] / h ** 2, rtol=1e-6, atol=1e-9)


def test_translated_bump():
    """rho1 = rho0 shifted by (a, b, c) voxels, support away from the walls: p = 1 gives
    W1 = (|a| + |b| + |c|) h mass (dual phi = -(sgn a x + sgn b y + sgn c z))."""
    n, h = 8, 1 / 8
    r0 = np.zeros((n, n, n))
    r0[2:4, 2:4, 2:4] = 1.0
    a, b, c = 2, 1, 2
    r1 = np.roll(np.roll(np.roll(r0, a, axis=2), b, axis=1), c, axis=0)
    mass = r0.sum() * h ** 3
    res = d3.multilevel(r0 + 0.5, r1 + 0.5, h=h, levels=1, norm=L1, tol=1e-18, theta=1.0, check_every=64,
                        max_iters=2_000_000)
    assert res.w1 == pytest.approx((a + b + c) * h * mass, rel=1e-6)


def test_restrict_prolong_identities():
    rng = np.random.default_rng(8)
    fine = rng.normal(size=(4, 6, 8))
    c = d3.restrict(fine)
    assert c.sum() * 8 == pytest.approx(fine.sum())
    # Interpolate commutes with the divergence under restriction: R div_f P m = div_c m
    m1c, m2c, m3c, pc = rng.normal(size=(4, 3, 2, 4))
    m1c[..., -1] = 0
    m2c[:, -1, :] = 0
    m3c[-1] = 0
    hc, hf = 1 / 4, 1 / 8
    f1, f2, f3, pf = d3.prolong(m1c, m2c, m3c, pc)
    np.testing.assert_allclose(d3.restrict(d3.div(f1, f2, f3, hf)), d3.div(m1c, m2c, m3c, hc), atol=1e-12)
    # Lemma 3.1: the interpolated potential is no larger in L2 (h^3 weights)
    assert (pf ** 2).sum() * hf ** 3 <= (pc ** 2).sum() * hc ** 3 * (1 + 1e-12)
    # affine potentials are reproduced away from the clamped boundary
    Z, Y, X = np.meshgrid(np.arange(3), np.arange(2), np.arange(4), indexing="ij")
    _, _, _, pa = d3.prolong(0 * m1c, 0 * m2c, 0 * m3c, 1.0 + 2.0 * X - 1.0 * Y + 0.5 * Z)
    zf, yf, xf = np.meshgrid(np.arange(6), np.arange(4), np.arange(8), indexing="ij")
    want = 1.0 + 2.0 * (xf - 0.5) / 2 - 1.0 * (yf - 0.5) / 2 + 0.5 * (zf - 0.5) / 2
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(pa[inner], want[inner], atol=1e-12)


def test_multilevel_matches_single_level_and_replays():
    rng = np.random.default_rng(12)
    n, h = 8, 1 / 8
    r0 = rng.uniform(0.2, 1.0, (n, n, n))
    r1 = rng.uniform(0.2, 1.0, (n, n, n))
    r0 /= r0.sum() * h ** 3
    r1 /= r1.sum() * h ** 3
    one = d3.multilevel(r0, r1, levels=1, norm=L2, tol=1e-16, theta=1.0, check_every=64, max_iters=2_000_000)
    ml = d3.multilevel(r0, r1, levels=2, norm=L2, tol=1e-16, theta=1.0, check_every=64, max_iters=2_000_000)
    assert ml.w1 == pytest.approx(one.w1, rel=1e-6)
    again = d3.multilevel(r0, r1, levels=2, norm=L2, theta=1.0, replay=ml.iters)
    assert again.w1 == ml.w1 and again.iters == ml.iters


def test_errors():
    z = np.ones((4, 4, 4))
    with pytest.raises(ValueError):
        d3.multilevel(z, 2 * z)
    with pytest.raises(ValueError):
        d3.multilevel(z, z, levels=4)
