"""Pins of the FP64 prox-PDHG oracle (Algorithms 2 and 4) against facts fixed
by the paper and by mathematics: the Poisson solve against the 5-point stencil
of the Algorithm 3 oracle (independent code), the two projections against their
defining minimisation, converged values against exact LPs, brute force, the 1-D
closed form and Algorithm 1, strong duality of the recovered potential."""
import numpy as np
import pytest

import oracle
from oracle import pdhg
from tests import lp_ref

L1, L2, LINF = oracle.NORM_L1, oracle.NORM_L2, oracle.NORM_LINF


def rand_zero_mass(rng, ny, nx):
    r = rng.normal(size=(ny, nx))
    return r - r.mean()


def converged(rho, h, norm, tol=1e-15, max_iters=200000):
    r = pdhg.solve_level(rho, h, norm, tol=tol, check_every=16, max_iters=max_iters)
    return r


@pytest.mark.parametrize("ny,nx", [(1, 8), (8, 1), (4, 6), (16, 16), (12, 20)])
def test_poisson_inverts_the_neumann_stencil(ny, nx):
    """(A A^*) psi = -div(grad psi) equals r - mean(r); the stencil is the C
    oracle's div and grad, not the DCT."""
    rng = np.random.default_rng(ny * 10 + nx)
    h = 1.0 / max(nx, ny)
    r = rng.normal(size=(ny, nx))
    psi = pdhg.poisson(r, h)
    g1, g2 = oracle.grad(psi, h)
    lap = -oracle.div(g1, g2, h)
    np.testing.assert_allclose(lap, r - r.mean(), atol=1e-9 * np.abs(r).max())
    assert abs(psi.mean()) < 1e-12


def test_operators_agree_with_the_c_oracle():
    rng = np.random.default_rng(3)
    m1, m2, p = rng.normal(size=(3, 7, 9))
    h = 1 / 9
    np.testing.assert_allclose(pdhg.div(m1, m2, h), oracle.div(m1, m2, h), rtol=1e-13, atol=1e-12)
    for a, b in zip(pdhg.grad(p, h), oracle.grad(p, h)):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-12)


def test_affine_projection_is_feasible_idempotent_and_nearest():
    rng = np.random.default_rng(5)
    ny, nx, h = 10, 14, 1 / 14
    rho = rand_zero_mass(rng, ny, nx)
    v1, v2 = rng.normal(size=(2, ny, nx))
    v1[:, -1] = 0
    v2[-1, :] = 0
    m1, m2 = pdhg.project_affine(v1, v2, rho, h)
    np.testing.assert_allclose(oracle.div(m1, m2, h), rho, atol=1e-9)
    assert np.all(m1[:, -1] == 0) and np.all(m2[-1, :] == 0)
    a1, a2 = pdhg.project_affine(m1, m2, rho, h)
    np.testing.assert_allclose(a1, m1, atol=1e-10)
    np.testing.assert_allclose(a2, m2, atol=1e-10)
    d0 = ((m1 - v1) ** 2 + (m2 - v2) ** 2).sum()
    for _ in range(5):  # any other feasible flux is farther from v
        w1, w2 = pdhg.project_affine(*rng.normal(size=(2, ny, nx)), rho, h)
        assert ((w1 - v1) ** 2 + (w2 - v2) ** 2).sum() >= d0 * (1 - 1e-12)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_dual_ball_projection_is_the_nearest_point(norm):
    rng = np.random.default_rng(norm)
    pts = rng.normal(scale=1.5, size=(2, 40))
    o1, o2 = pdhg.project_dual_ball(pts[0], pts[1], norm)
    q = {L1: np.inf, L2: 2, LINF: 1}[norm]
    # candidates: a fine grid of the ball plus its boundary
    t = np.linspace(-1, 1, 401)
    X, Y = np.meshgrid(t, t)
    cand = np.stack([X.ravel(), Y.ravel()])
    cand = cand[:, np.linalg.norm(cand, ord=q, axis=0) <= 1 + 1e-12]
    for k in range(pts.shape[1]):
        p = pts[:, k]
        got = np.array([o1[k], o2[k]])
        assert np.linalg.norm(got, ord=q) <= 1 + 1e-12
        best = np.min(np.sum((cand - p[:, None]) ** 2, axis=0))
        assert np.sum((got - p) ** 2) <= best + 1e-12
    i1, i2 = pdhg.project_dual_ball(o1, o2, norm)  # idempotent
    np.testing.assert_allclose(i1, o1, atol=1e-14)
    np.testing.assert_allclose(i2, o2, atol=1e-14)


@pytest.mark.parametrize("shape", [(2, 2), (4, 6), (8, 8)])
def test_p1_converges_to_the_exact_lp(shape):
    ny, nx = shape
    rng = np.random.default_rng(ny * 3 + nx)
    h = 1.0 / max(nx, ny)
    rho = rand_zero_mass(rng, ny, nx)
    exact = lp_ref.w1_lp(rho, h)
    r = converged(rho, h, L1)
    assert pdhg.objective(r.state.m1, r.state.m2, h, L1) == pytest.approx(exact, rel=1e-6)
    np.testing.assert_allclose(oracle.div(r.state.m1, r.state.m2, h), rho, atol=1e-8 * np.abs(rho).max())


@pytest.mark.parametrize("shape", [(4, 6), (8, 8)])
def test_pinf_converges_to_the_exact_lp(shape):
    ny, nx = shape
    rng = np.random.default_rng(ny * 5 + nx)
    h = 1.0 / max(nx, ny)
    rho = rand_zero_mass(rng, ny, nx)
    exact = lp_ref.w1_lp_linf(rho, h)
    r = converged(rho, h, LINF)
    assert pdhg.objective(r.state.m1, r.state.m2, h, LINF) == pytest.approx(exact, rel=1e-6)


@pytest.mark.parametrize("shape", [(2, 2), (2, 3)])
def test_p2_converges_to_the_bruteforce_minimum(shape):
    ny, nx = shape
    rng = np.random.default_rng(11 * nx + ny)
    h = 1.0 / max(nx, ny)
    rho = rand_zero_mass(rng, ny, nx)
    exact = lp_ref.w1_p2_bruteforce(rho, h)
    r = converged(rho, h, L2)
    assert pdhg.objective(r.state.m1, r.state.m2, h, L2) == pytest.approx(exact, rel=1e-6)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_strip_closed_form(norm):
    n = 16
    rng = np.random.default_rng(40 + norm)
    h = 1.0 / n
    r0 = rng.uniform(0.1, 1.0, n)
    r1 = rng.uniform(0.1, 1.0, n)
    r0 /= r0.sum() * h * h
    r1 /= r1.sum() * h * h
    C = np.cumsum((r0 - r1) * h * h)
    exact = np.abs(C[:-1]).sum() * h
    res = pdhg.multilevel(r0.reshape(1, n), r1.reshape(1, n), h=h, levels=1, norm=norm, tol=1e-20,
                          check_every=16, max_iters=20000)
    assert res.w1 == pytest.approx(exact, rel=1e-8)
    np.testing.assert_allclose(res.m1.ravel()[:-1], C[:-1] / h, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_agrees_with_algorithm_1_and_strong_duality(norm):
    """Algorithms 1 and 2 solve the same discrete problem: converged values agree;
    the potential recovered from phi (Appendix B) is dual feasible and attains it."""
    rng = np.random.default_rng(60 + norm)
    n, h = 16, 1 / 16
    r0 = rng.uniform(0.2, 1.0, (n, n))
    r1 = rng.uniform(0.2, 1.0, (n, n))
    r0 /= r0.sum() * h * h
    r1 /= r1.sum() * h * h
    a1 = oracle.multilevel(r0, r1, levels=1, norm=norm, tol=1e-9, stop=oracle.STOP_GAP, theta=1.0,
                           check_every=64, max_iters=3_000_000)
    res = pdhg.multilevel(r0, r1, levels=1, norm=norm, tol=1e-16, check_every=16, max_iters=100000)
    assert res.w1 == pytest.approx(a1.w1, rel=1e-6)
    rho = r0 - r1
    dual = -(res.phi * rho).sum() * h * h
    assert dual == pytest.approx(res.w1, rel=1e-6)
    g1, g2 = oracle.grad(res.phi, h)
    q = {L1: np.inf, L2: 2, LINF: 1}[norm]
    gn = np.linalg.norm(np.stack([g1.ravel(), g2.ravel()]), ord=q, axis=0)
    assert gn.max() <= 1 + 1e-6


def test_residual_goes_to_zero_and_multilevel_matches_single_level():
    rng = np.random.default_rng(9)
    n, h = 32, 1 / 32
    r0 = rng.uniform(0.2, 1.0, (n, n))
    r1 = rng.uniform(0.2, 1.0, (n, n))
    r0 /= r0.sum() * h * h
    r1 /= r1.sum() * h * h
    one = pdhg.multilevel(r0, r1, levels=1, norm=L2, tol=1e-14, check_every=16, max_iters=100000)
    ml = pdhg.multilevel(r0, r1, levels=2, norm=L2, tol=1e-14, check_every=16, max_iters=100000)
    assert ml.w1 == pytest.approx(one.w1, rel=1e-6)
    assert one.G[-1] < 1e-14 and ml.G[-1] < 1e-14
    again = pdhg.multilevel(r0, r1, levels=2, norm=L2, replay=ml.iters)
    assert again.w1 == ml.w1 and again.iters == ml.iters


def test_paper_tolerance_and_errors():
    assert pdhg.stop_tolerance(1 / 512) == pytest.approx(1e-4 / 32)
    assert pdhg.stop_tolerance(1 / 16) == pytest.approx(2e-4)
    z = np.ones((8, 8))
    with pytest.raises(ValueError):
        pdhg.multilevel(z, 2 * z, levels=1)
    with pytest.raises(ValueError):
        pdhg.multilevel(z, z, levels=5)
