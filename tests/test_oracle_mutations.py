"""Planted mistakes are caught by the oracle's pins.  Each test patches one step
of the oracle (on the CPU, for the duration of the test) with a plausible error
and checks that the pin covering that step fails: a dropped factor in the
Poisson eigenvalues, a sign error in the gradient, the wrong radius of the dual
ball, a wrong objective, a lost boundary condition, a wrong restriction weight
and a wrong Interpolate weight."""
import numpy as np
import pytest

import oracle
from oracle import d3, pdhg
from tests import test_oracle_3d as pins3
from tests import test_oracle_pdhg as pins

L1, L2, LINF = oracle.NORM_L1, oracle.NORM_L2, oracle.NORM_LINF


def caught(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_wrong_poisson_eigenvalues(monkeypatch):
    good = pdhg.laplacian_eigenvalues
    monkeypatch.setattr(pdhg, "laplacian_eigenvalues", lambda nx, ny, h: 2.0 * good(nx, ny, h))
    caught(pins.test_poisson_inverts_the_neumann_stencil, 4, 6)


def test_sign_error_in_the_gradient(monkeypatch):
    good = pdhg.grad
    monkeypatch.setattr(pdhg, "grad", lambda p, h: tuple(-g for g in good(p, h)))
    caught(pins.test_affine_projection_is_feasible_idempotent_and_nearest)
    caught(pins.test_operators_agree_with_the_c_oracle)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_dual_ball_of_radius_two(monkeypatch, norm):
    good = pdhg.project_dual_ball

    def radius_two(f1, f2, nrm):
        o1, o2 = good(np.asarray(f1) / 2.0, np.asarray(f2) / 2.0, nrm)
        return 2.0 * o1, 2.0 * o2

    monkeypatch.setattr(pdhg, "project_dual_ball", radius_two)
    caught(pins.test_dual_ball_projection_is_the_nearest_point, norm)


def test_objective_without_the_cell_area(monkeypatch):
    good = pdhg.objective
    monkeypatch.setattr(pdhg, "objective", lambda m1, m2, h, norm: good(m1, m2, h, norm) / (h * h))
    caught(pins.test_p1_converges_to_the_exact_lp, (4, 6))


def test_divergence_without_the_zero_flux_boundary(monkeypatch):
    def leaky_div(m1, m2, h):
        a = np.array(m1, dtype=np.float64)
        b = np.array(m2, dtype=np.float64)
        d = a.copy()
        d[:, 1:] -= a[:, :-1]
        d += b
        d[1:, :] -= b[:-1, :]
        return d / h

    monkeypatch.setattr(pdhg, "div", leaky_div)
    caught(pins.test_operators_agree_with_the_c_oracle)


def test_restriction_that_loses_mass(monkeypatch):
    good = d3.restrict
    monkeypatch.setattr(d3, "restrict", lambda fine: 0.5 * good(fine))
    caught(pins3.test_restrict_prolong_identities)


def test_interpolate_with_the_wrong_weights(monkeypatch):
    good = d3.prolong

    def half_weight(m1c, m2c, m3c, phic):
        f1, f2, f3, pf = good(m1c, m2c, m3c, phic)
        return f1, f2, f3, 0.5 * pf + 0.5 * np.kron(np.asarray(phic), np.ones((2, 2, 2)))

    monkeypatch.setattr(d3, "prolong", half_weight)
    caught(pins3.test_restrict_prolong_identities)
