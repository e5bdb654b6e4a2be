"""Planted mistakes are caught by the oracle's pins.  Each test patches one step
of an oracle (the prox-PDHG, 3-D and 2-D ones; on the CPU, for the duration of
the test) with a plausible error and checks that the pin covering that step
fails: a dropped factor in the Poisson eigenvalues, a sign error in the
gradient, the wrong radius of the dual ball, a wrong objective, a lost boundary
condition, a wrong shrink threshold, wrong restriction weights and wrong
Interpolate weights."""
import numpy as np
import pytest

import oracle
from oracle import d3, pdhg
from tests import test_oracle as pins2
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


# --- the 2-D oracle (planted through its Python wrappers) -------------------------


def test_2d_prox_with_twice_the_threshold(monkeypatch):
    good = oracle.prox
    monkeypatch.setattr(oracle, "prox", lambda norm, mu, v1, v2: good(norm, 2.0 * mu, v1, v2))
    caught(pins2.test_prox_is_the_argmin, L1)


def test_2d_gradient_with_the_wrong_sign(monkeypatch):
    good = oracle.grad
    monkeypatch.setattr(oracle, "grad", lambda phi, h: tuple(-g for g in good(phi, h)))
    caught(pins2.test_div_grad_adjoint, 3, 5)


def test_2d_restriction_by_sums_instead_of_means(monkeypatch):
    good = oracle.restrict
    monkeypatch.setattr(oracle, "restrict", lambda fine: 4.0 * good(fine))
    caught(pins2.test_restrict_conserves_mass_and_constants)


def test_2d_interpolate_that_copies_phi(monkeypatch):
    good = oracle.prolong

    def nearest_phi(m1c, m2c, phic):
        f1, f2, _ = good(m1c, m2c, phic)
        return f1, f2, np.kron(np.asarray(phic, dtype=np.float64), np.ones((2, 2)))

    monkeypatch.setattr(oracle, "prolong", nearest_phi)
    caught(pins2.test_prolong_golden_2x2)
    caught(pins2.test_prolong_phi_reproduces_affine_inside)
