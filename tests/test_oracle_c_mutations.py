"""Mistakes planted in the C oracle itself must fail its pins.

Each case copies oracle/w1_oracle.c, replaces one line of the arithmetic with a
plausible mistake (a dropped extrapolation, a wrong shrink threshold, a sign
error in the gradient, the divergence or the dual step, a wrong saddle term, a
wrong restriction or Interpolate weight), compiles the copy with gcc into a
temporary library, points the oracle's Python wrapper at it, and runs a small
set of pins: the exact LP with strong duality and dual feasibility, the 1-D
closed form, the saddle value of a feasible flux and of zero flux, mass
conservation of the restriction, and the divergence commutation of
Interpolate.  At least one pin must fail for every mutant; the unmutated
source passes all of them.  Nothing here touches a GPU.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from tests import lp_ref

SRC = os.path.join(os.path.dirname(oracle.__file__), "w1_oracle.c")
SRC3 = os.path.join(os.path.dirname(oracle.__file__), "w1_oracle3.c")

MUTATIONS = {
    "no extrapolation": ("s->b1[k] = 2.0 * s->n1[k] - m1[k];", "s->b1[k] = s->n1[k];"),
    "shrink threshold doubled": ("double a1 = fabs(v1) - mu, a2 = fabs(v2) - mu;",
                                 "double a1 = fabs(v1) - 2.0 * mu, a2 = fabs(v2) - 2.0 * mu;"),
    "divergence sign": ("if (i > 0) d1 -= AT(m1, j, i - 1);", "if (i > 0) d1 += AT(m1, j, i - 1);"),
    "dual step sign": ("s->dphi[k] = tau * (s->d[k] - rho[k]);", "s->dphi[k] = tau * (s->d[k] + rho[k]);"),
    "gradient sign": ("AT(g1, j, i) = (i < nx - 1) ? (AT(phi, j, i + 1) - AT(phi, j, i)) / h : 0.0;",
                      "AT(g1, j, i) = (i < nx - 1) ? (AT(phi, j, i) - AT(phi, j, i + 1)) / h : 0.0;"),
    "saddle term sign": ("out->saddle = out->f + inner;", "out->saddle = out->f - inner;"),
    "restriction by sums": ("coarse[(size_t)J * ncx + I] = 0.25 * (", "coarse[(size_t)J * ncx + I] = 1.0 * ("),
    "Interpolate copies the wrong coarse edge": ("v1 = C(m1c, J, I);", "v1 = 0.5 * C(m1c, J, I);"),
}


def _build(tmp_path, name, mutation):
    text = open(SRC).read()
    if mutation is not None:
        old, new = mutation
        assert text.count(old) == 1, f"mutation site not unique: {old}"
        text = text.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(text)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), SRC3, "-lm"], check=True)
    return oracle.bind(ctypes.CDLL(str(so)))


def _pins():
    """name -> callable returning True when the pin holds."""
    def lp_8x8():
        rng = np.random.default_rng(88)
        rho = rng.normal(size=(8, 8))
        rho -= rho.mean()
        h = 1.0 / 8
        exact = lp_ref.w1_lp(rho, h)
        res = oracle.solve_level(rho, h, oracle.NORM_L1, tol=1e-7, stop=oracle.STOP_GAP, check_every=64,
                                 max_iters=400_000, theta=1.0)
        # primal value, strong duality and dual feasibility (||grad phi||_inf <= 1) at the optimum
        return (res.status == oracle.OK and abs(res.stats.f - exact) <= 1e-6 * exact
                and abs(res.stats.dual - exact) <= 1e-5 * exact and res.stats.gmax <= 1.0 + 1e-4)

    def strip():
        rng = np.random.default_rng(5)
        n = 16
        h = 1.0 / n
        r0 = rng.uniform(0.1, 1.0, n)
        r1 = rng.uniform(0.1, 1.0, n)
        r0 /= r0.sum() * h * h
        r1 /= r1.sum() * h * h
        C = np.cumsum((r0 - r1) * h * h)
        exact = np.abs(C[:-1]).sum() * h
        res = oracle.multilevel(r0.reshape(1, n), r1.reshape(1, n), h=h, levels=1, norm=oracle.NORM_L2, tol=1e-9,
                                stop=oracle.STOP_GAP, theta=1.0, check_every=64, max_iters=2_000_000)
        return res.status == oracle.OK and abs(res.w1 - exact) <= 1e-7 * exact

    def saddle_feasible():
        rng = np.random.default_rng(7)
        n = 12
        h = 1.0 / n
        rho = rng.normal(size=n)
        rho -= rho.mean()
        C = np.cumsum(rho * h * h)
        m1 = np.zeros((1, n))
        m1[0, :-1] = C[:-1] / h
        s = oracle.stats(rho.reshape(1, n), m1, np.zeros((1, n)), rng.normal(size=(1, n)), h, oracle.NORM_L1)
        return abs(s.saddle - s.f) <= 1e-10 * s.f

    def saddle_zero_flux():
        rng = np.random.default_rng(8)
        rho = rng.normal(size=(5, 6))
        rho -= rho.mean()
        z = np.zeros((5, 6))
        s = oracle.stats(rho, z, z, rng.normal(size=(5, 6)), 0.2, oracle.NORM_L2)
        return abs(s.saddle - s.dual) <= 1e-12 * abs(s.dual)

    def restrict_mass():
        rng = np.random.default_rng(9)
        f = rng.uniform(size=(8, 6))
        return abs(oracle.restrict(f).sum() * 4.0 - f.sum()) <= 1e-12 * f.sum()

    def prolong_commutes():
        rng = np.random.default_rng(10)
        ncy, ncx = 4, 5
        m1c, m2c, phic = rng.normal(size=(3, ncy, ncx))
        m1c[:, -1] = 0.0
        m2c[-1, :] = 0.0
        hc = 0.2
        m1f, m2f, _ = oracle.prolong(m1c, m2c, phic)
        lhs = oracle.restrict(oracle.div(m1f, m2f, hc / 2))
        return np.abs(lhs - oracle.div(m1c, m2c, hc)).max() <= 1e-10

    return {"LP 8x8": lp_8x8, "1-D closed form": strip, "saddle of a feasible flux": saddle_feasible,
            "saddle of zero flux": saddle_zero_flux,
            "restriction keeps mass": restrict_mass, "Interpolate commutes with div": prolong_commutes}


@pytest.fixture
def use_lib(monkeypatch):
    def set_lib(lib):
        monkeypatch.setattr(oracle, "_lib", lib)
    return set_lib


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_unmutated_source_passes_every_pin(tmp_path, use_lib):
    use_lib(_build(tmp_path, "plain", None))
    failed = [name for name, pin in _pins().items() if not pin()]
    assert not failed, failed


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(tmp_path, use_lib, name):
    use_lib(_build(tmp_path, "mutant", MUTATIONS[name]))
    results = {}
    for pin_name, pin in _pins().items():
        try:
            results[pin_name] = bool(pin())
        except (RuntimeError, ValueError, AssertionError):
            results[pin_name] = False
    assert not all(results.values()), f"no pin caught '{name}': {results}"
