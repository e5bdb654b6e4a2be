"""The seeded synthetic inputs that both the oracle and the CUDA path take:
deterministic per seed, unit mass with the grid's cell weights, a positive floor,
the requested shapes, and distinct pairs for distinct seeds."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("workload", sorted(synth.WORKLOADS))
def test_pairs_are_deterministic_unit_mass_and_positive(workload):
    n = 64
    r0, r1 = synth.pair(workload, 3, n=n)
    s0, s1 = synth.pair(workload, 3, n=n)
    np.testing.assert_array_equal(r0, s0)
    np.testing.assert_array_equal(r1, s1)
    h = 1.0 / n
    for r in (r0, r1):
        assert r.shape == (n, n) and r.dtype == np.float64
        assert r.sum() * h * h == pytest.approx(1.0, rel=1e-12)
        assert r.min() > 0.0
    assert not np.array_equal(r0, r1)
    t0, _ = synth.pair(workload, 4, n=n)
    assert not np.array_equal(r0, t0)


def test_rectangular_grids_use_the_longer_side_for_h():
    r0, _ = synth.pair(1, 0, nx=48, ny=32)
    assert r0.shape == (32, 48)
    assert r0.sum() * (1.0 / 48) ** 2 == pytest.approx(1.0, rel=1e-12)


def test_3d_pairs():
    r0, r1 = synth.pair3(0, 2, nx=16, ny=8, nz=4)
    assert r0.shape == (4, 8, 16)
    h = 1.0 / 16
    for r in (r0, r1):
        assert r.sum() * h ** 3 == pytest.approx(1.0, rel=1e-12) and r.min() > 0.0
    a0, _ = synth.pair3(0, 2, nx=16, ny=8, nz=4)
    np.testing.assert_array_equal(a0, r0)


def test_float32_pair_is_the_same_values_widened():
    r0, r1 = synth.pair(2, 1, n=32)
    a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
    assert a0.dtype == np.float32 and d0.dtype == np.float64
    np.testing.assert_array_equal(a0.astype(np.float64), d0)
    np.testing.assert_array_equal(a1.astype(np.float64), d1)
