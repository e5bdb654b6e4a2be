"""Mixed-size batches: classes whose levels fit one CTA run in one persistent
launch (every level of a pair on one CTA); when a class has a level that needs
a cluster of four CTAs, that launch runs in clusters (those pairs on a whole
cluster, the others on one CTA each); classes that fit neither run as batched
plans beside it.  Each pair is checked against the FP64 oracle replaying its
step counts (W1 relative 1e-4, as the other full solves)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402


@pytest.fixture(scope="module")
def w1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_00118_gb300 import w1 as mod
    return mod


def make(classes, seed0=0):
    r0, r1, host = [], [], []
    for ci, (nx, ny, cnt) in enumerate(classes):
        pairs = [synth.pair(3, seed0 + 1000 * ci + k, nx=nx, ny=ny) for k in range(cnt)]
        a0 = np.ascontiguousarray(np.stack([p[0] for p in pairs]), dtype=np.float32)
        a1 = np.ascontiguousarray(np.stack([p[1] for p in pairs]), dtype=np.float32)
        host.append((a0, a1))
        r0.append(torch.from_numpy(a0).cuda())
        r1.append(torch.from_numpy(a1).cuda())
    return r0, r1, host


def solve(w1, classes, norm, **opt):
    r0, r1, host = make(classes)
    with w1.Mixed(classes, norm=norm, **opt) as mx:
        mx.solve_async(r0, r1)
        torch.cuda.synchronize()
        out = [mx.results(c) for c in range(len(classes))]
        pers = [mx.persistent(c) for c in range(len(classes))]
        info = mx.launch_info()
    # launch sizes: the coarse launch whenever some persistent class has levels of at
    # most 1024 nodes; clusters when a persistent class needs them, else single CTAs
    if any(pers):
        assert info["coarse_ctas"] > 0
        big = any(p and nx * ny > 16384 for p, (nx, ny, _) in zip(pers, classes))
        assert (info["clusters"] > 0) == big
        assert info["clusters"] > 0 or info["ctas"] > 0
    else:
        assert info == {"ctas": 0, "clusters": 0, "coarse_ctas": 0}
    return out, pers, host


@pytest.mark.parametrize("norm", [1, 2, 3])
def test_mixed_batch_matches_the_oracle(w1, norm):
    """The 256^2 class makes the persistent launch a cluster launch: its pairs
    run on four-CTA clusters (128^2 and 256^2 levels split in row bands), the
    other classes one pair per CTA in the same launch."""
    classes = [(64, 64, 5), (128, 128, 3), (32, 32, 4), (256, 256, 2)]
    out, pers, host = solve(w1, classes, norm)
    assert pers == [True, True, True, True]
    for ci, (vals, sts, statuses, _) in enumerate(out):
        a0, a1 = host[ci]
        for k, (v, st) in enumerate(zip(vals, sts)):
            assert statuses[k] == w1.OK and st.converged
            ref = oracle.multilevel(a0[k].astype(np.float64), a1[k].astype(np.float64), levels=st.levels, norm=norm,
                                    replay=st.iters)
            assert abs(v - ref.w1) <= 1e-4 * abs(ref.w1), (ci, k, v, ref.w1)
            assert st.lb <= st.ub


def test_cluster_launch_without_single_cta_classes(w1):
    """Only cluster classes (256^2 and a 128 x 512 grid whose 512-wide levels
    split in four row bands): the launch's second phase finds no work."""
    classes = [(256, 256, 3), (512, 128, 1)]
    out, pers, host = solve(w1, classes, 1)
    assert pers == [True, True]
    for ci, (vals, sts, statuses, _) in enumerate(out):
        a0, a1 = host[ci]
        for k, (v, st) in enumerate(zip(vals, sts)):
            assert statuses[k] == w1.OK and st.converged
            ref = oracle.multilevel(a0[k].astype(np.float64), a1[k].astype(np.float64), levels=st.levels, norm=1,
                                    replay=st.iters)
            assert abs(v - ref.w1) <= 1e-4 * abs(ref.w1), (ci, k, v, ref.w1)


def test_cluster_launch_rejects_a_bad_pair_alone(w1):
    """A rejected pair of a cluster class is skipped by its cluster; the others
    (cluster and single-CTA classes) are unaffected."""
    classes = [(256, 256, 3), (64, 64, 2)]
    r0, r1, host = make(classes, seed0=91)
    r1[0][1] *= 1.5
    with w1.Mixed(classes, norm=2) as mx:
        mx.solve_async(r0, r1)
        torch.cuda.synchronize()
        assert [mx.persistent(c) for c in range(2)] == [True, True]
        vals, sts, statuses, _ = mx.results(0)
        assert statuses == [w1.OK, w1.ERR_MASS, w1.OK]
        assert np.isnan(vals[1]) and np.isfinite(vals[0]) and np.isfinite(vals[2])
        _, _, st1, _ = mx.results(1)
        assert st1 == [w1.OK, w1.OK]


def test_persistent_launch_equals_the_batched_plan_with_the_same_kernels(w1):
    """A 64^2 class (every level on one CTA in both) gives the same bits in the
    persistent launch and in a batched plan."""
    classes = [(64, 64, 6)]
    out, pers, host = solve(w1, classes, 1)
    assert pers == [True]
    a0, a1 = host[0]
    with w1.Plan(64, 64, norm=1, batch=6) as plan:
        vals, sts, _, _ = plan.solve_batch(torch.from_numpy(a0).cuda(), torch.from_numpy(a1).cuda(),
                                           allow=(w1.OK, w1.ERR_NOT_CONVERGED))
    assert out[0][0] == vals
    assert [s.iters for s in out[0][1]] == [s.iters for s in sts]


def test_mixed_batch_rejects_a_bad_pair_alone(w1):
    classes = [(64, 64, 3), (32, 32, 2)]
    r0, r1, host = make(classes, seed0=77)
    r1[0][1] *= 1.5  # mass mismatch in class 0, pair 1
    with w1.Mixed(classes, norm=1) as mx:
        mx.solve_async(r0, r1)
        torch.cuda.synchronize()
        vals, sts, statuses, _ = mx.results(0)
        assert statuses == [w1.OK, w1.ERR_MASS, w1.OK]
        assert np.isnan(vals[1]) and np.isfinite(vals[0]) and np.isfinite(vals[2])
        vals1, _, st1, _ = mx.results(1)
        assert st1 == [w1.OK, w1.OK]


def test_mixed_batch_path_option_sends_every_class_to_plans(w1):
    classes = [(64, 64, 2), (32, 32, 2)]
    out, pers, host = solve(w1, classes, 1, path=2)
    assert pers == [False, False]
    for ci, (vals, sts, statuses, _) in enumerate(out):
        assert all(s == w1.OK for s in statuses)


def test_mixed_batch_bad_arguments(w1):
    with pytest.raises(w1.W1Error):
        w1.Mixed([(64, 64, 0)])
    with pytest.raises(w1.W1Error):
        w1.Mixed([(64, 64, 1)], norm=4)
