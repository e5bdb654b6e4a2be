"""Autotuner: it measures every configuration that can run a level, picks the
fastest for the batch it is asked about, and plans built on its choices solve
like the oracle."""
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


@pytest.mark.parametrize("n", [32, 128, 512])
@pytest.mark.parametrize("objective,batch", [(1, 1), (2, 1), (2, 48), (3, 1)])
def test_autotune_picks_the_fastest_candidate(w1, n, objective, batch):
    best, cands = w1.autotune_level(n, n, 1, objective, steps=64, batch=batch)
    assert len(cands) >= 3
    paths = {c["path"] for c in cands}
    assert {2, 3} <= paths  # both streaming kernels are always candidates here
    assert 1 in paths  # and every grid here fits on chip
    if objective == 3:  # least SM-time: time x CTAs on chip, time x all SMs when streaming
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        cost = lambda c: c["us_per_step"] * (c["cluster"] if c["path"] == 1 else sms)  # noqa: E731
        assert cost(best) == min(cost(c) for c in cands)
    else:
        assert best["us_per_step"] == min(c["us_per_step"] for c in cands)
    assert all(c["us_per_step"] > 0 for c in cands)
    assert all(c["batch"] == (batch if objective == 2 else 1) for c in cands)


def test_autotune_rejects_bad_arguments(w1):
    with pytest.raises(w1.W1Error):
        w1.autotune_level(64, 64, 4)
    with pytest.raises(w1.W1Error):
        w1.autotune_level(64, 64, 1, objective=4)
    with pytest.raises(w1.W1Error):
        w1.autotune_level(64, 64, 1, batch=0)


@pytest.mark.parametrize("tune,batch", [(1, 1), (2, 1), (2, 3), (3, 1)])
def test_tuned_plan_solves_like_the_oracle(w1, tune, batch):
    pairs = [synth.pair(2, 50 + k, n=256) for k in range(batch)]
    a0 = np.ascontiguousarray(np.stack([p[0] for p in pairs]), dtype=np.float32)
    a1 = np.ascontiguousarray(np.stack([p[1] for p in pairs]), dtype=np.float32)
    flux = torch.empty((batch, 2, 256, 256), device="cuda")
    with w1.Plan(256, 256, norm=1, tune=tune, batch=batch) as plan:
        vals, sts, _, _ = plan.solve_batch(torch.from_numpy(a0).cuda(), torch.from_numpy(a1).cuda(), flux=flux)
    for k in range(batch):
        v, st = vals[k], sts[k]
        ref = oracle.multilevel(a0[k].astype(np.float64), a1[k].astype(np.float64), levels=st.levels, norm=1,
                                replay=st.iters)
        assert st.converged and abs(v - ref.w1) <= 1e-4 * ref.w1
        f = flux[k].cpu().numpy().astype(np.float64)
        rel = (np.abs(f[0] - ref.m1).sum() + np.abs(f[1] - ref.m2).sum()) / \
            (np.abs(ref.m1).sum() + np.abs(ref.m2).sum())
        assert rel <= 1e-3
