"""Serving loop (continuous batching) on the GPU: every request's result is the
same alone and inside a mix of other requests of mixed sizes and norms; the
HBM budget rejects requests that cannot fit and evicts idle slots."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


@pytest.fixture(scope="module")
def w1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_00118_gb300 import w1 as mod
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def make_requests(n_each=3):
    reqs = []
    for size, norm in ((64, 1), (128, 2), (256, 1), (128, 1), (64, 2)):
        for k in range(n_each):
            r0, r1 = synth.pair(2, 500 + 10 * size + k, n=size)
            reqs.append((dev(r0), dev(r1), norm))
    return reqs


@pytest.mark.parametrize("max_batch", [1, 4])
def test_results_same_alone_and_in_the_mix(w1, max_batch):
    target0, target1 = (dev(x) for x in synth.pair(2, 777, n=128))
    with w1.Plan(128, 128, norm=1) as plan:
        ref, ref_st, _ = plan.solve(target0, target1)
    with w1.Server(max_slots=8, max_batch=max_batch) as srv:
        t = srv.submit(target0, target1, norm=1)
        st, alone, alone_st = srv.wait(t, 120)
        assert st == w1.OK
        mix = make_requests()
        tickets = []
        for k, (a, b, norm) in enumerate(mix):
            tickets.append(srv.submit(a, b, norm=norm))
            if k == 7:
                tx = srv.submit(target0, target1, norm=1)
        results = {tk: srv.wait(tk, 300) for tk in tickets}
        st2, in_mix, mix_st = srv.wait(tx, 300)
        info = srv.info()
    assert st2 == w1.OK and all(r[0] == w1.OK for r in results.values())
    assert alone == ref and in_mix == ref
    assert alone_st.iters == ref_st.iters == mix_st.iters
    assert info["completed"] == len(mix) + 2
    # every mixed request agrees with a plain solve of the same pair
    for (a, b, norm), tk in list(zip(mix, tickets))[::4]:
        n = a.shape[0]
        with w1.Plan(n, n, norm=norm) as p:
            v, _, _ = p.solve(a, b)
        assert results[tk][1] == v


def test_latency_slots_agree_within_tolerance(w1):
    """latency_below > 0: a lone request runs on a slot whose kernels the
    autotuner picked for one solve, requests under load on the configured slots;
    either way W1 agrees with a plain solve to 1e-4 (the kernels differ only in
    FP32 rounding order)."""
    target0, target1 = (dev(x) for x in synth.pair(2, 778, n=128))
    with w1.Plan(128, 128, norm=1) as plan:
        ref, _, _ = plan.solve(target0, target1)
    with w1.Server(max_slots=8, latency_below=2) as srv:
        st, alone, _ = srv.wait(srv.submit(target0, target1, norm=1), 120)
        assert st == w1.OK
        mix = make_requests(2)
        tickets = [srv.submit(a, b, norm=norm) for a, b, norm in mix]
        tx = srv.submit(target0, target1, norm=1)
        results = {tk: srv.wait(tk, 300) for tk in tickets}
        st2, in_mix, _ = srv.wait(tx, 300)
    assert st2 == w1.OK and all(r[0] == w1.OK for r in results.values())
    assert alone == pytest.approx(ref, rel=1e-4) and in_mix == pytest.approx(ref, rel=1e-4)
    for (a, b, norm), tk in list(zip(mix, tickets))[::3]:
        n = a.shape[0]
        with w1.Plan(n, n, norm=norm) as p:
            v, _, _ = p.solve(a, b)
        assert results[tk][1] == pytest.approx(v, rel=1e-4)


def test_budget_rejects_and_evicts(w1):
    small = w1.plan_bytes(64, 64, norm=1) + 2 * 64 * 64 * 4
    with w1.Server(hbm_budget_bytes=small + 1024, max_slots=4) as srv:
        big0, big1 = (dev(x) for x in synth.pair(2, 1, n=256))
        with pytest.raises(w1.W1Error, match="ERR_BUDGET"):
            srv.submit(big0, big1)
        # two size classes that cannot both be resident: the idle one is evicted
        a0, a1 = (dev(x) for x in synth.pair(0, 1, n=64))
        b0, b1 = (dev(x) for x in synth.pair(0, 2, n=64))
        t1 = srv.submit(a0, a1, norm=1)
        t2 = srv.submit(b0, b1, norm=2)
        assert srv.wait(t1, 120)[0] == w1.OK
        assert srv.wait(t2, 120)[0] == w1.OK
        info = srv.info()
        assert info["evictions"] >= 1 and info["bytes_in_use"] <= small + 1024


def test_poll_and_unknown_ticket(w1):
    with w1.Server(max_slots=2) as srv:
        a0, a1 = (dev(x) for x in synth.pair(0, 3, n=64))
        t = srv.submit(a0, a1)
        st = w1.PENDING
        import time
        end = time.time() + 120
        while st == w1.PENDING and time.time() < end:
            st, v, stats, lat = srv.poll(t)
        assert st == w1.OK and v > 0 and lat > 0
        st, *_ = srv.poll(t)  # already collected
        assert st == w1.ERR_INVALID_ARG
