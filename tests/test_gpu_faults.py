"""Failure handling of the on-chip cluster levels, without a GPU fault: the
host makes one CTA of every cluster skip its halo pushes (W1_FAULT_HALO_RANK,
read when a plan is built); its neighbours' bounded waits run out, the level
ends at its next stop test with a timeout status, and the context stays usable
for the next solve."""
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


# (grid side, levels): 128^2 finest level on a 4-CTA cluster (four nodes per
# thread); 512^2 on a 16-CTA cluster of wide bands
@pytest.mark.parametrize("n,levels", [(128, 2), (512, 1)])
def test_dropped_halo_ends_in_timeout_and_recovers(w1, monkeypatch, n, levels):
    r0, r1 = (dev(x) for x in synth.pair(2, 9, n=n))
    monkeypatch.setenv("W1_FAULT_HALO_RANK", "1")
    with w1.Plan(n, n, levels=levels, norm=1) as plan:
        _, st, status = plan.solve(r0, r1, allow=(w1.ERR_TIMEOUT,))
    assert status == w1.ERR_TIMEOUT and not st.converged
    assert st.path[-1] == 1 and st.cluster[-1] > 1
    assert 0 < st.iters[-1] <= 64  # stopped at the first or second stop test
    monkeypatch.delenv("W1_FAULT_HALO_RANK")
    with w1.Plan(n, n, levels=levels, norm=1) as plan:
        v, st2, status2 = plan.solve(r0, r1, allow=(w1.OK, w1.ERR_NOT_CONVERGED))
    assert status2 == w1.OK and st2.converged and np.isfinite(v) and v > 0
