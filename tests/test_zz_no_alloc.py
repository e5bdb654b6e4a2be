"""w1_state_stats_noalloc: certificate statistics for callers that cannot
allocate device memory (loops that must not pay cudaMalloc's implicit device
synchronisation, frameworks that own all device memory through their own
pools, services with a fixed preallocated footprint).  Its scratch is a static
device array; this test calls it through the C ABI and checks it against
w1_state_stats, several calls in a row with different grids and norms, so that
the contents a previous call left behind cannot leak into the next result.

Collected last on purpose (file name), so a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("w1", "primal", "saddle", "dual", "res_l1", "rho_l1", "gmax", "route", "lb", "ub")


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_00118_gb300 import w1
    return w1


def _state(rng, ny, nx):
    m1, m2, phi = rng.normal(scale=0.3, size=(3, ny, nx)).astype(np.float32)
    m1[:, -1] = 0
    m2[-1, :] = 0
    rho = rng.normal(size=(ny, nx))
    rho = (rho - rho.mean()).astype(np.float32)
    return [torch.from_numpy(a).cuda() for a in (rho, m1, m2, phi)]


def _call(fn, t, nx, ny, h, norm, stream):
    out = __import__("paper_1810_00118_gb300").w1._Stats()
    ptr = [ctypes.c_void_p(x.data_ptr()) for x in t]
    status = fn(nx, ny, h, norm, *ptr, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
    return status, out


def test_noalloc_stats_match_allocating_stats_two_calls_in_a_row():
    w1 = _lib()
    lib = w1.lib()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(2024)
    # a large grid first, then smaller ones: no call may see an earlier call's
    # leftovers; every norm; the maximum size as a square, a 1 x N strip and a
    # non-square grid; odd sides (the dyadic route of the bound stops early)
    for (ny, nx), norm in (((512, 512), 1), ((96, 80), 2), ((1, 262144), 3), ((1024, 256), 2), ((37, 53), 3),
                           ((256, 1024), 1), ((5, 7), 2)):
        t = _state(rng, ny, nx)
        h = 1.0 / max(nx, ny)
        s_ref, ref = _call(lib.w1_state_stats, t, nx, ny, h, norm, stream)
        s_new, new = _call(lib.w1_state_stats_noalloc, t, nx, ny, h, norm, stream)
        assert s_ref == 0 and s_new == 0, lib.w1_noalloc_last_error()
        for f in FIELDS:
            assert getattr(new, f) == pytest.approx(getattr(ref, f), rel=1e-9, abs=1e-13), f


def test_noalloc_rejects_grids_above_its_limit():
    w1 = _lib()
    lib = w1.lib()
    stream = torch.cuda.current_stream()
    t = [torch.zeros((520, 520), device="cuda") for _ in range(4)]
    status, _ = _call(lib.w1_state_stats_noalloc, t, 520, 520, 1 / 520, 1, stream)
    assert status == w1.ERR_INVALID_ARG
    assert b"262144" in lib.w1_noalloc_last_error()
