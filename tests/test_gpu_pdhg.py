"""GPU parity of the prox-PDHG path (Algorithms 2 and 4) against the FP64
oracle: the Neumann Poisson solve, steps of eq. pdhg from the same state, and
full multilevel solves with the oracle replaying the GPU's step counts.

Tolerances: the Poisson solve carries FP32 FFT rounding (about log2(n) * 6e-8
relative): 2e-5 of the solution's scale; a few steps from the same state: 5e-5
of the state's scale (the iteration is non-expansive); full solves as the other
full solves (W1 relative 1e-4, flux relative L1 1e-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import pdhg as opd  # noqa: E402

L1, L2, LINF = 1, 2, 3


@pytest.fixture(scope="module")
def w1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_00118_gb300 import w1 as mod
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", [(2, 2), (4, 8), (16, 16), (64, 32), (8, 1024), (512, 512), (1024, 1024)])
def test_poisson_matches_oracle(w1, shape):
    ny, nx = shape
    rng = np.random.default_rng(nx + 7 * ny)
    h = 1.0 / max(nx, ny)
    r = rng.normal(size=shape).astype(np.float32)
    psi = torch.empty(shape, device="cuda")
    w1.poisson(dev(r), psi, h)
    want = opd.poisson(r.astype(np.float64), h)
    assert np.abs(host(psi) - want).max() <= 2e-5 * np.abs(want).max()


def test_poisson_rejects_other_sizes(w1):
    z = torch.zeros((12, 16), device="cuda")
    with pytest.raises(w1.W1Error):
        w1.poisson(z, z, 1 / 16)


def rand_state(rng, ny, nx):
    m1, m2, f1, f2, g1, g2 = (rng.normal(scale=0.5, size=(6, ny, nx))).astype(np.float32)
    m1[:, -1] = m2[-1, :] = 0
    f1[:, -1] = f2[-1, :] = 0
    g1[:, -1] = g2[-1, :] = 0
    rho = rng.normal(size=(ny, nx))
    rho = (rho - rho.mean()).astype(np.float32)
    return rho, [m1, m2, f1, f2, g1, g2]


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape", [(8, 8), (16, 32), (64, 64), (128, 256)])
def test_pdhg_steps_match_oracle(w1, norm, shape):
    ny, nx = shape
    rng = np.random.default_rng(ny * 100 + nx + norm)
    rho, st = rand_state(rng, ny, nx)
    h = 1.0 / max(nx, ny)
    for iters in (1, 5, 40):
        g = [dev(a) for a in st]
        G = w1.pdhg_steps(dev(rho), *g, h, norm, iters)
        s = opd.State(*(a.astype(np.float64) for a in st))
        Gref = 0.0
        for _ in range(iters):
            s, Gref = opd.step(rho.astype(np.float64), s, h, norm, 0.5, 0.5)
        want = [s.m1, s.m2, s.f1, s.f2, s.g1, s.g2]
        scale = max(max(np.abs(x).max() for x in want), 1.0)
        for got, ref in zip(g, want):
            assert np.abs(host(got) - ref).max() <= 5e-5 * scale, iters
        assert G == pytest.approx(Gref, rel=2e-3, abs=1e-10)


def flux_rel_l1(f, m1, m2):
    return (np.abs(f[0] - m1).sum() + np.abs(f[1] - m2).sum()) / (np.abs(m1).sum() + np.abs(m2).sum())


def alg4_solve(w1, workload, k, n, norm, **opt):
    r0, r1 = synth.pair(workload, k, n=n)
    a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
    flux = torch.empty((2, n, n), device="cuda")
    phi = torch.empty((n, n), device="cuda")
    with w1.Plan(n, n, norm=norm, algorithm=4, **opt) as plan:
        val, st, _ = plan.solve(dev(a0), dev(a1), flux=flux)
        plan.potential(phi)
    ref = opd.multilevel(d0, d1, levels=st.levels, norm=norm, replay=st.iters)
    return val, st, host(flux), host(phi), ref


@pytest.mark.parametrize("norm,workload,n", [(L1, 0, 64), (L2, 1, 256), (LINF, 0, 64), (L1, 2, 512), (L2, 2, 512)])
def test_algorithm4_solve_matches_oracle_replay(w1, norm, workload, n):
    val, st, flux, phi, ref = alg4_solve(w1, workload, 3, n, norm)
    assert st.converged
    assert all(p == 4 for p in st.path)
    assert abs(val - ref.w1) <= 1e-4 * abs(ref.w1), (val, ref.w1, st.iters)
    assert flux_rel_l1(flux, ref.m1, ref.m2) <= 1e-3
    # the potential of Appendix B matches and brackets W1 with the flux
    assert np.abs(phi - ref.phi).max() <= 1e-3 * np.abs(ref.phi).max()
    assert st.lb <= st.ub


def test_algorithm4_default_tolerance_is_the_papers(w1):
    _, st, _, _, _ = alg4_solve(w1, 2, 1, 512, L1)
    # eq. stop_tol for Alg. 4 at h = 1/512: eps_L = 1e-4 / 32, eps_l = eps_L (h_l / h)^-1
    assert st.tol[-1] == pytest.approx(1e-4 / 32)
    assert st.tol[0] == pytest.approx(1e-4 / 32 / 32)
    assert all(f < t for f, t in zip(st.fpr, st.tol))


def test_algorithm4_batch_equals_single_and_eager_equals_graph(w1):
    pairs = [synth.pair(2, 20 + k, n=128) for k in range(3)]
    a0 = np.ascontiguousarray(np.stack([p[0] for p in pairs]), dtype=np.float32)
    a1 = np.ascontiguousarray(np.stack([p[1] for p in pairs]), dtype=np.float32)
    with w1.Plan(128, 128, norm=L1, algorithm=4, batch=3) as plan:
        vb, sb, _, _ = plan.solve_batch(dev(a0), dev(a1))
    for k in range(3):
        for eager in (0, 1):
            with w1.Plan(128, 128, norm=L1, algorithm=4, eager=eager) as plan:
                v, s, _ = plan.solve(dev(a0[k]), dev(a1[k]))
            assert v == vb[k] and s.iters == sb[k].iters


def test_algorithm4_rejects_other_sizes(w1):
    with pytest.raises(w1.W1Error):
        w1.Plan(96, 96, algorithm=4)
    with pytest.raises(w1.W1Error):
        w1.Plan(64, 64, algorithm=5)
