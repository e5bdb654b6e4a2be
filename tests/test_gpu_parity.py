"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Floating-point tolerances (FP32 iterates against FP64):
  - a few steps of eq. primaldual from the same state: max |diff| <= 2e-5 of the
    state's scale (rounding of order 1e-7 per step, non-expansive iteration);
  - full solves, oracle replaying the GPU's per-level iteration counts:
    W1 relative 1e-4, flux relative L1 1e-3 (the accuracy targets of the build);
  - FP64 statistics of the same FP32 state: relative 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402

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


def rand_state(rng, ny, nx, scale=0.5):
    m1, m2, phi = rng.normal(scale=scale, size=(3, ny, nx)).astype(np.float32)
    m1[:, -1] = 0
    m2[-1, :] = 0
    rho = rng.normal(size=(ny, nx))
    rho = (rho - rho.mean()).astype(np.float32)
    return rho, m1, m2, phi


def resident_fits(nx, ny):
    """A cluster of 1..16 CTAs, each holding whole rows, at most 4096 nodes per
    CTA (16384 when nx is a multiple of 4 and the band a multiple of 128 nodes,
    and nx <= 4096 in a cluster of several CTAs)."""
    def fits(c):
        band = (ny // c) * nx
        return ny % c == 0 and (band <= 4096 or (nx % 4 == 0 and band <= 16384 and band % 128 == 0
                                                 and (c == 1 or nx <= 4096)))
    return any(fits(c) for c in (1, 2, 4, 8, 16))


def mu_of(h, theta=0.5):
    return float(np.float32(theta * h / (2 * np.sqrt(2.0))))


def flux_rel_l1(f, m1, m2):
    return (np.abs(f[0] - m1).sum() + np.abs(f[1] - m2).sum()) / (np.abs(m1).sum() + np.abs(m2).sum())


# --------------------------------------------------------------------------------------
# Building blocks
# --------------------------------------------------------------------------------------

SHAPES = [(1, 37), (37, 1), (3, 5), (17, 33), (40, 33), (64, 64), (128, 96), (200, 300)]


SHAPES4 = [(1, 64), (3, 8), (40, 36), (64, 64), (96, 128), (200, 300), (130, 72), (512, 512), (256, 1024)]


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape", SHAPES + SHAPES4)
@pytest.mark.parametrize("path", [1, 2, 3])
def test_cp_steps_match_oracle(w1, norm, shape, path):
    """Steps of eq. primaldual from the same random state on odd shapes: 1xN and
    Nx1 strips, ragged widths, several warps and several cluster bands, tiles
    with ragged edges (path 3: 4 steps per launch)."""
    ny, nx = shape
    if path == 1 and not resident_fits(nx, ny):
        pytest.skip("larger than the resident path")
    if path == 3 and nx % 4:
        pytest.skip("temporal blocking needs nx % 4 == 0")
    rng = np.random.default_rng(ny * 1000 + nx + norm)
    rho, m1, m2, phi = rand_state(rng, ny, nx)
    h = 1.0 / max(nx, ny)
    mu = mu_of(h)
    for iters in ((4, 8, 64) if path == 3 else (1, 7, 64)):
        g = [dev(a) for a in (rho, m1, m2, phi)]
        fpr = w1.cp_steps(g[0], g[1], g[2], g[3], h, norm, mu, mu, iters, path=path)
        o1, o2, op, ofpr = oracle.cp_iterate(rho, m1, m2, phi, h, norm, iters, mu=mu, tau=mu)
        scale = max(np.abs(o1).max(), np.abs(o2).max(), np.abs(op).max(), 1.0)
        for got, want in ((g[1], o1), (g[2], o2), (g[3], op)):
            err = np.abs(host(got) - want).max()
            assert err <= 2e-5 * scale, (iters, err, scale)
        assert fpr == pytest.approx(ofpr, rel=2e-3, abs=1e-12 * scale)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape,cluster", [((64, 64), 1), ((64, 64), 16), ((128, 128), 1), ((128, 128), 2),
                                           ((128, 128), 4), ((128, 128), 8), ((256, 256), 4), ((512, 512), 16),
                                           ((96, 160), 1), ((16, 1024), 16), ((32, 4096), 16), ((64, 1024), 4),
                                           ((256, 512), 8)])
def test_resident_cluster_sizes_match_oracle(w1, norm, shape, cluster):
    """Every on-chip layout: one CTA or a cluster, four nodes per thread (up to
    4096 per CTA) or wide bands (up to 16384 per CTA, single CTA included),
    bands of one row (the halo rows above and below meet in one row), wide
    bands of two rows."""
    ny, nx = shape
    rng = np.random.default_rng(ny + nx + cluster + 10 * norm)
    rho, m1, m2, phi = rand_state(rng, ny, nx)
    h = 1.0 / max(nx, ny)
    mu = mu_of(h)
    g = [dev(a) for a in (rho, m1, m2, phi)]
    fpr = w1.cp_steps(*g, h, norm, mu, mu, 64, path=1, cluster=cluster)
    o1, o2, op, ofpr = oracle.cp_iterate(rho, m1, m2, phi, h, norm, 64, mu=mu, tau=mu)
    scale = max(np.abs(o1).max(), np.abs(o2).max(), np.abs(op).max(), 1.0)
    for got, want in ((g[1], o1), (g[2], o2), (g[3], op)):
        assert np.abs(host(got) - want).max() <= 2e-5 * scale
    assert fpr == pytest.approx(ofpr, rel=2e-3, abs=1e-12 * scale)


def test_resident_cluster_that_does_not_fit_is_refused(w1):
    g = [torch.zeros((256, 256), device="cuda") for _ in range(4)]
    with pytest.raises(w1.W1Error):
        w1.cp_steps(*g, 1 / 256, L1, 0.01, 0.01, 8, path=1, cluster=1)  # 65536 nodes in one CTA
    with pytest.raises(w1.W1Error):
        w1.cp_steps(*g, 1 / 256, L1, 0.01, 0.01, 8, path=1, cluster=3)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_resident_and_streaming_paths_agree(w1, norm):
    rng = np.random.default_rng(77)
    rho, m1, m2, phi = rand_state(rng, 96, 128)
    h = 1 / 128
    out = []
    for path in (1, 2, 3):
        g = [dev(a) for a in (rho, m1, m2, phi)]
        w1.cp_steps(*g, h, norm, mu_of(h), mu_of(h), 200, path=path)
        out.append([host(t) for t in g[1:]])
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.abs(a - b).max() <= 2e-5 * max(np.abs(b).max(), 1.0)


@pytest.mark.parametrize("shape", [(2, 2), (6, 10), (64, 64), (256, 130), (512, 512)])
def test_restrict_matches_oracle(w1, shape):
    rng = np.random.default_rng(3)
    f = rng.normal(size=shape).astype(np.float32)
    out = torch.empty((shape[0] // 2, shape[1] // 2), device="cuda")
    w1.restrict(dev(f), out)
    np.testing.assert_allclose(host(out), oracle.restrict(f.astype(np.float64)), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (3, 4), (32, 32), (64, 17)])
def test_prolong_matches_oracle(w1, shape):
    rng = np.random.default_rng(4)
    m1c, m2c, phic = rng.normal(size=(3,) + shape).astype(np.float32)
    m1c[:, -1] = 0
    m2c[-1, :] = 0
    fs = (2 * shape[0], 2 * shape[1])
    f = [torch.empty(fs, device="cuda") for _ in range(3)]
    w1.prolong(dev(m1c), dev(m2c), dev(phic), *f)
    want = oracle.prolong(m1c, m2c, phic)
    for got, ref in zip(f, want):
        np.testing.assert_allclose(host(got), ref, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape", [(1, 16), (5, 7), (64, 64), (96, 80), (32, 96), (160, 64), (512, 512)])
def test_state_stats_match_oracle(w1, norm, shape):
    """Certificate statistics of a random state against the oracle's: odd sides
    (no pooling), even sides (one route level pooled per thread), and sides that
    are multiples of 32 (route levels pooled per 32 x 32 tile, the coarse tree
    ending on a 3 x 1 grid and on a 2 x 5 grid with an odd side)."""
    rng = np.random.default_rng(5)
    rho, m1, m2, phi = rand_state(rng, *shape, scale=0.2)
    h = 1.0 / max(shape)
    g = w1.state_stats(dev(rho), dev(m1), dev(m2), dev(phi), h, norm)
    o = oracle.stats(rho, m1, m2, phi, h, norm)
    for name in ("f", "dual", "res_l1", "rho_l1", "gmax", "route", "lb", "ub", "saddle"):
        got = getattr(g, "primal" if name == "f" else name)
        assert got == pytest.approx(getattr(o, name), rel=1e-9, abs=1e-13), name
    assert g.w1 == g.saddle


# --------------------------------------------------------------------------------------
# Full solves (Algorithm 3) against the oracle replaying the GPU's iteration counts
# --------------------------------------------------------------------------------------

def solve_and_replay(w1, r0, r1, norm, levels, tol=0.0, **opt):
    a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
    ny, nx = a0.shape
    flux = torch.empty((2, ny, nx), device="cuda")
    phi = torch.empty((ny, nx), device="cuda")
    with w1.Plan(nx, ny, levels=levels, norm=norm, tol=tol, **opt) as plan:
        val, st, _ = plan.solve(dev(a0), dev(a1), flux=flux)
        plan.potential(phi)
    theta = opt.get("theta", 0.5)
    ratio = opt.get("step_ratio", 1.0)
    ref = oracle.multilevel(d0, d1, levels=levels, norm=norm, theta=theta, ratio=ratio, replay=st.iters)
    return val, st, host(flux), host(phi), ref


def assert_parity(val, st, flux, ref):
    assert st.converged
    assert val == st.w1
    assert abs(val - ref.w1) <= 1e-4 * abs(ref.w1), (val, ref.w1)
    assert flux_rel_l1(flux, ref.m1, ref.m2) <= 1e-3
    # the GPU's certificate brackets its own value consistently with the oracle's
    assert st.lb <= st.ub
    assert st.ub == pytest.approx(ref.stats.ub, rel=1e-3)


def test_solve_64_l1_three_levels(w1):
    """64x64, L1, 3-level cascade 16->32->64, FPR threshold 1e-6 on the finest level."""
    r0, r1 = synth.pair(0, 0)
    val, st, flux, phi, ref = solve_and_replay(w1, r0, r1, L1, 3, tol=1e-6)
    assert [s for s in st.sizes] == [(16, 16), (32, 32), (64, 64)]
    assert all(k % 32 == 0 and k > 0 for k in st.iters)
    assert_parity(val, st, flux, ref)
    # the potential is the oracle's (up to FP32 rounding)
    assert np.abs(phi - ref.phi).max() <= 1e-3 * max(np.abs(ref.phi).max(), 1.0)
    # free-running oracle (its own stop decisions) agrees as well
    a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
    free = oracle.multilevel(d0, d1, levels=3, norm=L1, tol=1e-6, stop=oracle.STOP_FPR)
    assert abs(val - free.w1) <= 1e-3 * free.w1
    for a, b in zip(st.iters, free.iters):
        assert abs(a - b) <= max(0.1 * b, 64)


def test_solve_64_linf_three_levels(w1):
    r0, r1 = synth.pair(0, 6)
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, LINF, 3, tol=1e-6)
    assert_parity(val, st, flux, ref)


def test_solve_256_l2_five_levels(w1):
    r0, r1 = synth.pair(1, 0)
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, L2, 5)
    assert st.sizes[0] == (16, 16) and st.sizes[-1] == (256, 256)
    assert_parity(val, st, flux, ref)


def test_cascade_against_single_level_256_l2(w1):
    """Algorithm 3 (5 levels, 16 -> 256) against Algorithm 1 from zero on one level
    with the same finest-level tolerance: far fewer finest-level steps for the
    same W1 (each stops at its own R^k < eps, so they agree to the tolerance's
    accuracy, not bitwise)."""
    r0, r1 = synth.pair(1, 0)
    a0, a1 = dev(r0), dev(r1)
    with w1.Plan(256, 256, levels=5, norm=L2) as p:
        v5, st5, _ = p.solve(a0, a1)
    with w1.Plan(256, 256, levels=1, norm=L2, max_iters=4_000_000) as p:
        v1, st1, status = p.solve(a0, a1, allow=(w1.OK, w1.ERR_NOT_CONVERGED))
    assert st5.converged
    assert st5.iters[-1] * 5 < st1.iters[0]
    if status == w1.OK:
        assert v5 == pytest.approx(v1, rel=5e-3)


@pytest.mark.parametrize("norm", [L2, L1, LINF])
def test_solve_512_six_levels(w1, norm):
    """The 512x512 image-shaped workload, 6 levels 16->512, the bench configuration."""
    r0, r1 = synth.pair(2, 0)
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, norm, 6)
    assert st.sizes[-1] == (512, 512)
    assert_parity(val, st, flux, ref)


@pytest.mark.parametrize("path", [1, 2, 3])
def test_forced_paths_give_the_same_solution(w1, path):
    r0, r1 = synth.pair(0, 1)
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, L1, 3, tol=1e-6, path=path)
    assert all(p == path for p in st.path)
    assert_parity(val, st, flux, ref)


@pytest.mark.parametrize("nx,ny,levels", [(128, 64, 3), (80, 48, 2), (33, 17, 1), (64, 1, 1), (1, 40, 1)])
def test_ragged_and_nonsquare(w1, nx, ny, levels):
    rng = np.random.default_rng(nx * ny)
    r0 = rng.uniform(0.1, 1.0, (ny, nx))
    r1 = rng.uniform(0.1, 1.0, (ny, nx))
    h = 1.0 / max(nx, ny)
    r0 /= r0.sum() * h * h
    r1 /= r1.sum() * h * h
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, L2 if nx % 2 else L1, levels, tol=1e-5)
    assert_parity(val, st, flux, ref)


def test_equal_densities_give_zero(w1):
    r0, _ = synth.pair(0, 2)
    a0 = dev(r0)
    with w1.Plan(64, 64, levels=3, norm=L1) as plan:
        val, st, _ = plan.solve(a0, a0)
    assert val == 0.0 and st.iters == [32, 32, 32]


def test_mass_imbalance_and_nonfinite_are_rejected(w1):
    r0, r1 = synth.pair(0, 3)
    with w1.Plan(64, 64, levels=3, norm=L1) as plan:
        val, st, status = plan.solve(dev(r0), dev(1.01 * r1), allow=(w1.ERR_MASS,))
        assert status == w1.ERR_MASS and np.isnan(val)
        bad = r1.copy()
        bad[5, 5] = np.inf
        _, _, status = plan.solve(dev(r0), dev(bad), allow=(w1.ERR_MASS,))
        assert status == w1.ERR_MASS
        # the plan is still usable afterwards
        val, st, status = plan.solve(dev(r0), dev(r1))
        assert status == w1.OK and val > 0


def test_shape_errors(w1):
    with pytest.raises(w1.W1Error, match="ERR_SHAPE"):
        w1.Plan(60, 64, levels=4)
    with pytest.raises(w1.W1Error, match="ERR_INVALID_ARG"):
        w1.Plan(64, 64, levels=3, norm=4)
    with pytest.raises(w1.W1Error, match="ERR_INVALID_ARG"):
        w1.Plan(64, 64, levels=3, check_every=7)
    with pytest.raises(w1.W1Error, match="ERR_INVALID_ARG"):
        w1.Plan(64, 64, levels=3, check_every=12)
    with pytest.raises(w1.W1Error, match="ERR_UNSUPPORTED"):
        w1.Plan(66, 64, levels=1, path=3)


def test_iteration_cap_and_time_budget_end_a_level(w1):
    """The device loops are bounded: an iteration cap and a wall-clock budget end
    a level with a status instead of running on."""
    r0, r1 = synth.pair(0, 4)
    for path in (1, 2, 3):
        with w1.Plan(64, 64, levels=3, norm=L1, tol=1e-12, max_iters=64, path=path) as plan:
            val, st, status = plan.solve(dev(r0), dev(r1), allow=(w1.ERR_NOT_CONVERGED,))
            assert status == w1.ERR_NOT_CONVERGED and val > 0 and not st.converged
            assert st.iters == [64, 64, 64]
        with w1.Plan(64, 64, levels=3, norm=L1, tol=1e-12, time_budget_s=1e-6, path=path) as plan:
            val, st, status = plan.solve(dev(r0), dev(r1), allow=(w1.ERR_TIMEOUT,))
            assert status == w1.ERR_TIMEOUT and val > 0
            assert all(0 < k <= 64 for k in st.iters)


def test_deterministic_and_host_entry_point(w1):
    r0, r1 = synth.pair(2, 1, n=256)
    a0, a1 = (np.ascontiguousarray(x, dtype=np.float32) for x in (r0, r1))
    with w1.Plan(256, 256, norm=L1) as plan:
        f1 = torch.empty((2, 256, 256), device="cuda")
        f2 = torch.empty_like(f1)
        v1, s1, _ = plan.solve(dev(a0), dev(a1), flux=f1)
        v2, s2, _ = plan.solve(dev(a0), dev(a1), flux=f2)
        fh = np.empty((2, 256, 256), dtype=np.float32)
        v3, s3, _ = plan.solve_host(a0, a1, flux=fh)
    assert v1 == v2 == v3 and s1.iters == s2.iters == s3.iters
    assert torch.equal(f1, f2)
    np.testing.assert_array_equal(fh, f1.cpu().numpy())


def test_caller_workspace(w1):
    r0, r1 = synth.pair(0, 5)
    with w1.Plan(64, 64, levels=3, norm=L2) as plan:
        v_own, _, _ = plan.solve(dev(r0), dev(r1))
        ws = torch.empty(plan.workspace_bytes // 4 + 64, dtype=torch.float32, device="cuda")
        plan.set_workspace(ws)
        v_ws, _, _ = plan.solve(dev(r0), dev(r1))
    assert v_own == v_ws


def test_resident_path_rejects_grids_it_cannot_hold(w1):
    g = [torch.zeros((200, 300), device="cuda") for _ in range(4)]
    with pytest.raises(w1.W1Error, match="ERR_UNSUPPORTED"):
        w1.cp_steps(*g, 1 / 300, 1, 1e-3, 1e-3, 2, path=1)


# --------------------------------------------------------------------------------------
# Batched solves
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("norm,n,levels", [(L1, 64, 3), (L2, 128, 4), (L1, 512, 6)])
def test_batch_results_equal_single_solves(w1, norm, n, levels):
    """A pair gives bitwise the same W1, flux and iteration counts alone and
    inside a batch (fixed per-pair reduction order)."""
    B = 3
    pairs = [synth.pair(2 if n == 512 else 0, 10 + k, n=n) for k in range(B)]
    a0 = np.stack([p[0] for p in pairs]).astype(np.float32)
    a1 = np.stack([p[1] for p in pairs]).astype(np.float32)
    fb = torch.empty((B, 2, n, n), device="cuda")
    with w1.Plan(n, n, levels=levels, norm=norm, batch=4) as plan:
        vals, stats, statuses, _ = plan.solve_batch(dev(a0), dev(a1), flux=fb)
    assert statuses == [w1.OK] * B
    with w1.Plan(n, n, levels=levels, norm=norm) as single:
        for k in range(B):
            f1 = torch.empty((2, n, n), device="cuda")
            v, st, _ = single.solve(dev(a0[k]), dev(a1[k]), flux=f1)
            assert v == vals[k] and st.iters == stats[k].iters
            assert torch.equal(f1, fb[k])


def test_batch_isolates_a_rejected_pair(w1):
    r = [synth.pair(0, 20 + k) for k in range(3)]
    a0 = np.stack([x[0] for x in r]).astype(np.float32)
    a1 = np.stack([x[1] for x in r]).astype(np.float32)
    a1[1] *= 1.01  # pair 1 loses mass balance
    with w1.Plan(64, 64, levels=3, norm=L1, batch=3) as plan:
        vals, stats, statuses, status = plan.solve_batch(dev(a0), dev(a1), allow=(w1.ERR_MASS,))
        assert status == w1.ERR_MASS and statuses == [w1.OK, w1.ERR_MASS, w1.OK]
        assert np.isnan(vals[1]) and vals[0] > 0 and vals[2] > 0
        with w1.Plan(64, 64, levels=3, norm=L1) as single:
            v0, _, _ = single.solve(dev(a0[0]), dev(a1[0]))
            v2, _, _ = single.solve(dev(a0[2]), dev(a1[2]))
        assert vals[0] == v0 and vals[2] == v2
        # a partial batch (fewer pairs than the plan holds) and the host entry point
        fh = np.empty((2, 2, 64, 64), dtype=np.float32)
        hv, _, hs, _ = plan.solve_batch_host(np.ascontiguousarray(a0[[0, 2]]), np.ascontiguousarray(a1[[0, 2]]),
                                             flux=fh)
        assert hv == [v0, v2] and hs == [w1.OK, w1.OK]


def test_batch_oracle_parity_512(w1):
    """Every pair of a 512x512 batch against the oracle replaying its counts (p = 2)."""
    B = 2
    pairs = [synth.pair(2, 30 + k) for k in range(B)]
    a0 = np.stack([p[0] for p in pairs]).astype(np.float32)
    a1 = np.stack([p[1] for p in pairs]).astype(np.float32)
    fb = torch.empty((B, 2, 512, 512), device="cuda")
    with w1.Plan(512, 512, levels=6, norm=L2, batch=B) as plan:
        vals, stats, _, _ = plan.solve_batch(dev(a0), dev(a1), flux=fb)
    for k in range(B):
        ref = oracle.multilevel(a0[k].astype(np.float64), a1[k].astype(np.float64), levels=6, norm=L2,
                                replay=stats[k].iters)
        assert_parity(vals[k], stats[k], host(fb[k]), ref)


@pytest.mark.parametrize("norm", [L1, L2])
def test_eager_mode_equals_graph_mode(w1, norm):
    """Launching the level kernels directly (profiling mode) runs the same
    kernels in the same order as the CUDA graph: bitwise equal results."""
    r0, r1 = synth.pair(2, 40, n=256)
    a0, a1 = dev(r0), dev(r1)
    out = []
    for eager in (0, 1):
        f = torch.empty((2, 256, 256), device="cuda")
        with w1.Plan(256, 256, norm=norm, eager=eager) as plan:
            v, st, _ = plan.solve(a0, a1, flux=f)
        out.append((v, st.iters, f))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert torch.equal(out[0][2], out[1][2])


# --------------------------------------------------------------------------------------
# Tolerance schedules (eq. tol_formula_propose, the alpha study of Sec. 6.2) and level
# counts other than the paper's L = log2(1/h) - 3 (Sec. 6.3)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,norm,levels,alpha", [(256, L2, 5, 0.0), (256, L1, 6, 0.0), (512, L2, 7, -1.0),
                                                 (128, LINF, 4, 1.0)])
def test_tolerance_schedule_and_level_count(w1, n, norm, levels, alpha):
    """eps_l = eps_L (h_l / h)^alpha on every level (checked against the formula),
    replay parity with the oracle at that schedule, and the oracle's own stop
    decisions under the same schedule land on about the same step counts."""
    workload = 1 if n == 256 else 2
    r0, r1 = synth.pair(workload, 3, n=n)
    eps_L = 1e-6 / 128 * (512.0 / n) ** 2
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, norm, levels, tol=eps_L, alpha=alpha)
    assert st.levels == levels and st.sizes[0] == (n >> (levels - 1),) * 2
    for lvl in range(levels):
        h_ratio = 2.0 ** (levels - 1 - lvl)
        assert st.tol[lvl] == pytest.approx(eps_L * h_ratio ** alpha, rel=1e-12)
    assert_parity(val, st, flux, ref)
    if n <= 256:
        a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
        free = oracle.multilevel(d0, d1, levels=levels, norm=norm, tol=eps_L, alpha=alpha, stop=oracle.STOP_FPR)
        assert abs(val - free.w1) <= 1e-4 * free.w1
        for a, b in zip(st.iters, free.iters):
            assert abs(a - b) <= max(0.1 * b, 64)


# --------------------------------------------------------------------------------------
# Tile shapes and depths of the temporally blocked kernel (picked per level by the
# autotuner or forced with w1_options.tile)
# --------------------------------------------------------------------------------------

TILES = [(1, "64x32, 4 steps"), (2, "128x16, 4"), (3, "32x64, 4"), (4, "64x32, 8"), (5, "32x32, 8")]


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("tile", [t for t, _ in TILES])
@pytest.mark.parametrize("shape", [(3, 8), (40, 36), (130, 72), (200, 300), (96, 256)])
def test_tile_variants_match_oracle(w1, norm, tile, shape):
    """Every tile variant against the oracle on ragged grids (tiles cut by the
    grid's edges, grids smaller than one tile), 8 and 16 steps."""
    ny, nx = shape
    rng = np.random.default_rng(ny * 7 + nx + 31 * tile + norm)
    rho, m1, m2, phi = rand_state(rng, ny, nx)
    h = 1.0 / max(nx, ny)
    mu = mu_of(h)
    for iters in (8, 16):
        g = [dev(a) for a in (rho, m1, m2, phi)]
        fpr = w1.cp_steps(g[0], g[1], g[2], g[3], h, norm, mu, mu, iters, path=3, cluster=tile)
        o1, o2, op, ofpr = oracle.cp_iterate(rho, m1, m2, phi, h, norm, iters, mu=mu, tau=mu)
        scale = max(np.abs(o1).max(), np.abs(o2).max(), np.abs(op).max(), 1.0)
        for got, want in ((g[1], o1), (g[2], o2), (g[3], op)):
            assert np.abs(host(got) - want).max() <= 2e-5 * scale, (iters, tile)
        assert fpr == pytest.approx(ofpr, rel=2e-3, abs=1e-12 * scale)


@pytest.mark.parametrize("tile", [2, 4, 5])
def test_plan_with_forced_tile_matches_replay(w1, tile):
    """A plan whose streaming levels all run a non-default tile (path 3 forced)
    against the oracle replaying its step counts; the tile is reported in
    stats.cluster of those levels."""
    r0, r1 = synth.pair(2, 9, n=256)
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, L2, 5, path=3, tile=tile)
    assert st.path == [3] * 5 and st.cluster == [tile] * 5
    assert_parity(val, st, flux, ref)


def test_autotuner_reports_tile_candidates(w1):
    """The tuner times every tile variant of a streaming level among its candidates."""
    best, cands = w1.autotune_level(1024, 1024, L1, objective=1, steps=64)
    tiles = sorted(c["tile"] for c in cands if c["path"] == 3)
    assert tiles == list(range(5))
    assert best["us_per_step"] == min(c["us_per_step"] for c in cands)


@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_calibrated_schedule_sets_level_tolerances(w1, norm):
    """w1_options.schedule = 1 with tol <= 0: eps_L = eq. stop_tol x the calibrated
    scale (for p = 1, 2 with stop_tol's (512 h)^2 capped at 1 on this 128^2 grid),
    eps_l = eps_L (h_l / h)^alpha and the step sizes theta / ||A_h||, all from
    w1_calibrated_schedule; the solve still meets the oracle replay."""
    r0, r1 = synth.pair(2, 4, n=128)
    scale, alpha, theta, ratio = w1.calibrated_schedule(norm)
    growth = (512.0 / 128) ** 2 if norm == LINF else 1.0
    eps_L = 1e-6 / 128 * growth * scale
    # the schedule sets the plan's theta and step ratio; the same go to the oracle replay
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, norm, 4, schedule=1, theta=theta, step_ratio=ratio)
    for lvl in range(4):
        assert st.tol[lvl] == pytest.approx(eps_L * (2.0 ** (3 - lvl)) ** alpha, rel=1e-12)
    assert_parity(val, st, flux, ref)


@pytest.mark.parametrize("norm,ratio", [(L1, 0.25), (L2, 4.0), (LINF, 2.0)])
def test_step_ratio_matches_replay(w1, norm, ratio):
    """Unequal step sizes (tau / mu = ratio at mu tau = (theta / ||A_h||)^2) on every
    level against the oracle replaying the same steps."""
    r0, r1 = synth.pair(2, 6, n=128)
    val, st, flux, _, ref = solve_and_replay(w1, r0, r1, norm, 4, step_ratio=ratio)
    assert_parity(val, st, flux, ref)
