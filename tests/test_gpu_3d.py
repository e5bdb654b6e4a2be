"""GPU parity of Algorithm 3 on 3-D grids: the CUDA path (through the C ABI)
against the FP64 3-D oracle.

Floating-point tolerances (FP32 iterates against FP64), as for 2-D grids:
  - a few steps of eq. primaldual from the same state: max |diff| <= 2e-5 of the
    state's scale; R^k of the last step relative 1e-3 (a sum of squared
    differences of FP32 iterates);
  - restriction: relative 1e-6 (a mean of eight FP32 values); Interpolate:
    absolute 1e-6 of the coarse state's scale;
  - full solves, the oracle replaying the GPU's per-level iteration counts:
    W1 relative 1e-4, flux relative L1 1e-3;
  - FP64 certificates of the returned FP32 state: relative 1e-9 (f, dual,
    gmax), 1e-7 (residual sums, which rounding of rho to FP32 can move).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import d3  # noqa: E402

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


def rand_state3(rng, nz, ny, nx, scale=0.5):
    m1, m2, m3, phi = rng.normal(scale=scale, size=(4, nz, ny, nx)).astype(np.float32)
    m1[..., -1] = 0
    m2[:, -1, :] = 0
    m3[-1] = 0
    rho = rng.normal(size=(nz, ny, nx))
    rho = (rho - rho.mean()).astype(np.float32)
    return rho, m1, m2, m3, phi


def mu3(h, theta=0.5):
    return float(np.float32(theta * h / (2 * np.sqrt(3.0))))


# (nz, ny, nx): one block, ragged tails, several blocks, strips along each axis
SHAPES3 = [(1, 1, 1), (2, 3, 5), (9, 10, 11), (16, 16, 16), (3, 40, 33), (1, 1, 300), (1, 300, 1), (300, 1, 1),
           (33, 17, 64)]


@pytest.mark.parametrize("path", [2, 3])
@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape", SHAPES3)
def test_cp_steps3d_match_oracle(w1, norm, shape, path):
    """Streamed steps, two launches (path 2) or one (path 3) per step, against the
    oracle: 7 steps (an odd count, so the one-launch step copies its state back)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(nx * 10007 + ny * 101 + nz + norm)
    rho, m1, m2, m3, phi = rand_state3(rng, nz, ny, nx)
    h = 1.0 / max(shape)
    mu = mu3(h)
    t = [dev(a) for a in (rho, m1, m2, m3, phi)]
    steps = 7
    r = w1.cp_steps3d(*t, h, norm, mu, mu, steps, path=path)
    o1, o2, o3, op, rf = d3.cp_iterate(rho.astype(np.float64), m1, m2, m3, phi, h, norm, steps, mu=mu, tau=mu)
    for got, want in zip(t[1:], (o1, o2, o3, op)):
        g = host(got)
        scale = max(1.0, np.abs(want).max())
        assert np.abs(g - want).max() <= 2e-5 * scale
    assert r == pytest.approx(rf, rel=1e-3, abs=1e-12)
    # the pinned faces stay zero
    assert not host(t[1])[..., -1].any() and not host(t[2])[:, -1, :].any() and not host(t[3])[-1].any()


# (shape, cluster): one CTA, clusters of 2..16 slabs (one-plane slabs included)
RESIDENT3 = [((1, 1, 4), 1), ((2, 3, 8), 1), ((8, 8, 8), 1), ((16, 16, 16), 1), ((4, 12, 16), 2), ((4, 12, 16), 4),
             ((32, 32, 32), 8), ((32, 32, 32), 16), ((16, 16, 16), 16), ((2, 40, 32), 2), ((16, 8, 64), 4),
             # wide slabs (up to 16384 voxels per CTA, own state in tensor memory)
             ((8, 32, 64), 1), ((32, 32, 32), 4), ((64, 64, 64), 16), ((16, 64, 64), 4), ((48, 48, 48), 16)]


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape,cluster", RESIDENT3)
def test_onchip_steps3d_match_oracle(w1, norm, shape, cluster):
    """Every step of a level in one launch (one CTA or a cluster of slabs whose
    halo planes move between CTAs): 40 steps against the oracle; R^k of the last."""
    nz, ny, nx = shape
    rng = np.random.default_rng(nx * 131 + ny * 17 + nz + cluster + 7 * norm)
    rho, m1, m2, m3, phi = rand_state3(rng, nz, ny, nx)
    h = 1.0 / max(shape)
    mu = mu3(h)
    t = [dev(a) for a in (rho, m1, m2, m3, phi)]
    steps = 40
    r = w1.cp_steps3d(*t, h, norm, mu, mu, steps, path=1, cluster=cluster)
    o1, o2, o3, op, rf = d3.cp_iterate(rho.astype(np.float64), m1, m2, m3, phi, h, norm, steps, mu=mu, tau=mu)
    for got, want in zip(t[1:], (o1, o2, o3, op)):
        scale = max(1.0, np.abs(want).max())
        assert np.abs(host(got) - want).max() <= 2e-5 * scale
    assert r == pytest.approx(rf, rel=2e-3, abs=1e-12)


def test_onchip_steps3d_refuses_what_does_not_fit(w1):
    g = [torch.zeros((32, 32, 32), device="cuda") for _ in range(5)]
    with pytest.raises(w1.W1Error):
        w1.cp_steps3d(*g, 1 / 32, L1, 0.01, 0.01, 8, path=1, cluster=1)  # 32768 voxels in one CTA
    g = [torch.zeros((4, 4, 6), device="cuda") for _ in range(5)]
    with pytest.raises(w1.W1Error):
        w1.cp_steps3d(*g, 1 / 6, L1, 0.01, 0.01, 8, path=1)  # nx % 4 != 0


@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 6, 8), (8, 34, 66), (64, 64, 64)])
def test_restrict3d_matches_oracle(w1, shape):
    rng = np.random.default_rng(sum(shape))
    fine = rng.normal(size=shape).astype(np.float32)
    out = torch.empty(tuple(s // 2 for s in shape), device="cuda")
    w1.restrict3d(dev(fine), out)
    torch.cuda.synchronize()
    want = d3.restrict(fine.astype(np.float64))
    np.testing.assert_allclose(host(out), want, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("cshape", [(1, 1, 1), (1, 2, 3), (3, 4, 5), (8, 17, 33), (32, 32, 32)])
def test_prolong3d_matches_oracle(w1, cshape):
    rng = np.random.default_rng(7 * sum(cshape))
    m1c, m2c, m3c, pc = rng.normal(size=(4,) + cshape).astype(np.float32)
    m1c[..., -1] = 0
    m2c[:, -1, :] = 0
    m3c[-1] = 0
    fs = tuple(2 * s for s in cshape)
    f = [torch.empty(fs, device="cuda") for _ in range(4)]
    w1.prolong3d(dev(m1c), dev(m2c), dev(m3c), dev(pc), *f)
    torch.cuda.synchronize()
    want = d3.prolong(m1c, m2c, m3c, pc)
    for g, w in zip(f, want):
        assert np.abs(host(g) - w).max() <= 1e-6 * max(1.0, np.abs(w).max())


# --------------------------------------------------------------------------------------
# Full solves against the oracle replaying the GPU's iteration counts
# --------------------------------------------------------------------------------------

def solve3_and_replay(w1, r0, r1, norm, levels, tol=0.0, **opt):
    a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
    nz, ny, nx = a0.shape
    flux = torch.empty((3, nz, ny, nx), device="cuda")
    phi = torch.empty((nz, ny, nx), device="cuda")
    val, st, status = w1.solve3d(dev(a0), dev(a1), norm=norm, levels=levels, tol=tol, flux=flux, potential=phi, **opt)
    theta = opt.get("theta", 0.5)
    ref = d3.multilevel(d0, d1, levels=st.levels, norm=norm, theta=theta, replay=st.iters)
    return val, st, status, host(flux), host(phi), ref


def flux3_rel_l1(f, ref):
    num = sum(np.abs(f[c] - w).sum() for c, w in enumerate((ref.m1, ref.m2, ref.m3)))
    return num / sum(np.abs(w).sum() for w in (ref.m1, ref.m2, ref.m3))


@pytest.mark.parametrize("path", [0, 2, 3])
@pytest.mark.parametrize("norm", [L1, L2, LINF])
def test_solve3d_16_two_levels(w1, norm, path):
    """16^3, two levels 8^3 -> 16^3, default tolerance of eq. stop_tol; both
    levels on chip (path 0), two launches per step (path 2) or one (path 3)."""
    r0, r1 = synth.pair3(16, norm)
    val, st, status, flux, phi, ref = solve3_and_replay(w1, r0, r1, norm, 2, path=path)
    assert status == w1.OK and st.converged
    assert st.levels == 2 and st.sizes == [(8, 8), (16, 16)]
    assert st.path == ([1, 1] if path == 0 else [path, path])
    assert all(k % 32 == 0 and k > 0 for k in st.iters)
    assert val == st.w1
    assert abs(val - ref.w1) <= 1e-4 * abs(ref.w1), (val, ref.w1)
    assert flux3_rel_l1(flux, ref) <= 1e-3
    assert np.abs(phi - ref.phi).max() <= 1e-3 * max(np.abs(ref.phi).max(), 1.0)
    assert st.lb <= st.ub and st.ub == pytest.approx(ref.stats.ub, rel=1e-3)
    # the oracle's own stop decision at the GPU's count: R^k is below eps_l there too
    for k in range(2):
        assert ref.fpr[k] < st.tol[k] * 1.5


def test_solve3d_32_cluster_level(w1):
    """32^3 with two levels: 16^3 on one CTA, 32^3 on an 8-CTA cluster of slabs."""
    r0, r1 = synth.pair3(32, 6)
    val, st, status, flux, phi, ref = solve3_and_replay(w1, r0, r1, L1, 2)
    assert status == w1.OK and st.converged
    assert st.path == [1, 1] and st.cluster == [1, 8]
    assert abs(val - ref.w1) <= 1e-4 * abs(ref.w1), (val, ref.w1)
    assert flux3_rel_l1(flux, ref) <= 1e-3


def test_solve3d_64_wide_level(w1):
    """64^3 with three levels: 16^3 on one CTA, 32^3 on 8 CTAs, 64^3 on a
    16-CTA cluster of wide slabs (four planes of 4096 voxels each)."""
    r0, r1 = synth.pair3(64, 0)
    val, st, status, flux, phi, ref = solve3_and_replay(w1, r0, r1, L1, 3)
    assert status == w1.OK and st.converged
    assert st.path == [1, 1, 1] and st.cluster == [1, 8, 16]
    assert abs(val - ref.w1) <= 1e-4 * abs(ref.w1), (val, ref.w1)
    assert flux3_rel_l1(flux, ref) <= 1e-3


def test_solve3d_ragged_three_levels(w1):
    """Unequal sides 32 x 16 x 8 (h = 1/32), three levels 8x4x2 -> 32x16x8, p = 2."""
    r0, r1 = synth.pair3(0, 3, nx=32, ny=16, nz=8)
    val, st, status, flux, phi, ref = solve3_and_replay(w1, r0, r1, L2, 3)
    assert status == w1.OK and st.converged
    assert st.sizes == [(8, 4), (16, 8), (32, 16)]
    assert abs(val - ref.w1) <= 1e-4 * abs(ref.w1), (val, ref.w1)
    assert flux3_rel_l1(flux, ref) <= 1e-3


def test_solve3d_certificates_match_oracle(w1):
    """The FP64 certificates of the returned FP32 state equal the oracle's
    certificates of the same state."""
    r0, r1 = synth.pair3(16, 5)
    a0, a1, d0, d1 = synth.to_f32_pair(r0, r1)
    flux = torch.empty((3, 16, 16, 16), device="cuda")
    phi = torch.empty((16, 16, 16), device="cuda")
    val, st, _ = w1.solve3d(dev(a0), dev(a1), norm=L1, levels=2, flux=flux, potential=phi)
    rho = (d0 - d1)
    rho = (rho - rho.mean()).astype(np.float32).astype(np.float64)
    f = host(flux)
    s = d3.stats(rho, f[0], f[1], f[2], host(phi), 1 / 16, L1)
    assert st.primal == pytest.approx(s.f, rel=1e-9)
    assert st.saddle == pytest.approx(s.saddle, rel=1e-9)
    assert st.w1 == st.saddle
    assert st.dual == pytest.approx(s.dual, rel=1e-9)
    assert st.gmax == pytest.approx(s.gmax, rel=1e-9)
    assert st.res_l1 == pytest.approx(s.res_l1, rel=1e-7)
    assert st.route == pytest.approx(s.route, rel=1e-7)
    assert st.ub == pytest.approx(s.ub, rel=1e-7)
    assert st.lb == pytest.approx(s.lb, rel=1e-9)
    assert st.mass0 == pytest.approx(1.0, rel=1e-6) and st.mass1 == pytest.approx(1.0, rel=1e-6)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_solve3d_strip_closed_form(w1, axis):
    """A strip of 16 voxels along one axis (levels chosen automatically: the
    other sides are 1, so one level): W1 = sum_k |C_k| h with C the cumulative
    mass difference, for every p (theta = 1, eps = 1e-10)."""
    n = 16
    rng = np.random.default_rng(40 + axis)
    h = 1.0 / n
    r0 = rng.uniform(0.1, 1.0, n)
    r1 = rng.uniform(0.1, 1.0, n)
    r0 = (r0 / (r0.sum() * h ** 3)).astype(np.float32)
    r1 = (r1 / (r1.sum() * h ** 3)).astype(np.float32)
    d = r0.astype(np.float64) - r1.astype(np.float64)
    C = np.cumsum((d - d.mean()) * h ** 3)
    exact = np.abs(C[:-1]).sum() * h
    shape = [1, 1, 1]
    shape[2 - axis] = n
    for norm in (L1, LINF):
        val, st, status = w1.solve3d(dev(r0.reshape(shape)), dev(r1.reshape(shape)), norm=norm, tol=1e-10,
                                     theta=1.0, max_iters=400_000)
        assert status == w1.OK and st.levels == 1
        assert val == pytest.approx(exact, rel=1e-4)
        assert st.lb <= exact * (1 + 1e-4) and st.ub >= exact * (1 - 1e-4)


def test_solve3d_single_voxel_and_identical(w1):
    one = dev(np.ones((1, 1, 1)))
    val, st, status = w1.solve3d(one, one, norm=L2)
    assert status == w1.OK and val == 0.0 and st.ub == 0.0
    r0, _ = synth.pair3(8, 1)
    a = dev(r0)
    val, st, status = w1.solve3d(a, a.clone(), norm=L1, levels=2)
    assert status == w1.OK and val == 0.0 and st.converged


def test_solve3d_workspace_reuse(w1):
    """Repeated solves of different sizes reuse the pooled workspace and give the
    same result as after the pool is freed."""
    r0, r1 = synth.pair3(16, 11)
    a0, a1 = dev(r0), dev(r1)
    v1, _, _ = w1.solve3d(a0, a1, norm=L2, levels=2)
    s0, s1 = synth.pair3(8, 12)
    w1.solve3d(dev(s0), dev(s1), norm=L1)
    v2, _, _ = w1.solve3d(a0, a1, norm=L2, levels=2)
    w1.release_workspace3d()
    v3, _, _ = w1.solve3d(a0, a1, norm=L2, levels=2)
    assert v1 == v2 == v3


def test_solve3d_errors(w1):
    z = dev(np.ones((4, 4, 4)))
    with pytest.raises(w1.W1Error) as e:
        w1.solve3d(z, 2 * z)
    assert e.value.status == w1.ERR_MASS
    with pytest.raises(w1.W1Error) as e:
        w1.solve3d(z, z, levels=4)
    assert e.value.status == w1.ERR_SHAPE
    with pytest.raises(w1.W1Error) as e:
        w1.solve3d(z, z, norm=7)
    assert e.value.status == w1.ERR_INVALID_ARG
    bad = np.ones((4, 4, 4), dtype=np.float32)
    bad[1, 2, 3] = np.nan
    with pytest.raises(w1.W1Error) as e:
        w1.solve3d(dev(bad), z)
    assert e.value.status == w1.ERR_MASS


def test_solve3d_max_iters_reports_not_converged(w1):
    r0, r1 = synth.pair3(8, 2)
    val, st, status = w1.solve3d(dev(r0), dev(r1), norm=L1, levels=1, tol=1e-30, max_iters=64)
    assert status == w1.ERR_NOT_CONVERGED and not st.converged
    assert st.iters == [64] and np.isfinite(val) and st.lb <= st.ub


@pytest.mark.parametrize("norm", [L1, L2, LINF])
@pytest.mark.parametrize("shape,steps", [((24, 20, 36), 6), ((9, 13, 7), 5)])
def test_one_launch_step_equals_two_launch_step(w1, norm, shape, steps):
    """The one-launch step recomputes m' on each voxel's lower neighbours with the
    two-launch step's arithmetic: the new state is the same bit for bit (even and
    odd step counts); R^k agrees to rounding."""
    nz, ny, nx = shape
    rng = np.random.default_rng(nx + 31 * ny + 977 * nz + norm)
    rho, m1, m2, m3, phi = rand_state3(rng, nz, ny, nx)
    h = 1.0 / max(shape)
    mu = mu3(h)
    a = [dev(x) for x in (rho, m1, m2, m3, phi)]
    b = [dev(x) for x in (rho, m1, m2, m3, phi)]
    ra = w1.cp_steps3d(*a, h, norm, mu, mu, steps, path=2)
    rb = w1.cp_steps3d(*b, h, norm, mu, mu, steps, path=3)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(host(x), host(y))
    assert rb == pytest.approx(ra, rel=1e-5, abs=1e-14)
