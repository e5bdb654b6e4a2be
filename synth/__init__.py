"""Seeded synthetic density pairs shaped like the paper's image workloads.

This module holds input generation only: no step of the W1 method is computed
here.  Both the oracle-side tests and the CUDA path take their inputs from it.

The paper measures on the "cat" pair (Sec. 5.1) and on the DOTmark "classic
images" (Sec. 5.3, 10 images, 45 pairs, up to 512x512); neither dataset is
available, so these generators stand in for them with the same grid sizes and
image-like structure (smooth blobs, filled shapes, texture, a positive floor).

Conventions:
  - a density is a float64 array [ny, nx] sampled at pixel centres
    ((i + 1/2) h, (j + 1/2) h) of [0,1]^2 with h = 1 / max(nx, ny);
  - it is floored, then normalised in float64 so that sum(rho) * h^2 = 1;
  - pair k of workload c is drawn from numpy's default_rng(1000 * c + k),
    rho0 first, rho1 second.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "centres", "normalise", "gaussian_mixture", "ellipse_texture", "pair",
    "WORKLOADS", "to_f32_pair", "gaussian_mixture3", "pair3",
]


def centres(nx: int, ny: int):
    h = 1.0 / max(nx, ny)
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(x, y)  # [ny, nx]
    return X, Y, h


def normalise(r: np.ndarray, h: float) -> np.ndarray:
    return r / (r.sum() * h * h)


def gaussian_mixture(nx: int, ny: int, k: int, floor: float, rng: np.random.Generator) -> np.ndarray:
    """Sum of k isotropic Gaussians w exp(-|x-c|^2 / (2 s^2)) with c ~ U[0.2,0.8]^2,
    s ~ U[0.03,0.1], w ~ U[0.5,1], plus a constant floor, unit mass."""
    X, Y, h = centres(nx, ny)
    r = np.zeros((ny, nx))
    for _ in range(k):
        cx, cy = rng.uniform(0.2, 0.8, 2)
        s = rng.uniform(0.03, 0.1)
        w = rng.uniform(0.5, 1.0)
        r += w * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * s * s))
    r += floor
    return normalise(r, h)


def _gauss_blur(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur (sigma in pixels), reflecting boundary."""
    rad = int(np.ceil(4 * sigma))
    t = np.arange(-rad, rad + 1)
    ker = np.exp(-t * t / (2.0 * sigma * sigma))
    ker /= ker.sum()
    out = a
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        p = np.pad(out, pad, mode="reflect")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for k, wk in enumerate(ker):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(k, k + n)
            acc += wk * p[tuple(sl)]
        out = acc
    return out


def ellipse_texture(nx: int, ny: int, rng: np.random.Generator) -> np.ndarray:
    """5-15 filled ellipses (semi-axes U[0.02,0.3], angle U[0,pi), intensity
    U[0.2,1], overlaps summed) plus uniform noise blurred with sigma = 4 px and
    rescaled to [0, 0.1]; clipped at 1e-4 and normalised to unit mass."""
    X, Y, h = centres(nx, ny)
    r = np.zeros((ny, nx))
    for _ in range(int(rng.integers(5, 16))):
        cx, cy = rng.uniform(0.1, 0.9, 2)
        a, b = rng.uniform(0.02, 0.3, 2)
        th = rng.uniform(0.0, np.pi)
        val = rng.uniform(0.2, 1.0)
        dx, dy = X - cx, Y - cy
        u = dx * np.cos(th) + dy * np.sin(th)
        v = -dx * np.sin(th) + dy * np.cos(th)
        r += val * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    noise = _gauss_blur(rng.uniform(0.0, 1.0, (ny, nx)), 4.0)
    lo, hi = noise.min(), noise.max()
    noise = 0.1 * (noise - lo) / (hi - lo if hi > lo else 1.0)
    r = np.maximum(r + noise, 1e-4)
    return normalise(r, h)


# Workload recipes: (name, grid side, density kind, kwargs)
WORKLOADS = {
    0: dict(name="gauss3_64", n=64, kind="gauss", k=3, floor=1e-3),
    1: dict(name="gauss8_256", n=256, kind="gauss", k=8, floor=1e-4),
    2: dict(name="ellipse_512", n=512, kind="ellipse"),
    3: dict(name="batch_mixed", n=None, kind="gauss", k=8, floor=1e-4),
    4: dict(name="serve_mixed", n=None, kind="ellipse"),
}


def pair(workload: int, k: int = 0, n: int | None = None, nx: int | None = None, ny: int | None = None):
    """Density pair k of a workload recipe (float64, unit mass each).  n (or
    nx, ny) overrides the grid side, e.g. for the mixed-size workloads."""
    spec = WORKLOADS[workload]
    side = n if n is not None else spec["n"]
    nx = nx if nx is not None else side
    ny = ny if ny is not None else side
    rng = np.random.default_rng(1000 * workload + k)
    if spec["kind"] == "gauss":
        r0 = gaussian_mixture(nx, ny, spec["k"], spec["floor"], rng)
        r1 = gaussian_mixture(nx, ny, spec["k"], spec["floor"], rng)
    else:
        r0 = ellipse_texture(nx, ny, rng)
        r1 = ellipse_texture(nx, ny, rng)
    return r0, r1


def to_f32_pair(r0: np.ndarray, r1: np.ndarray):
    """The float32 inputs the GPU takes, and the same values widened to float64
    for the oracle (so both solve the identical discrete problem)."""
    a0 = np.ascontiguousarray(r0, dtype=np.float32)
    a1 = np.ascontiguousarray(r1, dtype=np.float32)
    return a0, a1, a0.astype(np.float64), a1.astype(np.float64)


def gaussian_mixture3(nx: int, ny: int, nz: int, k: int, floor: float, rng: np.random.Generator) -> np.ndarray:
    """The 3-D counterpart of gaussian_mixture: k isotropic Gaussian blobs with
    centres ~ U[0.2,0.8]^3, s ~ U[0.05,0.12], w ~ U[0.5,1], a constant floor,
    sampled at voxel centres with h = 1 / max(nx, ny, nz), array [nz, ny, nx],
    normalised so that sum(rho) h^3 = 1."""
    h = 1.0 / max(nx, ny, nz)
    z, y, x = ((np.arange(m) + 0.5) * h for m in (nz, ny, nx))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.zeros((nz, ny, nx))
    for _ in range(k):
        cx, cy, cz = rng.uniform(0.2, 0.8, 3)
        s = rng.uniform(0.05, 0.12)
        w = rng.uniform(0.5, 1.0)
        r += w * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2.0 * s * s))
    r += floor
    return r / (r.sum() * h ** 3)


def pair3(n: int, k: int = 0, nx: int | None = None, ny: int | None = None, nz: int | None = None, blobs: int = 4,
          floor: float = 1e-3):
    """Density pair k of the 3-D recipe (float64, unit mass each), drawn from
    default_rng(7000 + k)."""
    nx = nx if nx is not None else n
    ny = ny if ny is not None else n
    nz = nz if nz is not None else n
    rng = np.random.default_rng(7000 + k)
    return (gaussian_mixture3(nx, ny, nz, blobs, floor, rng), gaussian_mixture3(nx, ny, nz, blobs, floor, rng))
