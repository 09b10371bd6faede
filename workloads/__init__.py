"""Seeded synthetic inputs for the Minimod acoustic-isotropic workloads.

This module only draws inputs: velocity models, source and receiver
positions, shot lists and arrival streams.  It holds none of the method's
arithmetic (no time step, no Courant number, no coefficients, no sponge, no
wavelet); the CPU oracle and the CUDA library each compute those themselves
from what is drawn here.

Arrays follow the library's host layout: a velocity model of an
``nx x ny x nz`` interior grid is a C-ordered ``float64`` array of shape
``(nz, ny, nx)`` (x fastest, then y, then z), in m/s.

Recipes (the paper only names the Minimod workload, a 1200^3 grid run for
1000 steps with the acoustic isotropic kernel, section 4.5; the shapes below
are the synthetic stand-ins for the velocity models it does not publish):

* layered: ``nlayers - 1`` interface depths drawn uniformly over the z
  extent and sorted, ``nlayers`` velocities drawn uniformly in
  [vmin, vmax]; a cell at depth index k belongs to the layer below every
  interface whose depth is <= k.
* perturbed: a model times ``1 + clip(sigma * N(0, 1), -clip, +clip)``,
  independently per cell.
* source position: uniform over the cells at least ``margin`` cells from
  every face.
* receivers: an ``n x n`` lattice spread evenly over x and y inside the
  margin, on one z plane.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "homogeneous",
    "layered",
    "layered_profile",
    "perturbed",
    "random_field",
    "source_position",
    "lattice_receivers",
    "BatchShot",
    "batch_shots",
    "Request",
    "arrival_stream",
]


def homogeneous(nx: int, ny: int, nz: int, v: float = 1500.0) -> np.ndarray:
    """Constant velocity ``v`` on an ``nx x ny x nz`` grid."""
    return np.full((nz, ny, nx), float(v), dtype=np.float64)


def _layer_profile(nz: int, rng: np.random.Generator, nlayers: int,
                   vmin: float, vmax: float) -> np.ndarray:
    depths = np.sort(rng.uniform(0.0, float(nz), size=nlayers - 1))
    # velocities rounded to FP32 values, so that a model passed in FP32 and
    # the same model passed in FP64 are the same numbers
    vels = rng.uniform(vmin, vmax, size=nlayers).astype(np.float32).astype(np.float64)
    k = np.arange(nz, dtype=np.float64)
    layer = np.searchsorted(depths, k, side="right")
    return vels[layer]


def layered(nx: int, ny: int, nz: int, seed: int, nlayers: int = 8,
            vmin: float = 1500.0, vmax: float = 4500.0) -> np.ndarray:
    """Horizontally layered model: velocity depends on the z index only."""
    rng = np.random.default_rng(seed)
    prof = _layer_profile(nz, rng, nlayers, vmin, vmax)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    out[...] = prof[:, None, None]
    return out


def layered_profile(nz: int, seed: int, nlayers: int = 8,
                    vmin: float = 1500.0, vmax: float = 4500.0) -> np.ndarray:
    """The z profile of ``layered`` with the same seed (nz values)."""
    rng = np.random.default_rng(seed)
    return _layer_profile(nz, rng, nlayers, vmin, vmax)


def perturbed(base: np.ndarray, seed: int, sigma: float = 0.05,
              clip: float = 0.2, out_dtype=np.float64) -> np.ndarray:
    """Multiply ``base`` cell by cell by ``1 + clip(sigma*N(0,1))``.

    The normals are drawn one z plane at a time so that a crop of a large
    model can be regenerated without drawing the whole volume.
    """
    rng = np.random.default_rng(seed)
    nz = base.shape[0]
    out = np.empty(base.shape, dtype=out_dtype)
    for k in range(nz):
        eps = rng.standard_normal(base.shape[1:]) * sigma
        np.clip(eps, -clip, clip, out=eps)
        out[k] = base[k] * (1.0 + eps)
    return out


def random_field(nx: int, ny: int, nz: int, seed: int,
                 lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random values, for initial wavefields in tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nz, ny, nx))


def source_position(seed: int, nx: int, ny: int, nz: int,
                    margin: int = 0) -> tuple[int, int, int]:
    """A cell drawn uniformly at least ``margin`` cells inside every face."""
    rng = np.random.default_rng(seed)
    lo = margin
    return (int(rng.integers(lo, max(lo + 1, nx - margin))),
            int(rng.integers(lo, max(lo + 1, ny - margin))),
            int(rng.integers(lo, max(lo + 1, nz - margin))))


def lattice_receivers(nx: int, ny: int, z: int, n: int = 8,
                      margin: int = 0) -> np.ndarray:
    """``n*n`` receivers on plane ``z``, evenly spread in x and y.

    Returns an ``(n*n, 3)`` int32 array of (x, y, z) interior indices.
    """
    xs = np.linspace(margin, nx - 1 - margin, n).round().astype(np.int32)
    ys = np.linspace(margin, ny - 1 - margin, n).round().astype(np.int32)
    gx, gy = np.meshgrid(xs, ys, indexing="xy")
    rec = np.stack([gx.ravel(), gy.ravel(),
                    np.full(n * n, z, dtype=np.int32)], axis=1)
    return np.ascontiguousarray(rec, dtype=np.int32)


@dataclass
class BatchShot:
    """One shot of a batched run: a cube of side ``side``."""
    side: int
    model_seed: int
    source: tuple[int, int, int]
    nsteps: int
    sponge: int = 20

    def model(self) -> np.ndarray:
        return layered(self.side, self.side, self.side, self.model_seed)


def batch_shots(seed: int, n: int = 64, sides=tuple(range(96, 257, 16)),
                nsteps: int = 300, sponge: int = 20) -> list[BatchShot]:
    """``n`` independent cubic shots with sides drawn from ``sides``."""
    rng = np.random.default_rng(seed)
    shots = []
    for _ in range(n):
        side = int(rng.choice(np.asarray(sides)))
        mseed = int(rng.integers(0, 2**31 - 1))
        src = source_position(int(rng.integers(0, 2**31 - 1)),
                              side, side, side, margin=sponge)
        shots.append(BatchShot(side, mseed, src, nsteps, sponge))
    return shots


@dataclass
class Request:
    """One request of a serving stream."""
    arrival_s: float
    nx: int
    ny: int
    nz: int
    nsteps: int
    dtype: str
    model_seed: int
    source: tuple[int, int, int]
    sponge: int = 20
    meta: dict = field(default_factory=dict)


def arrival_stream(seed: int, n: int = 2000, rate_per_s: float = 10.0,
                   side_lo: int = 64, side_hi: int = 384,
                   max_aspect: float = 2.0, steps_lo: int = 200,
                   steps_hi: int = 2000,
                   dtypes=("f32", "bf16"), sponge: int = 20) -> list[Request]:
    """A Poisson stream of shot requests.

    Inter-arrival times are exponential with mean ``1/rate_per_s``; the side
    is log-uniform on [side_lo, side_hi] rounded to a multiple of 16; the z
    extent is the side times an aspect drawn uniformly in [1, max_aspect],
    rounded to a multiple of 16; the step count is uniform on
    [steps_lo, steps_hi]; the storage type alternates at random between
    ``dtypes``.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        side = math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))
        side = max(16, int(round(side / 16.0)) * 16)
        aspect = float(rng.uniform(1.0, max_aspect))
        nz = max(16, int(round(side * aspect / 16.0)) * 16)
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        dt = str(dtypes[int(rng.integers(0, len(dtypes)))])
        mseed = int(rng.integers(0, 2**31 - 1))
        src = source_position(int(rng.integers(0, 2**31 - 1)),
                              side, side, nz, margin=sponge)
        out.append(Request(t, side, side, nz, steps, dt, mseed, src, sponge))
    return out


@dataclass
class ShotInputs:
    """Everything a single-shot run draws: model, source, receivers."""
    name: str
    vel: np.ndarray
    src: tuple[int, int, int]
    receivers: np.ndarray
    f_peak: float
    nsteps: int
    sponge: int
    h: float = 10.0


def plain_cube(n: int = 64, nsteps: int = 100) -> ShotInputs:
    """Homogeneous 1500 m/s cube, 15 Hz source at interior index n/2 in
    every axis, no sponge (zero halo only), receivers on the source line."""
    vel = homogeneous(n, n, n, 1500.0)
    c = n // 2
    rec = np.array([[c, c, c], [c // 3, c, c], [c, c, n - 1 - c // 4]],
                   dtype=np.int32)
    return ShotInputs(f"plain_{n}cubed", vel, (c, c, c), rec, 15.0, nsteps, 0)


def layered_cube(n: int = 512, seed: int = 2506, nsteps: int = 1000,
                 sponge: int = 20) -> ShotInputs:
    """8-layer model (1500-4500 m/s) on an n^3 grid, 20-cell sponge, 20 Hz
    source at a seeded cell outside the sponge, 8 x 8 receivers on the
    first plane below the top sponge."""
    vel = layered(n, n, n, seed)
    src = source_position(seed + 1, n, n, n, margin=sponge)
    rec = lattice_receivers(n, n, sponge, n=8, margin=sponge)
    return ShotInputs(f"layered_{n}cubed", vel, src, rec, 20.0, nsteps,
                      sponge)


def perturbed_box(nx: int = 1024, ny: int = 1024, nz: int = 512,
                  seed: int = 2507, nsteps: int = 500, sponge: int = 20,
                  vel_dtype=np.float32, crop=None) -> ShotInputs:
    """The layered model with 5% i.i.d. Gaussian perturbations (clipped at
    20%) on an nx x ny x nz grid; 20 Hz source at a seeded cell.

    crop = (cx, cy, cz) returns the corner [0, cx) x [0, cy) x [0, cz) of
    exactly that model (the same layers and the same per-cell draws), with
    the source at the centre of the crop."""
    rng = np.random.default_rng(seed)
    prof = _layer_profile(nz, rng, 8, 1500.0, 4500.0)
    cx, cy, cz = (nx, ny, nz) if crop is None else crop
    base = np.empty((cz, cy, cx), dtype=vel_dtype)
    pr = np.random.default_rng(seed + 1)
    for k in range(cz):
        eps = pr.standard_normal((ny, nx)) * 0.05
        np.clip(eps, -0.2, 0.2, out=eps)
        base[k] = prof[k] * (1.0 + eps[:cy, :cx])
    if crop is None:
        src = source_position(seed + 2, nx, ny, nz, margin=sponge)
        rec = lattice_receivers(nx, ny, sponge, n=8, margin=sponge)
    else:
        src = (cx // 2, cy // 2, cz // 2)
        rec = lattice_receivers(cx, cy, sponge, n=8, margin=sponge)
    return ShotInputs(f"perturbed_{cx}x{cy}x{cz}", base, src, rec, 20.0,
                      nsteps, sponge)
