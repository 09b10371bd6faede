"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs, element by element, at sizes the oracle finishes in
seconds that still span several tiles and ragged tails.

Tolerances: FP32 storage and arithmetic, relative L2 <= 1e-4 after 100
steps against FP64 (the accuracy bar of the plain 64^3 configuration);
FP64 kernel relative L2 <= 1e-10.  Each side computes its own time step
(Courant rule) and its own Ricker samples from the same peak frequency.
"""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import gpu_run, rel_l2, seg_for
from paper_2506_02486_gb300 import gbwave as gw

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


def oracle_for(vel, nsteps, *, h=10.0, src=None, f_peak=None, wavelet=None,
               receivers=None, sponge=0, periodic=False, u0=None, um1=None,
               dt=None, nthreads=8):
    if dt is None:
        dt = oracle.time_step(h, float(vel.max()))
    return oracle.run(vel, h, nsteps, dt=dt, sponge=sponge, periodic=periodic,
                      src=src, f_peak=f_peak, wavelet=wavelet,
                      receivers=receivers, u0=u0, um1=um1, norms=True,
                      nthreads=nthreads)


def test_plain_64cubed_matches_oracle():
    """64^3, h = 10 m, v = 1500 m/s, dt at half the Courant limit, 100
    steps, 15 Hz Ricker at the centre cell, zero halo, no sponge."""
    n = 64
    vel = workloads.homogeneous(n, n, n, 1500.0)
    src = (32, 32, 32)
    rec = np.array([[32, 32, 32], [10, 40, 32], [50, 5, 60], [0, 0, 0]],
                   dtype=np.int32)
    g = gpu_run(vel, 100, src=src, f_peak=15.0, receivers=rec)
    o = oracle_for(vel, 100, src=src, f_peak=15.0, receivers=rec)
    assert g["dt"] == pytest.approx(o["dt"], rel=1e-14)
    assert g["dt"] == pytest.approx(1.5095e-3, rel=1e-4)
    err = rel_l2(g["u"], o["u"])
    assert err <= TOL32, err
    assert np.abs(o["u"]).max() > 1e-6            # the wave is there
    assert rel_l2(g["traces"], o["traces"]) <= TOL32
    assert g["norms"] == pytest.approx(o["norms"], rel=TOL32)


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6, 7])
def test_ragged_layered_sponge_matches_oracle(tile):
    """Non-multiple sizes in every axis (ragged tiles and x tails), a
    layered model, a 6-cell sponge, an off-centre source, every FP32 tile."""
    nx, ny, nz = 75, 37, 29
    vel = workloads.layered(nx, ny, nz, seed=7)
    src = workloads.source_position(11, nx, ny, nz, margin=6)
    rec = workloads.lattice_receivers(nx, ny, 6, n=4, margin=6)
    g = gpu_run(vel, 60, src=src, f_peak=30.0, receivers=rec, sponge=6,
                tile=tile)
    o = oracle_for(vel, 60, src=src, f_peak=30.0, receivers=rec, sponge=6)
    assert rel_l2(g["u"], o["u"]) <= TOL32
    assert rel_l2(g["traces"], o["traces"]) <= TOL32


def test_tiles_and_graphs_do_not_change_bits():
    nx, ny, nz = 70, 45, 33
    vel = workloads.layered(nx, ny, nz, seed=3)
    src = (30, 20, 16)
    runs = [gpu_run(vel, 37, src=src, f_peak=25.0, sponge=5, tile=t,
                    chunk=c, zchunk=z)
            for t, c, z in [(1, 0, 0), (2, 7, 5), (3, -1, 0), (4, 4, 13),
                            (1, 25, 33)]]
    for r in runs[1:]:
        assert np.array_equal(r["u32"], runs[0]["u32"])


@pytest.mark.parametrize("dtype,tiles", [("f16s", [1, 2, 3, 4, 5]),
                                         ("bf16", [1, 2, 3, 4])])
def test_delta_tiles_do_not_change_bits(dtype, tiles):
    """16-bit delta storage: every tile, z-chunking and launch mode gives
    the same bits (the stored values and the traces)."""
    nx, ny, nz = 70, 45, 33
    vel = workloads.layered(nx, ny, nz, seed=3)
    rec = workloads.lattice_receivers(nx, ny, 5, n=3, margin=5)
    runs = [gpu_run(vel, 37, src=(30, 20, 16), f_peak=25.0, sponge=5,
                    receivers=rec, dtype=dtype, tile=t, chunk=c, zchunk=z)
            for t, c, z in [(tiles[0], 0, 0)] +
            [(t, 7, 5 + 4 * i) for i, t in enumerate(tiles[1:])] +
            [(tiles[0], -1, 33)]]
    for r in runs[1:]:
        assert np.array_equal(r["u32"], runs[0]["u32"])
        assert np.array_equal(r["traces"], runs[0]["traces"])


@pytest.mark.parametrize("shape", [(8, 8, 8), (9, 5, 3), (1, 1, 1),
                                   (130, 3, 4), (5, 70, 9)])
def test_small_and_degenerate_grids(shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(1)
    vel = rng.uniform(1500, 4500, (nz, ny, nx))
    u0 = rng.standard_normal((nz, ny, nx))
    um1 = rng.standard_normal((nz, ny, nx))
    g = gpu_run(vel, 12, u0=u0, um1=um1, courant=0.3)
    o = oracle_for(vel, 12, u0=u0, um1=um1,
                   dt=oracle.time_step(10.0, float(vel.max()), 0.3))
    assert rel_l2(g["u"], o["u"]) <= TOL32


def test_zero_steps_is_identity():
    rng = np.random.default_rng(2)
    vel = np.full((9, 10, 11), 2000.0)
    u0 = rng.standard_normal(vel.shape).astype(np.float32)
    g = gpu_run(vel, 0, u0=u0)
    assert np.array_equal(g["u32"], u0)


def test_fp64_kernel_matches_oracle():
    nx, ny, nz = 48, 40, 36
    vel = workloads.perturbed(workloads.layered(nx, ny, nz, seed=5), seed=6)
    src = (20, 21, 18)
    g = gpu_run(vel, 50, src=src, f_peak=30.0, sponge=5, dtype="f64")
    o = oracle_for(vel, 50, src=src, f_peak=30.0, sponge=5)
    assert rel_l2(g["u"], o["u"]) <= 1e-10


def test_centred_source_is_mirror_symmetric_bitwise():
    n = 65
    vel = workloads.homogeneous(n, n, n, 2500.0)
    g = gpu_run(vel, 80, src=(32, 32, 32), f_peak=25.0, sponge=8)
    u = g["u32"]
    assert np.abs(u).max() > 0
    for ax in range(3):
        assert np.array_equal(u, np.flip(u, axis=ax))
    # x <-> y swap keeps the pair-sum order: bitwise
    assert np.array_equal(u, u.transpose(0, 2, 1))
    # swapping z with x or y reorders the sums: equal to rounding only
    assert rel_l2(u, u.transpose(2, 1, 0)) <= 1e-6


def test_plane_wave_periodic_box_follows_discrete_dispersion():
    nx, ny, nz = 32, 24, 16
    h, v = 10.0, 2000.0
    nu = 0.8 * oracle.nu_max()
    dt = nu * h / v
    kx, ky, kz = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny, 2 * np.pi / nz
    c = oracle.coefficients()

    def L(t):
        return c[0] + 2 * sum(c[m] * np.cos(m * t) for m in range(1, 5))

    wdt = np.arccos(1 + 0.5 * nu ** 2 * (L(kx) + L(ky) + L(kz)))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    ph = kx * i + ky * j + kz * k
    vel = np.full((nz, ny, nx), v)
    n = 60
    g = gpu_run(vel, n, dt=dt, periodic=7, u0=np.cos(ph),
                um1=np.cos(ph + wdt))
    want = np.cos(ph - wdt * n)
    assert np.abs(g["u"] - want).max() <= 2e-5
    # the same periodic box cut into 2 x 2 x 2 subdomains: identical bits
    g2 = gpu_run(vel, n, dt=dt, periodic=7, u0=np.cos(ph),
                 um1=np.cos(ph + wdt), px=2, py=2, pz=2)
    assert np.array_equal(g2["u32"], g["u32"])


def test_energy_is_conserved_on_gpu():
    nx, ny, nz = 40, 36, 32
    rng = np.random.default_rng(4)
    vel = rng.uniform(1500, 4500, (nz, ny, nx))
    u0 = rng.standard_normal((nz, ny, nx))
    with seg_for(nx, ny, nz) as seg:
        from paper_2506_02486_gb300.runtime import Shot
        from paper_2506_02486_gb300 import gbwave as gw
        with Shot(seg, nx, ny, nz, nsteps=200, courant=0.4) as s:
            s.set_model(vel)
            s.write(gw.GW_FIELD_U, u0)
            s.write(gw.GW_FIELD_UPREV, u0)
            e = []
            for _ in range(10):
                s.step(20)
                e.append(s.check()[1])
    e = np.array(e)
    assert e[0] > 0
    assert np.abs(e / e[0] - 1).max() <= 1e-4


def test_checkpoint_resume_is_bitwise():
    from paper_2506_02486_gb300.runtime import Shot
    from paper_2506_02486_gb300 import gbwave as gw
    nx, ny, nz = 50, 40, 30
    vel = workloads.layered(nx, ny, nz, seed=9)
    with seg_for(nx, ny, nz, px=2, pz=2) as seg:
        with Shot(seg, nx, ny, nz, px=2, pz=2, nsteps=60, sponge=4) as s:
            s.set_model(vel)
            s.add_ricker((25, 20, 15), 30.0)
            s.set_receivers([[5, 5, 5], [40, 30, 20]])
            s.step(20)
            snap = gw.gw_save_state(s.dom)
            s.step(20)
            a = s.u(f64=False)
            ta = s.traces(40)
            gw.gw_load_state(s.dom, snap)
            s.step(20)
            b = s.u(f64=False)
            tb = s.traces(40)
    assert np.array_equal(a, b)
    assert np.array_equal(ta, tb)


def test_tall_thin_grid_matches_oracle():
    """Many z items over a narrow column (and a sponge only along z)."""
    nx, ny, nz = 20, 24, 700
    vel = workloads.layered(nx, ny, nz, seed=41)
    src = (10, 12, 350)
    rec = np.array([[10, 12, z] for z in range(300, 400, 7)], dtype=np.int32)
    g = gpu_run(vel, 40, src=src, f_peak=35.0, receivers=rec, sponge=4)
    o = oracle_for(vel, 40, src=src, f_peak=35.0, receivers=rec, sponge=4)
    assert rel_l2(g["u"], o["u"]) <= TOL32
    assert rel_l2(g["traces"], o["traces"]) <= TOL32


def test_dense_receivers_in_one_tile():
    """64 receivers in one tile column are recorded; 80 are refused up
    front with a clear message instead of being dropped on the device."""
    nx, ny, nz = 128, 28, 24           # two 64 x 28 tile columns
    vel = workloads.homogeneous(nx, ny, nz)
    src = (96, 14, 12)                 # in the other column
    rec = np.array([[x, y, 12] for x in range(8, 24) for y in range(4, 8)],
                   dtype=np.int32)                       # 64 cells
    g = gpu_run(vel, 20, src=src, f_peak=40.0, receivers=rec, zchunk=nz)
    o = oracle_for(vel, 20, src=src, f_peak=40.0, receivers=rec)
    assert rel_l2(g["traces"], o["traces"]) <= TOL32
    more = np.array([[x, y, 12] for x in range(8, 28) for y in range(4, 8)],
                    dtype=np.int32)                      # 80 cells
    with pytest.raises(gw.GWError) as e:
        gpu_run(vel, 20, src=src, f_peak=40.0, receivers=more, zchunk=nz)
    assert e.value.status == gw.GW_ERR_ARG and "one work item" in str(e.value)
