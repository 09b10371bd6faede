"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs, element by element, at sizes the oracle finishes in
seconds that still span several tiles and ragged tails.

Tolerances: FP32 storage and arithmetic, relative L2 <= 1e-4 after 100
steps against FP64 (the accuracy bar of the plain 64^3 configuration), and
the same bound point by point, max |g - o| <= 1e-4 max |o|, so that one
wrong row of a partial tile cannot hide in a whole-grid norm; FP64 kernel
<= 1e-10 both ways.  Each side computes its own time step
(Courant rule) and its own Ricker samples from the same peak frequency.
"""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import U32, assert_close, gamma, gpu_run, max_rel, rel_l2, seg_for
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
    assert_close(g["u"], o["u"], TOL32)
    assert np.abs(o["u"]).max() > 1e-6            # the wave is there
    assert_close(g["traces"], o["traces"], TOL32, "traces")
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
    assert_close(g["u"], o["u"], TOL32)
    assert_close(g["traces"], o["traces"], TOL32, "traces")


def test_tiles_graphs_and_schedules_do_not_change_bits():
    """Tiles, z-chunking, graph or plain launches, persistent launches and
    the static or dynamic work-item schedule: the same bits."""
    nx, ny, nz = 70, 45, 33
    vel = workloads.layered(nx, ny, nz, seed=3)
    src = (30, 20, 16)
    cases = [(1, 0, 0, 0, 0), (2, 7, 5, 2, 0), (3, -1, 0, 1, 0), (4, 4, 13, 2, 0),
             (1, 25, 33, 1, 0), (1, 6, 5, 2, 1), (2, 9, 7, 1, 1), (5, -1, 3, 2, 0)]
    runs = [gpu_run(vel, 37, src=src, f_peak=25.0, sponge=5, tile=t, chunk=c,
                    zchunk=z, schedule=sch, persistent=p)
            for t, c, z, sch, p in cases]
    for (t, c, z, sch, p), r in zip(cases, runs):
        assert np.array_equal(r["u32"], runs[0]["u32"]), (t, c, z, sch, p)
        if sch:
            assert r["info"]["schedule"] == sch
        # norms: each thread's plane partials depend on the tile (gamma_7)
        assert r["norms"] == pytest.approx(runs[0]["norms"],
                                           rel=2 * (gamma(7) + gamma(127) ** 2))


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
    assert_close(g["u"], o["u"], TOL32)


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
    assert_close(g["u"], o["u"], 1e-10)


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
    assert_close(g["u"], o["u"], TOL32)
    assert_close(g["traces"], o["traces"], TOL32, "traces")


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
    assert_close(g["traces"], o["traces"], TOL32, "traces")
    more = np.array([[x, y, 12] for x in range(8, 28) for y in range(4, 8)],
                    dtype=np.int32)                      # 80 cells
    with pytest.raises(gw.GWError) as e:
        gpu_run(vel, 20, src=src, f_peak=40.0, receivers=more, zchunk=nz)
    assert e.value.status == gw.GW_ERR_ARG and "one work item" in str(e.value)


def _state(vel, steps, dtype="f32", **kw):
    """A layered shot after `steps` steps: the library's checks and the
    fields as stored (u_n, u_{n-1}, coef), read back unscaled."""
    from paper_2506_02486_gb300.runtime import Shot
    nz, ny, nx = vel.shape
    with seg_for(nx, ny, nz, dtype) as seg:
        with Shot(seg, nx, ny, nz, nsteps=steps, dtype=dtype, **kw) as s:
            s.set_model(vel)
            s.add_ricker((nx // 2 - 3, ny // 2 + 2, nz // 2 + 1), 30.0)
            s.step(steps)
            s.sync()
            norm2, energy = s.check()
            out = {"norm2": norm2, "energy": energy,
                   "norms": s.norms(steps), "u": s.u(gw.GW_FIELD_U),
                   "coef": s.u(gw.GW_FIELD_COEF), "dt": s.info["dt"]}
            if dtype in ("f32", "f64"):
                out["up"] = s.u(gw.GW_FIELD_UPREV)
            return out


def _kin_pot(coef, u, up):
    """The two sums of the discrete energy E = kin - pot, written out from
    their definitions: kin = sum (u - up)^2 / coef, pot = sum u lap(up)."""
    d = u - up
    kin = float(np.sum(d * d / coef))
    pot = float(np.sum(u * oracle.laplacian(oracle.pad(up))))
    return kin, pot


def test_check_energy_equals_oracle_energy_on_the_same_state():
    """gw_check's FP64 energy and norm against the oracle's energy of the
    very fields the library holds (read back, with the coefficients as
    stored): the same sums in another order, so equal to FP64 rounding."""
    nx, ny, nz = 47, 39, 33
    vel = workloads.layered(nx, ny, nz, seed=12)
    st = _state(vel, 45, sponge=5)
    e_or = oracle.energy(st["coef"], st["u"], st["up"])
    kin, pot = _kin_pot(st["coef"], st["u"], st["up"])
    scale = abs(kin) + abs(pot)
    assert kin > 0 and scale > 0
    assert abs(st["energy"] - e_or) <= 1e-12 * scale
    assert st["norm2"] == pytest.approx(float(np.sum(st["u"] ** 2)), rel=1e-12)


def test_check_energy_follows_the_oracle_run():
    """gw_check's energy of the GPU state against the oracle's energy of
    its own FP64 run of the same shot (no sponge, so E is conserved once
    the source is quiet).  The kinetic sum is built from differences of
    consecutive fields, about omega dt = 0.2 of u in size here, so its
    relative error is a few times the field's: bound 10 * TOL32."""
    nx, ny, nz = 44, 40, 36
    vel = workloads.layered(nx, ny, nz, seed=13)
    steps = 90
    st = _state(vel, steps)
    src = (nx // 2 - 3, ny // 2 + 2, nz // 2 + 1)
    o = oracle_for(vel, steps, src=src, f_peak=30.0)
    e_or = oracle.energy((vel * o["dt"] / 10.0) ** 2, o["u"], o["u_prev"])
    kin, pot = _kin_pot((vel * o["dt"] / 10.0) ** 2, o["u"], o["u_prev"])
    assert kin > 0
    assert abs(st["energy"] - e_or) <= 10 * TOL32 * (abs(kin) + abs(pot))
    assert st["norm2"] == pytest.approx(o["norms"][-1], rel=2 * TOL32)


@pytest.mark.parametrize("dtype,u_store", [("f32", 0.0), ("f64", 0.0),
                                           ("f16s", 2.0 ** -11),
                                           ("bf16", 2.0 ** -8)])
def test_step_norms_are_fp64_sums_of_plane_partials(dtype, u_store):
    """The step kernel's per-step norm, against gw_check's FP64 sum of the
    same field.  Each thread sums its at most 8 points of a plane in the
    math type (positive terms: relative error <= gamma_7 = 7 u / (1 - 7 u)
    for FP32), accumulates the plane sums of an item (fewer than 128 planes
    on this grid) as a compensated pair (Ogita, Rump and Oishi's Sum2:
    error <= gamma_127^2 of the sum), and the items are added in FP64; so
    for FP32 storage the two
    agree to gamma_7 + gamma_127^2, 4.2e-7.  (A plain FP32 partial over an
    item of 64 planes would only be bound by gamma_511 = 3e-5.)  With 16-bit
    storage the kernel squares the values before they are rounded to the
    storage type (unit roundoff u_s, 2^-11 for FP16 and 2^-8 for BF16) and
    gw_check squares the stored ones: 2 u_s + u_s^2 more."""
    nx, ny, nz = 75, 37, 29
    vel = workloads.layered(nx, ny, nz, seed=14)
    st = _state(vel, 40, dtype=dtype, sponge=4)
    assert st["norm2"] > 0
    bound = gamma(7) + gamma(127) ** 2 + 2 * u_store + u_store ** 2 + 1e-12
    assert abs(st["norms"][-1] - st["norm2"]) <= bound * st["norm2"]
