"""Parity at the full size the benchmark times (512^3, 20-cell sponge,
layered model, 20 Hz source, 64 receivers, FP32, default launch
configuration), where the oracle cannot run the whole grid:

* sampled outputs: for the first n steps the wavefield is non-zero only
  within 4n cells of the source (the stencil reaches 4 cells per step), so
  the oracle run on a box around the source with a zero boundary computes
  those cells exactly; n is chosen so that the box stays in the undamped
  interior (sponge factor 1);
* a property that holds at any size: the 2 x 2 x 2 decomposition with
  fused one-sided halo puts reproduces the undecomposed run bit for bit.
"""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import assert_close, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shot():
    return workloads.layered_cube(512)


def test_light_cone_box_matches_oracle(shot):
    sx, sy, sz = shot.src
    d = min(min(c - shot.sponge, 512 - shot.sponge - 1 - c) for c in shot.src)
    n = min(12, (d - 1) // 4)
    assert n >= 4
    g = gpu_run(shot.vel, n, src=shot.src, f_peak=shot.f_peak,
                receivers=shot.receivers, sponge=shot.sponge)
    B = 4 * n + 8
    lo = [c - B for c in (sx, sy, sz)]
    hi = [c + B + 1 for c in (sx, sy, sz)]
    crop = shot.vel[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    dt = oracle.time_step(shot.h, float(shot.vel.max()))
    o = oracle.run(crop, shot.h, n, dt=dt, src=(B, B, B), f_peak=shot.f_peak,
                   nthreads=8)
    gu = g["u"][lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    assert_close(gu, o["u"], 1e-4)
    # nothing outside the light cone box
    outside = g["u"].copy()
    outside[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 0
    assert not outside.any()


def test_decomposed_2x2x2_is_bitwise_at_full_size(shot):
    n = 30
    a = gpu_run(shot.vel, n, src=shot.src, f_peak=shot.f_peak,
                receivers=shot.receivers, sponge=shot.sponge)
    b = gpu_run(shot.vel, n, src=shot.src, f_peak=shot.f_peak,
                receivers=shot.receivers, sponge=shot.sponge, px=2, py=2,
                pz=2)
    assert np.array_equal(a["u32"], b["u32"])
    assert np.array_equal(a["traces"], b["traces"])
    assert np.abs(a["u32"]).max() > 0


def test_light_cone_box_at_the_paper_minimod_grid():
    """The same light-cone check on the paper's own Minimod grid, 1200^3
    (section 4.5), with the 8-layer model set one value per plane (so no
    13.8 GB host model is built) and the default launch configuration,
    whose x and y edges leave partial tiles."""
    from paper_2506_02486_gb300 import gbwave as gw
    from paper_2506_02486_gb300.runtime import Segment, Shot, padded_bytes
    n, sponge, h = 1200, 20, 10.0
    vz = workloads.layered_profile(n, 2506)
    src = workloads.source_position(2507, n, n, n, margin=sponge)
    d = min(min(c - sponge, n - sponge - 1 - c) for c in src)
    steps = min(12, (d - 1) // 4)
    assert steps >= 4
    with Segment(4 * padded_bytes(n, n, n, "f32") + (1 << 30)) as seg:
        with Shot(seg, n, n, n, nsteps=steps, sponge=sponge) as s:
            gw.gw_set_model_layered(s.dom, vz)
            s.add_ricker(src, 20.0)
            s.step(steps)
            s.sync()
            u = s.u(f64=False)
    B = 4 * steps + 8
    sx, sy, sz = src
    lo = [c - B for c in (sx, sy, sz)]
    hi = [c + B + 1 for c in (sx, sy, sz)]
    crop = np.broadcast_to(vz[lo[2]:hi[2], None, None],
                           (hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])).copy()
    dt = oracle.time_step(h, float(vz.max()))
    o = oracle.run(crop, h, steps, dt=dt, src=(B, B, B), f_peak=20.0, nthreads=8)
    gu = u[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].astype(np.float64)
    assert_close(gu, o["u"], 1e-4)
    u[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 0
    assert not u.any()
