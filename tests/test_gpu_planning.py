"""How a shot's work is cut into items and handed to CTAs (the planner in
csrc/domain.cpp and csrc/batch.cpp): the documented policy, pinned on
grids small enough for a test.  Results do not depend on any of it (the
parity and decomposition tests run every schedule); these tests keep the
performance policy from drifting unnoticed.

* AUTO takes the static schedule for an undecomposed shot whose tile
  columns all fit in one round of CTAs, the dynamic one otherwise, and
  decomposed shots are always dynamic.
* At least two z-chunks per column (when nz >= 32) and at least 16 planes
  per item.
* The tile groups of a non-persistent batch, running side by side, get
  whole columns of up to 256 planes; a persistent batch keeps the model."""

import numpy as np
import pytest

from gpu_util import seg_for
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Batch, Segment, Shot, shot_bytes

pytestmark = pytest.mark.gpu

TX, TY = 64, 28            # the default FP32 tile


def _cols(nx, ny, tx=TX, ty=TY):
    return -(-nx // tx) * -(-ny // ty)


def _info(nx, ny, nz, **kw):
    with seg_for(nx, ny, nz, "f32", kw.get("px", 1), kw.get("py", 1),
                 kw.get("pz", 1)) as seg:
        with Shot(seg, nx, ny, nz, nsteps=2, sponge=0, **kw) as s:
            return s.info


def test_static_when_the_columns_fit_one_round():
    info = _info(1024, 200, 40)
    cols = _cols(1024, 200)
    assert cols <= info["ctas"]
    assert info["schedule"] == gw.GW_SCHED_STATIC
    # nz = 40: two z-chunks of 20 planes (at least two, at least 16 planes)
    assert info["items"] == 2 * cols


def test_dynamic_when_the_columns_outnumber_the_ctas():
    info = _info(1100, 250, 40)
    cols = _cols(1100, 250)
    assert cols > info["ctas"]
    assert info["schedule"] == gw.GW_SCHED_DYNAMIC
    assert info["items"] == 2 * cols


def test_decomposed_shots_are_dynamic_and_short_grids_one_chunk():
    info = _info(96, 80, 72, px=2, pz=2)
    assert info["schedule"] == gw.GW_SCHED_DYNAMIC
    # subdomains of 36 planes: two chunks of 18
    assert info["items"] == 2 * 2 * _cols(48, 80) * 2
    # nz < 32: one chunk per column
    info = _info(96, 80, 24)
    assert info["items"] == _cols(96, 80)


def test_forced_schedules_are_reported():
    for sched in (gw.GW_SCHED_STATIC, gw.GW_SCHED_DYNAMIC):
        assert _info(200, 100, 40, schedule=sched)["schedule"] == sched


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_items(persistent):
    """Two shots with different tiles form two groups.  Side by side (not
    persistent) each shot's columns are whole items (nz <= 256); persistent,
    the shots keep the single-shot model (at least two z-chunks here)."""
    sides = (96, 112)
    tiles = (1, 2)                       # 64 x 28 and 128 x 14 for FP32
    total = sum(shot_bytes(n, n, n, "f32", 4) for n in sides) + (1 << 30)
    with Segment(total) as seg:
        shots = [Shot(seg, n, n, n, nsteps=4, tile=t, sponge=4)
                 for n, t in zip(sides, tiles)]
        try:
            for s, n in zip(shots, sides):
                s.set_model(np.full((n, n, n), 2000.0))
            with Batch(seg, shots, persistent=persistent) as b:
                info = b.info
        finally:
            for s in shots:
                s.close()
    assert info["groups"] == 2
    cols = _cols(96, 96) + _cols(112, 112, 128, 14)
    if persistent:
        assert info["items"] >= 2 * cols
    else:
        assert info["items"] == cols
