"""The bounded stream pool of the non-blocking puts/gets (paper section 3.2,
"Bounded Concurrency": a MAX_ACTIVE_STREAMS threshold; at the threshold
half of the completed streams are synchronised and released while the
others keep running), checked on the library's host-side model of the same
policy code, with hand-derived schedules."""

import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2506_02486_gb300 import gbwave as gw  # noqa: E402

from test_abi_cpu import HostSeg, lib  # noqa: E402,F401


def sim(max_active, durations):
    return gw.gw_stream_pool_simulate(max_active, durations)


def test_instant_operations_release_half_of_the_completed(lib):
    # 4 streams made lazily; at each threshold all 4 are complete and only
    # the oldest 2 are released
    so, st = sim(4, [0] * 10)
    assert so.tolist() == [0, 1, 2, 3, 0, 1, 2, 3, 0, 1]
    assert st["created"] == 4 and st["peak_active"] == 4
    assert st["partial_syncs"] == 3 and st["released"] == 6
    assert st["waited_oldest"] == 0 and st["reuses"] == 6


def test_nothing_complete_waits_for_the_oldest(lib):
    # durations of 100 ticks: op 4 waits for stream 0 (clock -> 100); then
    # streams 1, 2, 3 have finished one at a time (each partial sync finds
    # exactly one complete); op 8 waits for stream 0 again (clock -> 200)
    so, st = sim(4, [100] * 10)
    assert so.tolist() == [0, 1, 2, 3, 0, 1, 2, 3, 0, 1]
    assert st["partial_syncs"] == 6 and st["waited_oldest"] == 2
    assert st["released"] == 6


def test_three_of_four_complete_releases_two(lib):
    # at op 4 (tick 4) streams 0, 1, 2 are complete and 3 runs until 103:
    # ceil(3 / 2) = 2 are released (0 and 1); op 5 then finds 3 active and
    # takes the idle stream 1 without a second partial sync
    d = [0, 0, 0, 100] + [0] * 2
    so, st = sim(4, d)
    assert so.tolist() == [0, 1, 2, 3, 0, 1]
    assert st["partial_syncs"] == 1 and st["released"] == 2
    assert st["active"] == 4 and st["idle"] == 0


def test_limit_one_serialises(lib):
    so, st = sim(1, [5, 5, 5])
    assert so.tolist() == [0, 0, 0]
    assert st["created"] == 1 and st["waited_oldest"] == 2


@pytest.mark.parametrize("max_active", [1, 2, 3, 8, 17])
def test_invariants_on_random_schedules(lib, max_active):
    rng = np.random.default_rng(2506 + max_active)
    d = rng.integers(0, 40, size=300)
    so, st = sim(max_active, d)
    assert st["created"] <= max_active
    assert st["peak_active"] <= max_active
    assert st["ops"] == 300 and st["reuses"] == 300 - st["created"]
    assert (so >= 0).all() and (so < st["created"]).all()
    assert len(set(so.tolist())) == st["created"]
    # every operation beyond the first max_active needed a released stream
    assert st["released"] >= 300 - max_active


def test_arguments_checked(lib):
    with pytest.raises(gw.GWError):
        sim(0, [1])
    with pytest.raises(gw.GWError):
        sim(65, [1])
    with pytest.raises(gw.GWError):
        sim(4, [1, -1])


def test_host_context_nbi_copies_and_limits(lib):
    s = HostSeg(1 << 20, 2)
    try:
        g = gw.gw_alloc_symmetric(s.ctx, 4096)
        src = np.arange(256, dtype=np.uint8)
        gw.gw_put_nbi(s.ctx, g, 1, 64, src, 256)
        gw.gw_fence(s.ctx)
        gw.gw_quiet(s.ctx)
        dst = np.zeros(256, dtype=np.uint8)
        gw.gw_get_nbi(s.ctx, dst, g, 1, 64, 256)
        assert np.array_equal(dst, src)
        with pytest.raises(gw.GWError):
            gw.gw_put_nbi(s.ctx, g, 1, 4000, src, 256)   # past the block
        gw.gw_set_max_active_streams(s.ctx, 3)
        assert gw.gw_pool_stats_get(s.ctx)["max_active"] == 3
        with pytest.raises(gw.GWError):
            gw.gw_set_max_active_streams(s.ctx, 0)
    finally:
        s.close()


def test_cannon_sizes_and_host_context_refusal(lib):
    """Host-side checks of the Cannon ring's boundary (section 5): segment
    bytes per rank (an A stripe, two B stripe buffers, a C stripe), argument
    validation, and a host-only context refused (the ring needs a device)."""
    n, p = 30240, 4
    ns = n // p
    per = gw.gw_cannon_bytes(n, p)
    assert per >= 3 * ns * n * 2 + ns * n * 4
    assert per <= 3 * ns * n * 2 + ns * n * 4 + 4096
    for bad in ((100, 3), (0, 1), (64, 0), (128, 65)):
        with pytest.raises(gw.GWError):
            gw.gw_cannon_bytes(*bad)
    s = HostSeg(1 << 20, 2)
    try:
        with pytest.raises(gw.GWError) as e:
            gw.gw_cannon_create(s.ctx, 64, 2)
        assert e.value.status == gw.GW_ERR_STATE
    finally:
        s.close()
