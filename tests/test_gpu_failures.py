"""Failure detection without a GPU fault.  Every wait of the step kernel
(mbarrier phases, the device-wide counter of persistent launches) is
bounded; one that runs out sets an error bit, the kernel returns and the
host reads GW_ERR_TIMEOUT.  The self-test entry point makes both kinds of
wait run out on purpose (nothing ever completes them) with a short limit;
the context must stay usable afterwards."""

import time

import numpy as np
import pytest

import workloads
from gpu_util import ensure_built, gpu_run, seg_for
from paper_2506_02486_gb300 import gbwave as gw

pytestmark = pytest.mark.gpu


def test_device_waits_give_up_and_the_context_survives():
    ensure_built()
    with seg_for(24, 24, 24) as seg:
        t0 = time.perf_counter()
        st, bits = gw.gw_selftest_timeout(seg.ctx, 50000)      # 50 ms each
        el = time.perf_counter() - t0
        assert st == gw.GW_ERR_TIMEOUT
        assert bits == 3                     # mbarrier and counter both gave up
        assert 0.09 <= el < 10.0
        # the context is still usable: a small shot runs to the same bits
        vel = workloads.homogeneous(24, 24, 24)
        a = gpu_run(vel, 12, src=(12, 12, 12), f_peak=40.0, seg=seg)
        b = gpu_run(vel, 12, src=(12, 12, 12), f_peak=40.0)
        assert np.abs(a["u"]).max() > 0
        assert np.array_equal(a["u32"], b["u32"])


def test_block_product_waits_give_up_and_the_context_survives():
    """The tensor-core kernel of the Cannon ring: a launch whose producer
    issues no loads runs its MMA and epilogue waits out (50 ms), latches
    the timeout, frees its tensor memory and returns; with either tile shape
    the next run is exact."""
    ensure_built()
    from oracle import cannon as oc
    from paper_2506_02486_gb300.runtime import Segment
    from workloads import matmul as mm
    n, p = 256, 2
    a_bits, bt_bits, a, b = mm.pair(n, 31, "dyadic")
    ref, _ = oc.cannon(a, b, p)
    with Segment(p * (gw.gw_cannon_bytes(n, p) + (1 << 20)), nranks=p) as seg:
        cn = gw.gw_cannon_create(seg.ctx, n, p)
        try:
            gw.gw_cannon_set(cn, a_bits, bt_bits)
            for tile_m in (256, 128):
                gw.gw_cannon_schedule(cn, tile_m, 8)
                t0 = time.perf_counter()
                st, expired = gw.gw_cannon_selftest_timeout(cn, 50000)
                el = time.perf_counter() - t0
                assert st == gw.GW_ERR_TIMEOUT and expired == 1
                assert 0.04 <= el < 10.0
                gw.gw_cannon_run(cn)
                c = np.empty((n, n), dtype=np.float32)
                gw.gw_cannon_read_c(cn, c)
                assert np.array_equal(c.astype(np.float64), ref)
        finally:
            gw.gw_cannon_destroy(cn)
