"""Non-blocking puts and gets on the bounded stream pool (section 3.2): the
copies are ordered after the producer stream given as `after`, overlap the
caller's later work, are complete after a fence on the consumer stream, and
the pool never holds more than MAX_ACTIVE_STREAMS active streams."""

import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Segment

pytestmark = pytest.mark.gpu

NR = 4
BLOCK = 1 << 20            # bytes per rank of the exchanged block


def _ring(seg, limit, rounds, producer, consumer):
    """`rounds` ring exchanges: every rank's source is refilled on the
    producer stream, put into the next rank's block, fenced on the consumer
    stream and read back there."""
    gw.gw_set_max_active_streams(seg.ctx, limit)
    g = gw.gw_alloc_symmetric(seg.ctx, BLOCK)
    n = BLOCK // 4
    src = torch.empty((NR, n), dtype=torch.float32, device="cuda")
    got = []
    for k in range(rounds):
        with torch.cuda.stream(producer):
            for r in range(NR):
                src[r].fill_(float(100 * k + r))
        for r in range(NR):
            # two halves per rank: more operations than streams
            for h in range(2):
                off = h * BLOCK // 2
                gw.gw_put_nbi(seg.ctx, g, (r + 1) % NR, off,
                              src[r].data_ptr() + off, BLOCK // 2, producer)
        gw.gw_fence(seg.ctx, consumer)
        with torch.cuda.stream(consumer):
            out = torch.empty((NR, n), dtype=torch.float32, device="cuda")
            for r in range(NR):
                gw.gw_get(seg.ctx, out[r].data_ptr(), g, r, 0, BLOCK, consumer)
            got.append(out)
        # the producer may not refill the sources before the puts read them
        producer.wait_stream(consumer)
    torch.cuda.synchronize()
    gw.gw_free(seg.ctx, g)
    return [o.cpu().numpy() for o in got]


@pytest.mark.parametrize("limit", [1, 3, 8])
def test_ring_exchange_through_the_pool(limit):
    ensure_built()
    producer = torch.cuda.Stream()
    consumer = torch.cuda.Stream()
    with Segment(64 << 20, nranks=NR) as seg:
        outs = _ring(seg, limit, 6, producer, consumer)
        for k, out in enumerate(outs):
            for r in range(NR):
                assert (out[r] == float(100 * k + (r - 1) % NR)).all(), (k, r)
        st = gw.gw_pool_stats_get(seg.ctx)
        assert st["ops"] == 6 * NR * 2
        assert st["created"] <= limit and st["peak_active"] <= limit
        assert st["fences"] == 6
        assert st["active"] == 0            # fences released them all
        if limit < NR * 2:
            assert st["partial_syncs"] > 0


def test_get_nbi_and_quiet():
    ensure_built()
    with Segment(16 << 20, nranks=2) as seg:
        g = gw.gw_alloc_symmetric(seg.ctx, 1 << 16)
        a = torch.arange(1 << 14, dtype=torch.int32, device="cuda")
        gw.gw_put(seg.ctx, g, 1, 0, a, 1 << 16, None)
        gw.gw_fence(seg.ctx, None)
        b = torch.zeros_like(a)
        torch.cuda.synchronize()
        gw.gw_get_nbi(seg.ctx, b, g, 1, 0, 1 << 16, None)
        gw.gw_quiet(seg.ctx)                # host wait: no stream join
        assert torch.equal(a.cpu(), b.cpu())
        st = gw.gw_pool_stats_get(seg.ctx)
        assert st["active"] == 0 and st["ops"] == 1
