"""Cannon's ring exchange on the tensor cores (section 5, matrix
multiplication) against the FP64 oracle: bit for bit on dyadic inputs (whose
FP32 sums are exact in any order), within the FP32 accumulation bound on
uniform BF16 inputs; the ring of P ranks gives the bits of the single
product (P = 1); ragged stripes and K tails; repeated runs."""

import numpy as np
import pytest

from gpu_util import ensure_built
from oracle import cannon as oc
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Segment
from workloads import matmul as mm

pytestmark = pytest.mark.gpu


def cannon_gpu(a_bits, bt_bits, n, p, runs=1, stats=False, tile_m=256, group=4):
    ensure_built()
    per = gw.gw_cannon_bytes(n, p)
    with Segment(p * (per + (1 << 20)), nranks=p) as seg:
        cn = gw.gw_cannon_create(seg.ctx, n, p)
        try:
            gw.gw_cannon_schedule(cn, tile_m, group)
            gw.gw_cannon_set(cn, a_bits, bt_bits)
            out = []
            for _ in range(runs):
                gw.gw_cannon_run(cn, None)
                c = np.empty((n, n), dtype=np.float32)
                gw.gw_cannon_read_c(cn, c)
                out.append(c)
            pool = gw.gw_pool_stats_get(seg.ctx)
        finally:
            gw.gw_cannon_destroy(cn)
    return (out, pool) if stats else out


@pytest.mark.parametrize("tile_m", [256, 128])
@pytest.mark.parametrize("n,p", [(256, 2), (328, 4), (384, 3), (512, 1),
                                 (1152, 3), (1800, 2)])
def test_dyadic_inputs_bit_exact(n, p, tile_m):
    """Ragged cases: 328 / 4 = 82 rows per stripe (one partial tile) and a
    K tail of 8; 1152 / 3 = 384 rows (one and a half 256-row tiles, three
    128-row tiles); 1800 / 2 = 900 rows and columns (3.5 tiles of 256 each
    way, 7.03 of 128) with a K tail of 8: more tiles than one CTA per SM
    when P = 2 at 128 rows."""
    a_bits, bt_bits, a, b = mm.pair(n, 100 + n + p, "dyadic")
    ref, _ = oc.cannon(a, b, p)
    (c,) = cannon_gpu(a_bits, bt_bits, n, p, tile_m=tile_m)
    assert np.array_equal(c.astype(np.float64), ref)


def test_uniform_inputs_within_fp32_bound():
    n, p = 640, 4
    a_bits, bt_bits, a, b = mm.pair(n, 7, "uniform")
    ref, _ = oc.cannon(a, b, p)
    (c,) = cannon_gpu(a_bits, bt_bits, n, p)
    bound = oc.fp32_sum_bound(n, np.abs(a) @ np.abs(b))
    err = np.abs(c.astype(np.float64) - ref)
    assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())
    rel = np.linalg.norm(c - ref) / np.linalg.norm(ref)
    assert rel < 1e-6


def test_ring_gives_the_bits_of_the_single_product():
    """Each element's sum runs over the same K blocks in the same order
    whatever the stripe, tile shape or raster group it falls in."""
    n = 768
    a_bits, bt_bits, _, _ = mm.pair(n, 17, "uniform")
    (one,) = cannon_gpu(a_bits, bt_bits, n, 1, tile_m=128)
    for p in (1, 2, 3, 4, 6):
        (c,) = cannon_gpu(a_bits, bt_bits, n, p)
        assert np.array_equal(c, one), p
    for tile_m, group in ((128, 1), (256, 1), (128, 3), (256, 2), (128, 64),
                          (256, 16), (256, 1024)):
        (c,) = cannon_gpu(a_bits, bt_bits, n, 2, tile_m=tile_m, group=group)
        assert np.array_equal(c, one), (tile_m, group)


def test_repeated_runs_and_pool_use():
    n, p = 512, 4
    a_bits, bt_bits, a, b = mm.pair(n, 23, "dyadic")
    ref, _ = oc.cannon(a, b, p)
    outs, pool = cannon_gpu(a_bits, bt_bits, n, p, runs=3, stats=True)
    for c in outs:
        assert np.array_equal(c.astype(np.float64), ref)
    # p puts per ring step, p - 1 steps with puts per run
    assert pool["ops"] == 3 * p * (p - 1)
    assert pool["fences"] == 3 * (p - 1)
    assert pool["peak_active"] <= pool["max_active"]


def test_arguments_checked():
    ensure_built()
    with pytest.raises(gw.GWError):
        gw.gw_cannon_bytes(100, 3)               # N not a multiple of P
    with Segment(8 << 20, nranks=2) as seg:
        with pytest.raises(gw.GWError):
            gw.gw_cannon_create(seg.ctx, 96, 4)  # more ranks than the segment
        with pytest.raises(gw.GWError):
            gw.gw_cannon_create(seg.ctx, 100, 2)  # rows not 16-byte multiples
        cn = gw.gw_cannon_create(seg.ctx, 96, 2)
        try:
            for bad in ((64, 8), (192, 8), (256, 0), (128, 2000), (512, 8)):
                with pytest.raises(gw.GWError):
                    gw.gw_cannon_schedule(cn, *bad)
        finally:
            gw.gw_cannon_destroy(cn)


def test_paper_size_sampled_entries_exact():
    """The paper's 30240 x 30240 product on 4 ring ranks, the launch
    configuration the benchmark times: sampled entries against the oracle's
    one-by-one FP64 sums (exact for dyadic inputs), plus the entries of the
    last rows and columns (ragged tiles: 7560 = 29 x 256 + 136 rows and
    columns per stripe block)."""
    n, p = 30240, 4
    ka = mm.dyadic_codes(n, n, 2506)
    kb = mm.dyadic_codes(n, n, 2507)
    (c,) = cannon_gpu(mm.dyadic_bits(ka), mm.dyadic_bits(kb), n, p)
    rng = np.random.default_rng(1)
    idx = [tuple(rng.integers(0, n, 2)) for _ in range(200)]
    idx += [(n - 1, n - 1), (n - 1, 0), (0, n - 1), (7559, 7560), (7560, 7559),
            (15119, 22679), (22680, 30239)]
    for i, j in idx:
        ref = oc.entry(mm.dyadic_values(ka[i:i + 1]), mm.dyadic_values(kb[j:j + 1]).T, 0, 0)
        assert c[i, j] == ref, (i, j, c[i, j], ref)
