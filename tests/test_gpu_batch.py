"""Batched multi-shot launches: shots of different sizes, tiles, sponge
settings and decompositions advanced together by gw_batch_step.

Each shot of a batch must end bit-identical (wavefield and receiver traces)
to the same shot stepped alone with the same kernel tile: the per-point
arithmetic does not depend on which launch, CTA or z-chunk computes a
point.  Per-step norms are FP64 sums over a different set of work items,
so they agree to rounding (1e-12 relative).  Every batched shot is also
checked against the FP64 oracle run of the same shot: FP32 within 1e-4,
FP64 within 1e-10 (relative L2 and point by point), the 16-bit storage
types within their stated bounds against FP64 (FP16 with power-of-two
scales 5e-3, BF16 6e-2).
"""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import assert_close, ensure_built, rel_l2
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Batch, Segment, Shot, shot_bytes

pytestmark = pytest.mark.gpu

STEPS = 60
# (nx, ny, nz, px, py, pz, sponge, tile)
SHOTS = [
    (48, 48, 48, 1, 1, 1, 8, 0),
    (64, 40, 56, 1, 1, 1, 8, 0),
    (37, 41, 29, 1, 1, 1, 0, 0),
    (64, 48, 40, 2, 1, 1, 8, 0),
    (40, 40, 72, 1, 1, 2, 8, 2),
]


def _make(seg, k, spec, dtype):
    nx, ny, nz, px, py, pz, sponge, tile = spec
    s = Shot(seg, nx, ny, nz, px=px, py=py, pz=pz, nsteps=STEPS,
             dtype=dtype, sponge=sponge, tile=tile)
    s.set_model(workloads.layered(nx, ny, nz, seed=100 + k))
    s.add_ricker((nx // 2, ny // 3, nz // 2), 30.0)
    s.set_receivers(_receivers(spec))
    return s


def _receivers(spec):
    """A cross through the source cell (distances 0, 2, 4 along each axis):
    within STEPS steps (shorter than the Ricker delay 1 / f) the wave has
    not travelled further, and ahead of it the values are ~1e-38 noise that
    16-bit storage rightly flushes to zero."""
    nx, ny, nz = spec[:3]
    sx, sy, sz = nx // 2, ny // 3, nz // 2
    pts = {(sx, sy, sz)}
    for d in (2, 4):
        pts |= {(sx + d, sy, sz), (sx, sy + d, sz), (sx, sy, sz + d)}
    return np.array(sorted(pts), dtype=np.int32)


def _result(s):
    return {"u": s.u(f64=True), "traces": s.traces(STEPS),
            "norms": s.norms(STEPS)}


# bound against the FP64 oracle per storage type
BOUND = {"f32": 1e-4, "f64": 1e-10, "f16s": 5e-3, "bf16": 6e-2}
_oracle_cache = {}


def _oracle(k):
    """FP64 oracle run of SHOTS[k] (the inputs _make gives the library)."""
    if k not in _oracle_cache:
        nx, ny, nz, px, py, pz, sponge, tile = SHOTS[k]
        vel = workloads.layered(nx, ny, nz, seed=100 + k)
        rec = _receivers(SHOTS[k])
        _oracle_cache[k] = oracle.run(
            vel, 10.0, STEPS, dt=oracle.time_step(10.0, float(vel.max())),
            src=(nx // 2, ny // 3, nz // 2), f_peak=30.0, sponge=sponge,
            receivers=rec, nthreads=8)
    return _oracle_cache[k]


def _against_oracle(k, r, dtype):
    o = _oracle(k)
    tol = BOUND[dtype]
    u = r["u"].astype(np.float64)
    assert np.abs(o["traces"]).max() > 1e-2 * np.abs(o["u"]).max(), k
    if dtype in ("f32", "f64"):
        assert_close(u, o["u"], tol, f"shot {k} u")
        # traces are recorded in FP32 for every storage type
        assert_close(r["traces"], o["traces"], max(tol, 2.0 ** -23), f"shot {k} traces")
    else:
        # 16-bit storage: the stated bounds are relative L2 bounds
        assert rel_l2(u, o["u"]) <= tol, (k, rel_l2(u, o["u"]))
        assert rel_l2(r["traces"], o["traces"]) <= tol, (k, rel_l2(r["traces"], o["traces"]))


def _seg_bytes(dtype):
    return sum(shot_bytes(nx, ny, nz, dtype, STEPS, 9, px, py, pz)
               for nx, ny, nz, px, py, pz, _, _ in SHOTS)


@pytest.mark.parametrize("dtype,mode", [
    ("f32", "graphs"), ("f32", "plain"), ("f32", "persistent"),
    ("bf16", "graphs"), ("bf16", "persistent"), ("f16s", "persistent"),
    ("f64", "graphs")])
def test_batched_shots_match_alone(dtype, mode):
    """Three groups (two tiles, with and without the sponge): side by side
    on forked streams, or one cooperative launch per group and chunk."""
    ensure_built()
    alone = []
    with Segment(2 * _seg_bytes(dtype), nranks=2) as seg:
        for k, spec in enumerate(SHOTS):
            with _make(seg, k, spec, dtype) as s:
                s.step(STEPS)
                s.sync()
                alone.append(_result(s))
    chunk = -25 if mode == "plain" else 0
    with Segment(2 * _seg_bytes(dtype), nranks=2) as seg:
        shots = [_make(seg, k, spec, dtype) for k, spec in enumerate(SHOTS)]
        try:
            with Batch(seg, shots, chunk=chunk,
                       persistent=(mode == "persistent")) as b:
                info = b.info
                # tile 2 and the sponge-free shot form their own groups
                assert info["groups"] == 3
                b.step(STEPS - 20)
                b.step(20)
                shots[0].sync()
            for k, s in enumerate(shots):
                r = _result(s)
                a = alone[k]
                assert np.array_equal(r["u"], a["u"]), k
                assert np.array_equal(r["traces"], a["traces"]), k
                np.testing.assert_allclose(r["norms"], a["norms"],
                                           rtol=1e-12, atol=0)
                assert np.abs(a["u"]).max() > 0
                _against_oracle(k, r, dtype)
        finally:
            for s in shots:
                s.close()


def test_batch_then_alone_continues_the_same_shot():
    """A shot stepped partly in a batch and partly alone equals a shot
    stepped alone throughout (the batch advances the shot's own step)."""
    ensure_built()
    spec = SHOTS[0]
    with Segment(_seg_bytes("f32")) as seg:
        with _make(seg, 0, spec, "f32") as s:
            s.step(STEPS)
            s.sync()
            ref = _result(s)
        with _make(seg, 0, spec, "f32") as s, _make(seg, 1, SHOTS[1],
                                                    "f32") as t:
            with Batch(seg, [s, t]) as b:
                b.step(30)
            s.step(STEPS - 30)
            s.sync()
            r = _result(s)
    assert np.array_equal(r["u"], ref["u"])
    assert np.array_equal(r["traces"], ref["traces"])


def test_batch_rejects_mixed_types():
    ensure_built()
    with Segment(_seg_bytes("f32") * 4, nranks=2) as seg:
        a = _make(seg, 0, SHOTS[0], "f32")
        b = _make(seg, 1, SHOTS[0], "bf16")
        try:
            with pytest.raises(gw.GWError) as e:
                Batch(seg, [a, b])
            assert e.value.status == gw.GW_ERR_ARG
        finally:
            for s in (a, b):
                s.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_separate_halo_shots_in_a_batch_match_alone(persistent):
    """Decomposed shots whose halos a copy kernel moves after each step
    (the compute-put-fence order of Listing 1) form their own group; the
    results equal the same shots alone, bit for bit."""
    ensure_built()
    specs = [(64, 48, 40, 2, 1, 1, 8, 0), (40, 56, 48, 1, 2, 2, 8, 0),
             (48, 48, 48, 1, 1, 1, 8, 0)]

    def make(seg, k, spec):
        nx, ny, nz, px, py, pz, sponge, tile = spec
        s = Shot(seg, nx, ny, nz, px=px, py=py, pz=pz, nsteps=STEPS,
                 sponge=sponge, halo_mode=gw.GW_HALO_SEPARATE)
        s.set_model(workloads.layered(nx, ny, nz, seed=200 + k))
        s.add_ricker((nx // 2, ny // 3, nz // 2), 30.0)
        s.set_receivers(workloads.lattice_receivers(nx, ny, nz // 4, n=3,
                                                    margin=2))
        return s

    nbytes = 8 * sum(shot_bytes(nx, ny, nz, "f32", STEPS, 9, px, py, pz)
                     for nx, ny, nz, px, py, pz, _, _ in specs)
    with Segment(nbytes, nranks=4) as seg:
        alone = []
        for k, spec in enumerate(specs):
            with make(seg, k, spec) as s:
                s.step(STEPS)
                s.sync()
                alone.append(_result(s))
        shots = [make(seg, k, spec) for k, spec in enumerate(specs)]
        try:
            with Batch(seg, shots, persistent=persistent) as b:
                assert b.info["groups"] == 2      # separate halos / none
                b.step(STEPS)
                shots[0].sync()
            for k, s in enumerate(shots):
                r = _result(s)
                assert np.array_equal(r["u"], alone[k]["u"]), k
                assert np.array_equal(r["traces"], alone[k]["traces"]), k
        finally:
            for s in shots:
                s.close()


def test_batch_timing_counts_steps():
    ensure_built()
    with Segment(_seg_bytes("f32")) as seg:
        shots = [_make(seg, k, spec, "f32")
                 for k, spec in enumerate(SHOTS[:2])]
        try:
            with Batch(seg, shots) as b:
                b.timing(True)
                b.step(10)
                st = b.stats()
            assert st["launches"] == 10
            assert st["total_ms"] > 0
        finally:
            for s in shots:
                s.close()


def test_autotune_picks_an_available_tile_and_caches_it():
    ensure_built()
    n = 96
    # room for the planner's full-occupancy scratch shot (96 x 96 x 4096)
    with Segment(6 * shot_bytes(n, n, n, "f32", 16) + (2 << 30)) as seg:
        d = gw.shot_desc(n, n, n, nsteps=16, sponge=10)
        t1, ms1, all1 = gw.gw_autotune(seg.ctx, d, 1, 1, 1, 5, all_times=True)
        t2, ms2 = gw.gw_autotune(seg.ctx, d, 1, 1, 1, 5)
        assert t1 >= 1 and ms1 > 0
        assert (t1, ms1) == (t2, ms2)
        assert len(all1) == gw.gw_tile_count("f32")
        assert ms1 == min(t for t in all1 if t > 0) == all1[t1 - 1]
        # planning: with an unreachable margin every shot gets one tile; with
        # margin 0 each shape keeps its own best tile unless one tile is
        # at least as fast in sum
        d2 = gw.shot_desc(n + 16, n, n, nsteps=16, sponge=10)
        uni = gw.gw_plan_tiles(seg.ctx, [d, d2, d], 5, margin=1.0)
        assert len(set(uni)) == 1
        own = gw.gw_plan_tiles(seg.ctx, [d, d2], 5, margin=0.0)
        # the plan times each shape at full occupancy: its x-y plane over
        # enough planes for 64 M points (cached, so this is the plan's own
        # timing)
        tall = gw.shot_desc(n, n, min(4096, (64 << 20) // (n * n)), nsteps=16, sponge=10)
        t_plan = gw.gw_autotune(seg.ctx, tall, 1, 1, 1, 5)[0]
        assert own[0] == t_plan or len(set(own)) == 1
        # the chosen tile builds and runs
        with Shot(seg, n, n, n, nsteps=16, sponge=10, tile=t1) as s:
            s.set_model(workloads.homogeneous(n, n, n))
            s.step(4)
            s.sync()
            assert s.info["tile"] == t1


def test_persistent_batch_with_a_one_row_per_thread_tile():
    """A persistent batch whose groups include a two-CTAs-per-SM tile
    (128 x 7, one row per thread) next to the default one: each group's
    cooperative launch covers its own occupancy; results are those of the
    shots alone."""
    ensure_built()
    specs = [(48, 48, 48, 1, 1, 1, 8, 0), (64, 40, 56, 1, 1, 1, 8, 7)]
    alone = []
    with Segment(2 * _seg_bytes("f32")) as seg:
        for k, spec in enumerate(specs):
            with _make(seg, k, spec, "f32") as s:
                s.step(STEPS)
                s.sync()
                alone.append(_result(s))
        shots = [_make(seg, k, spec, "f32") for k, spec in enumerate(specs)]
        try:
            with Batch(seg, shots, persistent=True) as b:
                assert b.info["groups"] == 2
                b.step(STEPS)
                shots[0].sync()
            for k, s in enumerate(shots):
                r = _result(s)
                assert np.array_equal(r["u"], alone[k]["u"]), k
                assert np.array_equal(r["traces"], alone[k]["traces"]), k
        finally:
            for s in shots:
                s.close()
