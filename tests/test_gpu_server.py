"""The continuous-batching shot server.

* Every result (receiver traces, final norm and energy) equals the same
  shot run alone through a domain of its own: bit-identical traces and
  identical FP64 checks, whether the shot ran in a mix of FP32 and BF16
  shots, joined a running batch, or waited for memory.
* Every result of the mix also matches the FP64 oracle run of that shot:
  traces within the storage type's bound (FP32 1e-4, FP16 with power-of-
  two scales 5e-3, BF16 6e-2; relative L2), the final sum of u^2 within
  twice that, and the energy within ten times that of the energy's two
  sums (its kinetic sum is built from differences of consecutive fields).
* Admission respects the HBM budget and the slot count, in arrival order.
* Requests that can never fit are refused at submission; waits time out.
"""

import time

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import ensure_built, rel_l2
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Segment, Server, Shot

pytestmark = pytest.mark.gpu

# (nx, ny, nz, steps, dtype, seed)
REQS = [
    (48, 48, 64, 70, "f32", 1),
    (64, 64, 48, 33, "bf16", 2),
    (40, 56, 40, 120, "f32", 3),
    (72, 40, 56, 50, "bf16", 4),
    (56, 56, 56, 90, "f32", 5),
    (32, 48, 80, 26, "f32", 6),
    (64, 48, 64, 61, "f16s", 7),
]
SPONGE = 8


def _vz(nz, seed):
    """Layered profile rounded to FP32 values, so that the FP32 full-model
    path and the FP64 profile path load the same velocities."""
    return workloads.layered_profile(nz, seed).astype(np.float32) \
        .astype(np.float64)


def _vel(nx, ny, nz, seed):
    return np.broadcast_to(_vz(nz, seed)[:, None, None], (nz, ny, nx))


def _src(nx, ny, nz, seed):
    return workloads.source_position(seed, nx, ny, nz, margin=SPONGE)


def _rec(nx, ny, nz, seed):
    """A cross through the source cell (distances 0, 3, 6 along each axis):
    the runs are shorter than the Ricker delay 1 / f, so the wave has not
    gone further."""
    sx, sy, sz = (int(c) for c in _src(nx, ny, nz, seed))
    pts = {(sx, sy, sz)}
    for d in (3, 6):
        pts |= {(sx + d, sy, sz), (sx, sy + d, sz), (sx, sy, sz + d)}
    return np.array(sorted(pts), dtype=np.int32)


def _alone(seg, spec):
    nx, ny, nz, steps, dtype, seed = spec
    with Shot(seg, nx, ny, nz, nsteps=steps, dtype=dtype,
              sponge=SPONGE) as s:
        s.set_model(_vel(nx, ny, nz, seed))
        s.add_ricker(_src(nx, ny, nz, seed), 25.0)
        s.set_receivers(_rec(nx, ny, nz, seed))
        s.step(steps)
        s.sync()
        n2, en = s.check()
        return s.traces(steps), n2, en


def _submit(srv, spec, full_model=False):
    nx, ny, nz, steps, dtype, seed = spec
    kw = {}
    if full_model:
        kw["vel"] = _vel(nx, ny, nz, seed)
    else:
        kw["vz"] = _vz(nz, seed)
    return srv.submit(nx, ny, nz, steps, src=_src(nx, ny, nz, seed),
                      f_peak=25.0, receivers=_rec(nx, ny, nz, seed), dtype=dtype,
                      sponge=SPONGE, **kw)


@pytest.fixture(scope="module")
def alone():
    ensure_built()
    with Segment(1 << 30) as seg:
        return [_alone(seg, spec) for spec in REQS]


BOUND = {"f32": 1e-4, "f16s": 5e-3, "bf16": 6e-2}


@pytest.fixture(scope="module")
def oracle_runs():
    out = []
    for nx, ny, nz, steps, dtype, seed in REQS:
        vel = np.ascontiguousarray(_vel(nx, ny, nz, seed))
        o = oracle.run(vel, 10.0, steps, dt=oracle.time_step(10.0, float(vel.max())),
                       src=_src(nx, ny, nz, seed), f_peak=25.0, sponge=SPONGE,
                       receivers=_rec(nx, ny, nz, seed), norms=True, nthreads=8)
        coef = (vel * o["dt"] / 10.0) ** 2
        d = o["u"] - o["u_prev"]
        kin = float(np.sum(d * d / coef))
        pot = float(np.sum(o["u"] * oracle.laplacian(oracle.pad(o["u_prev"]))))
        out.append({"traces": o["traces"], "norm2": float(o["norms"][-1]),
                    "energy": oracle.energy(coef, o["u"], o["u_prev"]),
                    "scale": abs(kin) + abs(pot)})
    return out


def _check_oracle(res, o, dtype):
    tol = BOUND[dtype]
    assert np.abs(o["traces"]).max() > 0
    assert rel_l2(res["traces"], o["traces"]) <= tol
    assert abs(res["norm2"] - o["norm2"]) <= 2 * tol * o["norm2"]
    assert abs(res["energy"] - o["energy"]) <= 10 * tol * o["scale"]


def _check_same(res, ref):
    traces, n2, en = ref
    assert res["status"] == gw.GW_OK
    assert np.array_equal(res["traces"], traces)
    assert res["norm2"] == n2 and res["energy"] == en
    assert n2 > 0


def test_mixed_shots_equal_alone(alone, oracle_runs):
    with Segment(2 << 30) as seg, Server(seg, 1 << 30, max_slots=8) as srv:
        tickets = [_submit(srv, spec, full_model=(i % 2 == 0))
                   for i, spec in enumerate(REQS)]
        results = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    for res, ref, o, spec in zip(results, alone, oracle_runs, REQS):
        _check_same(res, ref)
        _check_oracle(res, o, spec[4])
        assert res["submit_s"] <= res["admit_s"] <= res["done_s"]
    assert st["completed"] == len(REQS)
    assert st["max_active"] >= 2
    assert st["point_updates"] >= sum(nx * ny * nz * k
                                      for nx, ny, nz, k, _, _ in REQS)


def test_budget_and_slots_limit_admission(alone):
    """A budget that fits about two of these shots and two slots: admission
    waits for retirements, in arrival order, and results do not change."""
    fp = [gw.gw_domain_bytes(gw.shot_desc(nx, ny, nz, nsteps=k, dtype=dt,
                                          sponge=SPONGE), nrec=9)
          for nx, ny, nz, k, dt, _ in REQS]
    budget = max(fp) + sorted(fp)[-2]
    with Segment(2 << 30) as seg, Server(seg, budget, max_slots=2) as srv:
        tickets = [_submit(srv, spec) for spec in REQS]
        results = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    for res, ref in zip(results, alone):
        _check_same(res, ref)
    assert st["max_active"] <= 2
    assert st["peak_bytes"] <= budget
    admits = [r["admit_s"] for r in results]
    assert admits == sorted(admits)
    # some shot had to wait for another to retire
    assert any(r["admit_s"] >= min(q["done_s"] for q in results) for r in results)


def test_shots_joining_a_running_batch(alone):
    with Segment(2 << 30) as seg, Server(seg, 1 << 30, chunk=10) as srv:
        first = [_submit(srv, REQS[i]) for i in (2, 4)]
        time.sleep(0.05)
        later = [_submit(srv, REQS[i]) for i in (0, 1, 3, 5, 6)]
        res = {i: srv.wait(t, 60000) for i, t in zip((2, 4), first)}
        res.update({i: srv.wait(t, 60000)
                    for i, t in zip((0, 1, 3, 5, 6), later)})
        st = srv.stats()
    for i, r in res.items():
        _check_same(r, alone[i])
    assert st["rebuilds"] >= 2


def test_refusals_and_timeouts():
    ensure_built()
    with Segment(1 << 30) as seg, Server(seg, 64 << 20, max_slots=4) as srv:
        with pytest.raises(gw.GWError) as e:
            srv.submit(400, 400, 400, 10, src=(200, 200, 200),
                       vz=np.full(400, 2000.0))
        assert e.value.status == gw.GW_ERR_BUDGET
        t = srv.submit(64, 64, 64, 4000, src=(32, 32, 32),
                       vz=np.full(64, 2000.0))
        with pytest.raises(gw.GWError) as e:
            srv.wait(t, 0)
        assert e.value.status == gw.GW_ERR_TIMEOUT
        r = srv.wait(t, 120000)
        assert r["status"] == gw.GW_OK and r["steps"] == 4000
        with pytest.raises(gw.GWError) as e:
            srv.wait(t, 0)              # returned once
        assert e.value.status == gw.GW_ERR_ARG


def test_destroy_with_work_outstanding():
    ensure_built()
    with Segment(1 << 30) as seg:
        srv = Server(seg, 256 << 20, max_slots=1)
        for _ in range(3):
            srv.submit(96, 96, 96, 2000, src=(48, 48, 48),
                       vz=np.full(96, 2500.0))
        time.sleep(0.05)
        t0 = time.perf_counter()
        srv.close()
        assert time.perf_counter() - t0 < 30
