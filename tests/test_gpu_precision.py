"""Precision of the storage types on a 128^3 crop of the 1024 x 1024 x 512
perturbed layered model (20-cell sponge, 20 Hz source at the crop centre,
500 steps).

* The FP64 GPU path is checked against the FP64 oracle: relative L2
  <= 1e-10 (both FP64; the difference is summation order).
* The other storage types are measured against that FP64 GPU path: FP32
  (3-level) <= 1e-4; FP16 x 2^k delta storage <= 5e-3, the accuracy bar
  set for mixed-precision storage; BF16 delta storage is reported, with a
  loose bound (8 significand bits cannot meet 5e-3 over 500 steps).
"""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import gpu_run, rel_l2

pytestmark = pytest.mark.gpu

N = 128
STEPS = 500


@pytest.fixture(scope="module")
def crop():
    return workloads.perturbed_box(crop=(N, N, N), nsteps=STEPS)


@pytest.fixture(scope="module")
def fp64(crop):
    vel = crop.vel.astype(np.float64)
    return gpu_run(vel, STEPS, src=crop.src, f_peak=crop.f_peak,
                   receivers=crop.receivers, sponge=crop.sponge, dtype="f64")


def test_fp64_gpu_path_matches_oracle(crop, fp64):
    vel = crop.vel.astype(np.float64)
    dt = oracle.time_step(crop.h, float(vel.max()))
    o = oracle.run(vel, crop.h, STEPS, dt=dt, src=crop.src, f_peak=crop.f_peak,
                   sponge=crop.sponge, receivers=crop.receivers, nthreads=16)
    assert np.abs(o["u"]).max() > 0
    assert rel_l2(fp64["u"], o["u"]) <= 1e-10
    # traces are kept in FP32 whatever the arithmetic type: rounding only
    assert rel_l2(fp64["traces"], o["traces"]) <= 1e-7


@pytest.mark.parametrize("dtype,bound", [("f32", 1e-4), ("f16s", 5e-3),
                                         ("bf16", 6e-2)])
def test_storage_error_against_fp64(crop, fp64, dtype, bound):
    vel = crop.vel.astype(np.float64)
    g = gpu_run(vel, STEPS, src=crop.src, f_peak=crop.f_peak,
                receivers=crop.receivers, sponge=crop.sponge, dtype=dtype)
    err = rel_l2(g["u"], fp64["u"])
    maxabs = float(np.abs(g["u"] - fp64["u"]).max())
    print(f"\n{dtype}: rel L2 {err:.3e}, max abs {maxabs:.3e} "
          f"(max |u| {np.abs(fp64['u']).max():.3e}), traces rel L2 "
          f"{rel_l2(g['traces'], fp64['traces']):.3e}")
    assert err <= bound
