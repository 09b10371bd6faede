"""The model precompute (rows a1): the FP32 model call against the FP64 one,
and the integer FP64 -> FP32 rounding the FP32 path uses against IEEE 754
round-to-nearest-even (numpy's conversion)."""

import numpy as np
import pytest

import workloads
from gpu_util import seg_for
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Shot

pytestmark = pytest.mark.gpu


def _f32_bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def _rounding_cases(rng):
    """Doubles that exercise every branch of a narrowing conversion: random
    values over FP32's normal range (both signs), exact ties between two
    FP32 neighbours (even and odd lower neighbour), values a hair above and
    below a tie, carries into the exponent, the largest finite FP32 and the
    tie above it (which rounds to infinity), FP32 subnormals and values
    below them, zeros, infinities and NaN."""
    n = 200_000
    mag = np.exp2(rng.uniform(-125.9, 127.9, n))
    rnd = mag * rng.choice([-1.0, 1.0], n)
    f = rng.uniform(1.0, 2.0, 50_000).astype(np.float32)
    f = f * np.exp2(rng.integers(-120, 120, f.size)).astype(np.float32)
    lo = f.astype(np.float64)
    hi = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    tie = lo + (hi - lo) / 2                       # exact in FP64
    eps = np.abs(tie) * 2.0 ** -50
    near = np.concatenate([tie, tie + eps, tie - eps, -tie])
    # all-ones significands: rounding up carries into the exponent
    ones = (np.float32(2.0) - np.float32(2.0 ** -23)) * np.exp2(
        np.arange(-120, 127)).astype(np.float32)
    o64 = ones.astype(np.float64)
    carry = np.concatenate([o64 + o64 * 2.0 ** -25, o64 + o64 * 2.0 ** -24 * (1 - 2.0 ** -20)])
    fmax = float(np.finfo(np.float32).max)
    edge = np.array([fmax, fmax + 2.0 ** 103, fmax + 2.0 ** 102, -fmax - 2.0 ** 103,
                     2.0 ** 128, 2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -30),
                     2.0 ** -130, 2.0 ** -149, 2.0 ** -150, 2.0 ** -151, 1e-300,
                     0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, 1.5, 3.0e38, 1e39])
    return np.concatenate([rnd, near, carry, edge])


def test_round_to_f32_is_ieee_nearest_even():
    import torch
    rng = np.random.default_rng(2506)
    x = _rounding_cases(rng)
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)                # IEEE round to nearest even
    d_in = torch.from_numpy(x).cuda()
    d_out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    gw.gw_round_to_f32(d_in, d_out, x.size)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    assert np.array_equal(_f32_bits(got), _f32_bits(want))
    nan = torch.tensor([np.nan, -np.nan], dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    gw.gw_round_to_f32(nan, out, 2)
    assert torch.isnan(out).all()


def test_round_to_f32_rejects_null_arrays():
    with pytest.raises(gw.GWError) as e:
        gw.gw_round_to_f32(None, None, 4)
    assert e.value.status == gw.GW_ERR_ARG
    gw.gw_round_to_f32(None, None, 0)              # nothing to do


@pytest.mark.parametrize("dtype,dec", [("f32", (1, 1, 1)), ("f32", (2, 1, 2)),
                                       ("f64", (1, 1, 1)), ("f16s", (1, 1, 1)),
                                       ("bf16", (1, 1, 1))])
def test_fp32_model_call_gives_the_bits_of_the_fp64_call(dtype, dec):
    """gw_set_model_f32 on FP32 velocities and gw_set_model on the same
    values in FP64: the same time step, the same coefficient bits and so the
    same run.  For FP32 and FP64 storage the FP32 call stores v and forms
    (v dt / h)^2 in place (FP32 storage: converting to and from FP64 in
    integer arithmetic), the FP64 call forms it from its input; for 16-bit
    storage both take the same route.  The model carries a 5 % i.i.d.
    perturbation, so its values cover many significands."""
    nx, ny, nz = 71, 53, 67
    rng = np.random.default_rng(31)
    vel = workloads.layered(nx, ny, nz, seed=31)
    vel = vel * (1.0 + 0.05 * rng.standard_normal(vel.shape))
    v32 = np.ascontiguousarray(vel, dtype=np.float32)
    runs = []
    for f32 in (False, True):
        with seg_for(nx, ny, nz, dtype, *dec) as seg:
            with Shot(seg, nx, ny, nz, px=dec[0], py=dec[1], pz=dec[2],
                      nsteps=20, dtype=dtype, sponge=5) as s:
                if f32:
                    gw.gw_set_model_f32(s.dom, v32)
                else:
                    gw.gw_set_model(s.dom, v32.astype(np.float64))
                dt = s.info["dt"]
                coef = s.u(gw.GW_FIELD_COEF, f64=True)
                s.add_ricker((35, 26, 33), 30.0)
                s.step(20)
                s.sync()
                runs.append((dt, coef, s.u(f64=True)))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])
    assert np.abs(runs[0][2]).max() > 0
    # the coefficients themselves: (v dt / h)^2 in FP64, rounded once more
    # to storage (FP32 here; checked against numpy's rounding)
    if dtype == "f32":
        want = np.square(v32.astype(np.float64) * (dt / 10.0)).astype(np.float32)
        assert np.array_equal(runs[1][1].astype(np.float32), want)
