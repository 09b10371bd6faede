"""gw_check_fields_noalloc -- the allocation-free variant of gw_check, for
callers that cannot allocate device memory (for example code running while
another framework holds its memory pool).  Its per-plane partial sums live
in a built-in device array instead of memory the call would allocate.

For each storage type (FP32; FP16 with a power-of-two scale of 2^6; BF16)
the test runs a small shot, reads its fields back, lays the stored values
out again in device arrays of that storage type that the test owns, and
checks two calls in a row of the allocation-free entry point:

* against gw_check on the shot: bit for bit, since both run the same plane
  sums in the same order;
* against the oracle's energy of the same fields (FP64, another order of
  the same sums): to 1e-12 of the energy's two sums;
* that free device memory is the same before and after the two calls.

This file is collected last, so that a run stopping at the first failure
has already run every other test."""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import seg_for
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Shot

pytestmark = pytest.mark.gpu

# storage type -> (x offset of the interior in a padded row, element type of
# the fields, element type of coef, scale of u)
LAYOUT = {"f32": (8, "float32", "float32", 1.0),
          "f16s": (16, "float16", "float16", 64.0),
          "bf16": (16, "bfloat16", "float16", 1.0)}


def padded(a, px, xo, dtype):
    """Interior (nz, ny, nx) values in the library's padded layout, halo
    cells zero (the shot's zero boundary)."""
    import torch
    nz, ny, nx = a.shape
    out = torch.zeros((nz + 8, ny + 8, px), dtype=getattr(torch, dtype), device="cuda")
    out[4:4 + nz, 4:4 + ny, xo:xo + nx] = torch.from_numpy(
        np.ascontiguousarray(a, dtype=np.float64)).to("cuda", getattr(torch, dtype))
    return out


@pytest.mark.parametrize("dtype", ["f32", "f16s", "bf16"])
def test_noalloc_check_matches_gw_check_twice(dtype):
    import torch
    xo, ft, ct, su = LAYOUT[dtype]
    nx, ny, nz = 45, 38, 31
    vel = workloads.layered(nx, ny, nz, seed=17)
    with seg_for(nx, ny, nz, dtype, extra=64 << 20) as seg:
        desc = {"scale_u": su, "scale_w": su} if dtype == "f16s" else {}
        with Shot(seg, nx, ny, nz, nsteps=40, dtype=dtype, sponge=4, **desc) as s:
            s.set_model(vel)
            s.add_ricker((20, 19, 15), 40.0)
            s.step(30)
            norm2, energy = s.check()
            assert s.info["scale_u"] == su
            u = s.u(gw.GW_FIELD_U)               # unscaled, FP64
            up = s.u(gw.GW_FIELD_UPREV)
            coef = s.u(gw.GW_FIELD_COEF)
    assert norm2 > 0
    px = -(-(xo + nx + 4) // 32) * 32
    # the stored values: u scaled by su (exact: a power of two), coef as is
    du, dup = padded(u * su, px, xo, ft), padded(up * su, px, xo, ft)
    dcf = padded(coef, px, xo, ct)
    assert torch.equal(du[4:4 + nz, 4:4 + ny, xo:xo + nx].double().cpu(),
                       torch.from_numpy(u * su))
    kin0 = np.sum((u - up) ** 2 / coef)
    pot0 = np.sum(u * oracle.laplacian(oracle.pad(up)))
    e_oracle = oracle.energy(coef, u, up)
    outs = [torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            for _ in range(3)]
    # a first call loads the library's kernels on this device
    gw.gw_check_fields_noalloc(du, dup, dcf, dtype, nx, ny, nz, px, su, outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in (1, 2):
        gw.gw_check_fields_noalloc(du, dup, dcf, dtype, nx, ny, nz, px, su, outs[call])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for call in (1, 2):
        n2, kin, pot = outs[call].cpu().numpy()
        assert n2 == norm2, call
        assert kin - pot == energy, call
        assert abs((kin - pot) - e_oracle) <= 1e-12 * (abs(kin0) + abs(pot0)), call
        assert n2 == pytest.approx(float(np.sum(u * u)), rel=1e-12), call


def test_noalloc_rejects_more_planes_than_its_scratch():
    import torch
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(gw.GWError) as e:
        gw.gw_check_fields_noalloc(buf, buf, buf, "f32", 4, 4, 4097, 32, 1.0,
                                   out)
    assert e.value.status == gw.GW_ERR_ARG
    assert "4096" in str(e.value)
