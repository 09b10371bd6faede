"""gw_check_fields_noalloc -- the allocation-free variant of gw_check, for
callers that cannot allocate device memory (for example code running while
another framework holds its memory pool).  Its per-plane partial sums live
in a built-in device array instead of memory the call would allocate.

The test runs a small shot, reads its fields back, lays them out again in
device arrays the test owns, and checks that two calls in a row of the
allocation-free entry point give the norm and energy that gw_check gives
for the same state (FP64 sums in a different order: equal to 1e-10)."""

import numpy as np
import pytest

import workloads
from gpu_util import seg_for
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Shot

pytestmark = pytest.mark.gpu


def padded(a, px):
    """Interior (nz, ny, nx) FP32 values in the library's padded layout."""
    import torch
    nz, ny, nx = a.shape
    out = torch.zeros((nz + 8, ny + 8, px), dtype=torch.float32, device="cuda")
    out[4:4 + nz, 4:4 + ny, 8:8 + nx] = torch.from_numpy(
        np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return out


def test_noalloc_check_matches_gw_check_twice():
    import torch
    nx, ny, nz = 45, 38, 31
    vel = workloads.layered(nx, ny, nz, seed=17)
    with seg_for(nx, ny, nz, extra=64 << 20) as seg:
        with Shot(seg, nx, ny, nz, nsteps=40) as s:
            s.set_model(vel)
            s.add_ricker((20, 19, 15), 40.0)
            s.step(30)
            norm2, energy = s.check()
            u = s.u(gw.GW_FIELD_U, f64=False)
            up = s.u(gw.GW_FIELD_UPREV, f64=False)
            coef = s.u(gw.GW_FIELD_COEF, f64=False)
    assert norm2 > 0
    px = -(-(8 + nx + 4) // 32) * 32
    du, dup, dcf = padded(u, px), padded(up, px), padded(coef, px)
    # halo cells are zero, as in the shot (zero boundary); the reduction
    # divides by coef at interior cells only
    for call in range(2):
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        gw.gw_check_fields_noalloc(du, dup, dcf, "f32", nx, ny, nz, px, 1.0, out)
        torch.cuda.synchronize()
        n2, kin, pot = out.cpu().numpy()
        assert n2 == pytest.approx(norm2, rel=1e-10), call
        assert abs((kin - pot) - energy) <= 1e-10 * (abs(kin) + abs(pot)), call


def test_noalloc_rejects_more_planes_than_its_scratch():
    import torch
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(gw.GWError) as e:
        gw.gw_check_fields_noalloc(buf, buf, buf, "f32", 4, 4, 4097, 32, 1.0,
                                   out)
    assert e.value.status == gw.GW_ERR_ARG
    assert "4096" in str(e.value)
