"""Subdomain decomposition inside one HBM (the halo exchange of Listing 1,
section 4.5, with the symmetric and asymmetric allocation of section 3.2)
must reproduce the undecomposed run bit for bit, and the halo a put leaves
in a subdomain must equal the definition of the exchanged field."""

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import assert_close, gamma, gpu_run, seg_for
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Shot

pytestmark = pytest.mark.gpu

NX, NY, NZ = 96, 80, 72


@pytest.fixture(scope="module")
def reference():
    vel = workloads.layered(NX, NY, NZ, seed=21)
    src = workloads.source_position(22, NX, NY, NZ, margin=10)
    rec = workloads.lattice_receivers(NX, NY, 10, n=8, margin=10)
    base = gpu_run(vel, 60, src=src, f_peak=40.0, receivers=rec, sponge=10)
    return vel, src, rec, base


def test_undecomposed_reference_matches_oracle(reference):
    """The run every decomposition below must reproduce bit for bit, against
    the FP64 oracle (relative L2 and point by point)."""
    vel, src, rec, base = reference
    dt = oracle.time_step(10.0, float(vel.max()))
    o = oracle.run(vel, 10.0, 60, dt=dt, src=src, f_peak=40.0, sponge=10,
                   receivers=rec, nthreads=8)
    assert_close(base["u"], o["u"], 1e-4)
    assert_close(base["traces"], o["traces"], 1e-4, "traces")


def test_persistent_chunks_are_bitwise(reference):
    """K steps in one launch (device-wide barrier between steps) give the
    bits of one launch per step, undecomposed and 2 x 2 x 2, with the static
    and the dynamic work-item schedule (the dynamic one hands out a step's
    tickets and resets its counter between the steps of one launch)."""
    vel, src, rec, base = reference
    for dec, sched in (((1, 1, 1), 0), ((1, 1, 1), 2), ((2, 2, 2), 0), ((2, 2, 2), 1)):
        g = gpu_run(vel, 60, src=src, f_peak=40.0, receivers=rec, sponge=10,
                    px=dec[0], py=dec[1], pz=dec[2], persistent=1, chunk=7,
                    schedule=sched)
        assert np.array_equal(g["u32"], base["u32"]), (dec, sched)
        assert np.array_equal(g["traces"], base["traces"]), (dec, sched)


@pytest.mark.parametrize("px,py,pz,symmetric,mode,split", [
    (2, 2, 2, True, gw.GW_HALO_FUSED, (None, None, None)),
    (2, 2, 2, True, gw.GW_HALO_SEPARATE, (None, None, None)),
    (2, 2, 2, "static", gw.GW_HALO_FUSED, (None, None, None)),
    (4, 1, 1, True, gw.GW_HALO_FUSED, (None, None, None)),   # x slabs
    (1, 1, 6, False, gw.GW_HALO_FUSED, (None, None, None)),
    (3, 2, 1, False, gw.GW_HALO_FUSED, ([20, 41, 35], [30, 50], None)),
    (3, 2, 1, True, gw.GW_HALO_SEPARATE, ([20, 41, 35], [30, 50], None)),
    (2, 3, 2, False, gw.GW_HALO_SEPARATE, ([47, 49], [9, 60, 11], [36, 36])),
])
def test_decomposed_equals_undecomposed(reference, px, py, pz, symmetric,
                                        mode, split):
    """Decomposed shots take the dynamic work-item schedule unless asked
    (the "static" case: symmetric, static round robin)."""
    vel, src, rec, base = reference
    sched = gw.GW_SCHED_STATIC if symmetric == "static" else gw.GW_SCHED_AUTO
    g = gpu_run(vel, 60, src=src, f_peak=40.0, receivers=rec, sponge=10,
                px=px, py=py, pz=pz, symmetric=bool(symmetric), halo_mode=mode,
                split=split, schedule=sched)
    assert g["info"]["nsub"] == px * py * pz
    assert g["info"]["schedule"] == (gw.GW_SCHED_STATIC if sched else gw.GW_SCHED_DYNAMIC)
    assert np.array_equal(g["u32"], base["u32"])
    assert np.array_equal(g["traces"], base["traces"])
    # norms: per-thread, per-plane FP32 partials of at most 8 positive
    # terms, accumulated over an item's planes (fewer than 128 here) with
    # compensation and over items in FP64, grouped by tile: each run within
    # gamma_7 + gamma_127^2 of the exact sum, so the two within twice that
    assert g["norms"] == pytest.approx(base["norms"],
                                       rel=2 * (gamma(7) + gamma(127) ** 2))


@pytest.mark.parametrize("symmetric", [True, False])
def test_put_halo_fills_face_halos_by_definition(symmetric):
    nx, ny, nz = 30, 22, 18
    rng = np.random.default_rng(8)
    u = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    sx, sy, sz = [13, 17], [22], [5, 6, 7]
    with seg_for(nx, ny, nz, px=2, pz=3, extra=64 << 20) as seg:
        with Shot(seg, nx, ny, nz, px=2, py=1, pz=3, split=(sx, sy, sz),
                  symmetric=symmetric, nsteps=1) as s:
            s.set_model(np.full((nz, ny, nx), 2000.0))
            s.write(gw.GW_FIELD_U, u)          # scatters, then puts halos
            gw.gw_put_halo(s.dom)
            gw.gw_barrier(s.dom, None, True)
            import torch
            torch.cuda.synchronize()
            host = seg.buf.cpu().numpy()
            base = seg.buf.data_ptr()
            xr = oracle.split_points(nx, 2, sx)
            zr = oracle.split_points(nz, 3, sz)
            for k in range(3):
                for i in range(2):
                    r = k * 2 + i
                    snx, sny, snz = sx[i], ny, sz[k]
                    # the subdomain's u_0 buffer: first field allocation
                    want = oracle.halo_exchanged(u.astype(np.float64), xr[i],
                                                 (0, ny), zr[k])
                    got = read_padded(host, base, s, r, snx, sny, snz,
                                      symmetric, sx, sz)
                    m = ~np.isnan(want)
                    assert np.array_equal(got[m], want[m].astype(np.float32))


def read_padded(host, base, shot, rank, snx, sny, snz, symmetric, sx, sz):
    """Locate subdomain `rank`'s u_0 array inside the segment and return
    its (snz+8, sny+8, snx+8) window."""
    seginfo = gw.gw_segment_info(shot.seg.ctx)
    rank_bytes = seginfo[0]
    # fields were allocated first: u0 is the first allocation of the domain
    # (symmetric: offset 0 on every rank; asymmetric: top of each rank)
    lx = max(sx) if symmetric else snx
    ly = sny
    px = -(-(8 + lx + 4) // 8) * 8        # FP32: interior at x offset 8,
                                          # rows a multiple of 32 bytes
    py = ly + 8
    pzp = (max(sz) if symmetric else snz) + 8
    nbytes = px * py * pzp * 4
    if symmetric:
        off = rank * rank_bytes
    else:
        off = rank * rank_bytes + rank_bytes - (-(-nbytes // 256) * 256)
    arr = host[off:off + nbytes].view(np.float32).reshape(pzp, py, px)
    return arr[:snz + 8, :sny + 8, 4:snx + 12].astype(np.float64)
