"""Helpers shared by the GPU tests: a CUDA shot run through the C ABI and
the matching FP64 oracle run on the same seeded inputs."""

from __future__ import annotations

import numpy as np

import oracle
from paper_2506_02486_gb300 import buildlib
from paper_2506_02486_gb300 import gbwave as gw
from paper_2506_02486_gb300.runtime import Segment, Shot, padded_bytes

_built = False


def ensure_built():
    global _built
    if not _built:
        buildlib.build()
        _built = True


def seg_for(nx, ny, nz, dtype="f32", px=1, py=1, pz=1, extra=512 << 20):
    """A segment with room for one shot of this size and decomposition."""
    ensure_built()
    nsub = px * py * pz
    sx, sy, sz = -(-nx // px), -(-ny // py), -(-nz // pz)
    per = 4 * padded_bytes(sx, sy, sz, dtype) + extra
    return Segment(nsub * per, nranks=nsub)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b) -> float:
    """Largest point-by-point difference relative to the largest value of
    the reference: max |a - b| / max |b|.  Unlike the relative L2 norm it
    does not average a wrong row or a wrong halo cell away over the grid."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def assert_close(g, o, tol, what="u"):
    """Relative L2 <= tol and max |g - o| <= tol * max |o|."""
    e2, ei = rel_l2(g, o), max_rel(g, o)
    assert e2 <= tol, f"{what}: relative L2 {e2:.3e} > {tol:.1e}"
    assert ei <= tol, f"{what}: max |g - o| / max |o| = {ei:.3e} > {tol:.1e}"
    return e2, ei


# 2^-24: unit roundoff of FP32
U32 = 2.0 ** -24


def gamma(n: int, u: float = U32) -> float:
    """gamma_n = n u / (1 - n u): the relative error bound of a sum of n + 1
    positive terms in a precision of unit roundoff u (Higham, eq. 3.8)."""
    return n * u / (1.0 - n * u)


def gpu_run(vel, nsteps, *, h=10.0, src=None, f_peak=None, wavelet=None,
            receivers=None, sponge=0, dtype="f32", px=1, py=1, pz=1,
            split=(None, None, None), symmetric=True, seg=None, u0=None,
            um1=None, periodic=0, courant=0.0, dt=0.0, steps_per_call=None,
            **desc):
    """Run one shot on the GPU; returns u (FP64 copy), traces, norms, info."""
    nz, ny, nx = vel.shape
    own = seg is None
    if own:
        seg = seg_for(nx, ny, nz, dtype, px, py, pz)
    try:
        with Shot(seg, nx, ny, nz, px=px, py=py, pz=pz, split=split,
                  symmetric=symmetric, h=h, nsteps=max(nsteps, 1),
                  dtype=dtype, sponge=sponge, periodic=periodic,
                  courant=courant, dt=dt, **desc) as s:
            s.set_model(vel)
            info = s.info
            wl = None
            if src is not None:
                if wavelet is None:
                    wl = s.add_ricker(src, f_peak)
                else:
                    wl = np.asarray(wavelet, dtype=np.float32)
                    s.add_source(src, wl)
            if receivers is not None:
                s.set_receivers(receivers)
            if u0 is not None:
                s.write(gw.GW_FIELD_U, u0)
            if um1 is not None:
                s.write(gw.GW_FIELD_UPREV, um1)
            if steps_per_call:
                left = nsteps
                while left > 0:
                    k = min(left, steps_per_call)
                    s.step(k)
                    left -= k
            else:
                s.step(nsteps)
            s.sync()
            out = {
                "u": s.u(f64=True),
                "u32": s.u(f64=False),
                "traces": s.traces(nsteps) if receivers is not None else None,
                "norms": s.norms(min(nsteps, s.desc.nsteps)),
                "info": s.info,
                "dt": info["dt"],
                "wavelet": wl,
            }
            return out
    finally:
        if own:
            seg.close()
