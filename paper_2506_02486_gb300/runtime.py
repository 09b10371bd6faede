"""PyTorch-owned global segment and a one-shot helper over the C ABI.

PyTorch only provides the device memory (one ``uint8`` tensor that becomes
the PGAS global segment, paper section 3.2) and streams; every step of the
computation runs in the library's kernels.
"""

from __future__ import annotations

import numpy as np

from . import gbwave as gw


class Segment:
    """A device buffer attached as the global segment of a new context."""

    def __init__(self, nbytes: int, nranks: int = 1, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the gbwave library needs a CUDA device")
        self.device = device
        self.nbytes = int(nbytes)
        self.nranks = int(nranks)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8,
                               device=f"cuda:{device}")
        self.ctx = gw.gw_ctx_create(device)
        gw.gw_segment_attach(self.ctx, self.buf, self.nbytes, self.nranks)

    def close(self):
        if self.ctx:
            gw.gw_ctx_destroy(self.ctx)
            self.ctx = 0
        self.buf = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def padded_bytes(nx: int, ny: int, nz: int, dtype: str = "f32") -> int:
    """Bytes of one padded field array (x pitch a multiple of 32 bytes)."""
    es = {"f32": 4, "f64": 8, "f16s": 2, "bf16": 2}[dtype]
    xo = {2: 16, 4: 8, 8: 4}[es]
    mul = 32 // es
    px = -(-(xo + nx + 4) // mul) * mul
    return px * (ny + 8) * (nz + 8) * es


def shot_bytes(nx: int, ny: int, nz: int, dtype: str = "f32",
               nsteps: int = 1, nrec: int = 0, px=1, py=1, pz=1) -> int:
    """A generous segment size for one shot (fields + metadata + staging)."""
    nsub = px * py * pz
    sx, sy, sz = -(-nx // px), -(-ny // py), -(-nz // pz)
    f = padded_bytes(sx, sy, sz, dtype)
    nfields = 4 if dtype in ("f16s", "bf16") else 3
    meta = 64 << 20
    stage = min(256 << 20, nx * ny * nz * 8) + (1 << 20)
    items = (nx // 16 + 1) * (ny // 8 + 1) * 64 * 8 * 32
    return nsub * (nfields * f + (4 << 20)) + meta + stage + items \
        + nrec * nsteps * 4


class Shot:
    """One shot domain with its model, source and receivers."""

    def __init__(self, seg: Segment, nx, ny, nz, *, px=1, py=1, pz=1,
                 split=(None, None, None), symmetric=True, **desc):
        self.seg = seg
        self.shape = (nz, ny, nx)
        self.desc = gw.shot_desc(nx, ny, nz, **desc)
        self.dom = gw.gw_domain_create(seg.ctx, self.desc, px, py, pz,
                                       split[0], split[1], split[2],
                                       symmetric)
        self.nrec = 0

    @property
    def info(self) -> dict:
        return gw.gw_domain_info_get(self.dom)

    def set_model(self, vel: np.ndarray):
        gw.gw_set_model(self.dom, vel)

    def add_ricker(self, pos, f_peak: float):
        """The library's FP64 Ricker source (sampled at the domain's dt)."""
        gw.gw_inject_ricker(self.dom, *pos, f_peak)

    def add_source(self, pos, wavelet):
        gw.gw_inject_source(self.dom, *pos, wavelet)

    def set_receivers(self, xyz):
        xyz = np.asarray(xyz, dtype=np.int32).reshape(-1, 3)
        gw.gw_set_receivers(self.dom, xyz)
        self.nrec = xyz.shape[0]

    def step(self, n: int, stream=None):
        gw.gw_step(self.dom, n, stream)

    def sync(self):
        gw.gw_barrier(self.dom, None, True)

    def u(self, which=gw.GW_FIELD_U, f64=True) -> np.ndarray:
        return gw.gw_read_wavefield(self.dom, which, self.shape, f64)

    def write(self, which, arr):
        gw.gw_write_wavefield(self.dom, which, arr)

    def traces(self, nsteps: int) -> np.ndarray:
        return gw.gw_read_receivers(self.dom, self.nrec, nsteps)

    def norms(self, n: int) -> np.ndarray:
        return gw.gw_norms(self.dom, n)

    def check(self) -> tuple[float, float]:
        return gw.gw_check(self.dom)

    def close(self):
        if self.dom:
            gw.gw_domain_destroy(self.dom)
            self.dom = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Several shots of one segment advanced by shared launches."""

    def __init__(self, seg: Segment, shots, chunk: int = 0,
                 persistent: bool = False):
        self.seg = seg
        self.shots = list(shots)
        self.h = gw.gw_batch_create(seg.ctx, [s.dom for s in self.shots],
                                    chunk, persistent)

    @property
    def info(self) -> dict:
        return gw.gw_batch_info(self.h)

    def step(self, n: int, stream=None):
        gw.gw_batch_step(self.h, n, stream)

    def timing(self, enable: bool):
        gw.gw_batch_timing(self.h, enable)

    def stats(self) -> dict:
        return gw.gw_batch_stats_get(self.h)

    def close(self):
        if self.h:
            gw.gw_batch_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching shot server on a segment (one loop thread in the
    library).  Keeps each request's host buffers alive until it is
    waited for."""

    def __init__(self, seg: Segment, budget: int, max_slots: int = 64,
                 chunk: int = 0):
        self.seg = seg
        self.h = gw.gw_server_create(seg.ctx, budget, max_slots, chunk)
        self._keep = {}

    def submit(self, nx, ny, nz, nsteps, *, src, f_peak=20.0, vel=None,
               vz=None, receivers=None, dtype="f32", sponge=20, h=10.0,
               tile=0) -> int:
        req = gw.gw_request()
        req.desc = gw.shot_desc(nx, ny, nz, h=h, nsteps=nsteps, dtype=dtype,
                                sponge=sponge, tile=tile)
        keep = []
        if vel is not None:
            v = np.ascontiguousarray(vel, dtype=np.float32)
            assert v.size == nx * ny * nz
            req.vel = v.ctypes.data
            keep.append(v)
        else:
            v = np.ascontiguousarray(vz, dtype=np.float64)
            assert v.size == nz
            req.vz = v.ctypes.data
            keep.append(v)
        req.src[:] = [int(c) for c in src]
        req.f_peak = float(f_peak)
        traces = None
        if receivers is not None and len(receivers):
            r = np.ascontiguousarray(np.asarray(receivers, dtype=np.int32)
                                     .reshape(-1, 3))
            req.nrec = r.shape[0]
            req.rec = r.ctypes.data
            traces = np.zeros((r.shape[0], nsteps), dtype=np.float32)
            req.traces = traces.ctypes.data
            keep.append(r)
        t = gw.gw_submit(self.h, req)
        self._keep[t] = (keep, traces)
        return t

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        res = gw.gw_wait(self.h, ticket, timeout_ms)
        _, traces = self._keep.pop(ticket)
        res["traces"] = traces
        return res

    def stats(self) -> dict:
        return gw.gw_server_stats_get(self.h)

    def now(self) -> float:
        return gw.gw_server_now(self.h)

    def close(self):
        if self.h:
            gw.gw_server_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
