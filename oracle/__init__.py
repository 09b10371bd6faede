"""FP64 CPU oracle for the Minimod acoustic-isotropic time step.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` use it to check and to time against the
CUDA library; the library itself never imports, links or runs anything
here, and shares no code with it.

The arithmetic lives in ``minimod_oracle.c`` (plain C, FP64, one point at a
time); this module compiles it with gcc and binds it with ctypes, and adds
the NumPy definition of a halo exchange (what a subdomain's padded array
holds after the puts of the paper's Listing 1, section 4.5).

Parity status (see the CPU tests for each pin):

* coefficients, Laplacian, time stepping, energy, stability limit: pinned
  (polynomial exactness, brute-force Kronecker matrices, plane-wave
  dispersion, conservation, growth beyond the limit).
* Ricker wavelet: pinned by its defining properties (peak, zero crossings,
  zero mean).
* Cerjan sponge constants, wavelet delay, source form: readings of an
  unspecified paper; parity unpinned beyond the shape properties tested.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "minimod_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

R = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vectorisation flags, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_stencil_coefficients.argtypes = [dp]
            L.oracle_symbol.argtypes = [ctypes.c_double]
            L.oracle_symbol.restype = ctypes.c_double
            L.oracle_nu_max.restype = ctypes.c_double
            L.oracle_time_step.argtypes = [ctypes.c_double] * 3
            L.oracle_time_step.restype = ctypes.c_double
            L.oracle_ricker.argtypes = [ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, dp]
            L.oracle_cerjan_profile.argtypes = [ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, dp]
            L.oracle_laplacian.argtypes = [ctypes.c_int] * 3 + [dp, dp]
            L.oracle_energy.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp,
                                                             ctypes.c_int]
            L.oracle_energy.restype = ctypes.c_double
            L.oracle_run.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                ctypes.c_double, ctypes.c_double, ctypes.c_int,
                ctypes.c_int, ctypes.c_double, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                ctypes.c_int, ip, dp,
                ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int]
            L.oracle_run.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def coefficients() -> np.ndarray:
    c = np.zeros(5)
    lib().oracle_stencil_coefficients(_dp(c))
    return c


def symbol(theta: float) -> float:
    return lib().oracle_symbol(float(theta))


def nu_max() -> float:
    return lib().oracle_nu_max()


def time_step(h: float, vmax: float, courant: float = 0.0) -> float:
    return lib().oracle_time_step(float(h), float(vmax), float(courant))


def ricker(f: float, dt: float, n: int) -> np.ndarray:
    out = np.zeros(n)
    lib().oracle_ricker(float(f), float(dt), int(n), _dp(out))
    return out


def cerjan(n: int, width: int, a: float = 0.015) -> np.ndarray:
    g = np.zeros(n)
    lib().oracle_cerjan_profile(int(n), int(width), float(a), _dp(g))
    return g


def pad(u: np.ndarray, periodic: bool = False) -> np.ndarray:
    """Interior (nz, ny, nx) -> padded (nz+8, ny+8, nx+8), zero or wrapped."""
    mode = "wrap" if periodic else "constant"
    return np.pad(np.asarray(u, dtype=np.float64), R, mode=mode)


def laplacian(u_pad: np.ndarray) -> np.ndarray:
    u_pad = np.ascontiguousarray(u_pad, dtype=np.float64)
    nz, ny, nx = (s - 2 * R for s in u_pad.shape)
    out = np.zeros((nz, ny, nx))
    lib().oracle_laplacian(nx, ny, nz, _dp(u_pad), _dp(out))
    return out


def energy(coef, u_next, u_cur, periodic: bool = False) -> float:
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    u_next = np.ascontiguousarray(u_next, dtype=np.float64)
    u_cur = np.ascontiguousarray(u_cur, dtype=np.float64)
    nz, ny, nx = coef.shape
    return lib().oracle_energy(nx, ny, nz, _dp(coef), _dp(u_next),
                               _dp(u_cur), int(periodic))


def run(vel, h: float, nsteps: int, *, dt: float | None = None,
        courant: float = 0.0, sponge: int = 0, sponge_a: float = 0.015,
        periodic: bool = False, src=None, f_peak: float | None = None,
        wavelet=None, receivers=None, u0=None, um1=None,
        norms: bool = False, nthreads: int = 1) -> dict:
    """Run the FP64 recurrence; see ``oracle_run`` in the C source.

    ``dt`` defaults to the oracle's own Courant rule on ``max(vel)``; the
    source wavelet defaults to the oracle's Ricker of ``f_peak``.
    """
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    nz, ny, nx = vel.shape
    if dt is None:
        dt = time_step(h, float(vel.max()), courant)
    wl = None
    if src is not None:
        if wavelet is None:
            if f_peak is None:
                raise ValueError("source needs f_peak or wavelet")
            wavelet = ricker(f_peak, dt, nsteps)
        wl = np.ascontiguousarray(wavelet, dtype=np.float64)
        if wl.shape[0] < nsteps:
            raise ValueError("wavelet shorter than nsteps")
    rec = (np.zeros((0, 3), np.int32) if receivers is None
           else np.ascontiguousarray(receivers, dtype=np.int32))
    nrec = rec.shape[0]
    traces = np.zeros((nrec, max(nsteps, 1)))
    u = (np.zeros((nz, ny, nx)) if u0 is None
         else np.array(u0, dtype=np.float64, order="C", copy=True))
    up = (np.zeros((nz, ny, nx)) if um1 is None
          else np.array(um1, dtype=np.float64, order="C", copy=True))
    nrm = np.zeros(max(nsteps, 1)) if norms else None
    sx, sy, sz = (0, 0, 0) if src is None else (int(s) for s in src)
    rc = lib().oracle_run(
        nx, ny, nz, _dp(vel), float(h), float(dt), int(nsteps),
        int(sponge), float(sponge_a), int(periodic), sx, sy, sz,
        _dp(wl) if wl is not None else None,
        nrec, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        _dp(traces), int(u0 is not None), _dp(u), int(um1 is not None),
        _dp(up), _dp(nrm) if nrm is not None else None, int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_run failed ({rc})")
    return {"u": u, "u_prev": up, "traces": traces[:, :nsteps],
            "norms": None if nrm is None else nrm[:nsteps], "dt": dt,
            "wavelet": wl}


def split_points(n: int, parts: int, sizes=None) -> list[tuple[int, int]]:
    """Ranges [lo, hi) of an axis of n cells cut into ``parts`` pieces:
    the given ``sizes``, else as even as possible (larger pieces first)."""
    if sizes is not None:
        if sum(sizes) != n or len(sizes) != parts:
            raise ValueError("sizes must sum to n")
    else:
        q, r = divmod(n, parts)
        sizes = [q + (1 if i < r else 0) for i in range(parts)]
    out, lo = [], 0
    for s in sizes:
        out.append((lo, lo + s))
        lo += s
    return out


def halo_exchanged(u: np.ndarray, xr, yr, zr, periodic: bool = False):
    """Definition of a subdomain's field after the halo exchange.

    ``u`` is the global interior field; (xr, yr, zr) the subdomain's
    [lo, hi) ranges.  Listing 1 (section 4.5) has every rank put its
    boundary slabs into its neighbours' halos, then fence; afterwards each
    face halo cell of a subdomain holds the global field at that position
    (zero outside a non-periodic domain, wrapped in a periodic one).  Only
    face halos are defined: the star stencil never reads edge or corner
    halo cells, so those are returned as NaN.
    """
    P = pad(u, periodic)
    sub = P[zr[0]:zr[1] + 2 * R, yr[0]:yr[1] + 2 * R,
            xr[0]:xr[1] + 2 * R].copy()
    nz, ny, nx = (s - 2 * R for s in sub.shape)
    kk, jj, ii = np.meshgrid(np.arange(nz + 2 * R), np.arange(ny + 2 * R),
                             np.arange(nx + 2 * R), indexing="ij")
    outside = ((ii < R) | (ii >= nx + R)).astype(int) \
        + ((jj < R) | (jj >= ny + R)).astype(int) \
        + ((kk < R) | (kk >= nz + R)).astype(int)
    sub[outside >= 2] = np.nan
    return sub
