"""ctypes binding of the gbwave C ABI (``include/gbwave.h``).

Every ``gw_*`` function here has the name of the C entry point it calls and
only marshals arguments: NumPy arrays become host pointers, PyTorch tensors
device pointers, streams their ``cudaStream_t`` handles.  A non-zero status
raises :class:`GWError` carrying the library's message.  All arithmetic of
the time step runs in the library's CUDA kernels; if the library is not
built, loading fails loudly instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbwave.so")

GW_OK = 0
GW_ERR_ARG = -1
GW_ERR_BUDGET = -2
GW_ERR_ALIGN = -3
GW_ERR_CUDA = -4
GW_ERR_TIMEOUT = -5
GW_ERR_STATE = -6
GW_ERR_NUMERIC = -7
GW_ERR_NOMEM = -8

GW_F32, GW_F64, GW_F16S, GW_BF16 = 0, 1, 2, 3
GW_HALO_FUSED, GW_HALO_SEPARATE = 0, 1
GW_SCHED_AUTO, GW_SCHED_STATIC, GW_SCHED_DYNAMIC = 0, 1, 2
GW_FIELD_U, GW_FIELD_UPREV, GW_FIELD_W, GW_FIELD_COEF = 0, 1, 2, 3

DTYPES = {"f32": GW_F32, "f64": GW_F64, "f16s": GW_F16S, "bf16": GW_BF16}


class GWError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {msg} (status {status})")
        self.status = status


class gw_shot_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double), ("courant", ctypes.c_double),
        ("dt", ctypes.c_double), ("nsteps", ctypes.c_int),
        ("dtype", ctypes.c_int), ("sponge", ctypes.c_int),
        ("sponge_a", ctypes.c_double), ("periodic", ctypes.c_int),
        ("halo_mode", ctypes.c_int), ("chunk", ctypes.c_int),
        ("tile", ctypes.c_int), ("zchunk", ctypes.c_int),
        ("scale_u", ctypes.c_double), ("scale_w", ctypes.c_double),
        ("persistent", ctypes.c_int), ("schedule", ctypes.c_int),
    ]


class gw_domain_info(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("courant", ctypes.c_double),
        ("vmax", ctypes.c_double), ("nsub", ctypes.c_int),
        ("step", ctypes.c_int), ("tile", ctypes.c_int),
        ("ctas", ctypes.c_int), ("items", ctypes.c_int),
        ("scale_u", ctypes.c_double), ("scale_w", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t), ("schedule", ctypes.c_int),
    ]


class gw_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("halo_ms", ctypes.c_double)]


class gw_request(ctypes.Structure):
    _fields_ = [
        ("desc", gw_shot_desc), ("vel", ctypes.c_void_p),
        ("vz", ctypes.c_void_p), ("src", ctypes.c_int * 3),
        ("f_peak", ctypes.c_double), ("nrec", ctypes.c_int),
        ("rec", ctypes.c_void_p), ("traces", ctypes.c_void_p),
    ]


class gw_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("steps", ctypes.c_int),
        ("points", ctypes.c_longlong), ("submit_s", ctypes.c_double),
        ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
        ("norm2", ctypes.c_double), ("energy", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t), ("tile", ctypes.c_int),
    ]


class gw_server_stats(ctypes.Structure):
    _fields_ = [
        ("pending", ctypes.c_int), ("active", ctypes.c_int),
        ("completed", ctypes.c_int), ("max_active", ctypes.c_int),
        ("chunks", ctypes.c_int), ("rebuilds", ctypes.c_int),
        ("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
        ("peak_bytes", ctypes.c_size_t), ("point_updates", ctypes.c_longlong),
        ("busy_s", ctypes.c_double), ("now_s", ctypes.c_double),
    ]


class gw_pool_stats(ctypes.Structure):
    _fields_ = [
        ("created", ctypes.c_int), ("active", ctypes.c_int),
        ("idle", ctypes.c_int), ("max_active", ctypes.c_int),
        ("peak_active", ctypes.c_int), ("pad_", ctypes.c_int),
        ("ops", ctypes.c_longlong), ("reuses", ctypes.c_longlong),
        ("partial_syncs", ctypes.c_longlong), ("released", ctypes.c_longlong),
        ("waited_oldest", ctypes.c_longlong), ("fences", ctypes.c_longlong),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_D = ctypes.c_double
_U64 = ctypes.c_uint64

# name -> argtypes (all return gw_status unless listed in _RESTYPES)
_SIGS = {
    "gw_last_error": [],
    "gw_status_string": [_I],
    "gw_version": [],
    "gw_ctx_create": [ctypes.POINTER(_P), _I],
    "gw_ctx_destroy": [_P],
    "gw_segment_attach": [_P, _P, _SZ, _I, _I],
    "gw_segment_info": [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ),
                        ctypes.POINTER(_SZ)],
    "gw_alloc_symmetric": [_P, _SZ, ctypes.POINTER(_U64)],
    "gw_alloc_asymmetric": [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_U64)],
    "gw_free": [_P, _U64],
    "gw_resolve": [_P, _U64, _I, ctypes.POINTER(_P), ctypes.POINTER(_SZ)],
    "gw_ptr_cache_stats": [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64)],
    "gw_put": [_P, _U64, _I, _SZ, _P, _SZ, _P],
    "gw_get": [_P, _P, _U64, _I, _SZ, _SZ, _P],
    "gw_fence": [_P, _P],
    "gw_put_nbi": [_P, _U64, _I, _SZ, _P, _SZ, _P],
    "gw_get_nbi": [_P, _P, _U64, _I, _SZ, _SZ, _P],
    "gw_quiet": [_P],
    "gw_set_max_active_streams": [_P, _I],
    "gw_pool_stats_get": [_P, ctypes.POINTER(gw_pool_stats)],
    "gw_stream_pool_simulate": [_I, _I, _P, _P, ctypes.POINTER(gw_pool_stats)],
    "gw_cannon_bytes": [_I, _I, ctypes.POINTER(_SZ)],
    "gw_cannon_create": [_P, _I, _I, ctypes.POINTER(_P)],
    "gw_cannon_destroy": [_P],
    "gw_cannon_set": [_P, _P, _P, _I],
    "gw_cannon_run": [_P, _P],
    "gw_cannon_sync": [_P],
    "gw_cannon_schedule": [_P, _I, _I],
    "gw_cannon_read_c": [_P, _P, _I],
    "gw_cannon_timing": [_P, _I],
    "gw_cannon_selftest_timeout": [_P, ctypes.c_uint, ctypes.POINTER(_I)],
    "gw_cannon_stats": [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                        ctypes.POINTER(_I)],
    "gw_domain_create": [_P, ctypes.POINTER(gw_shot_desc), _I, _I, _I, _P,
                         _P, _P, _I, ctypes.POINTER(_P)],
    "gw_domain_destroy": [_P],
    "gw_domain_bytes": [ctypes.POINTER(gw_shot_desc), _I, _I, _I, _I,
                        ctypes.POINTER(_SZ)],
    "gw_domain_info_get": [_P, ctypes.POINTER(gw_domain_info)],
    "gw_set_model": [_P, _P],
    "gw_set_model_f32": [_P, _P],
    "gw_set_model_layered": [_P, _P],
    "gw_ricker": [_D, _D, _I, _P],
    "gw_round_to_f32": [_P, _P, _SZ, _P],
    "gw_inject_source": [_P, _I, _I, _I, _P, _I],
    "gw_inject_ricker": [_P, _I, _I, _I, _D],
    "gw_set_receivers": [_P, _I, _P],
    "gw_step": [_P, _I, _P],
    "gw_put_halo": [_P, _P],
    "gw_barrier": [_P, _P, _I],
    "gw_read_receivers": [_P, _P, _I, _I],
    "gw_read_wavefield": [_P, _I, _P, _I],
    "gw_write_wavefield": [_P, _I, _P, _I],
    "gw_norms": [_P, _P, _I],
    "gw_check": [_P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "gw_check_fields_noalloc": [_P, _P, _P, _I, _I, _I, _I, _I, _D, _P, _P],
    "gw_kernel_timing": [_P, _I],
    "gw_kernel_stats_get": [_P, ctypes.POINTER(gw_kernel_stats)],
    "gw_batch_create": [_P, _I, _P, _I, _I, ctypes.POINTER(_P)],
    "gw_batch_destroy": [_P],
    "gw_batch_step": [_P, _I, _P],
    "gw_batch_info": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I),
                      ctypes.POINTER(_I)],
    "gw_batch_timing": [_P, _I],
    "gw_batch_stats_get": [_P, ctypes.POINTER(gw_kernel_stats)],
    "gw_autotune": [_P, ctypes.POINTER(gw_shot_desc), _I, _I, _I, _I,
                    ctypes.POINTER(_I), ctypes.POINTER(_D), _P, _I],
    "gw_tile_count": [_I, ctypes.POINTER(_I)],
    "gw_pick_tile": [_I, _I, _I, ctypes.POINTER(_I)],
    "gw_plan_tiles": [_P, _I, _P, _I, _D, _P],
    "gw_server_create": [_P, _SZ, _I, _I, ctypes.POINTER(_P)],
    "gw_server_destroy": [_P],
    "gw_submit": [_P, ctypes.POINTER(gw_request), ctypes.POINTER(_U64)],
    "gw_wait": [_P, _U64, _I, ctypes.POINTER(gw_result)],
    "gw_server_stats_get": [_P, ctypes.POINTER(gw_server_stats)],
    "gw_server_now": [_P],
    "gw_selftest_timeout": [_P, ctypes.c_uint, ctypes.POINTER(_I)],
    "gw_state_bytes": [_P, ctypes.POINTER(_SZ)],
    "gw_save_state": [_P, _P],
    "gw_load_state": [_P, _P],
}
_RESTYPES = {"gw_last_error": ctypes.c_char_p,
             "gw_status_string": ctypes.c_char_p,
             "gw_version": ctypes.c_char_p,
             "gw_server_now": ctypes.c_double}

_lib = None
_lock = threading.Lock()


def symbols() -> list[str]:
    """Entry points the binding expects the library to export."""
    return list(_SIGS)


def lib():
    """Load libgbwave.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"gbwave CUDA library missing at {LIB_PATH}; build it "
                    "with paper_2506_02486_gb300.buildlib.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, ctypes.c_int)
            _lib = L
    return _lib


def _check(status: int, func: str):
    if status != GW_OK:
        msg = lib().gw_last_error().decode(errors="replace")
        raise GWError(status, func, msg)


def _ptr(a) -> int | None:
    """Address of a NumPy array, a torch tensor, or an integer."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if hasattr(a, "is_contiguous") and not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"cannot take the address of {type(a)!r}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream   # torch.cuda.Stream


# ---------------------------------------------------------------- errors

def gw_last_error() -> str:
    return lib().gw_last_error().decode(errors="replace")


def gw_status_string(s: int) -> str:
    return lib().gw_status_string(int(s)).decode()


def gw_version() -> str:
    return lib().gw_version().decode()


# ---------------------------------------------------------------- context

def gw_ctx_create(device: int = 0) -> int:
    h = _P()
    _check(lib().gw_ctx_create(ctypes.byref(h), int(device)), "gw_ctx_create")
    return h.value


def gw_ctx_destroy(ctx: int):
    _check(lib().gw_ctx_destroy(ctx), "gw_ctx_destroy")


def gw_segment_attach(ctx: int, base, nbytes: int, nranks: int,
                      zero: bool = True):
    _check(lib().gw_segment_attach(ctx, _ptr(base), int(nbytes), int(nranks),
                                   int(bool(zero))), "gw_segment_attach")


def gw_segment_info(ctx: int) -> tuple[int, int, int]:
    a, b, c = _SZ(), _SZ(), _SZ()
    _check(lib().gw_segment_info(ctx, ctypes.byref(a), ctypes.byref(b),
                                 ctypes.byref(c)), "gw_segment_info")
    return a.value, b.value, c.value


def gw_alloc_symmetric(ctx: int, nbytes: int) -> int:
    g = _U64()
    _check(lib().gw_alloc_symmetric(ctx, int(nbytes), ctypes.byref(g)),
           "gw_alloc_symmetric")
    return g.value


def gw_alloc_asymmetric(ctx: int, nbytes_per_rank) -> int:
    arr = (_SZ * len(nbytes_per_rank))(*[int(b) for b in nbytes_per_rank])
    g = _U64()
    _check(lib().gw_alloc_asymmetric(ctx, arr, ctypes.byref(g)),
           "gw_alloc_asymmetric")
    return g.value


def gw_free(ctx: int, g: int):
    _check(lib().gw_free(ctx, int(g)), "gw_free")


def gw_resolve(ctx: int, g: int, rank: int) -> tuple[int, int]:
    p, n = _P(), _SZ()
    _check(lib().gw_resolve(ctx, int(g), int(rank), ctypes.byref(p),
                            ctypes.byref(n)), "gw_resolve")
    return p.value or 0, n.value


def gw_ptr_cache_stats(ctx: int) -> tuple[int, int]:
    h, m = _U64(), _U64()
    _check(lib().gw_ptr_cache_stats(ctx, ctypes.byref(h), ctypes.byref(m)),
           "gw_ptr_cache_stats")
    return h.value, m.value


def gw_put(ctx: int, dst: int, dst_rank: int, dst_off: int, src,
           nbytes: int, stream=None):
    _check(lib().gw_put(ctx, int(dst), int(dst_rank), int(dst_off),
                        _ptr(src), int(nbytes), _stream(stream)), "gw_put")


def gw_get(ctx: int, dst, src: int, src_rank: int, src_off: int,
           nbytes: int, stream=None):
    _check(lib().gw_get(ctx, _ptr(dst), int(src), int(src_rank),
                        int(src_off), int(nbytes), _stream(stream)), "gw_get")


def gw_fence(ctx: int, stream=None):
    _check(lib().gw_fence(ctx, _stream(stream)), "gw_fence")


def gw_put_nbi(ctx: int, dst: int, dst_rank: int, dst_off: int, src,
               nbytes: int, after=None):
    _check(lib().gw_put_nbi(ctx, int(dst), int(dst_rank), int(dst_off),
                            _ptr(src), int(nbytes), _stream(after)),
           "gw_put_nbi")


def gw_get_nbi(ctx: int, dst, src: int, src_rank: int, src_off: int,
               nbytes: int, after=None):
    _check(lib().gw_get_nbi(ctx, _ptr(dst), int(src), int(src_rank),
                            int(src_off), int(nbytes), _stream(after)),
           "gw_get_nbi")


def gw_quiet(ctx: int):
    _check(lib().gw_quiet(ctx), "gw_quiet")


def gw_set_max_active_streams(ctx: int, n: int):
    _check(lib().gw_set_max_active_streams(ctx, int(n)),
           "gw_set_max_active_streams")


def _pool_dict(s: gw_pool_stats) -> dict:
    return {k: getattr(s, k) for k, _ in gw_pool_stats._fields_
            if k != "pad_"}


def gw_pool_stats_get(ctx: int) -> dict:
    s = gw_pool_stats()
    _check(lib().gw_pool_stats_get(ctx, ctypes.byref(s)), "gw_pool_stats_get")
    return _pool_dict(s)


def gw_stream_pool_simulate(max_active: int, durations):
    """The pool policy on the host model; returns (stream of each op,
    counters)."""
    d = np.ascontiguousarray(durations, dtype=np.int32)
    so = np.full(d.shape[0], -1, dtype=np.int32)
    s = gw_pool_stats()
    _check(lib().gw_stream_pool_simulate(int(max_active), int(d.shape[0]),
                                         _ptr(d), _ptr(so), ctypes.byref(s)),
           "gw_stream_pool_simulate")
    return so, _pool_dict(s)


# ---------------------------------------------------------------- Cannon

def gw_cannon_bytes(n: int, p: int) -> int:
    v = _SZ()
    _check(lib().gw_cannon_bytes(int(n), int(p), ctypes.byref(v)),
           "gw_cannon_bytes")
    return v.value


def gw_cannon_create(ctx: int, n: int, p: int) -> int:
    h = _P()
    _check(lib().gw_cannon_create(ctx, int(n), int(p), ctypes.byref(h)),
           "gw_cannon_create")
    return h.value


def gw_cannon_destroy(cn: int):
    _check(lib().gw_cannon_destroy(cn), "gw_cannon_destroy")


def gw_cannon_set(cn: int, a, bt, on_device: bool = False):
    _check(lib().gw_cannon_set(cn, _ptr(a), _ptr(bt), int(bool(on_device))),
           "gw_cannon_set")


def gw_cannon_run(cn: int, stream=None):
    _check(lib().gw_cannon_run(cn, _stream(stream)), "gw_cannon_run")


def gw_cannon_schedule(cn: int, tile_m: int = 256, group: int = 4):
    _check(lib().gw_cannon_schedule(cn, int(tile_m), int(group)),
           "gw_cannon_schedule")


def gw_cannon_sync(cn: int):
    _check(lib().gw_cannon_sync(cn), "gw_cannon_sync")


def gw_cannon_read_c(cn: int, out, on_device: bool = False):
    _check(lib().gw_cannon_read_c(cn, _ptr(out), int(bool(on_device))),
           "gw_cannon_read_c")
    return out


def gw_cannon_selftest_timeout(cn: int, limit_us: int):
    """(status, expired) of the block-product kernel's timeout self-test;
    a status of GW_ERR_TIMEOUT is the expected outcome, not raised."""
    e = _I()
    st = lib().gw_cannon_selftest_timeout(cn, int(limit_us), ctypes.byref(e))
    if st not in (GW_OK, GW_ERR_TIMEOUT):
        _check(st, "gw_cannon_selftest_timeout")
    return st, e.value


def gw_cannon_timing(cn: int, enable: bool):
    _check(lib().gw_cannon_timing(cn, int(bool(enable))), "gw_cannon_timing")


def gw_cannon_stats(cn: int) -> dict:
    ms, n, g = _D(), ctypes.c_longlong(), _I()
    _check(lib().gw_cannon_stats(cn, ctypes.byref(ms), ctypes.byref(n),
                                 ctypes.byref(g)), "gw_cannon_stats")
    return {"gemm_ms": ms.value, "launches": n.value, "grid": g.value}


# ---------------------------------------------------------------- domains

def shot_desc(nx, ny, nz, *, h=10.0, courant=0.0, dt=0.0, nsteps=0,
              dtype="f32", sponge=0, sponge_a=0.0, periodic=0,
              halo_mode=GW_HALO_FUSED, chunk=0, tile=0, zchunk=0,
              scale_u=0.0, scale_w=0.0, persistent=0,
              schedule=0) -> gw_shot_desc:
    d = gw_shot_desc()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.h, d.courant, d.dt = float(h), float(courant), float(dt)
    d.nsteps = int(nsteps)
    d.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    d.sponge, d.sponge_a = int(sponge), float(sponge_a)
    d.periodic, d.halo_mode = int(periodic), int(halo_mode)
    d.chunk, d.tile, d.zchunk = int(chunk), int(tile), int(zchunk)
    d.scale_u, d.scale_w = float(scale_u), float(scale_w)
    d.persistent = int(persistent)
    d.schedule = int(schedule)
    return d


def gw_domain_create(ctx: int, desc: gw_shot_desc, px=1, py=1, pz=1,
                     split_x=None, split_y=None, split_z=None,
                     symmetric=True) -> int:
    def arr(s):
        return None if s is None else (_I * len(s))(*[int(v) for v in s])
    h = _P()
    sx, sy, sz = arr(split_x), arr(split_y), arr(split_z)
    _check(lib().gw_domain_create(
        ctx, ctypes.byref(desc), int(px), int(py), int(pz),
        ctypes.cast(sx, _P) if sx is not None else None,
        ctypes.cast(sy, _P) if sy is not None else None,
        ctypes.cast(sz, _P) if sz is not None else None,
        int(bool(symmetric)), ctypes.byref(h)), "gw_domain_create")
    return h.value


def gw_domain_destroy(dom: int):
    _check(lib().gw_domain_destroy(dom), "gw_domain_destroy")


def gw_domain_bytes(desc: gw_shot_desc, px=1, py=1, pz=1, nrec=0) -> int:
    n = _SZ()
    _check(lib().gw_domain_bytes(ctypes.byref(desc), int(px), int(py),
                                 int(pz), int(nrec), ctypes.byref(n)),
           "gw_domain_bytes")
    return n.value


def gw_domain_info_get(dom: int) -> dict:
    i = gw_domain_info()
    _check(lib().gw_domain_info_get(dom, ctypes.byref(i)),
           "gw_domain_info_get")
    return {k: getattr(i, k) for k, _ in gw_domain_info._fields_}


def gw_set_model(dom: int, vel: np.ndarray):
    v = np.ascontiguousarray(vel, dtype=np.float64)
    _check(lib().gw_set_model(dom, _ptr(v)), "gw_set_model")


def gw_set_model_f32(dom: int, vel: np.ndarray):
    v = np.ascontiguousarray(vel, dtype=np.float32)
    _check(lib().gw_set_model_f32(dom, _ptr(v)), "gw_set_model_f32")


def gw_set_model_layered(dom: int, vz: np.ndarray):
    v = np.ascontiguousarray(vz, dtype=np.float64)
    _check(lib().gw_set_model_layered(dom, _ptr(v)), "gw_set_model_layered")


def gw_ricker(f_peak: float, dt: float, n: int) -> np.ndarray:
    out = np.zeros(int(n), dtype=np.float32)
    _check(lib().gw_ricker(float(f_peak), float(dt), int(n), _ptr(out)),
           "gw_ricker")
    return out


def gw_round_to_f32(in_dev, out_dev, n: int, stream=None):
    _check(lib().gw_round_to_f32(_ptr(in_dev), _ptr(out_dev), int(n),
                                 _stream(stream)), "gw_round_to_f32")


def gw_inject_source(dom: int, gx: int, gy: int, gz: int, wavelet):
    w = np.ascontiguousarray(wavelet, dtype=np.float32)
    _check(lib().gw_inject_source(dom, int(gx), int(gy), int(gz), _ptr(w),
                                  int(w.size)), "gw_inject_source")


def gw_inject_ricker(dom: int, gx: int, gy: int, gz: int, f_peak: float):
    _check(lib().gw_inject_ricker(dom, int(gx), int(gy), int(gz),
                                  float(f_peak)), "gw_inject_ricker")


def gw_set_receivers(dom: int, xyz):
    r = np.ascontiguousarray(np.asarray(xyz, dtype=np.int32).reshape(-1, 3))
    _check(lib().gw_set_receivers(dom, int(r.shape[0]),
                                  _ptr(r) if r.size else None),
           "gw_set_receivers")


def gw_step(dom: int, nsteps: int, stream=None):
    _check(lib().gw_step(dom, int(nsteps), _stream(stream)), "gw_step")


def gw_put_halo(dom: int, stream=None):
    _check(lib().gw_put_halo(dom, _stream(stream)), "gw_put_halo")


def gw_barrier(dom: int, stream=None, sync: bool = False):
    _check(lib().gw_barrier(dom, _stream(stream), int(bool(sync))),
           "gw_barrier")


def gw_read_receivers(dom: int, nrec: int, nsteps: int, out=None):
    if out is None:
        out = np.zeros((int(nrec), int(nsteps)), dtype=np.float32)
    _check(lib().gw_read_receivers(dom, _ptr(out), int(nrec), int(nsteps)),
           "gw_read_receivers")
    return out


def gw_read_wavefield(dom: int, which: int, shape, f64: bool = True,
                      out=None):
    if out is None:
        out = np.zeros(shape, dtype=np.float64 if f64 else np.float32)
    _check(lib().gw_read_wavefield(dom, int(which), _ptr(out),
                                   int(out.dtype == np.float64)),
           "gw_read_wavefield")
    return out


def gw_write_wavefield(dom: int, which: int, arr):
    a = np.ascontiguousarray(arr)
    if a.dtype not in (np.float64, np.float32):
        a = a.astype(np.float64)
    _check(lib().gw_write_wavefield(dom, int(which), _ptr(a),
                                    int(a.dtype == np.float64)),
           "gw_write_wavefield")


def gw_norms(dom: int, n: int) -> np.ndarray:
    out = np.zeros(int(n), dtype=np.float64)
    _check(lib().gw_norms(dom, _ptr(out) if n else None, int(n)), "gw_norms")
    return out


def gw_check(dom: int) -> tuple[float, float]:
    a, b = _D(), _D()
    _check(lib().gw_check(dom, ctypes.byref(a), ctypes.byref(b)), "gw_check")
    return a.value, b.value


def gw_check_fields_noalloc(u_cur, u_prev, coef, dtype, nx: int, ny: int,
                            nz: int, px: int, scale_u: float, out_dev,
                            stream=None):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(lib().gw_check_fields_noalloc(
        _ptr(u_cur), _ptr(u_prev), _ptr(coef), dt, int(nx), int(ny), int(nz),
        int(px), float(scale_u), _ptr(out_dev), _stream(stream)),
        "gw_check_fields_noalloc")


def gw_kernel_timing(dom: int, enable: bool):
    _check(lib().gw_kernel_timing(dom, int(bool(enable))), "gw_kernel_timing")


def gw_kernel_stats_get(dom: int) -> dict:
    s = gw_kernel_stats()
    _check(lib().gw_kernel_stats_get(dom, ctypes.byref(s)),
           "gw_kernel_stats_get")
    return {"launches": s.launches, "total_ms": s.total_ms,
            "halo_ms": s.halo_ms}


def gw_batch_create(ctx: int, doms, chunk: int = 0,
                    persistent: bool = False) -> int:
    arr = (_P * len(doms))(*doms)
    h = _P()
    _check(lib().gw_batch_create(ctx, len(doms), ctypes.cast(arr, _P),
                                 int(chunk), int(bool(persistent)),
                                 ctypes.byref(h)), "gw_batch_create")
    return h.value


def gw_batch_destroy(b: int):
    _check(lib().gw_batch_destroy(b), "gw_batch_destroy")


def gw_batch_step(b: int, nsteps: int, stream=None):
    _check(lib().gw_batch_step(b, int(nsteps), _stream(stream)),
           "gw_batch_step")


def gw_batch_info(b: int) -> dict:
    g, c, i = _I(), _I(), _I()
    _check(lib().gw_batch_info(b, ctypes.byref(g), ctypes.byref(c),
                               ctypes.byref(i)), "gw_batch_info")
    return {"groups": g.value, "ctas": c.value, "items": i.value}


def gw_batch_timing(b: int, enable: bool):
    _check(lib().gw_batch_timing(b, int(bool(enable))), "gw_batch_timing")


def gw_batch_stats_get(b: int) -> dict:
    s = gw_kernel_stats()
    _check(lib().gw_batch_stats_get(b, ctypes.byref(s)), "gw_batch_stats_get")
    return {"launches": s.launches, "total_ms": s.total_ms,
            "halo_ms": s.halo_ms}


def gw_pick_tile(dtype, nx: int, ny: int) -> int:
    t = _I()
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(lib().gw_pick_tile(dt, int(nx), int(ny), ctypes.byref(t)),
           "gw_pick_tile")
    return t.value


def gw_tile_count(dtype) -> int:
    n = _I()
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(lib().gw_tile_count(dt, ctypes.byref(n)), "gw_tile_count")
    return n.value


def gw_autotune(ctx: int, desc: gw_shot_desc, px: int = 1, py: int = 1,
                pz: int = 1, steps: int = 10, all_times: bool = False):
    """(best tile, ms per step), plus the list of every tile's ms per step
    (0 where a tile does not fit) when all_times is set."""
    n = gw_tile_count(desc.dtype)
    t, ms = _I(), _D()
    times = np.zeros(n, dtype=np.float64)
    _check(lib().gw_autotune(ctx, ctypes.byref(desc), int(px), int(py),
                             int(pz), int(steps), ctypes.byref(t),
                             ctypes.byref(ms), _ptr(times), n), "gw_autotune")
    if all_times:
        return t.value, ms.value, times.tolist()
    return t.value, ms.value


def gw_plan_tiles(ctx: int, descs, steps: int = 10,
                  margin: float = 0.05) -> list[int]:
    arr = (gw_shot_desc * len(descs))(*descs)
    out = np.zeros(len(descs), dtype=np.int32)
    _check(lib().gw_plan_tiles(ctx, len(descs), ctypes.cast(arr, _P),
                               int(steps), float(margin), _ptr(out)),
           "gw_plan_tiles")
    return [int(v) for v in out]


def gw_server_create(ctx: int, hbm_budget: int, max_slots: int,
                     chunk: int = 0) -> int:
    h = _P()
    _check(lib().gw_server_create(ctx, int(hbm_budget), int(max_slots),
                                  int(chunk), ctypes.byref(h)),
           "gw_server_create")
    return h.value


def gw_server_destroy(srv: int):
    _check(lib().gw_server_destroy(srv), "gw_server_destroy")


def gw_submit(srv: int, req: gw_request) -> int:
    """The caller keeps req.vel and req.traces valid until the ticket
    completes (gw_wait returned it)."""
    t = _U64()
    _check(lib().gw_submit(srv, ctypes.byref(req), ctypes.byref(t)),
           "gw_submit")
    return t.value


def gw_wait(srv: int, ticket: int, timeout_ms: int = -1) -> dict:
    r = gw_result()
    _check(lib().gw_wait(srv, int(ticket), int(timeout_ms), ctypes.byref(r)),
           "gw_wait")
    return {k: getattr(r, k) for k, _ in gw_result._fields_}


def gw_server_stats_get(srv: int) -> dict:
    st = gw_server_stats()
    _check(lib().gw_server_stats_get(srv, ctypes.byref(st)),
           "gw_server_stats_get")
    return {k: getattr(st, k) for k, _ in gw_server_stats._fields_}


def gw_server_now(srv: int) -> float:
    return float(lib().gw_server_now(srv))


def gw_selftest_timeout(ctx: int, limit_us: int) -> tuple[int, int]:
    """(status, expired bits): GW_ERR_TIMEOUT with bits 3 is the expected
    outcome (both device waits gave up)."""
    bits = _I()
    st = lib().gw_selftest_timeout(ctx, int(limit_us), ctypes.byref(bits))
    return st, bits.value


def gw_state_bytes(dom: int) -> int:
    n = _SZ()
    _check(lib().gw_state_bytes(dom, ctypes.byref(n)), "gw_state_bytes")
    return n.value


def gw_save_state(dom: int) -> np.ndarray:
    buf = np.zeros(gw_state_bytes(dom), dtype=np.uint8)
    _check(lib().gw_save_state(dom, _ptr(buf)), "gw_save_state")
    return buf


def gw_load_state(dom: int, buf: np.ndarray):
    _check(lib().gw_load_state(dom, _ptr(np.ascontiguousarray(buf))),
           "gw_load_state")
