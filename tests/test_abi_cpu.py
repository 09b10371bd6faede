"""CPU-only checks of the C ABI: the library builds and loads, exports every
entry point the header declares, and its host-side PGAS logic (symmetric
offsets, asymmetric second-level pointers, the remote pointer cache,
put/get/fence) behaves as section 3.2 of the paper describes, exercised on
a host-only context whose segment is host memory."""

import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_02486_gb300 import buildlib as build_mod
from paper_2506_02486_gb300 import gbwave as gw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbwave.h")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return gw.lib()


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gw_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree(lib):
    decl = declared_symbols()
    assert len(decl) > 30
    assert sorted(gw.symbols()) == decl


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gw.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gw_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_status_strings_and_errors(lib):
    assert gw.gw_status_string(gw.GW_ERR_BUDGET) == "GW_ERR_BUDGET"
    with pytest.raises(gw.GWError) as e:
        gw.gw_segment_attach(gw.gw_ctx_create(-1), 0, 1 << 20, 1)
    assert e.value.status == gw.GW_ERR_ARG


class HostSeg:
    def __init__(self, nbytes, nranks):
        self.buf = np.zeros(nbytes + 4096, dtype=np.uint8)
        base = self.buf.ctypes.data
        self.base = (base + 255) // 256 * 256
        self.ctx = gw.gw_ctx_create(-1)
        gw.gw_segment_attach(self.ctx, self.base, nbytes, nranks, False)
        self.rank_bytes = gw.gw_segment_info(self.ctx)[0]

    def close(self):
        gw.gw_ctx_destroy(self.ctx)


def test_symmetric_allocation_uses_one_offset_on_every_rank(lib):
    s = HostSeg(4 << 20, 4)
    try:
        a = gw.gw_alloc_symmetric(s.ctx, 1000)
        b = gw.gw_alloc_symmetric(s.ctx, 5000)
        for g in (a, b):
            addrs = [gw.gw_resolve(s.ctx, g, r)[0] for r in range(4)]
            offs = {p - s.base - r * s.rank_bytes for r, p in enumerate(addrs)}
            assert len(offs) == 1                      # same offset everywhere
            assert all(p % 256 == 0 for p in addrs)
        pa = gw.gw_resolve(s.ctx, a, 0)[0]
        pb = gw.gw_resolve(s.ctx, b, 0)[0]
        assert pb - pa >= 1000
        assert gw.gw_resolve(s.ctx, a, 2)[1] == 1024   # rounded to 256
    finally:
        s.close()


def test_asymmetric_allocation_via_second_level_pointers(lib):
    s = HostSeg(4 << 20, 3)
    try:
        sizes = [4096, 0, 10000]
        g = gw.gw_alloc_asymmetric(s.ctx, sizes)
        h0, m0 = gw.gw_ptr_cache_stats(s.ctx)
        p0, n0 = gw.gw_resolve(s.ctx, g, 0)
        p2, n2 = gw.gw_resolve(s.ctx, g, 2)
        h1, m1 = gw.gw_ptr_cache_stats(s.ctx)
        assert (h1 - h0, m1 - m0) == (0, 2)            # two record fetches
        # data sits at the end of each rank's segment
        assert p0 + n0 == s.base + s.rank_bytes
        assert p2 + n2 == s.base + 3 * s.rank_bytes
        assert n0 == 4096 and n2 == 10240
        # repeated translations are served by the pointer cache
        for _ in range(5):
            assert gw.gw_resolve(s.ctx, g, 2)[0] == p2
        h2, m2 = gw.gw_ptr_cache_stats(s.ctx)
        assert (h2 - h1, m2 - m1) == (5, 0)
        # the 32-byte record in rank 2's segment points at the data
        rec = None
        for off in range(0, s.rank_bytes, 256):
            raw = ctypes.string_at(s.base + 2 * s.rank_bytes + off, 32)
            addr, nb, rank, flags, _ = np.frombuffer(
                raw, dtype=[("a", "<u8"), ("b", "<u8"), ("r", "<u4"),
                            ("f", "<u4"), ("x", "<u8")])[0]
            if addr == p2:
                rec = (nb, rank, flags)
                break
        assert rec == (10240, 2, 1)
    finally:
        s.close()


def test_free_reuses_space_and_invalidates_cache(lib):
    s = HostSeg(1 << 20, 2)
    try:
        rb = s.rank_bytes
        a = gw.gw_alloc_symmetric(s.ctx, rb // 2)
        with pytest.raises(gw.GWError) as e:
            gw.gw_alloc_symmetric(s.ctx, rb // 2 + 4096)
        assert e.value.status == gw.GW_ERR_BUDGET
        pa = gw.gw_resolve(s.ctx, a, 0)[0]
        gw.gw_free(s.ctx, a)
        b = gw.gw_alloc_symmetric(s.ctx, rb // 2)
        assert gw.gw_resolve(s.ctx, b, 0)[0] == pa
        g = gw.gw_alloc_asymmetric(s.ctx, [1024, 2048])
        gw.gw_resolve(s.ctx, g, 1)
        gw.gw_free(s.ctx, g)
        with pytest.raises(gw.GWError):
            gw.gw_resolve(s.ctx, g, 1)
        # symmetric and asymmetric regions may not collide
        with pytest.raises(gw.GWError) as e:
            gw.gw_alloc_asymmetric(s.ctx, [rb // 2 + 4096, 0])
        assert e.value.status == gw.GW_ERR_BUDGET
        used = gw.gw_segment_info(s.ctx)
        assert used[1] == rb // 2 and used[2] == 0
    finally:
        s.close()


def test_put_get_fence_on_host_context(lib):
    s = HostSeg(1 << 20, 4)
    try:
        g = gw.gw_alloc_symmetric(s.ctx, 4096)
        a = gw.gw_alloc_asymmetric(s.ctx, [512, 1024, 0, 256])
        src = np.arange(256, dtype=np.uint8)
        gw.gw_put(s.ctx, g, 3, 100, src, 256)
        gw.gw_put(s.ctx, a, 1, 768, src, 256)
        gw.gw_fence(s.ctx)
        dst = np.zeros(256, dtype=np.uint8)
        gw.gw_get(s.ctx, dst, g, 3, 100, 256)
        assert np.array_equal(dst, src)
        dst[:] = 0
        gw.gw_get(s.ctx, dst, a, 1, 768, 256)
        assert np.array_equal(dst, src)
        with pytest.raises(gw.GWError):           # beyond the rank's block
            gw.gw_put(s.ctx, a, 1, 900, src, 256)
        with pytest.raises(gw.GWError):
            gw.gw_put(s.ctx, g, 4, 0, src, 16)    # no such rank
    finally:
        s.close()


def test_ricker_host_function(lib):
    w = gw.gw_ricker(20.0, 0.001, 200)
    assert w.dtype == np.float32
    assert int(np.argmax(w)) == 50            # t0 = 1/f = 50 dt
    assert w[50] == pytest.approx(1.0)


def test_domain_needs_device_context(lib):
    s = HostSeg(1 << 20, 1)
    try:
        with pytest.raises(gw.GWError) as e:
            gw.gw_domain_create(s.ctx, gw.shot_desc(8, 8, 8, nsteps=4))
        assert e.value.status == gw.GW_ERR_STATE
    finally:
        s.close()


STRUCTS = ["gw_shot_desc", "gw_domain_info", "gw_kernel_stats", "gw_request",
           "gw_result", "gw_server_stats"]


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and offsetof of every struct the binding mirrors, from a C
    program compiled against the header, equal the ctypes layout."""
    lines = ["#include <stdio.h>", "#include <stddef.h>",
             '#include "gbwave.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(gw, name)
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    for name in STRUCTS:
        cls = getattr(gw, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_domain_bytes_bounds_the_fields(lib):
    """The admission footprint covers the padded fields (two wavefields and
    coef; plus w and an FP16 coef in the delta form) and grows with the
    step count (traces, wavelet table)."""
    from paper_2506_02486_gb300.runtime import padded_bytes
    for dtype, nf in (("f32", 3), ("f64", 3), ("bf16", 4), ("f16s", 4)):
        d = gw.shot_desc(100, 90, 80, nsteps=10, dtype=dtype)
        b = gw.gw_domain_bytes(d)
        assert b >= nf * padded_bytes(100, 90, 80, dtype)
        assert b < nf * padded_bytes(100, 90, 80, dtype) * 1.2 + (4 << 20)
        d2 = gw.shot_desc(100, 90, 80, nsteps=1000, dtype=dtype)
        assert gw.gw_domain_bytes(d2, nrec=64) > b + 64 * 990 * 4
    with pytest.raises(gw.GWError):
        gw.gw_domain_bytes(gw.shot_desc(0, 8, 8))


def test_selftest_needs_a_device_context(lib):
    ctx = gw.gw_ctx_create(-1)
    try:
        st, bits = gw.gw_selftest_timeout(ctx, 1000)
        assert st == gw.GW_ERR_STATE and bits == 0
    finally:
        gw.gw_ctx_destroy(ctx)


def test_tile_model_prefers_fitting_tiles(lib):
    """The host-side tile model: the default tile on a large grid that it
    tiles well, a 32-wide tile where 64-wide tiles would leave half-empty
    columns, and only the type's own tiles."""
    assert gw.gw_pick_tile("f32", 512, 512) == 1            # 64 x 28
    assert gw.gw_pick_tile("f32", 96, 96) == 3              # 32 x 56
    assert gw.gw_pick_tile("bf16", 96, 112) == 4            # 32 x 56
    for dt in ("f32", "f64", "f16s", "bf16"):
        for n in (17, 64, 100, 333):
            assert 1 <= gw.gw_pick_tile(dt, n, n) <= gw.gw_tile_count(dt)
    with pytest.raises(gw.GWError):
        gw.gw_pick_tile("f32", 0, 8)


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the CUDA library the binding raises."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2506_02486_gb300 import gbwave as gw\n"
            "gw.LIB_PATH = %r\n"
            "try:\n"
            "    gw.lib()\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'missing' in str(e))\n" %
            (ROOT, str(tmp_path / "absent.so")))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True,
                         text=True, check=True).stdout
    assert out.strip() == "raised True"
