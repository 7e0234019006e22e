"""CPU-only checks of the C-ABI library: it builds, loads, exports every
symbol include/ooc.h declares, and its host-side planning logic (shape and
rate validation, budget-derived slab thickness) behaves as documented.  No
kernel is launched here."""
import ctypes
import os
import re

import pytest

import paper_2109_05410_gb300 as ooc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    ooc.build()
    return ooc.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ooc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ooc_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    assert ooc.ooc_status_string(0) == "ok"
    assert "budget" in ooc.ooc_status_string(2)
    assert ooc.ooc_status_string(99) == "unknown status"


def test_compressed_bytes(L):
    assert ooc.ooc_compressed_bytes(1024, 1024, 1024, 16) == 1024 ** 3 * 2
    assert ooc.ooc_compressed_bytes(8, 8, 8, 24) == 512 * 3
    assert ooc.ooc_compressed_bytes(6, 8, 8, 16) == 2 * 2 * 2 * 8 * 16  # partial blocks count whole
    assert ooc.ooc_compressed_bytes(1, 1, 1, 8) == 64
    assert ooc.ooc_compressed_bytes(0, 8, 8, 16) == 0
    assert ooc.ooc_compress_var_bound(5, 5, 5) == 8 * 130 * 4
    # the encoder's tile counter and one status word per tile of 128 blocks
    assert ooc.ooc_var_scratch_bytes(1024, 1024, 1024) == 8 * (256 ** 3 // 128 + 1)
    assert ooc.ooc_compressed_bytes(8, 8, 8, 65) == 0


def make_cfg(**kw):
    c = ooc.OocConfig()
    c.nx, c.ny, c.nz = kw.get("n", (64, 64, 64))
    c.stencil = kw.get("stencil", ooc.OOC_HEAT7)
    c.k = kw.get("k", 2)
    c.r = 1.0 / 6.0
    c.rw_format = kw.get("rw_format", ooc.OOC_FMT_FR4)
    c.rw_rate = kw.get("rw_rate", 16)
    c.ro_format = kw.get("ro_format", ooc.OOC_FMT_FP32)
    c.ro_rate = kw.get("ro_rate", 16)
    c.device_budget_bytes = kw.get("budget", 0)
    c.slab_planes = kw.get("slab_planes", 0)
    c.heat_steps_per_launch = kw.get("spl", 0)
    c.debug_checks = kw.get("debug", 0)
    return c


def plan_create(L, c):
    h = ctypes.c_void_p()
    d, hb = ctypes.c_size_t(), ctypes.c_size_t()
    s = L.ooc_plan_create(ctypes.byref(c), ctypes.byref(h), ctypes.byref(d), ctypes.byref(hb))
    info = None
    if s == 0:
        i = ooc.OocPlanInfo()
        assert L.ooc_plan_get_info(h, ctypes.byref(i)) == 0
        info = i.as_dict()
        L.ooc_plan_destroy(h)
    return s, d.value, hb.value, info


def test_plan_validation(L):
    assert plan_create(L, make_cfg(n=(64, 64, 62), slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(k=0, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(rw_rate=0, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(rw_rate=65, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(stencil=3, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(slab_planes=6))[0] == 1
    assert plan_create(L, make_cfg(rw_format=7, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg())[0] == 1  # neither a budget nor a slab thickness
    assert plan_create(L, make_cfg(spl=3, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(spl=-1, slab_planes=8))[0] == 1
    assert plan_create(L, make_cfg(spl=2, stencil=ooc.OOC_WAVE25, slab_planes=32, k=2))[0] == 1
    assert plan_create(L, make_cfg(spl=1, stencil=ooc.OOC_WAVE25, slab_planes=32, k=2))[0] == 0


def test_plan_side_limits(L):
    # Each side may be up to 2^20 points (a multiple of 4); one block more
    # is refused (plans with slabs of 4 planes).
    big = 1 << 20
    assert plan_create(L, make_cfg(n=(4, 4, big), k=1, slab_planes=4))[0] == 0
    assert plan_create(L, make_cfg(n=(big, 4, 4), k=1, slab_planes=4))[0] == 0
    for n in ((4, 4, big + 4), (4, big + 4, 4), (big + 4, 4, 4)):
        assert plan_create(L, make_cfg(n=n, k=1, slab_planes=4))[0] == 1


def test_fused_pairs_reserve_bands(L):
    # Fused heat7 pairs keep, per pair of the pass and slab parity, the 2h
    # top planes of the intermediate level for the next slab.
    plane = 64 * 64 * 4
    for k in (1, 2, 4, 5):
        s1, d1, _, _ = plan_create(L, make_cfg(k=k, slab_planes=16, spl=1))
        s2, d2, _, _ = plan_create(L, make_cfg(k=k, slab_planes=16, spl=2))
        s0, d0, _, _ = plan_create(L, make_cfg(k=k, slab_planes=16, spl=0))
        assert s1 == 0 and s2 == 0 and s0 == 0
        assert d2 - d1 == 2 * (k // 2) * 2 * plane
        # the default runs pairs whenever k >= 2
        assert d0 == (d2 if k >= 2 else d1)


def test_budget_derivation(L):
    # The device budget forces streaming even though the grid would fit:
    # the plan picks the largest 4-aligned slab that fits the arena.
    plane = 1024 * 1024 * 4
    s, dev, host, info = plan_create(L, make_cfg(n=(1024, 1024, 1024), k=4, rw_format=ooc.OOC_FMT_FR4, rw_rate=16,
                                                 budget=1 << 30))
    assert s == 0
    assert dev <= 1 << 30
    T = info["slab_planes"]
    assert T % 4 == 0 and T >= 32
    assert info["nslab"] == -(-1024 // T)
    assert info["common_planes"] == 4 and info["halo"] == 1
    assert info["ring_planes"] >= T + 4 + 2
    assert host == 1024 ** 3 * 2
    # one more slab plane would not fit
    s2, dev2, _, _ = plan_create(L, make_cfg(n=(1024, 1024, 1024), k=4, rw_rate=16, slab_planes=T + 4))
    assert s2 == 0 and dev2 > 1 << 30
    # FP32 storage lands slabs directly in a ring twice as deep
    s3, dev3, host3, info3 = plan_create(L, make_cfg(n=(1024, 1024, 1024), k=4, rw_format=ooc.OOC_FMT_FP32,
                                                     budget=1 << 30))
    assert s3 == 0 and host3 == 1024 ** 3 * 4
    assert info3["ring_planes"] >= 2 * info3["slab_planes"] + 4 + 2
    # a budget below one 4-plane slab is refused
    s4 = plan_create(L, make_cfg(n=(1024, 1024, 1024), k=4, budget=8 * plane))[0]
    assert s4 == 2


def test_wave_plan_geometry(L):
    s, dev, host, info = plan_create(L, make_cfg(n=(128, 128, 128), stencil=ooc.OOC_WAVE25, k=10,
                                                 rw_format=ooc.OOC_FMT_FR4, rw_rate=16, ro_format=ooc.OOC_FMT_FR4,
                                                 ro_rate=16, slab_planes=32))
    assert s == 0
    assert info["halo"] == 4 and info["common_planes"] == 40 and info["nrings"] == 3
    assert host == 3 * 128 ** 3 * 2


def test_trace_of_an_unstepped_plan_is_empty(L):
    # ooc_plan_get_trace: no profiled ooc_step yet, so no records; argument
    # errors are refused without touching the plan.
    c = make_cfg(slab_planes=8)
    h = ctypes.c_void_p()
    d, hb = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.ooc_plan_create(ctypes.byref(c), ctypes.byref(h), ctypes.byref(d), ctypes.byref(hb)) == 0
    try:
        n = ctypes.c_int64(-7)
        assert L.ooc_plan_get_trace(h, None, 0, ctypes.byref(n)) == 0 and n.value == 0
        recs = (ooc.OocTraceRec * 4)()
        assert L.ooc_plan_get_trace(h, recs, 4, ctypes.byref(n)) == 0 and n.value == 0
        assert L.ooc_plan_get_trace(h, None, 4, ctypes.byref(n)) == 1
        assert L.ooc_plan_get_trace(h, recs, -1, ctypes.byref(n)) == 1
        assert L.ooc_plan_get_trace(h, recs, 4, None) == 1
        assert L.ooc_plan_get_trace(None, recs, 4, ctypes.byref(n)) == 1
    finally:
        L.ooc_plan_destroy(h)
    assert ctypes.sizeof(ooc.OocTraceRec) == 40


def test_debug_checks_add_guard_regions(L):
    # debug_checks = 1 puts 256 guard bytes after every arena region (each
    # ring, each nonempty staging buffer, the fused-pair bands, the time and
    # source slot) plus a 256-byte flag; the geometry is otherwise the same.
    cases = [
        (dict(slab_planes=16, spl=1), 2 + 4 + 1),                                # heat7 FR4
        (dict(slab_planes=16, spl=1, rw_format=ooc.OOC_FMT_FP32), 2 + 1),        # FP32: no staging
        (dict(slab_planes=16, spl=2, k=4), 2 + 4 + 1 + 1),                       # fused pairs: bands
        (dict(slab_planes=16), 2 + 4 + 1 + 1),                                   # the default (k = 2): pairs
        (dict(slab_planes=32, stencil=ooc.OOC_WAVE25, k=2, ro_format=ooc.OOC_FMT_FR4), 3 + 2 * (3 + 2) + 1),
    ]
    for kw, nguard in cases:
        s0, d0, h0, i0 = plan_create(L, make_cfg(**kw))
        s1, d1, h1, i1 = plan_create(L, make_cfg(debug=1, **kw))
        assert s0 == 0 and s1 == 0, kw
        assert d1 - d0 == 256 * (nguard + 1), (kw, d1 - d0)
        assert h1 == h0 and i1["slab_planes"] == i0["slab_planes"] and i1["ring_planes"] == i0["ring_planes"]


def test_in_core_entry_points_reject_misaligned_or_aliased_buffers(L):
    # The argument checks run before any CUDA call, so fake device addresses
    # are enough: a buffer that is not 16-byte aligned, or the same buffer
    # passed twice, is refused with OOC_E_INVALID (1) and nothing launches.
    vp = ctypes.c_void_p
    a, b, c, odd = vp(1 << 20), vp(2 << 20), vp(3 << 20), vp((4 << 20) + 4)
    n = (ctypes.c_int64(8),) * 3
    for fn in (L.ooc_heat7_steps, L.ooc_heat7_steps_fused):
        assert fn(odd, b, *n, ctypes.c_double(1 / 6), ctypes.c_int64(2), None) == 1
        assert fn(a, odd, *n, ctypes.c_double(1 / 6), ctypes.c_int64(2), None) == 1
        assert fn(a, a, *n, ctypes.c_double(1 / 6), ctypes.c_int64(2), None) == 1
    w = L.ooc_wave25_steps
    src = (ctypes.c_int64(-1),) * 3
    assert w(odd, b, c, *n, *src, None, ctypes.c_int64(0), ctypes.c_int64(2), None) == 1
    assert w(a, b, odd, *n, *src, None, ctypes.c_int64(0), ctypes.c_int64(2), None) == 1
    assert w(a, a, c, *n, *src, None, ctypes.c_int64(0), ctypes.c_int64(2), None) == 1
    assert L.ooc_heat7_steps_noalloc(odd, *n, ctypes.c_double(1 / 6), ctypes.c_int64(2), None) == 1
