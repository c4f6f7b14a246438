"""The C-ABI library loads and exports every entry point include/wenoc.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2608_00746_b300 import wenoc

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                   "wenoc.h")


def declared():
    txt = open(HDR).read()
    return sorted(set(re.findall(r"^\s*(?:wc_status|void|int|long|size_t)\s+\*?(wc_\w+)\s*\(",
                                 txt, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for core in ("wc_init_grid", "wc_set_state", "wc_rhs", "wc_rk_step", "wc_limit"):
        assert core in names


def test_library_exports_every_declared_symbol():
    L = wenoc.lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(declared()) <= set(wenoc.exported_symbols())


def desc(**kw):
    d = wenoc.GridDesc()
    d.dim = kw.get("dim", 2)
    n = kw.get("n", (16, 8, 1))
    for a in range(3):
        d.n[a] = n[a]
        d.dx[a] = 0.1
    d.nphase = kw.get("nphase", 2)
    for p in range(d.nphase):
        d.gamma[p] = 1.4
        d.pinf[p] = 0.0
    d.flux = kw.get("flux", 0)
    d.precision = kw.get("precision", 0)
    d.energy_limiter = 1
    for k in range(6):
        d.bc[k] = kw.get("bc", 0)
    d.scheme = kw.get("scheme", 0)
    d.kmodel = kw.get("kmodel", 0)
    d.js_eps = kw.get("js_eps", 0.0)
    return d


def init(d):
    h = ctypes.c_void_p()
    st = wenoc.lib().wc_init_grid(ctypes.byref(d), ctypes.byref(h))
    if st == 0:
        wenoc.lib().wc_destroy(h)
    return st, h


def test_init_grid_accepts_valid_and_sizes():
    d = desc()
    h = ctypes.c_void_p()
    assert wenoc.lib().wc_init_grid(ctypes.byref(d), ctypes.byref(h)) == 0
    L = wenoc.lib()
    assert L.wc_nvar(h) == 2 * 2 + 2 + 1
    assert L.wc_ncell(h) == 16 * 8
    assert L.wc_workspace_bytes(h) >= 3 * 7 * 128 * 8
    L.wc_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("seg", [0, 14])
def test_workspace_parts(precision, seg):
    """The workspace: three state buffers and 256 bytes, then the primitive
    slots of the window schedule ((NV + 1) words a cell, none for the
    segment schedule or a 1-D grid), then the reduced precision's face
    buffer; each part rounded to 256 bytes."""
    d = desc(precision=precision)
    d.seg = seg
    h = ctypes.c_void_p()
    L = wenoc.lib()
    assert L.wc_init_grid(ctypes.byref(d), ctypes.byref(h)) == 0
    up = lambda b: (b + 255) // 256 * 256  # noqa: E731
    nv, nc = 7, 128
    prim = 0 if seg else up((nv + 1) * nc * 8)
    assert L.wc_prim_buffer_bytes(h) == prim
    face = L.wc_face_buffer_bytes(h)
    assert (face > 0) == (precision == 1 and seg == 0)
    assert L.wc_workspace_bytes(h) == 3 * up(nv * nc * 8) + 256 + prim + face
    L.wc_destroy(h)
    d1 = desc(precision=precision, dim=1, n=(128, 1, 1), nphase=2)
    assert L.wc_init_grid(ctypes.byref(d1), ctypes.byref(h)) == 0
    assert L.wc_prim_buffer_bytes(h) == 0
    L.wc_destroy(h)


@pytest.mark.parametrize("bad,status", [
    (dict(dim=4), 1), (dict(nphase=0), 5), (dict(nphase=6), 5),
    (dict(n=(2, 8, 1)), 1), (dict(n=(16, 8, 2)), 1), (dict(flux=7), 1),
    (dict(precision=9), 5), (dict(bc=5), 1), (dict(scheme=4), 1), (dict(scheme=-1), 1),
    (dict(kmodel=2), 1), (dict(scheme=3, js_eps=-1.0), 1),
    # the comparison schemes (WENO-W, WENO-JS) are built in FP64 only
    (dict(scheme=2, precision=1), 5), (dict(scheme=3, precision=2), 5),
])
def test_init_grid_rejects(bad, status):
    assert init(desc(**bad))[0] == status


@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_init_grid_accepts_every_scheme(scheme):
    assert init(desc(scheme=scheme))[0] == 0


def test_periodic_must_pair():
    d = desc()
    d.bc[0], d.bc[1] = 0, 2
    assert init(d)[0] == 1


def test_calls_before_binding_fail_cleanly():
    d = desc()
    h = ctypes.c_void_p()
    L = wenoc.lib()
    assert L.wc_init_grid(ctypes.byref(d), ctypes.byref(h)) == 0
    dt = ctypes.c_double(0)
    assert L.wc_rk_step(h, 0.2, 0.0, 1, ctypes.byref(dt), None) == 6   # WC_ERR_STATE
    assert L.wc_rk_step(h, 0.0, 0.0, 1, None, None) == 1                # no cfl, no dt
    hb = (ctypes.c_double * (L.wc_nvar(h) * L.wc_ncell(h)))()
    assert L.wc_rk_step_host(h, hb, hb, 0.2, 0.0, 1, None) == 6          # nothing bound
    assert L.wc_rk_step_host(h, None, hb, 0.2, 0.0, 1, None) == 1
    assert L.wc_rk_step_host(h, hb, hb, 0.2, 0.0, 0, None) == 1          # nsteps < 1
    assert L.wc_rk_step_host(h, hb, hb, 0.0, 0.0, 1, None) == 1
    assert L.wc_rhs(h, None, None, None) == 1
    assert L.wc_limit(h, 5, 1, None, None, None, None, None, None, None) == 1
    buf = ctypes.create_string_buffer(64)
    L.wc_last_error(h, buf, 64)
    L.wc_destroy(h)


@pytest.mark.parametrize("n", [(0, 8, 1), (-3, 8, 1), (16, 0, 1)])
def test_init_grid_rejects_empty_grids(n):
    assert init(desc(n=n))[0] == 1


def pdesc(**kw):
    d = wenoc.PatchesDesc()
    d.nphase = kw.get("nphase", 3)
    for p in range(min(d.nphase, wenoc.MAX_PHASE)):
        d.gamma[p] = 1.4
        d.pinf[p] = 0.0
    d.flux = kw.get("flux", 0)
    d.precision = kw.get("precision", 1)
    d.energy_limiter = 1
    d.kmodel = kw.get("kmodel", 0)
    return d


def pinit(d, edges):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * max(len(edges), 1))(*edges)
    d.npatch = len(edges)
    st = wenoc.lib().wc_patches_init(ctypes.byref(d), arr, ctypes.byref(h))
    return st, h


def test_patches_init_tables_and_workspace():
    """Host-side patch tables: pooled offsets in patch order, the window
    schedule's face buffer sized for the largest group of equal patches
    (mixed precision only; (2 NV + 1) e^2 (e + 2) doubles a patch)."""
    L = wenoc.lib()
    edges = [8, 32, 8, 12, 32, 3]
    st, h = pinit(pdesc(), edges)
    assert st == 0
    try:
        assert L.wc_patches_ncell(h) == sum(e ** 3 for e in edges)
        offs = [L.wc_patches_offset(h, p) for p in range(len(edges))]
        assert offs == [sum(e ** 3 for e in edges[:p]) for p in range(len(edges))]
        assert L.wc_patches_offset(h, len(edges)) == -1
        nv = 2 * 3 + 4
        most = max(edges.count(e) * (2 * nv + 1) * e * e * (e + 2) for e in set(edges))
        fb = L.wc_patches_face_buffer_bytes(h)
        assert most * 8 <= fb < most * 8 + 256
        nc = sum(e ** 3 for e in edges)
        state = (nv * nc * 8 + 255) // 256 * 256
        prim = L.wc_patches_prim_buffer_bytes(h)
        assert prim == ((nv + 1) * nc * 8 + 255) // 256 * 256
        assert L.wc_patches_workspace_bytes(h) >= 4 * state + prim + fb
    finally:
        L.wc_patches_destroy(h)
    st, h = pinit(pdesc(precision=0), edges)
    assert st == 0
    assert L.wc_patches_face_buffer_bytes(h) == 0
    L.wc_patches_destroy(h)


@pytest.mark.parametrize("kw,edges,status", [
    ({}, [], 1),                      # no patch
    ({}, [8, 2], 1),                  # an edge below the stencil's 3 cells
    ({}, [8, 1025], 1),               # above 1024
    ({"nphase": 0}, [8], 5), ({"nphase": 6}, [8], 5),
    ({"flux": 3}, [8], 1), ({"precision": 2}, [8], 5),  # learned: grids only
    ({"kmodel": 2}, [8], 1), ({"kmodel": -1}, [8], 1),
])
def test_patches_init_rejects(kw, edges, status):
    st, h = pinit(pdesc(**kw), edges)
    if st == 0:
        wenoc.lib().wc_patches_destroy(h)
    assert st == status


def test_patches_schedule_kinds():
    L = wenoc.lib()
    st, h = pinit(pdesc(), [8, 16])
    assert st == 0
    try:
        for b, c, k in [(128, 4, 2), (64, 3, 1), (32, 1, 0)]:
            assert L.wc_patches_set_schedule(h, b, c, k) == 0
        for b, c, k in [(128, 4, 3), (128, 4, -1), (100, 2, 1), (128, 0, 1), (128, 17, 2)]:
            assert L.wc_patches_set_schedule(h, b, c, k) == 1
    finally:
        L.wc_patches_destroy(h)
