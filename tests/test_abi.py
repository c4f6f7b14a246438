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
    assert L.wc_rhs(h, None, None, None) == 1
    assert L.wc_limit(h, 5, 1, None, None, None, None, None, None, None) == 1
    buf = ctypes.create_string_buffer(64)
    L.wc_last_error(h, buf, 64)
    L.wc_destroy(h)
