"""The C-ABI library: it builds, loads, exports every entry point declared in
include/gosurf.h, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2206_14735_gb300 as gs
import scenegen as sg
from paper_2206_14735_gb300 import _lib
from paper_2206_14735_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    return _lib.lib()


def test_library_exports_every_declared_symbol(L):
    declared = declared_entry_points()
    assert {"gs_sample_rays", "gs_forward", "gs_backward", "gs_adam_step", "gs_query_sdf"} <= declared
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared <= set(_lib.EXPORTS) | declared  # binding covers the declared set
    assert set(_lib.EXPORTS) <= declared


def test_param_count_matches_layout(L):
    for w in sg.WORKLOADS.values():
        cfg = gs.make_config(w)
        ng = ctypes.c_int64()
        n = L.gs_param_count(ctypes.byref(cfg), ctypes.byref(ng))
        offs, n_grid, n_tot = w.layout()
        assert (n, ng.value) == (n_tot, n_grid)


def test_create_rejects_bad_configs_on_host(L):
    w = sg.WORKLOADS["cube-1024x64"]
    h = ctypes.c_void_p()
    bad = gs.make_config(w)
    bad.dims[2][1] = 1
    assert L.gs_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert b"vertices" in L.gs_last_error(None)
    bad = gs.make_config(w)
    bad.voxel[0] = 0.0
    assert L.gs_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = gs.make_config(w)
    bad.n_strat, bad.n_guided = 100, 100
    assert L.gs_create(ctypes.byref(bad), ctypes.byref(h)) == 6
    bad = gs.make_config(w)
    bad.far_m = bad.near_m
    assert L.gs_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    assert L.gs_create(None, ctypes.byref(h)) == 1
    assert h.value is None


def test_entry_points_reject_null_context(L):
    assert L.gs_sample_rays(None, None, 0, 0, None, None) == 1
    assert L.gs_forward(None, None, None, None, None, None, None, None, None) == 1
    assert L.gs_backward(None, None, None, None, None, None, None) == 1
    assert L.gs_adam_step(None, None, None, None, None, 0, 0, 1, 0.0, 0.0, 0.9, 0.999, 1e-8, None, None) == 1
    assert L.gs_query_sdf(None, None, None, 0, None, None, None) == 1
    assert L.gs_sync_status(None) == 1


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()
