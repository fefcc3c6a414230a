"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/osann.h declares.  Only host-side calls are made
here (no kernel runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1509_03453_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "osann.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set()
    for line in text.splitlines():
        if line.lstrip().startswith("#"):
            continue
        names.update(re.findall(r"\b(osann_\w+)\s*\(", line))
    names.discard("osann_alloc_fn")
    names.discard("osann_free_fn")
    return names


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("osann_build", "osann_search", "osann_free", "osann_search_excl", "osann_bruteforce",
                 "osann_probes", "osann_keys", "osann_export"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding covers exactly the declared entry points
    assert set(_lib.SIGNATURES) == names


def test_host_only_entry_points(L):
    out = ctypes.c_int64()
    assert L.osann_num_cones(3, 2, ctypes.byref(out)) == 0 and out.value == 12
    assert L.osann_num_cones(16, 4, ctypes.byref(out)) == 0 and out.value == 29120
    assert L.osann_num_cones(128, 3, ctypes.byref(out)) == 0 and out.value == 2731008
    assert L.osann_num_cones(3, 4, ctypes.byref(out)) == -1          # L > d
    assert L.osann_num_cones(64, 16, ctypes.byref(out)) == -2        # N_C >= 2^31
    h = ctypes.c_void_p()
    assert L.osann_build(None, 10, 4, 2, None, ctypes.byref(h)) == -1
    assert b"invalid" in L.osann_last_error()
    assert L.osann_search(None, None, 1, 1, 1, 0, None, 0, None, None, None) == -1
    assert L.osann_free(None) == 0
    assert L.osann_search_workspace_size(None, 1, 1, 1, 0) == 0
    assert L.osann_stats_get(99, None, None) == -1
    assert L.osann_launch_count() >= 0


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(build, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        _lib.load()


def test_host_only_argument_checks_of_the_newer_entry_points(L):
    h = ctypes.c_void_p()
    c = ctypes
    # build with options: no data
    assert L.osann_build_ex(None, 10, 4, 2, None, None, c.byref(h)) == -1
    # build and search in one call: no output handle / no data
    assert L.osann_build_search(None, 10, 4, 2, None, None, 1, 1, 1, 0, None, 0, None, None, None, None) == -1
    assert L.osann_build_search(None, 10, 4, 2, None, None, 1, 1, 1, 0, None, 0, None, None, None, c.byref(h)) == -1
    # in-place rebuild and rebuild-and-search: no index
    assert L.osann_rebuild(None, None, None) == -1
    assert L.osann_rebuild_search(None, None, None, 1, 1, 1, 0, None, 0, None, None, None) == -1
    # ROSANNA+ search, cone table queries: no index
    assert L.osann_search_clusters(None, None, 1, 2, 1, 1, 0, None, 0, None, None, None) == -1
    assert L.osann_search_clusters_workspace_size(None, 1, 2, 1, 1, 0) == 0
    assert L.osann_cones(None, None, None, None, None, None) == -1
    assert L.osann_export_cones(None, None, None) == -1
    # 128-bit keys: bad sizes are rejected before any device work
    assert L.osann_keys_wide(None, 1, 0, 2, None, None) == -1
    assert L.osann_keys_wide(None, 1, 300, 2, None, None) == -1


def test_host_only_checks_of_the_layout_knob(L):
    c = ctypes
    # no index, or a layout outside OSANN_LAYOUT_DEFAULT..OSANN_LAYOUT_TMEM: refused on the host
    assert L.osann_search_layout(None, None, 1, 1, 1, 0, 0, 0, None, 0, None, None, None) == -1
    assert L.osann_search_layout(None, None, 1, 1, 1, 0, 0, 3, None, 0, None, None, None) == -1
    # the header's layout constants are the binding's
    text = open(HEADER).read()
    for name, v in (("OSANN_LAYOUT_DEFAULT", 0), ("OSANN_LAYOUT_SMEM", 1), ("OSANN_LAYOUT_TMEM", 2)):
        assert re.search(r"#define\s+%s\s+%d\b" % (name, v), text)
    assert _lib.LAYOUTS == {"default": 0, "smem": 1, "tmem": 2}
    # the tuner's choices of no server: none
    out = (c.c_int32 * 3)()
    assert L.osann_server_choices(None, out, 1) == 0
