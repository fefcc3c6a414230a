"""ctypes view of libosann.so (the C ABI in include/osann.h).

Argument marshalling only.  Loading fails loudly when the CUDA library has
not been built: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c = ctypes
_lib = None

OK = 0
ERRORS = {
    -1: "invalid argument",
    -2: "unsupported size",
    -3: "out of device memory",
    -4: "non-finite data",
    -5: "CUDA error",
    -6: "device wait timed out",
}
PATHS = {"auto": 0, "plain": 1, "batched": 2, "bf16": 3, "fp16": 4}
LAYOUTS = {"default": 0, "smem": 1, "tmem": 2}  # query tiles of the tensor-core screen
CONE_TABLES = {"auto": 0, "dense": 1, "hashed": 2}


class BuildOpts(c.Structure):
    """osann_build_opts."""
    _fields_ = [("d_basis", c.c_void_p), ("d_offset", c.c_void_p), ("m", c.c_int32), ("async_", c.c_int32),
                ("cone_table", c.c_int32), ("d_centroids", c.c_void_p), ("n_clusters", c.c_int32),
                ("key_mode", c.c_int32)]
KEY_MODES = {"set": 0, "ordered": 1}
STAGES = ["data_keys", "buckets", "gather", "query_order", "probes", "worklist", "tile_scan", "merge",
          "plain_scan", "bruteforce", "tc_prep", "tc_scan", "tc_rerank"]
STATUS_NONFINITE_DATA = 1
STATUS_NONFINITE_QUERY = 2
STATUS_TIMEOUT = 4
STATUS_BOUND = 16

# exported symbols and their signatures: (restype, argtypes)
SIGNATURES = {
    "osann_set_allocator": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_num_cones": (c.c_int, [c.c_int32, c.c_int32, c.POINTER(c.c_int64)]),
    "osann_keys": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_void_p]),
    "osann_query_order": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_build": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p,
                              c.POINTER(c.c_void_p)]),
    "osann_build_async": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p,
                                    c.POINTER(c.c_void_p)]),
    "osann_build_rot": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_int32,
                                  c.c_void_p, c.POINTER(c.c_void_p)]),
    "osann_build_proj": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_void_p,
                                   c.c_int32, c.c_int32, c.c_void_p, c.POINTER(c.c_void_p)]),
    "osann_build_ex": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_void_p,
                                 c.POINTER(c.c_void_p)]),
    "osann_cones": (c.c_int, [c.c_void_p, c.POINTER(c.c_int32), c.POINTER(c.c_uint64), c.POINTER(c.c_int64),
                              c.POINTER(c.c_int64), c.c_void_p]),
    "osann_export_cones": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_keys_wide": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_void_p]),
    "osann_search_clusters": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32,
                                        c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_search_clusters_workspace_size": (c.c_size_t, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32,
                                                          c.c_int32]),
    "osann_build_search": (c.c_int, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_void_p,
                                     c.c_int64, c.c_int32, c.c_int32, c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p,
                                     c.c_void_p, c.c_void_p, c.POINTER(c.c_void_p)]),
    "osann_rebuild": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_rebuild_search": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32,
                                       c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_free": (c.c_int, [c.c_void_p]),
    "osann_info": (c.c_int, [c.c_void_p, c.POINTER(c.c_int64), c.POINTER(c.c_int32), c.POINTER(c.c_int32),
                             c.POINTER(c.c_int64), c.POINTER(c.c_int64)]),
    "osann_export": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_probes": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_void_p, c.c_void_p,
                               c.c_size_t, c.c_void_p]),
    "osann_search_workspace_size": (c.c_size_t, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32]),
    "osann_search": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32, c.c_void_p,
                               c.c_size_t, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_search_excl": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32,
                                    c.c_int64, c.c_int32, c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p,
                                    c.c_void_p, c.c_void_p]),
    "osann_search_noalloc": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_void_p,
                                       c.c_void_p, c.c_void_p]),
    "osann_bruteforce_workspace_size": (c.c_size_t, [c.c_void_p, c.c_int64, c.c_int32]),
    "osann_bruteforce": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int64,
                                   c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_status": (c.c_int, [c.c_void_p, c.c_void_p, c.POINTER(c.c_uint32)]),
    "osann_screen_stats": (c.c_int, [c.c_void_p, c.c_void_p, c.POINTER(c.c_int64)]),
    "osann_last_error": (c.c_char_p, []),
    "osann_stats_enable": (c.c_int, [c.c_int]),
    "osann_stats_reset": (c.c_int, []),
    "osann_stats_get": (c.c_int, [c.c_int32, c.POINTER(c.c_double), c.POINTER(c.c_int64)]),
    "osann_launch_count": (c.c_int64, []),
    "osann_debug_wait_budget": (c.c_int, [c.c_int64]),
    "osann_search_group": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32,
                                     c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p, c.c_void_p, c.c_void_p]),
    "osann_search_workspace_size_group": (c.c_size_t, [c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32,
                                                       c.c_int32]),
    "osann_search_layout": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, c.c_int32, c.c_int32,
                                      c.c_int32, c.c_int32, c.c_void_p, c.c_size_t, c.c_void_p, c.c_void_p,
                                      c.c_void_p]),
    "osann_server_create": (c.c_int, [c.POINTER(c.c_void_p), c.c_int32, c.POINTER(c.c_int32),
                                      c.POINTER(c.c_int32), c.c_int32, c.c_int64, c.c_size_t, c.c_int32,
                                      c.POINTER(c.c_void_p)]),
    "osann_server_slots": (c.c_int, [c.c_void_p]),
    "osann_server_submit": (c.c_int, [c.c_void_p, c.c_int32, c.c_void_p, c.c_int64, c.c_void_p, c.c_void_p,
                                      c.POINTER(c.c_uint64)]),
    "osann_server_progress": (c.c_int, [c.c_void_p, c.c_int32, c.POINTER(c.c_uint64), c.c_int32,
                                        c.POINTER(c.c_int32)]),
    "osann_server_pending": (c.c_int, [c.c_void_p, c.POINTER(c.c_int64), c.POINTER(c.c_int32)]),
    "osann_server_tune": (c.c_int, [c.c_void_p, c.c_int32, c.POINTER(c.c_int32)]),
    "osann_server_tune_queries": (c.c_int, [c.c_void_p, c.POINTER(c.c_void_p), c.POINTER(c.c_int64), c.c_int32,
                                            c.POINTER(c.c_int32)]),
    "osann_server_buckets": (c.c_int, [c.c_void_p, c.POINTER(c.c_int64), c.c_int32]),
    "osann_server_choices": (c.c_int, [c.c_void_p, c.POINTER(c.c_int32), c.c_int32]),
    "osann_server_warmup": (c.c_int, [c.c_void_p]),
    "osann_server_free": (c.c_int, [c.c_void_p]),
    "osann_server_stats": (c.c_int, [c.c_void_p, c.POINTER(c.c_int64)]),
    "osann_merge_topk": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int32, c.c_int64, c.c_int32, c.c_void_p,
                                   c.c_void_p, c.c_void_p]),
}


class OsannError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB_PATH


def load():
    """Load libosann.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"libosann.so not found at {path}: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int):
    if rc != OK:
        msg = load().osann_last_error().decode(errors="replace")
        raise OsannError(rc, msg)
