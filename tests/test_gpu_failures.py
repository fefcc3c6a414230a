"""Failure detection without a GPU fault.

* A bounded wait that runs out: the plain scan's waits for its staged copies
  get a budget of a few clock cycles through osann_debug_wait_budget, so
  they give up; the kernel lets its copies land, the search reports
  OSANN_STATUS_TIMEOUT through osann_status, its outputs stay in range, and
  with the default budget restored the same index searches correctly again
  (the context is still usable).
* Device allocation failures injected on the host: an allocator installed
  through osann_set_allocator fails the n-th request.  Every build, rebuild
  and search that meets the failure returns OSANN_ERR_OOM and gives back
  every block it took (nothing leaks), and the library works once the
  allocator is restored.
"""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import assert_knn_match, to_dev, to_np

pytestmark = pytest.mark.gpu

OOM = -3
STATUS_TIMEOUT = 4
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


@pytest.fixture(scope="module")
def osann():
    import paper_1509_03453_gb300 as m
    from paper_1509_03453_gb300 import build
    build.build()
    m.load()
    yield m


def _data(N=60_000, Q=300, d=32, seed=31):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, d)).astype(np.float32), rng.standard_normal((Q, d)).astype(np.float32)


def test_plain_scan_wait_runs_out_and_reports_timeout(osann):
    from paper_1509_03453_gb300 import _lib
    L = _lib.load()
    X, Y = _data()
    idx = osann.Index(to_dev(X), 2)
    Yd = to_dev(Y)
    assert idx.status() == 0
    assert L.osann_debug_wait_budget(-1) == -1
    assert L.osann_debug_wait_budget(2) == 0
    try:
        ids, d2 = idx.search(Yd, 64, 4, path="plain")
        flags = idx.status()
    finally:
        assert L.osann_debug_wait_budget(0) == 0
    assert flags & STATUS_TIMEOUT
    ids = to_np(ids)
    assert ((ids >= -1) & (ids < X.shape[0])).all()
    # the default budget again: the same index and context give the oracle's answer
    ids, d2 = idx.search(Yd, 64, 4, path="plain")
    assert idx.status() == 0
    oids, od = oracle.Index(X, 2).search(Y, 64, 4)
    assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
    idx.close()


class _FailingAllocator:
    """Serves requests from torch's caching allocator and fails request
    number `fail_at` (1-based; 0: never).  Tracks live blocks."""

    def __init__(self, lib, fail_at=0):
        import torch
        self.torch = torch
        self.lib = lib
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(nbytes)
        self.live[p] = nbytes
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        # stream-ordered release: let the work that used the block finish first
        self.torch.cuda.synchronize()
        assert self.live.pop(ptr) == nbytes
        self.torch.cuda.caching_allocator_delete(ptr)

    def __enter__(self):
        assert self.lib.osann_set_allocator(ctypes.cast(self.alloc_cb, ctypes.c_void_p),
                                            ctypes.cast(self.free_cb, ctypes.c_void_p), None) == 0
        return self

    def __exit__(self, *exc):
        assert self.lib.osann_set_allocator(None, None, None) == 0


def _search_lib_ws(L, idx, Yd, P, k, path):
    """osann_search with no caller workspace: the library allocates it."""
    import torch

    from paper_1509_03453_gb300 import PATHS
    Q = Yd.shape[0]
    ids = torch.empty((Q, k), dtype=torch.int64, device=Yd.device)
    d2 = torch.empty((Q, k), dtype=torch.float32, device=Yd.device)
    rc = L.osann_search(idx._h, ctypes.c_void_p(Yd.data_ptr()), Q, P, k, PATHS[path], None, 0,
                        ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, ids, d2


def test_allocation_failures_return_oom_without_leaks(osann):
    import torch
    from paper_1509_03453_gb300 import OsannError, _lib
    L = _lib.load()
    X, Y = _data(N=30_000, Q=200)
    Xd, Yd = to_dev(X), to_dev(Y)
    torch.cuda.synchronize()

    # how many requests a build, a first rebuild and a search make
    with _FailingAllocator(L) as a:
        idx = osann.Index(Xd, 2)
        n_build = a.calls
        idx.rebuild(Xd)
        idx.status()
        n_rebuild = a.calls - n_build
        assert _search_lib_ws(L, idx, Yd, 32, 4, "fp16")[0] == 0
        torch.cuda.synchronize()
        n_search = a.calls - n_build - n_rebuild
        idx.close()
        torch.cuda.synchronize()
        assert a.live == {}
    assert n_build >= 3 and n_rebuild >= 1 and n_search >= 1

    # every build request failing in turn: OOM, nothing left behind
    for n in range(1, n_build + 1):
        with _FailingAllocator(L, fail_at=n) as a:
            with pytest.raises(OsannError) as e:
                osann.Index(Xd, 2)
            assert e.value.code == OOM
            torch.cuda.synchronize()
            assert a.live == {}, f"build failing at request {n} leaked {len(a.live)} blocks"

    ref = oracle.Index(X, 2)
    oids, od = ref.search(Y, 32, 4)
    for n in range(1, n_rebuild + 1):
        idx = osann.Index(Xd, 2)
        with _FailingAllocator(L, fail_at=n) as a:
            with pytest.raises(OsannError) as e:
                idx.rebuild(Xd)
            assert e.value.code == OOM
            torch.cuda.synchronize()
            assert a.live == {}
        # the index is intact after the failed rebuild
        ids, d2 = idx.search(Yd, 32, 4, path="plain")
        assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
        idx.close()

    idx = osann.Index(Xd, 2)
    for n in range(1, n_search + 1):
        with _FailingAllocator(L, fail_at=n) as a:
            assert _search_lib_ws(L, idx, Yd, 32, 4, "fp16")[0] == OOM
            torch.cuda.synchronize()
            assert a.live == {}
    # the default allocator again: everything works
    rc, ids, d2 = _search_lib_ws(L, idx, Yd, 32, 4, "fp16")
    assert rc == 0
    assert idx.status() == 0
    assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
    idx.close()


def test_misaligned_workspace_is_refused_before_any_launch(osann):
    """A caller workspace must be 256-byte aligned (the vector loads and
    16-byte asynchronous copies that read it): a misaligned one is refused
    with OSANN_ERR_INVALID, nothing runs, and an aligned one works."""
    import torch
    from paper_1509_03453_gb300 import OsannError
    X, Y = _data(N=20_000, Q=100)
    Xd, Yd = to_dev(X), to_dev(Y)
    idx = osann.Index(Xd, 2)
    for path in ("plain", "batched", "fp16"):
        need = idx.workspace_size(100, 32, 4, path)
        raw = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
        base = (-raw.data_ptr()) % 256
        with pytest.raises(OsannError) as e:
            idx.search(Yd, 32, 4, path=path, workspace=raw[base + 16:base + 16 + need])
        assert e.value.code == -1
        ids, d2 = idx.search(Yd, 32, 4, path=path, workspace=raw[base:base + need])
        ref = oracle.Index(X, 2)
        oids, od = ref.search(Y, 32, 4)
        assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
    assert idx.status() == 0
    idx.close()
