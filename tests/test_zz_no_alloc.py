"""osann_search_noalloc, the search entry point that allocates nothing, for
callers that cannot allocate device memory at query time (a plugin inside a
process that owns the allocator, a latency-critical thread that must not
take allocator locks, a program that reserved all device memory up front).

Called through the C ABI on two calls in a row (the shared scratch array
keeps the previous call's contents, which must not leak into the next
result) and checked three ways: against the CPU oracle under the suite's
tolerance, against osann_search on the plain path bit for bit, and, with a
counting allocator installed through osann_set_allocator, that the library
asked for no memory while it ran.  This file sorts last so that a run
stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import assert_knn_match, to_dev, to_np

pytestmark = pytest.mark.gpu

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def _noalloc(L, idx, Yd, Q, P, k, ids, d2, stream):
    return L.osann_search_noalloc(idx._h, ctypes.c_void_p(Yd.data_ptr()), Q, P, k,
                                  ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()), stream)


def test_noalloc_search_matches_oracle_twice_without_allocating():
    import torch

    import oracle
    import paper_1509_03453_gb300 as osann
    from paper_1509_03453_gb300 import _lib, build
    build.build()
    L = _lib.load()
    rng = np.random.default_rng(77)
    X = rng.standard_normal((50_021, 32)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2)
    ref = oracle.Index(X, 2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(1_000, 64, 4), (777, 33, 1)]
    inputs = []
    for Q, P, k in cases:
        Y = rng.standard_normal((Q, 32)).astype(np.float32)
        inputs.append((Y, to_dev(Y), torch.full((Q, k), -7, dtype=torch.int64, device="cuda"),
                       torch.full((Q, k), -7.0, dtype=torch.float32, device="cuda")))
    torch.cuda.synchronize()

    # every allocation or release the library asks for while the counting
    # allocator is installed is recorded (and served by torch, so that a
    # failure of this test still leaves a working process)
    calls = []

    def alloc(nbytes, st, ctx):
        calls.append(("alloc", nbytes))
        return torch.cuda.caching_allocator_alloc(nbytes)

    def free(ptr, nbytes, st, ctx):
        calls.append(("free", nbytes))
        torch.cuda.caching_allocator_delete(ptr)

    alloc_cb, free_cb = ALLOC_FN(alloc), FREE_FN(free)
    assert L.osann_set_allocator(ctypes.cast(alloc_cb, ctypes.c_void_p), ctypes.cast(free_cb, ctypes.c_void_p),
                                 None) == 0
    try:
        for (Q, P, k), (Y, Yd, ids, d2) in zip(cases, inputs):
            rc = _noalloc(L, idx, Yd, Q, P, k, ids, d2, stream)
            assert rc == 0, L.osann_last_error()
        torch.cuda.synchronize()
    finally:
        assert L.osann_set_allocator(None, None, None) == 0
    assert calls == [], f"osann_search_noalloc asked the allocator for memory: {calls[:5]}"

    for (Q, P, k), (Y, Yd, ids, d2) in zip(cases, inputs):
        # the oracle (fp64) under the suite's tolerance
        oids, od = ref.search(Y, P, k)
        assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
        # and the allocating plain search, bit for bit
        ref_ids, ref_d2 = idx.search(Yd, P, k, path="plain")
        assert np.array_equal(to_np(ids), to_np(ref_ids))
        assert np.array_equal(to_np(d2).view(np.int32), to_np(ref_d2).view(np.int32))

    # above the fixed scratch maximum: a clear error and the outputs untouched
    Qbig = 200_000
    Ybig = torch.zeros((Qbig, 32), dtype=torch.float32, device="cuda")
    ids = torch.full((Qbig, 1), -7, dtype=torch.int64, device="cuda")
    d2 = torch.full((Qbig, 1), -7.0, dtype=torch.float32, device="cuda")
    rc = _noalloc(L, idx, Ybig, Qbig, 64, 1, ids, d2, stream)
    assert rc == -1
    assert b"maximum" in L.osann_last_error()
    torch.cuda.synchronize()
    assert bool((ids == -7).all()) and bool((d2 == -7.0).all())
    idx.close()


@pytest.mark.skipif("__import__('torch').cuda.device_count() < 2")
def test_noalloc_rejects_another_current_device():
    import torch

    import paper_1509_03453_gb300 as osann
    from paper_1509_03453_gb300 import _lib
    L = _lib.load()
    X = np.random.default_rng(5).standard_normal((4096, 16)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2)
    Yd = to_dev(X[:8])
    ids = torch.full((8, 1), -7, dtype=torch.int64, device="cuda")
    d2 = torch.full((8, 1), -7.0, dtype=torch.float32, device="cuda")
    with torch.cuda.device(1):
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = _noalloc(L, idx, Yd, 8, 4, 1, ids, d2, stream)
    assert rc == -1 and b"device" in L.osann_last_error()
    idx.close()
