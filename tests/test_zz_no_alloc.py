"""osann_search_noalloc, the search entry point that allocates nothing, for
callers that cannot allocate device memory at query time (a plugin inside a
process that owns the allocator, a latency-critical thread that must not
take allocator locks, a program that reserved all device memory up front).

Called through the C ABI and compared with osann_search on the plain path,
on two calls in a row (the shared scratch array keeps the previous call's
contents, which must not leak into the next result).  This file sorts last
so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import assert_knn_match, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_noalloc_search_matches_search_twice():
    import torch

    import oracle
    import paper_1509_03453_gb300 as osann
    from paper_1509_03453_gb300 import _lib, build
    build.build()
    L = _lib.load()
    rng = np.random.default_rng(77)
    X = rng.standard_normal((50_021, 32)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (Q, P, k) in enumerate([(1_000, 64, 4), (777, 33, 1)]):
        Y = rng.standard_normal((Q, 32)).astype(np.float32)
        Yd = to_dev(Y)
        ids = torch.full((Q, k), -7, dtype=torch.int64, device="cuda")
        d2 = torch.full((Q, k), -7.0, dtype=torch.float32, device="cuda")
        rc = L.osann_search_noalloc(idx._h, ctypes.c_void_p(Yd.data_ptr()), Q, P, k,
                                    ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()), stream)
        assert rc == 0, L.osann_last_error()
        ref_ids, ref_d2 = idx.search(Yd, P, k, path="plain")
        # within the parity tolerance of the suite (and in fact bit-identical)
        ref_ids_np, ref_d2_np = to_np(ref_ids), to_np(ref_d2).astype(np.float64)
        assert_knn_match(X, Y, to_np(ids), to_np(d2), ref_ids_np, ref_d2_np)
        assert np.array_equal(to_np(ids), ref_ids_np)
        assert np.array_equal(to_np(d2), to_np(ref_d2))
    # above the fixed scratch maximum: a clear error, nothing written
    Qbig = 200_000
    Ybig = torch.zeros((Qbig, 32), dtype=torch.float32, device="cuda")
    ids = torch.empty((Qbig, 1), dtype=torch.int64, device="cuda")
    d2 = torch.empty((Qbig, 1), dtype=torch.float32, device="cuda")
    rc = L.osann_search_noalloc(idx._h, ctypes.c_void_p(Ybig.data_ptr()), Qbig, 64, 1,
                                ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()), stream)
    assert rc == -1
    assert b"maximum" in L.osann_last_error()
    del oracle
