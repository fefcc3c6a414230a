"""Parity at the full workload sizes, in the bench's launch configuration.

For the scale-up Gaussian case (the bench workload: N = 10^6, d = 32,
Q = 10^4, L = 2, P = 224, path auto = fp16 screening) the whole query batch
runs on the GPU as the bench runs it; the oracle then computes a sample of
the queries one by one at full N, and the keys, offsets and permutation are
compared in full.  The patch workload (about 10^6 mean-removed 8x8 patches,
L = 3, exclusion radius 8, k = 4) and the descriptor workload (N = 2*10^6,
d = 128, L = 3, k = 10) are checked the same way on query samples.
"""
import numpy as np
import pytest

import oracle
from helpers import assert_knn_match, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osann():
    import paper_1509_03453_gb300 as m
    from paper_1509_03453_gb300 import build
    build.build()
    m.load()
    yield m


def _sample(Q, n, seed):
    return np.sort(np.random.default_rng(seed).choice(Q, size=n, replace=False))


def test_gauss32_full_size_bench_configuration(osann):
    from paper_1509_03453_gb300 import datagen
    w = datagen.workload("gauss32")
    X, Y = w["X"], w["Y"]
    idx = osann.Index(to_dev(X), 2)
    ids, d2 = idx.search(to_dev(Y), 224, 1)  # the bench's call: path auto
    ids, d2 = to_np(ids), to_np(d2)
    o = oracle.Index(X, 2)
    keys, offs, perm = (to_np(t) for t in idx.export())
    assert np.array_equal(keys, o.keys)
    assert np.array_equal(offs, o.offsets)
    assert np.array_equal(perm, o.perm)
    s = _sample(Y.shape[0], 300, 1)
    oids, od = o.search(Y[s], 224, 1)
    assert_knn_match(X, Y[s], ids[s], d2[s], oids, od)
    # the same batch through the other paths: the same bits
    for path in ("plain", "batched"):
        pi, pd = idx.search(to_dev(Y), 224, 1, path=path)
        assert np.array_equal(to_np(pi), ids)
        assert np.array_equal(to_np(pd).view(np.uint32), d2.view(np.uint32))
    st = idx.screen_stats()
    assert st["bound_violations"] == 0
    idx.close()


def test_patch64_full_size_sampled(osann):
    import torch
    from paper_1509_03453_gb300 import datagen
    w = datagen.workload("patch64")
    X, Y, src = w["X"], w["Y"], w["query_src"]
    idx = osann.Index(to_dev(X), 3)
    kw = dict(query_src=torch.from_numpy(src).cuda(), grid_w=w["grid_w"], radius=w["radius"])
    ids, d2 = idx.search(to_dev(Y), 64, 4, **kw)
    ids, d2 = to_np(ids), to_np(d2)
    o = oracle.Index(X, 3)
    s = _sample(Y.shape[0], 200, 2)
    oids, od = o.search(Y[s], 64, 4, query_src=src[s], grid_w=w["grid_w"], radius=w["radius"])
    assert_knn_match(X, Y[s], ids[s], d2[s], oids, od)
    idx.close()


def test_desc128_full_size_sampled(osann):
    from paper_1509_03453_gb300 import datagen
    w = datagen.workload("desc128")
    X, Y = w["X"], w["Y"]
    idx = osann.Index(to_dev(X), 3)
    for path in ("auto", "fp16"):
        ids, d2 = idx.search(to_dev(Y), 128, 10, path=path)
        ids, d2 = to_np(ids), to_np(d2)
        if path == "auto":
            o = oracle.Index(X, 3)
            s = _sample(Y.shape[0], 200, 3)
            oids, od = o.search(Y[s], 128, 10)
            assert_knn_match(X, Y[s], ids[s], d2[s], oids, od)
            ref = (ids, d2)
        else:
            assert np.array_equal(ids, ref[0])
            assert np.array_equal(d2.view(np.uint32), ref[1].view(np.uint32))
    idx.close()
