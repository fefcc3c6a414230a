"""GPU parity of ROSANNA+ (Sec. 4-B): k-means clusters searched with the cone
hash of their residuals, a query visiting its M nearest clusters.

Against the oracle's clustered index: point order, offsets of the occupied
composite cones, each point's cluster (the nearest-centroid decision,
duplicate centroids included), and the search on every path (the same bits
on all of them); a composite table beyond 2^31 cones (second-level table);
one centroid at the origin against the plain index, bit for bit; all
clusters at the full budget against linear search.
"""
import numpy as np
import pytest

import oracle
from helpers import assert_knn_match, to_dev, to_np
from paper_1509_03453_gb300.kmeans import kmeans

pytestmark = pytest.mark.gpu

PATHS = ("plain", "batched", "fp16", "bf16")


@pytest.fixture(scope="module")
def osann():
    import paper_1509_03453_gb300 as m
    from paper_1509_03453_gb300 import build
    build.build()
    m.load()
    yield m


def _blobs(N, d, n_blobs, seed, spread=4.0):
    rng = np.random.default_rng(seed)
    centers = spread * rng.standard_normal((n_blobs, d))
    X = (centers[rng.integers(n_blobs, size=N)] + rng.standard_normal((N, d))).astype(np.float32)
    Y = (centers[rng.integers(n_blobs, size=200)] + rng.standard_normal((200, d))).astype(np.float32)
    return X, Y


def _check_table(idx, ci):
    keys, offs, perm = (to_np(t) for t in idx.export())
    assert np.array_equal(perm, ci.perm)
    if idx.hashed:
        n = ci.n_occ
        assert np.array_equal(offs[: n + 1], ci.offsets)
        assert idx.cone_ids()[:n] == ci.uniq
        ids = idx.cone_ids()
        assert [ids[c] for c in keys] == ci.keys
    else:
        uq = np.array(ci.uniq, np.int64)
        assert np.array_equal(offs[uq], ci.offsets[:-1])
        assert keys.tolist() == ci.keys
    assert idx.occupied() == ci.n_occ


@pytest.mark.parametrize("d,L,K", [(32, 2, 16), (30, 3, 24), (128, 2, 8), (16, 2, 64)])
def test_clustered_matches_oracle(osann, d, L, K):
    X, Y = _blobs(20000, d, 12, 700 + d)
    C = kmeans(X, K, iters=6, seed=K)
    C[K - 1] = C[1]  # a duplicate centroid: its points and queries go to index 1
    idx = osann.Index(to_dev(X), L, centroids=to_dev(C))
    ci = oracle.ClusteredIndex(X, L, C)
    assert idx.n_cones == K * oracle.num_cones_wide(d, L)
    _check_table(idx, ci)
    for M, P, k in ((1, 8, 1), (3, 24, 4)):
        oids, od = ci.search(Y, M, P, k)
        ref = None
        for path in PATHS:
            gi, gd = idx.search(to_dev(Y), P, k, path=path, clusters=M)
            gi, gd = to_np(gi), to_np(gd)
            assert_knn_match(X, Y, gi, gd, oids, od)
            if ref is None:
                ref = (gi, gd)
            else:
                assert np.array_equal(gi, ref[0]) and np.array_equal(gd.view(np.uint32), ref[1].view(np.uint32))
    assert idx.status() == 0
    idx.close()


def test_clustered_second_level_table(osann):
    d, L, K = 64, 4, 256  # K * N_C = 256 * 10,166,016 > 2^31
    X, Y = _blobs(30000, d, 40, 800)
    C = kmeans(X, K, iters=4, seed=2)
    idx = osann.Index(to_dev(X), L, centroids=to_dev(C))
    assert idx.hashed
    ci = oracle.ClusteredIndex(X, L, C)
    _check_table(idx, ci)
    oids, od = ci.search(Y, 4, 16, 3)
    for path in ("plain", "fp16"):
        gi, gd = idx.search(to_dev(Y), 16, 3, path=path, clusters=4)
        assert_knn_match(X, Y, to_np(gi), to_np(gd), oids, od)
    idx.close()


def test_one_centroid_at_origin_is_the_plain_index(osann):
    X, Y = _blobs(20000, 32, 1, 900, spread=0.0)
    a = osann.Index(to_dev(X), 2)
    b = osann.Index(to_dev(X), 2, centroids=to_dev(np.zeros((1, 32), np.float32)))
    for path in ("plain", "fp16"):
        ra = a.search(to_dev(Y), 40, 3, path=path)
        rb = b.search(to_dev(Y), 40, 3, path=path, clusters=5)  # clamped to K = 1
        assert np.array_equal(to_np(ra[0]), to_np(rb[0]))
        assert np.array_equal(to_np(ra[1]).view(np.uint32), to_np(rb[1]).view(np.uint32))
    a.close()
    b.close()


def test_all_clusters_full_budget_is_linear_search(osann):
    X, Y = _blobs(5000, 8, 6, 901)
    C = kmeans(X, 6, iters=4, seed=3)
    idx = osann.Index(to_dev(X), 2, centroids=to_dev(C))
    gi, gd = idx.search(to_dev(Y[:50]), oracle.num_cones(8, 2), 3, path="plain", clusters=6)
    ri, rd = idx.bruteforce(to_dev(Y[:50]), 3)
    assert np.array_equal(to_np(gi), to_np(ri))
    assert np.array_equal(to_np(gd).view(np.uint32), to_np(rd).view(np.uint32))
    idx.close()
