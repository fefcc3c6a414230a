"""Oracle pins for ROSANNA+ (Sec. 4-B: k-means clusters, each searched with
the cone hash of its residuals; a query visits its nearest clusters).

The fp32 distance that decides the nearest centroid is pinned to exact
integer arithmetic and to its rounding bound; the nearest centroids to a
numpy fp64 ranking (up to near-ties); one centroid at the origin reduces the
method to the one-basis search, bit for bit; the search equals the exact
top-k (numpy fp64) over the points of the selected clusters whose residual
cone is in the residual's probed list; all clusters at the full budget is
linear search."""
import numpy as np
import pytest

import oracle
from paper_1509_03453_gb300.kmeans import kmeans


def _d_pad(d):
    p = 16
    while p < d:
        p *= 2
    return p


@pytest.mark.parametrize("d", [3, 16, 30, 64, 128])
def test_sqdist_f32_exact_on_small_integers(d):
    rng = np.random.default_rng(d)
    for _ in range(20):
        x = rng.integers(-40, 41, size=d).astype(np.float32)
        y = rng.integers(-40, 41, size=d).astype(np.float32)
        assert oracle.sqdist_f32(x, y) == float(((x.astype(np.int64) - y.astype(np.int64)) ** 2).sum())


@pytest.mark.parametrize("d", [5, 32, 100, 256])
def test_sqdist_f32_within_rounding_bound(d):
    rng = np.random.default_rng(10 + d)
    bound = (5 + np.log2(_d_pad(d) / 4)) * 2.0 ** -24
    worst = 0.0
    for _ in range(200):
        x = rng.standard_normal(d).astype(np.float32)
        y = rng.standard_normal(d).astype(np.float32)
        ref = ((x.astype(np.float64) - y.astype(np.float64)) ** 2).sum()
        worst = max(worst, abs(oracle.sqdist_f32(x, y) - ref) / ref)
    assert worst <= bound
    assert worst > 0  # it is an fp32 evaluation, not the fp64 one


def test_nearest_centroids_match_fp64_ranking():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((500, 24)).astype(np.float32)
    C = rng.standard_normal((40, 24)).astype(np.float32)
    C[7] = C[3]  # duplicate centroid: the lower index first
    near = oracle.nearest_centroids(X, C, 5)
    D = ((X.astype(np.float64)[:, None, :] - C.astype(np.float64)[None]) ** 2).sum(-1)
    for i in range(X.shape[0]):
        exp = np.lexsort((np.arange(40), D[i]))[:5]
        got = near[i]
        assert np.allclose(D[i, got], D[i, exp], rtol=1e-6, atol=0)
        assert len(set(got.tolist())) == 5
        if 3 in got and 7 in got:
            assert list(got).index(3) < list(got).index(7)
    # M > K pads with -1
    assert (oracle.nearest_centroids(X[:3], C[:2], 4)[:, 2:] == -1).all()


def test_one_centroid_at_origin_is_the_one_basis_search():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((3000, 16)).astype(np.float32)
    Y = rng.standard_normal((60, 16)).astype(np.float32)
    ci = oracle.ClusteredIndex(X, 2, np.zeros((1, 16), np.float32))
    o = oracle.Index(X, 2)
    assert np.array_equal(ci.perm, o.perm)
    assert ci.keys == [int(v) for v in o.keys]
    a = ci.search(Y, 1, 9, 3)
    b = o.search(Y, 9, 3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("K,M,P,k", [(8, 1, 6, 1), (16, 3, 10, 4), (5, 5, 3, 2)])
def test_clustered_search_is_exact_topk_over_selected_cones(K, M, P, k):
    d, L = 16, 2
    rng = np.random.default_rng(20 + K)
    # clustered data: K0 blobs
    centers = 4.0 * rng.standard_normal((12, d))
    X = (centers[rng.integers(12, size=4000)] + rng.standard_normal((4000, d))).astype(np.float32)
    Y = (centers[rng.integers(12, size=40)] + rng.standard_normal((40, d))).astype(np.float32)
    C = kmeans(X, K, iters=8, seed=K)
    ci = oracle.ClusteredIndex(X, L, C)
    assert np.array_equal(ci.asg, oracle.nearest_centroids(X, C, 1)[:, 0])
    ids, dd, cnt = ci.search(Y, M, P, k, want_counts=True)
    # residual cone of every point, on its own cluster
    rk = oracle.keys_wide(X - C[ci.asg], L)
    X64 = X.astype(np.float64)
    for q in range(Y.shape[0]):
        near = oracle.nearest_centroids(Y[q], C, M)[0]
        cand = []
        for c in near:
            pset = set(oracle.probes_wide(Y[q] - C[c], L, P))
            cand += [n for n in np.flatnonzero(ci.asg == c) if rk[n] in pset]
        cand = np.array(sorted(cand), np.int64)
        assert cnt[q] == cand.size
        dist = ((X64[cand] - Y[q].astype(np.float64)) ** 2).sum(1) if cand.size else np.zeros(0)
        o = np.lexsort((cand, dist))[:k]
        exp = np.full(k, -1, np.int64)
        exp[:o.size] = cand[o]
        assert np.array_equal(ids[q], exp)
        assert np.allclose(dd[q][:o.size], dist[o], rtol=1e-12, atol=0)


def test_all_clusters_full_budget_is_linear_search():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((1500, 8)).astype(np.float32)
    Y = rng.standard_normal((30, 8)).astype(np.float32)
    C = kmeans(X, 6, iters=5, seed=1)
    ci = oracle.ClusteredIndex(X, 2, C)
    a = ci.search(Y, 6, oracle.num_cones(8, 2), 3)
    b = oracle.bruteforce(X, Y, 3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_kmeans_is_seeded_and_reduces_distortion():
    rng = np.random.default_rng(6)
    X = (np.repeat(8.0 * rng.standard_normal((5, 10)), 200, axis=0) + rng.standard_normal((1000, 10))).astype(np.float32)
    a = kmeans(X, 5, seed=3)
    assert np.array_equal(a, kmeans(X, 5, seed=3))
    D = ((X[:, None, :].astype(np.float64) - a[None].astype(np.float64)) ** 2).sum(-1).min(1).mean()
    D0 = ((X - X.mean(0)) ** 2).sum(1).mean()
    assert D < 0.2 * D0
