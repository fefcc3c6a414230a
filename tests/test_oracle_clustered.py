"""Oracle pins for ROSANNA+ (Sec. 4-B: k-means clusters, each searched with
the cone hash of its residuals; a query visits its nearest clusters).

The nearest centroid is the plain definition (fp64 squared distance, ties to
the lower index), pinned to a numpy fp64 ranking, to exact ties on a bisecting
hyperplane and to a difference below fp32 resolution; a given assignment and
given query clusters are followed; one centroid at the origin reduces the
method to the one-basis search, bit for bit; the search equals the exact
top-k (numpy fp64) over the points of the selected clusters whose residual
cone is in the residual's probed list; all clusters at the full budget is
linear search."""
import numpy as np
import pytest

import oracle
from paper_1509_03453_gb300.kmeans import kmeans


def _fp64_sqdists(X, C):
    return ((np.asarray(X, np.float64)[:, None, :] - np.asarray(C, np.float64)[None]) ** 2).sum(-1)


def test_nearest_centroids_are_the_fp64_ranking():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((500, 24)).astype(np.float32)
    C = rng.standard_normal((40, 24)).astype(np.float32)
    C[7] = C[3]  # duplicate centroid: the lower index first
    near = oracle.nearest_centroids(X, C, 5)
    D = _fp64_sqdists(X, C)
    for i in range(X.shape[0]):
        exp = np.lexsort((np.arange(40), D[i]))[:5]
        got = near[i]
        # numpy sums in another order: identical up to a last-bit near-tie
        same = got == exp
        assert np.all(same | (np.abs(D[i, got] - D[i, exp]) <= 1e-12 * D[i, exp]))
        assert len(set(got.tolist())) == 5
        if 3 in got and 7 in got:
            assert list(got).index(3) < list(got).index(7)
    # M > K pads with -1
    assert (oracle.nearest_centroids(X[:3], C[:2], 4)[:, 2:] == -1).all()


@pytest.mark.parametrize("d", [2, 16, 33])
def test_nearest_centroid_exact_ties_go_to_the_lower_index(d):
    # x on the bisecting hyperplane of two centroids mirrored through it: the
    # fp64 distances are equal exactly, so the lower index wins whatever the
    # order the centroids are listed in
    rng = np.random.default_rng(40 + d)
    c = np.zeros(d, np.float32)
    c[0] = 1.5
    X = rng.integers(-8, 9, size=(20, d)).astype(np.float32)
    X[:, 0] = 0.0
    far = np.full((3, d), 50.0, np.float32)
    for order in ([0, 1], [1, 0]):
        C = np.concatenate([far, np.stack([c, -c])[order]])
        near = oracle.nearest_centroids(X, C, 2)
        assert (near == [[3, 4]]).all()
    # one step off the hyperplane decides it
    X[:, 0] = 0.25
    C = np.concatenate([far, np.stack([-c, c])])
    assert (oracle.nearest_centroids(X, C, 1)[:, 0] == 4).all()


def test_nearest_centroid_is_not_an_fp32_decision():
    # two centroids whose fp64 distances differ by far less than an fp32 ulp
    # of the distance: fp64 decides it (an fp32 evaluation would call it a tie)
    x = np.zeros((1, 4), np.float32)
    c0 = np.array([4096.0, 0.0, 0.0, 0.0], np.float32)
    c1 = np.array([4096.0, 2.0 ** -12, 0.0, 0.0], np.float32)
    assert np.float32(4096.0) ** 2 == np.float32(4096.0) ** 2 + np.float32(2.0 ** -24)
    assert oracle.nearest_centroids(x, np.stack([c1, c0]), 1)[0, 0] == 1


def test_given_assignment_and_query_clusters_are_followed():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((2000, 16)).astype(np.float32)
    Y = rng.standard_normal((30, 16)).astype(np.float32)
    C = kmeans(X, 6, iters=4, seed=2)
    ci = oracle.ClusteredIndex(X, 2, C)
    same = oracle.ClusteredIndex(X, 2, C, asg=ci.asg)
    assert same.keys == ci.keys and np.array_equal(same.perm, ci.perm)
    # another assignment: each point keyed by its residual on the given cluster
    alt = (ci.asg + 1) % 6
    ca = oracle.ClusteredIndex(X, 2, C, asg=alt)
    assert np.array_equal(ca.asg, alt)
    nc = oracle.num_cones_wide(16, 2)
    rk = oracle.keys_wide(X - C[alt], 2)
    assert ca.keys == [int(a) * nc + r for a, r in zip(alt, rk)]
    with pytest.raises(ValueError):
        oracle.ClusteredIndex(X, 2, C, asg=np.full(2000, 6))
    # the query's own nearest clusters given explicitly: the default search
    near = oracle.nearest_centroids(Y, C, 3)
    a = ci.search(Y, 3, 8, 2)
    b = ci.search(Y, 3, 8, 2, near=near)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # other clusters given: the search over those
    other = near[:, ::-1].copy()
    other[:, 0] = -1  # skipped
    ids, dd, cnt = ci.search(Y, 3, 8, 2, near=other, want_counts=True)
    ref_ids, _, ref_cnt = ci.search(Y, 2, 8, 2, near=near[:, :2][:, ::-1].copy(), want_counts=True)
    assert np.array_equal(cnt, ref_cnt) and np.array_equal(ids, ref_ids)


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
