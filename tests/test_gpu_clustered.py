"""GPU parity of ROSANNA+ (Sec. 4-B): k-means clusters searched with the cone
hash of their residuals, a query visiting its M nearest clusters.

Against the oracle's clustered index.  The oracle decides the nearest
centroid in fp64 (the plain definition); the kernels decide it in fp32, so a
point's cluster may differ only where the two fp64 distances lie within the
fp32 rounding window, and the test checks exactly that.  The point order and
the offsets of the occupied composite cones are then compared bit for bit
with the oracle's table built on the GPU's (checked) assignment, and the
search on every path (the same bits on all of them) with the oracle
searching the query's fp64-nearest clusters (any admissible set where the
M-th cluster is a near-tie); a composite table beyond 2^31 cones (second-level table);
one centroid at the origin against the plain index, bit for bit; all
clusters at the full budget against linear search.
"""
import itertools

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


def _window(d):
    """Relative error bound of the kernels' fp32 squared distance (all terms
    nonnegative; float4 pieces and a pairwise tree over d_pad / 4 of them):
    two centroids whose fp64 distances lie this close may be ordered either
    way by an fp32 evaluation."""
    dp = 16
    while dp < d:
        dp *= 2
    return (5 + np.log2(dp / 4)) * 2.0 ** -24


def _fp64_sqdists(X, C):
    return ((np.asarray(X, np.float64)[:, None, :] - np.asarray(C, np.float64)[None]) ** 2).sum(-1)


def _gpu_clusters(idx, d, L):
    """Cluster of every point as the GPU assigned it (from its composite ids)."""
    nc = oracle.num_cones_wide(d, L)
    keys = to_np(idx.export()[0]).astype(np.int64)
    if idx.hashed:
        ids = idx.cone_ids()
        return np.array([ids[c] // nc for c in keys], np.int64)
    return keys // nc


def _accepted_assignment(X, C, gpu_asg):
    """The GPU's assignment, checked against the fp64 nearest centroid: a
    point may sit in another cluster only when the two fp64 distances are
    within the fp32 rounding window (a near-tie a float decides); the
    assignment returned is the GPU's, for building the oracle's table."""
    o_asg = oracle.nearest_centroids(X, C, 1)[:, 0].astype(np.int64)
    diff = np.flatnonzero(gpu_asg != o_asg)
    if diff.size:
        D = _fp64_sqdists(X[diff], C)
        dg = D[np.arange(diff.size), gpu_asg[diff]]
        do = D[np.arange(diff.size), o_asg[diff]]
        eps = _window(X.shape[1])
        assert np.all(dg - do <= eps * (dg + do)), "a point's cluster differs beyond the fp32 window"
    return gpu_asg, diff.size


def _query_cluster_sets(Y, C, M):
    """Per query, every set of M clusters an fp32 ranking may select: the
    fp64 M nearest, plus alternatives where the M-th and the next ones are
    within the rounding window.  Bitwise-identical centroids have equal fp32
    distances too, and both sides take the lower index first, so a set holds
    a centroid's higher-index twin only together with the lower one."""
    D = _fp64_sqdists(Y, C)
    K = C.shape[0]
    M = min(M, K)
    eps = _window(Y.shape[1])
    out = []
    for q in range(Y.shape[0]):
        order = np.lexsort((np.arange(K), D[q]))
        base = [int(c) for c in order[:M]]
        edge = D[q, order[M - 1]]
        near = [int(c) for c in order if abs(D[q, c] - edge) <= eps * (D[q, c] + edge)]
        if M == K or all(c in base for c in near):
            out.append([np.array(base)])
            continue
        fixed = [c for c in base if c not in near]
        sets = []
        for comb in itertools.combinations(near, M - len(fixed)):
            ok = all(any(np.array_equal(C[c], C[u]) and u < c for u in comb) or
                     not any(np.array_equal(C[c], C[u]) and u < c for u in near) for c in comb)
            if ok:
                sets.append(np.array(fixed + list(comb)))
        out.append(sets)
    return out


def _check_search(X, Y, ci, sets, M, P, k, gi, gd):
    """GPU results against the oracle searching the query's fp64 M nearest
    clusters, or, for a query with a near-tie at the M-th cluster, any of
    the sets an fp32 ranking may select."""
    plain = np.array([len(s) == 1 for s in sets])
    near = np.stack([np.pad(s[0], (0, M - len(s[0])), constant_values=-1) for s in sets]).astype(np.int32)
    oids, od = ci.search(Y, M, P, k, near=near)
    if plain.all():
        assert_knn_match(X, Y, gi, gd, oids, od)
        return 0
    assert_knn_match(X, Y[plain], gi[plain], gd[plain], oids[plain], od[plain])
    for q in np.flatnonzero(~plain):
        ok = False
        for s in sets[q]:
            nq = np.pad(s, (0, M - len(s)), constant_values=-1).astype(np.int32)[None]
            a, b = ci.search(Y[q:q + 1], M, P, k, near=nq)
            try:
                assert_knn_match(X, Y[q:q + 1], gi[q:q + 1], gd[q:q + 1], a, b)
                ok = True
                break
            except AssertionError:
                pass
        assert ok, f"query {q}: no admissible cluster set reproduces the GPU result"
    return int((~plain).sum())


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
    assert idx.n_cones == K * oracle.num_cones_wide(d, L)
    asg, _ = _accepted_assignment(X, C, _gpu_clusters(idx, d, L))
    ci = oracle.ClusteredIndex(X, L, C, asg=asg)
    _check_table(idx, ci)
    # the duplicate centroid holds nothing (its twin has the lower index)
    assert not np.any(asg == K - 1)
    for M, P, k in ((1, 8, 1), (3, 24, 4)):
        sets = _query_cluster_sets(Y, C, M)
        ref = None
        for path in PATHS:
            gi, gd = idx.search(to_dev(Y), P, k, path=path, clusters=M)
            gi, gd = to_np(gi), to_np(gd)
            _check_search(X, Y, ci, sets, M, P, k, gi, gd)
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
    asg, _ = _accepted_assignment(X, C, _gpu_clusters(idx, d, L))
    ci = oracle.ClusteredIndex(X, L, C, asg=asg)
    _check_table(idx, ci)
    sets = _query_cluster_sets(Y, C, 4)
    for path in ("plain", "fp16"):
        gi, gd = idx.search(to_dev(Y), 16, 3, path=path, clusters=4)
        _check_search(X, Y, ci, sets, 4, 16, 3, to_np(gi), to_np(gd))
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
