"""Oracle pins for the multi-basis search (Sec. 3-D, Algorithm 1 with R bases).

The rotated coordinates are checked against exact signed permutations and
against an fp64 matrix product; the R-basis search against its definition:
the exact top-k over the union of the bases' probed cones, computed here with
numpy from the per-basis probe lists and buckets."""
import numpy as np
import pytest

import oracle
from paper_1509_03453_gb300 import datagen


def _signed_perm(d, seed):
    rng = np.random.default_rng(seed)
    p = rng.permutation(d)
    while np.all(p[p] == np.arange(d)):  # not an involution, so a transpose shows
        p = rng.permutation(d)
    s = rng.choice([-1.0, 1.0], size=d)
    M = np.zeros((d, d), np.float32)
    M[np.arange(d), p] = s
    return M, p, s


def test_rotate_signed_permutation_is_exact():
    X = np.random.default_rng(3).standard_normal((400, 12)).astype(np.float32)
    M, p, s = _signed_perm(12, 5)
    Xr = oracle.rotate(M, X)
    assert np.array_equal(Xr, (X[:, p] * s).astype(np.float32))
    # keys on the new basis are the keys of the permuted, sign-flipped rows
    assert np.array_equal(oracle.keys(Xr, 3), oracle.keys((X[:, p] * s).astype(np.float32), 3))


def test_rotate_matches_fp64_product_and_not_its_transpose():
    d = 16
    Rm = datagen.rotations(2, d, 9)[1]
    assert np.allclose(Rm.astype(np.float64) @ Rm.T.astype(np.float64), np.eye(d), atol=1e-5)
    X = np.random.default_rng(4).standard_normal((300, d)).astype(np.float32)
    got = oracle.rotate(Rm, X).astype(np.float64)
    ref = X.astype(np.float64) @ Rm.astype(np.float64).T
    bound = d * 2.0 ** -23 * (np.abs(X) @ np.abs(Rm).T)
    assert np.all(np.abs(got - ref) <= bound)
    wrong = X.astype(np.float64) @ Rm.astype(np.float64)
    assert np.max(np.abs(got - wrong)) > 0.1


def test_one_identity_basis_is_the_single_basis_search():
    X = np.random.default_rng(6).standard_normal((3000, 16)).astype(np.float32)
    Y = np.random.default_rng(7).standard_normal((80, 16)).astype(np.float32)
    mi = oracle.MultiIndex(X, 2, datagen.rotations(1, 16, 0))
    a_ids, a_d = mi.search(Y, 12, 3)
    b_ids, b_d = oracle.Index(X, 2).search(Y, 12, 3)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_d, b_d)


@pytest.mark.parametrize("R,P,k", [(2, 4, 1), (3, 10, 5), (4, 2, 3)])
def test_multibasis_is_exact_topk_over_union(R, P, k):
    d, L = 12, 2
    X = np.random.default_rng(10 + R).standard_normal((2500, d)).astype(np.float32)
    Y = np.random.default_rng(20 + R).standard_normal((40, d)).astype(np.float32)
    rots = datagen.rotations(R, d, 30 + R)
    mi = oracle.MultiIndex(X, L, rots)
    ids, dist, cnt = mi.search(Y, P, k, want_counts=True)
    for q in range(Y.shape[0]):
        union = set()
        for r in range(R):
            yr = oracle.rotate(rots[r], Y[q:q + 1])[0]
            for c in oracle.probes(yr, L, P):
                o, pm = mi.offsets[r], mi.perms[r]
                union.update(int(v) for v in pm[o[c]:o[c + 1]])
        u = np.array(sorted(union), np.int64)
        assert cnt[q] == len(u)
        dd = ((X[u].astype(np.float64) - Y[q].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((u, dd))[:k]
        assert np.array_equal(ids[q, :len(order)], u[order])
        assert np.allclose(dist[q, :len(order)], dd[order], rtol=1e-12, atol=0)  # fp64 summation order


def test_full_budget_on_any_basis_is_linear_search():
    d, L = 8, 2
    X = np.random.default_rng(40).standard_normal((1500, d)).astype(np.float32)
    Y = np.random.default_rng(41).standard_normal((30, d)).astype(np.float32)
    mi = oracle.MultiIndex(X, L, datagen.rotations(3, d, 42))
    ids, dist = mi.search(Y, oracle.num_cones(d, L), 2)
    bi, bd = oracle.bruteforce(X, Y, 2)
    assert np.array_equal(ids, bi) and np.array_equal(dist, bd)


def test_more_bases_never_lose_the_best_candidate():
    d, L, P = 16, 2, 6
    X = np.random.default_rng(50).standard_normal((4000, d)).astype(np.float32)
    Y = np.random.default_rng(51).standard_normal((60, d)).astype(np.float32)
    rots = datagen.rotations(4, d, 52)
    prev = None
    for R in (1, 2, 4):
        _, dist = oracle.MultiIndex(X, L, rots[:R]).search(Y, P, 1)
        if prev is not None:
            assert np.all(dist[:, 0] <= prev)
        prev = dist[:, 0]


def test_projection_selects_and_offsets_exactly():
    X = np.random.default_rng(60).standard_normal((300, 20)).astype(np.float32)
    m = 7
    Pm = np.eye(20, dtype=np.float32)[:m]
    off = np.random.default_rng(61).standard_normal(m).astype(np.float32)
    assert np.array_equal(oracle.project(Pm, X), X[:, :m])
    assert np.array_equal(oracle.project(Pm, X, off), (X[:, :m] - off).astype(np.float32))


def test_projected_multibasis_is_exact_topk_over_union():
    from paper_1509_03453_gb300.pca import pca_basis
    d, m, L, P, k = 24, 8, 2, 6, 3
    rng = np.random.default_rng(70)
    # correlated data: a few strong directions
    X = (rng.standard_normal((3000, d)) @ rng.standard_normal((d, d))).astype(np.float32)
    Y = (rng.standard_normal((30, d)) @ rng.standard_normal((d, d))).astype(np.float32)
    axes, off = pca_basis(X, m, seed=1)
    assert np.allclose(axes.astype(np.float64) @ axes.T.astype(np.float64), np.eye(m), atol=1e-5)
    mi = oracle.MultiIndex(X, L, axes[None], off[None])
    assert mi.NC == oracle.num_cones(m, L)
    ids, dist, cnt = mi.search(Y, P, k, want_counts=True)
    Xp = oracle.project(axes, X, off)
    keys = oracle.keys(Xp, L)
    for q in range(Y.shape[0]):
        yp = oracle.project(axes, Y[q:q + 1], off)[0]
        cones = set(int(c) for c in oracle.probes(yp, L, P))
        u = np.array([n for n in range(X.shape[0]) if int(keys[n]) in cones], np.int64)
        assert cnt[q] == len(u)
        dd = ((X[u].astype(np.float64) - Y[q].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((u, dd))[:k]
        assert np.array_equal(ids[q, :len(order)], u[order])


@pytest.mark.parametrize("d", [16, 32, 128])
def test_walsh_hadamard_bases(d):
    """The structured bases: basis 0 the identity; the others orthonormal,
    every entry +-1/sqrt(d), entry (i, j) = s_j (-1)^popcount(i & j) / sqrt(d)
    (checked against the Sylvester recursion H_2n = [[H, H], [H, -H]]), with
    signs that differ between bases; the oracle's rotated coordinates match
    an fp64 product within the fp32 in-order FMA bound."""
    B = datagen.hadamard_rotations(3, d, 17)
    assert np.array_equal(B[0], np.eye(d, dtype=np.float32))
    H = np.array([[1.0]])
    while H.shape[0] < d:
        H = np.block([[H, H], [H, -H]])
    inv = np.float32(1.0 / np.sqrt(d))
    for r in (1, 2):
        Rm = B[r].astype(np.float64)
        assert np.allclose(Rm @ Rm.T, np.eye(d), atol=1e-6)
        assert np.all(np.abs(np.abs(B[r]) - inv) == 0)
        s = np.sign(Rm[0])  # row 0 of H is all ones: it carries the signs
        assert np.array_equal(np.sign(Rm), H * s[None, :])
    assert not np.array_equal(np.sign(B[1][0]), np.sign(B[2][0]))
    X = np.random.default_rng(d).standard_normal((200, d)).astype(np.float32)
    got = oracle.rotate(B[1], X).astype(np.float64)
    ref = X.astype(np.float64) @ B[1].astype(np.float64).T
    assert np.all(np.abs(got - ref) <= d * 2.0 ** -23 * (np.abs(X) @ np.abs(B[1]).T.astype(np.float64)))
    with pytest.raises(ValueError):
        datagen.hadamard_rotations(2, 24, 0)
