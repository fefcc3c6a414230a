"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
worked example of the paper, a closed form, a textbook/library routine
(numpy argsort, bincount, lexsort, itertools) or an invariant.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig2_toy.txt")


def _fig2_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            t = line.split()
            x = np.array([float(v) for v in t[:3]], np.float32)
            rows.append((x, t[3], int(t[4]), t[5], int(t[6])))
    assert len(rows) == 16
    return rows


def _label_set(label):
    return frozenset(int(v) - 1 for v in label.split("-"))


# ---------------------------------------------------------------- keys (Sec. 2)

@pytest.mark.parametrize("G", [1, 2])
def test_fig2_profiles_and_cones(G):
    """Fig. 2: profile membership and cone numbering of the toy dataset."""
    rows = _fig2_rows()
    for x, p1, c1, p2, c2 in rows:
        label, cone = (p1, c1) if G == 1 else (p2, c2)
        order = oracle.magnitude_order(x)
        assert frozenset(order[:G].tolist()) == _label_set(label), (x, label)
        key = oracle.key(x, G)
        assert key % (1 << G) == cone, (x, key, cone)
    # same (profile, cone) <=> same key: the partition of the figure exactly
    groups = {}
    for x, p1, c1, p2, c2 in rows:
        lab = (p1, c1) if G == 1 else (p2, c2)
        groups.setdefault(lab, set()).add(oracle.key(x, G))
    assert all(len(v) == 1 for v in groups.values())
    assert len({next(iter(v)) for v in groups.values()}) == len(groups)
    # profiles are numbered in the order the figure lists them (for K=3 the
    # colexicographic and lexicographic orders coincide)
    prof_rank = {}
    for x, p1, c1, p2, c2 in rows:
        lab = p1 if G == 1 else p2
        prof_rank[lab] = oracle.key(x, G) >> G
    labels = sorted(prof_rank, key=lambda s: [int(v) for v in s.split("-")])
    assert [prof_rank[s] for s in labels] == list(range(len(labels)))


def test_zero_counts_as_positive():
    """Fig. 2 caption: cone 0 holds x1<0, cone 1 'the others' (x1 >= 0)."""
    assert oracle.key(np.array([0.0, 0.0, 0.0], np.float32), 1) == 1
    assert oracle.key(np.array([-0.0, 0.0, 0.0], np.float32), 1) == 1
    assert oracle.key(np.array([-0.0, -0.0, -0.0], np.float32), 2) == 3
    assert oracle.key(np.array([-1.0, 0.0, 0.0], np.float32), 1) == 0


def test_ties_go_to_lower_index():
    x = np.array([1.0, -1.0, 1.0, 0.5], np.float32)
    assert oracle.magnitude_order(x).tolist() == [0, 1, 2, 3]
    assert oracle.key(x, 1) == 1                      # profile {1}, positive
    assert oracle.key(x, 2) >> 2 == 0                 # profile {1,2}
    y = np.array([0.5, -2.0, 2.0, 2.0], np.float32)
    assert oracle.magnitude_order(y).tolist() == [1, 2, 3, 0]


def test_num_cones_closed_forms():
    """N_C = C(K,G) 2^G (Sec. 2): 6 and 12 for the K=3 toy set, 'almost
    30000' for K=16, G=4, and 2K, 2K(K-1), 2^K for G = 1, 2, K."""
    assert oracle.num_cones(3, 1) == 6
    assert oracle.num_cones(3, 2) == 12
    assert oracle.num_cones(16, 4) == 29120
    for K in range(2, 20):
        assert oracle.num_cones(K, 1) == 2 * K
        assert oracle.num_cones(K, 2) == 2 * K * (K - 1)
        assert oracle.num_cones(K, K) == 2 ** K
    for n in range(0, 70):
        for k in range(0, min(n, 20) + 1):
            assert oracle.binom(n, k) == math.comb(n, k)


def _cone_vector(S, signs, d):
    """A vector whose G largest-magnitude components are S (distinct
    magnitudes) with the given signs; the rest small and positive."""
    x = np.full(d, 0.25, np.float32)
    for j, (s, sg) in enumerate(zip(S, signs)):
        x[s] = (10.0 + j) * (1.0 if sg else -1.0)
    return x


@pytest.mark.parametrize("d,L", [(3, 1), (3, 2), (5, 2), (6, 3), (7, 7), (8, 1)])
def test_keys_biject_onto_cones(d, L):
    """Every (profile, sign pattern) maps to a distinct key in [0, N_C)."""
    NC = oracle.num_cones(d, L)
    seen = set()
    for S in itertools.combinations(range(d), L):
        for signs in itertools.product([0, 1], repeat=L):
            x = _cone_vector(S, signs, d)
            k = oracle.key(x, L)
            assert 0 <= k < NC
            # the sign code reads the members by ascending component index,
            # the lowest index in the most significant bit
            code = sum(b << (L - 1 - j) for j, b in enumerate(signs))
            assert k % (1 << L) == code
            seen.add(k)
    assert len(seen) == NC


def _tie_free(rng, n, d):
    X = rng.standard_normal((n, d)).astype(np.float32)
    X[np.abs(X) < 1e-3] = 0.5
    for row in X:
        assert len(set(np.abs(row).tolist())) == d
    return X


def test_key_invariants():
    """Scaling by 2^m changes nothing; permuting coordinates or flipping
    signs permutes the cone partition consistently (Sec. 2: the partition is
    symmetric by construction)."""
    rng = np.random.default_rng(11)
    d, L = 7, 3
    X = _tie_free(rng, 600, d)
    k0 = oracle.keys(X, L)
    for m in (-3, 1, 5):
        assert np.array_equal(oracle.keys(X * np.float32(2.0 ** m), L), k0)

    def same_partition(a, b):
        pairs = {}
        for u, v in zip(a.tolist(), b.tolist()):
            if pairs.setdefault(u, v) != v:
                return False
        return len(set(a.tolist())) == len(set(b.tolist()))

    for _ in range(4):
        pi = rng.permutation(d)
        assert same_partition(k0, oracle.keys(X[:, pi], L))
        flips = np.where(rng.random(d) < 0.5, -1.0, 1.0).astype(np.float32)
        assert same_partition(k0, oracle.keys(X * flips, L))
    # one flipped coordinate: same key if it is outside the top-G set, else
    # the same profile with exactly one sign bit changed
    for x in X[:100]:
        top = set(oracle.magnitude_order(x)[:L].tolist())
        k = oracle.key(x, L)
        for j in range(d):
            z = x.copy()
            z[j] = -z[j]
            kz = oracle.key(z, L)
            if j in top:
                diff = k ^ kz
                assert kz >> L == k >> L and diff and diff & (diff - 1) == 0
            else:
                assert kz == k


# ------------------------------------------------------- buckets (Sec. 4 prep)

def test_buckets_partition_and_stable_order():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((5000, 6)).astype(np.float32)
    L = 2
    NC = oracle.num_cones(6, L)
    keys = oracle.keys(X, L)
    offsets, perm = oracle.buckets(keys, NC)
    assert np.array_equal(offsets, np.concatenate(
        [[0], np.cumsum(np.bincount(keys, minlength=NC))]).astype(np.uint32))
    assert np.array_equal(perm, np.argsort(keys, kind="stable").astype(np.uint32))
    assert offsets[-1] == 5000
    for c in range(NC):
        seg = perm[offsets[c]:offsets[c + 1]]
        assert np.all(keys[seg] == c)
        assert np.all(np.diff(seg.astype(np.int64)) > 0)


def test_cone_occupancy_uniform_for_iid_gaussian():
    """Sec. 2: under perfect symmetry every cone is equally likely."""
    from scipy import stats
    from paper_1509_03453_gb300 import datagen
    w = datagen.workload("gauss16")
    keys = oracle.keys(w["X"], 2)
    counts = np.bincount(keys, minlength=oracle.num_cones(16, 2))
    chi2 = stats.chisquare(counts)
    assert chi2.pvalue > 1e-4


# ------------------------------------------------------- probe order (Sec. 3-B)

def test_probe_order_hand_worked():
    """d=4, G=2, y=(0.1,-3,2,-0.5): order i = (2,3,4,1) in the paper's
    1-based numbering.  Worked by hand:
      delta 0: {2,3}                      signs (-,+)   -> cone 9
      delta 1: {2,4} (rank 3), {2,1} (rank 4)           -> 16, 2
      delta 2: {3,4}, {3,1}, {4,1}                      -> 22, 7, 14
    then the one-flip cones (smaller |y| member flipped first) and the
    two-flip cones, each sweep in the same profile order."""
    y = np.array([0.1, -3.0, 2.0, -0.5], np.float32)
    expect = [9, 16, 2, 22, 7, 14,
              8, 11, 17, 18, 0, 3, 23, 20, 5, 6, 12, 15,
              10, 19, 1, 21, 4, 13]
    assert oracle.probes(y, 2, 100).tolist() == expect
    assert oracle.probes(y, 2, 4).tolist() == expect[:4]


def _cone_table(d, L):
    table = {}
    for S in itertools.combinations(range(d), L):
        for signs in itertools.product([0, 1], repeat=L):
            table[oracle.key(_cone_vector(S, signs, d), L)] = (frozenset(S), signs)
    return table


@pytest.mark.parametrize("d,L", [(6, 2), (7, 3), (9, 4), (8, 1), (5, 5)])
def test_probe_classes(d, L):
    """Profile distance delta = G - level of the closest common ancestor with
    the query's profile {i_1..i_G}: non-decreasing along the list, class
    delta has C(K-G+delta-1, delta) members (summing to C(K,G)), the first
    C(K,G) probes keep the query's signs, and all N_C probes cover every cone
    exactly once."""
    rng = np.random.default_rng(d * 100 + L)
    table = _cone_table(d, L)
    NC = oracle.num_cones(d, L)
    nprof = math.comb(d, L)
    for y in _tie_free(rng, 20, d):
        order = oracle.magnitude_order(y).tolist()
        pr = oracle.probes(y, L, NC + 10)
        assert sorted(pr.tolist()) == list(range(NC))
        deltas = []
        for c in pr[:nprof].tolist():
            S, signs = table[c]
            g = 0
            while g < L and set(order[:g + 1]) <= S:
                g += 1
            deltas.append(L - g)
            members = sorted(S)
            assert list(signs) == [int(y[m] >= 0) for m in members]
        assert deltas == sorted(deltas)
        for delta in range(L + 1):
            if delta == 0:
                expect = 1
            else:
                expect = math.comb(d - L + delta - 1, delta) if d > L else 0
            assert deltas.count(delta) == expect
        assert sum(math.comb(d - L + t - 1, t) for t in range(1, L + 1)
                   if d > L) + 1 == nprof                # hockey stick
        # nested budgets: the first P probes never change with larger P
        for P in (1, 3, nprof, NC):
            assert oracle.probes(y, L, P).tolist() == pr[:min(P, NC)].tolist()


# ------------------------------------------------------- search (Eq. 1, Alg. 1)

def _np_knn(X, Y, k, mask=None):
    D = ((Y.astype(np.float64)[:, None, :] - X.astype(np.float64)[None]) ** 2).sum(-1)
    ids = np.empty((Y.shape[0], k), np.int64)
    ds = np.empty((Y.shape[0], k))
    for q in range(Y.shape[0]):
        row = D[q].copy()
        valid = np.arange(X.shape[0])
        if mask is not None:
            valid = valid[~mask[q]]
        o = valid[np.lexsort((valid, row[valid]))][:k]
        ids[q, :len(o)] = o
        ds[q, :len(o)] = row[o]
        ids[q, len(o):] = -1
        ds[q, len(o):] = np.inf
    return ids, ds


def test_bruteforce_matches_numpy_with_ties():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((300, 5)).astype(np.float32)
    X[150:160] = X[10]                               # exact duplicates: ties
    Y = rng.standard_normal((40, 5)).astype(np.float32)
    Y[0] = X[10]
    for k in (1, 4, 13):
        ids, ds = oracle.bruteforce(X, Y, k)
        eids, eds = _np_knn(X, Y, k)
        assert np.array_equal(ids, eids)
        assert np.array_equal(ds, eds)


def test_exclusion_matches_numpy():
    rng = np.random.default_rng(4)
    W = 20
    X = rng.standard_normal((W * 15, 4)).astype(np.float32)
    src = rng.choice(X.shape[0], 25, replace=False).astype(np.int64)
    Y = X[src]
    r, c = np.divmod(np.arange(X.shape[0]), W)
    sr, sc = np.divmod(src, W)
    mask = np.maximum(np.abs(r[None] - sr[:, None]), np.abs(c[None] - sc[:, None])) <= 2
    ids, ds = oracle.bruteforce(X, Y, 3, query_src=src, grid_w=W, radius=2)
    eids, eds = _np_knn(X, Y, 3, mask)
    assert np.array_equal(ids, eids) and np.array_equal(ds, eds)


@pytest.mark.parametrize("d,L,k", [(6, 2, 1), (5, 3, 3), (8, 1, 5)])
def test_full_budget_is_linear_search(d, L, k):
    """Visiting all N_C cones scans every point: ROSANNA = linear search."""
    rng = np.random.default_rng(d + L + k)
    X = rng.standard_normal((2000, d)).astype(np.float32)
    Y = rng.standard_normal((50, d)).astype(np.float32)
    idx = oracle.Index(X, L)
    ids, ds, cnt = idx.search(Y, idx.NC, k, want_counts=True)
    bids, bds = oracle.bruteforce(X, Y, k)
    assert np.array_equal(ids, bids) and np.array_equal(ds, bds)
    assert np.all(cnt == 2000)


def test_candidates_are_union_of_probed_cones_and_nest():
    rng = np.random.default_rng(21)
    d, L = 8, 2
    X = rng.standard_normal((4000, d)).astype(np.float32)
    Y = rng.standard_normal((60, d)).astype(np.float32)
    idx = oracle.Index(X, L)
    sizes = np.diff(idx.offsets.astype(np.int64))
    prev = None
    for P in (1, 2, 5, 17, 56, idx.NC):
        ids, ds, cnt = idx.search(Y, P, 1, want_counts=True)
        for q in range(Y.shape[0]):
            assert cnt[q] == sizes[oracle.probes(Y[q], L, P)].sum()
        if prev is not None:
            assert np.all(ds[:, 0] <= prev)          # nested candidate sets
        prev = ds[:, 0]
        hit = ids[:, 0] >= 0
        # returned distance is the exact distance of the returned id
        assert np.array_equal(oracle.pair_dists(X, Y, ids)[hit], ds[hit])
