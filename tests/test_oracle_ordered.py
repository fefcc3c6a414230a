"""Oracle pins for the ORDERED key (the other reading of the "ordered
(index, sign)" profile, Sec. 2): the tuple of the L largest-magnitude
components in decreasing magnitude, with their signs.

Pinned by: the closed form N_C = d!/(d-L)! 2^L; a hand-worked d = 4, L = 2
case (key and probe list derived from the definitions by hand, below); the
numbering equal to the position of the tuple in itertools' lexicographic
enumeration of L-permutations (an independent routine); the key surjective
onto [0, N_C); the set key recovered by sorting the tuple; equivariance under
coordinate permutation; the probe list a permutation of all cones whose
classes have the closed-form sizes and whose rank tuples ascend inside a
class; and the full budget equal to linear search."""
import itertools
import math

import numpy as np
import pytest

import oracle


def test_num_cones_closed_form():
    for d, L in [(1, 1), (4, 2), (6, 3), (16, 2), (32, 3), (7, 7), (128, 2)]:
        assert oracle.num_cones_ordered(d, L) == math.perm(d, L) * 2 ** L
    # the set key has C(d, L) 2^L cones: the ordered one L! times as many
    assert oracle.num_cones_ordered(16, 4) == math.factorial(4) * oracle.num_cones(16, 4)


# Hand-worked case, d = 4, L = 2, y = (0.5, -3, 2, 1).  Magnitude order
# i_1..i_4 = 1, 2, 3, 0.  Tuple (1, 2): c_0 = 1, c_1 = 2 - 1 (one earlier
# member below 2) = 1, rank = 1*3 + 1 = 4; signs (-, +) -> code 0b01; key 17.
# Probe order: delta 0: (1,2) -> 17.  delta 1 (prefix (1), next member any
# but i_2 = 2): (1,3) rank 1*3+2 = 5, code 01 -> 21; (1,0) rank 3, code 01 ->
# 13.  delta 2 (first member any but i_1 = 1, by rank: 2, 3, 0; second any
# unused, by rank): (2,1) rank 7 code 10 -> 30; (2,3) rank 8 code 11 -> 35;
# (2,0) rank 6 code 11 -> 27; (3,1) rank 10 code 10 -> 42; (3,2) rank 11
# code 11 -> 47; (3,0) rank 9 code 11 -> 39; (0,1) rank 0 code 10 -> 2; (0,2)
# rank 1 code 11 -> 7; (0,3) rank 2 code 11 -> 11.  Then one flip: (1,2) with
# its smaller-|y| member (2) flipped -> code 00 -> 16, its larger (1) flipped
# -> code 11 -> 19.
HAND_Y = np.array([0.5, -3.0, 2.0, 1.0], np.float32)
HAND_PROBES = [17, 21, 13, 30, 35, 27, 42, 47, 39, 2, 7, 11, 16, 19]


def test_hand_worked_case():
    assert oracle.key_ordered(HAND_Y, 2) == 17
    assert oracle.probes_ordered(HAND_Y, 2, len(HAND_PROBES)).tolist() == HAND_PROBES
    full = oracle.probes_ordered(HAND_Y, 2, 1000)
    assert sorted(full.tolist()) == list(range(48))


def _tuple_key(x, L):
    """Independent restatement: lexicographic position of the magnitude-ordered
    top-L tuple among itertools' L-permutations, then the sign code."""
    d = x.shape[0]
    order = sorted(range(d), key=lambda i: (-abs(float(x[i])), i))[:L]
    rank = {t: r for r, t in enumerate(itertools.permutations(range(d), L))}[tuple(order)]
    code = 0
    for j, c in enumerate(order):
        code |= (1 if x[c] >= 0 else 0) << (L - 1 - j)
    return rank * 2 ** L + code, order


@pytest.mark.parametrize("d,L", [(5, 2), (6, 3), (7, 1), (4, 4)])
def test_numbering_is_the_lexicographic_permutation_index(d, L):
    rng = np.random.default_rng(100 * d + L)
    X = rng.standard_normal((300, d)).astype(np.float32)
    X[::7, 0] = 0.0
    X[::11, 1] = -0.0
    got = oracle.keys_ordered(X, L)
    for x, g in zip(X, got):
        assert g == _tuple_key(x, L)[0]


def test_keys_cover_all_cones():
    d, L = 5, 2
    seen = set()
    for T in itertools.permutations(range(d), L):
        for signs in itertools.product((-1.0, 1.0), repeat=L):
            x = np.full(d, 0.01, np.float32) * (1 + np.arange(d, dtype=np.float32))
            for j, (c, sg) in enumerate(zip(T, signs)):
                x[c] = sg * (10.0 - j)
            seen.add(oracle.key_ordered(x, L))
    assert seen == set(range(oracle.num_cones_ordered(d, L)))


def test_sorting_the_tuple_gives_the_set_key():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((200, 9)).astype(np.float32)
    for x in X:
        _, order = _tuple_key(x, 3)
        s = sorted(order)
        rank = sum(math.comb(c, j + 1) for j, c in enumerate(s))
        code = sum((1 if x[c] >= 0 else 0) << (2 - j) for j, c in enumerate(s))
        assert oracle.key(x, 3) == rank * 8 + code


def test_permutation_equivariance():
    rng = np.random.default_rng(4)
    d, L = 8, 3
    X = rng.standard_normal((100, d)).astype(np.float32)
    pi = rng.permutation(d)
    Xp = np.empty_like(X)
    Xp[:, pi] = X  # component c moves to pi[c]
    perms = list(itertools.permutations(range(d), L))
    for x, xp in zip(X, Xp):
        k, kp = oracle.key_ordered(x, L), oracle.key_ordered(xp, L)
        T, Tp = perms[k >> L], perms[kp >> L]
        assert Tp == tuple(int(pi[c]) for c in T)
        assert (k & (2 ** L - 1)) == (kp & (2 ** L - 1))


@pytest.mark.parametrize("d,L", [(5, 2), (6, 3), (4, 4)])
def test_probe_classes(d, L):
    rng = np.random.default_rng(d * 10 + L)
    perms = list(itertools.permutations(range(d), L))
    nprof = math.perm(d, L)
    for _ in range(5):
        y = rng.standard_normal(d).astype(np.float32)
        order = sorted(range(d), key=lambda i: (-abs(float(y[i])), i))
        rank_of = {c: r for r, c in enumerate(order)}
        pr = oracle.probes_ordered(y, L, 10 ** 6)
        assert sorted(pr.tolist()) == list(range(oracle.num_cones_ordered(d, L)))  # every cone once
        assert pr[0] == oracle.key_ordered(y, L)
        own = tuple(order[:L])
        prev = None
        sizes = {}
        for c in pr[:nprof]:
            T = perms[int(c) >> L]
            code = int(c) & (2 ** L - 1)
            # the query's own signs
            assert code == sum((1 if y[t] >= 0 else 0) << (L - 1 - j) for j, t in enumerate(T))
            lcp = next((j for j in range(L) if T[j] != own[j]), L)
            delta = L - lcp
            key = (delta, tuple(rank_of[t] for t in T[lcp:]))
            assert prev is None or key > prev  # delta ascending, then the rank tuple lexicographic
            prev = key
            sizes[delta] = sizes.get(delta, 0) + 1
        for delta, cnt in sizes.items():
            n0 = d - (L - delta)
            exp = 1 if delta == 0 else (n0 - 1) * math.perm(n0 - 1, delta - 1)
            assert cnt == exp


def test_nesting_and_full_budget_is_linear_search():
    rng = np.random.default_rng(9)
    d, L = 6, 2
    X = rng.standard_normal((3000, d)).astype(np.float32)
    Y = rng.standard_normal((40, d)).astype(np.float32)
    ix = oracle.Index(X, L, key_mode=1)
    assert ix.NC == oracle.num_cones_ordered(d, L)
    assert np.array_equal(ix.keys, oracle.keys_ordered(X, L))
    # buckets partition the data, each point in its own cone
    assert ix.offsets[-1] == X.shape[0]
    for c in range(ix.NC):
        assert (ix.keys[ix.perm[ix.offsets[c]:ix.offsets[c + 1]]] == c).all()
    prev = None
    for P in (1, 4, 16, 64, ix.NC):
        ids, dd = ix.search(Y, P, 3)
        if prev is not None:
            assert (dd[:, 0] <= prev[:, 0]).all()
        prev = dd
    bf = oracle.bruteforce(X, Y, 3)
    assert np.array_equal(ids, bf[0]) and np.array_equal(dd, bf[1])
