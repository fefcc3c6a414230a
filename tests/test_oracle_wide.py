"""Oracle pins for the second-level cone table (Sec. 4: when N_C grows very
large, only the occupied cones are stored and probed cones are looked up).

The 128-bit cone ids are pinned where the direct table is pinned already
(N_C < 2^31: the same numbers, the same point order, the same search), and
on huge N_C by properties that fix the colexicographic rank without
binomials: the smallest and largest ids (hockey-stick identity), the
successor rule of the colexicographic order, the order itself (the largest
element of the symmetric difference decides), and the sign code's bits.
The search over the table is checked against its definition: the exact
top-k, by numpy in fp64, over the points whose id is in the probed list."""
import math

import numpy as np
import pytest

import oracle


def _vec_with_top(d, S, signs=None, seed=0):
    """A vector whose L largest magnitudes sit exactly on the members of S
    (distinct magnitudes in (1, 2)), with the given signs (+1 default), the
    other components in (-0.5, 0.5)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, size=d)
    S = list(S)
    mags = 1.0 + rng.permutation(len(S)) / (2.0 * len(S))
    for j, c in enumerate(S):
        s = 1.0 if signs is None else signs[j]
        x[c] = s * mags[j]
    return x.astype(np.float32)


def _colex_successor(S, d):
    """Next L-subset of {0..d-1} in colexicographic order, or None."""
    s = sorted(S)
    L = len(s)
    for j in range(L):
        nxt = s[j + 1] if j + 1 < L else d
        if s[j] + 1 < nxt:
            return list(range(j)) + [s[j] + 1] + s[j + 1:]
    return None


@pytest.mark.parametrize("d,L", [(16, 2), (32, 3), (64, 11), (128, 16), (256, 16), (300, 7)])
def test_num_cones_wide_closed_form(d, L):
    assert oracle.num_cones_wide(d, L) == math.comb(d, L) * 2 ** L


@pytest.mark.parametrize("d,L", [(1024, 16), (512, 32), (5, 6)])
def test_num_cones_wide_out_of_range(d, L):
    assert oracle.num_cones_wide(d, L) == -1


@pytest.mark.parametrize("name,L,P", [("gauss16", 2, 7), ("gauss32", 3, 40), ("ties", 3, 25)])
def test_wide_table_equals_direct_table(name, L, P):
    rng = np.random.default_rng(31)
    if name == "gauss16":
        X = rng.standard_normal((3000, 16)).astype(np.float32)
    elif name == "gauss32":
        X = rng.standard_normal((2500, 32)).astype(np.float32)
    else:  # integer magnitudes with many ties and zeros
        X = rng.integers(-3, 4, size=(2500, 24)).astype(np.float32)
    Y = X[rng.choice(X.shape[0], 30, replace=False)] + rng.standard_normal((30, X.shape[1])).astype(np.float32)
    o = oracle.Index(X, L)
    w = oracle.WideIndex(X, L)
    assert w.NC == o.NC
    assert w.keys == [int(v) for v in o.keys]
    assert np.array_equal(w.perm, o.perm)
    occ = np.unique(o.keys)
    assert w.uniq == [int(v) for v in occ]
    assert np.array_equal(w.offsets, np.append(o.offsets[occ], np.uint32(X.shape[0])))
    for y in Y[:5]:
        assert oracle.probes_wide(y, L, P) == [int(v) for v in oracle.probes(y, L, P)]
    a_ids, a_d = w.search(Y, P, 3)
    b_ids, b_d = o.search(Y, P, 3)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_d, b_d)
    # the full budget is brute force
    f_ids, f_d = w.search(Y, o.NC, 2)
    r_ids, r_d = oracle.bruteforce(X, Y, 2)
    assert np.array_equal(f_ids, r_ids) and np.array_equal(f_d, r_d)


@pytest.mark.parametrize("d,L", [(64, 11), (128, 16), (256, 16)])
def test_wide_key_extremes(d, L):
    NC = math.comb(d, L) * 2 ** L
    top = list(range(d - L, d))
    low = list(range(L))
    # largest profile, all signs positive: N_C - 1 (sum_j C(d-L+j, j+1) = C(d,L) - 1)
    assert oracle.keys_wide(_vec_with_top(d, top)[None], L) == [NC - 1]
    # smallest profile: rank 0; all negative -> 0, all positive -> 2^L - 1
    assert oracle.keys_wide(_vec_with_top(d, low, [-1.0] * L)[None], L) == [0]
    assert oracle.keys_wide(_vec_with_top(d, low)[None], L) == [2 ** L - 1]


@pytest.mark.parametrize("d,L,seed", [(64, 11, 1), (200, 16, 2), (256, 13, 3)])
def test_wide_key_colex_successor_and_order(d, L, seed):
    rng = np.random.default_rng(seed)
    for t in range(40):
        S = sorted(rng.choice(d, size=L, replace=False).tolist())
        T = _colex_successor(S, d)
        if T is None:
            continue
        ks, kt = oracle.keys_wide(np.stack([_vec_with_top(d, S, seed=t), _vec_with_top(d, T, seed=t + 99)]), L)
        assert kt - ks == 2 ** L  # rank(successor) = rank + 1
        # order of two random profiles: the larger max of the symmetric difference wins
        U = sorted(rng.choice(d, size=L, replace=False).tolist())
        ku = oracle.keys_wide(_vec_with_top(d, U, seed=t + 7)[None], L)[0]
        diff = set(S) ^ set(U)
        if diff:
            assert (ks < ku) == (max(diff) in U)


@pytest.mark.parametrize("d,L", [(64, 11), (200, 16)])
def test_wide_key_sign_bits(d, L):
    rng = np.random.default_rng(8)
    S = sorted(rng.choice(d, size=L, replace=False).tolist())
    base = oracle.keys_wide(_vec_with_top(d, S)[None], L)[0]
    assert base % 2 ** L == 2 ** L - 1
    for j in range(L):
        sg = [1.0] * L
        sg[j] = -1.0
        k = oracle.keys_wide(_vec_with_top(d, S, sg)[None], L)[0]
        # the member with the j-th smallest index owns bit L-1-j
        assert base - k == 2 ** (L - 1 - j)
    # zero counts as positive, -0.0 included: with L-1 nonzero components the
    # last member is the lowest-index zero, and its bit is set either way
    x = np.zeros(d, np.float32)
    x[S[1:]] = -1.0 - np.arange(L - 1, dtype=np.float32) / L
    c = min(set(range(d)) - set(S[1:]))
    xp, xn, xt = x.copy(), x.copy(), x.copy()
    xn[c] = -0.0
    xt[c] = 1e-30  # the same cone with an explicitly positive member
    kp, kn, kt = oracle.keys_wide(np.stack([xp, xn, xt]), L)
    assert kp == kn == kt
    assert kp % 2 ** L == 2 ** (L - 1 - sorted(S[1:] + [c]).index(c))


def test_wide_probe_prefix():
    d, L = 64, 11
    y = np.random.default_rng(77).standard_normal(d).astype(np.float32)
    order = oracle.magnitude_order(y).tolist()
    pr = oracle.probes_wide(y, L, 1 + (d - L) + 5)
    assert len(pr) == 1 + (d - L) + 5 and len(set(pr)) == len(pr)
    assert pr[0] == oracle.keys_wide(y[None], L)[0]
    # delta = 1: keep the top L-1, the last member the ranks L+1 .. d in order
    for r in range(L + 1, d + 1):
        S = order[:L - 1] + [order[r - 1]]
        x = _vec_with_top(d, S, [1.0 if y[c] >= 0 else -1.0 for c in S], seed=r)
        assert pr[r - L] == oracle.keys_wide(x[None], L)[0]


@pytest.mark.parametrize("d,L,P,k", [(64, 11, 64, 4), (48, 9, 200, 2)])
def test_wide_search_is_exact_topk_over_probed_cones(d, L, P, k):
    rng = np.random.default_rng(40 + d)
    X = rng.standard_normal((2500, d)).astype(np.float32)
    X[100:140] = X[0]  # a crowded cone (duplicates)
    Y = np.concatenate([X[rng.choice(2500, 10)] + 0.05 * rng.standard_normal((10, d)),
                        rng.standard_normal((10, d))]).astype(np.float32)
    w = oracle.WideIndex(X, L)
    assert w.NC > 2 ** 31 and w.n_occ <= X.shape[0]
    ids, dd, cnt = w.search(Y, P, k, want_counts=True)
    keys = np.array(w.keys, dtype=object)
    X64 = X.astype(np.float64)
    for q in range(Y.shape[0]):
        pset = set(oracle.probes_wide(Y[q], L, P))
        cand = np.array([n for n in range(X.shape[0]) if keys[n] in pset], np.int64)
        assert cnt[q] == cand.size
        dist = ((X64[cand] - Y[q].astype(np.float64)) ** 2).sum(1) if cand.size else np.zeros(0)
        o = np.lexsort((cand, dist))[:k]
        exp_ids = np.full(k, -1, np.int64)
        exp_d = np.full(k, np.inf)
        exp_ids[:o.size] = cand[o]
        exp_d[:o.size] = dist[o]
        assert np.array_equal(ids[q], exp_ids)
        assert np.allclose(dd[q], exp_d, rtol=1e-12, atol=0)
