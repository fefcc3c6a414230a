"""The oracle run over row or query slices in parallel threads (how the CPU
baseline uses the host's cores) gives exactly the single-threaded results."""
import numpy as np

import oracle


def test_threaded_oracle_equals_single_threaded():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((5003, 16)).astype(np.float32)
    Y = rng.standard_normal((97, 16)).astype(np.float32)
    a = oracle.Index(X, 2)
    b = oracle.Index(X, 2, threads=5)
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.perm, b.perm)
    ra = a.search(Y, 12, 3, want_counts=True)
    rb = a.search(Y, 12, 3, want_counts=True, threads=7)
    for u, v in zip(ra, rb):
        assert np.array_equal(u, v)
    # with an exclusion source per query
    src = rng.integers(-1, 5003, size=97)
    ea = a.search(Y, 12, 3, query_src=src, grid_w=71, radius=2)
    eb = a.search(Y, 12, 3, query_src=src, grid_w=71, radius=2, threads=4)
    assert np.array_equal(ea[0], eb[0]) and np.array_equal(ea[1], eb[1])
    # a projected (PCA-like) basis
    A = np.linalg.qr(rng.standard_normal((16, 16)))[0][:6].astype(np.float32)
    off = rng.standard_normal(6).astype(np.float32)
    ma = oracle.MultiIndex(X, 2, A[None], offsets=off[None])
    mb = oracle.MultiIndex(X, 2, A[None], offsets=off[None], threads=3)
    assert np.array_equal(ma.perms, mb.perms)
    sa = ma.search(Y, 9, 2, want_counts=True)
    sb = ma.search(Y, 9, 2, want_counts=True, threads=6)
    for u, v in zip(sa, sb):
        assert np.array_equal(u, v)
