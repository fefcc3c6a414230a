"""GPU parity of the second-level cone table (Sec. 4, large N_C).

128-bit cone ids against the oracle's; indexes whose N_C is far beyond 2^31
(d = 64, L = 11: N_C ~ 1.5e15; d = 128 and 256, L = 16: three and four id
words) against the oracle's occupied-cone table and search, on every path;
the second-level table forced on small N_C against the direct table, bit for
bit (keys, permutation, offsets over the occupied cones, probes, results).
"""
import numpy as np
import pytest

import oracle
from helpers import assert_knn_match, to_dev, to_np

pytestmark = pytest.mark.gpu

PATHS = ("plain", "batched", "fp16", "bf16")


@pytest.fixture(scope="module")
def osann():
    import paper_1509_03453_gb300 as m
    from paper_1509_03453_gb300 import build
    build.build()
    m.load()
    yield m


def _data(N, d, seed, dup=True):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, d)).astype(np.float32)
    if dup:
        X[10:60] = X[3]  # one crowded cone (exact duplicates)
    return X


def _queries(X, Q, seed):
    rng = np.random.default_rng(seed)
    near = X[rng.choice(X.shape[0], Q // 2, replace=False)] + 0.05 * rng.standard_normal((Q // 2, X.shape[1]))
    far = rng.standard_normal((Q - Q // 2, X.shape[1]))
    return np.concatenate([near, far]).astype(np.float32)


@pytest.mark.parametrize("d,L", [(64, 11), (128, 16), (256, 16), (30, 7), (32, 2)])
def test_keys_wide_match_oracle(osann, d, L):
    X = _data(3000, d, 100 + d)
    X[0] = 0.0                      # all zero: ties everywhere, signs positive
    X[1, : d // 2] = -0.0
    X[2] = np.round(X[2])           # integer magnitudes, many ties
    assert osann.keys_wide(to_dev(X), L) == oracle.keys_wide(X, L)


def _check_table(idx, w):
    keys, offs, perm = (to_np(t) for t in idx.export())
    assert np.array_equal(perm, w.perm)
    n_occ = w.n_occ
    assert idx.occupied() == n_occ
    assert np.array_equal(offs[: n_occ + 1], w.offsets)
    assert np.all(offs[n_occ:] == idx.N)          # compact cones past the occupied ones are empty
    ids = idx.cone_ids()
    assert ids[:n_occ] == w.uniq
    assert all(v == (1 << 128) - 1 for v in ids[n_occ:])
    # every point's compact cone holds its id
    assert [ids[c] for c in keys] == w.keys


@pytest.mark.parametrize("d,L,N,P,k", [(64, 11, 30000, 64, 4), (128, 16, 20000, 48, 3), (256, 16, 6000, 32, 2)])
def test_large_nc_table_and_search(osann, d, L, N, P, k):
    X = _data(N, d, 200 + d)
    Y = _queries(X, 120, 300 + d)
    idx = osann.Index(to_dev(X), L)
    assert idx.hashed and idx.n_cones == oracle.num_cones_wide(d, L) > 2 ** 31
    assert idx.NC == N + 1
    w = oracle.WideIndex(X, L)
    _check_table(idx, w)
    oids, od = w.search(Y, P, k)
    ref = None
    for path in PATHS if d <= 128 else ("plain", "batched"):
        gi, gd = idx.search(to_dev(Y), P, k, path=path)
        gi, gd = to_np(gi), to_np(gd)
        assert_knn_match(X, Y, gi, gd, oids, od)
        if ref is None:
            ref = (gi, gd)
        else:
            assert np.array_equal(gi, ref[0]) and np.array_equal(gd.view(np.uint32), ref[1].view(np.uint32))
    assert idx.status() == 0
    idx.close()


@pytest.mark.parametrize("d,L", [(32, 2), (16, 3), (24, 4)])
def test_forced_second_level_equals_direct_table(osann, d, L):
    X = _data(20000, d, 400 + d)
    Y = _queries(X, 300, 500 + d)
    dense = osann.Index(to_dev(X), L, cone_table="dense")
    hashed = osann.Index(to_dev(X), L, cone_table="hashed")
    assert not dense.hashed and hashed.hashed and hashed.n_cones == dense.NC
    dk, do, dp = (to_np(t) for t in dense.export())
    hk, ho, hp = (to_np(t) for t in hashed.export())
    assert np.array_equal(hp, dp)
    occ = np.unique(dk)
    n_occ = hashed.occupied()
    assert n_occ == occ.size == dense.occupied()
    assert np.array_equal(ho[: n_occ + 1], np.append(do[occ], X.shape[0]))
    assert hashed.cone_ids()[:n_occ] == [int(c) for c in occ]
    assert np.array_equal(occ[hk], dk)
    # probe lists: compact cones map back to the direct ids; unoccupied ids to the empty cone
    P = 40
    pd_ = to_np(dense.probes(to_dev(Y), P))
    ph = to_np(hashed.probes(to_dev(Y), P))
    lut = np.full(dense.NC, hashed.NC - 1, np.int64)
    lut[occ] = np.arange(occ.size)
    assert np.array_equal(ph, lut[pd_])
    for path in PATHS:
        for k in (1, 5):
            a = dense.search(to_dev(Y), P, k, path=path)
            b = hashed.search(to_dev(Y), P, k, path=path)
            assert np.array_equal(to_np(a[0]), to_np(b[0]))
            assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(b[1]).view(np.uint32))
    # the full budget reaches every point: brute force
    bi, bd = hashed.search(to_dev(Y[:40]), dense.NC, 2, path="plain")
    ri, rd = hashed.bruteforce(to_dev(Y[:40]), 2)
    assert np.array_equal(to_np(bi), to_np(ri))
    dense.close()
    hashed.close()


def test_second_level_edges(osann):
    d, L = 64, 11
    # one point
    X1 = _data(1, d, 1, dup=False)
    idx = osann.Index(to_dev(X1), L)
    assert idx.hashed and idx.NC == 2 and idx.occupied() == 1
    gi, gd = idx.search(to_dev(X1), 8, 3)
    assert to_np(gi).tolist() == [[0, -1, -1]]
    idx.close()
    # every point in one cone
    X = np.repeat(_data(1, d, 2, dup=False), 500, axis=0)
    idx = osann.Index(to_dev(X), L)
    w = oracle.WideIndex(X, L)
    assert w.n_occ == 1
    _check_table(idx, w)
    Y = _queries(X, 20, 3)
    oids, od = w.search(Y, 5, 4)
    gi, gd = idx.search(to_dev(Y), 5, 4, path="plain")
    assert_knn_match(X, Y, to_np(gi), to_np(gd), oids, od)
    idx.close()
    # asynchronous build, then the status check
    X = _data(5000, d, 4)
    idx = osann.Index(to_dev(X), L, sync=False)
    Y = _queries(X, 50, 5)
    gi, gd = idx.search(to_dev(Y), 32, 2)
    assert idx.status() == 0
    oids, od = oracle.WideIndex(X, L).search(Y, 32, 2)
    assert_knn_match(X, Y, to_np(gi), to_np(gd), oids, od)
    idx.close()
    # a direct table cannot hold this N_C
    with pytest.raises(osann.OsannError):
        osann.Index(to_dev(X), L, cone_table="dense")


def test_second_level_exclusion(osann):
    """Patch-like rows (mean-removed 8 x 8 patches, d = 64) with L = 8
    (N_C ~ 1.1e12) and the Chebyshev exclusion of the copy-move workload."""
    import torch
    from paper_1509_03453_gb300 import datagen
    img = datagen.patch_image(7, size=96)
    X = datagen.patches(img)
    grid_w = img.shape[1] - 8 + 1
    rng = np.random.default_rng(9)
    src = np.sort(rng.choice(X.shape[0], 200, replace=False)).astype(np.int64)
    Y = X[src]
    L, P, k, radius = 8, 32, 4, 8
    idx = osann.Index(to_dev(X), L)
    assert idx.hashed
    w = oracle.WideIndex(X, L)
    oids, od = w.search(Y, P, k, query_src=src, grid_w=grid_w, radius=radius)
    for path in ("plain", "batched", "fp16"):
        gi, gd = idx.search(to_dev(Y), P, k, path=path, query_src=torch.from_numpy(src).cuda(), grid_w=grid_w,
                            radius=radius)
        assert_knn_match(X, Y, to_np(gi), to_np(gd), oids, od)
    idx.close()


def test_second_level_rotated_basis(osann):
    """A rotated basis (Sec. 3-D) over a forced second-level table: the same
    bits as over the direct table."""
    from paper_1509_03453_gb300 import datagen
    d, L = 32, 3
    X = _data(20000, d, 600)
    Y = _queries(X, 200, 601)
    R = to_dev(datagen.rotations(2, d, 3)[1])
    a = osann.Index(to_dev(X), L, rot=R, cone_table="dense")
    b = osann.Index(to_dev(X), L, rot=R, cone_table="hashed")
    assert b.hashed
    for path in ("plain", "fp16"):
        ra = a.search(to_dev(Y), 24, 3, path=path)
        rb = b.search(to_dev(Y), 24, 3, path=path)
        assert np.array_equal(to_np(ra[0]), to_np(rb[0]))
        assert np.array_equal(to_np(ra[1]).view(np.uint32), to_np(rb[1]).view(np.uint32))
    a.close()
    b.close()
