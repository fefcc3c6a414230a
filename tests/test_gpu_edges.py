"""Edge cases and error behaviour of the C ABI on the GPU: empty and ragged
inputs, degenerate dimensions, ties and duplicates, clamping, padding, and
the loud errors (invalid arguments, non-finite data)."""
import numpy as np
import pytest

import oracle
from helpers import assert_knn_match, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osann():
    import paper_1509_03453_gb300 as m
    from paper_1509_03453_gb300 import build
    build.build()
    m.load()
    return m


def _check_all(osann, X, Y, L, P, k, paths=("plain", "batched")):
    ref = oracle.Index(X, L)
    idx = osann.Index(to_dev(X), L)
    keys, offsets, perm = (to_np(t) for t in idx.export())
    assert np.array_equal(keys, ref.keys.astype(np.int64))
    assert np.array_equal(offsets, ref.offsets.astype(np.int64))
    assert np.array_equal(perm, ref.perm.astype(np.int64))
    oids, od = ref.search(Y, P, k)
    for path in paths:
        gids, gd = idx.search(to_dev(Y), P, k, path=path)
        assert_knn_match(X, Y, to_np(gids), to_np(gd), oids, od)
    return idx


@pytest.mark.parametrize("d,L", [(1, 1), (3, 2), (5, 5), (7, 3), (20, 4), (33, 2), (100, 3), (256, 2)])
def test_odd_dimensions(osann, d, L):
    """Unaligned rows (scalar loads), padding to 16/32/64/128/256, L = d."""
    rng = np.random.default_rng(d * 31 + L)
    X = rng.standard_normal((3001, d)).astype(np.float32)
    Y = rng.standard_normal((57, d)).astype(np.float32)
    _check_all(osann, X, Y, L, 7, 3)


def test_ties_zeros_and_duplicates(osann):
    """Integer data: magnitude ties (lower index wins), zeros (positive sign),
    exact duplicate points (id order), duplicates of the queries (distance 0)."""
    rng = np.random.default_rng(3)
    X = rng.integers(-3, 4, size=(5000, 8)).astype(np.float32)
    X[4000:4100] = X[17]
    Y = np.concatenate([X[[17, 3, 4050]], rng.integers(-3, 4, size=(40, 8)).astype(np.float32)])
    _check_all(osann, X, Y, 3, 50, 8)


def test_k_beyond_candidates_pads(osann):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((200, 6)).astype(np.float32)
    Y = rng.standard_normal((30, 6)).astype(np.float32)
    idx = _check_all(osann, X, Y, 3, 1, 32)       # one cone, k = 32 > its size
    ids, d2 = idx.search(to_dev(Y), 1, 32)
    ids, d2 = to_np(ids), to_np(d2)
    assert (ids == -1).any()
    assert np.all(np.isinf(d2[ids == -1]))


def test_budget_clamped_to_cone_count(osann):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((777, 4)).astype(np.float32)
    Y = rng.standard_normal((20, 4)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2)
    a = idx.search(to_dev(Y), idx.NC, 5)
    b = idx.search(to_dev(Y), 10 * idx.NC, 5)
    assert np.array_equal(to_np(a[0]), to_np(b[0]))
    assert to_np(idx.probes(to_dev(Y), 10 ** 6)).shape == (20, idx.NC)


def test_single_point_and_empty_batch(osann):
    import torch
    X = np.array([[1.0, -2.0, 3.0, 0.5]], np.float32)
    idx = osann.Index(to_dev(X), 2)
    ids, d2 = idx.search(to_dev(X), 24, 2)
    assert to_np(ids).tolist() == [[0, -1]]
    assert to_np(d2)[0, 0] == 0.0
    e_ids, e_d = idx.search(torch.empty((0, 4), dtype=torch.float32, device="cuda"), 4, 1)
    assert e_ids.shape == (0, 1)


def test_errors_are_loud(osann):
    import torch
    from paper_1509_03453_gb300 import OsannError
    X = np.random.default_rng(1).standard_normal((100, 8)).astype(np.float32)
    bad = X.copy()
    bad[37, 3] = np.nan
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(bad), 2)
    assert e.value.code == -4
    bad[37, 3] = np.inf
    with pytest.raises(OsannError):
        osann.Index(to_dev(bad), 2)
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(X), 9)                  # L > d
    assert e.value.code == -1
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(np.zeros((10, 64), np.float32)), 16, cone_table="dense")   # N_C >= 2^31
    assert e.value.code == -2
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(np.zeros((10, 64), np.float32)), 17)   # L > 16
    assert e.value.code == -1
    idx = osann.Index(to_dev(X), 2)
    with pytest.raises(OsannError):
        idx.search(to_dev(X[:3]), 4, 33)          # k > 32
    with pytest.raises(OsannError):
        idx.search(to_dev(X[:3]), 0, 1)           # P < 1
    q = X[:4].copy()
    q[2, 0] = np.inf
    idx.search(to_dev(q), 4, 1)
    assert idx.status() & 2                        # non-finite query flagged
    assert idx.status() == 0                       # and cleared
    with pytest.raises(OsannError):
        idx.search(to_dev(X[:3]), 4, 1, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))


def test_many_queries_small_budget_and_big_groups(osann):
    """Cone groups larger than one CTA's query group (ragged last group)."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((20_011, 16)).astype(np.float32)
    Y = rng.standard_normal((3_001, 16)).astype(np.float32)
    ref = oracle.Index(X, 1)
    idx = osann.Index(to_dev(X), 1)
    oids, od = ref.search(Y, 3, 2)
    for path in ("plain", "batched"):
        gids, gd = idx.search(to_dev(Y), 3, 2, path=path)
        assert_knn_match(X, Y, to_np(gids), to_np(gd), oids, od)


def test_async_build_same_index_and_deferred_status(osann):
    rng = np.random.default_rng(41)
    X = rng.standard_normal((30_011, 32)).astype(np.float32)
    Y = rng.standard_normal((500, 32)).astype(np.float32)
    a = osann.Index(to_dev(X), 2)
    b = osann.Index(to_dev(X), 2, sync=False)
    assert b.max_bucket == -1
    ia, da = a.search(to_dev(Y), 40, 3)
    ib, db = b.search(to_dev(Y), 40, 3)
    assert b.status() == 0 and b.max_bucket == a.max_bucket
    for ta, tb in zip(a.export(), b.export()):
        assert np.array_equal(to_np(ta), to_np(tb))
    assert np.array_equal(to_np(ia), to_np(ib))
    assert np.array_equal(to_np(da).view(np.uint32), to_np(db).view(np.uint32))
    # non-finite data: the synchronous build refuses it, the asynchronous one
    # reports it at the status read
    X[123, 5] = np.nan
    with pytest.raises(osann.OsannError):
        osann.Index(to_dev(X), 2)
    c = osann.Index(to_dev(X), 2, sync=False)
    assert c.status() & 1
    a.close()
    b.close()
    c.close()
