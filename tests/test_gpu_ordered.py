"""GPU parity of the ORDERED key (the top-L components as a tuple in
magnitude order, N_C = d!/(d-L)! 2^L) against the oracle: keys, offsets and
permutation bit for bit, probe lists bit for bit (through the sign-flip
extension), the search on every path within the suite's tolerance and bit
identical across paths, the full budget equal to linear search; builds the
variant cannot serve are refused."""
import math

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


def _case(name):
    from paper_1509_03453_gb300 import datagen
    rng = np.random.default_rng(hash(name) % 2 ** 32)
    if name == "gauss16_L2":
        return rng.standard_normal((20_011, 16), dtype=np.float32), rng.standard_normal((150, 16), dtype=np.float32), 2
    if name == "gauss32_L3":
        return rng.standard_normal((60_007, 32), dtype=np.float32), rng.standard_normal((120, 32), dtype=np.float32), 3
    if name == "odd30_L2":  # d not a multiple of 4: the scalar key path; ties and zeros
        X = np.round(rng.standard_normal((30_001, 30)) * 4).astype(np.float32)
        return X, np.round(rng.standard_normal((120, 30)) * 4).astype(np.float32), 2
    if name == "desc128_L2":
        return datagen.descriptors(20_000, 1004), datagen.descriptor_queries(80, 2004), 2
    if name == "gauss8_L4":
        return rng.standard_normal((20_000, 8), dtype=np.float32), rng.standard_normal((100, 8), dtype=np.float32), 4
    raise KeyError(name)


NAMES = ["gauss16_L2", "gauss32_L3", "odd30_L2", "desc128_L2", "gauss8_L4"]


@pytest.mark.parametrize("name", NAMES)
def test_ordered_keys_buckets_probes_bit_exact(osann, name):
    X, Y, L = _case(name)
    d = X.shape[1]
    ref = oracle.Index(X, L, key_mode=1)
    idx = osann.Index(to_dev(X), L, key_mode="ordered")
    assert idx.n_cones == ref.NC == math.perm(d, L) * 2 ** L
    keys, offsets, perm = (to_np(t) for t in idx.export())
    assert np.array_equal(keys, ref.keys.astype(np.int64))
    assert np.array_equal(offsets, ref.offsets.astype(np.int64))
    assert np.array_equal(perm, ref.perm.astype(np.int64))
    nprof = math.perm(d, L)
    for P in sorted({1, 7, 64, min(nprof + 29, ref.NC)}):
        pr = to_np(idx.probes(to_dev(Y), P))
        for q in range(Y.shape[0]):
            assert np.array_equal(pr[q], oracle.probes_ordered(Y[q], L, P).astype(np.int64)), (name, P, q)
    assert idx.status() == 0
    idx.close()


@pytest.mark.parametrize("name", NAMES)
def test_ordered_search_matches_oracle_on_every_path(osann, name):
    X, Y, L = _case(name)
    ref = oracle.Index(X, L, key_mode=1)
    idx = osann.Index(to_dev(X), L, key_mode="ordered")
    Yd = to_dev(Y)
    paths = ["plain", "batched", "fp16", "bf16"] if X.shape[1] <= 128 else ["plain", "batched"]
    for P, k in ((16, 1), (96, 4)):
        oids, od = ref.search(Y, P, k)
        first = None
        for path in paths:
            gi, gd = (to_np(t) for t in idx.search(Yd, P, k, path=path))
            assert_knn_match(X, Y, gi, gd, oids, od)
            if first is None:
                first = (gi, gd)
            else:
                assert np.array_equal(gi, first[0]) and np.array_equal(gd.view(np.int32), first[1].view(np.int32))
    assert idx.status() == 0
    idx.close()


def test_ordered_full_budget_is_linear_search(osann):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((8000, 6)).astype(np.float32)
    Y = rng.standard_normal((60, 6)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2, key_mode="ordered")
    gi, gd = idx.search(to_dev(Y), idx.n_cones, 3, path="plain")
    bi, bd = idx.bruteforce(to_dev(Y), 3)
    assert np.array_equal(to_np(gi), to_np(bi))
    assert np.array_equal(to_np(gd).view(np.int32), to_np(bd).view(np.int32))
    idx.close()


def test_ordered_refuses_what_it_cannot_serve(osann):
    from paper_1509_03453_gb300 import OsannError
    X = np.random.default_rng(6).standard_normal((1000, 128)).astype(np.float32)
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(X), 4, key_mode="ordered")  # 128*127*126*125*16 >= 2^31
    assert e.value.code == -2
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(X[:, :16]), 2, key_mode="ordered", cone_table="hashed")
    assert e.value.code == -2
    with pytest.raises(OsannError) as e:
        osann.Index(to_dev(X[:, :16]), 2, key_mode="ordered", centroids=to_dev(X[:4, :16]))
    assert e.value.code == -2
