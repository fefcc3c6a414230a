"""Tensor-core screening paths (bf16 or scaled fp16 tcgen05 tiles + certified
bound + fp32 rerank): same bits as the fp32 paths, parity with the oracle,
and the on-device check of the error bound (OSANN_DEBUG_CHECKS=1) never
fails."""
import os

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
    os.environ["OSANN_DEBUG_CHECKS"] = "1"
    yield m
    os.environ.pop("OSANN_DEBUG_CHECKS", None)


def _cases():
    from paper_1509_03453_gb300 import datagen
    rng = np.random.default_rng(11)
    out = []
    w = datagen.workload("gauss16")
    out.append(("gauss16", w["X"], w["Y"], 2, [4, 64], 1, None))
    out.append(("gauss32", rng.standard_normal((120_011, 32), dtype=np.float32),
                rng.standard_normal((2_000, 32), dtype=np.float32), 2, [16, 128], 1, None))
    out.append(("gauss32_k5", rng.standard_normal((60_013, 32), dtype=np.float32),
                rng.standard_normal((1_500, 32), dtype=np.float32), 2, [64], 5, None))
    img = datagen.patch_image(1003, 192)
    X = datagen.patches(img)
    src = np.sort(rng.choice(X.shape[0], 600, replace=False)).astype(np.int64)
    out.append(("patch64", X, X[src].copy(), 3, [16, 64], 4, (src, 185, 8)))
    out.append(("desc128", datagen.descriptors(40_009, 1004), datagen.descriptor_queries(400, 2004), 3,
                [32], 10, None))
    out.append(("d20", rng.standard_normal((30_007, 20), dtype=np.float32),
                rng.standard_normal((700, 20), dtype=np.float32), 2, [40], 3, None))
    out.append(("d100", rng.standard_normal((20_011, 100), dtype=np.float32),
                rng.standard_normal((300, 100), dtype=np.float32), 1, [30], 2, None))
    # magnitudes far from 1: the fp16 scale must bring them into range exactly
    out.append(("tiny", (1e-6 * rng.standard_normal((30_011, 32))).astype(np.float32),
                (1e-6 * rng.standard_normal((600, 32))).astype(np.float32), 2, [48], 2, None))
    out.append(("huge", (3e4 * rng.standard_normal((30_011, 32))).astype(np.float32),
                (3e4 * rng.standard_normal((600, 32))).astype(np.float32), 2, [48], 2, None))
    return out


CASES = None


def case(i):
    global CASES
    if CASES is None:
        CASES = _cases()
    return CASES[i]


@pytest.mark.parametrize("path", ["bf16", "fp16"])
@pytest.mark.parametrize("i", range(9))
def test_tensor_screen_is_exact(osann, i, path):
    name, X, Y, L, Ps, k, ex = case(i)
    idx = osann.Index(to_dev(X), L)
    Yd = to_dev(Y)
    kw, okw = {}, {}
    if ex is not None:
        kw = dict(query_src=to_dev(ex[0]), grid_w=ex[1], radius=ex[2])
        okw = dict(query_src=ex[0], grid_w=ex[1], radius=ex[2])
    ref = oracle.Index(X, L)
    idx.screen_stats()
    for P in Ps:
        a = idx.search(Yd, P, k, path=path, **kw)
        b = idx.search(Yd, P, k, path="batched", **kw)
        assert np.array_equal(to_np(a[0]), to_np(b[0])), name
        assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(b[1]).view(np.uint32)), name
        oids, od = ref.search(Y, P, k, **okw)
        assert_knn_match(X, Y, to_np(a[0]), to_np(a[1]), oids, od)
    st = idx.screen_stats()
    assert st["bound_checks"] > 0
    assert st["bound_violations"] == 0, st
    assert idx.status() == 0
    print(name, path, st)


@pytest.mark.parametrize("path", ["bf16", "fp16"])
def test_tensor_full_budget_is_linear_search(osann, path):
    name, X, Y, L, Ps, k, ex = case(0)
    idx = osann.Index(to_dev(X), L)
    Yd = to_dev(Y)
    a = idx.search(Yd, idx.NC, k, path=path)
    bf = idx.bruteforce(Yd, k)
    assert np.array_equal(to_np(a[0]), to_np(bf[0]))
    assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(bf[1]).view(np.uint32))
    assert idx.screen_stats()["bound_violations"] == 0


def test_fp16_out_of_range_query_takes_the_full_scan(osann):
    """A query too large for the scaled fp16 range is rescanned in fp32."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal((20_011, 32)).astype(np.float32)
    Y = rng.standard_normal((300, 32)).astype(np.float32)
    Y[7] *= 1e5
    idx = osann.Index(to_dev(X), 2)
    Yd = to_dev(Y)
    idx.screen_stats()
    a = idx.search(Yd, 64, 3, path="fp16")
    b = idx.search(Yd, 64, 3, path="batched")
    assert np.array_equal(to_np(a[0]), to_np(b[0]))
    assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(b[1]).view(np.uint32))
    assert idx.screen_stats()["fallbacks"] >= 1


@pytest.mark.parametrize("Q,P", [(1, 1), (1, 7), (31, 3), (32, 64), (33, 5), (65, 130), (97, 1984), (300, 255)])
def test_query_set_work_list_shapes(osann, Q, P):
    """The tensor-core work list built from per-cone query sets: query counts
    around multiples of 32 (the query-set words), slot counts not divisible
    by 4 (the scalar loads), one query, every cone (P = N_C), and N_C = 1984
    cones in the shared-memory words: same bits as the batched fp32 path
    (whose list keeps the slots), parity with the oracle."""
    rng = np.random.default_rng(7 * Q + P)
    X = rng.standard_normal((30_011, 32)).astype(np.float32)
    Y = rng.standard_normal((Q, 32)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2)
    assert idx.NC == 1984
    Yd = to_dev(Y)
    ref = oracle.Index(X, 2)
    for k in (1, 3):
        a = idx.search(Yd, P, k, path="fp16")
        b = idx.search(Yd, P, k, path="batched")
        assert np.array_equal(to_np(a[0]), to_np(b[0]))
        assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(b[1]).view(np.uint32))
        oids, od = ref.search(Y, P, k)
        assert_knn_match(X, Y, to_np(a[0]), to_np(a[1]), oids, od)
    assert idx.screen_stats()["bound_violations"] == 0
    assert idx.status() == 0
    idx.close()


def test_work_lists_at_the_shared_memory_cone_limit(osann):
    """N_C = C(78, 2) 4 = 12012 cones, near the 12288 that the per-cone
    shared-memory arrays serve (their size then passes the default 48 KB of
    dynamic shared memory): both work lists (query sets for the screen,
    per-block histograms for the fp32 batched path) give the oracle's
    answer."""
    rng = np.random.default_rng(78)
    X = rng.standard_normal((40_000, 78)).astype(np.float32)
    Y = rng.standard_normal((150, 78)).astype(np.float32)
    idx = osann.Index(to_dev(X), 2)
    assert idx.NC == 12012
    ref = oracle.Index(X, 2)
    Yd = to_dev(Y)
    for P in (64, 700):
        oids, od = ref.search(Y, P, 2)
        a = idx.search(Yd, P, 2, path="fp16")
        b = idx.search(Yd, P, 2, path="batched")
        assert np.array_equal(to_np(a[0]), to_np(b[0]))
        assert_knn_match(X, Y, to_np(a[0]), to_np(a[1]), oids, od)
    assert idx.status() == 0
    idx.close()
