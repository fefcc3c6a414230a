"""The tensor-core screen's query-tile layouts (shared memory or tensor
memory, a tuning knob of the library's own): every layout returns the same
bits on both 16-bit precisions, the oracle's answer, and the server's tuner
chooses among them where both exist (64 < d <= 128)."""
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


@pytest.mark.parametrize("d,L", [(128, 2), (100, 2), (72, 1), (64, 2)])
def test_layouts_bit_identical(osann, d, L):
    rng = np.random.default_rng(d + 10 * L)
    X = rng.standard_normal((20_011, d)).astype(np.float32)
    Y = rng.standard_normal((300, d)).astype(np.float32)
    idx = osann.Index(to_dev(X), L)
    ref = oracle.Index(X, L)
    Yd = to_dev(Y)
    for P, k in ((24, 1), (40, 4)):
        oids, od = ref.search(Y, P, k)
        for path in ("fp16", "bf16"):
            res = [idx.search(Yd, P, k, path=path, layout=lay) for lay in ("default", "smem", "tmem")]
            for a in res[1:]:
                assert np.array_equal(to_np(a[0]), to_np(res[0][0]))
                assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(res[0][1]).view(np.uint32))
            assert_knn_match(X, Y, to_np(res[0][0]), to_np(res[0][1]), oids, od)
    with pytest.raises(KeyError):
        idx.search(Yd, 24, 1, layout="registers")
    assert idx.status() == 0
    idx.close()


def test_tuner_chooses_a_layout_where_both_exist(osann):
    rng = np.random.default_rng(128)
    X = rng.standard_normal((60_000, 128)).astype(np.float32)
    Z = rng.standard_normal((40_000, 32)).astype(np.float32)
    ia, ib = osann.Index(to_dev(X), 2), osann.Index(to_dev(Z), 2)
    srv = osann.Server([ia, ib], P=[48, 32], k=[1, 1], slots=1, max_batch=512)
    choices = srv.tune(reps=1)
    for i, per_index in enumerate(choices):
        for path, group, layout in per_index:
            if i == 0 and path == "fp16" and group == 128:
                assert layout in ("smem", "tmem")
            else:
                assert layout == "default"
    srv.close()
    ia.close()
    ib.close()
