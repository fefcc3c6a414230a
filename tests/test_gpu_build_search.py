"""osann_build_search: one call that builds an index and searches it, with the
query-side steps beside the build.  Same bits as a build followed by a
search, on every path and table kind; the build's errors reported with a
synchronous call; the search's own status flags kept for osann_status."""
import numpy as np
import pytest

from helpers import to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osann():
    import paper_1509_03453_gb300 as m
    from paper_1509_03453_gb300 import build
    build.build()
    m.load()
    yield m


def _same(a, b):
    assert np.array_equal(to_np(a[0]), to_np(b[0]))
    assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(b[1]).view(np.uint32))


@pytest.mark.parametrize("path", ["auto", "plain", "batched", "fp16", "bf16"])
@pytest.mark.parametrize("sync", [True, False])
def test_equals_build_then_search(osann, path, sync):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((60000, 32)).astype(np.float32)
    Y = rng.standard_normal((3000, 32)).astype(np.float32)
    ref_ix = osann.Index(to_dev(X), 2)
    ref = ref_ix.search(to_dev(Y), 96, 3, path=path)
    ix, ids, d2 = osann.build_search(to_dev(X), 2, to_dev(Y), 96, 3, path=path, sync=sync)
    if not sync:
        assert ix.status() == 0
    _same(ref, (ids, d2))
    # the index is an ordinary index afterwards
    _same(ref_ix.search(to_dev(Y[:100]), 40, 1), ix.search(to_dev(Y[:100]), 40, 1))
    assert np.array_equal(to_np(ix.export()[2]), to_np(ref_ix.export()[2]))
    ix.close()
    ref_ix.close()


def test_second_level_table_and_odd_sizes(osann):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((7001, 30)).astype(np.float32)   # d % 4 != 0
    Y = rng.standard_normal((333, 30)).astype(np.float32)
    for table in ("dense", "hashed"):
        ref_ix = osann.Index(to_dev(X), 3, cone_table=table)
        ref = ref_ix.search(to_dev(Y), 50, 4)
        ix, ids, d2 = osann.build_search(to_dev(X), 3, to_dev(Y), 50, 4, cone_table=table)
        assert ix.hashed == (table == "hashed")
        _same(ref, (ids, d2))
        ix.close()
        ref_ix.close()


def test_errors_and_flags(osann):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((5000, 16)).astype(np.float32)
    Y = rng.standard_normal((50, 16)).astype(np.float32)
    bad = X.copy()
    bad[10, 2] = np.nan
    with pytest.raises(osann.OsannError) as e:
        osann.build_search(to_dev(bad), 2, to_dev(Y), 8, 1)
    assert e.value.code == -4
    q = Y.copy()
    q[3, 0] = np.inf
    ix, _, _ = osann.build_search(to_dev(X), 2, to_dev(q), 8, 1)
    assert ix.status() & 2          # the non-finite query is still reported
    assert ix.status() == 0
    ix.close()
