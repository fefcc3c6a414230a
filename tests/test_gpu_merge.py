"""Row-sharded search on one GPU: shards built over row blocks, searched,
and merged by the CUDA merge, equal the unsharded search bit for bit."""
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


@pytest.mark.parametrize("G,k,path", [(2, 1, "auto"), (3, 4, "plain"), (4, 10, "batched"), (2, 3, "fp16")])
def test_sharded_equals_unsharded(osann, G, k, path):
    import torch
    from paper_1509_03453_gb300.shard import shard_rows, to_global
    rng = np.random.default_rng(31 + G)
    X = rng.standard_normal((40_003, 32)).astype(np.float32)
    Y = rng.standard_normal((700, 32)).astype(np.float32)
    P = 40
    Xd, Yd = to_dev(X), to_dev(Y)
    full = osann.Index(Xd, 2)
    f_ids, f_d = full.search(Yd, P, k, path=path)
    ids, ds = [], []
    for r in range(G):
        lo, hi = shard_rows(X.shape[0], r, G)
        ix = osann.Index(Xd[lo:hi].contiguous(), 2)
        i, d = ix.search(Yd, P, k, path=path)
        ids.append(to_global(i, lo))
        ds.append(d)
        ix.close()
    m_ids, m_d = osann.merge_topk(torch.stack(ids), torch.stack(ds))
    assert np.array_equal(to_np(m_ids), to_np(f_ids))
    assert np.array_equal(to_np(m_d).view(np.uint32), to_np(f_d).view(np.uint32))


def test_merge_padding(osann):
    import torch
    ids = torch.tensor([[[3, -1]], [[-1, -1]], [[7, 2]]], dtype=torch.int64, device="cuda")
    d = torch.tensor([[[1.0, float("inf")]], [[float("inf")] * 2], [[1.0, 0.5]]], device="cuda")
    m_ids, m_d = osann.merge_topk(ids, d)
    assert to_np(m_ids).tolist() == [[2, 3]]
    assert to_np(m_d).tolist() == [[0.5, 1.0]]
    ids = torch.full((2, 1, 3), -1, dtype=torch.int64, device="cuda")
    d = torch.full((2, 1, 3), float("inf"), device="cuda")
    m_ids, m_d = osann.merge_topk(ids, d)
    assert to_np(m_ids).tolist() == [[-1, -1, -1]]
    assert np.isinf(to_np(m_d)).all()
