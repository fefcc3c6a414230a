"""osann_rebuild: an index rebuilt in place from new data of the same shape
equals a fresh build on that data (keys, cone table, permutation, results on
every path), for every table kind and key basis; a rebuild and a search
captured in one CUDA graph replay to the same bits; a rebuild reports
non-finite data through the status word."""
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


def _kwargs(kind, d, X):
    import torch
    from paper_1509_03453_gb300 import datagen
    from paper_1509_03453_gb300.kmeans import kmeans
    from paper_1509_03453_gb300.pca import pca_basis
    if kind == "rot":
        return dict(rot=torch.from_numpy(datagen.rotations(2, d, 4)[1]).cuda())
    if kind == "pca":
        A, off = pca_basis(X, 8, seed=1)
        return dict(rot=torch.from_numpy(A).cuda(), rot_offset=torch.from_numpy(off).cuda())
    if kind == "clusters":
        return dict(centroids=torch.from_numpy(kmeans(X, 12, iters=4, seed=2)).cuda())
    if kind == "hashed":
        return dict(cone_table="hashed")
    return {}


@pytest.mark.parametrize("kind", ["plain", "hashed", "rot", "pca", "clusters"])
def test_rebuild_equals_fresh_build(osann, kind):
    d, L = 32, 2
    rng = np.random.default_rng(11)
    X0 = rng.standard_normal((30000, d)).astype(np.float32)
    X1 = (rng.standard_normal((30000, d)) * 1.5 + 0.2).astype(np.float32)  # other data, other scale
    Y = rng.standard_normal((1500, d)).astype(np.float32)
    kw = _kwargs(kind, d, X0)
    ix = osann.Index(to_dev(X0), L, **kw)
    ix.search(to_dev(Y), 32, 2, path="bf16")          # bf16 operands exist before the rebuild
    for X in (X1, X0, X1):
        ix.rebuild(to_dev(X))
        assert ix.status() == 0
        ref = osann.Index(to_dev(X), L, **kw)
        for a, b in zip(ix.export(), ref.export()):
            assert np.array_equal(to_np(a), to_np(b))
        for path in ("plain", "batched", "fp16", "bf16"):
            _same(ix.search(to_dev(Y), 32, 2, path=path), ref.search(to_dev(Y), 32, 2, path=path))
        ref.close()
    ix.close()


def test_rebuild_and_search_in_one_graph(osann):
    import torch
    d, L, P, k = 32, 2, 96, 1
    rng = np.random.default_rng(12)
    Xs = [rng.standard_normal((50000, d)).astype(np.float32) for _ in range(3)]
    Ys = [rng.standard_normal((4000, d)).astype(np.float32) for _ in range(3)]
    s = torch.cuda.Stream()
    xbuf, ybuf = to_dev(Xs[0]), to_dev(Ys[0])
    ix = osann.Index(xbuf, L)
    ids = torch.empty((4000, k), dtype=torch.int64, device="cuda")
    d2 = torch.empty((4000, k), dtype=torch.float32, device="cuda")
    ws = torch.empty(ix.workspace_size(4000, P, k, "fp16"), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        ix.rebuild(xbuf, stream=s)                    # allocates the rebuild's temporaries
        ix.search(ybuf, P, k, path="fp16", out=(ids, d2), workspace=ws, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        ix.rebuild(xbuf, stream=s)
        ix.search(ybuf, P, k, path="fp16", out=(ids, d2), workspace=ws, stream=s)
    for X, Y in zip(Xs[1:] + Xs[:1], Ys[1:] + Ys[:1]):
        xbuf.copy_(to_dev(X))
        ybuf.copy_(to_dev(Y))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        ref = osann.Index(to_dev(X), L)
        _same((ids, d2), ref.search(to_dev(Y), P, k, path="fp16"))
        ref.close()
    assert ix.status() == 0
    ix.close()


def test_rebuild_reports_nonfinite_data(osann):
    rng = np.random.default_rng(13)
    X = rng.standard_normal((4000, 16)).astype(np.float32)
    ix = osann.Index(to_dev(X), 2)
    bad = X.copy()
    bad[7, 3] = np.inf
    ix.rebuild(to_dev(bad))
    assert ix.status() & 1
    ix.rebuild(to_dev(X))
    assert ix.status() == 0
    with pytest.raises(ValueError):
        ix.rebuild(to_dev(X[:100]))
    ix.close()


@pytest.mark.parametrize("path", ["fp16", "batched", "plain"])
def test_rebuild_search_graph(osann, path):
    """osann_rebuild_search (query side beside the rebuild), eagerly and as
    one captured graph, against a fresh build and search."""
    import torch
    d, L, P, k = 32, 2, 64, 3
    rng = np.random.default_rng(14)
    Xs = [rng.standard_normal((40000, d)).astype(np.float32) for _ in range(3)]
    Ys = [rng.standard_normal((3000, d)).astype(np.float32) for _ in range(3)]
    s = torch.cuda.Stream()
    xbuf, ybuf = to_dev(Xs[0]), to_dev(Ys[0])
    ix = osann.Index(xbuf, L)
    ids = torch.empty((3000, k), dtype=torch.int64, device="cuda")
    d2 = torch.empty((3000, k), dtype=torch.float32, device="cuda")
    ws = torch.empty(ix.workspace_size(3000, P, k, path), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        ix.rebuild_search(xbuf, ybuf, P, k, path=path, out=(ids, d2), workspace=ws, stream=s)
    s.synchronize()
    ref = osann.Index(xbuf, L)
    _same((ids, d2), ref.search(ybuf, P, k, path=path))
    ref.close()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        ix.rebuild_search(xbuf, ybuf, P, k, path=path, out=(ids, d2), workspace=ws, stream=s)
    for X, Y in zip(Xs[1:] + Xs[:1], Ys[1:] + Ys[:1]):
        xbuf.copy_(to_dev(X))
        ybuf.copy_(to_dev(Y))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        ref = osann.Index(to_dev(X), L)
        _same((ids, d2), ref.search(to_dev(Y), P, k, path=path))
        ref.close()
    assert ix.status() == 0
    ix.close()
