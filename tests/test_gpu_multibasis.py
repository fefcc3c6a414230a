"""Multi-basis search (Sec. 3-D, Algorithm 1 with R bases) on the GPU against
the oracle: per-basis keys and buckets bit-exact (the rotated coordinates
are computed in the same fp32 order on both sides), results within the
distance contract of the exact top-k over the union of the bases' probed
cones, and R = 1 on the identity basis equal to the single-basis index;
with random (QR) and structured Walsh-Hadamard bases."""
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
    yield m


@pytest.mark.parametrize("d,L,R,P,k,kind", [(16, 2, 3, 8, 1, "qr"), (32, 2, 4, 16, 4, "qr"), (64, 3, 2, 32, 10, "qr"),
                                             (13, 2, 3, 6, 2, "qr"), (32, 2, 3, 16, 1, "wht"),
                                             (128, 3, 2, 24, 4, "wht")])
def test_multibasis_matches_oracle(osann, d, L, R, P, k, kind):
    """Random (QR) and structured Walsh-Hadamard ("wht") bases."""
    from paper_1509_03453_gb300 import datagen
    rng = np.random.default_rng(100 + d)
    X = rng.standard_normal((20_000, d)).astype(np.float32)
    Y = rng.standard_normal((400, d)).astype(np.float32)
    rots = datagen.rotations(R, d, 7 + d) if kind == "qr" else datagen.hadamard_rotations(R, d, 7 + d)
    mi = osann.MultiIndex(to_dev(X), L, rots)
    om = oracle.MultiIndex(X, L, rots)
    for r, ix in enumerate(mi.bases):
        keys, offs, perm = (to_np(t) for t in ix.export())
        assert np.array_equal(keys, oracle.keys(oracle.rotate(rots[r], X), L))
        assert np.array_equal(offs, om.offsets[r])
        assert np.array_equal(perm, om.perms[r])
        # the query's probe list on this basis
        pr = to_np(ix.probes(to_dev(Y[:50]), P))
        for q in range(50):
            yr = oracle.rotate(rots[r], Y[q:q + 1])[0]
            assert np.array_equal(pr[q], oracle.probes(yr, L, P))
    ids, d2 = mi.search(to_dev(Y), P, k)
    oids, od = om.search(Y, P, k)
    assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
    # every path, the same bits
    for path in ("plain", "batched"):
        pi, pd = mi.search(to_dev(Y), P, k, path=path)
        assert np.array_equal(to_np(pi), to_np(ids))
        assert np.array_equal(to_np(pd).view(np.uint32), to_np(d2).view(np.uint32))
    mi.close()


def test_identity_basis_is_the_single_index(osann):
    from paper_1509_03453_gb300 import datagen
    rng = np.random.default_rng(3)
    X = rng.standard_normal((30_000, 32)).astype(np.float32)
    Y = rng.standard_normal((500, 32)).astype(np.float32)
    mi = osann.MultiIndex(to_dev(X), 2, datagen.rotations(1, 32, 0))
    ix = osann.Index(to_dev(X), 2)
    a = mi.search(to_dev(Y), 24, 3)
    b = ix.search(to_dev(Y), 24, 3)
    assert np.array_equal(to_np(a[0]), to_np(b[0]))
    assert np.array_equal(to_np(a[1]).view(np.uint32), to_np(b[1]).view(np.uint32))
    mi.close()
    ix.close()


def test_merge_drops_repeated_points(osann):
    import torch
    ids = torch.tensor([[[0, 5, 9]], [[0, 5, 7]], [[5, 0, 8]]], dtype=torch.int64, device="cuda")
    d = torch.tensor([[[0.0, 1.0, 3.0]], [[0.0, 1.0, 2.0]], [[1.0, 0.0, 4.0]]], device="cuda")
    m_ids, m_d = osann.merge_topk(ids, d)
    assert to_np(m_ids).tolist() == [[0, 5, 7]]
    assert to_np(m_d).tolist() == [[0.0, 1.0, 2.0]]


@pytest.mark.parametrize("d,m,L,P,k", [(64, 16, 3, 24, 4), (128, 16, 3, 32, 10), (40, 9, 2, 8, 1)])
def test_pca_front_end_matches_oracle(osann, d, m, L, P, k):
    from paper_1509_03453_gb300.pca import pca_basis
    rng = np.random.default_rng(200 + d)
    A = rng.standard_normal((d, d)).astype(np.float32)
    X = (rng.standard_normal((30_000, d)).astype(np.float32) @ A) + 3.0
    Y = (rng.standard_normal((300, d)).astype(np.float32) @ A) + 3.0
    X, Y = X.astype(np.float32), Y.astype(np.float32)
    axes, off = pca_basis(X, m, seed=2)
    ix = osann.Index(to_dev(X), L, rot=to_dev(axes), rot_offset=to_dev(off))
    om = oracle.MultiIndex(X, L, axes[None], off[None])
    assert ix.NC == oracle.num_cones(m, L)
    keys, offs, perm = (to_np(t) for t in ix.export())
    assert np.array_equal(keys, oracle.keys(oracle.project(axes, X, off), L))
    assert np.array_equal(offs, om.offsets[0])
    assert np.array_equal(perm, om.perms[0])
    ids, d2 = ix.search(to_dev(Y), P, k)
    oids, od = om.search(Y, P, k)
    assert_knn_match(X, Y, to_np(ids), to_np(d2), oids, od)
    for path in ("plain", "batched", "fp16"):
        pi, pd = ix.search(to_dev(Y), P, k, path=path)
        assert np.array_equal(to_np(pi), to_np(ids))
        assert np.array_equal(to_np(pd).view(np.uint32), to_np(d2).view(np.uint32))
    ix.close()
