"""Host-side preparation that the library takes as inputs: PCA axes for the
front-end of Sec. 4-B and the seeded random rotations of Sec. 3-D."""
import numpy as np

from paper_1509_03453_gb300 import datagen
from paper_1509_03453_gb300.pca import pca_basis


def test_pca_axes_orthonormal_ordered_and_centred():
    rng = np.random.default_rng(3)
    d = 12
    scales = np.linspace(5.0, 0.5, d)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    X = ((rng.standard_normal((20000, d)) * scales) @ Q.T + 3.0).astype(np.float32)
    A, off = pca_basis(X, 4, seed=1)
    assert A.shape == (4, d) and off.shape == (4,)
    assert np.allclose(A.astype(np.float64) @ A.T.astype(np.float64), np.eye(4), atol=1e-5)
    # the leading axes are the directions of the largest spreads, in order
    for j in range(4):
        assert abs(abs(float(A[j].astype(np.float64) @ Q[:, j])) - 1.0) < 1e-2
    # a deterministic sign: the largest-magnitude entry of every axis is positive
    assert np.all(A[np.arange(4), np.abs(A).argmax(1)] > 0)
    # the offsets centre the projected coordinates
    proj = X.astype(np.float64) @ A.T.astype(np.float64) - off
    assert np.all(np.abs(proj.mean(0)) < 0.05 * proj.std(0))
    # seeded: the same sample and axes twice
    A2, off2 = pca_basis(X, 4, seed=1)
    assert np.array_equal(A, A2) and np.array_equal(off, off2)


def test_rotations_orthonormal_identity_first_and_seeded():
    R = datagen.rotations(4, 16, 9)
    assert R.shape == (4, 16, 16)
    assert np.array_equal(R[0], np.eye(16, dtype=np.float32))
    for r in R:
        assert np.allclose(r.astype(np.float64) @ r.T.astype(np.float64), np.eye(16), atol=1e-5)
    assert np.array_equal(R, datagen.rotations(4, 16, 9))
    assert not np.allclose(R[1], R[2])
