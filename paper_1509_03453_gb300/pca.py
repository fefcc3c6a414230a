"""Principal axes for the PCA front-end (Sec. 4-B): keys and query orders on
the first m principal components, search on all components.

Host-side preparation of the projection that osann_build_proj takes as an
input (computed once per dataset, like the random rotations of the
multi-basis search): the covariance of a seeded row sample in fp64, its
eigenvectors by decreasing eigenvalue, and the projected sample mean as the
offset (so the projected coordinates are centred).
"""
from __future__ import annotations

import numpy as np


def pca_basis(X, m: int, sample: int = 200_000, seed: int = 0):
    """(axes float32 [m, d], offset float32 [m]) of the rows of X (numpy)."""
    X = np.asarray(X)
    n, d = X.shape
    if not 1 <= m <= d:
        raise ValueError("need 1 <= m <= d")
    rng = np.random.default_rng(seed)
    idx = rng.choice(n, size=min(n, sample), replace=False) if n > sample else np.arange(n)
    S = X[idx].astype(np.float64)
    mu = S.mean(0)
    C = (S - mu).T @ (S - mu) / max(1, S.shape[0] - 1)
    w, V = np.linalg.eigh(C)
    axes = V[:, np.argsort(w)[::-1][:m]].T  # rows = principal axes
    # a deterministic sign per axis: the largest-magnitude entry positive
    sgn = np.sign(axes[np.arange(m), np.abs(axes).argmax(1)])
    axes = (axes * sgn[:, None]).astype(np.float32)
    offset = (axes.astype(np.float64) @ mu).astype(np.float32)
    return axes, offset
