"""Centroids for ROSANNA+ (Sec. 4-B: the data are clustered off line by
k-means, and a query searches only its nearest clusters).

Host-side preparation of the centroids that osann_build_ex takes as an input
(computed once per dataset, like the PCA axes and the random rotations):
Lloyd's iterations in fp64 on a seeded row sample, seeded k-means++
initialisation, an empty cluster re-seeded with the sample point farthest
from its centroid.
"""
from __future__ import annotations

import numpy as np


def _sqdist(S, C):
    # |s|^2 - 2 s.c + |c|^2, fp64, clipped at 0
    d = (S * S).sum(1)[:, None] - 2.0 * (S @ C.T) + (C * C).sum(1)[None, :]
    return np.maximum(d, 0.0)


def kmeans(X, K: int, iters: int = 20, sample: int = 100_000, seed: int = 0) -> np.ndarray:
    """float32 [K, d] centroids of the rows of X (numpy)."""
    X = np.asarray(X)
    n, d = X.shape
    if not 1 <= K <= n:
        raise ValueError("need 1 <= K <= number of rows")
    rng = np.random.default_rng(seed)
    idx = rng.choice(n, size=min(n, sample), replace=False) if n > sample else np.arange(n)
    S = X[idx].astype(np.float64)
    # k-means++ seeding
    C = np.empty((K, d))
    C[0] = S[rng.integers(S.shape[0])]
    best = _sqdist(S, C[:1])[:, 0]
    for j in range(1, K):
        tot = best.sum()
        pick = rng.choice(S.shape[0], p=best / tot) if tot > 0 else rng.integers(S.shape[0])
        C[j] = S[pick]
        best = np.minimum(best, _sqdist(S, C[j:j + 1])[:, 0])
    for _ in range(iters):
        D = _sqdist(S, C)
        a = D.argmin(1)
        far = D[np.arange(S.shape[0]), a]
        for j in range(K):
            m = a == j
            if m.any():
                C[j] = S[m].mean(0)
            else:
                i = int(far.argmax())
                C[j] = S[i]
                far[i] = 0.0
    return C.astype(np.float32)
