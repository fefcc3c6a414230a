"""Seeded synthetic workloads (numpy only).

This module holds none of the search method's arithmetic: it only draws the
data and query vectors that both the CUDA path and the CPU oracle consume.
All draws use ``numpy.random.default_rng(seed)`` (PCG64).

Workloads (seeds: data 1000 + n, queries 2000 + n):

* ``gauss16``  -- N=10,000 data / 1,000 queries, d=16, iid N(0,1) (the
  paper's running example of iid Gaussian data, Sec. 3-C and Sec. 4-A).
* ``gauss32``  -- N=1,000,000 / 10,000, d=32, iid N(0,1).
* ``patch64``  -- all 8x8 patches (d=64, mean removed) of a 1024x1024 image
  with a 1/f^2 power spectrum plus uniform noise (sigma 0.02); 20,000 query
  patches at distinct random positions, searched with self/near exclusion.
  Stands in for the copy-move forgery detection workload of Sec. 4-C.
* ``desc128``  -- N=2,000,000 / 10,000, d=128 nonnegative descriptor-like
  vectors: Gamma(0.5, scale 20) clipped to [0,255], L2-normalised to 512 and
  rounded half-to-even; queries are fresh draws plus N(0, sigma=2) noise,
  clipped to [0,512].  Stands in for the SIFT sets of Sec. 4-B.
"""
from __future__ import annotations

import numpy as np

PATCH_IMAGE = 1024
PATCH_SIZE = 8
PATCH_GRID_W = PATCH_IMAGE - PATCH_SIZE + 1      # 1017 patch positions per row
PATCH_RADIUS = 8                                  # exclusion: Chebyshev <= 8


def gaussian(n: int, d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d), dtype=np.float32)


def patch_image(seed: int, size: int = PATCH_IMAGE) -> np.ndarray:
    """Grayscale image with a 1/f^2 power spectrum (amplitude 1/f, DC = 0),
    min-max scaled to [0,1], plus uniform noise of standard deviation 0.02."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((size, size))
    spec = np.fft.fft2(white)
    fy = np.fft.fftfreq(size)[:, None]
    fx = np.fft.fftfreq(size)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    amp = np.zeros_like(f)
    amp[f > 0] = 1.0 / f[f > 0]
    img = np.real(np.fft.ifft2(spec * amp))
    img = (img - img.min()) / (img.max() - img.min())
    half = 0.02 * np.sqrt(3.0)
    img = img + rng.uniform(-half, half, size=img.shape)
    return img.astype(np.float32)


def patches(img: np.ndarray, p: int = PATCH_SIZE) -> np.ndarray:
    """All overlapping p x p patches, row-major by position, each flattened
    row-major and mean-removed.  Patch id n sits at (n // W, n % W) with
    W = img width - p + 1."""
    h, w = img.shape
    view = np.lib.stride_tricks.sliding_window_view(img, (p, p))
    X = np.ascontiguousarray(view.reshape((h - p + 1) * (w - p + 1), p * p),
                             dtype=np.float32)
    X -= X.mean(axis=1, keepdims=True, dtype=np.float64).astype(np.float32)
    return X


def descriptors(n: int, seed: int, d: int = 128, chunk: int = 1 << 18) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.empty((n, d), np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = _descriptor_rows(rng, e - s, d)
    return out


def _descriptor_rows(rng, n, d):
    g = np.clip(rng.gamma(0.5, 20.0, size=(n, d)), 0.0, 255.0)
    nrm = np.sqrt((g * g).sum(axis=1, keepdims=True))
    g = np.where(nrm > 0, g * (512.0 / np.where(nrm > 0, nrm, 1.0)), 0.0)
    return np.rint(g).astype(np.float32)


def descriptor_queries(q: int, seed: int, d: int = 128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    base = _descriptor_rows(rng, q, d).astype(np.float64)
    noisy = base + rng.normal(0.0, 2.0, size=base.shape)
    return np.clip(noisy, 0.0, 512.0).astype(np.float32)


def rotations(R: int, d: int, seed: int) -> np.ndarray:
    """R orthonormal d x d bases (float32, row i = basis vector i) for the
    multi-basis search: basis 0 is the identity, the others are random
    rotations (QR of a Gaussian matrix, signs fixed by the diagonal of R)."""
    rng = np.random.default_rng(seed)
    out = np.empty((R, d, d), np.float32)
    out[0] = np.eye(d, dtype=np.float32)
    for r in range(1, R):
        a = rng.standard_normal((d, d))
        q, t = np.linalg.qr(a)
        q = q * np.sign(np.diag(t))[None, :]
        out[r] = q.T.astype(np.float32)
    return out


def hadamard_rotations(R: int, d: int, seed: int) -> np.ndarray:
    """R structured orthonormal d x d bases (float32, row i = basis vector
    i) for the multi-basis search: basis 0 is the identity, basis r > 0 is
    H D_r / sqrt(d) with H the Sylvester-Hadamard matrix (entry (i, j) =
    (-1)^popcount(i & j)) and D_r a diagonal of random signs -- the cheap
    structured rotation (Walsh-Hadamard) the paper suggests instead of a
    dense random one.  d must be a power of two."""
    if d < 1 or d & (d - 1):
        raise ValueError("a Walsh-Hadamard basis needs d a power of two")
    rng = np.random.default_rng(seed)
    i = np.arange(d)
    pc = np.vectorize(lambda v: bin(int(v)).count("1"))(i[:, None] & i[None, :])
    H = np.where(pc % 2 == 0, 1.0, -1.0)
    out = np.empty((R, d, d), np.float32)
    out[0] = np.eye(d, dtype=np.float32)
    for r in range(1, R):
        s = rng.choice(np.array([-1.0, 1.0]), size=d)
        out[r] = (H * s[None, :] / np.sqrt(d)).astype(np.float32)
    return out


def workload(name: str, n: int | None = None, q: int | None = None) -> dict:
    """Named workload.  ``n``/``q`` shrink it (same recipe, prefix of the
    draws for Gaussian data) for tests that need a smaller case."""
    if name == "gauss16":
        N, Q = n or 10_000, q or 1_000
        return dict(name=name, X=gaussian(N, 16, 1001), Y=gaussian(Q, 16, 2001),
                    L=2, P=[1, 4, 16], k=1)
    if name == "gauss32":
        N, Q = n or 1_000_000, q or 10_000
        return dict(name=name, X=gaussian(N, 32, 1002), Y=gaussian(Q, 32, 2002),
                    L=2, P=[1, 4, 16, 64], k=1)
    if name == "patch64":
        img = patch_image(1003, PATCH_IMAGE)
        X = patches(img)
        Q = q or 20_000
        rng = np.random.default_rng(2003)
        src = np.sort(rng.choice(X.shape[0], size=Q, replace=False)).astype(np.int64)
        return dict(name=name, X=X, Y=X[src].copy(), L=3, P=[4, 16, 64], k=4,
                    query_src=src, grid_w=PATCH_GRID_W, radius=PATCH_RADIUS)
    if name == "desc128":
        N, Q = n or 2_000_000, q or 10_000
        return dict(name=name, X=descriptors(N, 1004), Y=descriptor_queries(Q, 2004),
                    L=3, P=[8, 32, 128], k=10)
    raise KeyError(name)
