"""Statistical pins of the oracle against numbers the paper states.

Each test draws iid Gaussian data (the paper's running example) and checks
a quantity the paper quotes; the tolerances are a few binomial or sampling
standard deviations of the estimate.
"""
import numpy as np

import oracle


def test_order_statistics_energy_share():
    """Fig. 5 (K=8 iid N(0,1), components sorted by decreasing magnitude):
    the first component holds 44% of the energy, the first four almost 90%."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((20000, 8)).astype(np.float32)
    order = np.array([oracle.magnitude_order(x) for x in X])
    e = np.take_along_axis(X.astype(np.float64) ** 2, order, axis=1).mean(axis=0)
    share = np.cumsum(e) / e.sum()
    assert 0.42 <= share[0] <= 0.45
    assert 0.88 <= share[3] <= 0.91
    assert np.all(np.diff(e) < 0)          # decreasing magnitude order


def _nn_study(n_queries=600):
    """K=16, log2 N = 16 (density rho = 1, Eq. 4), exact NN by linear search."""
    rng = np.random.default_rng(16)
    X = rng.standard_normal((1 << 16, 16)).astype(np.float32)
    Y = rng.standard_normal((n_queries, 16)).astype(np.float32)
    ids, _ = oracle.bruteforce(X, Y, 1)
    return X, Y, X[ids[:, 0]]


def test_classification_and_sign_agreement():
    """Sec. 3-C, Fig. 7 (one basis): the query's largest component is the
    NN's largest in just above 40% of cases; the signs of the query's first 3
    components almost surely agree with the NN's, about 60% for 8 of them,
    almost never for all 16."""
    X, Y, NN = _nn_study()
    q_order = np.array([oracle.magnitude_order(y) for y in Y])
    n_order = np.array([oracle.magnitude_order(x) for x in NN])
    p_f1g1 = np.mean(q_order[:, 0] == n_order[:, 0])
    assert 0.36 <= p_f1g1 <= 0.48

    def agree(G):
        idx = q_order[:, :G]
        sy = np.take_along_axis(Y, idx, 1) >= 0
        sx = np.take_along_axis(NN, idx, 1) >= 0
        return np.mean(np.all(sy == sx, axis=1))

    assert agree(3) >= 0.95
    assert 0.50 <= agree(8) <= 0.72
    assert agree(16) <= 0.08
    # the F=1 curve grows with G (query's top index among the NN's top G)
    f1 = [np.mean([q_order[i, 0] in n_order[i, :G] for i in range(len(Y))])
          for G in (1, 2, 3, 4)]
    assert all(a < b for a, b in zip(f1, f1[1:]))


def test_crossing_probability_bounds_k2_g1():
    """Appendix, 2-d case (K = 2, G = 1, iid standard Gaussian X, Y uniform on
    the circle of radius r around X): the probability that Y lies in another
    cone than X is at least the mean of theta(r, Delta)/pi over Delta < r
    (Delta the distance of X to its nearest cone boundary, theta =
    arccos(Delta/r)), at most the mean of min(2 theta/pi, (N_C-1)/N_C), close
    to the lower bound for small r and tends to 3/4 as r grows (N_C = 4)."""
    rng = np.random.default_rng(21)
    n = 200_000
    X = rng.standard_normal((n, 2))
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    a = np.abs(X)
    delta = (a.max(1) - a.min(1)) / np.sqrt(2.0)
    kx = oracle.keys(X.astype(np.float32), 1)
    assert oracle.num_cones(2, 1) == 4 and set(np.unique(kx)) == {0, 1, 2, 3}
    se = lambda p: np.sqrt(p * (1 - p) / n)
    for r in (0.05, 0.3, 1.0, 3.0, 100.0):
        Y = X + r * np.stack([np.cos(phi), np.sin(phi)], 1)
        p = np.mean(oracle.keys(Y.astype(np.float32), 1) != kx)
        theta = np.where(delta < r, np.arccos(np.minimum(delta / r, 1.0)), 0.0)
        lower = np.mean(theta / np.pi)
        upper = np.mean(np.minimum(2.0 * theta / np.pi, 3.0 / 4.0))
        tol = 5 * se(max(p, 1e-4)) + 1e-4
        assert lower - tol <= p <= upper + tol, (r, lower, p, upper)
        if r <= 0.05:
            assert p - lower <= 0.1 * lower + tol  # the nearest boundary dominates
    assert abs(p - 0.75) <= 5 * se(0.75) + 0.005  # r = 100: any cone alike
