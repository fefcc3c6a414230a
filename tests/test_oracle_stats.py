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
