"""Shared test utilities: device placement and the parity contract.

Tolerance contract (fp32 kernels vs the fp64 oracle):
  * keys, offsets, permutations, probe lists, candidate sets: bit-exact;
  * a returned distance is within 1e-5 relative of the fp64 distance of the
    same (query, id) pair (absolute floor 1e-7 * |q|^2 for exact duplicates);
  * ids agree rank by rank, except where the fp64 distances of the two ids
    differ by at most 1e-6 relative (a near-tie the fp32 rounding may order
    either way).
The 1e-5 bound follows from the arithmetic: all terms are nonnegative, each
squared difference carries the rounding of the subtraction (twice, once per
factor) and of its fused multiply-add, the 4-term chain adds up to 3 more and
the pairwise tree log2(d_pad/4), so the relative error stays below
(5 + log2(d_pad/4)) * 2^-24, about 6.6e-7 for d_pad <= 256.
"""
import numpy as np

import oracle

REL_D = 1e-5
REL_GAP = 1e-6


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_np(t):
    return t.detach().cpu().numpy()


def assert_knn_match(X, Y, gids, gd, oids, od, rel_d=REL_D, rel_gap=REL_GAP):
    """GPU (gids, gd fp32) against oracle (oids, od fp64) under the contract."""
    gids = np.asarray(gids, np.int64)
    gd = np.asarray(gd, np.float64)
    oids = np.asarray(oids, np.int64)
    od = np.asarray(od, np.float64)
    assert gids.shape == oids.shape
    # same number of results per query (padding -1 / +inf)
    assert np.array_equal(gids < 0, oids < 0), "result counts differ"
    assert np.all(np.isinf(gd[gids < 0]))
    d64 = oracle.pair_dists(X, Y, np.where(gids < 0, 0, gids))
    d64 = np.where(gids < 0, np.inf, d64)
    qn2 = (np.asarray(Y, np.float64) ** 2).sum(1)[:, None] * np.ones_like(d64)
    valid = gids >= 0
    floor = 1e-7 * qn2
    err = np.where(valid, np.abs(np.where(valid, gd, 0.0) - np.where(valid, d64, 0.0)), 0.0)
    bad = valid & (err > rel_d * d64 + floor)
    assert not bad.any(), f"distance error: {np.argwhere(bad)[:5]} gpu={gd[bad][:5]} fp64={d64[bad][:5]}"
    mism = valid & (gids != oids)
    if mism.any():
        gap = np.abs(d64[mism] - od[mism])
        tie = gap <= rel_gap * od[mism] + 1e-12 * qn2[mism]
        assert tie.all(), (f"{(~tie).sum()} id mismatches beyond the tie window: "
                           f"gpu={gids[mism][~tie][:5]} oracle={oids[mism][~tie][:5]} "
                           f"gap={gap[~tie][:5]} od={od[mism][~tie][:5]}")
    # no duplicate ids within a query
    for row in gids:
        r = row[row >= 0]
        assert len(np.unique(r)) == len(r)


def recall_at_1(gids, truth_ids, X, Y, truth_d):
    """Fraction of queries whose top-1 is the true NN (near-ties accepted)."""
    hit = gids[:, 0] == truth_ids[:, 0]
    miss = ~hit & (gids[:, 0] >= 0)
    if miss.any():
        d64 = oracle.pair_dists(X, Y[miss], gids[miss][:, :1])[:, 0]
        hit[miss] = np.abs(d64 - truth_d[miss, 0]) <= REL_GAP * truth_d[miss, 0]
    return float(hit.mean())
