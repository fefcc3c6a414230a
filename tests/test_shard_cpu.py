"""Row-sharded search among CPU ranks (gloo, world size 2).

The host logic of the sharded path -- row blocks, local-to-global ids, the
all-gather of every rank's k-best lists and their merge -- must reproduce
the unsharded search.  Each rank's local search is the oracle (CPU); the
merge here is a plain lexsort by (distance, id).
"""
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
dist = torch.distributed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class _OracleIndex:
    def __init__(self, X, L):
        self.o = oracle.Index(np.asarray(X), L)

    def search(self, Y, P, k):
        ids, d = self.o.search(np.asarray(Y), P, k)
        return torch.from_numpy(ids), torch.from_numpy(d)


def _merge_lexsort(gi, gd):
    G, Q, k = gi.shape
    ids = gi.permute(1, 0, 2).reshape(Q, G * k).numpy()
    d = gd.permute(1, 0, 2).reshape(Q, G * k).numpy()
    out_i = np.full((Q, k), -1, np.int64)
    out_d = np.full((Q, k), np.inf)
    for q in range(Q):
        live = ids[q] >= 0
        order = np.lexsort((ids[q][live], d[q][live]))[:k]
        out_i[q, :len(order)] = ids[q][live][order]
        out_d[q, :len(order)] = d[q][live][order]
    return torch.from_numpy(out_i), torch.from_numpy(out_d)


def _worker(rank, world, port, X, Y, L, P, k, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1509_03453_gb300.shard import ShardedIndex, shard_rows
    lo, hi = shard_rows(X.shape[0], rank, world)
    sh = ShardedIndex(X[lo:hi], L, lo, index_factory=_OracleIndex, merge=_merge_lexsort)
    ids, d = sh.search(Y, P, k)
    if rank == 0:
        out.put((ids.numpy(), d.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_rows_partition():
    from paper_1509_03453_gb300.shard import shard_rows
    for N in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            blocks = [shard_rows(N, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == N
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("k", [1, 4])
def test_two_rank_sharded_search_equals_unsharded(k):
    import multiprocessing as mp
    rng = np.random.default_rng(21)
    X = rng.standard_normal((3001, 16)).astype(np.float32)
    Y = rng.standard_normal((60, 16)).astype(np.float32)
    L, P = 2, 24
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, X, Y, L, P, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    ids, d = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    full_ids, full_d = oracle.Index(X, L).search(Y, P, k)
    assert np.array_equal(ids, full_ids)
    assert np.array_equal(d, full_d)


def _worker_drop(rank, world, port, X, Y, L, P, k, out):
    """Rank 1 leaves before the exchange (between steps, nothing of its own in
    flight); rank 0's all-gather must end with an error, not wait forever."""
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    from paper_1509_03453_gb300.shard import ShardedIndex, shard_rows
    lo, hi = shard_rows(X.shape[0], rank, world)
    sh = ShardedIndex(X[lo:hi], L, lo, index_factory=_OracleIndex, merge=_merge_lexsort)
    dist.barrier()
    if rank == 1:
        os._exit(0)  # the rank is gone: no search, no collective
    try:
        sh.search(Y, P, k)
        out.put("no error")
    except Exception as exc:  # the peer's loss surfaces as an error on the collective
        out.put("error: " + type(exc).__name__)
    # flush the queue's feeder thread before leaving without the group's teardown
    out.close()
    out.join_thread()
    os._exit(0)


def test_dropped_rank_fails_the_exchange_instead_of_hanging():
    import multiprocessing as mp
    import time
    rng = np.random.default_rng(22)
    X = rng.standard_normal((2001, 16)).astype(np.float32)
    Y = rng.standard_normal((20, 16)).astype(np.float32)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_drop, args=(r, 2, port, X, Y, 2, 8, 1, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert res.startswith("error"), res
    assert time.time() - t0 < 100
