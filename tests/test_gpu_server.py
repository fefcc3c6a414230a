"""Request server: continuous batching over resident indexes.

Every request's answer must be the same alone (one osann_search call on its
own queries) and in the mix (batched with other requests, split across
batches, run as a graph replay or directly, tuned or not), bit for bit.
"""
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


@pytest.fixture(scope="module")
def setup(osann):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(77)
    XA = rng.standard_normal((20_000, 16)).astype(np.float32)
    XB = rng.standard_normal((60_000, 32)).astype(np.float32)
    ia, ib = osann.Index(to_dev(XA), 2), osann.Index(to_dev(XB), 2)
    pools = [to_dev(rng.standard_normal((3000, 16)).astype(np.float32)),
             to_dev(rng.standard_normal((3000, 32)).astype(np.float32))]
    yield torch, rng, [ia, ib], pools
    ia.close()
    ib.close()


P = [16, 48]
K = [1, 3]


def make_requests(rng, n, max_q):
    reqs = []
    for _ in range(n):
        i = int(rng.integers(0, 2))
        q = int(np.exp(rng.uniform(0, np.log(max_q))))
        off = int(rng.integers(0, 3000 - q))
        reqs.append((i, off, q))
    return reqs


def run_mix(osann, torch, idx, pools, reqs, **kw):
    srv = osann.Server(idx, P=P, k=K, **kw)
    out = {}
    tickets = []
    # continuous: keep submitting while earlier batches are in flight
    for j, (i, off, q) in enumerate(reqs):
        tickets.append(srv.submit(i, pools[i][off:off + q]))
        if j % 3 == 2:
            srv.progress()
    srv.drain()
    for j, t in enumerate(tickets):
        out[j] = srv.result(t)
    st = srv.stats()
    assert st["queries"] == sum(q for _, _, q in reqs)
    if kw.get("graphs", True):
        assert st["capture_failures"] == 0 and st["graph_replays"] == st["batches"] > 0
    else:
        assert st["graph_replays"] == 0
    srv.close()
    return out


def check_against_alone(idx, pools, reqs, out):
    for j, (i, off, q) in enumerate(reqs):
        ids, d2 = idx[i].search(pools[i][off:off + q], P[i], K[i])
        gi, gd = out[j]
        assert np.array_equal(to_np(ids), to_np(gi)), (j, i, q)
        assert np.array_equal(to_np(d2).view(np.uint32), to_np(gd).view(np.uint32)), (j, i, q)


@pytest.mark.parametrize("graphs", [True, False])
def test_mix_equals_alone(osann, setup, graphs):
    torch, rng, idx, pools = setup
    reqs = make_requests(np.random.default_rng(5), 40, 1200)
    out = run_mix(osann, torch, idx, pools, reqs, slots=3, max_batch=512, graphs=graphs)
    check_against_alone(idx, pools, reqs, out)


def test_tuned_mix_equals_alone(osann, setup):
    torch, rng, idx, pools = setup
    reqs = make_requests(np.random.default_rng(6), 30, 1000)
    srv = osann.Server(idx, P=P, k=K, slots=2, max_batch=512)
    choices = srv.tune(reps=1)
    assert len(choices) == 2 and all(len(c) == len(srv.buckets()) for c in choices)
    for per_index in choices:
        for path, group, layout in per_index:
            assert path in ("plain", "batched", "fp16")
            assert layout in ("default", "smem", "tmem")
    assert srv.choices() == choices
    tickets = [srv.submit(i, pools[i][off:off + q]) for (i, off, q) in reqs]
    srv.drain()
    out = {j: srv.result(t) for j, t in enumerate(tickets)}
    srv.close()
    check_against_alone(idx, pools, reqs, out)


def test_memory_budget_bounds_slots(osann, setup):
    torch, rng, idx, pools = setup
    big = osann.Server(idx, P=P, k=K, slots=4, max_batch=256)
    assert big.slots == 4
    big.close()
    with pytest.raises(osann.OsannError):
        osann.Server(idx, P=P, k=K, slots=4, max_batch=256, mem_budget=1024)


def test_empty_and_single_requests(osann, setup):
    torch, rng, idx, pools = setup
    srv = osann.Server(idx, P=P, k=K, slots=2, max_batch=64)
    t0 = srv.submit(0, pools[0][:0])
    t1 = srv.submit(1, pools[1][5:6])
    got = srv.drain()
    assert set(got) >= {t1}
    ids, d2 = srv.result(t1)
    a_ids, a_d2 = idx[1].search(pools[1][5:6], P[1], K[1])
    assert np.array_equal(to_np(ids), to_np(a_ids))
    srv.close()


def test_graph_replays_count_their_kernels(osann, setup):
    torch, rng, idx, pools = setup
    srv = osann.Server(idx, P=P, k=K, slots=1, max_batch=128, graphs=True)
    srv.submit(1, pools[1][:100])
    srv.drain()  # captures the graph
    before = osann.launch_count()
    srv.submit(1, pools[1][100:200])
    srv.drain()  # replays it
    assert osann.launch_count() - before >= 3
    st = srv.stats()
    assert st["graphs_captured"] == 1 and st["graph_replays"] == 2 and st["capture_failures"] == 0
    srv.close()
