"""osann: order-statistics cone-hash approximate nearest-neighbour search
(ROSANNA, one basis) on GB300.

Python face of libosann (include/osann.h).  torch supplies device memory and
streams; every step of the search runs in the library's CUDA kernels.

    idx = Index(data_cuda_f32, L)            # cone keys, buckets, permuted copy
    ids, d2 = idx.search(queries, P, k)      # ordered probing, exact top-k
    gt_ids, gt_d2 = idx.bruteforce(queries, k)
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import OsannError, PATHS, STAGES, load

__all__ = ["Index", "MultiIndex", "Server", "OsannError", "build_search", "merge_topk", "keys", "keys_wide",
           "query_order", "num_cones", "stats", "launch_count", "load"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float32 tensor")
    return t.contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def num_cones(d: int, L: int) -> int:
    out = ctypes.c_int64()
    _lib.check(load().osann_num_cones(d, L, ctypes.byref(out)))
    return out.value


def keys(vectors, L: int, stream=None):
    """Cone id (uint32 as int64 tensor) of every row."""
    torch = _torch()
    v = _dev_f32(vectors, "vectors")
    out = torch.empty(v.shape[0], dtype=torch.int32, device=v.device)
    _lib.check(load().osann_keys(_ptr(v), v.shape[0], v.shape[1], L, _ptr(out), _stream_ptr(stream)))
    return out.to(torch.int64) & 0xFFFFFFFF


def _wide_to_ints(w) -> list:
    """[n, 4] uint32 words (least significant first, as int32) -> Python ints."""
    a = w.cpu().numpy().astype("uint32").astype(object)
    return [int(r[0]) | (int(r[1]) << 32) | (int(r[2]) << 64) | (int(r[3]) << 96) for r in a]


def keys_wide(vectors, L: int, stream=None) -> list:
    """128-bit cone id (Python int) of every row, for any N_C."""
    torch = _torch()
    v = _dev_f32(vectors, "vectors")
    out = torch.empty((v.shape[0], 4), dtype=torch.int32, device=v.device)
    _lib.check(load().osann_keys_wide(_ptr(v), v.shape[0], v.shape[1], L, _ptr(out), _stream_ptr(stream)))
    return _wide_to_ints(out)


def query_order(queries, stream=None):
    """(order uint8 [Q, d], sign words int64 [Q, 8])."""
    torch = _torch()
    q = _dev_f32(queries, "queries")
    Q, d = q.shape
    order = torch.empty((Q, d), dtype=torch.uint8, device=q.device)
    signs = torch.empty((Q, 8), dtype=torch.int32, device=q.device)
    _lib.check(load().osann_query_order(_ptr(q), Q, d, _ptr(order), _ptr(signs), _stream_ptr(stream)))
    return order, signs.to(torch.int64) & 0xFFFFFFFF


def stats(enable: bool | None = None, reset: bool = False) -> dict:
    L = load()
    if enable is not None:
        L.osann_stats_enable(1 if enable else 0)
    out = {}
    for i, name in enumerate(STAGES):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        L.osann_stats_get(i, ctypes.byref(ms), ctypes.byref(n))
        out[name] = (ms.value, n.value)
    if reset:
        L.osann_stats_reset()
    return out


def merge_topk(ids, sqdists, stream=None):
    """k best by (distance, id) of G per-shard result lists: ids int64 and
    sqdists float32 CUDA tensors of shape [G, Q, k]."""
    torch = _torch()
    if ids.dim() != 3 or sqdists.shape != ids.shape:
        raise ValueError("ids and sqdists must both be [G, Q, k]")
    G, Q, k = ids.shape
    ids = ids.contiguous()
    d2 = sqdists.contiguous()
    out_ids = torch.empty((Q, k), dtype=torch.int64, device=ids.device)
    out_d = torch.empty((Q, k), dtype=torch.float32, device=ids.device)
    _lib.check(load().osann_merge_topk(_ptr(ids), _ptr(d2), G, Q, k, _ptr(out_ids), _ptr(out_d),
                                       _stream_ptr(stream)))
    return out_ids, out_d


def launch_count() -> int:
    return int(load().osann_launch_count())


class Index:
    """A one-basis cone index over ``data`` (N x d float32 CUDA tensor)."""

    def __init__(self, data, L: int, stream=None, sync: bool = True, rot=None, rot_offset=None,
                 cone_table: str = "auto", centroids=None, key_mode: str = "set"):
        """sync=False: no final synchronisation (call status() before
        trusting results).  rot: d x d (a rotated basis) or m x d (a
        projection on m components, e.g. PCA axes) float32 CUDA tensor, the
        basis of the keys and query orders; rot_offset: m offsets subtracted
        after projecting.  cone_table: "auto" (a direct table when
        N_C < 2^31), "dense" or "hashed" (the second-level table of occupied
        cones); the results are the same.  centroids: K x d float32 CUDA
        tensor (ROSANNA+, e.g. from kmeans.kmeans): points hashed by their
        residual on their nearest centroid; search(..., clusters=M) visits
        a query's M nearest clusters.  key_mode: "set" (the paper's
        unordered profile) or "ordered" (the top-L components as a tuple in
        magnitude order; N_C = d!/(d-L)! 2^L, direct table only)."""
        torch = _torch()
        x = _dev_f32(data, "data")
        self.N, self.d = x.shape
        self.L = L
        self.device = x.device
        h = ctypes.c_void_p()
        opts = _lib.BuildOpts()
        opts.async_ = 0 if sync else 1
        opts.cone_table = _lib.CONE_TABLES[cone_table]
        opts.key_mode = _lib.KEY_MODES[key_mode]
        self.key_mode = key_mode
        with torch.cuda.device(x.device):
            if rot is not None:
                r = _dev_f32(rot, "rot")
                if r.shape[1] != self.d or not 1 <= r.shape[0] <= self.d:
                    raise ValueError("rot must be m x d with 1 <= m <= d")
                off = None
                if rot_offset is not None:
                    off = rot_offset.to(device=x.device, dtype=torch.float32).contiguous().reshape(-1)
                    if off.numel() != r.shape[0]:
                        raise ValueError("rot_offset must hold m values")
                self._basis = (r, off)  # read by the build in stream order
                opts.d_basis = r.data_ptr()
                opts.d_offset = off.data_ptr() if off is not None else None
                opts.m = r.shape[0]
            self.K = 0
            if centroids is not None:
                cc = _dev_f32(centroids, "centroids")
                if cc.shape[1] != self.d:
                    raise ValueError("centroids must be K x d")
                self._cent = cc  # read by the build in stream order
                opts.d_centroids = cc.data_ptr()
                opts.n_clusters = cc.shape[0]
                self.K = cc.shape[0]
            _lib.check(load().osann_build_ex(_ptr(x), self.N, self.d, L, ctypes.byref(opts), _stream_ptr(stream),
                                             ctypes.byref(h)))
        self._adopt(h, x, L, sync)

    def _adopt(self, h, x, L, sync):
        self._h = h
        self.N, self.d = x.shape
        self.L = L
        self.device = x.device
        if not hasattr(self, "K"):
            self.K = 0
        # an asynchronous build may still be reading the input: keep it until status()
        self._src = None if sync else x
        NC, mb = ctypes.c_int64(), ctypes.c_int64()
        _lib.check(load().osann_info(h, None, None, None, ctypes.byref(NC), ctypes.byref(mb)))
        self.NC, self.max_bucket = NC.value, mb.value
        hashed, ncw = ctypes.c_int32(), (ctypes.c_uint64 * 2)()
        _lib.check(load().osann_cones(h, ctypes.byref(hashed), ncw, None, None, None))
        self.hashed = bool(hashed.value)
        self.n_cones = int(ncw[0]) | (int(ncw[1]) << 64)  # N_C itself (NC: cones of the CSR table)

    def rebuild(self, data, stream=None):
        """Rebuild in place from new data of the same shape (osann_rebuild):
        asynchronous, allocation-free after the first call (graph-capturable);
        check status() before trusting results."""
        x = _dev_f32(data, "data")
        if tuple(x.shape) != (self.N, self.d):
            raise ValueError("rebuild needs data of the index's shape")
        _lib.check(load().osann_rebuild(self._h, _ptr(x), _stream_ptr(stream)))
        self._src = x  # read in stream order until status()
        self.max_bucket = -1

    def rebuild_search(self, data, queries, P: int, k: int, path: str = "auto", stream=None, out=None,
                       workspace=None):
        """rebuild(data) then search(queries, ...) in one call
        (osann_rebuild_search), the query-side steps beside the rebuild.
        With ``out`` and ``workspace`` given (and after one earlier call) it
        allocates nothing, so it can be captured in a CUDA graph."""
        torch = _torch()
        x = _dev_f32(data, "data")
        q = _dev_f32(queries, "queries")
        if tuple(x.shape) != (self.N, self.d) or q.shape[1] != self.d:
            raise ValueError("rebuild_search needs data of the index's shape and queries of its dimension")
        Q = q.shape[0]
        if out is None:
            ids = torch.empty((Q, k), dtype=torch.int64, device=q.device)
            d2 = torch.empty((Q, k), dtype=torch.float32, device=q.device)
        else:
            ids, d2 = out
        ws_ptr, ws_n = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel())
        _lib.check(load().osann_rebuild_search(self._h, _ptr(x), _ptr(q), Q, P, k, PATHS[path], ws_ptr, ws_n,
                                               _ptr(ids), _ptr(d2), _stream_ptr(stream)))
        self._src = x
        self.max_bucket = -1
        return ids, d2

    def occupied(self, stream=None) -> int:
        """Cones holding at least one point (synchronises)."""
        n = ctypes.c_int64()
        _lib.check(load().osann_cones(self._h, None, None, None, ctypes.byref(n), _stream_ptr(stream)))
        return n.value

    def cone_ids(self, stream=None) -> list:
        """128-bit id (Python int) of every compact cone of a second-level
        table (all ones past the occupied cones)."""
        torch = _torch()
        out = torch.empty((self.NC, 4), dtype=torch.int32, device=self.device)
        _lib.check(load().osann_export_cones(self._h, _ptr(out), _stream_ptr(stream)))
        return _wide_to_ints(out)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().osann_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- queries
    def workspace_size(self, Q: int, P: int, k: int, path: str = "auto", group: int = 0) -> int:
        return int(load().osann_search_workspace_size_group(self._h, Q, P, k, PATHS[path], group))

    def search(self, queries, P: int, k: int, path: str = "auto", query_src=None, grid_w: int = 0,
               radius: int = 0, stream=None, out=None, workspace=None, group: int = 0, clusters: int = 1,
               layout: str = "default"):
        """Top-k by exact squared distance over the first min(P, N_C)
        probed cones.  Returns (ids int64 [Q,k], sqdists float32 [Q,k]).
        ``group``: queries per work-list item on the batched paths (0 =
        default); ``layout``: the tensor-core screen's query tiles ("smem",
        "tmem" or "default"); both change the speed, not the result.
        ``clusters`` (ROSANNA+ index): nearest clusters visited, P cones in
        each."""
        torch = _torch()
        if clusters != 1:
            if query_src is not None or group or layout != "default":
                raise ValueError("clusters > 1 takes no exclusion, group size or layout")
            return self._search_clusters(queries, clusters, P, k, path, stream, out, workspace)
        q = _dev_f32(queries, "queries")
        Q = q.shape[0]
        if q.shape[1] != self.d:
            raise ValueError("query dimension differs from the index's")
        if out is None:
            ids = torch.empty((Q, k), dtype=torch.int64, device=q.device)
            d2 = torch.empty((Q, k), dtype=torch.float32, device=q.device)
        else:
            ids, d2 = out
        ws_bytes = self.workspace_size(Q, P, k, path, 0 if query_src is not None else group)
        ws = workspace if workspace is not None else torch.empty(ws_bytes, dtype=torch.uint8, device=q.device)
        L = load()
        if query_src is None:
            rc = L.osann_search_layout(self._h, _ptr(q), Q, P, k, PATHS[path], group, _lib.LAYOUTS[layout],
                                       _ptr(ws), ws.numel(), _ptr(ids), _ptr(d2), _stream_ptr(stream))
        else:
            if layout != "default":
                raise ValueError("the exclusion search takes the default layout")
            src = query_src.contiguous()
            rc = L.osann_search_excl(self._h, _ptr(q), _ptr(src), Q, P, k, grid_w, radius, PATHS[path],
                                     _ptr(ws), ws.numel(), _ptr(ids), _ptr(d2), _stream_ptr(stream))
        _lib.check(rc)
        return ids, d2

    def _search_clusters(self, queries, M, P, k, path, stream, out, workspace):
        torch = _torch()
        q = _dev_f32(queries, "queries")
        Q = q.shape[0]
        if q.shape[1] != self.d:
            raise ValueError("query dimension differs from the index's")
        if out is None:
            ids = torch.empty((Q, k), dtype=torch.int64, device=q.device)
            d2 = torch.empty((Q, k), dtype=torch.float32, device=q.device)
        else:
            ids, d2 = out
        L = load()
        ws_bytes = int(L.osann_search_clusters_workspace_size(self._h, Q, M, P, k, PATHS[path]))
        ws = workspace if workspace is not None else torch.empty(ws_bytes, dtype=torch.uint8, device=q.device)
        _lib.check(L.osann_search_clusters(self._h, _ptr(q), Q, M, P, k, PATHS[path], _ptr(ws), ws.numel(),
                                           _ptr(ids), _ptr(d2), _stream_ptr(stream)))
        return ids, d2

    def bruteforce(self, queries, k: int, query_src=None, grid_w: int = 0, radius: int = 0, stream=None):
        """Exact linear search over all N points (Eq. 1)."""
        torch = _torch()
        q = _dev_f32(queries, "queries")
        Q = q.shape[0]
        ids = torch.empty((Q, k), dtype=torch.int64, device=q.device)
        d2 = torch.empty((Q, k), dtype=torch.float32, device=q.device)
        L = load()
        ws = torch.empty(int(L.osann_bruteforce_workspace_size(self._h, Q, k)), dtype=torch.uint8,
                         device=q.device)
        src = query_src.contiguous() if query_src is not None else None
        _lib.check(L.osann_bruteforce(self._h, _ptr(q), _ptr(src), Q, k, grid_w, radius, _ptr(ws), ws.numel(),
                                      _ptr(ids), _ptr(d2), _stream_ptr(stream)))
        return ids, d2

    def probes(self, queries, P: int, stream=None):
        """Ordered cone ids visited per query: int64 [Q, min(P, N_C)]."""
        torch = _torch()
        q = _dev_f32(queries, "queries")
        Q = q.shape[0]
        P_eff = min(P, self.n_cones)
        out = torch.empty((Q, P_eff), dtype=torch.int32, device=q.device)
        ws = torch.empty(self.workspace_size(Q, P, 1, "plain"), dtype=torch.uint8, device=q.device)
        _lib.check(load().osann_probes(self._h, _ptr(q), Q, P, _ptr(out), _ptr(ws), ws.numel(),
                                       _stream_ptr(stream)))
        return out.to(torch.int64) & 0xFFFFFFFF

    def export(self, stream=None):
        """(keys [N], offsets [NC+1], perm [N]) as int64 tensors (NC: cones of
        the CSR table; compact cones for a second-level table)."""
        torch = _torch()
        k = torch.empty(self.N, dtype=torch.int32, device=self.device)
        o = torch.empty(self.NC + 1, dtype=torch.int32, device=self.device)
        p = torch.empty(self.N, dtype=torch.int32, device=self.device)
        _lib.check(load().osann_export(self._h, _ptr(k), _ptr(o), _ptr(p), _stream_ptr(stream)))
        m = 0xFFFFFFFF
        return k.to(torch.int64) & m, o.to(torch.int64) & m, p.to(torch.int64) & m

    def screen_stats(self, stream=None) -> dict:
        """Counters of the tensor-core screening path since the last call."""
        out = (ctypes.c_int64 * 4)()
        _lib.check(load().osann_screen_stats(self._h, _stream_ptr(stream), out))
        return {"survivors": out[0], "fallbacks": out[1], "bound_checks": out[2], "bound_violations": out[3]}

    def status(self, stream=None) -> int:
        """Synchronise and return (and clear) the device status flags."""
        f = ctypes.c_uint32()
        _lib.check(load().osann_status(self._h, _stream_ptr(stream), ctypes.byref(f)))
        self._src = None
        if self.max_bucket < 0:
            mb = ctypes.c_int64()
            _lib.check(load().osann_info(self._h, None, None, None, None, ctypes.byref(mb)))
            self.max_bucket = mb.value
        return f.value


def build_search(data, L: int, queries, P: int, k: int, path: str = "auto", stream=None, sync: bool = True,
                 out=None, cone_table: str = "auto"):
    """Build an Index over ``data`` and search ``queries`` in one call
    (osann_build_search): the same results as Index(...).search(...), with
    the query-side steps running beside the build.  Returns (index, ids,
    sqdists); sync=False leaves the build's status for index.status()."""
    torch = _torch()
    x = _dev_f32(data, "data")
    q = _dev_f32(queries, "queries")
    N, d = x.shape
    Q = q.shape[0]
    if q.shape[1] != d:
        raise ValueError("query dimension differs from the data's")
    if out is None:
        ids = torch.empty((Q, k), dtype=torch.int64, device=q.device)
        d2 = torch.empty((Q, k), dtype=torch.float32, device=q.device)
    else:
        ids, d2 = out
    opts = _lib.BuildOpts()
    opts.async_ = 0 if sync else 1
    opts.cone_table = _lib.CONE_TABLES[cone_table]
    h = ctypes.c_void_p()
    with torch.cuda.device(x.device):
        _lib.check(load().osann_build_search(_ptr(x), N, d, L, ctypes.byref(opts), _ptr(q), Q, P, k, PATHS[path],
                                             None, 0, _ptr(ids), _ptr(d2), _stream_ptr(stream), ctypes.byref(h)))
    ix = Index.__new__(Index)
    ix._adopt(h, x, L, sync)
    return ix, ids, d2


class MultiIndex:
    """R bases (Sec. 3-D, Algorithm 1 with R > 1): one rotated index per basis
    (``rots``: R x d x d, basis 0 usually the identity), a search on each and
    the merge of the per-basis k-best lists with repeated ids dropped.

        mi = MultiIndex(X, L, datagen.rotations(4, d, seed))
        ids, d2 = mi.search(Y, P, k)    # P cones per basis
    """

    def __init__(self, data, L: int, rots, stream=None, sync: bool = True, offsets=None):
        torch = _torch()
        x = _dev_f32(data, "data")
        r = rots if isinstance(rots, torch.Tensor) else torch.as_tensor(rots)
        r = r.to(device=x.device, dtype=torch.float32).contiguous()
        if r.dim() == 2:
            r = r.unsqueeze(0)
        o = None
        if offsets is not None:
            o = offsets if isinstance(offsets, torch.Tensor) else torch.as_tensor(offsets)
            o = o.to(device=x.device, dtype=torch.float32).reshape(r.shape[0], r.shape[1]).contiguous()
        self.R = r.shape[0]
        self.rots = r
        self.bases = [Index(x, L, stream=stream, sync=sync, rot=r[i], rot_offset=None if o is None else o[i])
                      for i in range(self.R)]
        self.N, self.d, self.L = x.shape[0], x.shape[1], L

    def search(self, queries, P: int, k: int, path: str = "auto", stream=None):
        torch = _torch()
        q = _dev_f32(queries, "queries")
        Q = q.shape[0]
        ids = torch.empty((self.R, Q, k), dtype=torch.int64, device=q.device)
        d2 = torch.empty((self.R, Q, k), dtype=torch.float32, device=q.device)
        for i, ix in enumerate(self.bases):
            ix.search(q, P, k, path=path, stream=stream, out=(ids[i], d2[i]))
        return merge_topk(ids, d2, stream=stream)

    def status(self, stream=None) -> int:
        f = 0
        for ix in self.bases:
            f |= ix.status(stream)
        return f

    def close(self):
        for ix in self.bases:
            ix.close()


class Server:
    """Continuous-batching request loop over resident indexes (osann_server_*
    in include/osann.h).  ``indexes``: list of Index; ``P``, ``k``: per index.

        srv = Server([ia, ib], P=[64, 32], k=[1, 1], slots=4, max_batch=4096)
        t = srv.submit(0, queries_cuda)          # -> ticket; results in srv.result(t)
        done = srv.progress(wait=True)           # finished tickets
    """

    def __init__(self, indexes, P, k, slots: int = 4, max_batch: int = 4096, mem_budget: int = 0,
                 graphs: bool = True):
        n = len(indexes)
        self.indexes = list(indexes)
        self.P, self.k = list(P), list(k)
        arr = (ctypes.c_void_p * n)(*[ix._h.value for ix in indexes])
        Pa = (ctypes.c_int32 * n)(*self.P)
        ka = (ctypes.c_int32 * n)(*self.k)
        h = ctypes.c_void_p()
        _lib.check(load().osann_server_create(arr, n, Pa, ka, slots, max_batch, mem_budget, 1 if graphs else 0,
                                              ctypes.byref(h)))
        self._h = h
        self._req = {}  # ticket -> (queries, ids, dists): kept alive until finished
        self._out = {}

    @property
    def slots(self) -> int:
        return int(load().osann_server_slots(self._h))

    def buckets(self):
        out = (ctypes.c_int64 * 64)()
        n = load().osann_server_buckets(self._h, out, 64)
        return [int(out[i]) for i in range(n)]

    def tune(self, reps: int = 3, queries=None):
        """Autotune (path, group, layout) per (index, bucket); returns the
        choices as (path name, group, layout name) triples per index and
        bucket.  queries: optional list (per index) of sample query tensors."""
        nb = len(self.buckets())
        n = len(self.indexes)
        out = (ctypes.c_int32 * (2 * n * nb))()
        if queries is None:
            _lib.check(load().osann_server_tune(self._h, reps, out))
        else:
            qs = [None if q is None else _dev_f32(q, "queries") for q in queries]
            ptrs = (ctypes.c_void_p * n)(*[None if q is None else q.data_ptr() for q in qs])
            cnt = (ctypes.c_int64 * n)(*[0 if q is None else q.shape[0] for q in qs])
            _lib.check(load().osann_server_tune_queries(self._h, ptrs, cnt, reps, out))
        return self.choices()

    def choices(self):
        """The current (path name, group, layout name) per (index, bucket)."""
        nb = len(self.buckets())
        n = len(self.indexes)
        out = (ctypes.c_int32 * (3 * n * nb))()
        got = load().osann_server_choices(self._h, out, n * nb)
        paths = {v: k for k, v in PATHS.items()}
        layouts = {v: k for k, v in _lib.LAYOUTS.items()}
        trip = [(paths[out[3 * j]], int(out[3 * j + 1]), layouts[out[3 * j + 2]]) for j in range(got)]
        return [trip[i * nb:(i + 1) * nb] for i in range(n)]

    def warmup(self):
        """Capture every (slot, index, bucket) graph now rather than while serving."""
        _lib.check(load().osann_server_warmup(self._h))

    def submit(self, index: int, queries, out=None) -> int:
        torch = _torch()
        q = _dev_f32(queries, "queries")
        Q = q.shape[0]
        kk = self.k[index]
        if out is None:
            ids = torch.empty((Q, kk), dtype=torch.int64, device=q.device)
            d2 = torch.empty((Q, kk), dtype=torch.float32, device=q.device)
        else:
            ids, d2 = out
        t = ctypes.c_uint64()
        _lib.check(load().osann_server_submit(self._h, index, _ptr(q), Q, _ptr(ids), _ptr(d2), ctypes.byref(t)))
        self._req[t.value] = (q, ids, d2)
        return t.value

    def progress(self, wait: bool = False, max_done: int = 1024):
        done = (ctypes.c_uint64 * max_done)()
        n = ctypes.c_int32()
        _lib.check(load().osann_server_progress(self._h, 1 if wait else 0, done, max_done, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            t = int(done[i])
            q, ids, d2 = self._req.pop(t)
            self._out[t] = (ids, d2)
            out.append(t)
        return out

    def pending(self):
        w, b = ctypes.c_int64(), ctypes.c_int32()
        _lib.check(load().osann_server_pending(self._h, ctypes.byref(w), ctypes.byref(b)))
        return w.value, b.value

    def stats(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        _lib.check(load().osann_server_stats(self._h, out))
        return {"batches": out[0], "queries": out[1], "graph_replays": out[2], "graphs_captured": out[3],
                "capture_failures": out[4]}

    def result(self, ticket: int):
        """(ids, sqdists) of a finished request (removed from the server)."""
        return self._out.pop(ticket)

    def drain(self):
        """Progress until every submitted request has finished; returns their tickets."""
        got = []
        while self._req:
            got += self.progress(wait=True)
        return got

    def close(self):
        if getattr(self, "_h", None):
            load().osann_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
