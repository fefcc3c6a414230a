"""CPU oracle for the order-statistics cone-hash search (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it shares
no code with the C source here (``osann_oracle.c``), which is compiled with
gcc into ``oracle/_build/libosann_oracle.so`` by :func:`build`.

The wrappers below only marshal numpy arrays; every step of the method is in
the C file, which cites the paper section each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osann_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libosann_oracle.so")
_lib = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it runs on x86 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # no contraction of a*b+c into fused multiply-adds: the same roundings on x86 and Arm
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        c = ctypes
        L.oracle_binom.restype = c.c_uint64
        L.oracle_binom.argtypes = [c.c_int64, c.c_int64]
        L.oracle_num_cones.restype = c.c_int64
        L.oracle_num_cones.argtypes = [c.c_int, c.c_int]
        L.oracle_magnitude_order.restype = None
        L.oracle_magnitude_order.argtypes = [_f32p, c.c_int, _i32p]
        L.oracle_key.restype = c.c_uint32
        L.oracle_key.argtypes = [_f32p, c.c_int, c.c_int]
        L.oracle_keys.restype = None
        L.oracle_keys.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, _u32p]
        L.oracle_buckets.restype = None
        L.oracle_buckets.argtypes = [_u32p, c.c_int64, c.c_int64, _u32p, _u32p]
        L.oracle_probes.restype = c.c_int64
        L.oracle_probes.argtypes = [_f32p, c.c_int, c.c_int, c.c_int64, _u32p]
        L.oracle_search.restype = None
        L.oracle_search.argtypes = [
            _f32p, c.c_int64, c.c_int, c.c_int, _u32p, _u32p, _f32p, c.c_int64,
            c.c_int64, c.c_int, c.c_void_p, c.c_int64, c.c_int64, _i64p, _f64p,
            c.c_void_p]
        L.oracle_num_cones_ordered.restype = c.c_int64
        L.oracle_num_cones_ordered.argtypes = [c.c_int, c.c_int]
        L.oracle_key_ordered.restype = c.c_uint32
        L.oracle_key_ordered.argtypes = [_f32p, c.c_int, c.c_int]
        L.oracle_keys_ordered.restype = None
        L.oracle_keys_ordered.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, _u32p]
        L.oracle_probes_ordered.restype = c.c_int64
        L.oracle_probes_ordered.argtypes = [_f32p, c.c_int, c.c_int, c.c_int64, _u32p]
        L.oracle_search_mode.restype = None
        L.oracle_search_mode.argtypes = [
            _f32p, c.c_int64, c.c_int, c.c_int, c.c_int, _u32p, _u32p, _f32p, c.c_int64,
            c.c_int64, c.c_int, c.c_void_p, c.c_int64, c.c_int64, _i64p, _f64p,
            c.c_void_p]
        L.oracle_bruteforce.restype = None
        L.oracle_bruteforce.argtypes = [
            _f32p, c.c_int64, c.c_int, _f32p, c.c_int64, c.c_int, c.c_void_p,
            c.c_int64, c.c_int64, _i64p, _f64p]
        L.oracle_rotate.restype = None
        L.oracle_rotate.argtypes = [_f32p, _f32p, c.c_int64, c.c_int, _f32p]
        L.oracle_project.restype = None
        L.oracle_project.argtypes = [_f32p, c.c_void_p, _f32p, c.c_int64, c.c_int, c.c_int, _f32p]
        L.oracle_search_multi_proj.restype = None
        L.oracle_search_multi_proj.argtypes = [
            _f32p, c.c_int64, c.c_int, c.c_int, c.c_int, c.c_int, _f32p, c.c_void_p, _u32p, _u32p, _f32p,
            c.c_int64, c.c_int64, c.c_int, _i64p, _f64p, c.c_void_p]
        L.oracle_search_multi.restype = None
        L.oracle_search_multi.argtypes = [
            _f32p, c.c_int64, c.c_int, c.c_int, c.c_int, _f32p, _u32p, _u32p, _f32p, c.c_int64,
            c.c_int64, c.c_int, _i64p, _f64p, c.c_void_p]
        _u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        L.oracle_num_cones_wide.restype = c.c_int
        L.oracle_num_cones_wide.argtypes = [c.c_int, c.c_int, _u64p]
        L.oracle_keys_wide.restype = None
        L.oracle_keys_wide.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, _u64p]
        L.oracle_probes_wide.restype = c.c_int64
        L.oracle_probes_wide.argtypes = [_f32p, c.c_int, c.c_int, c.c_int64, _u64p]
        L.oracle_buckets_wide.restype = c.c_int64
        L.oracle_buckets_wide.argtypes = [_u64p, c.c_int64, _u32p, _u64p, _u32p]
        L.oracle_search_wide.restype = None
        L.oracle_search_wide.argtypes = [
            _f32p, c.c_int64, c.c_int, c.c_int, c.c_int64, _u64p, _u32p, _u32p, _f32p, c.c_int64,
            c.c_int64, c.c_int, c.c_void_p, c.c_int64, c.c_int64, _i64p, _f64p, c.c_void_p]
        L.oracle_nearest_centroids.restype = None
        L.oracle_nearest_centroids.argtypes = [_f32p, c.c_int64, c.c_int, _f32p, c.c_int, c.c_int, _i32p]
        L.oracle_keys_clustered.restype = c.c_int
        L.oracle_keys_clustered.argtypes = [_f32p, c.c_int64, c.c_int, c.c_int, _f32p, c.c_int, _u64p, _i32p,
                                            c.c_void_p]
        L.oracle_search_clustered.restype = None
        L.oracle_search_clustered.argtypes = [
            _f32p, c.c_int64, c.c_int, c.c_int, _f32p, c.c_int, c.c_int, c.c_int64, _u64p, _u32p, _u32p,
            _f32p, c.c_int64, c.c_int64, c.c_int, _i64p, _f64p, c.c_void_p, c.c_void_p]
        L.oracle_pair_dists.restype = None
        L.oracle_pair_dists.argtypes = [_f32p, c.c_int, _f32p, c.c_int64,
                                        c.c_int, _i64p, _f64p]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def binom(n: int, k: int) -> int:
    return int(lib().oracle_binom(n, k))


def num_cones(d: int, L: int) -> int:
    return int(lib().oracle_num_cones(d, L))


def magnitude_order(y) -> np.ndarray:
    y = _f32(y)
    out = np.empty(y.shape[-1], np.int32)
    lib().oracle_magnitude_order(y, y.shape[-1], out)
    return out


def key(x, L: int) -> int:
    x = _f32(x)
    return int(lib().oracle_key(x, x.shape[-1], L))


def _sliced(n: int, threads: int, fn) -> None:
    """Run fn(lo, hi) on `threads` contiguous slices of range(n), one thread
    each.  The C calls release the GIL and share no state, so the slices run
    in parallel; each runs the same single-threaded code on its rows."""
    threads = max(1, min(int(threads), n))
    if threads == 1:
        fn(0, n)
        return
    import threading
    cuts = [n * t // threads for t in range(threads + 1)]
    errs = []

    def run(lo, hi):
        try:
            fn(lo, hi)
        except BaseException as e:  # re-raised below
            errs.append(e)
    ts = [threading.Thread(target=run, args=(cuts[t], cuts[t + 1])) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]


def keys(X, L: int, threads: int = 1) -> np.ndarray:
    X = _f32(X)
    N, d = X.shape
    out = np.empty(N, np.uint32)
    _sliced(N, threads, lambda lo, hi: lib().oracle_keys(X[lo:hi], hi - lo, d, L, out[lo:hi]))
    return out


def num_cones_ordered(d: int, L: int) -> int:
    """N_C of the ORDERED key: d!/(d-L)! 2^L (-1 if it does not fit)."""
    return int(lib().oracle_num_cones_ordered(d, L))


def key_ordered(x, L: int) -> int:
    x = _f32(x)
    return int(lib().oracle_key_ordered(x, x.shape[-1], L))


def keys_ordered(X, L: int, threads: int = 1) -> np.ndarray:
    X = _f32(X)
    N, d = X.shape
    out = np.empty(N, np.uint32)
    _sliced(N, threads, lambda lo, hi: lib().oracle_keys_ordered(X[lo:hi], hi - lo, d, L, out[lo:hi]))
    return out


def probes_ordered(y, L: int, P: int) -> np.ndarray:
    """The ordered cone list of y for the ORDERED key."""
    y = _f32(y)
    out = np.empty(max(P, 1), np.uint32)
    n = lib().oracle_probes_ordered(y, y.shape[-1], L, P, out)
    return out[:n].copy()


def buckets(k: np.ndarray, NC: int):
    k = np.ascontiguousarray(k, dtype=np.uint32)
    offsets = np.empty(NC + 1, np.uint32)
    perm = np.empty(k.shape[0], np.uint32)
    lib().oracle_buckets(k, k.shape[0], NC, offsets, perm)
    return offsets, perm


def probes(y, L: int, P: int) -> np.ndarray:
    y = _f32(y)
    out = np.empty(max(P, 1), np.uint32)
    n = lib().oracle_probes(y, y.shape[-1], L, P, out)
    return out[:n].copy()


def num_cones_wide(d: int, L: int) -> int:
    """N_C = C(d, L) 2^L as a Python int, or -1 when it reaches 2^127."""
    out = np.zeros(2, np.uint64)
    if lib().oracle_num_cones_wide(d, L, out) != 0:
        return -1
    return int(out[0]) | (int(out[1]) << 64)


def _wide_ints(w: np.ndarray) -> list:
    return [int(a) | (int(b) << 64) for a, b in w.reshape(-1, 2)]


def keys_wide(X, L: int) -> list:
    """128-bit cone ids of the rows of X, as Python ints."""
    X = _f32(X)
    N, d = X.shape
    out = np.empty(2 * N, np.uint64)
    lib().oracle_keys_wide(X, N, d, L, out)
    return _wide_ints(out)


def probes_wide(y, L: int, P: int) -> list:
    """The ordered cone list of y with 128-bit ids (Python ints)."""
    y = _f32(y)
    out = np.empty(2 * max(P, 1), np.uint64)
    n = lib().oracle_probes_wide(y, y.shape[-1], L, P, out)
    return _wide_ints(out[:2 * n])


def _src_ptr(query_src):
    if query_src is None:
        return None, None
    arr = np.ascontiguousarray(query_src, dtype=np.int64)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


class Index:
    """Oracle index: keys, stable counting sort into cone buckets."""

    def __init__(self, X, L: int, threads: int = 1, key_mode: int = 0):
        """threads > 1: the keys of row slices computed in parallel threads
        (the same single-threaded code per slice).  key_mode 1: the ORDERED
        key (the top-L components as a tuple in magnitude order)."""
        self.X = _f32(X)
        self.N, self.d = self.X.shape
        self.L = L
        self.key_mode = int(key_mode)
        self.NC = num_cones_ordered(self.d, L) if self.key_mode else num_cones(self.d, L)
        if self.NC < 0 or self.NC >= 1 << 32:
            raise ValueError("N_C does not fit a direct table")
        self.keys = (keys_ordered if self.key_mode else keys)(self.X, L, threads)
        self.offsets, self.perm = buckets(self.keys, self.NC)

    def search(self, Y, P: int, k: int, query_src=None, grid_w: int = 0,
               radius: int = 0, want_counts: bool = False, threads: int = 1):
        """threads > 1: query slices searched in parallel threads."""
        Y = _f32(Y)
        Q = Y.shape[0]
        ids = np.empty(Q * k, np.int64)
        dists = np.empty(Q * k, np.float64)
        counts = np.empty(Q, np.int64) if want_counts else None
        keep, src = _src_ptr(query_src)
        step = np.dtype(np.int64).itemsize

        def part(lo, hi):
            lib().oracle_search_mode(
                self.X, self.N, self.d, self.L, self.key_mode, self.offsets, self.perm, Y[lo:hi], hi - lo, P, k,
                None if src is None else src.value + lo * step, grid_w, radius, ids[lo * k:hi * k],
                dists[lo * k:hi * k],
                counts[lo:hi].ctypes.data_as(ctypes.c_void_p) if want_counts else None)
        _sliced(Q, threads, part)
        del keep
        ids, dists = ids.reshape(Q, k), dists.reshape(Q, k)
        return (ids, dists, counts) if want_counts else (ids, dists)


class WideIndex:
    """Oracle index over the second-level table: 128-bit cone ids, points
    sorted by (id, point), only the occupied cones stored (ascending ids)."""

    def __init__(self, X, L: int):
        self.X = _f32(X)
        self.N, self.d = self.X.shape
        self.L = L
        self.NC = num_cones_wide(self.d, L)
        if self.NC < 0:
            raise ValueError("N_C does not fit in 127 bits")
        kw = np.empty(2 * self.N, np.uint64)
        lib().oracle_keys_wide(self.X, self.N, self.d, L, kw)
        self.keys = _wide_ints(kw)
        self.perm = np.empty(self.N, np.uint32)
        uniq = np.empty(2 * max(self.N, 1), np.uint64)
        offs = np.empty(self.N + 1, np.uint32)
        self.n_occ = int(lib().oracle_buckets_wide(kw, self.N, self.perm, uniq, offs))
        self._uniq = np.ascontiguousarray(uniq[:2 * max(self.n_occ, 1)])
        self.uniq = _wide_ints(uniq[:2 * self.n_occ])
        self.offsets = offs[:self.n_occ + 1].copy()

    def search(self, Y, P: int, k: int, query_src=None, grid_w: int = 0,
               radius: int = 0, want_counts: bool = False):
        Y = _f32(Y)
        Q = Y.shape[0]
        ids = np.empty(Q * k, np.int64)
        dists = np.empty(Q * k, np.float64)
        counts = np.empty(Q, np.int64) if want_counts else None
        keep, src = _src_ptr(query_src)
        lib().oracle_search_wide(
            self.X, self.N, self.d, self.L, self.n_occ, self._uniq, self.offsets, self.perm, Y, Q, P, k,
            src, grid_w, radius, ids, dists,
            counts.ctypes.data_as(ctypes.c_void_p) if want_counts else None)
        del keep
        ids, dists = ids.reshape(Q, k), dists.reshape(Q, k)
        return (ids, dists, counts) if want_counts else (ids, dists)


def nearest_centroids(X, C, M: int) -> np.ndarray:
    """[n, M] indices of the M nearest centroids (fp64 squared distance, then
    index; -1 pads when M > K)."""
    X, C = _f32(np.atleast_2d(X)), _f32(C)
    out = np.empty((X.shape[0], M), np.int32)
    lib().oracle_nearest_centroids(X, X.shape[0], X.shape[1], C, C.shape[0], M, out)
    return out


class ClusteredIndex:
    """ROSANNA+ oracle (Sec. 4-B): points assigned to their nearest of K
    given centroids, hashed by their residual, stored under the composite
    id cluster * N_C + cone; the search visits the query's M nearest
    clusters."""

    def __init__(self, X, L: int, centroids, asg=None):
        """asg: optional cluster of every point (int, [N]) used instead of
        the nearest centroid."""
        self.X = _f32(X)
        self.N, self.d = self.X.shape
        self.L = L
        self.C = _f32(centroids)
        self.K = self.C.shape[0]
        self.NC = num_cones_wide(self.d, L)
        kw = np.empty(2 * self.N, np.uint64)
        self.asg = np.empty(self.N, np.int32)
        a_in = None if asg is None else np.ascontiguousarray(asg, dtype=np.int32)
        if a_in is not None and a_in.shape != (self.N,):
            raise ValueError("asg must hold one cluster per point")
        if lib().oracle_keys_clustered(self.X, self.N, self.d, L, self.C, self.K, kw, self.asg,
                                       None if a_in is None else a_in.ctypes.data_as(ctypes.c_void_p)) != 0:
            raise ValueError("K * N_C does not fit in 127 bits, or a given cluster is out of range")
        self.keys = _wide_ints(kw)
        self.perm = np.empty(self.N, np.uint32)
        uniq = np.empty(2 * max(self.N, 1), np.uint64)
        offs = np.empty(self.N + 1, np.uint32)
        self.n_occ = int(lib().oracle_buckets_wide(kw, self.N, self.perm, uniq, offs))
        self._uniq = np.ascontiguousarray(uniq[:2 * max(self.n_occ, 1)])
        self.uniq = _wide_ints(uniq[:2 * self.n_occ])
        self.offsets = offs[:self.n_occ + 1].copy()

    def search(self, Y, M: int, P: int, k: int, want_counts: bool = False, near=None):
        """near: optional [Q, M] clusters of each query (-1: none) used
        instead of its M nearest."""
        Y = _f32(Y)
        Q = Y.shape[0]
        ids = np.empty(Q * k, np.int64)
        dists = np.empty(Q * k, np.float64)
        counts = np.empty(Q, np.int64) if want_counts else None
        n_in = None if near is None else np.ascontiguousarray(near, dtype=np.int32)
        if n_in is not None and n_in.shape != (Q, M):
            raise ValueError("near must be [Q, M]")
        lib().oracle_search_clustered(
            self.X, self.N, self.d, self.L, self.C, self.K, M, self.n_occ, self._uniq, self.offsets, self.perm,
            Y, Q, P, k, ids, dists, counts.ctypes.data_as(ctypes.c_void_p) if want_counts else None,
            None if n_in is None else n_in.ctypes.data_as(ctypes.c_void_p))
        ids, dists = ids.reshape(Q, k), dists.reshape(Q, k)
        return (ids, dists, counts) if want_counts else (ids, dists)


def rotate(Rm, X) -> np.ndarray:
    """Coordinates of the rows of X on the basis Rm (fp32, in-order FMAs)."""
    Rm, X = _f32(Rm), _f32(X)
    n, d = X.shape
    out = np.empty((n, d), np.float32)
    lib().oracle_rotate(Rm, X, n, d, out)
    return out


def project(Pm, X, off=None, threads: int = 1) -> np.ndarray:
    """Rows of X projected on the m rows of Pm minus off (fp32, in-order FMAs,
    one final subtraction)."""
    Pm, X = _f32(Pm), _f32(X)
    m = Pm.shape[0]
    n, d = X.shape
    out = np.empty((n, m), np.float32)
    o = None if off is None else _f32(off)
    _sliced(n, threads, lambda lo, hi: lib().oracle_project(
        Pm, None if o is None else o.ctypes.data_as(ctypes.c_void_p), X[lo:hi], hi - lo, d, m, out[lo:hi]))
    return out


class MultiIndex:
    """Oracle index over R bases: per basis, keys of the rows' coordinates on
    the basis (R x m x d, m <= d: a projection, with optional offsets R x m)
    and a stable counting sort; the search is the exact top-k over the union
    of the points of the bases' probed cones (Sec. 3-D)."""

    def __init__(self, X, L: int, rots, offsets=None, threads: int = 1):
        self.X = _f32(X)
        self.N, self.d = self.X.shape
        self.L = L
        r = np.asarray(rots, np.float32)
        self.rots = _f32(r.reshape(-1, r.shape[-2], self.d))
        self.R, self.m = self.rots.shape[0], self.rots.shape[1]
        self.off = None if offsets is None else _f32(np.asarray(offsets, np.float32).reshape(self.R, self.m))
        self.NC = num_cones(self.m, L)
        offs, perms = [], []
        for b in range(self.R):
            ob = None if self.off is None else self.off[b]
            o, p = buckets(keys(project(self.rots[b], self.X, ob, threads), L, threads), self.NC)
            offs.append(o)
            perms.append(p)
        self.offsets = np.ascontiguousarray(np.stack(offs), np.uint32)
        self.perms = np.ascontiguousarray(np.stack(perms), np.uint32)

    def search(self, Y, P: int, k: int, want_counts: bool = False, threads: int = 1):
        Y = _f32(Y)
        Q = Y.shape[0]
        ids = np.empty(Q * k, np.int64)
        dists = np.empty(Q * k, np.float64)
        counts = np.empty(Q, np.int64) if want_counts else None

        def part(lo, hi):
            lib().oracle_search_multi_proj(
                self.X, self.N, self.d, self.L, self.R, self.m, self.rots,
                None if self.off is None else self.off.ctypes.data_as(ctypes.c_void_p), self.offsets, self.perms,
                Y[lo:hi], hi - lo, P, k, ids[lo * k:hi * k], dists[lo * k:hi * k],
                counts[lo:hi].ctypes.data_as(ctypes.c_void_p) if want_counts else None)
        _sliced(Q, threads, part)
        ids, dists = ids.reshape(Q, k), dists.reshape(Q, k)
        return (ids, dists, counts) if want_counts else (ids, dists)


def bruteforce(X, Y, k: int, query_src=None, grid_w: int = 0, radius: int = 0):
    X, Y = _f32(X), _f32(Y)
    N, d = X.shape
    Q = Y.shape[0]
    ids = np.empty(Q * k, np.int64)
    dists = np.empty(Q * k, np.float64)
    keep, src = _src_ptr(query_src)
    lib().oracle_bruteforce(X, N, d, Y, Q, k, src, grid_w, radius, ids, dists)
    del keep
    return ids.reshape(Q, k), dists.reshape(Q, k)


def pair_dists(X, Y, ids) -> np.ndarray:
    X, Y = _f32(X), _f32(Y)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    Q, k = ids.shape
    out = np.empty(Q * k, np.float64)
    lib().oracle_pair_dists(X, X.shape[1], Y, Q, k, ids.reshape(-1), out)
    return out.reshape(Q, k)
