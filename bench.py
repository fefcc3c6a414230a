"""Benchmark: queries/s at recall@1 >= 0.9 of the cone-hash search on GB300.

Workload (the scale-up Gaussian case): N = 1,000,000 data and Q = 10,000
query vectors, d = 32, iid N(0,1) (seeds 1002 / 2002, +rank under torchrun),
key depth L = 2, k = 1.  The probe budget P is the smallest of a fixed
ladder whose recall@1 against exact linear search reaches 0.9.

One step = the whole path over one batch: build the index of the N points
(cone keys, histogram + scan, stable sort, permuted copy) and search the Q
queries (query order, probe lists, cone-major work list, tile scan, merge).
`value` = Q / device time of a step (CUDA events on the stream, inputs
resident in HBM, L2 flushed by a 256 MiB write before every step);
`e2e` = the same through host buffers (pinned H2D of X and Y, D2H of the
results inside the timed region).

--impl reference times the CPU oracle (the single-threaded plain program)
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FULL, Q_FULL, D, L, K = 1_000_000, 10_000, 32, 2, 1
P_LADDER = [64, 96, 128, 160, 192, 224, 256, 320, 384, 512]
MB_LADDER = [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256]
WORKLOAD = "gauss32: N=1,000,000 x d=32 data, Q=10,000 queries, iid N(0,1), L=2 (N_C=1984), k=1"
METRIC = "queries/s at recall@1>=0.9"
FP32_LANES_PER_SM = 128


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def gen(rank, n=N_FULL, q=Q_FULL):
    from paper_1509_03453_gb300 import datagen
    X = datagen.gaussian(n, D, 1002 + rank)
    Y = datagen.gaussian(q, D, 2002 + rank)
    return X, Y


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def recall1(ids, d2, gt_ids, gt_d2):
    hit = ids[:, 0] == gt_ids[:, 0]
    near = np.abs(d2[:, 0].astype(np.float64) - gt_d2[:, 0]) <= 1e-6 * gt_d2[:, 0]
    return float(np.mean(hit | near))


def profiled_traffic(kernel_md, sources):
    """DRAM bytes per launch from a committed ncu summary under profiles/,
    or None when the kernel's sources changed since the capture (the
    summary records a hash of them)."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", kernel_md)).read()
        h = hashlib.sha1(b"".join(open(os.path.join(ROOT, f), "rb").read() for f in sources)).hexdigest()[:16]
        rec = dict(line.split(":", 1) for line in txt.splitlines() if line.startswith(("traffic_bytes_per_launch:",
                                                                                    "kernel_source_sha1_16:")))
        if rec.get("kernel_source_sha1_16", "").split()[0] != h:
            return None
        return int(rec["traffic_bytes_per_launch"].split()[0])
    except Exception:
        return None


TC_SOURCES = ["paper_1509_03453_gb300/csrc/tc_scan_kernel.cuh", "paper_1509_03453_gb300/csrc/osann_tc.cuh",
              "paper_1509_03453_gb300/csrc/osann_device.cuh"]


def run_profile(args):
    """Only the warm-up and timed steps (fixed P, chosen path): the command
    the ncu captures under profiles/ run, so that the launch list holds
    exactly the kernels of the step."""
    import torch

    import paper_1509_03453_gb300 as osann
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    osann.load()
    if args.workload == "desc128":
        # the descriptor recipe (N = 2*10^6, d = 128, 1.02 GB of rows), L = 3, k = 10
        from paper_1509_03453_gb300 import datagen
        w = datagen.workload("desc128")
        X, Y, Lw, Kw = w["X"], w["Y"], w["L"], w["k"]
    else:
        X, Y = gen(0)
        Lw, Kw = L, K
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    P = args.P or 224
    times = []
    for i in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ix, _, _ = osann.build_search(Xd, Lw, Yd, P, Kw, path=args.path, sync=False)
        b.record()
        b.synchronize()
        ix.status()
        ix.close()
        if i >= args.warmup:
            times.append(a.elapsed_time(b))
    print(json.dumps({"profile_run": True, "workload": args.workload, "P": P, "path": args.path,
                      "ms_per_step": float(np.mean(times))}))


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1509_03453_gb300 as osann
    from paper_1509_03453_gb300 import build as libbuild

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not libbuild.up_to_date() and rank == 0:
        libbuild.build()
    if ws > 1:
        dist.barrier()
    osann.load()

    X, Y = gen(rank)
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.from_numpy(Y).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # ground truth (exact linear search on the GPU) and the probe budget
    idx = osann.Index(Xd, L)
    gt_ids, gt_d2 = (t.cpu().numpy() for t in idx.bruteforce(Yd, K))
    P, rec = None, None
    if args.P:
        P = args.P
        ids, d2 = idx.search(Yd, P, K)
        rec = recall1(ids.cpu().numpy(), d2.cpu().numpy(), gt_ids, gt_d2)
    else:
        for cand in P_LADDER:
            ids, d2 = idx.search(Yd, cand, K)
            rec = recall1(ids.cpu().numpy(), d2.cpu().numpy(), gt_ids, gt_d2)
            P = cand
            if rec >= 0.9:
                break
    if ws > 1:
        t = torch.tensor([P], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        P = int(t.item())
    ws_bytes = idx.workspace_size(Q_FULL, P, K)
    idx.close()
    work = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    out_ids = torch.empty((Q_FULL, K), dtype=torch.int64, device=dev)
    out_d2 = torch.empty((Q_FULL, K), dtype=torch.float32, device=dev)

    def step(path="auto"):
        # build and search in one call (osann_build_search): the query-side
        # steps run beside the build; the build's status is read after the step
        ix, _, _ = osann.build_search(Xd, L, Yd, P, K, path=path, sync=False, out=(out_ids, out_d2))
        return ix

    def check(ix):
        if ix.status() & 5:  # non-finite data or a device wait timeout
            raise RuntimeError("index build reported an error status")

    def timed(path, steps, warmup, with_stats=False):
        times = []
        for i in range(warmup + steps):
            flush.zero_()
            if with_stats and i == warmup:
                osann.stats(enable=True, reset=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ix = step(path)
            b.record(stream)
            b.synchronize()
            check(ix)
            ix.close()
            if i >= warmup:
                times.append(a.elapsed_time(b))
        st = osann.stats(enable=False) if with_stats else None
        return times, st

    # the timed step: the index rebuilt in place from the data and the Q
    # queries searched (osann_rebuild_search, query side beside the rebuild),
    # captured once as a CUDA graph and replayed -- every build and search
    # kernel runs in every step; the graph only removes launch gaps
    gix = osann.Index(Xd, L)
    gws = torch.empty(gix.workspace_size(Q_FULL, P, K), dtype=torch.uint8, device=dev)
    cap = torch.cuda.Stream(device=dev)  # graphs are captured on a non-default stream
    cap.wait_stream(stream)
    for _ in range(2):  # the first call allocates the rebuild's temporaries
        gix.rebuild_search(Xd, Yd, P, K, out=(out_ids, out_d2), workspace=gws, stream=cap)
    cap.synchronize()
    check(gix)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    launches0 = osann.launch_count()
    with torch.cuda.graph(graph, stream=cap, capture_error_mode="thread_local"):
        gix.rebuild_search(Xd, Yd, P, K, out=(out_ids, out_d2), workspace=gws, stream=cap)
    launches_per_step = osann.launch_count() - launches0
    torch.cuda.synchronize()

    def timed_graph(steps, warmup):
        times = []
        for i in range(warmup + steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            b.record(stream)
            b.synchronize()
            check(gix)
            if i >= warmup:
                times.append(a.elapsed_time(b))
        return times

    # warm-up, then exactly `steps` timed steps bracketed by barrier + sync
    timed_graph(0, args.warmup)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    t_wall0 = time.perf_counter()
    times = timed_graph(args.steps, 0)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = launches_per_step * args.steps
    clocks = sampler.stop()
    rec_graph = recall1(out_ids.cpu().numpy(), out_d2.cpu().numpy(), gt_ids, gt_d2)
    del graph
    gix.close()
    # the same step without the graph: one osann_build_search call (fresh index)
    eager_times, _ = timed("auto", max(3, args.steps // 2), 2)
    if ws > 1:
        dist.barrier()
    ms = sum(times) / len(times)
    ms_max = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(ms_max, op=dist.ReduceOp.MAX)
    ms_step = float(ms_max.item())
    value = ws * Q_FULL / (ms_step / 1e3)

    # multi-basis search (Sec. 3-D): R rotated indexes, P per basis the
    # smallest of a ladder with recall@1 >= 0.9; step = R asynchronous builds
    # + R searches + the duplicate-free merge, timed the same way
    multi = []
    if rank == 0 and ws == 1 and not args.no_multi:
        from paper_1509_03453_gb300 import datagen
        for R in (2, 4):
            rots = torch.from_numpy(datagen.rotations(R, D, 6000 + R)).to(dev)
            mi = osann.MultiIndex(Xd, L, rots)
            Pm, recm = None, 0.0
            for cand in MB_LADDER:
                ids, d2 = mi.search(Yd, cand, K)
                recm = recall1(ids.cpu().numpy(), d2.cpu().numpy(), gt_ids, gt_d2)
                Pm = cand
                if recm >= 0.9:
                    break
            mi.close()
            mt = []
            for i in range(args.warmup + args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                mi = osann.MultiIndex(Xd, L, rots, sync=False)
                mi.search(Yd, Pm, K)
                b.record(stream)
                b.synchronize()
                if mi.status() & 5:
                    raise RuntimeError("multi-basis build reported an error status")
                mi.close()
                if i >= args.warmup:
                    mt.append(a.elapsed_time(b))
            mms = float(np.mean(mt))
            multi.append({"R": R, "P_per_basis": Pm, "recall_at_1": round(recm, 4),
                          "value": round(Q_FULL / (mms / 1e3), 1), "unit": "queries/s", "ms_per_step": round(mms, 4),
                          "bases": "identity + seeded random rotations (QR of Gaussian, seed 6000 + R)"})

    # per-stage device times, from a separate pass (the stage events stay out
    # of the timed steps above)
    n_stat = max(3, args.steps // 2)
    _, stats = timed("auto", n_stat, 0, with_stats=True)

    # plain per-query fp32 scan and exact linear search, same P, same clocking
    plain_times, _ = timed("plain", max(3, args.steps // 2), 1)
    bf_times = []
    for i in range(3):
        ix = osann.Index(Xd, L)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ix.bruteforce(Yd, K)
        b.record(stream)
        b.synchronize()
        ix.close()
        if i:
            bf_times.append(a.elapsed_time(b))

    # end to end through host buffers (pinned), copies inside the timed region
    Xh = torch.from_numpy(X).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    ids_h = torch.empty((Q_FULL, K), dtype=torch.int64).pin_memory()
    d2_h = torch.empty((Q_FULL, K), dtype=torch.float32).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xd = Xh.to(dev, non_blocking=True)
        yd = Yh.to(dev, non_blocking=True)
        ix, _, _ = osann.build_search(xd, L, yd, P, K, sync=False, out=(out_ids, out_d2))
        ids_h.copy_(out_ids, non_blocking=True)
        d2_h.copy_(out_d2, non_blocking=True)
        b.record(stream)
        b.synchronize()
        check(ix)
        ix.close()
        if i >= args.warmup:
            e2e_times.append(a.elapsed_time(b))
    e2e_ms = sum(e2e_times) / len(e2e_times)
    e2e_t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_ms = float(e2e_t.item())

    # roofline of the dominant stage
    peaks, peak_src = load_peaks()
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in stats.items() if v[1]}
    stage_n = {k: v[1] / n_stat for k, v in stats.items() if v[1]}
    dom = max(stats, key=lambda s: stats[s][0])
    path_used = "tensor-core screen (fp16 operands)" if stats.get("tc_scan", (0, 0))[1] else (
        "batched fp32" if stats.get("tile_scan", (0, 0))[1] else "plain fp32")
    pairs = None
    roof = None
    # candidate pairs of the timed search (exact count from the probe lists)
    ix = osann.Index(Xd, L)
    off = ix.export()[1]
    pr = ix.probes(Yd, P)
    sizes = (off[1:] - off[:-1])
    pairs = int(sizes[pr].sum().item())
    ix.search(Yd, P, K, out=(out_ids, out_d2), workspace=work)
    screen = ix.screen_stats() if path_used.startswith("tensor") else None
    ix.close()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    dom_ms = stage_ms[dom]
    if dom == "tc_scan":
        # the contraction: 2d flops per (query, candidate) pair on 16-bit tensor
        # cores (fp16 and bf16 share the dense rate)
        flops = 2.0 * D * pairs
        peak = peaks.get("bf16_tflops", 1900.0)
        achieved = flops / (dom_ms / 1e3) / 1e12
        roof = {"kernel": dom, "bound": "tensor", "achieved": round(achieved, 2), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic("tc_scan_gauss32_N1M_Q10k_P224.md", TC_SOURCES),
                "traffic_source": "ncu capture in profiles/tc_scan_gauss32_N1M_Q10k_P224.md (null if the kernel changed)",
                "peak_source": f"{peak_src} bf16 dense (burst; fp16 has the same nominal rate)",
                "algorithmic": f"{pairs} (query, candidate) pairs x 2d flops per launch "
                               f"(issued MMA work is larger: padded tiles and one extra K block of 16)",
                "avg_launch_ms": round(dom_ms, 4)}
    elif dom in ("tile_scan", "plain_scan", "bruteforce"):
        flops = 3.0 * D * pairs  # d subtractions, d squares, d additions per pair
        peak = sm_count * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        achieved = flops / (dom_ms / 1e3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} fp32 lanes x 2 (FMA) x "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz",
                "algorithmic": f"{pairs} (query, candidate) pairs x 3d flops per launch",
                "avg_launch_ms": round(dom_ms, 4)}
    else:
        byts = 4.0 * N_FULL * D * 3
        achieved = byts / (dom_ms / 1e3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "peak_source": f"{peak_src} copy bandwidth",
                "avg_launch_ms": round(dom_ms, 4)}

    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "eager_ms_per_step": round(float(np.mean(eager_times)), 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded iid N(0,1), generated on the host)",
        "config": {"workload": WORKLOAD, "N": N_FULL, "Q": Q_FULL, "d": D, "L": L, "k": K, "P": P,
                   "path": f"auto -> {path_used}",
                   "step": "index build (rebuilt in place from the data: keys, cone table, permuted rows, screening operands) + search of the Q queries, one osann_rebuild_search call (query side beside the build) captured as a CUDA graph and replayed; the build's status read after every step; eager_ms_per_step: the same step as one osann_build_search call on a fresh index, no graph",
                   "l2": "flushed before every step by a 256 MiB device write (untimed)",
                   "parallelism": f"replicas x{ws} (independent data per rank)"},
        "recall_at_1": round(rec, 4),
        "recall_at_1_timed_step": round(rec_graph, 4),
        "latency_ms": {"p50": round(float(np.percentile(times, 50)), 4),
                       "p99": round(float(np.percentile(times, 99)), 4),
                       "note": "per batch step of Q queries"},
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "multi_basis": multi,
        "screen": screen,
        "stage_launches_per_step": stage_n,
        "plain_fp32": {"value": round(Q_FULL / (np.mean(plain_times) / 1e3), 1), "unit": "queries/s",
                       "ms_per_step": round(float(np.mean(plain_times)), 4)},
        "bruteforce_fp32": {"value": round(Q_FULL / (np.mean(bf_times) / 1e3), 1), "unit": "queries/s",
                            "ms_per_search": round(float(np.mean(bf_times)), 4), "recall_at_1": 1.0},
        "e2e": {"value": round(ws * Q_FULL / (e2e_ms / 1e3), 1), "unit": "queries/s",
                "ms_per_step": round(e2e_ms, 4),
                "h2d_bytes_per_step": int(X.nbytes + Y.nbytes),
                "d2h_bytes_per_step": int(out_ids.numel() * 8 + out_d2.numel() * 4)},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed": round(t_wall, 3),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(P, budget_s=args.cpu_budget)
    if rank == 0 and ws == 1 and args.serve_requests > 0:
        # the serving workload (three resident indexes), shortened: its own
        # numbers, reported beside the step throughput
        try:
            del Xd, Yd, work, flush
            torch.cuda.empty_cache()
            args_s = argparse.Namespace(**vars(args))
            args_s.serve_requests = min(args.serve_requests, 2000)
            sv = run_serving(args_s, emit=False)
            line["serving"] = {k: sv[k] for k in ("indexes", "requests", "queries", "slots", "max_batch",
                                                  "capacity_qps", "sustained_qps", "loads", "server")}
        except Exception as exc:  # reported, never fatal to the main line
            line["serving"] = {"error": repr(exc)[:300]}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def cpu_baseline(P, budget_s=15.0, rank=0):
    """The oracle as it stands, single-threaded, on a bounded sample: the full
    build of the N points plus a sample of the queries, scaled to a step of
    the whole workload (build + Q queries)."""
    import oracle
    oracle.build()
    X, Y = gen(rank)
    t0 = time.perf_counter()
    ref = oracle.Index(X, L)
    t_build = time.perf_counter() - t0
    n, t_search = 0, 0.0
    chunk = 25
    while t_search < max(1.0, budget_s - t_build) and n < Q_FULL:
        t1 = time.perf_counter()
        ref.search(Y[n:n + chunk], P, K)
        t_search += time.perf_counter() - t1
        n += chunk
    t_step = t_build + t_search * Q_FULL / n
    return {"value": round(Q_FULL / t_step, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle build of all {N_FULL} points ({t_build:.2f} s) + search of {n} of {Q_FULL} "
                      f"queries at P={P} ({t_search:.2f} s), scaled to build + {Q_FULL} queries",
            "P": P}


def run_reference(args):
    """CPU oracle arm: each step = oracle build + a bounded query sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    P = args.P or 224  # the GPU arm's recall@1 >= 0.9 budget on this workload (its P ladder)
    X, Y = gen(0)
    sample = 40
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ref = oracle.Index(X, L)
        tb = time.perf_counter() - t0
        t1 = time.perf_counter()
        s = (i * sample) % (Q_FULL - sample)
        ref.search(Y[s:s + sample], P, K)
        tq = time.perf_counter() - t1
        if i >= args.warmup:
            times.append(tb + tq * Q_FULL / sample)
    t_step = float(np.mean(times))
    value = Q_FULL / t_step
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "queries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded iid N(0,1))",
            "config": {"workload": WORKLOAD, "N": N_FULL, "Q": Q_FULL, "d": D, "L": L, "k": K, "P": P},
            "cpu_baseline": {"value": round(value, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step: oracle build of all {N_FULL} points + {sample} queries at "
                                       f"P={P}, scaled to {Q_FULL} queries"},
            "e2e": {"value": round(value, 3), "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- serving

SERVE_SEED = 5000
SERVE_POOL = 8192
SERVE_LADDER = [16, 32, 64, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 6144, 8192, 12288,
                16384]


def serve_indexes():
    """The three resident indexes of the serving workload: (name, X, query
    pool, L, PCA components or 0).  Gaussian rows iid N(0,1); descriptor rows
    as the descriptor recipe, keyed on their first 16 principal components
    (the PCA front-end of Sec. 4-B); query pools are fresh draws (seeds
    5001..5003)."""
    from paper_1509_03453_gb300 import datagen
    return [
        ("gauss32 N=1M", datagen.gaussian(1_000_000, 32, 1002), datagen.gaussian(SERVE_POOL, 32, 5001), 2, 0),
        ("gauss64 N=4M", datagen.gaussian(4_000_000, 64, 1005), datagen.gaussian(SERVE_POOL, 64, 5002), 2, 0),
        ("desc128 N=2M (PCA 16)", datagen.descriptors(2_000_000, 1004), datagen.descriptor_queries(SERVE_POOL, 5003),
         3, 16),
    ]


def run_serving(args, emit=True):
    """Poisson-arriving requests of 1..4096 queries (log-uniform sizes,
    uniform index) through the request server; capacity first (all requests
    at once), then open-loop loads at 50/80/95% of it."""
    import torch

    import paper_1509_03453_gb300 as osann
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    osann.load()
    specs = serve_indexes()
    idx, pools, Ps, names, recalls = [], [], [], [], []
    for name, X, Y, Lk, m in specs:
        if m:
            from paper_1509_03453_gb300.pca import pca_basis
            axes, off = pca_basis(X, m, seed=SERVE_SEED)
            ix = osann.Index(torch.from_numpy(X).to(dev), Lk, rot=torch.from_numpy(axes).to(dev),
                             rot_offset=torch.from_numpy(off).to(dev))
        else:
            ix = osann.Index(torch.from_numpy(X).to(dev), Lk)
        pool = torch.from_numpy(Y).to(dev)
        gt_ids, gt_d2 = (t.cpu().numpy() for t in ix.bruteforce(pool[:1000], 1))
        P, rec = SERVE_LADDER[-1], 0.0
        for cand in SERVE_LADDER:
            ids, d2 = (t.cpu().numpy() for t in ix.search(pool[:1000], cand, 1))
            rec = recall1(ids, d2, gt_ids, gt_d2)
            if rec >= 0.9:
                P = cand
                break
        idx.append(ix)
        pools.append(pool)
        Ps.append(P)
        names.append(name)
        recalls.append(round(rec, 4))
    srv = osann.Server(idx, P=Ps, k=[1] * len(idx), slots=args.serve_slots, max_batch=4096,
                       mem_budget=int(args.serve_mem_gb * (1 << 30)), graphs=True)
    choices = srv.tune(reps=2, queries=pools)
    rng = np.random.default_rng(SERVE_SEED)
    n_req = args.serve_requests
    sizes = np.floor(np.exp(rng.uniform(0.0, np.log(4096.0), n_req))).astype(np.int64).clip(1, 4096)
    which = rng.integers(0, len(idx), n_req)
    offs = np.array([rng.integers(0, SERVE_POOL - s + 1) for s in sizes], dtype=np.int64)
    total_q = int(sizes.sum())

    def drive(arrivals):
        lat = np.zeros(n_req)
        t0 = time.perf_counter()
        nxt, done = 0, 0
        owner = {}
        while done < n_req:
            now = time.perf_counter() - t0
            while nxt < n_req and arrivals[nxt] <= now:
                i = int(which[nxt])
                t = srv.submit(i, pools[i][offs[nxt]:offs[nxt] + sizes[nxt]])
                owner[t] = nxt
                nxt += 1
            got = srv.progress(wait=False)
            tn = time.perf_counter() - t0
            for t in got:
                j = owner.pop(t)
                srv.result(t)
                lat[j] = tn - arrivals[j]
                done += 1
        return time.perf_counter() - t0, lat

    # warm-up: capture every graph the run needs
    srv.warmup()  # every (slot, index, bucket) graph captured before timing
    el, _ = drive(np.zeros(n_req))
    capacity = total_q / el  # closed loop: every request queued at once, full batches
    loads = []
    mean_size = total_q / n_req
    # open loop: Poisson arrivals at fractions of the closed-loop capacity; the
    # sustained capacity is the largest offered rate the server keeps up with
    # (achieved >= 95% of offered)
    sustained = 0.0
    for frac in (0.1, 0.2, 0.3, 0.45, 0.6, 0.8):
        rate = frac * capacity / mean_size
        arr = np.cumsum(rng.exponential(1.0 / rate, n_req))
        arr -= arr[0]
        el, lat = drive(arr)
        achieved = total_q / el
        offered = total_q / max(arr[-1], 1e-9)
        keeps_up = achieved >= 0.95 * offered
        if keeps_up:
            sustained = max(sustained, offered)
        loads.append({"offered_frac": frac, "offered_qps": round(offered, 1), "qps": round(achieved, 1),
                      "keeps_up": bool(keeps_up),
                      "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                      "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3)})
    st = srv.stats()
    out = {
        "serving": True,
        "metric": "request latency p50/p99 and queries/s at recall@1>=0.9",
        "indexes": [{"name": n, "P": p, "recall_at_1": r, "tuned": [list(c) for c in ch]}
                    for n, p, r, ch in zip(names, Ps, recalls, choices)],
        "requests": n_req, "queries": total_q, "sizes": "floor(exp(U(0, ln 4096))), index uniform",
        "slots": srv.slots, "max_batch": 4096, "graphs": True,
        "capacity_qps": round(capacity, 1), "capacity_note": "closed loop (all requests queued at once)",
        "sustained_qps": round(sustained, 1), "loads": loads,
        "server": st,
    }
    srv.close()
    for ix in idx:
        ix.close()
    if emit:
        print(json.dumps(out))
    return out


def run_rosanna_plus(args):
    """ROSANNA+ (Sec. 4-B) against the one-basis search and the PCA front-end,
    each at the smallest ladder budget with recall@1 >= 0.9 (search only,
    index prebuilt; median of 5 timed searches): the descriptor stand-in
    (N = 5*10^5 of the desc128 recipe, weakly structured) and a 256-component
    Gaussian mixture (d = 32, N = 10^6, means N(0, 9 I), unit spread)."""
    import torch

    import paper_1509_03453_gb300 as osann
    from paper_1509_03453_gb300 import build as libbuild
    from paper_1509_03453_gb300 import datagen
    from paper_1509_03453_gb300.kmeans import kmeans
    from paper_1509_03453_gb300.pca import pca_basis

    if not libbuild.up_to_date():
        libbuild.build()
    osann.load()
    dev = torch.device("cuda", 0)
    Qn = 2000
    ladder = [4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384]

    def measure(Xd, Yd, gt, make, cases):
        res = []
        for name, ix_args, M in cases:
            ix = make(ix_args)
            best = None
            for P in ladder:
                if P > ix.n_cones // max(ix.K, 1):
                    break
                f = (lambda: ix.search(Yd, P, 1, clusters=M)) if M > 1 else (lambda: ix.search(Yd, P, 1))
                ids, d2 = f()
                r = recall1(ids.cpu().numpy(), d2.cpu().numpy(), *gt)
                if r >= 0.9:
                    ts = []
                    for _ in range(5):
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record()
                        f()
                        b.record()
                        b.synchronize()
                        ts.append(a.elapsed_time(b))
                    best = {"case": name, "clusters_visited": M, "P": P, "recall_at_1": round(r, 4),
                            "search_ms": round(float(np.median(ts)), 4),
                            "queries_per_s": round(Qn / (float(np.median(ts)) / 1e3), 1)}
                    break
            res.append(best or {"case": name, "clusters_visited": M, "P": None,
                                "note": "recall@1 0.9 not reached on the ladder"})
            ix.close()
        return res

    out = {"rosanna_plus": True, "metric": "search time at recall@1>=0.9 (Q = 2000, k = 1)", "workloads": []}
    # descriptor stand-in
    w = datagen.workload("desc128", n=500_000, q=Qn)
    X, Y = w["X"], w["Y"]
    Xd, Yd = torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)
    ix0 = osann.Index(Xd, 3)
    gt = tuple(t.cpu().numpy() for t in ix0.bruteforce(Yd, 1))
    ix0.close()
    A, off = pca_basis(X, 16, seed=0)
    C = torch.from_numpy(kmeans(X, 64, iters=10, sample=50_000, seed=64)).to(dev)
    At, offt = torch.from_numpy(A).to(dev), torch.from_numpy(off).to(dev)

    def make_d(a):
        kind, L = a
        if kind == "plain":
            return osann.Index(Xd, L)
        if kind == "pca":
            return osann.Index(Xd, L, rot=At, rot_offset=offt)
        return osann.Index(Xd, L, centroids=C)
    cases = [("one basis, L=3", ("plain", 3), 1), ("PCA front-end (16 axes), L=3", ("pca", 3), 1)]
    cases += [(f"ROSANNA+ K=64, L=2, M={M}", ("plus", 2), M) for M in (4, 16)]
    out["workloads"].append({"workload": "desc128 recipe, N=500,000, d=128", "results": measure(Xd, Yd, gt, make_d, cases)})
    del Xd, Yd
    # Gaussian mixture
    N, d, B = 1_000_000, 32, 256
    rng = np.random.default_rng(1007)
    cent = 3.0 * rng.standard_normal((B, d))
    X = (cent[rng.integers(B, size=N)] + rng.standard_normal((N, d))).astype(np.float32)
    rq = np.random.default_rng(2007)
    Y = (cent[rq.integers(B, size=Qn)] + rq.standard_normal((Qn, d))).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)
    ix0 = osann.Index(Xd, 2)
    gt = tuple(t.cpu().numpy() for t in ix0.bruteforce(Yd, 1))
    ix0.close()
    C = torch.from_numpy(kmeans(X, 64, iters=10, sample=100_000, seed=64)).to(dev)

    def make_m(a):
        kind, L = a
        return osann.Index(Xd, L) if kind == "plain" else osann.Index(Xd, L, centroids=C)
    cases = [("one basis, L=2", ("plain", 2), 1)] + [(f"ROSANNA+ K=64, L=2, M={M}", ("plus", 2), M) for M in (1, 2)]
    out["workloads"].append({"workload": "Gaussian mixture, 256 components, N=10^6, d=32",
                             "results": measure(Xd, Yd, gt, make_m, cases)})
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="osann", choices=["osann", "reference"])
    ap.add_argument("--P", type=int, default=0, help="fixed probe budget (default: recall ladder)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="only warm-up + timed steps (for ncu captures)")
    ap.add_argument("--path", default="auto", choices=["auto", "plain", "batched", "bf16", "fp16"])
    ap.add_argument("--workload", default="gauss32", choices=["gauss32", "desc128"],
                    help="workload of --profile runs")
    ap.add_argument("--serving", action="store_true", help="the request-server workload (three resident indexes)")
    ap.add_argument("--no-multi", action="store_true", help="skip the multi-basis (R > 1) measurement")
    ap.add_argument("--rosanna-plus", action="store_true",
                    help="ROSANNA+ vs the one-basis search and the PCA front-end (search times at recall 0.9)")
    ap.add_argument("--serve-requests", type=int, default=10_000,
                    help="requests of the serving workload (0: skip it in the default run)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-mem-gb", type=float, default=8.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile(args)
    elif args.serving:
        run_serving(args)
    elif args.rosanna_plus:
        run_rosanna_plus(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
