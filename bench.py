"""Benchmark of the linear-BVH search path on the large mixture workload.

A step is one pass of the whole hot path over one batch: build the BVH over
N = 10M float32 3D points (bounds, Morton codes, radix sort, Apetrei build, top
levels), answer M = 10M radius queries as CRS with squared distances (query
sort, count, scan, fill) and M = 10M k=16 nearest queries.  The metric is
queries per second (radius + kNN queries per step / step time), inputs already
resident in HBM when the timed region starts; the inputs (points, queries and
the 640 MB node array) are larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched with torch.distributed.run, one rank per GPU.  By default the
ranks split one batch (strong scaling): every rank builds the same tree over all
points and computes the same Morton order of all M queries, takes its
contiguous range of that order and answers it; its CRS offsets are then shifted
by the matches of the ranks before it, one 8-byte value per rank exchanged per
step.  `--shard replicas` gives every rank the whole workload instead (weak
scaling).  Timing is the maximum over ranks; the value is all ranks' queries
over that time.  Rank 0 prints one JSON line.  `--impl reference` times the CPU oracle (the all-pairs
brute force) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Mqueries/s kNN k=16+radius @10M 3D pts, exact; batched vs plain same B300"
UNIT = "Mqueries/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", "--points", dest="n", type=int, default=10_000_000)
    ap.add_argument("--m", "--queries", dest="m", type=int, default=10_000_000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--e2e-batches", type=int, default=6, help="query slices of the end-to-end step")
    ap.add_argument("--e2e-growth", type=float, default=1.0,
                    help="size ratio of consecutive end-to-end radius slices (kNN slices shrink by it; 1 = equal)")
    ap.add_argument("--cpu-sample", type=int, default=1000, help="queries of each kind timed on the oracle")
    ap.add_argument("--ref-sample", type=int, default=200, help="queries of each kind per reference step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-stats", action="store_true", help="skip the instrumented traversal (profiling runs)")
    ap.add_argument("--tuning", type=str, default="", help="JSON tuning dict passed to every query")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's default launch settings instead of searching them first")
    ap.add_argument("--workload", choices=["mixture", "forest", "serving"], default="mixture")
    ap.add_argument("--shard", choices=["queries", "replicas"], default="queries",
                    help="N > 1: split one batch's Morton-ordered queries over the ranks, or run a replica per rank")
    ap.add_argument("--serve-requests", type=int, default=20_000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=int, default=96)
    ap.add_argument("--forest-scale", choices=["full", "small"], default="full")
    ap.add_argument("--plain-sets", type=int, default=None, help="sets timed in the plain loop (default all)")
    ap.add_argument("--no-forest", action="store_true", help="skip the batched-vs-plain forest comparison")
    ap.add_argument("--forest-subsample", type=int, default=256,
                    help="sets of the 4096-set forest plan in the default line's batched-vs-plain comparison")
    ap.add_argument("--no-heightfield", action="store_true", help="skip the terrain ray / box measurements")
    ap.add_argument("--no-dbscan", action="store_true", help="skip the DBSCAN measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement of the default line")
    ap.add_argument("--line-serve-requests", type=int, default=1000,
                    help="requests of the serving stream measured in the default line")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, ms_rank: float, world: int, device=None) -> tuple[float, float]:
    """Whole-job rate under weak scaling: every rank processed units_per_rank
    units; the job took the slowest rank's time.  Returns (units per second
    over all ranks, that time in ms)."""
    ms = reduce_max(ms_rank, world, device)
    return world * units_per_rank / (ms / 1e3), ms


def shard_bounds(m: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous range [lo, hi) of the processing order answered by
    `rank`: near-equal parts, the first m % world ranks one longer."""
    q, rem = divmod(m, world)
    lo = rank * q + min(rank, rem)
    return lo, lo + q + (1 if rank < rem else 0)


def offsets_shift(local_nnz: int, rank: int, world: int, device=None) -> tuple[int, int]:
    """The one exchange step of the query-sharded form: every rank's match
    count, gathered; returns (this rank's offset shift = the matches of the
    ranks before it, the total over all ranks)."""
    if world == 1:
        return 0, local_nnz
    import torch
    import torch.distributed as dist
    mine = torch.tensor([local_nnz], dtype=torch.int64, device=device)
    every = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(every, mine)
    counts = [int(t.item()) for t in every]
    return sum(counts[:rank]), sum(counts)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(n, m, r, k):
    return {
        "workload": f"large mixture: N={n} float32 3D points of a 64-component Gaussian mixture "
                    f"(sigma log-uniform 1e-3..1e-1), M={m} queries from the same mixture, "
                    f"radius r={r:.9g} (mean 32 neighbours, CRS with d2) + kNN k={k}",
        "n_points": n, "n_queries": m, "radius": r, "k": k,
        "step": "build + radius CRS (sort, count, scan, fill) + kNN",
        "l2": "inputs larger than L2 (points 120 MB, queries 120 MB, nodes 640 MB at full size)",
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline

def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6400.0, "source": "fallback"}


# the translation unit of the traversal kernels: query.cu and what it includes
TRAVERSAL_SOURCES = ("paper_2507_23700_b300/csrc/query.cu", "paper_2507_23700_b300/csrc/query.cuh",
                     "paper_2507_23700_b300/csrc/traverse.cuh", "paper_2507_23700_b300/csrc/primitives.cuh",
                     "paper_2507_23700_b300/csrc/common.cuh", "include/arbx.h")


def _code_only(text: str) -> str:
    """C/C++ source without comments and blank space (comment edits do not
    change a kernel)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_sha() -> str:
    """Hash of the code the traversal kernels are compiled from (a DRAM
    capture stays valid while it is unchanged)."""
    h = hashlib.sha256()
    for f in TRAVERSAL_SOURCES:
        h.update(_code_only((ROOT / f).read_text()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str) -> float | None:
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources."""
    p = ROOT / "profiles" / "ncu_traffic.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    if d.get("source_sha") != source_sha():
        return None
    e = d.get("kernels", {}).get(kernel)
    return None if e is None else float(e["dram_bytes_per_launch_full_size"])


def slice_bounds(m: int, nb: int, growth: float) -> list[int]:
    """Boundaries of nb consecutive query slices whose sizes grow by `growth`
    (first slice m / (1 + g + ... + g^(nb-1))), ending at m."""
    w = [growth ** b for b in range(nb)]
    tot = sum(w)
    acc, out = 0.0, [0]
    for b in range(nb - 1):
        acc += w[b]
        out.append(min(m, int(round(m * acc / tot))))
    out.append(m)
    return out


def algorithmic_bytes(kernel: str, stats: dict, m: int, k: int, node_bytes: int,
                      knn_nodes: str = "knn_optimal") -> float | None:
    """Algorithmic bytes of one launch: per query the query record (12 B),
    the node records the method must touch, and the outputs: an int32 count
    (count pass), int64 offset plus int32 index and float32 d2 per match (fill
    pass), k (index, d2) pairs (nearest).  The nodes: for the spatial passes
    every node whose box passes the predicate (the count pass skips the
    subtrees its sphere contains); for kNN the nodes whose box lies within the
    query's final k-th distance ("knn_optimal", the set any exact best-first
    search opens), or with knn_nodes="knn" every node the kernel fetched."""
    if kernel == "spatial_fill":
        s = stats["radius"]
        return m * (12 + 8) + s["nodes"] * node_bytes + s["matches"] * 8
    if kernel == "spatial_count":
        # the count pass walks less of the tree (contained subtrees counted whole)
        s = stats.get("radius_count", stats["radius"])
        return m * (12 + 4) + s["nodes"] * node_bytes
    if kernel == "knn":
        s = stats.get(knn_nodes, stats["knn"])
        return m * (12 + k * 8) + s["nodes"] * node_bytes
    return None


def build_bytes_per_step(n: int, m: int, dim: int) -> dict:
    """Algorithmic bytes per step of the build, query-order and sort kernels
    (points of `dim` float32 coordinates): bounds read the points; Morton codes
    read them and write a 64-bit key and a 32-bit index; the gather reads the
    permutation and the point and writes its box; the chunked Apetrei pass
    reads each sorted box, its input index and its key and writes every node
    once (the few nodes across chunk boundaries, completed by the second
    Apetrei kernel, are not counted); query codes as Morton codes for the
    m queries (one order per step, shared by the radius and kNN calls).  The
    reduce-then-scan radix passes read the keys (histogram) and read and write
    key + index (scatter): 8 passes over the n build keys, 6 over the m query
    keys (the fill pass's 32-bit chunk keys are sorted by the single-launch
    look-back passes, reported apart)."""
    pb = 4 * dim
    half = 2 * pb + 8
    return {"bounds": n * pb, "morton": n * (pb + 12), "gather": n * (4 + pb + 2 * pb),
            "apetrei": n * (2 * pb + 4 + 8) + (n - 1) * (2 * half),
            "query_codes": m * (pb + 12),
            "radix_upsweep": 8 * n * 8 + 6 * m * 8,
            "radix_downsweep": 8 * n * 24 + 6 * m * 24}


# ------------------------------------------------------------------ CPU oracle timing

def time_oracle(points, queries, r, k, sample: int, seed: int = 7) -> dict:
    import oracle
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(queries), min(sample, len(queries)), replace=False))
    qs = queries[sel]
    t0 = time.perf_counter()
    oracle.radius(points, qs, r)
    t1 = time.perf_counter()
    oracle.knn(points, qs, k)
    t2 = time.perf_counter()
    cores = oracle.threads_used()
    return {"value": 2 * len(qs) / (t2 - t0) / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(qs)} radius + {len(qs)} kNN k={k} queries (seeded subset) against all "
                      f"{len(points)} points; radius {t1 - t0:.2f} s, kNN {t2 - t1:.2f} s"}


# ------------------------------------------------------------------ reference arm

def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads
    wl = workloads.large_mixture(a.n, a.m)
    pts, qs, r, k = wl["points"], wl["queries"], wl["radius"], wl["k"]
    rng = np.random.default_rng(99)
    times = []
    for i in range(a.warmup + a.steps):
        sel = np.sort(rng.choice(len(qs), a.ref_sample, replace=False))
        t0 = time.perf_counter()
        import oracle
        oracle.radius(pts, qs[sel], r)
        oracle.knn(pts, qs[sel], k)
        if i >= a.warmup:
            times.append(time.perf_counter() - t0)
    import oracle
    t = statistics.mean(times)
    value = 2 * a.ref_sample / t / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": workload_config(a.n, a.m, r, k),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
                             "sample": f"each step: {a.ref_sample} radius + {a.ref_sample} kNN k={k} "
                                       f"seeded queries against all {a.n} points"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_ours(a):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2507_23700_b300 as arbx
    import workloads

    wl = workloads.large_mixture(a.n, a.m)
    pts_h, qs_h, r, k = wl["points"], wl["queries"], wl["radius"], wl["k"]
    n, m = len(pts_h), len(qs_h)
    tuning = json.loads(a.tuning) if a.tuning else None
    pts = torch.from_numpy(pts_h).to(dev)
    qs = torch.from_numpy(qs_h).to(dev)
    stream = torch.cuda.current_stream()

    # launch-setting search (outside the timed region): the records it leaves
    # apply to every later query of this (n, m, kind) given no tuning
    autotuned = None
    if tuning is None and not a.no_autotune:
        tree = arbx.Tree(pts)
        autotuned = {"radius": tree.autotune(arbx.SPHERE, qs, r, sample=m),
                     "knn": tree.autotune(arbx.NEAREST, qs, k=k, sample=m)}
        autotuned = {kind: {"setting": st, "ms": ms} for kind, (st, ms) in autotuned.items()}
        tree.close()
        torch.cuda.synchronize()

    shard = world > 1 and a.shard == "queries"
    s_lo, s_hi = shard_bounds(m, rank, world) if shard else (0, m)
    m_rank = s_hi - s_lo  # queries this rank answers per step

    def step(p_dev, q_dev, marks=None):
        if marks is not None:
            marks[0].record(stream)
        tree = arbx.Tree(p_dev)
        if marks is not None:
            marks[1].record(stream)
        # one Morton order of the queries, shared by the radius and kNN calls
        order = tree.query_order(arbx.SPHERE, q_dev, r)
        if shard:
            # this rank's contiguous range of the order: its queries, already in
            # Morton order (the identity is their processing order)
            mine = order[s_lo:s_hi].long()
            q_dev = q_dev.index_select(0, mine)
            order = torch.arange(m_rank, dtype=torch.int32, device=q_dev.device)
        crs = tree.query_crs(arbx.SPHERE, q_dev, r, want_d2=True, tuning=tuning, order=order)
        if shard:
            # global CRS offsets: shifted by the matches of the ranks before this one
            shift, _ = offsets_shift(int(crs.indices.numel()), rank, world, dev)
            crs.offsets.add_(shift)
        if marks is not None:
            marks[2].record(stream)
        kidx, kd2 = tree.knn(q_dev, k, tuning=tuning, order=order)
        if marks is not None:
            marks[3].record(stream)
        return tree, crs, kidx, kd2

    for _ in range(a.warmup):
        tree, crs, kidx, kd2 = step(pts, qs)
        nnz = int(crs.indices.numel())
        del crs, kidx, kd2
        tree.close()
    torch.cuda.synchronize()

    # instrumented traversal (outside the timed region): node fetches and matches
    tree = arbx.Tree(pts)
    stats = None
    if not a.no_stats:
        stats = {"radius": tree.stats(arbx.SPHERE, qs, r, tuning=tuning),
                 "radius_count": tree.stats(arbx.SPHERE, qs, r, tuning=tuning, counting=True),
                 "knn": tree.stats(arbx.NEAREST, qs, k=k, tuning=tuning)}
        # the nodes any exact best-first search opens: box within the final k-th distance
        _, kd2_all = tree.knn(qs, k, tuning=tuning)
        stats["knn_optimal"] = tree.stats_r2(qs, kd2_all[:, -1].contiguous())
        del kd2_all
    node_bytes = tree.layout()["node_stride"]
    tree.close()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs.  The headline steps run with
    # the library's per-launch profiling off (its two events per launch add
    # host time to the synchronising build); a second timed region of the same
    # steps with profiling on gives the per-kernel device times.
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    launches0 = arbx.launch_count()
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(a.steps)]
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(a.steps):
        tree, crs, kidx, kd2 = step(pts, qs, marks[i])
        nnz = int(crs.indices.numel())
        del crs, kidx, kd2
        tree.close()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = arbx.launch_count() - launches0
    clk = clocks.stop()
    if shard:  # one batch of m radius + m kNN queries over all ranks, in the slowest rank's time
        ms = reduce_max(ev0.elapsed_time(ev1) / a.steps, world, dev)
        rate = 2 * m / (ms / 1e3)
    else:
        rate, ms = aggregate_rate(2 * m, ev0.elapsed_time(ev1) / a.steps, world, dev)
    phases = {"build_ms": statistics.median(mk[0].elapsed_time(mk[1]) for mk in marks),
              "radius_ms": statistics.median(mk[1].elapsed_time(mk[2]) for mk in marks),
              "knn_ms": statistics.median(mk[2].elapsed_time(mk[3]) for mk in marks)}
    value = rate / 1e6
    # profiled region: per-kernel device times (CUDA events around each launch)
    arbx.profile_reset()
    arbx.profile_enable(True)
    torch.cuda.synchronize()
    pv0, pv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pv0.record(stream)
    for i in range(a.steps):
        tree, crs, kidx, kd2 = step(pts, qs)
        del crs, kidx, kd2
        tree.close()
    pv1.record(stream)
    torch.cuda.synchronize()
    arbx.profile_enable(False)
    prof = arbx.profile_read()
    profiled_ms = pv0.elapsed_time(pv1) / a.steps

    # count-only query (pure COUNT callback, no storage) on a tree built once,
    # the analogue of the paper's "Query (count)" line of Table 1
    tree = arbx.Tree(pts)
    for _ in range(2):
        tree.count(qs, r)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(a.steps):
        cnt = tree.count(qs, r)
    c1.record(stream)
    torch.cuda.synchronize()
    count_ms = c0.elapsed_time(c1) / a.steps
    count_nnz = int(cnt.sum(dtype=torch.int64).item())
    del cnt

    # stack vs stackless traversal (same bytes; section 2.6) on the same tree
    def timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            del out
        return statistics.median(ts)
    traversal_ab = {}
    for name, sl in (("stack", 0), ("stackless", 1)):
        tu = dict(tuning or {}, stackless=sl, single_pass=0)
        traversal_ab[name] = {
            "count_ms": timed(lambda: tree.count(qs, r, tuning=tu)),
            "radius_crs_ms": timed(lambda: tree.query_crs(arbx.SPHERE, qs, r, want_d2=True, tuning=tu))}
    tu1 = dict(tuning or {}, single_pass=1)
    traversal_ab["single_pass"] = {
        "radius_crs_ms": timed(lambda: tree.query_crs(arbx.SPHERE, qs, r, want_d2=True, tuning=tu1))}
    tree.close()

    # ---- roofline of the dominant kernel
    top = max(prof.items(), key=lambda kv: kv[1][1])
    kname, (klaunches, kms) = top
    per_launch_ms = kms / klaunches
    peaks = measured_peaks()
    alg = algorithmic_bytes(kname, stats, m, k, node_bytes) if stats else None
    achieved = alg / (per_launch_ms / 1e3) / 1e9 if alg is not None else None
    tree_bytes = (n - 1) * node_bytes
    out_bytes = nnz * 8 + m * 8 if kname == "spatial_fill" else m * k * 8 if kname == "knn" else m * 4
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"] if achieved else None,
                "credit": ("nodes whose box lies within the final k-th distance (the set any exact best-first "
                           "search opens)" if kname == "knn" else "nodes whose box passes the predicate"),
                "peak_source": f"{peaks['source']} HBM copy bandwidth (MEASURED_PEAKS.json)",
                "traffic": committed_traffic(kname),
                "algorithmic_bytes_per_launch": alg, "launch_ms": per_launch_ms,
                "compulsory_gbs": (m * 12 + tree_bytes + out_bytes) / (per_launch_ms / 1e3) / 1e9}
    if stats:
        # the same figures for each traversal kernel of the step
        per = {}
        for kn in ("spatial_count", "spatial_fill", "knn"):
            if kn in prof:
                ms_k = prof[kn][1] / prof[kn][0]
                alg_k = algorithmic_bytes(kn, stats, m, k, node_bytes)
                ach = alg_k / (ms_k / 1e3) / 1e9
                per[kn] = {"launch_ms": ms_k, "achieved": ach, "frac": ach / peaks["hbm_gbs"],
                           "traffic": committed_traffic(kn)}
                if kn == "knn":
                    alg_f = algorithmic_bytes(kn, stats, m, k, node_bytes, knn_nodes="knn")
                    per[kn]["frac_fetched_nodes"] = alg_f / (ms_k / 1e3) / 1e9 / peaks["hbm_gbs"]
        roofline["per_kernel"] = per
        if kname == "knn":
            alg_f = algorithmic_bytes(kname, stats, m, k, node_bytes, knn_nodes="knn")
            roofline["frac_fetched_nodes"] = alg_f / (per_launch_ms / 1e3) / 1e9 / peaks["hbm_gbs"]
        roofline["visits_per_query"] = {"radius_nodes": stats["radius"]["nodes"] / m,
                                        "radius_count_nodes": stats["radius_count"]["nodes"] / m,
                                        "knn_nodes": stats["knn"]["nodes"] / m,
                                        "knn_optimal_nodes": stats["knn_optimal"]["nodes"] / m,
                                        "radius_matches": stats["radius"]["matches"] / m}
    # build, query-order and sort kernels of the step (bytes per step / time per step)
    bk = {}
    for kn, b in build_bytes_per_step(n, m, 3).items():
        if kn in prof and prof[kn][1] > 0:
            ms_step = prof[kn][1] / a.steps
            ach = b / (ms_step / 1e3) / 1e9
            bk[kn] = {"launches_per_step": prof[kn][0] / a.steps, "ms_per_step": ms_step, "bytes_per_step": b,
                      "achieved": ach, "frac": ach / peaks["hbm_gbs"]}
    roofline["build_kernels"] = bk
    kernels = {kn: {"launches": l, "ms_total": t, "share": t / sum(v[1] for v in prof.values())}
               for kn, (l, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # ---- end to end through the public API with host buffers: every step
    # copies the inputs from pinned host memory and reads every result back.
    # The queries go in on a second stream while the tree is built; the
    # queries are then answered in `e2e_batches` slices whose results go back
    # on the copy stream while the next slice computes (the step is bound by
    # the 4.2 GB download at about 57 GB/s).  With `e2e_growth` > 1 the radius
    # slices grow by it and the kNN slices shrink by it (a shorter first compute
    # and last download); equal slices measured faster (4 slices: 90.6 ms per
    # step, ratio 2: 103 ms).
    e_times = []
    d2h = 0
    if a.e2e_steps > 0:
        nb = max(1, a.e2e_batches)
        pts_pin = torch.from_numpy(pts_h).pin_memory()
        qs_pin = torch.from_numpy(qs_h).pin_memory()
        out_off = torch.empty(m + nb, dtype=torch.int64, pin_memory=True)   # per-slice offsets, one after another
        cap = int(nnz * 1.05) + 1024
        out_idx = torch.empty(cap, dtype=torch.int32, pin_memory=True)
        out_d2 = torch.empty(cap, dtype=torch.float32, pin_memory=True)
        out_kidx = torch.empty((m, k), dtype=torch.int32, pin_memory=True)
        out_kd2 = torch.empty((m, k), dtype=torch.float32, pin_memory=True)
        p_dev = torch.empty_like(pts)
        q_dev = torch.empty_like(qs)
        copy = torch.cuda.Stream()
        bounds = slice_bounds(m, nb, a.e2e_growth)
        kbounds = slice_bounds(m, nb, 1.0 / a.e2e_growth)
        for i in range(a.e2e_steps + 1):  # the first pass is a warm-up
            torch.cuda.synchronize()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            copy.wait_stream(stream)
            p_dev.copy_(pts_pin, non_blocking=True)
            with torch.cuda.stream(copy):
                q_dev.copy_(qs_pin, non_blocking=True)
            tree = arbx.Tree(p_dev)
            stream.wait_stream(copy)
            keep = []
            z = 0
            for b in range(nb):
                lo, hi = bounds[b], bounds[b + 1]
                crs = tree.query_crs(arbx.SPHERE, q_dev[lo:hi], r, want_d2=True, tuning=tuning)
                zb = int(crs.indices.numel())
                copy.wait_stream(stream)
                with torch.cuda.stream(copy):
                    out_off[lo + b:hi + b + 1].copy_(crs.offsets, non_blocking=True)
                    out_idx[z:z + zb].copy_(crs.indices, non_blocking=True)
                    out_d2[z:z + zb].copy_(crs.d2, non_blocking=True)
                z += zb
                keep.append(crs)
            for b in range(nb):
                lo, hi = kbounds[b], kbounds[b + 1]
                kidx, kd2 = tree.knn(q_dev[lo:hi], k, tuning=tuning)
                copy.wait_stream(stream)
                with torch.cuda.stream(copy):
                    out_kidx[lo:hi].copy_(kidx, non_blocking=True)
                    out_kd2[lo:hi].copy_(kd2, non_blocking=True)
                keep.append((kidx, kd2))
            stream.wait_stream(copy)
            e1.record(stream)
            torch.cuda.synchronize()
            d2h = (m + nb) * 8 + z * 8 + m * k * 8
            del keep, crs, kidx, kd2
            tree.close()
            if i > 0:
                e_times.append(e0.elapsed_time(e1))
    e2e = None
    if e_times:
        e_ms = reduce_max(statistics.median(e_times), world, dev)
        e2e = {"value": world * 2 * m / (e_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": e_ms,
               "form": "the whole batch per rank" if world > 1 else "one GPU",
               "query_slices": max(1, a.e2e_batches), "slice_growth": a.e2e_growth,
               "h2d_bytes_per_step": int(pts.numel() * 4 + qs.numel() * 4), "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = time_oracle(pts_h, qs_h, r, k, a.cpu_sample)

    terrain = None
    if not a.no_heightfield:
        terrain = heightfield_measure(arbx, dev)

    # DBSCAN (section 2.4) on the same points: eps = the radius, minPts = 16;
    # each call builds its own tree (included)
    db = None
    if not a.no_dbscan:
        labels, nc = arbx.dbscan(pts, r, 16)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            labels, nc = arbx.dbscan(pts, r, 16)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        db_ms = statistics.median(ts)
        db = {"eps": r, "min_pts": 16, "ms": db_ms, "mpts_per_s": n / (db_ms / 1e3) / 1e6, "clusters": nc,
              "noise_fraction": float((labels < 0).float().mean()), "includes": "tree build, core count, union, labels"}
        del labels

    serving = None
    if not a.no_serving:
        serving = serving_measure(arbx, dev, a.line_serve_requests, a.serve_slots, a.serve_budget_gb)

    batched = None
    if not a.no_forest:
        del pts, qs
        torch.cuda.empty_cache()
        batched = forest_compare(arbx, "full", dev, steps=3, plain_sets=None, subsample=a.forest_subsample)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong" if shard else "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(n, m, r, k), "phases": phases,
                "radius_mqps": m / (phases["radius_ms"] / 1e3) / 1e6,
                "knn_mqps": m / (phases["knn_ms"] / 1e3) / 1e6,
                "count_only": {"ms": count_ms, "mqps": m / (count_ms / 1e3) / 1e6,
                               "matches_equal_nnz": count_nnz == int(nnz)},
                "build_gprims": n / (phases["build_ms"] / 1e3) / 1e9,
                "nnz_radius": int(nnz), "gpu_launches": int(launches), "clocks": clk,
                "profiled_region_ms_per_step": profiled_ms,
                # library launches before the first timed step (ncu -s for a launch list of one step)
                "launches_before_timed": int(launches0),
                "roofline": roofline, "kernels": kernels, "e2e": e2e, "cpu_baseline": cpu,
                "tuning": tuning if tuning is not None else {"autotuned": autotuned},
                "traversal_ab": traversal_ab, "heightfield": terrain, "dbscan": db,
                "batched_vs_plain": batched, "serving": serving}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def heightfield_measure(arbx, dev, reps: int = 3) -> dict:
    """Terrain of 4,188,162 triangles (2048 x 1024 fBm grid), 4M rays and 4M
    boxes: build and query times with both node formats (section 2.5 ray
    predicates; box-intersect on triangles), medians of `reps` runs."""
    import torch
    import workloads
    stream = torch.cuda.current_stream()
    tris = torch.from_numpy(workloads.heightfield_triangles().reshape(-1, 9)).to(dev).view(-1, 3, 3)
    rays = torch.from_numpy(workloads.heightfield_rays()).to(dev)
    boxes = torch.from_numpy(workloads.heightfield_boxes()).to(dev)

    def timed(fn):
        out = fn()
        del out
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            del out
        return statistics.median(ts)

    m = rays.shape[0]
    res = {"workload": f"heightfield: {tris.shape[0]} triangles (2048x1024 fBm grid), {m} cosine-weighted rays, "
                       f"{boxes.shape[0]} boxes", "unit": "Mqueries/s"}
    for name, q in (("fp32", False), ("q16", True), ("p16", "parent")):
        build_ms = timed(lambda: arbx.Tree(tris, kind="triangle", quantized=q))
        t = arbx.Tree(tris, kind="triangle", quantized=q)
        r = {"build_ms": build_ms}
        for key, fn in (("ray_nearest", lambda: t.ray_nearest(rays)),
                        ("ray_nearest_k4", lambda: t.ray_nearest(rays, k=4)),
                        ("ray_intersect", lambda: t.ray_intersect(rays, ordered=False)),
                        ("ray_ordered_intersect", lambda: t.ray_intersect(rays, ordered=True)),
                        ("box_crs", lambda: t.box(boxes))):
            ms = timed(fn)
            r[key] = {"ms": ms, "mqps": m / (ms / 1e3) / 1e6}
        r["hits_per_ray"] = float(t.callback(arbx.RAY_INTERSECT, rays, arbx.CB_COUNT).float().mean())
        res[name] = r
        t.close()
    return res


FOREST_SCALES = {"full": (1e3, 1e6), "small": (1e2, 1e4)}


def forest_compare(arbx, scale: str, dev, steps: int = 3, plain_sets: int | None = None,
                   subsample: int | None = None, autotune: bool = True) -> dict:
    """Batched vs plain on the forest workload (4096 independent sets, dims
    {2,3,6}, per-set radius for ~16 neighbours, k=8), or on `subsample` sets
    of its plan drawn with a fixed seed (the same size law, fewer sets).
    Batched: one forest build, the launch setting searched by the forest
    autotuner (outside the timed region), then one CUDA-graph launch per step
    running the radius query (count, scan, fill) and kNN over all sets.
    Plain: per set, a tree build, a radius CRS query and a kNN query through
    the single-tree entry points, one set after another on one stream (all
    sets, or the first `plain_sets`, scaled to all queries).  Throughput =
    (radius + kNN queries) / time."""
    import torch
    import workloads
    lo, hi = FOREST_SCALES[scale]
    full_plan = workloads.forest_plan(size_lo=lo, size_hi=hi)
    sel = list(range(len(full_plan)))
    if subsample is not None and subsample < len(full_plan):
        sel = sorted(np.random.default_rng(20260).choice(len(full_plan), subsample, replace=False).tolist())
    plan = [full_plan[i] for i in sel]
    dims = np.array([p[0] for p in plan], np.int32)
    ns = np.array([p[1] for p in plan], np.int64)
    ms = np.array([p[2] for p in plan], np.int64)
    pts_d = torch.empty(int((ns * dims).sum()), dtype=torch.float32, device=dev)
    qs_d = torch.empty(int((ms * dims).sum()), dtype=torch.float32, device=dev)
    radii, sets = [], []
    po = qo = 0
    for s in range(len(plan)):
        fs = workloads.forest_set(full_plan, sel[s])
        n, m, d = len(fs.points), len(fs.queries), fs.dim
        pts_d[po:po + n * d].copy_(torch.from_numpy(fs.points.reshape(-1)))
        qs_d[qo:qo + m * d].copy_(torch.from_numpy(fs.queries.reshape(-1)))
        sets.append((po, n, qo, m, d))
        po += n * d
        qo += m * d
        radii.append(fs.radius)
    total_q = int(ms.sum())
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        forest = arbx.Forest(packed=pts_d, dims=dims, counts=ns, stream=stream)
        batch = arbx.ForestBatch(forest, ms, radii, stream=stream)
        # the search allocates outputs of its own: run it before ours exist
        setting = batch.tuning()
        if autotune:
            setting, _ = batch.autotune(qs_d, 8, stream=stream)
        off, idx, d2 = batch.radius(qs_d, stream=stream)
        nnz = int(off[-1].item())
        kidx, kd2 = batch.knn(qs_d, 8, stream=stream)
        nnz_d = torch.zeros(1, dtype=torch.int64, device=dev)
        stream.synchronize()
        graph = batch.graph(qs_d, off, idx, d2, nnz, nnz_d, 8, kidx, kd2, stream=stream)
        graph.launch(stream)  # warm-up
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        stream.synchronize()
        e0.record(stream)
        for _ in range(steps):
            graph.launch(stream)
        e1.record(stream)
        stream.synchronize()
        q_ms = e0.elapsed_time(e1) / steps
        forest.close()
        e0.record(stream)
        forest = arbx.Forest(packed=pts_d, dims=dims, counts=ns, stream=stream)
        e2.record(stream)
        stream.synchronize()
        b_ms = e0.elapsed_time(e2)
        # plain: one tree and two queries per set
        nplain = len(sets) if plain_sets is None else min(plain_sets, len(sets))
        for (po, n, qo, m, d) in sets[:2]:  # warm-up
            t = arbx.Tree(pts_d[po:po + n * d].view(n, d), stream=stream)
            t.radius(qs_d[qo:qo + m * d].view(m, d), radii[0], stream=stream)
        stream.synchronize()
        e0.record(stream)
        pq = 0
        for si, (po, n, qo, m, d) in enumerate(sets[:nplain]):
            t = arbx.Tree(pts_d[po:po + n * d].view(n, d), stream=stream)
            q = qs_d[qo:qo + m * d].view(m, d)
            o, i_, dd = t.radius(q, radii[si], stream=stream)
            ki, kd = t.knn(q, 8, stream=stream)
            pq += m
            del t, o, i_, dd, ki, kd
        e1.record(stream)
        stream.synchronize()
        p_ms = e0.elapsed_time(e1) * total_q / max(pq, 1)
    graph.close()
    batch.close()
    forest.close()
    which = (f"{len(plan)} sets" if len(plan) == len(full_plan) else
              f"{len(plan)} of the {len(full_plan)} sets of the plan (seeded subsample, same size law)")
    return {"workload": f"forest: {which}, dims uniform over {{2,3,6}}, sizes log-uniform "
                        f"[{lo:g}, {hi:g}] ({int(ns.sum())} points), {total_q} queries (0.5-2x per set), "
                        f"per-set radius for ~16 neighbours + kNN k=8",
            "n_sets": len(plan), "n_points": int(ns.sum()), "n_queries": total_q,
            "batched_setting": setting, "batched_autotuned": bool(autotune),
            "batched_query_mqps": 2 * total_q / (q_ms / 1e3) / 1e6, "batched_query_ms": q_ms,
            "batched_build_ms": b_ms,
            "batched_build_query_mqps": 2 * total_q / ((q_ms + b_ms) / 1e3) / 1e6,
            "plain_build_query_mqps": 2 * total_q / (p_ms / 1e3) / 1e6, "plain_ms": p_ms,
            "plain_sets_timed": nplain,
            "speedup_build_query": p_ms / (q_ms + b_ms), "nnz_radius": nnz}


def run_forest(a):
    import torch
    torch.cuda.set_device(0)
    import paper_2507_23700_b300 as arbx
    res = forest_compare(arbx, a.forest_scale, torch.device("cuda", 0), steps=a.steps,
                         plain_sets=a.plain_sets)
    print(json.dumps({"metric": "Mqueries/s forest radius+kNN k=8, batched (graph) vs plain",
                      "value": res["batched_build_query_mqps"], "unit": UNIT, "n_gpus": 1,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic", **res}), flush=True)


def serve_replay(arbx, sv, reqs, gaps=None, rate=None):
    """Submit every request (all at once, or at Poisson arrival times
    cumsum(gaps)/rate on the server clock), wait for each in another thread and
    release its result.  Returns the server's statistics."""
    import threading
    sv.reset_stats()
    tickets = []
    lock = threading.Condition()
    done = []

    def waiter():
        i = 0
        while True:
            with lock:
                while i >= len(tickets) and not done:
                    lock.wait()
                if i >= len(tickets):
                    return
                t = tickets[i]
            res = sv.wait(t)
            del res
            i += 1

    th = threading.Thread(target=waiter)
    th.start()
    t0 = sv.now()
    arrivals = None if gaps is None else t0 + np.cumsum(gaps) / rate
    for i, (tree, kind, q, r, k) in enumerate(reqs):
        arr = -1.0
        if arrivals is not None:
            arr = float(arrivals[i])
            delay = arr - sv.now()
            if delay > 0:
                time.sleep(delay)
        if kind == "count":
            t = sv.submit(tree, arbx.SPHERE, q, radius=r, callback=arbx.CB_COUNT, arrival_s=arr)
        elif kind == "radius":
            t = sv.submit(tree, arbx.SPHERE, q, radius=r, arrival_s=arr)
        else:
            t = sv.submit(tree, arbx.NEAREST, q, k=k, arrival_s=arr)
        with lock:
            tickets.append(t)
            lock.notify()
    with lock:
        done.append(True)
        lock.notify()
    th.join()
    return sv.stats()


def serving_measure(arbx, dev, nreq: int, slots: int, budget_gb: int, sweep: bool = False) -> dict:
    """Serving workload: 8 resident mixture trees of 1M-50M points, a stream
    of `nreq` requests with sizes log-uniform in [1, 1e6] queries and kinds
    uniform over {radius CRS, kNN k=1, 8, 32, count}; admission by device
    memory (the budget, capped by what the device has free).  Saturated
    throughput (every request submitted at once), then p50/p99 latency and
    throughput with Poisson arrivals at 0.7x the saturated request rate (and
    0.3, 0.5, 0.9x with `sweep`), beside the one-request-at-a-time form (one
    slot) on the same stream."""
    import torch
    import workloads
    st = workloads.serving_stream(nreq=nreq)
    trees_pts = [workloads.serving_tree_points(st, t) for t in range(len(st.tree_sizes))]
    radii = [float(np.float32(workloads.LARGE_RADIUS * (1e7 / len(p)) ** (1.0 / 3.0))) for p in trees_pts]
    kinds = [workloads.SERVE_KINDS[int(x)] for x in st.kinds]
    reqs = []
    for i in range(len(st.sizes)):
        t = int(st.trees[i])
        q = torch.from_numpy(workloads.serving_request_queries(st, i)).to(dev)
        kind = kinds[i]
        k = {"knn1": 1, "knn8": 8, "knn32": 32}.get(kind, 0)
        reqs.append((t, "knn" if k else kind, q, radii[t], k))
    total_q = int(st.sizes.sum())
    out = {"workload": f"serving: {len(trees_pts)} resident mixture trees ({', '.join(str(len(p)) for p in trees_pts)} "
                       f"points), {len(reqs)} requests of log-uniform 1..1e6 queries ({total_q} total), kinds "
                       f"uniform over radius CRS / kNN k=1, 8, 32 / count",
           "requests": len(reqs), "queries": total_q, "slots": slots, "budget_gb": budget_gb}

    def server(n_slots):
        sv = arbx.Server(slots=n_slots, hbm_budget_bytes=budget_gb << 30)
        for p in trees_pts:
            sv.add_tree(arbx.Tree(torch.from_numpy(p).to(dev)))
        return sv

    sv = server(slots)
    serve_replay(arbx, sv, reqs[:20])  # warm-up
    sat = serve_replay(arbx, sv, reqs)
    sat_rate = len(reqs) / (total_q / (sat["mqps"] * 1e6))
    out["saturated"] = sat
    for frac in ((0.7, 0.3, 0.5, 0.9) if sweep else (0.7,)):
        out[f"poisson_{frac}"] = serve_replay(arbx, sv, reqs, gaps=st.interarrival, rate=frac * sat_rate)
        out[f"poisson_{frac}"]["rate_req_s"] = frac * sat_rate
    sv.close()
    sv1 = server(1)
    serve_replay(arbx, sv1, reqs[:20])
    out["plain_saturated"] = serve_replay(arbx, sv1, reqs)
    out["plain_poisson_0.7"] = serve_replay(arbx, sv1, reqs, gaps=st.interarrival, rate=0.7 * sat_rate)
    sv1.close()
    out["served_vs_plain_saturated"] = sat["mqps"] / max(out["plain_saturated"]["mqps"], 1e-12)
    del reqs
    torch.cuda.empty_cache()
    return out


def run_serving(a):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import paper_2507_23700_b300 as arbx
    out = serving_measure(arbx, dev, a.serve_requests, a.serve_slots, a.serve_budget_gb, sweep=True)
    print(json.dumps({"metric": "served Mqueries/s and p50/p99 latency (Poisson arrivals at 0.7x saturation)",
                      "value": out["poisson_0.7"]["mqps"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic", **out}), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "forest":
        run_forest(a)
    elif a.workload == "serving":
        run_serving(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
