"""The multi-rank logic of bench.py on CPU: two gloo ranks agree on the
slowest rank's time and on the whole-job rate, pass the barrier; the
query-sharded form splits the processing order into contiguous near-equal
ranges and shifts each rank's CRS offsets by the matches of the ranks before
it (one gathered 8-byte value per rank); the reference arm under torchrun
prints exactly one line from rank 0.  (Options
after the script that prefix torchrun's own, like --n, are taken by torchrun,
hence --points / --queries.)"""
from __future__ import annotations

import json
import os
import subprocess
import sys
from pathlib import Path

import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_rank = 10.0 + 5.0 * rank           # rank 1 is the slow one
        rate, ms = bench.aggregate_rate(1000.0, ms_rank, world)
        bench.barrier(world)
        peak = bench.reduce_max(float(rank), world)
        Path(out_dir, f"r{rank}.json").write_text(json.dumps({"rate": rate, "ms": ms, "peak": peak}))
    finally:
        dist.destroy_process_group()


def _shard_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = bench.shard_bounds(10, rank, world)
        local_nnz = [7, 0, 5][rank]  # matches found by each rank's range
        shift, total = bench.offsets_shift(local_nnz, rank, world)
        Path(out_dir, f"s{rank}.json").write_text(json.dumps({"lo": lo, "hi": hi, "shift": shift, "total": total}))
    finally:
        dist.destroy_process_group()


def test_shard_bounds_partition_the_order():
    for m in (0, 1, 7, 10, 10_000_000, 10_000_001):
        for world in (1, 2, 3, 8):
            b = [bench_mod().shard_bounds(m, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == m
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1


def bench_mod():
    sys.path.insert(0, str(ROOT))
    import bench
    return bench


def test_three_gloo_ranks_shift_offsets(tmp_path):
    """The query-sharded form's one exchange: each rank's CRS offsets move by
    the matches of the ranks before it."""
    port = 31500 + os.getpid() % 1000
    mp.spawn(_shard_main, args=(3, port, str(tmp_path)), nprocs=3, join=True)
    res = [json.loads((tmp_path / f"s{r}.json").read_text()) for r in range(3)]
    assert [(r["lo"], r["hi"]) for r in res] == [(0, 4), (4, 7), (7, 10)]
    assert [r["shift"] for r in res] == [0, 7, 7] and all(r["total"] == 12 for r in res)


def test_two_gloo_ranks_agree(tmp_path):
    port = 29500 + os.getpid() % 1000
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.loads((tmp_path / f"r{r}.json").read_text()) for r in range(2)]
    for r in res:
        assert r["ms"] == 15.0 and r["peak"] == 1.0
        assert r["rate"] == pytest.approx(2 * 1000.0 / 0.015)


def test_reference_arm_under_torchrun_prints_once():
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), str(ROOT / "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--points", "20000", "--queries", "20000", "--ref-sample", "20"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
