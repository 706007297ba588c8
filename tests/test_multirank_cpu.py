"""The multi-process paths of bench.py on the CPU (gloo, world size 2).

The work does not shard: several GPUs run independent replicas, and the only
exchange is the timing, the slowest rank's time against the units all ranks
processed.  Checked here: that reduction over two gloo ranks, and the reference
arm launched under torch.distributed.run with two processes (rank 0 alone
works and prints one line; the other rank exits 0 without output).
"""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _load_bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _load_bench()
        # rank r processed 8 + r units in 1 + r seconds
        value, slowest = bench.combine_over_ranks(8 + rank, 1.0 + rank, world)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"value": value, "slowest": slowest}, f)
    finally:
        dist.destroy_process_group()


def test_replica_rate_is_all_units_over_the_slowest_rank(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["slowest"] == 2.0
        assert d["value"] == pytest.approx((8 + 9) / 2.0)


def test_single_rank_rate():
    bench = _load_bench()
    assert bench.combine_over_ranks(10, 2.0, 1) == (5.0, 2.0)


def test_reference_arm_under_two_processes_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--workload", "c1", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "solves/s"
    assert d["cpu_baseline"]["kind"] == "oracle"
