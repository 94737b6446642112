"""The multi-process side of bench.py on the CPU (gloo, world size 2): replicas, no data-path exchange.

Each rank solves its own copy of the workload; the whole-job line takes the slowest rank's time and the
sum of the ranks' solved paths, and the reference arm runs on rank 0 only.
"""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        out[rank] = bench.combine_ranks(10.0 + 5.0 * rank, 1000 + rank, dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world_2():
    torch_mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = torch_mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    # both ranks see the slowest rank's time and the total of solved paths
    assert res[0] == res[1] == (15.0, 2001.0)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.combine_ranks(12.5, 7, None, "cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_its_line():
    """Rank 0 of the reference arm times the oracle on the host and prints the contract's JSON line."""
    import json

    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "solves/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert key in line
