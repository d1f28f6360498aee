"""The multi-process path of bench.py on the CPU (gloo, world size 2): the
max-over-ranks timing, the whole-job aggregation, and the reference arm under
torchrun (rank 0 alone runs the oracle and prints one line)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    world, r, local = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    ms = 10.0 * (rank + 1)           # rank 1 is the slower one
    ms_max = bench.dist_max(ms, world)
    bench.barrier(world)
    q.put((r, world, ms_max, bench.aggregate_mlups(world, 1000, 5, ms_max)))
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, world, ms_max, mlups in out:
        assert world == 2 and ms_max == 20.0
        # both ranks' nodes over the slowest rank's time
        assert mlups == pytest.approx(2 * 1000 * 5 / 20e-3 / 1e6)
    assert sorted(o[0] for o in out) == [0, 1]


def test_reference_arm_under_torchrun_prints_one_line():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    from oracle import build as OB
    OB.build()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--side", "64",
           "--steps", "10", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["config"]["parallelism"] == "replica per GPU"
    assert d["cpu_baseline"]["kind"] == "oracle"
