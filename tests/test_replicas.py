"""The N > 1 path on the CPU, world size 2 over gloo (127.0.0.1): the replica
aggregation that bench.py applies under torchrun (the job's time is the
slowest rank's, the job's throughput counts every rank's work), and the
reference arm under torchrun, where rank 0 alone runs and prints one line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1101_0809_gb300.replicas import job_rate, max_over_ranks
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    seconds = [1.5, 3.0][rank]
    slowest = max_over_ranks(dist, seconds)
    rate = job_rate(dist, 1000.0, seconds)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, rate))


def test_replica_aggregation_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == 3.0                    # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000.0 / 3.0)


def test_single_process_aggregation_is_the_plain_rate():
    sys.path.insert(0, ROOT)
    from paper_1101_0809_gb300.replicas import job_rate, max_over_ranks
    assert max_over_ranks(None, 2.5) == 2.5
    assert job_rate(None, 100.0, 4.0) == 25.0


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1"]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
