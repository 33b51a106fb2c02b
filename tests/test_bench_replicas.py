"""Host logic of the benchmark's multi-process path.  The method does not shard one
program, so N ranks run N independent replicas: the whole-job rate is the evaluations
of all ranks over the slowest rank's time (checked with two gloo ranks on the CPU), and
the reference arm (the CPU oracle) runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    value, ms = bench.job_rate(100.0 + 50.0 * rank, 64, dist, "cpu")
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_single_process():
    import bench
    assert bench.job_rate(200.0, 64) == (320.0, 200.0)


def test_job_rate_takes_the_slowest_of_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, value, ms in out:
        assert ms == 150.0
        assert value == pytest.approx(2 * 64 / 0.150)


def _bench(args, env):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          timeout=300, env=dict(os.environ, **env), cwd=ROOT)


def test_reference_arm_on_a_nonzero_rank_does_no_work():
    r = _bench(["--impl", "reference", "--gpus", "2", "--workload", "small_socp"],
               {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_line():
    r = _bench(["--impl", "reference", "--workload", "small_socp", "--steps", "2", "--warmup", "3"],
               {"RANK": "0", "LOCAL_RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
