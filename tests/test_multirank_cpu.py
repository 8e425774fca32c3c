"""Host logic of the multi-GPU bench path (independent replicas, max-over-ranks timing) on CPU
ranks with the gloo backend, and the reference arm of bench.py (the CPU oracle)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        m = bench.max_over_ranks(ms, world, "cpu")
        v = bench.whole_job_mlups(1000, world, m)
        # a rank that finished early still reports the slowest rank's time
        q.put((rank, m, v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, m, v in got:
        assert m == 20.0
        assert abs(v - 2 * 1000 / 0.020 / 1e6) < 1e-12


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_mlups(2_000_000, 1, 1000.0) == 2.0


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--workload", "manufactured32", "--no-extras"], capture_output=True,
                         text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "MLUP/s" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0
    assert rec["cpu_baseline"]["cores"] == (os.cpu_count() or 1) or rec["cpu_baseline"]["cores"] == 1
    assert rec["steps"] == 2 and rec["warmup"] == 1
    assert rec["cycles_per_step"] == 11 and rec["final_rel_residual"] < 1e-10
    # the same config dict as the GPU arm prints for this workload
    sys.path.insert(0, ROOT)
    import bench
    from paper_1410_6609_gb300 import synth
    assert rec["config"] == {**bench.workload_config(synth.WORKLOADS["manufactured32"]), "parallelism": "single"}


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--workload", "manufactured32"], capture_output=True, text=True, timeout=120, cwd=ROOT,
                         env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""
