"""Host logic of bench.py for N > 1 processes, on CPU with gloo ranks: the
job's time is the slowest rank's, its throughput all ranks' units over that
time; under torchrun the reference arm is run and printed by rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    secs = 1.0 + rank                      # rank 1 is the slower replica
    q.put((rank, bench.job_rate(100.0, secs, "cpu", world), bench.max_over_ranks(secs, "cpu", world)))
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_replica_rate_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, mx in out:
        assert mx == 2.0
        assert rate == 100.0          # 2 ranks x 100 units / 2 s


def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_other_workloads_run_only_without_the_headline_legs():
    """bench.py --workload torus3d is a profiling run of the curved-space
    kernels: without --no-e2e --no-extras --no-cpu-baseline it is refused
    before any device work, so the benchmark line is always turb3d's."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "torus3d"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "--no-e2e --no-extras --no-cpu-baseline" in (r.stdout + r.stderr)
