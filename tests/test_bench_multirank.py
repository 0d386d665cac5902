"""The multi-rank parts of bench.py on CPU (gloo, two ranks): the timed
region is the maximum over ranks, the whole-job rate counts every rank's
pixels, and the reference arm under torchrun prints one line from rank 0
while the other rank exits without work."""
import json
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


def _worker(rank, world, port, times, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total = bench.max_over_ranks(times[rank], dist)
    rate = bench.whole_job_mpix_per_s(1_000_000, 10, world, total)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"total": total, "rate": rate}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo(tmp_path):
    import torch.multiprocessing as mp
    times = [812.5, 1093.25]
    mp.spawn(_worker, args=(2, _free_port(), times, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["total"] == max(times)
        # 2 ranks x 1 Mpix x 10 steps over the slowest rank's 1093.25 ms
        assert r["rate"] == pytest.approx(2 * 1e6 * 10 / (max(times) * 1e3))


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_mpix_per_s(2_000_000, 4, 1, 1000.0) == pytest.approx(8.0)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--leaves", "box10k", "--cams", "4", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0
