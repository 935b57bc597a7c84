"""The multi-process path of bench.py on CPU (gloo, world size 2): process-group setup from the
torchrun environment, the barrier, the max over ranks of the timed region, and the reference
arm under torchrun (rank 0 alone prints one JSON line, every rank exits 0)."""
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


def _worker(rank, world, port, out_dir):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(float(rank + 1) * 0.5, w)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(m))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert vals == [1.0, 1.0]


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_clock_probe_parses_nvidia_smi(monkeypatch):
    # the bench's clock samples: one nvidia-smi query per sample, fields as the recipe's line
    sys.path.insert(0, ROOT)
    import bench

    class Out:
        stdout = "2032, 2032, Not Active, Not Active, Not Active, Active\n"

    calls = []
    monkeypatch.setattr(bench.subprocess, "run", lambda cmd, **kw: calls.append(cmd) or Out())
    p = bench.ClockProbe(3)
    p.sample()
    p.sample()
    s = p.summary()
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 2
    assert s["reasons"] == ["sw_power_cap"]
    assert calls[0][:3] == ["nvidia-smi", "-i", "3"] and all("-lms" not in c for c in calls[0])
    assert bench.ClockProbe(0).summary()["reasons"] == ["unsampled"]
