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


def test_sps_ladder_doubles_groups_then_runs_three_seeds(monkeypatch):
    # the wall-time protocol of the bench, on a stand-in simulator whose NSE falls as 1/sqrt(J)
    sys.path.insert(0, ROOT)
    import types
    import bench
    import paper_1304_4333_b300 as pkg

    runs = []

    class FakeSps:
        def __init__(self, X, y, C, prior_sd, seed, precision, mkernel):
            self.seed, self.form = seed, (precision, mkernel)

        def run(self, J, N, record=False):
            runs.append((self.form, J, self.seed))
            nse = 0.32 / (J / 16) ** 0.5 * (1.0 + 0.01 * self.seed)
            return types.SimpleNamespace(seconds=J / 100.0, log_ml=-1.0, log_ml_nse=nse, m_steps=7)

        def close(self):
            pass

    monkeypatch.setattr(pkg, "Sps", FakeSps)
    w = types.SimpleNamespace(X=None, y=None, C=2, J=16, N=4096)
    out = bench.sps_ladder(w, [("split", "mala"), ("fp32", "rw")], max_groups=256)
    m = out["split_mala"]
    # 0.32 / sqrt(J / 16) * 1.01 <= 0.05 first at J = 1024 > 256: not reached at 256
    assert not m["reached"] and m["rung"] == "256 groups x 4096"
    assert [r["groups"] for r in m["ladder_seed1"]] == [16, 32, 64, 128, 256]
    assert len(m["seeds"]) == 1
    out = bench.sps_ladder(w, [("split", "rw")], max_groups=4096)
    r = out["split_rw"]
    assert r["reached"] and r["rung"] == "1024 groups x 4096"
    assert [x["seed"] for x in r["seeds"]] == [1, 2, 3]
    assert r["median_wall_s"] == 10.24
    assert out["target_log_ml_nse"] == 0.05
