"""Host logic of bench.py on CPU: the clock probe's parsing, the wall-time ladder protocol on a
stand-in simulator, the BF16-exact column count behind the roofline's FLOPs per term, and the
refusal of more than one GPU."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_next_rung_doubles_far_from_the_target_then_predicts():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.next_rung(16, 0.40, 0.05, 1024) == 32          # far: double
    assert bench.next_rung(256, 0.0758, 0.05, 1024) == 512      # above 1.5x the target: double
    # 512 (0.0506 / 0.05)^2 1.15 = 603.0 -> 608 (a multiple of 16)
    assert bench.next_rung(512, 0.0506, 0.05, 1024) == 608
    assert bench.next_rung(512, 0.0501, 0.05, 1024) == 592      # at least 15 % more groups
    assert bench.next_rung(512, 0.0500001, 0.05, 4096) >= 528   # at least one step more
    assert bench.next_rung(128, 0.074, 0.05, 4096) == 256       # at most twice
    assert bench.next_rung(512, 0.06, 0.05, 600) == 600         # never above the cap


def test_sps_ladder_raises_groups_then_runs_three_seeds(monkeypatch):
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
    out = bench.sps_ladder(w, [("split", "mala"), ("fp32", "rw")], max_groups=256, seeds=3, seeds_other=1)
    m = out["split_mala"]
    # 0.32 / sqrt(J / 16) * 1.01 <= 0.05 first at J = 1024 > 256: not reached at 256
    assert not m["reached"] and m["rung"] == "256 groups x 4096"
    assert [r["groups"] for r in m["ladder_seed1"]] == [16, 32, 64, 128, 256]
    assert len(m["seeds"]) == 1
    out = bench.sps_ladder(w, [("split", "rw")], max_groups=4096, seeds=3, seeds_other=3)
    r = out["split_rw"]
    # doubling to 512 (NSE 0.0571 < 0.075), then 512 (0.0571 / 0.05)^2 1.15 = 768.3 -> 784 groups
    # (NSE 0.0462)
    assert [x["groups"] for x in r["ladder_seed1"]] == [16, 32, 64, 128, 256, 512, 784]
    assert r["reached"] and r["rung"] == "784 groups x 4096"
    assert [x["seed"] for x in r["seeds"]] == [1, 2, 3]
    assert r["median_wall_s"] == 7.84
    assert out["target_log_ml_nse"] == 0.05


def test_sps_ladder_fp32_starts_at_the_split_rung(monkeypatch):
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
            nse = 0.32 / (J / 16) ** 0.5
            return types.SimpleNamespace(seconds=J / 100.0, log_ml=-1.0, log_ml_nse=nse, m_steps=7)

        def close(self):
            pass

    monkeypatch.setattr(pkg, "Sps", FakeSps)
    w = types.SimpleNamespace(X=None, y=None, C=2, J=16, N=4096)
    out = bench.sps_ladder(w, [("split", "mala"), ("split", "rw"), ("fp32", "rw")], max_groups=4096,
                           seeds=3, seeds_other=1)
    assert [r["seed"] for r in out["split_mala"]["seeds"]] == [1, 2, 3]
    assert [r["seed"] for r in out["split_rw"]["seeds"]] == [1]
    fp = [r for r in runs if r[0] == ("fp32", "rw")]
    # the split random walk reached the target at 768 groups (512 -> 754.4 -> 768)
    assert fp == [(("fp32", "rw"), 768, 1)]
    assert out["speedup_split_mala_vs_fp32_rw"] == 1.0


def test_exact_columns_and_flops_per_term():
    sys.path.insert(0, ROOT)
    import types
    import bench
    rng = np.random.default_rng(0)
    X = np.column_stack([np.ones(50), rng.standard_normal((50, 3)), (rng.random((50, 2)) < 0.3) * 1.0,
                         np.full(50, 3.0), np.full(50, 1.0 + 2.0 ** -9)])
    ex = bench.bf16_exact_columns(X)
    # intercept, dummies and 3.0 are exact; N(0,1) draws and 1 + 2^-9 (9 fraction bits) are not
    assert ex.tolist() == [True, False, False, False, True, True, True, False]
    w = types.SimpleNamespace(X=X, C=3, k=X.shape[1])
    assert bench.split_flops_per_term(w) == 2 * 2 * (3 * 4 + 2 * 4)


def test_more_than_one_gpu_is_refused():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0
    d = json.loads(p.stdout.strip().splitlines()[-1])
    assert d["n_gpus"] == 2 and "unavailable" in d
