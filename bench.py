"""Benchmark of the SPS logit hot path on one B300 (or N independent replicas under torchrun).

Metric: particle-observation log-likelihood evaluations per second on the binary-logit workload
c2 (n = 20 000 observations, k = 30 covariates, 16 groups x 4096 particles; synthetic data,
seed 0). A step is one cycle of the simulator over one batch of new observations: the C phase
over the next 64 observations (reweighting, ESS, log-ML increment), the S phase (resampling
within each group and the gather), and one M step at the new prefix length (refresh of the
cached log-likelihood with the M-phase kernel, particle covariance, FP64 Cholesky, Philox
proposal, fused log-likelihood of the proposals, Metropolis accept, RNE of the monitoring
functions). Units counted per step: P x 64 (C phase) + 2 P t (the refresh and the proposals).

Between timed steps the L2 cache is flushed by writing a 512 MB buffer (X of c2 fits in L2);
each step is timed with CUDA events on the library's stream and the flush is outside the
timed events. `e2e` is the same metric through sps_loglik with pinned host buffers (theta in,
log-likelihoods out, copies inside the timed region). The oracle (plain FP64 numpy) is timed on
a bounded sample as the CPU baseline, and is the `--impl reference` arm.

The step's outputs stay on the device (no particle indices, Sigma or log-ML increments are
copied to the host; the M step's acceptance rate comes back for its step-size rule). SM clocks
and throttle reasons are sampled by one-shot nvidia-smi queries between timed steps (after the
first, middle and last step), never during one. `--sps-ladder` adds the wall time of whole
simulator runs to log-ML NSE <= 0.05 (groups doubled from 16 until seed 1 reaches it, then three
seeds at that rung).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle·obs loglik evals/s; SPS wall-s to log-ML NSE≤0.05 vs plain FP32"
UNIT = "particle-obs evals/s"
C_BLOCK = 64


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockProbe:
    """SM clocks and throttle reasons, sampled inside the timed loop between steps.

    Each sample is one `nvidia-smi --query-gpu` call made right after a timed step has finished
    on the GPU (its end event synchronised) and before the next one starts, so no query overlaps
    a timed step. A concurrent `nvidia-smi -lms` process was measured to slow this launch-bound
    step by about 60 % whatever its period (50, 200 or 1000 ms): while it runs, the host-side
    launches and synchronisations of the simulator take longer. Reads only: no setting is
    changed."""

    _NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    _QUERY = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.samples = []          # (sm_mhz, sm_max_mhz, reasons set)

    def sample(self):
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self._QUERY}",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                 timeout=20).stdout
        except Exception:
            return
        for line in out.splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 6 and f[0].replace(".", "").isdigit():
                self.samples.append((float(f[0]), float(f[1]),
                                     {self._NAMES[i] for i in range(4) if f[2 + i] == "Active"}))

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "reasons": sorted(set().union(*(s[2] for s in self.samples))),
                "samples": len(self.samples),
                "source": "nvidia-smi --query-gpu between timed steps (right after a step ends)"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- CPU oracle

def oracle_throughput(w, seconds: float = 12.0, particles: int = 256):
    """The oracle's log-likelihood (plain FP64 numpy) on a bounded sample of the workload."""
    import synthetic
    from oracle.logit import loglik
    th = synthetic.particles_around(w.theta_true, particles, 0.05, seed=3)
    loglik(w.X, w.y, th[:8], w.C, w.n)   # warm-up
    t0 = time.perf_counter()
    calls = 0
    while True:
        loglik(w.X, w.y, th, w.C, w.n)
        calls += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    units = calls * particles * w.n
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": units / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{calls} calls of loglik on {particles} particles x all {w.n} observations "
                      f"({el:.1f} s, numpy FP64; BLAS threads for X theta', one thread elsewhere)"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import synthetic
    w = synthetic.make_c2()
    per_step = []
    for i in range(args.warmup + args.steps):
        r = oracle_throughput(w, seconds=2.0, particles=128)
        if i >= args.warmup:
            per_step.append(r)
    value = statistics.median(r["value"] for r in per_step)
    ms = 1e3 * (128 * w.n) / value
    cpu = dict(per_step[-1])
    cpu["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c2 binary logit n=20000 k=30 P=65536 (oracle: 128-particle sample per step)",
                       "global_batch": 65536, "seq_len": w.n, "parallelism": "cpu"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def run_ours(args, world, rank, local):
    import torch
    import synthetic
    from paper_1304_4333_b300 import Sps
    from paper_1304_4333_b300 import _native as N
    import ctypes as C

    torch.cuda.set_device(local)
    w = synthetic.make_c2()
    P, n = w.P, w.n
    steps, warm = args.steps, args.warmup
    s = Sps(w.X, w.y, w.C, prior_sd=5.0, seed=1 + rank, precision=args.precision)
    # the fused kernel's default launch shape (the autotuner, sps_autotune, finds a shape 2 %
    # faster on this workload; it is not run here because it times candidates and would pick
    # differently inside a profiler, so that profiles would not show the timed kernel)
    tuned = None
    stream = torch.cuda.Stream()
    lib = s.lib
    lib.sps_set_stream(s.ctx, C.c_void_p(stream.cuda_stream))
    st = s.state(w.J, w.N, seed=100 + rank)
    t0 = n - C_BLOCK * (warm + steps + (1 if args.ncu_step else 0))
    theta0 = synthetic.particles_around(w.theta_true, P, 0.05, seed=2)
    st.set(theta0, None, t0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def counters(reset=0):
        a, b, c = C.c_int64(), C.c_int64(), C.c_double()
        lib.sps_counters(s.ctx, reset, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    # warm-up steps
    for _ in range(warm):
        with torch.cuda.stream(stream):
            flush.zero_()
        st.cphase(st.get_t() + C_BLOCK, outputs=False)
        st.sphase(indices=False)
        st.mstep(kernel=args.mkernel, sigma_used=False)
    torch.cuda.synchronize()
    if args.ncu_step:
        # one more step inside a profiler range: `ncu --profile-from-start off` captures exactly
        # the kernels of one step (C phase, S phase, M step)
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        st.cphase(st.get_t() + C_BLOCK, outputs=False)
        st.sphase(indices=False)
        st.mstep(kernel=args.mkernel, sigma_used=False)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    counters(reset=1)
    lib.sps_set_timing(s.ctx, 1)
    units = 0
    hot_units = 0
    ev_ms = []
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    clk = ClockProbe(local)
    probe_at = {0, steps // 2, steps - 1}      # three samples: start, middle and end of the loop
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        # the step's outputs stay on the device (no particle indices, Sigma or log-ML increments
        # copied to the host); the M step's acceptance rate still comes back for its rule
        t_new, _, _ = st.cphase(st.get_t() + C_BLOCK, outputs=False)
        st.sphase(indices=False)
        st.mstep(kernel=args.mkernel, sigma_used=False)
        b.record(stream)
        b.synchronize()
        ev_ms.append(a.elapsed_time(b))
        units += P * C_BLOCK + 2 * P * t_new
        hot_units += 2 * P * t_new
        if i in probe_at:
            clk.sample()
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    launches, hot_launches, hot_ms = counters(reset=1)
    lib.sps_set_timing(s.ctx, 0)
    dev_s = max_over_ranks(sum(ev_ms) / 1e3, world)
    total_units = units * world
    value = total_units / dev_s
    t_end = st.get_t()

    # e2e: sps_loglik through the C ABI with pinned host buffers, copies inside the timed region
    th_host = torch.from_numpy(synthetic.particles_around(w.theta_true, P, 0.05, seed=4)).pin_memory()
    ll_host = torch.empty(P, dtype=torch.float64).pin_memory()
    for _ in range(warm):
        s.loglik_host_ptr(th_host.data_ptr(), ll_host.data_ptr(), P, n, args.precision)
    e2e_t = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t1 = time.perf_counter()
        s.loglik_host_ptr(th_host.data_ptr(), ll_host.data_ptr(), P, n, args.precision)
        e2e_t.append(time.perf_counter() - t1)
    e2e_s = max_over_ranks(sum(e2e_t), world)
    e2e_value = world * steps * P * n / e2e_s

    if rank != 0:
        return
    pk = peaks()
    clock = clk.summary()
    # roofline of the fused log-likelihood kernel: SFU-bound (one ex2 per particle-observation
    # term for C = 2); peak = 148 SMs x 32 ex2/clk x max SM clock
    sm_max = pk.get("sm_max_mhz", 2032.0)
    sfu_peak = 148 * 32 * sm_max * 1e6 / 1e9        # Gop/s
    hot_avg_ms = hot_ms / max(hot_launches, 1)
    # algorithmic SFU work of the timed launches: one ex2 per particle-observation term (C = 2)
    achieved = hot_units * (w.C - 1) / (hot_ms * 1e-3) / 1e9 if hot_ms > 0 else 0.0
    tensor_ms = P * n * 2 * (w.C - 1) * (3 * 19 + 2 * 11) / (pk.get("bf16_tflops", 1778.4) * 1e12) * 1e3
    sfu_ms = P * n * (w.C - 1) / (sfu_peak * 1e9) * 1e3
    hbm_ms = n * 128 / (pk.get("hbm_gbs", 6496.8) * 1e9) * 1e3
    traffic, traffic_src = args.traffic, "--traffic" if args.traffic is not None else None
    if traffic is None:
        traffic, traffic_src = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * dev_s / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x2-split/f32/f64" if args.precision == "split" else "f32/f64", "data": "synthetic",
        "config": {"workload": "c2 binary logit n=20000 k=30 (intercept, 19 AR(1) N(0,1), 10 Bernoulli(0.3)), "
                               "16 groups x 4096 particles, one SPS cycle per step (C phase 64 obs, S phase, M step)",
                   "global_batch": P * world, "seq_len": n, "parallelism": f"replicas{world}",
                   "precision": args.precision, "mkernel": args.mkernel,
                   "tile_shape": ({"rows": tuned["tile_rows"], "cluster": tuned["cluster"],
                                   "chunk_obs": tuned["chunk_obs"], "source": "sps_autotune"} if tuned else None),
                   "l2": "flushed between steps (512 MB write)"},
        "wall_s": wall,
        "gpu_launches": launches,
        "clocks": clock,
        "ms_per_step_median": statistics.median(ev_ms),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": P * w.D * 8, "d2h_bytes_per_step": P * 8,
                "call": "sps_loglik(mem=HOST) on pinned buffers, full t = n"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": sfu_peak, "unit": "Gop/s (ex2)",
                     "frac": achieved / sfu_peak, "traffic": traffic,
                     "traffic_source": traffic_src,
                     "kernel": f"loglik_tc_kernel<1,{tuned['tile_rows'] if tuned else 256}>",
                     "launches_timed": hot_launches,
                     "avg_launch_ms": hot_avg_ms,
                     "bounds_ms_full_t": {"sfu": sfu_ms, "tensor_split": tensor_ms, "hbm": hbm_ms},
                     "peak_source": "148 SMs x 32 ex2/clk/SM x sm_max_mhz of MEASURED_PEAKS (ex2 rate from a probe)"},
    }
    if not args.no_sps:
        line["sps"] = sps_wall(w, rank)
    if args.sps_ladder:
        forms = [tuple(f.split("_")) for f in args.sps_ladder.split(",")]
        if any(f not in (("split", "rw"), ("split", "mala"), ("fp32", "rw"), ("fp32", "mala")) for f in forms):
            raise SystemExit(f"--sps-ladder: unknown form in {args.sps_ladder!r}")
        line.setdefault("sps", {})["ladder"] = sps_ladder(w, forms, args.sps_max_groups)
    if not args.no_cpu:
        line["cpu_baseline"] = oracle_throughput(w)
    print(json.dumps(line), flush=True)


def profiled_traffic():
    """DRAM bytes per launch of the fused kernel (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary, used only while the kernel source still hashes to the value
    recorded beside it; otherwise (None, reason)."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "loglik_tc_c2.md")
    csrc = os.path.join(ROOT, "paper_1304_4333_b300", "csrc")
    try:
        text = open(prof).read()
        h = hashlib.sha256()
        for f in ("loglik_tc.cu", "common.cuh"):
            h.update(open(os.path.join(csrc, f), "rb").read())
    except OSError:
        return None, "no ncu summary"
    tb = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    sh = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
    if not (tb and sh):
        return None, "no traffic figure in the ncu summary"
    if sh.group(1) != h.hexdigest()[:16]:
        return None, "kernel changed since the ncu capture"
    return float(tb.group(1)), "profiles/loglik_tc_c2.md (ncu, one launch of this workload)"


def sps_wall(w, rank):
    """Second half of the metric: wall time of the whole simulator (sps_run, Algorithm 2) on c2
    with the split-BF16 path (random-walk M kernel, and the MALA M kernel driven by the
    tensor-core gradient) and with the plain FP32 random-walk path, the log-ML NSE each reaches
    at the configured 16 x 4096 particles, and the projected wall time to NSE <= 0.05 (NSE
    scales as particles^-1/2 and the time as particles, so time x (NSE / 0.05)^2; labelled as
    projected)."""
    from paper_1304_4333_b300 import Sps
    out = {}
    for name, prec, mk in (("split", "split", "rw"), ("split_mala", "split", "mala"), ("fp32", "fp32", "rw")):
        s = Sps(w.X, w.y, w.C, prior_sd=5.0, seed=11 + rank, precision=prec, mkernel=mk)
        r = s.run(w.J, w.N, record=False)
        out[name] = {"wall_s": r.seconds, "log_ml": r.log_ml, "log_ml_nse": r.log_ml_nse,
                     "cycles": r.n_cycles, "m_steps": r.m_steps, "mkernel": mk,
                     "projected_wall_s_to_nse_0.05": r.seconds * max(1.0, (r.log_ml_nse / 0.05) ** 2)}
        s.close()
    out["speedup_vs_fp32"] = out["fp32"]["wall_s"] / out["split"]["wall_s"]
    out["speedup_mala_vs_fp32"] = out["fp32"]["wall_s"] / out["split_mala"]["wall_s"]
    out["projected_speedup_mala_vs_fp32"] = (out["fp32"]["projected_wall_s_to_nse_0.05"]
                                             / out["split_mala"]["projected_wall_s_to_nse_0.05"])
    out["particles"] = f"{w.J} groups x {w.N}"
    return out


def sps_ladder(w, forms, max_groups: int, target: float = 0.05):
    """The wall-time half of the metric as a measured protocol instead of a projection: for each
    form (precision, M kernel), run seed 1 at the workload's groups x particles and double the
    number of groups (particles per group stay at the workload's value, the resampling bound)
    until its log-ML NSE is at most the target; then run seeds 2 and 3 at that rung and report
    the median wall time of the three seeds with each seed's NSE. A form whose seed 1 misses the
    target at max_groups reports its last rung with "reached": false."""
    from paper_1304_4333_b300 import Sps
    out = {}
    for prec, mk in forms:
        def one(J, seed):
            s = Sps(w.X, w.y, w.C, prior_sd=5.0, seed=seed, precision=prec, mkernel=mk)
            try:
                r = s.run(J, w.N, record=False)
            finally:
                s.close()
            return {"groups": J, "seed": seed, "wall_s": r.seconds, "log_ml": r.log_ml,
                    "log_ml_nse": r.log_ml_nse, "m_steps": r.m_steps}
        rungs, J = [], w.J
        while True:
            rungs.append(one(J, 1))
            if rungs[-1]["log_ml_nse"] <= target or 2 * J > max_groups:
                break
            J *= 2
        reached = rungs[-1]["log_ml_nse"] <= target
        seeds = [rungs[-1]] + ([one(J, 2), one(J, 3)] if reached else [])
        walls = sorted(x["wall_s"] for x in seeds)
        out[f"{prec}_{mk}"] = {"reached": reached, "rung": f"{J} groups x {w.N}",
                               "median_wall_s": walls[len(walls) // 2], "seeds": seeds,
                               "ladder_seed1": [{k: x[k] for k in ("groups", "wall_s", "log_ml_nse")}
                                                for x in rungs]}
    out["target_log_ml_nse"] = target
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split", choices=["split", "fp32"])
    ap.add_argument("--mkernel", default="rw", choices=["rw", "mala"],
                    help="M kernel of the timed step (MALA evaluates through the gradient kernel)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sps", action="store_true", help="skip the whole-simulator wall-time runs")
    ap.add_argument("--sps-ladder", default="",
                    help="comma list of forms (split_rw, split_mala, fp32_rw) run to log-ML NSE <= 0.05 "
                         "by doubling the groups, three seeds at the rung reached (adds sps.ladder)")
    ap.add_argument("--sps-max-groups", type=int, default=1024)
    ap.add_argument("--ncu-step", action="store_true",
                    help="run one extra step after warm-up inside a CUDA profiler range (for ncu --profile-from-start off)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the fused kernel from an ncu capture")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
