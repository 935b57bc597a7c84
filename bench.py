"""Benchmark of the SPS logit hot path on one B300 (single GPU only).

Metric: particle-observation log-likelihood evaluations per second, and the wall time of the
whole simulator to log-ML NSE <= 0.05 against the plain FP32 form.

Headline workload (the largest configuration that fits one GPU): c4, binary logit with
n = 1 000 000 observations and k = 100 covariates (intercept, 69 equicorrelated N(0,1), 30
Bernoulli(0.1) dummies), 64 groups x 1024 particles, synthetic data (seed 0). A step is one
cycle of the simulator over one batch of new observations at the end of the data: the C phase
over the next 64 observations (reweighting, ESS, log-ML increment), the S phase (resampling
within each group and the gather), and one M step at the new prefix length (refresh of the
cached log-likelihood with the M-phase kernel, particle covariance, FP64 Cholesky, Philox
proposal, fused log-likelihood of the proposals, Metropolis accept, RNE of the monitoring
functions). Units counted per step: P x 64 (C phase) + 2 P t (the refresh and the proposals).
X of c4 (384 MB of split-BF16 operand rows) is larger than L2, so no flush is needed; the
second workload in the same line, c2 (n = 20 000, k = 30, 16 x 4096 particles, X 2.5 MB),
flushes L2 between steps by writing a 512 MB buffer outside the timed events. Steps are timed
with CUDA events on the library's stream.

`roofline` is the fused log-likelihood kernel's: for c4 tensor-bound (algorithmic split-BF16
FLOPs 2 (C-1)(3 k_cont + 2 k_exact) per term against the measured BF16 peak), for c2 bound by
its one ex2 per term (SFU). Each launch of the kernel is timed with CUDA events recorded by the
library on its stream (sps_set_timing). `e2e` is the same metric through sps_loglik with
pinned host buffers (theta in, log-likelihoods out, copies inside the timed region). The
oracle (plain FP64 numpy) is timed on a bounded sample as the CPU baseline, on all host cores
and on one, and is the `--impl reference` arm.

`sps.ladder`: the wall time of whole simulator runs (sps_run) on c2 to log-ML NSE <= 0.05:
seed 1 from 16 groups, the groups doubled while its NSE is above 1.5x the target, then set to
where NSE ~ 1/sqrt(groups) predicts the target (with a margin) until seed 1 reaches it (the plain
FP32 form starts at the rung the split random walk reached); then further seeds at that rung
(`--ladder-seeds`).

SM clocks and throttle reasons are sampled by one-shot nvidia-smi queries between timed steps
(after the first, middle and last step), never during one.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
TRAFFIC_SOURCES = ("loglik_tc.cu", "common.cuh")


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


def bf16_exact_columns(X: np.ndarray) -> np.ndarray:
    """Columns whose every value is exactly representable in BF16 (the 0/1 dummies and the
    intercept): an FP64 value is when it survives FP32 and its FP32 pattern has 16 zero low bits."""
    x32 = X.astype(np.float32)
    ok = (x32.astype(np.float64) == X) & ((x32.view(np.uint32) & 0xFFFF) == 0)
    return ok.all(axis=0)


def split_flops_per_term(w) -> int:
    """Algorithmic tensor work of one particle-observation term of the split-BF16 product:
    Th Xh' + Tl Xh' + Th Xl' per outcome (three products for a continuous column, two for an
    exact one), 2 FLOP per multiply-add."""
    exact = int(bf16_exact_columns(w.X).sum())
    return 2 * (w.C - 1) * (3 * (w.k - exact) + 2 * exact)


# ----------------------------------------------------------------------------- CPU oracle

def oracle_throughput(w, seconds: float = 10.0, particles: int = 16):
    """The oracle's log-likelihood (plain FP64 numpy) on a bounded sample of the workload: calls
    on `particles` particles over all n observations until `seconds` have passed (at least one).
    The product X theta' runs on the BLAS thread pool; the elementwise terms on one thread."""
    import synthetic
    from oracle.logit import loglik
    th = synthetic.particles_around(w.theta_true, particles, 0.05, seed=3)
    loglik(w.X[:1000], w.y[:1000], th[:2], w.C)   # warm-up
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
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "0")) or cores
    return {"value": units / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{calls} calls of loglik on {particles} particles x all {w.n} observations of "
                      f"{w.name} ({el:.1f} s, numpy FP64; {threads} BLAS thread(s) for X theta', one thread "
                      f"for the elementwise terms; {cores} cores available)"}


def oracle_single_thread(name: str, seconds: float, particles: int):
    """oracle_throughput in a child process whose BLAS pools are limited to one thread (the
    thread counts are read when numpy loads its BLAS, so they are set before the child starts)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench, synthetic; "
            f"print(json.dumps(bench.oracle_throughput(synthetic.make_workload({name!r}), {seconds}, {particles})))")
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    if p.returncode != 0:
        return {"error": p.stderr.strip().splitlines()[-1] if p.stderr.strip() else f"rc {p.returncode}"}
    return json.loads(p.stdout.strip().splitlines()[-1])


def oracle_sps():
    """The whole simulator against the oracle's. c1: one adaptive SPS run (random walk, 4 x 256
    particles, n = 500) in the oracle (plain FP64 numpy) and one on the GPU (split precision,
    after an untimed run). c2: the oracle's SPS time extrapolated -- labelled as such -- from the
    oracle's measured log-likelihood rate on c2 and the log-likelihood terms of a recorded GPU run
    (M steps: sum over cycles of R_l t_l P; C phases: n P); the oracle's other work is not
    counted, so the figure is a lower bound."""
    import numpy as np
    import synthetic
    from oracle import smc as OS
    from paper_1304_4333_b300 import Sps
    out = {}
    w1 = synthetic.make_c1()
    prior = OS.GaussianPrior.isotropic(w1.D, w1.prior_sd)
    t0 = time.perf_counter()
    ro = OS.sps_run(w1.X, w1.y, w1.C, prior, w1.J, w1.N, np.random.Generator(np.random.PCG64(1)))
    t_or = time.perf_counter() - t0
    s = Sps(w1.X, w1.y, w1.C, prior_sd=w1.prior_sd, seed=1)
    s.run(w1.J, w1.N, record=False)
    t0 = time.perf_counter()
    rg = s.run(w1.J, w1.N, record=False)
    t_gpu = time.perf_counter() - t0
    s.close()
    out["c1"] = {"groups_x_particles": f"{w1.J} x {w1.N}", "oracle_wall_s": t_or, "gpu_wall_s": t_gpu,
                 "oracle_log_ml": ro.log_ml, "oracle_log_ml_nse": ro.log_ml_nse,
                 "gpu_log_ml": rg.log_ml, "gpu_log_ml_nse": rg.log_ml_nse,
                 "oracle_m_steps": int(sum(c.R for c in ro.cycles)), "gpu_m_steps": int(rg.m_steps)}
    w2 = synthetic.make_c2()
    s = Sps(w2.X, w2.y, w2.C, prior_sd=5.0, seed=1)
    t0 = time.perf_counter()
    rg = s.run(w2.J, w2.N, record=True)
    t_gpu = time.perf_counter() - t0
    s.close()
    sch = rg.schedule
    terms = float(np.sum(np.asarray(sch.R, dtype=np.float64) * np.asarray(sch.t, dtype=np.float64))) * w2.P \
        + float(w2.n) * w2.P
    rate = oracle_throughput(w2, seconds=5.0, particles=64)
    out["c2"] = {"groups_x_particles": f"{w2.J} x {w2.N}", "gpu_wall_s": t_gpu, "gpu_m_steps": int(rg.m_steps),
                 "gpu_cycles": int(rg.n_cycles), "loglik_terms": terms, "oracle_terms_per_s": rate["value"],
                 "oracle_wall_s_extrapolated": terms / rate["value"],
                 "label": "extrapolated: the oracle's log-likelihood rate on c2 (" + rate["sample"] + ") times the "
                          "terms of the GPU run's M steps and C phases; a lower bound"}
    return out


def run_reference(args):
    """The oracle arm: the plain FP64 CPU log-likelihood on c4, each step a bounded sample (16
    particles over all 10^6 observations)."""
    import synthetic
    w = synthetic.make_c4()
    per_step = []
    for i in range(args.warmup + args.steps):
        r = oracle_throughput(w, seconds=0.0, particles=16)
        if i >= args.warmup:
            per_step.append(r)
    value = statistics.median(r["value"] for r in per_step)
    ms = 1e3 * (16 * w.n) / value
    cpu = dict(per_step[-1])
    cpu["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c4 binary logit n=1000000 k=100 P=65536 (oracle: 16-particle sample per step)",
                       "global_batch": 65536, "seq_len": w.n, "parallelism": "cpu"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def step_bench(w, args, flush_l2: bool, e2e: bool = True):
    """Time `args.steps` simulator cycles (C phase over C_BLOCK observations, S phase, one M
    step) at the end of the workload's data, after `args.warmup` untimed ones."""
    import ctypes as C
    import torch
    import synthetic
    from paper_1304_4333_b300 import Sps

    P, n = w.P, w.n
    steps, warm = args.steps, args.warmup
    s = Sps(w.X, w.y, w.C, prior_sd=5.0, seed=1, precision=args.precision)
    stream = torch.cuda.Stream()
    lib = s.lib
    lib.sps_set_stream(s.ctx, C.c_void_p(stream.cuda_stream))
    st = s.state(w.J, w.N, seed=100)
    t0 = n - C_BLOCK * (warm + steps + (1 if args.ncu_step else 0))
    theta0 = synthetic.particles_around(w.theta_true, P, 0.05, seed=2)
    st.set(theta0, None, t0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda") if flush_l2 else None

    def counters(reset=0):
        a, b, c = C.c_int64(), C.c_int64(), C.c_double()
        lib.sps_counters(s.ctx, reset, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def one_step():
        t_new, _, _ = st.cphase(st.get_t() + C_BLOCK, outputs=False)
        st.sphase(indices=False)
        st.mstep(kernel=args.mkernel, sigma_used=False)
        return t_new

    for _ in range(warm):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.zero_()
        one_step()
    torch.cuda.synchronize()
    if args.ncu_step:
        # one more step inside a profiler range: `ncu --profile-from-start off` captures exactly
        # the kernels of one step (C phase, S phase, M step)
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        one_step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    counters(reset=1)
    lib.sps_set_timing(s.ctx, 1)
    units = 0
    hot_units = 0
    ev_ms = []
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    clk = ClockProbe(0)
    probe_at = {0, steps // 2, steps - 1}      # three samples: start, middle and end of the loop
    for i in range(steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        # the step's outputs stay on the device (no particle indices, Sigma or log-ML increments
        # copied to the host); the M step's acceptance rate still comes back for its rule
        t_new = one_step()
        b.record(stream)
        b.synchronize()
        ev_ms.append(a.elapsed_time(b))
        units += P * C_BLOCK + 2 * P * t_new
        hot_units += 2 * P * t_new
        if i in probe_at:
            clk.sample()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches, hot_launches, hot_ms = counters(reset=1)
    lib.sps_set_timing(s.ctx, 0)
    dev_s = sum(ev_ms) / 1e3
    out = {"value": units / dev_s, "ms_per_step": 1e3 * dev_s / steps,
           "ms_per_step_median": statistics.median(ev_ms), "wall_s": wall, "gpu_launches": launches,
           "hot_launches": hot_launches, "hot_ms": hot_ms, "hot_units": hot_units, "units": units,
           "clocks": clk.summary(), "t_end": st.get_t()}
    del st
    if e2e:
        # sps_loglik through the C ABI with pinned host buffers, copies inside the timed region
        th_host = torch.from_numpy(synthetic.particles_around(w.theta_true, P, 0.05, seed=4)).pin_memory()
        ll_host = torch.empty(P, dtype=torch.float64).pin_memory()
        for _ in range(warm):
            s.loglik_host_ptr(th_host.data_ptr(), ll_host.data_ptr(), P, n, args.precision)
        e2e_t = []
        for _ in range(steps):
            if flush is not None:
                with torch.cuda.stream(stream):
                    flush.zero_()
            stream.synchronize()
            t1 = time.perf_counter()
            s.loglik_host_ptr(th_host.data_ptr(), ll_host.data_ptr(), P, n, args.precision)
            e2e_t.append(time.perf_counter() - t1)
        out["e2e"] = {"value": steps * P * n / sum(e2e_t), "unit": UNIT, "h2d_bytes_per_step": P * w.D * 8,
                      "d2h_bytes_per_step": P * 8,
                      "call": "sps_loglik(mem=HOST) on pinned buffers, full t = n"}
    s.close()
    return out


def profiled_traffic(name: str):
    """DRAM bytes per full launch of the fused kernel (dram__bytes_read.sum +
    dram__bytes_write.sum) from the committed ncu summary profiles/loglik_tc_<name>.md, used only
    while the kernel sources still hash to the value recorded there; otherwise (None, reason)."""
    prof = os.path.join(ROOT, "profiles", f"loglik_tc_{name}.md")
    csrc = os.path.join(ROOT, "paper_1304_4333_b300", "csrc")
    try:
        text = open(prof).read()
        h = hashlib.sha256()
        for f in TRAFFIC_SOURCES:
            h.update(open(os.path.join(csrc, f), "rb").read())
    except OSError:
        return None, "no ncu summary"
    tb = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    sh = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", text)
    if not (tb and sh):
        return None, "no traffic figure in the ncu summary"
    if sh.group(1) != h.hexdigest()[:16]:
        return None, "kernel changed since the ncu capture"
    return float(tb.group(1)), f"profiles/loglik_tc_{name}.md (ncu dram bytes of one launch)"


def roofline_tensor(w, r, pk):
    """c4: the fused kernel is bound by its split-BF16 tensor-core products."""
    fpt = split_flops_per_term(w)
    peak = pk.get("bf16_tflops", 1800.0)
    peak_src = "bf16_tflops (burst) of MEASURED_PEAKS.json" if "bf16_tflops" in pk else "fallback 1.8 PFLOP/s"
    achieved = r["hot_units"] * fpt / (r["hot_ms"] * 1e-3) / 1e12 if r["hot_ms"] > 0 else 0.0
    traffic, tsrc = profiled_traffic(w.name)
    sm_max = pk.get("sm_max_mhz", 2032.0)
    full_units = w.P * w.n
    out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic, "traffic_source": tsrc,
           "kernel": "loglik_tc_kernel (split BF16, tcgen05)", "flop_per_term": fpt,
           "launches_timed": r["hot_launches"], "avg_launch_ms": r["hot_ms"] / max(1, r["hot_launches"]),
           "peak_source": peak_src,
           "frac_of_sustained": (achieved / pk["bf16_tflops_sustained"]) if "bf16_tflops_sustained" in pk else None,
           "bounds_ms_full_t": {"tensor_split": full_units * fpt / (peak * 1e12) * 1e3,
                                "sfu": full_units * (w.C - 1) / (148 * 32 * sm_max * 1e6) * 1e3,
                                "hbm": w.n * (2 * 64 * ((w.k + 15) // 16 + 1)) / (pk.get("hbm_gbs", 6400.0) * 1e9) * 1e3}}
    return out


def roofline_sfu(w, r, pk):
    """c2: the fused kernel is bound by its one ex2 per term (peak 148 SMs x 32 ex2/clk x the
    maximum SM clock; 30 ex2/clk/SM measured by a probe)."""
    sm_max = pk.get("sm_max_mhz", 2032.0)
    sfu_peak = 148 * 32 * sm_max * 1e6 / 1e9        # Gop/s
    achieved = r["hot_units"] * (w.C - 1) / (r["hot_ms"] * 1e-3) / 1e9 if r["hot_ms"] > 0 else 0.0
    traffic, tsrc = profiled_traffic(w.name)
    full_units = w.P * w.n
    return {"bound": "alu", "achieved": achieved, "peak": sfu_peak, "unit": "Gop/s (ex2)",
            "frac": achieved / sfu_peak, "traffic": traffic, "traffic_source": tsrc,
            "kernel": "loglik_tc_kernel (split BF16, tcgen05)",
            "launches_timed": r["hot_launches"], "avg_launch_ms": r["hot_ms"] / max(1, r["hot_launches"]),
            "peak_source": "148 SMs x 32 ex2/clk/SM x sm_max_mhz of MEASURED_PEAKS (ex2 rate from a probe)",
            "bounds_ms_full_t": {"sfu": full_units * (w.C - 1) / (sfu_peak * 1e9) * 1e3,
                                 "tensor_split": full_units * split_flops_per_term(w) /
                                 (pk.get("bf16_tflops", 1800.0) * 1e12) * 1e3}}


def run_ours(args):
    import torch
    import synthetic

    torch.cuda.set_device(0)
    pk = peaks()
    w4 = synthetic.make_c4()
    r4 = step_bench(w4, args, flush_l2=False)
    dtype = "bf16x2-split/f32/f64" if args.precision == "split" else "f32/f64"
    line = {
        "metric": METRIC, "value": r4["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r4["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": "c4 binary logit n=1000000 k=100 (intercept, 69 equicorrelated(0.2) N(0,1), "
                               "30 Bernoulli(0.1)), 64 groups x 1024 particles, one SPS cycle per step "
                               "(C phase 64 obs, S phase, M step) at t = n - 64 (steps + warmup) .. n",
                   "global_batch": w4.P, "seq_len": w4.n, "parallelism": "single GPU",
                   "precision": args.precision, "mkernel": args.mkernel,
                   "l2": "inputs larger than L2 (X split-BF16 operand rows 384 MB); no flush"},
        "wall_s": r4["wall_s"],
        "gpu_launches": r4["gpu_launches"],
        "clocks": r4["clocks"],
        "ms_per_step_median": r4["ms_per_step_median"],
        "e2e": r4["e2e"],
        "roofline": roofline_tensor(w4, r4, pk),
    }
    if not args.no_c2:
        w2 = synthetic.make_c2()
        r2 = step_bench(w2, args, flush_l2=True)
        line["workloads"] = {"c2": {
            "workload": "c2 binary logit n=20000 k=30 (intercept, 19 AR(1) N(0,1), 10 Bernoulli(0.3)), "
                        "16 groups x 4096 particles, one SPS cycle per step; L2 flushed between steps (512 MB write)",
            "value": r2["value"], "unit": UNIT, "ms_per_step": r2["ms_per_step"],
            "ms_per_step_median": r2["ms_per_step_median"], "gpu_launches": r2["gpu_launches"],
            "clocks": r2["clocks"], "e2e": r2["e2e"], "roofline": roofline_sfu(w2, r2, pk)}}
        if args.sps_ladder:
            forms = [tuple(f.split("_")) for f in args.sps_ladder.split(",")]
            if any(f not in (("split", "rw"), ("split", "mala"), ("fp32", "rw"), ("fp32", "mala")) for f in forms):
                raise SystemExit(f"--sps-ladder: unknown form in {args.sps_ladder!r}")
            line["sps"] = {"workload": "c2", "ladder": sps_ladder(w2, forms, args.sps_max_groups,
                                                                  args.ladder_seeds, args.ladder_seeds_other)}
    if not args.no_cpu:
        try:
            line["cpu_baseline"] = oracle_throughput(w4, seconds=10.0, particles=16)
            line["cpu_baseline"]["single_thread"] = oracle_single_thread("c4", 6.0, 16)
            line["cpu_baseline"]["sps"] = oracle_sps()
        except Exception as exc:      # the GPU figures are reported whatever happens here
            line["cpu_baseline"] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)


def next_rung(J: int, nse: float, target: float, max_groups: int, step: int = 16) -> int:
    """Groups of the ladder's next rung after a run at J groups that ended at log-ML NSE `nse`
    above the target: twice J while nse > 1.5 target (an NSE estimated from few groups is too
    noisy to extrapolate from); closer in, the groups at which NSE ~ 1 / sqrt(groups) reaches the
    target, times 1.15 (about two standard errors of an NSE estimated from some hundred groups),
    rounded up to a multiple of `step`, at least J + step and at most 2 J; never above
    max_groups."""
    if nse > 1.5 * target:
        nxt = 2 * J
    else:
        want = J * (nse / target) ** 2 * 1.15
        nxt = min(max(int(math.ceil(want / step)) * step, J + step), 2 * J)
    return min(nxt, max_groups)


def sps_ladder(w, forms, max_groups: int, seeds: int, seeds_other: int, target: float = 0.05):
    """The wall-time half of the metric as a measured protocol: for each form (precision, M
    kernel), run seed 1 at the workload's groups x particles and raise the number of groups
    (`next_rung`; particles per group stay at the workload's value, the resampling bound) until
    its log-ML NSE is at most the target; then run seeds 2..`seeds` (split MALA) or
    2..`seeds_other` (the other forms) at that rung and report the median wall time with each
    seed's NSE. The plain FP32 random walk starts at the rung the split random walk reached (the
    same Metropolis kernel on the same data: the two differ only in rounding). A form whose seed
    1 misses the target at max_groups reports its last rung with "reached": false."""
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
        J = w.J
        if prec == "fp32" and out.get(f"split_{mk}", {}).get("reached"):
            J = out[f"split_{mk}"]["groups"]
        rungs = []
        while True:
            rungs.append(one(J, 1))
            if rungs[-1]["log_ml_nse"] <= target or J >= max_groups:
                break
            J = next_rung(J, rungs[-1]["log_ml_nse"], target, max_groups)
        reached = rungs[-1]["log_ml_nse"] <= target
        ns = seeds if (prec, mk) == ("split", "mala") else seeds_other
        runs = [rungs[-1]] + ([one(J, sd) for sd in range(2, ns + 1)] if reached else [])
        walls = sorted(x["wall_s"] for x in runs)
        out[f"{prec}_{mk}"] = {"reached": reached, "groups": J, "rung": f"{J} groups x {w.N}",
                               "median_wall_s": walls[len(walls) // 2], "seeds": runs,
                               "ladder_seed1": [{k: x[k] for k in ("groups", "wall_s", "log_ml_nse")}
                                                for x in rungs]}
    if "fp32_rw" in out:
        for name in ("split_rw", "split_mala"):
            if name in out and out[name]["reached"] and out["fp32_rw"]["reached"]:
                out[f"speedup_{name}_vs_fp32_rw"] = out["fp32_rw"]["median_wall_s"] / out[name]["median_wall_s"]
    out["target_log_ml_nse"] = target
    return out


def run_loglik_only(args):
    """Profiling entry: `--calls` calls of the fused split-precision log-likelihood (or, with
    `--grad`, of the log-likelihood and its gradient) on the named workload at t = n with
    `--particles` particles around the true coefficients (device memory), after one untimed call;
    prints the per-launch time of the fused kernel from the library's CUDA events."""
    import ctypes as C
    import torch
    import synthetic
    from paper_1304_4333_b300 import Sps
    torch.cuda.set_device(0)
    w = synthetic.make_workload(args.loglik_only)
    P = args.particles or w.P
    th = torch.from_numpy(synthetic.particles_around(w.theta_true, P, 0.05, seed=2)).cuda()
    s = Sps(w.X, w.y, w.C, prior_sd=5.0)
    call = (lambda: s.loglik_grad(th, w.n)) if args.grad else (lambda: s.loglik(th, w.n, "split"))
    call()
    torch.cuda.synchronize()
    s.lib.sps_set_timing(s.ctx, 1)
    s.lib.sps_counters(s.ctx, 1, None, None, None)
    for _ in range(args.calls):
        call()
    torch.cuda.synchronize()
    a, b, c = C.c_int64(), C.c_int64(), C.c_double()
    s.lib.sps_counters(s.ctx, 1, C.byref(a), C.byref(b), C.byref(c))
    ms = c.value / max(b.value, 1)
    print(json.dumps({"workload": w.name, "kernel": "gradient" if args.grad else "log-likelihood",
                      "particles": P, "t": w.n, "launches": b.value, "ms_per_launch": ms,
                      "terms_per_s": P * w.n / (ms * 1e-3)}), flush=True)
    s.close()


def run_phase_kernels(args):
    """Profiling entry for the simulator's other kernels: `--calls` cycles on the named workload's
    J x N particles (around the true coefficients, near the end of its data): C phase over 64
    observations, S phase, one random-walk and one MALA M step, then one standalone Philox
    generation of P x D / 4 words; after one untimed cycle. Prints the wall time per phase
    (host clock around a synchronised call) for the timed cycles."""
    import torch
    import synthetic
    from paper_1304_4333_b300 import Sps
    torch.cuda.set_device(0)
    w = synthetic.make_workload(args.phase_kernels)
    s = Sps(w.X, w.y, w.C, prior_sd=5.0, seed=1)
    st = s.state(w.J, w.N, seed=100)
    t0 = w.n - C_BLOCK * (args.calls + 1)
    st.set(synthetic.particles_around(w.theta_true, w.P, 0.05, seed=2), None, t0)
    words = max(1, w.P * w.D // 4)
    phases = {"cphase": lambda: st.cphase(st.get_t() + C_BLOCK, outputs=False),
              "sphase": lambda: st.sphase(indices=False),
              "mstep_rw": lambda: st.mstep("rw", sigma_used=False),
              "mstep_mala": lambda: st.mstep("mala", sigma_used=False),
              "philox": lambda: s.philox((7, 11), (0, 0, 0, 0), words)}
    ms = {k: [] for k in phases}
    for i in range(args.calls + 1):
        for k, f in phases.items():
            torch.cuda.synchronize()
            a = time.perf_counter()
            f()
            torch.cuda.synchronize()
            if i > 0:
                ms[k].append((time.perf_counter() - a) * 1e3)
    print(json.dumps({"workload": w.name, "particles": w.P, "D": w.D, "cycles": args.calls,
                      "ms_per_call": {k: (sum(v) / len(v) if v else None) for k, v in ms.items()}}), flush=True)
    s.close()


def run_batched_sps(args):
    """Model comparison on c5: the batched simulator over the first `--models` nested models
    (k = 5, 8, ...; the paper's g-prior with g = 1 for each model's covariates, 16 x 1024
    particles each), random walk or MALA (`--mkernel`). Prints one JSON line per model (log
    marginal likelihood, its NSE, cycles, M steps) and one with the wall time of the run."""
    import torch
    import synthetic
    from paper_1304_4333_b300 import Sps
    torch.cuda.set_device(0)
    w = synthetic.make_workload("c5")
    ks = [int(k) for k in w.model_k[:args.models]]
    s = Sps(w.X, w.y, w.C, prior_sd=5.0, seed=1, mkernel=args.mkernel)
    t0 = time.perf_counter()
    rs = s.run_batched(ks, w.J, w.N, g=1.0)
    wall = time.perf_counter() - t0
    for k, r in zip(ks, rs):
        print(json.dumps({"k": k, "log_ml": r.log_ml, "log_ml_nse": r.log_ml_nse, "cycles": r.n_cycles,
                          "m_steps": r.m_steps, "graph_steps": r.graph_steps}), flush=True)
    print(json.dumps({"workload": "c5", "models": len(ks), "mkernel": args.mkernel, "wall_s": wall}), flush=True)
    s.close()


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
    ap.add_argument("--no-c2", action="store_true", help="skip the c2 workload and the ladder")
    ap.add_argument("--sps-ladder", default="split_mala,split_rw,fp32_rw",
                    help="comma list of forms (split_rw, split_mala, fp32_rw) run on c2 to log-ML NSE <= 0.05 "
                         "by doubling the groups ('' to skip)")
    ap.add_argument("--ladder-seeds", type=int, default=3, help="seeds of the split MALA form at the rung reached")
    ap.add_argument("--ladder-seeds-other", type=int, default=1,
                    help="seeds of the other forms at the rung reached (each run of the plain FP32 form at "
                         "512 groups takes about 170 s)")
    ap.add_argument("--sps-max-groups", type=int, default=1024)
    ap.add_argument("--ncu-step", action="store_true",
                    help="run one extra step after warm-up inside a CUDA profiler range (for ncu --profile-from-start off)")
    ap.add_argument("--loglik-only", default="", choices=["", "c1", "c2", "c3", "c4", "c5"],
                    help="profiling entry: only time the fused log-likelihood on this workload")
    ap.add_argument("--particles", type=int, default=0, help="with --loglik-only: particles (0 = the workload's)")
    ap.add_argument("--calls", type=int, default=2, help="with --loglik-only / --phase-kernels: timed calls")
    ap.add_argument("--grad", action="store_true", help="with --loglik-only: the log-likelihood gradient kernel")
    ap.add_argument("--batched-sps", action="store_true",
                    help="model comparison on c5: the batched simulator over --models nested models")
    ap.add_argument("--models", type=int, default=24, help="with --batched-sps: the first m of c5's models")
    ap.add_argument("--phase-kernels", default="", choices=["", "c1", "c2", "c3", "c4"],
                    help="profiling entry: simulator cycles (C, S, random-walk and MALA M steps, Philox) on this workload")
    args = ap.parse_args()
    if args.loglik_only:
        run_loglik_only(args)
        return
    if args.phase_kernels:
        run_phase_kernels(args)
        return
    if args.batched_sps:
        run_batched_sps(args)
        return
    if args.gpus != 1:
        print(json.dumps({"metric": METRIC, "impl": args.impl, "n_gpus": args.gpus,
                          "unavailable": "single-GPU build: the simulator runs on one GPU"}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
