"""Python binding of the SPS library: thin wrappers over the C ABI (include/sps.h).

Every step of the simulator runs in the library's CUDA kernels; this module only converts
arguments. Host arrays (numpy) are passed with SPS_MEM_HOST; CUDA tensors (torch) with
SPS_MEM_DEVICE on torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import weakref
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import _native as N
from ._native import SpsError

PRECISIONS = {"split": N.PREC_SPLIT, "fp32": N.PREC_FP32}
MKERNELS = {"rw": N.MKERNEL_RW, "mala": N.MKERNEL_MALA}
RESAMPLING = {"multinomial": N.RESAMPLE_MULTINOMIAL, "residual": N.RESAMPLE_RESIDUAL}


def _check(lib, ctx, status: int):
    if status != N.SPS_OK:
        msg = lib.sps_last_error(ctx).decode() if ctx else ""
        base = lib.sps_status_string(status).decode()
        raise SpsError(status, f"{base}: {msg}" if msg else base)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a) -> C.c_void_p:
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _torch():
    import torch
    return torch


def default_options(**over) -> N.SpsOptions:
    lib = N.load()
    o = N.SpsOptions()
    lib.sps_options_default(C.byref(o))
    for k, v in over.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "mkernel" and isinstance(v, str):
            v = MKERNELS[v]
        if k == "resampling" and isinstance(v, str):
            v = RESAMPLING[v]
        setattr(o, k, v)
    return o


def prior_normalize(mu, Sigma):
    """Prior of theta_j - theta_0 (j = 1..C-1) from independent class priors N(mu_c, Sigma_c)
    (sps_prior_normalize): mu [C, k], Sigma [C, k, k] -> (mean [D], cov [D, D])."""
    lib = N.load()
    mu = _f64(mu)
    Sig = _f64(Sigma)
    Cn, k = mu.shape
    D = k * (Cn - 1)
    mean = np.empty(D)
    cov = np.empty((D, D))
    st = lib.sps_prior_normalize(k, Cn, _ptr(mu), _ptr(Sig), _ptr(mean), _ptr(cov))
    if st != N.SPS_OK:
        raise SpsError(st, lib.sps_status_string(st).decode())
    return mean, cov


@dataclass
class RunResult:
    mean: np.ndarray
    sd: np.ndarray
    nse: np.ndarray
    rne: np.ndarray
    log_ml_group: np.ndarray
    log_ml: float
    log_ml_nse: float
    log_ml_pooled: float
    n_cycles: int
    m_steps: int
    seconds: float
    schedule: Optional["Schedule"] = None
    log_pred: Optional[np.ndarray] = None       # [n] log p(y_s | y_1:s-1), mean over groups
    log_pred_nse: Optional[np.ndarray] = None   # [n] sd over groups / sqrt(J)
    graph_steps: int = 0                        # M steps run inside captured CUDA graphs


@dataclass
class Schedule:
    """Recorded cycles of an adaptive run (Algorithm 3 pass 1): t_l, R_l, Sigma_lr, h_lr, alpha_lr."""
    t: np.ndarray
    R: np.ndarray
    sigma: np.ndarray          # [sum R, D, D]
    h: np.ndarray
    accept: np.ndarray
    _keep: List = field(default_factory=list, repr=False)

    def as_struct(self) -> N.SpsSchedule:
        t = np.ascontiguousarray(self.t, dtype=np.int64)
        R = np.ascontiguousarray(self.R, dtype=np.int32)
        sig = np.ascontiguousarray(self.sigma, dtype=np.float64)
        h = np.ascontiguousarray(self.h, dtype=np.float64)
        a = np.ascontiguousarray(self.accept, dtype=np.float64)
        self._keep = [t, R, sig, h, a]
        s = N.SpsSchedule()
        s.n_cycles = len(t)
        s.cap_cycles = len(t)
        s.t = t.ctypes.data_as(C.POINTER(C.c_int64))
        s.R = R.ctypes.data_as(C.POINTER(C.c_int32))
        s.cap_steps = int(R.sum())
        s.sigma = sig.ctypes.data_as(C.POINTER(C.c_double))
        s.h = h.ctypes.data_as(C.POINTER(C.c_double))
        s.accept = a.ctypes.data_as(C.POINTER(C.c_double))
        return s


class Sps:
    """A context: data (X, y), number of outcomes C (base outcome 0) and a Gaussian prior."""

    def __init__(self, X, y, C_outcomes: int, prior_sd: float = 5.0, prior_mean=None, prior_cov=None,
                 prior_diag_sd=None, **options):
        self.lib = N.load()
        X = _f64(X)
        y = np.ascontiguousarray(y, dtype=np.int32)
        n, k = X.shape
        self.n, self.k, self.C = int(n), int(k), int(C_outcomes)
        self.D = self.k * (self.C - 1)
        pr = self._prior_struct(prior_sd, prior_mean, prior_cov, prior_diag_sd)
        self.options = default_options(**options)
        self._states = weakref.WeakSet()   # states are destroyed before the context
        ctx = C.c_void_p()
        st = self.lib.sps_init(C.byref(ctx), _ptr(X), n, k, _ptr(y), self.C, C.byref(pr), C.byref(self.options))
        if st != N.SPS_OK:
            raise SpsError(st, self.lib.sps_status_string(st).decode())
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            for st in list(getattr(self, "_states", ())):
                st.close()
            self.lib.sps_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ helpers
    def _sync_stream(self):
        torch = _torch()
        self.lib.sps_set_stream(self.ctx, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def _call(self, name, *args):
        _check(self.lib, self.ctx, getattr(self.lib, name)(self.ctx, *args))

    # ------------------------------------------------------------------ likelihood
    def loglik(self, theta, t: Optional[int] = None, precision: str = "split"):
        """ll [P] = sum_{s<=t} log P(y_s | x_s, theta_p). numpy in -> numpy out; CUDA tensor in ->
        CUDA tensor out (on torch's current stream)."""
        t = self.n if t is None else int(t)
        prec = PRECISIONS[precision]
        if _is_device(theta):
            torch = _torch()
            th = theta.contiguous().to(torch.float64)
            P = th.shape[0]
            out = torch.empty(P, dtype=torch.float64, device=th.device)
            self._sync_stream()
            self._call("sps_loglik", _ptr(th), P, t, _ptr(out), prec, N.MEM_DEVICE)
            return out
        th = _f64(theta).reshape(-1, self.D)
        out = np.empty(th.shape[0])
        self._call("sps_loglik", _ptr(th), th.shape[0], t, _ptr(out), prec, N.MEM_HOST)
        return out

    def loglik_host_ptr(self, theta_ptr: int, ll_ptr: int, P: int, t: Optional[int] = None,
                        precision: str = "split"):
        """sps_loglik on caller-owned host buffers given by address (e.g. pinned torch tensors)."""
        t = self.n if t is None else int(t)
        self._call("sps_loglik", C.c_void_p(theta_ptr), int(P), t, C.c_void_p(ll_ptr), PRECISIONS[precision],
                   N.MEM_HOST)

    def autotune(self, P: int, t: Optional[int] = None) -> dict:
        """Time the fused kernel's launch shapes on P particles at prefix t (default n) and keep
        the fastest for later calls (sps_autotune)."""
        r = N.SpsTuneResult()
        self._call("sps_autotune", int(P), int(self.n if t is None else t), C.byref(r))
        return {"tile_rows": r.tile_rows, "cluster": r.cluster, "chunk_obs": r.chunk_obs,
                "n_candidates": r.n_candidates, "ms": r.ms, "ms_default": r.ms_default}

    def loglik_batched(self, thetas, ks, ts):
        """Log-likelihoods of nested models in one launch (sps_loglik_batched): thetas is a list of
        CUDA float64 tensors [P_m, k_m (C-1)], ks the covariate counts, ts the prefixes. Returns a
        list of CUDA tensors [P_m]."""
        torch = _torch()
        M = len(thetas)
        flat = torch.cat([t.contiguous().to(torch.float64).reshape(-1) for t in thetas])
        P = np.array([int(t.shape[0]) for t in thetas], dtype=np.int64)
        km = np.array([int(k) for k in ks], dtype=np.int32)
        tm = np.array([int(t) for t in ts], dtype=np.int64)
        out = torch.empty(int(P.sum()), dtype=torch.float64, device=flat.device)
        self._sync_stream()
        self._call("sps_loglik_batched", M, _ptr(km), _ptr(P), _ptr(tm), _ptr(flat), _ptr(out))
        return list(torch.split(out, P.tolist()))

    def loglik_grad(self, theta, t: Optional[int] = None):
        t = self.n if t is None else int(t)
        if _is_device(theta):
            torch = _torch()
            th = theta.contiguous().to(torch.float64)
            P = th.shape[0]
            ll = torch.empty(P, dtype=torch.float64, device=th.device)
            g = torch.empty_like(th)
            self._sync_stream()
            self._call("sps_loglik_grad", _ptr(th), P, t, _ptr(ll), _ptr(g), N.MEM_DEVICE)
            return ll, g
        th = _f64(theta).reshape(-1, self.D)
        ll = np.empty(th.shape[0])
        g = np.empty_like(th)
        self._call("sps_loglik_grad", _ptr(th), th.shape[0], t, _ptr(ll), _ptr(g), N.MEM_HOST)
        return ll, g

    # ------------------------------------------------------------------ priors
    def _prior_struct(self, prior_sd=5.0, prior_mean=None, prior_cov=None, prior_diag_sd=None) -> N.SpsPrior:
        pr = N.SpsPrior()
        if prior_cov is not None:
            cov = _f64(prior_cov).reshape(self.D, self.D)
            pr.kind, self._prior_arrays = N.PRIOR_FULL, [cov]
        elif prior_diag_sd is not None:
            sd = _f64(prior_diag_sd).reshape(self.D)
            pr.kind, self._prior_arrays = N.PRIOR_DIAG, [sd]
        else:
            sd = np.array([float(prior_sd)])
            pr.kind, self._prior_arrays = N.PRIOR_ISO, [sd]
        pr.cov_or_sd = self._prior_arrays[0].ctypes.data_as(C.POINTER(C.c_double))
        if prior_mean is not None:
            m = _f64(prior_mean).reshape(self.D)
            self._prior_arrays.append(m)
            pr.mean = m.ctypes.data_as(C.POINTER(C.c_double))
        return pr

    def set_prior(self, prior_sd: float = 5.0, prior_mean=None, prior_cov=None, prior_diag_sd=None):
        """Replace the prior (sps_set_prior); states created afterwards draw from it."""
        pr = self._prior_struct(prior_sd, prior_mean, prior_cov, prior_diag_sd)
        self._call("sps_set_prior", C.byref(pr))

    def gprior(self, g: float):
        """Zellner's g-prior for this data, normalised on outcome 0 (sps_gprior): (mean, cov)."""
        mean = np.empty(self.D)
        cov = np.empty((self.D, self.D))
        self._call("sps_gprior", float(g), _ptr(mean), _ptr(cov))
        return mean, cov

    # ------------------------------------------------------------------ building blocks
    def resample(self, w, u, J: int, N_: int, scheme: str = "multinomial"):
        sch = RESAMPLING[scheme]
        if _is_device(w):
            torch = _torch()
            idx = torch.empty(J * N_, dtype=torch.int32, device=w.device)
            self._sync_stream()
            self._call("sps_resample", _ptr(w.contiguous()), _ptr(u.contiguous()), J, N_, sch, _ptr(idx),
                       N.MEM_DEVICE)
            return idx
        w = _f64(w); u = _f64(u)
        idx = np.empty(J * N_, dtype=np.int32)
        self._call("sps_resample", _ptr(w), _ptr(u), J, N_, sch, _ptr(idx), N.MEM_HOST)
        return idx

    def philox(self, key, ctr, count: int):
        out = np.empty((count, 4), dtype=np.uint32)
        self._call("sps_philox", key[0], key[1], ctr[0], ctr[1], ctr[2], ctr[3], count, _ptr(out), N.MEM_HOST)
        return out

    def ess(self, logw, J: int):
        logw = _f64(logw)
        e = np.empty(1)
        lme = np.empty(J)
        self._call("sps_ess", _ptr(logw), logw.shape[0], J, _ptr(e), _ptr(lme), N.MEM_HOST)
        return float(e[0]), lme

    def particle_cov(self, theta):
        th = _f64(theta).reshape(-1, self.D)
        V = np.empty((self.D, self.D))
        self._call("sps_particle_cov", _ptr(th), th.shape[0], _ptr(V), N.MEM_HOST)
        return V

    def rw_step_given(self, theta, ll, t: int, sigma, z, u, precision: str = "split"):
        th = _f64(theta).reshape(-1, self.D).copy()
        l = _f64(ll).copy()
        sig = _f64(sigma).reshape(self.D, self.D)
        z = _f64(z).reshape(th.shape)
        u = _f64(u)
        la = np.empty(th.shape[0])
        acc = np.empty(th.shape[0], dtype=np.int32)
        self._call("sps_rw_step_given", _ptr(th), _ptr(l), th.shape[0], int(t), _ptr(sig), _ptr(z), _ptr(u),
                   PRECISIONS[precision], _ptr(la), _ptr(acc), N.MEM_HOST)
        return th, l, la, acc.astype(bool)

    def mala_step_given(self, theta, t: int, sigma, z, u):
        """One MALA step with given normals z [P, D] and uniforms u [P] (sps_mala_step_given):
        returns (theta, ll, log alpha, accepted)."""
        th = _f64(theta).reshape(-1, self.D).copy()
        l = np.empty(th.shape[0])
        sig = _f64(sigma).reshape(self.D, self.D)
        z = _f64(z).reshape(th.shape)
        u = _f64(u)
        la = np.empty(th.shape[0])
        acc = np.empty(th.shape[0], dtype=np.int32)
        self._call("sps_mala_step_given", _ptr(th), _ptr(l), th.shape[0], int(t), _ptr(sig), _ptr(z), _ptr(u),
                   _ptr(la), _ptr(acc), N.MEM_HOST)
        return th, l, la, acc.astype(bool)

    # ------------------------------------------------------------------ simulator
    def run_batched(self, ks, J: int, N_: int, g: Optional[float] = None) -> List[RunResult]:
        """Adaptive SPS for nested models (sps_run_batched): model m uses the first ks[m]
        covariates, with the paper's g-prior of its covariates when g is given (else the marginal
        of the context's prior); the M phases of all models run in lockstep with one batched
        log-likelihood launch per step; with graphs (the default) each phase after its first step is
        one CUDA graph launch. Returns one RunResult per model (no schedule)."""
        ks = [int(v) for v in ks]
        M = len(ks)
        res = (N.SpsResult * M)()
        keep = []
        for m, km in enumerate(ks):
            dim = km * (self.C - 1) + self.C - 1
            arrs = {f: np.zeros(dim) for f in ("mean", "sd", "nse", "rne")}
            lmg = np.zeros(J)
            for f, a in arrs.items():
                setattr(res[m], f, a.ctypes.data_as(C.POINTER(C.c_double)))
            res[m].log_ml_group = lmg.ctypes.data_as(C.POINTER(C.c_double))
            keep.append((arrs, lmg))
        kk = np.ascontiguousarray(ks, dtype=np.int32)
        self._call("sps_run_batched", M, kk.ctypes.data_as(C.c_void_p), float(g or 0.0), J, N_, res)
        out = []
        for m in range(M):
            arrs, lmg = keep[m]
            r = res[m]
            out.append(RunResult(arrs["mean"], arrs["sd"], arrs["nse"], arrs["rne"], lmg, r.log_ml, r.log_ml_nse,
                                 r.log_ml_pooled, r.n_cycles, r.m_steps, r.seconds, graph_steps=r.graph_steps))
        return out

    def state(self, J: int, N_: int, seed: int = 0) -> "State":
        return State(self, J, N_, seed)

    def run(self, J: int, N_: int, schedule: Optional[Schedule] = None, record: bool = True,
            cap_cycles: int = 4096, cap_steps: int = 20000, log_pred: bool = False) -> RunResult:
        m = self.D + self.C - 1
        arrs = {k: np.zeros(m) for k in ("mean", "sd", "nse", "rne")}
        lmg = np.zeros(J)
        res = N.SpsResult()
        for k_, a in arrs.items():
            setattr(res, k_, a.ctypes.data_as(C.POINTER(C.c_double)))
        res.log_ml_group = lmg.ctypes.data_as(C.POINTER(C.c_double))
        lp = np.zeros(self.n) if log_pred else None
        lpn = np.zeros(self.n) if log_pred else None
        if log_pred:
            res.log_pred = lp.ctypes.data_as(C.POINTER(C.c_double))
            res.log_pred_nse = lpn.ctypes.data_as(C.POINTER(C.c_double))
        sched_in = schedule.as_struct() if schedule is not None else None
        rec = None
        if record:
            rt = np.zeros(cap_cycles, np.int64)
            rR = np.zeros(cap_cycles, np.int32)
            rs = np.zeros((cap_steps, self.D, self.D)) if self.D * self.D * cap_steps <= 400_000_000 else None
            rh = np.zeros(cap_steps)
            ra = np.zeros(cap_steps)
            rec = N.SpsSchedule()
            rec.cap_cycles = cap_cycles
            rec.t = rt.ctypes.data_as(C.POINTER(C.c_int64))
            rec.R = rR.ctypes.data_as(C.POINTER(C.c_int32))
            rec.cap_steps = cap_steps
            rec.sigma = rs.ctypes.data_as(C.POINTER(C.c_double)) if rs is not None else None
            rec.h = rh.ctypes.data_as(C.POINTER(C.c_double))
            rec.accept = ra.ctypes.data_as(C.POINTER(C.c_double))
        self._call("sps_run", J, N_, C.byref(sched_in) if sched_in is not None else None,
                   C.byref(rec) if rec is not None else None, C.byref(res))
        sched = None
        if rec is not None:
            L = rec.n_cycles
            S = int(rR[:L].sum())
            sched = Schedule(rt[:L].copy(), rR[:L].copy(),
                             rs[:S].copy() if rs is not None else np.zeros((0, self.D, self.D)),
                             rh[:S].copy(), ra[:S].copy())
        return RunResult(arrs["mean"], arrs["sd"], arrs["nse"], arrs["rne"], lmg, res.log_ml, res.log_ml_nse,
                         res.log_ml_pooled, res.n_cycles, res.m_steps, res.seconds, sched, lp, lpn,
                         res.graph_steps)


class State:
    """Particle state of J groups of N particles on the device (sps_state)."""

    def __init__(self, sps: Sps, J: int, N_: int, seed: int = 0):
        self.sps, self.J, self.N = sps, J, N_
        st = C.c_void_p()
        sps._call("sps_state_create", J, N_, seed, C.byref(st))
        self.st = st
        sps._states.add(self)

    def close(self):
        if getattr(self, "st", None):
            if getattr(self.sps, "ctx", None):   # a destroyed context already released its device
                self.sps.lib.sps_state_destroy(self.st)
            self.st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        P, D = self.J * self.N, self.sps.D
        th = np.empty((P, D)); ll = np.empty(P); lw = np.empty(P)
        t = C.c_int64(); h = C.c_double()
        self.sps._call("sps_state_get", self.st, _ptr(th), _ptr(ll), _ptr(lw), C.byref(t), C.byref(h))
        return {"theta": th, "ll": ll, "logw": lw, "t": t.value, "h": h.value}

    def get_t(self) -> int:
        t = C.c_int64()
        self.sps._call("sps_state_get", self.st, None, None, None, C.byref(t), None)
        return t.value

    def set(self, theta, ll=None, t: int = 0):
        th = _f64(theta)
        l = _f64(ll) if ll is not None else None
        self.sps._call("sps_state_set", self.st, _ptr(th), _ptr(l) if l is not None else None, int(t))

    def cphase(self, t_target: int = 0, log_pred: bool = False, outputs: bool = True):
        """C phase; returns (t_new, ess, logml_inc[J]) and, with log_pred, the per-group log
        predictive likelihoods [t_new - t, J] of the observations taken in. With outputs=False
        ess and logml_inc are not read back (None): a C phase with a target then returns without
        waiting for the GPU."""
        tn = C.c_int64(); e = C.c_double()
        inc = np.empty(self.J) if outputs else None
        lp = np.empty((self.sps.n - self.get_t(), self.J)) if log_pred else None
        self.sps._call("sps_cphase", self.st, int(t_target), C.byref(tn), C.byref(e) if outputs else None,
                       _ptr(inc) if outputs else None, _ptr(lp) if lp is not None else None)
        if not outputs:
            e = C.c_double(float("nan"))
        if lp is None:
            return tn.value, e.value, inc
        return tn.value, e.value, inc, lp[:tn.value - (self.sps.n - lp.shape[0])].copy()

    def sphase(self, uniforms=None, indices: bool = True):
        """S phase; returns the selected index within the group of every particle (None with
        indices=False, which skips their copy to the host)."""
        idx = np.empty(self.J * self.N, dtype=np.int32) if indices else None
        u = _f64(uniforms) if uniforms is not None else None
        self.sps._call("sps_sphase", self.st, _ptr(u) if u is not None else None,
                       _ptr(idx) if indices else None, N.MEM_HOST)
        return idx

    def mstep(self, kernel: str = "rw", sigma=None, sigma_used: bool = True):
        """One M step; returns its diagnostics and the Sigma used (None with sigma_used=False)."""
        info = N.SpsMstepInfo()
        sig = _f64(sigma) if sigma is not None else None
        used = np.empty((self.sps.D, self.sps.D)) if sigma_used else None
        self.sps._call("sps_mstep", self.st, MKERNELS[kernel], _ptr(sig) if sig is not None else None,
                       _ptr(used) if sigma_used else None, C.byref(info))
        return {"h": info.h, "accept": info.accept_rate, "rne_min": info.rne_min, "h_next": info.h_next,
                "sigma": used}

    def result(self) -> RunResult:
        """Outputs of the current particles as a run reports them (sps_state_result)."""
        m = self.sps.D + self.sps.C - 1
        arrs = {k: np.zeros(m) for k in ("mean", "sd", "nse", "rne")}
        lmg = np.zeros(self.J)
        res = N.SpsResult()
        for k_, a in arrs.items():
            setattr(res, k_, a.ctypes.data_as(C.POINTER(C.c_double)))
        res.log_ml_group = lmg.ctypes.data_as(C.POINTER(C.c_double))
        self.sps._call("sps_state_result", self.st, C.byref(res))
        return RunResult(arrs["mean"], arrs["sd"], arrs["nse"], arrs["rne"], lmg, res.log_ml, res.log_ml_nse,
                         res.log_ml_pooled, res.n_cycles, res.m_steps, 0.0)

    def mphase(self, kernel: str = "rw", fixed_steps: int = 0):
        steps = C.c_int32(); a = C.c_double(); r = C.c_double()
        self.sps._call("sps_mphase", self.st, MKERNELS[kernel], int(fixed_steps), C.byref(steps), C.byref(a),
                       C.byref(r))
        return steps.value, a.value, r.value
