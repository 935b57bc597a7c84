"""B300-native (sm_103a) sequential posterior simulator for logit models.

Geweke, Durham & Xu (2013), "Bayesian Inference for Logistic Regression Models using Sequential
Posterior Simulation". The compute path is the in-tree CUDA library libsps.so (C ABI in
include/sps.h); this package is its Python binding. Importing the binding loads the library and
raises if it is missing: there is no CPU fallback.
"""
from .api import Sps, State, RunResult, Schedule, SpsError, default_options, prior_normalize  # noqa: F401

__all__ = ["Sps", "State", "RunResult", "Schedule", "SpsError", "default_options"]
