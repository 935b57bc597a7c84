"""Two calls of the log-likelihood gradient on the c2 workload (binary logit, n = 20 000,
k = 30, 16 x 4096 particles around the true coefficients) for profiling the gradient kernel
with ncu; prints the per-launch kernel time of the second call from the library's CUDA events."""
import ctypes as C
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import synthetic  # noqa: E402
from paper_1304_4333_b300 import Sps  # noqa: E402


def main():
    w = synthetic.make_c2()
    th = torch.from_numpy(synthetic.particles_around(w.theta_true, w.P, 0.05, seed=1)).cuda()
    s = Sps(w.X, w.y, w.C, prior_sd=5.0)
    s.loglik_grad(th, w.n)
    torch.cuda.synchronize()
    s.lib.sps_set_timing(s.ctx, 1)
    s.lib.sps_counters(s.ctx, 1, None, None, None)
    s.loglik_grad(th, w.n)
    a, b, c = C.c_int64(), C.c_int64(), C.c_double()
    s.lib.sps_counters(s.ctx, 1, C.byref(a), C.byref(b), C.byref(c))
    print("gradient kernel ms per launch: %.4f" % (c.value / max(b.value, 1)))
    s.close()


if __name__ == "__main__":
    main()
