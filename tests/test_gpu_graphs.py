"""Graph-captured M phases (options.graphs): after its first step an adaptive M phase runs as
one CUDA graph launch, a conditional loop whose body is one M step and a device-side step-size
and stopping rule (Algorithm 2 step 2(c)ii-iii). The device rule rounds every operation as the
host path does and the Philox step words are the same, so a run with graphs and a run that
issues and reads back every step are bit-for-bit identical."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _logit_case(n, k, C, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    beta = 0.5 * g.standard_normal((k, C))
    beta[:, 0] = 0.0
    eta = X @ beta
    p = np.exp(eta - eta.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    y = np.array([g.choice(C, p=row) for row in p], dtype=np.int32)
    return X, y


def _run(X, y, C, J, N, graphs, **kw):
    from paper_1304_4333_b300 import Sps
    s = Sps(X, y, C, prior_sd=5.0, seed=11, graphs=graphs, **kw)
    try:
        return s.run(J, N)
    finally:
        s.close()


def _assert_identical(a, b):
    assert a.n_cycles == b.n_cycles and a.m_steps == b.m_steps
    np.testing.assert_array_equal(a.schedule.t, b.schedule.t)
    np.testing.assert_array_equal(a.schedule.R, b.schedule.R)
    np.testing.assert_array_equal(a.schedule.h, b.schedule.h)
    np.testing.assert_array_equal(a.schedule.accept, b.schedule.accept)
    np.testing.assert_array_equal(a.schedule.sigma, b.schedule.sigma)
    np.testing.assert_array_equal(a.log_ml_group, b.log_ml_group)
    for f in ("mean", "sd", "nse", "rne"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


@pytest.mark.parametrize("C,mkernel,prec", [(2, "rw", "split"), (2, "rw", "fp32"), (3, "rw", "split"),
                                            (3, "mala", "split"), (2, "mala", "fp32")])
def test_graph_run_identical_to_stepwise(cuda, C, mkernel, prec):
    X, y = _logit_case(400, 4, C, seed=C)
    g = _run(X, y, C, 8, 512, 1, mkernel=mkernel, precision=prec)
    e = _run(X, y, C, 8, 512, 0, mkernel=mkernel, precision=prec)
    assert e.graph_steps == 0
    # every cycle's first step runs eagerly; the rest of each phase inside the graph
    assert g.graph_steps == g.m_steps - g.n_cycles
    assert g.graph_steps > 0
    _assert_identical(g, e)


def test_graph_run_c1(cuda):
    w = synthetic.make_c1()
    g = _run(w.X, w.y, w.C, w.J, w.N, 1)
    e = _run(w.X, w.y, w.C, w.J, w.N, 0)
    assert g.graph_steps > 0
    _assert_identical(g, e)


def test_graph_run_hits_step_cap(cuda):
    # r_max = 3: the device rule stops the loop at the cap exactly as the host rule does
    X, y = _logit_case(300, 3, 2, seed=5)
    g = _run(X, y, 2, 4, 256, 1, r_max=3, rne_cycle=50.0, rne_final=50.0)
    e = _run(X, y, 2, 4, 256, 0, r_max=3, rne_cycle=50.0, rne_final=50.0)
    assert np.all(g.schedule.R == 3)
    _assert_identical(g, e)


def test_mphase_state_api_graph(cuda):
    # sps_mphase on a state: same steps, h and particles with and without graphs
    from paper_1304_4333_b300 import Sps
    X, y = _logit_case(300, 3, 2, seed=9)
    out = []
    for graphs in (1, 0):
        s = Sps(X, y, 2, prior_sd=5.0, seed=3, graphs=graphs)
        st = s.state(4, 256, seed=4)
        st.cphase()
        st.sphase()
        r = st.mphase()
        d = st.get()
        out.append((r, d))
        s.close()
    (r1, d1), (r0, d0) = out
    assert r1 == r0
    np.testing.assert_array_equal(d1["theta"], d0["theta"])
    np.testing.assert_array_equal(d1["ll"], d0["ll"])
    assert d1["h"] == d0["h"]


def test_graph_with_many_groups(cuda):
    # J F 3 doubles of control-kernel sums above the default 48 KB of shared memory (J = 1100,
    # F = 2): the limit is raised before the capture; results still equal the stepwise run
    X, y = _logit_case(200, 3, 2, seed=13)
    g = _run(X, y, 2, 1100, 4, 1, r_max=5)
    e = _run(X, y, 2, 1100, 4, 0, r_max=5)
    assert g.graph_steps > 0
    _assert_identical(g, e)
