"""The tensor-core gradient (split precision, C - 1 <= 3) against the FP64 oracle.

Bound per gradient entry (c, i): the operands are BF16 hi + lo splits (theta, X: dropped lo x lo
product, relative 2^-16 of each product; q: relative 2^-16) with FP32 accumulation within a work
item. An error of delta in eta changes q by at most delta / 4, so
  |G - G_oracle| <= 1e-5 |G_oracle| + 2^-13 sum_s (1 + |eta_s|) |x_si|
(a factor 8 above the worst-case sum of these relative errors). The log-likelihood uses the
bound of the split log-likelihood tests. Shapes span several tiles with a ragged last tile and
a ragged particle tile. The bound is a guarantee, far above the achieved error; the gradient is
also held to 1e-4 relative (norm-wise) against central finite differences of the
FP64 oracle log-likelihood."""
import numpy as np
import pytest

from oracle import logit as OL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _data(n, k, C, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    X[:, k - k // 3:] = (X[:, k - k // 3:] > 0.4).astype(float)   # exact 0/1 columns
    y = g.integers(0, C, n).astype(np.int32)
    return X, y


def _eta_bound(X, th, C, t):
    k = X.shape[1]
    Xt = X[:t]
    out = np.zeros_like(th)
    for c in range(C - 1):
        eta = th[:, c * k:(c + 1) * k] @ Xt.T                        # [P, t]
        out[:, c * k:(c + 1) * k] = (1.0 + np.abs(eta)) @ np.abs(Xt)  # [P, k]
    return out


@pytest.mark.parametrize("C,n,k,t", [(2, 1500, 30, 1500), (2, 1500, 30, 701), (2, 300, 7, 1),
                                      (3, 1300, 12, 1300), (3, 1300, 12, 555), (3, 900, 74, 900),
                                      (4, 1000, 50, 1000), (4, 700, 9, 333)])
def test_tensor_core_gradient_against_oracle(cuda, C, n, k, t):
    from paper_1304_4333_b300 import Sps
    X, y = _data(n, k, C, seed=n + k + C)
    s = Sps(X, y, C, prior_sd=5.0, precision="split")
    g = np.random.Generator(np.random.PCG64(7))
    D = k * (C - 1)
    th = (0.8 / np.sqrt(k)) * g.standard_normal((300, D))
    ll, G = s.loglik_grad(th, t)
    ll_o, G_o = OL.loglik_grad(X, y, th, C, t)
    bound = 1e-5 * np.abs(G_o) + 2.0 ** -13 * _eta_bound(X, th, C, t)
    assert np.all(np.abs(G - G_o) <= bound), np.max(np.abs(G - G_o) - bound)
    ll_bound = 1e-5 * np.abs(ll_o) + 3 * 2.0 ** -16 * np.abs(th @ np.tile(np.abs(X[:t]).sum(0), C - 1))
    assert np.all(np.abs(ll - ll_o) <= ll_bound + 1e-9)
    # and against the FP32 SIMT form of the same gradient
    s32 = Sps(X, y, C, prior_sd=5.0, precision="fp32")
    _, G32 = s32.loglik_grad(th, t)
    assert np.all(np.abs(G - G32) <= bound + 1e-5 * np.abs(G32))
    s.close()
    s32.close()


def test_tensor_core_gradient_fills_tensor_memory(cuda):
    # C = 3 with 74 alternating continuous / 0-1 columns (the largest nested model of c5): the
    # gradient accumulators take the 256 tensor-memory columns beside the forward ones exactly
    from paper_1304_4333_b300 import Sps
    g = np.random.Generator(np.random.PCG64(74))
    n, k, C = 900, 74, 3
    X = g.standard_normal((n, k))
    X[:, 1::2] = (g.random((n, k // 2)) < 0.25).astype(float)
    y = g.integers(0, C, n).astype(np.int32)
    D = k * (C - 1)
    th = (0.8 / np.sqrt(k)) * g.standard_normal((300, D))
    s = Sps(X, y, C, prior_sd=5.0, precision="split")
    ll, G = s.loglik_grad(th, n)
    ll_o, G_o = OL.loglik_grad(X, y, th, C, n)
    bound = 1e-5 * np.abs(G_o) + 2.0 ** -13 * _eta_bound(X, th, C, n)
    assert np.all(np.abs(G - G_o) <= bound), np.max(np.abs(G - G_o) - bound)
    s32 = Sps(X, y, C, prior_sd=5.0, precision="fp32")
    _, G32 = s32.loglik_grad(th, n)
    assert not np.array_equal(G, G32)      # the tensor-core kernel ran, not the FP32 form
    rel = np.linalg.norm(G - G_o, axis=1) / np.linalg.norm(G_o, axis=1)
    assert rel.max() < 1e-4
    s.close()
    s32.close()


def test_tensor_core_gradient_device_and_zero_theta(cuda):
    # theta = 0: p = 1/C for every term, so G_c = sum_s (1[y_s = c] - 1/C) x_s exactly up to the
    # BF16 split of X (exact for these columns) and FP32 accumulation
    torch = cuda
    from paper_1304_4333_b300 import Sps
    X, y = _data(1000, 9, 3, seed=3)
    X = np.round(X * 8) / 8            # exact in BF16
    s = Sps(X, y, 3, prior_sd=5.0)
    th = torch.zeros((200, 18), dtype=torch.float64, device="cuda")
    ll, G = s.loglik_grad(th, 1000)
    ref = np.zeros(18)
    for c in (1, 2):
        ref[(c - 1) * 9:c * 9] = ((y == c) - 1.0 / 3).astype(float) @ X
    np.testing.assert_allclose(G.cpu().numpy(), np.tile(ref, (200, 1)), rtol=0, atol=2e-3)
    np.testing.assert_allclose(ll.cpu().numpy(), -1000 * np.log(3.0), rtol=1e-6)
    s.close()


@pytest.mark.parametrize("C,n,k", [(2, 2000, 30), (2, 1200, 100), (3, 1500, 12), (4, 1000, 50)])
def test_tensor_core_gradient_against_finite_differences(cuda, C, n, k):
    # ||G - G_fd||_inf / ||G_fd||_inf <= 1e-4 with G_fd the central difference of the FP64 oracle
    # (step 1e-5 max(1, |theta_i|)); shapes of the binary (k = 30, k = 100), three- and
    # four-outcome (k = 50, D = 150) workloads
    from paper_1304_4333_b300 import Sps
    X, y = _data(n, k, C, seed=5 * n + k)
    s = Sps(X, y, C, prior_sd=5.0, precision="split")
    D = k * (C - 1)
    g = np.random.Generator(np.random.PCG64(11))
    th = (0.6 / np.sqrt(k)) * g.standard_normal((129, D))     # a full particle tile and one more
    _, G = s.loglik_grad(th, n)
    worst = 0.0
    for p in (0, 64, 128):
        fd = np.zeros(D)
        for i in range(D):
            h = 1e-5 * max(1.0, abs(th[p, i]))
            e = np.zeros(D)
            e[i] = h
            fd[i] = (OL.loglik(X, y, (th[p] + e)[None], C, n)[0] - OL.loglik(X, y, (th[p] - e)[None], C, n)[0]) / (2 * h)
        worst = max(worst, np.max(np.abs(G[p] - fd)) / np.max(np.abs(fd)))
    print(f"C={C} n={n} k={k}: max ||G - G_fd|| / ||G_fd|| = {worst:.2e}")
    assert worst <= 1e-4
    s.close()
