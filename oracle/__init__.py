"""Oracle for the sequential posterior simulator (SPS) for logit models.

Geweke, Durham & Xu (2013), "Bayesian Inference for Logistic Regression Models using
Sequential Posterior Simulation".

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. It is a plain, slow, FP64 CPU
restatement of what the simulator computes, written from the paper so that the CUDA library can
be checked against it. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and ``--impl reference`` legs) may import or run it. The CUDA library
(``paper_1304_4333_b300``) never imports it, and it imports nothing from that library: the two
share no code. Both are fed from the seeded generators in ``synthetic/``, which hold none of the
method's arithmetic.

Modules
-------
logit       multinomial-logit log-likelihood and its gradient (Eq. 1, Sec. 2.1).
smc         ESS (Eq. 14), group moments / NSE / RNE (Eqs. 3-10), multinomial resampling
            (Algorithm 1 S phase), the C/S/M phases and the adaptive simulator (Algorithm 2),
            with the fixed-schedule replay of the two-pass simulator (Algorithm 3).
philox      the Philox4x32-10 counter-based generator (Salmon et al., SC'11), used only to pin
            the library's generator bit for bit.
quadrature  brute-force grid posteriors for one- and two-parameter logits (pins for the
            simulator's moments and log marginal likelihood).

Parity status of each function (what pins it, in ``tests/test_oracle_*.py``):

* loglik: closed forms (theta = 0, X = 0, single observations with rational probabilities),
  the binary case against scipy's log_expit, outcome-relabelling symmetry.
* loglik_grad: central finite differences of loglik, the closed form at theta = 0.
* ess: bounds, equal weights, a single non-zero weight, shift invariance.
* resample_multinomial: offspring counts sum to N, degenerate weights, exact hand cases,
  unbiasedness of offspring counts over replications (chi-square).
* resample_residual: exact deterministic copies for weights with integral N w, copies never
  below floor(N w) (up to the 2^-40 quantisation), unbiasedness over replications.
* log predictive likelihoods (cphase / sps_run): the first observation's value against the
  direct formula log mean_n p(y_1 | theta_n), X = 0 (each equals -log C exactly), their sum over
  a cycle against the log-ML increment.
* normalise_prior / gprior_covariance: the normalised prior against Monte Carlo draws of the
  class differences; the paper's identity T^-1 sum_t x_t' (2 g T (X'X)^-1) x_t = 2 g.
* group_moments: hand-computed small arrays; calibration of NSE is statistical.
* sps_run: X = 0 (posterior = prior, log ML = -n log C exactly), a dogmatic prior
  (log ML -> loglik at the prior mean), grid quadrature on 1-2 parameter logits.
* philox4x32_10: the published known-answer vectors of Philox4x32-10.
"""
