"""Pins for the oracle's model functions against facts outside the oracle.

The HMM of Section 1.1 (eq. (HMM)) is specified by its densities: the
potential g(x, y) is the observation density and f(x, .) the transition
kernel, and pi_0 the initial law (Section 6.1 uses X_0 ~ N(0, I)).  Each
test below checks one oracle function against an independent statement of
that density or law, on a model where every matrix is non-trivial (dense
A, lower-triangular Lq / L0 / Lr with off-diagonal entries, a non-square H,
nonzero m0), so that a transposed factor, a dropped term or a wrong sign
fails:

* ``bpf.obs_terms`` (log g split as s(x) + c): against scipy's normal and
  multivariate-normal log densities of the observation model;
* ``bpf.mutate``: the sample mean and covariance of f(x, .) over 10^6 draws
  against A x and Lq Lq^T (residual regression on random x, 5 standard errors);
* ``bpf.initial_particles``: the sample moments of pi_0 against m0, L0 L0^T
  (linear-Gaussian) and the stationary law N(0, sigma^2 / (1 - phi^2)) (SV);
* the whole filter on the dense model: its log-likelihood estimate is
  consistent with the Kalman filter's (Jensen bias of an unbiased estimate) and
  the squared error of its filtering means falls as 1/N.
"""
import numpy as np
import pytest
from scipy import stats

import synthetic as S
from oracle import bpf, kalman


def dense_model():
    """d = 3, dy = 2: every matrix non-trivial and not symmetric."""
    model = S.lg_dense(3, seed=12)
    model.A = np.array([[0.8, 0.3, -0.1], [-0.2, 0.7, 0.25], [0.05, -0.3, 0.6]])
    model.Lq = np.array([[0.9, 0.0, 0.0], [0.6, 0.5, 0.0], [-0.4, 0.7, 0.3]])
    model.H = np.array([[1.0, 0.5, 0.0], [0.0, -1.0, 2.0]])
    model.Lr = np.array([[0.7, 0.0], [0.3, 0.9]])
    model.m0 = np.array([0.5, -1.0, 0.2])
    model.L0 = np.array([[1.0, 0, 0], [0.2, 0.8, 0], [0.1, -0.3, 1.1]])
    return model


def check_sv_obs(bpf_mod):
    """SV: Y = beta exp(X/2) W, W ~ N(0, 1), so g(x, y) = N(y; 0, beta^2 e^x)."""
    for model in (S.sv_model(), S.sv_model(phi=0.9, sigma=0.4, beta=1.7)):
        x = np.linspace(-5.0, 4.0, 37)[:, None]
        for y in (-2.3, -0.31, 0.0, 0.47, 3.1):
            s, c = bpf_mod.obs_terms(model, x, np.array([y]))
            want = stats.norm.logpdf(y, loc=0.0, scale=model.beta * np.exp(x[:, 0] / 2))
            np.testing.assert_allclose(s + c, want, rtol=1e-13, atol=1e-12)


def check_lg_obs(bpf_mod):
    """LG: Y = H X + Lr W, so g(x, y) = N(y; H x, Lr Lr^T)."""
    model = dense_model()
    rng = np.random.default_rng(3)
    x = rng.standard_normal((50, 3)) * 1.5
    R = model.Lr @ model.Lr.T
    for _ in range(4):
        y = rng.standard_normal(2) * 2.0
        s, c = bpf_mod.obs_terms(model, x, y)
        want = np.array([stats.multivariate_normal(mean=model.H @ xi, cov=R).logpdf(y) for xi in x])
        np.testing.assert_allclose(s + c, want, rtol=1e-12, atol=1e-12)


def _moments_within(sample, mean, cov, nse=5.0):
    """Sample mean and covariance of ``sample`` (n x d) within nse standard errors of
    (mean, cov); the standard error of a covariance entry is sqrt((C_ii C_jj + C_ij^2) / n)."""
    n = sample.shape[0]
    m = sample.mean(axis=0)
    se_m = np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(m - mean) < nse * se_m), (m, mean, se_m)
    C = np.cov(sample, rowvar=False).reshape(cov.shape)
    se_C = np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov ** 2) / n)
    assert np.all(np.abs(C - cov) < nse * se_C), (C, cov, se_C)


def check_mutate(bpf_mod):
    """f(x, .) = N(A x, Lq Lq^T): the residuals of the draws on random x."""
    model = dense_model()
    n = 1_000_000
    rng = np.random.default_rng(9)
    xhat = rng.standard_normal((n, 3))
    x1 = bpf_mod.mutate(model, xhat, 5, seed=77)
    resid = x1 - xhat @ model.A.T
    _moments_within(resid, np.zeros(3), model.Lq @ model.Lq.T)
    # the regression coefficients themselves: E[resid x^T] = 0
    cross = resid.T @ xhat / n
    assert np.all(np.abs(cross) < 5 * np.sqrt(np.diag(model.Lq @ model.Lq.T))[:, None] / np.sqrt(n))


def check_mutate_sv(bpf_mod):
    model = S.sv_model()
    n = 1_000_000
    xhat = np.linspace(-1.0, 1.0, n)[:, None]
    x1 = bpf_mod.mutate(model, xhat, 3, seed=5)
    resid = x1 - model.phi * xhat
    _moments_within(resid, np.zeros(1), np.array([[model.sigma ** 2]]))


def check_init_lg(bpf_mod):
    model = dense_model()
    x0 = bpf_mod.initial_particles(model, 1_000_000, seed=41)
    _moments_within(x0, model.m0, model.L0 @ model.L0.T)


def check_init_sv(bpf_mod):
    model = S.sv_model()
    x0 = bpf_mod.initial_particles(model, 1_000_000, seed=42)
    var = model.sigma ** 2 / (1 - model.phi ** 2)
    _moments_within(x0, np.zeros(1), np.array([[var]]))


CHECKS = dict(sv_obs=check_sv_obs, lg_obs=check_lg_obs, mutate=check_mutate, mutate_sv=check_mutate_sv,
              init_lg=check_init_lg, init_sv=check_init_sv)


@pytest.mark.parametrize("name", sorted(CHECKS))
def test_model_function_pin(name):
    CHECKS[name](bpf)


def test_dense_model_factors_are_not_symmetric():
    """The pins can tell a factor from its transpose: Lq^T Lq, L0^T L0 and Lr^T Lr
    differ from Lq Lq^T, L0 L0^T and Lr Lr^T by far more than the tolerances."""
    model = dense_model()
    for L in (model.Lq, model.L0, model.Lr):
        assert np.max(np.abs(L.T @ L - L @ L.T)) > 0.05
    assert np.max(np.abs(model.A - model.A.T)) > 0.1


@pytest.fixture(scope="module")
def dense_runs():
    model = dense_model()
    _, y = S.simulate(model, 20, seed=31)
    kf = kalman.kalman_filter(model, y)
    return model, y, kf


@pytest.mark.parametrize("schedule", ["global", "all_stages"])
def test_dense_model_loglik_consistent_with_kalman(dense_runs, schedule):
    """The likelihood estimate is unbiased in p^ (alpha-SMC with doubly stochastic
    stages), so log p^ sits below the Kalman value by about half its variance.
    Checked with global resampling (radices (N,)) and with every stage of
    Algorithm 3 per step, whose weights are equalised at every step; the
    one-digit schedule's log-estimate is too heavy-tailed on this sharp
    3-D likelihood for a 16-run check of its mean."""
    model, y, kf = dense_runs
    rad, kw = ((1024,), {}) if schedule == "global" else ((4, 4, 4, 4, 4), dict(all_stages=True))
    lls = np.array([bpf.run(model, 1024, rad, 500 + r, y, **kw)["loglik"] for r in range(16)])
    err = lls - kf["loglik"]
    se = err.std(ddof=1) / np.sqrt(len(err))
    assert abs(err.mean() + 0.5 * err.var(ddof=1)) < 4 * se + 0.05, (err.mean(), err.var())


def test_dense_model_mse_scales_as_one_over_n(dense_runs):
    model, y, kf = dense_runs
    Ns = [2 ** 8, 2 ** 10, 2 ** 12]
    mses = []
    for N in Ns:
        errs = [np.mean((bpf.run(model, N, (4,) * int(np.log2(N) // 2), 700 + r, y, all_stages=True)["mean"]
                         - kf["mean"]) ** 2) for r in range(6)]
        mses.append(np.mean(errs))
    slope = np.polyfit(np.log(Ns), np.log(mses), 1)[0]
    assert -1.35 < slope < -0.65, (slope, mses)
