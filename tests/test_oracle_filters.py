"""Pins for the oracle's filters against what mathematics and the paper fix.

* Kalman filter  == conditioning of the joint Gaussian law of (X_0..X_T, Y_0..Y_T)
  (log-likelihood and filtering means), and the scalar steady-state Riccati root;
* grid filter    == Kalman on a scalar linear-Gaussian model;
* butterfly BPF with one digit (radices = (N,))  == a textbook BPF (Algorithm 1 +
  Algorithm 2) written here with the same integer draw: identical ancestors and
  likelihood;
* butterfly BPF -> Kalman as N grows (MSE ~ 1/N), and -> grid filter on SV;
* Section 6.3: the raw-observation MSE printed in the paper (2396) against the
  closed-form expectation from the Kalman gains, and our data generator's value.
"""
import os

import numpy as np
import pytest
from scipy import stats

import synthetic as S
from oracle import bpf, gridfilter, kalman, philox, resample


def _joint_gaussian(model, T):
    d, dy = model.d, model.dy
    A, H = model.A, model.H
    Q = model.Lq @ model.Lq.T
    R = model.Lr @ model.Lr.T
    P0 = model.L0 @ model.L0.T
    Ap = [np.linalg.matrix_power(A, n) for n in range(T)]
    mx = np.concatenate([Ap[n] @ model.m0 for n in range(T)])
    Cx = np.zeros((T * d, T * d))
    for n in range(T):
        for m in range(T):
            c = Ap[n] @ P0 @ Ap[m].T
            for j in range(1, min(n, m) + 1):
                c = c + Ap[n - j] @ Q @ Ap[m - j].T
            Cx[n * d:(n + 1) * d, m * d:(m + 1) * d] = c
    Hb = np.kron(np.eye(T), H)
    Cy = Hb @ Cx @ Hb.T + np.kron(np.eye(T), R)
    Cxy = Cx @ Hb.T
    return mx, Hb @ mx, Cx, Cy, Cxy


def test_kalman_equals_joint_gaussian_conditioning():
    model = S.lg_dense(3, seed=12)
    model.H = np.array([[1.0, 0.5, 0.0], [0.0, -1.0, 2.0]])
    model.Lr = np.array([[0.7, 0.0], [0.3, 0.9]])
    model.m0 = np.array([0.5, -1.0, 0.2])
    model.L0 = np.array([[1.0, 0, 0], [0.2, 0.8, 0], [0.1, -0.3, 1.1]])
    T = 7
    _, y = S.simulate(model, T, seed=4)
    kf = kalman.kalman_filter(model, y)
    mx, my, Cx, Cy, Cxy = _joint_gaussian(model, T)
    yv = y.reshape(-1)
    want_ll = stats.multivariate_normal(mean=my, cov=Cy).logpdf(yv)
    assert abs(kf["loglik"] - want_ll) < 1e-9 * abs(want_ll)
    d, dy = model.d, model.dy
    for n in range(T):
        sl = slice(0, (n + 1) * dy)
        mean_n = mx[n * d:(n + 1) * d] + Cxy[n * d:(n + 1) * d, sl] @ np.linalg.solve(Cy[sl, sl], yv[sl] - my[sl])
        np.testing.assert_allclose(kf["mean"][n], mean_n, rtol=1e-9, atol=1e-11)


def test_kalman_scalar_steady_state_riccati():
    # x = a x + N(0,q), y = x + N(0,r): predicted variance P solves P = a^2 P r/(P+r) + q
    a, q, r = 0.9, 1.0, 1.0
    model = S.lg_scalar(a, q, r)
    _, y = S.simulate(model, 200, seed=1)
    kf = kalman.kalman_filter(model, y)
    # filtered variance F = P r / (P + r);  P = a^2 F + q  -> quadratic in P
    bq = r - a * a * r - q
    P = (-bq + np.sqrt(bq * bq + 4 * q * r)) / 2
    F = P * r / (P + r)
    assert abs(kf["cov"][-1, 0, 0] - F) < 1e-12


def test_grid_filter_matches_kalman_on_scalar_lg():
    model = S.lg_scalar()
    _, y = S.simulate(model, 60, seed=21)
    kf = kalman.kalman_filter(model, y)
    gf = gridfilter.lg_scalar_grid_filter(model, y, G=4096)
    np.testing.assert_allclose(gf["mean"], kf["mean"], atol=1e-8)
    assert abs(gf["loglik"] - kf["loglik"]) < 1e-8 * abs(kf["loglik"])


def _textbook_bpf(model, N, seed, y):
    """Algorithm 1 with Algorithm 2 (global multinomial) and the integer draw rule;
    written without groups, carried weights or normalisers."""
    x = bpf.initial_particles(model, N, seed)
    ll = 0.0
    ancs = []
    for n in range(len(y)):
        s_x, c = bpf.obs_terms(model, x, y[n])
        # loglik increment of the standard BPF: log N^-1 sum_i g_n(x_i)
        mx = s_x.max()
        ll += mx + np.log(np.mean(np.exp(s_x - mx))) + c
        q = resample.quantise(s_x, axis=0)
        if N <= resample.NARROW_MAX_RADIX:
            r = philox.resample_words(seed, n, N)
            u = resample.scaled_uniform(r, np.full(N, q.sum(), np.uint64), N)
        else:
            lo, hi = philox.resample_words_wide(seed, n, N)
            u = resample.scaled_uniform(lo, np.full(N, q.sum(), np.uint64), N, hi)
        P = np.cumsum(q)
        anc = np.searchsorted(P, u, side="right")
        ancs.append(anc)
        x = bpf.mutate(model, x[anc], n, seed)
    return ll, np.stack(ancs), x


@pytest.mark.parametrize("N", [64, 512])
def test_single_digit_reduces_to_textbook_bpf(N):
    model = S.lg_scalar()
    _, y = S.simulate(model, 25, seed=5)
    ll, ancs, x = _textbook_bpf(model, N, 31, y)
    o = bpf.run(model, N, (N,), 31, y, keep_ancestors=True)
    assert np.array_equal(o["anc"], ancs)
    np.testing.assert_allclose(o["state"].x, x, rtol=0, atol=0)
    assert abs(o["loglik"] - ll) < 1e-10 * abs(ll)


def test_single_digit_reduces_to_textbook_bpf_sv():
    model = S.sv_model()
    _, y = S.simulate(model, 20, seed=6)
    ll, ancs, x = _textbook_bpf(model, 128, 8, y)
    o = bpf.run(model, 128, (128,), 8, y, keep_ancestors=True)
    assert np.array_equal(o["anc"], ancs)
    assert abs(o["loglik"] - ll) < 1e-10 * abs(ll)


def test_butterfly_mse_against_kalman_scales_as_one_over_n():
    model = S.lg_scalar()
    _, y = S.simulate(model, 30, seed=8)
    kf = kalman.kalman_filter(model, y)
    Ns = [2 ** 7, 2 ** 9, 2 ** 11, 2 ** 13]
    mses = []
    for N in Ns:
        errs = []
        for r in range(6):
            o = bpf.run(model, N, (2,) * int(np.log2(N)), 100 + r, y)
            errs.append(np.mean((o["mean"] - kf["mean"]) ** 2))
        mses.append(np.mean(errs))
    slope = np.polyfit(np.log(Ns), np.log(mses), 1)[0]
    assert -1.3 < slope < -0.7, (slope, mses)


def test_loglik_consistent_with_kalman():
    """The estimate p^(y) is unbiased (alpha-SMC); in logs its mean sits below the truth
    by about half its variance.  Check both over independent seeds."""
    w = S.workload("lg1d_n1024")
    y = w.observations()
    kf = kalman.kalman_filter(w.model, y)
    lls = np.array([bpf.run(w.model, w.N, w.radices, 1000 + r, y)["loglik"] for r in range(16)])
    err = lls - kf["loglik"]
    se = err.std(ddof=1) / np.sqrt(len(err))
    assert abs(err.mean() + 0.5 * err.var(ddof=1)) < 4 * se + 0.05, (err.mean(), err.var())


def test_sv_butterfly_against_grid_filter():
    model = S.sv_model()
    _, y = S.simulate(model, 40, seed=3)
    gf = gridfilter.sv_grid_filter(model, y, G=2048)
    o = bpf.run(model, 1 << 14, (16, 16, 16, 4), 3000, y)
    rmse = np.sqrt(np.mean((o["mean"] - gf["mean"]) ** 2))
    assert rmse < 0.02, rmse
    assert abs(o["loglik"] - gf["loglik"]) < 0.3


def test_sv_grid_filter_converged_in_grid_size():
    model = S.sv_model()
    _, y = S.simulate(model, 40, seed=3)
    a = gridfilter.sv_grid_filter(model, y, G=1024)
    b = gridfilter.sv_grid_filter(model, y, G=4096)
    np.testing.assert_allclose(a["mean"], b["mean"], atol=1e-6)
    assert abs(a["loglik"] - b["loglik"]) < 1e-6


def test_paper_raw_observation_mse(golden_dir):
    """Section 6.3: raw-observation MSE 2396 for the d=7 random walk, R = I/4, n_max = 8000.
    Its expectation follows from the Kalman gains: y_n - xbar_n = (I - K_n) nu_n with
    independent innovations nu_n ~ N(0, S_n)."""
    vals = {}
    for line in open(os.path.join(golden_dir, "raw_mse_rw7d.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    d, T = int(vals["d"]), int(vals["n_max"])
    model = S.random_walk(d, obs_std=np.sqrt(vals["obs_var"]))
    # closed form of E[raw MSE] and its standard deviation
    P = model.L0 @ model.L0.T
    Q = model.Lq @ model.Lq.T
    R = model.Lr @ model.Lr.T
    mean_mse, var_mse = 0.0, 0.0
    for n in range(T):
        if n > 0:
            P = P + Q
        Sn = P + R
        K = P @ np.linalg.inv(Sn)
        C = (np.eye(d) - K) @ Sn @ (np.eye(d) - K).T
        mean_mse += np.trace(C)
        var_mse += 2 * np.trace(C @ C)
        P = P - K @ Sn @ K.T
    sd = np.sqrt(var_mse)
    assert abs(mean_mse - 2402.07) < 0.05          # value quoted for this closed form
    assert abs(vals["raw_mse"] - mean_mse) < 3 * sd  # the paper's realisation
    # our generator's realisation of the same data set
    x, y = S.simulate(model, T, seed=7)
    kf = kalman.kalman_filter(model, y)
    raw = np.sum((y - kf["mean"]) ** 2)
    assert abs(raw - mean_mse) < 4 * sd, (raw, mean_mse, sd)
