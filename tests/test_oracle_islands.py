"""Pins of the AIRPF oracle (Algorithms 4-7): the island-stage sampling law
against its closed form, the invariants of augmented island resampling, and
the filter against the Kalman filter."""
import numpy as np
import pytest
from scipy import stats

import synthetic as S
from oracle import bpf, kalman, resample


def _pair_outcomes(lW_pair, modified, K=1 << 13, n=3, seed=77):
    """Outcomes of stage 1 for K independent island pairs with the same weights:
    0 = both hold the first sample, 1 = both hold the second, 2 = each keeps its
    own, 3 = the two swapped."""
    lW = np.tile(np.asarray(lW_pair, dtype=np.float64), K)
    _, _, info = bpf.island_stages(lW, seed, n, modified)
    c = info[0]["choice"].reshape(K, 2) - 2 * np.arange(K)[:, None]
    out = np.full(K, -1)
    out[(c[:, 0] == 0) & (c[:, 1] == 0)] = 0
    out[(c[:, 0] == 1) & (c[:, 1] == 1)] = 1
    out[(c[:, 0] == 0) & (c[:, 1] == 1)] = 2
    out[(c[:, 0] == 1) & (c[:, 1] == 0)] = 3
    assert np.all(out >= 0)
    return np.bincount(out, minlength=4), resample.quantise(np.asarray(lW_pair)[None, :], axis=1)[0]


@pytest.mark.parametrize("modified", [False, True])
@pytest.mark.parametrize("lW_pair", [(0.0, 0.0), (0.0, -0.7), (-2.5, 0.3)])
def test_island_pair_law(lW_pair, modified):
    """Each island draws the pair member j with probability given by the integer
    rule's exact law; Algorithm 7 maps the swap outcome to 'each keeps its own',
    so the number of copies of each sample keeps its law."""
    counts, q = _pair_outcomes(lW_pair, modified)
    p1 = resample.exact_law(q)[1]               # probability of drawing the second member
    p0 = 1.0 - p1
    if modified:
        probs = np.array([p0 * p0, p1 * p1, 2 * p0 * p1, 0.0])
    else:
        probs = np.array([p0 * p0, p1 * p1, p0 * p1, p1 * p0])
    K = counts.sum()
    keep = probs > 0
    assert np.all(counts[~keep] == 0)
    chi2 = np.sum((counts[keep] - K * probs[keep]) ** 2 / (K * probs[keep]))
    assert chi2 < stats.chi2.ppf(0.999, keep.sum() - 1), (counts, K * probs)


@pytest.mark.parametrize("modified", [False, True])
def test_island_stages_invariants(modified):
    """After S stages every island weight equals the mean island weight (the
    island analogue of Lemma 3(c)); every stage moves samples only within its
    pairs; the copies of the input samples add up to m."""
    rng = np.random.default_rng(1)
    lW = rng.normal(scale=1.5, size=64)
    holder, V, info = bpf.island_stages(lW, 5, 2, modified)
    mx = lW.max()
    np.testing.assert_allclose(V, mx + np.log(np.mean(np.exp(lW - mx))), rtol=0, atol=1e-12)
    for st in info:
        b = 1 << (st["s"] - 1)
        i = np.arange(64)
        assert np.all((st["choice"] == i) | (st["choice"] == (i ^ b)))
    assert np.bincount(holder, minlength=64).sum() == 64


def test_within_island_weights_are_island_means():
    """Algorithm 5, eq. (out weight): every particle of island k gets the mean of
    g over island k, and draws only from its island."""
    model = S.lg_scalar()
    M, m = 8, 16
    y = S.simulate(model, 1, seed=2)[1]
    st = bpf.init_state(model, M * m, seed=4)
    _, o = bpf.step_islands(model, M, m, 4, st, y[0])
    s_x, _ = bpf.obs_terms(model, st.x, y[0])
    lw = s_x - st.mu
    g = np.exp(lw - lw.max()).reshape(m, M)
    np.testing.assert_allclose(np.exp(o["lW"] - lw.max()), g.mean(axis=1), rtol=1e-12)
    assert np.all(o["within"]["anc"] // M == np.arange(M * m) // M)


@pytest.mark.parametrize("modified", ["modified", "plain"])
def test_airpf_loglik_consistent_with_kalman(modified):
    """AIRPF's likelihood estimate against the Kalman filter over independent seeds
    (mean of the log error near minus half its variance, as for any unbiased p^)."""
    w = S.workload("lg1d_n1024")
    y = w.observations()[:60]
    kf = kalman.kalman_filter(w.model, y)
    lls = np.array([bpf.run(w.model, 1024, (32, 32), 4000 + r, y, islands=modified)["loglik"] for r in range(16)])
    err = lls - kf["loglik"]
    se = err.std(ddof=1) / np.sqrt(len(err))
    assert abs(err.mean() + 0.5 * err.var(ddof=1)) < 4 * se + 0.05, (err.mean(), err.var())


def test_airpf_mean_converges_to_kalman():
    w = S.workload("lg1d_n1024")
    y = w.observations()[:40]
    kf = kalman.kalman_filter(w.model, y)
    mses = []
    for M in (16, 256):
        errs = [np.sum((bpf.run(w.model, M * 16, (M, 16), 500 + r, y, islands="modified")["mean"][:, 0]
                        - kf["mean"][:, 0]) ** 2) for r in range(6)]
        mses.append(np.mean(errs))
    assert mses[1] < mses[0] / 6, mses       # 16x the particles: about 16x less error


def test_airpf2_theta_limits():
    """Fully adapted island stages: theta > 1 runs every stage (= AIRPF1), theta = 0
    none (each island keeps its own sample and its weight)."""
    model = S.sv_model()
    M, m = 8, 16
    y = S.simulate(model, 4, seed=5)[1]
    a = bpf.init_state(model, M * m, seed=3)
    b = bpf.init_state(model, M * m, seed=3)
    c = bpf.init_state(model, M * m, seed=3)
    for n in range(4):
        a, oa = bpf.step_islands(model, M, m, 3, a, y[n])
        b, ob = bpf.step_islands(model, M, m, 3, b, y[n], theta=1.5)
        np.testing.assert_array_equal(a.x, b.x)
        assert len(ob["island_info"]) == 4
        c, oc = bpf.step_islands(model, M, m, 3, c, y[n], theta=0.0)
        assert oc["island_info"] == [] and np.array_equal(oc["holder"], np.arange(m))
        np.testing.assert_allclose(c.lV.reshape(m, M), oc["lW"][:, None] * np.ones((1, M)), rtol=0, atol=0)


def test_airpf2_stops_at_threshold():
    rng = np.random.default_rng(3)
    lW = rng.normal(scale=2.0, size=64)
    theta = 0.6
    holder, V, info = bpf.island_stages(lW, 9, 1, True, theta)
    for st in info:
        assert st["ess_before"] < theta
    if len(info) < 6:
        assert bpf.ess_of(V) >= theta
