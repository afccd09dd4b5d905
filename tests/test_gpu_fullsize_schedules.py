"""The paper's schedules at the full headline size (SV, N = 2^24): every step's
likelihood increment, filter mean and ESS against the oracle's summaries of the
GPU's own pre-step state, and the properties that hold at any size -- after all
stages the carried weights are equal (Lemma 3(c)); stages preserve the total
weight, so log N^-1 sum exp(lV) after the step is the oracle's normaliser."""
import numpy as np
import pytest

import synthetic as S
from oracle import bpf
import lockstep as LS

pytestmark = pytest.mark.gpu


def _check_summaries(model, x0, lv_pp, sc, y_n, mean, inc, ess):
    lw, c_n = bpf.weigh(model, x0.astype(np.float64), lv_pp.astype(np.float64), sc["mu_used"], y_n)
    inc_o, mean_o, ess_o, lme = bpf.summaries(lw, x0.astype(np.float64), c_n, sc["mu_used"], sc["mu"])
    assert abs(inc - inc_o) <= LS.TOL_INC * max(1.0, abs(inc_o))
    assert LS.rel_err(mean, mean_o) <= LS.TOL_STATE
    assert abs(ess - ess_o) <= 1e-4 * ess_o
    return lme


def _log_mean_exp(v):
    v = np.asarray(v, dtype=np.float64)
    mx = v.max()
    return mx + np.log(np.mean(np.exp(v - mx)))


def _run(bfpf, w, steps, expand, after, radices=None, **kw):
    """Step the filter; expand(lV, n) gives the per-particle carried weights before step n,
    after(lV, normaliser) checks the carried weights after it."""
    y = w.observations(steps)
    f = bfpf.ButterflyFilter(w.model, w.N, radices or w.radices, w.filter_seed, **kw)
    for n in range(steps):
        x0, lv0, sc = f.state()
        mean, inc, ess = f.step(y[n])
        lme = _check_summaries(w.model, x0, expand(lv0, n), sc, y[n], mean, inc, ess)
        x1, lv1, sc1 = f.state()
        assert np.all(np.isfinite(x1))
        after(lv1, lme)
        assert abs(sc1["mu"] - lme) <= 1e-6 * max(1.0, abs(lme))
    f.close()


def _all_equal_to_normaliser(lv1, lme):
    """After every stage of a step the carried weights are all equal (Lemma 3(c))."""
    assert LS.rel_err(lv1, np.full(lv1.shape, lme)) <= LS.TOL_STATE


def test_fullsize_all_stages(bfpf):
    w = S.workload("sv_n16m")
    m = len(w.radices)
    _run(bfpf, w, 3, lambda lv0, n: LS.per_particle_lV(lv0, w.radices, n * m), _all_equal_to_normaliser,
         all_stages=True)


def test_fullsize_digit_sets(bfpf):
    w = S.workload("sv_n16m")
    radices = (64,) + (2,) * 18                    # 64 particles per PE, 2^18 PEs, 18 stages
    from oracle import butterfly
    gi = butterfly.set_group_index(np.arange(w.N), radices, len(radices) - 1)
    _run(bfpf, w, 2, lambda lv0, n: lv0[gi], _all_equal_to_normaliser, radices=radices, digit_sets=True)


@pytest.mark.parametrize("theta", [0.5, 0.9995])
def test_fullsize_adaptive(bfpf, theta):
    w = S.workload("sv_n16m")

    def after(lv1, lme):                           # stages preserve the total weight
        assert abs(_log_mean_exp(lv1) - lme) <= 1e-5 * max(1.0, abs(lme))
    _run(bfpf, w, 3, lambda lv0, n: lv0, after, adaptive=True, ess_threshold=theta)


def test_fullsize_islands(bfpf):
    w = S.workload("sv_n16m")
    M, mi = 1024, 16384
    _run(bfpf, w, 2, lambda lv0, n: LS.per_particle_lV(lv0, (M, mi), 2 * n), _all_equal_to_normaliser,
         radices=(M, mi), islands="modified")


def test_fullsize_airpf2(bfpf):
    w = S.workload("sv_n16m")
    M, mi = 1024, 16384

    def after(lv1, lme):                           # one weight per island, total weight preserved
        assert lv1.shape == (mi,)
        assert abs(_log_mean_exp(lv1) - lme) <= 1e-5 * max(1.0, abs(lme))
    _run(bfpf, w, 2, lambda lv0, n: lv0[np.arange(w.N) // M], after, radices=(M, mi), islands="modified",
         adaptive=True, ess_threshold=0.5)
