"""Pins for the integer multinomial draw and one augmented-resampling cycle.

* the exact law of the integer draw (closed-form counts) is within 2^-W of q_j/Q
  and the oracle's Philox-driven draws follow it (chi-square);
* Proposition 1 (unbiasedness) and Lemma 3 (V_S = N^-1 sum g) hold for a full
  digit cycle, computed by exact enumeration over ancestor vectors at N = 4, 8;
* invariants of every step: ancestors differ from the child only in digit k,
  offspring counts per group sum to a_k, and sum exp(lV') = sum exp(lw).
"""
import itertools

import numpy as np
import pytest
from scipy import stats

import synthetic as S
from oracle import bpf, butterfly, philox, resample


def test_exact_law_close_to_weights():
    rng = np.random.default_rng(0)
    for a in (2, 3, 16, 32, 300):
        lw = rng.normal(0, 3, a)
        q = resample.quantise(lw, axis=0)
        assert q.max() == 2 ** resample.qbits(a)
        law = resample.exact_law(q, a_bits_wide=a > 256)
        W = 64 if a > 256 else 32
        np.testing.assert_allclose(law, q / q.sum(), atol=2.0 ** -W * 2, rtol=1e-13)
        assert abs(law.sum() - 1) < 1e-12


def test_quantise_matches_fp32_exp_definition():
    lw = np.array([-1.25, 0.0, -30.0, -17.5, np.nan, -np.inf])
    q = resample.quantise(lw, axis=0)
    e = np.exp(np.float32(lw[:4] - 0.0).astype(np.float64)).astype(np.float32)
    assert np.array_equal(q[:4], np.floor(e.astype(np.float64) * 2 ** 24).astype(np.uint64))
    assert q[4] == 0 and q[5] == 0 and q[1] == 2 ** 24


def test_draw_is_upper_bound():
    q = np.array([0, 5, 0, 3, 2], dtype=np.uint64)   # P = 0 5 5 8 10
    u = np.array([0, 4, 5, 7, 9], dtype=np.uint64)
    got = resample.draw(q, u, axis=0)
    assert got.tolist() == [1, 1, 3, 3, 4]           # zero-weight members never drawn
    # all-zero group keeps particles in place
    assert resample.draw(np.zeros(3, np.uint64), np.zeros(3, np.uint64), 0).tolist() == [0, 1, 2]


def test_draw_wide_equals_searchsorted():
    rng = np.random.default_rng(5)
    a = 400
    q = resample.quantise(rng.normal(0, 2, a), axis=0)
    Q = int(q.sum())
    lo = rng.integers(0, 2 ** 32, a, dtype=np.uint64)
    hi = rng.integers(0, 2 ** 32, a, dtype=np.uint64)
    u = resample.scaled_uniform(lo, np.full(a, Q, np.uint64), a, hi)
    want = [((int(h) << 32 | int(l)) * Q) >> 64 for l, h in zip(lo, hi)]
    assert u.tolist() == want
    got = resample.draw(q, u, axis=0)
    P = np.cumsum(q)
    assert got.tolist() == [int(np.sum(P <= v)) for v in u]


def test_philox_draws_follow_exact_law():
    """10^5 oracle draws of one group against the closed-form law (chi-square)."""
    a = 4
    lw = np.log(np.array([0.1, 0.4, 0.2, 0.3]))
    q = resample.quantise(lw, axis=0)
    law = resample.exact_law(q)
    counts = np.zeros(a)
    Q = np.uint64(q.sum())
    for n in range(25):
        r = philox.resample_words(seed=77, n=n, N=4096)
        u = resample.scaled_uniform(r, np.full(r.shape, Q, np.uint64), a)
        j = resample.draw(np.broadcast_to(q, (1024, a)).T.copy(), u.reshape(1024, a).T, axis=0)
        counts += np.bincount(j.reshape(-1), minlength=a)
    chi2, p = stats.chisquare(counts, law * counts.sum())
    assert p > 1e-4, (counts, law)


def _exact_transition(lw, radices, k):
    """Row-stochastic matrix P[i, j] = exact probability that new particle i copies j
    at a stage on digit k, from the integer law of each group."""
    N = len(lw)
    P = np.zeros((N, N))
    for i in range(N):
        mem = butterfly.group_members(i, radices, k)
        q = resample.quantise(lw[mem], axis=0)
        law = resample.exact_law(q)
        for j, pj in zip(mem, law):
            P[i, j] += pj
    return P


def _cycle_models():
    """Potential g at step 0 only, flat afterwards; identity mutation (A = 1, Lq = 0).
    With y = 0, H = 1, Lr = 1 a particle at x has s(x) = -x^2/2, so x = -sqrt(-2 log g)."""
    one = np.ones((1, 1))
    m0 = S.LinearGaussian(A=one, Lq=0 * one, H=one, Lr=one, m0=np.zeros(1), L0=one)
    m1 = S.LinearGaussian(A=one, Lq=0 * one, H=0 * one, Lr=one, m0=np.zeros(1), L0=one)
    return m0, m1


def _run_cycle(g, radices, seed=5):
    N = len(g)
    m0, m1 = _cycle_models()
    x = -np.sqrt(-2 * np.log(g))[:, None]
    st = bpf.State(x=x.copy(), lV=np.zeros(N), mu=0.0, n=0)
    outs = []
    for k in range(len(radices)):
        st, o = bpf.step(m0 if k == 0 else m1, radices, seed, st, np.zeros(1))
        outs.append(o)
    return st, outs, x[:, 0]


@pytest.mark.parametrize("radices", [(2, 2), (2, 2, 2), (2, 4), (4, 2)])
def test_prop1_and_lemma3_by_exact_enumeration(radices):
    """One full cycle of stages with g applied at stage 0 only (Algorithm 3), run by the
    oracle's own step: Lemma 3(c) (V_S = N^-1 sum g: all final weights equal) and
    Prop. 1 (E[N^-1 sum phi(xi_S)] = sum g phi / sum g), the expectation computed by exact
    enumeration of the per-stage integer laws, up to the quantisation (< a 2^-24 per stage)."""
    rng = np.random.default_rng(sum(radices) * 10 + len(radices))
    N = int(np.prod(radices))
    g = rng.uniform(0.05, 1.0, N)
    phi = rng.normal(size=N)
    st, outs, x0 = _run_cycle(g, radices)
    # Lemma 3(c): the carried weights are all equal after the cycle ...
    np.testing.assert_allclose(st.lV, st.lV[0], rtol=0, atol=1e-12)
    # ... and the first step's likelihood increment is log N^-1 sum g (plus the constant)
    np.testing.assert_allclose(outs[0]["inc"] - outs[0]["c"], np.log(g.mean()), rtol=1e-12)
    # every particle drawn in the cycle is a copy of an original particle
    assert np.all(np.isin(st.x[:, 0], x0))
    # E[phi(xi_s^i)] = sum_j P_s[i, j] E[phi(xi_{s-1}^j)]: apply stage 0's law first
    E = phi.copy()
    for k in range(len(radices)):
        E = _exact_transition(outs[k]["lw"], radices, k) @ E
    want = np.sum(g * phi) / np.sum(g)
    tol = len(radices) * max(radices) * 2.0 ** -24 * np.abs(phi).max() * 4
    assert abs(E.mean() - want) < tol, (E.mean(), want)


def test_prop1_brute_force_paths_n4():
    """N = 4, radices (2,2): sum over every pair of ancestor vectors of the two stages,
    with the stage laws of the oracle's step."""
    rng = np.random.default_rng(11)
    radices = (2, 2)
    g = rng.uniform(0.1, 1, 4)
    phi = rng.normal(size=4)
    _, outs, _ = _run_cycle(g, radices)
    P1 = _exact_transition(outs[0]["lw"], radices, 0)
    P2 = _exact_transition(outs[1]["lw"], radices, 1)
    total = 0.0
    for anc1 in itertools.product(*[butterfly.group_members(i, radices, 0) for i in range(4)]):
        p1 = np.prod([P1[i, anc1[i]] for i in range(4)])
        for anc2 in itertools.product(*[butterfly.group_members(i, radices, 1) for i in range(4)]):
            p2 = np.prod([P2[i, anc2[i]] for i in range(4)])
            xi2 = [anc1[anc2[i]] for i in range(4)]
            total += p1 * p2 * np.mean(phi[xi2])
    want = np.sum(g * phi) / np.sum(g)
    assert abs(total - want) < 1e-6


@pytest.mark.parametrize("radices", [(2,) * 6, (4, 8, 2), (3, 5, 4)])
def test_step_invariants(radices):
    N = int(np.prod(radices))
    model = S.lg_scalar()
    y = S.simulate(model, 12, seed=3)[1]
    st = bpf.init_state(model, N, seed=9)
    for n in range(12):
        prev = st
        st, o = bpf.step(model, radices, 9, st, y[n])
        k, a, s = o["k"], o["a"], o["stride"]
        idx = np.arange(N)
        anc = o["anc"]
        # ancestor differs from the child only in digit k
        assert np.array_equal(idx // (a * s), anc // (a * s))
        assert np.array_equal(idx % s, anc % s)
        # offspring counts per group sum to a_k
        grp = (anc // (a * s)) * s + anc % s
        counts = np.bincount(grp, minlength=N // a)
        assert np.all(counts == a)
        # V_s = A_s V_{s-1}: total weight conserved (double stochasticity)
        np.testing.assert_allclose(np.sum(np.exp(o["lV_new"])), np.sum(np.exp(o["lw"])), rtol=1e-12)
        # the new weights are constant on the groups of digit k
        lvg = o["lV_new"].reshape(N // (a * s), a, s)
        assert np.all(lvg == lvg[:, :1, :])
        # the carried normaliser is the log-mean weight
        assert np.isclose(st.mu, np.log(np.mean(np.exp(st.lV))), rtol=0, atol=1e-12)


@pytest.mark.parametrize("radices,n", [((4, 8, 2), 0), ((4, 8, 2), 1), ((4, 8, 2), 2), ((3, 5), 1), ((300, 2), 0)])
def test_step_on_groups_equals_full_step(radices, n):
    """The group-restricted step (used to check full-size GPU runs) agrees with the full step."""
    N = int(np.prod(radices))
    model = S.lg_dense(3, seed=4)
    y = S.simulate(model, 4, seed=2)[1]
    st = bpf.init_state(model, N, seed=6)
    for t in range(n):
        st, _ = bpf.step(model, radices, 6, st, y[t])
    new, o = bpf.step(model, radices, 6, st, y[n])
    k = n % len(radices)
    a, s_k = radices[k], butterfly.strides(radices)[k]
    H = N // (a * s_k)
    groups = np.array([(h, l) for h in range(H) for l in range(s_k)])
    g = bpf.step_on_groups(model, radices, 6, n, st.x, st.lV, st.mu, y[n], groups)
    assert np.array_equal(np.sort(g["idx"].reshape(-1)), np.arange(N))
    flat = g["idx"].reshape(-1)
    assert np.array_equal(g["anc"].reshape(-1), o["anc"][flat])
    np.testing.assert_allclose(g["x_next"].reshape(-1, 3), new.x[flat], rtol=1e-13, atol=1e-13)
    lv_c = o["lV_new"].reshape(H, a, s_k)[:, 0, :].reshape(-1)
    np.testing.assert_allclose(g["lV_new"], lv_c[groups[:, 0] * s_k + groups[:, 1]], rtol=1e-13)


@pytest.mark.parametrize("radices", [(2, 2, 2), (4, 8), (3, 5, 2)])
def test_all_stages_schedule_lemma3_and_textbook_increment(radices):
    """The paper's schedule (all stages of Algorithm 3 per time step): after each
    step the carried weights are all equal (Lemma 3(c)), and the likelihood
    increment equals the textbook BPF's log N^-1 sum_i g_n(zeta_i) on the same
    particles (since V_S = N^-1 sum g)."""
    N = int(np.prod(radices))
    model = S.lg_scalar()
    y = S.simulate(model, 6, seed=13)[1]
    st = bpf.init_state(model, N, seed=21)
    for n in range(6):
        s_x, c = bpf.obs_terms(model, st.x, y[n])
        mx = s_x.max()
        textbook = mx + np.log(np.mean(np.exp(s_x - mx))) + c
        st, o = bpf.step_all_stages(model, radices, 21, st, y[n])
        np.testing.assert_allclose(st.lV, st.lV[0], rtol=0, atol=1e-12)
        assert abs(o["inc"] - textbook) < 1e-10
        # every stage moves particles only inside their digit-k groups
        for sg in o["stages"]:
            k = sg["k"]
            a, s = radices[k], butterfly.strides(radices)[k]
            idx = np.arange(N)
            assert np.array_equal(sg["anc"] // (a * s), idx // (a * s)) and np.array_equal(sg["anc"] % s, idx % s)


def test_all_stages_with_one_digit_is_the_one_digit_step():
    """With m = 1 the two schedules coincide, counters included (t = n)."""
    model = S.sv_model()
    y = S.simulate(model, 4, seed=3)[1]
    a = bpf.init_state(model, 64, seed=8)
    b = bpf.init_state(model, 64, seed=8)
    for n in range(4):
        a, oa = bpf.step(model, (64,), 8, a, y[n])
        b, ob = bpf.step_all_stages(model, (64,), 8, b, y[n])
        assert np.array_equal(a.x, b.x) and np.array_equal(oa["anc"], ob["stages"][0]["anc"])
        assert oa["inc"] == ob["inc"]


def test_adaptive_theta_above_one_is_all_stages():
    """ESS <= 1 < theta: every stage runs, so the step is the all-stages step."""
    model, radices = S.lg_scalar(), (4, 2, 8)
    y = S.simulate(model, 4, seed=5)[1]
    a = bpf.init_state(model, 64, seed=3)
    b = bpf.init_state(model, 64, seed=3)
    for n in range(4):
        a, oa = bpf.step_all_stages(model, radices, 3, a, y[n])
        b, ob = bpf.step_adaptive(model, radices, 3, b, y[n], theta=1.5, rotate=True)
        assert len(ob["stages"]) == 3 and b.start == 0
        assert np.array_equal(a.x, b.x) and np.array_equal(a.lV, b.lV) and oa["inc"] == ob["inc"]


def test_adaptive_theta_zero_is_sequential_importance_sampling():
    """theta <= 1/N never resamples: each particle keeps its own path and the
    likelihood estimate is log N^-1 sum_i prod_n g_n(x_i^n), computed here
    directly from the unresampled paths."""
    model = S.lg_dense(2, seed=6)
    radices, N, T = (4, 4), 16, 5
    y = S.simulate(model, T, seed=8)[1]
    st = bpf.init_state(model, N, seed=9)
    x = st.x.copy()
    logg = np.zeros(N)
    const = 0.0
    for n in range(T):
        s_x, c = bpf.obs_terms(model, x, y[n])
        logg += s_x
        const += c
        st, o = bpf.step_adaptive(model, radices, 9, st, y[n], theta=0.0)
        assert o["stages"] == []
        x = bpf.mutate(model, x, n, 9, idx=butterfly.group_major(N, radices, 1))
        np.testing.assert_allclose(st.x, x, rtol=0, atol=0)
    mx = logg.max()
    direct = mx + np.log(np.mean(np.exp(logg - mx))) + const
    assert abs(st.loglik - direct) < 1e-9 * max(1.0, abs(direct))


@pytest.mark.parametrize("rotate", [False, True])
def test_adaptive_stopping_rule_and_weight_mass(rotate):
    """Stages run in rotation order while the ESS is below theta and stop once it
    reaches theta; each stage preserves the total weight (doubly stochastic A)."""
    model, radices = S.sv_model(), (4, 4, 4)
    N, theta = 64, 0.7
    y = S.simulate(model, 12, seed=12)[1]
    st = bpf.init_state(model, N, seed=13)
    starts = []
    for n in range(12):
        start = st.start
        starts.append(start)
        st, o = bpf.step_adaptive(model, radices, 13, st, y[n], theta=theta, rotate=rotate)
        for j, sg in enumerate(o["stages"]):
            assert sg["j"] == j and sg["k"] == (start + j) % 3 and sg["ess_before"] < theta
            mx = sg["lw"].max()
            np.testing.assert_allclose(np.sum(np.exp(sg["lV_new"] - mx)), np.sum(np.exp(sg["lw"] - mx)),
                                       rtol=1e-12)
        if len(o["stages"]) < 3:
            assert o["ess_final"] >= theta
        if rotate and o["stages"]:
            assert st.start == (o["stages"][-1]["k"] + 1) % 3
        if not rotate:
            assert st.start == 0
    if rotate:
        assert len(set(starts)) > 1


def test_digit_set_matrix_is_the_papers_A():
    """With radices (M, 2, ..., 2) the digit set {0, s} has the paper's A_s (eq. (A matrices))."""
    for M, S_ in ((3, 2), (2, 3)):
        radices = (M,) + (2,) * S_
        for s in range(1, S_ + 1):
            np.testing.assert_allclose(butterfly.set_A(radices, s), butterfly.paper_A(S_, M, s), atol=1e-15)


@pytest.mark.parametrize("radices", [(3, 2, 2), (4, 2, 2, 2), (2, 3, 5)])
def test_digit_set_stage_weights_and_support(radices):
    """V_s = A V_{s-1} for the set's matrix, ancestors inside the set group, and after
    all S set stages every weight is equal (Lemma 3(c))."""
    N = int(np.prod(radices))
    model = S.lg_scalar()
    y = S.simulate(model, 3, seed=4)[1]
    st = bpf.init_state(model, N, seed=6)
    for n in range(3):
        new, o = bpf.step_digit_sets(model, radices, 6, st, y[n])
        for sg in o["stages"]:
            A = butterfly.set_A(radices, sg["k"])
            mx = sg["lw"].max()
            np.testing.assert_allclose(np.exp(sg["lV_new"] - mx), A @ np.exp(sg["lw"] - mx), rtol=1e-12)
            gi = butterfly.set_group_index(np.arange(N), radices, sg["k"])
            assert np.array_equal(gi[sg["anc"]], gi)
        np.testing.assert_allclose(new.lV, new.lV[0], atol=1e-12)
        st = new


def test_one_digit_set_is_global_resampling():
    """With two digits the one set {0, 1} is every particle: the step is the one-digit
    step on radices (N,), counters and numbering included."""
    model = S.sv_model()
    y = S.simulate(model, 4, seed=9)[1]
    a = bpf.init_state(model, 48, seed=2)
    b = bpf.init_state(model, 48, seed=2)
    for n in range(4):
        a, oa = bpf.step(model, (48,), 2, a, y[n])
        b, ob = bpf.step_digit_sets(model, (6, 8), 2, b, y[n])
        assert np.array_equal(oa["anc"], ob["stages"][0]["anc"])
        np.testing.assert_allclose(a.x, b.x, rtol=0, atol=0)
        assert oa["inc"] == ob["inc"]
