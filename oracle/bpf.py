"""FP64 bootstrap particle filter with butterfly (mixed-radix) interaction.

Algorithm 1 (particle filter) with its Resample step replaced by ONE stage of
Algorithm 3 (augmented resampling) per time step: at step n the stage matrix
is A_k with k = n mod m (digit k of the mixed-radix particle index), and the
stage weights V carry over to the next step, where they multiply the next
potential g_n.  This is the paper's "rotate the starting stage" idea
(Section 6.4) with the weight recursion V_s = A_s V_{s-1} of eq.
(V_defn_proofs), a reading this library takes for its one-digit-per-step
schedule.  With one digit (radices = (N,)) it is Algorithm 1 + Algorithm 2,
the textbook BPF.

Notation: zeta_n = prediction particles (N x d), lV = log V (carried stage
weights, constant on the groups of the previous digit), g_n = g(., y_n).
All arithmetic is float64 except the integer draw, whose quantisation is
taken in FP32 (see ``resample``).

Carried-weight normalisation (bookkeeping of this library, not in the paper):
the step subtracts a scalar mu_n from every log-weight so lV stays O(1);
mu_{n+1} = log(N^-1 sum_i exp(lw_i)).  The observation density's
state-independent constant c_n (e.g. -1/2 log|2 pi R|) is left out of the
log-weights and added to the likelihood increment only.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Optional, Sequence

import numpy as np

from . import philox, resample
from .butterfly import group_major, set_group_major, strides


@dataclass
class State:
    x: np.ndarray            # (N, d) prediction particles zeta_n
    lV: np.ndarray           # (N,) log carried weights (per particle)
    mu: float                # carried normaliser mu_n
    n: int                   # time index of the next observation
    loglik: float = 0.0      # log p^(y_0..y_{n-1})
    start: int = 0           # fully adapted schedule: digit the next step's stages start at


def obs_terms(model, x: np.ndarray, y: np.ndarray):
    """log g(x, y) split as (state-dependent part s(x) (N,), constant c).

    Linear-Gaussian: g = N(y; Hx, Lr Lr^T)
        s(x) = -1/2 || Lr^{-1} (y - H x) ||^2,  c = -sum log diag(Lr) - dy/2 log(2 pi).
    Stochastic volatility: y = beta exp(x/2) w, w ~ N(0, 1)
        s(x) = -x/2 - y^2 exp(-x) / (2 beta^2),  c = -1/2 log(2 pi beta^2).
    """
    if model.kind == "lg":
        resid = y[None, :] - x @ model.H.T                            # (N, dy)
        z = np.linalg.solve(model.Lr, resid.T).T                      # Lr z = resid
        s = -0.5 * np.sum(z * z, axis=1)
        c = -np.sum(np.log(np.abs(np.diag(model.Lr)))) - 0.5 * model.dy * np.log(2 * np.pi)
        return s, c
    if model.kind == "sv":
        xx = x[:, 0]
        yy = float(y[0])
        s = -0.5 * xx - yy * yy * np.exp(-xx) / (2.0 * model.beta ** 2)
        c = -0.5 * np.log(2 * np.pi * model.beta ** 2)
        return s, c
    raise ValueError(model.kind)


def initial_particles(model, N: int, seed: int) -> np.ndarray:
    """Algorithm 1, first loop: zeta_0^i ~ pi_0 (i.i.d.)."""
    d = model.d
    eps = philox.normals(seed, 0, philox.PURPOSE_INIT, N * d).reshape(N, d)
    if model.kind == "lg":
        return model.m0[None, :] + eps @ model.L0.T
    sd0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)
    return sd0 * eps


def mutate(model, xhat: np.ndarray, n: int, seed: int, idx=None) -> np.ndarray:
    """Algorithm 1, mutation: zeta_{n+1}^i ~ f(zeta_hat_n^i, .).

    ``idx`` (optional) are the counter numbers of the rows of xhat (their normals are
    idx*d + t); by default 0..N-1."""
    N, d = xhat.shape
    if idx is None:
        eps = philox.normals(seed, n, philox.PURPOSE_PROPAGATE, N * d).reshape(N, d)
    else:
        nu = np.asarray(idx, dtype=np.int64)[:, None] * d + np.arange(d)[None, :]
        eps = philox.normals_at(seed, n, philox.PURPOSE_PROPAGATE, nu.reshape(-1)).reshape(N, d)
    if model.kind == "lg":
        return xhat @ model.A.T + eps @ model.Lq.T
    return model.phi * xhat + model.sigma * eps


def init_state(model, N: int, seed: int) -> State:
    return State(x=initial_particles(model, N, seed), lV=np.zeros(N), mu=0.0, n=0)


def _log_mean_exp(v: np.ndarray) -> float:
    m = np.max(v)
    return float(m + np.log(np.mean(np.exp(v - m))))


def weigh(model, x: np.ndarray, lV: np.ndarray, mu_sub: float, y_n: np.ndarray):
    """lw_i = log V_i + log g_n(zeta_i) - c_n - mu  (Algorithm 3, V_0 = g).  Returns (lw, c_n)."""
    s_x, c_n = obs_terms(model, x, np.asarray(y_n, dtype=np.float64))
    lw = lV + s_x - mu_sub
    return np.where(np.isfinite(lw), lw, -np.inf), c_n


def summaries(lw: np.ndarray, x: np.ndarray, c_n: float, mu_sub: float, mu: float):
    """Likelihood increment, weighted filtering mean and ESS (Section 1.2) of weighted particles.

    inc = log(sum_i V_i g_n(zeta_i) / sum_i V_i) with log(N^-1 sum V) = mu; returns
    (inc, mean (d,), ess, lme) with lme = log(N^-1 sum_i exp(lw_i)) the next normaliser."""
    N = len(lw)
    lme = _log_mean_exp(lw)
    inc = lme + c_n + (mu_sub - mu)
    w = np.exp(lw - np.max(lw))
    mean = (w @ x) / np.sum(w)
    ess = float(np.sum(w) ** 2 / (N * np.sum(w * w)))
    return inc, mean, ess, lme


def stage(radices: Sequence[int], seed: int, x: np.ndarray, lw: np.ndarray, k: int, t: int):
    """One stage of Algorithm 3 on digit k with log-weights lw (V_{s-1} g, in logs):
    new stage weights V_s = A_k V_{s-1} (eq. (V_defn_proofs)) and the draws
    xi_s^i ~ (V_s^i)^{-1} sum_j A_k^{ij} V_{s-1}^j delta_{xi_{s-1}^j} (integer rule),
    keyed by the stage counter t.  Returns (x gathered, lV_new, ancestors, q, u, pi)."""
    N = x.shape[0]
    a = radices[k]
    s_k = strides(radices)[k]
    Hh = N // (a * s_k)
    lwg = lw.reshape(Hh, a, s_k)
    Mg = np.max(lwg, axis=1, keepdims=True)
    with np.errstate(invalid="ignore"):
        Lg = Mg + np.log(np.sum(np.exp(lwg - Mg), axis=1, keepdims=True))
    lV_new = np.broadcast_to(Lg - np.log(a), lwg.shape).reshape(N).copy()
    q = resample.quantise(lwg, axis=1)
    Q = np.sum(q, axis=1, keepdims=True, dtype=np.uint64)
    pi = group_major(N, radices, k)            # counter numbering of the draws at this stage
    if a <= resample.NARROW_MAX_RADIX:
        r = philox.resample_words_at(seed, t, pi).reshape(Hh, a, s_k)
        u = resample.scaled_uniform(r, Q, a)
    else:
        lo, hi = philox.resample_words_wide_at(seed, t, pi)
        u = resample.scaled_uniform(lo.reshape(Hh, a, s_k), Q, a, hi.reshape(Hh, a, s_k))
    member = resample.draw(q, u, axis=1)
    h_idx = np.arange(Hh)[:, None, None]
    l_idx = np.arange(s_k)[None, None, :]
    anc = (h_idx * (a * s_k) + member * s_k + l_idx).reshape(N)
    return x[anc], lV_new, anc, q.reshape(N), u.reshape(N), pi


def stage_set(radices: Sequence[int], seed: int, x: np.ndarray, lw: np.ndarray, k: int, t: int):
    """One stage of Algorithm 3 whose matrix is the digit set {0, k} (k >= 1): the
    group of i is every index sharing all digits but 0 and k (a_0 a_k members, digit
    k major, digit 0 minor), V_s = A V_{s-1} with A = set_A(radices, k) and the draws
    by the integer rule, words keyed by the stage counter t and numbered group by
    group (set_group_major).  With radices (M, 2, ..., 2) this is eq. (A matrices)."""
    N = x.shape[0]
    a0, a = radices[0], radices[k]
    s_k = strides(radices)[k]
    Hh = N // (a * s_k)
    L = s_k // a0
    G = a * a0
    # (H, a_k, L, a_0) -> (H, L, a_k, a_0) -> groups (H L) x members (a_k a_0)
    lwg = lw.reshape(Hh, a, L, a0).transpose(0, 2, 1, 3).reshape(Hh * L, G)
    Mg = np.max(lwg, axis=1, keepdims=True)
    with np.errstate(invalid="ignore"):
        Lg = Mg + np.log(np.sum(np.exp(lwg - Mg), axis=1, keepdims=True))
    q = resample.quantise(lwg, axis=1)
    Q = np.sum(q, axis=1, keepdims=True, dtype=np.uint64)
    pi = set_group_major(N, radices, k)
    # members' words in group order: member rho of group g is particle with pi = g G + rho
    order = np.argsort(pi)                     # order[g G + rho] = particle index
    if G <= resample.NARROW_MAX_RADIX:
        r = philox.resample_words_at(seed, t, np.arange(N)).reshape(Hh * L, G)
        u = resample.scaled_uniform(r, Q, G)
    else:
        lo, hi = philox.resample_words_wide_at(seed, t, np.arange(N))
        u = resample.scaled_uniform(lo.reshape(Hh * L, G), Q, G, hi.reshape(Hh * L, G))
    member = resample.draw(q, u, axis=1)       # (groups, G) member drawn by member rho
    ranks = np.arange(Hh * L)[:, None] * G
    anc_sorted = order[ranks + member]         # ancestor particle of the draw with number g G + rho
    anc = np.empty(N, dtype=np.int64)
    anc[order] = anc_sorted.reshape(N)
    lV_new = np.empty(N)
    lV_new[order] = np.broadcast_to(Lg - np.log(G), lwg.shape).reshape(N)
    q_p = np.empty(N, dtype=np.uint64)
    u_p = np.empty(N, dtype=np.uint64)
    q_p[order] = q.reshape(N)
    u_p[order] = u.reshape(N)
    return x[anc], lV_new, anc, q_p, u_p, pi


def step_digit_sets(model, radices: Sequence[int], seed: int, st: State, y_n: np.ndarray,
                    mu_used: Optional[float] = None) -> (State, Dict[str, np.ndarray]):
    """One time step of Algorithm 1 with Algorithm 3 exactly as the paper defines its
    stages (eq. (A matrices)): radices (a_0, a_1, ..., a_S), stage s = 1..S on the digit
    set {0, s} (the within-PE digit and PE bit s-1 when radices = (M, 2, ..., 2)).
    g_n weights stage 1, stage S mutates (normals numbered group by group on the set
    {0, S}); stage s draws with counter t = n S + s - 1.  Afterwards every weight is
    equal (Lemma 3(c))."""
    radices = [int(a) for a in radices]
    S_ = len(radices) - 1
    if S_ < 1:
        raise ValueError("digit sets need at least two digits")
    n = st.n
    mu_sub = st.mu if mu_used is None else float(mu_used)
    lw, c_n = weigh(model, st.x, st.lV, mu_sub, y_n)
    inc, mean, ess, lme = summaries(lw, st.x, c_n, mu_sub, st.mu)
    x = st.x
    stages = []
    for s in range(1, S_ + 1):
        x, lV_new, anc, q, u, pi = stage_set(radices, seed, x, lw, s, n * S_ + s - 1)
        stages.append(dict(k=s, anc=anc, q=q, u=u, lw=lw, lV_new=lV_new))
        lw = lV_new
    x_next = mutate(model, x, n, seed, idx=pi)
    new = State(x=x_next, lV=lw, mu=lme, n=n + 1, loglik=st.loglik + inc)
    return new, dict(stages=stages, inc=inc, mean=mean, ess=ess, lV_new=lw, c=c_n)


def step_all_stages(model, radices: Sequence[int], seed: int, st: State, y_n: np.ndarray,
                    mu_used: Optional[float] = None) -> (State, Dict[str, np.ndarray]):
    """One time step with the paper's schedule: Algorithm 1 whose Resample is the
    whole of Algorithm 3 - g_n weights stage 1 (V_0 = g), then all S = m stages
    s = 1..S on digits 0..m-1 in turn, then the mutation (Section 3).  Stage s of
    time step n draws with counter t = n m + s - 1; the mutation uses time n.
    By Lemma 3(c) the weights after the last stage are all equal."""
    radices = [int(a) for a in radices]
    m = len(radices)
    n = st.n
    mu_sub = st.mu if mu_used is None else float(mu_used)
    lw, c_n = weigh(model, st.x, st.lV, mu_sub, y_n)
    inc, mean, ess, lme = summaries(lw, st.x, c_n, mu_sub, st.mu)
    x = st.x
    stages = []
    for k in range(m):
        x, lV_new, anc, q, u, pi = stage(radices, seed, x, lw, k, n * m + k)
        stages.append(dict(k=k, anc=anc, q=q, u=u, lw=lw, lV_new=lV_new))
        lw = lV_new
    # the mutation's normals are numbered like the draws of the stage that mutates
    # (group-major on digit m-1), as in the one-digit step
    x_next = mutate(model, x, n, seed, idx=pi)
    new = State(x=x_next, lV=lw, mu=lme, n=n + 1, loglik=st.loglik + inc)
    return new, dict(stages=stages, inc=inc, mean=mean, ess=ess, lV_new=lw, c=c_n)


def ess_of(lv: np.ndarray) -> float:
    """Effective sample size (Section 1.2) of the weights exp(lv): (sum w)^2 / (N sum w^2)."""
    w = np.exp(lv - np.max(lv))
    return float(np.sum(w) ** 2 / (len(lv) * np.sum(w * w)))


def step_adaptive(model, radices: Sequence[int], seed: int, st: State, y_n: np.ndarray, theta: float,
                  rotate: bool = False, mu_used: Optional[float] = None) -> (State, Dict[str, np.ndarray]):
    """One time step with fully adapted augmented resampling (Section 1.2): weight
    with g_n, then run the stages of Algorithm 3 one after another, evaluating the
    ESS of the current weights before each stage and skipping the remaining
    stages once it reaches theta; then mutate.  Weights that were not equalised
    carry over to the next step (per particle).

    Launch j = 0..m-1 of step n works on digit k = (start + j) mod m and draws with
    stage counter t = n m + j; start = 0 unless ``rotate``, in which case the next
    step starts one digit after the last stage executed (Section 6.4's proposal),
    and stays put after a step without resampling.  The mutation's normals are
    numbered group-major on the digit of launch m-1, as in the other schedules.
    theta > 1 runs every stage (the all-stages step); theta <= 1/N runs none
    (sequential importance sampling)."""
    radices = [int(a) for a in radices]
    m = len(radices)
    n = st.n
    N = st.x.shape[0]
    mu_sub = st.mu if mu_used is None else float(mu_used)
    lw, c_n = weigh(model, st.x, st.lV, mu_sub, y_n)
    inc, mean, ess, lme = summaries(lw, st.x, c_n, mu_sub, st.mu)
    x = st.x
    cur = lw
    e = ess
    stages = []
    for j in range(m):
        if e >= theta:
            break
        k = (st.start + j) % m
        x, lV_new, anc, q, u, pi = stage(radices, seed, x, cur, k, n * m + j)
        stages.append(dict(k=k, j=j, anc=anc, q=q, u=u, lw=cur, lV_new=lV_new, ess_before=e))
        cur = lV_new
        e = ess_of(cur)
    k_last = (st.start + m - 1) % m
    x_next = mutate(model, x, n, seed, idx=group_major(N, radices, k_last))
    start = st.start
    if rotate and stages:
        start = (stages[-1]["k"] + 1) % m
    new = State(x=x_next, lV=cur, mu=lme, n=n + 1, loglik=st.loglik + inc, start=start)
    return new, dict(stages=stages, inc=inc, mean=mean, ess=ess, ess_final=e, lV_new=cur, c=c_n)


def island_stages(lW: np.ndarray, seed: int, n: int, modified: bool = True, theta: Optional[float] = None):
    """Augmented island resampling (Algorithm 6; Algorithm 7 when ``modified``) on the
    log island weights lW (m = 2^S islands).  Stage s = 1..S pairs island i with
    i xor 2^(s-1) (matrices bold-A_s); both members of a pair get the pair's mean
    weight, and each island draws, by the integer rule on the pair's two weights
    with its own uniform (island_words_at(seed, n, s, i)), the island whose whole
    sample it holds next.  Algorithm 7 undoes a draw in which the two islands
    would merely swap their samples.  With ``theta`` (fully adapted, Section 1.2)
    the ESS of the island weights is evaluated before every stage and the
    remaining stages are skipped once it reaches theta.  Returns (holder,
    lW_final, per-stage info): holder[i] = the island whose input sample island
    i ends up holding."""
    m = len(lW)
    S = int(np.log2(m))
    if 1 << S != m:
        raise ValueError("the number of islands must be a power of two")
    V = np.asarray(lW, dtype=np.float64).copy()
    holder = np.arange(m)
    info = []
    for s in range(1, S + 1):
        if theta is not None and ess_of(V) >= theta:
            break
        b = 1 << (s - 1)
        H = m // (2 * b)
        Vr = V.reshape(H, 2, b)
        q = resample.quantise(Vr, axis=1)
        Q = np.sum(q, axis=1, keepdims=True, dtype=np.uint64)
        u = resample.scaled_uniform(philox.island_words_at(seed, n, s, np.arange(m)).reshape(H, 2, b), Q, 2)
        member = resample.draw(q, u, axis=1)
        member = np.where(Q == 0, np.arange(2)[None, :, None], member)   # an all-zero pair keeps its samples
        swapped = np.zeros((H, 1, b), dtype=bool)
        if modified:
            swapped = ((member[:, 0, :] == 1) & (member[:, 1, :] == 0))[:, None, :]
            member = np.where(swapped, np.arange(2)[None, :, None], member)
        h_idx = np.arange(H)[:, None, None]
        l_idx = np.arange(b)[None, None, :]
        c = (h_idx * 2 * b + member * b + l_idx).reshape(m)
        Mx = np.max(Vr, axis=1, keepdims=True)
        with np.errstate(invalid="ignore", divide="ignore"):
            Lp = Mx + np.log(np.sum(np.exp(Vr - Mx), axis=1, keepdims=True)) - np.log(2.0)
        V = np.broadcast_to(Lp, Vr.shape).reshape(m).copy()
        holder = holder[c]
        info.append(dict(s=s, q=q.reshape(m), u=u.reshape(m), choice=c, swaps_undone=int(np.sum(swapped)),
                         ess_before=ess_of(Vr.reshape(m))))
    return holder, V, info


def step_islands(model, M: int, m: int, seed: int, st: State, y_n: np.ndarray, modified: bool = True,
                 mu_used: Optional[float] = None, theta: Optional[float] = None) -> (State, Dict[str, np.ndarray]):
    """One time step of AIRPF (Algorithm 4): N = M m particles in m islands of M
    consecutive particles.  Weight with g_n; within-island multinomial resampling
    (Algorithm 5: the stage on digit 0 of radices (M, m), island weight = mean g of
    the island, eq. (out weight)), drawn with stage counter t = 2n; augmented island
    resampling (Algorithm 6 / 7) over S = log2 m stages; every particle of island i
    takes the particle at the same place in the sample island i holds; mutation
    (normals numbered by the particle index).  Afterwards all weights are equal,
    unless ``theta`` (AIRPF2: fully adapted island stages) stopped the island
    stages early, in which case every particle carries its island's weight."""
    N = M * m
    radices = (M, m)
    n = st.n
    mu_sub = st.mu if mu_used is None else float(mu_used)
    lw, c_n = weigh(model, st.x, st.lV, mu_sub, y_n)
    inc, mean, ess, lme = summaries(lw, st.x, c_n, mu_sub, st.mu)
    x1, lV1, anc1, q1, u1, _ = stage(radices, seed, st.x, lw, 0, 2 * n)
    lW = lV1[::M]
    holder, V, info = island_stages(lW, seed, n, modified, theta)
    src = (holder[np.arange(N) // M] * M + np.arange(N) % M)
    x_hat = x1[src]
    x_next = mutate(model, x_hat, n, seed, idx=np.arange(N))
    new = State(x=x_next, lV=V[np.arange(N) // M], mu=lme, n=n + 1, loglik=st.loglik + inc)
    return new, dict(inc=inc, mean=mean, ess=ess, within=dict(anc=anc1, q=q1, u=u1, lV=lV1), holder=holder,
                     island_info=info, lW=lW, lW_final=V, x_within=x1, c=c_n)


def step(model, radices: Sequence[int], seed: int, st: State, y_n: np.ndarray,
         mu_used: Optional[float] = None) -> (State, Dict[str, np.ndarray]):
    """One time step n = st.n: weight, one augmented-resampling stage, mutate.

    ``mu_used`` (lockstep parity only) is the normaliser the caller's filter
    actually subtracted; the likelihood increment corrects for it.
    """
    radices = [int(a) for a in radices]
    N, d = st.x.shape
    m = len(radices)
    n = st.n
    k = n % m
    a = radices[k]
    s_k = strides(radices)[k]
    Hh = N // (a * s_k)
    mu_sub = st.mu if mu_used is None else float(mu_used)

    # V_{s-1}^j g_n(zeta^j), in logs: lw_j = log V_j + s(zeta_j) - mu    (Algorithm 3, V_0 = g)
    lw, c_n = weigh(model, st.x, st.lV, mu_sub, y_n)

    # Group view (h, r, l): digit k is the middle axis.
    lwg = lw.reshape(Hh, a, s_k)
    # V_s^i = sum_j A^{ij} V_{s-1}^j = (1/a) sum_{j in G(i)} V_{s-1}^j   (eq. V_defn_proofs)
    Mg = np.max(lwg, axis=1, keepdims=True)
    Lg = Mg + np.log(np.sum(np.exp(lwg - Mg), axis=1, keepdims=True))
    lV_new = np.broadcast_to(Lg - np.log(a), lwg.shape).reshape(N).copy()

    # xi_s^i ~ (V_s^i)^{-1} sum_j A^{ij} V_{s-1}^j delta_{xi_{s-1}^j}   (integer rule)
    q = resample.quantise(lwg, axis=1)
    Q = np.sum(q, axis=1, keepdims=True, dtype=np.uint64)
    pi = group_major(N, radices, k)            # counter numbering of the draws at this step
    if a <= resample.NARROW_MAX_RADIX:
        r = philox.resample_words_at(seed, n, pi).reshape(Hh, a, s_k)
        u = resample.scaled_uniform(r, Q, a)
    else:
        lo, hi = philox.resample_words_wide_at(seed, n, pi)
        u = resample.scaled_uniform(lo.reshape(Hh, a, s_k), Q, a, hi.reshape(Hh, a, s_k))
    member = resample.draw(q, u, axis=1)                                  # (Hh, a, s_k)
    h_idx = np.arange(Hh)[:, None, None]
    l_idx = np.arange(s_k)[None, None, :]
    anc = (h_idx * (a * s_k) + member * s_k + l_idx).reshape(N)

    # Likelihood increment, filter mean and ESS (Section 1.2) from the weighted particles.
    inc, mean, ess, lme = summaries(lw, st.x, c_n, mu_sub, st.mu)

    x_next = mutate(model, st.x[anc], n, seed, idx=pi)
    new = State(x=x_next, lV=lV_new, mu=lme, n=n + 1, loglik=st.loglik + inc)
    out = dict(k=k, a=a, stride=s_k, anc=anc, lw=lw, q=q.reshape(N), u=u.reshape(N),
               Q=np.broadcast_to(Q, q.shape).reshape(N), inc=inc, mean=mean, ess=ess,
               lV_new=lV_new, c=c_n)
    return new, out


def run(model, N: int, radices: Sequence[int], seed: int, y: np.ndarray,
        keep_ancestors: bool = False, all_stages: bool = False, theta: Optional[float] = None,
        rotate: bool = False, islands: Optional[str] = None) -> Dict[str, np.ndarray]:
    """Run the filter over y[0:T].  Returns per-step inc, mean, ess and the final loglik.
    all_stages: the paper's schedule (all m stages per time step) instead of one digit;
    theta: fully adapted resampling with ESS threshold theta (optionally rotated)."""
    if int(np.prod(radices)) != N:
        raise ValueError("product of radices must equal N")
    y = np.asarray(y, dtype=np.float64).reshape(len(y), -1)
    T = y.shape[0]
    st = init_state(model, N, seed)
    incs = np.empty(T)
    means = np.empty((T, model.d))
    ess = np.empty(T)
    ancs = [] if keep_ancestors else None
    executed = 0
    for t in range(T):
        if all_stages == "sets":     # Algorithm 3 with eq. (A matrices): digit sets {0, s}
            st, o = step_digit_sets(model, radices, seed, st, y[t])
        elif islands is not None:    # "modified" (Algorithm 7) or "plain" (Algorithm 6); radices = (M, m)
            st, o = step_islands(model, radices[0], radices[1], seed, st, y[t], islands == "modified",
                                 theta=theta)
            executed += len(o["island_info"])
        elif theta is not None:
            st, o = step_adaptive(model, radices, seed, st, y[t], theta, rotate)
            executed += len(o["stages"])
        else:
            st, o = (step_all_stages if all_stages else step)(model, radices, seed, st, y[t])
        incs[t], means[t], ess[t] = o["inc"], o["mean"], o["ess"]
        if keep_ancestors and not all_stages and theta is None and islands is None:
            ancs.append(o["anc"])
    out = dict(inc=incs, mean=means, ess=ess, loglik=st.loglik, state=st, stages_executed=executed)
    if keep_ancestors:
        out["anc"] = np.stack(ancs)
    return out


def step_on_groups(model, radices: Sequence[int], seed: int, n: int, x: np.ndarray, lV: np.ndarray,
                   mu_used: float, y_n: np.ndarray, groups: np.ndarray) -> Dict[str, np.ndarray]:
    """Step n (weight, one stage on digit k = n mod m, mutate) restricted to some groups.

    Used to check full-size runs one group at a time.  x: (N, d) prediction
    particles; lV: (N,) carried log weights; groups: (G, 2) array of (h, l), the
    digits above and below k that name a group.  Returns per-member arrays of
    shape (G, a): global index, lw, q, u, ancestor (global), and x_next (G, a, d),
    lV_new (G,).
    """
    radices = [int(a) for a in radices]
    m = len(radices)
    k = n % m
    a = radices[k]
    s_k = strides(radices)[k]
    d = x.shape[1]
    groups = np.asarray(groups, dtype=np.int64)
    idx = groups[:, :1] * (a * s_k) + np.arange(a)[None, :] * s_k + groups[:, 1:2]   # (G, a)
    flat = idx.reshape(-1)
    lw, _ = weigh(model, x[flat].astype(np.float64), lV[flat].astype(np.float64), mu_used, y_n)
    lw = lw.reshape(idx.shape)
    Mg = np.max(lw, axis=1, keepdims=True)
    Lg = Mg + np.log(np.sum(np.exp(lw - Mg), axis=1, keepdims=True))
    q = resample.quantise(lw, axis=1)
    Q = np.sum(q, axis=1, keepdims=True, dtype=np.uint64)
    pi = ((groups[:, :1] * s_k + groups[:, 1:2]) * a + np.arange(a)[None, :]).reshape(-1)
    if a <= resample.NARROW_MAX_RADIX:
        u = resample.scaled_uniform(philox.resample_words_at(seed, n, pi).reshape(idx.shape), Q, a)
    else:
        lo, hi = philox.resample_words_wide_at(seed, n, pi)
        u = resample.scaled_uniform(lo.reshape(idx.shape), Q, a, hi.reshape(idx.shape))
    member = resample.draw(q, u, axis=1)
    anc = groups[:, :1] * (a * s_k) + member * s_k + groups[:, 1:2]
    x_next = mutate(model, x[anc.reshape(-1)].astype(np.float64), n, seed, idx=pi).reshape(idx.shape + (d,))
    return dict(idx=idx, lw=lw, q=q, u=u, Q=np.broadcast_to(Q, q.shape), anc=anc, x_next=x_next,
                lV_new=(Lg - np.log(a))[:, 0])
