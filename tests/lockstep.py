"""Lockstep parity: the FP64 oracle re-runs each GPU time step from the GPU's own
state and checks every output of that step.

Ancestors are integers decided by floating-point weights.  Both sides take the
decision with the same integer rule and FP32 quantisation, but their weights
differ by FP32-versus-FP64 rounding, so a draw that lands within a few quanta
of a prefix-sum boundary may legitimately go either way.  If every integer
weight differs between the sides by at most a relative ETA (plus one quantum
from the floor), a boundary P_j moves, relative to Q, by at most
2 ETA min(P_j, Q - P_j) + a + 2 quanta, and the uniform u = floor(r Q / 2^32)
by one more.  A draw is *decidable* when every boundary lies farther than

    margin_j = 2 * ETA * min(P_j, Q - P_j) + a + 4

from its uniform.  Decidable draws must match bit for bit; every GPU ancestor
must lie among the oracle's plausible members.  States and log-weights must
agree to 1e-5 (relative, floor 1), likelihood increments to 1e-6.
"""
from __future__ import annotations

import numpy as np

from oracle import bpf, butterfly

ETA = 2.0 ** -15
TOL_STATE = 1e-5
TOL_INC = 1e-6


def plausible_members(q: np.ndarray, u: np.ndarray, axis: int):
    """(lo, hi) member indices an ancestor draw may take given boundary uncertainty."""
    P = np.cumsum(q, axis=axis, dtype=np.uint64).astype(np.float64)
    Q = np.take(P, [-1], axis=axis)
    a = q.shape[axis]
    margin = 2 * ETA * np.minimum(P, Q - P) + a + 4
    if a > 64:   # P +- margin are non-decreasing along the group: binary searches
        Pm = np.moveaxis(P, axis, -1).reshape(-1, a)
        Mm = np.moveaxis(margin, axis, -1).reshape(-1, a)
        um = np.moveaxis(u.astype(np.float64), axis, -1).reshape(-1, a)
        lo = np.empty(um.shape, dtype=np.int64)
        hi = np.empty(um.shape, dtype=np.int64)
        for g in range(Pm.shape[0]):
            lo[g] = np.searchsorted(Pm[g] + Mm[g], um[g], side="right")
            hi[g] = np.minimum(np.searchsorted(Pm[g] - Mm[g], um[g], side="right"), a - 1)
        shape = np.moveaxis(u, axis, -1).shape
        return np.moveaxis(lo.reshape(shape), -1, axis), np.moveaxis(hi.reshape(shape), -1, axis)
    Pm = np.moveaxis(P, axis, -1)
    um = np.moveaxis(u.astype(np.float64), axis, -1)
    mg = np.moveaxis(margin, axis, -1)
    lo = (Pm[..., None, :] + mg[..., None, :] <= um[..., :, None]).sum(-1)
    hi = np.minimum((Pm[..., None, :] - mg[..., None, :] <= um[..., :, None]).sum(-1), a - 1)
    return np.moveaxis(lo, -1, axis), np.moveaxis(hi, -1, axis)


def rel_err(a, b, floor=1.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    fin = np.isfinite(b)
    if not np.array_equal(np.isfinite(a), fin):
        return np.inf
    if not fin.any():
        return 0.0
    return float(np.max(np.abs(a[fin] - b[fin]) / np.maximum(np.abs(b[fin]), floor)))


def per_particle_lV(lv_compact, radices, n):
    """Expand the GPU's compact carried weights (groups of digit (n-1) mod m) to particles."""
    N = int(np.prod(radices))
    kp = (n - 1) % len(radices)
    return lv_compact[butterfly.group_index(np.arange(N), radices, kp)]


class Report(dict):
    def merge(self, other):
        for k, v in other.items():
            if k.startswith("max_"):
                self[k] = max(self.get(k, 0.0), v)
            else:
                self[k] = self.get(k, 0) + v


def check_step_full(filt, model, radices, seed, y_n, n):
    """Run GPU step n and check it against the oracle's step from the same state."""
    N = int(np.prod(radices))
    m = len(radices)
    x0, lv0, sc = filt.state()
    assert sc["n"] == n
    mean, inc, ess = filt.step(y_n)
    anc = filt.ancestors().astype(np.int64)
    x1, lv1, sc1 = filt.state()
    lV = per_particle_lV(lv0, radices, n).astype(np.float64)
    st = bpf.State(x=x0.astype(np.float64), lV=lV, mu=sc["mu"], n=n)
    new, o = bpf.step(model, radices, seed, st, y_n, mu_used=sc["mu_used"])
    k, a, s = o["k"], o["a"], o["stride"]
    H = N // (a * s)
    # ancestors
    q = o["q"].reshape(H, a, s)
    u = o["u"].reshape(H, a, s)
    lo, hi = plausible_members(q, u, axis=1)
    member_gpu = ((anc // s) % a).reshape(H, a, s)
    same_group = np.array_equal(anc // (a * s), np.arange(N) // (a * s)) and \
        np.array_equal(anc % s, np.arange(N) % s)
    assert same_group, "GPU ancestor outside its group"
    dec = (lo == hi)
    member_o = (o["anc"].reshape(H, a, s) // s) % a
    mism = member_gpu != member_o
    assert not np.any(mism & dec), f"step {n}: {int(np.sum(mism & dec))} decidable ancestors differ"
    assert np.all((member_gpu >= lo) & (member_gpu <= hi)), f"step {n}: implausible ancestor"
    # offspring counts sum to a in every group
    grp = (anc // (a * s)) * s + anc % s
    assert np.all(np.bincount(grp, minlength=N // a) == a)
    # states: oracle mutation of the GPU's own ancestors
    x_chk = bpf.mutate(model, x0.astype(np.float64)[anc], n, seed, idx=butterfly.group_major(N, radices, k))
    e_x = rel_err(x1, x_chk)
    lv_chk = o["lV_new"].reshape(H, a, s)[:, 0, :].reshape(-1)
    e_lv = rel_err(lv1, lv_chk)
    e_inc = abs(inc - o["inc"]) / max(1.0, abs(o["inc"]))
    e_mean = rel_err(mean, o["mean"])
    e_ess = abs(ess - o["ess"]) / max(o["ess"], 1e-12)
    assert e_x <= TOL_STATE, f"step {n}: state error {e_x}"
    assert e_lv <= TOL_STATE, f"step {n}: log-weight error {e_lv}"
    assert e_inc <= TOL_INC, f"step {n}: likelihood increment error {e_inc}"
    assert e_mean <= TOL_STATE, f"step {n}: mean error {e_mean}"
    assert e_ess <= 1e-4, f"step {n}: ess error {e_ess}"
    assert abs(sc1["mu"] - new.mu) <= 1e-6 * max(1.0, abs(new.mu))
    return Report(draws=N, undecidable=int(np.sum(~dec)), mismatched_undecidable=int(np.sum(mism)),
                  max_state_err=e_x, max_logweight_err=e_lv, max_inc_err=e_inc, max_mean_err=e_mean,
                  max_ess_err=e_ess)


def check_step_sampled(filt, model, radices, seed, y_n, n, n_groups, rng):
    """Run GPU step n at full size and check sampled groups (ancestors, states,
    log-weights) and the global outputs (increment, mean, ESS) against the oracle."""
    N = int(np.prod(radices))
    m = len(radices)
    k = n % m
    a = int(radices[k])
    s = butterfly.strides(radices)[k]
    H = N // (a * s)
    x0, lv0, sc = filt.state()
    mean, inc, ess = filt.step(y_n)
    anc = filt.ancestors().astype(np.int64)
    x1, lv1, _ = filt.state()
    lV = per_particle_lV(lv0, radices, n)
    # global outputs from the whole GPU state
    lw, c_n = bpf.weigh(model, x0.astype(np.float64), lV.astype(np.float64), sc["mu_used"], y_n)
    inc_o, mean_o, ess_o, _ = bpf.summaries(lw, x0.astype(np.float64), c_n, sc["mu_used"], sc["mu"])
    e_inc = abs(inc - inc_o) / max(1.0, abs(inc_o))
    e_mean = rel_err(mean, mean_o)
    e_ess = abs(ess - ess_o) / max(ess_o, 1e-12)
    assert e_inc <= TOL_INC, f"step {n}: likelihood increment error {e_inc}"
    assert e_mean <= TOL_STATE, f"step {n}: mean error {e_mean}"
    assert e_ess <= 1e-4, f"step {n}: ess error {e_ess}"
    gid = rng.choice(H * s, size=min(n_groups, H * s), replace=False)
    groups = np.stack([gid // s, gid % s], axis=1)
    o = bpf.step_on_groups(model, radices, seed, n, x0, lV, sc["mu_used"], y_n, groups)
    idx = o["idx"]
    lo, hi = plausible_members(o["q"], o["u"], axis=1)
    member_gpu = (anc[idx] // s) % a
    member_o = (o["anc"] // s) % a
    dec = lo == hi
    assert np.all(anc[idx] // (a * s) == idx // (a * s)) and np.all(anc[idx] % s == idx % s)
    assert not np.any((member_gpu != member_o) & dec), f"step {n}: decidable ancestors differ"
    assert np.all((member_gpu >= lo) & (member_gpu <= hi))
    pi = ((groups[:, :1] * s + groups[:, 1:2]) * a + np.arange(a)[None, :]).reshape(-1)
    x_chk = bpf.mutate(model, x0[anc[idx].reshape(-1)].astype(np.float64), n, seed,
                       idx=pi).reshape(idx.shape + (x0.shape[1],))
    e_x = rel_err(x1[idx], x_chk)
    e_lv = rel_err(lv1[groups[:, 0] * s + groups[:, 1]], o["lV_new"])
    assert e_x <= TOL_STATE, f"step {n}: state error {e_x}"
    assert e_lv <= TOL_STATE, f"step {n}: log-weight error {e_lv}"
    return Report(draws=int(idx.size), undecidable=int(np.sum(~dec)),
                  mismatched_undecidable=int(np.sum(member_gpu != member_o)),
                  max_state_err=e_x, max_logweight_err=e_lv, max_inc_err=e_inc, max_mean_err=e_mean,
                  max_ess_err=e_ess)


def check_step_all_stages(filt, model, radices, seed, y_n, n):
    """GPU time step n with every stage of Algorithm 3 (PF_ALL_STAGES) against the
    oracle's all-stages step from the same state.

    After the first stage the stage weights are group sums of the previous
    stage's weights, independent of which particles were drawn, so the integer
    weights and uniforms of every stage are comparable between the sides.  A
    particle's final state must match the oracle's when every draw on its line
    of ancestry (one per stage) is decidable; increment, mean, ESS and the new
    carried weights (all equal, Lemma 3(c)) must match always."""
    N = int(np.prod(radices))
    m = len(radices)
    x0, lv0, sc = filt.state()
    assert sc["n"] == n
    mean, inc, ess = filt.step(y_n)
    x1, lv1, sc1 = filt.state()
    lV = per_particle_lV(lv0, radices, n * m).astype(np.float64)
    st = bpf.State(x=x0.astype(np.float64), lV=lV, mu=sc["mu"], n=n)
    new, o = bpf.step_all_stages(model, radices, seed, st, y_n, mu_used=sc["mu_used"])
    strides = butterfly.strides(radices)
    line = None
    undecidable = 0
    for sg in o["stages"]:
        k = sg["k"]
        a, s = int(radices[k]), strides[k]
        H = N // (a * s)
        lo, hi = plausible_members(sg["q"].reshape(H, a, s), sg["u"].reshape(H, a, s), axis=1)
        dec = (lo == hi).reshape(N)
        undecidable += int(np.sum(~dec))
        line = dec if line is None else dec & line[sg["anc"]]
    e_x = rel_err(x1[line], new.x[line])
    e_lv = rel_err(lv1, np.full(lv1.shape, new.lV[0]))
    e_inc = abs(inc - o["inc"]) / max(1.0, abs(o["inc"]))
    e_mean = rel_err(mean, o["mean"])
    e_ess = abs(ess - o["ess"]) / max(o["ess"], 1e-12)
    assert e_x <= TOL_STATE, f"step {n}: state error {e_x}"
    assert e_lv <= TOL_STATE, f"step {n}: log-weight error {e_lv}"
    assert e_inc <= TOL_INC, f"step {n}: likelihood increment error {e_inc}"
    assert e_mean <= TOL_STATE, f"step {n}: mean error {e_mean}"
    assert e_ess <= 1e-4, f"step {n}: ess error {e_ess}"
    assert abs(sc1["mu"] - new.mu) <= 1e-6 * max(1.0, abs(new.mu))
    return Report(draws=N * m, undecidable=undecidable, undecided_lines=int(np.sum(~line)),
                  max_state_err=e_x, max_logweight_err=e_lv, max_inc_err=e_inc, max_mean_err=e_mean,
                  max_ess_err=e_ess)


def check_step_adaptive(filt, model, radices, seed, y_n, n, theta, rotate, start):
    """GPU time step n with fully adapted resampling (PF_ADAPTIVE) against the
    oracle's adaptive step from the same state (per-particle carried weights).

    Checks the summaries, the number of stages the ESS test let run, the new
    per-particle log-weights and the states on fully decidable lines of
    ancestry.  An ESS within 1e-5 (relative) of theta makes the run/skip
    decision a rounding question; such a step is reported as ambiguous and its
    stage decisions are not compared.  Returns (Report, oracle's next start)."""
    N = int(np.prod(radices))
    x0, lv0, sc = filt.state()
    assert sc["n"] == n and lv0.shape == (N,)
    c0 = filt.stage_count()
    mean, inc, ess = filt.step(y_n)
    x1, lv1, sc1 = filt.state()
    c1 = filt.stage_count()
    st = bpf.State(x=x0.astype(np.float64), lV=lv0.astype(np.float64), mu=sc["mu"], n=n, start=start)
    new, o = bpf.step_adaptive(model, radices, seed, st, y_n, theta, rotate, mu_used=sc["mu_used"])
    e_inc = abs(inc - o["inc"]) / max(1.0, abs(o["inc"]))
    e_mean = rel_err(mean, o["mean"])
    e_ess = abs(ess - o["ess"]) / max(o["ess"], 1e-12)
    assert e_inc <= TOL_INC, f"step {n}: likelihood increment error {e_inc}"
    assert e_mean <= TOL_STATE, f"step {n}: mean error {e_mean}"
    assert e_ess <= 1e-4, f"step {n}: ess error {e_ess}"
    tested = [o["ess"]] + [bpf.ess_of(sg["lV_new"]) for sg in o["stages"]]
    if any(abs(e - theta) <= 1e-5 * theta for e in tested):
        return Report(ambiguous_steps=1), None
    assert c1 - c0 == len(o["stages"]), f"step {n}: GPU ran {c1 - c0} stages, oracle {len(o['stages'])}"
    strides = butterfly.strides(radices)
    line = np.ones(N, dtype=bool)
    undecidable = 0
    for sg in o["stages"]:
        k = sg["k"]
        a, s = int(radices[k]), strides[k]
        H = N // (a * s)
        lo, hi = plausible_members(sg["q"].reshape(H, a, s), sg["u"].reshape(H, a, s), axis=1)
        dec = (lo == hi).reshape(N)
        undecidable += int(np.sum(~dec))
        line = dec & line[sg["anc"]]
    e_x = rel_err(x1[line], new.x[line])
    e_lv = rel_err(lv1, o["lV_new"])
    assert e_x <= TOL_STATE, f"step {n}: state error {e_x}"
    assert e_lv <= TOL_STATE, f"step {n}: log-weight error {e_lv}"
    assert abs(sc1["mu"] - new.mu) <= 1e-6 * max(1.0, abs(new.mu))
    return Report(draws=N * len(o["stages"]), stages=len(o["stages"]), undecidable=undecidable,
                  undecided_lines=int(np.sum(~line)), max_state_err=e_x, max_logweight_err=e_lv,
                  max_inc_err=e_inc, max_mean_err=e_mean, max_ess_err=e_ess), new.start


def check_step_islands(filt, model, M, m, seed, y_n, n, modified, theta=None):
    """GPU AIRPF step n (PF_ISLANDS) against the oracle's AIRPF step from the same
    state.  A particle's new state must match when its within-island draw and
    every island-stage draw on its island's line of holders is decidable (with
    Algorithm 7 an island's choice also depends on its partner's draw).  With
    ``theta`` (AIRPF2) the number of island stages run must match too, unless an
    ESS lies within 1e-5 of theta (then the step is reported as ambiguous)."""
    N = M * m
    x0, lv0, sc = filt.state()
    assert sc["n"] == n
    c0 = filt.stage_count() if theta is not None else 0
    mean, inc, ess = filt.step(y_n)
    x1, lv1, sc1 = filt.state()
    if theta is not None:       # one carried weight per island
        lV = lv0[np.arange(N) // M].astype(np.float64)
    else:
        lV = per_particle_lV(lv0, (M, m), 2 * n).astype(np.float64)
    st = bpf.State(x=x0.astype(np.float64), lV=lV, mu=sc["mu"], n=n)
    new, o = bpf.step_islands(model, M, m, seed, st, y_n, modified, mu_used=sc["mu_used"], theta=theta)
    e_inc = abs(inc - o["inc"]) / max(1.0, abs(o["inc"]))
    e_mean = rel_err(mean, o["mean"])
    e_ess = abs(ess - o["ess"]) / max(o["ess"], 1e-12)
    assert e_inc <= TOL_INC, f"step {n}: likelihood increment error {e_inc}"
    assert e_mean <= TOL_STATE, f"step {n}: mean error {e_mean}"
    assert e_ess <= 1e-4, f"step {n}: ess error {e_ess}"
    if theta is not None:
        tested = [i["ess_before"] for i in o["island_info"]]
        if len(o["island_info"]) < int(np.log2(m)):
            tested.append(bpf.ess_of(o["lW_final"]))
        if any(abs(e - theta) <= 1e-5 * theta for e in tested):
            return Report(ambiguous_steps=1)
        assert filt.stage_count() - c0 == len(o["island_info"]), f"step {n}: island stages run differ"
    w = o["within"]
    lo, hi = plausible_members(w["q"].reshape(m, M, 1), w["u"].reshape(m, M, 1), axis=1)
    dec_w = (lo == hi).reshape(N)
    undecidable = int(np.sum(~dec_w))
    line = np.ones(m, dtype=bool)
    isl = np.arange(m)
    for info in o["island_info"]:
        b = 1 << (info["s"] - 1)
        H = m // (2 * b)
        lo, hi = plausible_members(info["q"].reshape(H, 2, b), info["u"].reshape(H, 2, b), axis=1)
        dec = (lo == hi).reshape(m)
        undecidable += int(np.sum(~dec))
        if modified:
            dec = dec & dec[isl ^ b]
        line = dec & line[info["choice"]]
    src = o["holder"][np.arange(N) // M] * M + np.arange(N) % M
    ok = line[np.arange(N) // M] & dec_w[src]
    e_x = rel_err(x1[ok], new.x[ok])
    e_lv = rel_err(lv1, new.lV[::M] if theta is not None else np.full(lv1.shape, new.lV[0]))
    assert e_x <= TOL_STATE, f"step {n}: state error {e_x}"
    assert e_lv <= TOL_STATE, f"step {n}: log-weight error {e_lv}"
    assert abs(sc1["mu"] - new.mu) <= 1e-6 * max(1.0, abs(new.mu))
    swaps = sum(i["swaps_undone"] for i in o["island_info"])
    return Report(draws=N + m * len(o["island_info"]), undecidable=undecidable, undecided_particles=int(np.sum(~ok)),
                  swaps_undone=swaps, max_state_err=e_x, max_logweight_err=e_lv, max_inc_err=e_inc,
                  max_mean_err=e_mean, max_ess_err=e_ess)


def check_step_digit_sets(filt, model, radices, seed, y_n, n):
    """GPU time step n with the paper's stage matrices (PF_DIGIT_SETS: stage s on the
    digit set {0, s}) against the oracle's step from the same state; states must
    match on lines of ancestry whose every draw is decidable."""
    N = int(np.prod(radices))
    m = len(radices)
    x0, lv0, sc = filt.state()
    assert sc["n"] == n
    mean, inc, ess = filt.step(y_n)
    x1, lv1, sc1 = filt.state()
    lV = lv0[butterfly.set_group_index(np.arange(N), radices, m - 1)].astype(np.float64)
    st = bpf.State(x=x0.astype(np.float64), lV=lV, mu=sc["mu"], n=n)
    new, o = bpf.step_digit_sets(model, radices, seed, st, y_n, mu_used=sc["mu_used"])
    line = np.ones(N, dtype=bool)
    undecidable = 0
    for sg in o["stages"]:
        k = sg["k"]
        G = int(radices[0]) * int(radices[k])
        order = np.argsort(butterfly.set_group_major(N, radices, k))
        lo, hi = plausible_members(sg["q"][order].reshape(N // G, G), sg["u"][order].reshape(N // G, G), axis=1)
        dec = np.empty(N, dtype=bool)
        dec[order] = (lo == hi).reshape(N)
        undecidable += int(np.sum(~dec))
        line = dec & line[sg["anc"]]
    e_x = rel_err(x1[line], new.x[line])
    e_lv = rel_err(lv1, np.full(lv1.shape, new.lV[0]))
    e_inc = abs(inc - o["inc"]) / max(1.0, abs(o["inc"]))
    e_mean = rel_err(mean, o["mean"])
    e_ess = abs(ess - o["ess"]) / max(o["ess"], 1e-12)
    assert e_x <= TOL_STATE, f"step {n}: state error {e_x}"
    assert e_lv <= TOL_STATE, f"step {n}: log-weight error {e_lv}"
    assert e_inc <= TOL_INC, f"step {n}: likelihood increment error {e_inc}"
    assert e_mean <= TOL_STATE, f"step {n}: mean error {e_mean}"
    assert e_ess <= 1e-4, f"step {n}: ess error {e_ess}"
    assert abs(sc1["mu"] - new.mu) <= 1e-6 * max(1.0, abs(new.mu))
    return Report(draws=N * (m - 1), undecidable=undecidable, undecided_lines=int(np.sum(~line)),
                  max_state_err=e_x, max_logweight_err=e_lv, max_inc_err=e_inc, max_mean_err=e_mean,
                  max_ess_err=e_ess)
