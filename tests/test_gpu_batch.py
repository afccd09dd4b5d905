"""Batches of independent filters (pf_batch_*): parity with the oracle for
filters inside a batch, and independence of each filter from the rest."""
import numpy as np
import pytest

import synthetic as S
from oracle import bpf, butterfly
import lockstep as LS

pytestmark = pytest.mark.gpu


def _specs():
    out = []
    rng = np.random.default_rng(7)
    shapes = [(1, (2,) * 8), (1, (16, 16, 4)), (4, (4, 8, 8)), (8, (32, 8)), (2, (3, 5, 7)), (4, (64,)),
              (8, (2, 2, 4, 8)), (1, (256, 2)), (3, (8, 8, 8)), (1, (256,))]
    for f, (d, rad) in enumerate(shapes):
        model = S.sv_model() if (d == 1 and f % 3 == 1) else (S.lg_scalar() if d == 1 else S.lg_dense(d, seed=f))
        out.append((model, int(np.prod(rad)), rad, 9000 + f))
    return out


def _specs_group():
    """Filters whose digits run the group path inside the batch (a power-of-two
    radix <= 32 whose groups fill whole block iterations: groups per iteration
    = 256 / lanes per group, lanes = radix / members per lane, members per lane
    = the largest power of two m <= radix with m d <= 16), at d = 1, 2, 4 and 8,
    with every radix from 2 to 32, and two filters that mix both paths (a radix
    3 digit on the tile path)."""
    shapes = [(8, (32, 32)), (8, (16, 8, 8)), (4, (16, 16, 8)), (4, (16, 16, 16, 3)), (2, (32, 32, 2)),
              (1, (16, 16, 16)), (1, (2, 4, 32, 16)), (8, (32, 32, 3))]
    out = []
    for f, (d, rad) in enumerate(shapes):
        model = S.sv_model() if (d == 1 and f == 5) else (S.lg_scalar() if d == 1 else S.lg_dense(d, seed=20 + f))
        out.append((model, int(np.prod(rad)), rad, 9100 + f))
    return out


def _obs(specs, T):
    dy_max = max(s[0].dy for s in specs)
    y = np.zeros((len(specs), T, dy_max), dtype=np.float32)
    for f, (model, N, rad, seed) in enumerate(specs):
        y[f, :, :model.dy] = S.simulate(model, T, seed=100 + f)[1]
    return y


@pytest.mark.parametrize("which", ["mixed", "group"])
def test_each_filter_independent_of_the_batch(bfpf, which):
    specs = _specs() if which == "mixed" else _specs_group()
    T = 9
    y = _obs(specs, T)
    b = bfpf.FilterBatch(specs)
    r = b.run(y)
    ll = b.loglik()
    b.close()
    for f in ((0, 3, 5, 9) if which == "mixed" else (0, 3, 5, 7)):
        one = bfpf.FilterBatch([specs[f]])
        r1 = one.run(y[f:f + 1, :, :specs[f][0].dy])
        assert np.array_equal(r1["inc"][0], r["inc"][f])
        d = specs[f][0].d
        assert np.array_equal(r1["mean"][0, :, :d], r["mean"][f, :, :d])
        assert np.array_equal(r1["ess"][0], r["ess"][f])
        assert one.loglik()[0] == ll[f]
        one.close()


def test_batch_initial_states_equal_single_filter(bfpf):
    specs = _specs()[:6]
    b = bfpf.FilterBatch(specs)
    for f, (model, N, rad, seed) in enumerate(specs):
        single = bfpf.ButterflyFilter(model, N, rad, seed)
        assert np.array_equal(b.state(f)[0], single.state()[0])
        single.close()
    b.close()


@pytest.mark.parametrize("which", ["mixed", "group"])
def test_batch_lockstep_against_oracle(bfpf, which):
    """Every step of every filter re-run by the oracle from the batch's own state:
    likelihood increments, means, ESS and new carried weights to the parity
    tolerances; states of particles whose draw is decidable to 1e-5.  "group":
    filters on the batch's group path (every radix 2 to 32, d = 1 to 8)."""
    specs = _specs() if which == "mixed" else _specs_group()
    T = 6
    y = _obs(specs, T)
    b = bfpf.FilterBatch(specs)
    rep = LS.Report()
    for n in range(T):
        before = [b.state(f) for f in range(len(specs))]
        r = b.run(y[:, n:n + 1, :])
        for f, (model, N, rad, seed) in enumerate(specs):
            x0, lv0, sc = before[f]
            x1, lv1, _ = b.state(f)
            lV = LS.per_particle_lV(lv0, rad, n).astype(np.float64)
            st = bpf.State(x=x0.astype(np.float64), lV=lV, mu=sc["mu"], n=n)
            new, o = bpf.step(model, rad, seed, st, y[f, n, :model.dy], mu_used=sc["mu_used"])
            a, s = o["a"], o["stride"]
            H = N // (a * s)
            lo, hi = LS.plausible_members(o["q"].reshape(H, a, s), o["u"].reshape(H, a, s), axis=1)
            dec = (lo == hi).reshape(N)
            e_x = LS.rel_err(x1[dec], new.x[dec])
            e_lv = LS.rel_err(lv1, o["lV_new"].reshape(H, a, s)[:, 0, :].reshape(-1))
            inc = r["inc"][f, 0]
            e_inc = abs(inc - o["inc"]) / max(1.0, abs(o["inc"]))
            e_mean = LS.rel_err(r["mean"][f, 0, :model.d], o["mean"])
            assert e_x <= LS.TOL_STATE, (f, n, e_x)
            assert e_lv <= LS.TOL_STATE, (f, n, e_lv)
            assert e_inc <= LS.TOL_INC, (f, n, e_inc)
            assert e_mean <= LS.TOL_STATE, (f, n, e_mean)
            assert abs(r["ess"][f, 0] - o["ess"]) <= 1e-4 * o["ess"]
            rep.merge(LS.Report(draws=N, undecidable=int(np.sum(~dec)), max_state_err=e_x,
                                max_logweight_err=e_lv, max_inc_err=e_inc, max_mean_err=e_mean))
    b.close()
    print("batch lockstep", which, dict(rep))
    assert rep["undecidable"] <= 0.02 * rep["draws"]


def test_batch_of_uneven_filters_runs(bfpf):
    specs = [(w.model, w.N, w.radices, w.filter_seed) for w in S.batched_specs(256, T=20, log2n=(8, 13))]
    y = _obs(specs, 20)
    b = bfpf.FilterBatch(specs)
    r = b.run(y)
    b.close()
    assert np.all(np.isfinite(r["inc"]))
    assert np.all((r["ess"] > 0) & (r["ess"] <= 1 + 1e-6))


def test_batch_rejects_wide_radix(bfpf):
    with pytest.raises(bfpf.PFError):
        bfpf.FilterBatch([(S.lg_scalar(), 1024, (512, 2), 1)])
