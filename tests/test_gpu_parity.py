"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every test runs the library's kernels on the same seeded inputs as the oracle
and compares element by element (see tests/lockstep.py for the decidability
rule of ancestor draws and the tolerances).
"""
import numpy as np
import pytest

import synthetic as S
from oracle import bpf, philox
import lockstep as LS

pytestmark = pytest.mark.gpu


def _filter(bfpf, model, radices, seed, **kw):
    N = int(np.prod(radices))
    return bfpf.ButterflyFilter(model, N, radices, seed, record_ancestors=True, **kw)


def test_device_philox_matches_oracle(bfpf):
    for seed, ctr in [(0, (0, 0, 0, 0)), (2 ** 40 + 12345, (17, 3, 1, 0)), (2 ** 64 - 1, (2 ** 32 - 100, 9, 2, 7))]:
        dev = bfpf.philox_blocks(seed, ctr, 4096).cpu().numpy().astype(np.uint64)
        c = (np.arange(4096, dtype=np.uint64) + ctr[0]) & np.uint64(0xFFFFFFFF)
        host = np.stack(philox.philox4x32(c, ctr[1], ctr[2], ctr[3], philox.seed_key(seed)), 1)
        assert np.array_equal(dev, host.astype(np.uint64))


@pytest.mark.parametrize("case", [
    ("lg1d_radix2", S.lg_scalar(), (2,) * 10, 12),
    ("lg1d_mixed", S.lg_scalar(), (4, 2, 8, 4), 9),
    ("lg1d_nonpow2", S.lg_scalar(), (3, 5, 4, 3), 9),
    ("lg2d", S.lg_dense(2, seed=3), (8, 4, 4), 7),
    ("lg3d", S.lg_dense(3, seed=5), (16, 8, 2), 7),
    ("lg4d", S.lg_dense(4, seed=7), (32, 32), 5),
    ("lg8d", S.lg_dense(8, seed=2), (32, 32), 5),
    ("lg5d_obs2", None, (8, 8, 2), 6),
    ("sv", S.sv_model(), (16, 16, 4), 7),
    ("sv_nonpow2", S.sv_model(), (6, 7, 5), 7),
    ("global_256", S.lg_scalar(), (256,), 4),
    ("wide_512", S.sv_model(), (512,), 4),
    ("wide_mixed", S.lg_scalar(), (300, 4), 5),
    # Section 6.1's model: A = I, Q = I, R = I/4 (the diagonal-A and diagonal-Lr fast paths)
    ("rw7d_paper", S.random_walk(7), (16, 16, 16), 7),
    ("rw7d_paper_all_digits", S.random_walk(7), (4, 8, 2, 16), 9),
])
def test_lockstep_small(bfpf, case):
    name, model, radices, T = case
    if model is None:   # non-identity observation matrix and correlated noise factors
        model = S.lg_dense(5, seed=11)
        model.H = np.array([[1.0, 0.5, 0.0, -0.2, 0.0], [0.0, 0.3, 1.0, 0.0, 0.7]])
        model.Lr = np.array([[0.8, 0.0], [0.3, 0.6]])
        model.Lq = np.tril(np.full((5, 5), 0.1)) + 0.6 * np.eye(5)
        model.m0 = np.linspace(-1, 1, 5)
    y = S.simulate(model, T, seed=17)[1]
    seed = 4242
    f = _filter(bfpf, model, radices, seed)
    rep = LS.Report()
    for n in range(T):
        rep.merge(LS.check_step_full(f, model, radices, seed, y[n], n))
    f.close()
    print(name, dict(rep))
    # each draw is undecidable with probability about 2 ETA a (a boundaries, margin ~ ETA Q)
    a_max = max(radices)
    assert rep["undecidable"] <= max(8, 4 * 2 * LS.ETA * a_max * rep["draws"])


@pytest.mark.parametrize("d,radices", [
    (1, (2,) * 12), (1, (4, 8, 2, 16, 8)), (1, (32, 32, 4)), (2, (8, 8, 8, 8)), (3, (16, 2, 32)),
    (4, (32, 32)), (5, (4, 16, 8)), (7, (16, 16, 2)), (8, (32, 32)), (8, (2, 4, 8, 16))])
def test_lockstep_group_kernels(bfpf, d, radices):
    """Sizes at which the register-resident group kernel runs every digit."""
    model = S.lg_scalar() if d == 1 else S.lg_dense(d, seed=d)
    y = S.simulate(model, len(radices) + 2, seed=19)[1]
    f = _filter(bfpf, model, radices, 99)
    plan = f.describe()
    assert all(dg["kernel"] == "group" for dg in plan["digits"]), plan
    rep = LS.Report()
    for n in range(len(y)):
        rep.merge(LS.check_step_full(f, model, radices, 99, y[n], n))
    f.close()
    print("group", d, radices, dict(rep))
    assert rep["undecidable"] <= max(8, 4 * 2 * LS.ETA * max(radices) * rep["draws"])


def test_lockstep_sv_group_kernel(bfpf):
    model = S.sv_model()
    radices = (16, 16, 16, 4)
    y = S.simulate(model, 6, seed=23)[1]
    f = _filter(bfpf, model, radices, 7)
    digits = f.describe()["digits"]
    assert all(dg["kernel"] == "group" for dg in digits)
    # 16384 particles fill few thread blocks: two members per lane (8 lanes per radix-16 group)
    assert [dg["lanes"] for dg in digits] == [8, 8, 8, 2]
    rep = LS.Report()
    for n in range(len(y)):
        rep.merge(LS.check_step_full(f, model, radices, 7, y[n], n))
    f.close()
    print("sv group", dict(rep))


@pytest.mark.parametrize("all_stages", [False, True])
def test_lockstep_sv_group_kernel_default_split(bfpf, all_stages):
    """2^20 particles: the default split (a whole radix-16 group in one lane), every
    step checked in full against the oracle."""
    model = S.sv_model()
    radices = (16,) * 5
    y = S.simulate(model, 5 if not all_stages else 2, seed=29)[1]
    N = int(np.prod(radices))
    f = (bfpf.ButterflyFilter(model, N, radices, 17, all_stages=True) if all_stages
         else _filter(bfpf, model, radices, 17))
    digits = f.describe()["digits"]
    assert all(dg["kernel"] == "group" and dg["lanes"] == 1 for dg in digits)
    rep = LS.Report()
    for n in range(len(y)):
        if all_stages:
            rep.merge(LS.check_step_all_stages(f, model, radices, 17, y[n], n))
        else:
            rep.merge(LS.check_step_full(f, model, radices, 17, y[n], n))
    f.close()
    print("sv group default split", all_stages, dict(rep))


@pytest.mark.parametrize("d,N,T", [(1, 4096, 5), (1, 1 << 16, 3), (4, 5000, 3), (8, 1 << 14, 2), (0, 1 << 15, 4)])
def test_lockstep_global_resampling(bfpf, d, N, T):
    """radices = {N} above one block: the global path (d = 0 means SV)."""
    model = S.sv_model() if d == 0 else (S.lg_scalar() if d == 1 else S.lg_dense(d, seed=d))
    y = S.simulate(model, T, seed=41)[1]
    f = _filter(bfpf, model, (N,), 606)
    assert f.describe()["digits"][0]["kernel"] == "global"
    rep = LS.Report()
    for n in range(T):
        rep.merge(LS.check_step_full(f, model, (N,), 606, y[n], n))
    assert f.status() == 0
    f.close()
    print("global", d, N, dict(rep))
    # With one group of N members the worst-case margin (ETA times a cumulative sum)
    # spans several boundary spacings, so most draws count as undecidable; the
    # actual FP32/FP64 differences are far smaller: nearly all draws agree exactly.
    assert rep["mismatched_undecidable"] <= 0.001 * rep["draws"]


@pytest.mark.parametrize("d,N,T,small,outlier", [
    (1, 4099, 3, False, False),        # N not a multiple of 4: scalar weight loop, ragged scan tile
    (1, 1 << 15, 3, False, True),      # one far observation: most integer weights tiny or zero
    (2, 1 << 15, 2, True, False),      # 16 draws per bucket: the overflow list and global searches
    (0, 1 << 16, 2, True, False),
    (8, 5000, 2, True, True),
    (1, 1025, 2, False, False),        # the smallest global population: one scan tile, four buckets
])
def test_lockstep_global_bucket_paths(bfpf, d, N, T, small, outlier):
    """The global draws are resolved per bucket of their uniform; every layout
    of buckets (staged in shared memory, searched in global memory, overflow)
    must give the oracle's ancestors."""
    model = S.sv_model() if d == 0 else (S.lg_scalar() if d == 1 else S.lg_dense(d, seed=d))
    y = S.simulate(model, T, seed=43)[1]
    if outlier:
        y = y.copy()
        y[0] = 8.0
    flags = bfpf.PF_TEST_SMALL_BUCKETS if small else 0
    f = _filter(bfpf, model, (N,), 607, extra_flags=flags)
    dg = f.describe()["digits"][0]
    assert dg["kernel"] == "global"
    if small:
        assert dg["bucket_cap"] == 16 and dg["stage_cap"] == 64
    rep = LS.Report()
    for n in range(T):
        rep.merge(LS.check_step_full(f, model, (N,), 607, y[n], n))
    assert f.status() == 0
    f.close()
    print("global buckets", d, N, small, outlier, dict(rep))
    assert rep["mismatched_undecidable"] <= 0.001 * rep["draws"]


def test_config1_lockstep_all_steps(bfpf):
    """1-D LG, N = 2^10 radix 2, T = 100: every step checked from the GPU's state."""
    w = S.workload("lg1d_n1024")
    y = w.observations()
    f = _filter(bfpf, w.model, w.radices, w.filter_seed)
    rep = LS.Report()
    for n in range(w.T):
        rep.merge(LS.check_step_full(f, w.model, w.radices, w.filter_seed, y[n], n))
    f.close()
    print("lg1d_n1024 lockstep", dict(rep))


def test_config1_free_running_parity(bfpf):
    """Free-running GPU and oracle from the same seed: ancestors agree bit for bit
    up to the first undecidable draw (none expected at this size); the FP64
    log-likelihood agrees to 1e-6 relative."""
    w = S.workload("lg1d_n1024")
    y = w.observations()
    ref = bpf.run(w.model, w.N, w.radices, w.filter_seed, y, keep_ancestors=True)
    f = _filter(bfpf, w.model, w.radices, w.filter_seed)
    first_diff = None
    incs = []
    for n in range(w.T):
        _, inc, _ = f.step(y[n])
        incs.append(inc)
        if first_diff is None and not np.array_equal(f.ancestors(), ref["anc"][n]):
            first_diff = n
    ll = f.loglik()
    f.close()
    if first_diff is not None:
        pytest.fail(f"ancestors diverged at step {first_diff}")
    assert abs(ll - ref["loglik"]) <= 1e-6 * abs(ref["loglik"]), (ll, ref["loglik"])
    np.testing.assert_allclose(incs, ref["inc"], rtol=1e-6, atol=1e-6)


def test_run_graph_equals_steps(bfpf):
    """pf_run (CUDA-graph chunks, several chunk lengths) equals step-by-step pf_step."""
    model = S.lg_dense(4, seed=9)
    radices = (8, 16, 4)
    y = S.simulate(model, 37, seed=2)[1]
    outs = []
    for chunk in (0, 5, 16):
        f = bfpf.ButterflyFilter(model, int(np.prod(radices)), radices, 77, chunk_len=chunk)
        r = f.run(y)
        outs.append((r, f.loglik(), f.state()[0]))
        f.close()
    f = bfpf.ButterflyFilter(model, int(np.prod(radices)), radices, 77)
    step_incs = [f.step(y[n])[1] for n in range(len(y))]
    x_step = f.state()[0]
    f.close()
    for r, ll, x in outs:
        assert np.array_equal(r["inc"], np.array(step_incs))
        assert np.array_equal(x, x_step)


def test_run_with_device_inputs(bfpf):
    import torch
    model = S.sv_model()
    radices = (16, 16)
    y = S.simulate(model, 20, seed=5)[1]
    f1 = bfpf.ButterflyFilter(model, 256, radices, 3)
    r1 = f1.run(y)
    f2 = bfpf.ButterflyFilter(model, 256, radices, 3)
    r2 = f2.run(torch.tensor(y, dtype=torch.float32, device="cuda"))
    assert np.array_equal(r1["inc"], r2["inc"].cpu().numpy())
    assert np.array_equal(r1["mean"], r2["mean"].cpu().numpy())
    f1.close()
    f2.close()


def test_tile_choice_does_not_change_ancestors(bfpf):
    model = S.lg_dense(2, seed=1)
    radices = (4, 8, 16)
    y = S.simulate(model, 9, seed=8)[1]
    ancs = []
    for tile in (64, 512, 4096):
        f = _filter(bfpf, model, radices, 5, tile=tile)
        a = []
        for n in range(9):
            f.step(y[n])
            a.append(f.ancestors())
        ancs.append(np.stack(a))
        f.close()
    # ancestors can only differ through last-bit differences of the normaliser
    for a in ancs[1:]:
        assert np.mean(a == ancs[0]) > 0.999


def test_nonfinite_observation_sets_status(bfpf):
    model = S.lg_scalar()
    f = bfpf.ButterflyFilter(model, 64, (4, 4, 4), 1)
    f.step(np.array([0.3]))
    assert f.status() == 0
    f.step(np.array([np.nan]))
    assert f.status() & 1
    f.close()


def test_invalid_arguments_raise(bfpf):
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 64, (4, 4, 2), 1)      # product != N
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 4096, (2048, 2), 1)    # radix too large for m > 1
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_dense(9, seed=1), 64, (8, 8), 1)  # d > 8
