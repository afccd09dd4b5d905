"""Unit parity of the integer draw: every ancestor, exactly.

The draw of Algorithm 2 (and of Algorithm 3's sampling line) is integer
arithmetic once the quantised weights are fixed: with the prefix sums P of
the integer weights of a group, its total Q and a particle's uniform word(s)
r, the ancestor is member #{j : P_j <= floor(r Q / 2^W)}.  The GPU path and
the oracle compute the weights in different precisions, so the lockstep tests
can only ask for agreement on draws far from a boundary.  Here the filter is
created with PF_RECORD_DRAWS and hands back the integer prefix sums it used;
the oracle redoes every draw of the step from those integers and from its own
Philox words, and every ancestor must agree: no tolerance, no exceptions.

The recorded weights are also checked against the oracle's own FP64-derived
quantisation of the same pre-step state (they may differ by the FP32 rounding
the lockstep margin allows, 2^-15 relative plus two quanta), and the first
states against the oracle's draw from pi_0.

Cases cover the register-resident group kernel (radices 2 to 32, both SV and
linear-Gaussian models), the shared-memory tile kernel (non-power-of-two
radices, groups of 300, 512 and 1024 members with 32-bit weights and 64-bit
draws) and the global-resampling path (one group of N = 2^16, 2^20 and 2^24
particles, every bucket layout).
"""
import numpy as np
import pytest

import synthetic as S
from oracle import bpf, butterfly, philox, resample
import lockstep as LS

pytestmark = pytest.mark.gpu


def _dense_lg():
    model = S.lg_dense(3, seed=12)
    model.A = np.array([[0.8, 0.3, -0.1], [-0.2, 0.7, 0.25], [0.05, -0.3, 0.6]])
    model.Lq = np.array([[0.9, 0.0, 0.0], [0.6, 0.5, 0.0], [-0.4, 0.7, 0.3]])
    model.H = np.array([[1.0, 0.5, 0.0], [0.0, -1.0, 2.0]])
    model.Lr = np.array([[0.7, 0.0], [0.3, 0.9]])
    model.m0 = np.array([0.5, -1.0, 0.2])
    model.L0 = np.array([[1.0, 0, 0], [0.2, 0.8, 0], [0.1, -0.3, 1.1]])
    return model


def redo_draws(prefix, anc, radices, seed, n):
    """The oracle's draws of step n from the GPU's integer prefix sums.
    Returns (number of draws, number that differ from the GPU's ancestors)."""
    N = int(np.prod(radices))
    m = len(radices)
    k = n % m
    a = int(radices[k])
    s = butterfly.strides(radices)[k]
    H = N // (a * s)
    P = prefix.reshape(H, a, s)
    q = np.diff(P, axis=1, prepend=np.zeros((H, 1, s), dtype=np.uint64))
    Q = P[:, -1:, :]
    B = resample.qbits(a)
    assert np.all(q <= np.uint64(1 << B)), "an integer weight above 2^B"
    live = Q[:, 0, :] > 0
    assert np.all(q.max(axis=1)[live] == np.uint64(1 << B)), "the group maximum must weigh exactly 2^B"
    pi = butterfly.group_major(N, radices, k)
    if a <= resample.NARROW_MAX_RADIX:
        r = philox.resample_words_at(seed, n, pi).reshape(H, a, s)
        u = resample.scaled_uniform(r, Q, a)
    else:
        lo, hi = philox.resample_words_wide_at(seed, n, pi)
        u = resample.scaled_uniform(lo.reshape(H, a, s), Q, a, hi.reshape(H, a, s))
    member = resample.draw(q, u, axis=1)
    idx = np.arange(N).reshape(H, a, s)
    anc = anc.astype(np.int64).reshape(H, a, s)
    assert np.array_equal(anc // (a * s), idx // (a * s)) and np.array_equal(anc % s, idx % s), \
        "an ancestor outside its group"
    member_gpu = (anc // s) % a
    return N, int(np.sum(member_gpu != member))


def quantisation_gap(model, radices, seed, n, x0, lv0, mu_used, y_n, prefix):
    """Largest |q_gpu - q_oracle| - (2^-15 q_oracle + 2) over the step's weights,
    with q_oracle the oracle's quantisation of the GPU's own pre-step state."""
    N = int(np.prod(radices))
    k = n % len(radices)
    a = int(radices[k])
    s = butterfly.strides(radices)[k]
    H = N // (a * s)
    lV = LS.per_particle_lV(lv0, radices, n).astype(np.float64)
    lw, _ = bpf.weigh(model, x0.astype(np.float64), lV, mu_used, y_n)
    q_or = resample.quantise(lw.reshape(H, a, s), axis=1).astype(np.float64)
    P = prefix.reshape(H, a, s)
    q_gpu = np.diff(P, axis=1, prepend=np.zeros((H, 1, s), dtype=np.uint64)).astype(np.float64)
    return float(np.max(np.abs(q_gpu - q_or) - (LS.ETA * q_or + 2)))


def run_exact(bfpf, model, radices, seed, T, y=None, check_quant=True, extra_flags=0):
    N = int(np.prod(radices))
    if y is None:
        y = S.simulate(model, T, seed=seed % 1000 + 3)[1]
    f = bfpf.ButterflyFilter(model, N, radices, seed, extra_flags=bfpf.PF_RECORD_DRAWS | extra_flags)
    draws = differ = 0
    worst_gap = -np.inf
    for n in range(T):
        x0, lv0, sc = f.state() if check_quant else (None, None, None)
        f.step(y[n])
        prefix = f.draw_prefix()
        anc = f.ancestors()
        d, bad = redo_draws(prefix, anc, radices, seed, n)
        draws += d
        differ += bad
        if check_quant:
            worst_gap = max(worst_gap, quantisation_gap(model, radices, seed, n, x0, lv0, sc["mu_used"], y[n], prefix))
    f.close()
    return draws, differ, worst_gap


@pytest.mark.parametrize("name,model,radices,T", [
    ("sv_radix2", S.sv_model(), (2,) * 12, 14),
    ("sv_radix4", S.sv_model(), (4,) * 6, 8),
    ("sv_radix8", S.sv_model(), (8,) * 5, 7),
    ("sv_radix16", S.sv_model(), (16,) * 4, 6),
    ("sv_radix32", S.sv_model(), (32,) * 3, 5),
    ("lg1d_radix16", S.lg_scalar(), (16, 16, 8), 5),
    ("lg3d_dense", "dense", (16, 8, 16), 5),
    ("lg8d_radix32", S.lg_dense(8, seed=2), (32, 32), 4),
])
def test_group_kernel_draws_exact(bfpf, name, model, radices, T):
    if model == "dense":
        model = _dense_lg()
    draws, differ, gap = run_exact(bfpf, model, radices, 9001, T)
    print(name, "draws", draws, "differ", differ, "quantisation gap", gap)
    assert differ == 0
    assert gap <= 0.0


@pytest.mark.parametrize("name,model,radices,T", [
    ("sv_3_5_7_4", S.sv_model(), (3, 5, 7, 4), 6),
    ("lg_6_64", S.lg_scalar(), (6, 64), 4),
    ("lg3d_dense_12_9", "dense", (12, 9, 10), 4),
    ("sv_300_4", S.sv_model(), (300, 4), 4),
    ("lg_512_2", S.lg_scalar(), (512, 2), 3),
    ("sv_1024_4", S.sv_model(), (1024, 4), 3),
    ("lg_1024_single", S.lg_scalar(), (1024,), 3),
])
def test_tile_kernel_draws_exact(bfpf, name, model, radices, T):
    if model == "dense":
        model = _dense_lg()
    draws, differ, gap = run_exact(bfpf, model, radices, 9002, T)
    print(name, "draws", draws, "differ", differ, "quantisation gap", gap)
    assert differ == 0
    assert gap <= 0.0


@pytest.mark.parametrize("N,T,small", [(1025, 3, False), (4096, 3, False), (4099, 3, False), (1 << 16, 3, False),
                                       (1 << 16, 2, True), (1 << 20, 2, False), (1 << 24, 2, False)])
def test_global_draws_exact(bfpf, N, T, small):
    """One group of all N particles (Algorithm 2): the GPU's 64-bit prefix sums
    over the whole population and the oracle's 64-bit uniforms.  N = 1025 and
    4096 fit one scan tile (no reduce pass); 4099 ends in a ragged tile."""
    model = S.sv_model()
    flags = bfpf.PF_TEST_SMALL_BUCKETS if small else 0
    draws, differ, gap = run_exact(bfpf, model, (N,), 9003, T, check_quant=N <= (1 << 20), extra_flags=flags)
    print("global", N, small, "draws", draws, "differ", differ, "quantisation gap", gap)
    assert differ == 0
    if N <= (1 << 20):
        assert gap <= 0.0


def test_headline_draws_exact_at_full_size(bfpf):
    """SV, N = 2^24, radix 16: two full steps, every one of the 2^25 draws."""
    w = S.workload("sv_n16m")
    y = w.observations()[:2]
    draws, differ, _ = run_exact(bfpf, w.model, w.radices, w.filter_seed, 2, y=y, check_quant=False)
    print("headline", "draws", draws, "differ", differ)
    assert differ == 0 and draws == 2 * w.N


@pytest.mark.parametrize("name,model", [("sv", S.sv_model()), ("lg3d_dense", "dense"),
                                        ("lg7d_random_walk", S.random_walk(7))])
def test_initial_particles_match_oracle(bfpf, name, model):
    """Algorithm 1's first loop: the GPU's draw from pi_0 against the oracle's (SV:
    the stationary law; linear-Gaussian: m0 + L0 eps with non-trivial m0, L0)."""
    if model == "dense":
        model = _dense_lg()
    N = 1 << 14
    f = bfpf.ButterflyFilter(model, N, (16, 16, 64), 777)
    x0, _, _ = f.state()
    f.close()
    want = bpf.initial_particles(model, N, 777)
    assert LS.rel_err(x0, want) <= LS.TOL_STATE
