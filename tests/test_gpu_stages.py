"""The paper's schedule (PF_ALL_STAGES): every stage of Algorithm 3 inside each
time step, checked step by step against the oracle's all-stages step."""
import numpy as np
import pytest

import synthetic as S
import lockstep as LS

pytestmark = pytest.mark.gpu


# launches: fused launches per step (consecutive digits of one power-of-two
# radix <= 32 share a launch while their tile fits), or m without fusion
@pytest.mark.parametrize("name,model,radices,T,launches", [
    ("lg_radix2", S.lg_scalar(), (2,) * 10, 5, 1),
    ("sv_group", S.sv_model(), (16, 16, 4), 5, 3),            # N < 2^16, 2 of 3 launches: not fused
    ("sv_mixed_radices", S.sv_model(), (32, 32, 16, 4), 3, 3),
    ("lg4_group", S.lg_dense(4, seed=3), (8, 8, 4), 4, 3),
    ("lg4_two_launches", S.lg_dense(4, seed=3), (8,) * 5, 3, 2),
    ("lg8_group", S.lg_dense(8, seed=4), (32, 32), 3, 1),
    ("lg8_two_launches", S.lg_dense(8, seed=6), (32, 32, 8, 8), 2, 2),
    ("sv_three_digits", S.sv_model(), (16, 16, 16, 16), 3, 2),
    ("lg3_radix4", S.lg_dense(3, seed=7), (4,) * 7, 3, 2),
    ("lg1_lone_radix2", S.lg_scalar(), (2, 4, 4, 4, 4), 4, 2),  # a one-digit launch of 2 on a tile of 4
    ("lg1_mixed_tile", S.lg_scalar(), (3, 5, 7), 5, 3),
    ("lg2_tile", S.lg_dense(2, seed=5), (64, 16), 4, 2),
    ("sv_wide", S.sv_model(), (300, 4), 4, 2),
])
@pytest.mark.parametrize("per_launch", [False, True])
def test_all_stages_lockstep(bfpf, name, model, radices, T, launches, per_launch):
    N = int(np.prod(radices))
    y = S.simulate(model, T, seed=23)[1]
    seed = 777
    f = bfpf.ButterflyFilter(model, N, radices, seed, all_stages=True,
                             extra_flags=bfpf.PF_TEST_STAGE_PER_LAUNCH if per_launch else 0)
    d = f.describe()
    assert d["stages_per_step"] == len(radices)
    assert d["launches_per_step"] == (len(radices) if per_launch else launches), d
    rep = LS.Report()
    for n in range(T):
        rep.merge(LS.check_step_all_stages(f, model, radices, seed, y[n], n))
    f.close()
    print(name, dict(rep))
    assert rep["undecided_lines"] <= max(8, 0.02 * N * T)


@pytest.mark.parametrize("model,radices,T", [
    (S.sv_model(), (16,) * 5, 6),                 # fused launches on digits {0, 1, 2} and {3, 4}
    (S.lg_dense(8, seed=4), (32, 32, 8, 8), 3),   # {0, 1} and {2, 3}; groups over 16 and 4 lanes
    (S.lg_scalar(), (4,) * 9, 4),                 # {0 .. 5} and {6, 7, 8}
])
def test_fused_launches_equal_one_launch_per_stage(bfpf, model, radices, T):
    """Fused launches split each group over lanes as the one-stage group
    kernel does, so from the same state the two forms of the schedule give the
    same particles and carried weights bit for bit (step 0).  The step
    summaries add the same terms in another block order, so from step 1 on the
    normaliser mu subtracted from the log-weights may differ in its last bits:
    then the carried weights agree to rounding and a draw may fall on the other
    side of a boundary, rarely."""
    N = int(np.prod(radices))
    y = S.simulate(model, T, seed=41)[1]
    a = bfpf.ButterflyFilter(model, N, radices, 99, all_stages=True)
    b = bfpf.ButterflyFilter(model, N, radices, 99, all_stages=True, extra_flags=bfpf.PF_TEST_STAGE_PER_LAUNCH)
    assert a.describe()["launches_per_step"] < len(radices) == b.describe()["launches_per_step"]
    for n in range(T):
        ma, ia, ea = a.step(y[n])
        mb, ib, eb = b.step(y[n])
        xa, lva, _ = a.state()
        xb, lvb, _ = b.state()
        if n == 0:
            assert np.array_equal(xa, xb), f"step {n}: states differ at {np.argwhere(xa != xb)[:5]}"
            assert np.array_equal(lva, lvb)
        else:
            assert np.mean(xa != xb) <= 1e-3, f"step {n}: {np.mean(xa != xb)} of the states differ"
            assert LS.rel_err(lva, lvb) <= 1e-6
        assert abs(ia - ib) <= 1e-6 * max(1.0, abs(ib))
        assert np.allclose(ma, mb, rtol=1e-5, atol=1e-6) and abs(ea - eb) <= 1e-4 * eb
    assert a.stage_count() == b.stage_count() == T * len(radices)
    a.close()
    b.close()


@pytest.mark.parametrize("model,radices", [
    (S.sv_model(), (16, 8, 4)),              # one launch per stage
    (S.lg_scalar(), (2,) * 10),              # one fused launch per step
    (S.sv_model(), (32, 32, 16, 4)),         # three fused launches per step
])
def test_all_stages_graph_equals_steps(bfpf, model, radices):
    """Chunks replayed from CUDA graphs (every launch of a step) equal single steps."""
    N = int(np.prod(radices))
    y = S.simulate(model, 40, seed=29)[1]
    a = bfpf.ButterflyFilter(model, N, radices, 31, all_stages=True, chunk_len=8)
    ra = a.run(y)
    b = bfpf.ButterflyFilter(model, N, radices, 31, all_stages=True)
    inc_b = [b.step(y[n])[1] for n in range(len(y))]
    assert np.array_equal(ra["inc"], np.array(inc_b))
    assert np.array_equal(a.state()[0], b.state()[0])
    a.close()
    b.close()


def test_all_stages_single_digit_is_default(bfpf):
    """With one digit the two schedules are the same filter."""
    model = S.lg_scalar()
    y = S.simulate(model, 12, seed=31)[1]
    a = bfpf.ButterflyFilter(model, 512, (512,), 5, all_stages=True)
    b = bfpf.ButterflyFilter(model, 512, (512,), 5)
    ra, rb = a.run(y), b.run(y)
    assert np.array_equal(ra["inc"], rb["inc"]) and np.array_equal(a.state()[0], b.state()[0])
    a.close()
    b.close()


def test_all_stages_rejects_ancestor_recording(bfpf):
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 64, (8, 8), 1, all_stages=True, record_ancestors=True)


@pytest.mark.parametrize("name,model,radices,T", [
    ("sv_paper_4x8pe", S.sv_model(), (4, 2, 2, 2), 5),
    ("lg_paper_8x16pe", S.lg_scalar(), (8, 2, 2, 2, 2), 5),
    ("lg3_mixed", S.lg_dense(3, seed=8), (16, 4, 4, 2), 4),
    ("sv_m100", S.sv_model(), (100, 2, 2, 2), 4),
    ("lg1_wide_300", S.lg_scalar(r=0.2), (300, 2, 2), 4),
    ("lg2_32x8x4", S.lg_dense(2, seed=9), (32, 8, 4), 4),
    ("sv_two_digits", S.sv_model(), (32, 16), 4),
    ("lg1_paper_64x1024pe", S.lg_scalar(), (64,) + (2,) * 10, 3),
])
def test_digit_sets_lockstep(bfpf, name, model, radices, T):
    N = int(np.prod(radices))
    y = S.simulate(model, T, seed=59)[1]
    seed = 828
    f = bfpf.ButterflyFilter(model, N, radices, seed, digit_sets=True)
    d = f.describe()
    assert d["digit_sets"] and d["stages_per_step"] == len(radices) - 1
    rep = LS.Report()
    for n in range(T):
        rep.merge(LS.check_step_digit_sets(f, model, radices, seed, y[n], n))
    f.close()
    print(name, dict(rep))
    # a draw is undecidable with probability about eta * (group size); a line crosses m - 1 stages
    expected = sum(radices[0] * a for a in radices[1:]) * LS.ETA * N * T
    assert rep["undecided_lines"] <= max(16, 3 * expected)


def test_digit_sets_graph_equals_steps(bfpf):
    model, radices = S.sv_model(), (16, 2, 2, 2, 2)
    N = int(np.prod(radices))
    y = S.simulate(model, 30, seed=61)[1]
    a = bfpf.ButterflyFilter(model, N, radices, 3, digit_sets=True, chunk_len=8)
    ra = a.run(y)
    b = bfpf.ButterflyFilter(model, N, radices, 3, digit_sets=True)
    inc_b = [b.step(y[n])[1] for n in range(len(y))]
    assert np.array_equal(ra["inc"], np.array(inc_b))
    assert np.array_equal(a.state()[0], b.state()[0])
    a.close()
    b.close()


def test_digit_sets_invalid(bfpf):
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 2048, (64, 32), 1, digit_sets=True)       # a_0 a_1 > 1024
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 64, (8, 8), 1, digit_sets=True, all_stages=True)
