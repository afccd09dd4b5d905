"""AIRPF (PF_ISLANDS): within-island resampling, augmented island resampling
(Algorithm 7, or 6 with PF_ISLANDS_PLAIN) and the island gather, checked step by
step against the oracle's AIRPF step from the GPU's own state."""
import numpy as np
import pytest

import synthetic as S
import lockstep as LS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,model,M,m,modified,T", [
    ("sv_16x64", S.sv_model(), 16, 64, True, 5),
    ("lg4_32x256", S.lg_dense(4, seed=3), 32, 256, True, 4),
    ("lg1_30x16_plain", S.lg_scalar(r=0.1), 30, 16, False, 5),
    ("lg1_100x16", S.lg_scalar(r=0.1), 100, 16, True, 5),
    ("sv_wide_300x8", S.sv_model(), 300, 8, True, 4),
    ("lg2_8x2048", S.lg_dense(2, seed=6), 8, 2048, True, 4),
    ("lg1_4x16384", S.lg_scalar(), 4, 16384, True, 3),
])
def test_islands_lockstep(bfpf, name, model, M, m, modified, T):
    N = M * m
    y = S.simulate(model, T, seed=47)[1]
    seed = 616
    f = bfpf.ButterflyFilter(model, N, (M, m), seed, islands="modified" if modified else "plain")
    desc = f.describe()
    assert desc["islands"] == m
    rep = LS.Report()
    for n in range(T):
        rep.merge(LS.check_step_islands(f, model, M, m, seed, y[n], n, modified))
    f.close()
    print(name, dict(rep))
    assert rep["undecided_particles"] <= max(16, 0.02 * N * T)


@pytest.mark.parametrize("name,model,M,m,theta,T", [
    ("sv_16x64_half", S.sv_model(), 16, 64, 0.5, 6),
    ("lg4_32x256_09", S.lg_dense(4, seed=3), 32, 256, 0.9, 4),
    ("lg1_30x16_all", S.lg_scalar(r=0.1), 30, 16, 1.5, 4),
    ("lg1_64x128_none", S.lg_scalar(r=0.1), 64, 128, 1e-9, 4),
    ("lg2_8x2048_07", S.lg_dense(2, seed=6), 8, 2048, 0.7, 4),
])
def test_airpf2_lockstep(bfpf, name, model, M, m, theta, T):
    """AIRPF2: the island stages run while the ESS of the island weights is below theta."""
    N = M * m
    y = S.simulate(model, T, seed=71)[1]
    seed = 717
    f = bfpf.ButterflyFilter(model, N, (M, m), seed, islands="modified", adaptive=True, ess_threshold=theta)
    assert "adapted" in f.describe()["island_resampling"]
    rep = LS.Report()
    for n in range(T):
        r = LS.check_step_islands(f, model, M, m, seed, y[n], n, True, theta=theta)
        rep.merge(r)
        if r.get("ambiguous_steps"):
            break
    stages = f.stage_count()
    f.close()
    print(name, dict(rep), "island stages", stages)
    if theta > 1:
        assert stages == int(np.log2(m)) * T
    if theta < 1e-6:
        assert stages == 0


def test_islands_graph_equals_steps(bfpf):
    model, M, m = S.sv_model(), 64, 32
    y = S.simulate(model, 30, seed=53)[1]
    a = bfpf.ButterflyFilter(model, M * m, (M, m), 17, islands="modified", chunk_len=7)
    ra = a.run(y)
    b = bfpf.ButterflyFilter(model, M * m, (M, m), 17, islands="modified")
    inc_b = [b.step(y[n])[1] for n in range(len(y))]
    assert np.array_equal(ra["inc"], np.array(inc_b))
    assert np.array_equal(a.state()[0], b.state()[0])
    a.close()
    b.close()


def test_islands_invalid(bfpf):
    m = S.lg_scalar()
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(m, 96, (8, 12), 1, islands="modified")            # m not a power of two
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(m, 64, (4, 4, 4), 1, islands="modified")          # not (M, m)
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(m, 64, (8, 8), 1, islands="modified", all_stages=True)
