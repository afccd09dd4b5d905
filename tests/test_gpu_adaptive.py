"""Fully adapted augmented resampling (PF_ADAPTIVE): every step checked against
the oracle's adaptive step from the GPU's own state."""
import numpy as np
import pytest

import synthetic as S
import lockstep as LS

pytestmark = pytest.mark.gpu


def _informative_lg(d, seed):
    model = S.lg_dense(d, seed=seed)
    model.Lr = 0.3 * np.eye(d)          # sharp observations: the ESS falls quickly
    return model


@pytest.mark.parametrize("name,model,radices,theta,rotate,T", [
    ("sv_half", S.sv_model(), (16, 16, 4), 0.5, False, 8),
    ("sv_rot", S.sv_model(), (16, 16, 4), 0.97, True, 8),
    ("lg4_rot", _informative_lg(4, 3), (8, 8, 4), 0.8, True, 6),
    ("lg1_mixed", S.lg_scalar(r=0.05), (3, 5, 7), 0.9, False, 6),
    ("lg2_all", _informative_lg(2, 5), (32, 32), 1.5, False, 4),
    ("lg1_none", S.lg_scalar(), (16, 16), 1e-9, True, 4),
    ("sv_wide", S.sv_model(), (300, 4), 0.9, True, 4),
    # sizes at which every digit runs on the register-resident group kernel (no rotation)
    ("sv_group_half", S.sv_model(), (16, 16, 16), 0.5, False, 5),
    ("sv_group_all", S.sv_model(), (16, 16, 16), 1.5, False, 3),
    ("lg4_group_09", _informative_lg(4, 3), (8, 8, 8, 8), 0.9, False, 4),
])
def test_adaptive_lockstep(bfpf, name, model, radices, theta, rotate, T):
    N = int(np.prod(radices))
    y = S.simulate(model, T, seed=41)[1]
    seed = 515
    f = bfpf.ButterflyFilter(model, N, radices, seed, adaptive=True, ess_threshold=theta, rotate=rotate)
    desc = f.describe()
    assert desc["adaptive"] and desc["rotate"] == rotate
    if name.startswith(("sv_group", "lg4_group")):
        assert all(dg["kernel"] == "group" for dg in desc["digits"])
    rep = LS.Report()
    start = 0
    for n in range(T):
        r, start = LS.check_step_adaptive(f, model, radices, seed, y[n], n, theta, rotate, start)
        rep.merge(r)
        if start is None:      # ambiguous decision: the schedules may part from here
            break
    f.close()
    print(name, dict(rep))
    if theta > 1:
        assert rep["stages"] == len(radices) * T
    if theta < 1.0 / N:
        assert rep.get("stages", 0) == 0
    assert rep.get("undecided_lines", 0) <= max(8, 0.02 * N * T)


def test_adaptive_graph_equals_steps(bfpf):
    model, radices = _informative_lg(3, 7), (8, 8, 4)
    N = int(np.prod(radices))
    y = S.simulate(model, 24, seed=43)[1]
    a = bfpf.ButterflyFilter(model, N, radices, 9, adaptive=True, ess_threshold=0.7, rotate=True, chunk_len=6)
    ra = a.run(y)
    b = bfpf.ButterflyFilter(model, N, radices, 9, adaptive=True, ess_threshold=0.7, rotate=True)
    inc_b = [b.step(y[n])[1] for n in range(len(y))]
    assert np.array_equal(ra["inc"], np.array(inc_b))
    assert a.stage_count() == b.stage_count() > 0
    assert np.array_equal(a.state()[0], b.state()[0])
    a.close()
    b.close()


def test_adaptive_invalid_combinations(bfpf):
    m = S.lg_scalar()
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(m, 64, (8, 8), 1, adaptive=True, all_stages=True)
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(m, 64, (8, 8), 1, adaptive=True, record_ancestors=True)
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(m, 4096, (4096,), 1, adaptive=True)
