"""Checkpoint / resume (pf_save / pf_load): a filter resumed from a checkpoint
continues bit for bit as the uninterrupted one, for every schedule; a
checkpoint is refused by a filter with other parameters."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,model,radices,kw", [
    ("one_digit_sv", S.sv_model(), (16, 16, 16), {}),
    ("tile_mixed", S.lg_dense(3, seed=2), (3, 5, 7), {}),
    ("global", S.lg_scalar(), (1 << 14,), {}),
    ("all_stages", S.sv_model(), (8, 8, 4), {"all_stages": True}),
    ("all_stages_one_fused_launch", S.lg_scalar(), (2,) * 10, {"all_stages": True}),
    ("all_stages_three_fused_launches", S.sv_model(), (32, 32, 16, 4), {"all_stages": True}),
    ("adaptive_rot", S.lg_dense(2, seed=3), (8, 8, 4), {"adaptive": True, "ess_threshold": 0.8, "rotate": True}),
    ("airpf2", S.sv_model(), (32, 64), {"islands": "modified", "adaptive": True, "ess_threshold": 0.5}),
    ("digit_sets", S.lg_scalar(), (16, 2, 2, 2, 2), {"digit_sets": True}),
])
def test_resume_is_bit_identical(bfpf, name, model, radices, kw):
    N = int(np.prod(radices))
    y = S.simulate(model, 30, seed=81)[1]
    a = bfpf.ButterflyFilter(model, N, radices, 99, **kw)
    a.run(y[:12])
    blob = a.save()
    ra = a.run(y[12:30])
    xa, lva, sca = a.state()
    lla = a.loglik()
    a.close()
    b = bfpf.ButterflyFilter(model, N, radices, 99, **kw)
    b.load(blob)
    assert b.steps == 12
    rb = b.run(y[12:30])
    xb, lvb, scb = b.state()
    assert np.array_equal(ra["inc"], rb["inc"]) and np.array_equal(ra["mean"], rb["mean"])
    assert np.array_equal(xa, xb) and np.array_equal(lva, lvb)
    assert b.loglik() == lla
    b.close()


def test_checkpoint_refused_by_other_parameters(bfpf):
    model = S.sv_model()
    a = bfpf.ButterflyFilter(model, 1024, (16, 64), 5)
    a.run(S.simulate(model, 3, seed=1)[1])
    blob = a.save()
    a.close()
    for radices, seed in (((64, 16), 5), ((16, 64), 6)):
        b = bfpf.ButterflyFilter(model, 1024, radices, seed)
        with pytest.raises(bfpf.PFError):
            b.load(blob)
        b.close()
    c = bfpf.ButterflyFilter(S.sv_model(phi=0.9), 1024, (16, 64), 5)   # another model
    with pytest.raises(bfpf.PFError):
        c.load(blob)
    c.close()
