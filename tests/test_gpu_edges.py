"""Edge cases of the boundary: no observations, the smallest filter, the
largest group one thread block resamples, the most digits, and arguments
outside the documented limits."""
import numpy as np
import pytest

import synthetic as S
import lockstep as LS

pytestmark = pytest.mark.gpu


def test_zero_observations_is_a_no_op(bfpf):
    f = bfpf.ButterflyFilter(S.sv_model(), 256, (16, 16), 3)
    x0 = f.state()[0]
    r = f.run(np.zeros((0, 1)))
    assert r["inc"].shape == (0,) and r["mean"].shape[0] == 0
    assert f.loglik() == 0.0 and np.array_equal(f.state()[0], x0)
    f.close()


@pytest.mark.parametrize("model,radices,T", [
    (S.lg_scalar(), (2,), 6),                      # two particles, one digit
    (S.sv_model(), (1024,), 3),                    # the largest group of one thread block
    (S.lg_scalar(), (2,) * 16, 3),                 # sixteen digits
    (S.lg_dense(8, seed=4), (2, 2), 4),            # largest state dimension, four particles
])
def test_extreme_shapes_lockstep(bfpf, model, radices, T):
    N = int(np.prod(radices))
    y = S.simulate(model, T, seed=91)[1]
    f = bfpf.ButterflyFilter(model, N, radices, 44, record_ancestors=True)
    for n in range(T):
        LS.check_step_full(f, model, radices, 44, y[n], n)
    f.close()


def test_arguments_outside_the_limits(bfpf):
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 2 ** 31, (2 ** 31,), 1)                          # N >= 2^31
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 2 ** 33, (2,) * 33, 1)                           # more than 32 digits
    with pytest.raises(bfpf.PFError):
        bfpf.ButterflyFilter(S.lg_scalar(), 1, (1,), 1)                                       # N < 2


def test_filter_keeps_running_after_a_smaller_tile_is_created(bfpf):
    """The shared-memory limit of a kernel is shared by every handle: creating a
    filter with a smaller tile must not break a running filter with a larger one."""
    model = S.lg_scalar()
    big = bfpf.ButterflyFilter(model, 4096, (64, 64), 1, tile=4096)
    small = bfpf.ButterflyFilter(model, 4096, (64, 64), 2, tile=256)
    y = S.simulate(model, 3, seed=3)[1]
    for n in range(3):
        big.step(y[n])
        small.step(y[n])
    assert np.isfinite(big.loglik()) and np.isfinite(small.loglik())
    big.close()
    small.close()
