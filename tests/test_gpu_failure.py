"""Failure reporting without a GPU fault.  No kernel of the library waits on
another block (the global path's prefix sum is reduce-then-scan), so the
failures a step can meet are in its data: a non-finite observation makes
every log-weight NaN.  The step treats them as weight zero (status bit 0),
the all-zero population keeps its particles (status bit 1, every ancestor is
the particle itself), the bits are sticky on the handle, and the context and
the handle stay usable: the following finite steps run normally."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("radices", [(1 << 16,), (16, 16, 16, 16)])
def test_nan_observation_is_reported_and_the_filter_goes_on(bfpf, radices):
    model = S.lg_scalar()
    N = int(np.prod(radices))
    y = S.simulate(model, 4, seed=3)[1]
    f = bfpf.ButterflyFilter(model, N, radices, 11, record_ancestors=True)
    f.step(y[0])
    assert f.status() == 0
    x_before, _, _ = f.state()
    bad = np.full_like(y[1], np.nan)
    f.step(bad)
    assert f.status() & 1 and f.status() & 2, f.status()
    anc = f.ancestors()
    assert np.array_equal(anc, np.arange(N)), "an all-zero population must keep its particles"
    x_after, _, _ = f.state()
    assert np.all(np.isfinite(x_after))
    # the propagation still moved every particle (the mutation ran on the kept states)
    assert not np.array_equal(x_after, x_before)
    for n in (2, 3):
        f.step(y[n])
    assert np.all(np.isfinite(f.state()[0]))
    assert f.status() & 1, "the status bits are sticky"
    f.close()
    # another filter in the same context is unaffected
    g = bfpf.ButterflyFilter(model, N, radices, 11)
    g.run(y)
    assert g.status() == 0
    assert np.isfinite(g.loglik())
    g.close()
