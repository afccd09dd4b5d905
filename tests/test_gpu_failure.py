"""Failure reporting without a GPU fault: the global-resampling scan's bounded
wait is made to run out (a test hook makes one tile wait on a flag that nothing
sets); the kernel gives up, records status bit 2 and returns, the host reports
PF_ETIMEOUT, and the context stays usable."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def test_scan_wait_runs_out_and_is_reported(bfpf):
    model = S.lg_scalar()
    N = 1 << 16                                  # 16 scan tiles
    y = S.simulate(model, 2, seed=3)[1]
    f = bfpf.ButterflyFilter(model, N, (N,), 11, extra_flags=bfpf.PF_TEST_SCAN_TIMEOUT)
    f.step(y[0])
    assert f.status() & 4
    with pytest.raises(bfpf.PFError) as e:
        f.loglik()
    assert e.value.status == bfpf.PF_ETIMEOUT
    f.close()
    # the context is still usable: a normal filter runs and reports no timeout
    g = bfpf.ButterflyFilter(model, N, (N,), 11)
    g.run(y)
    assert g.status() & 4 == 0
    assert np.isfinite(g.loglik())
    g.close()
