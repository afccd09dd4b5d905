"""The all-core CPU baseline of the bench splits the groups of every step of the
FP64 oracle over a pool of processes; it must compute exactly what the
single-process oracle step computes (states, carried weights, normaliser)."""
import numpy as np

import bench
import synthetic as S
from oracle import bpf, butterfly


def test_pool_step_equals_single_process_oracle():
    w = S.workload("sv_n16m")
    N = 1 << 12
    x, lv, mu, _, _, radices = bench.oracle_pool_run("sv_n16m", N, procs=3, steps=4)
    st = bpf.init_state(w.model, N, w.filter_seed)
    y = w.observations(4)
    for n in range(4):
        st, _ = bpf.step(w.model, radices, w.filter_seed, st, y[n])
    assert np.array_equal(x, st.x)
    assert np.allclose(lv, st.lV, rtol=0, atol=1e-12)
    assert abs(mu - st.mu) < 1e-12
