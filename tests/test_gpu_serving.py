"""Serving loop: continuous batching with memory admission; every request's
result is the same alone and in the mix."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _requests(serve, n=12, seed=11):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n):
        kind = r % 4
        model = [S.lg_scalar(), S.lg_dense(4, seed=r), S.lg_dense(8, seed=r), S.sv_model()][kind]
        N = int(2 ** rng.integers(10, 15))
        radices = (16,) * (int(np.log2(N)) // 4) + ((2 ** (int(np.log2(N)) % 4),) if np.log2(N) % 4 else ())
        T = int(rng.integers(100, 260))
        y = S.simulate(model, T, seed=500 + r)[1]
        reqs.append(serve.Request(rid=r, arrival=0.002 * r, model=model, N=N, radices=radices,
                                  seed=7000 + r, y=y))
    return reqs


def test_results_same_alone_and_in_the_mix(bfpf):
    from paper_1812_01502_gb300 import serve
    mix = _requests(serve)
    srv = serve.Server(memory_budget=8 << 30, slots=6)
    done = {r.rid: r for r in srv.run(mix)}
    assert len(done) == len(mix)
    assert srv.max_active > 1                        # requests overlapped on the device
    for rid in (0, 3, 7, 10):
        alone = _requests(serve)[rid]
        alone.arrival = 0.0
        one = serve.Server(memory_budget=8 << 30, slots=1).run([alone])[0]
        assert np.array_equal(one.means, done[rid].means)
        assert np.array_equal(one.incs, done[rid].incs)
        assert one.loglik == done[rid].loglik
    s = serve.summarize(list(done.values()), srv.wall)
    print("serving", s)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_memory_admission_limits_concurrency(bfpf):
    from paper_1812_01502_gb300 import serve
    reqs = _requests(serve, n=8, seed=3)
    need = max(serve.workspace_bytes(r.model, r.N, r.radices) for r in reqs)
    budget = 2 * need + 1
    srv = serve.Server(memory_budget=budget, slots=8)
    done = srv.run(reqs)
    assert len(done) == len(reqs)
    assert srv.max_in_use <= budget              # admission never exceeded the budget
    assert srv.max_active < len(reqs)            # so some requests had to wait
    assert all(np.all(np.isfinite(r.incs)) for r in done)


def test_request_larger_than_budget_is_refused(bfpf):
    from paper_1812_01502_gb300 import serve
    req = _requests(serve, n=1)[0]
    with pytest.raises(MemoryError):
        serve.Server(memory_budget=1024, slots=2).run([req])


def test_failed_request_is_isolated(bfpf):
    """A request with NaN observations finishes with an error; every other request
    in the mix gets exactly its result alone."""
    from paper_1812_01502_gb300 import serve
    mix = _requests(serve, n=8, seed=5)
    bad = mix[2]
    bad.y = bad.y.copy()
    bad.y[40:45] = np.nan
    done = {r.rid: r for r in serve.Server(memory_budget=8 << 30, slots=6).run(mix)}
    assert done[2].error is not None and done[2].status & 1
    for rid in (0, 5):
        assert done[rid].error is None
        alone = _requests(serve, n=8, seed=5)[rid]
        alone.arrival = 0.0
        one = serve.Server(memory_budget=8 << 30, slots=1).run([alone])[0]
        assert np.array_equal(one.incs, done[rid].incs)
    assert serve.summarize(list(done.values()), 1.0)["failed_requests"] == 1



def test_admission_by_device_free_memory(bfpf):
    """Without a fixed budget the server admits against the device's free memory
    (less a reserve); results are those of each request alone."""
    from paper_1812_01502_gb300 import serve
    mix = _requests(serve, n=8, seed=13)
    srv = serve.Server(slots=4)
    assert srv.available() > 0
    done = {r.rid: r for r in srv.run(mix)}
    assert len(done) == len(mix) and srv.max_active > 1
    alone = _requests(serve, n=8, seed=13)[6]
    alone.arrival = 0.0
    one = serve.Server(slots=1).run([alone])[0]
    assert np.array_equal(one.means, done[6].means)


def test_chunks_arrive_after_admission(bfpf):
    """Observation chunks that arrive every 20 ms are enqueued only once they have
    arrived: a request of k chunks finishes no earlier than arrival + k * 20 ms,
    and its result is the same as with every observation available at once."""
    from paper_1812_01502_gb300 import serve
    reqs = _requests(serve, n=3, seed=17)
    for r in reqs:
        r.chunk_interval = 0.02
    done = {r.rid: r for r in serve.Server(memory_budget=8 << 30, slots=3).run(reqs)}
    for r in reqs:
        k = -(-len(r.y) // r.chunk)
        assert done[r.rid].finished >= r.arrival + k * 0.02 - 1e-9
        assert len(done[r.rid].chunk_latencies) == k
    instant = _requests(serve, n=3, seed=17)[1]
    instant.arrival = 0.0
    one = serve.Server(memory_budget=8 << 30, slots=1).run([instant])[0]
    assert np.array_equal(one.incs, done[1].incs)
