"""The solve server on the GPU: every request's result is the same alone and in a mix of
concurrent requests (bit for bit: a column's arithmetic in the batched kernels does not depend on
the other columns, and a grouped solve of several operators gives each the bits of its own
solve), every result meets its tolerance (true residual from the oracle's product), and the
hierarchy cache is used."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2512_15121_gb300 import serve  # noqa: E402


def test_alone_equals_in_the_mix():
    reqs, ops = serve.synthetic_stream(24, seed=3, rate_per_s=1e9, max_rhs=3, meshes=(3, 4), orders=(2, 4),
                                       lambdas=(0.0, 1000.0))
    # alone: one request at a time through a one-slot server
    alone = serve.Server(slots=1)
    ref = {}
    for r in reqs:
        rr = serve.Request(rid=r.rid, key=r.key, make_operator=r.make_operator, rhs=r.rhs)
        alone.submit(rr)
        alone.drain()
        ref[r.rid] = rr
    alone.close()
    # the mix: every operator built by one request first, then everything submitted at once to a
    # three-slot server, whose workers solve the batches of cached operators in groups
    mix = serve.Server(slots=3)
    for key in sorted({r.key for r in reqs}):
        first = next(r for r in reqs if r.key == key)
        mix.submit(serve.Request(rid=-1, key=key, make_operator=first.make_operator, rhs=first.rhs))
    mix.drain()
    for r in reqs:
        r.arrival = 0.0
        mix.submit(r)
    mix.drain()
    mix.close()
    batched = sum(1 for r in reqs if sum(q.batch_id == r.batch_id for q in reqs) > 1)
    assert batched > 0  # some requests really shared a batch
    assert mix.stats["grouped_solves"] > 0  # and some batches of different operators a grouped solve
    for r in reqs:
        a = ref[r.rid]
        assert r.error is None and a.error is None
        assert np.array_equal(r.x, a.x), r.rid
        assert np.array_equal(r.iters, a.iters) and np.all(r.relres <= 1e-8)
    # true residuals of a few results through the oracle's product
    for r in reqs[:6]:
        n, p, lam = int(r.key[0][len("jitter"):-2]), r.key[1], r.key[2]
        prob = ops[(n, p, lam)]
        H = oracle.Hierarchy.from_problem(prob, cheb_degree=3 if lam > 0 else 2)
        for j in range(r.columns):
            res = r.rhs[:, j] - H.spmv(0, r.x[:, j])
            assert np.linalg.norm(res) <= 1.5e-8 * np.linalg.norm(r.rhs[:, j])


def test_stream_statistics_and_cache():
    reqs, ops = serve.synthetic_stream(40, seed=5, rate_per_s=400.0, max_rhs=4, meshes=(3, 4), orders=(2,),
                                       lambdas=(1.0,))
    srv = serve.Server(slots=2)
    stats = serve.run_stream(srv, reqs)
    srv.close()
    assert stats["requests"] == 40 and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert srv.stats["setups"] == 2 and srv.stats["cache_hits"] > 0
    assert all(r.error is None for r in reqs)
