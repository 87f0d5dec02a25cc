"""Host logic of the solve server with a fake clock, a fake free-memory figure and a fake solver:
batching of requests for one operator, the column limit, admission by free memory, LRU eviction
and completion of every request.  No GPU is used."""
import threading
import time

import numpy as np

from paper_2512_15121_gb300 import serve


class FakeSolver:
    def __init__(self, key):
        self.key = key
        self.closed = False

    def close(self):
        self.closed = True


class Memory:
    """free bytes = capacity - bytes of live fake hierarchies"""

    def __init__(self, capacity):
        self.capacity = capacity
        self.live = {}
        self.lock = threading.Lock()

    def info(self):
        with self.lock:
            return self.capacity - sum(self.live.values()), self.capacity


def make_request(rid, key, n=100, cols=1):
    op = dict(n=n, row_ptr=None, col=None, val=np.zeros(10 * n), elem_dof=None, p=2)
    return serve.Request(rid=rid, key=key, make_operator=lambda: op, rhs=np.full((n, cols), float(rid)))


def server_with_fakes(capacity, slots=2, delay=0.002, max_columns=32):
    mem = Memory(capacity)
    batches = []

    def factory(op):
        s = FakeSolver(None)
        mem.live[id(s)] = serve.estimate_bytes(op["n"], len(op["val"]), max_columns)
        orig = s.close

        def close():
            mem.live.pop(id(s), None)
            orig()
        s.close = close
        return s, None

    def runner(e, B, rtol, precision):
        batches.append(B.shape[1])
        time.sleep(delay)
        m = B.shape[1]
        return B * 2.0, np.full(m, 3, np.int32), np.full(m, 1e-9)

    srv = serve.Server(slots=slots, reserve_bytes=0, max_columns=max_columns, mem_info=mem.info,
                       solver_factory=factory, runner=runner)
    return srv, mem, batches


def test_every_request_completes_with_its_own_columns():
    srv, mem, batches = server_with_fakes(capacity=1 << 40)
    reqs = [make_request(i, key=("mesh", i % 3, 1.0), cols=1 + i % 4) for i in range(40)]
    for r in reqs:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    for r in reqs:
        assert r.error is None and r.x.shape == r.rhs.shape
        assert np.array_equal(r.x, 2.0 * r.rhs)           # the columns come back to their owner
        assert np.all(r.iters == 3)
    assert sum(batches) == sum(r.columns for r in reqs)
    assert max(batches) <= 32
    assert srv.stats["setups"] == 3 and srv.stats["cache_hits"] >= 1


def test_requests_for_one_operator_are_batched():
    srv, mem, batches = server_with_fakes(capacity=1 << 40, slots=1, delay=0.05)
    first = make_request(0, ("A", 2, 0.0))
    srv.submit(first)
    time.sleep(0.01)  # the first batch is running; these queue up and run together next
    rest = [make_request(i, ("A", 2, 0.0)) for i in range(1, 9)]
    for r in rest:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert batches[0] == 1 and batches[1] == 8
    assert len({r.batch_id for r in rest}) == 1


def test_column_limit_splits_batches():
    srv, mem, batches = server_with_fakes(capacity=1 << 40, slots=1, delay=0.02, max_columns=8)
    reqs = [make_request(i, ("A", 2, 0.0), cols=3) for i in range(6)]
    for r in reqs:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert all(b <= 8 for b in batches) and sum(batches) == 18


def test_admission_waits_for_memory_and_evicts_idle_hierarchies():
    one = serve.estimate_bytes(100, 1000, 32)
    srv, mem, batches = server_with_fakes(capacity=int(1.5 * one), slots=1)
    reqs = [make_request(i, (f"mesh{i % 3}", 2, 0.0)) for i in range(9)]
    for r in reqs:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert all(r.error is None for r in reqs)
    # only one hierarchy fits: switching operators evicts the idle one
    assert srv.stats["evictions"] >= 2
    assert len(mem.live) == 0


def test_latency_summary():
    reqs = [make_request(i, ("A", 2, 0.0)) for i in range(4)]
    for i, r in enumerate(reqs):
        r.arrival, r.finish = 0.0, 0.001 * (i + 1)
    s = serve.latency_summary(reqs)
    assert s["requests"] == 4 and abs(s["p50_ms"] - 3.0) < 1e-9 and abs(s["p99_ms"] - 4.0) < 1e-9


def test_failed_setup_fails_its_requests_and_the_server_goes_on():
    mem = Memory(1 << 40)

    def factory(op):
        if op["p"] == 7:
            raise RuntimeError("element order outside 1..12")
        return FakeSolver(None), None

    def runner(e, B, rtol, precision):
        m = B.shape[1]
        return B * 2.0, np.full(m, 3, np.int32), np.full(m, 1e-9)

    srv = serve.Server(slots=2, reserve_bytes=0, mem_info=mem.info, solver_factory=factory, runner=runner)
    bad_op = dict(n=10, row_ptr=None, col=None, val=np.zeros(100), elem_dof=None, p=7)
    bad = [serve.Request(rid=100 + i, key=("bad", 7, 0.0), make_operator=lambda: bad_op, rhs=np.ones((10, 1)))
           for i in range(3)]
    good = [make_request(i, ("A", 2, 0.0)) for i in range(6)]
    for r in bad + good:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert all(r.error and "setup failed" in r.error and r.finish >= 0 for r in bad)
    assert all(r.error is None and np.array_equal(r.x, 2.0 * r.rhs) for r in good)
    assert srv.stats["setup_errors"] >= 1 and srv.stats["failed_requests"] == 3
    assert ("bad", 7, 0.0) not in srv.cache and all(w.is_alive() is False for w in srv.workers)


def test_setups_of_different_operators_overlap():
    """A setup runs outside the server lock: two slow builds for two operators run at once."""
    mem = Memory(1 << 40)
    active, peak = [0], [0]
    lock = threading.Lock()

    def factory(op):
        with lock:
            active[0] += 1
            peak[0] = max(peak[0], active[0])
        time.sleep(0.1)
        with lock:
            active[0] -= 1
        return FakeSolver(None), None

    def runner(e, B, rtol, precision):
        m = B.shape[1]
        return B, np.ones(m, np.int32), np.zeros(m)

    srv = serve.Server(slots=2, reserve_bytes=0, mem_info=mem.info, solver_factory=factory, runner=runner)
    reqs = [make_request(0, ("A", 2, 0.0)), make_request(1, ("B", 2, 0.0))]
    for r in reqs:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert peak[0] == 2 and srv.stats["setups"] == 2
    assert all(r.error is None for r in reqs)


def test_malformed_requests_are_refused_at_submit():
    """A right-hand side that is not an n x r array with 1 <= r <= max_columns is refused by
    submit (it would otherwise stop a worker or wait forever); the server goes on."""
    import pytest
    srv, mem, batches = server_with_fakes(capacity=1 << 40, max_columns=8)
    for rhs in (np.zeros(100), np.zeros((100, 0)), np.zeros((100, 9)), [[0.0]]):
        r = make_request(1, key=("mesh", 0, 1.0))
        r.rhs = rhs
        with pytest.raises(ValueError, match="rhs"):
            srv.submit(r)
    good = make_request(2, key=("mesh", 0, 1.0), cols=8)
    srv.submit(good)
    srv.drain(30)
    srv.close()
    assert good.error is None and np.array_equal(good.x, 2.0 * good.rhs)


def test_request_with_the_wrong_row_count_fails_alone():
    """In a batch for one operator, a request whose rows are not the operator's n fails with its
    own error; the other requests of the batch are solved."""
    srv, mem, batches = server_with_fakes(capacity=1 << 40, delay=0.05)
    inner = srv.solver_factory

    def factory(op):
        s, stream = inner(op)
        s.n = op["n"]
        return s, stream
    srv.solver_factory = factory
    key = ("mesh", 0, 1.0)
    reqs = [make_request(i, key=key, n=100) for i in range(3)]
    reqs[1].rhs = np.ones((101, 1))
    for r in reqs:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert "rows" in reqs[1].error and reqs[1].x is None
    for r in (reqs[0], reqs[2]):
        assert r.error is None and np.array_equal(r.x, 2.0 * r.rhs)
    assert srv.stats["failed_requests"] == 1


def test_size_hint_admits_by_size_and_builds_outside_the_lock():
    """A request that states its operator's (n, nnz) is admitted by that size, and its operator is
    materialised by the worker that builds the hierarchy, outside the server's lock (other workers
    keep serving meanwhile): once per setup."""
    srv, mem, batches = server_with_fakes(capacity=1 << 40, slots=2)
    made, held = [], []
    n = 100

    def maker(key):
        def make():
            held.append(srv.cv._is_owned())
            made.append(key)
            return dict(n=n, row_ptr=None, col=None, val=np.zeros(10 * n), elem_dof=None, p=2)
        return make

    reqs = [serve.Request(rid=i, key=("mesh", i % 2, 1.0), make_operator=maker(i % 2),
                          rhs=np.full((n, 1), float(i)), size=(n, 10 * n)) for i in range(12)]
    for r in reqs:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert all(r.error is None and np.array_equal(r.x, 2.0 * r.rhs) for r in reqs)
    assert sorted(made) == [0, 1] and srv.stats["setups"] == 2
    assert held == [False, False]
    # admission by the stated size: larger than the whole device memory with nothing cached, built
    # or running (nothing will ever be freed), the request fails at once instead of waiting
    # forever, and its operator is never built
    srv2, mem2, _ = server_with_fakes(capacity=serve.estimate_bytes(n, 10 * n) - 1, slots=1)
    called = []
    big = serve.Request(rid=99, key=("mesh", 9, 1.0), make_operator=lambda: called.append(1),
                        rhs=np.ones((n, 1)), size=(n, 10 * n))
    srv2.submit(big)
    srv2.drain(10)
    srv2.close()
    assert not called and big.error is not None and "device memory" in big.error


def test_shared_operators_combine_stiffness_and_mass():
    """The large-stream generator's operators share one stiffness and one mass matrix per mesh and
    order: K + lambda M equals the directly assembled operator of that lambda (to rounding, the
    element sums grouped differently), with the Dirichlet identity rows kept, and its nodal
    right-hand sides are the generator's own nodal Fourier fields."""
    import fegen
    so = serve._SharedOperator(3, 2)
    try:
        for lam in (0.0, 1.0, 1000.0):
            direct = fegen.make(3, 2, mesh="jitter", mesh_seed=3, lam=lam, rhs="none")
            v = so.values(lam)
            assert np.array_equal(direct.row_ptr, so.K.row_ptr) and np.array_equal(direct.col, so.K.col)
            assert np.max(np.abs(v - direct.val)) <= 1e-13 * np.max(np.abs(direct.val))
            assert np.all(v[so.diag_rows] == 1.0)
            direct.close()
        F = so.rhs_nodal([5, 6])
        for j, sd in enumerate((5, 6)):
            assert np.allclose(F[:, j], so.K.rhs_nodal(sd), rtol=0, atol=1e-12 * np.abs(F).max())
    finally:
        so.close()


def test_cached_operators_are_solved_in_groups():
    """A worker that takes a batch also takes the waiting batches of other cached, idle operators
    with the same precision and tolerance (up to max_group) and solves them in one grouped call;
    every request still gets its own columns back.  Requests with another tolerance or precision,
    and operators not yet built, are not pulled into a group."""
    mem = Memory(1 << 40)
    groups, singles = [], []

    def factory(op):
        s = FakeSolver(None)
        s.n = op["n"]
        return s, None

    def runner(e, B, rtol, precision):
        singles.append(B.shape[1])
        return B * 2.0, np.full(B.shape[1], 3, np.int32), np.full(B.shape[1], 1e-9)

    def group_runner(items):
        groups.append([(it[1].shape[1], it[2], it[3]) for it in items])
        assert len({(it[2], it[3]) for it in items}) == 1  # one tolerance and precision per group
        return [(it[1] * 2.0, np.full(it[1].shape[1], 3, np.int32), np.full(it[1].shape[1], 1e-9), 0) for it in items]

    srv = serve.Server(slots=1, reserve_bytes=0, mem_info=mem.info, solver_factory=factory, runner=runner,
                       group_runner=group_runner, max_group=3)
    # build four operators first (one request each), then a burst for all of them
    warm = [make_request(i, key=("mesh", i, 1.0)) for i in range(4)]
    for r in warm:
        srv.submit(r)
    srv.drain(30)
    burst = [make_request(10 + i, key=("mesh", i % 4, 1.0), cols=2) for i in range(8)]
    odd = make_request(99, key=("mesh", 0, 1.0))
    odd.rtol = 1e-6                                             # another tolerance: its own batch
    for r in burst + [odd]:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    for r in warm + burst + [odd]:
        assert r.error is None and np.array_equal(r.x, 2.0 * r.rhs), r.rid
    assert groups and all(len(g) <= 3 for g in groups)
    assert all(t[1] == 1e-8 for g in groups for t in g)
    assert srv.stats["grouped_solves"] == len(groups)
    assert srv.stats["grouped_batches"] == sum(len(g) for g in groups)
    assert srv.stats["setups"] == 4


def test_large_operators_are_not_grouped():
    """Operators above group_max_nnz are solved on their own: their kernels fill the GPU, and a
    grouped call would hold its small members until the large one is done."""
    mem = Memory(1 << 40)
    groups = []

    def factory(op):
        s = FakeSolver(None)
        s.n = op["n"]
        return s, None

    def runner(e, B, rtol, precision):
        return B * 2.0, np.full(B.shape[1], 3, np.int32), np.full(B.shape[1], 1e-9)

    def group_runner(items):
        groups.append(sorted(it[1].shape[0] for it in items))
        return [(it[1] * 2.0, np.full(it[1].shape[1], 3, np.int32), np.full(it[1].shape[1], 1e-9), 0) for it in items]

    srv = serve.Server(slots=1, reserve_bytes=0, mem_info=mem.info, solver_factory=factory, runner=runner,
                       group_runner=group_runner, max_group=4, group_max_nnz=5000)
    sizes = {0: 100, 1: 100, 2: 100, 3: 800}  # nnz 10 n: the last one is large
    warm = [make_request(i, key=("mesh", i, 1.0), n=sizes[i]) for i in range(4)]
    for r in warm:
        srv.submit(r)
    srv.drain(30)
    burst = [make_request(10 + i, key=("mesh", i % 4, 1.0), n=sizes[i % 4]) for i in range(12)]
    for r in burst:
        srv.submit(r)
    srv.drain(30)
    srv.close()
    assert all(r.error is None and np.array_equal(r.x, 2.0 * r.rhs) for r in warm + burst)
    assert groups and all(800 not in g for g in groups)
