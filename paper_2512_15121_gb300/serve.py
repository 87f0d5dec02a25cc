"""Continuous-batching solve server over the C ABI.

Requests (an assembled operator, its element map, and 1..32 right-hand sides) arrive over time.
The server

* caches hierarchies on the device, keyed by (mesh key, order, lambda): a request whose operator
  is cached skips setup;
* admits work only while free device memory covers it (a hierarchy's estimated footprint plus a
  reserve), evicting idle cached hierarchies least recently used first;
* batches: requests for the same operator that are waiting when a worker slot frees up are
  solved together as one multi-right-hand-side solve (giamg_solve_batch, up to 32 columns);
  requests that arrive while a batch runs join the next batch -- continuous batching;
* overlaps: every cached hierarchy owns a CUDA stream and every worker slot is a host thread,
  so batches for different operators run concurrently on the device;
* groups: a worker that takes a batch also takes the other waiting batches (same precision and
  tolerance) whose hierarchies are cached and idle, up to max_group, and solves them together
  with giamg_solve_grouped -- one kernel launch per phase of the V-cycle and the CG iteration
  for all of them, each with the bits of its own multi-right-hand-side solve.

A column's arithmetic in the batched kernels does not depend on the other columns, so a request
gets the same bits alone and in a mix (tests/test_gpu_serve.py checks this).  The clock and the
free-memory probe are injectable so admission can be tested deterministically on the host.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    key: tuple                      # (mesh key, order, lambda)
    make_operator: Callable         # () -> dict(n, row_ptr, col, val, elem_dof, p, cheb_degree)
    rhs: np.ndarray                 # n x r (r <= 32)
    rtol: float = 1e-8
    precision: int = 1
    arrival: float = 0.0
    size: tuple | None = None       # (n, nnz) of the operator, if known without building it: the
                                    # server then admits by it and calls make_operator outside its lock
    # filled in by the server
    start: float = -1.0
    finish: float = -1.0
    x: np.ndarray | None = None
    iters: np.ndarray | None = None
    relres: np.ndarray | None = None
    error: str | None = None
    batch_id: int = -1

    @property
    def columns(self) -> int:
        return int(self.rhs.shape[1])


def estimate_bytes(n: int, nnz: int, columns: int = 32) -> int:
    """Device footprint of a served hierarchy plus batch work: the finest CSR (FP64 + FP32 values,
    column indices, row pointers) with a third more for the coarse levels, row patterns and
    groups, and the n x 32 FP64 / FP32 work blocks of the multi-right-hand-side solve."""
    matrix = nnz * (8 + 4 + 4) + 16 * n
    work = n * columns * (12 * 8 + 5 * 4)
    return int(1.35 * matrix + work)


class _Entry:
    def __init__(self, solver, stream, nbytes, nnz=0):
        self.solver = solver
        self.stream = stream
        self.nbytes = nbytes
        self.nnz = nnz
        self.lock = threading.Lock()
        self.last_used = 0.0
        self.busy = False


class Server:
    def __init__(self, slots: int = 4, reserve_bytes: int = 2 << 30, max_columns: int = 32,
                 mem_info: Callable | None = None, clock: Callable | None = None,
                 solver_factory: Callable | None = None, runner: Callable | None = None, device: int = 0,
                 solver_options: dict | None = None, max_group: int = 8, group_runner: Callable | None = None,
                 group_max_nnz: int = 20_000_000):
        self.slots = slots
        self.solver_options = dict(solver_options or {})
        self.reserve = reserve_bytes
        self.max_columns = max_columns
        self.clock = clock or time.perf_counter
        self.device = device
        self.release_cache = None
        if mem_info is None:
            import torch
            mem_info = lambda: torch.cuda.mem_get_info(device)  # noqa: E731
            self.release_cache = torch.cuda.empty_cache  # torch's unused cached blocks back to the device
        self.mem_info = mem_info
        self.solver_factory = solver_factory or self._default_factory
        self.runner = runner or self._default_runner
        # grouped solves: the library's by default, none with an injected runner unless given one
        self.group_runner = group_runner or (self._default_group_runner if runner is None else None)
        self.max_group = max_group if self.group_runner is not None else 1
        # only operators this small are grouped: their solves are bound by kernel launches, which
        # a group shares; a large operator's kernels fill the GPU alone, and a grouped call
        # returns when its slowest member is done, so a large member would hold the small ones
        self.group_max_nnz = group_max_nnz
        self.cache: dict = {}
        self.pending: dict = collections.OrderedDict()   # key -> deque of requests
        self.done: list = []
        self.cv = threading.Condition()
        self.closed = False
        self.stats = collections.Counter()
        self.batch_seq = 0
        self._running = 0
        self._building_bytes = 0
        self.workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(slots)]
        for w in self.workers:
            w.start()

    # ------------------------------------------------------------------ hierarchy cache
    def _default_factory(self, op: dict):
        """A hierarchy on its own stream.  The operator is handed over as host arrays, which the
        library copies into memory it owns (no torch temporaries: freed blocks in torch's caching
        allocator would stay invisible to the free-memory probe that admission relies on); solves
        then take device arrays."""
        import torch
        from . import Solver
        stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.device(self.device):
            opts = dict(self.solver_options)
            opts.setdefault("cheb_degree", op.get("cheb_degree", 3))
            # served solves are multi-right-hand-side solves, whose kernels read the CSR values and
            # row patterns: the single-right-hand-side row forms' value copies (group-major,
            # sliced) would take a third of a large hierarchy's memory for nothing
            opts.setdefault("row_form", 2)
            S = Solver(op["n"], op["row_ptr"], op["col"], op["val"], op["elem_dof"], op["p"],
                       stream=stream.cuda_stream, device_ptrs=0, **opts)
            S.set_device_ptrs(True)
        return S, stream

    def _free_bytes(self) -> int:
        free, _total = self.mem_info()
        return int(free)

    def _evict_for(self, need: int) -> bool:
        """Evict idle cached hierarchies (least recently used first) until `need` bytes fit next
        to the hierarchies that are being built (their memory is not allocated yet)."""
        released = False
        while self._free_bytes() - self.reserve - self._building_bytes < need:
            idle = [(e.last_used, k) for k, e in self.cache.items() if not e.busy]
            if not idle:
                if self.release_cache is None or released:
                    return False
                self.release_cache()  # right-hand-side blocks torch keeps cached are not free to the library
                released = True
                continue
            _, k = min(idle)
            e = self.cache.pop(k)
            e.solver.close()
            self.stats["evictions"] += 1
        return True

    def _never_fits(self, need: int) -> bool:
        """Under the lock, after _evict_for failed: nothing is cached, built or running, so no
        memory will be released and a request needing `need` bytes would wait forever."""
        return not self.cache and self._building_bytes == 0 and self._running == 0

    def _claim(self, key, req: Request):
        """Under the lock: the cached hierarchy for `key` (marked busy), a new placeholder entry
        that the caller must build, or None if memory does not allow a new one now."""
        e = self.cache.get(key)
        if e is not None:
            self.stats["cache_hits"] += 1
            e.busy = True
            return e, None
        if req.size is not None:  # materialised by _build, outside the lock
            op = req.make_operator
            nnz = int(req.size[1])
            need = estimate_bytes(int(req.size[0]), nnz, self.max_columns)
        else:
            op = req.make_operator()
            nnz = len(op["val"])
            need = estimate_bytes(op["n"], nnz, self.max_columns)
        if not self._evict_for(need):
            if self._never_fits(need):
                raise MemoryError(f"the operator needs about {need} bytes of device memory, {self._free_bytes()} "
                                  f"are free with nothing left to evict")
            self.stats["admission_waits"] += 1
            return None, None
        e = _Entry(None, None, need, nnz)
        e.busy = True
        self.cache[key] = e
        self._building_bytes += need
        return e, op

    def _build(self, key, e: _Entry, op) -> str | None:
        """Outside the lock: run the solver factory for a claimed placeholder (materialising the
        operator first when the request gave only its size); the error text, or None.  A failed
        build leaves no cache entry."""
        t0 = time.perf_counter()
        try:
            if callable(op):
                op = op()
            e.solver, e.stream = self.solver_factory(op)
            err = None
        except Exception as ex:
            err = f"setup failed: {ex}"
        with self.cv:
            self.stats["setup_ms"] += (time.perf_counter() - t0) * 1e3
            self._building_bytes -= e.nbytes
            if err is None:
                self.stats["setups"] += 1
            else:
                self.cache.pop(key, None)
                self.stats["setup_errors"] += 1
        return err

    # ------------------------------------------------------------------ requests
    def submit(self, req: Request):
        """Queue a request.  Its right-hand sides must be an n x r array with 1 <= r <= max_columns
        (ValueError otherwise, raised here: a malformed request never reaches a batch)."""
        rhs = req.rhs
        if not isinstance(rhs, np.ndarray) or rhs.ndim != 2 or not 1 <= rhs.shape[1] <= self.max_columns:
            shape = getattr(rhs, "shape", None)
            raise ValueError(f"request {req.rid}: rhs must be an n x r array with 1 <= r <= "
                             f"{self.max_columns}, got shape {shape}")
        with self.cv:
            req.arrival = self.clock() if req.arrival <= 0 else req.arrival
            # requests share a batch only when they share the operator, precision and tolerance
            self.pending.setdefault((req.key, req.precision, req.rtol), collections.deque()).append(req)
            self.cv.notify_all()

    def _next_batch(self):
        """Oldest waiting key whose hierarchy is not busy; its requests up to max_columns."""
        best = None
        for key, q in self.pending.items():
            if not q:
                continue
            e = self.cache.get(key[0])
            if e is not None and e.busy:
                continue
            if best is None or q[0].arrival < self.pending[best][0].arrival:
                best = key
        if best is None:
            return None, []
        q = self.pending[best]
        batch, cols = [], 0
        while q and cols + q[0].columns <= self.max_columns:
            r = q.popleft()
            batch.append(r)
            cols += r.columns
        if not q:
            del self.pending[best]
        return best, batch

    def _take(self, pkey):
        """Under the lock: the requests of pending key pkey for one batch (up to max_columns)."""
        q = self.pending[pkey]
        batch, cols = [], 0
        while q and cols + q[0].columns <= self.max_columns:
            r = q.popleft()
            batch.append(r)
            cols += r.columns
        if not q:
            del self.pending[pkey]
        return batch

    def _claim_group(self, pkey):
        """Under the lock: further waiting batches to solve with pkey's in one grouped solve -- the
        same precision and tolerance, hierarchies cached, built and idle (no setup in the group),
        all of them small (group_max_nnz) -- oldest first, up to max_group - 1; each is marked busy
        and given its batch id."""
        extra = []
        first = self.cache.get(pkey[0])
        if self.max_group <= 1 or pkey[1] != 1 or first is None or first.nnz > self.group_max_nnz:
            return extra
        for k in sorted((k for k, q in self.pending.items() if q and k != pkey and k[1:] == pkey[1:]),
                        key=lambda k: self.pending[k][0].arrival):
            if len(extra) >= self.max_group - 1:
                break
            e = self.cache.get(k[0])
            if e is None or e.busy or e.solver is None or e.nnz > self.group_max_nnz:
                continue
            batch = self._take(k)
            e.busy = True
            self.stats["cache_hits"] += 1
            self.batch_seq += 1
            self._running += 1
            extra.append((e, batch, self.batch_seq))
        return extra

    def _worker(self):
        while True:
            extra = []
            with self.cv:
                while True:
                    if self.closed and not any(self.pending.values()):
                        return
                    key, batch = self._next_batch()
                    if batch:
                        try:
                            e, op = self._claim(key[0], batch[0])
                        except Exception as ex:  # the operator could not even be described
                            self._fail(batch, f"setup failed: {ex}")
                            continue
                        if e is None:  # not enough memory now: put the batch back and wait
                            self.pending.setdefault(key, collections.deque()).extendleft(reversed(batch))
                            self.pending.move_to_end(key, last=False)
                            self.cv.wait(timeout=0.01)
                            continue
                        self.batch_seq += 1
                        self._running += 1
                        bid = self.batch_seq
                        extra = self._claim_group(key)
                        break
                    self.cv.wait(timeout=0.05)
            err = self._build(key[0], e, op) if op is not None else None
            if err is None:
                if extra:
                    self._run_group([(e, batch, bid)] + extra)
                else:
                    self._run(e, batch, bid)
            with self.cv:
                if err is not None:
                    self._fail(batch, err, bid)
                for ee, _, _ in [(e, batch, bid)] + extra:
                    ee.busy = False
                    self._running -= 1
                    ee.last_used = self.clock()
                if err is None:
                    for _, bb, _ in [(e, batch, bid)] + extra:
                        self.done.extend(bb)
                else:  # the group's other batches were not solved: back to the front of their queues
                    for _, bb, _ in extra:
                        q = self.pending.setdefault((bb[0].key, bb[0].precision, bb[0].rtol), collections.deque())
                        q.extendleft(reversed(bb))
                self.cv.notify_all()

    def _fail(self, batch: list, err: str, bid: int = -1):
        """Under the lock: finish every request of a batch with an error."""
        t = self.clock()
        for r in batch:
            r.start = r.start if r.start >= 0 else t
            r.finish, r.batch_id, r.error = t, bid, err
        self.done.extend(batch)
        self.stats["failed_requests"] += len(batch)
        self.cv.notify_all()

    def _default_runner(self, e: _Entry, B: np.ndarray, rtol: float, precision: int):
        """One multi-right-hand-side solve.  The batch is padded with zero columns to the next
        power of two (a zero column retires before the first iteration, and a column's bits do not
        depend on the batch width), so each hierarchy sees at most six batch shapes and reuses
        their captured CUDA graphs."""
        import torch
        m = B.shape[1]
        mp = 1 << (m - 1).bit_length()
        if mp > m:
            B = np.concatenate([B, np.zeros((B.shape[0], mp - m))], axis=1)
        with torch.cuda.stream(e.stream):
            Bd = torch.from_numpy(np.ascontiguousarray(B)).to(f"cuda:{self.device}")
            X, it, rr = e.solver.solve_batch(Bd, rtol=rtol, precision=precision)
            return X[:, :m].cpu().numpy(), it[:m], rr[:m]

    def _default_group_runner(self, items):
        """One grouped solve (giamg_solve_grouped) of several hierarchies' batches: items are
        (entry, B, rtol, precision) with one precision and tolerance; each B padded as in
        _default_runner.  Returns [(X, iters, relres, status)]."""
        import torch
        from . import solve_grouped
        e0 = items[0][0]
        Bs, ms = [], []
        with torch.cuda.stream(e0.stream):
            for e, B, rtol, precision in items:
                m = B.shape[1]
                mp = 1 << (m - 1).bit_length()
                if mp > m:
                    B = np.concatenate([B, np.zeros((B.shape[0], mp - m))], axis=1)
                Bs.append(torch.from_numpy(np.ascontiguousarray(B)).to(f"cuda:{self.device}"))
                ms.append(m)
            res = solve_grouped([it[0].solver for it in items], Bs, rtol=items[0][2])
            return [(X[:, :m].cpu().numpy(), it[:m], rr[:m], st) for (X, it, rr, st), m in zip(res, ms)]

    def _run_group(self, members: list):
        """Solve several hierarchies' batches in one grouped solve; each request gets its columns,
        iterations and residuals (or its member's error)."""
        t0 = self.clock()
        w0 = time.perf_counter()
        items, kept = [], []
        for e, batch, bid in members:
            rows = getattr(e.solver, "n", None)
            rows = batch[0].rhs.shape[0] if rows is None else rows
            ok = [r for r in batch if r.rhs.shape[0] == rows]
            for r in batch:
                if r.rhs.shape[0] != rows:
                    r.start, r.finish, r.batch_id = t0, self.clock(), bid
                    r.error = f"rhs has {r.rhs.shape[0]} rows, the operator {rows}"
                    with self.cv:
                        self.stats["failed_requests"] += 1
            if ok:
                items.append((e, np.concatenate([r.rhs for r in ok], axis=1), min(r.rtol for r in ok), ok[0].precision))
                kept.append((ok, bid))
        if not items:
            return
        try:
            res = self.group_runner(items)
            err = None
        except Exception as ex:  # a failed group fails its requests, not the server
            res, err = None, str(ex)
        t1 = self.clock()
        c_total = 0
        for i, (ok, bid) in enumerate(kept):
            merr = err
            if res is not None and res[i][3] not in (0, -8):  # GIAMG_OK, GIAMG_ERR_MAXITER
                merr = f"grouped solve failed (status {res[i][3]})"
            c = 0
            for r in ok:
                k = r.columns
                r.start, r.finish, r.batch_id, r.error = t0, t1, bid, merr
                if merr is None:
                    Xh, it, rr, _ = res[i]
                    r.x = Xh[:, c:c + k].copy()
                    r.iters = np.asarray(it[c:c + k]).copy()
                    r.relres = np.asarray(rr[c:c + k]).copy()
                c += k
            c_total += c
            if merr is not None:
                with self.cv:
                    self.stats["failed_requests"] += len(ok)
        with self.cv:
            self.stats["batches"] += len(kept)
            self.stats["grouped_solves"] += 1
            self.stats["grouped_batches"] += len(kept)
            self.stats["columns"] += c_total
            self.stats["solve_ms"] += (time.perf_counter() - w0) * 1e3

    def _run(self, e: _Entry, batch: list, bid: int):
        t0 = self.clock()
        w0 = time.perf_counter()
        # a request whose row count is not the operator's fails alone; the others are solved
        rows = getattr(e.solver, "n", None)
        rows = batch[0].rhs.shape[0] if rows is None else rows
        misfit = [r for r in batch if r.rhs.shape[0] != rows]
        batch = [r for r in batch if r.rhs.shape[0] == rows]
        for r in misfit:
            r.start, r.finish, r.batch_id = t0, self.clock(), bid
            r.error = f"rhs has {r.rhs.shape[0]} rows, the operator {rows}"
        if misfit:
            with self.cv:
                self.stats["failed_requests"] += len(misfit)
        if not batch:
            return
        prec = batch[0].precision
        rtol = min(r.rtol for r in batch)
        try:
            B = np.concatenate([r.rhs for r in batch], axis=1)
            Xh, it, rr = self.runner(e, B, rtol, prec)
            err = None
        except Exception as ex:  # a failed batch fails its requests, not the server
            Xh, it, rr, err = None, None, None, str(ex)
        t1 = self.clock()
        c = 0
        for r in batch:
            k = r.columns
            r.start, r.finish, r.batch_id, r.error = t0, t1, bid, err
            if err is None:
                r.x = Xh[:, c:c + k].copy()
                r.iters = np.asarray(it[c:c + k]).copy()
                r.relres = np.asarray(rr[c:c + k]).copy()
            c += k
        with self.cv:
            self.stats["batches"] += 1
            self.stats["columns"] += c
            self.stats["solve_ms"] += (time.perf_counter() - w0) * 1e3
            if err is not None:
                self.stats["failed_requests"] += len(batch)

    def drain(self, timeout: float = 600.0):
        """Wait until every submitted request is done."""
        t_end = time.perf_counter() + timeout
        with self.cv:
            while any(self.pending.values()) or any(e.busy for e in self.cache.values()) or self._running:
                left = t_end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError("server did not drain")
                self.cv.wait(timeout=min(left, 0.05))

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for w in self.workers:
            w.join(timeout=60)
        for e in self.cache.values():
            e.solver.close()
        self.cache.clear()


def latency_summary(requests: list) -> dict:
    ok = [r for r in requests if r.finish >= 0 and r.error is None]
    lat = sorted((r.finish - r.arrival) * 1e3 for r in ok)
    if not lat:
        return {}
    pick = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]  # noqa: E731
    span = max(r.finish for r in ok) - min(r.arrival for r in ok)
    cols = sum(r.columns for r in ok)
    return {"requests": len(lat), "solves": cols, "p50_ms": pick(0.5), "p99_ms": pick(0.99),
            "solves_per_s": cols / span if span > 0 else None, "makespan_s": span}


# ---------------------------------------------------------------------- synthetic request stream
STREAM_MESHES = (4, 6, 8)
STREAM_ORDERS = (2, 4, 6)
STREAM_LAMBDAS = (0.0, 1.0, 1000.0)


def _combine(K: np.ndarray, M: np.ndarray, lam: float, diag_rows: np.ndarray) -> np.ndarray:
    """K + lam M in chunks on host threads (numpy releases the GIL on large arrays), the Dirichlet
    identity rows (rows holding only their diagonal) reset to 1."""
    from concurrent.futures import ThreadPoolExecutor
    out = np.empty_like(K)
    step = max(1 << 22, (len(K) + 63) // 64)

    def part(lo):
        hi = min(lo + step, len(K))
        np.multiply(M[lo:hi], lam, out=out[lo:hi])
        np.add(out[lo:hi], K[lo:hi], out=out[lo:hi])

    with ThreadPoolExecutor(16) as ex:
        list(ex.map(part, range(0, len(K), step)))
    out[diag_rows] = 1.0
    return out


class _SharedOperator:
    """One mesh and order assembled once as stiffness K (lambda = 0) and mass M: the operator of
    any lambda is K + lambda M with the same pattern, formed when it is needed."""

    def __init__(self, n, p):
        import fegen
        self.K = fegen.make(n, p, mesh="jitter", mesh_seed=n, lam=0.0, rhs="none")
        mass = fegen.make(n, p, mesh="jitter", mesh_seed=n, lam=1.0, kappa=2, rhs="none")
        assert np.array_equal(mass.row_ptr, self.K.row_ptr) and np.array_equal(mass.col, self.K.col)
        self.M = mass.val
        mass.close()
        lens = np.diff(self.K.row_ptr)
        self.diag_rows = self.K.row_ptr[:-1][lens == 1]  # value index of each identity row's diagonal
        self.n, self.nnz, self.p = self.K.n, self.K.nnz, self.K.p
        self._basis = None

    def values(self, lam):
        return self.K.val.copy() if lam == 0.0 else _combine(self.K.val, self.M, lam, self.diag_rows)

    def rhs_nodal(self, seeds):
        """prob.rhs_nodal(seed) for each seed (the same Fourier fields at the nodes, c ~ N(0, 1)
        from numpy's PCG64 with that seed), as one product with a table of the 64 mode products at
        the nodes, built once per mesh and order: n x len(seeds)."""
        if self._basis is None:
            k = np.arange(1, 5)[:, None] * np.pi
            sx, sy, sz = (np.sin(k * self.K.coords[None, :, d]) for d in range(3))  # 4 x n each
            T = (sx[:, None, None, :] * sy[None, :, None, :]) * sz[None, None, :, :]
            self._basis = T.reshape(64, self.n)
        C = np.stack([np.random.default_rng(sd).standard_normal((4, 4, 4)).ravel() for sd in seeds])
        F = (C @ self._basis).T.copy()
        F[self.K.boundary != 0, :] = 0.0
        return F

    def close(self):
        self.K.close()


def synthetic_stream(n_requests: int = 128, seed: int = 7, rate_per_s: float = 200.0, max_rhs: int = 8,
                     meshes=STREAM_MESHES, orders=STREAM_ORDERS, lambdas=STREAM_LAMBDAS, rhs_kind: str = "fourier"):
    """Requests for Helmholtz / Poisson operators on jittered hex meshes (mesh seed = mesh size, so
    a (mesh, order, lambda) triple always names the same operator), 1..max_rhs smooth Fourier
    right-hand sides seeded by request id (rhs_kind "fourier": loaded by quadrature; "nodal": the
    same fields evaluated at the nodes, for large streams: the operators of one mesh and order
    then share one stiffness and one mass matrix on the host, each lambda's values formed when the
    server builds that operator), Poisson arrivals (exponential gaps) at rate_per_s."""
    import fegen
    if rhs_kind == "nodal":
        return _shared_stream(n_requests, seed, rate_per_s, max_rhs, meshes, orders, lambdas)
    rng = np.random.default_rng(seed)
    ops = {}

    def operator(n, p, lam):
        key = (n, p, lam)
        if key not in ops:
            prob = fegen.make(n, p, mesh="jitter", mesh_seed=n, lam=lam, rhs="none")
            ops[key] = prob
        return ops[key]

    t = 0.0
    reqs = []
    for rid in range(n_requests):
        n = int(rng.choice(meshes))
        p = int(rng.choice(orders))
        lam = float(rng.choice(lambdas))
        r = int(rng.integers(1, max_rhs + 1))
        t += float(rng.exponential(1.0 / rate_per_s))
        prob = operator(n, p, lam)
        load = prob.rhs_nodal if rhs_kind == "nodal" else (lambda sd, prob=prob: prob.rhs("fourier", sd))
        rhs = np.stack([load(100000 + 64 * rid + j) for j in range(r)], axis=1)
        k = 3 if lam > 0 else 2

        def make(prob=prob, k=k):
            return dict(n=prob.n, row_ptr=prob.row_ptr, col=prob.col, val=prob.val, elem_dof=prob.elem_dof,
                        p=prob.p, cheb_degree=k)
        reqs.append(Request(rid=rid, key=(f"jitter{n}^3", p, lam), make_operator=make, rhs=rhs, arrival=t))
    return reqs, ops


def _shared_stream(n_requests, seed, rate_per_s, max_rhs, meshes, orders, lambdas):
    """synthetic_stream's draws (the same mesh, order, lambda, column count and arrival of every
    request) with operators shared across lambda and nodal right-hand sides."""
    rng = np.random.default_rng(seed)
    shared = {}
    t = 0.0
    reqs, keys = [], set()
    for rid in range(n_requests):
        n = int(rng.choice(meshes))
        p = int(rng.choice(orders))
        lam = float(rng.choice(lambdas))
        r = int(rng.integers(1, max_rhs + 1))
        t += float(rng.exponential(1.0 / rate_per_s))
        if (n, p) not in shared:
            shared[(n, p)] = _SharedOperator(n, p)
        so = shared[(n, p)]
        rhs = so.rhs_nodal([100000 + 64 * rid + j for j in range(r)])
        k = 3 if lam > 0 else 2

        def make(so=so, lam=lam, k=k):
            return dict(n=so.n, row_ptr=so.K.row_ptr, col=so.K.col, val=so.values(lam), elem_dof=so.K.elem_dof,
                        p=so.p, cheb_degree=k)
        keys.add((n, p, lam))
        reqs.append(Request(rid=rid, key=(f"jitter{n}^3", p, lam), make_operator=make, rhs=rhs, arrival=t,
                            size=(so.n, so.nnz)))
    return reqs, {key: shared[key[:2]] for key in sorted(keys)}


def run_stream(server: Server, reqs: list, time_scale: float = 1.0, drain_timeout: float = 600.0):
    """Submit the requests at their arrival times (relative to now) and wait for all of them
    (TimeoutError if they are not all done drain_timeout seconds after the last submission)."""
    t0 = server.clock()
    offs = [r.arrival for r in reqs]
    for r, off in zip(reqs, offs):
        target = t0 + off * time_scale
        while server.clock() < target:
            time.sleep(min(0.001, max(0.0, target - server.clock())))
        r.arrival = 0.0
        server.submit(r)
    server.drain(drain_timeout)
    return latency_summary(reqs)
