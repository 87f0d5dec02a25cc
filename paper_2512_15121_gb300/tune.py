"""Tuning by measured time to solution: every candidate is timed as whole solves on the same
hierarchy, never as an isolated kernel.

* The smoother degree.  The paper fixes it per problem class (3 for Helmholtz, 2 for the flow
  operators, Sec. 3) and compares degrees by V-cycle time and iteration count (Sec. 3.2.2).  A
  higher degree costs more products per V-cycle and saves iterations; which wins depends on the
  operator and on how fast the products run.  `tune_cheb_degree` times the solve for each
  degree (giamg_set_cheb_degree keeps the setup) and keeps the fastest.
* The finest level's row kernel (form and threads per row), per precision: `tune_row_kernels`
  (giamg_set_row_kernel).
* The multi-right-hand-side FP32 products' rows per work item: `tune_batch_rows`
  (giamg_set_batch_rows), timed as whole multi-RHS solves.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass
class DegreeTiming:
    degree: int
    iterations: int
    relres: float
    ms: float  # median solve time


def _cuda_event_timer(fn):
    """Run fn() between two CUDA events on the current stream; (fn's result, milliseconds)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = fn()
    e1.record()
    torch.cuda.synchronize()
    return res, e0.elapsed_time(e1)


def tune_cheb_degree(solver, b, degrees=(1, 2, 3, 4, 5), precision: int = 1, rtol: float = 1e-8,
                     reps: int = 5, warmup: int = 2, timer=None):
    """Time solves of A x = b for each smoother degree, set the fastest one that reaches rtol on
    the solver and return (best degree, [DegreeTiming, ...]).  b: a device vector of the solver's
    pointer mode.  Times are CUDA-event medians on the current stream (`timer` replaces the
    CUDA-event timer: a function of a callable returning (its result, milliseconds))."""
    import statistics

    timer = timer or _cuda_event_timer
    out = []
    for k in degrees:
        solver.set_cheb_degree(k)
        for _ in range(warmup):
            solver.solve(b, rtol=rtol, precision=precision)
        ts = []
        for _ in range(reps):
            (_, it, rr), ms = timer(lambda: solver.solve(b, rtol=rtol, precision=precision))
            ts.append(ms)
        out.append(DegreeTiming(k, int(it), float(rr), statistics.median(ts)))
    ok = [t for t in out if t.relres <= rtol]
    best = min(ok or out, key=lambda t: t.ms)
    solver.set_cheb_degree(best.degree)
    return best.degree, out


@dataclasses.dataclass
class KernelTiming:
    choice: tuple        # (form, threads) for row kernels, (rows_per_item,) for batch rows
    kernel: tuple        # what ran: giamg_level_kernel's (threads per row, form name), or ()
    iterations: int
    relres: float
    ms: float


def _time_solves(fn, reps, warmup, timer):
    import statistics
    for _ in range(warmup):
        fn()
    ts, res = [], None
    for _ in range(reps):
        res, ms = timer(fn)
        ts.append(ms)
    return res, statistics.median(ts)


ROW_CANDIDATES = ((0, 0), (1, 16), (1, 32), (2, 8), (2, 32), (4, 0), (5, 0), (6, 0))


def tune_row_kernels(solver, b, precision: int = 1, candidates=ROW_CANDIDATES, rtol: float = 1e-8, reps: int = 5,
                     warmup: int = 2, level: int = 0, timer=None):
    """Time whole solves of A x = b (precision 0 FP64 or 1 FP32 V-cycle) with each row-kernel
    candidate (form, threads) on `level` for that precision -- the precision's own V-cycle levels
    and, for precision 1, its FP32 products; set the fastest that reaches rtol and return
    ((form, threads), [KernelTiming, ...]).  A candidate whose form does not apply runs the
    level's default kernel and is timed as what ran."""
    timer = timer or _cuda_event_timer
    out = []
    for form, threads in candidates:
        solver.set_row_kernel(level, precision, form, threads)
        (_, it, rr), ms = _time_solves(lambda: solver.solve(b, rtol=rtol, precision=precision), reps, warmup, timer)
        out.append(KernelTiming((form, threads), tuple(solver.kernel(level, precision)), int(it), float(rr), ms))
    ok = [t for t in out if t.relres <= rtol]
    best = min(ok or out, key=lambda t: t.ms)
    solver.set_row_kernel(level, precision, *best.choice)
    return best.choice, out


def tune_batch_rows(solver, B, precision: int = 1, choices=(1, 2), rtol: float = 1e-8, reps: int = 3,
                    warmup: int = 1, levels=(0,), timer=None):
    """Time whole multi-right-hand-side solves of the n x m block B with each rows-per-item choice
    of the FP32 products on `levels`; set the fastest whose columns all reach rtol and return
    (rows_per_item, [KernelTiming, ...])."""
    timer = timer or _cuda_event_timer
    out = []
    for rows in choices:
        for l in levels:
            solver.set_batch_rows(l, rows)
        (_, it, rr), ms = _time_solves(lambda: solver.solve_batch(B, rtol=rtol, precision=precision), reps, warmup,
                                       timer)
        out.append(KernelTiming((rows,), (), int(max(it)), float(max(rr)), ms))
    ok = [t for t in out if t.relres <= rtol]
    best = min(ok or out, key=lambda t: t.ms)
    for l in levels:
        solver.set_batch_rows(l, best.choice[0])
    return best.choice[0], out
