"""Chebyshev-degree tuning by measured time to solution.

The paper fixes the smoother degree per problem class (3 for Helmholtz, 2 for the flow
operators, Sec. 3) and compares degrees by V-cycle time and iteration count (Sec. 3.2.2).  A
higher degree costs more products per V-cycle and saves iterations; which wins depends on the
operator and on how fast the products run.  `tune_cheb_degree` times the whole solve for each
candidate degree on the same hierarchy (giamg_set_cheb_degree keeps the setup) and keeps the
fastest.
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
