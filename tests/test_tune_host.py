"""Host logic of the Chebyshev-degree tuner: the fastest degree that reaches the tolerance wins
and is left set on the solver (a fake solver and timer stand in for the GPU)."""
import paper_2512_15121_gb300.tune as tune


class FakeSolver:
    """Degree k: iterations and time per solve from tables; degree 1 misses the tolerance."""
    ITERS = {1: 40, 2: 12, 3: 9, 4: 7, 5: 6}
    MS = {1: 20.0, 2: 28.6, 3: 27.7, 4: 26.4, 5: 26.8}

    def __init__(self):
        self.k = 3
        self.calls = []

    def set_cheb_degree(self, k):
        self.k = k

    def solve(self, b, rtol, precision):
        self.calls.append(self.k)
        rr = 1e-6 if self.k == 1 else 0.5 * rtol
        return None, self.ITERS[self.k], rr


def test_fastest_degree_that_reaches_rtol_is_kept():
    S = FakeSolver()
    timer = lambda fn: (fn(), FakeSolver.MS[S.k])
    best, timings = tune.tune_cheb_degree(S, None, degrees=(1, 2, 3, 4, 5), rtol=1e-8, reps=3, warmup=1,
                                          timer=timer)
    # degree 1 is the fastest per solve but misses rtol; of the others 4 is fastest
    assert best == 4 and S.k == 4
    assert [t.degree for t in timings] == [1, 2, 3, 4, 5]
    assert [t.iterations for t in timings] == [40, 12, 9, 7, 6]
    assert timings[3].ms == 26.4
    # warm-up plus timed solves for every degree, in order
    assert S.calls == [k for k in (1, 2, 3, 4, 5) for _ in range(4)]


def test_when_no_degree_reaches_rtol_the_fastest_is_kept():
    S = FakeSolver()
    best, _ = tune.tune_cheb_degree(S, None, degrees=(1,), rtol=1e-8, reps=1, warmup=0,
                                    timer=lambda fn: (fn(), 1.0))
    assert best == 1 and S.k == 1
