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


class FakeKernelSolver:
    """Row kernels and batch rows: times per choice from tables; one form misses the tolerance."""
    MS = {(0, 0): 10.0, (1, 16): 12.0, (5, 0): 9.0, (6, 0): 8.0, (2, 8): 7.0}
    BMS = {1: 5.0, 2: 4.0}

    def __init__(self):
        self.form = {0: (0, 0), 1: (0, 0)}
        self.rows = {}
        self.log = []

    def set_row_kernel(self, level, precision, form, threads=0):
        self.form[precision] = (form, threads)
        self.log.append(("set", level, precision, form, threads))

    def kernel(self, level, precision):
        return (1, "sliced") if self.form[precision][0] == 6 else (32, "other")

    def solve(self, b, rtol, precision):
        rr = 1e-6 if self.form[precision] == (2, 8) else 0.5 * rtol  # (2, 8) is fast but wrong
        return None, 9, rr

    def set_batch_rows(self, level, rows):
        self.rows[level] = rows

    def solve_batch(self, B, rtol, precision):
        import numpy as np
        return None, np.array([11, 12]), np.array([1e-9, 2e-9])


def test_row_kernel_tuner_keeps_the_fastest_valid_choice():
    S = FakeKernelSolver()
    timer = lambda fn: (fn(), FakeKernelSolver.MS[S.form[1]])
    cands = ((0, 0), (1, 16), (2, 8), (5, 0), (6, 0))
    best, timings = tune.tune_row_kernels(S, None, precision=1, candidates=cands, reps=2, warmup=1, timer=timer)
    # (2, 8) is fastest but misses rtol; of the rest the sliced form (6, 0) wins and stays set
    assert best == (6, 0) and S.form[1] == (6, 0) and S.form[0] == (0, 0)
    assert [t.choice for t in timings] == list(cands)
    assert timings[-1].kernel == (1, "sliced") and timings[0].ms == 10.0
    assert S.log[-1] == ("set", 0, 1, 6, 0)


def test_batch_rows_tuner_sets_every_level():
    S = FakeKernelSolver()
    timer = lambda fn: (fn(), FakeKernelSolver.BMS[S.rows[0]])
    best, timings = tune.tune_batch_rows(S, None, choices=(1, 2), levels=(0, 1), reps=1, warmup=0, timer=timer)
    assert best == 2 and S.rows == {0: 2, 1: 2}
    assert [t.iterations for t in timings] == [12, 12] and timings[0].ms == 5.0
