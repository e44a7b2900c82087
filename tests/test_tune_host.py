"""The measured choice of the preconditioner sweep count (tune.py), on the host
with a stand-in solver and clock: the candidate with the fastest residual
decay per second is kept and left set on the solver."""
from paper_2505_20968_gb300.tune import tune_precond_sweeps


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class _Solver:
    """m sweeps: each iteration costs (1 + m) time units and gains 0.1 (1 + 4 m) / (1 + m^2)
    decades, so m = 1 decays fastest per unit time (0.125 decades per unit; m = 0: 0.1)."""
    def __init__(self, clock):
        self.clock, self.m, self.calls = clock, None, []

    def set_precond_sweeps(self, m):
        self.m = m

    def solve(self, tol, max_iter, restart, check):
        assert check is False and max_iter == 40
        m = self.m
        self.clock.t += max_iter * (1 + m)
        self.calls.append(m)
        return None, {"true_rel_res": 10.0 ** (-max_iter * 0.1 * (1 + 4 * m) / (1 + m * m)), "iters": max_iter}


def test_fastest_decay_is_chosen_and_set():
    clock = _Clock()
    S = _Solver(clock)
    best, res = tune_precond_sweeps(S, candidates=(0, 1, 2, 3), clock=clock)
    rates = {m: r[0] for m, r in res.items()}
    assert best == max(rates, key=rates.get) == 1
    assert S.m == 1 and S.calls == [0, 1, 2, 3]
