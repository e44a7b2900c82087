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


class _Applier:
    """Apply time per ring depth: 5 units for the deepest (0), depth 3 fastest."""
    cost = {0: 5.0, 2: 6.0, 3: 4.0, 4: 4.5, 5: 5.0}

    def __init__(self, clock):
        self.clock, self.st, self.set_calls = clock, None, []

    def set_tile_stages(self, n):
        self.st = n
        self.set_calls.append(n)

    def apply_operator(self, x, out=None):
        self.clock.t += self.cost[self.st] * 1e-3
        return out


def test_fastest_tile_ring_is_chosen_and_set():
    from paper_2505_20968_gb300.tune import tune_tile_stages
    clock = _Clock()
    A = _Applier(clock)
    best, res = tune_tile_stages(A, clock=clock)
    assert best == 3 and A.st == 3
    assert abs(res[3] - 4.0) < 1e-9 and abs(res[2] - 6.0) < 1e-9
