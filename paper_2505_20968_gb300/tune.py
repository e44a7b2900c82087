"""Measured choice of the preconditioner's inner sweep count m_in (Sect. 5.2:
P^-1 is applied as m_in Richardson sweeps with App. F's block inverse).

More sweeps make P^-1 a better inverse of P and cut GMRES iterations, but cost
one Lambda* Sigma* application each.  The best count depends on the atmosphere,
so it is measured: every candidate runs a short solve from zero, and the one
with the fastest decay of the true residual per second is kept.
"""
import math
import time


def _cuda_clock():
    import torch
    torch.cuda.synchronize()
    return time.perf_counter()


def tune_precond_sweeps(P, candidates=(1, 2, 3), probe_iters=40, restart=60, tol=1e-12, clock=None):
    """Set on P, and return, the m_in of `candidates` with the fastest residual
    decay: -log10(true relative residual) per second over a solve of at most
    probe_iters iterations.  Returns (m_in, {m: (decades_per_s, iters, seconds, residual)})."""
    clock = clock or _cuda_clock
    results = {}
    best = None
    for m in candidates:
        P.set_precond_sweeps(m)
        t0 = clock()
        _, info = P.solve(tol=tol, max_iter=probe_iters, restart=restart, check=False)
        dt = max(clock() - t0, 1e-9)
        res = max(float(info["true_rel_res"]), 1e-300)
        rate = -math.log10(res) / dt
        results[m] = (rate, int(info["iters"]), dt, res)
        if best is None or rate > results[best][0]:
            best = m
    P.set_precond_sweeps(best)
    return best, results
