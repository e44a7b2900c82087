"""Measured choices of the solver's schedule parameters.

* The preconditioner's inner sweep count m_in (Sect. 5.2: P^-1 is applied as
  m_in Richardson sweeps with App. F's block inverse).
* The tile-ring depth of the tensor-core R_II contraction (how many tile K
  steps are in flight per SM), per problem shape: the deepest ring that fits
  is not always the fastest, since a shallower one leaves the thread blocks
  the same work but less shared memory to contend for.

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


def tune_tile_stages(P, candidates=(0, 2, 3, 4, 5), reps=3, clock=None):
    """Set on P, and return, the tile-ring depth of `candidates` (0 = the
    deepest that fits; larger values are capped by the library) with the
    shortest operator apply, timed over `reps` applies after one warm-up.
    Returns (depth, {depth: ms per apply})."""
    clock = clock or _cuda_clock
    x = P.empty().fill_(1.0) if hasattr(P, "empty") else None
    results = {}
    best = None
    for st in candidates:
        P.set_tile_stages(st)
        y = P.apply_operator(x)
        t0 = clock()
        for _ in range(reps):
            y = P.apply_operator(x, y)
        ms = (clock() - t0) * 1e3 / reps
        results[st] = ms
        if best is None or ms < results[best]:
            best = st
    P.set_tile_stages(best)
    return best, results
