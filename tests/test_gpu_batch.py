"""S12: batched solve of independent ragged instances (prd_solve_batch).

Each instance of a batch must give the solution its own prd_solve gives: in
FP64 mode to 1e-9 relative (both are converged to 1e-12; they differ only by
the order of floating-point atomics), in FP32 mode to the refinement's
accuracy on emergent I; and every instance must match the oracle's solution
(tests/golden/twolevel.npz, batch_*.npz): FP64 within 1e-8, FP32 emergent I
within 1e-5 relative and Q/I, U/I, V/I within 1e-4 absolute.
"""
import os
import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ragged(prec):
    cfgs = [inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2),
            inputs.mgii(n_z=7, n_core_each=7, n_wing=6, n_mu_half=2, n_chi=4, seed=401),
            inputs.mgii(n_z=9, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=402),
            inputs.hi_lya(n_z=6, n_core=9, n_wing=6, n_mu_half=2, n_chi=4, seed=403)]
    from paper_2505_20968_gb300.binding import PRD
    return [PRD(c, precision=prec, device=0) for c in cfgs]


@pytest.mark.parametrize("prec,tol,agree", [("fp64", 1e-12, 1e-9), ("fp32", 1e-10, 2e-5)])
def test_batch_matches_single_solves(prec, tol, agree):
    from paper_2505_20968_gb300.binding import solve_batch
    Ps = _ragged(prec)
    xs, infos = solve_batch(Ps, tol=tol, max_iter=800, restart=60)
    for P, x, info in zip(Ps, xs, infos):
        assert info["rc"] == 0 and info["true_rel_res"] < tol, info
        ref, rinfo = P.solve(tol=tol, max_iter=800, restart=60)
        a, b = x.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        top = P.mu > 0
        d = np.max(np.abs(a[-1, top, :, 0] - b[-1, top, :, 0]) / np.abs(b[-1, top, :, 0]))
        assert d < agree, (P.shape, d)
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for P, x, name in zip(Ps, xs, ("twolevel", "batch_mgii7", "batch_mgii9", "batch_hi6")):
        ref = np.load(os.path.join(gold, name + ".npz"))["sol"]
        a = x.cpu().numpy().astype(np.float64)
        if prec == "fp64":
            assert np.max(np.abs(a - ref)) / np.max(np.abs(ref)) < 1e-8, name
        else:
            top = P.mu > 0
            g, o = a[-1, top], ref[-1, top]
            assert np.max(np.abs(g[..., 0] - o[..., 0]) / o[..., 0]) < 1e-5, name
            for s_ in (1, 2, 3):
                assert np.max(np.abs(g[..., s_] / g[..., 0] - o[..., s_] / o[..., 0])) < 1e-4, name
    for P in Ps:
        P.close()


def test_batch_rejects_repeated_ctx():
    from paper_2505_20968_gb300.binding import PRD, lib
    import ctypes
    P = PRD(inputs.twolevel_slab(n_z=6, n_x=9, n_mu_half=1, n_chi=4, eps=1e-2), device=0)
    x = P.empty()
    hs = (ctypes.c_void_p * 2)(P.h, P.h)
    xs = (ctypes.c_void_p * 2)(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()))
    assert lib().prd_solve_batch(hs, 2, 1e-8, 10, 10, xs, None, None, None) == -1   # PRD_E_ARG
    P.close()
