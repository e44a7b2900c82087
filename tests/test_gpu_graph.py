"""S10/S12: the GMRES iteration as one CUDA-graph launch (PRD_OPT_GRAPH).

The Arnoldi step (operator, preconditioner, both Gram-Schmidt passes, the
rotation kernel and the next basis vector, step index on the device) is
captured once per context and replayed.  With the graph on, every Arnoldi
iteration is one graph launch (the launch counter grows by the iteration
count); the solution equals the one from direct launches of the same kernels
(FP64: 1e-12 relative, the order of the FP64 atomics in the reductions being
the only difference), with the same iteration count; and the oracle's solution
is met (FP64 two-level slab within 1e-8).  A batched solve replays one graph
per instance, each on its own stream.
"""
import os

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _twolevel():
    return inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2)


def test_graph_step_matches_direct_launches_fp64():
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(_twolevel(), precision="fp64", device=0)
    n0 = P.graph_launches()
    xg, ig = P.solve(tol=1e-12, max_iter=400, restart=30)
    n1 = P.graph_launches()
    assert n1 - n0 == ig["iters"] > 0, (n0, n1, ig)
    P.set_graph(False)
    xd, idr = P.solve(tol=1e-12, max_iter=400, restart=30)
    assert P.graph_launches() == n1                      # direct launches only
    assert idr["iters"] == ig["iters"]
    a, b = xg.cpu().numpy(), xd.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    ref = np.load(os.path.join(GOLD, "twolevel.npz"))["sol"]
    assert np.max(np.abs(a - ref)) / np.max(np.abs(ref)) < 1e-8
    P.set_graph(True)                                    # re-captured on the next solve
    x2, i2 = P.solve(tol=1e-12, max_iter=400, restart=30)
    assert P.graph_launches() - n1 == i2["iters"]
    P.close()


def test_graph_step_in_refined_fp32_and_adjoint_solves():
    """FP32 mode: the inner GMRES iterations of the refinement are graph
    launches (one per apply), and the adjoint solve captures its own graph
    (the transposed operator) beside the forward one."""
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(inputs.mgii(n_z=7, n_core_each=7, n_wing=6, n_mu_half=2, n_chi=4, seed=401), precision="fp32", device=0)
    n0 = P.graph_launches()
    x, info = P.solve(tol=1e-10, max_iter=600, restart=60)
    assert P.graph_launches() - n0 == info["iters"] > 0
    ref = np.load(os.path.join(GOLD, "batch_mgii7.npz"))["sol"]
    top = P.mu > 0
    g, o = x.cpu().numpy().astype(np.float64)[-1, top], ref[-1, top]
    assert np.max(np.abs(g[..., 0] - o[..., 0]) / o[..., 0]) < 1e-5
    P.close()
    Q = PRD(_twolevel(), precision="fp64", device=0)
    g = torch.from_numpy(inputs.seeded_vector(Q.shape, 9, 0.1, 1.0)).to(Q.device, Q.dtype)
    n0 = Q.graph_launches()
    lam, info = Q.solve_adjoint(g, tol=1e-11, max_iter=400, restart=30)
    assert Q.graph_launches() - n0 == info["iters"] > 0
    Q.set_graph(False)
    lam2, info2 = Q.solve_adjoint(g, tol=1e-11, max_iter=400, restart=30)
    a, b = lam.cpu().numpy(), lam2.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))
    Q.close()


def test_batch_replays_one_graph_per_instance():
    from paper_2505_20968_gb300.binding import PRD, solve_batch
    Ps = [PRD(_twolevel(), precision="fp64", device=0),
          PRD(inputs.twolevel_slab(n_z=10, n_x=13, n_mu_half=2, n_chi=4, eps=1e-3, seed=5), precision="fp64",
              device=0)]
    n0 = [P.graph_launches() for P in Ps]
    xs, infos = solve_batch(Ps, tol=1e-12, max_iter=400, restart=30)
    for P, k, info in zip(Ps, n0, infos):
        assert info["rc"] == 0 and P.graph_launches() - k == info["iters"] > 0, info
    for P in Ps:
        P.close()
