"""prd_set_allocator: the library's device memory from PyTorch's caching
allocator gives the same results as cudaMalloc'd memory, and is returned to
the allocator when the context is destroyed."""
import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 4e-6)])
def test_torch_allocator_same_results(prec, tol):
    from paper_2505_20968_gb300.binding import PRD
    cfg = (inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2) if prec == "fp64" else
           inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31))
    Pt = PRD(cfg, precision=prec, device=0, allocator="torch")
    held = sum(Pt.alloc_stats["live"].values())
    assert held >= Pt.workspace_bytes() > 0, (held, Pt.workspace_bytes())
    Pd = PRD(cfg, precision=prec, device=0)
    x = torch.from_numpy(inputs.seeded_vector(Pt.shape, 9, 0.1, 1.0)).to(device=Pt.device, dtype=Pt.dtype)
    a = Pt.apply_operator(x).double()
    b = Pd.apply_operator(x).double()
    assert float((a - b).abs().max() / b.abs().max()) < tol
    xa, ia = Pt.solve(tol=1e-10, max_iter=400, restart=60)
    xb, ib = Pd.solve(tol=1e-10, max_iter=400, restart=60)
    assert ia["true_rel_res"] < 1e-10 and ib["true_rel_res"] < 1e-10
    d = (xa.double() - xb.double()).abs().max() / xb.double().abs().max()
    assert float(d) < (1e-8 if prec == "fp64" else 1e-5)
    stats = Pt.alloc_stats
    Pt.close()
    Pd.close()
    assert stats["bytes"] > held and not stats["live"]     # solve temporaries too; all handed back
