"""S13 through torch autograd: binding.solve_with_field, the
torch.autograd.Function whose forward is prd_solve for a given magnetic field
and whose backward is the adjoint gradient prd_grad_B, against central
differences of the oracle's forward solves (tests/golden/grad_mgii_small.npz).
"""
import os

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_autograd_field_gradient_matches_oracle():
    """J = sum of the emergent intensities of the top layer on a small Mg II
    case, as in the gradient test of test_gpu_adjoint.py; its gradient taken by
    torch autograd through solve_with_field, against the Richardson combination
    of the oracle's central differences at h and h/2; bound 2e-4 of the largest
    component of each kind (prd_grad_B called directly measured <= 2.4e-5)."""
    from paper_2505_20968_gb300.binding import PRD, solve_with_field
    G = dict(np.load(os.path.join(GOLD, "grad_mgii_small.npz")))
    cfg = inputs.mgii(n_z=6, n_core_each=5, n_wing=4, n_mu_half=1, n_chi=4, seed=23)
    P = PRD(cfg, precision="fp64", device=0)
    top = torch.from_numpy(P.mu > 0)
    P.close()
    a = cfg["atm"]
    field = torch.tensor(np.stack([a["B_G"], a["thetaB"], a["chiB"]], 1), dtype=torch.float64,
                         requires_grad=True)
    x = solve_with_field(cfg, field)
    x[-1, top.to(x.device), :, 0].sum().backward()
    g = field.grad.numpy()
    fd = (4.0 * G["fd_half"] - G["fd"]) / 3.0
    for k, kind in enumerate(("B", "theta_B", "chi_B")):
        d = np.max(np.abs(g[:, k] - fd[:, k])) / np.max(np.abs(fd[:, k]))
        print(f"autograd dJ/d{kind}: {d:.2e}")
        assert d < 2e-4, f"dJ/d{kind}: {d:.2e}"
