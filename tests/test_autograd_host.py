"""The autograd wrapper of the adjoint gradient (binding.solve_with_field), on
the host with a stand-in solver of known derivative: the field reaches the
problem set-up, the upstream gradient dJ/dI reaches grad_B, and grad_B's
result becomes the field's gradient (checked against torch's own autograd of
the same stand-in)."""
import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")

_W = np.random.default_rng(3).uniform(0.5, 1.5, (2, 3, 4))
_C = np.array([0.7, -1.3, 0.4])


class _Quadratic:
    """x[z, o, n, s] = W[o, n, s] sum_k C_k p[z, k]^2, with p the field."""
    made = []

    def __init__(self, cfg):
        a = cfg["atm"]
        self.p = np.stack([a["B_G"], a["thetaB"], a["chiB"]], 1)
        self.closed = False
        _Quadratic.made.append(self)

    def solve(self, tol, max_iter, restart):
        x = _W[None] * ((self.p ** 2) @ _C)[:, None, None, None]
        return torch.from_numpy(x), {}

    def grad_B(self, x, gx):
        assert gx.is_contiguous() and gx.shape == x.shape
        s = np.einsum("zons,ons->z", gx.numpy(), _W)
        return 2.0 * _C[None, :] * self.p * s[:, None]

    def close(self):
        self.closed = True


def test_field_gradient_reaches_the_field():
    from paper_2505_20968_gb300.binding import solve_with_field
    cfg = inputs.mgii(n_z=5, n_core_each=3, n_wing=4, n_mu_half=1, n_chi=4, seed=9)
    p0 = np.stack([cfg["atm"]["B_G"], cfg["atm"]["thetaB"], cfg["atm"]["chiB"]], 1) * 1.1
    field = torch.tensor(p0, requires_grad=True)
    x = solve_with_field(cfg, field, make=_Quadratic)
    P = _Quadratic.made[-1]
    assert np.array_equal(P.p, p0)                        # the field reached the set-up
    v = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, tuple(x.shape)))
    (x[:, :, 1:] * v[:, :, 1:]).sum().backward()          # a non-contiguous upstream gradient
    assert P.closed
    ref_field = torch.tensor(p0, requires_grad=True)
    xr = torch.from_numpy(_W)[None] * ((ref_field ** 2) @ torch.from_numpy(_C))[:, None, None, None]
    (xr[:, :, 1:] * v[:, :, 1:]).sum().backward()
    assert torch.allclose(field.grad, ref_field.grad, rtol=1e-14, atol=0)
