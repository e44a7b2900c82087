"""S13: the transposed operator and the adjoint solve, through the C ABI.

A^T is fixed by A, and A is pinned to the oracle (test_gpu_parity.py), so the
transpose is checked by the identity <y, A x> = <A^T y, x> on seeded vectors
(a property of any size), in FP64 mode on the two-level slab and on the
two-term Mg II and H I physics.  The adjoint solve is checked by its residual
and by <g, x> = <lam, b> for A x = b and A^T lam = g.
"""
import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "twolevel": lambda: inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2),
    "mgii": lambda: inputs.mgii(n_z=10, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=21),
    "hi": lambda: inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31),
    "hi_aa": lambda: inputs.hi_lya(n_z=8, n_core=11, n_wing=6, n_mu_half=2, n_chi=4, seed=32,
                                   mode=inputs.MODE_AA),
}


def _vec(P, seed):
    v = inputs.seeded_vector(P.shape, seed, 0.1, 1.0)
    v[..., 1:] = v[..., 1:] * 0.1 - 0.05
    return torch.from_numpy(np.ascontiguousarray(v)).to(device=P.device, dtype=P.dtype)


def _dot(a, b):
    return float(torch.sum(a.double() * b.double()).item())


@pytest.mark.parametrize("name", ["twolevel", "mgii", "hi", "hi_aa"])
def test_adjoint_identity_fp64(name):
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(CASES[name](), precision="fp64", device=0)
    for sx, sy in ((1, 2), (3, 4)):
        x, y = _vec(P, sx), _vec(P, sy)
        Ax = P.apply_operator(x)
        ATy = P.apply_operator_T(y)
        lhs, rhs = _dot(y, Ax), _dot(ATy, x)
        scale = float(torch.linalg.norm(y.double()) * torch.linalg.norm(Ax.double()))
        assert abs(lhs - rhs) < 1e-12 * scale, (lhs, rhs, scale)
    P.close()


@pytest.mark.parametrize("name", ["mgii", "hi"])
def test_adjoint_identity_fp32_mode(name):
    """FP32 mode: A^T is the FP64 transpose of the operator the refinement
    solves (FP64 tables); the FP32 forward apply differs from it by the FP32
    apply error (stage bounds of test_gpu_parity.py), so the identity holds to
    that level."""
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(CASES[name](), device=0)
    x, y = _vec(P, 5), _vec(P, 6)
    Ax = P.apply_operator(x)
    ATy = P.apply_operator_T(y)
    lhs, rhs = _dot(y, Ax), _dot(ATy, x)
    scale = float(torch.linalg.norm(y.double()) * torch.linalg.norm(Ax.double()))
    assert abs(lhs - rhs) < 5e-4 * scale, (lhs, rhs, scale)
    P.close()


@pytest.mark.parametrize("name,tol", [("twolevel", 1e-12), ("mgii", 1e-10)])
def test_adjoint_solve_fp64(name, tol):
    """The forward preconditioner is only an approximate inverse of A^T, so the
    two-term case is solved to 1e-10 (more iterations than the forward solve)."""
    from paper_2505_20968_gb300.binding import PRD
    P = PRD(CASES[name](), precision="fp64", device=0)
    b = P.rhs()
    x, info = P.solve(tol=1e-12, max_iter=600, restart=80)
    g = _vec(P, 7)
    lam, ainfo = P.solve_adjoint(g, tol=tol, max_iter=3000, restart=120, check=False)
    assert ainfo["rc"] == 0, ainfo
    r = g - P.apply_operator_T(lam)
    assert float(torch.linalg.norm(r.double()) / torch.linalg.norm(g.double())) < 10 * tol
    lhs, rhs = _dot(g, x), _dot(lam, b)
    assert abs(lhs - rhs) < 1e3 * tol * abs(lhs), (lhs, rhs, ainfo["iters"])
    P.close()


def test_grad_B_matches_finite_differences_of_J():
    """dJ/d(B, theta_B) from prd_grad_B (one adjoint solve) against central
    differences of J over two forward solves, for J = sum of the emergent
    intensities of the top layer (linear in I) on a small two-term case."""
    from paper_2505_20968_gb300.binding import PRD
    mk = lambda: inputs.mgii(n_z=6, n_core_each=5, n_wing=4, n_mu_half=1, n_chi=4, seed=23)
    cfg = mk()
    P = PRD(cfg, precision="fp64", device=0)
    x, _ = P.solve(tol=1e-12, max_iter=600, restart=80)
    top = P.mu > 0
    dJdI = torch.zeros_like(x)
    dJdI[-1, torch.from_numpy(top).to(x.device), :, 0] = 1.0
    g = P.grad_B(x, dJdI)
    assert np.all(np.isfinite(g))

    def J_of(atm_key, iz, val):
        c = mk()
        c["atm"][atm_key] = np.array(c["atm"][atm_key], dtype=np.float64)
        c["atm"][atm_key][iz] = val
        Q = PRD(c, precision="fp64", device=0)
        xq, _ = Q.solve(tol=1e-12, max_iter=600, restart=80)
        v = float(xq[-1, torch.from_numpy(top).to(xq.device), :, 0].sum().item())
        Q.close()
        return v

    for key, k, iz in (("B_G", 0, 2), ("thetaB", 1, 4)):
        p0 = float(cfg["atm"][key][iz])
        h = max(1e-3 * abs(p0), 0.1 if k == 0 else 1e-3)
        lo = p0 if (k == 0 and p0 - h < 0) else p0 - h
        fd = (J_of(key, iz, p0 + h) - J_of(key, iz, lo)) / (p0 + h - lo)
        scale = float(x[-1, torch.from_numpy(top).to(x.device), :, 0].sum().item())
        assert abs(g[iz, k] - fd) < 1e-4 * abs(fd) + 1e-9 * scale, (key, iz, g[iz, k], fd)
    P.close()
