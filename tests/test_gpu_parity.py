"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

FP64 mode (two-level slab): every stage within 1e-9 relative.
FP32 mode (two-term Mg II / H I physics on reduced grids): the emissivity
within 2e-5 of its scale, and after a solve the emergent I within 1e-5
relative and Q/I, U/I, V/I within 1e-4 absolute (the stated FP32 tolerance).
"""
import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs
from oracle.problem import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _prd(cfg, **kw):
    from paper_2505_20968_gb300.binding import PRD
    return PRD(cfg, device=0, **kw)


def _t(x, P):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device=P.device, dtype=P.dtype)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


CASES = {
    "twolevel": lambda: inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2),
    "twolevel_1mu": lambda: inputs.twolevel_slab(n_z=7, n_x=9, n_mu_half=1, n_chi=4, eps=1e-3),
    "mgii": lambda: inputs.mgii(n_z=10, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=21),
    "hi": lambda: inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31),
    "hi_aa": lambda: inputs.hi_lya(n_z=8, n_core=11, n_wing=6, n_mu_half=2, n_chi=4, seed=32,
                                   mode=inputs.MODE_AA),
}
_cache = {}


def pair(name):
    if name not in _cache:
        cfg = CASES[name]()
        _cache[name] = (cfg, _prd(cfg), Problem(cfg))
    return _cache[name]


@pytest.mark.parametrize("name", ["twolevel", "twolevel_1mu"])
def test_fp64_stages(name):
    cfg, P, O = pair(name)
    x = inputs.seeded_vector(P.shape, 3, 0.1, 1.0)
    x[..., 1:] *= 0.1
    tol = 1e-9
    assert _rel(P.apply_sigma(_t(x, P)).cpu().numpy(), O.apply_sigma(x)) < tol
    assert _rel(P.apply_lambda(_t(x, P)).cpu().numpy(), O.formal_solution(x)) < tol
    assert _rel(P.rhs().cpu().numpy(), O.rhs()) < tol
    assert _rel(P.apply_operator(_t(x, P)).cpu().numpy(), O.apply_A(x)) < tol


@pytest.mark.parametrize("name", ["twolevel", "twolevel_1mu"])
def test_fp64_solve(name):
    cfg, P, O = pair(name)
    xg, info = P.solve(tol=1e-11, max_iter=400, restart=80)
    xo, _ = O.solve(tol=1e-13)
    assert info["true_rel_res"] < 1e-11
    assert _rel(xg.cpu().numpy(), xo) < 1e-8


@pytest.mark.parametrize("name", ["mgii", "hi", "hi_aa"])
def test_fp32_sigma_and_operator(name):
    cfg, P, O = pair(name)
    x = inputs.seeded_vector(P.shape, 5, 0.1, 1.0)
    x[..., 1:] *= 0.05
    eg = P.apply_sigma(_t(x, P)).cpu().numpy().astype(np.float64)
    eo = O.apply_sigma(x)
    for iz in range(P.nz):
        scale = np.max(np.abs(eo[iz, ..., 0]))
        assert np.max(np.abs(eg[iz] - eo[iz])) < 2e-5 * scale, f"height {iz}"
    lg = P.apply_lambda(_t(eo, P)).cpu().numpy()
    lo = O.formal_solution(eo)
    assert _rel(lg, lo) < 2e-5
    ag = P.apply_operator(_t(x, P)).cpu().numpy()
    assert _rel(ag, O.apply_A(x)) < 2e-5


@pytest.mark.parametrize("name", ["mgii", "hi", "hi_aa"])
def test_fp32_emergent_stokes_after_solve(name):
    cfg, P, O = pair(name)
    xg, info = P.solve(tol=1e-9, max_iter=300, restart=100, check=False)
    xo, _ = O.solve(tol=1e-12)
    top = P.mu > 0
    Ig = xg.cpu().numpy()[-1, top].astype(np.float64)
    Io = xo[-1, top]
    assert np.max(np.abs(Ig[..., 0] - Io[..., 0]) / Io[..., 0]) < 1e-5
    for s in (1, 2, 3):
        assert np.max(np.abs(Ig[..., s] / Ig[..., 0] - Io[..., s] / Io[..., 0])) < 1e-4
