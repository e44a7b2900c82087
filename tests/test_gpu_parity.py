"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Reference values come from tests/golden/*.npz, written by
tests/golden/make_golden.py, which calls only oracle/ (inputs are regenerated
here from the same seeds).

FP64 mode (two-level slab): every stage within 1e-9 relative, the solution
within 1e-8.  FP32 mode (two-term Mg II / H I physics on reduced grids, and
sampled rows of the full Mg II workload): the emissivity within 4e-6 of its
scale per height (1e-6 on the CUDA-core path) and within a point-wise bound,
the operator within that bound propagated through |Lambda|; after a solve with
mixed-precision refinement (residuals from the FP64 copy of the Sigma tables)
the emergent I within 1e-5 relative and Q/I, U/I, V/I within 1e-4 absolute.
"""
import os

import numpy as np
import pytest

from paper_2505_20968_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

CASES = {
    "twolevel": lambda: inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2),
    "twolevel_1mu": lambda: inputs.twolevel_slab(n_z=7, n_x=9, n_mu_half=1, n_chi=4, eps=1e-3),
    "mgii": lambda: inputs.mgii(n_z=10, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=21),
    "hi": lambda: inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31),
    "hi_aa": lambda: inputs.hi_lya(n_z=8, n_core=11, n_wing=6, n_mu_half=2, n_chi=4, seed=32,
                                   mode=inputs.MODE_AA),
}
_cache = {}


def get(name):
    if name not in _cache:
        from paper_2505_20968_gb300.binding import PRD
        cfg = CASES[name]()
        _cache[name] = (cfg, PRD(cfg, device=0), dict(np.load(os.path.join(GOLD, name + ".npz"))))
    return _cache[name]


def _t(x, P):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device=P.device, dtype=P.dtype)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("name", ["twolevel", "twolevel_1mu"])
def test_fp64_stages(name):
    cfg, P, G = get(name)
    x = G["x"]
    tol = 1e-9
    assert _rel(P.apply_sigma(_t(x, P)).cpu().numpy(), G["sigma"]) < tol
    assert _rel(P.apply_lambda(_t(G["sigma"], P)).cpu().numpy(), G["lam"]) < tol
    assert _rel(P.rhs().cpu().numpy(), G["rhs"]) < tol
    assert _rel(P.apply_operator(_t(x, P)).cpu().numpy(), G["Ax"]) < tol


@pytest.mark.parametrize("name", ["twolevel", "twolevel_1mu"])
def test_fp64_solve(name):
    cfg, P, G = get(name)
    xg, info = P.solve(tol=1e-11, max_iter=400, restart=80)
    assert info["true_rel_res"] < 1e-11
    assert _rel(xg.cpu().numpy(), G["sol"]) < 1e-8


_lam_abs_cache = {}


def _lambda_abs(name):
    """|Lambda| of the oracle, ray by ray ((4 nz) x (4 nz) per (Omega, nu)),
    as a map v -> |Lambda| v on [z][Omega][nu][4] arrays."""
    if name not in _lam_abs_cache:
        from oracle.problem import Problem
        O = Problem(CASES[name](), normalise=False)       # K and DELO tables only
        L = np.abs(O.lambda_rays())
        nz, nO, nN = O.nz, O.nO, O.nN

        def lam_abs(v):
            vr = v.transpose(1, 2, 0, 3).reshape(nO, nN, 4 * nz)
            return np.einsum("onij,onj->oni", L, vr).reshape(nO, nN, nz, 4).transpose(2, 0, 1, 3)
        _lam_abs_cache[name] = lam_abs
    return _lam_abs_cache[name]


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "simt"])
@pytest.mark.parametrize("name", ["mgii", "hi", "hi_aa"])
def test_fp32_sigma_and_operator(name, tc):
    """FP32 stages.

    Sigma, per height: absolute error below a bound relative to the height's
    largest emissivity: 1e-6 for the CUDA-core contraction (FP32 rounding of
    the largest terms; measured 4e-7) and 4e-6 for the tcgen05 contraction,
    whose 3xTF32 split leaves <= 3 * 2^-22 per product and whose products are
    summed in the tensor pipe's FP32 accumulator (measured 2.1e-6).

    Sigma, point by point: |d eps| <= 1e-5 |eps_I| + 1e-7 max_z |eps_I| (every
    Stokes parameter measured against the point's own intensity).  Away from
    the far wings the error is ~2e-6 relative to the point itself; the FP32
    tables leave an absolute floor of ~5e-8 of the height's maximum where the
    dispersion terms of nearly degenerate components cancel.  This catches a
    wrong Kirchhoff factor at any point carrying more than ~1e-7 of its
    height's emissivity.

    The operator y = x - Lambda Sigma x, point by point, by propagating those
    bounds: |d y| <= |Lambda| (1e-5 |eps_I| + 1e-7 max_z |eps_I|) + 2e-5 |Lambda| |eps|
    + 1e-6 |x|, with |Lambda| the oracle's formal solution ray by ray with
    every entry replaced by its magnitude, 2e-5 the FP32 bound of Lambda
    (measured against the oracle's on its own emissivity) and 1e-6 the FP32
    rounding of x - Lambda eps.  (y itself nearly cancels, |y_I| / |x_I| down to
    2e-4, and in the far wings Lambda multiplies the absolute Sigma floor by
    1/eta_I, so no relative bound on y can be tight there; the
    mixed-precision refinement of prd_solve removes this at solution level,
    test_fp32_emergent_stokes_after_solve.)"""
    cfg, P, G = get(name)
    x = G["x"]
    P.set_tensor_cores(tc)
    eg = P.apply_sigma(_t(x, P)).cpu().numpy().astype(np.float64)
    eo = G["sigma"]
    for iz in range(P.nz):
        scale = np.max(np.abs(eo[iz, ..., 0]))
        d = np.max(np.abs(eg[iz] - eo[iz])) / scale
        assert d < (4e-6 if tc else 1e-6), f"height {iz}: {d:.2e}"
    hmax = np.max(np.abs(eo[..., 0]).reshape(P.nz, -1), axis=1)[:, None, None, None]
    b_sig = 1e-5 * np.abs(eo[..., :1]) + 1e-7 * hmax
    r = np.max(np.abs(eg - eo) / b_sig)
    assert r < 1.0, f"Sigma point-wise: {r:.2f} of the bound"
    d = _rel(P.apply_lambda(_t(eo, P)).cpu().numpy(), G["lam"])
    assert d < 2e-5, f"lambda {d:.2e}"
    yg = P.apply_operator(_t(x, P)).cpu().numpy().astype(np.float64)
    P.set_tensor_cores(True)
    lam_abs = _lambda_abs(name)
    b_y = lam_abs(np.broadcast_to(b_sig, eo.shape)) + 2e-5 * lam_abs(np.abs(eo)) + 1e-6 * np.abs(x)
    r = np.max(np.abs(yg - G["Ax"]) / b_y)
    print(f"{name} tc={tc}: operator error at most {r:.2f} of its point-wise bound")
    assert r < 1.0, f"operator point-wise: {r:.2f} of the bound"


@pytest.mark.parametrize("name", ["mgii", "hi", "hi_aa"])
def test_fp32_emergent_stokes_after_solve(name):
    """FP32 mode at the accuracy target: emergent I within 1e-5 relative and
    Q/I, U/I, V/I within 1e-4 absolute of the oracle's converged solution.
    GMRES tol 1e-10 is the largest that meets it on the Mg II case (a sweep
    measured 2e-4 at 1e-9 and 3e-6 at 1e-10: the small-epsilon scattering
    problem amplifies the residual by ~1e5 into the top-layer intensity)."""
    cfg, P, G = get(name)
    xg, info = P.solve(tol=1e-10, max_iter=600, restart=60)
    top = P.mu > 0
    Ig = xg.cpu().numpy()[-1, top].astype(np.float64)
    Io = G["sol"][-1, top]
    d = np.max(np.abs(Ig[..., 0] - Io[..., 0]) / Io[..., 0])
    assert d < 1e-5, f"I {d:.2e}"
    for s in (1, 2, 3):
        d = np.max(np.abs(Ig[..., s] / Ig[..., 0] - Io[..., s] / Io[..., 0]))
        assert d < 1e-4, f"Stokes {s} {d:.2e}"


def test_full_size_mgii_sampled_rows():
    """The full Mg II workload (70 x 64 x 200, FP32, the configuration bench.py
    times): Sigma x at sampled (height, direction) rows and Lambda x on sampled
    rays, against the oracle's one-by-one evaluation."""
    from paper_2505_20968_gb300.binding import PRD
    G = np.load(os.path.join(GOLD, "mgii_full.npz"))
    P = PRD(inputs.mgii(), device=0)
    x = inputs.seeded_vector(P.shape, 5, 0.1, 1.0)
    x[..., 1:] *= 0.05
    xt = _t(x, P)
    eg = P.apply_sigma(xt).cpu().numpy().astype(np.float64)
    lg = P.apply_lambda(xt).cpu().numpy().astype(np.float64)
    for key in G.files:
        if key.startswith("sigma_"):
            iz, o = map(int, key.split("_")[1:])
            ref = G[key]
            assert np.max(np.abs(eg[iz, o] - ref)) < 2e-5 * np.max(np.abs(ref[:, 0])), key
        if key.startswith("lam_"):
            o, n = map(int, key.split("_")[1:])
            ref = G[key]
            assert np.max(np.abs(lg[:, o, n] - ref)) < 2e-5 * np.max(np.abs(ref)), key
    P.close()


def test_full_size_twolevel_fp64_sampled_rows():
    from paper_2505_20968_gb300.binding import PRD
    G = np.load(os.path.join(GOLD, "twolevel_full.npz"))
    P = PRD(inputs.twolevel_slab(), device=0)
    x = inputs.seeded_vector(P.shape, 5, 0.1, 1.0)
    x[..., 1:] *= 0.05
    xt = _t(x, P)
    eg = P.apply_sigma(xt).cpu().numpy()
    lg = P.apply_lambda(xt).cpu().numpy()
    for key in G.files:
        if key.startswith("sigma_"):
            iz, o = map(int, key.split("_")[1:])
            assert _rel(eg[iz, o], G[key]) < 1e-9, key
        if key.startswith("lam_"):
            o, n = map(int, key.split("_")[1:])
            assert _rel(lg[:, o, n], G[key]) < 1e-9, key


@pytest.mark.parametrize("name", ["twolevel", "mgii", "hi", "hi_aa"])
def test_emergent_stokes_off_grid(name):
    """S11: emergent Stokes along lines of sight off the grid (mu = 0.1, 1,
    0.55) from the oracle's converged field."""
    cfg, P, G = get(name)
    los = G["los"]
    out = P.emergent_stokes(_t(G["sol"], P), los[:, 0], los[:, 1]).cpu().numpy().astype(np.float64)
    ref = G["emergent"]
    tol = 1e-9 if P.prec == 0 else 1e-5
    d = np.max(np.abs(out[..., 0] - ref[..., 0]) / ref[..., 0])
    assert d < tol, f"I {d:.2e}"
    for s in (1, 2, 3):
        d = np.max(np.abs(out[..., s] / out[..., 0] - ref[..., s] / ref[..., 0]))
        assert d < (1e-9 if P.prec == 0 else 1e-5), f"Stokes {s} {d:.2e}"


@pytest.mark.parametrize("name", ["mgii", "hi", "hi_aa"])
def test_tensor_core_contraction(name):
    """tcgen05 R_II contraction (3xTF32) against the CUDA-core contraction and
    the oracle; no bounded wait may expire."""
    cfg, P, G = get(name)
    x = _t(G["x"], P)
    P.set_tensor_cores(False)
    e_simt = P.apply_sigma(x).cpu().numpy().astype(np.float64)
    P.set_tensor_cores(True)
    e_tc = P.apply_sigma(x).cpu().numpy().astype(np.float64)
    P.device_status()
    eo = G["sigma"]
    for iz in range(P.nz):
        scale = np.max(np.abs(eo[iz, ..., 0]))
        d_simt = np.max(np.abs(e_tc[iz] - e_simt[iz])) / scale
        d_or = np.max(np.abs(e_tc[iz] - eo[iz])) / scale
        # bounds of test_fp32_sigma_and_operator: 4e-6 (tcgen05) and 1e-6 (CUDA cores)
        assert d_simt < 5e-6, f"height {iz}: tc vs simt {d_simt:.2e}"
        assert d_or < 4e-6, f"height {iz}: tc vs oracle {d_or:.2e}"


@pytest.mark.parametrize("name", ["mgii", "hi", "hi_aa"])
def test_bf16x3_contraction_and_solve(name):
    """Split-BF16 products (PRD_FP32_BF16X3, the compensated bf16 precision mode):
    Sigma within 1e-4 of each height's largest emissivity (each product
    hi*hi + hi*lo + lo*hi of bf16 halves leaves <= 3 * 2^-18 = 1.1e-5; the
    3xTF32 path measures ~3x its own per-product bound, so 1e-4 leaves room),
    and the refined solve, whose FP64 residuals do not use the contraction,
    at the FP32 accuracy target: emergent I within 1e-5 relative, Q/I, U/I,
    V/I within 1e-4 absolute of the oracle's solution."""
    from paper_2505_20968_gb300.binding import PRD
    G = dict(np.load(os.path.join(GOLD, name + ".npz")))
    P = PRD(CASES[name](), precision="fp32_bf16x3", device=0)
    eg = P.apply_sigma(_t(G["x"], P)).cpu().numpy().astype(np.float64)
    P.device_status()
    worst = 0.0
    for iz in range(P.nz):
        scale = np.max(np.abs(G["sigma"][iz, ..., 0]))
        worst = max(worst, np.max(np.abs(eg[iz] - G["sigma"][iz])) / scale)
    print(f"BF16x3 Sigma {name}: {worst:.2e} of the height maximum")
    assert worst < 1e-4
    # the context's tiles are stored as bf16 planes: the same products as a
    # PRD_FP32 context splitting its FP32 tiles on the fly (to FP32 atomics order)
    from paper_2505_20968_gb300.binding import PrdError
    Q = PRD(CASES[name](), precision="fp32", device=0)
    Q.set_contraction("bf16x3")
    eq = Q.apply_sigma(_t(G["x"], P)).cpu().numpy().astype(np.float64)
    Q.close()
    for iz in range(P.nz):
        scale = np.max(np.abs(eq[iz, ..., 0]))
        assert np.max(np.abs(eg[iz] - eq[iz])) <= 1e-6 * scale, iz
    with pytest.raises(PrdError):
        P.set_contraction("tf32x3")
    xg, info = P.solve(tol=1e-10, max_iter=900, restart=200)
    top = P.mu > 0
    Ig = xg.cpu().numpy()[-1, top].astype(np.float64)
    Io = G["sol"][-1, top]
    d = np.max(np.abs(Ig[..., 0] - Io[..., 0]) / Io[..., 0])
    print(f"BF16x3 solve {name}: {info['iters']} applies, emergent I {d:.2e}")
    assert d < 1e-5
    for s in (1, 2, 3):
        assert np.max(np.abs(Ig[..., s] / Ig[..., 0] - Io[..., s] / Io[..., 0])) < 1e-4
    P.close()


@pytest.mark.parametrize("name", ["mgii", "hi"])
def test_bf16x2_contraction_and_solve(name):
    """BF16x2 (PRD_FP32_BF16X2): tiles stored as the bf16 hi plane alone and two
    products hi(B) hi(A) + lo(B) hi(A).  The tile keeps its rounding to bf16
    (<= 2^-9 relative per entry), so Sigma is good to ~1e-3: within 1e-2 of
    each height's largest emissivity (measured 8.9e-4 on Mg II).  As the inner
    operator of the refinement that error is amplified by the scattering
    problem's ~1/eps, and on the Mg II case the outer FP64 iteration stalls
    (PRD_E_NOCONV); prd_solve never returns a solution it has not checked, so
    the test asserts: either PRD_E_NOCONV, or a solution at the FP32 target
    (emergent I within 1e-5 relative, Q/I, U/I, V/I within 1e-4 absolute)."""
    from paper_2505_20968_gb300.binding import PRD
    G = dict(np.load(os.path.join(GOLD, name + ".npz")))
    P = PRD(CASES[name](), precision="fp32_bf16x2", device=0)
    eg = P.apply_sigma(_t(G["x"], P)).cpu().numpy().astype(np.float64)
    P.device_status()
    worst = 0.0
    for iz in range(P.nz):
        scale = np.max(np.abs(G["sigma"][iz, ..., 0]))
        worst = max(worst, np.max(np.abs(eg[iz] - G["sigma"][iz])) / scale)
    print(f"BF16x2 Sigma {name}: {worst:.2e} of the height maximum")
    assert worst < 1e-2
    xg, info = P.solve(tol=1e-10, max_iter=400, restart=200, check=False)
    print(f"BF16x2 solve {name}: rc {info['rc']}, {info['iters']} applies, residual {info['true_rel_res']:.2e}")
    assert info["rc"] in (0, -5), info
    if info["rc"] == 0:
        assert info["true_rel_res"] < 1e-10
        top = P.mu > 0
        Ig = xg.cpu().numpy()[-1, top].astype(np.float64)
        Io = G["sol"][-1, top]
        assert np.max(np.abs(Ig[..., 0] - Io[..., 0]) / Io[..., 0]) < 1e-5
        for s in (1, 2, 3):
            assert np.max(np.abs(Ig[..., s] / Ig[..., 0] - Io[..., s] / Io[..., 0])) < 1e-4
    P.close()
