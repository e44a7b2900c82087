"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test states the passage or the closed form it checks.  None of them
calls the CUDA library.
"""
import numpy as np
import pytest
from scipy import special
from scipy.integrate import quad_vec, quad
from scipy.interpolate import CubicSpline

from paper_2505_20968_gb300 import inputs
from oracle.faddeeva import wofz, voigt_faraday
from oracle.spline import NaturalSpline
from oracle.geometry import angular_grid, theta_classes
from oracle import redistribution as RD
from oracle.problem import Problem, delo_coeffs, gmres
from oracle.constants import MU_B_OVER_H, GAUSS
from oracle.atom import states


# ---------------------------------------------------------------- Faddeeva
def test_faddeeva_closed_forms():
    y = np.geomspace(1e-4, 30, 200)
    np.testing.assert_allclose(wofz(1j * y), special.erfcx(y), rtol=2e-14)
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(wofz(x).real, np.exp(-x * x), atol=2e-15)
    np.testing.assert_allclose(wofz(x).imag, 2 / np.sqrt(np.pi) * special.dawsn(x), atol=2e-15)
    z = 300.0 * np.exp(1j * np.linspace(0.01, np.pi - 0.01, 50))
    np.testing.assert_allclose(wofz(z), 1j / (np.sqrt(np.pi) * z) * (1 + 0.5 / z ** 2 + 0.75 / z ** 4),
                               rtol=1e-10)


def test_faddeeva_vs_scipy():
    rng = np.random.default_rng(0)
    x = rng.uniform(-60, 60, 20000)
    y = 10 ** rng.uniform(-6, 1.5, 20000)
    z = x + 1j * y
    ref = special.wofz(z)
    assert np.max(np.abs(wofz(z) - ref) / np.abs(ref)) < 1e-13


# ---------------------------------------------------------------- spline
def test_spline_natural_vs_scipy_and_linear_exactness():
    rng = np.random.default_rng(1)
    u = np.sort(rng.uniform(-5, 5, 17))
    y = rng.normal(size=17)
    s = NaturalSpline(u)
    xs = np.linspace(u[0], u[-1], 400)
    np.testing.assert_allclose(s(y, xs), CubicSpline(u, y, bc_type="natural")(xs), atol=1e-12)
    np.testing.assert_allclose(s(2.0 - 0.3 * u, xs), 2.0 - 0.3 * xs, atol=1e-12)
    # constant extension outside the grid
    assert s(y, np.array([u[0] - 3.0]))[0] == y[0] and s(y, np.array([u[-1] + 1.0]))[0] == y[-1]


# ---------------------------------------------------------------- angles
def test_number_of_scattering_angles_paper_grid():
    """Sect. 6.2: 2 x 6 GL mu x 9 chi gives N_Theta = 205 (with Theta = 0)."""
    mu, chi, w = angular_grid(6, 9)
    th, _ = theta_classes(mu, chi)
    assert th.size == 205
    assert abs(w.sum() - 1.0) < 1e-14
    assert 4 * 70 * 210 * mu.size == 6350400     # "N ~ 6e6" (Sect. 6.2)


# ---------------------------------------------------------------- F kernel
@pytest.mark.parametrize("theta", [0.1, 0.7, 1.6, 2.6, 0.9 * np.pi, np.pi - 1e-3, np.pi])
@pytest.mark.parametrize("a", [1e-2, 1e-4])
def test_F_marginal_is_complex_voigt(theta, a):
    """int F(Theta, x', x) dx' = sqrt(pi) W(a, x) for every Theta: the complex
    form of Hummer's R_II-A marginal (R_II-A = Re F / pi, Sect. 2.4)."""
    for x in (0.0, 0.8, -2.5, 4.0):
        g = 2 * np.sin(theta / 2)
        pts = sorted([x, -x])
        val, _ = quad_vec(lambda xp: np.array([RD.F_kernel(theta, xp, x, a).real,
                                               RD.F_kernel(theta, xp, x, a).imag]),
                          x - 7 * g, x + 7 * g, points=[p for p in pts if abs(p - x) < 7 * g],
                          epsabs=1e-13, epsrel=1e-12, limit=5000)
        ref = np.sqrt(np.pi) * voigt_faraday(a, x)
        assert abs(val[0] + 1j * val[1] - ref) < 2e-9 * max(1.0, abs(ref))


def test_F_symmetry_and_pi_limit():
    xp = np.linspace(-3, 3, 13)
    for theta in (0.3, 1.9, 3.0):
        np.testing.assert_allclose(RD.F_kernel(theta, xp, 0.7, 1e-3), RD.F_kernel(theta, 0.7, xp, 1e-3),
                                   rtol=1e-13)
    # Theta -> pi approaches the exact limit kernel
    f_lim = RD.F_kernel(np.pi, xp, 0.4, 1e-2)
    f_near = RD.F_kernel(np.pi - 1e-6, xp, 0.4, 1e-2)
    np.testing.assert_allclose(f_near, f_lim, rtol=2e-5)


def test_small_theta_tile_tends_to_delta_form():
    """App. C rule i: F(0,u,u') = sqrt(pi) delta(u-u') W(a,u')."""
    t = -1.0 + np.arange(21) / 10.0
    u = 8.0 * np.sinh(3 * t) / np.sinh(3)
    s = NaturalSpline(u)
    T0 = RD.tile(s, 0.0, 1e-3, 0.01, -0.02)
    Ts = RD.tile(s, 2e-4, 1e-3, 0.01, -0.02)
    assert np.max(np.abs(Ts - T0)) < 1e-3 * np.max(np.abs(T0))


def test_composite_quadrature_vs_adaptive_gk_fig1():
    """Fig. 1 setting (a = 0.01, Theta = 0.9 pi, u_{ku,kl} = -11.1,
    u_{ku,kl'} = -11.2); the paper's grids reach 1e-8, the oracle's 1e-10."""
    u = np.linspace(-25.0, 25.0, 61) + 11.15
    s = NaturalSpline(u)
    theta, a, s_in, s_out = 0.9 * np.pi, 0.01, -11.1, -11.2
    for un in (u[5], 11.15 - 0.3, 11.2, u[40]):
        row = RD.tile_row(s, theta, a, s_in, s_out, un)
        x = un + s_out
        g = 2 * np.sin(theta / 2)
        L, R = x - s_in - 6.5 * g, x - s_in + 6.5 * g
        pts = [p for p in list(u) + [-x - s_in] if L < p < R]

        def f(up):
            v = RD.F_kernel(theta, np.array([up + s_in]), x, a)[0] * s.basis(np.array([up]))[0]
            return np.concatenate([v.real, v.imag])
        ref, _ = quad_vec(f, L, R, points=sorted(pts), epsabs=1e-14, epsrel=1e-12, limit=20000)
        ref = ref[:u.size] + 1j * ref[u.size:]
        assert np.max(np.abs(row - ref)) < 1e-10 * np.max(np.abs(ref))


def test_r3_weights_vs_adaptive():
    u = np.linspace(-12, 12, 31)
    s = NaturalSpline(u)
    r = RD.r3_in_weights(s, 3e-3, 0.3, -0.2)
    for m in (0, 7, 15, 30):
        e = np.zeros(u.size)
        e[m] = 1.0
        f = lambda x: (voigt_faraday(3e-3, x + 0.3) + np.conj(voigt_faraday(3e-3, x - 0.2))) * s(e, np.array([x]))[0]
        re = quad(lambda x: f(x).real, u[0], u[-1], points=list(u[1:-1]) + [-0.3, 0.2], limit=2000,
                  epsabs=1e-14)[0]
        im = quad(lambda x: f(x).imag, u[0], u[-1], points=list(u[1:-1]) + [-0.3, 0.2], limit=2000,
                  epsabs=1e-14)[0]
        assert abs(r[m] - (re + 1j * im)) < 1e-11


# ---------------------------------------------------------------- DELO
def test_delo_constant_source_exact():
    """DELO-linear reproduces I = S (1 - e^-tau) + I0 e^-tau for constant S."""
    d = np.array([1e-6, 1e-4, 1e-3, 0.3, 2.0, 40.0])
    e, al, be = delo_coeffs(d)
    np.testing.assert_allclose(e + al + be, 1.0, atol=1e-15)
    # linear source S = t: exact solution of dI/dt = -I + t over one step
    I0 = 0.4
    exact = I0 * np.exp(-d) + (d - 1.0) + np.exp(-d)   # S(t)=t from t=0 to d
    np.testing.assert_allclose(e * I0 + al * 0.0 + be * d, exact, rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- atom / K
def test_paschen_back_levels():
    """Sect. 2.2: at B = 0 the two-term upper levels sit at the Table-1
    energies; the dipole strengths sum to one per upper state."""
    cfg = inputs.mgii(n_z=2)
    Eu, D, El = states(cfg["atom"], 0.0)
    E = np.array(cfg["atom"]["E_u_cm"]) * 2.99792458e10
    nu0 = (2 * E[0] + 4 * E[1]) / 6
    np.testing.assert_allclose(np.sort(Eu), np.sort([E[0] - nu0] * 2 + [E[1] - nu0] * 4), rtol=1e-12)
    np.testing.assert_allclose((D ** 2).sum(axis=(0, 2)), 1.0, rtol=1e-12)
    # weak field: Zeeman splitting with Lande factors 2/3 (P1/2) and 4/3 (P3/2)
    Eu1, _, _ = states(cfg["atom"], 1.0)
    nuL = MU_B_OVER_H * GAUSS
    split = np.sort(Eu1 - np.sort(Eu))
    assert abs(np.ptp(np.sort(Eu1)[:2]) - 2 * (2 / 3) * 0.5 * nuL) < 1e-3 * nuL


def test_weak_field_stokes_V():
    """V(lambda) = -dlambda_B g cos(theta_B) dI/dlambda (weak field, LL04 Ch. 9):
    in reduced frequency eta_V = -(nu_L/dnu_D) g cos(theta_B) d eta_I/du."""
    cfg = inputs.twolevel_slab(n_z=2, n_x=9)
    cfg["atm"]["B_G"][:] = 10.0
    P = Problem(cfg)
    u = np.linspace(-4, 4, 801)
    for mu in (0.8, -0.35):
        K = P.K_from_kappa(P.kappa(0, P.amplitudes(0, mu, 0.3), 0.0, u))
        pred = -(MU_B_OVER_H * GAUSS * 10.0 / P.dnuD[0]) * mu * np.gradient(K[:, 0, 0], u)
        assert np.max(np.abs(K[:, 3, 0] - pred)) < 1e-3 * np.max(np.abs(pred))


# ---------------------------------------------------------------- phase matrices
def _integrated_phase(P, iz, amp_o, amp_i, subset=None, hanle=True):
    """Frequency-integrated R^II: 3/(4(2S+1)) sum Tr(...) alpha/alpha_0 (Eq. RQIIKKp
    with int int [G(k_u') + G(k_u)^*] du' du = 2 pi)."""
    nu_ = P.nu_states
    ks = range(nu_) if subset is None else subset
    al = P.alpha[iz] / P.alpha[iz][0, 0].real
    M = np.zeros((4, 4), dtype=complex)
    for kl in range(P.nl_states):
        for klp in range(P.nl_states):
            for ku in ks:
                for kv in ks:
                    M += P._tr(amp_o, amp_i, ku, kv, kl, klp) * (al[ku, kv] if hanle else 1.0)
    M *= 3.0 / (4.0 * P.S2)
    assert np.max(np.abs(M.imag)) < 1e-12
    return M.real


def test_rayleigh_and_polarisabilities():
    """Zero-field polarisability W2 (Sect. 2.2 atoms): 90-degree scattering of
    unpolarised light gives Q/I = 3 W2 / (4 - W2): W2 = 1 for J 0->1 and for
    the spinless-limit two-term atom, 1/2 for J_u = 3/2, 0 for J_u = 1/2."""
    cfg = inputs.twolevel_slab(n_z=2, n_x=5)
    P = Problem(cfg)
    ao, ai = P.amplitudes(0, 0.0, 0.0), P.amplitudes(0, 1.0, 0.0)   # out: +x, in: +z
    M = _integrated_phase(P, 0, ao, ai)
    assert abs(M[1, 0] / M[0, 0] - 1.0) < 1e-12      # W2 = 1
    # Theta-averaged I->I coefficient is 1 (normalisation of App. E)
    mu, chi, w = angular_grid(4, 8)
    tot = sum(wi * _integrated_phase(P, 0, ao, P.amplitudes(0, m, c))[0, 0] for m, c, wi in zip(mu, chi, w))
    assert abs(tot - 1.0) < 1e-12
    cfg2 = inputs.mgii(n_z=2, n_core_each=3, n_wing=6, n_mu_half=1, n_chi=2)
    cfg2["atm"]["B_G"][:] = 0.0
    P2 = Problem(cfg2)
    ao, ai = P2.amplitudes(0, 0.0, 0.0), P2.amplitudes(0, 1.0, 0.0)
    Eu, _, _ = states(cfg2["atom"], 0.0)
    j12 = [k for k in range(6) if Eu[k] < 0]
    j32 = [k for k in range(6) if Eu[k] > 0]
    M32 = _integrated_phase(P2, 0, ao, ai, j32, hanle=False)
    M12 = _integrated_phase(P2, 0, ao, ai, j12, hanle=False)
    Mall = _integrated_phase(P2, 0, ao, ai, None, hanle=False)
    assert abs(M32[1, 0] / M32[0, 0] - 3 * 0.5 / (4 - 0.5)) < 1e-12
    assert abs(M12[1, 0] / M12[0, 0]) < 1e-12
    assert abs(Mall[1, 0] / Mall[0, 0] - 1.0) < 1e-12   # spin as spectator


def test_hanle_rotation_and_depolarisation():
    """Hanle effect of the J 0->1 atom (Sect. 1), 90-degree scattering with B
    along the line of sight: (Q + iU)/I = 1/(1 + 2 i H), H = 2 pi nu_L / Gamma,
    i.e. |p| = 1/sqrt(1 + 4H^2), |U/Q| = 2H."""
    cfg = inputs.twolevel_slab(n_z=2, n_x=5, a=1e-2)
    cfg["atm"]["B_G"][:] = 3.0
    cfg["atm"]["thetaB"][:] = np.pi / 2
    cfg["atm"]["chiB"][:] = 0.0
    P = Problem(cfg)
    H = 2 * np.pi * MU_B_OVER_H * GAUSS * 3.0 / (4 * np.pi * P.dnuD[0] * P.a[0])
    M = _integrated_phase(P, 0, P.amplitudes(0, 0.0, 0.0), P.amplitudes(0, 1.0, 0.0))
    q, uu = M[1, 0] / M[0, 0], M[2, 0] / M[0, 0]
    assert abs(np.hypot(q, uu) - 1 / np.sqrt(1 + 4 * H * H)) < 1e-12
    assert abs(abs(uu / q) - 2 * H) < 1e-10


# ---------------------------------------------------------------- operator-level pins
def _static_twolevel(n_z=3, n_x=11, B=0.0, r_el=1e-9, eps=1e-3, n_mu_half=2, n_chi=4):
    cfg = inputs.twolevel_slab(n_z=n_z, n_x=n_x, n_mu_half=n_mu_half, n_chi=n_chi, r_el=r_el, eps=eps)
    cfg["atm"]["B_G"][:] = B
    cfg["atm"]["thetaB"][:] = 0.7
    cfg["atm"]["chiB"][:] = 1.1
    return cfg


def test_kirchhoff_normalisation_is_one_at_zero_field():
    """App. E: at B = 0, v = 0 and with an angular rule exact for P_2, the
    discrete Sigma applied to (W_T, 0, 0, 0) already gives (1-eps) W_T eta_I,
    so f = 1 (R_III is switched off: its incident integral stops at the grid
    edges)."""
    P = Problem(_static_twolevel())
    assert np.max(np.abs(P.f - 1.0)) < 1e-9


def test_generalised_kirchhoff_all_stokes_magnetic():
    """App. E (generalised Kirchhoff law, LL04 Sect. 9.1): for an isotropic
    unpolarised W_T field eps_sc = (1-eps) W_T (eta_I, eta_Q, eta_U, eta_V), in
    a magnetic field as well; this ties the scattering amplitudes of R to the
    absorption matrix K.  Checked away from the two outermost frequencies."""
    P = Problem(_static_twolevel(B=40.0, n_x=15))
    for iz in range(P.nz):
        Il = np.zeros((P.nO, P.nN, 4))
        Il[..., 0] = P.WT[iz]
        num = (P.sigma_matrix(iz, normalised=False) @ Il.ravel()).reshape(P.nO, P.nN, 4)
        ref = (1 - P.eps[iz]) * P.WT[iz] * P.K[iz][..., :, 0]
        sl = slice(2, -2)
        assert np.max(np.abs(num[:, sl] - ref[:, sl])) < 1e-8 * np.max(np.abs(ref[..., 0]))


def test_crd_limit():
    """r_E -> 1 (alpha = 0): R = (1-eps) phi(u') phi(u) x Rayleigh (Sect. 2.4):
    the I->I part of Sigma_bar is rank one in frequency."""
    P = Problem(_static_twolevel(r_el=1 - 1e-12, n_x=9))
    blk = P.block(1, 0, 5)[:, 0, :, 0]
    sv = np.linalg.svd(blk, compute_uv=False)
    assert sv[1] < 1e-9 * sv[0]


def test_zero_field_1d_symmetries():
    """Static, unmagnetised 1D slab: U = V = 0 and no chi dependence; at the
    disk centre Q = 0 (axial symmetry), and near the limb the line-core
    scattering polarisation is parallel to the limb, Q/I > 0 (positive Q
    along the limb, as the figures of Sect. 6.3 take it; the radiation field
    at the surface is limb-darkened, so its anisotropy is positive)."""
    cfg = inputs.twolevel_slab(n_z=8, n_x=9, n_mu_half=2, n_chi=4, eps=1e-2)
    P = Problem(cfg)
    x, _ = P.solve(tol=1e-12)
    assert np.max(np.abs(x[..., 2:])) < 1e-12 * np.max(np.abs(x[..., 0]))
    xi = x.reshape(P.nz, 4, 4, P.nN, 4)          # [z, mu, chi, n, s]
    assert np.max(np.abs(xi - xi[:, :, :1])) < 1e-10 * np.max(np.abs(x))
    centre = P.emergent(x, 1.0, 0.0)
    assert np.max(np.abs(centre[:, 1:])) < 1e-12 * np.max(centre[:, 0])
    limb = P.emergent(x, 0.1, 0.0)
    core = P.nN // 2                               # x = 0 on the symmetric grid
    assert limb[core, 1] / limb[core, 0] > 1e-3


def test_r2_marginal_is_doppler_averaged_kramers_heisenberg():
    """Fixes which factor of Eq. RQIIKKp carries the conjugate, with alpha of
    App. B, by the physics of one atom rather than by the printed formula.

    An atom at rest scatters lower state k_l -> k_l' with the amplitude
    (Kramers-Heisenberg) T = sum_{k_u} M(k_u) / (x_{k_u} - i a), x in Doppler
    units, a = Gamma / (4 pi Dnu_D).  Partial fractions give
        A_u A_v^* = alpha_uv / (2a) [Phi(x_u) + Phi(x_v)^*],  Phi(x) = 1/(a + i x),
    with alpha_uv = 1 / (1 + i (x_u - x_v) / (2a)), and the Doppler average of
    Phi(x)^* is sqrt(pi) W(a, x).  Under a flat incident spectrum F integrates
    to sqrt(pi) W, so the block of R_II (R_III off: eps = 0, no elastic
    collisions) must equal 2a times the Doppler average of Tr(sigma_i T
    sigma_j T^+), which is computed here directly by quadrature over the
    velocity, without alpha or W.  Zeeman splittings comparable to the
    damping width (B = 360 G, a = 0.05) make the upper-level interference
    matter.  Swapping the conjugated factor changes the result at O(1),
    conjugating alpha by 5e-4; the oracle agrees to ~1e-13."""
    cfg = inputs.mgii(n_z=2, n_core_each=8, n_wing=3, n_mu_half=1, n_chi=4, seed=7)
    atm = cfg["atm"]
    nz = len(atm["z_km"])
    for key, val in (("a", 0.05), ("eps", 0.0), ("r_el", 0.0), ("B_G", 360.0), ("thetaB", 0.7),
                     ("chiB", 0.4)):
        atm[key] = np.full(nz, val)
    atm["v_kms"] = np.zeros((nz, 3))
    P = Problem(cfg, normalise=False)
    from oracle.problem import SIG
    iz, o, op = 0, 1, 6
    assert 0.0 < P.thetas[P.cls[o, op]] < np.pi
    N, a = P.nN, P.a[iz]
    c2 = 3.0 / (8.0 * np.pi * P.S2)
    flat = P.block(iz, o, op).reshape(N, 4, N, 4).sum(axis=2) / (P.k[iz] * P.wang[op] * c2 * 2.0 * a)
    ampO, ampI, s = P.amp[iz][o], P.amp[iz][op], P.shift[iz]

    def kramers_heisenberg(xn):
        def f(y):
            acc = np.zeros((4, 4))
            for kl in range(P.nl_states):
                for klp in range(P.nl_states):
                    T = np.zeros((2, 2), complex)
                    for ku in range(P.nu_states):
                        T += np.outer(ampO[:, ku, klp].conj(), ampI[:, ku, kl]) / (xn + s[ku, klp] - y - 1j * a)
                    acc += np.einsum("iab,bc,jcd,ad->ij", SIG, T, SIG, T.conj()).real
            return acc * np.exp(-y * y) / np.sqrt(np.pi)
        poles = sorted({xn + s[ku, klp] for ku in range(P.nu_states) for klp in range(P.nl_states)})
        pts = [-12.0] + [q for q in poles if -12.0 < q < 12.0] + [12.0]
        return sum(quad_vec(f, lo, hi, epsabs=1e-14, epsrel=1e-12, limit=2000)[0]
                   for lo, hi in zip(pts[:-1], pts[1:]))

    for n in (0, 4, 9, 14, N - 1):           # wings and both line cores
        k = kramers_heisenberg(P.u[iz][n])
        assert np.max(np.abs(k - flat[n])) < 1e-10 * np.max(np.abs(k)), n


def test_aa_tile_marginal_and_theta_convergence():
    """Angle-averaged tiles (Eq. R_AA): every Theta's F integrates to
    sqrt(pi) W(a, x) over the incident frequency and 1/2 int_0^pi sin(Theta)
    dTheta = 1, so under a flat incident spectrum (the spline basis sums to
    one, including its constant continuation) a row of the tile is exactly
    sqrt(pi) W(a, u_n + s_out); doubling the Theta nodes moves the tile by less
    than 1e-11 (measured 1e-13; halving them, 3e-10)."""
    u = np.concatenate([-np.geomspace(30, 2, 5), np.linspace(-1.5, 1.5, 9), np.geomspace(2, 30, 5)])
    spl = NaturalSpline(u)
    a, s_in, s_out = 0.01, 0.3, -0.2
    T = RD.aa_tile(spl, a, s_in, s_out)
    ref = np.sqrt(np.pi) * voigt_faraday(a, u + s_out)
    assert np.max(np.abs(T.sum(axis=1) - ref)) < 1e-12 * np.max(np.abs(ref))
    T2 = RD.aa_tile(spl, a, s_in, s_out, n_theta=96)
    assert np.max(np.abs(T - T2)) < 1e-11 * np.max(np.abs(T))


def test_sampled_rows_match_the_full_operator():
    """The one-by-one evaluations that write the full-size reference values
    (Sigma at one (height, direction) with its own Kirchhoff factor f; Lambda
    along one ray) equal the rows of the full operator on a small case with
    bulk velocities, so that the frame changes enter."""
    cfg = inputs.mgii(n_z=3, n_core_each=5, n_wing=4, n_mu_half=1, n_chi=4, seed=13)
    P = Problem(cfg)
    assert np.max(np.abs(P.ub)) > 0.1
    x = inputs.seeded_vector(P.shape(), 5, 0.1, 1.0)
    x[..., 1:] *= 0.05
    full = P.apply_sigma(x)
    for iz, o in ((1, 2), (2, 6)):
        eps, f = P.sigma_sample(x, iz, o)
        assert np.max(np.abs(f - P.f[iz, o])) < 1e-12
        assert np.max(np.abs(eps - full[iz, o])) < 1e-12 * np.max(np.abs(full[iz, o, :, 0]))
    lam = P.formal_solution(x)
    for o, n in ((0, 3), (5, 9)):
        assert np.max(np.abs(P.lambda_ray(x, o, n) - lam[:, o, n])) < 1e-14 * np.max(np.abs(lam))


@pytest.mark.parametrize("case", ["mgii", "twolevel"])
def test_preconditioner_oracle(case):
    """Sect. 5.2 / App. F preconditioner (oracle/preconditioner.py):
    * one sweep from zero is P_hat^-1, which equals the dense inverse of
      Id - Lambda_ii Sigma_hat at every height (brute force);
    * the Richardson sweeps converge to the exact inverse of P: P (P^-1 y) = y;
    * Q, U, V pass through, and zero sweeps are the identity;
    * Sigma*'s photon budget: under a flat isotropic field the R_II part of
      Phi_bar returns alpha0 k phi* exactly (every F integrates to sqrt(pi) W)
      and the R_III part (beta0 - alpha0) k phi* times the profile's area
      inside the grid span (adaptive quadrature here)."""
    from oracle.preconditioner import Preconditioner, _levels
    if case == "mgii":
        cfg = inputs.mgii(n_z=4, n_core_each=4, n_wing=4, n_mu_half=1, n_chi=4, seed=19)
    else:
        cfg = inputs.twolevel_slab(n_z=6, n_x=9, n_mu_half=1, n_chi=4, eps=1e-2)
    P = Problem(cfg, normalise=False)
    C = Preconditioner(P)
    nz, nO, N = P.nz, P.nO, P.nN
    y = inputs.seeded_vector(P.shape(), 3, -1.0, 1.0)
    x1 = C.apply_inv(y, 1)
    for iz in range(nz):
        S = np.broadcast_to(C.Phi[iz][None, :, None, :] * P.wang[None, None, :, None], (nO, N, nO, N))
        B = np.eye(nO * N) - C.lii[iz].ravel()[:, None] * S.reshape(nO * N, nO * N)
        ref = np.linalg.solve(B, y[iz, ..., 0].ravel())
        assert np.max(np.abs(x1[iz, ..., 0].ravel() - ref)) < 1e-12 * np.max(np.abs(ref))
    x = C.apply_inv(y, 60)
    assert np.linalg.norm(C.apply_P(x) - y) < 1e-12 * np.linalg.norm(y)
    assert np.array_equal(x[..., 1:], y[..., 1:]) and np.array_equal(C.apply_inv(y, 0), y)
    E, cg = _levels(P.atom, P.nu0)
    for iz in range(nz):
        a, u = P.a[iz], P.u[iz]
        prof = lambda v: sum(c * voigt_faraday(a, v + Eg / P.dnuD[iz]).real for Eg, c in zip(E, cg)) / np.sqrt(np.pi)
        span = quad(prof, u[0], u[-1], limit=400, points=[-Eg / P.dnuD[iz] for Eg in E], epsabs=1e-13)[0]
        a0 = (1 - P.eps[iz]) * (1 - P.rE[iz])
        b0 = 1 - P.eps[iz]
        ref = P.k[iz] * prof(u) * (a0 + (b0 - a0) * span)
        assert np.max(np.abs(C.Phi[iz].sum(axis=1) - ref)) < 1e-9 * np.max(ref)


def test_gmres_matches_dense_solve():
    """Brute force on a tiny grid: assemble A column by column, solve by LU;
    the same for A^T and the adjoint solve."""
    cfg = inputs.mgii(n_z=4, n_core_each=5, n_wing=6, n_mu_half=1, n_chi=2, seed=11)
    P = Problem(cfg)
    n = int(np.prod(P.shape()))
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = P.apply_A(e.reshape(P.shape())).ravel()
    b = P.rhs().ravel()
    xd = np.linalg.solve(A, b)
    xg, hist = P.solve(tol=1e-13)
    assert np.max(np.abs(xg.ravel() - xd)) < 1e-10 * np.max(np.abs(xd))
    # the transposed operator (adjoint, not in the paper) against the transpose
    # of the same brute-force matrix, and its GMRES solve against LU on A^T
    y = inputs.seeded_vector(P.shape(), 3, -1.0, 1.0)
    ATy = P.apply_AT(y).ravel()
    assert np.max(np.abs(ATy - A.T @ y.ravel())) < 1e-13 * np.max(np.abs(ATy))
    g = inputs.seeded_vector(P.shape(), 4, 0.1, 1.0)
    ld = np.linalg.solve(A.T, g.ravel())
    lg, _ = P.solve_adjoint(g, tol=1e-13)
    assert np.max(np.abs(lg.ravel() - ld)) < 1e-10 * np.max(np.abs(ld))


@pytest.mark.slow
def test_sqrt_eps_law():
    """Isothermal CRD two-level atmosphere, constant eps: S(0) = sqrt(eps) B
    (the sqrt(eps) law, exact for isotropic scattering in a semi-infinite
    medium); 8 % allows for the Rayleigh phase matrix and the discretisation."""
    eps = 1e-2
    cfg = inputs.twolevel_slab(n_z=60, n_x=15, n_mu_half=2, n_chi=4, eps=eps, r_el=1 - 1e-12,
                               tau_min=1e-5, tau_max=1e5)
    P = Problem(cfg)
    x, _ = P.solve(tol=1e-11)
    S = (P.apply_sigma(x) + P.eps_th)[..., 0] / P.eta1
    assert abs(S[-1, 0, P.nN // 2] / np.sqrt(eps) - 1.0) < 0.08
    assert abs(S[0, 0, P.nN // 2] - 1.0) < 0.01          # thermalised at depth


def test_emergent_along_grid_direction_is_the_solution():
    """The extra formal solution of Sect. 6.2, taken along a direction of the
    grid, must return the solution's own emergent Stokes vector."""
    cfg = inputs.twolevel_slab(n_z=6, n_x=9, n_mu_half=2, n_chi=4, eps=1e-2)
    cfg["atm"]["B_G"][:] = 30.0
    P = Problem(cfg)
    x, _ = P.solve(tol=1e-13)
    for o in [i for i in range(P.nO) if P.mu[i] > 0][:3]:
        e = P.emergent(x, P.mu[o], P.chi[o])
        assert np.max(np.abs(e - x[-1, o])) < 1e-10 * np.max(np.abs(x[-1, o]))


def test_gradient_reference_differences_converged():
    """The stored oracle derivatives of the gradient test (central differences
    of J over forward solves at steps h and h/2, tests/golden/make_golden.py)
    differ by their O(h^2) truncation alone: within 1e-4 of the largest
    component of each kind (measured 2.3e-5 for B, 4.8e-6 for theta_B, 5.5e-5
    for chi_B)."""
    import os
    G = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grad_mgii_small.npz"))
    for k in range(3):
        fd, fh = G["fd"][:, k], G["fd_half"][:, k]
        assert np.max(np.abs(fd - fh)) < 1e-4 * np.max(np.abs(fd)), k


# ---------------------------------------------------------------- polarised formal solution
def _magnetised_homogeneous_slab(n_z, formal_solver="delo_linear"):
    """Two-level slab with every height alike (T, a, k, B): K is constant
    along each ray, so the transfer equation has a closed-form solution."""
    cfg = inputs.twolevel_slab(n_z=n_z, n_x=9, n_mu_half=2, n_chi=4, a=2e-2)
    atm = cfg["atm"]
    atm["z_km"] = np.linspace(0.0, 4.0, n_z)
    atm["B_G"][:] = 900.0
    atm["thetaB"][:] = 0.6
    atm["chiB"][:] = 0.9
    return Problem(cfg, normalise=False, formal_solver=formal_solver)


def _delo_error_vs_matrix_exponential(n_z, formal_solver="delo_linear"):
    """Max error of the emergent Stokes vectors of formal_solution for a
    constant emissivity e against I = exp(-K l) I0 + (Id - exp(-K l)) K^-1 e."""
    from scipy.linalg import expm
    P = _magnetised_homogeneous_slab(n_z, formal_solver)
    e = np.array([1.0, 0.3, -0.2, 0.15])
    out = P.formal_solution(np.broadcast_to(e, P.shape()).copy(), boundary=True)
    err = scale = 0.0
    for o in range(P.nO):
        l = (P.z[-1] - P.z[0]) / abs(P.mu[o])
        up = P.mu[o] > 0
        I0 = np.array([P.WT[0], 0.0, 0.0, 0.0]) if up else np.zeros(4)
        for n in range(P.nN):
            K = P.K[0, o, n]
            E = expm(-K * l)
            exact = E @ I0 + (np.eye(4) - E) @ np.linalg.solve(K, e)
            got = out[-1 if up else 0, o, n]
            err = max(err, np.max(np.abs(got - exact)))
            scale = max(scale, np.max(np.abs(exact)))
    return err / scale, P


def test_polarised_delo_converges_to_matrix_exponential():
    """Sect. 3: the DELO-linear step with K' = K/eta_I - Id, in a homogeneous
    slab with a 900 G field (Zeeman absorption in Q, U, V and magneto-optical
    terms up to 17 eta_I in the wings) and a constant emissivity with all four
    Stokes parameters, against the exact solution of dI/ds = e - K I,
        I(l) = exp(-K l) I0 + (Id - exp(-K l)) K^-1 e,
    from the lower boundary (W_T, 0, 0, 0) upwards and from zero downwards.
    DELO-linear is second order: halving the step divides the error by 4
    (measured 5.2e-5, 1.3e-5, 3.3e-6 at 21, 41, 81 heights).  A flipped sign
    of alpha K'_{k-1} or of beta K'_k, or a transposed K', stalls at ~0.1-0.2."""
    e21, _ = _delo_error_vs_matrix_exponential(21)
    e41, P = _delo_error_vs_matrix_exponential(41)
    off = np.abs(P.K * (1.0 - np.eye(4))) / P.K[..., :1, :1]
    assert np.max(off) > 1.0          # polarised: off-diagonal K above eta_I in places
    assert e41 < 2e-5
    assert 3.5 < e21 / e41 < 4.5


# ---------------------------------------------------------------- redistribution symmetry
def _point_kernels(P):
    """Replace the spline-basis integrals of the discrete operator by point
    values at the frequency nodes: R_II tiles become F(Theta, u_m + s, u_n + s')
    and the R_III incident weights W(a, u_m + s1) + W(a, u_m + s2)^*, so that
    a block is the redistribution matrix R(u_n, Omega; u_m, Omega') itself
    (times k w_Omega')."""
    u = P.u

    def tile(iz, theta, s_in, s_out):
        if theta == 0.0:
            return np.zeros((u[iz].size, u[iz].size), complex)
        return RD.F_kernel(theta, u[iz][None, :] + s_in, u[iz][:, None] + s_out, P.a[iz])
    P.tile = tile
    P.r3 = lambda iz, s1, s2: voigt_faraday(P.a[iz], u[iz] + s1) + np.conj(voigt_faraday(P.a[iz], u[iz] + s2))
    return P


@pytest.mark.parametrize("case", ["twolevel", "mgii"])
def test_redistribution_symmetry_zero_field(case):
    """R(nu, Omega; nu', Omega') = R(nu', Omega'; nu, Omega)^T for a static
    atom without a magnetic field (reciprocity of the scattering: the
    Rayleigh-type phase matrix of an isotropic atom is symmetric, and F is
    symmetric in its frequencies), for R_II + R_III with J-state interference
    (two-term atom).  Checked on R at the nodes (point-valued kernels; the
    spline-basis integrals of the discrete operator are not symmetric by
    construction): block(o, o')/w_o' against the transposed block(o', o)/w_o,
    for every pair off the forward direction (measured 2e-17 two-level,
    1.7e-12 two-term)."""
    if case == "twolevel":
        cfg = inputs.twolevel_slab(n_z=2, n_x=7, n_mu_half=2, n_chi=4, eps=1e-2, r_el=0.3)
    else:
        cfg = inputs.mgii(n_z=2, n_core_each=3, n_wing=2, n_mu_half=2, n_chi=4, seed=3)
    atm = cfg["atm"]
    nz = len(atm["z_km"])
    atm["B_G"] = np.zeros(nz)
    atm["v_kms"] = np.zeros((nz, 3))
    P = _point_kernels(Problem(cfg, normalise=False))
    err = scale = 0.0
    for o in range(P.nO):
        for op in range(P.nO):
            if P.cls[o, op] == 0:
                continue
            b1 = P.block(0, o, op) / P.wang[op]                  # [n, i, m, j]
            b2 = P.block(0, op, o) / P.wang[o]
            err = max(err, np.max(np.abs(b1 - np.einsum("mjni->nimj", b2))))
            scale = max(scale, np.max(np.abs(b1)))
    assert err < 1e-10 * scale


# ---------------------------------------------------------------- R_III conjugate pairing
def _kh_case():
    """The Mg II atom of the Kramers-Heisenberg pin: B = 360 G, a = 0.05, so
    that the upper-state coherences (k_u != k_u') carry weight."""
    cfg = inputs.mgii(n_z=2, n_core_each=6, n_wing=3, n_mu_half=1, n_chi=4, seed=7)
    atm = cfg["atm"]
    nz = len(atm["z_km"])
    for key, val in (("a", 0.05), ("eps", 0.0), ("r_el", 0.0), ("B_G", 360.0), ("thetaB", 0.7),
                     ("chiB", 0.4)):
        atm[key] = np.full(nz, val)
    atm["v_kms"] = np.zeros((nz, 3))
    return Problem(cfg, normalise=False)


def _r2_and_r3_parts(P, reduce):
    """Sum over direction pairs of reduce(block) with R_II alone (alpha =
    beta = X) and with R_III alone (alpha = 0, beta - alpha = X), X the
    height's alpha: the same coefficients on both sides."""
    iz = 0
    X = P.alpha[iz].copy()
    out = []
    for al, be in ((X, X), (0.0 * X, X)):
        P.alpha[iz], P.beta[iz] = al, be.copy()
        out.append(sum(reduce(P.block(iz, o, op), o, op) for o in range(P.nO) for op in range(P.nO)))
    P.alpha[iz], P.beta[iz] = X, X
    return out


def test_r3_emission_bracket_matches_r2_under_white_light():
    """Eq. RIIIQKKp's emission bracket [W(u + s_{k_u' k_l'}) + W(u + s_{k_u k_l'})^*]
    against Eq. RQIIKKp (whose pairing the Kramers-Heisenberg pin fixes).
    Under incident light flat in frequency, frequency-coherent (R_II) and
    collisionally redistributed (R_III) scattering emit the same spectrum:
    every F integrates over the incident frequency to sqrt(pi) W(a, u + s_out)
    (the Def-B tiles do so exactly), and the R_III incident bracket to
    2 sqrt(pi) over the whole line.  With equal coefficients (c3 = c2 / 2) the
    two emissivities must agree, for an anisotropic, polarised incident field
    in a field that makes the upper-state coherences matter.  The R_III
    weights are rescaled to the full-line integral 2 sqrt(pi) (the oracle
    stops them at the grid span; they are pinned against adaptive quadrature
    separately).  Measured 5e-14; swapping which W of the emission bracket is
    conjugated gives 0.11."""
    P = _kh_case()
    N = P.nN
    r3 = P.r3
    P.r3 = lambda iz, s1, s2: r3(iz, s1, s2) * (2.0 * np.sqrt(np.pi) / r3(iz, s1, s2).sum())
    rng = np.random.default_rng(3)
    inc = rng.uniform(0.5, 1.5, (P.nO, 4))
    inc[:, 1:] *= 0.3

    def emit(blk, o, op):
        e = np.zeros((P.nO, N, 4))
        e[o] = blk.reshape(N, 4, N, 4).sum(axis=2) @ inc[op]
        return e
    e2, e3 = _r2_and_r3_parts(P, emit)
    assert np.max(np.abs(e2 - e3)) < 1e-12 * np.max(np.abs(e2[..., 0]))


def test_r3_incident_bracket_matches_r2_under_flat_emission():
    """Eq. RIIIQKKp's incident bracket [W(u' + s_{k_u' k_l}) + W(u' + s_{k_u k_l})^*]
    against Eq. RQIIKKp: integrated over the outgoing frequency, R_II becomes
    c2 X sqrt(pi) [W(u' + s_{k_u' k_l}) + W(u' + s_{k_u k_l})^*] (F is symmetric
    in its frequencies, so it integrates over u to sqrt(pi) W(a, u' + s_in);
    both pinned above), and R_III c3 X 2 sqrt(pi) times its incident bracket
    (every W integrates to sqrt(pi) over u).  Here every kernel is replaced by
    that exact integral and the incident side by its values at the nodes; the
    absorption sides must then agree per incident frequency, Stokes parameter
    and direction pair.  Measured 4e-16; swapping the arguments of the R_III
    incident weights, or the conjugated G of R_II, gives 1.0."""
    import oracle.problem as OP
    P = _kh_case()
    u = P.u[0]
    sp = np.sqrt(np.pi)
    P.tile = lambda iz, th, s_in, s_out: np.broadcast_to(sp * voigt_faraday(P.a[iz], u + s_in), (u.size, u.size))
    P.r3 = lambda iz, s1, s2: voigt_faraday(P.a[iz], u + s1) + np.conj(voigt_faraday(P.a[iz], u + s2))
    vf = OP.voigt_faraday
    OP.voigt_faraday = lambda a, x: sp * np.ones(np.shape(x), dtype=complex)   # int W(a, u + s) du
    try:
        a2, a3 = _r2_and_r3_parts(P, lambda blk, o, op: blk[0])   # every outgoing row is the integral
    finally:
        OP.voigt_faraday = vf
    assert np.max(np.abs(a2 - a3)) < 1e-12 * np.max(np.abs(a2))


# ---------------------------------------------------------------- narrow-band CLV signals
def test_narrowband_closed_forms():
    """Sect. 6.5's Gaussian-weighted wavelength integral (FWHM 35 A, limits
    +-30 A around 1215.67 A) on ascending wavelength nodes: a constant profile
    c gives c erf(Delta / (sqrt(2) sigma)) (the constant continuation covers
    the limits beyond the grid); an odd profile about lambda_0 on a symmetric
    grid covering the limits gives 0; a Gaussian profile of width tau gives
    (rho / sigma) erf(Delta / (sqrt(2) rho)), 1/rho^2 = 1/sigma^2 + 1/tau^2
    (to the spline's interpolation error, 1e-6 on a 0.2 A grid)."""
    from oracle.narrowband import narrowband, sigma_of_fwhm
    from scipy.special import erf
    lam0, fwhm, dl = 1215.67, 35.0, 30.0
    s = sigma_of_fwhm(fwhm)
    assert abs(2 * np.sqrt(2 * np.log(2)) * s - fwhm) < 1e-12
    lam = lam0 + np.concatenate([-np.geomspace(20, 1.5, 8), np.linspace(-1.4, 1.4, 9), np.geomspace(1.5, 20, 8)])
    X = np.full((lam.size, 4), 0.7)
    np.testing.assert_allclose(narrowband(lam, X, lam0, fwhm, dl), 0.7 * erf(dl / (np.sqrt(2) * s)), rtol=1e-10)
    lam = lam0 + np.linspace(-40.0, 40.0, 161)
    X = np.stack([lam - lam0, (lam - lam0) ** 3] * 2, axis=1)
    assert np.max(np.abs(narrowband(lam, X, lam0, fwhm, dl))) < 1e-9 * np.max(np.abs(X))
    lam = lam0 + np.arange(-40.0, 40.0 + 1e-9, 0.2)
    tau = 3.0
    X = np.exp(-0.5 * ((lam - lam0) / tau) ** 2)[:, None] * np.ones(4)
    rho = 1.0 / np.sqrt(1.0 / s ** 2 + 1.0 / tau ** 2)
    np.testing.assert_allclose(narrowband(lam, X, lam0, fwhm, dl), rho / s * erf(dl / (np.sqrt(2) * rho)),
                               rtol=1e-6)


def test_delopar_parabolic_source_exact_and_linear_limit():
    """DELOPAR (Sect. 3; the source vector parabolic through the upwind,
    current and downwind points, K'I linear): in an unmagnetised homogeneous
    slab (K' = 0) a source quadratic in height, hence in optical depth along
    every ray, is integrated exactly at every point whose step has a
    downwind neighbour (the last step of a ray is linear):
        I(T) = I0 e^{-T} + int_0^T e^{-(T - t)} S(t) dt  in closed form;
    a linear source gives DELO-linear's solution at every point."""
    from oracle.problem import delo_coeffs
    cfg = inputs.twolevel_slab(n_z=9, n_x=7, n_mu_half=2, n_chi=4, a=2e-2)
    cfg["atm"]["z_km"] = np.linspace(0.0, 3.0, 9) + np.array([0, .1, -.05, .2, 0, -.1, .05, 0, 0])
    par = Problem(cfg, normalise=False, formal_solver="delopar")
    lin = Problem(cfg, normalise=False)
    z = par.z
    S = 0.3 + 0.8 * (z - z[0]) - 0.15 * (z - z[0]) ** 2
    eps = np.zeros(par.shape())
    eps[..., 0] = (S[:, None, None] * par.eta1[:, :, :])
    out = par.formal_solution(eps, boundary=True)
    for o in range(par.nO):
        mu = par.mu[o]
        for n in range(par.nN):
            eta = par.eta1[0, o, n]
            # along the ray: tau = eta (z - z_start) / |mu| from the entry point
            if mu > 0:
                zs, k = z[0], par.nz - 2
                I0 = par.WT[0]
                Sf = lambda t: 0.3 + 0.8 * (mu * t / eta) - 0.15 * (mu * t / eta) ** 2
            else:
                zs, k = z[-1], 1
                I0 = 0.0
                Sf = lambda t: 0.3 + 0.8 * (z[-1] - z[0] + mu * t / eta) - 0.15 * (z[-1] - z[0] + mu * t / eta) ** 2
            T = eta * abs(z[k] - zs) / abs(mu)
            exact = I0 * np.exp(-T) + quad(lambda t: np.exp(-(T - t)) * Sf(t), 0, T, epsabs=1e-14, epsrel=1e-13)[0]
            assert abs(out[k, o, n, 0] - exact) < 1e-11 * max(1.0, abs(exact)), (o, n)
    S = 0.3 + 0.8 * (z - z[0])
    eps[..., 0] = S[:, None, None] * par.eta1
    np.testing.assert_allclose(par.formal_solution(eps, boundary=True), lin.formal_solution(eps, boundary=True),
                               rtol=1e-12, atol=1e-13)


def test_delopar_polarised_slab_converges_to_matrix_exponential():
    """DELOPAR in the magnetised homogeneous slab of the DELO-linear pin: the
    K'I term is linear over a step, so the error falls at second order too
    (the source there is constant, which both schemes integrate exactly, so
    the errors equal DELO-linear's: 5.2e-5, 1.3e-5, 3.3e-6 at 21, 41, 81
    heights).  Swapping psi_M and psi_P fails the parabolic-source pin."""
    e21, _ = _delo_error_vs_matrix_exponential(21, "delopar")
    e41, _ = _delo_error_vs_matrix_exponential(41, "delopar")
    assert e41 < 2e-5
    assert 3.5 < e21 / e41 < 4.5


# ---------------------------------------------------------------- continuum (App. A)
def test_continuum_phase_matrix_and_photon_budget():
    """App. A's coherent continuum scattering uses the dipole phase matrix
    (sum over K <= 2 of (-1)^Q T^K_Q T^K_-Q, every W_K = 1).  The oracle builds
    it from the polarisation bases (3/4 Tr(sigma_i J sigma_j J^T)); it must
    equal the frequency-integrated R_II phase matrix of the J 0 -> 1 atom at
    B = 0 (W_1 = W_2 = 1), built from the atom's scattering amplitudes, for
    every direction pair; integrate to one over incident directions; obey
    reciprocity; and under an isotropic unpolarised field W return sigma_c W
    on Stokes I and nothing on Q, U, V."""
    cfg = inputs.with_continuum(inputs.twolevel_slab(n_z=3, n_x=7, n_mu_half=2, n_chi=4, eps=1e-2), 1e-3, 0.4)
    P = Problem(cfg, normalise=False)
    for o in range(P.nO):
        tot = np.zeros((4, 4))
        for op in range(P.nO):
            R = P.rayleigh(P.mu[o], P.chi[o], P.mu[op], P.chi[op])
            A = _integrated_phase(P, 0, P.amplitudes(0, P.mu[o], P.chi[o]), P.amplitudes(0, P.mu[op], P.chi[op]))
            assert np.max(np.abs(R - A)) < 1e-12
            assert np.max(np.abs(R - P.rayleigh(P.mu[op], P.chi[op], P.mu[o], P.chi[o]).T)) < 1e-13
            tot += P.wang[op] * R
        assert abs(tot[0, 0] - 1.0) < 1e-12 and np.max(np.abs(tot[1:, 0])) < 1e-12
    W = np.zeros(P.shape())
    W[..., 0] = 0.8
    full = Problem(cfg, normalise=False)
    for iz in range(P.nz):
        C = np.stack([full.continuum_block(iz, P.mu[o], P.chi[o]) for o in range(P.nO)])  # [o, n, i, o', j]
        e = np.einsum("onipj,pnj->oni", C, W[iz])
        np.testing.assert_allclose(e[..., 0], 0.8 * P.sig_c[iz][None, :] * np.ones((P.nO, 1)), rtol=1e-12)
        assert np.max(np.abs(e[..., 1:])) < 1e-12 * 0.8 * np.max(P.sig_c[iz])
