"""Seeded synthetic inputs for the five workloads (numpy only).

This module only draws and lays out input arrays: atmospheres, atoms and
grids.  It holds none of the method's arithmetic (no Doppler widths, no
profiles, no optical depths, no quadrature), so both the CUDA library and the
FP64 oracle can consume what it returns without sharing any computation.

Workloads (the synthetic stand-ins for the paper's FAL-C Mg II h&k and
H I Ly-alpha runs, Sect. 6.1-6.2 and Table 1):

* ``twolevel_slab``   two-level J=0->1 atom, static, unmagnetised, isothermal
                      slab, 40 heights, 21 reduced frequencies in [-8, 8],
                      2 mu x 4 chi directions.  FP64.
* ``mgii``            Mg II h&k-like two-term atom (Table 1), 70 heights,
                      200 wavelengths, 4+4 mu x 8 chi, B <= 100 G, |v| <= 5 km/s.
* ``hi_lya``          H I Ly-alpha-like two-term atom (Table 1), 90 heights,
                      150 wavelengths, 6+6 mu x 8 chi, B <= 50 G.
* ``mgii_batch``      256 Mg II-like instances with 50..130 heights and
                      120..220 wavelengths (seeds 400 + i).
* ``mgii_adjoint``    the Mg II atmosphere with a seeded +-20 % perturbation
                      of the magnetic parameters (target profiles).

All sizes can be reduced with keyword arguments so that tests can run the
same physics on grids the FP64 oracle finishes in seconds.
"""
import numpy as np

# grid kinds understood by set_quadrature
GRID_LAMBDA = 0   # vacuum wavelengths in Angstrom, ascending
GRID_X = 1        # reduced frequencies x = (nu0 - nu)/dnuD_ref, ascending,
                  # dnuD_ref = Doppler width at the first (lowest) height

ATOM_TWO_LEVEL = 0
ATOM_TWO_TERM = 1

MODE_AD = 0
MODE_AA = 1

MU_GL_HEMISPHERES = 0   # one Gauss-Legendre rule of n_mu_half nodes per hemisphere
MU_GL_FULL = 1          # one Gauss-Legendre rule of 2 n_mu_half nodes on [-1, 1]

# Table 1 of the paper (NIST energies, vacuum wavelengths, A_ul averages)
MGII_TABLE = dict(mass_amu=24.305, E_u_cm=(35669.31, 35760.88), A_ul=2.59e8)
HI_TABLE = dict(mass_amu=1.008, E_u_cm=(82258.92, 82259.29), A_ul=6.265e8)


def _smooth(rng, z, amp=0.1, ncos=4):
    """1 + sum of `ncos` cosines in z with seeded phases; relative amplitude `amp`."""
    zn = (z - z.min()) / max(z.max() - z.min(), 1e-30)
    out = np.zeros_like(zn)
    for k in range(1, ncos + 1):
        out += np.cos(np.pi * k * zn + rng.uniform(0, 2 * np.pi)) / ncos
    return 1.0 + amp * out


def _geom(lo, hi, n):
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))


def twolevel_slab(n_z=40, n_x=21, n_mu_half=1, n_chi=4, tau_min=1e-4, tau_max=1e4,
                  a=1e-3, eps=1e-4, r_el=0.1, seed=1):
    """Two-level 0->1 isothermal static slab (reduced-frequency grid).

    Heights are placed so that the line-centre vertical optical depth
    (k_line * z / sqrt(pi) in the a -> 0 limit) runs log-spaced from tau_min at
    the top to tau_max at the bottom.  k_line = sqrt(pi) km^-1.
    """
    tau = np.geomspace(tau_min, tau_max, n_z)
    z = np.sort(-tau)                      # km, ascending (bottom first)
    t = -1.0 + np.arange(n_x) / ((n_x - 1) / 2.0)
    x = 8.0 * np.sinh(3.0 * t) / np.sinh(3.0)
    ones = np.ones(n_z)
    atm = dict(
        z_km=z, T_K=5000.0 * ones, xi_kms=0.0 * ones, a=a * ones, eps=eps * ones,
        r_el=r_el * ones, k_line=np.sqrt(np.pi) * ones, W_T=ones.copy(),
        B_G=0.0 * ones, thetaB=0.0 * ones, chiB=0.0 * ones, v_kms=np.zeros((n_z, 3)))
    atom = dict(kind=ATOM_TWO_LEVEL, twoS=0, E_u_cm=(1e8 / 4226.728, 1e8 / 4226.728),
                mass_amu=40.078, g_s=2.0, nu0_hz=0.0)
    quad = dict(grid=x, grid_kind=GRID_X, n_mu_half=n_mu_half, n_chi=n_chi, mode=MODE_AD,
                mu_rule=MU_GL_FULL if n_mu_half == 1 else MU_GL_HEMISPHERES)
    return dict(name="twolevel_slab", atom=atom, atm=atm, quad=quad, precision="fp64",
                gmres_tol=1e-10, seed=seed)


def _chromosphere(rng, n_z, T_top_extra, z_lo=-100.0, z_hi=2219.43):
    z = np.linspace(z_lo, z_hi, n_z)
    T = 4500.0 + 2000.0 * np.exp(-(z - z_lo) / 150.0) \
        + T_top_extra * 0.5 * (1.0 + np.tanh((z - 1600.0) / 350.0))
    T = T * _smooth(rng, z, 0.03)
    xi = np.linspace(1.0, 5.0, n_z)
    return z, T, xi


def _velocity(z, vmax):
    """Bulk velocity law of Sect. 6.4 (v_z Gaussian x erf, horizontal 0.7|v_z|
    rotating with height), rescaled to max|v| = vmax km/s."""
    from math import erf
    zmin, zmax = z.min(), z.max()
    vz = -10.0 * np.exp(-((z - 2100.0) / 500.0) ** 2) * \
        (1.0 + np.array([erf((2100.0 - zz) / 150.0) for zz in z]))
    chiv = -2.0 * np.pi * (z - zmin) / (zmax - zmin) + np.pi
    vx = 0.7 * np.abs(vz) * np.cos(chiv)
    vy = 0.7 * np.abs(vz) * np.sin(chiv)
    v = np.stack([vx, vy, vz], axis=1)
    vmag = np.sqrt((v ** 2).sum(1)).max()
    return v * (vmax / vmag) if vmag > 0 else v


def _wien(T, lam_A):
    """Wien function exp(-h nu0/(k T)) normalised to 1 at the lowest height."""
    hc_over_k = 1.438776877e8          # K Angstrom
    return np.exp(-hc_over_k / lam_A * (1.0 / T - 1.0 / T[0]))


def _lines_grid(centers, n_core_each, half_core, n_wing_total, wing_out, d0):
    """Uniform cores of +-half_core around each line + log-spaced wings."""
    centers = sorted(centers)
    parts = [np.linspace(c - half_core, c + half_core, n_core_each) for c in centers]
    lo_edge, hi_edge = centers[0] - half_core, centers[-1] + half_core
    if len(centers) == 1:
        nb = n_wing_total // 2
        parts.append(lo_edge - _geom(d0, wing_out, nb))
        parts.append(hi_edge + _geom(d0, wing_out, n_wing_total - nb))
    else:
        nb = n_wing_total // 3
        nm = n_wing_total - 2 * nb
        parts.append(lo_edge - _geom(d0, wing_out, nb))
        parts.append(hi_edge + _geom(d0, wing_out, nb))
        gap_lo, gap_hi = centers[0] + half_core, centers[1] - half_core
        half = 0.5 * (gap_hi - gap_lo)
        d = _geom(d0, 0.95 * half, nm // 2)
        parts.append(gap_lo + d)
        parts.append(gap_hi - _geom(d0, 0.95 * half, nm - nm // 2))
    lam = np.sort(np.concatenate(parts))
    assert np.all(np.diff(lam) > 0)
    return lam


def mgii(n_z=70, n_core_each=70, n_wing=60, n_mu_half=4, n_chi=8, Bmax=100.0, vmax=5.0,
         seed=2, T_top_extra=5500.0, k_span=(1e-3, 1e6)):
    """Mg II h&k-like two-term atom (Table 1) in a synthetic chromosphere."""
    rng = np.random.default_rng(seed)
    z, T, xi = _chromosphere(rng, n_z, T_top_extra)
    lam_h = 1e8 / MGII_TABLE["E_u_cm"][0]
    lam_k = 1e8 / MGII_TABLE["E_u_cm"][1]
    # line-centre k-line opacity: exponential in z with a smooth factor, scaled
    # so that (roughly) k_line * H * 0.38 spans k_span from top to bottom
    H = (z[-1] - z[0]) / np.log(k_span[1] / k_span[0])
    k_line = (k_span[1] / (0.38 * H)) * np.exp(-(z - z[0]) / H) * _smooth(rng, z, 0.1)
    eps = np.exp(np.linspace(np.log(1e-3), np.log(1e-6), n_z))
    a = np.exp(np.linspace(np.log(1e-2), np.log(1e-4), n_z)) * _smooth(rng, z, 0.1)
    r_el = np.clip(0.3 * _smooth(rng, z, 0.5), 0.02, 0.9)
    B = rng.uniform(0.0, Bmax, n_z)
    thetaB = np.arccos(rng.uniform(-1.0, 1.0, n_z))
    chiB = rng.uniform(0.0, 2.0 * np.pi, n_z)
    v = _velocity(z, vmax)
    W_T = _wien(T, 0.5 * (lam_h + lam_k))
    atm = dict(z_km=z, T_K=T, xi_kms=xi, a=a, eps=eps, r_el=r_el, k_line=k_line, W_T=W_T,
               B_G=B, thetaB=thetaB, chiB=chiB, v_kms=v)
    lam = _lines_grid([lam_k, lam_h], n_core_each, 1.0, n_wing, 10.0, 0.05)
    atom = dict(kind=ATOM_TWO_TERM, twoS=1, E_u_cm=MGII_TABLE["E_u_cm"],
                mass_amu=MGII_TABLE["mass_amu"], g_s=2.0, nu0_hz=0.0)
    quad = dict(grid=lam, grid_kind=GRID_LAMBDA, n_mu_half=n_mu_half, n_chi=n_chi, mode=MODE_AD)
    return dict(name="mgii", atom=atom, atm=atm, quad=quad, precision="fp32",
                gmres_tol=1e-6, seed=seed)


def hi_lya(n_z=90, n_core=90, n_wing=60, n_mu_half=6, n_chi=8, Bmax=50.0, vmax=5.0,
           seed=3, mode=MODE_AD):
    """H I Ly-alpha-like two-term atom (Table 1), atmosphere up to ~2e4 K."""
    rng = np.random.default_rng(seed)
    z, T, xi = _chromosphere(rng, n_z, 15500.0)
    lam0 = 1e8 / (HI_TABLE["E_u_cm"][0] / 3.0 + 2.0 * HI_TABLE["E_u_cm"][1] / 3.0)
    H = (z[-1] - z[0]) / np.log(1e9)
    k_line = (1e6 / (0.56 * H)) * np.exp(-(z - z[0]) / H) * _smooth(rng, z, 0.1)
    eps = np.exp(np.linspace(np.log(1e-3), np.log(1e-6), n_z))
    a = np.exp(np.linspace(np.log(1e-2), np.log(1e-4), n_z)) * _smooth(rng, z, 0.1)
    r_el = np.clip(0.3 * _smooth(rng, z, 0.5), 0.02, 0.9)
    B = rng.uniform(0.0, Bmax, n_z)
    thetaB = np.arccos(rng.uniform(-1.0, 1.0, n_z))
    chiB = rng.uniform(0.0, 2.0 * np.pi, n_z)
    v = _velocity(z, vmax)
    W_T = _wien(T, lam0)
    atm = dict(z_km=z, T_K=T, xi_kms=xi, a=a, eps=eps, r_el=r_el, k_line=k_line, W_T=W_T,
               B_G=B, thetaB=thetaB, chiB=chiB, v_kms=v)
    lam = _lines_grid([lam0], n_core, 1.5, n_wing, 20.0, 0.05)
    atom = dict(kind=ATOM_TWO_TERM, twoS=1, E_u_cm=HI_TABLE["E_u_cm"],
                mass_amu=HI_TABLE["mass_amu"], g_s=2.0, nu0_hz=0.0)
    quad = dict(grid=lam, grid_kind=GRID_LAMBDA, n_mu_half=n_mu_half, n_chi=n_chi, mode=mode)
    return dict(name="hi_lya", atom=atom, atm=atm, quad=quad, precision="fp32",
                gmres_tol=1e-6, seed=seed)


def with_continuum(cfg, opacity=1e-4, albedo=0.3, seed=7):
    """The workload with continuum arrays added (App. A): per height a
    continuum extinction opacity * k_line (10 % smooth seeded modulation),
    flat over the line's narrow frequency range, of which the share `albedo`
    is scattering (sigma_c) and the rest absorption (kappa_c), and the LTE
    thermal continuum emissivity kappa_c W_T.  Arrays [z][nu], km^-1."""
    rng = np.random.default_rng(seed)
    atm = dict(cfg["atm"])
    z = np.asarray(atm["z_km"], float)
    nnu = len(cfg["quad"]["grid"])
    ext = opacity * np.asarray(atm["k_line"], float) * _smooth(rng, z, 0.1)
    kap = (1.0 - albedo) * ext
    atm["kappa_c"] = np.repeat(kap[:, None], nnu, axis=1)
    atm["sigma_c"] = np.repeat((albedo * ext)[:, None], nnu, axis=1)
    atm["eps_c_th"] = np.repeat((kap * np.asarray(atm["W_T"], float))[:, None], nnu, axis=1)
    return dict(cfg, atm=atm)


def mgii_batch(n_inst=256, base_seed=400, n_mu_half=4, n_chi=8, nz_range=(50, 130),
               nnu_range=(120, 220)):
    """Ragged batch of Mg II-like instances (config-2 physics)."""
    out = []
    for i in range(n_inst):
        rng = np.random.default_rng(base_seed + i)
        n_z = int(rng.integers(nz_range[0], nz_range[1] + 1))
        n_nu = int(rng.integers(nnu_range[0], nnu_range[1] + 1))
        n_wing = max(6, int(round(0.3 * n_nu)))
        n_core = (n_nu - n_wing) // 2
        n_wing = n_nu - 2 * n_core
        out.append(mgii(n_z=n_z, n_core_each=n_core, n_wing=n_wing, n_mu_half=n_mu_half,
                        n_chi=n_chi, seed=base_seed + i))
    return out


def mgii_adjoint(seed=5, perturb=0.2, **kw):
    """Mg II atmosphere plus a seeded +-20 % perturbation of (B, thetaB, chiB)."""
    cfg = mgii(seed=2, **kw)
    rng = np.random.default_rng(seed)
    atm = cfg["atm"]
    tgt = {k: np.array(v, copy=True) for k, v in atm.items()}
    n = len(atm["z_km"])
    tgt["B_G"] = atm["B_G"] * (1.0 + perturb * rng.uniform(-1, 1, n))
    tgt["thetaB"] = np.clip(atm["thetaB"] * (1.0 + perturb * rng.uniform(-1, 1, n)), 0, np.pi)
    tgt["chiB"] = atm["chiB"] * (1.0 + perturb * rng.uniform(-1, 1, n))
    cfg["target_atm"] = tgt
    cfg["name"] = "mgii_adjoint"
    return cfg


def seeded_vector(shape, seed, lo=0.0, hi=1.0, dtype=np.float64):
    """Seeded uniform test vector (used for operator parity inputs)."""
    return np.random.default_rng(seed).uniform(lo, hi, shape).astype(dtype)
