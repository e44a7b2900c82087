"""Angular grid, scattering angles and polarisation reference frames (oracle).

Sect. 4.2: tensor product of a trapezoidal rule in chi over [0, 2 pi) and one
Gauss-Legendre rule on each hemisphere of mu (on [-1,0] and on [0,1]).
Weights are normalised to the solid-angle average  oint dOmega / (4 pi).
Directions are ordered Omega = i_mu * N_chi + i_chi with mu ascending
(downward rays first) and chi_k = 2 pi k / N_chi.

Stokes reference (Sect. 6.3, Fig. 3 caption): positive Q is parallel to the
limb, i.e. along e_a = (-sin chi, cos chi, 0); e_b = (cos th cos chi,
cos th sin chi, -sin th) completes the transverse pair.
"""
import numpy as np


def angular_grid(n_mu_half, n_chi, mu_rule=0):
    """mu_rule 0: one GL rule of n_mu_half nodes on each hemisphere (Sect. 4.2);
    mu_rule 1: a single GL rule of 2 n_mu_half nodes on [-1, 1] (used when one
    node per hemisphere is asked for: the per-hemisphere 1-node rule puts
    mu = 1/2 and integrates P_2(mu) to -1/8 instead of 0, which feeds a
    spurious I <-> Q coupling; the full-range rule puts mu = 1/sqrt(3))."""
    if mu_rule == 1:
        x, w = np.polynomial.legendre.leggauss(2 * n_mu_half)
        mu, wmu = x, w                   # weights sum to 2 on [-1, 1]
    else:
        x, w = np.polynomial.legendre.leggauss(n_mu_half)
        mu_pos = 0.5 * (x + 1.0)
        w_pos = 0.5 * w                  # GL weights on [0, 1]
        mu = np.concatenate([-mu_pos[::-1], mu_pos])
        wmu = np.concatenate([w_pos[::-1], w_pos])
    chi = 2.0 * np.pi * np.arange(n_chi) / n_chi
    MU, CHI = np.meshgrid(mu, chi, indexing="ij")
    W = np.outer(0.5 * wmu, np.full(n_chi, 1.0 / n_chi))
    return MU.ravel(), CHI.ravel(), W.ravel()


def unit_vector(mu, chi):
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([s * np.cos(chi), s * np.sin(chi), mu * np.ones_like(chi)], axis=-1)


def pol_basis(mu, chi):
    """(e_a, e_b): e_a horizontal (Q reference, parallel to the limb)."""
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    ea = np.array([-np.sin(chi), np.cos(chi), 0.0])
    eb = np.array([mu * np.cos(chi), mu * np.sin(chi), -s])
    return ea, eb


def scattering_angle(n1, n2):
    """Theta = angle between unit vectors, robust at 0 and pi."""
    return 2.0 * np.arctan2(np.linalg.norm(n1 - n2, axis=-1), np.linalg.norm(n1 + n2, axis=-1))


def theta_classes(mu, chi, tol=1e-10):
    """Distinct scattering angles over all (Omega, Omega') pairs.

    Returns (thetas, cls) with cls[o, o'] the class index.  Values within `tol`
    rad are merged; classes within `tol` of 0 or pi are set to exactly 0 or pi.
    """
    n = unit_vector(mu, chi)
    th = scattering_angle(n[:, None, :], n[None, :, :])
    flat = np.sort(th.ravel())
    reps = [flat[0]]
    for v in flat[1:]:
        if v - reps[-1] > tol:
            reps.append(v)
    reps = np.array(reps)
    reps[np.abs(reps) < tol] = 0.0
    reps[np.abs(reps - np.pi) < tol] = np.pi
    cls = np.abs(th[..., None] - reps[None, None, :]).argmin(-1)
    assert np.all(np.abs(th - reps[cls]) <= tol * 1.0001 + 1e-15)
    return reps, cls
