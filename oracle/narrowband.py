"""Wavelength-integrated narrow-band Stokes signals of Sect. 6.5 (oracle;
test infrastructure: nothing in the library imports or calls this module).

The paper weights the emergent profiles X(z_max, mu, lambda) (X = I, Q, U) by
a Gaussian of standard deviation sigma (full width at half maximum
2 sqrt(2 ln 2) sigma) centred on lambda_0 and integrates over
[lambda_0 - Delta, lambda_0 + Delta]:
    Xbar(mu) = 1 / (sqrt(2 pi) sigma) int exp(-(lambda - lambda_0)^2 / (2 sigma^2)) X(lambda) dlambda.
It leaves open how X is continued between and beyond the wavelength nodes.
Reading: X is the natural cubic spline through its node values in lambda,
continued by its end values outside the grid (the same continuation the frame
changes of Sect. 4.1 use).  The integral is taken by adaptive Gauss-Kronrod
quadrature of the spline basis (scipy, every node at once); pinned in tests by
closed forms (a constant, an odd profile, a Gaussian profile).
"""
import numpy as np
from scipy.integrate import quad_vec

from . import constants as C
from .spline import NaturalSpline


def sigma_of_fwhm(fwhm):
    return fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))


def weights(lam, lam0, fwhm, half_width):
    """w[n] with Xbar = sum_n w[n] X[n] for profiles X on the ascending
    wavelength nodes lam (Angstrom)."""
    lam = np.asarray(lam, dtype=np.float64)
    spl = NaturalSpline(lam)
    s = sigma_of_fwhm(fwhm)
    a, b = lam0 - half_width, lam0 + half_width
    pts = [p for p in lam if a < p < b]
    norm = 1.0 / (np.sqrt(2.0 * np.pi) * s)
    f = lambda l: norm * np.exp(-0.5 * ((l - lam0) / s) ** 2) * spl.basis(np.array([l]))[0]
    w, _ = quad_vec(f, a, b, points=pts, limit=4 * lam.size + 200, epsabs=1e-15, epsrel=1e-13)
    return w


def narrowband(lam, X, lam0, fwhm, half_width):
    """Xbar for profiles X[..., n, s] on the wavelength nodes lam (axis -2)."""
    w = weights(lam, lam0, fwhm, half_width)
    return np.einsum("n,...ns->...s", w, np.asarray(X, dtype=np.float64))


def grid_wavelengths(P):
    """Vacuum wavelengths (Angstrom) of the frequency nodes of an oracle
    Problem, ascending in wavelength (the grid is ascending in wavelength or
    in reduced frequency, both descending in frequency)."""
    lam = C.C_LIGHT / P.nu * 1e10
    assert np.all(np.diff(lam) > 0)
    return lam
