"""Faddeeva function w(z) = exp(-z^2) erfc(-i z) for Im z >= 0, in FP64.

Test infrastructure: only tests/, the smoke check and bench.py's CPU-baseline
leg may import anything under oracle/.

The paper writes the Voigt-Faraday pair as W(a, v) := w(v + i a) (Sect. 2.4,
F after Eq. G; Eq. RIIIQKKp).  It does not say how W is evaluated, so this
module follows a named published method: J.A.C. Weideman, "Computation of the
complex error function", SIAM J. Numer. Anal. 31 (1994) 1497, written here from
its derivation rather than from its listing:

  psi(t) = exp(-t^2) (L^2 + t^2) is expanded in powers of Z(t) = (L+it)/(L-it),
  psi = sum_n a_n Z^n (a_n real, a_-n = a_n);
  inserting this in w(z) = (i/pi) int exp(-t^2)/(z-t) dt and closing the
  contour in the upper half plane leaves only the terms n >= 0:
      w(z) = 2 sum_{n>=1} a_n Z(z)^(n-1) / (L - i z)^2 + 1/(sqrt(pi) (L - i z)),
  with a_n the Fourier coefficients of psi(L tan(theta/2)) over theta in
  (-pi, pi], computed here by the (spectrally accurate) trapezoidal rule.

Parity is pinned in tests against closed forms (w(iy) = exp(y^2) erfc(y),
Re w(x) = exp(-x^2) on the real axis, the large-|z| asymptote i/(sqrt(pi) z))
and against scipy.special.wofz, used only as a check.
"""
import numpy as np

_N = 40                       # terms kept in the expansion
_L = 2.0 ** (-0.25) * np.sqrt(_N)   # Weideman's recommended scale


def _coefficients(n_terms=_N, L=_L, m_points=None):
    """a_1..a_N of psi(L tan(theta/2)) = sum a_n e^{i n theta}."""
    if m_points is None:
        m_points = 8 * n_terms
    k = np.arange(-m_points + 1, m_points + 1)
    theta = np.pi * k / m_points
    with np.errstate(over="ignore", invalid="ignore"):
        t = L * np.tan(theta / 2.0)
        psi = np.exp(-t * t) * (L * L + t * t)
    psi[k == m_points] = 0.0          # theta = pi  <=>  t = infinity
    n = np.arange(1, n_terms + 1)
    a = (np.cos(np.outer(n, theta)) @ psi) / (2.0 * m_points)
    return a


_A = _coefficients()


def wofz(z):
    """w(z) for Im z >= 0 (vectorised, complex128)."""
    z = np.asarray(z, dtype=np.complex128)
    d = _L - 1j * z
    Z = (_L + 1j * z) / d
    p = np.zeros_like(z)
    for a in _A[::-1]:            # Horner in Z: sum_{n>=1} a_n Z^(n-1)
        p = p * Z + a
    return 2.0 * p / (d * d) + 1.0 / (np.sqrt(np.pi) * d)


def voigt_faraday(a, v):
    """W(a, v) = w(v + i a): real part H(a,v) (Voigt), imaginary part L(a,v)."""
    return wofz(np.asarray(v, dtype=np.float64) + 1j * np.asarray(a, dtype=np.float64))
