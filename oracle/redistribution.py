"""R_II-AD kernel F, its Theta = 0 and Theta = pi limits, and the integrals of
F and of the R_III profiles against the natural-spline basis (oracle).

Sect. 2.4 (after Eq. G):
    F(Theta, u', u) = 1/sin(Theta) exp[-((u-u')/(2 sin(Theta/2)))^2]
                      W(a/cos(Theta/2), (u+u')/(2 cos(Theta/2)))
Sect. 4.3 / App. C rule i:  F(0, u, u') = sqrt(pi) delta(u-u') W(a, u').
Theta = pi (the back-scattering pairs every even-N_chi grid contains, which
the paper's odd N_chi avoids): w(Z) ~ i/(sqrt(pi) Z) as |Z| -> infinity gives
    F(pi, u', u) = exp[-(u-u')^2/4] (a + i v) / (2 sqrt(pi) (v^2 + a^2)),
    v = (u+u')/2.

Discrete operator (reading "Def-B"): the incident field enters only through
its natural spline S[I~] on the comoving grid, continued by its end values,
and the frequency integral of R_II is exact over the whole real line:
    T[n, m] = int F(Theta, u'+s, u_n+s') phi_m(u') du'
with phi_m the cardinal spline basis.  The R_III incident integral (Eq.
RIIIQKKp) is taken over the grid span [u_1, u_N] (the paper integrates R_III
over a finite interval, Sect. 4.3).

Quadrature: composite 16-point Gauss-Legendre on panels that never straddle a
grid node, graded towards the centre of the W factor (v = 0) and no wider than
a quarter of the Gaussian width 2 sin(Theta/2); the Gaussian factor is cut
where it is below exp(-6.5^2).  Pinned in tests against adaptive
Gauss-Kronrod (scipy.integrate.quad_vec) to 1e-10 relative, on the Fig. 1
parameters among others.
"""
import numpy as np
from .faddeeva import voigt_faraday

SQRT_PI = np.sqrt(np.pi)
_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)
GAUSS_CUT = 6.5


def F_kernel(theta, xp, x, a):
    """F(Theta, x', x) for 0 < Theta <= pi (Theta = pi uses the exact limit)."""
    xp = np.asarray(xp, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if theta >= np.pi:
        v = 0.5 * (x + xp)
        return np.exp(-0.25 * (x - xp) ** 2) * (a + 1j * v) / (2.0 * SQRT_PI * (v * v + a * a))
    s2 = np.sin(0.5 * theta)
    c2 = np.cos(0.5 * theta)
    g = np.exp(-((x - xp) / (2.0 * s2)) ** 2) / np.sin(theta)
    return g * voigt_faraday(a / c2, (x + xp) / (2.0 * c2))


def _panels(L, R, breaks, uV, hV, hG):
    """Panel edges on [L, R]: split at every break, graded towards uV."""
    pts = sorted(set([L, R] + [b for b in breaks if L < b < R]))
    edges = [L]
    for a0, b0 in zip(pts[:-1], pts[1:]):
        x = a0
        while x < b0 - 1e-14 * max(1.0, abs(b0)):
            d = abs(x - uV) if uV is not None else np.inf
            # width limited by Gaussian scale and by distance to the W centre;
            # when approaching uV from the left, stop exactly at the midpoint
            w = min(hG, max(0.25 * hV, 0.5 * d))
            if uV is not None and x < uV < b0:
                w = min(w, max(0.5 * (uV - x), 0.25 * hV) if uV - x > 0.25 * hV else uV - x)
            x = min(x + w, b0)
            edges.append(x)
    return np.array(edges)


def _nodes(edges):
    a0, b0 = edges[:-1], edges[1:]
    half = 0.5 * (b0 - a0)
    mid = 0.5 * (b0 + a0)
    x = (mid[:, None] + half[:, None] * _GL_X[None, :]).ravel()
    w = (half[:, None] * _GL_W[None, :]).ravel()
    return x, w


def tile_row(spl, theta, a, s_in, s_out, u_n):
    """Row T[n, :] = int F(Theta, u'+s_in, u_n+s_out) phi(u') du' (complex, len N)."""
    x = u_n + s_out                     # outgoing detuning
    if theta == 0.0:
        return SQRT_PI * voigt_faraday(a, x) * spl.basis(np.array([x - s_in]))[0]
    s2 = np.sin(0.5 * theta)
    c2 = np.cos(0.5 * theta)
    g = 2.0 * s2                        # Gaussian width in (x - x')
    uG = x - s_in                       # Gaussian centre in u'
    L, R = uG - GAUSS_CUT * g, uG + GAUSS_CUT * g
    uV = -x - s_in                      # v = 0  <=>  x' = -x
    hV = 2.0 * max(c2 if theta < np.pi else 0.0, a)
    edges = _panels(L, R, list(spl.u) + ([uV] if L < uV < R else []),
                    uV if (L - 10 * hV) < uV < (R + 10 * hV) else None, hV, 0.25 * g)
    up, w = _nodes(edges)
    f = F_kernel(theta, up + s_in, x, a) * w
    return f @ spl.basis(up)


def tile(spl, theta, a, s_in, s_out):
    return np.array([tile_row(spl, theta, a, s_in, s_out, un) for un in spl.u])


def r3_in_weights(spl, a, s1, s2):
    """r[m] = int_{u_1}^{u_N} [W(a, u'+s1) + conj W(a, u'+s2)] phi_m(u') du'."""
    u = spl.u
    edges = [u[0]]
    centers = np.array([-s1, -s2])
    for a0, b0 in zip(u[:-1], u[1:]):
        x = a0
        while x < b0 - 1e-14 * max(1.0, abs(b0)):
            d = np.min(np.abs(centers - x))
            w = max(0.25, 0.25 * d)
            # do not jump over a profile centre with a wide panel
            ahead = centers[(centers > x) & (centers < x + w)]
            if ahead.size:
                w = max(ahead.min() - x, 0.05) if ahead.min() - x > 1e-12 else 0.25
            x = min(x + w, b0)
            edges.append(x)
    up, wq = _nodes(np.array(edges))
    p = voigt_faraday(a, up + s1) + np.conj(voigt_faraday(a, up + s2))
    return (p * wq) @ spl.basis(up)


def aa_tile(spl, a, s_in, s_out, n_theta=48):
    """Angle-averaged tile 1/2 int_0^pi sin(Theta) T(Theta) dTheta (Eq. R_AA).

    Composite Gauss-Legendre in Theta on [0, pi/2] and [pi/2, pi] with
    n_theta nodes each (the integrand is smooth in Theta once integrated
    against the spline basis); convergence is checked in tests by doubling.
    """
    x, w = np.polynomial.legendre.leggauss(n_theta)
    acc = 0.0
    for lo, hi in ((0.0, 0.5 * np.pi), (0.5 * np.pi, np.pi)):
        th = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        wt = 0.5 * (hi - lo) * w
        for t_, w_ in zip(th, wt):
            acc = acc + 0.5 * w_ * np.sin(t_) * tile(spl, t_, a, s_in, s_out)
    return acc
