"""Physics-based preconditioner of Sect. 5.2, P = Id - Lambda* Sigma*, applied
as m_in Richardson sweeps with the block-diagonal inner preconditioner P_hat
of App. F (oracle; test infrastructure).

The paper leaves the simplified operators to the implementer (Sect. 5.2); the
reading written out here is:

* Sigma* is unpolarised and unmagnetised, with angle-averaged R_II (Eq. R_AA),
  and acts on Stokes I only (App. F keeps K = Q = 0).  In the comoving frame
      eps_bar*(z, u_n) = sum_m Phi_bar[n, m] J_bar(z, u_m),
      J_bar(z, u_m)    = sum_Omega w_Omega I~(z, Omega, u_m)           (Phi^Omega),
      Phi_bar[n, m]    = k [alpha0 sum_g c_g (1/pi) int Re F_AA(u'+s_g, u_n+s_g) phi_m(u') du'
                            + (beta0 - alpha0) phi*(u_n) int phi*(u') phi_m(u') du'],
  where g runs over the J levels of the upper term at B = 0 (shift s_g, weight
  c_g = (2J+1)/(2(2L+1)); one level of weight 1 for the two-level atom),
  phi*(u) = sum_g c_g H(a, u + s_g)/sqrt(pi), phi_m the spline basis, and the
  incident integral of the R_III-like term runs over the grid span.  The frame
  changes of Sect. 4.1 sit on either side (I -> I~, eps_bar* -> eps*).
* Lambda* is the DELO-linear formal solution (Sect. 3) of the scalar problem
  (K = eta_I Id).
* P x = x - Lambda* Sigma* x on Stokes I, the identity on Q, U, V.
* P^-1 y: x <- x + P_hat^-1 (y - P x) from x = 0 (Q, U, V = y), m_in times,
      P_hat^-1 = Id + Lambda_ii Phi_bar (Id - A)^-1 Phi^Omega,   A = Phi^Omega Lambda_ii Phi_bar,
  App. F's local block inverse with its frame changes dropped (they only shape
  the approximation P_hat); Lambda_ii = beta / eta_I is the DELO weight of the
  source function at the point itself.

Pinned in tests: P_hat^-1 against the dense inverse of Id - Lambda_ii Sigma_hat
per height (brute force), and the sweeps converging to the exact inverse of P.
"""
import numpy as np

from . import constants as C
from . import redistribution as RD
from .faddeeva import voigt_faraday
from .problem import delo_coeffs


def _levels(atom, nu0):
    """(energy of each J level relative to nu0 [Hz], weight c_g) at B = 0."""
    E = atom["E_u_cm"]
    if atom["twoS"] == 0:
        return [E[0] * C.CM_TO_HZ - nu0], [1.0]
    return [E[0] * C.CM_TO_HZ - nu0, E[1] * C.CM_TO_HZ - nu0], [2.0 / 6.0, 4.0 / 6.0]


class Preconditioner:
    def __init__(self, P):
        self.P = P
        nz, nO, N = P.nz, P.nO, P.nN
        E, cg = _levels(P.atom, P.nu0)
        _, _, beta = delo_coeffs(P.dtau)
        self.lii = beta / P.eta1                                   # [z][Omega][n]
        self.Phi = np.zeros((nz, N, N))
        self.M = np.zeros((nz, N, N))
        for iz in range(nz):
            spl, a, u = P.spl[iz], P.a[iz], P.u[iz]
            a0 = (1.0 - P.eps[iz]) * (1.0 - P.rE[iz])
            b0 = 1.0 - P.eps[iz]
            aa = np.zeros((N, N))
            phis = np.zeros(N)
            rs = np.zeros(N)
            for Eg, c in zip(E, cg):
                s = Eg / P.dnuD[iz]
                aa += c * RD.aa_tile(spl, a, s, s).real / np.pi
                phis += c * voigt_faraday(a, u + s).real / np.sqrt(np.pi)
                rs += c * RD.r3_in_weights(spl, a, s, s).real / (2.0 * np.sqrt(np.pi))
            Phi = P.k[iz] * (a0 * aa + (b0 - a0) * np.outer(phis, rs))
            lbar = P.wang @ self.lii[iz]                           # Phi^Omega Lambda_ii
            A = lbar[:, None] * Phi
            self.Phi[iz] = Phi
            self.M[iz] = Phi @ np.linalg.inv(np.eye(N) - A)

    def sigma_star(self, xI):
        """eps* (observer frame) of the Stokes-I field xI[z][Omega][n]."""
        P = self.P
        out = np.zeros_like(xI)
        for iz in range(P.nz):
            It = np.stack([P.interp_in(iz, o) @ xI[iz, o] for o in range(P.nO)])
            eb = self.Phi[iz] @ (P.wang @ It)
            for o in range(P.nO):
                out[iz, o] = P.interp_back(iz, o) @ eb
        return out

    def lambda_star(self, eps):
        """Scalar DELO-linear formal solution of eps[z][Omega][n], zero boundary."""
        P = self.P
        K = np.zeros_like(P.K)
        for s in range(4):
            K[..., s, s] = P.eta1
        e4 = np.zeros(eps.shape + (4,))
        e4[..., 0] = eps
        return P.formal_solution(e4, K=K)[..., 0]

    def apply_P(self, x):
        y = x.copy()
        y[..., 0] = x[..., 0] - self.lambda_star(self.sigma_star(x[..., 0]))
        return y

    def apply_Phat_inv(self, r):
        """P_hat^-1 on a Stokes-I field r[z][Omega][n]."""
        v = np.einsum("znm,zm->zn", self.M, np.einsum("o,zon->zn", self.P.wang, r))
        return r + self.lii * v[:, None, :]

    def apply_inv(self, y, m_in):
        """The preconditioner applied to y (m_in Richardson sweeps from zero)."""
        x = y.copy()
        if m_in <= 0:
            return x
        x[..., 0] = 0.0
        for sweep in range(m_in):
            if sweep == 0:
                r = y[..., 0].copy()
            else:
                r = y[..., 0] - self.apply_P(x)[..., 0]
            x[..., 0] += self.apply_Phat_inv(r)
        return x
