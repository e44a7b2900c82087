"""Discrete linear problem (Id - Lambda Sigma) I = Lambda eps_th + t (Eq.
linear_system), assembled plainly in FP64 (oracle).

Vectors are arrays I[z, Omega, n, s] (s = I, Q, U, V), heights ascending,
directions as in geometry.angular_grid, reduced frequencies per height.

Redistribution matrix ("Jones" or amplitude route; the paper cites
Alsina Ballester 2022 / Bommier 1997b for the phase matrix and A_Q^KK' (App.
B) without printing them).  Scattering amplitudes of the two-term atom with an
unpolarised lower term, reference basis (e_a, e_b) of each direction:
    M_{alpha gamma}(k_u; k_l, k_l') = <k_l'| e_alpha* . d |k_u> <k_u| e'_gamma . d |k_l>
    R^II_ij = 3/(8 pi (2S+1)) sum_{k_u k_u' k_l k_l'}
              Tr(sigma_i M(k_u) sigma_j M(k_u')^+) alpha_{k_u k_u'}
              [G(k_u', k_l, k_l') + G(k_u, k_l, k_l')^*]          (Eq. RQIIKKp)
    R^III_ij = 3/(16 pi (2S+1)) sum Tr(...) (beta - alpha)_{k_u k_u'}
              [W(u'+s_{k_u' k_l}) + W(u'+s_{k_u k_l})^*]
              [W(u +s_{k_u' k_l'}) + W(u +s_{k_u k_l'})^*]        (Eq. RIIIQKKp)
with alpha, beta the branching ratios of App. B, G = F evaluated at the
shifted reduced frequencies (Eq. G), Stokes I = Tr(rho), Q = Tr(sigma_z rho),
U = Tr(sigma_x rho), V = S_V Tr(sigma_y rho) and rho the coherency matrix of
(E_a, E_b).  The factor 3/2 makes oint R_11 = (1 - eps) phi at B = 0 (App. E).
The conjugate pairing of R^II is pinned by the Kramers-Heisenberg limit of a
single atom (tests); both brackets of R^III are pinned against R^II: under
incident light flat in frequency the two emit the same spectrum, and
integrated over the outgoing frequency they absorb alike (tests).  At B = 0
and v = 0 the point-valued R is symmetric, R(nu, Omega; nu', Omega') =
R(nu', Omega'; nu, Omega)^T (tests).  The polarised DELO-linear step converges
at second order to the matrix-exponential solution of a homogeneous slab
(tests).

Test infrastructure only: nothing in the library imports or calls this module.

Propagation matrix from the forward-scattering amplitude (LL04 Ch. 7, cited in
Sect. 2.2): kappa = k/(2 sqrt(pi)(2S+1)) sum_{k_u k_l} (a_l^*)(a_l)^T W(x)^*,
K_ij = 1/2 Tr(sigma_i kappa sigma_j + sigma_i sigma_j kappa^+); then
eps_th = eps W_T (K_11, K_21, K_31, K_41) (Sect. 2.3).

Continuum (App. A, optional atmosphere arrays kappa_c, sigma_c, eps_c_th of
shape [z, nu], km^-1 like k_line): eta_c = kappa_c + sigma_c is added to the
diagonal of K; the thermal continuum emissivity to Stokes I of eps_th; and
coherent scattering in the observer frame,
    eps_c(Omega, nu) = sigma_c(nu) oint P(Omega, Omega') I(Omega', nu) dOmega'/4pi,
with P the dipole (Rayleigh) phase matrix P_ij = 3/4 Tr(sigma_i J sigma_j J^T),
J_ab = e_a(Omega) . e_b(Omega') (the sum over K <= 2 of (-1)^Q T^K_Q T^K_-Q of
App. A with every W_K = 1).  The Kirchhoff factor f normalises the line part
only, with the line's eta_I.
"""
import numpy as np
from . import constants as C
from .faddeeva import voigt_faraday
from .spline import NaturalSpline
from .geometry import angular_grid, unit_vector, pol_basis, theta_classes, scattering_angle
from .atom import nu0_of, states
from . import redistribution as RD

GRID_LAMBDA, GRID_X = 0, 1
S_V = 1.0   # sign convention of Stokes V (fixed by the weak-field pin)

SIG = np.array([[[1, 0], [0, 1]],
                [[1, 0], [0, -1]],
                [[0, 1], [1, 0]],
                [[0, -1j * S_V], [1j * S_V, 0]]], dtype=np.complex128)
# spherical unit vectors e_q (q = -1, 0, +1) in the magnetic frame
EQ = np.array([[1, -1j, 0], [0, 0, np.sqrt(2)], [-1, -1j, 0]], dtype=np.complex128) / np.sqrt(2)


def magnetic_frame(thB, chB):
    """Rows (x_B, y_B, z_B): components of a vector in the magnetic frame."""
    b = np.array([np.sin(thB) * np.cos(chB), np.sin(thB) * np.sin(chB), np.cos(thB)])
    xB = np.array([np.cos(thB) * np.cos(chB), np.cos(thB) * np.sin(chB), -np.sin(thB)])
    yB = np.array([-np.sin(chB), np.cos(chB), 0.0])
    return np.stack([xB, yB, b])


def delo_coeffs(d):
    """DELO-linear weights (exp(-d), alpha, beta), series below d = 1e-3."""
    d = np.asarray(d, dtype=np.float64)
    e = np.exp(-d)
    small = d < 1e-3
    w0 = -np.expm1(-d)
    with np.errstate(divide="ignore", invalid="ignore"):
        beta = np.where(small, 0.0, 1.0 - w0 / d)
        alpha = np.where(small, 0.0, w0 - beta)
    ds = d[small]
    beta[small] = ds / 2 - ds ** 2 / 6 + ds ** 3 / 24 - ds ** 4 / 120 + ds ** 5 / 720
    alpha[small] = ds / 2 - ds ** 2 / 3 + ds ** 3 / 8 - ds ** 4 / 30 + ds ** 5 / 144
    return e, alpha, beta


def delopar_coeffs(dM, dP):
    """Weights (psi_M, psi_O, psi_P) of the upwind, current and downwind source
    values for one step of DELOPAR: the source vector is the parabola through
    the three points and its contribution int_0^dM e^{-t} S(t) dt is taken
    exactly, t measured from the current point back towards the upwind one
    (upwind at t = dM, downwind at t = -dP).  From the moments
    I_n = int_0^dM t^n e^{-t} dt = n! P(n + 1, dM) (regularised incomplete
    gamma) and the Lagrange basis through t = dM, 0, -dP."""
    from scipy.special import gammainc
    dM = np.asarray(dM, dtype=np.float64)
    dP = np.asarray(dP, dtype=np.float64)
    I0 = gammainc(1.0, dM)
    I1 = gammainc(2.0, dM)
    I2 = 2.0 * gammainc(3.0, dM)
    psiM = (I2 + dP * I1) / (dM * (dM + dP))
    psiO = -(I2 + (dP - dM) * I1 - dM * dP * I0) / (dM * dP)
    psiP = (I2 - dM * I1) / (dP * (dM + dP))
    return psiM, psiO, psiP


class Problem:
    # formal solvers: DELO-linear (source vector and K'I linear over a step) and
    # DELOPAR (source vector parabolic through the upwind, current and downwind
    # points, K'I linear; linear at the last point of a ray)
    FORMAL_SOLVERS = ("delo_linear", "delopar")

    def __init__(self, cfg, mode=None, normalise=True, formal_solver="delo_linear"):
        self.cfg = cfg
        assert formal_solver in self.FORMAL_SOLVERS
        self.formal_solver = formal_solver
        atom, atm, quad = cfg["atom"], cfg["atm"], cfg["quad"]
        self.atom = atom
        self.mode = quad.get("mode", 0) if mode is None else mode
        self.z = np.asarray(atm["z_km"], dtype=np.float64)
        nz = self.nz = self.z.size
        self.mu, self.chi, self.wang = angular_grid(quad["n_mu_half"], quad["n_chi"], quad.get("mu_rule", 0))
        self.nO = self.mu.size
        self.nvec = unit_vector(self.mu, self.chi)
        self.thetas, self.cls = theta_classes(self.mu, self.chi)
        self.S2 = 2 if atom["twoS"] == 1 else 1          # 2S+1 of the lower term
        nu0 = self.nu0 = nu0_of(atom)
        T = np.asarray(atm["T_K"], float)
        xi = np.asarray(atm["xi_kms"], float) * 1e3
        vD = np.sqrt(2.0 * C.K_BOLTZ * T / (atom["mass_amu"] * C.AMU) + xi * xi)   # m/s
        self.vD_kms = vD / 1e3
        self.dnuD = nu0 * vD / C.C_LIGHT
        grid = np.asarray(quad["grid"], float)
        if quad["grid_kind"] == GRID_LAMBDA:
            nu = C.C_LIGHT / (grid * 1e-10)
        else:
            nu = nu0 - grid * self.dnuD[0]
        self.nu = nu
        self.nN = nu.size
        self.u = (nu0 - nu[None, :]) / self.dnuD[:, None]            # [z, n]
        self.spl = [NaturalSpline(self.u[k]) for k in range(nz)]
        self.a = np.asarray(atm["a"], float)
        self.eps = np.asarray(atm["eps"], float)
        self.rE = np.asarray(atm["r_el"], float)
        self.k = np.asarray(atm["k_line"], float)
        self.WT = np.asarray(atm["W_T"], float)
        zn = (nz, self.nN)
        self.kap_c = np.asarray(atm.get("kappa_c", np.zeros(zn)), float).reshape(zn)
        self.sig_c = np.asarray(atm.get("sigma_c", np.zeros(zn)), float).reshape(zn)
        self.epsc_th = np.asarray(atm.get("eps_c_th", np.zeros(zn)), float).reshape(zn)
        v = np.asarray(atm["v_kms"], float)
        self.ub = (v @ self.nvec.T) / self.vD_kms[:, None]           # [z, Omega]
        # atom per height
        self.shift, self.alpha, self.beta, self.amp, self.D, self.Rm = [], [], [], [], [], []
        Bv = np.asarray(atm["B_G"], float)
        thB = np.asarray(atm["thetaB"], float)
        chB = np.asarray(atm["chiB"], float)
        for iz in range(nz):
            Eu, D, El = states(atom, Bv[iz])
            self.shift.append((Eu[:, None] - El[None, :]) / self.dnuD[iz])    # s[ku, kl]
            Gtot = 4.0 * np.pi * self.dnuD[iz] * self.a[iz]
            a0 = (1.0 - self.eps[iz]) * (1.0 - self.rE[iz])
            b0 = 1.0 - self.eps[iz]
            dnu = Eu[:, None] - Eu[None, :]
            self.alpha.append(a0 / (1.0 + 2j * np.pi * dnu / Gtot))
            self.beta.append(b0 / (1.0 + 2j * np.pi * dnu / (Gtot * (1.0 - self.rE[iz]))))
            self.D.append(D)
            self.Rm.append(magnetic_frame(thB[iz], chB[iz]))
            self.amp.append(np.stack([self.amplitudes(iz, self.mu[o], self.chi[o])
                                      for o in range(self.nO)]))
        self.nu_states = self.amp[0].shape[2]
        self.nl_states = self.amp[0].shape[3]
        self._tiles = {}
        self._r3 = {}
        self._build_K()
        self._build_delo()
        self.f = np.ones((nz, self.nO, self.nN))
        if normalise:
            self.f = self._normalisation()

    def amplitudes(self, iz, mu, chi):
        """a[alpha, ku, kl] = <k_u| e_alpha . d |k_l> for direction (mu, chi)."""
        out = []
        for e in pol_basis(mu, chi):
            proj = EQ.conj() @ (self.Rm[iz] @ e)       # e . e_q^*  for q = -1, 0, +1
            out.append(np.einsum("q,qul->ul", proj, self.D[iz]))
        return np.stack(out)

    # ------------------------------------------------------------------ K, eps_th
    def kappa(self, iz, o_amp, ub, un):
        """kappa[n, 2, 2] for one direction (amplitudes o_amp[2, ku, kl], shift ub)."""
        s = self.shift[iz]
        W = voigt_faraday(self.a[iz], un[:, None, None] + ub + s[None])       # [n, ku, kl]
        kap = np.einsum("aul,bul,nul->nab", o_amp.conj(), o_amp, W.conj())
        return kap * self.k[iz] / (2.0 * np.sqrt(np.pi) * self.S2)

    @staticmethod
    def K_from_kappa(kap):
        K1 = np.einsum("iab,nbc,jcd->nijad", SIG, kap, SIG)
        K1 = np.einsum("nijaa->nij", K1)
        kd = np.conj(np.swapaxes(kap, -1, -2))
        K2 = np.einsum("iab,jbc,ncd->nijad", SIG, SIG, kd)
        K2 = np.einsum("nijaa->nij", K2)
        K = 0.5 * (K1 + K2)
        assert np.max(np.abs(K.imag)) <= 1e-12 * max(1.0, np.max(np.abs(K.real)))
        return K.real

    def _build_K(self):
        nz, nO, nN = self.nz, self.nO, self.nN
        self.K = np.zeros((nz, nO, nN, 4, 4))
        for iz in range(nz):
            for o in range(nO):
                self.K[iz, o] = self.K_from_kappa(self.kappa(iz, self.amp[iz][o], self.ub[iz, o],
                                                             self.u[iz]))
        self.eta1_line = self.K[..., 0, 0].copy()
        self.eps_th = (self.eps * self.WT)[:, None, None, None] * self.K[..., :, 0]
        for s_ in range(4):
            self.K[..., s_, s_] += (self.kap_c + self.sig_c)[:, None, :]
        self.eta1 = self.K[..., 0, 0]
        self.eps_th[..., 0] += self.epsc_th[:, None, :]

    # ------------------------------------------------------------------ Lambda
    def _build_delo(self):
        z = self.z
        nz = self.nz
        self.dtau = np.zeros((nz, self.nO, self.nN))   # step arriving at each point
        for o in range(self.nO):
            mu = self.mu[o]
            order = np.arange(nz) if mu > 0 else np.arange(nz)[::-1]
            for p in range(1, nz):
                k1, k0 = order[p], order[p - 1]
                self.dtau[k1, o] = 0.5 * (self.eta1[k0, o] + self.eta1[k1, o]) * abs(z[k1] - z[k0]) / abs(mu)

    def formal_solution(self, eps, boundary=False, K=None, eta1=None, dtau=None, mu=None):
        """I = Lambda eps (+ t if boundary) along every ray (Sect. 3), with the
        problem's formal solver: DELO-linear,
            (Id + b K'_k) I_k = (e Id - a K'_{k-1}) I_{k-1} + a S_{k-1} + b S_k,
        or DELOPAR, whose source terms are psi_M S_{k-1} + psi_O S_k + psi_P S_{k+1}
        (delopar_coeffs; DELO-linear's a, b at the last point of the ray)."""
        K = self.K if K is None else K
        eta1 = self.eta1 if eta1 is None else eta1
        dtau = self.dtau if dtau is None else dtau
        mus = self.mu if mu is None else mu
        nz = self.nz
        nO, nN = eps.shape[1], eps.shape[2]
        out = np.zeros_like(eps)
        Id = np.eye(4)
        for o in range(nO):
            up = mus[o] > 0
            order = np.arange(nz) if up else np.arange(nz)[::-1]
            I = np.zeros((nN, 4))
            if boundary and up:
                I[:, 0] = self.WT[0]
            k0 = order[0]
            out[k0, o] = I
            for p in range(1, nz):
                k1 = order[p]
                e, al, be = delo_coeffs(dtau[k1, o])
                Kp0 = K[k0, o] / eta1[k0, o][:, None, None] - Id
                Kp1 = K[k1, o] / eta1[k1, o][:, None, None] - Id
                S0 = eps[k0, o] / eta1[k0, o][:, None]
                S1 = eps[k1, o] / eta1[k1, o][:, None]
                lhs = Id[None] + be[:, None, None] * Kp1
                rhs = np.einsum("nij,nj->ni", e[:, None, None] * Id[None] - al[:, None, None] * Kp0, I)
                if self.formal_solver == "delopar" and p + 1 < nz:
                    k2 = order[p + 1]
                    pM, pO, pP = delopar_coeffs(dtau[k1, o], dtau[k2, o])
                    S2 = eps[k2, o] / eta1[k2, o][:, None]
                    rhs = rhs + pM[:, None] * S0 + pO[:, None] * S1 + pP[:, None] * S2
                else:
                    rhs = rhs + al[:, None] * S0 + be[:, None] * S1
                I = np.linalg.solve(lhs, rhs[..., None])[..., 0]
                out[k1, o] = I
                k0 = k1
        return out

    # ------------------------------------------------------------------ Sigma
    def tile(self, iz, theta, s_in, s_out):
        key = (iz, round(theta, 13), round(s_in, 13), round(s_out, 13), self.mode)
        if key not in self._tiles:
            if self.mode == 1:
                self._tiles[key] = RD.aa_tile(self.spl[iz], self.a[iz], s_in, s_out)
            else:
                self._tiles[key] = RD.tile(self.spl[iz], theta, self.a[iz], s_in, s_out)
        return self._tiles[key]

    def r3(self, iz, s1, s2):
        key = (iz, round(s1, 13), round(s2, 13))
        if key not in self._r3:
            self._r3[key] = RD.r3_in_weights(self.spl[iz], self.a[iz], s1, s2)
        return self._r3[key]

    def _tr(self, ampO, ampI, ku, kv, kl, klp):
        """Tr(sigma_i M(ku) sigma_j M(kv)^+) for all i, j  (4x4 complex)."""
        Mu = np.outer(ampO[:, ku, klp].conj(), ampI[:, ku, kl])
        Mv = np.outer(ampO[:, kv, klp].conj(), ampI[:, kv, kl])
        return np.einsum("iab,bc,jcd,ad->ij", SIG, Mu, SIG, Mv.conj())

    def block(self, iz, o, op, amp_o=None, theta=None, ub_o=None):
        """Comoving-frame block (N x 4) x (N x 4) coupling I~(Omega') -> eps_bar(Omega)."""
        amp = self.amp[iz]
        ampO = amp[o] if amp_o is None else amp_o
        ampI = amp[op]
        th = self.thetas[self.cls[o, op]] if theta is None else theta
        if self.mode == 1:
            th = -1.0
        s = self.shift[iz]
        nu_, nl = self.nu_states, self.nl_states
        N = self.nN
        un = self.u[iz]
        blk = np.zeros((N, 4, N, 4), dtype=np.complex128)
        c2 = 3.0 / (8.0 * np.pi * self.S2)
        c3 = 3.0 / (16.0 * np.pi * self.S2)
        al, be = self.alpha[iz], self.beta[iz]
        for kl in range(nl):
            for klp in range(nl):
                for ku in range(nu_):
                    if not np.any(ampI[:, ku, kl]) or not np.any(ampO[:, ku, klp]):
                        continue
                    for kv in range(nu_):
                        if not np.any(ampI[:, kv, kl]) or not np.any(ampO[:, kv, klp]):
                            continue
                        tr = self._tr(ampO, ampI, ku, kv, kl, klp)
                        if np.max(np.abs(tr)) == 0.0:
                            continue
                        Gv = self.tile(iz, th, s[kv, kl], s[kv, klp])
                        Gu = self.tile(iz, th, s[ku, kl], s[ku, klp])
                        prof2 = al[ku, kv] * (Gv + Gu.conj())
                        blk += c2 * np.einsum("ij,nm->nimj", tr, prof2)
                        out3 = voigt_faraday(self.a[iz], un + s[kv, klp]) + \
                            np.conj(voigt_faraday(self.a[iz], un + s[ku, klp]))
                        in3 = self.r3(iz, s[kv, kl], s[ku, kl])
                        blk += c3 * (be[ku, kv] - al[ku, kv]) * np.einsum("ij,n,m->nimj", tr, out3, in3)
        assert np.max(np.abs(blk.imag)) <= 1e-10 * max(1e-300, np.max(np.abs(blk.real)))
        return self.k[iz] * self.wang[op] * blk.real

    def sigma_bar(self, iz):
        """Dense comoving operator at one height, shape (nO*N*4, nO*N*4)."""
        nO, N = self.nO, self.nN
        S = np.zeros((nO, N, 4, nO, N, 4))
        for o in range(nO):
            for op in range(nO):
                S[o, :, :, op] = self.block(iz, o, op)
        return S.reshape(nO * N * 4, nO * N * 4)

    def interp_in(self, iz, o):
        """I(Omega',.) on the observer grid -> I~ at comoving nodes u_m (I(u_m - u_b))."""
        return self.spl[iz].basis(self.u[iz] - self.ub[iz, o])

    def interp_back(self, iz, o):
        return self.spl[iz].basis(self.u[iz] + self.ub[iz, o])

    @staticmethod
    def rayleigh(mu_o, chi_o, mu_p, chi_p):
        """Dipole phase matrix P[i, j] from direction Omega' (mu_p, chi_p) into
        Omega (mu_o, chi_o), normalised to oint P_00 dOmega'/4pi = 1."""
        eo, ep = pol_basis(mu_o, chi_o), pol_basis(mu_p, chi_p)
        J = np.array([[eo[a] @ ep[b] for b in range(2)] for a in range(2)])
        P = 0.75 * np.einsum("iab,bc,jcd,ad->ij", SIG, J, SIG, J)    # Tr(sigma_i J sigma_j J^T)
        assert np.max(np.abs(P.imag)) < 1e-13
        return P.real

    def continuum_block(self, iz, mu_o, chi_o):
        """sigma_c-weighted continuum scattering into one direction:
        C[n, i, o', j] with eps_c(n, i) = sum C[n, i, o', j] I(o', n, j)."""
        P = np.stack([self.rayleigh(mu_o, chi_o, self.mu[p], self.chi[p]) * self.wang[p] for p in range(self.nO)])
        return self.sig_c[iz][:, None, None, None] * P.transpose(1, 0, 2)[None]

    def sigma_matrix(self, iz, normalised=True, continuum=True):
        nO, N = self.nO, self.nN
        Sb = self.sigma_bar(iz).reshape(nO, N, 4, nO, N, 4)
        Uin = np.stack([self.interp_in(iz, o) for o in range(nO)])      # [o', m, n']
        Ub = np.stack([self.interp_back(iz, o) for o in range(nO)])     # [o, n, m]
        S = np.einsum("onm,omipkj,pkl->oniplj", Ub, Sb, Uin)   # eps(o,n,i) <- I(p,l,j)
        S = S.reshape(nO, N, 4, nO, N, 4)
        if normalised:
            S[:, :, 0] *= self.f[iz][:, :, None, None, None]
        if continuum and np.any(self.sig_c[iz]):
            for o in range(nO):
                C = self.continuum_block(iz, self.mu[o], self.chi[o])           # [n, i, o', j]
                for n in range(N):
                    S[o, n, :, :, n, :] += C[n]
        return S.reshape(nO * N * 4, nO * N * 4)

    def sigma_sample(self, x, iz, o):
        """eps(z, Omega, :) = Sigma x at one height and direction (normalised
        with f computed at the same point); for spot checks at full size."""
        N = self.nN
        sb = np.zeros((N, 4))
        sw = np.zeros((N, 4))
        Il = np.zeros((N, 4))
        Il[:, 0] = self.WT[iz]
        for op in range(self.nO):
            blk = self.block(iz, o, op).reshape(N * 4, N * 4)
            It = self.interp_in(iz, op) @ x[iz, op]
            sb += (blk @ It.ravel()).reshape(N, 4)
            sw += (blk @ (self.interp_in(iz, op) @ Il).ravel()).reshape(N, 4)
        Ub = self.interp_back(iz, o)
        eps = Ub @ sb
        num = (Ub @ sw)[:, 0]
        f = (1.0 - self.eps[iz]) * self.WT[iz] * self.eta1_line[iz, o] / num
        eps[:, 0] *= f
        eps += np.einsum("nipj,pnj->ni", self.continuum_block(iz, self.mu[o], self.chi[o]), x[iz])
        return eps, f

    def lambda_ray(self, eps, o, n):
        """Lambda eps along one ray (Omega, nu) for every height."""
        sub = eps[:, o:o + 1, n:n + 1]
        out = self.formal_solution(sub, K=self.K[:, o:o + 1, n:n + 1], eta1=self.eta1[:, o:o + 1, n:n + 1],
                                   dtau=self.dtau[:, o:o + 1, n:n + 1], mu=self.mu[o:o + 1])
        return out[:, 0, 0]

    def emergent(self, x, mu, chi):
        """Emergent Stokes vector at z_max along a line of sight (mu > 0, chi)
        off the grid (Sect. 6.2): scattering emissivity rows for the new
        direction, Kirchhoff factor from the same rows, thermal part, and one
        DELO-linear formal solution from the lower boundary."""
        nz, N = self.nz, self.nN
        n_l = unit_vector(np.array([mu]), np.array([chi]))[0]
        v = np.asarray(self.cfg["atm"]["v_kms"], float)
        eps = np.zeros((nz, 1, N, 4))
        K = np.zeros((nz, 1, N, 4, 4))
        for iz in range(nz):
            amp = self.amplitudes(iz, mu, chi)
            ub = (v[iz] @ n_l) / self.vD_kms[iz]
            K[iz, 0] = self.K_from_kappa(self.kappa(iz, amp, ub, self.u[iz]))
            eta_line = K[iz, 0, :, 0, 0].copy()
            sb = np.zeros((N, 4))
            sw = np.zeros((N, 4))
            Il = np.zeros((N, 4))
            Il[:, 0] = self.WT[iz]
            for op in range(self.nO):
                th = scattering_angle(n_l, self.nvec[op])
                th = 0.0 if th < 1e-10 else (np.pi if abs(th - np.pi) < 1e-10 else th)
                blk = self.block(iz, None, op, amp_o=amp, theta=th).reshape(N * 4, N * 4)
                Uin = self.interp_in(iz, op)
                sb += (blk @ (Uin @ x[iz, op]).ravel()).reshape(N, 4)
                sw += (blk @ (Uin @ Il).ravel()).reshape(N, 4)
            Ub = self.spl[iz].basis(self.u[iz] + ub)
            e = Ub @ sb
            f = (1.0 - self.eps[iz]) * self.WT[iz] * eta_line / (Ub @ sw)[:, 0]
            e[:, 0] *= f
            eps[iz, 0] = e + (self.eps[iz] * self.WT[iz]) * K[iz, 0, :, :, 0]
            eps[iz, 0, :, 0] += self.epsc_th[iz]
            eps[iz, 0] += np.einsum("nipj,pnj->ni", self.continuum_block(iz, mu, chi), x[iz])
            for s_ in range(4):
                K[iz, 0, :, s_, s_] += self.kap_c[iz] + self.sig_c[iz]
        eta1 = K[..., 0, 0]
        dtau = np.zeros((nz, 1, N))
        for k in range(1, nz):
            dtau[k, 0] = 0.5 * (eta1[k - 1, 0] + eta1[k, 0]) * (self.z[k] - self.z[k - 1]) / mu
        out = self.formal_solution(eps, boundary=True, K=K, eta1=eta1, dtau=dtau, mu=np.array([mu]))
        return out[-1, 0]

    def _normalisation(self):
        f = np.ones((self.nz, self.nO, self.nN))
        for iz in range(self.nz):
            Il = np.zeros((self.nO, self.nN, 4))
            Il[..., 0] = self.WT[iz]
            num = (self.sigma_matrix(iz, normalised=False, continuum=False) @ Il.ravel()).reshape(self.nO, self.nN, 4)
            ref = (1.0 - self.eps[iz]) * self.WT[iz] * self.eta1_line[iz]
            f[iz] = ref / num[..., 0]
        return f

    # ------------------------------------------------------------------ operator
    def sigma_mats(self):
        if not hasattr(self, "_smats"):
            self._smats = [self.sigma_matrix(iz) for iz in range(self.nz)]
        return self._smats

    def apply_sigma(self, x):
        mats = self.sigma_mats()
        out = np.zeros_like(x)
        for iz in range(self.nz):
            out[iz] = (mats[iz] @ x[iz].ravel()).reshape(x.shape[1:])
        return out

    def apply_A(self, x):
        return x - self.formal_solution(self.apply_sigma(x))

    def rhs(self):
        return self.formal_solution(self.eps_th, boundary=True)

    def solve(self, tol=1e-12, maxiter=2000, restart=400, x0=None):
        b = self.rhs()
        x, hist = gmres(lambda v: self.apply_A(v.reshape(b.shape)).ravel(), b.ravel(),
                        tol=tol, maxiter=maxiter, restart=restart,
                        x0=None if x0 is None else x0.ravel())
        return x.reshape(b.shape), hist

    def shape(self):
        return (self.nz, self.nO, self.nN, 4)

    # ------------------------------------------------------------------ transpose
    # Not in the paper (which solves forward problems only): the transposed
    # operator A^T = Id - Sigma^T Lambda^T, written out as the definition.
    # Sigma is block diagonal over heights (sigma_mats); Lambda is block
    # diagonal over rays (Omega, n), each block the (4 nz) x (4 nz) matrix whose
    # column (k, s) is the formal solution of a unit emissivity at height k in
    # Stokes s on that ray.
    def lambda_rays(self):
        if not hasattr(self, "_Lrays"):
            nz = self.nz
            L = np.zeros((self.nO, self.nN, nz, 4, nz, 4))
            for k in range(nz):
                for s in range(4):
                    e = np.zeros(self.shape())
                    e[k, :, :, s] = 1.0
                    L[:, :, :, :, k, s] = self.formal_solution(e).transpose(1, 2, 0, 3)
            self._Lrays = L.reshape(self.nO, self.nN, 4 * nz, 4 * nz)
        return self._Lrays

    def apply_AT(self, y):
        L = self.lambda_rays()
        yr = y.transpose(1, 2, 0, 3).reshape(self.nO, self.nN, 4 * self.nz)
        w = np.einsum("onji,onj->oni", L, yr)            # Lambda^T y, ray by ray
        w = w.reshape(self.nO, self.nN, self.nz, 4).transpose(2, 0, 1, 3)
        mats = self.sigma_mats()
        out = np.empty_like(y)
        for iz in range(self.nz):
            out[iz] = (mats[iz].T @ w[iz].ravel()).reshape(y.shape[1:])
        return y - out

    def solve_adjoint(self, g, tol=1e-13, maxiter=4000, restart=400):
        lam, hist = gmres(lambda v: self.apply_AT(v.reshape(g.shape)).ravel(), g.ravel(),
                          tol=tol, maxiter=maxiter, restart=restart)
        return lam.reshape(g.shape), hist


def gmres(A, b, tol, maxiter, restart, x0=None):
    """Restarted GMRES with modified Gram-Schmidt (plain FP64)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bn = np.linalg.norm(b)
    hist = []
    it = 0
    while it < maxiter:
        r = b - A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta / bn < tol:
            break
        m = min(restart, maxiter - it)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = A(V[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w -= H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            j_done = j + 1
            it += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / bn
            hist.append(res)
            if H[j + 1, j] > 1e-300:
                V[j + 1] = w / H[j + 1, j]
            if res < tol or H[j + 1, j] <= 1e-300:
                break
        x = x + V[:j_done].T @ y
    r = b - A(x)
    hist.append(np.linalg.norm(r) / bn)
    return x, hist
