"""Two-level / two-term atom with an unpolarised, infinitely sharp lower term
(Sect. 2.2) and Paschen-Back upper-term levels (oracle).

Upper term L_u = 1 with spin S (S = 0: two-level atom J_l = 0 -> J_u = 1;
S = 1/2: the S_1/2 -> P_1/2,3/2 doublets of Table 1).  In the magnetic frame
(z_B along B) the upper-term Hamiltonian in the uncoupled basis |M_L, M_S> is
    H_u = zeta L.S + nu_L (L_z + g_s S_z),      nu_L = mu_B B / h,
diagonalised numerically (full Paschen-Back regime, "j" label of Sect. 2.2).
zeta follows from the two J-level energies: E(3/2) - E(1/2) = (3/2) zeta.
The lower term (L_l = 0) has states |M_S> with energies nu_L g_s M_S.

Dipole matrix elements in the uncoupled basis: spin is a spectator and
<L_u=1 M_L | d_q | L_l=0> = delta(M_L, q) (Wigner-Eckart, reduced element 1),
so <k_u | d_q | k_l=M_S> is the eigenvector component on |M_L=q, M_S>.
"""
import numpy as np
from .constants import CM_TO_HZ, MU_B_OVER_H, GAUSS


def nu0_of(atom):
    """Reference frequency: (2J+1)-weighted centroid of the upper levels (Sect. 2.4)."""
    if atom.get("nu0_hz", 0.0):
        return float(atom["nu0_hz"])
    E = atom["E_u_cm"]
    if atom["twoS"] == 0:
        return E[0] * CM_TO_HZ
    return (2.0 * E[0] + 4.0 * E[1]) / 6.0 * CM_TO_HZ


def states(atom, B_gauss):
    """Return (E_u [Hz rel. nu0], D[q, ku, kl], E_l [Hz]) with q index 0,1,2 <-> q=-1,0,+1."""
    nu0 = nu0_of(atom)
    nuL = MU_B_OVER_H * GAUSS * B_gauss
    gs = atom.get("g_s", 2.0)
    E = atom["E_u_cm"]
    if atom["twoS"] == 0:
        basis = [(ml, 0.0) for ml in (-1, 0, 1)]
        H = np.diag([nuL * ml for ml, _ in basis]) + (E[0] * CM_TO_HZ - nu0) * np.eye(3)
        lower_ms = [0.0]
    else:
        zeta = (E[1] - E[0]) * CM_TO_HZ / 1.5
        Ec = E[0] * CM_TO_HZ + zeta - nu0
        basis = [(ml, ms) for ml in (-1, 0, 1) for ms in (-0.5, 0.5)]
        nb = len(basis)
        H = np.zeros((nb, nb))
        for i, (ml, ms) in enumerate(basis):
            H[i, i] = Ec + zeta * ml * ms + nuL * (ml + gs * ms)
            for j, (ml2, ms2) in enumerate(basis):
                # (zeta/2)(L+ S- + L- S+)
                if ml2 == ml + 1 and ms2 == ms - 1:      # L+ S- |ml,ms> -> |ml+1, ms-1>
                    H[j, i] += 0.5 * zeta * np.sqrt(2 - ml * (ml + 1)) * np.sqrt(0.75 - ms * (ms - 1))
                if ml2 == ml - 1 and ms2 == ms + 1:      # L- S+
                    H[j, i] += 0.5 * zeta * np.sqrt(2 - ml * (ml - 1)) * np.sqrt(0.75 - ms * (ms + 1))
        lower_ms = [-0.5, 0.5]
    Eu, V = np.linalg.eigh(H)
    nu_, nl = len(basis), len(lower_ms)
    D = np.zeros((3, nu_, nl))
    for kl, msl in enumerate(lower_ms):
        for qi, q in enumerate((-1, 0, 1)):
            for b, (ml, ms) in enumerate(basis):
                if ml == q and ms == msl:
                    D[qi, :, kl] += V[b, :]
    El = np.array([nuL * gs * ms for ms in lower_ms])
    return Eu, D, El
