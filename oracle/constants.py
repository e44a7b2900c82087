"""Physical constants (CODATA 2018, SI unless stated).  Oracle-only copy."""
C_LIGHT = 2.99792458e8          # m/s
K_BOLTZ = 1.380649e-23          # J/K
AMU = 1.66053906660e-27         # kg
MU_B_OVER_H = 1.39962449361e10  # Hz per tesla (Bohr magneton / Planck)
GAUSS = 1e-4                    # tesla per gauss
CM_TO_HZ = 2.99792458e10        # wavenumber (cm^-1) -> Hz
