"""Write the oracle reference values used by the GPU parity tests.

Calls only oracle/ and the seeded input generator; never the CUDA library.
Run from the repository root:  python tests/golden/make_golden.py [names...]
Outputs tests/golden/<name>.npz (forward operator and solution),
twolevel_full_sol.npz (the solution of the full two-level slab), <name>_nb.npz
(narrow-band signals along lines of sight), <name>_par.npz (the DELOPAR
formal solver), batch_*.npz (oracle solutions of the batched solve's instances),
<name>_adj.npz (transposed operator and adjoint solve), <name>_pc.npz (the
preconditioner with 1 and 2 sweeps) and grad_mgii_small.npz
(derivatives of an emergent-intensity functional by central differences of
forward solves).
"""
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from paper_2505_20968_gb300 import inputs   # noqa: E402
from oracle.problem import Problem          # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# reduced grids that span several tiles and a ragged tail, same physics as the workloads
CASES = {
    "twolevel": lambda: inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2),
    "twolevel_1mu": lambda: inputs.twolevel_slab(n_z=7, n_x=9, n_mu_half=1, n_chi=4, eps=1e-3),
    "mgii": lambda: inputs.mgii(n_z=10, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=21),
    "hi": lambda: inputs.hi_lya(n_z=10, n_core=13, n_wing=8, n_mu_half=2, n_chi=4, seed=31),
    "hi_aa": lambda: inputs.hi_lya(n_z=8, n_core=11, n_wing=6, n_mu_half=2, n_chi=4, seed=32,
                                   mode=inputs.MODE_AA),
    # with continuum absorption, emission and coherent scattering (App. A)
    "twolevel_cont": lambda: inputs.with_continuum(
        inputs.twolevel_slab(n_z=8, n_x=11, n_mu_half=2, n_chi=4, eps=1e-2), 1e-3, 0.4),
    "mgii_cont": lambda: inputs.with_continuum(
        inputs.mgii(n_z=10, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=21), 1e-5, 0.3),
}
# full-size workloads: sampled outputs the oracle can compute one by one
SAMPLES = {
    "mgii_full": (lambda: inputs.mgii(), [(35, 45)], [(45, 120), (3, 60)]),
    "twolevel_full": (lambda: inputs.twolevel_slab(), [(20, 5), (0, 2)], [(6, 10), (1, 0)]),
    # H I Ly-alpha size (90 x 96 x 150): work items with more than 32 incident directions
    "hi_full": (lambda: inputs.hi_lya(), [(45, 60)], [(60, 75), (5, 10)]),
    "hi_aa_full": (lambda: inputs.hi_lya(mode=inputs.MODE_AA), [(45, 60)], []),
}


def seeded_x(shape, seed):
    x = inputs.seeded_vector(shape, seed, 0.1, 1.0)
    x[..., 1:] *= 0.05
    return x


def make_case(name):
    cfg = CASES[name]()
    P = Problem(cfg)
    x = seeded_x(P.shape(), 5)
    eo = P.apply_sigma(x)
    sol, hist = P.solve(tol=1e-13)
    los = np.array([[0.1, 0.0], [1.0, 0.0], [0.55, 1.3]])
    em = np.stack([P.emergent(sol, m, c) for m, c in los])
    np.savez_compressed(os.path.join(HERE, name + ".npz"), x=x, sigma=eo, lam=P.formal_solution(eo),
                        rhs=P.rhs(), Ax=P.apply_A(x), sol=sol, mu=P.mu, f=P.f, los=los, emergent=em)


# transposed operator and adjoint solve, on the reduced forward cases; y and g
# are drawn as the GPU tests draw their vectors (polarisation 10x smaller)
ADJOINT = ("twolevel", "mgii", "hi", "hi_aa")


def adj_vec(shape, seed):
    v = inputs.seeded_vector(shape, seed, 0.1, 1.0)
    v[..., 1:] = v[..., 1:] * 0.1 - 0.05
    return v


def make_adjoint(name):
    P = Problem(CASES[name]())
    y, g = adj_vec(P.shape(), 2), adj_vec(P.shape(), 7)
    lam, hist = P.solve_adjoint(g, tol=1e-13)
    np.savez_compressed(os.path.join(HERE, name + "_adj.npz"), y=y, ATy=P.apply_AT(y), g=g, lam=lam,
                        res=hist[-1])


# preconditioner (Sect. 5.2, App. F) applied to a seeded vector with 1 and 2 sweeps
PRECOND = ("twolevel", "mgii", "hi")


def make_precond(name):
    from oracle.preconditioner import Preconditioner
    P = Problem(CASES[name](), normalise=False)
    C = Preconditioner(P)
    y = inputs.seeded_vector(P.shape(), 11, -1.0, 1.0)
    np.savez_compressed(os.path.join(HERE, name + "_pc.npz"), y=y, m1=C.apply_inv(y, 1), m2=C.apply_inv(y, 2))


# dJ/d(B, theta_B, chi_B) per height for J = sum of the emergent Stokes I
# (top height, mu > 0, every frequency) of the forward solution: central
# differences of J at steps h and h/2, h = max(1e-3 |p|, 0.1 G for B, 1e-3 rad)
GRAD_KEYS = ("B_G", "thetaB", "chiB")


def grad_case():
    return inputs.mgii(n_z=6, n_core_each=5, n_wing=4, n_mu_half=1, n_chi=4, seed=23)


def grad_step(k, p0):
    return max(1e-3 * abs(p0), 0.1 if k == 0 else 1e-3)


def J_of(job):
    k, iz, val = job
    cfg = grad_case()
    if k >= 0:
        cfg["atm"][GRAD_KEYS[k]] = np.array(cfg["atm"][GRAD_KEYS[k]], dtype=np.float64)
        cfg["atm"][GRAD_KEYS[k]][iz] = val
    P = Problem(cfg)
    x, _ = P.solve(tol=1e-13)
    return float(x[-1, P.mu > 0, :, 0].sum())


def make_grad():
    cfg = grad_case()
    nz = len(cfg["atm"]["z_km"])
    jobs, steps = [(-1, 0, 0.0)], np.zeros((nz, 3))
    for iz in range(nz):
        for k in range(3):
            p0 = float(cfg["atm"][GRAD_KEYS[k]][iz])
            h = steps[iz, k] = grad_step(k, p0)
            jobs += [(k, iz, p0 + h), (k, iz, p0 - h), (k, iz, p0 + h / 2), (k, iz, p0 - h / 2)]
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=get_context("spawn")) as ex:
        J = list(ex.map(J_of, jobs))
    Jp = np.array(J[1:]).reshape(nz, 3, 4)
    fd = (Jp[..., 0] - Jp[..., 1]) / (2 * steps)
    fd_half = (Jp[..., 2] - Jp[..., 3]) / steps
    np.savez_compressed(os.path.join(HERE, "grad_mgii_small.npz"), fd=fd, fd_half=fd_half, step=steps, J0=J[0])


# narrow-band signals (Sect. 6.5) of the reduced cases' oracle solutions along
# lines of sight at chi = 0: the H I cases with the paper's band (lambda_0 =
# 1215.67 A, FWHM 35 A, +-30 A), the two-level slab with a band of its own width
NB = {"hi": (1215.67, 35.0, 30.0), "hi_aa": (1215.67, 35.0, 30.0), "twolevel": (None, 0.08, 0.1)}
NB_MU = np.array([0.1, 0.3, 0.5, 0.7, 0.9, 1.0])


def make_narrowband(name):
    from oracle.narrowband import narrowband, grid_wavelengths
    P = Problem(CASES[name]())
    sol = np.load(os.path.join(HERE, name + ".npz"))["sol"]
    lam = grid_wavelengths(P)
    lam0, fwhm, half = NB[name]
    if lam0 is None:
        lam0 = 0.5 * (lam[0] + lam[-1])
    em = np.stack([P.emergent(sol, m, 0.0) for m in NB_MU])
    np.savez_compressed(os.path.join(HERE, name + "_nb.npz"), mu=NB_MU, lam0=lam0, fwhm=fwhm, half=half, em=em,
                        xbar=narrowband(lam, em, lam0, fwhm, half))


# the DELOPAR formal solver (Sect. 3) on reduced cases: Lambda of the stored
# emissivity, the right-hand side and the solution to 1e-13
PAR = ("twolevel", "hi")


def make_delopar(name):
    P = Problem(CASES[name](), formal_solver="delopar")
    G = np.load(os.path.join(HERE, name + ".npz"))
    sol, hist = P.solve(tol=1e-13)
    np.savez_compressed(os.path.join(HERE, name + "_par.npz"), lam=P.formal_solution(G["sigma"]), rhs=P.rhs(),
                        sol=sol, res=hist[-1])


# ragged instances of the batched solve (the config-2 physics at reduced sizes):
# the oracle's solutions to 1e-13
BATCH = {
    "batch_mgii7": lambda: inputs.mgii(n_z=7, n_core_each=7, n_wing=6, n_mu_half=2, n_chi=4, seed=401),
    "batch_mgii9": lambda: inputs.mgii(n_z=9, n_core_each=9, n_wing=8, n_mu_half=2, n_chi=4, seed=402),
    "batch_hi6": lambda: inputs.hi_lya(n_z=6, n_core=9, n_wing=6, n_mu_half=2, n_chi=4, seed=403),
}


def make_batch(name):
    P = Problem(BATCH[name]())
    sol, hist = P.solve(tol=1e-13)
    np.savez_compressed(os.path.join(HERE, name + ".npz"), sol=sol, res=hist[-1])


# the full two-level slab (40 heights x 8 directions x 21 frequencies, FP64):
# the solution to tol 1e-12 and its emergent Stokes vectors
def make_full_solve():
    P = Problem(inputs.twolevel_slab())
    sol, hist = P.solve(tol=1e-12)
    los = np.array([[0.1, 0.0], [1.0, 0.0], [0.55, 1.3]])
    em = np.stack([P.emergent(sol, m, c) for m, c in los])
    np.savez_compressed(os.path.join(HERE, "twolevel_full_sol.npz"), sol=sol, rhs=P.rhs(), res=hist[-1],
                        iters=len(hist), los=los, emergent=em)


def make_sample(name):
    mk, sig_pts, ray_pts = SAMPLES[name]
    cfg = mk()
    P = Problem(cfg, normalise=False)
    x = seeded_x(P.shape(), 5)
    out = {}
    for iz, o in sig_pts:
        eps, f = P.sigma_sample(x, iz, o)
        out[f"sigma_{iz}_{o}"] = eps
        out[f"f_{iz}_{o}"] = f
    for o, n in ray_pts:
        out[f"lam_{o}_{n}"] = P.lambda_ray(x, o, n)
    np.savez_compressed(os.path.join(HERE, name + ".npz"), **out)


if __name__ == "__main__":
    names = sys.argv[1:] or (list(CASES) + list(SAMPLES) + [a + "_adj" for a in ADJOINT] + ["grad"]
                             + [a + "_pc" for a in PRECOND] + ["twolevel_full_sol"] + [a + "_nb" for a in NB]
                             + [a + "_par" for a in PAR] + list(BATCH))
    for nm in names:
        t0 = time.time()
        if nm in CASES:
            make_case(nm)
        elif nm in SAMPLES:
            make_sample(nm)
        elif nm.endswith("_adj"):
            make_adjoint(nm[:-4])
        elif nm.endswith("_pc"):
            make_precond(nm[:-3])
        elif nm == "grad":
            make_grad()
        elif nm == "twolevel_full_sol":
            make_full_solve()
        elif nm.endswith("_nb"):
            make_narrowband(nm[:-3])
        elif nm.endswith("_par"):
            make_delopar(nm[:-4])
        elif nm in BATCH:
            make_batch(nm)
        else:
            raise SystemExit(f"unknown golden set {nm}")
        print(f"{nm}: {time.time() - t0:.1f} s", flush=True)
