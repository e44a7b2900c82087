"""Write the oracle reference values used by the GPU parity tests.

Calls only oracle/ and the seeded input generator; never the CUDA library.
Run from the repository root:  python tests/golden/make_golden.py [names...]
Outputs tests/golden/<name>.npz.
"""
import os
import sys
import time

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
}
# full-size workloads: sampled outputs the oracle can compute one by one
SAMPLES = {
    "mgii_full": (lambda: inputs.mgii(), [(35, 45)], [(45, 120), (3, 60)]),
    "twolevel_full": (lambda: inputs.twolevel_slab(), [(20, 5), (0, 2)], [(6, 10), (1, 0)]),
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
    names = sys.argv[1:] or list(CASES) + list(SAMPLES)
    for nm in names:
        t0 = time.time()
        (make_case if nm in CASES else make_sample)(nm)
        print(f"{nm}: {time.time() - t0:.1f} s", flush=True)
