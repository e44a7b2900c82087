"""Host logic of the library, without a GPU: the angular grid, the
scattering-angle classes and the class -> output direction -> incident
direction tables (build_host_tables in csrc/host_setup.cpp) that every Sigma
kernel indexes through.  A small C++ driver fills a context through the C ABI
setters (host copies only), calls build_host_tables and checks:

* N_Theta = 205 on the paper's 2 x 6 Gauss-Legendre mu x 9 chi grid (Sect. 6.2);
* the weights integrate the sphere (sum = 1) and P_2(mu) to zero;
* every ordered pair (o, o') appears exactly once, under the class whose angle
  equals the pair's scattering angle to 1e-10, on the paper's odd-N_chi grid
  (no back-scattering pairs) and on an even one (whose Theta = pi class is
  exactly pi);
* per class, the output entries and their pair ranges are consistent CSR.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cmath>
#include <cstdio>
#include <vector>
#include "prd_internal.h"
static double angle(const prd::Ctx* c, int o, int p) {
  double a[3], b[3];
  const int idx[2] = {o, p};
  double* v[2] = {a, b};
  for (int s = 0; s < 2; ++s) {
    const double m = c->mu[idx[s]], ch = c->chi[idx[s]], sn = std::sqrt(std::fmax(0.0, 1.0 - m * m));
    v[s][0] = sn * std::cos(ch); v[s][1] = sn * std::sin(ch); v[s][2] = m;
  }
  // half-chord forms, well conditioned near 0 and near pi
  const double dm = std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
  const double dp = std::sqrt((a[0] + b[0]) * (a[0] + b[0]) + (a[1] + b[1]) * (a[1] + b[1]) + (a[2] + b[2]) * (a[2] + b[2]));
  return dm <= dp ? 2.0 * std::asin(0.5 * dm) : prd::kPi - 2.0 * std::asin(0.5 * dp);
}
// every ordered pair once, under the class of its angle; CSR consistent
static int check_pairs(const prd::Ctx* c) {
  const int nO = c->nO;
  if ((int)c->cout_ptr.size() != c->ncls + 1 || c->cout_ptr[0] != 0) return 23;
  for (int cl = 1; cl < c->ncls; ++cl)
    if (!(c->theta[cl] > c->theta[cl - 1])) return 32;                // classes ascending
  if (c->theta.front() != 0.0 || c->theta.back() > prd::kPi) return 31;
  std::vector<int> seen((size_t)nO * nO, 0);
  for (int cl = 0; cl < c->ncls; ++cl)
    for (int e = c->cout_ptr[cl]; e < c->cout_ptr[cl + 1]; ++e) {
      const int o = c->cout_dir[e];
      if (c->pair_ptr[e + 1] <= c->pair_ptr[e]) return 24;           // an output entry has pairs
      for (int q = c->pair_ptr[e]; q < c->pair_ptr[e + 1]; ++q) {
        const int p = c->pair_in[q];
        if (o < 0 || o >= nO || p < 0 || p >= nO) return 25;
        if (seen[(size_t)o * nO + p]++) return 26;                   // each pair once
        if (c->cls[(size_t)o * nO + p] != cl) return 27;
        if (std::fabs(angle(c, o, p) - c->theta[cl]) > 1e-10) { std::printf("pair %d %d\n", o, p); return 28; }
      }
    }
  for (int i = 0; i < nO * nO; ++i) if (seen[i] != 1) return 29;     // every pair present
  if (c->npairs != nO * nO || c->pair_ptr.back() != nO * nO) return 30;
  return 0;
}
int main() {
  prd_ctx* h = new prd_ctx();
  prd::Ctx* c = &h->c;
  prd_atom at{};
  at.kind = PRD_TWO_LEVEL; at.twoS = 0; at.E_u_cm[0] = 35760.88; at.mass_amu = 24.305; at.g_s = 2.0;
  if (prd_set_atom(h, &at)) return 10;
  const int nz = 2;
  std::vector<double> z = {0.0, 100.0}, T(nz, 6000.0), xi(nz, 1.0), a(nz, 1e-3), eps(nz, 1e-3), r(nz, 0.1),
      k(nz, 1.0), W(nz, 1.0), B(nz, 10.0), th(nz, 0.5), chb(nz, 0.2), v(3 * nz, 0.0);
  if (prd_set_atmosphere(h, nz, z.data(), T.data(), xi.data(), a.data(), eps.data(), r.data(), k.data(), W.data(),
                         B.data(), th.data(), chb.data(), v.data())) return 11;
  std::vector<double> x;
  for (int i = 0; i < 9; ++i) x.push_back(-4.0 + i);
  // the paper's grid: odd N_chi, so no direction has its antipode on the grid
  if (prd_set_quadrature(h, 9, x.data(), PRD_GRID_X, 6, 9, PRD_MU_GL_HEMISPHERES, PRD_MODE_AD)) return 12;
  if (prd::build_host_tables(c)) return 13;
  if (c->nO != 108) return 20;
  if (c->ncls != 205) { std::printf("ncls %d\n", c->ncls); return 21; }
  double sw = 0, sp2 = 0;
  for (int o = 0; o < c->nO; ++o) { sw += c->wang[o]; sp2 += c->wang[o] * 0.5 * (3 * c->mu[o] * c->mu[o] - 1); }
  if (std::fabs(sw - 1.0) > 1e-14 || std::fabs(sp2) > 1e-14) return 22;
  int rc = check_pairs(c);
  if (rc) return rc;
  if (!(c->theta.back() < prd::kPi - 1e-3)) return 33;
  // an even N_chi grid has back-scattering pairs: their class is exactly pi
  if (prd_set_quadrature(h, 9, x.data(), PRD_GRID_X, 4, 8, PRD_MU_GL_HEMISPHERES, PRD_MODE_AD)) return 14;
  if (prd::build_host_tables(c)) return 15;
  if ((rc = check_pairs(c))) return 100 + rc;
  if (c->theta.back() != prd::kPi) return 34;
  std::printf("ok\n");
  delete h;
  return 0;
}
'''


def test_angle_classes_and_pair_tables(tmp_path):
    from paper_2505_20968_gb300 import build
    gxx = shutil.which("g++")
    cuda = "/usr/local/cuda"
    if not gxx or not os.path.isdir(os.path.join(cuda, "include")):
        pytest.skip("g++ or the CUDA toolkit is missing")
    lib = build.build()
    libdir = os.path.dirname(lib)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    if cudalib is None:
        pytest.skip("libcudart.so not found")
    src, exe = tmp_path / "tables.cpp", tmp_path / "tables"
    src.write_text(SRC)
    csrc = os.path.join(ROOT, "paper_2505_20968_gb300", "csrc")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", csrc, "-I", os.path.join(cuda, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lprd", "-Wl,-rpath," + libdir, "-L", cudalib, "-lcudart",
                        "-Wl,-rpath," + cudalib], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stdout, r.stderr[-2000:])


DUMP = r'''
#include <cstdio>
#include <vector>
#include "prd_internal.h"
// reads a problem (text), builds the library's host tables and prints them
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "r");
  if (!f) return 2;
  prd_atom at{};
  int twoS, nz;
  if (std::fscanf(f, "%d %lf %lf %lf %lf %d", &twoS, &at.E_u_cm[0], &at.E_u_cm[1], &at.mass_amu, &at.g_s, &nz) != 6)
    return 3;
  at.twoS = twoS;
  at.kind = twoS ? PRD_TWO_TERM : PRD_TWO_LEVEL;
  std::vector<std::vector<double>> A(11, std::vector<double>(nz));
  for (auto& arr : A) for (auto& x : arr) if (std::fscanf(f, "%lf", &x) != 1) return 4;
  std::vector<double> v(3 * nz);
  for (auto& x : v) if (std::fscanf(f, "%lf", &x) != 1) return 5;
  int nnu, kind, nmu, nchi;
  if (std::fscanf(f, "%d %d %d %d", &nnu, &kind, &nmu, &nchi) != 4) return 6;
  std::vector<double> grid(nnu);
  for (auto& x : grid) if (std::fscanf(f, "%lf", &x) != 1) return 7;
  std::fclose(f);
  prd_ctx* h = new prd_ctx();
  prd::Ctx* c = &h->c;
  if (prd_set_atom(h, &at)) return 8;
  if (prd_set_atmosphere(h, nz, A[0].data(), A[1].data(), A[2].data(), A[3].data(), A[4].data(), A[5].data(),
                         A[6].data(), A[7].data(), A[8].data(), A[9].data(), A[10].data(), v.data())) return 9;
  if (prd_set_quadrature(h, nnu, grid.data(), kind, nmu, nchi, PRD_MU_GL_HEMISPHERES, PRD_MODE_AD)) return 10;
  if (prd::build_host_tables(c)) return 11;
  const int nu = c->nu_st, nl = c->nl_st, nO = c->nO;
  std::printf("%d %d %d %d\n", nz, nO, nu, nl);
  for (int iz = 0; iz < nz; ++iz) std::printf("%.17g\n", c->dnuD[iz]);
  for (double x : c->shift) std::printf("%.17g\n", x);
  for (auto z : c->alpha) std::printf("%.17g %.17g\n", z.real(), z.imag());
  for (auto z : c->beta) std::printf("%.17g %.17g\n", z.real(), z.imag());
  for (auto z : c->amp) std::printf("%.17g %.17g\n", z.real(), z.imag());
  delete h;
  return 0;
}
'''


def _build_exe(tmp_path, name, src_text):
    from paper_2505_20968_gb300 import build
    gxx = shutil.which("g++")
    cuda = "/usr/local/cuda"
    if not gxx or not os.path.isdir(os.path.join(cuda, "include")):
        pytest.skip("g++ or the CUDA toolkit is missing")
    libdir = os.path.dirname(build.build())
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    if cudalib is None:
        pytest.skip("libcudart.so not found")
    src, exe = tmp_path / (name + ".cpp"), tmp_path / name
    src.write_text(src_text)
    csrc = os.path.join(ROOT, "paper_2505_20968_gb300", "csrc")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", csrc, "-I", os.path.join(cuda, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lprd", "-Wl,-rpath," + libdir, "-L", cudalib, "-lcudart",
                        "-Wl,-rpath," + cudalib], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def test_atom_tables_match_the_oracle(tmp_path):
    """S0 host tables of the library against the oracle, on Mg II physics with
    a strong-field (Paschen-Back) height added: Doppler widths, the upper-state
    energies seen as shifts from each lower state, the branching ratios
    alpha/beta of every upper-state pair (App. B), and the products of
    polarisation amplitudes conj(a(k_u, k_l')) a(k_u, k_l) of every direction
    pair, which do not depend on the phase of each eigenvector.  The library
    diagonalises the Hamiltonian in fixed-M 2 x 2 blocks, the oracle as a full
    matrix; states are matched by energy."""
    import numpy as np
    from paper_2505_20968_gb300 import inputs
    from oracle.problem import Problem
    cfg = inputs.mgii(n_z=4, n_core_each=4, n_wing=4, n_mu_half=1, n_chi=4, seed=17)
    atm = cfg["atm"]
    atm["B_G"] = np.array(atm["B_G"], dtype=np.float64)
    atm["B_G"][2] = 3000.0
    exe = _build_exe(tmp_path, "dump", DUMP)
    at = cfg["atom"]
    keys = ("z_km", "T_K", "xi_kms", "a", "eps", "r_el", "k_line", "W_T", "B_G", "thetaB", "chiB")
    lines = [f"{at['twoS']} {at['E_u_cm'][0]!r} {at['E_u_cm'][1]!r} {at['mass_amu']!r} {at['g_s']!r} {len(atm['z_km'])}"]
    lines += [" ".join(repr(float(x)) for x in np.asarray(atm[k], dtype=np.float64)) for k in keys]
    lines.append(" ".join(repr(float(x)) for x in np.asarray(atm["v_kms"], dtype=np.float64).ravel()))
    q = cfg["quad"]
    lines.append(f"{len(q['grid'])} {q['grid_kind']} {q['n_mu_half']} {q['n_chi']}")
    lines.append(" ".join(repr(float(x)) for x in q["grid"]))
    (tmp_path / "problem.txt").write_text("\n".join(lines) + "\n")
    r = subprocess.run([str(exe), str(tmp_path / "problem.txt")], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    tok = r.stdout.split()
    nz, nO, nu, nl = map(int, tok[:4])
    vals = np.array([float(t) for t in tok[4:]])
    pos = 0

    def take(n):
        nonlocal pos
        out = vals[pos:pos + n]
        pos += n
        return out
    dnuD = take(nz)
    shift = take(nz * nu * nl).reshape(nz, nu, nl)
    cz = lambda n: take(2 * n).reshape(-1, 2) @ np.array([1.0, 1j])
    alpha = cz(nz * nu * nu).reshape(nz, nu, nu)
    beta = cz(nz * nu * nu).reshape(nz, nu, nu)
    amp = cz(nz * nO * 2 * nu * nl).reshape(nz, nO, 2, nu, nl)
    assert pos == vals.size
    P = Problem(cfg, normalise=False)
    assert P.nO == nO and P.nu_states == nu and P.nl_states == nl
    assert np.max(np.abs(dnuD / P.dnuD - 1.0)) < 1e-14
    for iz in range(nz):
        pl = np.argsort(shift[iz][:, 0], kind="stable")
        po = np.argsort(P.shift[iz][:, 0], kind="stable")
        assert np.max(np.abs(shift[iz][pl] - P.shift[iz][po])) < 1e-9 * np.max(np.abs(P.shift[iz]))
        # energies ~3e12 Hz carry ~6e-4 Hz of rounding; over Gamma ~1e8 s^-1 that is ~4e-11 in alpha
        assert np.max(np.abs(alpha[iz][np.ix_(pl, pl)] - P.alpha[iz][np.ix_(po, po)])) < 1e-10
        assert np.max(np.abs(beta[iz][np.ix_(pl, pl)] - P.beta[iz][np.ix_(po, po)])) < 1e-10
        if P.cfg["atm"]["B_G"][iz] < 1.0:
            continue                      # near-degenerate states: per-state products are not unique
        for o, op in ((0, 1), (2, 7), (5, 5)):
            for kl in range(nl):
                for klp in range(nl):
                    ml = np.einsum("au,gu->uag", amp[iz, o, :, :, klp].conj(), amp[iz, op, :, :, kl])[pl]
                    mo = np.einsum("au,gu->uag", P.amp[iz][o][:, :, klp].conj(), P.amp[iz][op][:, :, kl])[po]
                    assert np.max(np.abs(ml - mo)) < 1e-12, (iz, o, op, kl, klp)


LOS = DUMP.replace('''  const int nu = c->nu_st, nl = c->nl_st, nO = c->nO;
  std::printf("%d %d %d %d\\n", nz, nO, nu, nl);
  for (int iz = 0; iz < nz; ++iz) std::printf("%.17g\\n", c->dnuD[iz]);
  for (double x : c->shift) std::printf("%.17g\\n", x);
  for (auto z : c->alpha) std::printf("%.17g %.17g\\n", z.real(), z.imag());
  for (auto z : c->beta) std::printf("%.17g %.17g\\n", z.real(), z.imag());
  for (auto z : c->amp) std::printf("%.17g %.17g\\n", z.real(), z.imag());''', '''  prd::LosTables L;
  const double mu = std::atof(argv[2]), chi = std::atof(argv[3]);
  prd::los_tables(c, mu, chi, L);
  std::printf("%d %d\\n", nz, nnu);
  for (double x : L.kt) std::printf("%.17g\\n", x);
  for (double x : L.epsth) std::printf("%.17g\\n", x);''').replace("#include <cstdio>", "#include <cstdio>\n#include <cstdlib>")


def test_line_of_sight_tables_match_the_oracle(tmp_path):
    """S11 host tables of an off-grid line of sight (los_tables in
    csrc/host_tables.cpp) against the oracle's emergent-Stokes set-up, on
    magnetised Mg II physics with bulk velocities: the propagation matrix K
    (absorption and magneto-optical terms, Sect. 2.1; from the forward
    scattering amplitudes) as K_ij / eta_I and 1 / eta_I, the thermal
    emissivity eps W_T K[:, 0] (Sect. 2.3) and the DELO-linear weights of
    every step along the line of sight (Sect. 3)."""
    import numpy as np
    from paper_2505_20968_gb300 import inputs
    from oracle.problem import Problem, delo_coeffs
    from oracle.geometry import unit_vector
    cfg = inputs.mgii(n_z=4, n_core_each=4, n_wing=4, n_mu_half=1, n_chi=4, seed=17)
    cfg["atm"]["B_G"] = np.array(cfg["atm"]["B_G"], dtype=np.float64)
    cfg["atm"]["B_G"][1] = 800.0
    exe = _build_exe(tmp_path, "los", LOS)
    at, atm, q = cfg["atom"], cfg["atm"], cfg["quad"]
    keys = ("z_km", "T_K", "xi_kms", "a", "eps", "r_el", "k_line", "W_T", "B_G", "thetaB", "chiB")
    lines = [f"{at['twoS']} {at['E_u_cm'][0]!r} {at['E_u_cm'][1]!r} {at['mass_amu']!r} {at['g_s']!r} {len(atm['z_km'])}"]
    lines += [" ".join(repr(float(x)) for x in np.asarray(atm[k], dtype=np.float64)) for k in keys]
    lines.append(" ".join(repr(float(x)) for x in np.asarray(atm["v_kms"], dtype=np.float64).ravel()))
    lines.append(f"{len(q['grid'])} {q['grid_kind']} {q['n_mu_half']} {q['n_chi']}")
    lines.append(" ".join(repr(float(x)) for x in q["grid"]))
    (tmp_path / "problem.txt").write_text("\n".join(lines) + "\n")
    P = Problem(cfg, normalise=False)
    nz, N = P.nz, P.nN
    v = np.asarray(atm["v_kms"], dtype=np.float64)
    for mu, chi in ((0.3, 0.7), (0.95, 4.0)):
        r = subprocess.run([str(exe), str(tmp_path / "problem.txt"), repr(mu), repr(chi)],
                           capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
        tok = r.stdout.split()
        assert (int(tok[0]), int(tok[1])) == (nz, N)
        vals = np.array([float(t) for t in tok[2:]])
        kt = vals[:nz * N * 10].reshape(nz, N, 10)
        epsth = vals[nz * N * 10:].reshape(nz, N, 4)
        n_l = unit_vector(np.array([mu]), np.array([chi]))[0]
        K = np.stack([P.K_from_kappa(P.kappa(iz, P.amplitudes(iz, mu, chi), (v[iz] @ n_l) / P.vD_kms[iz], P.u[iz]))
                      for iz in range(nz)])                           # [z][n][4][4]
        e1 = K[..., 0, 0]
        ref = np.stack([K[..., 0, 1], K[..., 0, 2], K[..., 0, 3], K[..., 1, 2], K[..., 1, 3], K[..., 2, 3]], -1)
        # Far in the wings eta_I is ~1e-9 of its core value, and both sides' Faddeeva values
        # carry ~1e-15 |w| of absolute error, i.e. up to ~1e-9 relative in H = Re w (|w| / H ~ v / a);
        # the magneto-optical ratios there are differences of nearly equal dispersion profiles.
        # K / eta_I multiplies I in the transfer equation: 1e-8 relative plus 1e-9 absolute.
        r = ref / e1[..., None]
        assert np.all(np.abs(kt[..., :6] - r) <= 1e-8 * np.abs(r) + 1e-9)
        assert np.max(np.abs(kt[..., 6] * e1 - 1.0)) < 1e-8
        eth = (P.eps * P.WT)[:, None, None] * K[..., :, 0]
        assert np.max(np.abs(epsth - eth)) < 1e-12 * np.max(np.abs(eth))
        dtau = 0.5 * (e1[:-1] + e1[1:]) * np.diff(P.z)[:, None] / mu
        e, al, be = delo_coeffs(dtau)
        # the optical depths inherit eta_I's far-wing difference (~1e-9 relative)
        for got, want in ((kt[1:, :, 7], e), (kt[1:, :, 8], al), (kt[1:, :, 9], be)):
            assert np.max(np.abs(got - want)) < 1e-10


FAD = r'''
#include <complex>
#include <cstdio>
#include <cstdlib>
namespace prd { std::complex<double> faddeeva_host(std::complex<double>); }
int main(int argc, char** argv) {
  for (int i = 1; i + 1 < argc; i += 2) {
    const std::complex<double> w = prd::faddeeva_host({std::atof(argv[i]), std::atof(argv[i + 1])});
    std::printf("%.17g %.17g\n", w.real(), w.imag());
  }
  return 0;
}
'''


def test_host_faddeeva_against_scipy(tmp_path):
    """The library's FP64 Faddeeva function W(a, v) = w(v + i a) (Sect. 2.4;
    Weideman's rational series) against scipy.special.wofz: L = Im w to 1e-14
    everywhere; H = Re w to 1e-12 in the core (|v| <= 2) and, in the wings, to
    the floor of evaluating H as Re w (absolute ~1e-15 |w|, so ~1e-15 v / a
    relative; measured 6e-10 at a = 1e-4)."""
    import numpy as np
    from scipy.special import wofz
    exe = _build_exe(tmp_path, "fad", FAD)
    pts = [(v, a) for a in (1e-4, 1e-3, 1e-2, 0.3) for v in (0.0, 0.5, 2.0, 3.0, 10.0, 30.0, 150.0, 1000.0, -7.5)]
    args = [repr(x) for v, a in pts for x in (v, a)]
    r = subprocess.run([str(exe)] + args, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0
    got = np.array([[float(s) for s in line.split()] for line in r.stdout.strip().splitlines()])
    for (v, a), (H, L) in zip(pts, got):
        ref = wofz(v + 1j * a)
        assert abs(L - ref.imag) <= 1e-14 * abs(ref) + 1e-300, (v, a)
        bound = 1e-12 if abs(v) <= 2.0 else max(1e-12, 1e-14 * abs(v) / a)
        assert abs(H - ref.real) <= bound * abs(ref.real), (v, a, abs(H - ref.real) / abs(ref.real))


YDUMP = DUMP.replace('''  const int nu = c->nu_st, nl = c->nl_st, nO = c->nO;
  std::printf("%d %d %d %d\\n", nz, nO, nu, nl);
  for (int iz = 0; iz < nz; ++iz) std::printf("%.17g\\n", c->dnuD[iz]);
  for (double x : c->shift) std::printf("%.17g\\n", x);
  for (auto z : c->alpha) std::printf("%.17g %.17g\\n", z.real(), z.imag());
  for (auto z : c->beta) std::printf("%.17g %.17g\\n", z.real(), z.imag());
  for (auto z : c->amp) std::printf("%.17g %.17g\\n", z.real(), z.imag());''', '''  prd::LosTables L;
  const double mu = std::atof(argv[2]), chi = std::atof(argv[3]);
  prd::los_tables(c, mu, chi, L);
  const int nu = c->nu_st, nl = c->nl_st, nO = c->nO, nt = c->ntrip, ng = c->ngrp;
  std::printf("%d %d %d %d %d %d\\n", nz, nO, nu, nl, nt, ng);
  for (int t = 0; t < nt; ++t) std::printf("%d %d %d\\n", c->trip_k[t], c->trip_l[t], c->trip_lp[t]);
  for (double x : c->shift) std::printf("%.17g\\n", x);
  for (double x : L.theta) std::printf("%.17g\\n", x);
  for (double x : L.Y) std::printf("%.17g\\n", x);''').replace("#include <cstdio>", "#include <cstdio>\n#include <cstdlib>")


def test_rii_coefficients_rebuild_the_oracle_block(tmp_path):
    """S3+S4 regrouping: the library writes R_II between a line of sight and a
    grid direction as Re sum_t Y^t G_t over triples t = (k, k_l, k_l') (one
    coefficient matrix per triple, Eq. RQIIKKp with the amplitude products
    factorised), the oracle as the trace over upper-state pairs with
    alpha [G(k_u') + G(k_u)^*].  Y^t from los_tables, combined with the oracle's
    own tiles G_t, must rebuild the oracle's comoving block (R_III switched off
    by r_E = 0, so that beta = alpha), on magnetised Mg II physics."""
    import numpy as np
    from paper_2505_20968_gb300 import inputs
    from oracle.problem import Problem
    from oracle.geometry import unit_vector, scattering_angle
    cfg = inputs.mgii(n_z=3, n_core_each=4, n_wing=3, n_mu_half=1, n_chi=4, seed=29)
    atm = cfg["atm"]
    atm["r_el"] = np.zeros(3)
    atm["B_G"] = np.array([40.0, 700.0, 5.0])
    exe = _build_exe(tmp_path, "ydump", YDUMP)
    at, q = cfg["atom"], cfg["quad"]
    keys = ("z_km", "T_K", "xi_kms", "a", "eps", "r_el", "k_line", "W_T", "B_G", "thetaB", "chiB")
    lines = [f"{at['twoS']} {at['E_u_cm'][0]!r} {at['E_u_cm'][1]!r} {at['mass_amu']!r} {at['g_s']!r} {len(atm['z_km'])}"]
    lines += [" ".join(repr(float(x)) for x in np.asarray(atm[k], dtype=np.float64)) for k in keys]
    lines.append(" ".join(repr(float(x)) for x in np.asarray(atm["v_kms"], dtype=np.float64).ravel()))
    lines.append(f"{len(q['grid'])} {q['grid_kind']} {q['n_mu_half']} {q['n_chi']}")
    lines.append(" ".join(repr(float(x)) for x in q["grid"]))
    (tmp_path / "problem.txt").write_text("\n".join(lines) + "\n")
    mu, chi = 0.4, 2.2
    r = subprocess.run([str(exe), str(tmp_path / "problem.txt"), repr(mu), repr(chi)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    tok = r.stdout.split()
    nz, nO, nu, nl, nt, ng = map(int, tok[:6])
    pos = 6
    trip = np.array(tok[pos:pos + 3 * nt], dtype=int).reshape(nt, 3)
    pos += 3 * nt
    vals = np.array([float(s) for s in tok[pos:]])
    shift = vals[:nz * nu * nl].reshape(nz, nu, nl)
    theta = vals[nz * nu * nl:nz * nu * nl + nO]
    Y = vals[nz * nu * nl + nO:].reshape(nz, nO, ng + nt, 4, 4, 2)
    Y = Y[..., 0] + 1j * Y[..., 1]
    P = Problem(cfg, normalise=False)
    N = P.nN
    n_l = unit_vector(np.array([mu]), np.array([chi]))[0]
    for iz in range(nz):
        pl = np.argsort(shift[iz][:, 0], kind="stable")
        po = np.argsort(P.shift[iz][:, 0], kind="stable")
        to_oracle = dict(zip(pl, po))                      # library upper state -> oracle state
        amp = P.amplitudes(iz, mu, chi)
        for op in (1, 6):
            th = scattering_angle(n_l, P.nvec[op])
            assert abs(th - theta[op]) < 1e-12
            ref = P.block(iz, None, op, amp_o=amp, theta=th).reshape(N, 4, N, 4)
            rebuilt = np.zeros((N, 4, N, 4))
            for t, (k, l, lp) in enumerate(trip):
                ku = to_oracle[k]
                G = P.tile(iz, th, P.shift[iz][ku, l], P.shift[iz][ku, lp])
                rebuilt += np.einsum("ij,nm->nimj", Y[iz, op, ng + t], G).real
            assert np.max(np.abs(rebuilt - ref)) < 1e-10 * np.max(np.abs(ref)), (iz, op)


PAR = r'''
#include <cstdio>
#include <cstdlib>
namespace prd { void delopar_weights(double dM, double dP, double* psi); }
int main(int argc, char** argv) {
  for (int i = 1; i + 1 < argc; i += 2) {
    double psi[3];
    prd::delopar_weights(std::atof(argv[i]), std::atof(argv[i + 1]), psi);
    std::printf("%.17g %.17g %.17g\n", psi[0], psi[1], psi[2]);
  }
  return 0;
}
'''


def test_host_delopar_weights_match_the_oracle(tmp_path):
    """DELOPAR's source weights (Sect. 3) of the library (power series of the
    moments int_0^d t^n e^{-t} dt below d = 0.5, closed forms above) against
    the oracle's (regularised incomplete gamma), from optically thin to thick
    steps and for downwind steps thinner and thicker than the current one:
    1e-12 of the largest weight."""
    import numpy as np
    from oracle.problem import delopar_coeffs
    exe = _build_exe(tmp_path, "par", PAR)
    pts = [(dM, dP) for dM in (1e-6, 3e-4, 0.02, 0.3, 0.49, 0.51, 1.7, 12.0, 300.0)
           for dP in (1e-5, 0.01, 0.5, 2.0, 50.0)]
    args = [repr(x) for dM, dP in pts for x in (dM, dP)]
    r = subprocess.run([str(exe)] + args, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0
    got = np.array([[float(s) for s in line.split()] for line in r.stdout.strip().splitlines()])
    for (dM, dP), g in zip(pts, got):
        want = np.array(delopar_coeffs(dM, dP), dtype=float)
        assert np.max(np.abs(g - want)) <= 1e-12 * np.max(np.abs(want)), (dM, dP, g, want)
