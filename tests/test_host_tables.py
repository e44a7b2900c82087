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
