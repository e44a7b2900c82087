// Host-side setup (step S0): grids, scattering-angle classes, Paschen-Back
// states, branching ratios, polarisation amplitudes, propagation matrices,
// DELO-linear weights, redistribution coefficients and interpolation tables.
// Everything here runs once per prd_setup in FP64; the per-apply work is in
// the CUDA kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include "prd_internal.h"

namespace prd {

namespace {

// Stokes "Pauli" matrices: I = Tr(rho), Q = Tr(s_z rho), U = Tr(s_x rho),
// V = Tr(s_y rho), rho the coherency matrix of (E_a, E_b).
const cplx kSig[4][2][2] = {
    {{1.0, 0.0}, {0.0, 1.0}},
    {{1.0, 0.0}, {0.0, -1.0}},
    {{0.0, 1.0}, {1.0, 0.0}},
    {{0.0, cplx(0.0, -1.0)}, {cplx(0.0, 1.0), 0.0}}};

struct States {
  std::vector<double> E;          // upper energies rel. nu0 [Hz]
  std::vector<int> M2;            // 2*M of each upper state
  std::vector<double> D;          // [3 (q=-1,0,1)][ku][kl]
  std::vector<double> El;         // lower energies [Hz]
  std::vector<int> ml2;           // 2*M of lower states
};

// Paschen-Back upper term H = zeta L.S + nu_L (L_z + g_s S_z), diagonalised in
// blocks of fixed M = M_L + M_S (H conserves M): blocks are 1x1 or 2x2.
States pb_states(const prd_atom& at, double nu0, double B_gauss) {
  States s;
  const double nuL = kMuBoverH * kGauss * B_gauss;
  const double gs = at.g_s;
  if (at.twoS == 0) {
    const double E0 = at.E_u_cm[0] * kCmToHz - nu0;
    for (int ml = -1; ml <= 1; ++ml) {
      s.E.push_back(E0 + nuL * ml);
      s.M2.push_back(2 * ml);
    }
    s.D.assign(3 * 3 * 1, 0.0);
    // D[q][ku][kl]: <ku=ml| d_q |0> = delta(ml, q)
    for (int q = 0; q < 3; ++q) s.D[q * 3 + q] = 1.0;
    s.El = {0.0};
    s.ml2 = {0};
    return s;
  }
  const double zeta = (at.E_u_cm[1] - at.E_u_cm[0]) * kCmToHz / 1.5;
  const double Ec = at.E_u_cm[0] * kCmToHz + zeta - nu0;
  // uncoupled basis index b = (ml+1)*2 + (ms2+1)/2, ms2 = 2 M_S
  auto diag = [&](int ml, int ms2) { return Ec + zeta * ml * 0.5 * ms2 + nuL * (ml + gs * 0.5 * ms2); };
  std::vector<double> V;   // eigenvectors in uncoupled basis, [b][ku]
  std::vector<double> E;
  std::vector<int> M2;
  std::vector<std::vector<double>> vecs;
  // M = +3/2: |1,+>
  {
    std::vector<double> v(6, 0.0);
    v[(1 + 1) * 2 + 1] = 1.0;
    E.push_back(diag(1, 1));
    M2.push_back(3);
    vecs.push_back(v);
  }
  // M = -3/2: |-1,->
  {
    std::vector<double> v(6, 0.0);
    v[(-1 + 1) * 2 + 0] = 1.0;
    E.push_back(diag(-1, -1));
    M2.push_back(-3);
    vecs.push_back(v);
  }
  // M = +1/2: {|1,->, |0,+>} ; M = -1/2: {|0,->, |-1,+>}
  const int blocks[2][2][2] = {{{1, -1}, {0, 1}}, {{0, -1}, {-1, 1}}};
  for (int bI = 0; bI < 2; ++bI) {
    const int ml_a = blocks[bI][0][0], ms_a = blocks[bI][0][1];
    const int ml_b = blocks[bI][1][0], ms_b = blocks[bI][1][1];
    const double haa = diag(ml_a, ms_a), hbb = diag(ml_b, ms_b);
    // off-diagonal (zeta/2)(L+S- + L-S+): <ml_a, ms_a| ... |ml_b, ms_b>
    // ml_a = ml_b + 1, ms_a = ms_b - 1 (L+ S-):  sqrt(2 - ml_b(ml_b+1)) * 1
    const double hab = 0.5 * zeta * std::sqrt(2.0 - ml_b * (ml_b + 1.0)) * 1.0;
    const double tr = 0.5 * (haa + hbb), df = 0.5 * (haa - hbb);
    const double r = std::sqrt(df * df + hab * hab);
    const double e1 = tr - r, e2 = tr + r;
    // eigenvector for e: (hab, e - haa) or (e - hbb, hab)
    for (double e : {e1, e2}) {
      double va = hab, vb = e - haa;
      if (std::fabs(va) + std::fabs(vb) < 1e-300 * (1 + std::fabs(e))) {
        va = e - hbb;
        vb = hab;
      }
      if (std::fabs(hab) == 0.0) {   // uncoupled: pick the basis vector with this energy
        if (std::fabs(e - haa) <= std::fabs(e - hbb)) { va = 1; vb = 0; } else { va = 0; vb = 1; }
      }
      const double nrm = std::sqrt(va * va + vb * vb);
      std::vector<double> v(6, 0.0);
      v[(ml_a + 1) * 2 + (ms_a + 1) / 2] = va / nrm;
      v[(ml_b + 1) * 2 + (ms_b + 1) / 2] = vb / nrm;
      E.push_back(e);
      M2.push_back(2 * ml_a + ms_a);
      vecs.push_back(v);
    }
    if (r == 0.0 && std::fabs(hab) == 0.0 && haa == hbb) {
      // exactly degenerate and uncoupled: make sure the two vectors differ
      auto& v1 = vecs[vecs.size() - 2];
      auto& v2 = vecs[vecs.size() - 1];
      std::fill(v1.begin(), v1.end(), 0.0);
      std::fill(v2.begin(), v2.end(), 0.0);
      v1[(ml_a + 1) * 2 + (ms_a + 1) / 2] = 1.0;
      v2[(ml_b + 1) * 2 + (ms_b + 1) / 2] = 1.0;
    }
  }
  const int nu = 6, nl = 2;
  s.E = E;
  s.M2 = M2;
  s.D.assign(3 * nu * nl, 0.0);
  for (int ku = 0; ku < nu; ++ku)
    for (int kl = 0; kl < nl; ++kl) {
      const int ms_l = kl == 0 ? -1 : 1;
      for (int q = -1; q <= 1; ++q) s.D[((q + 1) * nu + ku) * nl + kl] = vecs[ku][(q + 1) * 2 + (ms_l + 1) / 2];
    }
  s.El = {nuL * gs * -0.5, nuL * gs * 0.5};
  s.ml2 = {-1, 1};
  return s;
}

}  // namespace

size_t nvec(const Ctx* c) { return (size_t)4 * c->nz * c->nO * c->nnu; }

void dir_amplitudes(const Ctx* c, int iz, double m, double ch, cplx* out) {
  const int nu_ = c->nu_st, nl = c->nl_st;
  const double isq2 = 1.0 / std::sqrt(2.0);
  const cplx eqc[3][3] = {{isq2, cplx(0, isq2), 0.0}, {0.0, 0.0, 1.0}, {-isq2, cplx(0, isq2), 0.0}};
  const double* R = &c->Rmag[(size_t)iz * 9];
  const double sn = std::sqrt(std::max(0.0, 1.0 - m * m));
  const double e[2][3] = {{-std::sin(ch), std::cos(ch), 0.0}, {m * std::cos(ch), m * std::sin(ch), -sn}};
  for (int al = 0; al < 2; ++al) {
    double eB[3];
    for (int r = 0; r < 3; ++r) eB[r] = R[r * 3] * e[al][0] + R[r * 3 + 1] * e[al][1] + R[r * 3 + 2] * e[al][2];
    cplx proj[3];
    for (int q = 0; q < 3; ++q) proj[q] = eqc[q][0] * eB[0] + eqc[q][1] * eB[1] + eqc[q][2] * eB[2];
    for (int ku = 0; ku < nu_; ++ku)
      for (int l = 0; l < nl; ++l) {
        cplx sum = 0.0;
        for (int q = 0; q < 3; ++q) sum += proj[q] * c->Dmat[(size_t)iz * 3 * nu_ * nl + ((size_t)q * nu_ + ku) * nl + l];
        out[((size_t)al * nu_ + ku) * nl + l] = sum;
      }
  }
}

int build_host_tables(Ctx* c) {
  const int nz = c->nz, N = c->nnu;
  // ---------------- angular grid (Sect. 4.2)
  std::vector<double> mu, wmu;
  if (c->mu_rule == PRD_MU_GL_FULL) {
    gauss_legendre(2 * c->n_mu_half, mu, wmu);
  } else {
    std::vector<double> x, w;
    gauss_legendre(c->n_mu_half, x, w);
    for (int i = c->n_mu_half - 1; i >= 0; --i) { mu.push_back(-0.5 * (x[i] + 1.0)); wmu.push_back(0.5 * w[i]); }
    for (int i = 0; i < c->n_mu_half; ++i) { mu.push_back(0.5 * (x[i] + 1.0)); wmu.push_back(0.5 * w[i]); }
  }
  const int nmu = (int)mu.size();
  c->nO = nmu * c->n_chi;
  const int nO = c->nO;
  c->mu.resize(nO);
  c->chi.resize(nO);
  c->wang.resize(nO);
  for (int i = 0; i < nmu; ++i)
    for (int k = 0; k < c->n_chi; ++k) {
      c->mu[i * c->n_chi + k] = mu[i];
      c->chi[i * c->n_chi + k] = 2.0 * kPi * k / c->n_chi;
      c->wang[i * c->n_chi + k] = 0.5 * wmu[i] / c->n_chi;
    }
  std::vector<double> nv(3 * nO);
  for (int o = 0; o < nO; ++o) {
    const double s = std::sqrt(std::max(0.0, 1.0 - c->mu[o] * c->mu[o]));
    nv[3 * o] = s * std::cos(c->chi[o]);
    nv[3 * o + 1] = s * std::sin(c->chi[o]);
    nv[3 * o + 2] = c->mu[o];
  }
  // ---------------- scattering-angle classes
  std::vector<double> th(nO * nO);
  for (int o = 0; o < nO; ++o)
    for (int p = 0; p < nO; ++p) {
      double dm = 0, ds = 0;
      for (int d = 0; d < 3; ++d) {
        dm += (nv[3 * o + d] - nv[3 * p + d]) * (nv[3 * o + d] - nv[3 * p + d]);
        ds += (nv[3 * o + d] + nv[3 * p + d]) * (nv[3 * o + d] + nv[3 * p + d]);
      }
      th[o * nO + p] = 2.0 * std::atan2(std::sqrt(dm), std::sqrt(ds));
    }
  std::vector<double> sorted(th);
  std::sort(sorted.begin(), sorted.end());
  c->theta.clear();
  c->theta.push_back(sorted[0]);
  for (double v : sorted)
    if (v - c->theta.back() > 1e-10) c->theta.push_back(v);
  for (auto& v : c->theta) {
    if (std::fabs(v) < 1e-10) v = 0.0;
    if (std::fabs(v - kPi) < 1e-10) v = kPi;
  }
  if (c->mode == PRD_MODE_AA) {
    // one class: the angle-averaged kernel does not depend on Theta
    c->theta.assign(1, -1.0);
  }
  c->ncls = (int)c->theta.size();
  c->cls.assign(nO * nO, 0);
  for (int i = 0; i < nO * nO; ++i) {
    if (c->mode == PRD_MODE_AA) { c->cls[i] = 0; continue; }
    int best = 0;
    for (int k = 1; k < c->ncls; ++k)
      if (std::fabs(th[i] - c->theta[k]) < std::fabs(th[i] - c->theta[best])) best = k;
    c->cls[i] = best;
  }
  // CSR: class -> out dirs -> in dirs
  c->cout_ptr.assign(c->ncls + 1, 0);
  c->cout_dir.clear();
  c->pair_ptr.assign(1, 0);
  c->pair_in.clear();
  c->max_cout = 0;
  for (int k = 0; k < c->ncls; ++k) {
    int cnt = 0;
    for (int o = 0; o < nO; ++o) {
      int np = 0;
      for (int p = 0; p < nO; ++p)
        if (c->cls[o * nO + p] == k) { c->pair_in.push_back(p); ++np; }
      if (np) {
        c->cout_dir.push_back(o);
        c->pair_ptr.push_back((int)c->pair_in.size());
        ++cnt;
      }
    }
    c->cout_ptr[k + 1] = c->cout_ptr[k] + cnt;
    c->max_cout = std::max(c->max_cout, cnt);
  }
  c->npairs = (int)c->pair_in.size();
  // AA Theta rule: composite GL on [0, pi/2] and [pi/2, pi]
  if (c->mode == PRD_MODE_AA) {
    std::vector<double> x, w;
    gauss_legendre(kAAThetaNodes, x, w);
    c->aa_theta.clear();
    c->aa_w.clear();
    for (int h = 0; h < 2; ++h) {
      const double lo = h * 0.5 * kPi, hi = lo + 0.5 * kPi;
      for (int i = 0; i < kAAThetaNodes; ++i) {
        const double t = 0.5 * (hi - lo) * x[i] + 0.5 * (hi + lo);
        c->aa_theta.push_back(t);
        c->aa_w.push_back(0.5 * 0.5 * (hi - lo) * w[i] * std::sin(t));
      }
    }
  }

  // ---------------- frequencies, Doppler widths (Sect. 6.1)
  const prd_atom& at = c->atom;
  c->nu0 = at.nu0_hz != 0.0 ? at.nu0_hz
                            : (at.twoS == 0 ? at.E_u_cm[0] * kCmToHz
                                            : (2.0 * at.E_u_cm[0] + 4.0 * at.E_u_cm[1]) / 6.0 * kCmToHz);
  c->dnuD.resize(nz);
  c->vD.resize(nz);
  for (int iz = 0; iz < nz; ++iz) {
    const double xi = c->xi[iz] * 1e3;
    const double vd = std::sqrt(2.0 * kKB * c->T[iz] / (at.mass_amu * kAMU) + xi * xi);
    c->vD[iz] = vd / 1e3;
    c->dnuD[iz] = c->nu0 * vd / kC;
  }
  std::vector<double> nu(N);
  for (int n = 0; n < N; ++n)
    nu[n] = (c->grid_kind == PRD_GRID_LAMBDA) ? kC / (c->grid[n] * 1e-10) : c->nu0 - c->grid[n] * c->dnuD[0];
  c->u.resize((size_t)nz * N);
  for (int iz = 0; iz < nz; ++iz)
    for (int n = 0; n < N; ++n) c->u[(size_t)iz * N + n] = (c->nu0 - nu[n]) / c->dnuD[iz];
  for (int iz = 0; iz < nz; ++iz)
    for (int n = 1; n < N; ++n)
      if (!(c->u[(size_t)iz * N + n] > c->u[(size_t)iz * N + n - 1]))
        return fail(c, PRD_E_ARG, "frequency grid must be strictly ascending in reduced frequency");
  c->ub.resize((size_t)nz * nO);
  for (int iz = 0; iz < nz; ++iz)
    for (int o = 0; o < nO; ++o)
      c->ub[(size_t)iz * nO + o] =
          (c->v[3 * iz] * nv[3 * o] + c->v[3 * iz + 1] * nv[3 * o + 1] + c->v[3 * iz + 2] * nv[3 * o + 2]) / c->vD[iz];
  c->Q.resize((size_t)nz * N * N);
  for (int iz = 0; iz < nz; ++iz) natural_spline_Q(&c->u[(size_t)iz * N], N, &c->Q[(size_t)iz * N * N]);

  // ---------------- atom per height (Sect. 2.2, App. B)
  States s0 = pb_states(at, c->nu0, c->B[0]);
  c->nu_st = (int)s0.E.size();
  c->nl_st = (int)s0.El.size();
  const int nu_ = c->nu_st, nl = c->nl_st;
  // triples (k, kl, kl') allowed by the dipole selection rules |M_k - M_l| <= 1
  c->trip_k.clear(); c->trip_l.clear(); c->trip_lp.clear();
  for (int k = 0; k < nu_; ++k)
    for (int l = 0; l < nl; ++l)
      for (int lp = 0; lp < nl; ++lp)
        if (std::abs(s0.M2[k] - s0.ml2[l]) <= 2 && std::abs(s0.M2[k] - s0.ml2[lp]) <= 2) {
          c->trip_k.push_back(k);
          c->trip_l.push_back(l);
          c->trip_lp.push_back(lp);
        }
  c->ntrip = (int)c->trip_k.size();
  // group of each upper state: the J level whose B = 0 energy is closest
  {
    std::vector<int> grp_of(nu_, 0);
    c->ngrp = 1;
    if (at.twoS == 1) {
      c->ngrp = 2;
      const double E12 = at.E_u_cm[0] * kCmToHz - c->nu0, E32 = at.E_u_cm[1] * kCmToHz - c->nu0;
      States sb = pb_states(at, c->nu0, 0.0);
      for (int k = 0; k < nu_; ++k) grp_of[k] = std::fabs(sb.E[k] - E12) <= std::fabs(sb.E[k] - E32) ? 0 : 1;
    }
    c->trip_grp.resize(c->ntrip);
    for (int t = 0; t < c->ntrip; ++t) c->trip_grp[t] = grp_of[c->trip_k[t]];
  }
  c->shift.assign((size_t)nz * nu_ * nl, 0.0);
  c->alpha.assign((size_t)nz * nu_ * nu_, 0.0);
  c->beta.assign((size_t)nz * nu_ * nu_, 0.0);
  c->amp.assign((size_t)nz * nO * 2 * nu_ * nl, 0.0);
  c->Dmat.assign((size_t)nz * 3 * nu_ * nl, 0.0);
  c->Rmag.assign((size_t)nz * 9, 0.0);
  const double isq2 = 1.0 / std::sqrt(2.0);
  // spherical unit vectors e_q (q=-1,0,1) in the magnetic frame, conjugated
  const cplx eqc[3][3] = {{isq2, cplx(0, isq2), 0.0}, {0.0, 0.0, 1.0}, {-isq2, cplx(0, isq2), 0.0}};
  for (int iz = 0; iz < nz; ++iz) {
    States st = pb_states(at, c->nu0, c->B[iz]);
    for (int ku = 0; ku < nu_; ++ku)
      for (int l = 0; l < nl; ++l) c->shift[((size_t)iz * nu_ + ku) * nl + l] = (st.E[ku] - st.El[l]) / c->dnuD[iz];
    const double Gt = 4.0 * kPi * c->dnuD[iz] * c->a[iz];
    const double a0 = (1.0 - c->eps[iz]) * (1.0 - c->rE[iz]);
    const double b0 = 1.0 - c->eps[iz];
    for (int ku = 0; ku < nu_; ++ku)
      for (int kv = 0; kv < nu_; ++kv) {
        const double dnu = st.E[ku] - st.E[kv];
        c->alpha[((size_t)iz * nu_ + ku) * nu_ + kv] = a0 / cplx(1.0, 2.0 * kPi * dnu / Gt);
        c->beta[((size_t)iz * nu_ + ku) * nu_ + kv] = b0 / cplx(1.0, 2.0 * kPi * dnu / (Gt * (1.0 - c->rE[iz])));
      }
    // magnetic frame rows
    const double tb = c->thB[iz], cb = c->chB[iz];
    const double R[3][3] = {{std::cos(tb) * std::cos(cb), std::cos(tb) * std::sin(cb), -std::sin(tb)},
                            {-std::sin(cb), std::cos(cb), 0.0},
                            {std::sin(tb) * std::cos(cb), std::sin(tb) * std::sin(cb), std::cos(tb)}};
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) c->Rmag[(size_t)iz * 9 + r * 3 + q] = R[r][q];
    for (size_t i = 0; i < st.D.size(); ++i) c->Dmat[(size_t)iz * 3 * nu_ * nl + i] = st.D[i];
    for (int o = 0; o < nO; ++o) {
      const double m = c->mu[o], ch = c->chi[o];
      const double sn = std::sqrt(std::max(0.0, 1.0 - m * m));
      const double e[2][3] = {{-std::sin(ch), std::cos(ch), 0.0}, {m * std::cos(ch), m * std::sin(ch), -sn}};
      for (int al = 0; al < 2; ++al) {
        double eB[3];
        for (int r = 0; r < 3; ++r) eB[r] = R[r][0] * e[al][0] + R[r][1] * e[al][1] + R[r][2] * e[al][2];
        cplx proj[3];
        for (int q = 0; q < 3; ++q) proj[q] = eqc[q][0] * eB[0] + eqc[q][1] * eB[1] + eqc[q][2] * eB[2];
        for (int ku = 0; ku < nu_; ++ku)
          for (int l = 0; l < nl; ++l) {
            cplx s = 0.0;
            for (int q = 0; q < 3; ++q) s += proj[q] * st.D[((size_t)q * nu_ + ku) * nl + l];
            c->amp[((((size_t)iz * nO + o) * 2 + al) * nu_ + ku) * nl + l] = s;
          }
      }
    }
  }
  return PRD_OK;
}

}  // namespace prd
