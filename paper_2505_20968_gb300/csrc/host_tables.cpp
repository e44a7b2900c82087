// Host-side per-height tables uploaded at prd_setup: propagation matrices and
// DELO-linear weights (Sect. 3), thermal emissivity (Sect. 2.3), the complex
// coefficients of the R_II contraction (Eq. RQIIKKp, phase part), the
// separable R_III factors (Eq. RIIIQKKp) and the spline tables of the frame
// changes (Sect. 4.1).  FP64 on the host, stored in the ctx precision.
#include <cmath>
#include <cstring>
#include <vector>
#include "prd_internal.h"

namespace prd {

namespace {

const cplx kI(0.0, 1.0);
// sigma matrices: I, Q (s_z), U (s_x), V (s_y)
inline cplx sig(int i, int a, int b) {
  switch (i) {
    case 0: return a == b ? 1.0 : 0.0;
    case 1: return a == b ? (a == 0 ? 1.0 : -1.0) : 0.0;
    case 2: return a != b ? 1.0 : 0.0;
    default: return a == b ? 0.0 : (a == 0 ? -kI : kI);
  }
}

template <typename T>
int upload_conv(Ctx* c, DBuf& b, const std::vector<double>& v) {
  std::vector<T> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = (T)v[i];
  return upload(c, b, h.data(), h.size() * sizeof(T));
}

int upload_T(Ctx* c, DBuf& b, const std::vector<double>& v) {
  return c->prec == PRD_FP64 ? upload_conv<double>(c, b, v) : upload_conv<float>(c, b, v);
}

// DELO-linear weights (exp(-d), alpha, beta) with a series for small d.
void delo(double d, double* e, double* al, double* be) {
  *e = std::exp(-d);
  if (d < 2e-3) {
    const double d2 = d * d, d3 = d2 * d, d4 = d3 * d, d5 = d4 * d;
    *be = d / 2 - d2 / 6 + d3 / 24 - d4 / 120 + d5 / 720;
    *al = d / 2 - d2 / 3 + d3 / 8 - d4 / 30 + d5 / 144;
  } else {
    const double w0 = -std::expm1(-d);
    *be = 1.0 - w0 / d;
    *al = w0 - *be;
  }
}

}  // namespace

// DELOPAR source weights for a step of optical thickness dM (upwind point at
// t = dM, current point at t = 0) and the next step downwind of thickness dP
// (downwind point at t = -dP): psi_j = int_0^dM e^{-t} L_j(t) dt with L_j the
// quadratic Lagrange basis through the three points.  The moments
// J_n = int_0^dM t^n e^{-t} dt come from their power series for small dM
// (alternating, terms dM^(n+1+k) / (k! (n+1+k))) and in closed form otherwise.
void delopar_weights(double dM, double dP, double* psi) {
  double J0, J1, J2;
  if (dM < 0.5) {
    J0 = J1 = J2 = 0.0;
    double term = 1.0;                     // (-1)^k dM^k / k!
    for (int k = 0; k < 30; ++k) {
      J0 += term * std::pow(dM, 1) / (1 + k);
      J1 += term * std::pow(dM, 2) / (2 + k);
      J2 += term * std::pow(dM, 3) / (3 + k);
      term *= -dM / (k + 1);
    }
  } else {
    const double e = std::exp(-dM);
    J0 = 1.0 - e;
    J1 = 1.0 - e * (1.0 + dM);
    J2 = 2.0 - e * (dM * dM + 2.0 * dM + 2.0);
  }
  psi[0] = (J2 + dP * J1) / (dM * (dM + dP));
  psi[1] = (dM * dP * J0 - J2 - (dP - dM) * J1) / (dM * dP);
  psi[2] = (J2 - dM * J1) / (dP * (dM + dP));
}

// Dipole phase matrix of coherent continuum scattering (App. A: the sum over
// K <= 2 of (-1)^Q T^K_Q(o) T^K_-Q(o') with every W_K = 1): the field scattered
// into o is the projection of the incident one, J_ab = e_a(o) . e_b(o') in the
// polarisation bases of the two directions (e_a parallel to the limb), and
// P_ij = 3/4 Tr(sig_i J sig_j J^T), normalised to oint P_00 dOmega'/4pi = 1.
void dipole_phase(double mu_o, double chi_o, double mu_p, double chi_p, double* P) {
  auto basis = [](double mu, double chi, double e[2][3]) {
    const double s = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
    e[0][0] = -std::sin(chi); e[0][1] = std::cos(chi); e[0][2] = 0.0;
    e[1][0] = mu * std::cos(chi); e[1][1] = mu * std::sin(chi); e[1][2] = -s;
  };
  double eo[2][3], ep[2][3], J[2][2];
  basis(mu_o, chi_o, eo);
  basis(mu_p, chi_p, ep);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) J[a][b] = eo[a][0] * ep[b][0] + eo[a][1] * ep[b][1] + eo[a][2] * ep[b][2];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cplx tr = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int cc = 0; cc < 2; ++cc)
            for (int d = 0; d < 2; ++d) tr += sig(i, a, b) * J[b][cc] * sig(j, cc, d) * J[a][d];
      P[i * 4 + j] = 0.75 * tr.real();
    }
}

// Outgoing factor O_i(o; ku, kv, kl') = sum_ab a_b(kv,kl') sig_i[b][a] conj(a_a(ku,kl'))
// Incoming factor I_j(o'; ku, kv, kl) = sum_gd conj(a_d(kv,kl)) sig_j[g][d] a_g(ku,kl)
static void phase_factors_amp(const Ctx* c, const cplx* A, std::vector<cplx>& O, std::vector<cplx>& I) {
  const int nu_ = c->nu_st, nl = c->nl_st;
  O.assign((size_t)nu_ * nu_ * nl * 4, 0.0);
  I.assign((size_t)nu_ * nu_ * nl * 4, 0.0);
  auto amp = [&](int al, int ku, int kl) { return A[((size_t)al * nu_ + ku) * nl + kl]; };
  for (int ku = 0; ku < nu_; ++ku)
    for (int kv = 0; kv < nu_; ++kv)
      for (int l = 0; l < nl; ++l)
        for (int s = 0; s < 4; ++s) {
          cplx so = 0.0, si = 0.0;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
              so += amp(b, kv, l) * sig(s, b, a) * std::conj(amp(a, ku, l));
              si += std::conj(amp(b, kv, l)) * sig(s, a, b) * amp(a, ku, l);
            }
          O[(((size_t)ku * nu_ + kv) * nl + l) * 4 + s] = so;
          I[(((size_t)ku * nu_ + kv) * nl + l) * 4 + s] = si;
        }
}

static void phase_factors(const Ctx* c, int iz, int o, std::vector<cplx>& O, std::vector<cplx>& I) {
  phase_factors_amp(c, &c->amp[(((size_t)iz * c->nO + o) * 2) * c->nu_st * c->nl_st], O, I);
}

// propagation matrix K (4x4) for amplitudes A at shift ub and reduced frequency un
static void kmatrix(const Ctx* c, int iz, const cplx* A, double ub, double un, double K[4][4]) {
  const int nu_ = c->nu_st, nl = c->nl_st;
  const double S2 = (c->atom.twoS == 1) ? 2.0 : 1.0;
  cplx kap[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int ku = 0; ku < nu_; ++ku)
    for (int l = 0; l < nl; ++l) {
      const double x = un + ub + c->shift[((size_t)iz * nu_ + ku) * nl + l];
      const cplx w = std::conj(faddeeva_host(cplx(x, c->a[iz])));
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          kap[a][b] += std::conj(A[((size_t)a * nu_ + ku) * nl + l]) * A[((size_t)b * nu_ + ku) * nl + l] * w;
    }
  const double norm = c->k[iz] / (2.0 * kSqrtPi * S2);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cplx tr = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int d = 0; d < 2; ++d) {
            tr += sig(i, a, b) * kap[b][d] * norm * sig(j, d, a);
            tr += sig(i, a, b) * sig(j, b, d) * std::conj(kap[a][d] * norm);
          }
      K[i][j] = 0.5 * tr.real();
    }
}

void los_tables(const Ctx* c, double mu, double chi, LosTables& L) {
  const int nz = c->nz, nO = c->nO, N = c->nnu, nu_ = c->nu_st, nl = c->nl_st, nt = c->ntrip, ng = c->ngrp;
  const int nti = c->ntile(), nuv = nu_ * nu_;
  const double S2 = (c->atom.twoS == 1) ? 2.0 : 1.0;
  const double c2 = 3.0 / (4.0 * kPi * S2);
  const double sn = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  const double nl_[3] = {sn * std::cos(chi), sn * std::sin(chi), mu};
  L.theta.assign(nO, 0.0);
  for (int op = 0; op < nO; ++op) {
    const double so = std::sqrt(std::max(0.0, 1.0 - c->mu[op] * c->mu[op]));
    const double np_[3] = {so * std::cos(c->chi[op]), so * std::sin(c->chi[op]), c->mu[op]};
    double dm = 0, ds = 0;
    for (int d = 0; d < 3; ++d) {
      dm += (nl_[d] - np_[d]) * (nl_[d] - np_[d]);
      ds += (nl_[d] + np_[d]) * (nl_[d] + np_[d]);
    }
    double th = 2.0 * std::atan2(std::sqrt(dm), std::sqrt(ds));
    if (th < 1e-10) th = 0.0;
    if (std::fabs(th - kPi) < 1e-10) th = kPi;
    L.theta[op] = c->mode == PRD_MODE_AA ? -1.0 : th;
  }
  L.Y.assign((size_t)nz * nO * nti * 32, 0.0);
  L.rout.assign((size_t)nz * nuv * nl * 8, 0.0);
  L.kt.assign((size_t)nz * N * 10, 0.0);
  L.epsth.assign((size_t)nz * N * 4, 0.0);
  L.kidx.assign((size_t)nz * N, 0);
  L.tt.assign((size_t)nz * N, 0.0);
  L.eta_line.assign((size_t)nz * N, 0.0);
  L.cont_pw.assign((size_t)nO * 16, 0.0);
  if (c->has_cont())
    for (int op = 0; op < nO; ++op) {
      dipole_phase(mu, chi, c->mu[op], c->chi[op], &L.cont_pw[(size_t)op * 16]);
      for (int e = 0; e < 16; ++e) L.cont_pw[(size_t)op * 16 + e] *= c->wang[op];
    }
  std::vector<double> eta((size_t)nz * N);
  for (int iz = 0; iz < nz; ++iz) {
    std::vector<cplx> A((size_t)2 * nu_ * nl);
    dir_amplitudes(c, iz, mu, chi, A.data());
    std::vector<cplx> O, Id, Oo, Io;
    phase_factors_amp(c, A.data(), O, Id);
    const cplx* al = &c->alpha[(size_t)iz * nu_ * nu_];
    for (int op = 0; op < nO; ++op) {
      phase_factors(c, iz, op, Oo, Io);
      const double fac = c2 * c->k[iz] * c->wang[op];
      for (int t = 0; t < nt; ++t) {
        const int k = c->trip_k[t], l = c->trip_l[t], lp = c->trip_lp[t];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) {
            cplx y = 0.0;
            for (int ku = 0; ku < nu_; ++ku)
              y += O[(((size_t)ku * nu_ + k) * nl + lp) * 4 + i] * Io[(((size_t)ku * nu_ + k) * nl + l) * 4 + j] *
                   al[(size_t)ku * nu_ + k];
            y *= fac;
            const size_t idx = ((((size_t)iz * nO + op) * nti + ng + t) * 16 + i * 4 + j) * 2;
            L.Y[idx] = y.real();
            L.Y[idx + 1] = y.imag();
            const size_t ig = ((((size_t)iz * nO + op) * nti + c->trip_grp[t]) * 16 + i * 4 + j) * 2;
            L.Y[ig] += y.real();
            L.Y[ig + 1] += y.imag();
          }
      }
    }
    for (int q = 0; q < nuv * nl; ++q)
      for (int s = 0; s < 4; ++s) {
        L.rout[(((size_t)iz * nuv * nl + q) * 4 + s) * 2] = O[(size_t)q * 4 + s].real();
        L.rout[(((size_t)iz * nuv * nl + q) * 4 + s) * 2 + 1] = O[(size_t)q * 4 + s].imag();
      }
    const double ub = (c->v[3 * iz] * nl_[0] + c->v[3 * iz + 1] * nl_[1] + c->v[3 * iz + 2] * nl_[2]) / c->vD[iz];
    const double* u = &c->u[(size_t)iz * N];
    for (int n = 0; n < N; ++n) {
      double K[4][4];
      kmatrix(c, iz, A.data(), ub, u[n], K);
      L.eta_line[(size_t)iz * N + n] = K[0][0];
      for (int s = 0; s < 4; ++s) L.epsth[((size_t)iz * N + n) * 4 + s] = c->eps[iz] * c->WT[iz] * K[s][0];
      if (c->has_cont()) {
        const size_t q = (size_t)iz * N + n;
        for (int s = 0; s < 4; ++s) K[s][s] += c->kapc[q] + c->sigc[q];
        L.epsth[q * 4] += c->epsc[q];
      }
      const double e1 = K[0][0];
      L.eta_line[(size_t)iz * N + n] /= e1;   // the line's share of eta_I
      double* t = &L.kt[((size_t)iz * N + n) * 10];
      t[0] = K[0][1] / e1; t[1] = K[0][2] / e1; t[2] = K[0][3] / e1;
      t[3] = K[1][2] / e1; t[4] = K[1][3] / e1; t[5] = K[2][3] / e1;
      t[6] = 1.0 / e1;
      eta[(size_t)iz * N + n] = e1;
      const double x = u[n] + ub;
      int kk;
      double tv = 0.0;
      if (x <= u[0]) kk = -1;
      else if (x >= u[N - 1]) kk = N - 1;
      else {
        int lo = 0, hi = N - 1;
        while (hi - lo > 1) { const int md = (lo + hi) / 2; if (u[md] <= x) lo = md; else hi = md; }
        kk = lo;
        tv = (x - u[kk]) / (u[kk + 1] - u[kk]);
      }
      L.kidx[(size_t)iz * N + n] = kk;
      L.tt[(size_t)iz * N + n] = tv;
    }
  }
  // DELO weights along the line of sight (upward, mu > 0), and DELOPAR's
  L.par.assign((size_t)nz * N * 3, 0.0);
  auto dtau = [&](int n, int p) {
    return 0.5 * (eta[(size_t)(p - 1) * N + n] + eta[(size_t)p * N + n]) * std::fabs(c->z[p] - c->z[p - 1]) / mu;
  };
  for (int n = 0; n < N; ++n)
    for (int p = 1; p < nz; ++p) {
      const double d = dtau(n, p);
      double e, a, b;
      delo(d, &e, &a, &b);
      L.kt[((size_t)p * N + n) * 10 + 7] = e;
      L.kt[((size_t)p * N + n) * 10 + 8] = a;
      L.kt[((size_t)p * N + n) * 10 + 9] = b;
      double* ps = &L.par[((size_t)p * N + n) * 3];
      if (p + 1 < nz) delopar_weights(d, dtau(n, p + 1), ps);
      else { ps[0] = a; ps[1] = b; ps[2] = 0.0; }
    }
}

int build_device_tables(Ctx* c) {
  const int nz = c->nz, nO = c->nO, N = c->nnu, nu_ = c->nu_st, nl = c->nl_st;
  const double S2 = (c->atom.twoS == 1) ? 2.0 : 1.0;
  const size_t npt = (size_t)nz * nO * N;
  std::vector<double> kt(npt * 10), epsth(npt * 4), eta(npt), etal(npt);
  // ---- propagation matrix from the forward-scattering amplitude
#pragma omp parallel for schedule(dynamic)
  for (int iz = 0; iz < nz; ++iz) {
    for (int o = 0; o < nO; ++o) {
      const cplx* A = &c->amp[(((size_t)iz * nO + o) * 2) * nu_ * nl];
      for (int n = 0; n < N; ++n) {
        cplx kap[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int ku = 0; ku < nu_; ++ku)
          for (int l = 0; l < nl; ++l) {
            const double x = c->u[(size_t)iz * N + n] + c->ub[(size_t)iz * nO + o] +
                             c->shift[((size_t)iz * nu_ + ku) * nl + l];
            const cplx w = std::conj(faddeeva_host(cplx(x, c->a[iz])));
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b)
                kap[a][b] += std::conj(A[((size_t)a * nu_ + ku) * nl + l]) * A[((size_t)b * nu_ + ku) * nl + l] * w;
          }
        const double norm = c->k[iz] / (2.0 * kSqrtPi * S2);
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) kap[a][b] *= norm;
        // K_ij = 1/2 Tr(sig_i kap sig_j + sig_i sig_j kap^+)
        double K[4][4];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) {
            cplx tr = 0.0;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b)
                for (int d = 0; d < 2; ++d)
                  for (int e = 0; e < 2; ++e) {
                    if (e != a) continue;
                    tr += sig(i, a, b) * kap[b][d] * sig(j, d, e);
                    tr += sig(i, a, b) * sig(j, b, d) * std::conj(kap[e][d]);
                  }
            K[i][j] = 0.5 * tr.real();
          }
        const size_t pt = ((size_t)iz * nO + o) * N + n;
        etal[pt] = K[0][0];
        for (int s = 0; s < 4; ++s) epsth[pt * 4 + s] = c->eps[iz] * c->WT[iz] * K[s][0];
        if (c->has_cont()) {
          // continuum (App. A): extinction on the diagonal, thermal emission in Stokes I
          const size_t q = (size_t)iz * N + n;
          for (int s = 0; s < 4; ++s) K[s][s] += c->kapc[q] + c->sigc[q];
          epsth[pt * 4] += c->epsc[q];
        }
        const double e1 = K[0][0];
        eta[pt] = e1;
        etal[pt] /= e1;   // the line's share of eta_I
        double* t = &kt[pt * 10];
        t[0] = K[0][1] / e1; t[1] = K[0][2] / e1; t[2] = K[0][3] / e1;
        t[3] = K[1][2] / e1; t[4] = K[1][3] / e1; t[5] = K[2][3] / e1;
        t[6] = 1.0 / e1;
      }
    }
  }
  // ---- DELO-linear weights of the step arriving at each point (Sect. 3), and the
  // DELOPAR source weights of the same step (linear at the last point of a ray)
  std::vector<double> par(npt * 3, 0.0);
  for (int o = 0; o < nO; ++o) {
    const bool up = c->mu[o] > 0;
    // optical thickness of the step arriving at the p-th point along the ray
    auto dtau = [&](int n, int p) {
      const int k1 = up ? p : nz - 1 - p, k0 = up ? p - 1 : nz - p;
      const size_t pt1 = ((size_t)k1 * nO + o) * N + n, pt0 = ((size_t)k0 * nO + o) * N + n;
      return 0.5 * (eta[pt0] + eta[pt1]) * std::fabs(c->z[k1] - c->z[k0]) / std::fabs(c->mu[o]);
    };
    for (int n = 0; n < N; ++n)
      for (int p = 0; p < nz; ++p) {
        const int k1 = up ? p : nz - 1 - p;
        const size_t pt1 = ((size_t)k1 * nO + o) * N + n;
        double e = 0, al = 0, be = 0;
        if (p > 0) {
          const double d = dtau(n, p);
          delo(d, &e, &al, &be);
          double* ps = &par[pt1 * 3];
          if (p + 1 < nz) delopar_weights(d, dtau(n, p + 1), ps);
          else { ps[0] = al; ps[1] = be; ps[2] = 0.0; }
        }
        kt[pt1 * 10 + 7] = e;
        kt[pt1 * 10 + 8] = al;
        kt[pt1 * 10 + 9] = be;
      }
  }
  int rc;
  // the DELOPAR weights stay FP64 in both modes: with uneven steps they are large and of
  // opposite sign, and their FP32 rounding would reach the FP64 residuals of the refinement
  if ((rc = upload_T(c, c->kt, kt)) || (rc = upload_T(c, c->epsth, epsth)) ||
      (rc = upload(c, c->par, par.data(), par.size() * 8)) ||
      (rc = upload(c, c->eta_line, etal.data(), npt * 8)))
    return rc;
  if (c->prec == PRD_FP32 &&
      ((rc = upload(c, c->kt64, kt.data(), kt.size() * 8)) || (rc = upload(c, c->epsth64, epsth.data(), epsth.size() * 8))))
    return rc;
  if (c->has_cont()) {
    std::vector<double> pw((size_t)nO * nO * 16);
    for (int o = 0; o < nO; ++o)
      for (int op = 0; op < nO; ++op) {
        double* P = &pw[((size_t)o * nO + op) * 16];
        dipole_phase(c->mu[o], c->chi[o], c->mu[op], c->chi[op], P);
        for (int e = 0; e < 16; ++e) P[e] *= c->wang[op];
      }
    if ((rc = upload(c, c->cont_pw, pw.data(), pw.size() * 8)) ||
        (rc = upload(c, c->cont_sig, c->sigc.data(), c->sigc.size() * 8)))
      return rc;
  }
  {
    std::vector<double> ones(npt, 1.0);
    if ((rc = upload(c, c->f, ones.data(), npt * 8))) return rc;   // FP64 in both modes
  }
  // ---- preconditioner scalar formal-solver tables: eta1 and DELO weights
  {
    std::vector<double> pe(npt), pd(npt * 3), lii(npt);
    for (size_t i = 0; i < npt; ++i) {
      pe[i] = eta[i];
      pd[3 * i] = kt[10 * i + 7];
      pd[3 * i + 1] = kt[10 * i + 8];
      pd[3 * i + 2] = kt[10 * i + 9];
      lii[i] = kt[10 * i + 9] / eta[i];     // local DELO weight of S = eps/eta1
    }
    if ((rc = upload_T(c, c->pc_eta, pe)) || (rc = upload_T(c, c->pc_delo, pd)) || (rc = upload_T(c, c->pc_lii, lii)))
      return rc;
    c->pc_lii_host = lii;
  }
  // ---- R_II contraction coefficients Y[z][pair][t][i][j] (complex)
  if (!c->lambda_only) {
    const double c2 = 3.0 / (4.0 * kPi * S2);
    const int nt = c->ntrip, nti = c->ntile(), ng = c->ngrp;
    std::vector<double> Y((size_t)nz * c->npairs * nti * 32, 0.0);
#pragma omp parallel for schedule(dynamic)
    for (int iz = 0; iz < nz; ++iz) {
      std::vector<std::vector<cplx>> O(nO), I(nO);
      for (int o = 0; o < nO; ++o) phase_factors(c, iz, o, O[o], I[o]);
      const cplx* al = &c->alpha[(size_t)iz * nu_ * nu_];
      int pidx = 0;
      for (int cl = 0; cl < c->ncls; ++cl)
        for (int e = c->cout_ptr[cl]; e < c->cout_ptr[cl + 1]; ++e) {
          const int o = c->cout_dir[e];
          for (int pp = c->pair_ptr[e]; pp < c->pair_ptr[e + 1]; ++pp, ++pidx) {
            const int op = c->pair_in[pp];
            const double fac = c2 * c->k[iz] * c->wang[op];
            for (int t = 0; t < nt; ++t) {
              const int k = c->trip_k[t], l = c->trip_l[t], lp = c->trip_lp[t];
              for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                  cplx y = 0.0;
                  for (int ku = 0; ku < nu_; ++ku)
                    y += O[o][(((size_t)ku * nu_ + k) * nl + lp) * 4 + i] *
                         I[op][(((size_t)ku * nu_ + k) * nl + l) * 4 + j] * al[(size_t)ku * nu_ + k];
                  y *= fac;
                  // deviation tile of triple t, and the group-mean tile of its J level
                  const size_t idx = ((((size_t)iz * c->npairs + pidx) * nti + ng + t) * 16 + i * 4 + j) * 2;
                  Y[idx] = y.real();
                  Y[idx + 1] = y.imag();
                  const size_t ig = ((((size_t)iz * c->npairs + pidx) * nti + c->trip_grp[t]) * 16 + i * 4 + j) * 2;
                  Y[ig] += y.real();
                  Y[ig + 1] += y.imag();
                }
            }
          }
        }
    }
    if ((rc = upload_T(c, c->Y, Y))) return rc;
    if (c->has64 && (rc = upload(c, c->Y64, Y.data(), Y.size() * 8))) return rc;
  }
  // ---- R_III separable factors
  if (!c->lambda_only) {
    const double c3 = 3.0 / (16.0 * kPi * S2);
    const int nuv = nu_ * nu_, nq = nuv * nl;
    std::vector<double> rin((size_t)nz * nO * nq * 4 * 2), rout((size_t)nz * nO * nuv * nl * 4 * 2),
        prof((size_t)nz * nuv * nl * N * 2), ab((size_t)nz * nuv * 2);
#pragma omp parallel for schedule(dynamic)
    for (int iz = 0; iz < nz; ++iz) {
      std::vector<cplx> O, I;
      for (int o = 0; o < nO; ++o) {
        phase_factors(c, iz, o, O, I);
        for (int q = 0; q < nq; ++q)
          for (int s = 0; s < 4; ++s) {
            const cplx v = I[(size_t)q * 4 + s] * c->wang[o];
            const size_t idx = ((((size_t)iz * nO + o) * nq + q) * 4 + s) * 2;
            rin[idx] = v.real();
            rin[idx + 1] = v.imag();
            const cplx w = O[(size_t)q * 4 + s];
            rout[idx] = w.real();
            rout[idx + 1] = w.imag();
          }
      }
      for (int ku = 0; ku < nu_; ++ku)
        for (int kv = 0; kv < nu_; ++kv) {
          const cplx b = c->k[iz] * c3 * (c->beta[((size_t)iz * nu_ + ku) * nu_ + kv] - c->alpha[((size_t)iz * nu_ + ku) * nu_ + kv]);
          const size_t ia = ((size_t)iz * nuv + ku * nu_ + kv) * 2;
          ab[ia] = b.real();
          ab[ia + 1] = b.imag();
          for (int lp = 0; lp < nl; ++lp)
            for (int n = 0; n < N; ++n) {
              const double un = c->u[(size_t)iz * N + n];
              const cplx p = faddeeva_host(cplx(un + c->shift[((size_t)iz * nu_ + kv) * nl + lp], c->a[iz])) +
                             std::conj(faddeeva_host(cplx(un + c->shift[((size_t)iz * nu_ + ku) * nl + lp], c->a[iz])));
              const size_t ip = ((((size_t)iz * nuv + ku * nu_ + kv) * nl + lp) * N + n) * 2;
              prof[ip] = p.real();
              prof[ip + 1] = p.imag();
            }
        }
    }
    if ((rc = upload_T(c, c->r3in, rin)) || (rc = upload_T(c, c->r3out, rout)) || (rc = upload_T(c, c->r3prof, prof)) ||
        (rc = upload_T(c, c->r3ab, ab)))
      return rc;
    if (c->has64 &&
        ((rc = upload(c, c->r3in64, rin.data(), rin.size() * 8)) || (rc = upload(c, c->r3out64, rout.data(), rout.size() * 8)) ||
         (rc = upload(c, c->r3prof64, prof.data(), prof.size() * 8)) || (rc = upload(c, c->r3ab64, ab.data(), ab.size() * 8))))
      return rc;
    if ((rc = dalloc(c, c->r3J, (size_t)nz * nuv * 2 * sizeof(double)))) return rc;
  }
  // ---- spline tables: per height h, Thomas factors (cp, den), grid
  {
    std::vector<double> sp((size_t)nz * 3 * N, 0.0), ug((size_t)nz * N);
    for (int iz = 0; iz < nz; ++iz) {
      const double* u = &c->u[(size_t)iz * N];
      double* h = &sp[(size_t)iz * 3 * N];
      double* cp = h + N;
      double* den = cp + N;
      for (int i = 0; i < N - 1; ++i) h[i] = u[i + 1] - u[i];
      const int m = N - 2;
      for (int r = 0; r < m; ++r) {
        const int i = r + 1;
        const double sub = (r > 0) ? h[i - 1] : 0.0;
        const double dn = 2.0 * (h[i - 1] + h[i]) - sub * (r > 0 ? cp[r - 1] : 0.0);
        den[r] = dn;
        cp[r] = (r < m - 1) ? h[i] / dn : 0.0;
      }
      for (int n = 0; n < N; ++n) ug[(size_t)iz * N + n] = u[n];
    }
    if ((rc = upload(c, c->sp, sp.data(), sp.size() * 8))) return rc;   // FP64 always
    if ((rc = upload_T(c, c->ugrid, ug))) return rc;
    // interpolation points: in  = u_n - u_b(o) (observer -> comoving, Sect. 4.1)
    //                        back = u_n + u_b(o) (comoving -> observer)
    std::vector<int> iin(npt), ibk(npt);
    std::vector<double> tin(npt), tbk(npt);
    for (int iz = 0; iz < nz; ++iz) {
      const double* u = &c->u[(size_t)iz * N];
      for (int o = 0; o < nO; ++o)
        for (int n = 0; n < N; ++n) {
          const size_t pt = ((size_t)iz * nO + o) * N + n;
          for (int dir = 0; dir < 2; ++dir) {
            const double x = u[n] + (dir == 0 ? -1.0 : 1.0) * c->ub[(size_t)iz * nO + o];
            int k;
            double t = 0.0;
            if (x <= u[0]) k = -1;
            else if (x >= u[N - 1]) k = N - 1;
            else {
              int lo = 0, hi = N - 1;
              while (hi - lo > 1) { const int md = (lo + hi) / 2; if (u[md] <= x) lo = md; else hi = md; }
              k = lo;
              t = (x - u[k]) / (u[k + 1] - u[k]);
            }
            (dir == 0 ? iin : ibk)[pt] = k;
            (dir == 0 ? tin : tbk)[pt] = t;
          }
        }
    }
    if ((rc = upload(c, c->iin, iin.data(), npt * 4)) || (rc = upload(c, c->ibk, ibk.data(), npt * 4)) ||
        (rc = upload(c, c->tin, tin.data(), npt * 8)) || (rc = upload(c, c->tbk, tbk.data(), npt * 8)))
      return rc;
  }
  // ---- class structure on the device
  {
    std::vector<int> all;
    all.insert(all.end(), c->cout_ptr.begin(), c->cout_ptr.end());
    all.insert(all.end(), c->cout_dir.begin(), c->cout_dir.end());
    all.insert(all.end(), c->pair_ptr.begin(), c->pair_ptr.end());
    all.insert(all.end(), c->pair_in.begin(), c->pair_in.end());
    if ((rc = upload(c, c->cls_dev, all.data(), all.size() * 4))) return rc;
  }
  // ---- scratch vectors
  const size_t vb = nvec(c) * c->esz;
  if ((rc = dalloc(c, c->scratch1, vb)) || (rc = dalloc(c, c->scratch2, vb)) || (rc = dalloc(c, c->scratch3, vb)))
    return rc;
  return PRD_OK;
}

}  // namespace prd
