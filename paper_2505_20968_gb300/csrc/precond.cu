// Physics-based preconditioner P = Id - Lambda* Sigma* (Sect. 5.2) with the
// block-diagonal inner preconditioner of App. F.
//
//  Sigma*: unpolarised, unmagnetised PRD-AA on Stokes I only (K = Q = 0):
//     eps_bar*(z,u) = k [alpha0 sum_g c_g r_AA(u'+s_g, u+s_g) + (beta0-alpha0) phi*(u) phi*(u')] J_bar(u')
//     with J_bar the angle average of the comoving I, r_AA = (1/pi) 1/2 int sin(Theta) Re F dTheta
//     (Eq. R_AA), c_g the J-level weights (2J+1)/(2(2L+1)) and phi* = sum_g c_g H(a,u+s_g)/sqrt(pi);
//     eps* = eps_bar* back in the observer frame.  Lambda*: scalar DELO-linear with eta_I.
//  P^-1 y: m_in Richardson sweeps x <- x + P_hat^-1 (y - P x) from x = 0, with
//     P_hat_i^-1 = Id + Lambda_ii Phi_bar_i (Id - A_i)^-1 Phi^Omega,  A_i = Phi^Omega Lambda_ii Phi_bar_i
//     (App. F, without the frame-change interpolations inside P_hat).
//  Q, U, V pass through unchanged (P is the identity there).
#include <cmath>
#include <vector>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

int launch_pc_tiles(Ctx* c, const std::vector<double>& shift_g, std::vector<double>& aa_tiles,
                    std::vector<double>& r3g);

// The sweeps run in FP64 in both modes: the residual y - P x of a later sweep
// cancels almost completely, and the block inverse amplifies whatever rounding
// it carries, so in FP32 it would leave P^-1 neither accurate nor linear.  The
// vectors of P^-1 are Stokes I only and its tables small; the FP32 tables of
// the ctx (K/DELO weights, Lambda_ii) enter as fixed coefficients.

// J[z][m] = sum_o w_o X[z][o][m][0]
__global__ void pc_angle_avg_kernel(const double* __restrict__ X, const double* __restrict__ w, double* __restrict__ J,
                                    int nz, int nO, int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nz * N) return;
  const int iz = idx / N, m = idx - iz * N;
  double s = 0.0;
  for (int o = 0; o < nO; ++o) s += w[o] * X[(((size_t)iz * nO + o) * N + m) * 4];
  J[idx] = s;
}

// V[z][o][n][0] = sum_m A[z][n][m] J[z][m]  (broadcast over o; Q,U,V zero)
__global__ void pc_matvec_bcast_kernel(const double* __restrict__ A, const double* __restrict__ J, double* __restrict__ V,
                                       int nz, int nO, int N) {
  const int iz = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double* a = A + ((size_t)iz * N + n) * N;
  const double* j = J + (size_t)iz * N;
  double s = 0.0;
  for (int m = 0; m < N; ++m) s += a[m] * j[m];
  for (int o = 0; o < nO; ++o) {
    double* v = V + (((size_t)iz * nO + o) * N + n) * 4;
    v[0] = s;
    v[1] = v[2] = v[3] = 0.0;
  }
}

// Scalar DELO-linear sweep of Stokes I: out = Lambda* eps (zero boundary).
template <typename T>
__global__ void pc_delo_kernel(const double* __restrict__ eps, const T* __restrict__ kt, const double* __restrict__ mu,
                               double* __restrict__ out, int nz, int nO, int N) {
  const int ray = blockIdx.x * blockDim.x + threadIdx.x;
  if (ray >= nO * N) return;
  const int o = ray / N, n = ray - o * N;
  const bool up = mu[o] > 0.0;
  double I = 0, Sp = 0;
  for (int p = 0; p < nz; ++p) {
    const int k = up ? p : nz - 1 - p;
    const size_t pt = ((size_t)k * nO + o) * N + n;
    const T* t = kt + pt * 10;
    const double S = eps[pt * 4] * (double)t[6];
    const double e = (double)t[7], al = (double)t[8], be = (double)t[9];
    if (p == 0) I = 0;
    else if (e <= 0.5) I = S + e * (I - S) + al * (Sp - S);   // thick: photon-exact form
    else I = e * I + al * Sp + be * S;                          // thin: standard form
    out[pt * 4] = I;
    Sp = S;
  }
}

// x[.][0] += r[.][0] + lii * v[.][0]  (Richardson update with P_hat^-1)
template <typename T>
__global__ void pc_update_kernel(double* __restrict__ x, const double* __restrict__ r, const T* __restrict__ lii,
                                 const double* __restrict__ v, long long npt) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  x[pt * 4] += r[pt * 4] + (double)lii[pt] * v[pt * 4];
}

// r[.][0] = y[.][0] - x[.][0] + LS[.][0]   (residual of P x = y on Stokes I)
template <typename T>
__global__ void pc_resid_kernel(const T* __restrict__ y, const double* __restrict__ x, const double* __restrict__ ls,
                                double* __restrict__ r, long long npt) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  r[pt * 4] = ((double)y[pt * 4] - x[pt * 4]) + ls[pt * 4];
}

// x = 0 on Stokes I; r = y on Stokes I (the first sweep's residual)
template <typename T>
__global__ void pc_init_kernel(const T* __restrict__ y, double* __restrict__ x, double* __restrict__ r, long long npt) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  x[pt * 4] = 0.0;
  r[pt * 4] = (double)y[pt * 4];
}

// out = (x on Stokes I, y on Q, U, V) in the ctx precision
template <typename T>
__global__ void pc_out_kernel(const T* __restrict__ y, const double* __restrict__ x, T* __restrict__ out, long long npt) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  out[pt * 4] = (T)x[pt * 4];
  out[pt * 4 + 1] = y[pt * 4 + 1];
  out[pt * 4 + 2] = y[pt * 4 + 2];
  out[pt * 4 + 3] = y[pt * 4 + 3];
}

// observer <-> comoving frame change of an FP64 vector (kernels_apply.cu)
int spline_frame_change_d(Ctx* c, const double* in, double* out, double* Mscratch, bool to_comoving);

static int lu_inverse(std::vector<double>& A, int n) {
  std::vector<int> piv(n);
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > std::fabs(A[(size_t)p * n + k])) p = i;
    piv[k] = p;
    if (A[(size_t)p * n + k] == 0.0) return -1;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      const double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = f;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
    }
  }
  for (int col = 0; col < n; ++col) {
    std::vector<double> b(n, 0.0);
    b[col] = 1.0;
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) b[i] -= A[(size_t)i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) b[i] -= A[(size_t)i * n + j] * b[j];
      b[i] /= A[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + col] = b[i];
  }
  A.swap(inv);
  return 0;
}

int launch_precond_setup(Ctx* c) {
  const int nz = c->nz, N = c->nnu, nO = c->nO, ng = c->ngrp;
  // J-level shifts at B = 0 and weights
  std::vector<double> sg((size_t)nz * ng), cg(ng);
  const prd_atom& at = c->atom;
  for (int g = 0; g < ng; ++g) {
    const double E = (at.twoS == 0 ? at.E_u_cm[0] : at.E_u_cm[g]) * kCmToHz - c->nu0;
    cg[g] = (at.twoS == 0) ? 1.0 : (g == 0 ? 1.0 / 3.0 : 2.0 / 3.0);
    for (int iz = 0; iz < nz; ++iz) sg[(size_t)iz * ng + g] = E / c->dnuD[iz];
  }
  std::vector<double> aa, r3;   // aa: [z][g][N][2N]; r3: [z][g*g][2N]
  int rc = launch_pc_tiles(c, sg, aa, r3);
  if (rc) return rc;
  std::vector<double> phi((size_t)nz * N * N), Mm((size_t)nz * N * N);
  std::vector<int> bad(nz, 0);
#pragma omp parallel for schedule(dynamic)
  for (int iz = 0; iz < nz; ++iz) {
    const double a0 = (1.0 - c->eps[iz]) * (1.0 - c->rE[iz]);
    const double b0 = 1.0 - c->eps[iz];
    std::vector<double> ph(N), rs(N, 0.0);
    for (int n = 0; n < N; ++n) {
      double s = 0.0;
      for (int g = 0; g < ng; ++g)
        s += cg[g] * faddeeva_host(cplx(c->u[(size_t)iz * N + n] + sg[(size_t)iz * ng + g], c->a[iz])).real() / kSqrtPi;
      ph[n] = s;
    }
    for (int g = 0; g < ng; ++g) {
      const double* rr = &r3[((size_t)iz * ng * ng + g * ng + g) * 2 * N];
      for (int m = 0; m < N; ++m) rs[m] += cg[g] * rr[m] / (2.0 * kSqrtPi);
    }
    double* P = &phi[(size_t)iz * N * N];
    for (int n = 0; n < N; ++n)
      for (int m = 0; m < N; ++m) {
        double v = 0.0;
        for (int g = 0; g < ng; ++g) v += cg[g] * aa[(((size_t)iz * ng + g) * N + n) * 2 * N + m] / kPi;
        P[(size_t)n * N + m] = c->k[iz] * (a0 * v + (b0 - a0) * ph[n] * rs[m]);
      }
    // lambda_bar(n) = sum_o w_o Lambda_ii(z, o, n)
    std::vector<double> lb(N, 0.0);
    for (int o = 0; o < nO; ++o)
      for (int n = 0; n < N; ++n) lb[n] += c->wang[o] * c->pc_lii_host[((size_t)iz * nO + o) * N + n];
    std::vector<double> A((size_t)N * N);
    for (int n = 0; n < N; ++n)
      for (int m = 0; m < N; ++m) A[(size_t)n * N + m] = (n == m ? 1.0 : 0.0) - lb[n] * P[(size_t)n * N + m];
    if (lu_inverse(A, N)) { bad[iz] = 1; continue; }
    double* Mz = &Mm[(size_t)iz * N * N];
    for (int n = 0; n < N; ++n)
      for (int m = 0; m < N; ++m) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += P[(size_t)n * N + k] * A[(size_t)k * N + m];
        Mz[(size_t)n * N + m] = s;
      }
  }
  for (int iz = 0; iz < nz; ++iz)
    if (bad[iz]) return fail(c, PRD_E_ARG, "block-Jacobi matrix (Id - A_i) is singular at height " + std::to_string(iz));
  if ((rc = upload(c, c->pc_phi, phi.data(), phi.size() * 8)) || (rc = upload(c, c->pc_M, Mm.data(), Mm.size() * 8)))
    return rc;
  DBuf w;
  if ((rc = upload(c, w, c->wang.data(), nO * 8))) return rc;
  c->owned.push_back(w);     // angular weights (double), freed with the ctx
  c->pc_w = w.p;
  const size_t vb = nvec(c) * sizeof(double);
  if ((rc = dalloc(c, c->pc_s1, vb)) || (rc = dalloc(c, c->pc_s2, vb)) || (rc = dalloc(c, c->pc_s3, vb)) ||
      (rc = dalloc(c, c->pc_s4, vb)) || (rc = dalloc(c, c->pc_s5, vb)) ||
      (rc = dalloc(c, c->gm_w, (size_t)nz * N * sizeof(double))))
    return rc;
  return PRD_OK;
}

template <typename T>
static int precond_T(Ctx* c, const T* y, T* x) {
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  const long long npt = (long long)nz * nO * N;
  double* r = (double*)c->pc_s1.p;
  double* t1 = (double*)c->pc_s2.p;
  double* t2 = (double*)c->pc_s3.p;
  double* xd = (double*)c->pc_s4.p;
  double* Ms = (double*)c->pc_s5.p;
  double* J = (double*)c->gm_w.p;
  const double* w = (const double*)c->pc_w;
  const int g1 = ceil_div(npt, 256);
  pc_init_kernel<T><<<g1, 256, 0, c->stream>>>(y, xd, r, npt);
  for (int sweep = 0; sweep < c->m_in; ++sweep) {
    // r = y - P x on Stokes I (P x = x - Lambda* Sigma* x); the first sweep starts from x = 0
    if (sweep > 0) {
      int rc = spline_frame_change_d(c, xd, t1, Ms, true);                  // comoving I~
      if (rc) return rc;
      pc_angle_avg_kernel<<<ceil_div(nz * N, 128), 128, 0, c->stream>>>(t1, w, J, nz, nO, N);
      pc_matvec_bcast_kernel<<<dim3(ceil_div(N, 128), nz), 128, 0, c->stream>>>((const double*)c->pc_phi.p, J, t2, nz,
                                                                               nO, N);
      if ((rc = spline_frame_change_d(c, t2, t1, Ms, false))) return rc;    // eps* (observer)
      pc_delo_kernel<T><<<ceil_div(nO * N, 128), 128, 0, c->stream>>>(t1, (const T*)c->kt.p, (const double*)c->dmu.p,
                                                                      t2, nz, nO, N);
      pc_resid_kernel<T><<<g1, 256, 0, c->stream>>>(y, xd, t2, r, npt);
    }
    // x += P_hat^-1 r
    pc_angle_avg_kernel<<<ceil_div(nz * N, 128), 128, 0, c->stream>>>(r, w, J, nz, nO, N);
    pc_matvec_bcast_kernel<<<dim3(ceil_div(N, 128), nz), 128, 0, c->stream>>>((const double*)c->pc_M.p, J, t2, nz, nO, N);
    pc_update_kernel<T><<<g1, 256, 0, c->stream>>>(xd, r, (const T*)c->pc_lii.p, t2, npt);
  }
  pc_out_kernel<T><<<g1, 256, 0, c->stream>>>(y, xd, x, npt);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

int apply_precond(Ctx* c, const void* y, void* x) {
  if (c->m_in <= 0) {
    PRD_CUDA_TRY(c, cudaMemcpyAsync(x, y, nvec(c) * c->esz, cudaMemcpyDeviceToDevice, c->stream));
    return PRD_OK;
  }
  if (c->prec == PRD_FP64) return precond_T<double>(c, (const double*)y, (double*)x);
  return precond_T<float>(c, (const float*)y, (float*)x);
}

}  // namespace prd
