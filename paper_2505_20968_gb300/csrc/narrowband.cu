// Wavelength-integrated narrow-band Stokes signals (Sect. 6.5): the emergent
// profiles X(z_max, mu, lambda) along lines of sight, weighted by a Gaussian
// of full width at half maximum `fwhm` centred on lambda_0 and integrated over
// [lambda_0 - Delta, lambda_0 + Delta], normalised by 1/(sqrt(2 pi) sigma).
//
// X between the wavelength nodes is its natural cubic spline in lambda and
// beyond the grid its end value (the continuation of the frame changes), so
// Xbar = sum_n w_n X_n with w_n the integral of the Gaussian against the n-th
// spline basis function.  The weights are computed once per call on the host
// in FP64 (16-point Gauss-Legendre on every grid interval inside the limits,
// the error function on the constant continuations); the reduction over the
// emergent profiles runs on the device with FP64 accumulation.
#include <cmath>
#include <vector>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

// out[l][s] = sum_n w[n] em[l][n][s]   (one warp per (l, s))
template <typename T>
__global__ void narrowband_kernel(const T* __restrict__ em, const double* __restrict__ w, double* __restrict__ out,
                                  int nlos, int N) {
  const int ls = blockIdx.x;                 // (l, s)
  if (ls >= nlos * 4) return;
  const int l = ls >> 2, s = ls & 3;
  double acc = 0.0;
  for (int n = threadIdx.x; n < N; n += 32) acc += w[n] * (double)em[((size_t)l * N + n) * 4 + s];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) out[ls] = acc;
}

// Vacuum wavelengths (Angstrom) of the frequency nodes, ascending.
static std::vector<double> grid_wavelengths(const Ctx* c) {
  const int N = c->nnu;
  std::vector<double> lam(N);
  for (int n = 0; n < N; ++n) {
    if (c->grid_kind == PRD_GRID_LAMBDA) lam[n] = c->grid[n];
    else lam[n] = kC / (c->nu0 - c->grid[n] * c->dnuD[0]) * 1e10;
  }
  return lam;
}

// w[n]: the weight of node n in the Gaussian-weighted integral.
static int narrowband_weights(Ctx* c, double lam0, double fwhm, double half, std::vector<double>& w) {
  const int N = c->nnu;
  const std::vector<double> lam = grid_wavelengths(c);
  for (int n = 0; n + 1 < N; ++n)
    if (!(lam[n + 1] > lam[n])) return fail(c, PRD_E_ARG, "wavelength nodes are not ascending");
  std::vector<double> Q((size_t)N * N);
  natural_spline_Q(lam.data(), N, Q.data());
  const double sig = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  const double norm = 1.0 / (std::sqrt(2.0 * kPi) * sig);
  const double a = lam0 - half, b = lam0 + half;
  auto g = [&](double l) { const double d = (l - lam0) / sig; return norm * std::exp(-0.5 * d * d); };
  // integral of g over [p, q]
  auto gint = [&](double p, double q) {
    return 0.5 * (std::erf((q - lam0) / (std::sqrt(2.0) * sig)) - std::erf((p - lam0) / (std::sqrt(2.0) * sig)));
  };
  std::vector<double> xg, wg;
  gauss_legendre(16, xg, wg);
  w.assign(N, 0.0);
  std::vector<double> cM(N, 0.0);   // coefficient of the second derivative M_j = sum_m Q[j][m] X_m
  for (int j = 0; j + 1 < N; ++j) {
    const double x0 = std::max(a, lam[j]), x1 = std::min(b, lam[j + 1]);
    if (!(x1 > x0)) continue;
    const double h = lam[j + 1] - lam[j], half_w = 0.5 * (x1 - x0), mid = 0.5 * (x1 + x0);
    for (int k = 0; k < 16; ++k) {
      const double l = mid + half_w * xg[k];
      const double f = g(l) * half_w * wg[k];
      const double t = (l - lam[j]) / h, omt = 1.0 - t, k6 = h * h / 6.0;
      w[j] += f * omt;
      w[j + 1] += f * t;
      cM[j] += f * k6 * (omt * omt * omt - omt);
      cM[j + 1] += f * k6 * (t * t * t - t);
    }
  }
  for (int j = 0; j < N; ++j)
    if (cM[j] != 0.0)
      for (int m = 0; m < N; ++m) w[m] += cM[j] * Q[(size_t)j * N + m];
  if (a < lam[0]) w[0] += gint(a, std::min(b, lam[0]));
  if (b > lam[N - 1]) w[N - 1] += gint(std::max(a, lam[N - 1]), b);
  return PRD_OK;
}

int narrowband(Ctx* c, const void* x, int nlos, const double* mu, const double* chi, double lam0, double fwhm,
               double half, double* out) {
  std::vector<double> w;
  int rc = narrowband_weights(c, lam0, fwhm, half, w);
  if (rc) return rc;
  const int N = c->nnu;
  DBuf em, dw, dout;
  auto cleanup = [&]() { dfree(em); dfree(dw); dfree(dout); };
  if ((rc = dalloc(c, em, (size_t)nlos * N * 4 * c->esz)) || (rc = upload(c, dw, w.data(), w.size() * 8)) ||
      (rc = dalloc(c, dout, (size_t)nlos * 4 * 8))) {
    cleanup();
    return rc;
  }
  if ((rc = emergent(c, x, nlos, mu, chi, em.p))) { cleanup(); return rc; }
  if (c->prec == PRD_FP64)
    narrowband_kernel<double><<<nlos * 4, 32, 0, c->stream>>>((const double*)em.p, (const double*)dw.p,
                                                              (double*)dout.p, nlos, N);
  else
    narrowband_kernel<float><<<nlos * 4, 32, 0, c->stream>>>((const float*)em.p, (const double*)dw.p,
                                                             (double*)dout.p, nlos, N);
  cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout.p, (size_t)nlos * 4 * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cleanup();
  if (e != cudaSuccess) return fail(c, PRD_E_CUDA, std::string("narrow-band signals: ") + cudaGetErrorString(e));
  return PRD_OK;
}

}  // namespace prd
