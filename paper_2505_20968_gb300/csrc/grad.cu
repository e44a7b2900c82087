// S13: gradient of a functional J(I) of the solution with respect to the
// magnetic-field parameters (B, theta_B, chi_B) of every height, by the adjoint
// method on the discrete system A(p) I = b(p) of Eq. linear_system:
//   dJ/dp = lam^T (db/dp - (dA/dp) I),   A^T lam = dJ/dI.
// lam comes from one adjoint solve; the parameter derivative of the residual
// b(p) - A(p) I (I fixed) is a central difference per parameter, each side a
// full FP64 setup of the perturbed atmosphere (steps: 1e-3 relative; 0.1 G for
// B = 0, where the difference is one-sided; 1e-3 rad for angles at 0).  The
// cost is 6 setups per height, which suits reduced problems; the paper has no
// gradient (it solves forward problems only).
#include <cmath>
#include <vector>
#include "prd_internal.h"

namespace prd {

namespace {

__global__ void f2d_kernel2(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}
// out += sum_i lam_i (b_i - y_i)
__global__ void resdot_kernel(const double* __restrict__ lam, const double* __restrict__ b,
                              const double* __restrict__ y, size_t n, double* out) {
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += lam[i] * (b[i] - y[i]);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

}  // namespace

// lam^T (b(p') - A(p') x) for the atmosphere of c with B, theta_B, chi_B replaced;
// x64, lam64: FP64 device vectors of c's shape.
static int residual_dot(Ctx* c, const std::vector<double>& B, const std::vector<double>& thB,
                        const std::vector<double>& chB, const double* x64, const double* lam64, double* out) {
  prd_ctx* h = nullptr;
  int rc = prd_create(&h, c->device, PRD_FP64);
  if (rc) return fail(c, rc, "gradient: cannot create the perturbed context");
  const size_t n = nvec(c);
  DBuf b, y, acc;
  auto done = [&](int code) {
    dfree(b); dfree(y); dfree(acc);
    if (code && h) fail(c, code, std::string("gradient: perturbed setup or apply: ") + prd_last_error(h));
    prd_destroy(h);
    return code;
  };
  if ((rc = prd_set_atom(h, &c->atom))) return done(rc);
  if ((rc = prd_set_atmosphere(h, c->nz, c->z.data(), c->T.data(), c->xi.data(), c->a.data(), c->eps.data(),
                               c->rE.data(), c->k.data(), c->WT.data(), B.data(), thB.data(), chB.data(),
                               c->v.data())))
    return done(rc);
  if ((rc = prd_set_quadrature(h, c->nnu, c->grid.data(), c->grid_kind, c->n_mu_half, c->n_chi, c->mu_rule,
                               c->mode)))
    return done(rc);
  if ((rc = prd_set_stream(h, c->stream))) return done(rc);
  if ((rc = prd_setup(h))) return done(rc);
  if ((rc = dalloc(c, b, n * 8)) || (rc = dalloc(c, y, n * 8)) || (rc = dalloc(c, acc, 8))) return done(rc);
  if ((rc = prd_rhs(h, b.p)) || (rc = prd_apply_operator(h, x64, y.p))) return done(rc);
  if (cudaMemsetAsync(acc.p, 0, 8, c->stream) != cudaSuccess) return done(PRD_E_CUDA);
  resdot_kernel<<<c->grid_ew(), 256, 0, c->stream>>>(lam64, (const double*)b.p, (const double*)y.p, n, (double*)acc.p);
  if (cudaMemcpyAsync(out, acc.p, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return done(PRD_E_CUDA);
  return done(PRD_OK);
}

int grad_b(Ctx* c, const void* x, const void* dJdI, double tol, double* dJdp) {
  const size_t n = nvec(c);
  const int nz = c->nz;
  DBuf lam, x64, lam64;
  auto cleanup = [&]() { dfree(lam); dfree(x64); dfree(lam64); };
  int rc;
  if ((rc = dalloc(c, lam, n * c->esz)) || (rc = dalloc(c, x64, n * 8)) || (rc = dalloc(c, lam64, n * 8))) {
    cleanup();
    return rc;
  }
  int its = 0;
  double res = 0.0;
  if ((rc = solve_adjoint(c, dJdI, tol, 3000, 120, lam.p, &its, &res, nullptr))) { cleanup(); return rc; }
  if (c->prec == PRD_FP64) {
    PRD_CUDA_TRY(c, cudaMemcpyAsync(x64.p, x, n * 8, cudaMemcpyDeviceToDevice, c->stream));
    PRD_CUDA_TRY(c, cudaMemcpyAsync(lam64.p, lam.p, n * 8, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    f2d_kernel2<<<c->grid_ew(), 256, 0, c->stream>>>((const float*)x, (double*)x64.p, n);
    f2d_kernel2<<<c->grid_ew(), 256, 0, c->stream>>>((const float*)lam.p, (double*)lam64.p, n);
  }
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<double>* par[3] = {&c->B, &c->thB, &c->chB};
  for (int iz = 0; iz < nz && !rc; ++iz)
    for (int k = 0; k < 3 && !rc; ++k) {
      const double p0 = (*par[k])[iz];
      const double step = k == 0 ? std::max(1e-3 * std::fabs(p0), 0.1) : std::max(1e-3 * std::fabs(p0), 1e-3);
      const double lo = (k == 0 && p0 - step < 0.0) ? p0 : p0 - step;   // B >= 0: one-sided at B = 0
      const double hi = p0 + step;
      double rp = 0.0, rm = 0.0;
      std::vector<double> B = c->B, th = c->thB, ch = c->chB;
      std::vector<double>* q[3] = {&B, &th, &ch};
      (*q[k])[iz] = hi;
      if ((rc = residual_dot(c, B, th, ch, (const double*)x64.p, (const double*)lam64.p, &rp))) break;
      (*q[k])[iz] = lo;
      if ((rc = residual_dot(c, B, th, ch, (const double*)x64.p, (const double*)lam64.p, &rm))) break;
      dJdp[iz * 3 + k] = (rp - rm) / (hi - lo);
    }
  cleanup();
  return rc;
}

}  // namespace prd
