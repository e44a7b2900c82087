// S13: gradient of a functional J(I) of the solution with respect to the
// magnetic-field parameters (B, theta_B, chi_B) of every height, by the adjoint
// method on the discrete system A(p) I = b(p) of Eq. linear_system:
//   dJ/dp = lam^T (db/dp - (dA/dp) I),   A^T lam = dJ/dI.
// lam comes from one adjoint solve; the parameter derivative of the residual
// b(p) - A(p) I (I fixed) is a central difference per parameter (steps: 1e-3
// relative; 0.1 G for B = 0, where the difference is one-sided; 1e-3 rad for
// angles at 0).  Each side re-sets up, in FP64, only what the perturbed height
// changes: its Sigma rows (a two-height context) and the formal solver's
// tables of the whole atmosphere (no Sigma tables); PRD_OPT_GRAD_FULL_SETUP
// takes a full setup of the perturbed atmosphere per side instead.  The paper
// has no gradient (it solves forward problems only).
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

__global__ void row_sum_kernel(double* __restrict__ dst, const double* __restrict__ a, const double* __restrict__ b,
                               size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = a[i] + b[i];
}

// The same residual dot, re-setting up only what the perturbed height iz
// changes.  Sigma is local in height (every table of its rows, f included,
// comes from that height's own state), so its rows at iz come from a context
// of two heights, height 0 (the reference of a reduced-frequency grid) and iz
// (or iz = 0 and 1), with the perturbed field at iz; the rest of
// eps' = eps_th + Sigma' x is the unperturbed e.  The formal solution sees the
// perturbed K at iz (and the DELO weights of its two steps), so it runs in a
// context of the whole perturbed atmosphere that holds the formal solver's
// tables only.  Then b' - A' x = Lambda'_b eps' - x.
static int residual_dot_local(Ctx* c, int iz, const std::vector<double>& B, const std::vector<double>& thB,
                              const std::vector<double>& chB, const double* x64, const double* lam64,
                              const double* e64, double* out) {
  const int nz = c->nz;
  const size_t n = nvec(c), row = n / nz;
  prd_ctx* hs = nullptr;   // two heights
  prd_ctx* hl = nullptr;   // the whole atmosphere, formal solver only
  DBuf xs, ss, ep, y, acc;
  auto done = [&](int code, prd_ctx* who) {
    dfree(xs); dfree(ss); dfree(ep); dfree(y); dfree(acc);
    if (code && who) fail(c, code, std::string("gradient: perturbed height set-up or apply: ") + prd_last_error(who));
    else if (code) fail(c, code, "gradient: perturbed height contexts");
    if (hs) prd_destroy(hs);
    if (hl) prd_destroy(hl);
    return code;
  };
  int rc;
  if ((rc = prd_create(&hs, c->device, PRD_FP64)) || (rc = prd_create(&hl, c->device, PRD_FP64))) return done(rc, nullptr);
  hl->c.lambda_only = true;
  const int i0 = 0, i1 = iz == 0 ? 1 : iz;   // rows of the two-height atmosphere
  const int j = iz == 0 ? 0 : 1;              // the row of iz in it
  auto pick = [&](const std::vector<double>& v) { return std::vector<double>{v[i0], v[i1]}; };
  std::vector<double> z2 = pick(c->z), T2 = pick(c->T), xi2 = pick(c->xi), a2 = pick(c->a), e2 = pick(c->eps),
                      r2 = pick(c->rE), k2 = pick(c->k), w2 = pick(c->WT), B2 = pick(B), th2 = pick(thB),
                      ch2 = pick(chB);
  std::vector<double> v2 = {c->v[3 * i0], c->v[3 * i0 + 1], c->v[3 * i0 + 2], c->v[3 * i1], c->v[3 * i1 + 1],
                            c->v[3 * i1 + 2]};
  for (prd_ctx* h : {hs, hl}) {
    if ((rc = prd_set_atom(h, &c->atom))) return done(rc, h);
    if ((rc = prd_set_quadrature(h, c->nnu, c->grid.data(), c->grid_kind, c->n_mu_half, c->n_chi, c->mu_rule,
                                 c->mode)))
      return done(rc, h);
    if ((rc = prd_set_stream(h, c->stream))) return done(rc, h);
  }
  if ((rc = prd_set_atmosphere(hs, 2, z2.data(), T2.data(), xi2.data(), a2.data(), e2.data(), r2.data(), k2.data(),
                               w2.data(), B2.data(), th2.data(), ch2.data(), v2.data())))
    return done(rc, hs);
  if ((rc = prd_set_atmosphere(hl, nz, c->z.data(), c->T.data(), c->xi.data(), c->a.data(), c->eps.data(),
                               c->rE.data(), c->k.data(), c->WT.data(), B.data(), thB.data(), chB.data(),
                               c->v.data())))
    return done(rc, hl);
  if ((rc = prd_setup(hs))) return done(rc, hs);
  if ((rc = prd_setup(hl))) return done(rc, hl);
  if ((rc = dalloc(c, xs, 2 * row * 8)) || (rc = dalloc(c, ss, 2 * row * 8)) || (rc = dalloc(c, ep, n * 8)) ||
      (rc = dalloc(c, y, n * 8)) || (rc = dalloc(c, acc, 8)))
    return done(rc, nullptr);
  // Sigma' x at iz from the two-height context, on the rows i0, i1 of x
  if (cudaMemcpyAsync(xs.p, x64 + (size_t)i0 * row, row * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync((double*)xs.p + row, x64 + (size_t)i1 * row, row * 8, cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(ep.p, e64, n * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return done(PRD_E_CUDA, nullptr);
  if ((rc = apply_sigma(&hs->c, xs.p, ss.p, true))) return done(rc, hs);
  row_sum_kernel<<<c->grid_ew(), 256, 0, c->stream>>>((double*)ep.p + (size_t)iz * row, (const double*)ss.p + j * row,
                                                       (const double*)hs->c.epsth.p + j * row, row);
  // Lambda'_b eps' in the perturbed atmosphere, then lam^T (Lambda'_b eps' - x)
  if ((rc = apply_lambda(&hl->c, ep.p, y.p, nullptr, true))) return done(rc, hl);
  if (cudaMemsetAsync(acc.p, 0, 8, c->stream) != cudaSuccess) return done(PRD_E_CUDA, nullptr);
  resdot_kernel<<<c->grid_ew(), 256, 0, c->stream>>>(lam64, (const double*)y.p, x64, n, (double*)acc.p);
  if (cudaMemcpyAsync(out, acc.p, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return done(PRD_E_CUDA, nullptr);
  return done(PRD_OK, nullptr);
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
  // the unperturbed emissivity eps_th + Sigma x (FP64), shared by the per-height residuals
  DBuf e64, ws;
  if (!c->grad_full_setup) {
    if ((rc = dalloc(c, e64, n * 8)) || (rc = dalloc(c, ws, 3 * n * 8)) ||
        (rc = emissivity_acc(c, (const double*)x64.p, (double*)e64.p, (double*)ws.p))) {
      dfree(e64); dfree(ws); cleanup();
      return rc;
    }
  }
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  dfree(ws);
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
      auto rdot = [&](double* out) {
        return c->grad_full_setup
                   ? residual_dot(c, B, th, ch, (const double*)x64.p, (const double*)lam64.p, out)
                   : residual_dot_local(c, iz, B, th, ch, (const double*)x64.p, (const double*)lam64.p,
                                        (const double*)e64.p, out);
      };
      (*q[k])[iz] = hi;
      if ((rc = rdot(&rp))) break;
      (*q[k])[iz] = lo;
      if ((rc = rdot(&rm))) break;
      dJdp[iz * 3 + k] = (rp - rm) / (hi - lo);
    }
  dfree(e64);
  cleanup();
  return rc;
}

}  // namespace prd
