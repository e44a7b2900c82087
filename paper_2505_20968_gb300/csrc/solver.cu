// Krylov solver (S10): left-preconditioned restarted GMRES with classical
// Gram-Schmidt applied twice (CGS2), inner products accumulated in FP64 on the
// device, Givens rotations and the least-squares update in FP64 on the host
// (Sect. 5.1-5.2).  The stopping test is the unpreconditioned relative residual
// ||b - A x|| / ||b|| of Sect. 5.1, recomputed in FP64 before returning.
#include <cmath>
#include <cstring>
#include <vector>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

// dots[k] += sum_i V[k][i] * w[i]   for k < nv   (FP64 accumulation)
template <typename T>
__global__ void multidot_kernel(const T* __restrict__ V, size_t ld, const T* __restrict__ w, size_t n, double* dots) {
  const int k = blockIdx.y;
  const T* v = V + (size_t)k * ld;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += (double)v[i] * (double)w[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&dots[k], red[0]);
}

// w -= sum_k h[k] V[k]
template <typename T>
__global__ void multiaxpy_kernel(const T* __restrict__ V, size_t ld, const double* __restrict__ h, int nv, T* w,
                                 size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = (double)w[i];
    for (int k = 0; k < nv; ++k) s -= h[k] * (double)V[(size_t)k * ld + i];
    w[i] = (T)s;
  }
}

template <typename T>
__global__ void scale_copy_kernel(const T* __restrict__ a, double s, T* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (T)((double)a[i] * s);
}

// x += sum_k y[k] V[k]
template <typename T>
__global__ void update_kernel(const T* __restrict__ V, size_t ld, const double* __restrict__ y, int nv, T* x, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = (double)x[i];
    for (int k = 0; k < nv; ++k) s += y[k] * (double)V[(size_t)k * ld + i];
    x[i] = (T)s;
  }
}

// r = b - r   (r holds A x on entry)
template <typename T>
__global__ void rsub_kernel(const T* __restrict__ b, T* r, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    r[i] = b[i] - r[i];
}

namespace {

struct Vops {
  Ctx* c;
  size_t n;
  int grid;
  DBuf dots;
  int cap = 0;   // capacity of `dots` in doubles
  int init(int capacity) {
    grid = 152 * 4;
    cap = capacity;
    return dalloc(c, dots, (size_t)capacity * sizeof(double));
  }
  int dot_many(const void* V, size_t ld, int nv, const void* w, double* out) {
    if (nv > cap) return fail(c, PRD_E_ARG, "internal: dot buffer too small");
    PRD_CUDA_TRY(c, cudaMemsetAsync(dots.p, 0, nv * sizeof(double), c->stream));
    if (c->prec == PRD_FP64)
      multidot_kernel<double><<<dim3(grid, nv), 256, 0, c->stream>>>((const double*)V, ld, (const double*)w, n, (double*)dots.p);
    else
      multidot_kernel<float><<<dim3(grid, nv), 256, 0, c->stream>>>((const float*)V, ld, (const float*)w, n, (double*)dots.p);
    PRD_CUDA_TRY(c, cudaMemcpyAsync(out, dots.p, nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PRD_OK;
  }
  int axpy_many(const void* V, size_t ld, const double* h, int nv, void* w) {
    if (nv > cap) return fail(c, PRD_E_ARG, "internal: dot buffer too small");
    PRD_CUDA_TRY(c, cudaMemcpyAsync(dots.p, h, nv * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->prec == PRD_FP64)
      multiaxpy_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)V, ld, (const double*)dots.p, nv, (double*)w, n);
    else
      multiaxpy_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)V, ld, (const double*)dots.p, nv, (float*)w, n);
    PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PRD_OK;
  }
  int update(const void* V, size_t ld, const double* y, int nv, void* x) {
    if (nv > cap) return fail(c, PRD_E_ARG, "internal: dot buffer too small");
    PRD_CUDA_TRY(c, cudaMemcpyAsync(dots.p, y, nv * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->prec == PRD_FP64)
      update_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)V, ld, (const double*)dots.p, nv, (double*)x, n);
    else
      update_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)V, ld, (const double*)dots.p, nv, (float*)x, n);
    PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PRD_OK;
  }
  int scale(const void* a, double s, void* b) {
    if (c->prec == PRD_FP64)
      scale_copy_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)a, s, (double*)b, n);
    else
      scale_copy_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)a, s, (float*)b, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  int rsub(const void* b, void* r) {
    if (c->prec == PRD_FP64) rsub_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)b, (double*)r, n);
    else rsub_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)b, (float*)r, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  int norm(const void* a, double* out) {
    double d;
    int rc = dot_many(a, 0, 1, a, &d);
    *out = std::sqrt(d);
    return rc;
  }
};

}  // namespace

int apply_operator_t(Ctx* c, const void* x, void* y);
// the operator GMRES iterates with: A, or A^T for the adjoint solve
static int op_apply(Ctx* c, const void* x, void* y) {
  return c->op_transpose ? apply_operator_t(c, x, y) : apply_operator(c, x, y);
}

// GMRES on A x = b in the ctx precision; x holds the initial guess on entry.
// inner: correction solve of the mixed-precision refinement.  x is zero on
// entry and the solve ends as soon as the Arnoldi estimate is below tol (the
// refinement's FP64 residual is the true check), so no apply is spent on a
// residual the caller recomputes anyway.
static int gmres_core(Ctx* c, const void* bvec, void* x, double tol, int max_iter, int restart, int* iters,
                      double* true_res, double* hist, double hist_scale, int* nh_io, bool inner = false) {
  const size_t n = nvec(c);
  const size_t vb = n * c->esz;
  const int m = std::max(1, std::min(restart, 200));
  Vops ops{c, n};
  int rc = ops.init(m + 2);
  if (rc) return rc;
  DBuf V, r, w;
  struct { void* p; } b{const_cast<void*>(bvec)};
  auto cleanup = [&]() { dfree(V); dfree(r); dfree(w); dfree(ops.dots); };
  if ((rc = dalloc(c, V, vb * (m + 1))) || (rc = dalloc(c, r, vb)) || (rc = dalloc(c, w, vb))) {
    cleanup();
    return rc;
  }
  auto vec = [&](int k) { return (void*)((char*)V.p + (size_t)k * vb); };
  double bnorm;
  if ((rc = ops.norm(b.p, &bnorm))) { cleanup(); return rc; }
  if (!(bnorm > 0) || !std::isfinite(bnorm)) { cleanup(); return fail(c, PRD_E_NAN, "right-hand side norm is zero or not finite"); }
  int it = 0, nh = nh_io ? *nh_io : 0;
  double tol_in = tol;
  double tr = 1.0;
  int status = PRD_E_NOCONV;
  bool first = true;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h(m + 1), h2(m + 1);
  while (it < max_iter) {
    // r = P^-1 (b - A x)
    if (inner && first) {
      PRD_CUDA_TRY(c, cudaMemcpyAsync(w.p, b.p, vb, cudaMemcpyDeviceToDevice, c->stream));
      tr = 1.0;
    } else {
      if ((rc = op_apply(c, x, w.p)) || (rc = ops.rsub(b.p, w.p))) break;
      double rn_true;
      if ((rc = ops.norm(w.p, &rn_true))) break;
      tr = rn_true / bnorm;
    }
    first = false;
    if (!std::isfinite(tr)) { rc = fail(c, PRD_E_NAN, "residual is not finite"); break; }
    if (tr < tol) { status = PRD_OK; break; }
    if ((rc = apply_precond(c, w.p, r.p))) break;
    double beta;
    if ((rc = ops.norm(r.p, &beta))) break;
    if (!(beta > 0)) { status = PRD_OK; break; }
    if ((rc = ops.scale(r.p, 1.0 / beta, vec(0)))) break;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    const double beta0 = beta;
    int j = 0;
    bool breakdown = false, est_ok = false;
    for (; j < m && it < max_iter; ++j) {
      if ((rc = op_apply(c, vec(j), w.p)) || (rc = apply_precond(c, w.p, r.p))) break;
      ++it;
      // CGS2
      if ((rc = ops.dot_many(V.p, n, j + 1, r.p, h.data())) || (rc = ops.axpy_many(V.p, n, h.data(), j + 1, r.p))) break;
      if ((rc = ops.dot_many(V.p, n, j + 1, r.p, h2.data())) || (rc = ops.axpy_many(V.p, n, h2.data(), j + 1, r.p))) break;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i] + h2[i];
      double hn;
      if ((rc = ops.norm(r.p, &hn))) break;
      if (!std::isfinite(hn)) { rc = fail(c, PRD_E_NAN, "Arnoldi vector is not finite"); break; }
      H[(size_t)(j + 1) * m + j] = hn;
      // Givens
      for (int i = 0; i < j; ++i) {
        const double a0 = H[(size_t)i * m + j], a1 = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a0 + sn[i] * a1;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
      }
      const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
      const double den = std::hypot(a0, a1);
      cs[j] = den > 0 ? a0 / den : 1.0;
      sn[j] = den > 0 ? a1 / den : 0.0;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      const double est = tr * std::fabs(g[j + 1]) / beta0;   // estimate of the true relative residual
      if (hist && nh <= max_iter) hist[nh++] = est * hist_scale;
      if (hn <= 1e-300 * std::max(1.0, beta0)) { breakdown = true; ++j; break; }
      if ((rc = ops.scale(r.p, 1.0 / hn, vec(j + 1)))) break;
      if (est < 0.5 * tol_in) { ++j; est_ok = true; break; }
    }
    if (rc) break;
    // back substitution H y = g, x += V y
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
      y[i] = s / H[(size_t)i * m + i];
    }
    if ((rc = ops.update(V.p, n, y.data(), j, x))) break;
    if (inner && (est_ok || breakdown)) {
      status = PRD_OK;
      tr = std::fabs(g[j]) / beta0 * tr;
      break;
    }
    if (breakdown) {
      if ((rc = op_apply(c, x, w.p)) || (rc = ops.rsub(b.p, w.p))) break;
      double rn;
      if ((rc = ops.norm(w.p, &rn))) break;
      tr = rn / bnorm;
      status = tr < tol ? PRD_OK : PRD_E_BREAKDOWN;
      break;
    }
    tol_in *= 0.5;
  }
  if (!rc && status == PRD_E_NOCONV && !inner) {
    // final true residual
    if (!(rc = op_apply(c, x, w.p)) && !(rc = ops.rsub(b.p, w.p))) {
      double rn;
      if (!(rc = ops.norm(w.p, &rn))) {
        tr = rn / bnorm;
        if (tr < tol) status = PRD_OK;
      }
    }
  }
  if (iters) *iters = it;
  if (true_res) *true_res = tr;
  if (nh_io) *nh_io = nh;
  cleanup();
  if (rc) return rc;
  if (status == PRD_E_NOCONV) return fail(c, PRD_E_NOCONV, "GMRES reached max_iter before tol");
  if (status == PRD_E_BREAKDOWN) return fail(c, PRD_E_BREAKDOWN, "GMRES breakdown before tol");
  return PRD_OK;
}

__global__ void d2f_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f2d_add_kernel(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] += (double)a[i];
}
__global__ void f2d_kernel(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void sub_kernel(const double* __restrict__ b, double* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = b[i] - y[i];
}
__global__ void dnorm2_kernel(const double* __restrict__ a, size_t n, double* out) {
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += a[i] * a[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

int apply_operator_acc(Ctx* c, const double* x, double* y, double* ws);
int rhs_acc(Ctx* c, double* b);

static int dnorm(Ctx* c, const double* a, size_t n, double* dsum, double* out) {
  PRD_CUDA_TRY(c, cudaMemsetAsync(dsum, 0, 8, c->stream));
  dnorm2_kernel<<<608, 256, 0, c->stream>>>(a, n, dsum);
  double h;
  PRD_CUDA_TRY(c, cudaMemcpyAsync(&h, dsum, 8, cudaMemcpyDeviceToHost, c->stream));
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *out = std::sqrt(h);
  return PRD_OK;
}

int solve(Ctx* c, double tol, int max_iter, int restart, const void* x0, void* x, int* iters, double* true_res,
          double* hist) {
  const size_t n = nvec(c);
  const size_t vb = n * c->esz;
  int rc;
  if (c->prec == PRD_FP64) {
    DBuf b;
    if ((rc = dalloc(c, b, vb))) return rc;
    if ((rc = rhs(c, b.p))) { dfree(b); return rc; }
    if (x0) PRD_CUDA_TRY(c, cudaMemcpyAsync(x, x0, vb, cudaMemcpyDeviceToDevice, c->stream));
    else PRD_CUDA_TRY(c, cudaMemsetAsync(x, 0, vb, c->stream));
    rc = gmres_core(c, b.p, x, tol, max_iter, restart, iters, true_res, hist, 1.0, nullptr);
    dfree(b);
    return rc;
  }
  // FP32 mode: mixed-precision iterative refinement.  Residuals b - A x are
  // formed with FP64 vectors and FP64 accumulation over the FP32-stored
  // operator (the FP64 residual check); corrections come from FP32 GMRES.
  DBuf b64, x64, r64, ws, d32, r32, dsum;
  auto cleanup = [&]() { dfree(b64); dfree(x64); dfree(r64); dfree(ws); dfree(d32); dfree(r32); dfree(dsum); };
  if ((rc = dalloc(c, b64, n * 8)) || (rc = dalloc(c, x64, n * 8)) || (rc = dalloc(c, r64, n * 8)) ||
      (rc = dalloc(c, ws, 4 * n * 8)) || (rc = dalloc(c, d32, vb)) || (rc = dalloc(c, r32, vb)) ||
      (rc = dalloc(c, dsum, 8))) {
    cleanup();
    return rc;
  }
  const int G = 608;
  if ((rc = rhs_acc(c, (double*)b64.p))) { cleanup(); return rc; }
  if (x0) f2d_kernel<<<G, 256, 0, c->stream>>>((const float*)x0, (double*)x64.p, n);
  else PRD_CUDA_TRY(c, cudaMemsetAsync(x64.p, 0, n * 8, c->stream));
  double bn;
  if ((rc = dnorm(c, (const double*)b64.p, n, (double*)dsum.p, &bn))) { cleanup(); return rc; }
  if (!(bn > 0) || !std::isfinite(bn)) { cleanup(); return fail(c, PRD_E_NAN, "right-hand side norm is zero or not finite"); }
  int it_total = 0, nh = 0, status = PRD_E_NOCONV;
  double res = 1.0;
  for (int outer = 0; outer < 12 && it_total < max_iter; ++outer) {
    double rn;
    if (outer == 0 && !x0) {
      // x = 0: the residual is b itself (no FP64 apply)
      PRD_CUDA_TRY(c, cudaMemcpyAsync(r64.p, b64.p, n * 8, cudaMemcpyDeviceToDevice, c->stream));
      rn = bn;
    } else {
      if ((rc = apply_operator_acc(c, (const double*)x64.p, (double*)r64.p, (double*)ws.p))) break;
      sub_kernel<<<G, 256, 0, c->stream>>>((const double*)b64.p, (double*)r64.p, n);
      if ((rc = dnorm(c, (const double*)r64.p, n, (double*)dsum.p, &rn))) break;
    }
    res = rn / bn;
    if (!std::isfinite(res)) { rc = fail(c, PRD_E_NAN, "residual is not finite"); break; }
    if (res < tol) { status = PRD_OK; break; }
    d2f_kernel<<<G, 256, 0, c->stream>>>((const double*)r64.p, (float*)r32.p, n);
    PRD_CUDA_TRY(c, cudaMemsetAsync(d32.p, 0, vb, c->stream));
    const double tin = std::max(0.3 * tol / res, 3e-5);
    int its = 0;
    double tr_in = 0;
    const int cap_in = std::min(max_iter - it_total, std::max(2 * restart, 40));
    int rci = gmres_core(c, r32.p, d32.p, tin, cap_in, restart, &its, &tr_in, hist, res, &nh, true);
    it_total += its;
    if (rci && rci != PRD_E_NOCONV) { rc = rci; break; }
    f2d_add_kernel<<<G, 256, 0, c->stream>>>((const float*)d32.p, (double*)x64.p, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
  }
  if (!rc) {
    d2f_kernel<<<G, 256, 0, c->stream>>>((const double*)x64.p, (float*)x, n);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = fail(c, PRD_E_CUDA, cudaGetErrorString(e));
  }
  if (iters) *iters = it_total;
  if (true_res) *true_res = res;
  cleanup();
  if (rc) return rc;
  if (status != PRD_OK) return fail(c, PRD_E_NOCONV, "refined GMRES reached max_iter before tol");
  return PRD_OK;
}

// Adjoint solve A^T lam = g (S13): GMRES in the ctx precision on the FP64
// transposed operator, left-preconditioned with the forward P^-1 (any fixed
// linear map keeps GMRES exact; it only changes the iteration count).
int solve_adjoint(Ctx* c, const void* g, double tol, int max_iter, int restart, void* lam, int* iters,
                  double* true_res, double* hist) {
  PRD_CUDA_TRY(c, cudaMemsetAsync(lam, 0, nvec(c) * c->esz, c->stream));
  c->op_transpose = true;
  const int rc = gmres_core(c, g, lam, tol, max_iter, restart, iters, true_res, hist, 1.0, nullptr);
  c->op_transpose = false;
  return rc;
}

}  // namespace prd
