// C ABI entry points (include/prd.h): argument checks, ordering, setup
// orchestration.  No exception leaves this file.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include "prd_internal.h"

namespace prd {

int fail(Ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int dalloc(Ctx* c, DBuf& b, size_t bytes) {
  dfree(b);
  if (bytes == 0) bytes = 16;
  if (c->alloc_fn) {
    b.p = c->alloc_fn(bytes, c->alloc_user, (void*)c->stream);
    if (!b.p) return fail(c, PRD_E_NOMEM, "the caller's allocator returned NULL for " + std::to_string(bytes) + " bytes");
    if (reinterpret_cast<uintptr_t>(b.p) & 255u) {   // bulk copies and vector loads need the alignment
      c->free_fn(b.p, c->alloc_user);
      b.p = nullptr;
      return fail(c, PRD_E_ARG, "the caller's allocator returned a pointer that is not 256-byte aligned");
    }
    b.fr = c->free_fn;
    b.user = c->alloc_user;
    b.bytes = bytes;
    return PRD_OK;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail(c, PRD_E_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  b.fr = nullptr;
  b.user = nullptr;
  b.bytes = bytes;
  return PRD_OK;
}

void dfree(DBuf& b) {
  if (b.p) {
    if (b.fr) b.fr(b.p, b.user);
    else cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
  b.fr = nullptr;
  b.user = nullptr;
}

int upload(Ctx* c, DBuf& b, const void* host, size_t bytes) {
  int rc = dalloc(c, b, bytes);
  if (rc) return rc;
  PRD_CUDA_TRY(c, cudaMemcpy(b.p, host, bytes, cudaMemcpyHostToDevice));
  return PRD_OK;
}

static void free_all(Ctx* c) {
  DBuf* bufs[] = {&c->tiles, &c->Y, &c->r3w, &c->r3in, &c->r3out, &c->r3prof, &c->r3J, &c->r3ab, &c->kt,
                  &c->epsth, &c->f, &c->sp, &c->ugrid, &c->iin, &c->ibk, &c->tin, &c->tbk, &c->cls_dev, &c->dmu,
                  &c->scratch1, &c->scratch2, &c->scratch3, &c->pc_phi, &c->pc_M, &c->pc_lii, &c->pc_eta,
                  &c->pc_delo, &c->pc_s1, &c->pc_s2, &c->pc_s3, &c->pc_s4, &c->pc_s5, &c->gm_w, &c->gm_r, &c->gm_t, &c->gm_dots,
                  &c->tc_err, &c->tc_work, &c->tiles64, &c->Y64, &c->r3w64, &c->r3in64, &c->r3out64,
                  &c->r3prof64, &c->r3ab64, &c->par, &c->eta_line, &c->cont_pw, &c->cont_sig,
                  &c->gk_V, &c->gk_r, &c->gk_w, &c->gk_cur, &c->gk_S, &c->kt64, &c->epsth64};
  invalidate_graphs(c);
  c->gk_m = 0;
  c->has64 = false;
  c->tc_ready = false;
  for (DBuf* b : bufs) dfree(*b);
  for (auto& b : c->adj) dfree(b);
  for (auto& b : c->krylov) dfree(b);
  c->krylov.clear();
  for (auto& b : c->owned) dfree(b);
  c->owned.clear();
}

void stage_begin(Ctx* c, int stage, cudaEvent_t* out) {
  *out = nullptr;
  if (!c->prof) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, c->stream);
  *out = e;
}

void stage_end(Ctx* c, int stage, cudaEvent_t start) {
  if (!c->prof || !start) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, c->stream);
  c->ev_pending.push_back({stage, {start, e}});
}

void stage_collect(Ctx* c) {
  for (auto& p : c->ev_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.second.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
      c->stage_ms[p.first] += ms;
      c->stage_n[p.first] += 1;
    }
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  c->ev_pending.clear();
}

Ctx::~Ctx() {
  stage_collect(this);
  free_all(this);
  if (gk_host) cudaFreeHost(gk_host);
  if (gk_cap) cudaStreamDestroy(gk_cap);
}

int launch_precond_setup(Ctx* c);

static int setup(Ctx* c) {
  c->ready = false;
  free_all(c);
  int rc = build_host_tables(c);
  if (rc) return rc;
  if (c->lambda_only) {
    // the field gradient's perturbed formal solver: K, DELO weights, thermal emissivity
    if ((rc = upload(c, c->dmu, c->mu.data(), c->mu.size() * 8)) || (rc = build_device_tables(c)) ||
        (rc = r2_tc_prepare(c)))
      return rc;
    PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->ready = true;
    return PRD_OK;
  }
  // memory check for the tiles
  const size_t tile_bytes = (size_t)c->nz * c->ncls * c->ntile() * c->nnu * c->ld() * c->tile_esz();
  size_t fr = 0, tot = 0;
  PRD_CUDA_TRY(c, cudaMemGetInfo(&fr, &tot));
  if (tile_bytes > fr * 0.9)
    return fail(c, PRD_E_NOMEM, "R_II tiles need " + std::to_string(tile_bytes >> 20) + " MiB, device has " +
                                    std::to_string(fr >> 20) + " MiB free");
  if ((rc = dalloc(c, c->tiles, tile_bytes))) return rc;
  PRD_CUDA_TRY(c, cudaMemset(c->tiles.p, 0, tile_bytes));   // row padding (ld > 2N) stays zero
  const int nq = c->nu_st * c->nu_st * c->nl_st;
  if ((rc = dalloc(c, c->r3w, (size_t)c->nz * nq * 2 * c->nnu * c->esz))) return rc;
  // FP64 Sigma tables for the refinement residuals (FP32 mode), if they fit with room to spare
  if (c->prec == PRD_FP32) {
    const size_t t64 = (size_t)c->nz * c->ncls * c->ntile() * c->nnu * c->ld64() * 8;
    PRD_CUDA_TRY(c, cudaMemGetInfo(&fr, &tot));
    if (t64 < fr * 0.6) {
      if ((rc = dalloc(c, c->tiles64, t64))) return rc;
      if ((rc = dalloc(c, c->r3w64, (size_t)c->nz * nq * 2 * c->nnu * 8))) return rc;
      c->has64 = true;
    }
  }
  if ((rc = upload(c, c->dmu, c->mu.data(), c->mu.size() * 8))) return rc;
  if ((rc = build_device_tables(c))) return rc;
  if ((rc = dalloc(c, c->gm_t, nvec(c) * c->esz))) return rc;
  if ((rc = launch_tiles(c))) return rc;
  if ((rc = r2_tc_prepare(c))) return rc;
  if ((rc = compute_normalisation(c))) return rc;
  if ((rc = launch_precond_setup(c))) return rc;
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->ready = true;
  return PRD_OK;
}

}  // namespace prd

using prd::Ctx;
using prd::fail;


#define CTX_OR_ARG(ctx)                 \
  if (!(ctx)) return PRD_E_ARG;         \
  Ctx* c = &(ctx)->c;                   \
  cudaSetDevice(c->device);

#define NEED_READY()                                              \
  if (!c->ready) return fail(c, PRD_E_STATE, "call prd_setup first");

#define NEED_ALIGNED(p)                 \
  if (!prd::point_aligned(c, (p)))      \
    return fail(c, PRD_E_ARG, #p " does not start on a whole Stokes point (4 elements)");

extern "C" {

int prd_create(prd_ctx** out, int device, int precision) {
  if (!out) return PRD_E_ARG;
  *out = nullptr;
  if (precision != PRD_FP64 && precision != PRD_FP32 && precision != PRD_FP32_BF16X3 &&
      precision != PRD_FP32_BF16X2)
    return PRD_E_ARG;
  const bool bf16x2 = precision == PRD_FP32_BF16X2;
  const bool bf16x3 = precision == PRD_FP32_BF16X3 || bf16x2;
  if (bf16x3) precision = PRD_FP32;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return PRD_E_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return PRD_E_CUDA;
  prd_ctx* h = new (std::nothrow) prd_ctx();
  if (!h) return PRD_E_NOMEM;
  h->c.device = device;
  h->c.prec = precision;
  h->c.esz = precision == PRD_FP64 ? 8 : 4;
  h->c.use_tc = precision == PRD_FP32 ? 1 : 0;   // tcgen05 contraction by default in FP32
  h->c.tc_bf16 = bf16x3 ? 1 : 0;
  h->c.split_tiles = bf16x3;                    // tiles stored as bf16 planes (hi and lo, or hi only)
  h->c.hi_only = bf16x2;
  if (cudaDeviceGetAttribute(&h->c.nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete h;
    return PRD_E_CUDA;
  }
  *out = h;
  return PRD_OK;
}

int prd_destroy(prd_ctx* ctx) {
  if (!ctx) return PRD_OK;
  cudaSetDevice(ctx->c.device);
  delete ctx;
  return PRD_OK;
}

const char* prd_last_error(const prd_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null ctx"; }

int prd_set_stream(prd_ctx* ctx, void* stream) {
  CTX_OR_ARG(ctx);
  c->stream = (cudaStream_t)stream;
  return PRD_OK;
}

int prd_set_allocator(prd_ctx* ctx, prd_alloc_fn alloc, prd_free_fn free_fn, void* user) {
  CTX_OR_ARG(ctx);
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(c, PRD_E_ARG, "give both alloc and free, or neither");
  c->alloc_fn = alloc;
  c->free_fn = free_fn;
  c->alloc_user = user;
  return PRD_OK;
}

int prd_set_atom(prd_ctx* ctx, const prd_atom* atom) {
  CTX_OR_ARG(ctx);
  if (!atom) return fail(c, PRD_E_ARG, "atom is NULL");
  if (!(atom->twoS == 0 || atom->twoS == 1)) return fail(c, PRD_E_ARG, "twoS must be 0 or 1");
  if (atom->kind != (atom->twoS == 0 ? PRD_TWO_LEVEL : PRD_TWO_TERM))
    return fail(c, PRD_E_ARG, "kind must be PRD_TWO_LEVEL for twoS=0 and PRD_TWO_TERM for twoS=1");
  if (!(atom->mass_amu > 0) || !(atom->E_u_cm[0] > 0) || (atom->twoS == 1 && !(atom->E_u_cm[1] > 0)))
    return fail(c, PRD_E_ARG, "mass and energies must be positive");
  c->atom = *atom;
  if (c->atom.g_s == 0.0) c->atom.g_s = 2.0;
  c->have_atom = true;
  c->ready = false;
  return PRD_OK;
}

int prd_set_atmosphere(prd_ctx* ctx, int nz, const double* z_km, const double* T_K, const double* xi_kms,
                       const double* a, const double* eps, const double* r_el, const double* k_line,
                       const double* W_T, const double* B_G, const double* thetaB, const double* chiB,
                       const double* v_kms) {
  CTX_OR_ARG(ctx);
  if (nz < 2) return fail(c, PRD_E_ARG, "nz must be >= 2");
  const double* arrs[] = {z_km, T_K, xi_kms, a, eps, r_el, k_line, W_T, B_G, thetaB, chiB, v_kms};
  for (const double* p : arrs)
    if (!p) return fail(c, PRD_E_ARG, "atmosphere array is NULL");
  for (int i = 0; i < nz; ++i) {
    if (i > 0 && !(z_km[i] > z_km[i - 1])) return fail(c, PRD_E_ARG, "z_km must be strictly ascending");
    if (!(T_K[i] > 0) || !(a[i] > 0) || !(k_line[i] > 0) || !(W_T[i] >= 0) || !(eps[i] >= 0 && eps[i] < 1) ||
        !(r_el[i] >= 0 && r_el[i] < 1) || !(B_G[i] >= 0) || !std::isfinite(xi_kms[i]))
      return fail(c, PRD_E_ARG, "atmosphere value out of range at height " + std::to_string(i));
  }
  c->nz = nz;
  c->z.assign(z_km, z_km + nz);
  c->T.assign(T_K, T_K + nz);
  c->xi.assign(xi_kms, xi_kms + nz);
  c->a.assign(a, a + nz);
  c->eps.assign(eps, eps + nz);
  c->rE.assign(r_el, r_el + nz);
  c->k.assign(k_line, k_line + nz);
  c->WT.assign(W_T, W_T + nz);
  c->B.assign(B_G, B_G + nz);
  c->thB.assign(thetaB, thetaB + nz);
  c->chB.assign(chiB, chiB + nz);
  c->v.assign(v_kms, v_kms + 3 * nz);
  c->have_atm = true;
  c->ready = false;
  return PRD_OK;
}

int prd_set_quadrature(prd_ctx* ctx, int nnu, const double* grid, int grid_kind, int n_mu_half, int n_chi,
                       int mu_rule, int mode) {
  CTX_OR_ARG(ctx);
  if (nnu < 4 || nnu > 256 || !grid) return fail(c, PRD_E_ARG, "nnu must be in [4, 256] and grid non-NULL");
  if (grid_kind != PRD_GRID_LAMBDA && grid_kind != PRD_GRID_X) return fail(c, PRD_E_ARG, "bad grid_kind");
  if (n_mu_half < 1 || n_mu_half > 32 || n_chi < 1 || n_chi > 64) return fail(c, PRD_E_ARG, "bad angular sizes");
  if (mu_rule != PRD_MU_GL_HEMISPHERES && mu_rule != PRD_MU_GL_FULL) return fail(c, PRD_E_ARG, "bad mu_rule");
  if (mode != PRD_MODE_AD && mode != PRD_MODE_AA) return fail(c, PRD_E_ARG, "bad mode");
  for (int i = 1; i < nnu; ++i)
    if (!(grid[i] > grid[i - 1])) return fail(c, PRD_E_ARG, "grid must be strictly ascending");
  c->nnu = nnu;
  c->grid.assign(grid, grid + nnu);
  c->grid_kind = grid_kind;
  c->n_mu_half = n_mu_half;
  c->n_chi = n_chi;
  c->mu_rule = mu_rule;
  c->mode = mode;
  c->have_quad = true;
  c->ready = false;
  return PRD_OK;
}

int prd_set_continuum(prd_ctx* ctx, const double* kappa_c, const double* sigma_c, const double* eps_c_th) {
  CTX_OR_ARG(ctx);
  if (!kappa_c && !sigma_c && !eps_c_th) {
    c->kapc.clear(); c->sigc.clear(); c->epsc.clear();
    c->ready = false;
    return PRD_OK;
  }
  if (!kappa_c || !sigma_c || !eps_c_th) return fail(c, PRD_E_ARG, "continuum: give all three arrays or none");
  if (!c->have_atm || !c->have_quad) return fail(c, PRD_E_STATE, "continuum: set the atmosphere and quadrature first");
  const size_t n = (size_t)c->nz * c->nnu;
  for (size_t i = 0; i < n; ++i)
    if (!(kappa_c[i] >= 0) || !(sigma_c[i] >= 0) || !(eps_c_th[i] >= 0))
      return fail(c, PRD_E_ARG, "continuum coefficients must be finite and non-negative");
  c->kapc.assign(kappa_c, kappa_c + n);
  c->sigc.assign(sigma_c, sigma_c + n);
  c->epsc.assign(eps_c_th, eps_c_th + n);
  c->cont_nz = c->nz;
  c->cont_nnu = c->nnu;
  c->ready = false;
  return PRD_OK;
}

int prd_setup(prd_ctx* ctx) {
  CTX_OR_ARG(ctx);
  if (!c->have_atom || !c->have_atm || !c->have_quad)
    return fail(c, PRD_E_STATE, "set_atom, set_atmosphere and set_quadrature must precede setup");
  if (c->grid_kind == PRD_GRID_LAMBDA && !(c->grid[0] > 0)) return fail(c, PRD_E_ARG, "wavelengths must be positive");
  if (c->has_cont() && (c->cont_nz != c->nz || c->cont_nnu != c->nnu))
    return fail(c, PRD_E_STATE, "continuum arrays were set for another atmosphere or frequency grid");
  try {
    return prd::setup(c);
  } catch (const std::exception& e) {
    return fail(c, PRD_E_NOMEM, std::string("host exception in setup: ") + e.what());
  }
}

int prd_sizes(const prd_ctx* ctx, int* nz, int* n_omega, int* nnu, int* n_theta, int64_t* n) {
  if (!ctx) return PRD_E_ARG;
  const Ctx* c = &ctx->c;
  if (!c->ready) return PRD_E_STATE;
  if (nz) *nz = c->nz;
  if (n_omega) *n_omega = c->nO;
  if (nnu) *nnu = c->nnu;
  if (n_theta) *n_theta = c->ncls;
  if (n) *n = (int64_t)prd::nvec(c);
  return PRD_OK;
}

int prd_directions(const prd_ctx* ctx, double* mu, double* chi, double* w) {
  if (!ctx) return PRD_E_ARG;
  const Ctx* c = &ctx->c;
  if (!c->ready) return PRD_E_STATE;
  for (int o = 0; o < c->nO; ++o) {
    if (mu) mu[o] = c->mu[o];
    if (chi) chi[o] = c->chi[o];
    if (w) w[o] = c->wang[o];
  }
  return PRD_OK;
}

int prd_workspace_bytes(const prd_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return PRD_E_ARG;
  const Ctx* c = &ctx->c;
  const prd::DBuf* bufs[] = {&c->tiles, &c->Y, &c->r3w, &c->r3in, &c->r3out, &c->r3prof, &c->r3J, &c->r3ab,
                             &c->kt, &c->kt64, &c->epsth64, &c->epsth, &c->f, &c->sp, &c->ugrid, &c->iin, &c->ibk,
                             &c->tin, &c->tbk,
                             &c->cls_dev, &c->scratch1, &c->scratch2, &c->scratch3, &c->pc_phi, &c->pc_M,
                             &c->pc_lii, &c->pc_eta, &c->pc_delo, &c->gm_t, &c->dmu, &c->pc_s1, &c->pc_s2,
                             &c->pc_s3, &c->pc_s4, &c->pc_s5, &c->tc_err, &c->tc_work, &c->tiles64, &c->Y64, &c->r3w64, &c->r3in64,
                             &c->r3out64, &c->r3prof64, &c->r3ab64, &c->par, &c->eta_line, &c->cont_pw,
                             &c->cont_sig, &c->gm_w, &c->gk_V, &c->gk_r, &c->gk_w, &c->gk_cur, &c->gk_S};
  int64_t s = 0;
  for (auto* b : bufs) s += (int64_t)b->bytes;
  for (const auto& b : c->adj) s += (int64_t)b.bytes;   // scratch of the transposed operator, once used
  *bytes = s;
  return PRD_OK;
}

int prd_contraction_work(const prd_ctx* ctx, double* flops, double* bytes) {
  if (!ctx) return PRD_E_ARG;
  const Ctx* c = &ctx->c;
  if (!c->ready) return PRD_E_STATE;
  const double N = c->nnu, per_tile_out = (double)c->ntile() * N * 2.0 * N;   // tile elements per class
  double outs = 0;                                                               // Stokes outputs per class
  for (int k = 0; k < c->ncls; ++k) outs += 4.0 * (c->cout_ptr[k + 1] - c->cout_ptr[k]);
  if (flops) *flops = 2.0 * c->nz * per_tile_out * outs;
  if (bytes) *bytes = (double)c->nz * c->ncls * per_tile_out * c->tile_esz();
  return PRD_OK;
}

int prd_rhs(prd_ctx* ctx, void* b_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!b_dev) return fail(c, PRD_E_ARG, "b_dev is NULL");
  NEED_ALIGNED(b_dev);
  return prd::rhs(c, b_dev);
}

int prd_apply_sigma(prd_ctx* ctx, const void* x_dev, void* eps_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!x_dev || !eps_dev || x_dev == eps_dev) return fail(c, PRD_E_ARG, "x_dev/eps_dev NULL or aliased");
  NEED_ALIGNED(x_dev);
  NEED_ALIGNED(eps_dev);
  return prd::apply_sigma(c, x_dev, eps_dev, true);
}

int prd_apply_lambda(prd_ctx* ctx, const void* eps_dev, void* out_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!eps_dev || !out_dev || eps_dev == out_dev) return fail(c, PRD_E_ARG, "eps_dev/out_dev NULL or aliased");
  NEED_ALIGNED(eps_dev);
  NEED_ALIGNED(out_dev);
  return prd::apply_lambda(c, eps_dev, out_dev, nullptr, false);
}

int prd_apply_operator(prd_ctx* ctx, const void* x_dev, void* y_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!x_dev || !y_dev || x_dev == y_dev) return fail(c, PRD_E_ARG, "x_dev/y_dev NULL or aliased");
  NEED_ALIGNED(x_dev);
  NEED_ALIGNED(y_dev);
  return prd::apply_operator(c, x_dev, y_dev);
}

int prd_apply_preconditioner(prd_ctx* ctx, const void* y_dev, void* x_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!x_dev || !y_dev || x_dev == y_dev) return fail(c, PRD_E_ARG, "x_dev/y_dev NULL or aliased");
  NEED_ALIGNED(x_dev);
  NEED_ALIGNED(y_dev);
  return prd::apply_precond(c, y_dev, x_dev);
}

int prd_set_precond_sweeps(prd_ctx* ctx, int m_in) {
  CTX_OR_ARG(ctx);
  if (m_in < 0 || m_in > 64) return fail(c, PRD_E_ARG, "m_in must be in [0, 64]");
  prd::invalidate_graphs(c);
  c->m_in = m_in;
  return PRD_OK;
}

int prd_graph_launches(const prd_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return PRD_E_ARG;
  *n = ctx->c.gk_launches;
  return PRD_OK;
}

int prd_solve(prd_ctx* ctx, double tol, int max_iter, int restart, const void* x0_dev, void* x_dev, int* iters,
              double* true_rel_res, double* res_history) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!x_dev || !(tol > 0) || max_iter < 1 || restart < 1) return fail(c, PRD_E_ARG, "bad solve arguments");
  NEED_ALIGNED(x0_dev);
  NEED_ALIGNED(x_dev);
  try {
    int rc = prd::solve(c, tol, max_iter, restart, x0_dev, x_dev, iters, true_rel_res, res_history);
    if (c->tc_err.p) {
      const int rt = prd::r2_tc_check_error(c);
      if (rt) return rt;
    }
    return rc;
  } catch (const std::exception& e) {
    return fail(c, PRD_E_NOMEM, std::string("host exception in solve: ") + e.what());
  }
}

int prd_grad_B(prd_ctx* ctx, const void* x_dev, const void* dJdI_dev, double* dJ_dp) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (c->formal != PRD_DELO_LINEAR)
    return fail(c, PRD_E_STATE, "the transposed operator is built for the DELO-linear formal solver");
  if (c->has_cont()) return fail(c, PRD_E_STATE, "the transposed operator is built without continuum");
  if (!x_dev || !dJdI_dev || !dJ_dp) return fail(c, PRD_E_ARG, "NULL argument");
  NEED_ALIGNED(x_dev);
  NEED_ALIGNED(dJdI_dev);
  try {
    return prd::grad_b(c, x_dev, dJdI_dev, 1e-10, dJ_dp);
  } catch (const std::exception& e) {
    c->op_transpose = false;
    return fail(c, PRD_E_NOMEM, std::string("host exception in gradient: ") + e.what());
  }
}

int prd_solve_batch(prd_ctx* const* ctxs, int n, double tol, int max_iter, int restart, void* const* x_devs,
                    int* iters, double* true_rel_res, int* rcs) {
  if (!ctxs || !x_devs || n < 1 || !(tol > 0) || max_iter < 1 || restart < 1) return PRD_E_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !x_devs[i]) return PRD_E_ARG;
    if (!prd::point_aligned(&ctxs[i]->c, x_devs[i]))
      return fail(&ctxs[i]->c, PRD_E_ARG, "x_devs[i] does not start on a whole Stokes point (4 elements)");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return PRD_E_ARG;
  }
  std::vector<int> rc(n, PRD_OK), it(n, 0);
  std::vector<double> res(n, 0.0);
  // lockstep rounds (one graph launch runs every waiting instance's Arnoldi
  // step) when all instances sit on one device; else each replays its own graph
  bool one_device = true;
  for (int i = 1; i < n; ++i) one_device = one_device && ctxs[i]->c.device == ctxs[0]->c.device;
  prd::BatchRound* round = nullptr;
  if (one_device && n > 1) {
    cudaSetDevice(ctxs[0]->c.device);
    round = prd::batch_round_create(n);
  }
  for (int i = 0; i < n; ++i) ctxs[i]->c.batch = round;
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      Ctx* c = &ctxs[i]->c;
      auto leave = [&]() {
        if (c->batch) prd::batch_round_leave(c->batch);
        c->batch = nullptr;
      };
      if (!c->ready) { rc[i] = fail(c, PRD_E_STATE, "call prd_setup first"); leave(); return; }
      if (cudaSetDevice(c->device) != cudaSuccess) { rc[i] = fail(c, PRD_E_CUDA, "cudaSetDevice failed"); leave(); return; }
      try {
        rc[i] = prd::solve(c, tol, max_iter, restart, nullptr, x_devs[i], &it[i], &res[i], nullptr);
        leave();
        if (!rc[i] && c->tc_err.p) rc[i] = prd::r2_tc_check_error(c);
      } catch (const std::exception& e) {
        leave();
        rc[i] = fail(c, PRD_E_NOMEM, std::string("host exception in solve: ") + e.what());
      }
    });
  for (auto& t : th) t.join();
  prd::batch_round_destroy(round);
  int first = PRD_OK;
  for (int i = 0; i < n; ++i) {
    if (iters) iters[i] = it[i];
    if (true_rel_res) true_rel_res[i] = res[i];
    if (rcs) rcs[i] = rc[i];
    if (first == PRD_OK && rc[i] != PRD_OK) first = rc[i];
  }
  return first;
}

int prd_apply_operator_T(prd_ctx* ctx, const void* x_dev, void* y_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (c->formal != PRD_DELO_LINEAR)
    return fail(c, PRD_E_STATE, "the transposed operator is built for the DELO-linear formal solver");
  if (c->has_cont()) return fail(c, PRD_E_STATE, "the transposed operator is built without continuum");
  if (!x_dev || !y_dev) return fail(c, PRD_E_ARG, "NULL vector");
  NEED_ALIGNED(x_dev);
  NEED_ALIGNED(y_dev);
  try {
    return prd::apply_operator_t(c, x_dev, y_dev);
  } catch (const std::exception& e) {
    return fail(c, PRD_E_NOMEM, std::string("host exception: ") + e.what());
  }
}

int prd_solve_adjoint(prd_ctx* ctx, const void* g_dev, double tol, int max_iter, int restart, void* lam_dev,
                      int* iters, double* true_rel_res, double* res_history) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (c->formal != PRD_DELO_LINEAR)
    return fail(c, PRD_E_STATE, "the transposed operator is built for the DELO-linear formal solver");
  if (c->has_cont()) return fail(c, PRD_E_STATE, "the transposed operator is built without continuum");
  if (!g_dev || !lam_dev || !(tol > 0) || max_iter < 1 || restart < 1)
    return fail(c, PRD_E_ARG, "bad adjoint solve arguments");
  NEED_ALIGNED(g_dev);
  NEED_ALIGNED(lam_dev);
  try {
    return prd::solve_adjoint(c, g_dev, tol, max_iter, restart, lam_dev, iters, true_rel_res, res_history);
  } catch (const std::exception& e) {
    c->op_transpose = false;
    return fail(c, PRD_E_NOMEM, std::string("host exception in adjoint solve: ") + e.what());
  }
}

int prd_emergent_stokes(prd_ctx* ctx, const void* x_dev, int nlos, const double* mu, const double* chi,
                        void* out_dev) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!x_dev || !out_dev || nlos < 1 || !mu || !chi) return fail(c, PRD_E_ARG, "bad emergent_stokes arguments");
  NEED_ALIGNED(x_dev);
  NEED_ALIGNED(out_dev);
  for (int i = 0; i < nlos; ++i)
    if (!(mu[i] > 0 && mu[i] <= 1)) return fail(c, PRD_E_ARG, "line-of-sight mu must be in (0, 1]");
  try {
    return prd::emergent(c, x_dev, nlos, mu, chi, out_dev);
  } catch (const std::exception& e) {
    return fail(c, PRD_E_NOMEM, std::string("host exception: ") + e.what());
  }
}

int prd_narrowband(prd_ctx* ctx, const void* x_dev, int nlos, const double* mu, const double* chi, double lambda0_A,
                   double fwhm_A, double half_width_A, double* out) {
  CTX_OR_ARG(ctx);
  NEED_READY();
  if (!x_dev || !out || nlos < 1 || !mu || !chi) return fail(c, PRD_E_ARG, "bad narrowband arguments");
  if (!(fwhm_A > 0) || !(half_width_A > 0) || !std::isfinite(lambda0_A))
    return fail(c, PRD_E_ARG, "narrowband needs fwhm > 0, half width > 0 and a finite centre");
  NEED_ALIGNED(x_dev);
  for (int i = 0; i < nlos; ++i)
    if (!(mu[i] > 0 && mu[i] <= 1)) return fail(c, PRD_E_ARG, "line-of-sight mu must be in (0, 1]");
  try {
    return prd::narrowband(c, x_dev, nlos, mu, chi, lambda0_A, fwhm_A, half_width_A, out);
  } catch (const std::exception& e) {
    return fail(c, PRD_E_NOMEM, std::string("host exception: ") + e.what());
  }
}

int prd_set_option(prd_ctx* ctx, int option, int value) {
  CTX_OR_ARG(ctx);
  prd::invalidate_graphs(c);   // the captured solver step bakes in every option
  if (option == PRD_OPT_GRAPH) {
    c->use_graph = value ? 1 : 0;
    return PRD_OK;
  }
  if (option == PRD_OPT_STAGED_SWEEP) {
    c->staged_sweep = value ? 1 : 0;
    return PRD_OK;
  }
  if (option == PRD_OPT_GRAD_FULL_SETUP) {
    c->grad_full_setup = value ? 1 : 0;
    return PRD_OK;
  }
  if (option == PRD_OPT_TENSOR_CORES) {
    if (value && c->prec != PRD_FP32) return fail(c, PRD_E_ARG, "tensor-core contraction needs PRD_FP32");
    if (!value && c->split_tiles)
      return fail(c, PRD_E_ARG, "PRD_FP32_BF16X3 stores its tiles as bf16 planes for the tensor cores only");
    c->use_tc = value ? 1 : 0;
    return PRD_OK;
  }
  if (option == PRD_OPT_PRECOND_SWEEPS) {
    if (value < 0 || value > 64) return fail(c, PRD_E_ARG, "m_in must be in [0, 64]");
    c->m_in = value;
    return PRD_OK;
  }
  if (option == PRD_OPT_WAIT_POLLS) {
    if (value < 0) return fail(c, PRD_E_ARG, "poll limit must be >= 0");
    c->tc_spin = value;
    return PRD_OK;
  }
  if (option == PRD_OPT_REFINE_FLOOR) {
    if (value < 1 || value > 1000000) return fail(c, PRD_E_ARG, "refinement floor must be in [1, 1e6] x 1e-8");
    c->refine_floor = value * 1e-8;
    return PRD_OK;
  }
  if (option == PRD_OPT_FORMAL_SOLVER) {
    if (value != PRD_DELO_LINEAR && value != PRD_DELOPAR) return fail(c, PRD_E_ARG, "unknown formal solver");
    c->formal = value;
    return PRD_OK;
  }
  if (option == PRD_OPT_CONTRACTION) {
    if (value != PRD_CONTRACTION_TF32X3 && value != PRD_CONTRACTION_BF16X3)
      return fail(c, PRD_E_ARG, "unknown contraction product");
    if (c->prec != PRD_FP32) return fail(c, PRD_E_ARG, "the split products are for PRD_FP32 contexts");
    if (c->split_tiles && value != PRD_CONTRACTION_BF16X3)
      return fail(c, PRD_E_ARG, "PRD_FP32_BF16X3/X2 store their tiles as bf16 planes: their own products only");
    c->tc_bf16 = value == PRD_CONTRACTION_BF16X3 ? 1 : 0;
    return PRD_OK;
  }
  if (option == PRD_OPT_TILE_STAGES) {
    if (value != 0 && (value < 2 || value > 5)) return fail(c, PRD_E_ARG, "tile stages must be 0 or in [2, 5]");
    c->tc_stages = value;
    return PRD_OK;
  }
  if (option == PRD_OPT_TEST_ZERO_OPERATOR) {
    c->test_zero_op = value ? 1 : 0;
    return PRD_OK;
  }
  return fail(c, PRD_E_ARG, "unknown option");
}

int prd_device_status(prd_ctx* ctx) {
  CTX_OR_ARG(ctx);
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  PRD_CUDA_TRY(c, cudaGetLastError());
  if (c->tc_err.p) return prd::r2_tc_check_error(c);
  return PRD_OK;
}

int prd_set_profiling(prd_ctx* ctx, int on) {
  CTX_OR_ARG(ctx);
  prd::stage_collect(c);
  c->prof = on != 0;
  for (int i = 0; i < 8; ++i) { c->stage_ms[i] = 0; c->stage_n[i] = 0; }
  return PRD_OK;
}

int prd_stage_times(prd_ctx* ctx, double* ms, int64_t* count, int n) {
  CTX_OR_ARG(ctx);
  if (!ms || n < 1) return fail(c, PRD_E_ARG, "bad stage_times arguments");
  prd::stage_collect(c);
  for (int i = 0; i < n && i < 8; ++i) {
    ms[i] = c->stage_ms[i];
    if (count) count[i] = c->stage_n[i];
  }
  return PRD_OK;
}

}  // extern "C"
