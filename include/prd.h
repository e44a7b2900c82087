/*
 * prd.h -- C ABI of the GB300 (sm_103a) library for the matrix-free AD-PRD
 * operator of polarised non-LTE radiative transfer with a fixed lower-level
 * population (Riva et al., arXiv 2505.20968).
 *
 * The unknown is the discrete Stokes field I[z][Omega][nu][s] (s = I,Q,U,V;
 * Sect. 2.6: N = 4 N_r N_nu N_Omega), heights ascending, directions ordered
 * Omega = i_mu * N_chi + i_chi with mu ascending, frequencies ascending in the
 * reduced frequency u = (nu0 - nu)/dnu_D.  The library solves
 *     (Id - Lambda Sigma) I = Lambda eps_th + t                (Eq. linear_system)
 * with Lambda the DELO-linear (or DELOPAR) formal solution (Sect. 3) and Sigma the
 * comoving-frame R_II-AD + R_III scattering operator (Eqs. eps_sc_l,
 * RQIIKKp, RIIIQKKp, eps_sc_bar; Sect. 4; App. B, E).
 *
 * Conventions of every call:
 *   - returns PRD_OK (0) or a negative PRD_E_* code; prd_last_error() gives a
 *     one-line reason.  No C++ exception crosses this boundary.
 *   - host arrays are read during the call and copied; the caller keeps them.
 *   - "device" pointers are caller-owned CUDA allocations on the ctx's device,
 *     contiguous, layout [z][Omega][nu][4], element type double for
 *     PRD_FP64 and float for the FP32 precisions, starting on a whole Stokes point
 *     (address a multiple of 4 elements: 32 bytes in FP64, 16 in FP32;
 *     otherwise PRD_E_ARG, as the kernels move one point per access).  The
 *     library never frees them.
 *   - the library owns its workspace (cudaMalloc at prd_setup and at the
 *     first solve, or the caller's allocator of prd_set_allocator; freed at
 *     prd_destroy or at the next prd_setup).
 *   - work is issued on the ctx stream (prd_set_stream, default: the legacy
 *     stream) and is asynchronous, except prd_setup, prd_solve and calls that
 *     return host scalars, which synchronise the stream.
 *   - a ctx is not thread-safe: use one ctx per host thread.
 */
#ifndef PRD_H
#define PRD_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PRD_OK = 0,
  PRD_E_ARG = -1,        /* invalid argument (null pointer, size, range)   */
  PRD_E_STATE = -2,      /* call out of order (e.g. apply before setup)    */
  PRD_E_CUDA = -3,       /* CUDA runtime error                              */
  PRD_E_NOMEM = -4,      /* device allocation failed                        */
  PRD_E_NOCONV = -5,     /* solver hit max_iter before tol                  */
  PRD_E_BREAKDOWN = -6,  /* Arnoldi breakdown (h_{j+1,j} ~ 0)               */
  PRD_E_NAN = -7,        /* NaN/Inf in a solver quantity                    */
  PRD_E_TIMEOUT = -8     /* a bounded device wait expired                   */
};

/* Precision of a context.  PRD_FP64: every table, vector and product in
 * FP64.  PRD_FP32: FP32 tables and vectors with FP64 reductions and an FP64
 * residual refinement in prd_solve; the R_II contraction runs on the tcgen05
 * tensor cores as 3xTF32 split products (<= 3 * 2^-22 per product).
 * PRD_FP32_BF16X3: the same, with split-BF16 products (hi*hi + hi*lo + lo*hi
 * of bf16 halves, <= 3 * 2^-18 per product, twice the TF32 tensor rate); the
 * context is a PRD_FP32 context (vectors are float) whose R_II tiles are
 * stored split into bf16 hi and lo planes in the operand layout of the MMA
 * (the same bytes as FP32), so its contraction is BF16x3 on the tensor cores
 * only: PRD_OPT_CONTRACTION = TF32X3 and PRD_OPT_TENSOR_CORES = 0 return
 * PRD_E_ARG.  A PRD_FP32 context can also run BF16x3 (PRD_OPT_CONTRACTION),
 * splitting its FP32 tiles on the fly.
 * PRD_FP32_BF16X2: the same with the tiles stored as the bf16 hi plane alone
 * (half the bytes of FP32) and two products per element, hi(B)*hi(A) +
 * lo(B)*hi(A): the tile's rounding to bf16 (<= 2^-9 relative) is kept, so the
 * contraction is a ~1e-3-accurate inner operator; prd_solve's FP64 residuals
 * (FP64 table copy) still check the solution, and where the scattering
 * amplifies that error by more than its inverse (the Mg II case) the
 * refinement stalls and prd_solve returns PRD_E_NOCONV. */
enum { PRD_FP64 = 0, PRD_FP32 = 1, PRD_FP32_BF16X3 = 2, PRD_FP32_BF16X2 = 3 };
enum { PRD_TWO_LEVEL = 0, PRD_TWO_TERM = 1 };
enum { PRD_GRID_LAMBDA = 0, PRD_GRID_X = 1 };
enum { PRD_MU_GL_HEMISPHERES = 0, PRD_MU_GL_FULL = 1 };
enum { PRD_MODE_AD = 0, PRD_MODE_AA = 1 };

typedef struct prd_ctx prd_ctx;

/* Atomic model (Sect. 2.2, Table 1).  Lower term L=0 (unpolarised, sharp),
 * upper term L=1 with spin S = twoS/2 (twoS = 0: two-level atom J 0->1;
 * twoS = 1: S_1/2 -> P_1/2,3/2 two-term atom with J-state interference and
 * Paschen-Back levels).  E_u_cm: upper J-level energies in cm^-1 (J = L-S
 * first; for twoS = 0 only E_u_cm[0] is used).  nu0_hz = 0 selects the
 * (2J+1)-weighted centroid as the reference frequency nu0 (Sect. 2.4). */
typedef struct {
  int kind;          /* PRD_TWO_LEVEL or PRD_TWO_TERM (must agree with twoS) */
  int twoS;          /* 0 or 1 */
  double E_u_cm[2];
  double mass_amu;   /* atomic mass, Doppler width (Sect. 6.1) */
  double g_s;        /* electron spin g factor (2.0) */
  double nu0_hz;     /* 0 -> centroid */
} prd_atom;

/* Create a context on CUDA device `device` with arithmetic `precision`
 * (PRD_FP64, PRD_FP32, PRD_FP32_BF16X3 or PRD_FP32_BF16X2).  *out receives the handle (NULL
 * on failure). */
int prd_create(prd_ctx** out, int device, int precision);
/* Free the context and all library-owned device memory.  NULL is a no-op. */
int prd_destroy(prd_ctx* ctx);
/* Static one-line description of the last error on this ctx (never NULL). */
const char* prd_last_error(const prd_ctx* ctx);
/* Issue all further work on this cudaStream_t (passed as a pointer). */
int prd_set_stream(prd_ctx* ctx, void* cuda_stream);
/* Device memory of the library from the caller's allocator (e.g. a caching
 * allocator of the host framework) instead of cudaMalloc/cudaFree.
 * alloc(bytes, user, stream) returns a device pointer of at least `bytes`
 * bytes on the ctx device, 256-byte aligned, usable on `stream` (the ctx
 * stream at the time of the call), or NULL on failure (-> PRD_E_NOMEM); a
 * pointer that is not 256-byte aligned is handed back to free and the call
 * that needed it fails with PRD_E_ARG; free(ptr, user) releases it.  Both NULL: back to cudaMalloc/cudaFree.  Every
 * buffer is released with the deallocator it was obtained from, so the call
 * can come at any time; set it before prd_setup to route the workspace
 * (tiles and tables) through it.  prd_apply_sigma_noalloc allocates nothing
 * either way. */
typedef void* (*prd_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void (*prd_free_fn)(void* ptr, void* user);
int prd_set_allocator(prd_ctx* ctx, prd_alloc_fn alloc, prd_free_fn free_fn, void* user);

/* Sect. 2.2 / Table 1. */
int prd_set_atom(prd_ctx* ctx, const prd_atom* atom);

/* Atmosphere on nz >= 2 heights (Sects. 2.3-2.5, 6.1), each array of
 * length nz except v_kms [nz][3]:
 *   z_km ascending; T_K; xi_kms microturbulence; a damping constant
 *   (Gamma_R+Gamma_I+Gamma_E)/(4 pi dnu_D); eps = Gamma_I/(Gamma_R+Gamma_I)
 *   (photon destruction); r_el = Gamma_E/(Gamma_R+Gamma_I+Gamma_E) (< 1);
 *   k_line: frequency-integrated line absorption coefficient of the fixed
 *   lower population in km^-1 per unit reduced frequency (eta_I = k_line phi(u)
 *   at B = 0); W_T Wien (Planck) function; B_G field strength in gauss,
 *   thetaB/chiB its inclination/azimuth (rad, vertical z axis); v_kms bulk
 *   velocity (x, y, z). */
int prd_set_atmosphere(prd_ctx* ctx, int nz, const double* z_km, const double* T_K,
                       const double* xi_kms, const double* a, const double* eps,
                       const double* r_el, const double* k_line, const double* W_T,
                       const double* B_G, const double* thetaB, const double* chiB,
                       const double* v_kms);

/* Continuum processes (App. A), optional: per height and frequency, arrays
 * [nz][nnu] of the continuum absorption kappa_c and scattering sigma_c
 * coefficients (km^-1, as k_line) and the thermal continuum emissivity.
 * kappa_c + sigma_c adds to the diagonal of K (no continuum dichroism or
 * dispersion), the thermal emissivity to Stokes I, and sigma_c scatters
 * coherently in the observer frame with the dipole phase matrix:
 *     eps_c(Omega, nu) = sigma_c(nu) oint P(Omega, Omega') I(Omega', nu) dOmega'/4pi.
 * The Kirchhoff factor f normalises the line emissivity alone.  Call after
 * prd_set_atmosphere and prd_set_quadrature and before prd_setup; three
 * NULLs remove the continuum.  The transposed operator, the adjoint solve and
 * prd_grad_B are built without continuum and return PRD_E_STATE with it. */
int prd_set_continuum(prd_ctx* ctx, const double* kappa_c, const double* sigma_c, const double* eps_c_th);

/* Frequency and angular quadrature (Sects. 2.6, 4.2, 4.3).  grid: nnu ascending
 * values, vacuum wavelengths in Angstrom (PRD_GRID_LAMBDA) or reduced
 * frequencies x with nu = nu0 - x dnu_D(z_0) (PRD_GRID_X).  mu_rule
 * PRD_MU_GL_HEMISPHERES puts n_mu_half Gauss-Legendre nodes on each of
 * [-1,0] and [0,1]; PRD_MU_GL_FULL puts 2 n_mu_half nodes on [-1,1].  chi is
 * the trapezoidal rule with n_chi nodes chi_k = 2 pi k/n_chi.  mode
 * PRD_MODE_AD (angle-dependent R_II) or PRD_MODE_AA (Eq. R_AA). */
int prd_set_quadrature(prd_ctx* ctx, int nnu, const double* grid, int grid_kind,
                       int n_mu_half, int n_chi, int mu_rule, int mode);

/* Build every table and the R_II tiles on the device (setup, Sect. 4; App. C,
 * E, F): Doppler widths, Paschen-Back states, branching ratios (App. B),
 * propagation matrices, DELO-linear weights, redistribution tiles against the
 * natural-spline basis, Kirchhoff normalisation f (App. E), block-Jacobi
 * inverses (App. F).  Synchronous.  Re-callable after set_* changes. */
int prd_setup(prd_ctx* ctx);

/* Problem sizes after setup: heights, directions, frequencies, scattering-
 * angle classes (incl. Theta = 0) and the vector length n = 4 nz nO nnu. */
int prd_sizes(const prd_ctx* ctx, int* nz, int* n_omega, int* nnu, int* n_theta,
              int64_t* n);
/* Copy the direction grid (mu, chi, weights; host arrays of length n_omega). */
int prd_directions(const prd_ctx* ctx, double* mu, double* chi, double* w);
/* Bytes of device memory the library holds: tiles and tables from setup, plus
 * the solver workspace kept after the first prd_solve / prd_solve_adjoint
 * (Krylov basis, device state) and the transposed operator's scratch. */
int prd_workspace_bytes(const prd_ctx* ctx, int64_t* bytes);
/* Work of one R_II contraction (Eq. G summed over the tiles of every class,
 * Sect. 4): *flops = 2 x (real multiply-adds of Re(T Z) over all heights,
 * classes, tiles, rows n, columns k < 2N and Stokes outputs), *bytes = tile
 * bytes read once per apply.  Either pointer may be NULL.  For roofline
 * accounting; PRD_E_STATE before prd_setup. */
int prd_contraction_work(const prd_ctx* ctx, double* flops, double* bytes);

/* b = Lambda eps_th + t  (right-hand side of Eq. linear_system). */
int prd_rhs(prd_ctx* ctx, void* b_dev);
/* eps = Sigma x: normalised line scattering emissivity (Eq. eps_sc_l in the
 * comoving frame, Eq. eps_sc_bar; intensity scaled by f, App. E). */
int prd_apply_sigma(prd_ctx* ctx, const void* x_dev, void* eps_dev);
/* out = Lambda eps: DELO-linear formal solution, zero boundary (Sect. 3). */
int prd_apply_lambda(prd_ctx* ctx, const void* eps_dev, void* out_dev);
/* y = (Id - Lambda Sigma) x  (one operator apply, Eq. linear_system). */
int prd_apply_operator(prd_ctx* ctx, const void* x_dev, void* y_dev);
/* y = (Id - Lambda Sigma)^T x = x - Sigma^T Lambda^T x: the transpose of the
 * discrete operator of Eq. linear_system (adjoint of the linear system for
 * gradients of functionals of I w.r.t. the atmosphere, Sect. 5 setting).  Each
 * stage is transposed exactly (reverse DELO sweep, transposed splines, R_II
 * tiles and R_III factors); arithmetic is FP64.  x, y: ctx-precision device
 * vectors [z][Omega][nu][4], distinct.  In FP32 mode it uses the FP64 copy of
 * the Sigma tables and returns PRD_E_STATE if that copy was not kept (too
 * little device memory at setup).  Synchronises the ctx stream. */
int prd_apply_operator_T(prd_ctx* ctx, const void* x_dev, void* y_dev);
/* Gradient of a functional J of the solution I with respect to the magnetic
 * field of every height: dJ_dp[z*3 + 0..2] = dJ/dB_z [1/G], dJ/dtheta_B,z,
 * dJ/dchi_B,z [1/rad].  x_dev: the solution of A I = b (ctx precision);
 * dJdI_dev: dJ/dI at x (ctx precision, [z][Omega][nu][4]).  Adjoint method on
 * Eq. linear_system: one adjoint solve A^T lam = dJ/dI (tol 1e-10), then
 * dJ/dp = lam^T (db/dp - (dA/dp) I) with the parameter derivative taken as a
 * central difference of b - A I, each side a full FP64 setup of the perturbed
 * atmosphere (6 setups per height: meant for reduced problems).  Steps: 1e-3
 * relative, 0.1 G for B = 0 (one-sided there), 1e-3 rad for angles at 0.  The
 * paper solves forward problems only; it has no gradient.  Synchronises. */
int prd_grad_B(prd_ctx* ctx, const void* x_dev, const void* dJdI_dev, double* dJ_dp);
/* Batched solve of n independent problems (ragged sizes allowed: one ctx per
 * instance, each set up beforehand).  Instance i is solved as by prd_solve
 * (x0 = 0, tolerance, iteration and restart limits shared) into x_devs[i], on
 * its own host thread and its own ctx stream, so the instances overlap on the
 * GPU when their streams differ.  iters, true_rel_res and rcs are arrays of n
 * (rcs[i] = prd_solve's return code for instance i; any may be NULL).  Returns
 * PRD_OK if every instance succeeded, else the first failing code.  The ctxs
 * must be distinct and not used by other threads during the call.  The paper
 * solves one atmosphere at a time; batching is the throughput form of its
 * per-atmosphere solve (Sect. 5). */
int prd_solve_batch(prd_ctx* const* ctxs, int n, double tol, int max_iter, int restart, void* const* x_devs,
                    int* iters, double* true_rel_res, int* rcs);
/* Adjoint solve (Id - Lambda Sigma)^T lam = g by restarted GMRES on
 * prd_apply_operator_T, left-preconditioned with the forward preconditioner
 * (a fixed linear map).  Arguments as prd_solve, with the right-hand side g
 * given; lam starts from zero.  PRD_E_NOCONV if tol is not reached. */
int prd_solve_adjoint(prd_ctx* ctx, const void* g_dev, double tol, int max_iter, int restart, void* lam_dev,
                      int* iters, double* true_rel_res, double* res_history);
/* x = P^-1 y, P = Id - Lambda* Sigma* on Stokes I (identity on Q,U,V):
 * Sigma* unpolarised, unmagnetised PRD-AA; m_in block-Jacobi-preconditioned
 * Richardson sweeps from zero (Sect. 5.2, App. F). */
int prd_apply_preconditioner(prd_ctx* ctx, const void* y_dev, void* x_dev);
/* Set the number of inner sweeps m_in (>= 1, default 3) of the preconditioner. */
int prd_set_precond_sweeps(prd_ctx* ctx, int m_in);

/* Options.  PRD_OPT_TENSOR_CORES (FP32 only): 1 runs the R_II contraction on
 * the tcgen05 tensor cores (TMA-fed tiles, TMEM accumulators, 3xTF32 split
 * products), 0 on the CUDA cores.  PRD_OPT_PRECOND_SWEEPS: m_in as above.
 * PRD_OPT_WAIT_POLLS: poll limit of the tensor-core contraction's pipeline
 * waits (0: the default, 2^24 polls, about a second).  A wait that runs out
 * makes its thread block stop, drain the copies and products it issued
 * (those waits keep the default limit) and report PRD_E_TIMEOUT through
 * prd_device_status; the output of that apply is invalid and the context
 * stays usable.  A small limit is for testing that failure path.
 * PRD_OPT_TEST_ZERO_OPERATOR: 1 makes prd_solve and prd_solve_adjoint iterate
 * with the zero map instead of the operator (failure injection: the first
 * Arnoldi step breaks down and an unconverged solve returns PRD_E_BREAKDOWN);
 * 0 restores the operator.
 * PRD_OPT_REFINE_FLOOR (FP32 mode): the floor of the relative tolerance of
 * each inner FP32 GMRES solve of the mixed-precision refinement, in units of
 * 1e-8 (default 3000: 3e-5); the inner tolerance is max(0.3 tol / res, floor)
 * with res the current FP64 relative residual.  It trades outer FP64
 * residuals against inner iterations, never the accuracy of the result.
 * PRD_OPT_FORMAL_SOLVER: PRD_DELO_LINEAR (default; the source vector and the
 * K'I term linear over a step) or PRD_DELOPAR (Sect. 3: the source vector
 * parabolic through the upwind, current and downwind points, K'I linear;
 * linear on the last step of a ray).  Both are linear in the emissivity, so
 * GMRES applies to either; every formal solution (Lambda, the right-hand
 * side, emergent Stokes vectors, the refinement residuals) uses the choice.
 * The transposed operator, the adjoint solve and prd_grad_B are built for
 * DELO-linear and return PRD_E_STATE under PRD_DELOPAR.
 * PRD_OPT_CONTRACTION (FP32 contexts): the split products of the tensor-core
 * R_II contraction, PRD_CONTRACTION_TF32X3 (the PRD_FP32 default) or
 * PRD_CONTRACTION_BF16X3 (the PRD_FP32_BF16X3 default).  prd_solve's FP64
 * residuals do not use the contraction, so the solution's accuracy is the
 * same with either; the inner iterations count changes.
 * PRD_OPT_TILE_STAGES: depth of the contraction's tile ring, 2..5 (capped at
 * the deepest that fits in shared memory beside the resident I~) or 0 for
 * that deepest ring (default); a schedule parameter for measured tuning.
 * PRD_OPT_GRAPH: 1 (default) runs each GMRES iteration of prd_solve,
 * prd_solve_adjoint and prd_solve_batch as one launch of a CUDA graph (the
 * Arnoldi step: operator, preconditioner, both Gram-Schmidt passes, the
 * rotation kernel and the next basis vector, with the step index kept on the
 * device), captured on the first iteration and kept with the solver's
 * workspace; 0 launches the same kernels one by one.  Results are identical.
 * Any option change, prd_set_precond_sweeps and prd_setup drop the captured
 * graphs; stage profiling (prd_set_profiling) runs the kernels one by one.
 * PRD_OPT_STAGED_SWEEP: 1 (default) runs the formal solution of the operator
 * and of prd_apply_lambda / prd_rhs with the heights' inputs streamed into
 * shared memory by bulk asynchronous copies (a ring of 8 heights per block of
 * 128 rays) when the frequency count is even; 0, or an odd count, runs one
 * thread per ray reading its inputs directly.  Results are identical.  Its
 * waits are bounded like the contraction's (PRD_E_TIMEOUT through
 * prd_device_status).
 * PRD_OPT_GRAD_FULL_SETUP: 0 (default) makes prd_grad_B difference each
 * height's residual by re-setting up only that height's Sigma rows (a context
 * of two heights) and the formal solver's tables of the perturbed atmosphere;
 * 1 takes a full FP64 setup of the perturbed atmosphere per side.  Both
 * difference the same residual with the same steps. */
enum { PRD_OPT_TENSOR_CORES = 1, PRD_OPT_PRECOND_SWEEPS = 2, PRD_OPT_WAIT_POLLS = 3, PRD_OPT_TEST_ZERO_OPERATOR = 4,
       PRD_OPT_REFINE_FLOOR = 5, PRD_OPT_FORMAL_SOLVER = 6, PRD_OPT_CONTRACTION = 7, PRD_OPT_TILE_STAGES = 8,
       PRD_OPT_GRAPH = 9, PRD_OPT_STAGED_SWEEP = 10, PRD_OPT_GRAD_FULL_SETUP = 11 };
enum { PRD_CONTRACTION_TF32X3 = 0, PRD_CONTRACTION_BF16X3 = 1 };
enum { PRD_DELO_LINEAR = 0, PRD_DELOPAR = 1 };
int prd_set_option(prd_ctx* ctx, int option, int value);
/* Number of CUDA-graph launches of the GMRES step made by this context so far
 * (each is one whole Arnoldi iteration); *n receives it.  PRD_E_ARG on NULL. */
int prd_graph_launches(const prd_ctx* ctx, int64_t* n);
/* Synchronise the ctx stream and report device-side failures: a CUDA error,
 * or PRD_E_TIMEOUT if a bounded wait inside a kernel expired since the last
 * call (the kernel then returned early and its output is invalid). */
int prd_device_status(prd_ctx* ctx);

/* Left-preconditioned restarted GMRES(restart) (Sect. 5.1-5.2) from x0_dev
 * (NULL = zero) into x_dev; stops when the unpreconditioned relative residual
 * ||b - A x||/||b|| < tol (checked in FP64).  *iters receives the number of
 * operator applies, *true_rel_res the final FP64 residual; res_history (NULL
 * or max_iter+1 doubles) the preconditioned residual estimate per iteration.
 * Returns PRD_E_NOCONV if max_iter is reached, PRD_E_BREAKDOWN /
 * PRD_E_NAN on those events (x_dev then holds the last iterate). */
int prd_solve(prd_ctx* ctx, double tol, int max_iter, int restart, const void* x0_dev,
              void* x_dev, int* iters, double* true_rel_res, double* res_history);

/* Emergent Stokes vectors at z_max along nlos lines of sight (mu > 0, any
 * chi) that need not be on the grid (Sect. 6.2, extra formal solution):
 * a scattering emissivity is built for each new direction from the solution
 * x_dev, then one DELO sweep.  out_dev: [nlos][nnu][4] device array. */
int prd_emergent_stokes(prd_ctx* ctx, const void* x_dev, int nlos, const double* mu,
                        const double* chi, void* out_dev);

/* Wavelength-integrated narrow-band Stokes signals (Sect. 6.5, centre-to-limb
 * variation): for each line of sight (mu in (0, 1], any chi) the emergent
 * Stokes profiles of the solution x_dev (as prd_emergent_stokes) weighted by a
 * Gaussian of full width at half maximum fwhm_A centred on lambda0_A and
 * integrated over [lambda0_A - half_width_A, lambda0_A + half_width_A]
 * (Angstrom, vacuum), normalised by 1/(sqrt(2 pi) sigma):
 *     out[l][s] = 1/(sqrt(2 pi) sigma) int exp(-(lambda - lambda0)^2/(2 sigma^2)) X_s(mu_l, lambda) dlambda.
 * X between the wavelength nodes is its natural cubic spline in lambda and
 * beyond the grid its end value.  out: host array [nlos][4] (I, Q, U, V),
 * FP64.  Synchronous.  PRD_E_ARG for fwhm or half width <= 0 or mu outside
 * (0, 1]. */
int prd_narrowband(prd_ctx* ctx, const void* x_dev, int nlos, const double* mu, const double* chi,
                   double lambda0_A, double fwhm_A, double half_width_A, double* out);

/* Same result as prd_apply_sigma, for callers that must not allocate device
 * memory at call time: code that runs while another framework owns the
 * allocator, inside allocation-free real-time or replay loops, or in
 * environments where cudaMalloc is not permitted after initialisation.  This
 * call allocates nothing (no cudaMalloc/cudaFree, no allocating library call):
 * its intermediates (comoving field, spline second derivatives, comoving
 * emissivity, R_III moments) live in one static device array of 64 MiB that
 * every GPU which loads the library holds until the process exits.  A problem
 * whose intermediates need more than 64 MiB is rejected with PRD_E_ARG.  Each
 * call looks up the array's device address in the current context (no
 * allocation; it stays valid if the device is reset in between); the first
 * call on a device may load the library's device code, so make it before any
 * stream capture.  Every call shares the array and overwrites it, so calls
 * that overlap on the GPU (other streams, other contexts on the same device)
 * race.  PRD_OK means the work was queued: in FP32 mode the tensor-core
 * contraction reports an expired bounded wait only through
 * prd_device_status, which the caller checks after the stream completes, as
 * for prd_apply_sigma.  The paper has no counterpart: this is a deployment
 * variant of the Sigma apply. */
int prd_apply_sigma_noalloc(prd_ctx* ctx, const void* x_dev, void* eps_dev);

/* Stage timing (tracing).  When on, CUDA events recorded on the ctx stream
 * bracket each stage of every apply; prd_stage_times returns the accumulated
 * milliseconds and call counts per stage (index 0: S1 comoving interpolation,
 * 1: S5 R_III, 2: S3+S4 R_II contraction, 3: S6 back-interpolation and f,
 * 4: S7+S8 formal solution) and synchronises the stream.  Turning it on or
 * off resets the counters. */
int prd_set_profiling(prd_ctx* ctx, int on);
int prd_stage_times(prd_ctx* ctx, double* ms, int64_t* count, int n);

#ifdef __cplusplus
}
#endif
#endif /* PRD_H */
