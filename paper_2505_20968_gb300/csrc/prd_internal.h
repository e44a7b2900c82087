// Internal declarations shared by the library's translation units (host C++
// and CUDA).  Nothing here is part of the C ABI (include/prd.h).
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/prd.h"

namespace prd {

using cplx = std::complex<double>;

// physical constants (CODATA 2018), library copy
constexpr double kC = 2.99792458e8;            // m/s
constexpr double kKB = 1.380649e-23;           // J/K
constexpr double kAMU = 1.66053906660e-27;     // kg
constexpr double kMuBoverH = 1.39962449361e10; // Hz/T
constexpr double kGauss = 1e-4;                // T/G
constexpr double kCmToHz = 2.99792458e10;
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;

constexpr int kWeidemanN64 = 36;   // Faddeeva expansion terms, FP64 paths
constexpr int kWeidemanN32 = 20;   // Faddeeva expansion terms, FP32 paths
// Angle-averaged R_II (Eq. R_AA): composite Gauss-Legendre in Theta with this
// many nodes on each of [0, pi/2] and [pi/2, pi]
constexpr int kAAThetaNodes = 48;

// device buffer with byte size
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  prd_free_fn fr = nullptr;     // caller's deallocator (NULL: cudaFree)
  void* user = nullptr;
};

struct Ctx {
  int device = 0;
  int nsm = 1;                  // streaming multiprocessors of the device (queried at create)
  // grid of the grid-stride elementwise and reduction kernels: 4 CTAs per SM
  int grid_ew() const { return 4 * (nsm > 0 ? nsm : 1); }
  int prec = PRD_FP32;
  size_t esz = 4;               // element size of vectors (4 or 8)
  cudaStream_t stream = nullptr;
  std::string err = "ok";

  // ---- inputs
  bool have_atom = false, have_atm = false, have_quad = false, ready = false;
  prd_atom atom{};
  int nz = 0;
  std::vector<double> z, T, xi, a, eps, rE, k, WT, B, thB, chB, v;
  // continuum (App. A), [z][nu] each, empty if none: absorption, scattering, thermal emissivity
  std::vector<double> kapc, sigc, epsc;
  bool has_cont() const { return !sigc.empty(); }
  int cont_nz = 0, cont_nnu = 0;      // sizes the continuum arrays were given for
  int nnu = 0;
  std::vector<double> grid;
  int grid_kind = 0, n_mu_half = 0, n_chi = 0, mu_rule = 0, mode = 0;
  int m_in = 3;   // preconditioner sweeps (the fastest Mg II solve of a sweep over 1..3)

  // ---- derived on host
  int nO = 0;
  std::vector<double> mu, chi, wang;
  int ncls = 0;                       // scattering-angle classes (class 0: Theta = 0)
  std::vector<double> theta;          // per class
  std::vector<int> cls;               // [o][o'] class index
  // per class: output directions (CSR) and, per output direction, input dirs
  std::vector<int> cout_ptr, cout_dir;    // cout_ptr[c]..cout_ptr[c+1]
  std::vector<int> pair_ptr, pair_in;     // per (class, out-entry): pairs
  int npairs = 0, max_cout = 0;
  int nu_st = 0, nl_st = 0;             // upper / lower states
  int ntrip = 0;                         // R_II triples (k, kl, kl')
  std::vector<int> trip_k, trip_l, trip_lp;
  // Tiles are stored as one mean tile per group of triples whose upper state
  // belongs to the same J level, followed by each triple's deviation from it
  // (tile index ti < ngrp: group mean; ti = ngrp + t: deviation of triple t).
  int ngrp = 1;
  std::vector<int> trip_grp;
  int ntile() const { return ngrp + ntrip; }
  // Stored tile row length: FP32 tiles are kept in the tensor-core layout of
  // tile_off (the Re and Im halves each padded to a multiple of 16 columns,
  // K chunks of 16, each a contiguous [n][16] block), FP64 tiles as plain rows
  // of 2N rounded up to 4; so every row or chunk starts on 16 bytes.
  bool tiled() const { return prec == PRD_FP32; }
  int np16() const { return (nnu + 15) / 16 * 16; }
  int ld() const { return tiled() ? 2 * np16() : (2 * nnu + 3) / 4 * 4; }
  int nq3 = 0;                           // R_III incident combos (ku, kv, kl)
  double nu0 = 0;
  std::vector<double> dnuD, vD;          // per z (Hz, km/s)
  std::vector<double> u;                 // [z][n]
  std::vector<double> ub;                // [z][o]
  std::vector<double> shift;             // [z][ku][kl]
  std::vector<cplx> alpha, beta;         // [z][ku][kv]
  std::vector<cplx> amp;                 // [z][o][2][ku][kl]
  std::vector<double> Dmat;              // [z][3][ku][kl] dipole elements <ku|d_q|kl>
  std::vector<double> Rmag;              // [z][3][3] rows of the magnetic frame
  std::vector<double> Q;                 // [z][n][n] natural-spline 2nd-derivative map
  std::vector<int> theta_node_cls;       // AA: unused
  int n_aa_theta = 0;
  std::vector<double> aa_theta, aa_w;     // AA Theta rule

  // ---- device
  // FP32 mode keeps an FP64 copy of the Sigma tables (plain tile layout) for the
  // residuals of the mixed-precision refinement, when it fits (has64)
  DBuf tiles64, Y64, r3w64, r3in64, r3out64, r3prof64, r3ab64;
  bool has64 = false;
  bool op_transpose = false;   // GMRES iterates with A^T (adjoint solve)
  int test_zero_op = 0;        // GMRES iterates with the zero map (failure injection for tests)
  double refine_floor = 3e-5;  // FP32 refinement: floor of the inner GMRES relative tolerance
  int ld64() const { return (2 * nnu + 3) / 4 * 4; }
  DBuf tiles;        // [z][c][t][n][2N]    (T)
  DBuf Y;            // [z][pair][t][16]    complex (T2)
  DBuf r3w;          // [z][q3][N] complex  (T2)  R_III incident weights
  DBuf r3in;         // [z][o'][q3][4] complex: w_o' * I_j(o'; ku, kv, kl)
  DBuf r3out;        // [z][o][uv][kl'][4] complex: O_i(o; ku, kv, kl') * c
  DBuf r3prof;       // [z][uv][kl'][N] complex: outgoing profile
  DBuf r3J;          // [z][uv] complex scratch
  DBuf r3ab;         // [z][uv] complex (beta-alpha) * k * c3
  DBuf kt;           // [z][o][n][10] K'/eta1 (6), 1/eta1, exp(-d), alpha, beta
  // FP32 mode: FP64 copies of kt and epsth for the refinement's FP64 residuals,
  // the right-hand side and f (the formal solution of the residual operator
  // then carries no FP32 table rounding)
  DBuf kt64, epsth64;
  DBuf adj[7];       // scratch of the transposed operator (allocated on first use)
  DBuf par;          // [z][o][n][3] DELOPAR source weights psi_M, psi_O, psi_P of the step arriving there (double)
  DBuf eta_line;     // [z][o][n] the line's share eta_line/eta_total of eta_I (double): f normalises the line only
  DBuf cont_pw;      // [o][o'][4][4] w_o' P(o, o') dipole phase matrix of continuum scattering (double)
  DBuf cont_sig;     // [z][n] sigma_c (double)
  int formal = 0;    // formal solver: 0 DELO-linear, 1 DELOPAR (PRD_OPT_FORMAL_SOLVER)
  const void* par_active() const { return formal ? par.p : nullptr; }
  DBuf epsth;        // [z][o][n][4]
  DBuf f;            // [z][o][n]
  DBuf sp;           // spline tables: per z  h[N-1], cp[N], den[N]  (T) -> [z][3][N]
  DBuf ugrid;        // [z][N] (T)
  DBuf iin, ibk;     // interpolation [z][o][n]: int k | flag, and t (T)  -> int2/ T pairs
  DBuf tin, tbk;
  DBuf cls_dev;      // cout_ptr, cout_dir, pair_ptr, pair_in  (int)
  DBuf dmu;          // [nO] mu of each direction (double)
  DBuf scratch1, scratch2, scratch3;  // N-vector scratch (T)
  // preconditioner
  DBuf pc_phi;       // [z][N][N] Phi_bar (double)
  DBuf pc_M;         // [z][N][N] Phi_bar (Id - A)^-1 (double)
  DBuf pc_lii;       // [z][o][n] Lambda_ii (T)
  DBuf pc_eta;       // [z][o][n]: eta1 (T)  (scalar Lambda*)
  DBuf pc_delo;      // [z][o][n][3] (T)
  DBuf pc_s1, pc_s2, pc_s3, pc_s4, pc_s5;   // FP64 N-vector scratch of the sweeps
  std::vector<double> pc_lii_host;
  void* pc_w = nullptr;   // device angular weights (double), owned via `owned`
  // GMRES
  std::vector<DBuf> krylov;
  DBuf gm_w, gm_r, gm_t, gm_dots;
  // GMRES workspace kept across solves (basis V[m+1], residual r, operator
  // output w, current basis vector, device state), and the Arnoldi step
  // captured once as a CUDA graph over it: [0] A, [1] A^T
  DBuf gk_V, gk_r, gk_w, gk_cur, gk_S;
  int gk_m = 0;
  double* gk_host = nullptr;               // pinned copy of the step's scalars
  cudaGraphExec_t gk_exec[2] = {nullptr, nullptr};
  cudaGraph_t gk_graph[2] = {nullptr, nullptr};   // the captured steps (children of a batch round)
  int use_graph = 1;                       // PRD_OPT_GRAPH
  int staged_sweep = 1;                    // PRD_OPT_STAGED_SWEEP: bulk-copy-staged formal solution
  // internal context of the field gradient holding only the formal solver's
  // tables (no Sigma tables, tiles, normalisation or preconditioner)
  bool lambda_only = false;
  int grad_full_setup = 0;                 // PRD_OPT_GRAD_FULL_SETUP
  cudaStream_t gk_cap = nullptr;           // private stream the step is captured on
  struct BatchRound* batch = nullptr;      // set while prd_solve_batch runs this context in lockstep
  long long gk_launches = 0;               // graph launches (prd_graph_launches)
  std::vector<DBuf> owned;
  prd_alloc_fn alloc_fn = nullptr;   // caller's allocator (prd_set_allocator), NULL: cudaMalloc
  prd_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  // tensor-core contraction (r2_tc.cu)
  DBuf tc_err;
  DBuf tc_work;      // tcgen05 contraction work items: (class, first output entry) pairs
  int tc_nwork = 0;
  bool tc_ready = false;
  int use_tc = 0;
  long long tc_spin = 0;   // poll limit of the contraction's pipeline waits (0: the default)
  int tc_bf16 = 0;         // contraction products: 0 3xTF32, 1 split-BF16 (BF16x3)
  bool split_tiles = false;   // PRD_FP32_BF16X3/X2: R_II tiles stored as bf16 planes (tile_off_split)
  bool hi_only = false;       // PRD_FP32_BF16X2: the hi plane only (tile_off_hi), two products
  // bytes of one stored tile element (tile_bytes / elements of the padded layout)
  size_t tile_esz() const { return hi_only ? 2 : esz; }
  int tc_stages = 0;       // tile ring depth of the contraction (0: the deepest that fits)
  // stage timing (prd_set_profiling): events on the ctx stream around each stage
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long stage_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  ~Ctx();
};

// Caller vectors [z][Omega][nu][4] are moved one Stokes point (4 elements) per
// access, so each must start on a multiple of 4 * esz bytes (NULL passes).
inline bool point_aligned(const Ctx* c, const void* p) {
  return !p || reinterpret_cast<uintptr_t>(p) % (4 * c->esz) == 0;
}

// ---- errors
int fail(Ctx* c, int code, const std::string& msg);
#define PRD_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess)                                                          \
      return ::prd::fail((ctx), PRD_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

int dalloc(Ctx* c, DBuf& b, size_t bytes);
void dfree(DBuf& b);
int upload(Ctx* c, DBuf& b, const void* host, size_t bytes);

// ---- host math (host_math.cpp)
cplx faddeeva_host(cplx z);
void weideman_coeffs(int n, double* a_out, double* L_out);
void natural_spline_Q(const double* u, int n, double* Q);
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// ---- setup pieces (host_setup.cpp)
int build_host_tables(Ctx* c);
int build_device_tables(Ctx* c);
int emissivity_acc(Ctx* c, const double* x, double* eps, double* ws);
// polarisation amplitudes a[alpha][ku][kl] = <ku| e_alpha . d |kl> of any direction
void dir_amplitudes(const Ctx* c, int iz, double mu, double chi, cplx* out);
// tables of one extra line of sight (emergent_stokes)
struct LosTables {
  std::vector<double> Y;       // [z][nO][ntile][32]  pairs (LOS, o')
  std::vector<double> theta;   // [z? no: nO]  scattering angle LOS-o'
  std::vector<double> rout;    // [z][nuv][nl][4][2]
  std::vector<double> kt;      // [z][N][10]
  std::vector<double> par;     // [z][N][3]  DELOPAR source weights
  std::vector<double> eta_line;   // [z][N]  the line's share eta_line/eta_total of eta_I
  std::vector<double> cont_pw;    // [nO][4][4]  w_o' P(LOS, o') (continuum scattering)
  std::vector<double> epsth;   // [z][N][4]
  std::vector<int> kidx;       // [z][N]   back-interpolation intervals
  std::vector<double> tt;      // [z][N]
};
void los_tables(const Ctx* c, double mu, double chi, LosTables& L);
int gen_tiles_z(Ctx* c, int iz, const std::vector<double>& thetas, void* outT);
// DELOPAR source weights of a step of optical thickness dM followed downwind by dP
void delopar_weights(double dM, double dP, double* psi);
// dipole (Rayleigh) phase matrix P[4][4] from direction (mu_p, chi_p) into (mu_o, chi_o)
void dipole_phase(double mu_o, double chi_o, double mu_p, double chi_p, double* P);
// eps[z][o][n] += sigma_c sum_o' w_o' P(o, o') x[z][o'][n] (continuum scattering, App. A)
int add_continuum_scattering(Ctx* c, const void* x, void* eps, bool fp64_vectors);

// ---- device launchers (kernels_*.cu)
int launch_tiles(Ctx* c);
int launch_setup_tables(Ctx* c);   // normalisation etc. (needs apply)
int apply_sigma(Ctx* c, const void* x, void* eps, bool normalised);
int apply_lambda(Ctx* c, const void* eps, void* out, const void* sub_from, bool boundary);
int apply_operator(Ctx* c, const void* x, void* y);
int apply_precond(Ctx* c, const void* y, void* x);
int apply_operator_t(Ctx* c, const void* x, void* y);   // y = A^T x (FP64 arithmetic)
int solve_adjoint(Ctx* c, const void* g, double tol, int max_iter, int restart, void* lam, int* iters,
                  double* true_res, double* hist);
int grad_b(Ctx* c, const void* x, const void* dJdI, double tol, double* dJdp);
int compute_normalisation(Ctx* c);
int rhs(Ctx* c, void* b);
int solve(Ctx* c, double tol, int max_iter, int restart, const void* x0, void* x, int* iters,
          double* true_res, double* hist);
int emergent(Ctx* c, const void* x, int nlos, const double* mu, const double* chi, void* out);
int narrowband(Ctx* c, const void* x, int nlos, const double* mu, const double* chi, double lam0, double fwhm,
               double half, double* out);
int upload_faddeeva_coeffs(Ctx* c);

size_t nvec(const Ctx* c);   // 4*nz*nO*nnu
int r2_tc_prepare(Ctx* c);
int r2_tc_launch(Ctx* c, const float* Ic, float* eb);
// drop the captured solver graphs (options, tables or workspace changed)
void invalidate_graphs(Ctx* c);
// Lockstep rounds of a batched solve (solver.cu): every context of the batch
// that is inside an Arnoldi step waits until all contexts still solving have
// either reached their step or left; then one launch of a graph whose
// children are their captured steps runs all of them.
BatchRound* batch_round_create(int n);
void batch_round_leave(BatchRound* b);
void batch_round_destroy(BatchRound* b);
int r2_tc_check_error(Ctx* c);

// Stage ids for prd_stage_times.
enum Stage { ST_S1 = 0, ST_S5 = 1, ST_S3 = 2, ST_S6 = 3, ST_S7 = 4, ST_PRE = 5 };
// Begin / end a timed stage (no-ops unless profiling is on).
void stage_begin(Ctx* c, int stage, cudaEvent_t* out);
void stage_end(Ctx* c, int stage, cudaEvent_t start);
void stage_collect(Ctx* c);

// Offset of tile element (row n, column k in [0, 2N): Re | Im halves) within
// one tile of N rows.  Plain layout: n * ld + k.  Tensor-core layout (FP32,
// ld = 2 NP with NP = N rounded up to 16): column k sits at kp = k in the Re
// half and kp = NP + k - N in the Im half (the columns N..NP-1 of each half
// stay zero), so no K chunk mixes the halves; the tile is cut into K chunks of
// 16 columns of kp, chunk kc a contiguous block of N rows of 64 bytes, each
// row's four 16-byte groups permuted by the 64-byte shared-memory swizzle of
// its row index (group g stored at g ^ ((n >> 1) & 3)), so one bulk copy of
// N * 64 bytes lands a K step in the operand layout.
__host__ __device__ inline int tile_col(int k, int N, int NP) { return k < N ? k : NP + (k - N); }
__host__ __device__ inline size_t tile_off(int n, int k, int N, int ld, bool tiled) {
  if (!tiled) return (size_t)n * ld + k;
  const int kp = tile_col(k, N, ld >> 1);
  const int kc = kp >> 4, kl = kp & 15;
  return (size_t)kc * N * 16 + (size_t)n * 16 + (size_t)((((kl >> 2) ^ ((n >> 1) & 3)) << 2) | (kl & 3));
}

// Offset, in bf16 units, of the hi (lo = false) or lo plane entry of tile
// element (row n, column k) in the split layout of a BF16x3 context: the tile
// is cut into K chunks of 16 padded columns kp like the FP32 tensor-core layout, and
// chunk kc (N x 64 bytes, the same bytes as FP32) holds two planes of N rows
// x 32 bytes, hi = rn_bf16(v) then lo = rn_bf16(v - hi) for v the FP32 value;
// each row's two 16-byte halves are exchanged in rows whose bit 2 is set (the
// 32-byte shared-memory swizzle), so one bulk copy per plane lands a K step
// in the operand layout of a kind::f16 MMA.
__host__ __device__ inline size_t tile_off_split(int n, int k, int N, int ld, bool lo) {
  const int kp = tile_col(k, N, ld >> 1);
  const int kc = kp >> 4, kl = kp & 15, g = kl >> 2;
  const size_t base = (size_t)kc * N * 32 + (lo ? (size_t)N * 16 : 0);
  return base + (size_t)n * 16 + (size_t)(((g >> 1) ^ ((n >> 2) & 1)) * 8 + (g & 1) * 4 + (kl & 3));
}

// Offset, in bf16 units, of tile element (row n, column k) in the hi-only
// layout of a BF16x2 context: the hi plane of tile_off_split alone, K chunk kc
// a contiguous block of N rows x 32 bytes under the 32-byte swizzle.
__host__ __device__ inline size_t tile_off_hi(int n, int k, int N, int ld) {
  const int kp = tile_col(k, N, ld >> 1);
  const int kc = kp >> 4, kl = kp & 15, g = kl >> 2;
  return (size_t)kc * N * 16 + (size_t)n * 16 + (size_t)(((g >> 1) ^ ((n >> 2) & 1)) * 8 + (g & 1) * 4 + (kl & 3));
}

}  // namespace prd

// The opaque handle of the C ABI.
struct prd_ctx {
  prd::Ctx c;
};
