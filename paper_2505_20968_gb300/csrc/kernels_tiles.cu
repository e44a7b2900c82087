// Setup kernels: redistribution tiles of the R_II-AD kernel against the
// natural-spline basis (Eq. G, F after it; App. C rule i for Theta = 0; the
// Theta = pi limit kernel), R_III incident weights (Eq. RIIIQKKp) and the
// angle-averaged tiles (Eq. R_AA).
//
// A tile row n of class c and triple t = (k, kl, kl') is
//     T[n][m] = int F(Theta_c, u' + s_in, u_n + s_out) phi_m(u') du',
// s_in = s_{k kl}, s_out = s_{k kl'}, phi_m the cardinal natural cubic
// spline on the height's reduced-frequency grid continued by its end values.
// On grid interval j the spline is (1-t) y_j + t y_{j+1}
// + h_j^2/6 [((1-t)^3-(1-t)) M_j + (t^3-t) M_{j+1}], M = Q y; so a row is
// P_y + P_M Q with P_y, P_M the four moments of F on each interval.
//
// One warp per row: lanes take grid intervals, march Gauss-Legendre panels
// (8 nodes) whose width is at most a quarter of the Gaussian width
// 2 sin(Theta/2) and shrinks geometrically towards the centre of the W factor
// (v = 0), accumulate the moments in FP64, then the warp folds P_M Q and
// writes the row (Re in [0, N), Im in [N, 2N)).
#include <cstdio>
#include <cuda_bf16.h>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

__constant__ WeidemanConst c_wc;
__constant__ double c_gl8x[8];
__constant__ double c_gl8w[8];

enum RowKind { ROW_R2 = 0, ROW_R3 = 1 };

struct TileJob {
  const double* u;       // [N] grid of this height
  const double* Q;       // [N][N]
  double a;              // damping
  int N;
};

// F(Theta, x', x) (complex) at detunings x' (incident), x (outgoing); FP32
// kernels evaluate the Gaussian and W in float from FP64 arguments.
template <typename WT>
__device__ __forceinline__ Cx<double> F_eval(double theta, double s2, double c2, double sinth, double a,
                                             double xp, double x) {
  if (theta >= 3.14159265358979) {
    const double v = 0.5 * (x + xp), d = x - xp;
    const double g = exp(-0.25 * d * d) / (2.0 * 1.7724538509055160 * (v * v + a * a));
    return {g * a, g * v};
  }
  const double d = (x - xp) / (2.0 * s2);
  const WT gw = (WT)exp(-(double)d * d) ;
  const Cx<WT> w = faddeeva<WT>((WT)((x + xp) / (2.0 * c2)), (WT)(a / c2), c_wc);
  const double g = (double)gw / sinth;
  return {g * (double)w.re, g * (double)w.im};
}

template <typename WT>
__device__ __forceinline__ Cx<double> R3_eval(double a, double s1, double s2v, double up) {
  const Cx<WT> w1 = faddeeva<WT>((WT)(up + s1), (WT)a, c_wc);
  const Cx<WT> w2 = faddeeva<WT>((WT)(up + s2v), (WT)a, c_wc);
  return {(double)w1.re + (double)w2.re, (double)w1.im - (double)w2.im};
}

// Accumulate moments of one kernel over [x0, x1] inside interval j (or an
// extension region, j = -1 left / j = N-1 right).
template <typename WT>
__device__ void interval_moments(int kind, double theta, double s2, double c2, double sinth, double a,
                                 double s_in, double s_out, double x, double uV, double hV, double hG,
                                 const double* u, int N, int j, double x0, double x1, double* PyR,
                                 double* PyI, double* PmR, double* PmI, double wscale) {
  const bool ext = (j < 0 || j >= N - 1);
  const double uj = ext ? 0.0 : u[j];
  const double hj = ext ? 1.0 : u[j + 1] - u[j];
  double Ar = 0, Ai = 0, Br = 0, Bi = 0, Cr = 0, Ci = 0, Dr = 0, Di = 0;
  double xl = x0;
  int guard = 0;
  while (xl < x1 && guard < 4096) {
    ++guard;
    double w;
    if (kind == ROW_R2) {
      const double dist = fabs(xl - uV);
      w = fmin(hG, fmax(0.25 * hV, 0.5 * dist));
      if (uV > xl && uV < x1) {
        const double gap = uV - xl;
        // never wider than the Gaussian limit: a panel that stopped at the W centre
        // but spanned several Gaussian widths was under-resolved by 8 nodes
        w = (gap > 0.25 * hV) ? fmin(w, fmax(0.5 * gap, 0.25 * hV)) : fmin(w, gap);
      }
    } else {
      // R_III profiles: smooth on scale 1 around -s1, -s2
      const double d1 = fabs(xl + s_in), d2 = fabs(xl + s_out);
      w = fmax(0.25, 0.25 * fmin(d1, d2));
      const double c1 = -s_in, cc2 = -s_out;
      if (c1 > xl && c1 < xl + w) w = fmax(c1 - xl, 0.05);
      if (cc2 > xl && cc2 < xl + w) w = fmax(cc2 - xl, 0.05);
    }
    double xr = fmin(xl + w, x1);
    if (xr - xl <= 0.0) break;
    const double half = 0.5 * (xr - xl), mid = 0.5 * (xr + xl);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const double up = mid + half * c_gl8x[g];
      const double wq = half * c_gl8w[g] * wscale;
      Cx<double> f;
      if (kind == ROW_R2) f = F_eval<WT>(theta, s2, c2, sinth, a, up + s_in, x);
      else f = R3_eval<WT>(a, s_in, s_out, up);
      const double fr = f.re * wq, fi = f.im * wq;
      if (ext) {
        Ar += fr;
        Ai += fi;
      } else {
        const double t = (up - uj) / hj;
        const double omt = 1.0 - t;
        const double k6 = hj * hj / 6.0;
        const double cA = omt, cB = t, cC = k6 * (omt * omt * omt - omt), cD = k6 * (t * t * t - t);
        Ar += fr * cA; Ai += fi * cA;
        Br += fr * cB; Bi += fi * cB;
        Cr += fr * cC; Ci += fi * cC;
        Dr += fr * cD; Di += fi * cD;
      }
    }
    xl = xr;
  }
  if (ext) {
    const int m = (j < 0) ? 0 : N - 1;
    atomicAdd(&PyR[m], Ar);
    atomicAdd(&PyI[m], Ai);
  } else {
    atomicAdd(&PyR[j], Ar); atomicAdd(&PyI[j], Ai);
    atomicAdd(&PyR[j + 1], Br); atomicAdd(&PyI[j + 1], Bi);
    atomicAdd(&PmR[j], Cr); atomicAdd(&PmI[j], Ci);
    atomicAdd(&PmR[j + 1], Dr); atomicAdd(&PmI[j + 1], Di);
  }
}

__device__ __forceinline__ int find_interval(const double* u, int N, double x) {
  // largest j with u[j] <= x, clamped to [0, N-2]; -1 if x < u[0]; N-1 if x >= u[N-1]
  if (x < u[0]) return -1;
  if (x >= u[N - 1]) return N - 1;
  int lo = 0, hi = N - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (u[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Moments of one row over the support [L, R] (R2) or the grid span (R3),
// distributed over the lanes of the warp by interval.
template <typename WT>
__device__ void row_moments(int kind, double theta, double a, double s_in, double s_out, double un,
                            const double* u, int N, double* PyR, double* PyI, double* PmR, double* PmI,
                            double wscale) {
  const int lane = threadIdx.x & 31;
  if (kind == ROW_R2 && theta == 0.0) {
    if (lane == 0) {
      // App. C rule i: sqrt(pi) W(a, x) delta(u' - (x - s_in))
      const double x = un + s_out, p = x - s_in;
      const Cx<double> w = faddeeva<double>(x, a, c_wc);
      const double cr = 1.7724538509055160 * w.re * wscale, ci = 1.7724538509055160 * w.im * wscale;
      const int j = find_interval(u, N, p);
      if (j < 0) { PyR[0] += cr; PyI[0] += ci; }
      else if (j >= N - 1) { PyR[N - 1] += cr; PyI[N - 1] += ci; }
      else {
        const double h = u[j + 1] - u[j], t = (p - u[j]) / h, omt = 1.0 - t, k6 = h * h / 6.0;
        PyR[j] += cr * omt; PyI[j] += ci * omt;
        PyR[j + 1] += cr * t; PyI[j + 1] += ci * t;
        PmR[j] += cr * k6 * (omt * omt * omt - omt); PmI[j] += ci * k6 * (omt * omt * omt - omt);
        PmR[j + 1] += cr * k6 * (t * t * t - t); PmI[j + 1] += ci * k6 * (t * t * t - t);
      }
    }
    return;
  }
  double L, R, uV = 0, hV = 1, hG = 1, s2 = 0, c2 = 0, sinth = 1, x = un + s_out;
  if (kind == ROW_R2) {
    const bool pi_ = theta >= 3.14159265358979;
    s2 = pi_ ? 1.0 : sin(0.5 * theta);
    c2 = pi_ ? 0.0 : cos(0.5 * theta);
    sinth = pi_ ? 0.0 : sin(theta);
    const double g = 2.0 * s2;
    const double uG = x - s_in;
    L = uG - 6.5 * g;
    R = uG + 6.5 * g;
    uV = -x - s_in;
    hV = 2.0 * fmax(c2, a);
    hG = 0.25 * g;
  } else {
    L = u[0];
    R = u[N - 1];
  }
  // regions: left extension, intervals 0..N-2, right extension
  const int jlo = find_interval(u, N, L);
  const int jhi = find_interval(u, N, R);
  for (int j = jlo + lane; j <= jhi; j += 32) {
    double x0, x1;
    if (j < 0) { x0 = L; x1 = fmin(R, u[0]); }
    else if (j >= N - 1) { x0 = fmax(L, u[N - 1]); x1 = R; }
    else { x0 = fmax(L, u[j]); x1 = fmin(R, u[j + 1]); }
    if (x1 <= x0) continue;
    interval_moments<WT>(kind, theta, s2, c2, sinth, a, s_in, s_out, x, uV, hV, hG, u, N, j, x0, x1,
                         PyR, PyI, PmR, PmI, wscale);
  }
}

// Fold the moments into one output row: out[m] = Py[m] + sum_j Pm[j] Q[j][m].
template <typename T>
__device__ void fold_row(const double* PyR, const double* PyI, const double* PmR, const double* PmI,
                         const double* Q, int N, T* out_re, T* out_im) {
  const int lane = threadIdx.x & 31;
  for (int m0 = 0; m0 < N; m0 += 32) {
    const int m = m0 + lane;
    if (m >= N) break;
    double ar = PyR[m], ai = PyI[m];
    for (int j = 0; j < N; ++j) {
      const double pr = PmR[j], pi = PmI[j];
      if (pr == 0.0 && pi == 0.0) continue;
      const double q = Q[(size_t)j * N + m];
      ar += pr * q;
      ai += pi * q;
    }
    out_re[m] = (T)ar;
    out_im[m] = (T)ai;
  }
}

struct TileParams {
  const double* u;        // [nz][N]
  const double* Q;        // [nz][N][N]
  const double* a;        // [nz]
  const double* shift;    // [nz][nu][nl]
  const int* trip;        // [ntrip][3] (k, kl, kl')
  const double* theta;    // [ncls] (AA: unused)
  const double* aa_th;    // AA Theta nodes
  const double* aa_w;     // AA weights (1/2 sin(Theta) dTheta)
  int n_aa;
  int N, nu, nl, ntrip, ncls, z0;
  int aa;
};

constexpr int kRowsPerBlock = 4;

template <typename T, typename WT>
__global__ void __launch_bounds__(32 * kRowsPerBlock) tile_kernel(TileParams p, T* tiles, int nrows_total) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = p.N;
  double* PyR = sm + (size_t)warp * 4 * N;
  double* PyI = PyR + N;
  double* PmR = PyI + N;
  double* PmI = PmR + N;
  const long long row = (long long)blockIdx.x * kRowsPerBlock + warp;
  if (row >= nrows_total) return;
  // row -> (zl, c, t, n)
  const int n = (int)(row % N);
  long long r2 = row / N;
  const int t = (int)(r2 % p.ntrip);
  r2 /= p.ntrip;
  const int c = (int)(r2 % p.ncls);
  const int iz = p.z0 + (int)(r2 / p.ncls);
  for (int i = lane; i < 4 * N; i += 32) PyR[i] = 0.0;
  __syncwarp();
  const double* u = p.u + (size_t)iz * N;
  const int k = p.trip[3 * t], kl = p.trip[3 * t + 1], klp = p.trip[3 * t + 2];
  const double s_in = p.shift[((size_t)iz * p.nu + k) * p.nl + kl];
  const double s_out = p.shift[((size_t)iz * p.nu + k) * p.nl + klp];
  const double a = p.a[iz];
  if (p.aa) {
    for (int g = 0; g < p.n_aa; ++g) {
      row_moments<WT>(ROW_R2, p.aa_th[g], a, s_in, s_out, u[n], u, N, PyR, PyI, PmR, PmI, p.aa_w[g]);
      __syncwarp();
    }
  } else {
    row_moments<WT>(ROW_R2, p.theta[c], a, s_in, s_out, u[n], u, N, PyR, PyI, PmR, PmI, 1.0);
  }
  __syncwarp();
  T* out = tiles + (size_t)row * 2 * N;
  fold_row<T>(PyR, PyI, PmR, PmI, p.Q + (size_t)iz * N * N, N, out, out + N);
}

struct R3Params {
  const double* u;
  const double* Q;
  const double* a;
  const double* shift;
  int N, nu, nl;
};

// R_III incident weights r[z][q][m], q = (ku, kv, kl):
// int_{u_1}^{u_N} [W(a, u'+s_{kv kl}) + W(a, u'+s_{ku kl})^*] phi_m(u') du'.
template <typename T, typename WT>
__global__ void __launch_bounds__(32 * kRowsPerBlock) r3_kernel(R3Params p, T* out, int nz) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = p.N, nq = p.nu * p.nu * p.nl;
  double* PyR = sm + (size_t)warp * 4 * N;
  double* PyI = PyR + N;
  double* PmR = PyI + N;
  double* PmI = PmR + N;
  const long long row = (long long)blockIdx.x * kRowsPerBlock + warp;
  if (row >= (long long)nz * nq) return;
  const int q = (int)(row % nq), iz = (int)(row / nq);
  const int kl = q % p.nl, kv = (q / p.nl) % p.nu, ku = q / (p.nl * p.nu);
  for (int i = lane; i < 4 * N; i += 32) PyR[i] = 0.0;
  __syncwarp();
  const double* u = p.u + (size_t)iz * N;
  const double s1 = p.shift[((size_t)iz * p.nu + kv) * p.nl + kl];
  const double s2 = p.shift[((size_t)iz * p.nu + ku) * p.nl + kl];
  row_moments<WT>(ROW_R3, 0.0, p.a[iz], s1, s2, 0.0, u, N, PyR, PyI, PmR, PmI, 1.0);
  __syncwarp();
  T* o = out + (size_t)row * 2 * N;
  fold_row<T>(PyR, PyI, PmR, PmI, p.Q + (size_t)iz * N * N, N, o, o + N);
}

// Group-mean / deviation split of the FP64 tiles of one height:
//   tiles[c][g][.]        = mean over the triples t of group g of G_t
//   tiles[c][ngrp + t][.] = G_t - mean of its group
// so that the large dispersion parts that cancel between Zeeman components
// of one J level are summed once, in FP64, before rounding to the storage type.
// the FP32 value v of a tile entry stored as bf16 planes hi = rn(v), lo = rn(v - hi)
__device__ __forceinline__ void store_split(__nv_bfloat16* t, int n, int k, int N, int ld, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  t[tile_off_split(n, k, N, ld, false)] = hi;
  t[tile_off_split(n, k, N, ld, true)] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// split: 0 the storage type T (plain or tiled), 1 the bf16 hi and lo planes of
// BF16x3 contexts (the bytes of an FP32 tile), 2 the hi plane alone (BF16x2:
// half the bytes; dst is then read as bf16 with tiles of N ld elements)
template <typename T>
__global__ void group_split_kernel(const double* __restrict__ src, T* __restrict__ dst, const int* __restrict__ grp,
                                   int ncls, int ntrip, int ngrp, int N, int ld, int tiled, int split) {
  const int rowlen = 2 * N * N;                 // one FP64 scratch tile: N rows of 2N
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (c, n*2N + k)
  if (idx >= (long long)ncls * rowlen) return;
  const int c = (int)(idx / rowlen);
  const int e = (int)(idx - (long long)c * rowlen);
  const int n = e / (2 * N), kk = e - n * 2 * N;
  const size_t o = tile_off(n, kk, N, ld, tiled != 0);
  const size_t tsz = (size_t)N * ld;
  double mean[2] = {0.0, 0.0};
  int cnt[2] = {0, 0};
  for (int t = 0; t < ntrip; ++t) {
    const int g = grp[t];
    mean[g] += src[((size_t)c * ntrip + t) * rowlen + e];
    cnt[g] += 1;
  }
  for (int g = 0; g < ngrp; ++g) mean[g] = cnt[g] ? mean[g] / cnt[g] : 0.0;
  if (split == 2) {
    __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(dst);
    const size_t oh = tile_off_hi(n, kk, N, ld);
    for (int g = 0; g < ngrp; ++g) h[((size_t)c * (ngrp + ntrip) + g) * tsz + oh] = __float2bfloat16_rn((float)mean[g]);
    for (int t = 0; t < ntrip; ++t)
      h[((size_t)c * (ngrp + ntrip) + ngrp + t) * tsz + oh] =
          __float2bfloat16_rn((float)(src[((size_t)c * ntrip + t) * rowlen + e] - mean[grp[t]]));
    return;
  }
  if (split) {
    // split layout (BF16x3 contexts): T is float, each tile's bytes hold the two bf16 planes
    for (int g = 0; g < ngrp; ++g)
      store_split(reinterpret_cast<__nv_bfloat16*>(dst + ((size_t)c * (ngrp + ntrip) + g) * tsz), n, kk, N, ld,
                  (float)mean[g]);
    for (int t = 0; t < ntrip; ++t)
      store_split(reinterpret_cast<__nv_bfloat16*>(dst + ((size_t)c * (ngrp + ntrip) + ngrp + t) * tsz), n, kk, N, ld,
                  (float)(src[((size_t)c * ntrip + t) * rowlen + e] - mean[grp[t]]));
    return;
  }
  for (int g = 0; g < ngrp; ++g) dst[((size_t)c * (ngrp + ntrip) + g) * tsz + o] = (T)mean[g];
  for (int t = 0; t < ntrip; ++t)
    dst[((size_t)c * (ngrp + ntrip) + ngrp + t) * tsz + o] =
        (T)(src[((size_t)c * ntrip + t) * rowlen + e] - mean[grp[t]]);
}

// -------------------------------------------------------------- launchers
static int upload_consts(Ctx* c) {
  WeidemanConst wc;
  double a64[36], L64;
  weideman_coeffs(kWeidemanN64, a64, &L64);
  for (int i = 0; i < 36; ++i) wc.a64[i] = a64[i];
  wc.L64 = L64;
  double a32[20], L32;
  weideman_coeffs(kWeidemanN32, a32, &L32);
  for (int i = 0; i < 20; ++i) wc.a32[i] = (float)a32[i];
  wc.L32 = (float)L32;
  PRD_CUDA_TRY(c, cudaMemcpyToSymbol(c_wc, &wc, sizeof(wc)));
  // 8-point Gauss-Legendre on [-1, 1]
  const double x8[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                        0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
  const double w8[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                        0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
  PRD_CUDA_TRY(c, cudaMemcpyToSymbol(c_gl8x, x8, sizeof(x8)));
  PRD_CUDA_TRY(c, cudaMemcpyToSymbol(c_gl8w, w8, sizeof(w8)));
  return PRD_OK;
}

int launch_tiles(Ctx* c) {
  int rc = upload_consts(c);
  if (rc) return rc;
  const int nz = c->nz, N = c->nnu;
  // device copies of the FP64 setup inputs
  DBuf du, dQ, da, dsh, dtr, dth, dath, daw;
  std::vector<int> trip;
  for (int t = 0; t < c->ntrip; ++t) { trip.push_back(c->trip_k[t]); trip.push_back(c->trip_l[t]); trip.push_back(c->trip_lp[t]); }
  std::vector<double> aath = c->aa_theta, aaw = c->aa_w;
  if (aath.empty()) { aath.push_back(0); aaw.push_back(0); }
  if ((rc = upload(c, du, c->u.data(), c->u.size() * 8)) ||
      (rc = upload(c, dQ, c->Q.data(), c->Q.size() * 8)) ||
      (rc = upload(c, da, c->a.data(), nz * 8)) ||
      (rc = upload(c, dsh, c->shift.data(), c->shift.size() * 8)) ||
      (rc = upload(c, dtr, trip.data(), trip.size() * 4)) ||
      (rc = upload(c, dth, c->theta.data(), c->theta.size() * 8)) ||
      (rc = upload(c, dath, aath.data(), aath.size() * 8)) ||
      (rc = upload(c, daw, aaw.data(), aaw.size() * 8))) {
    dfree(du); dfree(dQ); dfree(da); dfree(dsh); dfree(dtr); dfree(dth); dfree(dath); dfree(daw);
    return rc;
  }
  TileParams p{(const double*)du.p, (const double*)dQ.p, (const double*)da.p, (const double*)dsh.p,
               (const int*)dtr.p, (const double*)dth.p, (const double*)dath.p, (const double*)daw.p,
               (int)c->aa_theta.size(), N, c->nu_st, c->nl_st, c->ntrip, c->ncls, 0,
               c->mode == PRD_MODE_AA ? 1 : 0};
  const size_t smem = (size_t)kRowsPerBlock * 4 * N * sizeof(double);
  const long long rows_per_z = (long long)c->ncls * c->ntrip * N;
  int err = 0;
  cudaFuncSetAttribute(tile_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(r3_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(r3_kernel<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  DBuf scr, dgrp;
  if ((rc = dalloc(c, scr, (size_t)rows_per_z * 2 * N * sizeof(double))) ||
      (rc = upload(c, dgrp, c->trip_grp.data(), c->trip_grp.size() * 4))) {
    dfree(du); dfree(dQ); dfree(da); dfree(dsh); dfree(dtr); dfree(dth); dfree(dath); dfree(daw); dfree(scr);
    return rc;
  }
  const int rowlen = 2 * N * N;     // one FP64 scratch tile (n rows of 2N)
  const size_t ztile = (size_t)c->ncls * c->ntile() * N * c->ld();
  for (int iz = 0; iz < nz && !err; ++iz) {
    p.z0 = iz;
    const long long nrows = rows_per_z;
    const int blocks = (int)((nrows + kRowsPerBlock - 1) / kRowsPerBlock);
    // W in FP64 in both modes: the per-triple tiles are differenced against
    // their group mean, so their errors must be far below the storage epsilon
    tile_kernel<double, double><<<blocks, 32 * kRowsPerBlock, smem, c->stream>>>(p, (double*)scr.p, (int)nrows);
    const int sb = ceil_div((long long)c->ncls * rowlen, 256);
    if (c->prec == PRD_FP64)
      group_split_kernel<double><<<sb, 256, 0, c->stream>>>((const double*)scr.p, (double*)c->tiles.p + iz * ztile,
                                                            (const int*)dgrp.p, c->ncls, c->ntrip, c->ngrp, N, c->ld(),
                                                            c->tiled(), 0);
    else {
      group_split_kernel<float><<<sb, 256, 0, c->stream>>>(
          (const double*)scr.p, (float*)((char*)c->tiles.p + iz * ztile * c->tile_esz()), (const int*)dgrp.p, c->ncls,
          c->ntrip, c->ngrp, N, c->ld(), c->tiled(), c->hi_only ? 2 : (c->split_tiles ? 1 : 0));
      if (c->has64)
        group_split_kernel<double><<<sb, 256, 0, c->stream>>>(
            (const double*)scr.p, (double*)c->tiles64.p + (size_t)iz * c->ncls * c->ntile() * N * c->ld64(),
            (const int*)dgrp.p, c->ncls, c->ntrip, c->ngrp, N, c->ld64(), 0, 0);
    }
    if (cudaPeekAtLastError() != cudaSuccess) err = 1;
  }
  cudaStreamSynchronize(c->stream);
  dfree(scr);
  dfree(dgrp);
  if (!err) {
    R3Params q{(const double*)du.p, (const double*)dQ.p, (const double*)da.p, (const double*)dsh.p, N,
               c->nu_st, c->nl_st};
    const int nq = c->nu_st * c->nu_st * c->nl_st;
    const int blocks = ceil_div((long long)nz * nq, kRowsPerBlock);
    if (c->prec == PRD_FP64)
      r3_kernel<double, double><<<blocks, 32 * kRowsPerBlock, smem, c->stream>>>(q, (double*)c->r3w.p, nz);
    else
      r3_kernel<float, double><<<blocks, 32 * kRowsPerBlock, smem, c->stream>>>(q, (float*)c->r3w.p, nz);
    if (c->prec != PRD_FP64 && c->has64)
      r3_kernel<double, double><<<blocks, 32 * kRowsPerBlock, smem, c->stream>>>(q, (double*)c->r3w64.p, nz);
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  dfree(du); dfree(dQ); dfree(da); dfree(dsh); dfree(dtr); dfree(dth); dfree(dath); dfree(daw);
  if (err || e != cudaSuccess)
    return fail(c, PRD_E_CUDA, std::string("tile generation: ") + cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
  return PRD_OK;
}

// Tiles of one height for an arbitrary list of scattering angles (one class
// per entry), stored like the main tiles: [class][group means, deviations][n][2N].
int gen_tiles_z(Ctx* c, int iz, const std::vector<double>& thetas, void* outT) {
  int rc = upload_consts(c);
  if (rc) return rc;
  const int N = c->nnu, ncl = (int)thetas.size();
  std::vector<int> trip;
  for (int t = 0; t < c->ntrip; ++t) { trip.push_back(c->trip_k[t]); trip.push_back(c->trip_l[t]); trip.push_back(c->trip_lp[t]); }
  std::vector<double> aath = c->aa_theta, aaw = c->aa_w;
  if (aath.empty()) { aath.push_back(0); aaw.push_back(0); }
  DBuf du, dQ, da, dsh, dtr, dth, dath, daw, scr, dgrp;
  auto cleanup = [&]() { dfree(du); dfree(dQ); dfree(da); dfree(dsh); dfree(dtr); dfree(dth); dfree(dath);
                         dfree(daw); dfree(scr); dfree(dgrp); };
  const long long nrows = (long long)ncl * c->ntrip * N;
  if ((rc = upload(c, du, c->u.data(), c->u.size() * 8)) || (rc = upload(c, dQ, c->Q.data(), c->Q.size() * 8)) ||
      (rc = upload(c, da, c->a.data(), c->nz * 8)) || (rc = upload(c, dsh, c->shift.data(), c->shift.size() * 8)) ||
      (rc = upload(c, dtr, trip.data(), trip.size() * 4)) || (rc = upload(c, dth, thetas.data(), thetas.size() * 8)) ||
      (rc = upload(c, dath, aath.data(), aath.size() * 8)) || (rc = upload(c, daw, aaw.data(), aaw.size() * 8)) ||
      (rc = dalloc(c, scr, (size_t)nrows * 2 * N * 8)) ||
      (rc = upload(c, dgrp, c->trip_grp.data(), c->trip_grp.size() * 4))) {
    cleanup();
    return rc;
  }
  TileParams p{(const double*)du.p, (const double*)dQ.p, (const double*)da.p, (const double*)dsh.p,
               (const int*)dtr.p, (const double*)dth.p, (const double*)dath.p, (const double*)daw.p,
               (int)c->aa_theta.size(), N, c->nu_st, c->nl_st, c->ntrip, ncl, iz, c->mode == PRD_MODE_AA ? 1 : 0};
  const size_t smem = (size_t)kRowsPerBlock * 4 * N * sizeof(double);
  cudaFuncSetAttribute(tile_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  tile_kernel<double, double><<<ceil_div(nrows, kRowsPerBlock), 32 * kRowsPerBlock, smem, c->stream>>>(
      p, (double*)scr.p, (int)nrows);
  const int rowlen = 2 * N * N;
  const int sb = ceil_div((long long)ncl * rowlen, 256);
  if (c->prec == PRD_FP64)
    group_split_kernel<double><<<sb, 256, 0, c->stream>>>((const double*)scr.p, (double*)outT, (const int*)dgrp.p, ncl,
                                                          c->ntrip, c->ngrp, N, c->ld(), c->tiled(), 0);
  else
    group_split_kernel<float><<<sb, 256, 0, c->stream>>>((const double*)scr.p, (float*)outT, (const int*)dgrp.p, ncl,
                                                         c->ntrip, c->ngrp, N, c->ld(), c->tiled(), 0);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  cleanup();
  if (e != cudaSuccess) return fail(c, PRD_E_CUDA, std::string("line-of-sight tiles: ") + cudaGetErrorString(e));
  return PRD_OK;
}

// Angle-averaged tiles and R_III incident weights of the unmagnetised J-level
// components (shifts shift_g[z][g]) for the preconditioner, returned in FP64.
int launch_pc_tiles(Ctx* c, const std::vector<double>& shift_g, std::vector<double>& aa_tiles,
                    std::vector<double>& r3g) {
  int rc = upload_consts(c);
  if (rc) return rc;
  const int nz = c->nz, N = c->nnu, ng = c->ngrp;
  std::vector<double> x, w, th, tw;
  gauss_legendre(kAAThetaNodes, x, w);
  for (int h = 0; h < 2; ++h) {
    const double lo = h * 0.5 * kPi, hi = lo + 0.5 * kPi;
    for (int i = 0; i < kAAThetaNodes; ++i) {
      const double t = 0.5 * (hi - lo) * x[i] + 0.5 * (hi + lo);
      th.push_back(t);
      tw.push_back(0.5 * 0.5 * (hi - lo) * w[i] * std::sin(t));
    }
  }
  std::vector<int> trip;
  for (int g = 0; g < ng; ++g) { trip.push_back(g); trip.push_back(0); trip.push_back(0); }
  const double th0 = 0.0;
  DBuf du, dQ, da, dsh, dtr, dth, dath, daw, out, out3;
  auto cleanup = [&]() { dfree(du); dfree(dQ); dfree(da); dfree(dsh); dfree(dtr); dfree(dth); dfree(dath);
                         dfree(daw); dfree(out); dfree(out3); };
  const long long rows_per_z = (long long)ng * N;
  if ((rc = upload(c, du, c->u.data(), c->u.size() * 8)) || (rc = upload(c, dQ, c->Q.data(), c->Q.size() * 8)) ||
      (rc = upload(c, da, c->a.data(), nz * 8)) || (rc = upload(c, dsh, shift_g.data(), shift_g.size() * 8)) ||
      (rc = upload(c, dtr, trip.data(), trip.size() * 4)) || (rc = upload(c, dth, &th0, 8)) ||
      (rc = upload(c, dath, th.data(), th.size() * 8)) || (rc = upload(c, daw, tw.data(), tw.size() * 8)) ||
      (rc = dalloc(c, out, (size_t)nz * rows_per_z * 2 * N * 8)) ||
      (rc = dalloc(c, out3, (size_t)nz * ng * ng * 2 * N * 8))) {
    cleanup();
    return rc;
  }
  TileParams p{(const double*)du.p, (const double*)dQ.p, (const double*)da.p, (const double*)dsh.p,
               (const int*)dtr.p, (const double*)dth.p, (const double*)dath.p, (const double*)daw.p,
               (int)th.size(), N, ng, 1, ng, 1, 0, 1};
  const size_t smem = (size_t)kRowsPerBlock * 4 * N * sizeof(double);
  cudaFuncSetAttribute(tile_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(r3_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int iz = 0; iz < nz; ++iz) {
    p.z0 = iz;
    tile_kernel<double, double><<<ceil_div(rows_per_z, kRowsPerBlock), 32 * kRowsPerBlock, smem, c->stream>>>(
        p, (double*)out.p + (size_t)iz * rows_per_z * 2 * N, (int)rows_per_z);
  }
  R3Params q{(const double*)du.p, (const double*)dQ.p, (const double*)da.p, (const double*)dsh.p, N, ng, 1};
  r3_kernel<double, double><<<ceil_div((long long)nz * ng * ng, kRowsPerBlock), 32 * kRowsPerBlock, smem,
                              c->stream>>>(q, (double*)out3.p, nz);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) {
    aa_tiles.resize((size_t)nz * rows_per_z * 2 * N);
    r3g.resize((size_t)nz * ng * ng * 2 * N);
    e = cudaMemcpy(aa_tiles.data(), out.p, aa_tiles.size() * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r3g.data(), out3.p, r3g.size() * 8, cudaMemcpyDeviceToHost);
  }
  cleanup();
  if (e != cudaSuccess) return fail(c, PRD_E_CUDA, std::string("preconditioner tiles: ") + cudaGetErrorString(e));
  return PRD_OK;
}

}  // namespace prd
