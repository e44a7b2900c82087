// S13: the adjoint (transposed) operator A^T = Id - Sigma^T Lambda^T of the
// discrete system of Eq. linear_system, in FP64, and the adjoint solve.
//
// Each forward stage is linear, so its transpose is written stage by stage
// (Sect. 4 discretisation, the same tables as the forward apply):
//   Lambda^T  reverse sweep of the DELO-linear recurrence per ray (Sect. 3),
//   S6^T      back-interpolation spline transposed, with the Kirchhoff factor f,
//   S3^T      R_II tiles transposed: Zbar = T^T g per tile, then the Y coefficients,
//   S5^T      R_III separable factors transposed,
//   S1^T      comoving interpolation spline transposed.
// The natural-spline system matrix is symmetric, so its transposed solve is
// the forward Thomas solve.  In FP32 mode the adjoint reads the FP64 copy of the
// Sigma tables, so it is the transpose of the operator whose solution
// prd_solve returns.
#include <cstdio>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

namespace {

constexpr int kTB = 256;

// ---------------------------------------------------------------- Lambda^T
// Forward, per ray in sweep order p (point k(p)), zero boundary:
//   I_p = M_p^-1 [(e_p Id - a_p K'_{p-1}) I_{p-1} + a_p S_{p-1} + b_p S_p],  M_p = Id + b_p K'_p,
//   S_p = eps_p / eta1_p,  I_0 = 0  (e, a, b of the step arriving at p).
// Transpose for output cotangents g_p:
//   lam_p = g_p + (e_{p+1} Id - a_{p+1} K'_p)^T w_{p+1},  w_p = M_p^-T lam_p  (p >= 1),
//   Sbar_p = b_p w_p + a_{p+1} w_{p+1},  epsbar_p = Sbar_p / eta1_p.
template <typename T>
__device__ __forceinline__ void kprime_t(const T* t, double K[4][4]) {
  K[0][0] = 0; K[1][1] = 0; K[2][2] = 0; K[3][3] = 0;
  K[0][1] = K[1][0] = t[0];
  K[0][2] = K[2][0] = t[1];
  K[0][3] = K[3][0] = t[2];
  K[1][2] = t[3]; K[2][1] = -t[3];
  K[1][3] = t[4]; K[3][1] = -t[4];
  K[2][3] = t[5]; K[3][2] = -t[5];
}

// solve (Id + b K)^T w = v  (4x4, Gaussian elimination without pivoting: the
// matrix is Id plus a small multiple of the propagation matrix)
__device__ __forceinline__ void solve_t(const double K[4][4], double b, const double v[4], double w[4]) {
  double M[4][4], r[4];
  for (int i = 0; i < 4; ++i) {
    r[i] = v[i];
    for (int j = 0; j < 4; ++j) M[i][j] = (i == j ? 1.0 : 0.0) + b * K[j][i];
  }
  for (int c0 = 0; c0 < 4; ++c0) {
    const double inv = 1.0 / M[c0][c0];
    for (int rr = c0 + 1; rr < 4; ++rr) {
      const double f = M[rr][c0] * inv;
      for (int cc = c0; cc < 4; ++cc) M[rr][cc] -= f * M[c0][cc];
      r[rr] -= f * r[c0];
    }
  }
  for (int rr = 3; rr >= 0; --rr) {
    double s = r[rr];
    for (int cc = rr + 1; cc < 4; ++cc) s -= M[rr][cc] * w[cc];
    w[rr] = s / M[rr][rr];
  }
}

template <typename T>
__global__ void delo_t_kernel(const double* __restrict__ g, const T* __restrict__ kt, const double* __restrict__ mu,
                              double* __restrict__ epsbar, int nz, int nO, int N) {
  const int ray = blockIdx.x * blockDim.x + threadIdx.x;
  if (ray >= nO * N) return;
  const int o = ray / N, n = ray - o * N;
  const bool up = mu[o] > 0.0;
  auto pt_of = [&](int p) { return ((size_t)(up ? p : nz - 1 - p) * nO + o) * N + n; };
  double wn[4] = {0, 0, 0, 0};     // w_{p+1}
  double en = 0.0, an = 0.0;       // e_{p+1}, a_{p+1}
  for (int p = nz - 1; p >= 0; --p) {
    const size_t pt = pt_of(p);
    const T* t = kt + pt * 10;
    double K[4][4];
    kprime_t(t, K);
    const double ie = t[6];
    double w[4] = {0, 0, 0, 0};
    if (p >= 1) {
      double lam[4];
      for (int i = 0; i < 4; ++i) {
        double v = g[pt * 4 + i] + en * wn[i];
        for (int j = 0; j < 4; ++j) v -= an * K[j][i] * wn[j];
        lam[i] = v;
      }
      solve_t(K, (double)t[9], lam, w);
    }
    const double b = p >= 1 ? (double)t[9] : 0.0;
    for (int i = 0; i < 4; ++i) epsbar[pt * 4 + i] = (b * w[i] + an * wn[i]) * ie;
    for (int i = 0; i < 4; ++i) wn[i] = w[i];
    en = p >= 1 ? (double)t[7] : 0.0;
    an = p >= 1 ? (double)t[8] : 0.0;
  }
}

// ---------------------------------------------------------------- splines^T
// Forward per row (z, Omega, s): M = T^-1 D y (natural spline, T symmetric
// tridiagonal), then r(pt) = y_k + t (y_{k+1} - y_k) + c2 M_k + c3 M_{k+1}, with
// constant extension outside the grid; the intensity row is scaled by fI.
// Transpose: scatter gbar into ybar and Mbar, w = T^-1 Mbar, ybar += D^T w.
// ybar and Mbar are per-row scratch rows in global memory.
__global__ void spline_t_kernel(const double* __restrict__ gbar, const int* __restrict__ kidx,
                                const double* __restrict__ tt, const double* __restrict__ sp,
                                const double* __restrict__ fI, double* __restrict__ ybar, double* __restrict__ Mbar,
                                int nz, int nO, int N) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;   // (z, o, s)
  if (row >= nz * nO * 4) return;
  const int s = row & 3, zo = row >> 2, iz = zo / nO;
  const double* h = sp + (size_t)iz * 3 * N;
  const double* cp = h + N;
  const double* den = cp + N;
  double* yb = ybar + (size_t)row * N;
  double* mb = Mbar + (size_t)row * N;
  for (int i = 0; i < N; ++i) { yb[i] = 0.0; mb[i] = 0.0; }
  for (int n = 0; n < N; ++n) {
    const size_t pt = (size_t)zo * N + n;
    double gv = gbar[pt * 4 + s];
    if (fI && s == 0) gv *= fI[pt];
    const int k = kidx[pt];
    if (k < 0) yb[0] += gv;
    else if (k >= N - 1) yb[N - 1] += gv;
    else {
      const double t = tt[pt], omt = 1.0 - t;
      const double hk = h[k], k6 = hk * hk / 6.0;
      yb[k] += (1.0 - t) * gv;
      yb[k + 1] += t * gv;
      mb[k] += k6 * (omt * omt * omt - omt) * gv;
      mb[k + 1] += k6 * (t * t * t - t) * gv;
    }
  }
  if (N <= 2) return;
  // w = T^-1 Mbar on the interior nodes (M_0 = M_{N-1} = 0 are constants)
  double gprev = 0.0;
  for (int r = 0; r < N - 2; ++r) {
    const int i = r + 1;
    const double sub = (r > 0) ? h[i - 1] : 0.0;
    const double gg = (mb[i] - sub * gprev) / den[r];
    mb[i] = gg;
    gprev = gg;
  }
  double mnext = 0.0;
  for (int r = N - 3; r >= 0; --r) {
    const int i = r + 1;
    const double m = mb[i] - cp[r] * mnext;
    mb[i] = m;
    mnext = m;
  }
  // ybar += D^T w,  (D y)_i = 6 [(y_{i+1} - y_i) / h_i - (y_i - y_{i-1}) / h_{i-1}]
  for (int i = 1; i <= N - 2; ++i) {
    const double w = 6.0 * mb[i];
    yb[i + 1] += w / h[i];
    yb[i] -= w * (1.0 / h[i] + 1.0 / h[i - 1]);
    yb[i - 1] += w / h[i - 1];
  }
}

// scratch rows [row][n] -> vector [z][o][n][s]
__global__ void rows_to_vec_kernel(const double* __restrict__ rows, double* __restrict__ v, int nrows, int N) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (row, n)
  if (idx >= (long long)nrows * N) return;
  const int row = (int)(idx / N), n = (int)(idx - (long long)row * N);
  const int s = row & 3, zo = row >> 2;
  v[((size_t)zo * N + n) * 4 + s] = rows[idx];
}

// ---------------------------------------------------------------- R_II^T
// Forward: eps_bar[e][n][i] += sum_m Re(T[n][m] Z[m][(e,i)]),
//          Z[m][(e,i)] = sum_{pairs p of e} sum_j Y_p[i][j] I~[o'_p][m][j].
// Transpose: Zr[m][(e,i)] = sum_n T_r[n][m] g[e][n][i],  Zi = -sum_n T_i[n][m] g[e][n][i],
//            Ibar[o'][m][j] += sum_i (Y_r[i][j] Zr + Y_i[i][j] Zi).
// Block per (chunk of kCE outputs, class, z); 16 incident frequencies m per pass.
constexpr int kCE = 8;
constexpr int kMB2 = 16;

__global__ void __launch_bounds__(256) r2_t_kernel(const double* __restrict__ tiles, const double* __restrict__ Y,
                                                   const double* __restrict__ g, const int* __restrict__ cls,
                                                   double* __restrict__ Ibar, int ncls, int ntile, int nO, int N,
                                                   int npairs, int ld) {
  const int chunk = blockIdx.x, c = blockIdx.y, iz = blockIdx.z;
  const int* cout_ptr = cls;
  const int* cout_dir = cls + ncls + 1;
  const int ne_tot = cout_ptr[ncls];
  const int* pair_ptr = cout_dir + ne_tot;
  const int* pair_in = pair_ptr + ne_tot + 1;
  const int e0 = cout_ptr[c] + chunk * kCE;
  const int e_end = cout_ptr[c + 1];
  if (e0 >= e_end) return;
  const int E = min(kCE, e_end - e0);
  extern __shared__ __align__(16) unsigned char smraw[];
  double* gs = reinterpret_cast<double*>(smraw);          // [e][n][i]
  double* zs = gs + (size_t)kCE * N * 4;                   // [m][e*4+i][2]
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kCE * N * 4; idx += blockDim.x) {
    const int e = idx / (N * 4), rem = idx - e * N * 4;
    gs[idx] = e < E ? g[((size_t)iz * nO + cout_dir[e0 + e]) * N * 4 + rem] : 0.0;
  }
  __syncthreads();
  const size_t tsz = (size_t)N * ld;
  const double* tb = tiles + ((size_t)iz * ncls + c) * ntile * tsz;
  for (int ti = 0; ti < ntile; ++ti) {
    const double* T = tb + (size_t)ti * tsz;
    for (int m0 = 0; m0 < N; m0 += kMB2) {
      // Zbar block: kMB2 m x (kCE * 4) columns, two entries per thread
      for (int q = tid; q < kMB2 * kCE * 4; q += blockDim.x) {
        const int mm = q / (kCE * 4), col = q - mm * (kCE * 4);
        const int m = m0 + mm, e = col >> 2, i = col & 3;
        double zr = 0.0, zi = 0.0;
        if (m < N && e < E)
          for (int n = 0; n < N; ++n) {
            const double gv = gs[((size_t)e * N + n) * 4 + i];
            zr += T[(size_t)n * ld + m] * gv;
            zi -= T[(size_t)n * ld + N + m] * gv;
          }
        zs[q * 2] = zr;
        zs[q * 2 + 1] = zi;
      }
      __syncthreads();
      // Y contraction into Ibar: items (m, pair, j)
      const int pa = pair_ptr[e0], pb = pair_ptr[e0 + E];
      const int np = pb - pa;
      for (int q = tid; q < kMB2 * np * 4; q += blockDim.x) {
        const int mm = q / (np * 4), rem = q - mm * np * 4;
        const int pl = rem >> 2, j = rem & 3;
        const int m = m0 + mm;
        if (m >= N) continue;
        const int p = pa + pl;
        int e = 0;
        while (e + 1 < E && pair_ptr[e0 + e + 1] <= p) ++e;
        const double* y = Y + (((size_t)iz * npairs + p) * ntile + ti) * 32;
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int col = e * 4 + i;
          acc += y[(i * 4 + j) * 2] * zs[(mm * (kCE * 4) + col) * 2] + y[(i * 4 + j) * 2 + 1] * zs[(mm * (kCE * 4) + col) * 2 + 1];
        }
        atomicAdd(&Ibar[(((size_t)iz * nO + pair_in[p]) * N + m) * 4 + j], acc);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- R_III^T
// Forward: J[uv] = sum_{l', o', j, m} rin_j(o'; q) w[q][m] I~_j(o', m),  q = (uv, l'),
//          eps_bar[o][n][i] += Re sum_{uv, l'} rout_i(o; uv, l') ab[uv] J[uv] prof[uv][l'][n].
// Transpose: E[uv] = sum_{o, n, i, l'} g[o][n][i] rout_i prof[uv][l'][n],  F = ab E,
//            Ibar_j(o', m) += sum_q Re(rin_j(o'; q) w[q][m] F[uv(q)]).
__global__ void r3_e_kernel(const double* __restrict__ g, const double* __restrict__ rout,
                            const double* __restrict__ prof, const double* __restrict__ ab, double* __restrict__ F,
                            int nO, int N, int nuv, int nl) {
  const int uv = blockIdx.x, iz = blockIdx.y;
  double er = 0.0, ei = 0.0;
  for (int idx = threadIdx.x; idx < nO * N; idx += blockDim.x) {
    const int o = idx / N, n = idx - o * N;
    const double* gv = g + (((size_t)iz * nO + o) * N + n) * 4;
    for (int lp = 0; lp < nl; ++lp) {
      const double* pp = prof + ((((size_t)iz * nuv + uv) * nl + lp) * N + n) * 2;
      const double* ro = rout + ((((size_t)iz * nO + o) * nuv + uv) * nl + lp) * 8;
      double sr = 0.0, si = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        sr += gv[i] * ro[2 * i];
        si += gv[i] * ro[2 * i + 1];
      }
      er += sr * pp[0] - si * pp[1];
      ei += sr * pp[1] + si * pp[0];
    }
  }
  __shared__ double red[2][kTB];
  red[0][threadIdx.x] = er;
  red[1][threadIdx.x] = ei;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ar = ab[((size_t)iz * nuv + uv) * 2], ai = ab[((size_t)iz * nuv + uv) * 2 + 1];
    F[((size_t)iz * nuv + uv) * 2] = ar * red[0][0] - ai * red[1][0];
    F[((size_t)iz * nuv + uv) * 2 + 1] = ar * red[1][0] + ai * red[0][0];
  }
}

__global__ void r3_ibar_kernel(const double* __restrict__ F, const double* __restrict__ rin,
                               const double* __restrict__ r3w, double* __restrict__ Ibar, int nz, int nO, int N,
                               int nq, int nl) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (z, o', m)
  if (pt >= (long long)nz * nO * N) return;
  const int m = (int)(pt % N);
  const int zo = (int)(pt / N), iz = zo / nO;
  double acc[4] = {0, 0, 0, 0};
  for (int q = 0; q < nq; ++q) {
    const double* w = r3w + ((size_t)iz * nq + q) * 2 * N;
    const double* f = F + ((size_t)iz * (nq / nl) + q / nl) * 2;
    const double wr = w[m], wi = w[N + m];
    const double cr = wr * f[0] - wi * f[1], ci = wr * f[1] + wi * f[0];   // w F
    const double* ri = rin + ((size_t)zo * nq + q) * 8;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += ri[2 * j] * cr - ri[2 * j + 1] * ci;
  }
  for (int j = 0; j < 4; ++j) Ibar[pt * 4 + j] += acc[j];
}

__global__ void to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = a[i];
}
__global__ void sub_out_kernel(const double* __restrict__ x, const double* __restrict__ s, void* __restrict__ y,
                               size_t n, int fp32) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i] - s[i];
    if (fp32) ((float*)y)[i] = (float)v;
    else ((double*)y)[i] = v;
  }
}

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

// y = (Id - Sigma^T Lambda^T) x, arithmetic in FP64 (x, y in the ctx precision).
int apply_operator_t(Ctx* c, const void* x, void* y) {
  const bool fp32 = c->prec == PRD_FP32;
  if (fp32 && !c->has64)
    return fail(c, PRD_E_STATE, "adjoint needs the FP64 copy of the Sigma tables (not kept: too little memory)");
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  const size_t nv = nvec(c);
  const int nrows = nz * nO * 4;
  const double* tiles = (const double*)(fp32 ? c->tiles64.p : c->tiles.p);
  const double* Y = (const double*)(fp32 ? c->Y64.p : c->Y.p);
  const double* r3w = (const double*)(fp32 ? c->r3w64.p : c->r3w.p);
  const double* r3in = (const double*)(fp32 ? c->r3in64.p : c->r3in.p);
  const double* r3out = (const double*)(fp32 ? c->r3out64.p : c->r3out.p);
  const double* r3prof = (const double*)(fp32 ? c->r3prof64.p : c->r3prof.p);
  const double* r3ab = (const double*)(fp32 ? c->r3ab64.p : c->r3ab.p);
  const int ld = fp32 ? c->ld64() : c->ld();
  const int nuv = c->nu_st * c->nu_st, nq = nuv * c->nl_st;
  // scratch kept by the context (allocated on first use), so that the apply
  // allocates nothing and can be captured into the adjoint solver's graph
  DBuf& x64 = c->adj[0];
  DBuf& g1 = c->adj[1];
  DBuf& g2 = c->adj[2];
  DBuf& ib = c->adj[3];
  DBuf& ybr = c->adj[4];
  DBuf& mbr = c->adj[5];
  DBuf& F = c->adj[6];
  int rc;
  if (!F.p && ((rc = dalloc(c, x64, nv * 8)) || (rc = dalloc(c, g1, nv * 8)) || (rc = dalloc(c, g2, nv * 8)) ||
               (rc = dalloc(c, ib, nv * 8)) || (rc = dalloc(c, ybr, (size_t)nrows * N * 8)) ||
               (rc = dalloc(c, mbr, (size_t)nrows * N * 8)) || (rc = dalloc(c, F, (size_t)nz * nuv * 2 * 8)))) {
    for (auto& b : c->adj) dfree(b);
    return rc;
  }
  const double* xd = (const double*)x;
  if (fp32) {
    to_f64_kernel<<<c->grid_ew(), 256, 0, c->stream>>>((const float*)x, (double*)x64.p, nv);
    xd = (const double*)x64.p;
  }
  // Lambda^T (FP32 mode: on the FP64 copy of the tables, as the forward residuals)
  delo_t_kernel<double><<<cdiv((long long)nO * N, 128), 128, 0, c->stream>>>(
      xd, (const double*)(fp32 ? c->kt64.p : c->kt.p), (const double*)c->dmu.p, (double*)g1.p, nz, nO, N);
  // S6^T (with f): cotangent of the comoving emissivity
  spline_t_kernel<<<cdiv(nrows, 64), 64, 0, c->stream>>>((const double*)g1.p, (const int*)c->ibk.p,
                                                         (const double*)c->tbk.p, (const double*)c->sp.p,
                                                         (const double*)c->f.p, (double*)ybr.p, (double*)mbr.p, nz,
                                                         nO, N);
  rows_to_vec_kernel<<<cdiv((long long)nrows * N, 256), 256, 0, c->stream>>>((const double*)ybr.p, (double*)g2.p,
                                                                              nrows, N);
  // S3^T + S5^T: cotangent of the comoving field
  PRD_CUDA_TRY(c, cudaMemsetAsync(ib.p, 0, nv * 8, c->stream));
  {
    const size_t smem = sizeof(double) * ((size_t)kCE * N * 4 + (size_t)kMB2 * kCE * 4 * 2);
    PRD_CUDA_TRY(c, cudaFuncSetAttribute(r2_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nchunk = (c->max_cout + kCE - 1) / kCE;
    r2_t_kernel<<<dim3(nchunk, c->ncls, nz), 256, smem, c->stream>>>(tiles, Y, (const double*)g2.p,
                                                                     (const int*)c->cls_dev.p, (double*)ib.p, c->ncls,
                                                                     c->ntile(), nO, N, c->npairs, ld);
  }
  r3_e_kernel<<<dim3(nuv, nz), kTB, 0, c->stream>>>((const double*)g2.p, r3out, r3prof, r3ab, (double*)F.p, nO, N,
                                                    nuv, c->nl_st);
  r3_ibar_kernel<<<cdiv((long long)nz * nO * N, 128), 128, 0, c->stream>>>((const double*)F.p, r3in, r3w,
                                                                            (double*)ib.p, nz, nO, N, nq, c->nl_st);
  // S1^T
  spline_t_kernel<<<cdiv(nrows, 64), 64, 0, c->stream>>>((const double*)ib.p, (const int*)c->iin.p,
                                                         (const double*)c->tin.p, (const double*)c->sp.p, nullptr,
                                                         (double*)ybr.p, (double*)mbr.p, nz, nO, N);
  rows_to_vec_kernel<<<cdiv((long long)nrows * N, 256), 256, 0, c->stream>>>((const double*)ybr.p, (double*)g1.p,
                                                                              nrows, N);
  sub_out_kernel<<<c->grid_ew(), 256, 0, c->stream>>>(xd, (const double*)g1.p, y, nv, fp32 ? 1 : 0);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

}  // namespace prd
