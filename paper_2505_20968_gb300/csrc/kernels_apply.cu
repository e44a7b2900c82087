// Per-apply kernels of y = (Id - Lambda Sigma) x.
//   S1  frame change observer -> comoving: natural spline of I(z,Omega',.)
//       evaluated at u_m - u_b(z,Omega')                     (Sect. 4.1)
//   S3+S4  R_II contraction over (Theta class, Omega', triple, frequency)
//       with the Stokes-route coefficients folded in          (Eq. RQIIKKp)
//   S5  R_III, separable in incident and outgoing frequency  (Eq. RIIIQKKp)
//   S6  frame change back (u_n + u_b(z,Omega)) and Kirchhoff factor f (App. E)
//   S7+S8  DELO-linear sweep per ray, y = x - Lambda eps      (Sect. 3)
#include <cstdio>
#include <mutex>
#include <type_traits>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

// ------------------------------------------------------------------ splines
// Second derivatives of the natural spline of every (z, Omega, s) row.
template <typename T>
__global__ void spline_M_kernel(const T* __restrict__ y, T* __restrict__ M, const double* __restrict__ sp,
                                int nz, int nO, int N) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;   // (z, o, s)
  if (row >= nz * nO * 4) return;
  const int s = row & 3, zo = row >> 2, iz = zo / nO;
  const double* h = sp + (size_t)iz * 3 * N;
  const double* cp = h + N;
  const double* den = cp + N;
  const T* yr = y + (size_t)zo * N * 4 + s;
  T* Mr = M + (size_t)zo * N * 4 + s;
  Mr[0] = (T)0;
  Mr[(size_t)(N - 1) * 4] = (T)0;
  if (N <= 2) return;
  // forward sweep: g_r stored in M[i], i = r + 1
  double gprev = 0.0;
  double y0 = (double)yr[0], y1 = (double)yr[4];
  for (int r = 0; r < N - 2; ++r) {
    const int i = r + 1;
    const double y2 = (double)yr[(size_t)(i + 1) * 4];
    const double rhs = 6.0 * ((y2 - y1) / h[i] - (y1 - y0) / h[i - 1]);
    const double sub = (r > 0) ? h[i - 1] : 0.0;
    const double g = (rhs - sub * gprev) / den[r];
    Mr[(size_t)i * 4] = (T)g;
    gprev = g;
    y0 = y1;
    y1 = y2;
  }
  double mnext = 0.0;
  for (int r = N - 3; r >= 0; --r) {
    const int i = r + 1;
    const double m = (double)Mr[(size_t)i * 4] - cp[r] * mnext;
    Mr[(size_t)i * 4] = (T)m;
    mnext = m;
  }
}

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4_16a; };

// Evaluate the spline of every (z, Omega) row at the tabulated points; the
// intensity component is multiplied by fI (nullable).
template <typename T, typename F = T>
__global__ void spline_eval_kernel(const T* __restrict__ y, const T* __restrict__ M, const int* __restrict__ kidx,
                                   const double* __restrict__ tt, const double* __restrict__ sp,
                                   const F* __restrict__ fI, T* __restrict__ out, int nz, int nO, int N) {
  using V = typename V4<T>::type;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (z, o, n)
  if (pt >= (long long)nz * nO * N) return;
  const int zo = (int)(pt / N), iz = zo / nO;
  const int k = kidx[pt];
  const V* yr = reinterpret_cast<const V*>(y) + (size_t)zo * N;
  const V* Mr = reinterpret_cast<const V*>(M) + (size_t)zo * N;
  V r;
  if (k < 0) r = yr[0];
  else if (k >= N - 1) r = yr[N - 1];
  else {
    const double t = tt[pt], omt = 1.0 - t;
    const double h = sp[(size_t)iz * 3 * N + k];
    const double k6 = h * h / 6.0;
    // y_k + t (y_{k+1} - y_k) + ...: reproduces a constant exactly in any precision
    const T c1 = (T)t, c2 = (T)(k6 * (omt * omt * omt - omt)), c3 = (T)(k6 * (t * t * t - t));
    const V a = yr[k], b = yr[k + 1], ma = Mr[k], mb = Mr[k + 1];
    r.x = a.x + c1 * (b.x - a.x) + c2 * ma.x + c3 * mb.x;
    r.y = a.y + c1 * (b.y - a.y) + c2 * ma.y + c3 * mb.y;
    r.z = a.z + c1 * (b.z - a.z) + c2 * ma.z + c3 * mb.z;
    r.w = a.w + c1 * (b.w - a.w) + c2 * ma.w + c3 * mb.w;
  }
  if (fI) r.x *= (T)fI[pt];
  reinterpret_cast<V*>(out)[pt] = r;
}

// ------------------------------------------------------------------ R_III
// J[z][ku kv] += sum_{o', j} rin[z][o'][q][j] * sum_m r3w[z][q][m] I~[z][o'][m][j],  q = (ku kv, l')
// One block per (o', z): the direction's comoving row I~[z][o'][.][.] is staged in
// shared memory and thread q forms S_j = sum_m r3w[q][m] I~_j(m) (arithmetic in A,
// so the FP32 path runs on the FP32 pipe), then adds sum_j rin_j S_j to J in FP64.
template <typename T, typename A>
__global__ void r3_J_kernel(const A* __restrict__ Ic, const T* __restrict__ r3w, const T* __restrict__ rin,
                            double* __restrict__ J, int nO, int N, int nq, int nl) {
  using V = typename V4<A>::type;
  const int o = blockIdx.x, iz = blockIdx.y;
  extern __shared__ __align__(16) unsigned char r3smem[];
  V* row = reinterpret_cast<V*>(r3smem);
  const V* src = reinterpret_cast<const V*>(Ic) + ((size_t)iz * nO + o) * N;
  for (int m = threadIdx.x; m < N; m += blockDim.x) row[m] = src[m];
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const T* w = r3w + ((size_t)iz * nq + q) * 2 * N;
    A sr[4] = {0, 0, 0, 0}, si[4] = {0, 0, 0, 0};
    for (int m = 0; m < N; ++m) {
      const A wr = (A)w[m], wi = (A)w[N + m];
      const V iv = row[m];
      sr[0] += wr * iv.x; sr[1] += wr * iv.y; sr[2] += wr * iv.z; sr[3] += wr * iv.w;
      si[0] += wi * iv.x; si[1] += wi * iv.y; si[2] += wi * iv.z; si[3] += wi * iv.w;
    }
    const T* ri = rin + (((size_t)iz * nO + o) * nq + q) * 8;
    double jr = 0.0, ji = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double rr = (double)ri[2 * j], rm = (double)ri[2 * j + 1];
      jr += rr * (double)sr[j] - rm * (double)si[j];
      ji += rr * (double)si[j] + rm * (double)sr[j];
    }
    const int uv = q / nl;
    atomicAdd(&J[((size_t)iz * (nq / nl) + uv) * 2], jr);
    atomicAdd(&J[((size_t)iz * (nq / nl) + uv) * 2 + 1], ji);
  }
}

// eps_bar[z][o][n][i] = Re sum_uv ab[uv] J[uv] sum_l' O_i(o; uv, l') prof[uv][l'][n]
// One block per (o, z), one thread per n: C = ab J per uv and the direction's
// O_i coefficients are staged in shared memory; the profile rows are read
// coalesced along n.  Arithmetic in A.
template <typename T, typename A>
__global__ void r3_out_kernel(const double* __restrict__ J, const T* __restrict__ ab, const T* __restrict__ rout,
                              const T* __restrict__ prof, A* __restrict__ eb, int nz, int nO, int N, int nuv,
                              int nl) {
  const int o = blockIdx.x, iz = blockIdx.y;
  const int zo = iz * nO + o;
  extern __shared__ __align__(16) unsigned char r3smem[];
  A* C = reinterpret_cast<A*>(r3smem);                 // [uv][2]
  A* R = C + 2 * nuv;                                  // [uv][l'][8]
  for (int uv = threadIdx.x; uv < nuv; uv += blockDim.x) {
    const double jr = J[((size_t)iz * nuv + uv) * 2], ji = J[((size_t)iz * nuv + uv) * 2 + 1];
    const double ar = (double)ab[((size_t)iz * nuv + uv) * 2], ai = (double)ab[((size_t)iz * nuv + uv) * 2 + 1];
    C[2 * uv] = (A)(ar * jr - ai * ji);
    C[2 * uv + 1] = (A)(ar * ji + ai * jr);
  }
  for (int k = threadIdx.x; k < nuv * nl * 8; k += blockDim.x) R[k] = (A)rout[(size_t)zo * nuv * nl * 8 + k];
  __syncthreads();
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    A acc[4] = {0, 0, 0, 0};
    for (int uv = 0; uv < nuv; ++uv) {
      const A cr = C[2 * uv], ci = C[2 * uv + 1];
      for (int lp = 0; lp < nl; ++lp) {
        const T* pp = prof + ((((size_t)iz * nuv + uv) * nl + lp) * N + n) * 2;
        const A pr = (A)pp[0], pi = (A)pp[1];
        const A dr = cr * pr - ci * pi, di = cr * pi + ci * pr;
        const A* ro = R + (uv * nl + lp) * 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += ro[2 * i] * dr - ro[2 * i + 1] * di;
      }
    }
    A* out = eb + ((size_t)zo * N + n) * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = acc[i];
  }
}

// The Sigma tables an apply reads: the ctx precision's, or (FP32 mode, t64) the
// FP64 copies kept for the refinement residuals.
struct SigmaTables {
  const void *tiles, *Y, *r3w, *r3in, *r3out, *r3prof, *r3ab;
  int ld, tiled;
};
static SigmaTables sigma_tables(const Ctx* c, bool t64) {
  if (t64)
    return {c->tiles64.p, c->Y64.p, c->r3w64.p, c->r3in64.p, c->r3out64.p, c->r3prof64.p, c->r3ab64.p, c->ld64(), 0};
  return {c->tiles.p, c->Y.p, c->r3w.p, c->r3in.p, c->r3out.p, c->r3prof.p, c->r3ab.p, c->ld(), c->tiled() ? 1 : 0};
}

// launchers (shared by the apply and the line-of-sight paths)
template <typename T, typename A>
static void launch_r3_J(Ctx* c, const A* Ic, double* J, int nO, const SigmaTables& tb) {
  const int nuv = c->nu_st * c->nu_st, nq = nuv * c->nl_st, N = c->nnu;
  r3_J_kernel<T, A><<<dim3(nO, c->nz), 128, (size_t)N * 4 * sizeof(A), c->stream>>>(
      Ic, (const T*)tb.r3w, (const T*)tb.r3in, J, nO, N, nq, c->nl_st);
}
template <typename T, typename A>
static void launch_r3_out(Ctx* c, const double* J, const T* rout, A* eb, int nO, const SigmaTables& tb) {
  const int nuv = c->nu_st * c->nu_st, N = c->nnu;
  const size_t smem = sizeof(A) * ((size_t)2 * nuv + (size_t)nuv * c->nl_st * 8);
  r3_out_kernel<T, A><<<dim3(nO, c->nz), N <= 128 ? 128 : 256, smem, c->stream>>>(
      J, (const T*)tb.r3ab, rout, (const T*)tb.r3prof, eb, c->nz, nO, N, nuv, c->nl_st);
}

// ------------------------------------------------------------------ R_II (SIMT)
// One CTA per (z, class, chunk of 16 output directions).  Over the triples t
// and blocks of 16 incident frequencies m it builds, in shared memory,
//   Z_t[m][(o,i)] = sum_{o' : Theta(o,o') = class} sum_j Y_t,ij(o,o') I~_j(o', m)
// and accumulates  eps_bar[n][(o,i)] += sum_m Re(T_t[n][m] Z_t[m][(o,i)])
// with the tile T_t of (z, class) streamed from global memory.
constexpr int kCW = 16;      // output directions per CTA
constexpr int kMB = 16;      // incident-frequency block
constexpr int kMaxRows = 16; // rows per thread (N <= 256)

template <typename T, typename A>
__global__ void __launch_bounds__(256) r2_simt_kernel(const T* __restrict__ tiles, const T* __restrict__ Y,
                                                      const A* __restrict__ Ic, const int* __restrict__ cls,
                                                      A* __restrict__ eb, int ncls, int ntrip, int nO, int N,
                                                      int npairs, int ld, int tiled) {
  const int chunk = blockIdx.x, c = blockIdx.y, iz = blockIdx.z;
  const int* cout_ptr = cls;
  const int* cout_dir = cls + ncls + 1;
  const int ne_tot = cout_ptr[ncls];
  const int* pair_ptr = cout_dir + ne_tot;
  const int* pair_in = pair_ptr + ne_tot + 1;
  const int e0 = cout_ptr[c] + chunk * kCW;
  const int e_end = cout_ptr[c + 1];
  if (e0 >= e_end) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  A (*Zs)[2][kCW * 4] = reinterpret_cast<A (*)[2][kCW * 4]>(smraw);
  T* Asb = reinterpret_cast<T*>(smraw + sizeof(A) * kMB * 2 * kCW * 4);
  // As[h][n][mm] -> Asb[(h * N + n) * (kMB + 1) + mm]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int e_mine = e0 + tx;
  A acc[kMaxRows][4];
#pragma unroll
  for (int r = 0; r < kMaxRows; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[r][i] = (A)0;
  const int nrows = (N + 15) / 16;
  const size_t tile_sz = (size_t)N * ld;
  const T* tbase = tiles + ((size_t)iz * ncls + c) * ntrip * tile_sz;
  // Z-building role: thread -> (e = tid & 15, m = tid >> 4)
  const int ze = tid & 15, zm = tid >> 4;
  const int e_z = e0 + ze;
  for (int t = 0; t < ntrip; ++t) {
    const T* tile = tbase + (size_t)t * tile_sz;
    for (int m0 = 0; m0 < N; m0 += kMB) {
      // ---- Z block
      {
        const int m = m0 + zm;
        A zr[4] = {0, 0, 0, 0}, zi[4] = {0, 0, 0, 0};
        if (e_z < e_end && m < N) {
          for (int p = pair_ptr[e_z]; p < pair_ptr[e_z + 1]; ++p) {
            const int op = pair_in[p];
            const A* iv = Ic + (((size_t)iz * nO + op) * N + m) * 4;
            const T* y = Y + (((size_t)iz * npairs + p) * ntrip + t) * 32;
            const A i0 = iv[0], i1 = iv[1], i2 = iv[2], i3 = iv[3];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const T* yi = y + i * 8;
              zr[i] += (A)yi[0] * i0 + (A)yi[2] * i1 + (A)yi[4] * i2 + (A)yi[6] * i3;
              zi[i] += (A)yi[1] * i0 + (A)yi[3] * i1 + (A)yi[5] * i2 + (A)yi[7] * i3;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          Zs[zm][0][ze * 4 + i] = zr[i];
          Zs[zm][1][ze * 4 + i] = zi[i];
        }
      }
      // ---- tile block: rows n, columns m0..m0+15 (Re and Im halves)
      for (int idx = tid; idx < N * 2 * kMB; idx += 256) {
        const int mm = idx % kMB;
        const int h = (idx / kMB) & 1;
        const int n = idx / (2 * kMB);
        const int m = m0 + mm;
        Asb[(h * N + n) * (kMB + 1) + mm] = (m < N) ? tile[tile_off(n, h * N + m, N, ld, tiled != 0)] : (T)0;
      }
      __syncthreads();
#pragma unroll 4
      for (int mm = 0; mm < kMB; ++mm) {
        A zr[4], zi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          zr[i] = Zs[mm][0][tx * 4 + i];
          zi[i] = Zs[mm][1][tx * 4 + i];
        }
#pragma unroll
        for (int r = 0; r < kMaxRows; ++r) {
          if (r < nrows) {
            const int n = ty + 16 * r;
            if (n < N) {
              const A ar = Asb[n * (kMB + 1) + mm], ai = Asb[(N + n) * (kMB + 1) + mm];
#pragma unroll
              for (int i = 0; i < 4; ++i) acc[r][i] += ar * zr[i] - ai * zi[i];
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (e_mine < e_end) {
    const int o = cout_dir[e_mine];
#pragma unroll
    for (int r = 0; r < kMaxRows; ++r) {
      const int n = ty + 16 * r;
      if (r < nrows && n < N) {
        A* dst = eb + (((size_t)iz * nO + o) * N + n) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) atomicAdd(dst + i, acc[r][i]);
      }
    }
  }
}

// ------------------------------------------------------------------ R_II, double-float
// The same contraction for the FP64 refinement residuals, run on the FP32 pipes
// (GB300's FP64 rate is 1/64 of its FP32 rate).  Every FP64 operand a is split
// into a = hi + lo (two floats, |lo| <= 2^-24 |a|); a product of two operands
// is hi*hi exactly (FMA error term) plus the hi*lo cross terms, and the sum is
// kept as an unevaluated float pair (s, c) with the error-free two-sum of s
// (Dekker / Knuth double-single arithmetic).  Dropped: lo*lo (2^-48 relative)
// and the rounding of c; the result carries ~2^-44 relative error per term,
// far below the 1e-10 residuals the refinement needs.
struct F2 { float hi, lo; };
__device__ __forceinline__ F2 split2(double a) {
  const float h = (float)a;
  return {h, (float)(a - (double)h)};
}
// (s, c) += x (x exact float); error-free two-sum of s and x into s, error into c
__device__ __forceinline__ void dd_add(float& s, float& c, float x) {
  const float t = s + x;
  const float bb = t - s;
  c += (s - (t - bb)) + (x - bb);
  s = t;
}

__global__ void __launch_bounds__(256) r2_dd_kernel(const double* __restrict__ tiles, const double* __restrict__ Y,
                                                    const double* __restrict__ Ic, const int* __restrict__ cls,
                                                    double* __restrict__ eb, int ncls, int ntrip, int nO, int N,
                                                    int npairs, int ld) {
  const int chunk = blockIdx.x, c = blockIdx.y, iz = blockIdx.z;
  const int* cout_ptr = cls;
  const int* cout_dir = cls + ncls + 1;
  const int ne_tot = cout_ptr[ncls];
  const int* pair_ptr = cout_dir + ne_tot;
  const int* pair_in = pair_ptr + ne_tot + 1;
  const int e0 = cout_ptr[c] + chunk * kCW;
  const int e_end = cout_ptr[c + 1];
  if (e0 >= e_end) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4 (*Zs)[kCW * 4] = reinterpret_cast<float4 (*)[kCW * 4]>(smraw);        // [mm][col]: zr hi/lo, zi hi/lo
  float2* Asb = reinterpret_cast<float2*>(smraw + sizeof(float4) * kMB * kCW * 4);  // [(h N + n)(kMB+1) + mm]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int e_mine = e0 + tx;
  float accs[kMaxRows][4], accc[kMaxRows][4];
#pragma unroll
  for (int r = 0; r < kMaxRows; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) { accs[r][i] = 0.f; accc[r][i] = 0.f; }
  const int nrows = (N + 15) / 16;
  const size_t tile_sz = (size_t)N * ld;
  const double* tbase = tiles + ((size_t)iz * ncls + c) * ntrip * tile_sz;
  const int ze = tid & 15, zm = tid >> 4;
  const int e_z = e0 + ze;
  for (int t = 0; t < ntrip; ++t) {
    const double* tile = tbase + (size_t)t * tile_sz;
    for (int m0 = 0; m0 < N; m0 += kMB) {
      {
        const int m = m0 + zm;
        double zr[4] = {0, 0, 0, 0}, zi[4] = {0, 0, 0, 0};
        if (e_z < e_end && m < N) {
          for (int p = pair_ptr[e_z]; p < pair_ptr[e_z + 1]; ++p) {
            const double* iv = Ic + (((size_t)iz * nO + pair_in[p]) * N + m) * 4;
            const double* y = Y + (((size_t)iz * npairs + p) * ntrip + t) * 32;
            const double i0 = iv[0], i1 = iv[1], i2 = iv[2], i3 = iv[3];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const double* yi = y + i * 8;
              zr[i] += yi[0] * i0 + yi[2] * i1 + yi[4] * i2 + yi[6] * i3;
              zi[i] += yi[1] * i0 + yi[3] * i1 + yi[5] * i2 + yi[7] * i3;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const F2 a = split2(zr[i]), b = split2(zi[i]);
          Zs[zm][ze * 4 + i] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
      }
      for (int idx = tid; idx < N * 2 * kMB; idx += 256) {
        const int mm = idx % kMB;
        const int h = (idx / kMB) & 1;
        const int n = idx / (2 * kMB);
        const int m = m0 + mm;
        const F2 v = split2(m < N ? tile[(size_t)n * ld + h * N + m] : 0.0);
        Asb[(h * N + n) * (kMB + 1) + mm] = make_float2(v.hi, v.lo);
      }
      __syncthreads();
#pragma unroll 2
      for (int mm = 0; mm < kMB; ++mm) {
        float4 z[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) z[i] = Zs[mm][tx * 4 + i];
#pragma unroll
        for (int r = 0; r < kMaxRows; ++r) {
          if (r < nrows) {
            const int n = ty + 16 * r;
            if (n < N) {
              const float2 ar = Asb[n * (kMB + 1) + mm], ai = Asb[(N + n) * (kMB + 1) + mm];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                // ar * zr - ai * zi
                const float p1 = ar.x * z[i].x;
                const float q1 = fmaf(ar.x, z[i].x, -p1);
                const float p2 = -ai.x * z[i].z;
                const float q2 = fmaf(-ai.x, z[i].z, -p2);
                const float lo = q1 + q2 + fmaf(ar.x, z[i].y, ar.y * z[i].x) - fmaf(ai.x, z[i].w, ai.y * z[i].z);
                dd_add(accs[r][i], accc[r][i], p1);
                dd_add(accs[r][i], accc[r][i], p2);
                accc[r][i] += lo;
              }
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (e_mine < e_end) {
    const int o = cout_dir[e_mine];
#pragma unroll
    for (int r = 0; r < kMaxRows; ++r) {
      const int n = ty + 16 * r;
      if (r < nrows && n < N) {
        double* dst = eb + (((size_t)iz * nO + o) * N + n) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) atomicAdd(dst + i, (double)accs[r][i] + (double)accc[r][i]);
      }
    }
  }
}

// ------------------------------------------------------------------ DELO
// One thread per ray (Omega, nu): I_k = (Id + b K'_k)^-1 [(e Id - a K'_{k-1}) I_{k-1}
//   + a S_{k-1} + b S_k], S = eps/eta1, K' = K/eta1 - Id.  Optional: out = x - I.
template <typename T, typename A>
__device__ __forceinline__ void kprime(const T* t, A K[4][4]) {
  K[0][0] = 0; K[1][1] = 0; K[2][2] = 0; K[3][3] = 0;
  K[0][1] = K[1][0] = t[0];
  K[0][2] = K[2][0] = t[1];
  K[0][3] = K[3][0] = t[2];
  K[1][2] = t[3]; K[2][1] = -t[3];
  K[1][3] = t[4]; K[3][1] = -t[4];
  K[2][3] = t[5]; K[3][2] = -t[5];
}

// Per-point inputs of one step of the formal solution.
template <typename T, typename A>
struct DeloPoint {
  T t[10];          // K'/eta1 (6), 1/eta1, exp(-dtau), alpha, beta
  A e[4];           // emissivity
  A xs[4];          // x of y = x - Lambda eps (zero if unused)
  double ps[3];     // DELOPAR source weights
};

template <typename T, typename A>
__device__ __forceinline__ void delo_load(DeloPoint<T, A>& d, const A* __restrict__ eps, const T* __restrict__ kt,
                                          const double* __restrict__ par, const A* __restrict__ x_sub, size_t pt) {
  for (int i = 0; i < 10; ++i) d.t[i] = kt[pt * 10 + i];
  for (int s = 0; s < 4; ++s) d.e[s] = eps[pt * 4 + s];
  for (int s = 0; s < 4; ++s) d.xs[s] = x_sub ? x_sub[pt * 4 + s] : (A)0;
  if (par)
    for (int i = 0; i < 3; ++i) d.ps[i] = par[pt * 3 + i];
}

// LU factors of M = Id + b K'_k of a point (no pivoting: M is the identity plus
// b times the antisymmetric-off-diagonal K', as in the step's original form):
// strictly lower multipliers l, strictly upper entries u and the reciprocals
// of the pivots.  M depends on the tables only, so a sweep factors the next
// point while the current one is solved, and only the substitutions, which
// carry the intensity, stay on the serial chain from step to step.
template <typename A>
struct DeloFact {
  A l10, l20, l30, l21, l31, l32;
  A u01, u02, u03, u12, u13, u23;
  A i0, i1, i2, i3;
};

template <typename T, typename A>
__device__ __forceinline__ void delo_factor(const DeloPoint<T, A>& d, DeloFact<A>& F) {
  A K[4][4];
  kprime(d.t, K);
  const A be = d.t[9];
  A M[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) M[i][j] = (i == j ? (A)1 : (A)0) + be * K[i][j];
  A l[4][4], piv[4];
  for (int c0 = 0; c0 < 4; ++c0) {
    piv[c0] = (A)1 / M[c0][c0];
    for (int r = c0 + 1; r < 4; ++r) {
      const A f = M[r][c0] * piv[c0];
      l[r][c0] = f;
      for (int cc = c0; cc < 4; ++cc) M[r][cc] -= f * M[c0][cc];
    }
  }
  F.l10 = l[1][0]; F.l20 = l[2][0]; F.l30 = l[3][0]; F.l21 = l[2][1]; F.l31 = l[3][1]; F.l32 = l[3][2];
  F.u01 = M[0][1]; F.u02 = M[0][2]; F.u03 = M[0][3]; F.u12 = M[1][2]; F.u13 = M[1][3]; F.u23 = M[2][3];
  F.i0 = piv[0]; F.i1 = piv[1]; F.i2 = piv[2]; F.i3 = piv[3];
}

// One step of the formal solution (Sect. 3) at the p-th point of a ray: DELO-
// linear, or DELOPAR when `par` (the parabolic source weights psi_M, psi_O,
// psi_P of the step arriving at the point; the source vector parabolic through
// the upwind, current and downwind points, the K'I term linear with DELO-
// linear's a, b; psi = (a, b, 0) at the last point) is set; `nxt` is the next
// point (read only under DELOPAR, p + 1 < nz); F the factors of cur's
// Id + b K'.  I, Sp, Kp carry the upwind intensity, source and K' from step
// to step.
template <typename T, typename A>
__device__ __forceinline__ void delo_step(const DeloPoint<T, A>& cur, const DeloFact<A>& F,
                                          const DeloPoint<T, A>& nxt, bool par, bool has_next, int p, bool up,
                                          int boundary, double WT0, A I[4], A Sp[4], A Kp[4][4]) {
  const T* t = cur.t;
  A Kk[4][4];
  kprime(t, Kk);
  const A ie = t[6];
  A S[4];
  for (int s = 0; s < 4; ++s) S[s] = cur.e[s] * ie;
  if (p == 0) {
    I[0] = (boundary && up) ? (A)WT0 : (A)0;
    I[1] = I[2] = I[3] = (A)0;
  } else {
    // Optically thick step (e = exp(-dtau) <= 1/2): solve for D = I_k - S_k,
    //   (Id + b K'_k) D = e (I_{k-1} - S_k) + a (S_{k-1} - S_k) - a K'_{k-1} I_{k-1} - b K'_k S_k,
    // which reproduces a constant unpolarised source exactly whatever the
    // rounding of the stored weights (b = 1 - e - a enters only the dichroic
    // terms).  Thin step: the standard form for I_k, free of the
    // cancellation I_{k-1} - S_k when I << S.
    const A e = t[7], al = t[8], be = t[9];
    const bool thick = e <= (A)0.5;
    // source weights: DELO-linear (a, b, 0) or DELOPAR's parabolic ones, with the
    // downwind source S_P; psi_M + psi_O + psi_P = 1 - e in both
    A pM = al, pO = be, pP = (A)0;
    A SP[4] = {0, 0, 0, 0};
    if (par) {
      pM = (A)cur.ps[0];
      pO = (A)cur.ps[1];
      pP = (A)cur.ps[2];
      if (has_next) {
        const A ie2 = nxt.t[6];
        for (int s = 0; s < 4; ++s) SP[s] = nxt.e[s] * ie2;
      }
    }
    A rhs[4];
    for (int i = 0; i < 4; ++i) {
      A v = thick ? e * (I[i] - S[i]) + pM * (Sp[i] - S[i]) + pP * (SP[i] - S[i])
                  : e * I[i] + pM * Sp[i] + pO * S[i] + pP * SP[i];
      for (int j = 0; j < 4; ++j) v -= al * Kp[i][j] * I[j] + (thick ? be * Kk[i][j] * S[j] : (A)0);
      rhs[i] = v;
    }
    // forward substitution with the unit lower factor, back substitution with the upper one
    const A y0 = rhs[0];
    const A y1 = rhs[1] - F.l10 * y0;
    const A y2 = rhs[2] - F.l20 * y0 - F.l21 * y1;
    const A y3 = rhs[3] - F.l30 * y0 - F.l31 * y1 - F.l32 * y2;
    A D[4];
    D[3] = y3 * F.i3;
    D[2] = (y2 - F.u23 * D[3]) * F.i2;
    D[1] = (y1 - F.u12 * D[2] - F.u13 * D[3]) * F.i1;
    D[0] = (y0 - F.u01 * D[1] - F.u02 * D[2] - F.u03 * D[3]) * F.i0;
    for (int i = 0; i < 4; ++i) I[i] = thick ? S[i] + D[i] : D[i];
  }
  for (int i = 0; i < 4; ++i) {
    Sp[i] = S[i];
    for (int j = 0; j < 4; ++j) Kp[i][j] = Kk[i][j];
  }
}

// Formal solution along every ray, one thread per ray (Omega, nu); the sweep is
// sequential in height, so the inputs of the next two points are loaded while
// a point is solved.  Used where the staged sweep below does not apply (odd
// frequency counts, lines of sight, the FP64 residual path).
template <typename T, typename A>
__global__ void delo_kernel(const A* __restrict__ eps, const T* __restrict__ kt, const double* __restrict__ par,
                            const double* __restrict__ mu, const A* __restrict__ x_sub, A* __restrict__ out, int nz,
                            int nO, int N, int boundary, double WT0) {
  const int ray = blockIdx.x * blockDim.x + threadIdx.x;
  if (ray >= nO * N) return;
  const int o = ray / N, n = ray - o * N;
  const bool up = mu[o] > 0.0;
  auto point = [&](int p) { return ((size_t)(up ? p : nz - 1 - p) * nO + o) * N + n; };
  A I[4] = {0, 0, 0, 0};
  A Sp[4] = {0, 0, 0, 0};
  A Kp[4][4];
  DeloPoint<T, A> cur, nx1, nx2;
  DeloFact<A> fc, fn;
  delo_load(cur, eps, kt, par, x_sub, point(0));
  delo_factor(cur, fc);
  if (nz > 1) delo_load(nx1, eps, kt, par, x_sub, point(1));
  for (int p = 0; p < nz; ++p) {
    const size_t pt = point(p);
    if (p + 2 < nz) delo_load(nx2, eps, kt, par, x_sub, point(p + 2));
    if (p + 1 < nz) delo_factor(nx1, fn);          // off the serial chain of this step
    delo_step(cur, fc, nx1, par != nullptr, p + 1 < nz, p, up, boundary, WT0, I, Sp, Kp);
    for (int s = 0; s < 4; ++s) out[pt * 4 + s] = x_sub ? cur.xs[s] - I[s] : I[s];
    cur = nx1;
    nx1 = nx2;
    fc = fn;
  }
}

// ---- staged sweep: one CTA per (direction, chunk of kDR frequencies).  Warp 0
// lane 0 streams each height's slices of the inputs (K'/eta1 and DELO weights,
// emissivity, the x of y = x - Lambda eps, DELOPAR weights: contiguous runs of
// kDR points) with bulk asynchronous copies into a ring of kDStages heights;
// the kDR consumer threads (one per ray) take their point from shared memory.
// Needs an even frequency count (16-byte aligned slices).  Every wait is
// bounded: on expiry the CTA stops, the producer drains its copies, and the
// error flag is raised (PRD_E_TIMEOUT through prd_device_status).
constexpr int kDR = 128;                       // rays per CTA
constexpr int kDStages = 8;                    // heights in flight per CTA
constexpr long long kDSpin = 1ll << 24;

__device__ __forceinline__ uint32_t dsm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool dbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.b32 %0, 1, 0, P;\n\t}\n"
      : "=r"(ok)
      : "r"(dsm_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool dbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  for (long long i = 0; i < kDSpin; ++i) {
    if (dbar_try(b, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

template <typename T, typename A>
struct DeloStage {
  // byte offsets of the slices inside one stage (each a multiple of 16)
  static constexpr int kKT = 0;
  static constexpr int kEps = kKT + kDR * 10 * (int)sizeof(T);
  static constexpr int kXs = kEps + kDR * 4 * (int)sizeof(A);
  static constexpr int kPar = kXs + kDR * 4 * (int)sizeof(A);
  static constexpr int kBytes = kPar + kDR * 3 * 8;
};

template <typename T, typename A>
__global__ void __launch_bounds__(32 + kDR) delo_staged_kernel(const A* __restrict__ eps, const T* __restrict__ kt,
                                                               const double* __restrict__ par,
                                                               const double* __restrict__ mu,
                                                               const A* __restrict__ x_sub, A* __restrict__ out,
                                                               int nz, int nO, int N, int boundary, double WT0,
                                                               int* err) {
  using L = DeloStage<T, A>;
  extern __shared__ __align__(128) unsigned char dsm[];
  uint64_t* full = (uint64_t*)(dsm + kDStages * L::kBytes);
  uint64_t* empty = full + kDStages;
  volatile int* abort_flag = (volatile int*)(empty + kDStages);
  const int o = blockIdx.y, n0 = blockIdx.x * kDR;
  const int R = min(kDR, N - n0);                // rays of this CTA (even)
  const bool up = mu[o] > 0.0;
  if (threadIdx.x == 0) {
    for (int d = 0; d < kDStages; ++d) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(dsm_u32(&full[d])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(dsm_u32(&empty[d])), "r"(kDR));
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto row = [&](int p) { return ((size_t)(up ? p : nz - 1 - p) * nO + o) * N + n0; };
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      const uint32_t bkt = (uint32_t)R * 10 * sizeof(T), bv = (uint32_t)R * 4 * sizeof(A), bp = (uint32_t)R * 24;
      const uint32_t bytes = bkt + bv + (x_sub ? bv : 0u) + (par ? bp : 0u);
      int p = 0;
      for (; p < nz; ++p) {
        const int d = p % kDStages;
        if (p >= kDStages && !dbar_wait(&empty[d], ((p / kDStages) - 1) & 1, abort_flag)) break;
        unsigned char* st = dsm + d * L::kBytes;
        const size_t r0 = row(p);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(dsm_u32(&full[d])), "r"(bytes)
                     : "memory");
        auto copy = [&](unsigned char* dst, const void* src, uint32_t nb) {
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  dsm_u32(dst)),
              "l"((uint64_t)src), "r"(nb), "r"(dsm_u32(&full[d]))
              : "memory");
        };
        copy(st + L::kKT, kt + r0 * 10, bkt);
        copy(st + L::kEps, eps + r0 * 4, bv);
        if (x_sub) copy(st + L::kXs, x_sub + r0 * 4, bv);
        if (par) copy(st + L::kPar, par + r0 * 3, bp);
      }
      if (*abort_flag)   // drain copies that were issued and may not have been consumed
        for (int q = max(0, p - kDStages); q < p; ++q)
          for (long long i = 0; i < kDSpin && !dbar_try(&full[q % kDStages], (q / kDStages) & 1); ++i) {
          }
    }
  } else {
    const int r = threadIdx.x - 32;
    const bool live = r < R;
    A I[4] = {0, 0, 0, 0};
    A Sp[4] = {0, 0, 0, 0};
    A Kp[4][4];
    DeloPoint<T, A> cur, nxt;
    // take point p of this ray from its stage, then release the stage
    auto take = [&](int p, DeloPoint<T, A>& dp) -> bool {
      const int d = p % kDStages;
      if (!dbar_wait(&full[d], (p / kDStages) & 1, abort_flag)) return false;
      const unsigned char* st = dsm + d * L::kBytes;
      if (live) {
        const T* tk = (const T*)(st + L::kKT) + r * 10;
        for (int i = 0; i < 10; ++i) dp.t[i] = tk[i];
        const A* ev = (const A*)(st + L::kEps) + r * 4;
        for (int s = 0; s < 4; ++s) dp.e[s] = ev[s];
        const A* xv = (const A*)(st + L::kXs) + r * 4;
        for (int s = 0; s < 4; ++s) dp.xs[s] = x_sub ? xv[s] : (A)0;
        if (par) {
          const double* pv = (const double*)(st + L::kPar) + r * 3;
          for (int i = 0; i < 3; ++i) dp.ps[i] = pv[i];
        }
      }
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(dsm_u32(&empty[d])) : "memory");
      return true;
    };
    DeloFact<A> fc, fn;
    bool ok = take(0, cur);
    if (ok && live) delo_factor(cur, fc);
    for (int p = 0; p < nz && ok; ++p) {
      if (p + 1 < nz) ok = take(p + 1, nxt);
      if (!ok) break;
      if (live) {
        if (p + 1 < nz) delo_factor(nxt, fn);      // off the serial chain of this step
        delo_step(cur, fc, nxt, par != nullptr, p + 1 < nz, p, up, boundary, WT0, I, Sp, Kp);
        A* dst = out + (row(p) + r) * 4;
        for (int s = 0; s < 4; ++s) dst[s] = x_sub ? cur.xs[s] - I[s] : I[s];
      }
      cur = nxt;
      fc = fn;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag && err) atomicExch(err, 1);
}

template <typename T, typename A>
static int launch_delo(Ctx* c, const A* eps, const T* kt, const double* par, const double* mu, const A* x_sub, A* out,
                       int boundary, bool allow_staged) {
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  if (allow_staged && c->staged_sweep && N % 2 == 0 && c->tc_err.p) {
    using L = DeloStage<T, A>;
    const int smem = kDStages * L::kBytes + 2 * kDStages * 8 + 16;
    PRD_CUDA_TRY(c, cudaFuncSetAttribute(delo_staged_kernel<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    delo_staged_kernel<T, A><<<dim3(ceil_div(N, kDR), nO), 32 + kDR, smem, c->stream>>>(
        eps, kt, par, mu, x_sub, out, nz, nO, N, boundary, c->WT[0], (int*)c->tc_err.p);
  } else {
    delo_kernel<T, A><<<ceil_div(nO * N, 128), 128, 0, c->stream>>>(eps, kt, par, mu, x_sub, out, nz, nO, N, boundary,
                                                                    c->WT[0]);
  }
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

// f = (1 - eps) W_T eta_I / [Sigma (W_T, 0, 0, 0)]_I with the line's eta_I (App. E),
// written as (1 - eps) W_T rho / (kt6 num) with rho = eta_line / eta_total (FP64)
// and kt6 the stored 1/eta_total of the formal solver's tables: the source
// f num kt6 then holds the photon budget exactly whatever the rounding of kt6
// (an FP32 1/eta against an FP64 eta would break it at 1e-7, which the
// scattering amplifies by ~1/eps).
template <typename T, typename A>
__global__ void normalise_kernel(const A* __restrict__ num, const T* __restrict__ kt, const double* __restrict__ rho,
                                 const double* __restrict__ fac, double* __restrict__ f, int nz, int nO, int N) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= (long long)nz * nO * N) return;
  const int iz = (int)(pt / ((long long)nO * N));
  f[pt] = fac[iz] * rho[pt] / ((double)kt[pt * 10 + 6] * (double)num[pt * 4]);
}

// Coherent continuum scattering in the observer frame (App. A):
//   eps[z][o][n][i] += sigma_c[z][n] sum_{o', j} PW[o][o'][i][j] x[z][o'][n][j]
// PW = w_o' P(o, o') (dipole phase matrix); nOut output directions (the grid,
// or one line of sight), the input x on the grid's nO directions.
template <typename A>
__global__ void continuum_kernel(const A* __restrict__ x, const double* __restrict__ pw,
                                 const double* __restrict__ sig, A* __restrict__ eps, int nz, int nOut, int nO, int N) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (z, o, n), n fastest
  if (pt >= (long long)nz * nOut * N) return;
  const int n = (int)(pt % N);
  const int o = (int)((pt / N) % nOut);
  const int iz = (int)(pt / ((long long)N * nOut));
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int op = 0; op < nO; ++op) {
    const A* xv = x + (((size_t)iz * nO + op) * N + n) * 4;
    const double* P = pw + ((size_t)o * nO + op) * 16;
    const double x0 = xv[0], x1 = xv[1], x2 = xv[2], x3 = xv[3];
    for (int i = 0; i < 4; ++i) acc[i] += P[i * 4] * x0 + P[i * 4 + 1] * x1 + P[i * 4 + 2] * x2 + P[i * 4 + 3] * x3;
  }
  const double sc = sig[(size_t)iz * N + n];
  A* e = eps + pt * 4;
  for (int i = 0; i < 4; ++i) e[i] = (A)((double)e[i] + sc * acc[i]);
}

template <typename T>
__global__ void fill_planck_kernel(T* __restrict__ x, const double* __restrict__ WT, int nz, int nO, int N) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= (long long)nz * nO * N) return;
  const int iz = (int)(pt / ((long long)nO * N));
  x[pt * 4] = (T)WT[iz];
  x[pt * 4 + 1] = x[pt * 4 + 2] = x[pt * 4 + 3] = (T)0;
}

// ------------------------------------------------------------------ launchers
template <typename T, typename A>
static int sigma_T(Ctx* c, const A* x, A* eps, bool normalised, A* eb_ext = nullptr, A* M_ext = nullptr,
                   A* Ic_ext = nullptr, double* J_ext = nullptr, bool t64 = false) {
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  const SigmaTables tb = sigma_tables(c, t64);
  const long long npt = (long long)nz * nO * N;
  A* Mb = M_ext ? M_ext : (A*)c->scratch1.p;
  A* M = Mb;
  A* Ic = Ic_ext ? Ic_ext : (A*)c->scratch2.p;
  A* eb = eb_ext ? eb_ext : (A*)c->scratch3.p;
  const double* sp = (const double*)c->sp.p;
  cudaEvent_t e0;
  // S1
  stage_begin(c, ST_S1, &e0);
  spline_M_kernel<A><<<ceil_div(nz * nO * 4, 128), 128, 0, c->stream>>>(x, M, sp, nz, nO, N);
  spline_eval_kernel<A, A><<<ceil_div(npt, 256), 256, 0, c->stream>>>(x, M, (const int*)c->iin.p, (const double*)c->tin.p,
                                                                  sp, nullptr, Ic, nz, nO, N);
  stage_end(c, ST_S1, e0);
  // S5 (initialises eps_bar)
  stage_begin(c, ST_S5, &e0);
  const int nuv = c->nu_st * c->nu_st;
  double* J = J_ext ? J_ext : (double*)c->r3J.p;
  PRD_CUDA_TRY(c, cudaMemsetAsync(J, 0, (size_t)nz * nuv * 2 * sizeof(double), c->stream));
  launch_r3_J<T, A>(c, Ic, J, nO, tb);
  launch_r3_out<T, A>(c, (const double*)J, (const T*)tb.r3out, eb, nO, tb);
  stage_end(c, ST_S5, e0);
  // S3 + S4
  stage_begin(c, ST_S3, &e0);
  const int nchunk = (c->max_cout + kCW - 1) / kCW;
  bool s3_done = false;   // the tensor-core or double-float contraction ran
  if constexpr (std::is_same<T, float>::value && std::is_same<A, float>::value) {
    if (c->use_tc && c->tc_ready && !t64) {
      int rc = r2_tc_launch(c, Ic, eb);
      if (rc) return rc;
      s3_done = true;
    }
  }
  if constexpr (std::is_same<T, double>::value && std::is_same<A, double>::value) {
    if (t64) {
      const size_t smem = sizeof(float4) * (size_t)kMB * kCW * 4 + sizeof(float2) * (size_t)2 * N * (kMB + 1);
      cudaFuncSetAttribute(r2_dd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      r2_dd_kernel<<<dim3(nchunk, c->ncls, nz), 256, smem, c->stream>>>(
          (const double*)tb.tiles, (const double*)tb.Y, Ic, (const int*)c->cls_dev.p, eb, c->ncls, c->ntile(), nO, N,
          c->npairs, tb.ld);
      s3_done = true;
    }
  }
  if (!s3_done) {
    const size_t smem = sizeof(A) * (size_t)kMB * 2 * kCW * 4 + sizeof(T) * (size_t)2 * N * (kMB + 1);
    cudaFuncSetAttribute(r2_simt_kernel<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    r2_simt_kernel<T, A><<<dim3(nchunk, c->ncls, nz), 256, smem, c->stream>>>(
        (const T*)tb.tiles, (const T*)tb.Y, Ic, (const int*)c->cls_dev.p, eb, c->ncls, c->ntile(), nO, N, c->npairs,
        tb.ld, tb.tiled);
  }
  stage_end(c, ST_S3, e0);
  // S6
  stage_begin(c, ST_S6, &e0);
  spline_M_kernel<A><<<ceil_div(nz * nO * 4, 128), 128, 0, c->stream>>>(eb, Mb, sp, nz, nO, N);
  spline_eval_kernel<A, double><<<ceil_div(npt, 256), 256, 0, c->stream>>>(eb, Mb, (const int*)c->ibk.p,
                                                                     (const double*)c->tbk.p, sp,
                                                                     normalised ? (const double*)c->f.p : nullptr, eps, nz,
                                                                     nO, N);
  // continuum scattering (App. A) joins the normalised emissivity; the
  // Kirchhoff factor is computed from the line alone (normalised = false)
  if (normalised && c->has_cont())
    continuum_kernel<A><<<ceil_div(npt, 256), 256, 0, c->stream>>>(x, (const double*)c->cont_pw.p,
                                                                 (const double*)c->cont_sig.p, eps, nz, nO, nO, N);
  stage_end(c, ST_S6, e0);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

// Spline frame change of a whole vector: to the comoving frame (I(u_n - u_b))
// or back (eps(u_n + u_b)); uses scratch1 for the second derivatives.
int spline_frame_change(Ctx* c, const void* in, void* out, bool to_comoving) {
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  const long long npt = (long long)nz * nO * N;
  const double* sp = (const double*)c->sp.p;
  const int* kk = (const int*)(to_comoving ? c->iin.p : c->ibk.p);
  const double* tt = (const double*)(to_comoving ? c->tin.p : c->tbk.p);
  if (c->prec == PRD_FP64) {
    spline_M_kernel<double><<<ceil_div(nz * nO * 4, 128), 128, 0, c->stream>>>((const double*)in, (double*)c->scratch1.p, sp, nz, nO, N);
    spline_eval_kernel<double, double><<<ceil_div(npt, 256), 256, 0, c->stream>>>((const double*)in, (const double*)c->scratch1.p, kk, tt,
                                                                         sp, nullptr, (double*)out, nz, nO, N);
  } else {
    spline_M_kernel<float><<<ceil_div(nz * nO * 4, 128), 128, 0, c->stream>>>((const float*)in, (float*)c->scratch1.p, sp, nz, nO, N);
    spline_eval_kernel<float, float><<<ceil_div(npt, 256), 256, 0, c->stream>>>((const float*)in, (const float*)c->scratch1.p, kk, tt,
                                                                        sp, nullptr, (float*)out, nz, nO, N);
  }
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

// The same frame change for an FP64 vector in either mode (the preconditioner's
// sweeps), with the caller's FP64 scratch for the spline second derivatives.
int spline_frame_change_d(Ctx* c, const double* in, double* out, double* Mscratch, bool to_comoving) {
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  const long long npt = (long long)nz * nO * N;
  const double* sp = (const double*)c->sp.p;
  const int* kk = (const int*)(to_comoving ? c->iin.p : c->ibk.p);
  const double* tt = (const double*)(to_comoving ? c->tin.p : c->tbk.p);
  spline_M_kernel<double><<<ceil_div(nz * nO * 4, 128), 128, 0, c->stream>>>(in, Mscratch, sp, nz, nO, N);
  spline_eval_kernel<double, double><<<ceil_div(npt, 256), 256, 0, c->stream>>>(in, Mscratch, kk, tt, sp, nullptr, out,
                                                                               nz, nO, N);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

int apply_sigma(Ctx* c, const void* x, void* eps, bool normalised) {
  if (c->prec == PRD_FP64) return sigma_T<double, double>(c, (const double*)x, (double*)eps, normalised);
  return sigma_T<float, float>(c, (const float*)x, (float*)eps, normalised);
}

int apply_lambda(Ctx* c, const void* eps, void* out, const void* sub_from, bool boundary) {
  const double* dmu = (const double*)c->dmu.p;
  cudaEvent_t e0;
  stage_begin(c, ST_S7, &e0);
  int rc;
  if (c->prec == PRD_FP64)
    rc = launch_delo<double, double>(c, (const double*)eps, (const double*)c->kt.p, (const double*)c->par_active(), dmu,
                                     (const double*)sub_from, (double*)out, boundary ? 1 : 0, true);
  else
    rc = launch_delo<float, float>(c, (const float*)eps, (const float*)c->kt.p, (const double*)c->par_active(), dmu,
                                   (const float*)sub_from, (float*)out, boundary ? 1 : 0, true);
  stage_end(c, ST_S7, e0);
  return rc;
}

// Kirchhoff factor f = (1-eps) W_T eta_I / [Sigma (W_T,0,0,0)]_I (App. E).  In
// FP32 mode the unnormalised Sigma is applied to the Planck field in FP64, with
// the tables the refinement residuals use, so that f corrects the photon budget
// of exactly the operator whose solution is returned (the FP32 apply that
// drives the inner iterations differs from it only at FP32 rounding level).
int compute_normalisation(Ctx* c) {
  const int nz = c->nz, nO = c->nO, N = c->nnu;
  const long long npt = (long long)nz * nO * N;
  DBuf wt, fac, xin, num, eb, Mb, Ic;
  std::vector<double> f(nz);
  for (int iz = 0; iz < nz; ++iz) f[iz] = (1.0 - c->eps[iz]) * c->WT[iz];
  int rc;
  const size_t vb64 = nvec(c) * 8;
  auto cleanup = [&]() { dfree(wt); dfree(fac); dfree(xin); dfree(num); dfree(eb); dfree(Mb); dfree(Ic); };
  if ((rc = upload(c, wt, c->WT.data(), nz * 8)) || (rc = upload(c, fac, f.data(), nz * 8)) ||
      (rc = dalloc(c, xin, vb64)) || (rc = dalloc(c, num, vb64)) || (rc = dalloc(c, eb, vb64)) ||
      (rc = dalloc(c, Mb, vb64)) || (rc = dalloc(c, Ic, vb64))) {
    cleanup();
    return rc;
  }
  if (c->prec == PRD_FP64) {
    fill_planck_kernel<double><<<ceil_div(npt, 256), 256, 0, c->stream>>>((double*)xin.p, (const double*)wt.p, nz, nO, N);
    rc = sigma_T<double, double>(c, (const double*)xin.p, (double*)num.p, false);
    if (!rc)
      normalise_kernel<double, double><<<ceil_div(npt, 256), 256, 0, c->stream>>>(
          (const double*)num.p, (const double*)c->kt.p, (const double*)c->eta_line.p, (const double*)fac.p,
          (double*)c->f.p, nz, nO, N);
  } else {
    fill_planck_kernel<double><<<ceil_div(npt, 256), 256, 0, c->stream>>>((double*)xin.p, (const double*)wt.p, nz, nO, N);
    rc = c->has64 ? sigma_T<double, double>(c, (const double*)xin.p, (double*)num.p, false, (double*)eb.p,
                                            (double*)Mb.p, (double*)Ic.p, nullptr, true)
                  : sigma_T<float, double>(c, (const double*)xin.p, (double*)num.p, false, (double*)eb.p, (double*)Mb.p,
                                           (double*)Ic.p);
    if (!rc)
      normalise_kernel<double, double><<<ceil_div(npt, 256), 256, 0, c->stream>>>(
          (const double*)num.p, (const double*)c->kt64.p, (const double*)c->eta_line.p, (const double*)fac.p,
          (double*)c->f.p, nz, nO, N);
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  cleanup();
  if (rc) return rc;
  if (e != cudaSuccess) return fail(c, PRD_E_CUDA, std::string("normalisation: ") + cudaGetErrorString(e));
  return PRD_OK;
}

int apply_operator(Ctx* c, const void* x, void* y) {
  int rc = apply_sigma(c, x, c->gm_t.p, true);
  if (rc) return rc;
  return apply_lambda(c, c->gm_t.p, y, x, false);
}

int rhs(Ctx* c, void* b) { return apply_lambda(c, c->epsth.p, b, nullptr, true); }

// FP32 mode only: y = (Id - Lambda Sigma) x with FP64 vectors, FP64 arithmetic
// and the FP64 copy of the Sigma tables when it was kept (else the FP32 tables):
// the residuals of the refinement, which fix the accuracy of the solution.
int apply_operator_acc(Ctx* c, const double* x, double* y, double* ws /* 4 x nvec doubles */) {
  const size_t nv = nvec(c);
  double* eps = ws;
  int rc = c->has64 ? sigma_T<double, double>(c, x, eps, true, ws + nv, ws + 2 * nv, ws + 3 * nv, nullptr, true)
                     : sigma_T<float, double>(c, x, eps, true, ws + nv, ws + 2 * nv, ws + 3 * nv);
  if (rc) return rc;
  delo_kernel<double, double><<<ceil_div(c->nO * c->nnu, 128), 128, 0, c->stream>>>(
      eps, (const double*)c->kt64.p, (const double*)c->par_active(), (const double*)c->dmu.p, x, y, c->nz, c->nO,
      c->nnu, 0, c->WT[0]);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

__global__ void add_kernel(double* __restrict__ a, const double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] += b[i];
}

// eps = eps_th + Sigma x in FP64 arithmetic on the FP64 tables (the residual
// path of the refinement in FP32 mode): the emissivity whose formal solution,
// with the boundary term, minus x is the residual b - A x.  ws: 3 N-vectors.
int emissivity_acc(Ctx* c, const double* x, double* eps, double* ws) {
  const size_t nv = nvec(c);
  int rc;
  if (c->prec == PRD_FP64) rc = sigma_T<double, double>(c, x, eps, true);
  else if (c->has64) rc = sigma_T<double, double>(c, x, eps, true, ws, ws + nv, ws + 2 * nv, nullptr, true);
  else rc = sigma_T<float, double>(c, x, eps, true, ws, ws + nv, ws + 2 * nv);
  if (rc) return rc;
  add_kernel<<<c->grid_ew(), 256, 0, c->stream>>>(eps, (const double*)(c->prec == PRD_FP64 ? c->epsth.p : c->epsth64.p),
                                                  nv);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

int rhs_acc(Ctx* c, double* b) {
  delo_kernel<double, double><<<ceil_div(c->nO * c->nnu, 128), 128, 0, c->stream>>>(
      (const double*)c->epsth64.p, (const double*)c->kt64.p, (const double*)c->par_active(), (const double*)c->dmu.p,
      nullptr, b, c->nz, c->nO, c->nnu, 1, c->WT[0]);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, PRD_E_CUDA, std::string("rhs_acc: ") + cudaGetErrorString(e));
  return PRD_OK;
}

// ------------------------------------------------------------------ S11
// Emergent Stokes vectors along extra lines of sight (Sect. 6.2): for each
// LOS the comoving emissivity eps_bar(z, LOS, .) is built from the solution's
// comoving field with new tiles for the angles Theta(LOS, Omega'), normalised
// with f computed from the same rows on the Planck field, moved to the
// observer frame, and one DELO sweep from the bottom boundary gives I at z_max.
template <typename T>
__global__ void planck_comoving_kernel(T* __restrict__ Ic, const double* __restrict__ WT, int nz, int nO, int N) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= (long long)nz * nO * N) return;
  const int iz = (int)(pt / ((long long)nO * N));
  Ic[pt * 4] = (T)WT[iz];
  Ic[pt * 4 + 1] = Ic[pt * 4 + 2] = Ic[pt * 4 + 3] = (T)0;
}

// eps(z, n) = (eps_sc with f) + eps_th;  f = (1-eps) W_T eta_I / num_I, formed
// as in normalise_kernel from rho = eta_line / eta_total and the stored 1/eta_total
template <typename T, typename A>
__global__ void los_combine_kernel(const A* __restrict__ es, const A* __restrict__ ew, const T* __restrict__ kt,
                                   const double* __restrict__ rho, const T* __restrict__ eth,
                                   const double* __restrict__ fac, A* __restrict__ out, int nz, int N) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= nz * N) return;
  const int iz = pt / N;
  const double f = fac[iz] * rho[pt] / ((double)kt[pt * 10 + 6] * (double)ew[pt * 4]);
  out[pt * 4] = (A)((double)es[pt * 4] * f + (double)eth[pt * 4]);
  for (int s = 1; s < 4; ++s) out[pt * 4 + s] = es[pt * 4 + s] + (A)eth[pt * 4 + s];
}

template <typename S, typename D>
__global__ void cast_kernel(const S* __restrict__ in, D* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (D)in[i];
}

// T: precision of the stored tables and of x / out; A: precision of the fields
// along the line of sight (double in FP32 mode, like the FP64-accumulated
// residual path, so the emergent spectrum carries no FP32 cancellation).

template <typename T, typename A>
static int emergent_T(Ctx* c, const T* x, int nlos, const double* mus, const double* chis, T* out) {
  const int nz = c->nz, nO = c->nO, N = c->nnu, nti = c->ntile(), nuv = c->nu_st * c->nu_st;
  const long long npt = (long long)nz * nO * N;
  const size_t tz = (size_t)nO * nti * N * c->ld() * sizeof(T);   // tiles of one height, all LOS classes
  DBuf Icx, Icw, Jx, Jw, tiles, Yd, rout, ktd, ethd, kidx, ttd, es_bar, ew_bar, es, ew, M, eps, lam, fac, dmu, clsd,
      xa, Mx, pard, etald, cpwd;
  auto cleanup = [&]() {
    DBuf* bs[] = {&Icx, &Icw, &Jx, &Jw, &tiles, &Yd, &rout, &ktd, &ethd, &kidx, &ttd, &es_bar, &ew_bar, &es, &ew,
                  &M, &eps, &lam, &fac, &dmu, &clsd, &xa, &Mx, &pard, &etald, &cpwd};
    for (DBuf* b : bs) dfree(*b);
  };
  const size_t vb = nvec(c) * sizeof(A), lb = (size_t)nz * N * 4 * sizeof(A);
  int rc;
  std::vector<double> facv(nz), wt(c->WT);
  for (int iz = 0; iz < nz; ++iz) facv[iz] = (1.0 - c->eps[iz]) * c->WT[iz];
  // class structure of one LOS: class o' has the single output entry 0 and the single pair (LOS, o')
  std::vector<int> cls;
  for (int i = 0; i <= nO; ++i) cls.push_back(i);
  for (int i = 0; i < nO; ++i) cls.push_back(0);
  for (int i = 0; i <= nO; ++i) cls.push_back(i);
  for (int i = 0; i < nO; ++i) cls.push_back(i);
  if ((rc = dalloc(c, Icx, vb)) || (rc = dalloc(c, Icw, vb)) || (rc = dalloc(c, Jx, (size_t)nz * nuv * 16)) ||
      (rc = dalloc(c, Jw, (size_t)nz * nuv * 16)) || (rc = dalloc(c, tiles, tz)) || (rc = dalloc(c, es_bar, lb)) ||
      (rc = dalloc(c, ew_bar, lb)) || (rc = dalloc(c, es, lb)) || (rc = dalloc(c, ew, lb)) || (rc = dalloc(c, M, lb)) ||
      (rc = dalloc(c, eps, lb)) || (rc = dalloc(c, lam, lb)) || (rc = upload(c, fac, facv.data(), nz * 8)) ||
      (rc = dalloc(c, xa, vb)) || (rc = dalloc(c, Mx, (size_t)nz * nO * N * 4 * sizeof(A))) ||
      (rc = upload(c, clsd, cls.data(), cls.size() * 4))) {
    cleanup();
    return rc;
  }
  DBuf wtd;
  if ((rc = upload(c, wtd, wt.data(), nz * 8))) { cleanup(); return rc; }
  // comoving fields of the solution and of the Planck function, and their R_III moments
  cast_kernel<T, A><<<ceil_div(npt * 4, 256), 256, 0, c->stream>>>(x, (A*)xa.p, npt * 4);
  spline_M_kernel<A><<<ceil_div(nz * nO * 4, 128), 128, 0, c->stream>>>((const A*)xa.p, (A*)Mx.p, (const double*)c->sp.p, nz, nO, N);
  spline_eval_kernel<A, A><<<ceil_div(npt, 256), 256, 0, c->stream>>>((const A*)xa.p, (const A*)Mx.p, (const int*)c->iin.p,
                                                                     (const double*)c->tin.p, (const double*)c->sp.p,
                                                                     nullptr, (A*)Icx.p, nz, nO, N);
  planck_comoving_kernel<A><<<ceil_div(npt, 256), 256, 0, c->stream>>>((A*)Icw.p, (const double*)wtd.p, nz, nO, N);
  PRD_CUDA_TRY(c, cudaMemsetAsync(Jx.p, 0, Jx.bytes, c->stream));
  PRD_CUDA_TRY(c, cudaMemsetAsync(Jw.p, 0, Jw.bytes, c->stream));
  const SigmaTables tb = sigma_tables(c, false);
  launch_r3_J<T, A>(c, (const A*)Icx.p, (double*)Jx.p, nO, tb);
  launch_r3_J<T, A>(c, (const A*)Icw.p, (double*)Jw.p, nO, tb);
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const double mu1 = 1.0;
  for (int l = 0; l < nlos && !rc; ++l) {
    LosTables L;
    los_tables(c, mus[l], chis[l], L);
    auto up = [&](DBuf& b, const std::vector<double>& v) {
      std::vector<T> h(v.begin(), v.end());
      return upload(c, b, h.data(), h.size() * sizeof(T));
    };
    if ((rc = up(Yd, L.Y)) || (rc = up(rout, L.rout)) || (rc = up(ktd, L.kt)) || (rc = up(ethd, L.epsth)) ||
        (rc = upload(c, pard, L.par.data(), L.par.size() * 8)) ||
        (rc = upload(c, etald, L.eta_line.data(), L.eta_line.size() * 8)) ||
        (rc = upload(c, cpwd, L.cont_pw.data(), L.cont_pw.size() * 8)) ||
        (rc = upload(c, kidx, L.kidx.data(), L.kidx.size() * 4)) || (rc = upload(c, ttd, L.tt.data(), L.tt.size() * 8)) ||
        (rc = upload(c, dmu, &mus[l], 8)))
      break;
    (void)mu1;
    // R_III parts initialise the comoving rows
    launch_r3_out<T, A>(c, (const double*)Jx.p, (const T*)rout.p, (A*)es_bar.p, 1, tb);
    launch_r3_out<T, A>(c, (const double*)Jw.p, (const T*)rout.p, (A*)ew_bar.p, 1, tb);
    // R_II: tiles of every height for the LOS classes, then the contraction
    for (int iz = 0; iz < nz && !rc; ++iz) {
      std::vector<double> th(L.theta);
      if ((rc = gen_tiles_z(c, iz, th, tiles.p))) break;
      const size_t smem = sizeof(A) * (size_t)kMB * 2 * kCW * 4 + sizeof(T) * (size_t)2 * N * (kMB + 1);
      cudaFuncSetAttribute(r2_simt_kernel<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      const T* Yz = (const T*)Yd.p + (size_t)iz * nO * nti * 32;
      r2_simt_kernel<T, A><<<dim3(1, nO, 1), 256, smem, c->stream>>>(
          (const T*)tiles.p, Yz, (const A*)Icx.p + (size_t)iz * nO * N * 4, (const int*)clsd.p,
          (A*)es_bar.p + (size_t)iz * N * 4, nO, nti, nO, N, nO, c->ld(), c->tiled());
      r2_simt_kernel<T, A><<<dim3(1, nO, 1), 256, smem, c->stream>>>(
          (const T*)tiles.p, Yz, (const A*)Icw.p + (size_t)iz * nO * N * 4, (const int*)clsd.p,
          (A*)ew_bar.p + (size_t)iz * N * 4, nO, nti, nO, N, nO, c->ld(), c->tiled());
      PRD_CUDA_TRY(c, cudaPeekAtLastError());
    }
    if (rc) break;
    // observer frame, normalisation, thermal part, formal solution along the LOS
    spline_M_kernel<A><<<ceil_div(nz * 4, 128), 128, 0, c->stream>>>((const A*)es_bar.p, (A*)M.p, (const double*)c->sp.p, nz, 1, N);
    spline_eval_kernel<A, A><<<ceil_div((long long)nz * N, 256), 256, 0, c->stream>>>(
        (const A*)es_bar.p, (const A*)M.p, (const int*)kidx.p, (const double*)ttd.p, (const double*)c->sp.p, nullptr,
        (A*)es.p, nz, 1, N);
    spline_M_kernel<A><<<ceil_div(nz * 4, 128), 128, 0, c->stream>>>((const A*)ew_bar.p, (A*)M.p, (const double*)c->sp.p, nz, 1, N);
    spline_eval_kernel<A, A><<<ceil_div((long long)nz * N, 256), 256, 0, c->stream>>>(
        (const A*)ew_bar.p, (const A*)M.p, (const int*)kidx.p, (const double*)ttd.p, (const double*)c->sp.p, nullptr,
        (A*)ew.p, nz, 1, N);
    los_combine_kernel<T, A><<<ceil_div(nz * N, 128), 128, 0, c->stream>>>((const A*)es.p, (const A*)ew.p,
                                                                          (const T*)ktd.p, (const double*)etald.p,
                                                                          (const T*)ethd.p,
                                                                          (const double*)fac.p, (A*)eps.p, nz, N);
    if (c->has_cont())
      continuum_kernel<A><<<ceil_div(nz * N, 128), 128, 0, c->stream>>>((const A*)xa.p, (const double*)cpwd.p,
                                                                       (const double*)c->cont_sig.p, (A*)eps.p, nz,
                                                                       1, nO, N);
    delo_kernel<T, A><<<ceil_div(N, 128), 128, 0, c->stream>>>((const A*)eps.p, (const T*)ktd.p,
                                                             c->formal ? (const double*)pard.p : nullptr,
                                                             (const double*)dmu.p, nullptr, (A*)lam.p, nz, 1, N, 1,
                                                             c->WT[0]);
    cast_kernel<A, T><<<ceil_div(N * 4, 128), 128, 0, c->stream>>>((const A*)lam.p + (size_t)(nz - 1) * N * 4,
                                                                  out + (size_t)l * N * 4, (long long)N * 4);
    PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  dfree(wtd);
  cleanup();
  return rc;
}

int emergent(Ctx* c, const void* x, int nlos, const double* mu, const double* chi, void* out) {
  if (c->prec == PRD_FP64) return emergent_T<double, double>(c, (const double*)x, nlos, mu, chi, (double*)out);
  return emergent_T<float, double>(c, (const float*)x, nlos, mu, chi, (float*)out);
}

// ------------------------------------------------------------------ static scratch
// Scratch of prd_apply_sigma_noalloc: one file-scope device array, present on
// every GPU that loads the library until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_sigma_scratch[kStaticScratchBytes];

// Device address of the static scratch in the current CUDA context.  The
// host-side symbol is only a stand-in and must not be passed to a kernel.  The
// address is looked up on every call (cudaGetSymbolAddress allocates nothing):
// a cached address would dangle after the host framework resets the device or
// re-creates its primary context, which reloads the library's device code.
static int static_scratch(Ctx* c, void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_sigma_scratch);
  if (e != cudaSuccess || !p)
    return fail(c, PRD_E_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
  *out = p;
  return PRD_OK;
}

template <typename T>
static int sigma_static_T(Ctx* c, const T* x, T* eps) {
  const size_t nv = nvec(c);
  const size_t nuv = (size_t)c->nu_st * c->nu_st;
  const size_t jbytes = ((size_t)c->nz * nuv * 2 * sizeof(double) + 255) / 256 * 256;
  const size_t vb = (nv * sizeof(T) + 255) / 256 * 256;
  if (jbytes + 3 * vb > kStaticScratchBytes)
    return fail(c, PRD_E_ARG, "problem needs " + std::to_string((jbytes + 3 * vb) >> 20) +
                                  " MiB of scratch; prd_apply_sigma_noalloc supports at most 64 MiB");
  void* base = nullptr;
  int rc = static_scratch(c, &base);
  if (rc) return rc;
  unsigned char* b = (unsigned char*)base;
  double* J = (double*)b;
  T* M = (T*)(b + jbytes);
  T* Ic = (T*)(b + jbytes + vb);
  T* eb = (T*)(b + jbytes + 2 * vb);
  return sigma_T<T, T>(c, x, eps, true, eb, M, Ic, J);
}

}  // namespace prd

extern "C" int prd_apply_sigma_noalloc(prd_ctx* ctx, const void* x_dev, void* eps_dev) {
  if (!ctx) return PRD_E_ARG;
  prd::Ctx* c = &ctx->c;
  cudaSetDevice(c->device);
  if (!c->ready) return prd::fail(c, PRD_E_STATE, "call prd_setup first");
  if (!x_dev || !eps_dev || x_dev == eps_dev) return prd::fail(c, PRD_E_ARG, "x_dev/eps_dev NULL or aliased");
  if (!prd::point_aligned(c, x_dev) || !prd::point_aligned(c, eps_dev))
    return prd::fail(c, PRD_E_ARG, "x_dev/eps_dev do not start on a whole Stokes point (4 elements)");
  if (c->prec == PRD_FP64) return prd::sigma_static_T<double>(c, (const double*)x_dev, (double*)eps_dev);
  return prd::sigma_static_T<float>(c, (const float*)x_dev, (float*)eps_dev);
}
