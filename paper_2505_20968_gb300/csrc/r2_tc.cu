// S3+S4 R_II contraction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// For one (height z, scattering-angle class c, chunk of <= 64 output
// directions) the CTA computes the real product
//     eps_bar[n][(o,i)] += sum_{ti, k} A[ti][n][k] * B[ti][k][(o,i)],   k in [0, 2N)
// where A[ti] is the stored tile (Re | Im halves of the tile against the spline
// basis, Eq. RQIIKKp / Eq. G) and
//     B[ti][k][(o,i)] = sum_{o' in class, j} Ycomp_{ti,ij}(o,o') I~_j(o', m)
// with Ycomp = Re Y for k = m < N and -Im Y for k = N + m (so that the sum is
// Re(T Z) over the complex tile T and Z = Y I~).
//
// Roles (192 threads): warp 0 streams A with TMA (box 16 x 128 fp32, 64-byte
// swizzle) and owns the TMEM allocation; warp 1 issues tcgen05.mma; warps 2-5
// build B in shared memory, split A and B into TF32 hi/lo parts (3 products:
// hi*hi + hi*lo + lo*hi, FP32-level accuracy) and run the epilogue from TMEM.
// Accumulators: two M = 128 blocks (rows n < 256) x NCP columns of TMEM.
// Every mbarrier wait is bounded; on expiry the CTA records an error flag,
// drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdio>
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

namespace tc {

constexpr int kStages = 3;
constexpr int kKC = 16;                       // fp32 per stage along K (64-byte rows)
constexpr int kABytes = 2 * 128 * kKC * 4;    // two M blocks
constexpr int kBBytes = 256 * kKC * 4;        // up to 256 columns
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;   // A, A_lo, B_hi, B_lo
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr int kMaxE = 64;                     // output directions per CTA
constexpr long long kSpin = 1ll << 24;        // bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.b32 %0, 1, 0, P;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false (and raises the CTA abort flag) on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  for (long long i = 0; i < kSpin; ++i) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t addr = (smem_u32(p) & 0x3FFFF) >> 4;
  const uint64_t lbo = 1;            // unused for swizzled K-major
  const uint64_t sbo = 512 >> 4;
  return addr | (lbo << 16) | (sbo << 32) | (1ull << 46) | (4ull << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// byte offset of element (row, k) in a K-major 64-byte-swizzled operand (k < 16)
__device__ __forceinline__ uint32_t swz64(int row, int k) {
  const uint32_t chunk = (uint32_t)(k >> 2) ^ (uint32_t)((row >> 1) & 3);
  return (uint32_t)((row >> 3) * 512 + (row & 7) * 64) + chunk * 16 + (uint32_t)(k & 3) * 4;
}

struct Params {
  const float* Y;       // [z][pair][ntile][16][2]
  const float* Ic;      // [z][o][N][4]
  const int* cls;
  float* eb;            // [z][o][N][4]
  int* err;
  int ncls, ntile, nO, N, npairs;
};

__global__ void __launch_bounds__(192, 1) r2_tc_kernel(const __grid_constant__ CUtensorMap tmap, Params p) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + kStages * kStageBytes);
  uint64_t* ready = full + kStages;
  uint64_t* empty = ready + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int chunk = blockIdx.x, c = blockIdx.y, iz = blockIdx.z;
  const int* cout_ptr = p.cls;
  const int* cout_dir = p.cls + p.ncls + 1;
  const int ne_tot = cout_ptr[p.ncls];
  const int* pair_ptr = cout_dir + ne_tot;
  const int* pair_in = pair_ptr + ne_tot + 1;
  const int e0 = cout_ptr[c] + chunk * kMaxE;
  const int e_end = cout_ptr[c + 1];
  if (e0 >= e_end) return;                       // uniform for the CTA
  const int E = min(kMaxE, e_end - e0);
  const int NCP = ((4 * E + 15) / 16) * 16;      // MMA N (multiple of 16, <= 256)
  const int N = p.N;
  const int KCH = (2 * N + kKC - 1) / kKC;
  const int iters = p.ntile * KCH;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tm_cols = (NCP > 128) ? 512u : 256u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tm_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const long long slab0 = ((long long)iz * p.ncls + c) * p.ntile;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int it = 0;
      for (; it < iters; ++it) {
        const int s = it % kStages;
        if (it >= kStages && !mbar_wait(&empty[s], ((it / kStages) - 1) & 1, abort_flag)) break;
        const int ti = it / KCH, kc = it - ti * KCH;
        unsigned char* A = sm + s * kStageBytes;
        mbar_expect_tx(&full[s], kABytes);
        tma_load_3d(A, &tmap, kc * kKC, 0, (int)(slab0 + ti), &full[s]);
        tma_load_3d(A + kABytes / 2, &tmap, kc * kKC, 128, (int)(slab0 + ti), &full[s]);
      }
      if (*abort_flag) {
        // drain loads that were issued and may not have been consumed
        for (int j = max(0, it - kStages); j < it; ++j) {
          const int s = j % kStages;
          for (long long i = 0; i < kSpin && !mbar_try(&full[s], (j / kStages) & 1); ++i) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NCP >> 3) << 17) | ((128u >> 4) << 24);
      int issued = 0;
      for (int it = 0; it < iters; ++it) {
        const int s = it % kStages;
        if (!mbar_wait(&ready[s], (it / kStages) & 1, abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* A = sm + s * kStageBytes;
        unsigned char* Alo = A + kABytes;
        unsigned char* Bhi = Alo + kABytes;
        unsigned char* Blo = Bhi + kBBytes;
        for (int mb = 0; mb < 2; ++mb) {
          const uint32_t d = tmem + (uint32_t)(mb * NCP);
          for (int ks = 0; ks < 2; ++ks) {
            const int ao = mb * (kABytes / 2) + ks * 32, bo = ks * 32;
            const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(d, sdesc(A + ao), sdesc(Bhi + bo), idesc, acc);
            mma_tf32(d, sdesc(A + ao), sdesc(Blo + bo), idesc, 1u);
            mma_tf32(d, sdesc(Alo + ao), sdesc(Bhi + bo), idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
        issued = it + 1;
      }
      if (issued > 0) mma_commit(done);
      else *abort_flag = 1;
    }
  } else {
    // ---------------- B builders / A splitters, then epilogue
    const int gt = threadIdx.x - 64;            // 0..127
    const int e_l = gt >> 1, half = gt & 1;     // output direction, k half (8 k each)
    const int e = e0 + e_l;
    const bool have = e_l < E;
    const int p0 = have ? pair_ptr[e] : 0, p1 = have ? pair_ptr[e + 1] : 0;
    for (int it = 0; it < iters; ++it) {
      const int s = it % kStages;
      if (!mbar_wait(&full[s], (it / kStages) & 1, abort_flag)) break;
      const int ti = it / KCH, kc = it - ti * KCH;
      unsigned char* A = sm + s * kStageBytes;
      unsigned char* Alo = A + kABytes;
      unsigned char* Bhi = Alo + kABytes;
      unsigned char* Blo = Bhi + kBBytes;
      // A_lo = A - tf32(A): same byte layout as A
      {
        const float4* a4 = (const float4*)A;
        float4* l4 = (float4*)Alo;
        for (int q = gt; q < kABytes / 16; q += 128) {
          float4 v = a4[q];
          v.x -= tf32_hi(v.x); v.y -= tf32_hi(v.y); v.z -= tf32_hi(v.z); v.w -= tf32_hi(v.w);
          l4[q] = v;
        }
      }
      // B rows (e_l*4 + i), k = kc*16 + half*8 + q
      float z[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) z[i][q] = 0.f;
      if (have) {
        for (int pp = p0; pp < p1; ++pp) {
          const int op = pair_in[pp];
          const float* y = p.Y + (((size_t)iz * p.npairs + pp) * p.ntile + ti) * 32;
          float yr[16], yi[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) { yr[q] = y[2 * q]; yi[q] = -y[2 * q + 1]; }
          const float* ib = p.Ic + ((size_t)iz * p.nO + op) * N * 4;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int k = kc * kKC + half * 8 + q;
            if (k >= 2 * N) continue;
            const bool re = k < N;
            const int m = re ? k : k - N;
            const float4 iv = *(const float4*)(ib + (size_t)m * 4);
            const float* yc = re ? yr : yi;
#pragma unroll
            for (int i = 0; i < 4; ++i)
              z[i][q] += yc[i * 4] * iv.x + yc[i * 4 + 1] * iv.y + yc[i * 4 + 2] * iv.z + yc[i * 4 + 3] * iv.w;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = e_l * 4 + i;
        if (row >= NCP) continue;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int k = half * 8 + g * 4;
          float4 hi, lo;
          hi.x = tf32_hi(z[i][g * 4]);     lo.x = z[i][g * 4] - hi.x;
          hi.y = tf32_hi(z[i][g * 4 + 1]); lo.y = z[i][g * 4 + 1] - hi.y;
          hi.z = tf32_hi(z[i][g * 4 + 2]); lo.z = z[i][g * 4 + 2] - hi.z;
          hi.w = tf32_hi(z[i][g * 4 + 3]); lo.w = z[i][g * 4 + 3] - hi.w;
          *(float4*)(Bhi + swz64(row, k)) = hi;
          *(float4*)(Blo + swz64(row, k)) = lo;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&ready[s]);
    }
    // ---------------- epilogue: TMEM -> registers -> eps_bar
    const bool ok = mbar_wait(done, 0, abort_flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int q = warp & 3;                    // TMEM lane quarter of this warp
      const int r = q * 32 + lane;
      for (int mb = 0; mb < 2; ++mb) {
        const int n = mb * 128 + r;
        for (int c0 = 0; c0 < NCP; c0 += 16) {
          uint32_t v[16];
          const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(mb * NCP + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(ta));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (n < N) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = c0 + j;
              if (col < 4 * E) {
                const int o = cout_dir[e0 + col / 4];
                atomicAdd(p.eb + (((size_t)iz * p.nO + o) * N + n) * 4 + (col & 3), __uint_as_float(v[j]));
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(p.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tm_cols));
  }
}

}  // namespace tc

// Tensor map over the tiles viewed as [slab][n][k] fp32, k = 2N innermost.
int r2_tc_prepare(Ctx* c) {
  if (c->prec != PRD_FP32) return PRD_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess)
    return fail(c, PRD_E_CUDA, "cuTensorMapEncodeTiled entry point not available");
  auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  const int N = c->nnu;
  const cuuint64_t nslab = (cuuint64_t)c->nz * c->ncls * c->ntile();
  cuuint64_t dims[3] = {(cuuint64_t)(2 * N), (cuuint64_t)N, nslab};
  cuuint64_t strides[2] = {(cuuint64_t)2 * N * 4, (cuuint64_t)N * 2 * N * 4};
  cuuint32_t box[3] = {tc::kKC, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode((CUtensorMap*)c->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->tiles.p, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, PRD_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  if (!c->tc_err.p) {
    int rc = dalloc(c, c->tc_err, sizeof(int));
    if (rc) return rc;
  }
  PRD_CUDA_TRY(c, cudaMemset(c->tc_err.p, 0, sizeof(int)));
  c->tc_ready = true;
  return PRD_OK;
}

int r2_tc_launch(Ctx* c, const float* Ic, float* eb) {
  tc::Params p{(const float*)c->Y.p, Ic, (const int*)c->cls_dev.p, eb, (int*)c->tc_err.p, c->ncls, c->ntile(),
               c->nO, c->nnu, c->npairs};
  static bool attr_set = false;
  if (!attr_set) {
    PRD_CUDA_TRY(c, cudaFuncSetAttribute(tc::r2_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    attr_set = true;
  }
  const int nchunk = (c->max_cout + tc::kMaxE - 1) / tc::kMaxE;
  tc::r2_tc_kernel<<<dim3(nchunk, c->ncls, c->nz), 192, tc::kSmemBytes, c->stream>>>(*(const CUtensorMap*)c->tmap, p);
  PRD_CUDA_TRY(c, cudaPeekAtLastError());
  return PRD_OK;
}

int r2_tc_check_error(Ctx* c) {
  int h = 0;
  PRD_CUDA_TRY(c, cudaMemcpy(&h, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(c->tc_err.p, 0, sizeof(int));
    return fail(c, PRD_E_TIMEOUT, "tensor-core contraction: a bounded wait expired");
  }
  return PRD_OK;
}

}  // namespace prd
